"""Pins of the oracle's coarse stage (quarter-size input, ZNCC Eq. 1-3, WTA Eq. 6)
against facts that do not come from the oracle itself: numpy's Pearson correlation
(ZNCC of two windows is their Pearson correlation coefficient), exact integer
arithmetic, invariances of the definition, and recovery of a known shift."""
import numpy as np
import pytest

import oracle
from paper_2305_11566_gb300 import synth


def _rng(seed):
    return np.random.default_rng(seed)


def test_downsample_brute_force():
    img = _rng(1).integers(0, 256, size=(23, 41), dtype=np.uint8)
    S = oracle.downsample4(img)
    assert S.shape == (5, 10)
    ref = img[:20, :40].astype(np.int64).reshape(5, 4, 10, 4).sum(axis=(1, 3))
    assert np.array_equal(S, ref)
    assert oracle.downsample4(np.full((8, 8), 255, np.uint8)).max() == 4080


def _window(S, x, y, r):
    h, w = S.shape
    ys = np.clip(np.arange(y - r, y + r + 1), 0, h - 1)
    xs = np.clip(np.arange(x - r, x + r + 1), 0, w - 1)
    return S[np.ix_(ys, xs)].astype(np.float64).ravel()


@pytest.mark.parametrize("k", [3, 5, 7])
def test_zncc_is_pearson_correlation(k):
    """Eq. 1-3 normalise the window covariance by both deviations: that is the
    Pearson correlation of the two k x k windows (numpy.corrcoef)."""
    rng = _rng(k)
    h, w, D = 7, 12, 5
    SL = rng.integers(0, 4081, size=(h, w)).astype(np.int32)
    SR = rng.integers(0, 4081, size=(h, w)).astype(np.int32)
    rho = oracle.zncc_volume(SL, SR, k, D)
    r = k // 2
    for y in range(h):
        for x in range(w):
            for d in range(D):
                if x - d < 0:
                    assert np.isnan(rho[y, x, d])
                    continue
                ref = np.corrcoef(_window(SL, x, y, r), _window(SR, x - d, y, r))[0, 1]
                assert abs(rho[y, x, d] - ref) < 1e-12


def test_zncc_range_and_self_match():
    p = synth.workload_small()
    SL = oracle.downsample4(p.left)
    rho = oracle.zncc_volume(SL, SL, 7, 16)
    v = rho[~np.isnan(rho)]
    assert v.min() >= -1.0 - 1e-12 and v.max() <= 1.0 + 1e-12
    assert np.allclose(rho[:, :, 0], 1.0, atol=1e-12)  # identical windows


def test_zncc_gain_offset_invariance():
    rng = _rng(5)
    SL = rng.integers(0, 4081, size=(9, 14)).astype(np.int32)
    SR = rng.integers(0, 4081, size=(9, 14)).astype(np.int32)
    base = oracle.zncc_volume(SL, SR, 5, 6)
    pos = oracle.zncc_volume(SL, 3 * SR + 17, 5, 6)
    neg = oracle.zncc_volume(SL, -2 * SR + 9000, 5, 6)
    ok = ~np.isnan(base)
    assert np.allclose(pos[ok], base[ok], atol=1e-12)
    assert np.allclose(neg[ok], -base[ok], atol=1e-12)
    left_gain = oracle.zncc_volume(5 * SL + 1, SR, 5, 6)
    assert np.allclose(left_gain[ok], base[ok], atol=1e-12)


def test_zncc_zero_variance_is_zero():
    SL = np.full((6, 10), 1234, np.int32)
    SR = _rng(3).integers(0, 4081, size=(6, 10)).astype(np.int32)
    rho = oracle.zncc_volume(SL, SR, 3, 4)
    assert np.all(rho[~np.isnan(rho)] == 0.0)
    disp, best, second = oracle.zncc_wta(SL, SR, 3, 4)
    assert np.all(disp == 0) and np.all(best == 0.0)


@pytest.mark.parametrize("s", [0, 3, 7])
def test_wta_recovers_constant_coarse_shift(s):
    """R(x) = L(x + s): for d = s the two windows are identical (rho = 1), so WTA
    must return s wherever neither window touches a border and the window varies."""
    rng = _rng(10 + s)
    h, w, k, D = 12, 48, 7, 12
    big = rng.integers(0, 4081, size=(h, w + s)).astype(np.int32)
    SL = big[:, :w].copy()       # L(x) = big(x)
    SR = big[:, s:s + w].copy()  # R(u) = big(u + s), so R(x - s) = L(x)
    disp, best, second = oracle.zncc_wta(SL, SR, k, D)
    r = k // 2
    interior = disp[:, s + r:w - r]
    assert np.all(interior == s)
    assert np.allclose(best[:, s + r:w - r], 1.0, atol=1e-12)


def test_wta_recovers_full_resolution_shift():
    """A full-resolution shift by 4 s pixels is a coarse shift by s after the 4x4 box sum."""
    p = synth.make_pair(256, 64, 0.0, 77)
    s = 5
    L = p.left
    R = np.zeros_like(L)
    R[:, :256 - 4 * s] = L[:, 4 * s:]  # R(X) = L(X + 4s)  => L(X) = R(X - 4s)
    disp, best, _ = oracle.coarse_match(L, R, 7, 16)
    r = 3
    w = 64
    assert np.all(disp[:, s + r:w - r - s] == s)


def test_wta_exact_agrees_with_fp64_argmax():
    p = synth.workload_small()
    SL = oracle.downsample4(p.left)
    SR = oracle.downsample4(p.right)
    k, D = 7, 16
    rho = oracle.zncc_volume(SL, SR, k, D)
    disp, best, second = oracle.zncc_wta(SL, SR, k, D)
    r2 = np.where(np.isnan(rho), -np.inf, rho)
    am = np.argmax(r2, axis=2)
    srt = np.sort(r2, axis=2)
    margin = srt[:, :, -1] - srt[:, :, -2]
    clear = margin > 1e-9
    assert clear.mean() > 0.95
    assert np.array_equal(disp[clear], am[clear])
    assert np.allclose(best, np.take_along_axis(r2, disp[..., None], 2)[..., 0], atol=0)
    # second best is the max over the other valid candidates
    oth = r2.copy()
    np.put_along_axis(oth, disp[..., None], -np.inf, 2)
    sec = oth.max(axis=2)
    sec[np.isinf(sec)] = -2.0
    assert np.array_equal(second, sec)


def test_wta_ties_take_lowest_d():
    """A right image that repeats with period 2 gives exactly equal scores for d and
    d + 2: the lowest d must win."""
    rng = _rng(9)
    h, w = 8, 30
    row = rng.integers(0, 4081, size=(h, 2)).astype(np.int32)
    SR = np.tile(row, (1, w // 2))
    SL = np.roll(SR, 1, axis=1)  # SL[x] = SR[x - 1]: d = 1, 3, 5 ... tie exactly
    disp, best, second = oracle.zncc_wta(SL, SR, 3, 6)
    r = 1
    inner = disp[:, 6:w - r]
    assert np.all(inner == 1)
    assert np.all(best[:, 6:w - r] == second[:, 6:w - r])


def test_wta_border_candidates():
    """Columns x < D only search d <= x; column 0 always returns 0."""
    p = synth.workload_small(1001)
    disp, best, second = oracle.coarse_match(p.left, p.right, 7, 16)
    x = np.arange(disp.shape[1])[None, :]
    assert np.all(disp <= x)
    assert np.all(disp[:, 0] == 0) and np.all(second[:, 0] == -2.0)
