"""Pins of the oracle's census cost and domain-transform (DT) aggregation (Sec. IV-C,
settings S1 Census+DT, S2 Census+SGM, S3 ZNCC+DT), on the CPU.

The paper names both methods without defining them; the readings (textbook census
transform on the quarter-size images; DT = cost aggregation by the recursive filter of
the domain transform, guided by the left image) are pinned here by facts that do not
re-type the oracle's loops: hand-computed codes, invariances, a mirror identity of the
matching geometry, a library recursive filter (scipy.signal.lfilter) for a uniform guide,
the variance-splitting property of the iteration schedule, edge separation, linearity
and bounds."""
import numpy as np
import pytest
import scipy.signal

import oracle


def test_census_hand_computed_centre():
    # 3 x 3 ramp: the centre (5) is larger than 1, 2, 3, 4 (first four offsets in raster
    # order); the reversed ramp's centre is larger than the last four.  Their codes differ
    # in all 8 bits.
    S = np.arange(1, 10, dtype=np.int32).reshape(3, 3)
    C = oracle.census_volume(S, 10 - S, 3, 1)
    assert C[1, 1, 0] == 8.0
    assert oracle.census_volume(S, S, 3, 1)[1, 1, 0] == 0.0
    # corner (0, 0) with clamping: the window reads 1 1 2 / 1 1 2 / 4 4 5 around the value 1,
    # nothing is smaller; in 10 - S the corner 9 sees 9 9 8 / 9 9 8 / 6 6 5: five smaller.
    assert C[0, 0, 0] == 5.0


@pytest.mark.parametrize("kc", [3, 5, 7])
def test_census_invariant_under_increasing_maps(kc):
    rng = np.random.default_rng(kc)
    SL = rng.integers(0, 4081, size=(9, 23), dtype=np.int32)
    SR = rng.integers(0, 4081, size=(9, 23), dtype=np.int32)
    ref = oracle.census_volume(SL, SR, kc, 6)
    for f in (lambda a: 3 * a + 7, lambda a: a * a, lambda a: 2 * a + 5 * (a > 2000)):  # strictly increasing
        np.testing.assert_array_equal(oracle.census_volume(f(SL), f(SR), kc, 6), ref)
    assert ref.min() >= 0 and ref.max() <= kc * kc - 1
    for d in range(6):
        assert np.all(ref[:, :d, d] == kc * kc - 1)


def test_census_zero_at_the_true_shift():
    rng = np.random.default_rng(5)
    h, w, s, kc = 7, 30, 4, 5
    r = kc // 2
    SL = rng.integers(0, 4081, size=(h, w), dtype=np.int32)
    SR = rng.integers(0, 4081, size=(h, w), dtype=np.int32)
    SR[:, :w - s] = SL[:, s:]          # R(x) = L(x + s): the match of L(x) is R(x - s)
    C = oracle.census_volume(SL, SR, kc, 8)
    assert np.all(C[:, s + r:w - r, s] == 0)
    assert np.all(oracle.census_volume(SL, SL, kc, 1) == 0)


def test_census_mirror_identity():
    # Flipping both images and swapping their roles maps the match of left (x, y) with right
    # (x - d, y) to the match of left' (w - 1 - x + d) with right' (w - 1 - x): same cost.
    rng = np.random.default_rng(9)
    h, w, D, kc = 6, 17, 5, 5
    SL = rng.integers(0, 4081, size=(h, w), dtype=np.int32)
    SR = rng.integers(0, 4081, size=(h, w), dtype=np.int32)
    C = oracle.census_volume(SL, SR, kc, D)
    M = oracle.census_volume(SR[:, ::-1].copy(), SL[:, ::-1].copy(), kc, D)
    for x in range(w):
        for d in range(min(D, x + 1)):
            np.testing.assert_array_equal(C[:, x, d], M[:, w - 1 - x + d, d])


def _rf_uniform(line, a):
    """Left-to-right then right-to-left first-order recursive filter with constant weight a,
    the first output equal to the first input: scipy's lfilter with the matching state."""
    b, den = [1.0 - a], [1.0, -a]
    f = scipy.signal.lfilter(b, den, line, zi=[a * line[0]])[0]
    g = scipy.signal.lfilter(b, den, f[::-1], zi=[a * f[-1]])[0]
    return g[::-1]


def _dt_uniform(C, sigmas):
    out = C.copy()
    for sig in sigmas:
        a = np.exp(-np.sqrt(2.0) / sig)
        out = np.apply_along_axis(_rf_uniform, 1, out, a)
        out = np.apply_along_axis(_rf_uniform, 0, out, a)
    return out


def test_dt_uniform_guide_is_a_recursive_filter():
    rng = np.random.default_rng(1)
    C = rng.random((7, 19, 3)) * 2.0
    g = np.full((7, 19), 1600, np.int32)
    s = 3.0
    # one iteration: the filter's scale is sigma_s itself
    np.testing.assert_allclose(oracle.dt_aggregate(C, g, s, 10.0, 1), _dt_uniform(C, [s]), rtol=0, atol=1e-12)
    # two iterations: the scales halve from one iteration to the next and their squares add
    # up to sigma_s^2, i.e. 2 s / sqrt(5) then s / sqrt(5)
    np.testing.assert_allclose(oracle.dt_aggregate(C, g, s, 10.0, 2),
                               _dt_uniform(C, [2 * s / np.sqrt(5), s / np.sqrt(5)]), rtol=0, atol=1e-12)


def test_dt_keeps_constant_slices_and_bounds():
    rng = np.random.default_rng(2)
    g = rng.integers(0, 4081, size=(8, 13), dtype=np.int32)
    C = np.broadcast_to(np.array([0.25, 1.5, 2.0]), (8, 13, 3)).copy()
    np.testing.assert_allclose(oracle.dt_aggregate(C, g, 5.0, 20.0, 3), C, rtol=0, atol=1e-12)
    R = rng.random((8, 13, 3))
    out = oracle.dt_aggregate(R, g, 5.0, 20.0, 3)
    for d in range(3):
        assert out[..., d].min() >= R[..., d].min() - 1e-12 and out[..., d].max() <= R[..., d].max() + 1e-12


def test_dt_hard_edge_separates_the_sides():
    # sigma_r -> 0 makes the transformed distance across an intensity edge infinite: the
    # two sides of a vertical edge are filtered as if they were separate images
    rng = np.random.default_rng(4)
    h, w, c = 6, 16, 7
    g = np.zeros((h, w), np.int32)
    g[:, c:] = 4080
    C = rng.random((h, w, 2))
    out = oracle.dt_aggregate(C, g, 4.0, 1e-9, 2)
    np.testing.assert_allclose(out[:, :c], oracle.dt_aggregate(C[:, :c].copy(), g[:, :c].copy(), 4.0, 1e-9, 2),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, c:], oracle.dt_aggregate(C[:, c:].copy(), g[:, c:].copy(), 4.0, 1e-9, 2),
                               rtol=0, atol=1e-12)


def test_dt_is_linear_in_the_cost():
    rng = np.random.default_rng(6)
    g = rng.integers(0, 4081, size=(5, 11), dtype=np.int32)
    A, B = rng.random((5, 11, 4)), rng.random((5, 11, 4))
    lhs = oracle.dt_aggregate(2.0 * A - 0.5 * B, g, 6.0, 15.0, 2)
    rhs = 2.0 * oracle.dt_aggregate(A, g, 6.0, 15.0, 2) - 0.5 * oracle.dt_aggregate(B, g, 6.0, 15.0, 2)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)
