"""GPU parity of the coarse matcher (sv_coarse_match: 4x4 box downsample, ZNCC Eq. 1-3,
WTA Eq. 6) against the FP64 oracle, through the C ABI.

Bar: integer disparities bit-exact wherever the oracle's best and second-best scores
differ by more than 1e-4; |d rho| <= 1e-5 on the best and second-best scores
everywhere."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MARGIN = 1e-4
RHO_TOL = 1e-5


def gpu_coarse(ctx, pairs_np, Ds):
    dps = [binding.to_device(p, D) for p, D in zip(pairs_np, Ds)]
    disp, best, second = ctx.coarse_match(dps, scores=True)
    torch.cuda.synchronize()
    return [(d.cpu().numpy().astype(np.int32), b.cpu().numpy(), s.cpu().numpy()) for d, b, s in
            zip(disp, best, second)]


def check(gpu, orc, label=""):
    dg, bg, sg = gpu
    do, bo, so = orc
    assert dg.shape == do.shape, label
    clear = (bo - so) > MARGIN
    bad = clear & (dg != do)
    assert not bad.any(), f"{label}: {bad.sum()} WTA mismatches where the margin is > 1e-4"
    assert np.abs(bg - bo).max() <= RHO_TOL, label
    assert np.abs(sg - so).max() <= RHO_TOL, label
    return int((dg != do).sum())


@pytest.fixture(scope="module")
def ctx_factory(svlib):
    made = {}

    def get(window):
        if window not in made:
            made[window] = binding.Context(synth.NET_SMALL, window, "fp32")
        return made[window]
    yield get
    for c in made.values():
        c.close()


@pytest.mark.parametrize("name,W,H,dmax,k,D", [
    ("256x128 k7 D16", 256, 128, 60.0, 7, 16),
    ("1242x375 k9 D48", 1242, 375, 190.0, 9, 48),
    ("ragged 258x131 k5 D33", 258, 131, 120.0, 5, 33),
    ("k3 D65", 400, 96, 200.0, 3, 65),
    ("k15 D100", 640, 193, 300.0, 15, 100),
    ("D128", 1024, 64, 400.0, 11, 128),
    ("D1", 256, 64, 30.0, 7, 1),
    ("minimum size 28x28 k7 D7", 28, 28, 10.0, 7, 7),
    ("D = w", 128, 64, 100.0, 5, 32),
])
def test_coarse_matches_oracle(ctx_factory, name, W, H, dmax, k, D):
    p = synth.make_pair(W, H, dmax, 3000 + W + H + k)
    g = gpu_coarse(ctx_factory(k), [p], [D])[0]
    o = oracle.coarse_match(p.left, p.right, k, D)
    flips = check(g, o, name)
    assert flips <= max(2, g[0].size // 1000), name


def test_coarse_batch_of_uneven_pairs_in_one_call(ctx_factory):
    """Pairs of widths {320, 640, 960, 1242} with D = ceil(W / 26), one launch."""
    batch = synth.batch_uneven(8, seed=2100)
    pairs = [p for p, _ in batch]
    Ds = [D for _, D in batch]
    gs = gpu_coarse(ctx_factory(9), pairs, Ds)
    for (p, D), g in zip(batch, gs):
        check(g, oracle.coarse_match(p.left, p.right, 9, D), f"{p.width}x{p.height}")


def test_constant_shift_recovered_exactly(ctx_factory):
    p = synth.make_pair(512, 128, 0.0, 99)
    s = 9
    L = p.left
    R = np.zeros_like(L)
    R[:, :512 - 4 * s] = L[:, 4 * s:]
    q = synth.Pair(L, R, p.gt, p.occ, 0)
    dg, bg, _ = gpu_coarse(ctx_factory(7), [q], [24])[0]
    r, w = 3, 128
    assert np.all(dg[:, s + r:w - r - s] == s)
    assert np.abs(bg[:, s + r:w - r - s] - 1.0).max() <= RHO_TOL


def test_exact_ties_take_lowest_d(ctx_factory):
    """A right image of period 8 px (2 coarse px) gives identical windows for d and
    d + 2: the lowest d must win, exactly as in the oracle."""
    rng = np.random.default_rng(5)
    W, H = 256, 64
    cols = rng.integers(0, 256, size=(H, 8), dtype=np.uint8)
    R = np.tile(cols, (1, W // 8))
    L = np.roll(R, 4, axis=1)  # L(X) = R(X - 4): coarse shift 1, ties at 3, 5, ...
    q = synth.Pair(L, R, np.zeros((H, W), np.float32), np.zeros((H, W), bool), 0)
    dg, bg, sg = gpu_coarse(ctx_factory(3), [q], [6])[0]
    do, bo, so = oracle.coarse_match(L, R, 3, 6)
    inner = (slice(None), slice(6, W // 4 - 1))
    assert np.all(do[inner] == 1)
    assert np.array_equal(dg[inner], do[inner])


def test_invalid_arguments_launch_nothing(ctx_factory, svlib):
    ctx = ctx_factory(7)
    p = synth.make_pair(128, 64, 20.0, 1)
    dp = binding.to_device(p, 8)
    out = torch.full((16, 32), -7, dtype=torch.int16, device="cuda")

    def call(sp, outs=(out,)):
        arr = (binding.SvPair * 1)(sp)
        ptrs = binding._ptrs(list(outs))
        return svlib.sv_coarse_match(ctx.handle, arr, 1, ptrs, None, None, None)

    base = dp.sv()
    cases = []
    sp = binding.SvPair.from_buffer_copy(base); sp.max_disp = 0; cases.append(sp)
    sp = binding.SvPair.from_buffer_copy(base); sp.max_disp = 33; cases.append(sp)     # > W / 4
    sp = binding.SvPair.from_buffer_copy(base); sp.pitch = 136; cases.append(sp)      # not a multiple of 16
    sp = binding.SvPair.from_buffer_copy(base); sp.left = None; cases.append(sp)
    sp = binding.SvPair.from_buffer_copy(base); sp.width = 20; cases.append(sp)        # < 4 * window
    sp = binding.SvPair.from_buffer_copy(base); sp.right = base.right + 4; cases.append(sp)  # misaligned
    for sp in cases:
        assert call(sp) == binding.SV_ERR_INVALID_ARG
    assert call(base, (None,)) == binding.SV_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((out == -7).all())
    # an empty batch is a no-op
    assert svlib.sv_coarse_match(ctx.handle, None, 0, None, None, None, None) == binding.SV_OK
    assert call(base) == binding.SV_OK
