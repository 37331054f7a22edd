"""Pins of the oracle's FP8 (E4M3) quantised refinement (Sec. V future work), on the CPU.

The E4M3 rounding is checked against torch's float8_e4m3fn conversion over the finite
range (round to nearest, ties to even) and against the saturation the form defines above
448; the quantised network with its roundings switched off must equal the plain FP64
refinement (the phase-folded decoder interior plus the unfolded border recompute is the
nearest-x2 convolution); with them on, the activations it passes between layers lie on
the E4M3 grid (d3 on the BF16 grid)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_11566_gb300 import synth


def test_e4m3_matches_torch_float8():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-448, 448, 4000), rng.uniform(-1, 1, 4000), rng.uniform(-0.02, 0.02, 4000),
                        np.ldexp(rng.uniform(-1, 1, 2000), -8)]).astype(np.float32)
    # exact ties: midpoints between neighbouring E4M3 values (ties go to the even code)
    grid = torch.arange(0, 127, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    grid = grid[np.isfinite(grid)]
    mids = ((grid[1:] + grid[:-1]) / 2).astype(np.float32)
    x = np.concatenate([x, mids, -mids, np.float32([0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10])])
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    got = np.array([oracle.e4m3(float(v)) for v in x])
    np.testing.assert_array_equal(got, want)
    for big in (448.0, 449.0, 464.0, 1e6):
        assert oracle.e4m3(big) == 448.0 and oracle.e4m3(-big) == -448.0


@pytest.mark.parametrize("W,H", [(128, 64), (130, 75), (250, 131)])
def test_quantised_form_without_rounding_is_the_plain_refinement(W, H):
    shape = synth.NET_WIDE
    params = synth.he_normal_weights(shape, 7)
    p = synth.make_pair(W, H, 40.0, 600 + W)
    rng = np.random.default_rng(W)
    coarse = rng.integers(0, 12, size=(H // 4, W // 4)).astype(np.float64)
    a = oracle.refine_forward_q(shape, params, p.left, coarse, quant=False)["Y"]
    b = oracle.refine_forward(shape, params, p.left, coarse)["Y"]
    # the folded weights are FP32 sums (as the GPU packs them): ~1e-7 relative on a decoder
    # output; a wrong phase, tap or border pixel would be off by whole pixels
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-5)


def test_quantised_activations_lie_on_the_grids():
    shape = synth.NET_WIDE
    params = synth.he_normal_weights(shape, 7)
    p = synth.make_pair(130, 75, 40.0, 700)
    coarse = np.full((75 // 4, 130 // 4), 5.0)
    for name in ("e1", "e2", "e3", "z", "d1", "d2"):
        a = oracle.refine_forward_q(shape, params, p.left, coarse, act=name)[name]
        sample = a.ravel()[:: max(1, a.size // 3000)]
        assert all(oracle.e4m3(v) == v for v in sample), name
        assert np.abs(a).max() <= 448.0
    d3 = oracle.refine_forward_q(shape, params, p.left, coarse, act="d3")["d3"]
    bf = torch.from_numpy(d3.astype(np.float32)).bfloat16().double().numpy()
    np.testing.assert_array_equal(d3, bf)
