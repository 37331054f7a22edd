"""Pins of the oracle's FP8 (E4M3) quantised refinement (Sec. V future work), on the CPU.

The E4M3 rounding is checked against torch's float8_e4m3fn conversion over the finite
range (round to nearest, ties to even) and against the saturation the form defines above
448; the quantised network with its roundings switched off must equal the plain FP64
refinement (the phase-folded decoder interior plus the unfolded border recompute is the
nearest-x2 convolution); with them on, the activations it passes between layers lie on
the E4M3 grid (d2 and d3, the last decoder layer's input and output, on the BF16 grid)."""
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
    for name in ("e1", "e2", "e3", "z", "d1"):
        a = oracle.refine_forward_q(shape, params, p.left, coarse, act=name)[name]
        sample = a.ravel()[:: max(1, a.size // 3000)]
        assert all(oracle.e4m3(v) == v for v in sample), name
        assert np.abs(a).max() <= 448.0
    for name in ("d2", "d3"):
        a = oracle.refine_forward_q(shape, params, p.left, coarse, act=name)[name]
        bf = torch.from_numpy(a.astype(np.float32)).bfloat16().double().numpy()
        np.testing.assert_array_equal(a, bf, err_msg=name)


def _grid_weights(rng, co, k, ci):
    """Weights E4M3 value x 2^-8 with every output channel reaching 448 x 2^-8."""
    grid = torch.arange(0, 127, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    grid = grid[np.isfinite(grid)]
    c = rng.choice(np.concatenate([grid, -grid]), size=(co, k, k, ci))
    c.reshape(co, -1)[:, 0] = 448.0
    return (c * 2.0 ** -8).astype(np.float32)


@pytest.mark.parametrize("mode,k,stride", [(0, 3, 2), (1, 1, 1)])
def test_qconv_layer_with_exact_codes_is_conv2d(mode, k, stride):
    rng = np.random.default_rng(5 + mode)
    co, ci, Hi, Wi = 24, 16, 13, 18
    wt = _grid_weights(rng, co, k, ci)
    b = rng.normal(size=co).astype(np.float32)
    x = rng.normal(size=(Hi, Wi, ci))
    Ho, Wo = ((Hi + 1) // 2, (Wi + 1) // 2) if mode == 0 else (Hi, Wi)
    got = oracle.qconv_layer(x, wt, b, mode, (Ho, Wo), relu=False, out_round="none")
    xt = torch.from_numpy(x).permute(2, 0, 1)[None]
    wt_t = torch.from_numpy(wt.astype(np.float64)).permute(0, 3, 1, 2)
    want = torch.nn.functional.conv2d(xt, wt_t, torch.from_numpy(b.astype(np.float64)), stride=stride,
                                      padding=k // 2)[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_qconv_layers_chain_to_the_quantised_forward():
    shape = synth.NET_WIDE
    params = synth.he_normal_weights(shape, 7)
    H, W = 75, 130
    p = synth.make_pair(W, H, 40.0, 701)
    coarse = np.random.default_rng(3).integers(0, 12, size=(H // 4, W // 4)).astype(np.float64)
    sl = oracle.param_slices(shape)
    (_, _), L1, L2, L3 = oracle.level_sizes(H, W)
    acts = {a: oracle.refine_forward_q(shape, params, p.left, coarse, act=a)[a]
            for a in ("e1", "e2", "e3", "z", "d1", "d2", "d3")}
    chain = [("enc2", "e1", "e2", 0, L2, "e4m3", True, True), ("enc3", "e2", "e3", 0, L3, "e4m3", True, True),
             ("mu", "e3", "z", 1, L3, "e4m3", False, True), ("dec1", "z", "d1", 2, L2, "e4m3", True, True),
             ("dec2", "d1", "d2", 2, L1, "bf16", True, True), ("dec3", "d2", "d3", 2, (H, W), "bf16", True, False)]
    names = [n for n, *_ in shape.layers()]
    for layer, a_in, a_out, mode, hw, rnd, relu, qw in chain:
        assert layer in names, layer
        ow, wshape, ob, co = sl[layer]
        wt = params[ow:ow + int(np.prod(wshape))].reshape(wshape)
        b = params[ob:ob + co]
        got = oracle.qconv_layer(acts[a_in], wt, b, mode, hw, relu=relu, out_round=rnd, quant_weights=qw)
        np.testing.assert_array_equal(got, acts[a_out], err_msg=layer)
