"""GPU parity of the FP8 (E4M3) form, the quantised refinement of Sec. V, against the
oracle's quantised refinement, through the C ABI.

Layer by layer: each quantised layer's output (enc2 .. dec2) is compared with the oracle's
same layer (`oracle.qconv_layer`: per-output-channel weight scales, E4M3 weight codes, FP64
sums) applied to the GPU's own input codes, so that a wrong scale, code, byte layout, phase,
tap or border pixel shows in the layer where it happens.  The GPU sums E4M3 products in
FP32 on the tensor cores, the oracle in FP64: a value within a few FP32 ulps of a rounding
midpoint can land on either side.  Bar: at most 1e-3 of a layer's codes differ, and each
differing code is a neighbour on its grid (E4M3; dec2's output: BF16).  The last decoder
layer runs as in the BF16 form (BF16 weights): its d3 against the oracle's unquantised layer
on the GPU's own d2, within the BF16 form's layer bar (3 % of the largest magnitude).

End to end (refined disparity against `oracle.refine_forward_q` on the same coarse map):
such single-step differences propagate through the later layers, so the bar is statistical
-- mean |dY| <= 0.005 px, max |dY| <= 0.25 px, EPE within 0.01 px of the oracle's -- where
the quantisation itself moves the disparity by about 0.03 px on average and 0.25 px at most
from the unquantised FP64 refinement (measured: 0.0013 / 0.10 px against the quantised
oracle at 1242 x 375)."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SHAPE = synth.NET_WIDE
CODE_DIFF_FRAC = 1e-3
MEAN_PX, MAX_PX, EPE_PX = 0.005, 0.25, 0.01
QUANT_MEAN_PX = 0.1  # the FP8 form against the unquantised FP64 refinement (quantisation error)


@pytest.fixture(scope="module")
def ctx(svlib):
    c = binding.Context(SHAPE, 5, "fp8")
    c.set_weights(synth.he_normal_weights(SHAPE, 7))
    yield c
    c.close()


def act_shape(H, W, name):
    L0, L1, L2, L3 = oracle.level_sizes(H, W)
    c1, c2, c3 = SHAPE.enc
    d1, d2, d3 = SHAPE.dec
    return {"e1": (*L1, c1), "e2": (*L2, c2), "e3": (*L3, c3), "z": (*L3, SHAPE.latent), "d1": (*L2, d1),
            "d2": (*L1, d2), "d3": (*L0, d3)}[name]


def e4m3_ordinal(v):
    """Position of E4M3 values on the signed grid (neighbours differ by 1)."""
    c = torch.from_numpy(np.asarray(v, dtype=np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    mag = (c & 0x7F).astype(np.int64)
    return np.where(c & 0x80, -mag, mag)


def bf16_ordinal(v):
    u = torch.from_numpy(np.asarray(v, dtype=np.float32)).bfloat16().view(torch.int16).numpy().astype(np.int64)
    mag = u & 0x7FFF
    return np.where(u < 0, -mag, mag)


def check_codes(g, o, ordinal, label):
    """g, o: values on the same grid; at most CODE_DIFF_FRAC differ, each by one grid step."""
    diff = g != o
    frac = diff.mean()
    assert frac <= CODE_DIFF_FRAC, f"{label}: {frac:.2e} of the codes differ"
    if diff.any():
        steps = np.abs(ordinal(g[diff]) - ordinal(o[diff]))
        assert steps.max() <= 1, f"{label}: a code differs by {steps.max()} grid steps"


def layer_weights(params, name):
    ow, wshape, ob, co = oracle.param_slices(SHAPE)[name]
    return params[ow:ow + int(np.prod(wshape))].reshape(wshape), params[ob:ob + co]


@pytest.mark.parametrize("W,H,D,enc1_tc", [(256, 128, 16, 1), (333, 97, 24, 1), (250, 131, 20, 1), (333, 97, 24, 0)])
def test_fp8_layers_match_the_quantised_oracle(ctx, W, H, D, enc1_tc):
    """enc1_tc 1: the tensor-core first layer writes the E4M3 codes of e1 itself; 0: the
    CUDA-core first layer writes BF16 and a separate kernel converts it."""
    p = synth.make_pair(W, H, 50.0, 8100 + W)
    disp_o = oracle.coarse_match(p.left, p.right, 5, D)[0]
    params = synth.he_normal_weights(SHAPE, 7)
    dp = binding.to_device(p, D)
    ctx.set_option("enc1_tensor", enc1_tc)
    ctx.set_option("fused_final", 0)  # keep d3 in HBM so that it can be compared
    try:
        Y = ctx.refine([dp], [torch.from_numpy(disp_o.astype(np.int16)).cuda()])[0]
        ctx.synchronize()
    finally:
        ctx.set_option("enc1_tensor", 1)
        ctx.set_option("fused_final", 1)
    g = {a: ctx.debug_activation(i, 0, act_shape(H, W, a)).astype(np.float64)
         for i, a in enumerate(["e1", "e2", "e3", "z", "d1", "d2", "d3"])}
    # e1: E4M3 codes of the first layer's BF16-rounded output, against the oracle's
    e1_o = oracle.refine_forward_q(SHAPE, params, p.left, disp_o.astype(np.float64), act="e1")["e1"]
    check_codes(g["e1"], e1_o, e4m3_ordinal, f"{W}x{H} enc1")
    (_, _), L1, L2, L3 = oracle.level_sizes(H, W)
    chain = [("enc2", g["e1"], "e2", 0, L2, "e4m3", True), ("enc3", g["e2"], "e3", 0, L3, "e4m3", True),
             ("mu", g["e3"], "z", 1, L3, "e4m3", False), ("dec1", g["z"], "d1", 2, L2, "e4m3", True),
             ("dec2", g["d1"], "d2", 2, L1, "bf16", True)]
    for name, x, out, mode, hw, rnd, relu in chain:
        wt, b = layer_weights(params, name)
        o = oracle.qconv_layer(x, wt, b, mode, hw, relu=relu, out_round=rnd)
        check_codes(g[out], o, e4m3_ordinal if rnd == "e4m3" else bf16_ordinal, f"{W}x{H} {name}")
    wt, b = layer_weights(params, "dec3")
    o = oracle.qconv_layer(g["d2"], wt, b, 2, (H, W), relu=True, out_round="bf16", quant_weights=False)
    assert np.abs(g["d3"] - o).max() <= 3e-2 * np.abs(o).max(), f"{W}x{H} dec3"
    # the refined disparity against the oracle's whole quantised forward
    refq = oracle.refine_forward_q(SHAPE, params, p.left, disp_o.astype(np.float64))["Y"]
    keep = np.ones((H, W), dtype=bool)
    parity.compare_refined(Y.cpu().numpy(), refq, keep, MAX_PX, MEAN_PX, p.gt, EPE_PX, f"fp8 {W}x{H}")


def test_fp8_full_size_against_the_quantised_and_plain_oracle(ctx):
    """1242 x 375 through the default plan (the last decoder layer fused with the final conv)."""
    W, H, D = 1242, 375, 48
    p = synth.make_pair(W, H, 60.0, 8300)
    disp_o = oracle.coarse_match(p.left, p.right, 5, D)[0]
    params = synth.he_normal_weights(SHAPE, 7)
    Y = ctx.refine([binding.to_device(p, D)], [torch.from_numpy(disp_o.astype(np.int16)).cuda()])[0]
    ctx.synchronize()
    Yg = Y.cpu().numpy().astype(np.float64)
    refq = oracle.refine_forward_q(SHAPE, params, p.left, disp_o.astype(np.float64))["Y"]
    keep = np.ones((H, W), dtype=bool)
    parity.compare_refined(Yg, refq, keep, MAX_PX, MEAN_PX, p.gt, EPE_PX, "fp8 1242x375")
    ref = oracle.refine_forward(SHAPE, params, p.left, disp_o.astype(np.float64))
    assert np.abs(Yg - ref["Y"]).mean() <= QUANT_MEAN_PX


def test_fp8_batched_graph_pipeline(ctx):
    """Ragged pairs in one batched call, captured into a CUDA graph and replayed; every pair
    against the quantised oracle on the oracle's own WTA map (outside the reach of near ties)."""
    sizes = [(256, 128, 16), (333, 97, 24), (250, 131, 20), (75, 37, 8)]
    pairs = [synth.make_pair(W, H, 40.0, 8500 + i) for i, (W, H, _) in enumerate(sizes)]
    dps = [binding.to_device(p, D) for p, (_, _, D) in zip(pairs, sizes)]
    params = synth.he_normal_weights(SHAPE, 7)
    s = torch.cuda.Stream()
    outs = [torch.empty((p.height, p.width), dtype=torch.float32, device="cuda") for p in pairs]
    with torch.cuda.stream(s):
        ctx.pipeline(dps, out=outs)          # capture + first replay
        first = [o.clone() for o in outs]
        for o in outs:
            o.fill_(-1)
        ctx.pipeline(dps, out=outs)          # replay
    s.synchronize()
    ctx.synchronize(s)
    for a, b in zip(outs, first):
        assert torch.equal(a, b)
    coarse = ctx.coarse_match(dps)
    for p, (_, _, D), o, d in zip(pairs, sizes, outs, coarse):
        disp_o, best_o, sec_o = oracle.coarse_match(p.left, p.right, 5, D)
        keep = parity.keep_mask(parity.wta_differences(d.cpu().numpy(), disp_o, best_o, sec_o), p.height, p.width)
        refq = oracle.refine_forward_q(SHAPE, params, p.left, disp_o.astype(np.float64))["Y"]
        parity.compare_refined(o.cpu().numpy(), refq, keep, MAX_PX, MEAN_PX, p.gt, EPE_PX,
                               f"fp8 graph {p.width}x{p.height}")


def test_fp8_autotuned_plans_give_the_same_result(svlib):
    """Tuned launch shapes (strip heights, N slices, CTAs per SM) change no arithmetic of an
    output element: the tuned batch must equal the untuned one bit for bit, with the decoder
    tail fused and unfused."""
    pairs = synth.batch_uneven(6, seed=8800)
    dps = [binding.to_device(p, D) for p, D in pairs]
    s = torch.cuda.Stream()
    plain = binding.Context(SHAPE, 9, "fp8")
    tuned = binding.Context(SHAPE, 9, "fp8")
    try:
        for c in (plain, tuned):
            c.set_weights(synth.he_normal_weights(SHAPE, 7))
        tuned.autotune(dps, stream=s)
        for fused in (1, 0):
            outs = []
            for c in (plain, tuned):
                c.set_option("fused_final", fused)
                with torch.cuda.stream(s):
                    o = c.pipeline(dps)
                s.synchronize()
                c.synchronize(s)
                outs.append([x.clone() for x in o])
            for a, b in zip(*outs):
                assert torch.equal(a, b), f"fused_final {fused}"
    finally:
        plain.close()
        tuned.close()


def test_fp8_is_inference_only(ctx):
    p = synth.make_pair(128, 64, 20.0, 8700)
    dp = binding.to_device(p, 8)
    h3, w3 = binding.latent_hw(64, 128)
    coarse = torch.zeros((16, 32), dtype=torch.float32, device="cuda")
    eps = torch.zeros((h3, w3, SHAPE.latent), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.SvError) as ei:
        ctx.refine_train([dp], [coarse], [eps])
    assert ei.value.status == binding.SV_ERR_UNSUPPORTED
