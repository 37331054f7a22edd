"""GPU parity of the BF16 tensor-core form (tcgen05 implicit-GEMM convolutions) against
the FP64 oracle, through the C ABI.

Bar for the refined disparity: max |dY| <= 0.05 px, mean |dY| <= 0.01 px and an EPE
(against the synthetic ground truth) within 0.01 px of the oracle's.  Each BF16
activation is also compared layer by layer with the oracle's FP64 activation (relative
to its largest magnitude), so a wrong tap, phase or channel slice shows up where it
happens."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MAX_PX, MEAN_PX, EPE_PX = 0.05, 0.01, 0.01
LAYER_REL = 3e-2
ACTS = ["e1", "e2", "e3", "z", "d1", "d2", "d3"]


@pytest.fixture(scope="module")
def contexts(svlib):
    made = {}

    def get(shape, k):
        if (shape, k) not in made:
            c = binding.Context(shape, k, "bf16")
            c.set_weights(synth.he_normal_weights(shape, 7))
            made[(shape, k)] = c
        return made[(shape, k)]
    yield get
    for c in made.values():
        c.close()


def act_shape(shape, H, W, name):
    L0, L1, L2, L3 = oracle.level_sizes(H, W)
    c1, c2, c3 = shape.enc
    d1, d2, d3 = shape.dec
    return {"e1": (*L1, c1), "e2": (*L2, c2), "e3": (*L3, c3), "z": (*L3, shape.latent), "d1": (*L2, d1),
            "d2": (*L1, d2), "d3": (*L0, d3)}[name]


def check_output(Yg, ref, gt, label):
    d = np.abs(Yg - ref["Y"])
    assert d.max() <= MAX_PX, f"{label}: max |dY| = {d.max():.4f}"
    assert d.mean() <= MEAN_PX, f"{label}: mean |dY| = {d.mean():.5f}"
    epe_g = np.abs(Yg - gt).mean()
    epe_o = np.abs(ref["Y"] - gt).mean()
    assert abs(epe_g - epe_o) <= EPE_PX, label


@pytest.mark.parametrize("name,shape,W,H,dmax,k,D", [
    ("256x128 small net", synth.NET_SMALL, 256, 128, 60.0, 7, 16),
    ("ragged 250x131 small net", synth.NET_SMALL, 250, 131, 50.0, 5, 20),
    ("ragged 333x97 wide net", synth.NET_WIDE, 333, 97, 60.0, 5, 24),
])
def test_bf16_layers_match_oracle(contexts, name, shape, W, H, dmax, k, D):
    p = synth.make_pair(W, H, dmax, 7000 + W)
    disp_o = oracle.coarse_match(p.left, p.right, k, D)[0]
    params = synth.he_normal_weights(shape, 7)
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    ctx.set_option("fused_final", 0)  # keep d3 in HBM so that it can be compared
    try:
        Y = ctx.refine([dp], [torch.from_numpy(disp_o.astype(np.int16)).cuda()])[0]
        ctx.synchronize()
    finally:
        ctx.set_option("fused_final", 1)
    for wi, a in enumerate(ACTS):
        g = ctx.debug_activation(wi, 0, act_shape(shape, H, W, a))
        ref = oracle.refine_activation(shape, params, p.left, disp_o.astype(np.float64), a)
        scale = max(1e-6, np.abs(ref).max())
        err = np.abs(g - ref).max() / scale
        assert err <= LAYER_REL, f"{name}: layer {a} rel err {err:.4f}"
    ref = oracle.refine_forward(shape, params, p.left, disp_o.astype(np.float64))
    check_output(Y.cpu().numpy().astype(np.float64), ref, p.gt, name)


@pytest.mark.parametrize("name,shape,W,H,dmax,k,D", [
    ("1242x375 wide net", synth.NET_WIDE, 1242, 375, 190.0, 9, 48),
    ("1242x375 small net", synth.NET_SMALL, 1242, 375, 190.0, 9, 48),
])
def test_bf16_refine_full_size(contexts, name, shape, W, H, dmax, k, D):
    p = synth.make_pair(W, H, dmax, 7100 + W)
    disp_o = oracle.coarse_match(p.left, p.right, k, D)[0]
    ref = oracle.refine_forward(shape, synth.he_normal_weights(shape, 7), p.left, disp_o.astype(np.float64))
    ctx = contexts(shape, k)
    Y = ctx.refine([binding.to_device(p, D)], [torch.from_numpy(disp_o.astype(np.int16)).cuda()])[0]
    ctx.synchronize()
    check_output(Y.cpu().numpy().astype(np.float64), ref, p.gt, name)


def test_bf16_uneven_batch_one_call(contexts):
    """Pairs of widths {320, 640, 960, 1242} refined together (one launch per layer)."""
    shape, k = synth.NET_WIDE, 9
    batch = synth.batch_uneven(6, seed=7300)
    params = synth.he_normal_weights(shape, 7)
    ctx = contexts(shape, k)
    coarse, dps, refs = [], [], []
    for p, D in batch:
        d = oracle.coarse_match(p.left, p.right, k, D)[0]
        coarse.append(torch.from_numpy(d.astype(np.int16)).cuda())
        dps.append(binding.to_device(p, D))
        refs.append(oracle.refine_forward(shape, params, p.left, d.astype(np.float64)))
    Ys = ctx.refine(dps, coarse)
    ctx.synchronize()
    for (p, D), Y, ref in zip(batch, Ys, refs):
        check_output(Y.cpu().numpy().astype(np.float64), ref, p.gt, f"{p.width}x{p.height}")


def test_bf16_pipeline(contexts):
    shape, k, D = synth.NET_WIDE, 9, 48
    p = synth.make_pair(1242, 375, 190.0, 7400)
    params = synth.he_normal_weights(shape, 7)
    Y_o, disp_o, best_o, sec_o = oracle.pipeline(shape, params, p.left, p.right, k, D)
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    Y = ctx.pipeline([dp])[0]
    dg = ctx.coarse_match([dp])[0].cpu().numpy()
    ctx.synchronize()
    keep = parity.keep_mask(parity.wta_differences(dg, disp_o, best_o, sec_o), 375, 1242)
    parity.compare_refined(Y.cpu().numpy(), Y_o, keep, MAX_PX, MEAN_PX, p.gt, EPE_PX, "BF16 pipeline 1242x375")


def test_device_wait_timeout_is_reported_and_recoverable(contexts):
    """A one-cycle spin limit makes every bounded wait of the tensor-core kernels give up:
    the kernels record the failure and return, sv_synchronize reports SV_ERR_TIMEOUT,
    and the context works again with the default limit.  No fault, no hang."""
    shape, k, D = synth.NET_SMALL, 7, 16
    p = synth.make_pair(256, 128, 60.0, 7500)
    disp_o = oracle.coarse_match(p.left, p.right, k, D)[0]
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    coarse = torch.from_numpy(disp_o.astype(np.int16)).cuda()
    ctx.set_option("spin_limit", 1)
    try:
        ctx.refine([dp], [coarse])
        with pytest.raises(binding.SvError) as ei:
            ctx.synchronize()
        assert ei.value.status == binding.SV_ERR_TIMEOUT
    finally:
        ctx.set_option("spin_limit", 4000000000)
    ctx.synchronize()
    Y = ctx.refine([dp], [coarse])[0]
    ctx.synchronize()
    ref = oracle.refine_forward(shape, synth.he_normal_weights(shape, 7), p.left, disp_o.astype(np.float64))
    check_output(Y.cpu().numpy().astype(np.float64), ref, p.gt, "after timeout")


@pytest.mark.parametrize("name,shape,W,H,dmax,k,D,rows", [
    ("1242x375 wide net, default strips", synth.NET_WIDE, 1242, 375, 190.0, 9, 48, 0),
    ("1242x375 wide net, 7-row strips", synth.NET_WIDE, 1242, 375, 190.0, 9, 48, 7),
    ("256x128 small net, 5-row strips", synth.NET_SMALL, 256, 128, 60.0, 7, 16, 5),
])
def test_bf16_fused_final(contexts, name, shape, W, H, dmax, k, D, rows):
    """The fused last-decoder-layer + final-conv kernel (d3 kept in shared memory, final conv
    on the tensor cores; odd output height handled by negated-weight MMAs on the last row,
    even height by the carried sums below; column strips overlapping by one input pixel;
    halo tiles above row strips) against the unfused kernels of the same context and
    against the FP64 oracle."""
    p = synth.make_pair(W, H, dmax, 8100 + W + rows)
    disp_o = oracle.coarse_match(p.left, p.right, k, D)[0]
    params = synth.he_normal_weights(shape, 7)
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    cm = [torch.from_numpy(disp_o.astype(np.int16)).cuda()]
    ctx.set_option("tc_strip_rows", rows)
    try:
        ctx.set_option("fused_final", 0)
        Yu = ctx.refine([dp], cm)[0].cpu().numpy().astype(np.float64)
        ctx.set_option("fused_final", 1)
        Yf = ctx.refine([dp], cm)[0].cpu().numpy().astype(np.float64)
        ctx.synchronize()
        with pytest.raises(binding.SvError):  # d3 was not materialised
            ctx.debug_activation(6, 0, act_shape(shape, H, W, "d3"))
    finally:
        ctx.set_option("tc_strip_rows", 0)
        ctx.set_option("fused_final", 1)
    d = np.abs(Yf - Yu)
    assert d.max() <= 5e-3, f"{name}: fused vs unfused max |dY| = {d.max():.2e}"
    ref = oracle.refine_forward(shape, params, p.left, disp_o.astype(np.float64))
    check_output(Yf, ref, p.gt, name)


def test_bf16_kernel_variants_agree(contexts):
    """Variants of the same layers behind options: the channel-block staging ring of dec1
    (split_rows) must give bit-identical results to whole-row staging (same MMAs, same
    order); enc1 on the tensor cores (high/low BF16 parts, FP32 accumulation) against the
    CUDA-core FP32 kernel: e1 within one BF16 rounding, and both refined outputs at the
    oracle's bar."""
    shape, W, H, dmax, k, D = synth.NET_WIDE, 333, 97, 60.0, 5, 24
    p = synth.make_pair(W, H, dmax, 7400)
    disp_o = oracle.coarse_match(p.left, p.right, k, D)[0]
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    cm = [torch.from_numpy(disp_o.astype(np.int16)).cuda()]
    out = {}
    try:
        for key, val in (("split_rows", 0), ("split_rows", 1), ("enc1_tensor", 0), ("enc1_tensor", 1)):
            ctx.set_option(key, val)
            y = ctx.refine([dp], cm)[0].cpu().numpy().astype(np.float64)
            ctx.synchronize()
            out[(key, val)] = (y, ctx.debug_activation(0, 0, act_shape(shape, H, W, "e1")))
    finally:
        ctx.set_option("split_rows", 1)
        ctx.set_option("enc1_tensor", 1)
    assert np.array_equal(out[("split_rows", 0)][0], out[("split_rows", 1)][0])
    e_t, e_c = out[("enc1_tensor", 1)][1], out[("enc1_tensor", 0)][1]
    scale = np.abs(e_c).max()
    assert np.abs(e_t - e_c).max() <= scale * 2.0 ** -7, "enc1 tensor-core vs CUDA-core"
    ref = oracle.refine_forward(shape, synth.he_normal_weights(shape, 7), p.left, disp_o.astype(np.float64))
    for v in (0, 1):
        check_output(out[("enc1_tensor", v)][0], ref, p.gt, f"enc1_tensor {v}")
