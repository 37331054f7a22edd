"""GPU parity of the paper's Table I network (Sec. III-B1, Eq. 8) and its loss (Eq. 9-11)
against the FP64 oracle, through the C ABI (contexts created with SV_NET_TABLE1).

Bars: the refined disparity within 1e-4 px + 2e-6 max |Y|.  Unlike the small net's residual
output (1e-4 px on top of the exactly upsampled coarse map), the Table I network's output is
the disparity itself, 256 Y, with a scale of hundreds of pixels at random initialisation; 13
layers of FP32 sums of up to 2400 products each leave a few tens of FP32 ulps of that scale
(2e-6 of it, ~1e-3 px at 400 px).  mu and sigma within 1e-5; the loss within 1e-6 relative and
its gradients equal to their closed forms."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu

PARAMS = synth.table1_weights(7)


@pytest.fixture(scope="module")
def t1ctx(svlib):
    made = {}

    def get(k):
        if k not in made:
            c = binding.Context("table1", k, "fp32")
            c.set_weights(PARAMS)
            made[k] = c
        return made[k]
    yield get
    for c in made.values():
        c.close()


def close(got, want, label):
    err = np.abs(got.astype(np.float64) - want)
    bar = 1e-4 + 2e-6 * np.abs(want).max()
    assert (err <= bar).all(), f"{label}: max |dY| = {err.max():.3g} px, worst ratio {(err / bar).max():.3g}"


def test_param_count_and_layout(t1ctx):
    assert t1ctx(7).n_params == oracle.t1_param_count() == 162380
    assert np.array_equal(t1ctx(7).get_weights(), PARAMS)


@pytest.mark.parametrize("W,H,dmax,k,D", [(256, 128, 60.0, 7, 16), (1242, 375, 190.0, 9, 48),
                                          (250, 131, 50.0, 5, 20), (75, 37, 20.0, 3, 5)])
def test_t1_refine_matches_oracle(t1ctx, W, H, dmax, k, D):
    p = synth.make_pair(W, H, dmax, 12000 + W)
    disp_o = oracle.coarse_match(p.left, p.right, k, D)[0]
    ref = oracle.t1_forward(PARAMS, p.left, disp_o.astype(np.float64))
    ctx = t1ctx(k)
    Y = ctx.refine([binding.to_device(p, D)], [torch.from_numpy(disp_o.astype(np.int16)).cuda()])[0]
    close(Y.cpu().numpy(), 256.0 * ref["Y"], f"{W}x{H}")


def test_t1_uneven_batch_one_call(t1ctx):
    batch = synth.batch_uneven(5, seed=12100)
    ctx = t1ctx(9)
    dps, cms, refs = [], [], []
    for p, D in batch:
        d = oracle.coarse_match(p.left, p.right, 9, D)[0]
        dps.append(binding.to_device(p, D))
        cms.append(torch.from_numpy(d.astype(np.int16)).cuda())
        refs.append(oracle.t1_forward(PARAMS, p.left, d.astype(np.float64)))
    Ys = ctx.refine(dps, cms)
    for (p, _), Y, ref in zip(batch, Ys, refs):
        close(Y.cpu().numpy(), 256.0 * ref["Y"], f"{p.width}x{p.height}")


def test_t1_pipeline_against_oracle(t1ctx):
    """sv_pipeline on a Table I context: coarse match + the Table I refinement, compared
    outside the reach of WTA near ties."""
    p = synth.make_pair(1242, 375, 190.0, 12200)
    k, D = 9, 48
    d_o, b_o, s_o = oracle.coarse_match(p.left, p.right, k, D)
    ref = oracle.t1_forward(PARAMS, p.left, d_o.astype(np.float64))
    ctx = t1ctx(k)
    dp = binding.to_device(p, D)
    Y = ctx.pipeline([dp])[0]
    dg = ctx.coarse_match([dp])[0].cpu().numpy()
    keep = parity.keep_mask(parity.wta_differences(dg, d_o, b_o, s_o), 375, 1242, radius=24)
    err = np.abs(Y.cpu().numpy().astype(np.float64) - 256.0 * ref["Y"])[keep]
    assert err.max() <= 1e-4 + 2e-6 * np.abs(256.0 * ref["Y"]).max()


def test_t1_training_forward_with_noise(t1ctx):
    """sv_refine_train: the decoder input (mu - 1) + eps exp(sigma - 1) of Eq. 8."""
    W, H, k, D = 256, 128, 7, 16
    p = synth.make_pair(W, H, 60.0, 12300)
    rng = np.random.default_rng(4)
    coarse = (rng.random((H // 4, W // 4)) * 12.0).astype(np.float32)
    H8, W8 = oracle.t1_levels(H, W)[3]
    eps = synth.reparam_noise(H8 * W8, 77)
    ref = oracle.t1_forward(PARAMS, p.left, coarse.astype(np.float64), eps)
    ctx = t1ctx(k)
    Y, mu, sg = ctx.refine_train([binding.to_device(p, D)], [torch.from_numpy(coarse).cuda()],
                                 [torch.from_numpy(eps).cuda().reshape(H8, W8, 1)])
    close(Y[0].cpu().numpy(), 256.0 * ref["Y"], "train forward")
    np.testing.assert_allclose(mu[0].cpu().numpy()[..., 0], ref["mu"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(sg[0].cpu().numpy()[..., 0], ref["sigma"], rtol=0, atol=1e-5)


def test_t1_loss_matches_oracle_and_closed_form_gradients(t1ctx):
    rng = np.random.default_rng(6)
    pairs = [synth.make_pair(256, 128, 60.0, 12400), synth.make_pair(120, 64, 30.0, 12401)]
    dps = [binding.to_device(p, 8) for p in pairs]
    Ys, gts, nocs, mus, sgs = [], [], [], [], []
    for p in pairs:
        H, W = p.left.shape
        H8, W8 = oracle.t1_levels(H, W)[3]
        Ys.append((p.gt + rng.standard_normal((H, W)) * 3.0).astype(np.float32))
        gts.append(p.gt.astype(np.float32))
        nocs.append((~p.occ).astype(np.uint8))
        mus.append((1.0 + 0.3 * rng.standard_normal((H8, W8))).astype(np.float32))
        sgs.append((1.0 + 0.2 * rng.standard_normal((H8, W8))).astype(np.float32))
    cuda = lambda a: [torch.from_numpy(x).cuda() for x in a]
    ctx = t1ctx(7)
    out, gY, gmu, gsg = ctx.loss_paper(dps, cuda(Ys), cuda(gts), cuda(nocs), cuda(mus), cuda(sgs))
    out = out.cpu().numpy()
    # the oracle's loss over the concatenated batch
    cat = lambda a: np.concatenate([x.ravel() for x in a])
    want = oracle.t1_loss(cat(Ys).astype(np.float64) / 256.0, cat(gts), cat(nocs), cat(mus).astype(np.float64),
                          cat(sgs).astype(np.float64))
    np.testing.assert_allclose(out, want, rtol=1e-6, atol=0)
    P = sum(y.size for y in Ys)
    nl = sum(m.size for m in mus)
    for y, g, n, gy in zip(Ys, gts, nocs, gY):
        wgt = np.where(n != 0, 2.0, 1.0)
        np.testing.assert_allclose(gy.cpu().numpy(), -wgt * np.sign(g - y) / P, rtol=1e-6, atol=1e-12)
    for m, s, gm, gs in zip(mus, sgs, gmu, gsg):
        np.testing.assert_allclose(gm.cpu().numpy(), 256.0 * (m.astype(np.float64) - 1.0) / nl, rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose(gs.cpu().numpy(), 256.0 * (np.exp(2.0 * (s.astype(np.float64) - 1.0)) - 1.0) / nl,
                                   rtol=1e-5, atol=1e-9)
    again = ctx.loss_paper(dps, cuda(Ys), cuda(gts), cuda(nocs), cuda(mus), cuda(sgs), want_grads=False)[0]
    assert torch.equal(again.cpu(), torch.from_numpy(out))  # fixed reduction order


def test_t1_context_refuses_what_it_does_not_have(t1ctx, svlib):
    ctx = t1ctx(7)
    z = [torch.zeros(4, 4, device="cuda")]
    with pytest.raises(binding.SvError) as ei:
        ctx.refine_backward(z, z, z, False, None)
    assert ei.value.status == binding.SV_ERR_UNSUPPORTED
    bad = binding.make_config("table1", 7, "bf16")
    assert svlib.sv_param_count(__import__("ctypes").byref(bad)) == 0
