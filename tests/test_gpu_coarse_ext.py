"""GPU parity of the coarse-stage variants (Sec. III-A, Eq. 4-7; robustness settings S1-S4
of Sec. IV-C) against the FP64 oracle, through the C ABI (sv_coarse_match_ex,
sv_postprocess, sv_pipeline_ex).

Bars:
  * census cost volume and its winner-take-all: bit-exact (integers);
  * census + SGM with integer penalties: every sum is an integer below 2^24, exact in FP32,
    so the aggregated volume, the map and the whole chain with the occlusion check and the
    median filter are bit-exact;
  * ZNCC / fractional penalties and DT: the volume within an absolute bar (FP32 sums of FP32
    costs against FP64), the map equal to the oracle's wherever its best and second-best
    aggregated costs differ by more than twice that bar;
  * occlusion check and median filter on given maps: bit-exact (integer work);
  * sv_pipeline_ex: the refined map at the form's bar against the oracle's refinement of the
    oracle's coarse chain (census + SGM + SMP + median, exact coarse maps)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_for(svlib):
    made = {}

    def get(k, prec="fp32", shape=synth.NET_SMALL):
        key = (k, prec, shape)
        if key not in made:
            c = binding.Context(shape, k, prec)
            c.set_weights(synth.he_normal_weights(shape, 7))
            made[key] = c
        return made[key]
    yield get
    for c in made.values():
        c.close()


def decisions_agree(disp, A, tol):
    s = np.sort(A, axis=2)
    sure = (s[:, :, 1] - s[:, :, 0]) > 2 * tol
    want = oracle.sgm_wta(A)
    assert np.array_equal(disp[sure], want[sure])
    picked = np.take_along_axis(A, disp[:, :, None].astype(np.int64), axis=2)[:, :, 0]
    assert (picked - s[:, :, 0]).max() <= 2 * tol


SIZES = [(256, 128, 60.0, 16), (250, 131, 50.0, 20), (1242, 375, 190.0, 48)]


@pytest.mark.parametrize("kc", [3, 5, 7])
@pytest.mark.parametrize("W,H,dmax,D", SIZES)
def test_census_cost_and_wta_bit_exact(ctx_for, W, H, dmax, D, kc):
    p = synth.make_pair(W, H, dmax, 9400 + W + kc)
    C = oracle.census_volume(oracle.downsample4(p.left), oracle.downsample4(p.right), kc, D)
    ctx = ctx_for(9)
    disp, vols = ctx.coarse_match_ex([binding.to_device(p, D)], binding.coarse_opts("census", census_window=kc),
                                     costs=True)
    assert np.array_equal(vols[0].cpu().numpy(), C)
    assert np.array_equal(disp[0].cpu().numpy(), oracle.sgm_wta(C))


@pytest.mark.parametrize("W,H,dmax,D", SIZES)
def test_census_sgm_chain_bit_exact(ctx_for, W, H, dmax, D):
    """Census + SGM (integer penalties: exact in FP32) + occlusion check + median filter."""
    p = synth.make_pair(W, H, dmax, 9500 + W)
    C = oracle.census_volume(oracle.downsample4(p.left), oracle.downsample4(p.right), 5, D)
    A = oracle.sgm(C, 2.0, 12.0, 4)
    wta = oracle.sgm_wta(A)
    ctx = ctx_for(9)
    dp = binding.to_device(p, D)
    disp, vols = ctx.coarse_match_ex([dp], binding.coarse_opts("census", "sgm", census_window=5, P1=2.0, P2=12.0),
                                     costs=True)
    assert np.array_equal(vols[0].cpu().numpy(), A)
    assert np.array_equal(disp[0].cpu().numpy(), wta)
    for smp, med in ((True, False), (False, True), (True, True)):
        want = wta
        if smp:
            want = oracle.smp(want, D)
        if med:
            want = oracle.median3(want)
        got = ctx.coarse_match_ex([dp], binding.coarse_opts("census", "sgm", census_window=5, P1=2.0, P2=12.0,
                                                            smp=smp, median=med))[0]
        assert np.array_equal(got.cpu().numpy(), want), (smp, med)


@pytest.mark.parametrize("cost,tol", [("zncc", 2e-5), ("census", 2e-3)])
@pytest.mark.parametrize("W,H,dmax,D", SIZES)
def test_dt_aggregation(ctx_for, cost, tol, W, H, dmax, D):
    """Domain-transform aggregation (settings S1, S3): FP32 recursive filter against FP64.
    The bar is relative to the cost's scale (2 for ZNCC, kc^2 - 1 = 24 for census)."""
    p = synth.make_pair(W, H, dmax, 9600 + W)
    k = 9 if W > 1000 else 7
    C = oracle.coarse_cost(p.left, p.right, cost, k, D, census_window=5)
    A = oracle.dt_aggregate(C, oracle.downsample4(p.left), 8.0, 20.0, 2)
    ctx = ctx_for(k)
    disp, vols = ctx.coarse_match_ex([binding.to_device(p, D)],
                                     binding.coarse_opts(cost, "dt", census_window=5, dt_sigma_s=8.0, dt_sigma_r=20.0,
                                                         dt_iters=2), costs=True)
    np.testing.assert_allclose(vols[0].cpu().numpy(), A, rtol=0, atol=tol)
    decisions_agree(disp[0].cpu().numpy(), A, tol)


def test_zncc_sgm_dt_mixed_batch_and_iterations(ctx_for):
    specs = [(256, 128, 60.0, 16), (250, 131, 50.0, 20), (96, 64, 20.0, 9)]
    pairs = [synth.make_pair(W, H, dm, 9700 + W) for W, H, dm, _ in specs]
    dps = [binding.to_device(p, D) for p, (_, _, _, D) in zip(pairs, specs)]
    ctx = ctx_for(5)
    for iters in (1, 3):
        disp, vols = ctx.coarse_match_ex(dps, binding.coarse_opts("zncc", "dt", dt_sigma_s=5.0, dt_sigma_r=30.0,
                                                                  dt_iters=iters), costs=True)
        for i, (p, (_, _, _, D)) in enumerate(zip(pairs, specs)):
            C = oracle.coarse_cost(p.left, p.right, "zncc", 5, D)
            A = oracle.dt_aggregate(C, oracle.downsample4(p.left), 5.0, 30.0, iters)
            np.testing.assert_allclose(vols[i].cpu().numpy(), A, rtol=0, atol=2e-5)
            decisions_agree(disp[i].cpu().numpy(), A, 2e-5)


@pytest.mark.parametrize("W,H,D", [(256, 128, 16), (1242, 375, 48), (250, 131, 20), (64, 16, 16), (16, 16, 1),
                                   (4096, 8, 128)])
def test_postprocess_bit_exact(ctx_for, W, H, D):
    """The occlusion check and the median filter on maps from the oracle (random disparities:
    many target collisions, rows without any kept pixel are not excluded)."""
    rng = np.random.default_rng(W + H + D)
    q = synth.make_pair(W, H, 4.0 * D, W + D)
    maps = [rng.integers(0, D, size=(H // 4, W // 4)).astype(np.int16),
            oracle.zncc_wta(oracle.downsample4(q.left), oracle.downsample4(q.right), 3, D)[0].astype(np.int16)]
    ctx = ctx_for(3)
    img = torch.zeros((1, 16), dtype=torch.uint8, device="cuda")  # not read by sv_postprocess
    dp = binding.DevicePair(img, img, W, H, D)
    for m in maps:
        dm = torch.from_numpy(m).cuda()
        for smp, med in ((True, False), (False, True), (True, True), (False, False)):
            want = m.astype(np.int32)
            if smp:
                want = oracle.smp(want, D)
            if med:
                want = oracle.median3(want)
            got = ctx.postprocess([dp], [dm], smp, med)[0]
            assert np.array_equal(got.cpu().numpy(), want), (W, H, D, smp, med)


def test_zncc_sgm_post_chain_consistent(ctx_for):
    """The paper's coarse chain (ZNCC + SGM + SMP + median): the map before post-processing
    agrees with the oracle's decisions, and the chain equals sv_postprocess of that map."""
    p = synth.make_pair(1242, 375, 190.0, 9800)
    D, k = 48, 9
    C = oracle.coarse_cost(p.left, p.right, "zncc", k, D)
    A = oracle.sgm(C, 0.1, 0.5, 4)
    ctx = ctx_for(k)
    dp = binding.to_device(p, D)
    pre = ctx.coarse_match_ex([dp], binding.coarse_opts("zncc", "sgm", P1=0.1, P2=0.5))[0]
    decisions_agree(pre.cpu().numpy(), A, 1e-3)
    chain = ctx.coarse_match_ex([dp], binding.coarse_opts("zncc", "sgm", P1=0.1, P2=0.5, smp=True, median=True))[0]
    assert torch.equal(chain, ctx.postprocess([dp], [pre], True, True)[0])


@pytest.mark.parametrize("prec,bar", [("fp32", 1e-4), ("bf16", 0.05)])
def test_pipeline_ex_census_sgm_post(ctx_for, prec, bar):
    """sv_pipeline_ex on the exact census chain: coarse maps bit-exact, so the refined map is
    held to the form's bar everywhere."""
    shape = synth.NET_SMALL
    W, H, D, k = 256, 128, 16, 7
    p = synth.make_pair(W, H, 60.0, 9900)
    C = oracle.census_volume(oracle.downsample4(p.left), oracle.downsample4(p.right), 5, D)
    m = oracle.median3(oracle.smp(oracle.sgm_wta(oracle.sgm(C, 2.0, 12.0, 4)), D))
    ref = oracle.refine_forward(shape, synth.he_normal_weights(shape, 7), p.left, m.astype(np.float64))
    ctx = ctx_for(k, prec)
    Y = ctx.pipeline_ex([binding.to_device(p, D)],
                        binding.coarse_opts("census", "sgm", census_window=5, P1=2.0, P2=12.0, smp=True,
                                            median=True))[0]
    torch.cuda.synchronize()
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref["Y"])
    assert err.max() <= bar, err.max()


def test_coarse_ex_rejects_bad_options(ctx_for):
    ctx = ctx_for(5)
    dp = binding.to_device(synth.make_pair(96, 64, 20.0, 9950), 9)
    bad = [binding.coarse_opts("census", census_window=9), binding.coarse_opts("zncc", "sgm", P1=-1.0),
           binding.coarse_opts("zncc", "sgm", npaths=5), binding.coarse_opts("zncc", "dt", dt_sigma_s=0.0),
           binding.coarse_opts("zncc", "dt", dt_iters=9)]
    o = binding.coarse_opts()
    o.post = 4
    bad.append(o)
    o = binding.coarse_opts()
    o.aggregation = 3
    bad.append(o)
    for o in bad:
        with pytest.raises(binding.SvError) as ei:
            ctx.coarse_match_ex([dp], o)
        assert ei.value.status == binding.SV_ERR_INVALID_ARG
    assert ctx.coarse_match_ex([], binding.coarse_opts()) == []
