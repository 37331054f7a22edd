"""GPU parity of the semi-global matching coarse stage (Sec. III-A, Eq. 1 and 4-6) against
the FP64 oracle, through the C ABI (sv_coarse_match_sgm).

Bars: the ZNCC cost volume (npaths = 1, no penalties, which returns the cost itself)
within 1e-6 of 1 - rho; the aggregated volume within 1e-4 (coarse 64 x 32) and 1e-3
(310 x 93: FP32 sums along 310-step paths); the winner-take-all disparity equal to the
oracle's wherever the oracle's best and second-best aggregated costs differ by more than
twice the volume bar, and within that bar of the oracle's minimum everywhere."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_for(svlib):
    made = {}

    def get(k):
        if k not in made:
            c = binding.Context(synth.NET_SMALL, k, "bf16")
            made[k] = c
        return made[k]
    yield get
    for c in made.values():
        c.close()


def oracle_volume(p, k, D):
    rho = oracle.zncc_volume(oracle.downsample4(p.left), oracle.downsample4(p.right), k, D)
    return oracle.sgm_cost(rho)


def check_decisions(disp, A_oracle, tol):
    s = np.sort(A_oracle, axis=2)
    margin = s[:, :, 1] - s[:, :, 0]
    want = oracle.sgm_wta(A_oracle)
    sure = margin > 2 * tol
    assert np.array_equal(disp[sure], want[sure])
    picked = np.take_along_axis(A_oracle, disp[:, :, None].astype(np.int64), axis=2)[:, :, 0]
    assert (picked - s[:, :, 0]).max() <= 2 * tol


@pytest.mark.parametrize("W,H,dmax,k,D,tol", [
    (256, 128, 60.0, 7, 16, 1e-4),
    (250, 131, 50.0, 5, 20, 1e-4),
    (1242, 375, 190.0, 9, 48, 1e-3),
])
def test_sgm_matches_oracle(ctx_for, W, H, dmax, k, D, tol):
    p = synth.make_pair(W, H, dmax, 9000 + W)
    C = oracle_volume(p, k, D)
    ctx = ctx_for(k)
    dp = binding.to_device(p, D)
    # npaths = 1 without penalties returns the ZNCC cost itself
    _, vols = ctx.coarse_match_sgm([dp], 0.0, 0.0, 1, costs=True)
    np.testing.assert_allclose(vols[0].cpu().numpy(), C, rtol=0, atol=1e-6)
    P1, P2 = 0.1, 0.5
    disp, vols = ctx.coarse_match_sgm([dp], P1, P2, 4, costs=True)
    A = oracle.sgm(C, P1, P2, 4)
    np.testing.assert_allclose(vols[0].cpu().numpy(), A, rtol=0, atol=tol)
    check_decisions(disp[0].cpu().numpy(), A, tol)


def test_sgm_directions_and_mixed_batch(ctx_for):
    # pairs of different sizes and disparity ranges in one call; every direction count
    k = 5
    specs = [(256, 128, 60.0, 16), (250, 131, 50.0, 20), (96, 64, 20.0, 9)]
    pairs = [synth.make_pair(W, H, dm, 9100 + W) for W, H, dm, _ in specs]
    dps = [binding.to_device(p, D) for p, (_, _, _, D) in zip(pairs, specs)]
    Cs = [oracle_volume(p, k, D) for p, (_, _, _, D) in zip(pairs, specs)]
    ctx = ctx_for(k)
    for npaths in (1, 2, 3, 4):
        disp, vols = ctx.coarse_match_sgm(dps, 0.05, 0.3, npaths, costs=True)
        for i, C in enumerate(Cs):
            A = oracle.sgm(C, 0.05, 0.3, npaths)
            np.testing.assert_allclose(vols[i].cpu().numpy(), A, rtol=0, atol=1e-4)
            check_decisions(disp[i].cpu().numpy(), A, 1e-4)
    # without the volumes requested, the same disparities
    disp2 = ctx.coarse_match_sgm(dps, 0.05, 0.3, 4)
    for a, b in zip(disp, disp2):
        assert torch.equal(a, b)


def test_sgm_rejects_bad_arguments(ctx_for):
    ctx = ctx_for(5)
    dp = binding.to_device(synth.make_pair(96, 64, 20.0, 9200), 9)
    for P1, P2, npaths in ((-0.1, 0.3, 4), (0.1, 0.3, 0), (0.1, 0.3, 5)):
        with pytest.raises(binding.SvError):
            ctx.coarse_match_sgm([dp], P1, P2, npaths)


def test_sgm_edges(ctx_for):
    # an empty batch is a no-op; the largest disparity range (128) at a wide, short map
    ctx = ctx_for(11)
    assert ctx.coarse_match_sgm([], 0.1, 0.5) == []
    W, H, D = 1024, 64, 128
    p = synth.make_pair(W, H, 400.0, 9300)
    C = oracle_volume(p, 11, D)
    disp, vols = ctx.coarse_match_sgm([binding.to_device(p, D)], 0.1, 0.5, 4, costs=True)
    A = oracle.sgm(C, 0.1, 0.5, 4)
    np.testing.assert_allclose(vols[0].cpu().numpy(), A, rtol=0, atol=1e-3)
    check_decisions(disp[0].cpu().numpy(), A, 1e-3)
