"""GPU parity of the plain FP32 refinement (sv_refine) and the whole FP32 pipeline
(sv_pipeline) against the FP64 oracle, through the C ABI.

Bar: within 1e-4 px of the oracle on every output pixel.  sv_refine is fed the
oracle's own coarse map, so the comparison is independent of WTA near-ties."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu

TOL_PX = 1e-4


@pytest.fixture(scope="module")
def contexts(svlib):
    made = {}

    def get(shape, k, prec="fp32"):
        key = (shape, k, prec)
        if key not in made:
            c = binding.Context(shape, k, prec)
            c.set_weights(synth.he_normal_weights(shape, 7))
            made[key] = c
        return made[key]
    yield get
    for c in made.values():
        c.close()


@pytest.mark.parametrize("name,shape,W,H,dmax,k,D", [
    ("256x128 small net", synth.NET_SMALL, 256, 128, 60.0, 7, 16),
    ("1242x375 wide net", synth.NET_WIDE, 1242, 375, 190.0, 9, 48),
    ("ragged 250x131", synth.NET_SMALL, 250, 131, 50.0, 5, 20),
    ("ragged 333x97 wide", synth.NET_WIDE, 333, 97, 60.0, 5, 24),
])
def test_refine_fp32_matches_oracle(contexts, name, shape, W, H, dmax, k, D):
    p = synth.make_pair(W, H, dmax, 4000 + W)
    disp_o, _, _ = oracle.coarse_match(p.left, p.right, k, D)
    ref = oracle.refine_forward(shape, synth.he_normal_weights(shape, 7), p.left, disp_o.astype(np.float64))
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    coarse = torch.from_numpy(disp_o.astype(np.int16)).cuda()
    Y = ctx.refine([dp], [coarse])[0]
    torch.cuda.synchronize()
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref["Y"])
    assert err.max() <= TOL_PX, f"{name}: max |dY| = {err.max():.3g}"


@pytest.mark.parametrize("name,shape,W,H,dmax,k,D", [
    ("256x128 small net", synth.NET_SMALL, 256, 128, 60.0, 7, 16),
    ("1242x375 wide net", synth.NET_WIDE, 1242, 375, 190.0, 9, 48),
])
def test_pipeline_fp32_matches_oracle(contexts, name, shape, W, H, dmax, k, D):
    p = synth.make_pair(W, H, dmax, 5000 + W)
    Y_o, disp_o, best_o, sec_o = oracle.pipeline(shape, synth.he_normal_weights(shape, 7), p.left, p.right, k, D)
    ctx = contexts(shape, k)
    dp = binding.to_device(p, D)
    Y = ctx.pipeline([dp])[0]
    disp_g = ctx.coarse_match([dp])[0]
    torch.cuda.synchronize()
    # WTA differences only on near ties; the refined output is compared outside their reach
    keep = parity.keep_mask(parity.wta_differences(disp_g.cpu().numpy(), disp_o, best_o, sec_o), H, W)
    parity.compare_refined(Y.cpu().numpy(), Y_o, keep, TOL_PX, label=name)


def test_pipeline_batch_of_pairs(contexts):
    shape, k = synth.NET_SMALL, 7
    pairs = [synth.make_pair(W, H, 40.0, 6000 + W) for W, H in ((256, 128), (320, 97), (200, 60))]
    dps = [binding.to_device(p, 12) for p in pairs]
    ctx = contexts(shape, k)
    Ys = ctx.pipeline(dps)
    torch.cuda.synchronize()
    params = synth.he_normal_weights(shape, 7)
    coarse = ctx.coarse_match(dps)
    for p, Y, d in zip(pairs, Ys, coarse):
        Y_o, disp_o, best_o, sec_o = oracle.pipeline(shape, params, p.left, p.right, k, 12)
        keep = parity.keep_mask(parity.wta_differences(d.cpu().numpy(), disp_o, best_o, sec_o), p.height, p.width)
        parity.compare_refined(Y.cpu().numpy(), Y_o, keep, TOL_PX, label=f"batch {p.width}x{p.height}")
