"""Pins of the oracle's Table I network (Sec. III-B1) and its loss (Eq. 8-11), on the CPU.

Every layer kind is checked against torch's FP64 library routines (conv2d,
conv_transpose2d, leaky_relu); the inputs against avg_pool2d / interpolate where the sizes
are exact multiples; the whole network against the same graph composed from those
routines (with and without the reparameterisation noise); the loss against closed forms
and torch.distributions' KL divergence of two normal distributions."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from paper_2305_11566_gb300 import synth


def tw(wt):
    """[Co, k, k, Ci] -> torch conv2d weight [Co, Ci, k, k]."""
    return torch.from_numpy(np.ascontiguousarray(wt.transpose(0, 3, 1, 2))).double()


def t(x):
    """[H, W, C] -> [1, C, H, W]."""
    return torch.from_numpy(np.ascontiguousarray(x.transpose(2, 0, 1)))[None].double()


def un(x):
    return x[0].permute(1, 2, 0).numpy()


def torch_layer(x, wt, b, mode, out_hw, act):
    k = wt.shape[1]
    bb = torch.from_numpy(b).double()
    if mode == 2:
        wT = torch.from_numpy(np.ascontiguousarray(wt.transpose(3, 0, 1, 2))).double()  # [Ci, Co, k, k]
        y = F.conv_transpose2d(x, wT, bb, stride=2, padding=k // 2, output_padding=1)
        y = y[:, :, :out_hw[0], :out_hw[1]]
    else:
        y = F.conv2d(x, tw(wt), bb, stride=1 + mode, padding=k // 2)
    return F.leaky_relu(y, 0.1) if act else y


@pytest.mark.parametrize("mode,Hi,Wi,Ci,Co,k,out_hw,act", [
    (0, 9, 13, 3, 4, 5, (9, 13), True),
    (1, 9, 13, 3, 4, 5, (5, 7), True),
    (1, 10, 12, 2, 3, 5, (5, 6), False),
    (2, 5, 7, 3, 2, 5, (10, 14), True),
    (2, 5, 7, 3, 2, 5, (9, 13), False),    # deconv output cropped to an odd size
    (0, 6, 5, 7, 2, 1, (6, 5), False),
])
def test_t1_layer_matches_torch(mode, Hi, Wi, Ci, Co, k, out_hw, act):
    rng = np.random.default_rng(Hi * 7 + mode)
    x = rng.standard_normal((Hi, Wi, Ci))
    wt = rng.standard_normal((Co, k, k, Ci)).astype(np.float32)
    b = rng.standard_normal(Co).astype(np.float32)
    got = oracle.t1_layer(x, wt, b, mode, out_hw, act)
    want = un(torch_layer(t(x), wt, b, mode, out_hw, act))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_t1_inputs_match_library_routines():
    p = synth.make_pair(128, 64, 30.0, 41)
    rng = np.random.default_rng(2)
    coarse = rng.random((16, 32)) * 7.0
    X0, X1 = oracle.t1_inputs(p.left, coarse)
    L = torch.from_numpy(p.left.astype(np.float64))[None, None]
    np.testing.assert_allclose(X1, F.avg_pool2d(L, 2)[0, 0].numpy() / 256.0, rtol=0, atol=1e-15)
    c = torch.from_numpy(coarse)[None, None]
    up = F.interpolate(c, scale_factor=2, mode="bilinear", align_corners=False)[0, 0].numpy()
    np.testing.assert_allclose(X0, 4.0 * up / 256.0, rtol=0, atol=1e-14)


def torch_t1(params, left, coarse, eps=None):
    """The Table I network composed from torch FP64 routines (sizes multiples of 8 and the
    coarse map a quarter of the input, so that pooling / interpolation are exact)."""
    sl = oracle.t1_param_slices()
    P = {n: (params[a].reshape(co, k, k, ci), params[b_])
         for (n, co, ci, k), (a, b_) in zip(synth.TABLE1_LAYERS, [sl[n] for n, *_ in synth.TABLE1_LAYERS])}
    H, W = left.shape
    (_, _), (H2, W2), (H4, W4), (H8, W8) = oracle.t1_levels(H, W)
    L = torch.from_numpy(left.astype(np.float64))[None, None]
    X1 = F.avg_pool2d(L, 2) / 256.0
    X0 = 4.0 * F.interpolate(torch.from_numpy(coarse)[None, None], scale_factor=2, mode="bilinear",
                             align_corners=False) / 256.0

    def lay(x, n, mode, hw, act=True):
        return torch_layer(x, P[n][0], P[n][1], mode, hw, act)
    fe1 = lay(X0, "FE_1", 0, (H2, W2))
    fe2 = lay(X1, "FE_2", 0, (H2, W2))
    en1 = lay(torch.cat([fe1, fe2], 1), "EN_1", 1, (H4, W4))
    en1r = lay(en1, "EN_1_R", 0, (H4, W4))
    en2 = lay(torch.cat([en1, en1r], 1), "EN_2", 1, (H8, W8))
    en2r = lay(en2, "EN_2_R", 0, (H8, W8))
    heads = lay(torch.cat([en2, en2r], 1), "heads", 0, (H8, W8), act=False)
    mu, sg = heads[:, 0:1], heads[:, 1:2]
    g = mu - 1.0
    if eps is not None:
        g = g + torch.from_numpy(eps.reshape(H8, W8).astype(np.float64))[None, None] * torch.exp(sg - 1.0)
    d1 = lay(g, "D_1", 0, (H8, W8))
    d1r = lay(torch.cat([d1, en2, en2r], 1), "D_1_R", 0, (H8, W8))
    d2 = lay(torch.cat([d1, en2, en2r, d1r], 1), "D_2", 2, (H4, W4))
    d2r = lay(torch.cat([d2, en1, en1r], 1), "D_2_R", 0, (H4, W4))
    dd = lay(torch.cat([d2, en1, en1r, d2r], 1), "D", 2, (H2, W2))
    Y = lay(torch.cat([dd, X0, fe1, fe2], 1), "Y", 2, (H, W), act=False)
    return Y[0, 0].numpy(), mu[0, 0].numpy(), sg[0, 0].numpy(), un(d1)


@pytest.mark.parametrize("with_eps", [False, True])
def test_t1_forward_matches_torch_composition(with_eps):
    H, W = 64, 128
    p = synth.make_pair(W, H, 30.0, 43)
    rng = np.random.default_rng(3)
    coarse = rng.random((H // 4, W // 4)) * 7.0
    params = synth.table1_weights(7)
    H8, W8 = oracle.t1_levels(H, W)[3]
    eps = synth.reparam_noise(H8 * W8, 5) if with_eps else None
    got = oracle.t1_forward(params, p.left, coarse, eps, act="D_1")
    Y, mu, sg, d1 = torch_t1(params, p.left, coarse, eps)
    np.testing.assert_allclose(got["Y"], Y, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["mu"], mu, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["sigma"], sg, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["D_1"], d1, rtol=0, atol=1e-12)
    assert np.abs(got["Y"]).max() > 1e-3  # the network does something


def test_t1_forward_odd_sizes_crop_consistently():
    # odd sizes: the deconvolutions' 2n outputs are cropped; the output has the input's size
    p = synth.make_pair(75, 37, 20.0, 44)
    coarse = np.full((37 // 4, 75 // 4), 3.0)
    out = oracle.t1_forward(synth.table1_weights(7), p.left, coarse)
    assert out["Y"].shape == (37, 75) and out["mu"].shape == oracle.t1_levels(37, 75)[3]
    assert np.isfinite(out["Y"]).all()


def test_t1_loss_closed_forms_and_library_kl():
    rng = np.random.default_rng(8)
    H, W = 12, 20
    gt = (rng.random((H, W)) * 100).astype(np.float32)
    noc = (rng.random((H, W)) > 0.3).astype(np.uint8)
    mu = np.ones((2, 3))
    sg = np.ones((2, 3))
    delta = 0.25
    tot, l1, l2 = oracle.t1_loss(gt.astype(np.float64) / 256.0 + delta, gt, noc, mu, sg)
    # a constant error delta: non-occluded pixels count twice
    assert abs(l1 - delta * (H * W + noc.sum()) / (H * W)) < 1e-15
    assert l2 == 0.0 and abs(tot - 256.0 * l1) < 1e-12
    mu = 1.0 + rng.standard_normal((2, 3))
    sg = 1.0 + 0.5 * rng.standard_normal((2, 3))
    _, _, l2 = oracle.t1_loss(gt.astype(np.float64) / 256.0, gt, noc, mu, sg)
    kl = torch.distributions.kl_divergence(
        torch.distributions.Normal(torch.from_numpy(mu - 1.0), torch.exp(torch.from_numpy(sg - 1.0))),
        torch.distributions.Normal(torch.zeros(2, 3, dtype=torch.float64), torch.ones(2, 3, dtype=torch.float64)))
    assert abs(l2 - kl.mean().item()) < 1e-14
