"""Pins of the oracle's refinement stage: bilinear x4 against affine ramps and
torch interpolate, convolutions against torch.nn.functional.conv2d in FP64 (a
library routine), the composed net against torch FP64, the hand-derived backward
against central finite differences and torch FP64 autograd, the KL term against
its closed form and Adam against torch.optim.Adam."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from paper_2305_11566_gb300 import synth

torch.set_default_dtype(torch.float64)


def test_upsample_affine_ramp_exact():
    h, w = 9, 13
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    a, b, c = 0.75, -1.25, 20.0
    disp = a * xx + b * yy + c
    H, W = 4 * h + 2, 4 * w + 3
    U = oracle.upsample4(disp, W, H)
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    sx = (X + 0.5) / 4 - 0.5
    sy = (Y + 0.5) / 4 - 0.5
    inner = (sx >= 0) & (sx <= w - 1) & (sy >= 0) & (sy <= h - 1)
    ref = 4 * (a * sx + b * sy + c)
    assert np.abs(U[inner] - ref[inner]).max() < 1e-12
    # outside the interior the coordinate clamps to the edge value
    assert np.allclose(U[0, 0], 4 * disp[0, 0])


def test_upsample_matches_torch_when_sizes_divide():
    rng = np.random.default_rng(0)
    disp = rng.integers(0, 16, size=(8, 11)).astype(np.float64)
    U = oracle.upsample4(disp, 44, 32)
    ref = 4 * F.interpolate(torch.from_numpy(disp)[None, None], scale_factor=4, mode="bilinear",
                            align_corners=False)[0, 0].numpy()
    assert np.abs(U - ref).max() < 1e-12


def test_upsample_backward_is_transpose():
    rng = np.random.default_rng(1)
    h, w, H, W = 5, 7, 22, 30
    d = rng.normal(size=(h, w))
    g = rng.normal(size=(H, W))
    lhs = (oracle.upsample4(d, W, H) * g).sum()
    rhs = (d * oracle.upsample4_backward(g, w, h)).sum()
    assert abs(lhs - rhs) < 1e-10 * max(1, abs(lhs))


def _torch_conv(x, wt, b, stride, pad, relu=False, up2=False, out_hw=None):
    t = torch.from_numpy(x).permute(2, 0, 1)[None]
    if up2:
        t = F.interpolate(t, scale_factor=2, mode="nearest")[:, :, :out_hw[0], :out_hw[1]]
    wt_t = torch.from_numpy(wt.astype(np.float64)).permute(0, 3, 1, 2)
    bt = None if b is None else torch.from_numpy(b.astype(np.float64))
    o = F.conv2d(t, wt_t, bt, stride=stride, padding=pad)
    if relu:
        o = F.relu(o)
    return o[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("Hi,Wi,Ci,Co,k,stride,pad,relu", [
    (9, 13, 3, 5, 3, 1, 1, True), (9, 13, 4, 6, 3, 2, 1, True), (10, 12, 2, 4, 3, 2, 1, False),
    (7, 5, 6, 3, 1, 1, 0, False), (11, 17, 8, 1, 3, 1, 1, False)])
def test_conv2d_matches_torch(Hi, Wi, Ci, Co, k, stride, pad, relu):
    rng = np.random.default_rng(Hi * Wi + Co)
    x = rng.normal(size=(Hi, Wi, Ci))
    wt = rng.normal(size=(Co, k, k, Ci)).astype(np.float32)
    b = rng.normal(size=Co).astype(np.float32)
    ref = _torch_conv(x, wt, b, stride, pad, relu)
    got = oracle.conv2d(x, wt, b, stride, pad, relu)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("Hi,Wi,Ho,Wo", [(5, 7, 10, 14), (5, 7, 9, 13), (24, 78, 47, 155)])
def test_conv2d_up2_crop_matches_torch(Hi, Wi, Ho, Wo):
    rng = np.random.default_rng(Ho)
    x = rng.normal(size=(Hi, Wi, 4))
    wt = rng.normal(size=(3, 3, 3, 4)).astype(np.float32)
    b = rng.normal(size=3).astype(np.float32)
    ref = _torch_conv(x, wt, b, 1, 1, True, up2=True, out_hw=(Ho, Wo))
    got = oracle.conv2d(x, wt, b, 1, 1, True, up2=True, out_hw=(Ho, Wo))
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("stride,up2", [(1, False), (2, False), (1, True)])
def test_conv2d_backward_matches_autograd(stride, up2):
    rng = np.random.default_rng(3 + stride + 2 * up2)
    Hi, Wi, Ci, Co = 6, 9, 3, 4
    x = rng.normal(size=(Hi, Wi, Ci))
    wt = rng.normal(size=(Co, 3, 3, Ci)).astype(np.float32)
    out_hw = (11, 17) if up2 else None
    o = oracle.conv2d(x, wt, None, stride, 1, False, up2, out_hw)
    g = rng.normal(size=o.shape)
    gin, gw, gb = oracle.conv2d_backward(x, wt, stride, 1, g, up2)
    xt = torch.from_numpy(x).permute(2, 0, 1)[None].requires_grad_(True)
    wtt = torch.from_numpy(wt.astype(np.float64)).permute(0, 3, 1, 2).detach().requires_grad_(True)
    bt = torch.zeros(Co, requires_grad=True)
    t = xt
    if up2:
        t = F.interpolate(t, scale_factor=2, mode="nearest")[:, :, :out_hw[0], :out_hw[1]]
    ot = F.conv2d(t, wtt, bt, stride=stride, padding=1)
    (ot * torch.from_numpy(g).permute(2, 0, 1)[None]).sum().backward()
    assert np.abs(gin - xt.grad[0].permute(1, 2, 0).numpy()).max() < 1e-11
    assert np.abs(gw - wtt.grad.permute(0, 2, 3, 1).numpy()).max() < 1e-11
    assert np.abs(gb - bt.grad.numpy()).max() < 1e-11


# ------------------------------------------------------------------ the net in torch FP64
def _torch_net(shape, params, left, coarse, eps=None):
    """The same network composed from torch library routines (FP64)."""
    sl = oracle.param_slices(shape)
    P = torch.from_numpy(params.astype(np.float64))

    def wb(name):
        ow, wshape, ob, co = sl[name]
        n = int(np.prod(wshape))
        return P[ow:ow + n].reshape(wshape).permute(0, 3, 1, 2), P[ob:ob + co]

    H, W = left.shape
    h, w = coarse.shape
    L0, L1, L2, L3 = oracle.level_sizes(H, W)
    U = torch.from_numpy(oracle.upsample4(coarse, W, H))
    x0 = torch.stack([torch.from_numpy(left.astype(np.float64)) / 256.0, U / 256.0])[None]
    e1 = F.relu(F.conv2d(x0, *wb("enc1"), stride=2, padding=1))
    e2 = F.relu(F.conv2d(e1, *wb("enc2"), stride=2, padding=1))
    e3 = F.relu(F.conv2d(e2, *wb("enc3"), stride=2, padding=1))
    mu = F.conv2d(e3, *wb("mu"))
    lv = F.conv2d(e3, *wb("logvar"))
    z = mu if eps is None else mu + torch.from_numpy(eps.astype(np.float64)).reshape(
        L3[0], L3[1], -1).permute(2, 0, 1)[None] * torch.exp(0.5 * lv)

    def up(t, hw):
        return F.interpolate(t, scale_factor=2, mode="nearest")[:, :, :hw[0], :hw[1]]

    d1 = F.relu(F.conv2d(up(z, L2), *wb("dec1"), padding=1))
    d2 = F.relu(F.conv2d(up(d1, L1), *wb("dec2"), padding=1))
    d3 = F.relu(F.conv2d(up(d2, L0), *wb("dec3"), padding=1))
    Y = U + F.conv2d(d3, *wb("final"), padding=1)[0, 0]
    return Y, mu[0].permute(1, 2, 0), lv[0].permute(1, 2, 0)


@pytest.mark.parametrize("W,H", [(64, 32), (70, 45)])
def test_refine_forward_matches_torch(W, H):
    shape = synth.NET_SMALL
    params = synth.he_normal_weights(shape, 7)
    p = synth.make_pair(W, H, 30.0, 5)
    disp, _, _ = oracle.coarse_match(p.left, p.right, 5, 6)
    out = oracle.refine_forward(shape, params, p.left, disp.astype(np.float64))
    Y, mu, lv = _torch_net(shape, params, p.left, disp.astype(np.float64))
    assert np.abs(out["Y"] - Y.numpy()).max() < 1e-10
    assert np.abs(out["mu"] - mu.numpy()).max() < 1e-10
    assert np.abs(out["logvar"] - lv.numpy()).max() < 1e-10
    d3 = oracle.refine_activation(shape, params, p.left, disp.astype(np.float64), "d3")
    assert d3.shape == (H, W, shape.dec[2])


def test_kl_closed_form_zero():
    """KL(N(mu, e^lv) || N(0, 1)) = 0 exactly at mu = 0, lv = 0: with all latent
    weights and biases zero, the loss is the reconstruction term alone."""
    shape = synth.NET_SMALL
    params = synth.he_normal_weights(shape, 7)
    sl = oracle.param_slices(shape)
    for name in ("mu", "logvar"):
        ow, wshape, ob, co = sl[name]
        params[ow:ow + int(np.prod(wshape))] = 0
        params[ob:ob + co] = 0
    p = synth.make_pair(64, 32, 20.0, 9)
    coarse = np.full((8, 16), 3.0)
    L0, L1, L2, L3 = oracle.level_sizes(32, 64)
    nlat = L3[0] * L3[1] * shape.latent
    with_kl = oracle.refine_loss(shape, params, p.left, coarse, None, p.gt, 32 * 64, nlat, 1e-3)
    without = oracle.refine_loss(shape, params, p.left, coarse, None, p.gt, 32 * 64, nlat, 0.0)
    assert with_kl == without


def _training_case(seed=11, W=64, H=32):
    shape = synth.NET_SMALL
    params = synth.he_normal_weights(shape, 7)
    rng = np.random.default_rng(seed)
    # give the latent heads non-trivial biases so exp(lv / 2) matters
    sl = oracle.param_slices(shape)
    ob, co = sl["logvar"][2], sl["logvar"][3]
    params[ob:ob + co] = rng.normal(scale=0.3, size=co).astype(np.float32)
    p = synth.make_pair(W, H, 30.0, seed)
    coarse = oracle.coarse_match(p.left, p.right, 5, 6)[0].astype(np.float64)
    coarse += rng.uniform(0.1, 0.4, size=coarse.shape)  # off the integer grid
    L3 = oracle.level_sizes(H, W)[3]
    nlat = L3[0] * L3[1] * shape.latent
    eps = synth.reparam_noise(nlat, seed)
    return shape, params, p, coarse, eps, nlat


def test_backward_matches_torch_autograd():
    shape, params, p, coarse, eps, nlat = _training_case()
    H, W = p.left.shape
    L, g, gc = oracle.refine_backward(shape, params, p.left, coarse, eps, p.gt, H * W, nlat, 1e-3, True)
    Pt = torch.from_numpy(params.astype(np.float64)).requires_grad_(True)

    def loss_fn(Pv):
        sl = oracle.param_slices(shape)

        def wb(name):
            ow, wshape, ob, co = sl[name]
            n = int(np.prod(wshape))
            return Pv[ow:ow + n].reshape(wshape).permute(0, 3, 1, 2), Pv[ob:ob + co]

        L0, L1, L2, L3 = oracle.level_sizes(H, W)
        U = torch.from_numpy(oracle.upsample4(coarse, W, H))
        x0 = torch.stack([torch.from_numpy(p.left.astype(np.float64)) / 256.0, U / 256.0])[None]
        e1 = F.relu(F.conv2d(x0, *wb("enc1"), stride=2, padding=1))
        e2 = F.relu(F.conv2d(e1, *wb("enc2"), stride=2, padding=1))
        e3 = F.relu(F.conv2d(e2, *wb("enc3"), stride=2, padding=1))
        mu = F.conv2d(e3, *wb("mu"))
        lv = F.conv2d(e3, *wb("logvar"))
        ep = torch.from_numpy(eps.astype(np.float64)).reshape(L3[0], L3[1], -1).permute(2, 0, 1)[None]
        z = mu + ep * torch.exp(0.5 * lv)

        def up(t, hw):
            return F.interpolate(t, scale_factor=2, mode="nearest")[:, :, :hw[0], :hw[1]]

        d1 = F.relu(F.conv2d(up(z, L2), *wb("dec1"), padding=1))
        d2 = F.relu(F.conv2d(up(d1, L1), *wb("dec2"), padding=1))
        d3 = F.relu(F.conv2d(up(d2, L0), *wb("dec3"), padding=1))
        Yt = U + F.conv2d(d3, *wb("final"), padding=1)[0, 0]
        rec = F.smooth_l1_loss(Yt, torch.from_numpy(p.gt.astype(np.float64)), beta=1.0, reduction="sum") / (H * W)
        kl = 0.5 * (mu ** 2 + torch.exp(lv) - 1 - lv).sum() / nlat
        return rec + 1e-3 * kl

    Lt = loss_fn(Pt)
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-12 * max(1.0, abs(L))
    ref = Pt.grad.numpy()
    assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()


def test_backward_matches_finite_differences():
    shape, params, p, coarse, eps, nlat = _training_case(seed=12)
    H, W = p.left.shape
    L, g, gc = oracle.refine_backward(shape, params, p.left, coarse, eps, p.gt, H * W, nlat, 1e-3, True)
    rng = np.random.default_rng(0)
    sl = oracle.param_slices(shape)
    # parameters: a few entries of every layer.  FD runs on a float64 copy of the
    # parameters, so the oracle is given float32 params that equal params64 exactly
    # only at the base point; perturbations are applied in float64 through a second
    # evaluation path: perturb the float32 value by a representable step.
    idx = []
    for name, (ow, wshape, ob, co) in sl.items():
        n = int(np.prod(wshape))
        idx += list(ow + rng.choice(n, size=3, replace=False)) + [ob + rng.integers(co)]
    worst = 0.0
    for i in idx:
        base = params[i]
        h = np.float32(max(abs(base), 1e-2) * 2.0 ** -10)
        pp = params.copy(); pp[i] = base + h
        pm = params.copy(); pm[i] = base - h
        step = float(np.float64(pp[i]) - np.float64(pm[i]))
        Lp = oracle.refine_loss(shape, pp, p.left, coarse, eps, p.gt, H * W, nlat, 1e-3)
        Lm = oracle.refine_loss(shape, pm, p.left, coarse, eps, p.gt, H * W, nlat, 1e-3)
        fd = (Lp - Lm) / step
        if abs(g[i]) > 1e-8:
            worst = max(worst, abs(fd - g[i]) / abs(g[i]))
    assert worst < 1e-4  # central difference truncation with h ~ 1e-3 relative
    # coarse map: FP64 perturbations are exact here (coarse is float64)
    for (y, x) in [(1, 1), (3, 7), (7, 15), (0, 15)]:
        h = 1e-5
        cp = coarse.copy(); cp[y, x] += h
        cm = coarse.copy(); cm[y, x] -= h
        fd = (oracle.refine_loss(shape, params, p.left, cp, eps, p.gt, H * W, nlat, 1e-3)
              - oracle.refine_loss(shape, params, p.left, cm, eps, p.gt, H * W, nlat, 1e-3)) / (2 * h)
        assert abs(fd - gc[y, x]) <= 1e-6 * max(abs(gc[y, x]), 1e-6)


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    n = 50
    p0 = rng.normal(size=n)
    p = p0.copy(); m = np.zeros(n); v = np.zeros(n)
    pt = torch.from_numpy(p0.copy()).requires_grad_(True)
    opt = torch.optim.Adam([pt], lr=5e-4, betas=(0.99, 0.999), eps=1e-8)
    for t in range(1, 4):
        g = rng.normal(size=n)
        oracle.adam(p, m, v, g, t)
        opt.zero_grad()
        pt.grad = torch.from_numpy(g.copy())
        opt.step()
    assert np.abs(p - pt.detach().numpy()).max() < 1e-14
