"""GPU parity of the differentiation form (sv_refine_train, sv_loss, sv_refine_backward,
sv_adam_step) against the FP64 oracle and against finite differences.

FP64 (SV_FP64_CHECK) on a 64x32 crop: loss equal to the oracle's to 1e-12, the analytic
gradient equal to the oracle's hand-derived gradient to 1e-9 (relative to the largest
entry), and to central finite differences of the GPU's own FP64 loss within 1e-6
relative (coarse-map entries: the loss is piecewise quadratic in them; parameters:
two-step extrapolated differences on entries whose gradient is at least 1e-3 of the
largest, where FP64 roundoff of the loss cannot reach 1e-6; entries whose two step sizes
disagree -- a ReLU kink inside the step -- are skipped and counted).  FP32: gradient within 1e-4 of the
oracle's (relative to each layer's largest entry), one Adam step within 1e-6."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_11566_gb300 import autograd, binding, synth

pytestmark = pytest.mark.gpu


def case(W=64, H=32, seed=21, shape=synth.NET_SMALL, k=5, D=6):
    params = synth.he_normal_weights(shape, 7)
    sl = oracle.param_slices(shape)
    rng = np.random.default_rng(seed)
    ob, co = sl["logvar"][2], sl["logvar"][3]
    params[ob:ob + co] = rng.normal(scale=0.3, size=co).astype(np.float32)
    p = synth.make_pair(W, H, 30.0, seed)
    coarse = oracle.coarse_match(p.left, p.right, k, D)[0].astype(np.float64)
    coarse += rng.uniform(0.1, 0.4, size=coarse.shape)
    L3 = oracle.level_sizes(H, W)[3]
    eps = synth.reparam_noise(L3[0] * L3[1] * shape.latent, seed)
    return shape, params, p, coarse, eps, k, D


def gpu_loss_grad(ctx, dp, coarse, eps, gt, dt, want_coarse=True):
    c = torch.from_numpy(coarse).to("cuda", dt)
    e = torch.from_numpy(eps.astype(np.float64)).to("cuda", dt)
    H3, W3 = binding.latent_hw(dp.height, dp.width)
    e = e.reshape(H3, W3, -1)
    Y, mu, lv = ctx.refine_train([dp], [c], [e])
    out, gY, gmu, glv = ctx.loss([dp], Y, [torch.from_numpy(gt).cuda()], mu, lv, 1e-3)
    gp, gc = ctx.refine_backward(gY, gmu, glv, want_coarse, [c])
    ctx.synchronize()
    return out.cpu().numpy(), gp.cpu().numpy(), (gc[0].cpu().numpy() if want_coarse else None)


@pytest.fixture(scope="module")
def fp64(svlib):
    shape, params, p, coarse, eps, k, D = case()
    ctx = binding.Context(shape, k, "fp64")
    ctx.set_weights(params)
    yield ctx, shape, params, p, coarse, eps, k, D
    ctx.close()


def test_fp64_gradient_equals_oracle(fp64):
    ctx, shape, params, p, coarse, eps, k, D = fp64
    H, W = p.left.shape
    dp = binding.to_device(p, D)
    out, gp, gc = gpu_loss_grad(ctx, dp, coarse, eps, p.gt, torch.float64)
    L3 = oracle.level_sizes(H, W)[3]
    nlat = L3[0] * L3[1] * shape.latent
    Lo, go, gco = oracle.refine_backward(shape, params, p.left, coarse, eps, p.gt, H * W, nlat, 1e-3, True)
    assert abs(out[0] - Lo) <= 1e-12 * abs(Lo)
    assert np.abs(gp - go).max() <= 1e-9 * np.abs(go).max()
    assert np.abs(gc - gco).max() <= 1e-9 * np.abs(gco).max()


def test_fp64_gradient_matches_finite_differences(fp64):
    """Central differences of the GPU's own FP64 loss.  The ground truth is the oracle's
    prediction plus 0.05 px noise, so the loss (~1e-3) and its FP64 roundoff are small and
    tiny steps (~1e-6) resolve the derivative; a ReLU kink inside a step shows as
    disagreement between steps h and h/2 and the entry is skipped (and counted)."""
    ctx, shape, params, p, coarse, eps, k, D = fp64
    dp = binding.to_device(p, D)
    H, W = p.left.shape
    Yo = oracle.refine_forward(shape, params, p.left, coarse, eps)["Y"]
    noise = np.random.default_rng(5).normal(scale=0.05, size=Yo.shape)
    gt = (Yo + noise).astype(np.float32)
    _, g, gc = gpu_loss_grad(ctx, dp, coarse, eps, gt, torch.float64)

    def L(par=None, c=None):
        if par is not None:
            ctx.set_weights(par)
        return gpu_loss_grad(ctx, dp, coarse if c is None else c, eps, gt, torch.float64, want_coarse=False)[0][0]

    skips = []

    def check(fd_pair, gi):
        (d1, d2) = fd_pair
        if abs(d1 - d2) > 3e-7 * abs(gi):
            skips.append((d1, d2, gi))
            return None  # kink inside the step
        return abs(d2 - gi) / abs(gi)

    rng = np.random.default_rng(1)
    results, skipped = [], 0
    # coarse map entries (FP64 inputs)
    for (y, x) in [(1, 1), (3, 7), (7, 15), (0, 15), (4, 0)]:
        ests = []
        for h in (2e-6, 1e-6):
            cp = coarse.copy(); cp[y, x] += h
            cm = coarse.copy(); cm[y, x] -= h
            ests.append((L(c=cp) - L(c=cm)) / (2 * h))
        r = check(ests, gc[y, x])
        if r is None:
            skipped += 1
        else:
            results.append(r)
    # parameters (FP32 master copy: the actual step is taken from the FP32 values)
    sl = oracle.param_slices(shape)
    gmax = np.abs(g).max()
    idx = []
    for name, (ow, wshape, ob, co) in sl.items():
        n = int(np.prod(wshape))
        cand = np.concatenate([np.arange(ow, ow + n), np.arange(ob, ob + co)])
        cand = cand[np.abs(g[cand]) >= 1e-3 * gmax]
        if cand.size:
            idx += list(rng.choice(cand, size=min(4, cand.size), replace=False))
    try:
        for i in idx:
            ests = []
            base = params[i]
            for rel in (2.0 ** -16, 2.0 ** -17):
                hh = np.float32(max(abs(base), 1e-2) * rel)
                pp = params.copy(); pp[i] = base + hh
                pm = params.copy(); pm[i] = base - hh
                step = float(np.float64(pp[i]) - np.float64(pm[i]))
                ests.append((L(par=pp) - L(par=pm)) / step)
            r = check(ests, g[i])
            if r is None:
                skipped += 1
            else:
                results.append(r)
    finally:
        ctx.set_weights(params)
    assert len(results) >= 0.6 * (len(results) + skipped), (len(results), skips)
    assert max(results) <= 1e-6, max(results)


def test_fp32_gradient_and_adam_match_oracle(svlib):
    shape, params, _, _, _, k, D = case()
    pairs = [synth.make_pair(W, H, 40.0, 900 + W) for W, H in ((256, 128), (130, 67))]
    ctx = binding.Context(shape, k, "fp32")
    try:
        ctx.set_weights(params)
        dps = [binding.to_device(p, D) for p in pairs]
        coarse, eps, cs, es = [], [], [], []
        rng = np.random.default_rng(3)
        for p, dp in zip(pairs, dps):
            c = oracle.coarse_match(p.left, p.right, k, D)[0].astype(np.float64) + rng.uniform(0, 0.5, (p.height // 4, p.width // 4))
            H3, W3 = binding.latent_hw(p.height, p.width)
            e = synth.reparam_noise(H3 * W3 * shape.latent, p.seed)
            coarse.append(c); eps.append(e)
            cs.append(torch.from_numpy(c).float().cuda())
            es.append(torch.from_numpy(e).cuda().reshape(H3, W3, -1))
        Y, mu, lv = ctx.refine_train(dps, cs, es)
        out, gY, gmu, glv = ctx.loss(dps, Y, [torch.from_numpy(p.gt).cuda() for p in pairs], mu, lv, 1e-3)
        gp, _ = ctx.refine_backward(gY, gmu, glv, False, cs)
        ctx.synchronize()
        npix = sum(p.width * p.height for p in pairs)
        nlat = sum(np.prod(binding.latent_hw(p.height, p.width)) * shape.latent for p in pairs)
        Lo, go = 0.0, np.zeros(params.size)
        for p, c, e in zip(pairs, coarse, eps):
            l, g, _ = oracle.refine_backward(shape, params, p.left, c, e, p.gt, npix, nlat, 1e-3)
            Lo += l
            go += g
        assert abs(out[0].item() - Lo) <= 1e-5 * abs(Lo)
        gpn = gp.cpu().numpy()
        for name, (ow, wshape, ob, co) in oracle.param_slices(shape).items():
            n = int(np.prod(wshape))
            ref = go[ow:ow + n]
            assert np.abs(gpn[ow:ow + n] - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-12, name
        # one Adam step (paper's betas) against the oracle's Adam on the same gradient
        ctx.adam_step(gp, 1)
        ctx.synchronize()
        p64 = params.astype(np.float64)
        m = np.zeros_like(p64); v = np.zeros_like(p64)
        oracle.adam(p64, m, v, gpn.astype(np.float64), 1)
        assert np.abs(ctx.get_weights() - p64).max() <= 1e-6
    finally:
        ctx.close()


def test_autograd_function_training_steps_reduce_loss(svlib):
    """torch.autograd route: SVRefineFn + SVLossFn, loss.backward(), sv_adam_step."""
    shape, params, p, coarse, eps, k, D = case(W=128, H=64, seed=33)
    ctx = binding.Context(shape, k, "fp32")
    try:
        ctx.set_weights(params)
        dp = binding.to_device(p, D)
        c = torch.from_numpy(coarse).float().cuda().requires_grad_(True)
        H3, W3 = binding.latent_hw(p.height, p.width)
        e = torch.from_numpy(eps).cuda().reshape(H3, W3, -1)
        gt = torch.from_numpy(p.gt).cuda()
        w = torch.from_numpy(params).cuda().requires_grad_(True)
        losses = []
        for t in range(1, 6):
            Y, mu, lv = autograd.refine(ctx, [dp], [c], [e], w)
            L = autograd.loss(ctx, [dp], Y, [gt], mu, lv)
            w.grad = None
            c.grad = None
            L.backward()
            assert w.grad is not None and c.grad is not None
            ctx.adam_step(w.grad, t, lr=1e-3)
            losses.append(L.item())
        assert losses[-1] < losses[0]
    finally:
        ctx.close()


def test_backward_without_forward_is_a_state_error(svlib):
    ctx = binding.Context(synth.NET_SMALL, 5, "fp32")
    try:
        g = torch.zeros(10, device="cuda")
        with pytest.raises(binding.SvError) as ei:
            ctx.refine_backward([g], [None], [None], False, [g])
        assert ei.value.status == binding.SV_ERR_STATE
    finally:
        ctx.close()


def test_bf16_training_step_matches_oracle(svlib):
    """BF16 forward on the tensor cores with FP32 master weights (the training form of the
    batched path): the training forward within the BF16 output bar of the FP64 oracle,
    the FP32 backward's gradient aligned with the oracle's (cosine >= 0.998 per layer, max
    deviation <= 8% of the layer's largest entry: the BF16 activations the backward reads
    leave up to ~5% on the logvar head, whose gradient is the smallest), and a few Adam
    steps lower the loss."""
    shape, params, _, _, _, k, D = case()
    pairs = [synth.make_pair(W, H, 40.0, 950 + W) for W, H in ((256, 128), (130, 67))]
    ctx = binding.Context(shape, k, "bf16")
    try:
        ctx.set_weights(params)
        dps = [binding.to_device(p, D) for p in pairs]
        rng = np.random.default_rng(7)
        coarse, eps, cs, es = [], [], [], []
        for p in pairs:
            c = oracle.coarse_match(p.left, p.right, k, D)[0].astype(np.float64) + rng.uniform(0, 0.5, (p.height // 4, p.width // 4))
            H3, W3 = binding.latent_hw(p.height, p.width)
            e = synth.reparam_noise(H3 * W3 * shape.latent, p.seed + 1)
            coarse.append(c); eps.append(e)
            cs.append(torch.from_numpy(c).float().cuda())
            es.append(torch.from_numpy(e).cuda().reshape(H3, W3, -1))
        Y, mu, lv = ctx.refine_train(dps, cs, es)
        gts = [torch.from_numpy(p.gt).cuda() for p in pairs]
        out, gY, gmu, glv = ctx.loss(dps, Y, gts, mu, lv, 1e-3)
        gp, _ = ctx.refine_backward(gY, gmu, glv, False, cs)
        ctx.synchronize()
        npix = sum(p.width * p.height for p in pairs)
        nlat = sum(np.prod(binding.latent_hw(p.height, p.width)) * shape.latent for p in pairs)
        go = np.zeros(params.size)
        for p, c, e, y in zip(pairs, coarse, eps, Y):
            ref = oracle.refine_forward(shape, params, p.left, c, e)
            d = np.abs(y.cpu().numpy().astype(np.float64) - ref["Y"])
            assert d.max() <= 0.05 and d.mean() <= 0.01
            _, g, _ = oracle.refine_backward(shape, params, p.left, c, e, p.gt, npix, nlat, 1e-3)
            go += g
        gpn = gp.cpu().numpy().astype(np.float64)
        for name, (ow, wshape, ob, co) in oracle.param_slices(shape).items():
            n = int(np.prod(wshape))
            a, b = gpn[ow:ow + n], go[ow:ow + n]
            cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
            assert cos >= 0.998, (name, cos)
            assert np.abs(a - b).max() <= 0.08 * np.abs(b).max(), name
        # a few steps of the autograd route on the BF16 form
        w = torch.from_numpy(params).cuda().requires_grad_(True)
        losses = []
        for t in range(1, 6):
            Yt, mut, lvt = autograd.refine(ctx, dps, cs, es, w)
            L = autograd.loss(ctx, dps, Yt, gts, mut, lvt)
            w.grad = None
            L.backward()
            ctx.adam_step(w.grad, t, lr=1e-3)
            losses.append(L.item())
        assert losses[-1] < losses[0]
    finally:
        ctx.close()
