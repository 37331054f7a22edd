"""torch.autograd bindings of the differentiation form.

SVRefineFn: training forward (sv_refine_train) and its hand-written backward
(sv_refine_backward) for a batch of pairs.  The network weights live in the library
context; a `params` tensor is passed through so that autograd delivers d loss / d params
to it.  SVLossFn: the loss of sv_loss with its gradients.  Both only marshal arguments:
all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import torch


class SVRefineFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sv, pairs, eps, params, *coarse):
        Y, mu, lv = sv.refine_train(pairs, list(coarse), list(eps))
        fctx.sv = sv
        fctx.n = len(pairs)
        fctx.coarse = coarse
        return (*Y, *mu, *lv)

    @staticmethod
    def backward(fctx, *grads):
        n = fctx.n
        gY = [g.contiguous() for g in grads[:n]]
        gmu = [None if g is None else g.contiguous() for g in grads[n:2 * n]]
        glv = [None if g is None else g.contiguous() for g in grads[2 * n:3 * n]]
        want_c = any(fctx.needs_input_grad[4:])
        gparams, gc = fctx.sv.refine_backward(gY, gmu, glv, want_c, fctx.coarse)
        return (None, None, None, gparams, *(gc if want_c else [None] * n))


def refine(sv, pairs, coarse, eps, params):
    """Differentiable refinement: returns (Y list, mu list, logvar list)."""
    out = SVRefineFn.apply(sv, pairs, eps, params, *coarse)
    n = len(pairs)
    return list(out[:n]), list(out[n:2 * n]), list(out[2 * n:])


class SVLossFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sv, pairs, gt, kl_weight, n, *tensors):
        Y, mu, lv = list(tensors[:n]), list(tensors[n:2 * n]), list(tensors[2 * n:])
        out, gY, gmu, glv = sv.loss(pairs, Y, gt, mu, lv, kl_weight, want_grads=True)
        fctx.save_for_backward(*gY, *gmu, *glv)
        return out[0].clone()

    @staticmethod
    def backward(fctx, g):
        return (None, None, None, None, None, *[t * g for t in fctx.saved_tensors])


def loss(sv, pairs, Y, gt, mu, lv, kl_weight=1e-3):
    return SVLossFn.apply(sv, pairs, gt, kl_weight, len(pairs), *Y, *mu, *lv)
