"""torch.autograd.Functions over librosar's forward and adjoint kernels.

SparseAzimuthPhase:  out = sparse_azimuth(S * exp(j*eps), w, o) for a stack of scans sharing w;
                     gradients in S, eps (per scan and pulse) and w.
RangeCompress:       S = range_compress(raw, win); gradient in raw through the adjoint FFT tile.

Both follow torch's convention for complex tensors (the gradient passed around is the
conjugate-Wirtinger derivative of the real loss), so they compose with torch ops on either side.
The backward passes call only librosar kernels.
"""

from __future__ import annotations

import torch

from . import ops


class SparseAzimuthPhase(torch.autograd.Function):
    @staticmethod
    def forward(ctx, S, eps, w, o):
        S_t = ops.phase_apply(S.contiguous(), eps.contiguous())
        out = ops.sparse_azimuth_scans(S_t, w.contiguous(), o)
        ctx.save_for_backward(S_t, eps, w, o)
        return out

    @staticmethod
    def backward(ctx, g):
        S_t, eps, w, o = ctx.saved_tensors
        need_S, need_eps, need_w = ctx.needs_input_grad[:3]
        g = g.contiguous()
        grad_S_t, grad_w = ops.sparse_azimuth_adjoint(g, S_t, w.contiguous(), o, want_S=need_S or need_eps,
                                                      want_w=need_w)
        grad_eps = grad_S = None
        if need_S or need_eps:
            grad_eps, grad_S = ops.phase_grad(S_t, grad_S_t, eps.contiguous(), want_eps=need_eps, want_S=need_S)
        return grad_S, grad_eps, grad_w, None


class RangeCompress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, raw, win, centred=True):
        ctx.win = win
        ctx.centred = centred
        return ops.range_compress(raw.contiguous(), win, centred=centred)

    @staticmethod
    def backward(ctx, g):
        return ops.range_compress_adjoint(g.contiguous(), ctx.win, centred=ctx.centred), None, None


def sparse_azimuth_phase(S, eps, w, o):
    """Differentiable sparse azimuth filter with per-pulse phase correction, S [n_scans, n_rng, n_az]."""
    return SparseAzimuthPhase.apply(S, eps, w, o)


def range_compress(raw, win=None, centred=True):
    """Differentiable range compression of one scan, raw [n_az, L] -> S [L, n_az]."""
    return RangeCompress.apply(raw, win, centred)
