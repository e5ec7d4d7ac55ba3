"""torch.autograd.Functions over librosar's forward and adjoint kernels.

SparseAzimuthPhase:  out = sparse_azimuth(S * exp(j*eps), w, o) for a stack of scans sharing w;
                     gradients in S, eps (per scan and pulse) and w; gather or frequency-domain kernels.
RangeCompress:       S = range_compress(raw, win); gradient in raw through the adjoint FFT tile.
ImageL2Loss:         sum |out - ref|^2 and its gradient, one library pass each way.

Both follow torch's convention for complex tensors (the gradient passed around is the
conjugate-Wirtinger derivative of the real loss), so they compose with torch ops on either side.
The backward passes call only librosar kernels.
"""

from __future__ import annotations

import torch

from . import ops


class SparseAzimuthPhase(torch.autograd.Function):
    """method "gather": the gather kernels (rosar_sparse_azimuth_scans / _adjoint); "fft": the frequency-domain
    forms (plan H from w every forward, filter and adjoint filter with H and conj(H), weight gradient from the
    per-row cross-spectrum).  Both compute the same sums; "auto" picks "fft" where the row length allows it."""

    @staticmethod
    def forward(ctx, S, eps, w, o, method):
        S_t = ops.phase_apply(S.contiguous(), eps.contiguous())
        w = w.contiguous()
        H = None
        if method == "fft":
            H = ops.azimuth_plan(w, o, S.shape[2])
            out = ops.sparse_azimuth_fft_scans(S_t, H)
        else:
            out = ops.sparse_azimuth_scans(S_t, w, o)
        ctx.method = method
        ctx.save_for_backward(S_t, eps, w, o, H)
        return out

    @staticmethod
    def backward(ctx, g):
        S_t, eps, w, o, H = ctx.saved_tensors
        need_S, need_eps, need_w = ctx.needs_input_grad[:3]
        g = g.contiguous()
        if ctx.method == "fft":
            grad_S_t = ops.sparse_azimuth_fft_scans(g, H, adjoint=True) if (need_S or need_eps) else None
            grad_w = ops.azimuth_weight_grad_fft(g, S_t, o, w.shape[1]) if need_w else None
        else:
            grad_S_t, grad_w = ops.sparse_azimuth_adjoint(g, S_t, w, o, want_S=need_S or need_eps, want_w=need_w)
        grad_eps = grad_S = None
        if need_S or need_eps:
            grad_eps, grad_S = ops.phase_grad(S_t, grad_S_t, eps.contiguous(), want_eps=need_eps, want_S=need_S)
        return grad_S, grad_eps, grad_w, None, None


class RangeCompress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, raw, win, centred=True):
        ctx.win = win
        ctx.centred = centred
        return ops.range_compress(raw.contiguous(), win, centred=centred)

    @staticmethod
    def backward(ctx, g):
        return ops.range_compress_adjoint(g.contiguous(), ctx.win, centred=ctx.centred), None, None


class ImageL2Loss(torch.autograd.Function):
    """loss = sum |out - ref|^2 in one library pass each way (rosar_image_l2_loss / _grad); ref may also
    require a gradient (its gradient is the negative of out's)."""

    @staticmethod
    def forward(ctx, out, ref):
        out, ref = out.contiguous(), ref.contiguous()
        ctx.save_for_backward(out, ref)
        return ops.image_l2_loss(out, ref)

    @staticmethod
    def backward(ctx, g):
        out, ref = ctx.saved_tensors
        grad = ops.image_l2_loss_grad(out, ref, g.to(torch.float32).contiguous())
        return grad, (-grad if ctx.needs_input_grad[1] else None)


def image_l2_loss(out, ref):
    """Differentiable squared L2 distance between two complex stacks (e.g. images and reference images)."""
    return ImageL2Loss.apply(out, ref)


# the frequency-domain forms keep three rows of n_az in shared memory for the weight gradient
_FFT_MAX_N_AZ = 8400


def sparse_azimuth_phase(S, eps, w, o, method="auto"):
    """Differentiable sparse azimuth filter with per-pulse phase correction, S [n_scans, n_rng, n_az].
    method: "auto", "fft" or "gather" (see SparseAzimuthPhase)."""
    n_az = S.shape[2]
    if method == "auto":
        method = "fft" if (ops.azimuth_fft_supported(n_az) and n_az <= _FFT_MAX_N_AZ) else "gather"
    if method not in ("fft", "gather"):
        raise ValueError("method must be 'auto', 'fft' or 'gather'")
    return SparseAzimuthPhase.apply(S, eps, w, o, method)


def range_compress(raw, win=None, centred=True):
    """Differentiable range compression of one scan, raw [n_az, L] -> S [L, n_az], or of a stack of scans,
    raw [n_scans, n_az, L] -> S [n_scans, L, n_az] (one launch each way)."""
    return RangeCompress.apply(raw, win, centred)
