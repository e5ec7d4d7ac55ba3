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


# The frequency-domain form keeps no phase-corrected copy S_t = S exp(j eps) in memory: the phase factors are
# computed once per (scan, pulse) and applied as the filter and the phase gradient load S.  When the weights
# need a gradient, the forward filter and the adjoint filter also store their rows' transforms, and the weight
# gradient is one inverse transform per row of their cross-spectrum.
FUSED_PHASE = True
SPECTRA = True


class SparseAzimuthPhase(torch.autograd.Function):
    """method "gather": the gather kernels (rosar_sparse_azimuth_scans / _adjoint) on S_t = S exp(j eps) from
    rosar_phase_apply; "fft": the frequency-domain forms (plan H from w every forward, filter and adjoint filter with
    H and conj(H), weight gradient from the per-row cross-spectrum), each forming S exp(j eps) as it loads S.  Both
    compute the same sums; "auto" picks "fft" where the row length allows it."""

    @staticmethod
    def forward(ctx, S, eps, w, o, method, keep_spectra):
        S = S.contiguous()
        w = w.contiguous()
        ctx.method = method
        if method == "fft":
            P = ops.phasors(eps.contiguous())
            H = ops.azimuth_plan(w, o, S.shape[2])
            X = torch.empty_like(S) if (keep_spectra and ctx.needs_input_grad[2]) else None
            out = ops.sparse_azimuth_fft_scans_ex(S, H, P=P, spectrum=X)
            ctx.save_for_backward(S, P, w, o, H, X)
        else:
            S_t = ops.phase_apply(S, eps.contiguous())
            out = ops.sparse_azimuth_scans(S_t, w, o)
            ctx.save_for_backward(S_t, eps, w, o)
        return out

    @staticmethod
    def backward(ctx, g):
        need_S, need_eps, need_w = ctx.needs_input_grad[:3]
        g = g.contiguous()
        grad_eps = grad_S = grad_w = None
        if ctx.method == "fft":
            S, P, w, o, H, X = ctx.saved_tensors
            G = torch.empty_like(g) if need_w else None
            grad_S_t = ops.sparse_azimuth_fft_scans_ex(g, H, adjoint=True, spectrum=G) if (need_S or need_eps or need_w) \
                else None
            grad_w = ops.azimuth_weight_grad_spectra(G, X, o, w.shape[1]) if need_w else None
            if need_S or need_eps:
                grad_eps, grad_S = ops.phase_grad_phasor(S, P, grad_S_t, want_eps=need_eps, want_S=need_S)
        else:
            S_t, eps, w, o = ctx.saved_tensors
            grad_S_t, grad_w = ops.sparse_azimuth_adjoint(g, S_t, w, o, want_S=need_S or need_eps, want_w=need_w)
            if need_S or need_eps:
                grad_eps, grad_S = ops.phase_grad(S_t, grad_S_t, eps.contiguous(), want_eps=need_eps, want_S=need_S)
        return grad_S, grad_eps, grad_w, None, None, None


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
    # the forward filter keeps its spectra only when a backward pass can follow (grad mode on)
    return SparseAzimuthPhase.apply(S, eps, w, o, method, torch.is_grad_enabled())


def range_compress(raw, win=None, centred=True):
    """Differentiable range compression of one scan, raw [n_az, L] -> S [L, n_az], or of a stack of scans,
    raw [n_scans, n_az, L] -> S [n_scans, L, n_az] (one launch each way)."""
    return RangeCompress.apply(raw, win, centred)
