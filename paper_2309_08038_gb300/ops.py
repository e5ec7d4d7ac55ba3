"""Python entry points with the C ABI's names (rosar_range_compress -> range_compress, ...).

Each function validates tensor metadata, allocates outputs with torch when none
are given, and calls one C-ABI entry point; all arithmetic is in librosar's kernels.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import check, ptr, require, stream_handle

C_LIGHT = 299792458.0


@dataclass(frozen=True)
class Radar:
    """FMCW radar on a rotating arm (mirrors the C struct rosar_radar)."""

    fc_hz: float
    slope_hz_per_s: float
    t_sample_s: float
    t_start_s: float
    r0_m: float
    c_mps: float = C_LIGHT

    def as_struct(self) -> _lib.RadarStruct:
        return _lib.RadarStruct(self.fc_hz, self.slope_hz_per_s, self.t_sample_s, self.t_start_s, self.r0_m,
                                self.c_mps)

    def bin_spacing(self, L: int) -> float:
        return self.c_mps / (2.0 * self.slope_hz_per_s * self.t_sample_s * L)


def range_compress(raw, win=None, centred=True, out=None, stream=None):
    """rosar_range_compress: raw [n_az, L] complex64 -> S [L, n_az] complex64 (range-major); a stack
    raw [n_scans, n_az, L] -> S [n_scans, L, n_az] goes through rosar_range_compress_scans (one launch)."""
    lib = _lib.load()
    if not isinstance(raw, torch.Tensor) or raw.dim() not in (2, 3):
        raise ValueError("raw must be a [n_az, L] or [n_scans, n_az, L] tensor")
    require(raw, torch.complex64, "raw", ndim=raw.dim())
    *lead, n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    shape = (*lead, L, n_az)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex64, device=raw.device)
    require(out, torch.complex64, "out", shape=shape)
    if lead:
        check(lib.rosar_range_compress_scans(ptr(raw), ptr(win), lead[0], n_az, L, int(bool(centred)), ptr(out),
                                             stream_handle(stream)))
    else:
        check(lib.rosar_range_compress(ptr(raw), ptr(win), n_az, L, int(bool(centred)), ptr(out),
                                       stream_handle(stream)))
    return out


def _offsets(o, n_rng, K):
    require(o, torch.int32, "o")
    if o.dim() == 1:
        if o.shape[0] != K:
            raise ValueError(f"shared offsets must have shape ({K},), got {tuple(o.shape)}")
        return 0
    if o.dim() == 2 and o.shape == (n_rng, K):
        return K
    raise ValueError(f"offsets must be [K] or [n_rng, K], got {tuple(o.shape)}")


def sparse_azimuth(S, w, o, out=None, stream=None):
    """rosar_sparse_azimuth: out[r, t] = sum_k w[r, k] * S[r, (t + o_k) mod n_az]."""
    lib = _lib.load()
    require(S, torch.complex64, "S", ndim=2)
    n_rng, n_az = S.shape
    require(w, torch.complex64, "w", ndim=2)
    if w.shape[0] != n_rng:
        raise ValueError(f"w must have {n_rng} rows, got {tuple(w.shape)}")
    K = w.shape[1]
    stride = _offsets(o, n_rng, K)
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=S.device)
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    check(lib.rosar_sparse_azimuth(ptr(S), ptr(w), ptr(o), stride, n_rng, n_az, K, ptr(out), stream_handle(stream)))
    return out


def bpa(S, radar: Radar, n_rng, M_ap, interp="linear", dphi=None, dr=None, out=None, stream=None):
    """rosar_bpa: back-projection of the centred range-compressed S [L, n_az] onto rows 0..n_rng-1."""
    lib = _lib.load()
    require(S, torch.complex64, "S", ndim=2)
    L, n_az = S.shape
    if dphi is not None:
        require(dphi, torch.float32, "dphi", shape=(n_az,))
    if dr is not None:
        require(dr, torch.float32, "dr", shape=(n_az,))
    if interp not in ("linear", "nearest"):
        raise ValueError("interp must be 'linear' or 'nearest'")
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=S.device)
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    st = radar.as_struct()
    check(lib.rosar_bpa(ptr(S), ctypes.byref(st), ptr(dphi), ptr(dr), L, n_rng, n_az, M_ap,
                        1 if interp == "linear" else 0, ptr(out), stream_handle(stream)))
    return out


def image_fft_host(raw_host, win, H, raw_dev, workspace, out_dev, out_host, stream=None):
    """rosar_image_fft_host: raw_host (CPU tensor, page-locked for asynchronous copies) -> H2D into raw_dev,
    range compression + frequency-domain azimuth filter into out_dev, D2H into out_host (CPU tensor), all
    enqueued on `stream`; out_host is valid once the stream is synchronised."""
    import torch
    lib = _lib.load()
    if not isinstance(raw_host, torch.Tensor) or raw_host.is_cuda or not isinstance(out_host, torch.Tensor) or \
            out_host.is_cuda:
        raise ValueError("raw_host and out_host must be CPU tensors")
    if raw_host.dtype != torch.complex64 or out_host.dtype != torch.complex64 or raw_host.dim() != 2 or \
            not raw_host.is_contiguous() or not out_host.is_contiguous():
        raise ValueError("raw_host and out_host must be contiguous complex64 matrices")
    n_az, L = raw_host.shape
    if tuple(out_host.shape) != (L, n_az):
        raise ValueError(f"out_host must have shape ({L}, {n_az})")
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(H, torch.complex64, "H", shape=(L, n_az))
    require(raw_dev, torch.complex64, "raw_dev", shape=(n_az, L))
    require(workspace, torch.complex64, "workspace", shape=(L, n_az))
    require(out_dev, torch.complex64, "out_dev", shape=(L, n_az))
    check(lib.rosar_image_fft_host(ctypes.c_void_p(raw_host.data_ptr()), ptr(win), ptr(H), n_az, L, ptr(raw_dev),
                                   ptr(workspace), ptr(out_dev), ctypes.c_void_p(out_host.data_ptr()),
                                   stream_handle(stream)))
    return out_host


def bpa_time(raw, win, radar: Radar, n_rng, M_ap, out=None, stream=None):
    """rosar_bpa_time: time-domain back-projection (Eq. (14)) of the raw cube [n_az, L] onto rows 0..n_rng-1."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=raw.device)
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    st = radar.as_struct()
    check(lib.rosar_bpa_time(ptr(raw), ptr(win), ctypes.byref(st), n_az, L, n_rng, M_ap, ptr(out),
                             stream_handle(stream)))
    return out


def sas_time(raw, win, w, o, radar: Radar, centred=True, out=None, stream=None):
    """rosar_sas_time: time-domain sparse-aperture imaging (Algorithm 2) of the raw cube [n_az, L]; one output
    row per row of w [n_rng, K]."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(w, torch.complex64, "w", ndim=2)
    n_rng, K = w.shape
    stride = _offsets(o, n_rng, K)
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=raw.device)
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    st = radar.as_struct()
    check(lib.rosar_sas_time(ptr(raw), ptr(win), ptr(w), ptr(o), stride, ctypes.byref(st), n_az, L, n_rng, K,
                             1 if centred else 0, ptr(out), stream_handle(stream)))
    return out


@dataclass(frozen=True)
class TimeDomainPlan:
    """The precomputed B operand of the tensor-core time-domain forms (rosar_*_time_plan): a uint8 device tensor
    of rosar_time_domain_plan_bytes(n_rng, L, K) bytes (the taps' B tiles in ascending offset order and the
    sorted offsets), with the shape it was made for."""

    data: torch.Tensor
    n_az: int
    L: int
    n_rng: int
    K: int


def _plan_tensor(n_rng, L, K, device):
    nbytes = int(_lib.load().rosar_time_domain_plan_bytes(n_rng, L, K))
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def sas_time_plan(win, w, o, radar: Radar, n_az, L, centred=True, stream=None):
    """rosar_sas_time_plan: the B operand of rosar_sas_time for the weights w [n_rng, K] and shared offsets o [K]."""
    lib = _lib.load()
    require(w, torch.complex64, "w", ndim=2)
    n_rng, K = w.shape
    require(o, torch.int32, "o", shape=(K,))
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    data = _plan_tensor(n_rng, L, K, w.device)
    st = radar.as_struct()
    check(lib.rosar_sas_time_plan(ptr(win), ptr(w), ptr(o), ctypes.byref(st), n_az, L, n_rng, K, 1 if centred else 0,
                                  ptr(data), data.numel(), stream_handle(stream)))
    return TimeDomainPlan(data, n_az, L, n_rng, K)


def sas_time_planned(raw, plan: TimeDomainPlan, out=None, stream=None):
    """rosar_sas_time_planned: rosar_sas_time of raw [n_az, L] with a plan from sas_time_plan (which holds the
    offsets)."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", shape=(plan.n_az, plan.L))
    if out is None:
        out = torch.empty((plan.n_rng, plan.n_az), dtype=torch.complex64, device=raw.device)
    require(out, torch.complex64, "out", shape=(plan.n_rng, plan.n_az))
    check(lib.rosar_sas_time_planned(ptr(raw), ptr(plan.data), plan.n_az, plan.L, plan.n_rng, plan.K, ptr(out),
                                     stream_handle(stream)))
    return out


def bpa_time_plan(win, radar: Radar, n_az, L, n_rng, M_ap, device=None, stream=None):
    """rosar_bpa_time_plan: the B operand of rosar_bpa_time (M_ap taps of the nominal geometry)."""
    lib = _lib.load()
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    device = win.device if win is not None else (device or torch.device("cuda"))
    data = _plan_tensor(n_rng, L, M_ap, device)
    st = radar.as_struct()
    check(lib.rosar_bpa_time_plan(ptr(win), ctypes.byref(st), n_az, L, n_rng, M_ap, ptr(data), data.numel(),
                                  stream_handle(stream)))
    return TimeDomainPlan(data, n_az, L, n_rng, M_ap)


def bpa_time_planned(raw, plan: TimeDomainPlan, out=None, stream=None):
    """rosar_bpa_time_planned: rosar_bpa_time of raw [n_az, L] with a plan from bpa_time_plan."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", shape=(plan.n_az, plan.L))
    if out is None:
        out = torch.empty((plan.n_rng, plan.n_az), dtype=torch.complex64, device=raw.device)
    require(out, torch.complex64, "out", shape=(plan.n_rng, plan.n_az))
    check(lib.rosar_bpa_time_planned(ptr(raw), ptr(plan.data), plan.n_az, plan.L, plan.n_rng, plan.K, ptr(out),
                                     stream_handle(stream)))
    return out


def image(raw, win, w, o, workspace=None, out=None, stream=None):
    """rosar_image: range compression into `workspace`, then the sparse azimuth filter into `out`."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(w, torch.complex64, "w", shape=(L, w.shape[1]) if w.dim() == 2 else None)
    K = w.shape[1]
    stride = _offsets(o, L, K)
    if workspace is None:
        workspace = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    if out is None:
        out = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    require(workspace, torch.complex64, "workspace", shape=(L, n_az))
    require(out, torch.complex64, "out", shape=(L, n_az))
    check(lib.rosar_image(ptr(raw), ptr(win), ptr(w), ptr(o), stride, n_az, L, K, ptr(workspace), ptr(out),
                          stream_handle(stream)))
    return out


def image_noalloc(raw, win, w, o, out=None, stream=None):
    """rosar_image_noalloc: the same image as `image`, for callers that cannot allocate device
    scratch (the range-compressed intermediate lives in a fixed 16 MiB array inside librosar).
    L * n_az must not exceed NOALLOC_MAX_ELEMS; concurrent calls on different streams race."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(w, torch.complex64, "w", ndim=2)
    K = w.shape[1]
    stride = _offsets(o, L, K)
    if out is None:
        out = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    require(out, torch.complex64, "out", shape=(L, n_az))
    check(lib.rosar_image_noalloc(ptr(raw), ptr(win), ptr(w), ptr(o), stride, n_az, L, K, ptr(out),
                                  stream_handle(stream)))
    return out


def azimuth_fft_supported(n_az: int) -> bool:
    """True if the frequency-domain azimuth filter handles n_az (2^a 3^b 5^c <= 16384)."""
    return bool(_lib.load().rosar_azimuth_fft_supported(int(n_az)))


def azimuth_plan(w, o, n_az, out=None, stream=None):
    """rosar_azimuth_plan: H [n_rng, n_az] = FFT(g_r)/n_az for the weights w [n_rng, K] and offsets o."""
    lib = _lib.load()
    require(w, torch.complex64, "w", ndim=2)
    n_rng, K = w.shape
    stride = _offsets(o, n_rng, K)
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=w.device)
    require(out, torch.complex64, "H", shape=(n_rng, n_az))
    check(lib.rosar_azimuth_plan(ptr(w), ptr(o), stride, n_rng, n_az, K, ptr(out), stream_handle(stream)))
    return out


def sparse_azimuth_fft(S, H, out=None, stream=None):
    """rosar_sparse_azimuth_fft: the sparse azimuth filter of S [n_rng, n_az] through its plan H."""
    lib = _lib.load()
    require(S, torch.complex64, "S", ndim=2)
    n_rng, n_az = S.shape
    require(H, torch.complex64, "H", shape=(n_rng, n_az))
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=S.device)
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    check(lib.rosar_sparse_azimuth_fft(ptr(S), ptr(H), n_rng, n_az, ptr(out), stream_handle(stream)))
    return out


def image_fft(raw, win, H, workspace=None, out=None, stream=None):
    """rosar_image_fft: range compression, then the frequency-domain azimuth filter with plan H [L, n_az]."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(H, torch.complex64, "H", shape=(L, n_az))
    if workspace is None:
        workspace = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    if out is None:
        out = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    require(workspace, torch.complex64, "workspace", shape=(L, n_az))
    require(out, torch.complex64, "out", shape=(L, n_az))
    check(lib.rosar_image_fft(ptr(raw), ptr(win), ptr(H), n_az, L, ptr(workspace), ptr(out), stream_handle(stream)))
    return out


def image_fft_scans(raw, win, H, workspace=None, out=None, stream=None):
    """rosar_image_fft_scans: rosar_image_fft of every scan of raw [n_scans, n_az, L] with one plan H [L, n_az],
    consecutive scans overlapped where a pipelined plan exists; workspace [2, L, n_az], out [n_scans, L, n_az]."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=3)
    n_scans, n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(H, torch.complex64, "H", shape=(L, n_az))
    if workspace is None:
        workspace = torch.empty((2, L, n_az), dtype=torch.complex64, device=raw.device)
    if out is None:
        out = torch.empty((n_scans, L, n_az), dtype=torch.complex64, device=raw.device)
    require(workspace, torch.complex64, "workspace", shape=(2, L, n_az))
    require(out, torch.complex64, "out", shape=(n_scans, L, n_az))
    check(lib.rosar_image_fft_scans(ptr(raw), ptr(win), ptr(H), n_scans, n_az, L, ptr(workspace), ptr(out),
                                    stream_handle(stream)))
    return out


def image_fft_scans_pipelined(L, n_az):
    """rosar_image_fft_scans_pipelined: True if image_fft_scans overlaps consecutive scans for (L, n_az)."""
    return bool(_lib.load().rosar_image_fft_scans_pipelined(int(L), int(n_az)))


# ------------------------------------------------------------------ differentiable form --

def _stack(S, name):
    require(S, torch.complex64, name, ndim=3)
    return S.shape


def phase_apply(S, eps, out=None, stream=None):
    """rosar_phase_apply: S_t [n_scans, n_rng, n_az] = S * exp(j*eps[:, None, :])."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S, "S")
    require(eps, torch.float32, "eps", shape=(n_scans, n_az))
    if out is None:
        out = torch.empty_like(S)
    require(out, torch.complex64, "S_t", shape=(n_scans, n_rng, n_az))
    check(lib.rosar_phase_apply(ptr(S), ptr(eps), n_scans, n_rng, n_az, ptr(out), stream_handle(stream)))
    return out


def sparse_azimuth_scans(S, w, o, out=None, stream=None):
    """rosar_sparse_azimuth_scans: the sparse azimuth filter of each scan of S [n_scans, n_rng, n_az]."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S, "S")
    require(w, torch.complex64, "w", ndim=2)
    K = w.shape[1]
    stride = _offsets(o, n_rng, K)
    if out is None:
        out = torch.empty_like(S)
    require(out, torch.complex64, "out", shape=(n_scans, n_rng, n_az))
    check(lib.rosar_sparse_azimuth_scans(ptr(S), ptr(w), ptr(o), stride, n_scans, n_rng, n_az, K, ptr(out),
                                         stream_handle(stream)))
    return out


def sparse_azimuth_adjoint(g, S_t, w, o, want_S=True, want_w=True, stream=None):
    """rosar_sparse_azimuth_adjoint: (grad_S_t or None, grad_w or None) for the image gradient g."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(g, "g")
    require(w, torch.complex64, "w", ndim=2)
    K = w.shape[1]
    stride = _offsets(o, n_rng, K)
    if want_w:
        require(S_t, torch.complex64, "S_t", shape=(n_scans, n_rng, n_az))
    gS = torch.empty_like(g) if want_S else None
    gw = torch.empty_like(w) if want_w else None
    check(lib.rosar_sparse_azimuth_adjoint(ptr(g), ptr(S_t) if want_w else None, ptr(w), ptr(o), stride, n_scans,
                                           n_rng, n_az, K, ptr(gS), ptr(gw), stream_handle(stream)))
    return gS, gw


def sparse_azimuth_fft_scans(S, H, adjoint=False, out=None, stream=None):
    """rosar_sparse_azimuth_fft_scans: the frequency-domain filter of every scan of S [n_scans, n_rng, n_az]
    with the shared plan H [n_rng, n_az]; adjoint=True filters with conj(H) (the filter's adjoint)."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S, "S")
    require(H, torch.complex64, "H", shape=(n_rng, n_az))
    if out is None:
        out = torch.empty_like(S)
    require(out, torch.complex64, "out", shape=(n_scans, n_rng, n_az))
    check(lib.rosar_sparse_azimuth_fft_scans(ptr(S), ptr(H), n_scans, n_rng, n_az, 1 if adjoint else 0, ptr(out),
                                             stream_handle(stream)))
    return out


def azimuth_weight_grad_fft(g, S_t, o, K, out=None, stream=None):
    """rosar_azimuth_weight_grad_fft: grad_w [n_rng, K] from the per-row cross-spectrum of g and S_t."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(g, "g")
    require(S_t, torch.complex64, "S_t", shape=(n_scans, n_rng, n_az))
    stride = _offsets(o, n_rng, K)
    if out is None:
        out = torch.empty((n_rng, K), dtype=torch.complex64, device=g.device)
    require(out, torch.complex64, "grad_w", shape=(n_rng, K))
    check(lib.rosar_azimuth_weight_grad_fft(ptr(g), ptr(S_t), ptr(o), stride, n_scans, n_rng, n_az, K, ptr(out),
                                            stream_handle(stream)))
    return out


def phasors(eps, out=None, stream=None):
    """rosar_phasors: P = exp(j*eps) elementwise (eps float32, any shape; P complex64 of the same shape)."""
    lib = _lib.load()
    require(eps, torch.float32, "eps", ndim=eps.dim())
    if out is None:
        out = torch.empty(eps.shape, dtype=torch.complex64, device=eps.device)
    require(out, torch.complex64, "P", shape=tuple(eps.shape))
    check(lib.rosar_phasors(ptr(eps), eps.numel(), ptr(out), stream_handle(stream)))
    return out


def sparse_azimuth_fft_scans_ex(S, H, P=None, adjoint=False, spectrum=None, out=None, stream=None):
    """rosar_sparse_azimuth_fft_scans_ex: the frequency-domain filter (adjoint: with conj(H)) of S [n_scans, n_rng,
    n_az], each scan's columns multiplied by P [n_scans, n_az] as they are loaded (P None: none); spectrum (a tensor
    like S, or None) receives the rows' forward transforms."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S, "S")
    if P is not None:
        require(P, torch.complex64, "P", shape=(n_scans, n_az))
    require(H, torch.complex64, "H", shape=(n_rng, n_az))
    if spectrum is not None:
        require(spectrum, torch.complex64, "spectrum", shape=(n_scans, n_rng, n_az))
    if out is None:
        out = torch.empty_like(S)
    require(out, torch.complex64, "out", shape=(n_scans, n_rng, n_az))
    check(lib.rosar_sparse_azimuth_fft_scans_ex(ptr(S), ptr(P), ptr(H), n_scans, n_rng, n_az, int(bool(adjoint)),
                                                ptr(out), ptr(spectrum), stream_handle(stream)))
    return out


def azimuth_weight_grad_spectra(G, X, o, K, workspace=None, out=None, stream=None):
    """rosar_azimuth_weight_grad_spectra: grad_w [n_rng, K] from the adjoint call's spectrum G and the forward call's
    spectrum X (both [n_scans, n_rng, n_az]); workspace [n_rng, n_az] holds the cross-spectrum."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(X, "X")
    require(G, torch.complex64, "G", shape=(n_scans, n_rng, n_az))
    stride = _offsets(o, n_rng, K)
    if workspace is None:
        workspace = torch.empty((n_rng, n_az), dtype=torch.complex64, device=X.device)
    require(workspace, torch.complex64, "workspace", shape=(n_rng, n_az))
    if out is None:
        out = torch.empty((n_rng, K), dtype=torch.complex64, device=X.device)
    require(out, torch.complex64, "grad_w", shape=(n_rng, K))
    check(lib.rosar_azimuth_weight_grad_spectra(ptr(G), ptr(X), ptr(o), stride, n_scans, n_rng, n_az, K,
                                                ptr(workspace), ptr(out), stream_handle(stream)))
    return out


def azimuth_weight_grad_fft_phase(g, S, P, o, K, out=None, stream=None):
    """rosar_azimuth_weight_grad_fft_phase: rosar_azimuth_weight_grad_fft with S_t = S * P formed at load."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S, "S")
    require(g, torch.complex64, "g", shape=(n_scans, n_rng, n_az))
    require(P, torch.complex64, "P", shape=(n_scans, n_az))
    stride = _offsets(o, n_rng, K)
    if out is None:
        out = torch.empty((n_rng, K), dtype=torch.complex64, device=S.device)
    require(out, torch.complex64, "grad_w", shape=(n_rng, K))
    check(lib.rosar_azimuth_weight_grad_fft_phase(ptr(g), ptr(S), ptr(P), ptr(o), stride, n_scans, n_rng, n_az, K,
                                                  ptr(out), stream_handle(stream)))
    return out


def phase_grad_phasor(S, P, grad_S_t, want_eps=True, want_S=False, stream=None):
    """rosar_phase_grad_phasor: (grad_eps [n_scans, n_az] or None, grad_S or None) with S_t = S * P formed at load."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S, "S")
    require(P, torch.complex64, "P", shape=(n_scans, n_az))
    require(grad_S_t, torch.complex64, "grad_S_t", shape=(n_scans, n_rng, n_az))
    ge = torch.empty((n_scans, n_az), dtype=torch.float32, device=S.device) if want_eps else None
    gS = torch.empty_like(S) if want_S else None
    check(lib.rosar_phase_grad_phasor(ptr(S), ptr(P), ptr(grad_S_t), n_scans, n_rng, n_az, ptr(ge), ptr(gS),
                                      stream_handle(stream)))
    return ge, gS


def phase_grad(S_t, grad_S_t, eps, want_eps=True, want_S=False, stream=None):
    """rosar_phase_grad: (grad_eps [n_scans, n_az] or None, grad_S or None)."""
    lib = _lib.load()
    n_scans, n_rng, n_az = _stack(S_t, "S_t")
    require(grad_S_t, torch.complex64, "grad_S_t", shape=(n_scans, n_rng, n_az))
    require(eps, torch.float32, "eps", shape=(n_scans, n_az))
    ge = torch.empty((n_scans, n_az), dtype=torch.float32, device=S_t.device) if want_eps else None
    gS = torch.empty_like(S_t) if want_S else None
    check(lib.rosar_phase_grad(ptr(S_t), ptr(grad_S_t), ptr(eps), n_scans, n_rng, n_az, ptr(ge), ptr(gS),
                               stream_handle(stream)))
    return ge, gS


def range_compress_adjoint(g, win=None, centred=True, out=None, stream=None):
    """rosar_range_compress_adjoint: g [L, n_az] -> grad_raw [n_az, L]; a stack g [n_scans, L, n_az] ->
    grad_raw [n_scans, n_az, L] goes through rosar_range_compress_adjoint_scans (one launch)."""
    lib = _lib.load()
    if not isinstance(g, torch.Tensor) or g.dim() not in (2, 3):
        raise ValueError("g must be a [L, n_az] or [n_scans, L, n_az] tensor")
    require(g, torch.complex64, "g", ndim=g.dim())
    *lead, L, n_az = g.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    shape = (*lead, n_az, L)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex64, device=g.device)
    require(out, torch.complex64, "grad_raw", shape=shape)
    if lead:
        check(lib.rosar_range_compress_adjoint_scans(ptr(g), ptr(win), lead[0], n_az, L, int(bool(centred)),
                                                     ptr(out), stream_handle(stream)))
    else:
        check(lib.rosar_range_compress_adjoint(ptr(g), ptr(win), n_az, L, int(bool(centred)), ptr(out),
                                               stream_handle(stream)))
    return out


def image_l2_loss(out, ref, stream=None):
    """rosar_image_l2_loss: sum |out - ref|^2 over two complex stacks of one shape, as a 0-d float32 tensor
    (deterministic order)."""
    lib = _lib.load()
    require(out, torch.complex64, "out")
    require(ref, torch.complex64, "ref", shape=tuple(out.shape))
    ws = torch.empty(int(lib.rosar_image_l2_loss_workspace_bytes()) // 8, dtype=torch.float64, device=out.device)
    loss = torch.empty((), dtype=torch.float32, device=out.device)
    check(lib.rosar_image_l2_loss(ptr(out), ptr(ref), out.numel(), ptr(ws), ptr(loss), stream_handle(stream)))
    return loss


def image_l2_loss_grad(out, ref, g, grad=None, stream=None):
    """rosar_image_l2_loss_grad: 2 g (out - ref) for the upstream gradient g (a 0-d float32 CUDA tensor)."""
    lib = _lib.load()
    require(out, torch.complex64, "out")
    require(ref, torch.complex64, "ref", shape=tuple(out.shape))
    require(g, torch.float32, "g", shape=())
    if grad is None:
        grad = torch.empty_like(out)
    require(grad, torch.complex64, "grad", shape=tuple(out.shape))
    check(lib.rosar_image_l2_loss_grad(ptr(out), ptr(ref), out.numel(), ptr(g), ptr(grad), stream_handle(stream)))
    return grad


# ------------------------------------------------------------ range-migration-aware taps --

def sparse_azimuth_migrating(S, w, o, dl, n_rng=None, out=None, stream=None):
    """rosar_sparse_azimuth_migrating: tap k of row r reads row r + dl[r, k] of S [n_bins, n_az]."""
    lib = _lib.load()
    require(S, torch.complex64, "S", ndim=2)
    n_bins, n_az = S.shape
    require(w, torch.complex64, "w", ndim=2)
    n_rng = w.shape[0] if n_rng is None else n_rng
    K = w.shape[1]
    stride = _offsets(o, n_rng, K)
    require(dl, torch.int32, "dl", shape=(n_rng, K))
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=S.device)
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    check(lib.rosar_sparse_azimuth_migrating(ptr(S), n_bins, ptr(w), ptr(o), stride, ptr(dl), n_rng, n_az, K,
                                             ptr(out), stream_handle(stream)))
    return out


def image_migrating(raw, win, w, o, dl, workspace=None, out=None, stream=None):
    """rosar_image_migrating: range compression, then the migration-aware azimuth filter."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(w, torch.complex64, "w", ndim=2)
    K = w.shape[1]
    stride = _offsets(o, L, K)
    require(dl, torch.int32, "dl", shape=(L, K))
    if workspace is None:
        workspace = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    if out is None:
        out = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    check(lib.rosar_image_migrating(ptr(raw), ptr(win), ptr(w), ptr(o), stride, ptr(dl), n_az, L, K, ptr(workspace),
                                    ptr(out), stream_handle(stream)))
    return out


@dataclass(frozen=True)
class MigratingPlan:
    """The planes of rosar_azimuth_plan_migrating: H [n_d, n_rng, n_az] for row offsets d_lo .. d_lo + n_d - 1."""

    H: torch.Tensor
    d_lo: int
    n_d: int


def azimuth_plan_migrating(w, o, dl, n_az, stream=None):
    """rosar_azimuth_plan_migrating: the frequency-domain planes of the range-migration-aware taps (w [n_rng, K],
    offsets o, row offsets dl [n_rng, K]); the planes span the full range of dl (read once on the host)."""
    lib = _lib.load()
    require(w, torch.complex64, "w", ndim=2)
    n_rng, K = w.shape
    stride = _offsets(o, n_rng, K)
    require(dl, torch.int32, "dl", shape=(n_rng, K))
    d_lo, d_hi = int(dl.min().item()), int(dl.max().item())
    n_d = d_hi - d_lo + 1
    H = torch.empty((n_d, n_rng, n_az), dtype=torch.complex64, device=w.device)
    check(lib.rosar_azimuth_plan_migrating(ptr(w), ptr(o), stride, ptr(dl), d_lo, n_d, n_rng, n_az, K, ptr(H),
                                           stream_handle(stream)))
    return MigratingPlan(H, d_lo, n_d)


def sparse_azimuth_migrating_fft(S, plan: MigratingPlan, spectrum=None, out=None, stream=None):
    """rosar_sparse_azimuth_migrating_fft: the range-migration-aware filter of S [n_bins, n_az] through its planes."""
    lib = _lib.load()
    require(S, torch.complex64, "S", ndim=2)
    n_bins, n_az = S.shape
    n_d, n_rng = plan.H.shape[0], plan.H.shape[1]
    require(plan.H, torch.complex64, "H", shape=(n_d, n_rng, n_az))
    if spectrum is None:
        spectrum = torch.empty_like(S)
    if out is None:
        out = torch.empty((n_rng, n_az), dtype=torch.complex64, device=S.device)
    require(spectrum, torch.complex64, "spectrum", shape=(n_bins, n_az))
    require(out, torch.complex64, "out", shape=(n_rng, n_az))
    check(lib.rosar_sparse_azimuth_migrating_fft(ptr(S), n_bins, ptr(plan.H), plan.d_lo, plan.n_d, n_rng, n_az,
                                                 ptr(spectrum), ptr(out), stream_handle(stream)))
    return out


def image_migrating_fft(raw, win, plan: MigratingPlan, workspace=None, out=None, stream=None):
    """rosar_image_migrating_fft: range compression, then the migration-aware filter in the frequency domain;
    workspace [2, L, n_az]."""
    lib = _lib.load()
    require(raw, torch.complex64, "raw", ndim=2)
    n_az, L = raw.shape
    if win is not None:
        require(win, torch.float32, "win", shape=(L,))
    require(plan.H, torch.complex64, "H", shape=(plan.n_d, L, n_az))
    if workspace is None:
        workspace = torch.empty((2, L, n_az), dtype=torch.complex64, device=raw.device)
    if out is None:
        out = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
    require(workspace, torch.complex64, "workspace", shape=(2, L, n_az))
    require(out, torch.complex64, "out", shape=(L, n_az))
    check(lib.rosar_image_migrating_fft(ptr(raw), ptr(win), ptr(plan.H), plan.d_lo, plan.n_d, n_az, L, ptr(workspace),
                                        ptr(out), stream_handle(stream)))
    return out
