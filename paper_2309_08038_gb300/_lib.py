"""ctypes binding to librosar.so: argument marshalling only, every step runs in the CUDA kernels.

Loading fails loudly (RuntimeError) if the library has not been built; there is
no CPU fallback.  Tensors are torch CUDA tensors: complex64 for complex arrays,
float32 for windows and pulse errors, int32 for offsets, all contiguous.  Work
is enqueued on torch's current CUDA stream unless a stream is passed.
"""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "librosar.so")

_lib = None
_lock = threading.Lock()


class RosarError(RuntimeError):
    def __init__(self, status: int, name: str, detail: str):
        super().__init__(f"{name}: {detail}" if detail else name)
        self.status = status


class RadarStruct(ctypes.Structure):
    _fields_ = [("fc_hz", ctypes.c_double), ("slope_hz_per_s", ctypes.c_double), ("t_sample_s", ctypes.c_double),
                ("t_start_s", ctypes.c_double), ("r0_m", ctypes.c_double), ("c_mps", ctypes.c_double)]


class ScanStruct(ctypes.Structure):
    _fields_ = [("raw", ctypes.c_void_p), ("win", ctypes.c_void_p), ("w", ctypes.c_void_p), ("o", ctypes.c_void_p),
                ("o_row_stride", ctypes.c_int), ("n_az", ctypes.c_int), ("L", ctypes.c_int), ("K", ctypes.c_int),
                ("S", ctypes.c_void_p), ("out", ctypes.c_void_p), ("H", ctypes.c_void_p)]


class BatchTuningStruct(ctypes.Structure):
    _fields_ = [("az_tile", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("interleave", ctypes.c_int),
                ("spin_limit", ctypes.c_int), ("debug_unmet_scan", ctypes.c_int), ("mix", ctypes.c_int),
                ("flags", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_PROTOS = {
    "rosar_status_string": (ctypes.c_char_p, [_I]),
    "rosar_last_error": (ctypes.c_char_p, []),
    "rosar_version": (_I, []),
    "rosar_range_compress": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "rosar_range_compress_scans": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_sparse_azimuth": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_bpa": (_I, [_P, ctypes.POINTER(RadarStruct), _P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "rosar_image": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "rosar_image_fft_host": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P]),
    "rosar_sparse_azimuth_fft_scans": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_azimuth_weight_grad_fft": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "rosar_bpa_time": (_I, [_P, _P, ctypes.POINTER(RadarStruct), _I, _I, _I, _I, _P, _P]),
    "rosar_sas_time": (_I, [_P, _P, _P, _P, _I, ctypes.POINTER(RadarStruct), _I, _I, _I, _I, _I, _P, _P]),
    "rosar_image_noalloc": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_sparse_azimuth_migrating": (_I, [_P, _I, _P, _P, _I, _P, _I, _I, _I, _P, _P]),
    "rosar_image_migrating": (_I, [_P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _P]),
    "rosar_azimuth_fft_supported": (_I, [_I]),
    "rosar_azimuth_plan": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_phasors": (_I, [_P, ctypes.c_longlong, _P, _P]),
    "rosar_sparse_azimuth_fft_scans_ex": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "rosar_azimuth_weight_grad_spectra": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "rosar_azimuth_weight_grad_fft_phase": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "rosar_phase_grad_phasor": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "rosar_time_domain_plan_bytes": (ctypes.c_size_t, [_I, _I, _I]),
    "rosar_sas_time_plan": (_I, [_P, _P, _P, ctypes.POINTER(RadarStruct), _I, _I, _I, _I, _I, _P, ctypes.c_size_t, _P]),
    "rosar_sas_time_planned": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_bpa_time_plan": (_I, [_P, ctypes.POINTER(RadarStruct), _I, _I, _I, _I, _P, ctypes.c_size_t, _P]),
    "rosar_bpa_time_planned": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_azimuth_plan_migrating": (_I, [_P, _P, _I, _P, _I, _I, _I, _I, _I, _P, _P]),
    "rosar_sparse_azimuth_migrating_fft": (_I, [_P, _I, _P, _I, _I, _I, _I, _P, _P, _P]),
    "rosar_image_migrating_fft": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "rosar_sparse_azimuth_fft": (_I, [_P, _P, _I, _I, _P, _P]),
    "rosar_image_fft": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "rosar_image_fft_scans": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "rosar_image_fft_scans_pipelined": (_I, [_I, _I]),
    "rosar_phase_apply": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "rosar_sparse_azimuth_scans": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "rosar_sparse_azimuth_adjoint": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "rosar_phase_grad": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "rosar_image_l2_loss_workspace_bytes": (ctypes.c_size_t, []),
    "rosar_image_l2_loss": (_I, [_P, _P, ctypes.c_longlong, _P, _P, _P]),
    "rosar_image_l2_loss_grad": (_I, [_P, _P, ctypes.c_longlong, _P, _P, _P]),
    "rosar_range_compress_adjoint": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "rosar_range_compress_adjoint_scans": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "rosar_batch_workspace_bytes": (ctypes.c_size_t, [_I]),
    "rosar_batch_create": (_I, [ctypes.POINTER(ScanStruct), _I, ctypes.POINTER(BatchTuningStruct), _P,
                                ctypes.c_size_t, ctypes.POINTER(_P)]),
    "rosar_batch_launch": (_I, [_P, _P]),
    "rosar_batch_status": (_I, [_P, _P]),
    "rosar_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rosar_batch_destroy": (_I, [_P]),
}

NOALLOC_MAX_ELEMS = 1 << 21


def load(path: str = LIB_PATH):
    """Loads librosar.so once; raises RuntimeError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"librosar.so is not built ({path}); run `python -m paper_2309_08038_gb300.build` "
                                   "or __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _PROTOS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int):
    if status != 0:
        lib = load()
        raise RosarError(status, lib.rosar_status_string(status).decode(), lib.rosar_last_error().decode())


# ------------------------------------------------------------ marshalling --

def ptr(t):
    """Device pointer of a tensor (None -> NULL)."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def require(t, dtype, name, ndim=None, shape=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims, got shape {tuple(t.shape)}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t
