"""Batched form: many uneven scans imaged by one persistent, graph-captured launch (rosar_batch_*)."""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import check, require, stream_handle


@dataclass
class Tuning:
    """Mirrors rosar_batch_tuning.  az_tile in {256, 512, 1024, 2048}; ctas_per_sm 0 = occupancy limit;
    interleave 0 = all range tiles first, 1 = scan by scan, d >= 2 = range tiles d-1 scans ahead of the azimuth
    tiles; spin_limit 0 = default; mix = chunks per scan in which the two kinds of tile alternate (interleave
    >= 2); flags = DISCARD_S bit."""

    az_tile: int = 1024
    ctas_per_sm: int = 0
    interleave: int = 0
    spin_limit: int = 0
    debug_unmet_scan: int = -1
    mix: int = 1
    flags: int = 0

    def as_struct(self):
        return _lib.BatchTuningStruct(self.az_tile, self.ctas_per_sm, self.interleave, self.spin_limit,
                                      self.debug_unmet_scan, self.mix, self.flags)


DISCARD_S = 2     # ROSAR_BATCH_DISCARD_S


class Batch:
    """A set of scans bound to one CUDA graph [counter reset -> persistent kernel].

    Each scan is a dict with CUDA tensors raw [n_az, L], w [L, K], o [K] or [L, K], and optionally
    win [L], S [L, n_az] (workspace), out [L, n_az] (allocated here when missing) and H [L, n_az]
    (the scan's plan from azimuth_plan: its azimuth filter then runs as whole-row FFT tiles).  The tensors are
    referenced for the lifetime of the batch; `launch()` re-reads whatever they hold.
    """

    def __init__(self, scans, tuning: Tuning | None = None):
        lib = _lib.load()
        self._keep = []
        arr = (_lib.ScanStruct * len(scans))()
        self.outs = []
        for i, sc in enumerate(scans):
            raw = require(sc["raw"], torch.complex64, f"scans[{i}].raw", ndim=2)
            n_az, L = raw.shape
            w = require(sc["w"], torch.complex64, f"scans[{i}].w", ndim=2)
            K = w.shape[1]
            o = require(sc["o"], torch.int32, f"scans[{i}].o")
            stride = 0 if o.dim() == 1 else K
            win = sc.get("win")
            if win is not None:
                require(win, torch.float32, f"scans[{i}].win", shape=(L,))
            S = sc.get("S")
            if S is None:
                S = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
            out = sc.get("out")
            if out is None:
                out = torch.empty((L, n_az), dtype=torch.complex64, device=raw.device)
            require(S, torch.complex64, f"scans[{i}].S", shape=(L, n_az))
            require(out, torch.complex64, f"scans[{i}].out", shape=(L, n_az))
            H = sc.get("H")
            if H is not None:
                require(H, torch.complex64, f"scans[{i}].H", shape=(L, n_az))
            arr[i] = _lib.ScanStruct(raw.data_ptr(), win.data_ptr() if win is not None else None, w.data_ptr(),
                                     o.data_ptr(), stride, n_az, L, K, S.data_ptr(), out.data_ptr(),
                                     H.data_ptr() if H is not None else None)
            self._keep += [raw, w, o, win, S, out, H]
            self.outs.append(out)
        nbytes = lib.rosar_batch_workspace_bytes(len(scans))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.outs[0].device)
        self.tuning = tuning or Tuning()
        ts = self.tuning.as_struct()
        h = ctypes.c_void_p()
        check(lib.rosar_batch_create(arr, len(scans), ctypes.byref(ts), ctypes.c_void_p(self.workspace.data_ptr()),
                                     nbytes, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        check(_lib.load().rosar_batch_launch(self._h, stream_handle(stream)))

    def status(self, stream=None):
        """Waits for the stream; raises RosarError (ROSAR_ERR_TIMEOUT) if a dependency wait gave up."""
        check(_lib.load().rosar_batch_status(self._h, stream_handle(stream)))

    def info(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(_lib.load().rosar_batch_info(self._h, *[ctypes.byref(x) for x in v]))
        return {"range_tiles": v[0].value, "azimuth_tiles": v[1].value, "ctas": v[2].value, "smem_bytes": v[3].value}

    def close(self):
        if getattr(self, "_h", None):
            check(_lib.load().rosar_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
