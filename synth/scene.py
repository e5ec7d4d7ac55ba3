"""Seeded synthetic scenes: random draws, the raw IF cube, window and sparse offsets.

Every random number comes from numpy's PCG64 (``default_rng(seed)``) in a fixed
order, so a (config, seed) pair always gives the same bits.  The draws are
returned with the cube so a second implementation can rebuild it.
"""

from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import build as _build
from .configs import ScanConfig, deg2rad

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_raw_cube.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       dp, dp, dp, dp, dp, dp, dp, dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
        lib.synth_raw_cube.restype = None
        lib.synth_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Scene:
    cfg: ScanConfig
    tgt_R: np.ndarray        # target distance from the rotation centre, m
    tgt_phi: np.ndarray      # target angle, rad
    tgt_amp: np.ndarray      # complex reflectivity
    clut_R: np.ndarray
    clut_phi: np.ndarray
    clut_amp: np.ndarray
    dphi: np.ndarray         # per-pulse angle error, rad (phi_hat_n = 2 pi n/N + dphi[n])
    dr: np.ndarray           # per-pulse radius error, m
    noise: np.ndarray | None  # complex128 [n_az, L]
    raw: np.ndarray | None = None   # complex64 [n_az, L]


def draw_scene(cfg: ScanConfig, with_noise: bool = True) -> Scene:
    """Draws targets, clutter, rotation jitter and receiver noise for ``cfg``."""
    rng = np.random.default_rng(cfg.seed_scene)
    nt = cfg.n_targets
    tgt_R = rng.uniform(cfg.R_lo, cfg.R_hi, nt)
    tgt_phi = rng.uniform(0.0, 2.0 * math.pi, nt)
    if cfg.amp == "unit":
        tgt_amp = np.ones(nt, dtype=np.complex128)
    elif cfg.amp == "rayleigh":
        tgt_amp = rng.standard_normal(nt) + 1j * rng.standard_normal(nt)   # sigma = 1, E|A|^2 = 2
    else:
        raise ValueError(cfg.amp)
    mean_tgt_power = 1.0 if cfg.amp == "unit" else 2.0
    if cfg.clutter_db is not None:
        dR = cfg.radar.bin_spacing(cfg.L)
        r_lo = max(cfg.R_lo, cfg.radar.r0 + dR)
        cells = int((cfg.R_hi - r_lo) / dR) * cfg.n_az
        nc = min(cells, cfg.clutter_cap)
        p_cell = 10.0 ** (cfg.clutter_db / 10.0) * mean_tgt_power
        sigma2 = p_cell * cells / nc                       # same clutter power per cell
        clut_R = np.sqrt(rng.uniform(r_lo ** 2, cfg.R_hi ** 2, nc))   # uniform over the annulus area
        clut_phi = rng.uniform(0.0, 2.0 * math.pi, nc)
        clut_amp = math.sqrt(sigma2 / 2.0) * (rng.standard_normal(nc) + 1j * rng.standard_normal(nc))
    else:
        clut_R = clut_phi = np.zeros(0)
        clut_amp = np.zeros(0, dtype=np.complex128)
    dphi = rng.standard_normal(cfg.n_az) * deg2rad(cfg.jitter_phi_deg) if cfg.jitter_phi_deg > 0 else np.zeros(cfg.n_az)
    dr = rng.standard_normal(cfg.n_az) * cfg.jitter_r_m if cfg.jitter_r_m > 0 else np.zeros(cfg.n_az)
    noise = None
    if with_noise and cfg.noise_var > 0:
        s = math.sqrt(cfg.noise_var / 2.0)
        noise = s * (rng.standard_normal((cfg.n_az, cfg.L)) + 1j * rng.standard_normal((cfg.n_az, cfg.L)))
    return Scene(cfg, tgt_R, tgt_phi, tgt_amp, clut_R, clut_phi, clut_amp, dphi, dr, noise)


def synth_if(cfg: ScanConfig, R, phi, amp, dphi=None, dr=None, n_threads: int = 0) -> np.ndarray:
    """Noise-free IF cube [n_az, L] complex128 of point scatterers at polar (R, phi) with reflectivity amp."""
    lib = _load()
    rad = cfg.radar
    n = np.arange(cfg.n_az, dtype=np.float64)
    ph = 2.0 * math.pi * n / cfg.n_az + (np.zeros(cfg.n_az) if dphi is None else np.asarray(dphi, np.float64))
    rr = rad.r0 + (np.zeros(cfg.n_az) if dr is None else np.asarray(dr, np.float64))
    ux = np.ascontiguousarray(np.cos(ph))
    uy = np.ascontiguousarray(np.sin(ph))
    px = np.ascontiguousarray(rr * ux)
    py = np.ascontiguousarray(rr * uy)
    R = np.asarray(R, np.float64)
    phi = np.asarray(phi, np.float64)
    amp = np.asarray(amp, np.complex128)
    sx = np.ascontiguousarray(R * np.cos(phi))
    sy = np.ascontiguousarray(R * np.sin(phi))
    are = np.ascontiguousarray(amp.real)
    aim = np.ascontiguousarray(amp.imag)
    out = np.zeros((cfg.n_az, cfg.L, 2), dtype=np.float64)
    lib.synth_raw_cube(cfg.n_az, cfg.L, int(R.shape[0]), _dp(sx), _dp(sy), _dp(are), _dp(aim),
                       _dp(px), _dp(py), _dp(ux), _dp(uy), rad.fc, rad.slope, rad.t_sample(cfg.L),
                       rad.t_start, rad.c, _dp(out), int(n_threads))
    return out[..., 0] + 1j * out[..., 1]


def make_scene(cfg: ScanConfig, with_noise: bool = True) -> Scene:
    """Draws a scene and synthesises its complex64 raw cube [n_az, L] (pulse-major)."""
    sc = draw_scene(cfg, with_noise)
    R = np.concatenate([sc.tgt_R, sc.clut_R])
    phi = np.concatenate([sc.tgt_phi, sc.clut_phi])
    amp = np.concatenate([sc.tgt_amp, sc.clut_amp])
    raw = synth_if(cfg, R, phi, amp, sc.dphi, sc.dr)
    if sc.noise is not None:
        raw = raw + sc.noise
    sc.raw = raw.astype(np.complex64)
    return sc


def hann_window(L: int) -> np.ndarray:
    """Symmetric Hann window, float32 [L]."""
    m = np.arange(L, dtype=np.float64)
    return (0.5 - 0.5 * np.cos(2.0 * math.pi * m / (L - 1))).astype(np.float32)


def draw_offsets(cfg: ScanConfig) -> np.ndarray:
    """Sparse pulse offsets, int32: K of the M_ap positions [-M_ap/2, M_ap/2), uniform without
    replacement, sorted.  Shape [K], or [L, K] (one draw per range row) if cfg.per_row_offsets."""
    rng = np.random.default_rng(cfg.seed_offsets)
    if not cfg.per_row_offsets:
        return (np.sort(rng.choice(cfg.M_ap, cfg.K, replace=False)) - cfg.M_ap // 2).astype(np.int32)
    o = np.empty((cfg.L, cfg.K), dtype=np.int32)
    for r in range(cfg.L):
        o[r] = np.sort(rng.choice(cfg.M_ap, cfg.K, replace=False)) - cfg.M_ap // 2
    return o
