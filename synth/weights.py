"""Default sparse-aperture weights: conjugate ideal rotation manifold with a Taylor taper.

The paper designs robust sparse weights offline with FPP-SCA (Sec. III-A..C,
Algorithm 1); that design stays off the imaging path.  The default used here is
the conjugate of the near-field steering vector of Eq. (16) at the chosen
sparse positions, tapered by a Taylor window (nbar = 4, -30 dB) laid over the
dense aperture and normalised to unit 2-norm per range row (constraint C3,
Eq. (20)).  Computed once in FP64 and stored as complex64.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.signal.windows import taylor

from .configs import ScanConfig


def default_weights(cfg: ScanConfig, offsets: np.ndarray, nbar: int = 4, sll_db: float = 30.0) -> np.ndarray:
    """Weights w[r, k] (complex64 [L, K]) applied as sum_k w[r,k] * S[r, theta + o_k].

    Row r images the ring at R_r = r0 + r*dR.  Tap k sits at pulse angle
    2*pi*o_k/n_az from the pixel; its distance to the pixel is rho and the cosine
    of its off-bore-sight angle is (R_r*cos(dphi) - r0)/rho (zero behind the antenna,
    one when rho = 0).  The matched phase uses the wavenumber at the centre of the
    ADC window, which is the phase reference of the centred range DFT.
    """
    rad = cfg.radar
    L = cfg.L
    dR = rad.bin_spacing(L)
    f_mid = rad.fc + rad.slope * (rad.t_start + rad.t_sample(L) * (L - 1) / 2.0)
    k_mid = 2.0 * math.pi * f_mid / rad.c
    o = np.asarray(offsets, dtype=np.int64)
    if o.ndim == 1:
        o = np.broadcast_to(o, (L, o.shape[0]))
    R = rad.r0 + np.arange(L, dtype=np.float64)[:, None] * dR            # [L, 1]
    dphi = 2.0 * math.pi * o / cfg.n_az                                  # [L, K]
    rho = np.sqrt(np.maximum(R * R + rad.r0 ** 2 - 2.0 * R * rad.r0 * np.cos(dphi), 0.0))
    proj = R * np.cos(dphi) - rad.r0
    with np.errstate(divide="ignore", invalid="ignore"):
        p = np.where(rho > 0, np.maximum(proj, 0.0) / np.where(rho > 0, rho, 1.0), 1.0)
    T = taylor(cfg.M_ap, nbar=nbar, sll=sll_db, norm=True)[o + cfg.M_ap // 2]
    v = T * p * np.exp(-2j * k_mid * rho)
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    w = np.where(nrm > 0, v / np.where(nrm > 0, nrm, 1.0), 0.0)
    return w.astype(np.complex64)


def migration_offsets(cfg: ScanConfig, offsets: np.ndarray) -> np.ndarray:
    """Row offsets dl[r, k] (int32 [L, K]) of the range-migration-aware filter: tap k of row r reads the
    bin where a point at that pixel peaks for the tap's phase centre, round(rho/dR) - r (the peak-bin
    rule of the paper's range FFT), with rho the nominal slant range used by default_weights."""
    rad = cfg.radar
    L = cfg.L
    dR = rad.bin_spacing(L)
    o = np.asarray(offsets, dtype=np.int64)
    if o.ndim == 1:
        o = np.broadcast_to(o, (L, o.shape[0]))
    R = rad.r0 + np.arange(L, dtype=np.float64)[:, None] * dR
    dphi = 2.0 * math.pi * o / cfg.n_az
    rho = np.sqrt(np.maximum(R * R + rad.r0 ** 2 - 2.0 * R * rad.r0 * np.cos(dphi), 0.0))
    return (np.floor(rho / dR + 0.5) - np.arange(L)[:, None]).astype(np.int32)
