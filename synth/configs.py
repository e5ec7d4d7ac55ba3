"""Workload definitions for the synthetic ROSAR scenes.

Five workloads, shaped like the paper's point-target simulation and indoor
testbed scans (Sec. IV-D, Sec. V) but on a 77 GHz / 4 GHz radar:

  tiny      360 pulses x 64 samples,   K=16 of M=60,     3 unit point targets
  indoor    3600 x 256,                K=64 of M=600,    20 Rayleigh targets + clutter, jitter
  highres   14400 x 1024,              K=128 of M=2400,  per-row taps, 200 targets + clutter
  batched   256 scans, n_az in {1800,3600,7200}, L in {128..1024}, K in {32,64,128}
  diff      16 indoor scans with per-pulse phase errors

Radar (shared): fc = 77 GHz ramp start, 4 GHz sweep over a 40 us ramp
(slope 1e14 Hz/s), rotation radius 0.25 m.  The ADC window is centred in the
ramp and covers 60 % of it, so t_s = 24 us / L and every L gives the same bin
spacing dR = c/(2*slope*t_s*L) = 6.246 cm and maximum range L*dR.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

C_LIGHT = 299792458.0


@dataclass(frozen=True)
class RadarParams:
    fc: float = 77e9
    bandwidth: float = 4e9
    t_ramp: float = 40e-6
    adc_fraction: float = 0.6
    r0: float = 0.25
    c: float = C_LIGHT

    @property
    def slope(self) -> float:
        return self.bandwidth / self.t_ramp

    def t_sample(self, L: int) -> float:
        return self.adc_fraction * self.t_ramp / L

    @property
    def t_start(self) -> float:
        return 0.5 * (1.0 - self.adc_fraction) * self.t_ramp

    def bin_spacing(self, L: int) -> float:
        return self.c / (2.0 * self.slope * self.t_sample(L) * L)


@dataclass(frozen=True)
class ScanConfig:
    name: str
    n_az: int                 # pulses (phase centres) per rotation
    L: int                    # ADC samples per pulse = FFT length = image rows
    K: int                    # sparse taps
    M_ap: int                 # dense aperture length in pulses; offsets in [-M_ap/2, M_ap/2)
    per_row_offsets: bool = False
    n_targets: int = 3
    R_lo: float = 0.5
    R_hi: float = 3.0
    amp: str = "unit"         # "unit": amplitude 1, phase 0; "rayleigh": CN(0, 2)
    clutter_db: float | None = None   # clutter power per image cell vs. mean target power
    clutter_cap: int = 16384  # scatterers actually synthesised (power rescaled to match)
    noise_var: float = 0.01   # complex AWGN variance per raw sample (20 dB vs a unit boresight target)
    jitter_phi_deg: float = 0.0
    jitter_r_m: float = 0.0
    seed_scene: int = 0
    seed_offsets: int = 100
    radar: RadarParams = field(default_factory=RadarParams)

    @property
    def n_rng(self) -> int:
        return self.L

    @property
    def pixels(self) -> int:
        return self.L * self.n_az


TINY = ScanConfig("tiny", 360, 64, 16, 60, n_targets=3, R_lo=0.5, R_hi=3.0, amp="unit",
                  seed_scene=0, seed_offsets=100)

INDOOR = ScanConfig("indoor", 3600, 256, 64, 600, n_targets=20, R_lo=0.5, R_hi=14.0,
                    amp="rayleigh", clutter_db=-20.0, clutter_cap=16384,
                    jitter_phi_deg=0.05, jitter_r_m=1e-3, seed_scene=1, seed_offsets=101)

HIGHRES = ScanConfig("highres", 14400, 1024, 128, 2400, per_row_offsets=True, n_targets=200,
                     R_lo=0.5, R_hi=57.0, amp="rayleigh", clutter_db=-15.0, clutter_cap=16384,
                     jitter_phi_deg=0.02, jitter_r_m=0.0, seed_scene=2, seed_offsets=102)

CONFIGS = {c.name: c for c in (TINY, INDOOR, HIGHRES)}

BATCH_N_AZ = (1800, 3600, 7200)
BATCH_L = (128, 256, 512, 1024)
BATCH_K = (32, 64, 128)


def batched_configs(n_scans: int = 256, seed: int = 3):
    """Per-scan shapes of the batched workload: n_az, L, K drawn uniformly; M_ap = n_az/6.

    Scene statistics follow the indoor scan; the target range is clipped to the
    unambiguous range of each L.  Scans sharing (n_az, L) share one scene cube.
    """
    import numpy as np

    rng = np.random.default_rng(seed)
    n_az = rng.choice(BATCH_N_AZ, n_scans)
    L = rng.choice(BATCH_L, n_scans)
    K = rng.choice(BATCH_K, n_scans)
    out = []
    for s in range(n_scans):
        L_s = int(L[s])
        R_hi = min(INDOOR.R_hi, INDOOR.radar.r0 + 0.9 * L_s * INDOOR.radar.bin_spacing(L_s))
        out.append(replace(INDOOR, name=f"batched{s}", n_az=int(n_az[s]), L=L_s, K=int(K[s]),
                           M_ap=int(n_az[s]) // 6, R_hi=R_hi, clutter_cap=4096,
                           seed_scene=1000 + BATCH_N_AZ.index(int(n_az[s])) * 10 + BATCH_L.index(L_s),
                           seed_offsets=103 + s))
    return out


def diff_configs(n_scans: int = 16):
    """The differentiable workload: indoor geometry, 16 scans with their own scenes."""
    return [replace(INDOOR, name=f"diff{s}", seed_scene=200 + s, clutter_cap=4096) for s in range(n_scans)]


def max_range(cfg: ScanConfig) -> float:
    return cfg.radar.r0 + cfg.L * cfg.radar.bin_spacing(cfg.L)


def deg2rad(x: float) -> float:
    return x * math.pi / 180.0
