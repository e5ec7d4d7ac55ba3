"""Plain FP64 restatement of the ROSAR imaging chain of arXiv 2309.08038.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  No blocking, fusion or
reordering beyond what each definition states; loops are vectorised over the
independent output index only (a numpy array op stands for "for every theta").

Notation follows the paper: N phase centres per rotation (here ``n_az``), M ADC
samples per pulse (here ``L``, equal to the FFT length), chirp slope K (here
``slope``), rotation radius r (here ``r0``).  The sparse tap count is ``K`` and
the dense aperture length in pulses is ``M_ap``.

Readings of the paper that the oracle fixes (the paper is silent or loose):
  * fixed-row azimuth filter: every tap of output row r reads range bin r
    (the paper picks the per-pulse peak bin l*_n of Eq. (40) in Eq. (43));
  * the range DFT may be taken about the window centre: bin l is multiplied by
    c_l = exp(+j*pi*l*(L-1)/L) ("centred"); centred=False is Eq. (38) verbatim;
  * the matched wavenumber is the one at the centre of the ADC window,
    k_mid = 2*pi*(fc + K*(T_start + t_s*(L-1)/2))/c, instead of Sec. II-B's
    k = 2*pi*(fc + K*T_start)/c, because the centred DFT references the phase
    to the window centre;
  * polar image grid: pixel (r, theta) sits at distance R_r = r0 + r*dR from
    the rotation centre and angle 2*pi*theta/n_az, dR = c/(2*K*t_s*L);
  * p(theta) = 1 when the slant range is exactly zero (degenerate row 0).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

C_LIGHT = 299792458.0

__all__ = [
    "C_LIGHT", "Radar", "phase_centre_angle", "slant_range", "off_boresight_angle",
    "antenna_pattern", "visibility_half_angle", "visible_pulses", "range_bin_spacing",
    "peak_range_bin", "wavenumber", "wavenumber_centred", "if_cube", "hann_symmetric",
    "dft_matrix", "range_compress", "sparse_azimuth", "bpa_pixels", "bpa",
    "taylor_taper", "default_weights", "sparse_azimuth_adjoint_S",
    "sparse_azimuth_adjoint_w", "phase_error_grad", "range_compress_adjoint",
    "apply_phase_errors", "image_entropy", "pisr", "half_mainlobe_width",
    "sparse_azimuth_migrating", "migration_offsets", "bpa_time_pixels", "bpa_time",
    "sas_time_pixels", "sas_time",
]


@dataclass(frozen=True)
class Radar:
    """FMCW radar on a rotating arm (Sec. II, Table "Parameters of the ROSAR System").

    fc       carrier frequency at the start of the ramp, Hz (Eq. (6))
    slope    chirp slope K, Hz/s (Eq. (6))
    t_s      ADC sampling interval, s (Sec. II-B, Eq. (10))
    t_start  delay from ramp start to the first ADC sample, s (T_Start, Eq. (10))
    r0       rotation radius r, m (Sec. II-A)
    c        propagation speed, m/s
    """

    fc: float
    slope: float
    t_s: float
    t_start: float
    r0: float
    c: float = C_LIGHT


# ---------------------------------------------------------------- geometry --

def phase_centre_angle(n, n_az):
    """Bore-sight direction of the n-th phase centre, phi_n = 2*pi*n/N (Sec. II-A, Eq. (1))."""
    return 2.0 * math.pi * np.asarray(n, dtype=np.float64) / n_az


def slant_range(R_t, phi_t, r, phi_n):
    """Distance from a phase centre at (r, phi_n) to a point at (R_t, phi_t) (Sec. II-A, Eq. (2))."""
    R_t = np.asarray(R_t, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    return np.sqrt(R_t * R_t + r * r - 2.0 * r * R_t * np.cos(np.asarray(phi_n) - np.asarray(phi_t)))


def off_boresight_angle(R_t, phi_t, r, phi_n):
    """Angle between the bore-sight of phase centre n and the direction to the point (Sec. II-A, Eq. (3)).

    Eq. (3) is written as arctan(R_t sin|dphi| / (R_t cos|dphi| - r)); the two-argument
    arctangent keeps the quadrant, so points behind the antenna get |theta| > pi/2.
    """
    d = np.abs(np.asarray(phi_n, dtype=np.float64) - np.asarray(phi_t, dtype=np.float64))
    R_t = np.asarray(R_t, dtype=np.float64)
    return np.arctan2(R_t * np.sin(d), R_t * np.cos(d) - np.asarray(r, dtype=np.float64))


def antenna_pattern(theta):
    """Cosine antenna pattern p(theta): cos(theta) inside (-pi/2, pi/2), else 0 (Sec. II-B, Eq. (8))."""
    theta = np.asarray(theta, dtype=np.float64)
    return np.where(np.abs(theta) < 0.5 * math.pi, np.cos(theta), 0.0)


def visibility_half_angle(R_t, r):
    """phi_v = arccos(r / R_t) (Sec. II-A, Eq. (4))."""
    return math.acos(r / R_t)


def visible_pulses(R_t, r, n_az):
    """Indices N_min..N_max of the phase centres that see a target at (pi/2, R_t) (Sec. II-A, Eq. (5))."""
    phi_v = visibility_half_angle(R_t, r)
    step = 2.0 * math.pi / n_az
    n_min = math.ceil((0.5 * math.pi - phi_v) / step)
    n_max = math.floor((0.5 * math.pi + phi_v) / step)
    return n_min, n_max


def range_bin_spacing(radar: Radar, L):
    """Range covered by one FFT bin: bin l holds ranges near l*c/(2*K*t_s*L) (from Eq. (40))."""
    return radar.c / (2.0 * radar.slope * radar.t_s * L)


def peak_range_bin(R_n, radar: Radar, L):
    """l*_n = round(2*R_n*K*t_s*L/c), the bin where a target at slant range R_n peaks (Sec. III-D, Eq. (40))."""
    x = 2.0 * np.asarray(R_n, dtype=np.float64) * radar.slope * radar.t_s * L / radar.c
    return np.floor(x + 0.5).astype(np.int64)


def wavenumber(radar: Radar):
    """k = 2*pi*(K*T_Start + fc)/c (Sec. II-B, text after Eq. (11); Sec. III-D before Eq. (39))."""
    return 2.0 * math.pi * (radar.slope * radar.t_start + radar.fc) / radar.c


def wavenumber_centred(radar: Radar, L):
    """Wavenumber at the centre of the ADC window, the phase reference of the centred DFT."""
    f_mid = radar.fc + radar.slope * (radar.t_start + radar.t_s * (L - 1) / 2.0)
    return 2.0 * math.pi * f_mid / radar.c


# ------------------------------------------------------------ signal model --

def if_cube(radar: Radar, n_az, L, tgt_R, tgt_phi, tgt_amp, phi_hat=None, r_hat=None):
    """Noise-free sampled IF signal of point scatterers (Sec. II-B, Eq. (10)).

    raw[n, m] = sum_t A_t * p(theta_{t,n}) * exp(j*2*pi*[tau*K*(m*t_s + T_Start) + fc*tau]),
    tau = 2*R_{t,n}/c, with R_{t,n} from Eq. (2) and theta_{t,n} from Eq. (3) evaluated at the
    actual (possibly jittered, Eq. (37)) phase-centre position (r_hat[n], phi_hat[n]).
    The amplitude is alpha_n of Eq. (15) times the target's complex reflectivity A_t; the
    residual video phase is dropped as in Eq. (9).
    """
    n = np.arange(n_az)
    if phi_hat is None:
        phi_hat = phase_centre_angle(n, n_az)
    if r_hat is None:
        r_hat = np.full(n_az, radar.r0)
    m = np.arange(L, dtype=np.float64)
    raw = np.zeros((n_az, L), dtype=np.complex128)
    for R_t, phi_t, A in zip(np.atleast_1d(tgt_R), np.atleast_1d(tgt_phi), np.atleast_1d(tgt_amp)):
        R_n = slant_range(R_t, phi_t, r_hat, phi_hat)                      # [n_az]
        alpha = A * antenna_pattern(off_boresight_angle(R_t, phi_t, r_hat, phi_hat))
        tau = 2.0 * R_n / radar.c
        ph = tau[:, None] * radar.slope * (m[None, :] * radar.t_s + radar.t_start) + radar.fc * tau[:, None]
        raw += alpha[:, None] * np.exp(2j * math.pi * ph)
    return raw


# ------------------------------------------------------- range compression --

def hann_symmetric(L):
    """Symmetric Hann window 0.5 - 0.5*cos(2*pi*m/(L-1)), m = 0..L-1 (the paper applies none)."""
    m = np.arange(L, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * math.pi * m / (L - 1))


def dft_matrix(L):
    """F[l, m] = exp(-j*2*pi*l*m/L), the range FFT of Sec. III-D, Eq. (38)."""
    lm = np.outer(np.arange(L), np.arange(L)) % L       # exact integer phase index
    return np.exp(-2j * math.pi * lm / L)


def range_compress(raw, win, centred=True, bins=None):
    """Range compression of every pulse (Sec. III-D, Eq. (38)).

    raw: [n_az, L] complex, pulse-major.  Returns S: [L, n_az], range-major, with
    S[l, n] = c_l * sum_m win[m] * raw[n, m] * exp(-j*2*pi*l*m/L),
    c_l = exp(+j*pi*l*(L-1)/L) if centred else 1.
    ``bins`` (optional) evaluates only those rows l, returning [len(bins), n_az].
    """
    raw = np.asarray(raw, dtype=np.complex128)
    n_az, L = raw.shape
    win = np.ones(L) if win is None else np.asarray(win, dtype=np.float64)
    l = np.arange(L) if bins is None else np.asarray(bins, dtype=np.int64)
    F = np.exp(-2j * math.pi * (np.outer(l, np.arange(L)) % L) / L)     # rows l of the DFT matrix
    Y = (raw * win[None, :]) @ F.T                      # [n_az, len(l)]: Y[n, l]
    if centred:
        Y = Y * np.exp(1j * math.pi * l.astype(np.float64) * (L - 1) / L)[None, :]
    return np.ascontiguousarray(Y.T)


# ----------------------------------------------------- sparse azimuth filter --

def _offsets_per_row(o, n_rng):
    o = np.asarray(o, dtype=np.int64)
    if o.ndim == 1:
        return np.broadcast_to(o, (n_rng, o.shape[0]))
    return o


def sparse_azimuth(S, w, o):
    """Sparse-aperture azimuth matched filter (Sec. III-D, Eq. (43); Algorithm 2).

    out[r, theta] = sum_k w[r, k] * S[r, (theta + o_k) mod n_az], the taps summed in k order.
    Eq. (43) writes w^H y with the paper's weights; ``w`` here is that conjugate already.
    S: [n_rng, n_az]; w: [n_rng, K]; o: [K] (shared) or [n_rng, K] integer pulse offsets.
    """
    S = np.asarray(S, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    n_rng, n_az = S.shape
    o = _offsets_per_row(o, n_rng)
    theta = np.arange(n_az)
    out = np.zeros((n_rng, n_az), dtype=np.complex128)
    for r in range(n_rng):
        for k in range(w.shape[1]):
            out[r] += w[r, k] * S[r, (theta + o[r, k]) % n_az]
    return out


def sparse_azimuth_migrating(S, w, o, dl):
    """Eq. (43) with each tap reading the pulse's own peak bin (Sec. III-D; l*_n of Eq. (40)):
    out[r, theta] = sum_k w[r, k] * S[r + dl[r, k], (theta + o_k) mod n_az], rows outside
    0 .. n_bins-1 reading zero.  S: [n_bins, n_az]; w, dl: [n_rng, K]; o: [K] or [n_rng, K]."""
    S = np.asarray(S, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    n_bins, n_az = S.shape
    n_rng = w.shape[0]
    o = _offsets_per_row(o, n_rng)
    dl = np.asarray(dl, dtype=np.int64)
    theta = np.arange(n_az)
    out = np.zeros((n_rng, n_az), dtype=np.complex128)
    for r in range(n_rng):
        for k in range(w.shape[1]):
            row = r + dl[r, k]
            if 0 <= row < n_bins:
                out[r] += w[r, k] * S[row, (theta + o[r, k]) % n_az]
    return out


def migration_offsets(radar: Radar, L, n_az, n_rng, o):
    """dl[r, k] = l*_{r,k} - r: the peak bin of Eq. (40) at the slant range from the tap's phase centre
    (offset o_k, nominal radius r0) to the pixel of row r (distance r0 + r*dR), minus the row."""
    o = _offsets_per_row(o, n_rng)
    dR = range_bin_spacing(radar, L)
    dl = np.zeros(o.shape, dtype=np.int64)
    for r in range(n_rng):
        R_n = slant_range(radar.r0 + r * dR, 0.0, radar.r0, phase_centre_angle(o[r], n_az))
        dl[r] = peak_range_bin(R_n, radar, L) - r
    return dl


# -------------------------------------------------------- back-projection --

def bpa_pixels(S, radar: Radar, n_az, M_ap, rows, thetas, interp="linear", dphi=None, dr=None):
    """Range-compressed back-projection at selected polar pixels ("FFT+BPA", Sec. III-D after Eq. (43)).

    I(phi, R) = sum over the M_ap pulses n = (theta + d) mod n_az, d = -M_ap/2 .. M_ap/2-1, of
    alpha_n * exp(-j*2*k_mid*R_n) * S(R_n/dR, n): the BPA weight w_BP = alpha*exp(-j2kR) applied
    to the range-compressed sample at the target's range (Eq. (43) with w_BP; Eq. (14) summed
    over fast time by the range FFT).  R_n by Eq. (2), alpha_n = p(theta_n) by Eqs. (3), (8), (15),
    both at the actual phase-centre position phi_n + dphi[n], r0 + dr[n] (Eq. (37)).
    S(x, n) reads bin x: linear interpolation between floor(x) and floor(x)+1, or the nearest
    bin floor(x + 0.5) (the paper's l*_n, Eq. (40)); bins outside 0..L-1 read zero.
    Pixel (r, theta) is at R = r0 + r*dR, phi = 2*pi*theta/n_az.
    """
    S = np.asarray(S, dtype=np.complex128)
    L = S.shape[0]
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    thetas = np.asarray(thetas, dtype=np.int64).reshape(-1)
    dR = range_bin_spacing(radar, L)
    k_mid = wavenumber_centred(radar, L)
    d = np.arange(-(M_ap // 2), M_ap - M_ap // 2)
    n = (thetas[:, None] + d[None, :]) % n_az                          # [P, M_ap]
    phi_n = phase_centre_angle(n, n_az)
    r_n = np.full(n.shape, radar.r0)
    if dphi is not None:
        phi_n = phi_n + np.asarray(dphi, dtype=np.float64)[n]
    if dr is not None:
        r_n = r_n + np.asarray(dr, dtype=np.float64)[n]
    R_pix = (radar.r0 + rows * dR).astype(np.float64)[:, None]
    phi_pix = phase_centre_angle(thetas, n_az)[:, None]
    R_n = slant_range(R_pix, phi_pix, r_n, phi_n)
    theta_n = off_boresight_angle(R_pix, phi_pix, r_n, phi_n)
    alpha = np.where(R_n == 0.0, 1.0, antenna_pattern(theta_n))
    x = R_n / dR
    if interp == "linear":
        l0 = np.floor(x).astype(np.int64)
        f = x - l0
        s0 = _read_bins(S, l0, n)
        s1 = _read_bins(S, l0 + 1, n)
        s = (1.0 - f) * s0 + f * s1
    elif interp == "nearest":
        s = _read_bins(S, np.floor(x + 0.5).astype(np.int64), n)
    else:
        raise ValueError(interp)
    return np.sum(alpha * np.exp(-2j * k_mid * R_n) * s, axis=1)


def _read_bins(S, l, n):
    L = S.shape[0]
    ok = (l >= 0) & (l < L)
    return np.where(ok, S[np.clip(l, 0, L - 1), n], 0.0)


def bpa(S, radar: Radar, n_rng, M_ap, interp="linear", dphi=None, dr=None):
    """Full polar BPA image [n_rng, n_az] by ``bpa_pixels`` row by row."""
    S = np.asarray(S)
    n_az = S.shape[1]
    thetas = np.arange(n_az)
    out = np.zeros((n_rng, n_az), dtype=np.complex128)
    for r in range(n_rng):
        out[r] = bpa_pixels(S, radar, n_az, M_ap, np.full(n_az, r), thetas, interp, dphi, dr)
    return out


# ------------------------------------------------ time-domain BPA and SAS --

def _fast_time_compensation(radar: Radar, rho, win, L, m_ref):
    """win[m] * exp(-j*2*pi*tau*K*t_s*(m - m_ref)), tau = 2*rho/c, for every slant range in ``rho``.

    This is one column of W_BP (Eq. (14)) or W_SA (Sec. III-A) without its per-pulse factor: the
    fast-time phase of a return from slant range rho, removed sample by sample.  Returns
    rho.shape + (L,)."""
    rho = np.asarray(rho, dtype=np.float64)
    m = np.arange(L, dtype=np.float64) - m_ref
    tau = 2.0 * rho / radar.c
    return win * np.exp(-2j * math.pi * (tau * radar.slope * radar.t_s)[..., None] * m)


def _window(win, L):
    return np.ones(L) if win is None else np.asarray(win, dtype=np.float64)


def bpa_time_pixels(raw, win, radar: Radar, n_az, M_ap, rows, thetas):
    """Time-domain back-projection at selected polar pixels, the paper's "BPA" (Sec. II-C, Eq. (14)).

    I(phi, R) = sum over the M_ap pulses n = (theta + d) mod n_az, d = -M_ap/2 .. M_ap/2-1, and the
    L fast-time samples m of alpha_n * exp(-j*2*pi*tau_n*K*m*t_s) * exp(-j*2*k*R_n) * win[m] * raw[n, m]:
    the Hadamard product of W_BP and Y_IF summed over both axes.  R_n by Eq. (2) at the nominal
    phase-centre position (r0, 2*pi*n/n_az), tau_n = 2*R_n/c, alpha_n = p(theta_n) by Eqs. (3), (8),
    (15), k = 2*pi*(K*T_Start + fc)/c.  ``win`` = None is Eq. (14) verbatim; a window multiplies the
    fast-time samples as in the range compression.  raw: [n_az, L] pulse-major.
    """
    raw = np.asarray(raw, dtype=np.complex128)
    L = raw.shape[1]
    win = _window(win, L)
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    thetas = np.asarray(thetas, dtype=np.int64).reshape(-1)
    dR = range_bin_spacing(radar, L)
    k = wavenumber(radar)
    d = np.arange(-(M_ap // 2), M_ap - M_ap // 2)
    out = np.zeros(rows.shape[0], dtype=np.complex128)
    for p in range(rows.shape[0]):
        n = (thetas[p] + d) % n_az
        R = radar.r0 + rows[p] * dR
        phi = phase_centre_angle(thetas[p], n_az)
        phi_n = phase_centre_angle(n, n_az)
        R_n = slant_range(R, phi, radar.r0, phi_n)
        alpha = np.where(R_n == 0.0, 1.0, antenna_pattern(off_boresight_angle(R, phi, radar.r0, phi_n)))
        W = (alpha * np.exp(-2j * k * R_n))[:, None] * _fast_time_compensation(radar, R_n, win, L, 0.0)
        out[p] = np.sum(W * raw[n])
    return out


def bpa_time(raw, win, radar: Radar, n_rng, M_ap):
    """Full polar time-domain BPA image [n_rng, n_az] (Eq. (14) at every pixel).

    Row by row: with nominal geometry, tap d of every pixel in row r sees the same slant range R_d,
    so the fast-time sums D[n, d] = sum_m W_BP[m, d] * raw[n, m] are one matrix product and
    I(r, theta) = sum_d D[(theta + d) mod n_az, d]."""
    raw = np.asarray(raw, dtype=np.complex128)
    n_az, L = raw.shape
    win = _window(win, L)
    dR = range_bin_spacing(radar, L)
    k = wavenumber(radar)
    d = np.arange(-(M_ap // 2), M_ap - M_ap // 2)
    theta = np.arange(n_az)
    phi_d = phase_centre_angle(d, n_az)
    out = np.zeros((n_rng, n_az), dtype=np.complex128)
    for r in range(n_rng):
        R = radar.r0 + r * dR
        R_d = slant_range(R, 0.0, radar.r0, phi_d)
        alpha = np.where(R_d == 0.0, 1.0, antenna_pattern(off_boresight_angle(R, 0.0, radar.r0, phi_d)))
        W = (alpha * np.exp(-2j * k * R_d))[:, None] * _fast_time_compensation(radar, R_d, win, L, 0.0)
        D = raw @ W.T                                                   # [n_az, M_ap]
        out[r] = np.sum(D[(theta[:, None] + d[None, :]) % n_az, np.arange(M_ap)[None, :]], axis=1)
    return out


def sas_time_pixels(raw, win, w, o, radar: Radar, n_az, rows, thetas, centred=True):
    """Time-domain sparse-aperture imaging at selected pixels, the paper's "SAS" (Algorithm 2).

    I(r, theta) = sum_k w[r, k] * sum_m W_SA[m, k] * win[m] * raw[(theta + o_k) mod n_az, m], the
    Khatri-Rao form 1^T (w^H o (W_SA . Y_IF')) 1 of Sec. III-A with the stored weights w = conj of the
    paper's w (as in Eq. (43) here).  W_SA[m, k] = exp(-j*2*pi*tau_k*K*t_s*(m - m_ref)) with tau_k
    = 2*rho_k/c and rho_k the nominal slant range from the phase centre at pulse offset o_k to the
    pixel (Eq. (2)).  m_ref = 0 is W_SA verbatim (it pairs with weights built with k of Sec. II-B);
    centred=True takes m_ref = (L-1)/2, which pairs with weights built with k_mid.
    w: [n_rng, K]; o: [K] shared or [n_rng, K] per row.
    """
    raw = np.asarray(raw, dtype=np.complex128)
    L = raw.shape[1]
    win = _window(win, L)
    m_ref = (L - 1) / 2.0 if centred else 0.0
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    thetas = np.asarray(thetas, dtype=np.int64).reshape(-1)
    w = np.asarray(w, dtype=np.complex128)
    orow = _offsets_per_row(o, w.shape[0])
    dR = range_bin_spacing(radar, L)
    out = np.zeros(rows.shape[0], dtype=np.complex128)
    for p in range(rows.shape[0]):
        r = rows[p]
        ok = orow[r]
        rho = slant_range(radar.r0 + r * dR, 0.0, radar.r0, phase_centre_angle(ok, n_az))
        E = _fast_time_compensation(radar, rho, win, L, m_ref)           # [K, L]
        n = (thetas[p] + ok) % n_az
        out[p] = np.sum(w[r] * np.sum(E * raw[n], axis=1))
    return out


def sas_time(raw, win, w, o, radar: Radar, n_rng, centred=True):
    """Full polar time-domain SAS image [n_rng, n_az] (Algorithm 2 at every pixel), row by row:
    D[n, k] = sum_m W_SA[m, k] * win[m] * raw[n, m] is one matrix product per row, and
    I(r, theta) = sum_k w[r, k] * D[(theta + o_k) mod n_az, k]."""
    raw = np.asarray(raw, dtype=np.complex128)
    n_az, L = raw.shape
    win = _window(win, L)
    m_ref = (L - 1) / 2.0 if centred else 0.0
    w = np.asarray(w, dtype=np.complex128)
    orow = _offsets_per_row(o, n_rng)
    dR = range_bin_spacing(radar, L)
    theta = np.arange(n_az)
    out = np.zeros((n_rng, n_az), dtype=np.complex128)
    for r in range(n_rng):
        ok = orow[r]
        rho = slant_range(radar.r0 + r * dR, 0.0, radar.r0, phase_centre_angle(ok, n_az))
        D = raw @ _fast_time_compensation(radar, rho, win, L, m_ref).T   # [n_az, K]
        out[r] = np.sum(w[r][None, :] * D[(theta[:, None] + ok[None, :]) % n_az, np.arange(ok.shape[0])[None, :]],
                        axis=1)
    return out


# -------------------------------------------------------- default weights --

def taylor_taper(M, nbar=4, sll_db=30.0):
    """Taylor line-source taper of length M (Taylor 1955), peak-normalised to 1.

    A = acosh(10^(SLL/20))/pi, sigma^2 = nbar^2/(A^2 + (nbar-1/2)^2),
    F_m = (-1)^(m+1) prod_{i<nbar} [1 - m^2/(sigma^2 (A^2 + (i-1/2)^2))] / (2 prod_{i<nbar, i!=m} [1 - m^2/i^2]),
    T(x) = 1 + 2 sum_{m<nbar} F_m cos(2 pi m x), x = (i - (M-1)/2)/M.
    The paper names no taper; the Taylor taper is the default weight design's reading.
    """
    A = math.acosh(10.0 ** (sll_db / 20.0)) / math.pi
    sigma2 = nbar * nbar / (A * A + (nbar - 0.5) ** 2)
    F = []
    for m in range(1, nbar):
        num = 1.0
        den = 1.0
        for i in range(1, nbar):
            num *= 1.0 - m * m / (sigma2 * (A * A + (i - 0.5) ** 2))
            if i != m:
                den *= 1.0 - m * m / float(i * i)
        F.append((-1.0) ** (m + 1) * num / (2.0 * den))
    x = (np.arange(M, dtype=np.float64) - (M - 1) / 2.0) / M

    def T(xx):
        v = np.ones_like(xx)
        for m, Fm in enumerate(F, start=1):
            v = v + 2.0 * Fm * np.cos(2.0 * math.pi * m * xx)
        return v

    return T(x) / T(np.zeros(1))[0]


def default_weights(radar: Radar, L, n_az, n_rng, o, M_ap, nbar=4, sll_db=30.0):
    """Conjugate ideal rotation manifold at the sparse taps, Taylor-tapered, unit norm per row.

    For row r (pixel distance R_r = r0 + r*dR) and tap k (pulse offset o_k, angle 2*pi*o_k/n_az
    from the pixel), the near-field steering entry of Eq. (16) is
    a_k = p(theta'_k) * exp(+j*2*k_mid*rho_k), rho_k from Eq. (2) and theta'_k from Eq. (3) at
    the nominal position (r0, phi_n).  The weight applied as sum_k w*S (Eq. (43) after
    conjugation) is w[r,k] = g_r * T[o_k + M_ap/2] * conj(a_k), with T the Taylor taper on the
    dense aperture and g_r making ||w_r||_2 = 1 (constraint C3, Eq. (20)).  p = 1 when rho_k = 0.
    """
    dR = range_bin_spacing(radar, L)
    k_mid = wavenumber_centred(radar, L)
    o = _offsets_per_row(o, n_rng)
    T = taylor_taper(M_ap, nbar, sll_db)
    w = np.zeros(o.shape, dtype=np.complex128)
    for r in range(n_rng):
        R_r = radar.r0 + r * dR
        phi_k = phase_centre_angle(o[r], n_az)                 # pulse angle relative to the pixel at 0
        rho = slant_range(R_r, 0.0, radar.r0, phi_k)
        p = np.where(rho == 0.0, 1.0, antenna_pattern(off_boresight_angle(R_r, 0.0, radar.r0, phi_k)))
        a = p * np.exp(2j * k_mid * rho)
        v = T[o[r] + M_ap // 2] * np.conj(a)
        nrm = np.linalg.norm(v)
        w[r] = v / nrm if nrm > 0 else 0.0
    return w


# ---------------------------------------------------------------- adjoints --
# For a holomorphic linear map y = A x and a real loss, the gradient in the
# conjugate-Wirtinger convention (the one torch uses) is grad_x = A^H grad_y.

def apply_phase_errors(S, eps):
    """S_tilde[r, n] = S[r, n] * exp(j*eps[n]): per-pulse phase correction before the azimuth filter."""
    return np.asarray(S, dtype=np.complex128) * np.exp(1j * np.asarray(eps, dtype=np.float64))[None, :]


def sparse_azimuth_adjoint_S(g, w, o):
    """grad_S[r, n] = sum_k conj(w[r,k]) * g[r, (n - o_k) mod n_az]: adjoint of Eq. (43) in S."""
    g = np.asarray(g, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    n_rng, n_az = g.shape
    o = _offsets_per_row(o, n_rng)
    n = np.arange(n_az)
    out = np.zeros_like(g)
    for r in range(n_rng):
        for k in range(w.shape[1]):
            out[r] += np.conj(w[r, k]) * g[r, (n - o[r, k]) % n_az]
    return out


def sparse_azimuth_adjoint_w(g, S, o):
    """grad_w[r, k] = sum_theta g[r, theta] * conj(S[r, (theta + o_k) mod n_az]): adjoint of Eq. (43) in w."""
    g = np.asarray(g, dtype=np.complex128)
    S = np.asarray(S, dtype=np.complex128)
    n_rng, n_az = g.shape
    o = _offsets_per_row(o, n_rng)
    th = np.arange(n_az)
    out = np.zeros(o.shape, dtype=np.complex128)
    for r in range(n_rng):
        for k in range(o.shape[1]):
            out[r, k] = np.sum(g[r] * np.conj(S[r, (th + o[r, k]) % n_az]))
    return out


def phase_error_grad(S_tilde, grad_S_tilde):
    """d loss / d eps[n] = sum_r Im(conj(S_tilde[r, n]) * grad_S_tilde[r, n]) for S_tilde = S*exp(j*eps)."""
    return np.sum(np.imag(np.conj(np.asarray(S_tilde)) * np.asarray(grad_S_tilde)), axis=0)


def range_compress_adjoint(g, win, centred=True):
    """grad_raw[n, m] = win[m] * sum_l conj(c_l) * exp(+j*2*pi*l*m/L) * g[l, n]: adjoint of Eq. (38)."""
    g = np.asarray(g, dtype=np.complex128)
    L, n_az = g.shape
    if centred:
        l = np.arange(L, dtype=np.float64)
        g = g * np.exp(-1j * math.pi * l * (L - 1) / L)[:, None]
    G = np.conj(dft_matrix(L)).T @ g                   # [m, n] = sum_l exp(+j2pi l m/L) g[l, n]
    return np.ascontiguousarray((G * np.asarray(win, dtype=np.float64)[:, None]).T)


# ----------------------------------------------------------------- metrics --

def image_entropy(I):
    """E_I = -sum d ln d, d = |I|^2 / sum |I|^2, with 0 ln 0 = 0 (Sec. IV-C, Eq. (45))."""
    p = np.abs(np.asarray(I, dtype=np.complex128)) ** 2
    E = p.sum()
    d = p[p > 0] / E
    return float(-np.sum(d * np.log(d)))


def pisr(I_row, main_idx, side_idx):
    """Peak-to-integral sidelobe ratio |I(phi_m)|^2 / sum_s |I(phi_s)|^2 (Sec. IV-C, Eq. (44))."""
    I_row = np.asarray(I_row)
    return float(np.abs(I_row[main_idx]) ** 2 / np.sum(np.abs(I_row[np.asarray(side_idx)]) ** 2))


def half_mainlobe_width(I_row, peak_idx):
    """Samples from the peak to the closest local minimum of |I| on either side (Sec. IV-C, phi_MW)."""
    a = np.abs(np.asarray(I_row))
    n = a.shape[0]
    best = n
    for step in (-1, 1):
        i = peak_idx
        cnt = 0
        while cnt < n - 1 and a[(i + step) % n] < a[i % n]:
            i += step
            cnt += 1
        best = min(best, cnt)
    return best
