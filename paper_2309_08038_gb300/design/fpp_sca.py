"""Robust sparse-aperture weight design by FPP-SCA (arXiv 2309.08038, Sec. III-A to III-C, Algorithm 1).

For one range bin (pixel distance R from the rotation centre) the design picks complex weights w over
the visible phase centres of a dense aperture so that, under array errors of norm <= Delta_R,
  C1  the main-lobe response at the target direction stays >= U,
  C2  every sidelobe direction outside +-phi_MW stays <= eta * U,
  C3  ||w||_2 = 1 (no noise gain),  C4/C5  U >= U_min,
while ||w||_1 (the convex stand-in for the number of phase centres, Sec. III-B) is minimal.  The
worst-case forms of C1/C2 (Eqs. (26)-(27)), the square-rooted constraints (Eqs. (28)-(32)), the slacked
surrogate (Eq. (33)) and the first-order upper bounds of its concave terms (Eqs. (34)-(35)) give the
convex sub-problem of Eq. (36), a second-order cone program solved here by ``socp.solve``.
Algorithm 1 repeats it ITER times from w_0 = 1/sqrt(N), U'_0 = |w_0^H a(phi_m)|; entries below a
threshold are then set to zero (Sec. III-C) and the slacks are checked (b + b1 + b2 < b_min).

Conventions of this package: the target sits at angle 0 and phase centre o (an offset in pulses) at
angle 2*pi*o/n_az; the steering vector is Eq. (16) with the wavenumber k_mid of the centred range DFT;
the imaging path applies sum_k w[r, k] * S[r, theta + o_k], i.e. the conjugate of the paper's w^H y.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import socp


@dataclass
class Geometry:
    """Rotating-radar geometry for the design: rotation radius r0 (m), pulses per turn n_az, matched
    wavenumber k (rad/m; k_mid for the centred range DFT), dense aperture of M_ap pulses."""
    r0: float
    n_az: int
    k: float
    M_ap: int


@dataclass
class Params:
    phi_mw_deg: float = 1.0         # half width of the main lobe, phi_MW
    eta_db: float = -20.0           # sidelobe to main-lobe power ratio, eta
    u_min_frac: float = 0.5         # U'_min = u_min_frac * ||a(phi_m)||, the matched-filter gain
    lambda_b: float | None = None   # slack penalty; default 10 * sqrt(N) (several times max ||w||_1)
    n_side: int | None = None       # sidelobe directions S; default 2 * N
    iters: int = 100                # ITER (the paper uses 50 to 100)
    threshold: float = 1e-3         # |w_n| < threshold * max |w| is set to zero
    b_min: float = 1e-5
    sigma_deg: float = 0.005        # rotation-angle jitter (Eq. (37)) for Delta_R
    mc_draws: int = 2000
    quantile: float = 0.99
    seed: int = 0


@dataclass
class RowDesign:
    R: float
    offsets: np.ndarray             # candidate phase-centre offsets (visible, within the aperture)
    w: np.ndarray                   # paper's w over the candidates (complex, after thresholding)
    U: float                        # U' of the last iterate
    delta: float                    # Delta_R
    slack: float                    # b + b1 + b2 of the last iterate
    objective: list = field(default_factory=list)   # J^(i) per iteration
    ok: bool = False                # slack < b_min

    @property
    def support(self) -> np.ndarray:
        return np.flatnonzero(self.w != 0)


def steering(geo: Geometry, R: float, phi, offsets, dphi=None) -> np.ndarray:
    """a(phi; R) of Eq. (16) over the phase centres at angles 2*pi*o/n_az (+ dphi): cos(theta'_n) *
    exp(j*2*k*rho_n), rho_n from Eq. (2), theta'_n from Eq. (3) (zero response behind the antenna).
    ``phi`` may be an array: the result is [len(phi), len(offsets)]."""
    phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
    ang = 2.0 * math.pi * np.asarray(offsets, dtype=np.float64) / geo.n_az
    if dphi is not None:
        ang = ang + dphi
    d = phi[:, None] - ang[None, :]
    rho = np.sqrt(R * R + geo.r0 * geo.r0 - 2.0 * R * geo.r0 * np.cos(d))
    proj = R * np.cos(d) - geo.r0
    p = np.where(rho > 0, np.maximum(proj, 0.0) / np.where(rho > 0, rho, 1.0), 1.0)
    return p * np.exp(2j * geo.k * rho)


def candidates(geo: Geometry, R: float) -> np.ndarray:
    """Offsets of the dense aperture [-M/2, M/2) whose phase centre sees the target at angle 0
    (Eqs. (4)-(5): cos(theta') > 0)."""
    o = np.arange(-(geo.M_ap // 2), geo.M_ap - geo.M_ap // 2)
    a = steering(geo, R, 0.0, o)[0]
    return o[np.abs(a) > 0]


def delta_R(geo: Geometry, R: float, offsets, p: Params) -> float:
    """Delta_R of Sec. III-C: the `quantile` of ||a_hat - a|| with phase-centre angles drawn from
    N(2*pi*n/N, sigma) (Eq. (37)), by seeded Monte Carlo."""
    rng = np.random.default_rng(p.seed)
    a = steering(geo, R, 0.0, offsets)[0]
    sig = math.radians(p.sigma_deg)
    norms = np.empty(p.mc_draws)
    for i in range(p.mc_draws):
        ah = steering(geo, R, 0.0, offsets, dphi=rng.standard_normal(len(offsets)) * sig)[0]
        norms[i] = np.linalg.norm(ah - a)
    return float(np.quantile(norms, p.quantile))


def sidelobe_directions(geo: Geometry, offsets, p: Params, n_side: int) -> np.ndarray:
    """S directions spread uniformly over [phi_min, -phi_MW] and [phi_MW, phi_max], phi_min/max the
    angles of the outermost candidate phase centres."""
    ang = 2.0 * math.pi * np.asarray(offsets, dtype=np.float64) / geo.n_az
    lo, hi = float(ang.min()), float(ang.max())
    mw = math.radians(p.phi_mw_deg)
    left = max(0.0, -mw - lo)
    right = max(0.0, hi - mw)
    if left + right <= 0:
        return np.zeros(0)
    n_left = int(round(n_side * left / (left + right)))
    n_right = n_side - n_left
    parts = []
    if n_left:
        parts.append(np.linspace(lo, -mw, n_left))
    if n_right:
        parts.append(np.linspace(mw, hi, n_right))
    return np.concatenate(parts)


def subproblem(a_m, a_s, w_i, U_i, delta, eta, U_min, lam):
    """Eq. (36) as a cone program over x = [Re w, Im w, t, U', b, b1, b2]; returns the socp result and
    the unpacked (w, U', b, b1, b2).  Cone rows (s = h - G x):
      orthant   b, b1, b2 >= 0;  U' >= U'_min (C5);  C4 with -||w||^2 replaced by its bound (Eq. (35))
      Q^3 x N   (t_n, Re w_n, Im w_n): |w_n| <= t_n, so sum t = ||w||_1
      Q^(2N+2)  (b + 2, 2w, b): ||w||^2 <= 1 + b (C3)
      Q^3       (v + 1, 2(U' + Delta), v - 1): (U' + Delta)^2 <= v, v = 2 Re{g^H w} + b1 - |gamma|^2,
                gamma = a_m^H w_i, g = gamma a_m (C1 with Eq. (34))
      Q^4 x S   (v_s + 1, 2 Re a_s^H w, 2 Im a_s^H w, v_s - 1): |a_s^H w|^2 <= v_s,
                v_s = kappa U' + b2 + Delta^2 - eta U_i^2, kappa = 2 (eta U_i - sqrt(eta) Delta) (C2 with Eq. (35))
    """
    N = a_m.shape[0]
    S = a_s.shape[0]
    n = 3 * N + 4
    wr, wi, tt = slice(0, N), slice(N, 2 * N), slice(2 * N, 3 * N)
    iU, ib, ib1, ib2 = 3 * N, 3 * N + 1, 3 * N + 2, 3 * N + 3
    c = np.zeros(n)
    c[tt] = 1.0
    c[ib] = c[ib1] = c[ib2] = lam
    n_rows = 5 + 3 * N + (2 * N + 2) + 3 + 4 * S
    G = np.zeros((n_rows, n))
    h = np.zeros(n_rows)
    # orthant
    G[0, ib] = G[1, ib1] = G[2, ib2] = -1.0
    G[3, iU] = -1.0
    h[3] = -U_min
    G[4, wr] = -2.0 * w_i.real
    G[4, wi] = -2.0 * w_i.imag
    G[4, ib] = -1.0
    h[4] = -1.0 - float(np.vdot(w_i, w_i).real)
    row = 5
    # |w_n| <= t_n
    k = np.arange(N)
    G[row + 3 * k, 2 * N + k] = -1.0
    G[row + 3 * k + 1, k] = -1.0
    G[row + 3 * k + 2, N + k] = -1.0
    row += 3 * N
    # C3
    G[row, ib] = -1.0
    h[row] = 2.0
    G[row + 1 + k, k] = -2.0
    G[row + 1 + N + k, N + k] = -2.0
    G[row + 2 * N + 1, ib] = -1.0
    row += 2 * N + 2
    # C1
    gamma = np.vdot(a_m, w_i)
    g = gamma * a_m
    g2 = float(abs(gamma) ** 2)
    for j, h0 in ((0, 1.0 - g2), (2, -1.0 - g2)):
        G[row + j, wr] = -2.0 * g.real
        G[row + j, wi] = -2.0 * g.imag
        G[row + j, ib1] = -1.0
        h[row + j] = h0
    G[row + 1, iU] = -2.0
    h[row + 1] = 2.0 * delta
    row += 3
    # C2
    kappa = 2.0 * (eta * U_i - math.sqrt(eta) * delta)
    const = delta * delta - eta * U_i * U_i
    r = row + 4 * np.arange(S)
    for j, h0 in ((0, const + 1.0), (3, const - 1.0)):
        G[r + j, iU] = -kappa
        G[r + j, ib2] = -1.0
        h[r + j] = h0
    G[r + 1, wr] = -2.0 * a_s.real
    G[r + 1, wi] = -2.0 * a_s.imag
    G[r + 2, wr] = 2.0 * a_s.imag
    G[r + 2, wi] = -2.0 * a_s.real
    cones = socp.Cones(l=5, q=(3,) * N + (2 * N + 2, 3) + (4,) * S)
    res = socp.solve(c, G, h, cones)
    x = res.x
    w = x[wr] + 1j * x[wi]
    return res, w, float(x[iU]), float(x[ib]), float(x[ib1]), float(x[ib2])


def design_row(geo: Geometry, R: float, p: Params = Params()) -> RowDesign:
    """Algorithm 1 for one range bin at distance R from the rotation centre."""
    offs = candidates(geo, R)
    N = len(offs)
    a_m = steering(geo, R, 0.0, offs)[0]
    if N <= 2:                                   # nothing to thin out: the matched filter
        w = a_m / np.linalg.norm(a_m)
        return RowDesign(R=R, offsets=offs, w=w, U=float(abs(np.vdot(w, a_m))), delta=0.0, slack=0.0, ok=True)
    delta = delta_R(geo, R, offs, p)
    S = p.n_side if p.n_side is not None else 2 * N
    phis = sidelobe_directions(geo, offs, p, S)
    a_s = steering(geo, R, phis, offs)
    eta = 10.0 ** (p.eta_db / 10.0)
    U_min = p.u_min_frac * float(np.linalg.norm(a_m))
    lam = p.lambda_b if p.lambda_b is not None else 10.0 * math.sqrt(N)
    w = np.full(N, 1.0 / math.sqrt(N), dtype=np.complex128)
    U = float(abs(np.vdot(w, a_m)))
    J = []
    slack = np.inf
    for _ in range(p.iters):
        res, w, U, b, b1, b2 = subproblem(a_m, a_s, w, U, delta, eta, U_min, lam)
        slack = b + b1 + b2
        J.append(float(np.sum(np.abs(w)) + lam * slack))
    wt = np.where(np.abs(w) < p.threshold * np.max(np.abs(w)), 0.0, w)
    return RowDesign(R=R, offsets=offs, w=wt, U=U, delta=delta, slack=float(slack), objective=J,
                     ok=bool(slack < p.b_min))


def to_taps(designs, K: int | None = None):
    """Per-row taps for the imaging path: offsets o[r, k] (int32) and weights w[r, k] = conj(paper's w)
    (complex64) over each row's support, padded to a common K with zero weights (padding repeats the
    row's first offset so the offset span does not grow)."""
    sup = [d.support for d in designs]
    K = max(max(len(s) for s in sup), 1) if K is None else K
    o = np.zeros((len(designs), K), dtype=np.int32)
    w = np.zeros((len(designs), K), dtype=np.complex64)
    for r, (d, s) in enumerate(zip(designs, sup)):
        if len(s) > K:
            raise ValueError(f"row {r}: support {len(s)} exceeds K={K}")
        if len(s) == 0:
            continue
        o[r, :len(s)] = d.offsets[s]
        o[r, len(s):] = d.offsets[s[0]]
        w[r, :len(s)] = np.conj(d.w[s])
    return w, o


def design(geo: Geometry, R_rows, p: Params = Params(), log=None):
    """Algorithm 1 over a list of range bins (pixel distances R); returns one RowDesign per bin."""
    out = []
    for i, R in enumerate(R_rows):
        d = design_row(geo, float(R), p)
        out.append(d)
        if log is not None:
            log(f"bin {i}: R={R:.3f} m  N={len(d.offsets)}  kept={len(d.support)}  slack={d.slack:.2e}  "
                f"ok={d.ok}")
    return out


def main(argv=None):
    """Offline design for rows of a synthetic scan configuration, written as an .npz of per-row taps
    (w [rows, K] complex64, o [rows, K] int32, rows, slack, ok) for rosar_sparse_azimuth /
    rosar_azimuth_plan with per-row offsets."""
    import argparse
    import sys
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--config", default="indoor")
    ap.add_argument("--rows", default="1:256:32", help="start:stop:step of image rows")
    ap.add_argument("--M-ap", type=int, default=None, help="dense aperture (default: the config's)")
    ap.add_argument("--iters", type=int, default=Params.iters)
    ap.add_argument("--eta-db", type=float, default=Params.eta_db)
    ap.add_argument("--phi-mw-deg", type=float, default=Params.phi_mw_deg)
    ap.add_argument("--sigma-deg", type=float, default=Params.sigma_deg)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    import synth
    cfg = synth.CONFIGS[a.config]
    rad = cfg.radar
    L = cfg.L
    f_mid = rad.fc + rad.slope * (rad.t_start + rad.t_sample(L) * (L - 1) / 2.0)
    geo = Geometry(r0=rad.r0, n_az=cfg.n_az, k=2.0 * math.pi * f_mid / rad.c, M_ap=a.M_ap or cfg.M_ap)
    start, stop, step = (int(x) for x in a.rows.split(":"))
    rows = np.arange(start, min(stop, L), step)
    p = Params(iters=a.iters, eta_db=a.eta_db, phi_mw_deg=a.phi_mw_deg, sigma_deg=a.sigma_deg)
    ds = design(geo, rad.r0 + rows * rad.bin_spacing(L), p, log=lambda m: print(m, file=sys.stderr))
    w, o = to_taps(ds)
    np.savez(a.out, w=w, o=o, rows=rows, slack=np.array([d.slack for d in ds]), ok=np.array([d.ok for d in ds]))


if __name__ == "__main__":
    main()
