"""Offline weight design (FPP-SCA, Sec. III / Algorithm 1) and its cone solver (CPU only).

The solver is pinned to scipy's LP solver, closed-form cone programs and the defining identities of
its Nesterov-Todd scaling; the FPP-SCA sub-problem (Eq. (36)) to an independent general-purpose
solver; Algorithm 1 to the properties the paper states (monotone objective, slacks vanishing, the
robust main-lobe/sidelobe constraints met, fewer than half of the phase centres kept), and the taps
it emits to the imaging path's convention through the oracle's filter.
"""

import math

import numpy as np
import pytest
from scipy.optimize import linprog, minimize

import oracle as O
import synth
from paper_2309_08038_gb300.design import fpp_sca as F
from paper_2309_08038_gb300.design import socp


# ------------------------------------------------------------------ solver --

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_socp_solves_random_lps_like_scipy(seed):
    rng = np.random.default_rng(seed)
    n, m = 8, 20
    G = rng.standard_normal((m, n))
    h = G @ rng.standard_normal(n) + rng.uniform(0.1, 1.0, m)     # strictly feasible primal
    c = -G.T @ rng.uniform(0.1, 1.0, m)                           # strictly feasible dual: bounded
    r = socp.solve(c, G, h, socp.Cones(l=m, q=()))
    ref = linprog(c, A_ub=G, b_ub=h, bounds=[(None, None)] * n, method="highs")
    assert r.status == "optimal"
    assert r.primal_objective == pytest.approx(ref.fun, rel=1e-7, abs=1e-7)


def test_socp_unit_ball_closed_form():
    """min c^T x s.t. ||x|| <= 1 has x = -c/||c||."""
    rng = np.random.default_rng(3)
    n = 5
    c = rng.standard_normal(n)
    G = np.vstack([np.zeros((1, n)), -np.eye(n)])
    h = np.r_[1.0, np.zeros(n)]
    r = socp.solve(c, G, h, socp.Cones(l=0, q=(n + 1,)))
    np.testing.assert_allclose(r.x, -c / np.linalg.norm(c), atol=1e-7)


def test_socp_projection_onto_affine_set_with_equalities():
    """min ||x - p|| s.t. A x = b is the orthogonal projection p - A^T (A A^T)^-1 (A p - b)."""
    rng = np.random.default_rng(4)
    n, k = 6, 2
    A = rng.standard_normal((k, n))
    b = rng.standard_normal(k)
    pt = rng.standard_normal(n)
    c = np.r_[np.zeros(n), 1.0]
    G = np.zeros((n + 1, n + 1))
    G[0, n] = -1.0
    G[1:, :n] = -np.eye(n)
    h = np.r_[0.0, -pt]
    r = socp.solve(c, G, h, socp.Cones(l=0, q=(n + 1,)), A=np.c_[A, np.zeros(k)], b=b)
    ref = pt - A.T @ np.linalg.solve(A @ A.T, A @ pt - b)
    np.testing.assert_allclose(r.x[:n], ref, atol=1e-8)


def _interior(rng, cones):
    u = rng.standard_normal(cones.size)
    u[:cones.l] = rng.uniform(0.2, 2.0, cones.l)
    off = cones.l
    for d in cones.q:
        u[off] = np.linalg.norm(u[off + 1:off + d]) + rng.uniform(0.1, 1.0)
        off += d
    return u


def test_nt_scaling_and_jordan_identities():
    """W z = W^-1 s (the Nesterov-Todd point), W^-1 W = I, and lam o (lam <> u) = u."""
    rng = np.random.default_rng(5)
    cones = socp.Cones(l=3, q=(4, 2, 3, 3, 5))
    s, z = _interior(rng, cones), _interior(rng, cones)
    W = socp.Scaling(s, z, cones)
    np.testing.assert_allclose(W.apply(z), W.apply(s, inverse=True), atol=1e-12)
    u = rng.standard_normal(cones.size)
    np.testing.assert_allclose(W.apply(W.apply(u), inverse=True), u, atol=1e-12)
    M = rng.standard_normal((cones.size, 4))
    np.testing.assert_allclose(W.apply(M)[:, 2], W.apply(M[:, 2]), atol=1e-12)
    lam = W.apply(z)
    np.testing.assert_allclose(socp.jordan(lam, socp.jordan_solve(lam, u, cones), cones), u, atol=1e-10)


def test_max_step_lands_on_the_cone_boundary():
    rng = np.random.default_rng(6)
    cones = socp.Cones(l=4, q=(3, 4, 6))
    hit = 0
    for _ in range(50):
        u = _interior(rng, cones)
        d = rng.standard_normal(cones.size) * 3
        a = socp.max_step(u, d, cones)
        if np.isfinite(a):
            assert socp.min_eig(u + a * d, cones) == pytest.approx(0.0, abs=1e-9)
            assert socp.min_eig(u + 0.999 * a * d, cones) > 0
            hit += 1
        else:
            assert socp.min_eig(u + 1e6 * d, cones) >= 0
    assert hit > 30


# ------------------------------------------------------------- sub-problem --

def _geometry(M_ap=60):
    cfg = synth.INDOOR
    rad = cfg.radar
    L = cfg.L
    orad = O.Radar(fc=rad.fc, slope=rad.slope, t_s=rad.t_sample(L), t_start=rad.t_start, r0=rad.r0, c=rad.c)
    return F.Geometry(r0=rad.r0, n_az=cfg.n_az, k=O.wavenumber_centred(orad, L), M_ap=M_ap), rad, L


def test_subproblem_matches_a_general_purpose_solver():
    """Eq. (36) on a small instance: the cone program's optimum equals SLSQP's on the constraints
    written out directly (|w_n| <= t_n, ||w||^2 <= 1 + b, the linearised C1, C2, C4, and C5)."""
    rng = np.random.default_rng(7)
    N, S = 5, 3
    a_m = (rng.uniform(0.5, 1.0, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N)))
    a_s = rng.standard_normal((S, N)) * 0.3 + 1j * rng.standard_normal((S, N)) * 0.3
    w_i = np.exp(1j * rng.uniform(0, 2 * np.pi, N)) / math.sqrt(N)
    U_i, delta, eta, U_min, lam = 0.8, 0.05, 0.1, 0.7, 5.0
    res, w, U, b, b1, b2 = F.subproblem(a_m, a_s, w_i, U_i, delta, eta, U_min, lam)
    assert res.status == "optimal"
    J_cone = float(np.sum(np.abs(w)) + lam * (b + b1 + b2))

    gamma = np.vdot(a_m, w_i)
    g = gamma * a_m

    def unpack(x):
        return x[:N] + 1j * x[N:2 * N], x[2 * N:3 * N], x[3 * N], x[3 * N + 1], x[3 * N + 2], x[3 * N + 3]

    def obj(x):
        _, t, _, bb, bb1, bb2 = unpack(x)
        return np.sum(t) + lam * (bb + bb1 + bb2)

    cons = []
    cons.append({"type": "ineq", "fun": lambda x: unpack(x)[1] ** 2 - np.abs(unpack(x)[0]) ** 2})
    cons.append({"type": "ineq", "fun": lambda x: unpack(x)[1]})
    cons.append({"type": "ineq", "fun": lambda x: np.array(unpack(x)[3:])})
    cons.append({"type": "ineq", "fun": lambda x: unpack(x)[2] - U_min})
    cons.append({"type": "ineq", "fun": lambda x: -(1 - unpack(x)[3] + np.vdot(w_i, w_i).real
                                                    - 2 * np.vdot(w_i, unpack(x)[0]).real)})
    cons.append({"type": "ineq", "fun": lambda x: 1 + unpack(x)[3] - np.vdot(unpack(x)[0], unpack(x)[0]).real})
    cons.append({"type": "ineq", "fun": lambda x: -((unpack(x)[2] + delta) ** 2 + abs(gamma) ** 2
                                                    - 2 * np.vdot(g, unpack(x)[0]).real - unpack(x)[4])})
    cons.append({"type": "ineq", "fun": lambda x: -(np.abs(a_s.conj() @ unpack(x)[0]) ** 2
                                                    + 2 * (math.sqrt(eta) * delta - eta * U_i) * unpack(x)[2]
                                                    + eta * U_i ** 2 - delta ** 2 - unpack(x)[5])})
    # the cone solution satisfies the constraints as written out
    x_cone = np.r_[w.real, w.imag, np.abs(w), U, b, b1, b2]
    for con in cons:
        assert np.min(con["fun"](x_cone)) >= -1e-7
    # and a general-purpose local solver from a generic start reaches the same optimum
    x0 = np.r_[w_i.real, w_i.imag, np.abs(w_i) + 0.1, U_min + 0.1, 2.0, 5.0, 5.0]
    ref = minimize(obj, x0, constraints=cons, method="SLSQP", options={"ftol": 1e-10, "maxiter": 1000})
    viol = min(float(np.min(con["fun"](ref.x))) for con in cons)
    assert viol >= -1e-6
    assert ref.fun == pytest.approx(J_cone, rel=1e-4)


# ------------------------------------------------------------- Algorithm 1 --

@pytest.fixture(scope="module")
def row_design():
    geo, rad, L = _geometry(M_ap=80)
    R = rad.r0 + 30 * rad.bin_spacing(L)
    p = F.Params(phi_mw_deg=2.5, eta_db=-18.0, iters=60, mc_draws=300)
    return geo, R, p, F.design_row(geo, R, p)


def test_fpp_sca_objective_is_monotone_and_slacks_vanish(row_design):
    """SCA with tight upper bounds (Eqs. (34)-(35)): each iterate is feasible for the next surrogate,
    so J^(i) never increases; FPP drives the slacks below b_min (Sec. III-C)."""
    _, _, p, d = row_design
    J = np.array(d.objective)
    assert len(J) == p.iters
    assert np.all(np.diff(J) <= 1e-6 * J[:-1])
    assert d.ok and d.slack < p.b_min


def test_fpp_sca_meets_the_robust_pattern_constraints(row_design):
    """Worst case over the error ball: (|w^H a_m| - Delta)^2 >= U >= U_min and (|w^H a_s| + Delta)^2 <=
    eta U for every sidelobe direction (Eqs. (26)-(27)); ||w|| = 1 (C3); under half the phase centres."""
    geo, R, p, d = row_design
    offs = d.offsets
    a_m = F.steering(geo, R, 0.0, offs)[0]
    phis = F.sidelobe_directions(geo, offs, p, 2 * len(offs))
    a_s = F.steering(geo, R, phis, offs)
    w = d.w
    U = d.U ** 2
    eta = 10 ** (p.eta_db / 10)
    tol = 1e-3
    assert d.U >= p.u_min_frac * np.linalg.norm(a_m) * (1 - 1e-6)
    assert (abs(np.vdot(w, a_m)) - d.delta) ** 2 >= U * (1 - tol)
    assert np.max((np.abs(a_s.conj() @ w) + d.delta) ** 2) <= eta * U * (1 + tol)
    assert np.linalg.norm(w) == pytest.approx(1.0, abs=1e-3)
    assert 0 < len(d.support) < len(offs) / 2


def test_delta_R_is_first_order_in_the_jitter():
    """Delta_R of Sec. III-C scales linearly with small angle jitter and vanishes without it."""
    geo, rad, L = _geometry(M_ap=60)
    R = rad.r0 + 40 * rad.bin_spacing(L)
    offs = F.candidates(geo, R)
    d1 = F.delta_R(geo, R, offs, F.Params(sigma_deg=1e-4, mc_draws=400))
    d2 = F.delta_R(geo, R, offs, F.Params(sigma_deg=2e-4, mc_draws=400))
    assert F.delta_R(geo, R, offs, F.Params(sigma_deg=0.0, mc_draws=10)) == 0.0
    assert d2 / d1 == pytest.approx(2.0, rel=1e-3)


def test_taps_apply_the_paper_weights_through_the_imaging_filter(row_design):
    """to_taps stores conj(w) at the support's offsets: the oracle's sparse filter applied to pulses
    that carry a(phi_m) returns w^H a(phi_m), the paper's pattern value (Eq. (17))."""
    geo, R, _, d = row_design
    w_t, o_t = F.to_taps([d, d], K=len(d.support) + 3)
    assert np.all(w_t[:, len(d.support):] == 0)
    n_az = geo.n_az
    a_m = F.steering(geo, R, 0.0, d.offsets)[0]
    S = np.zeros((2, n_az), dtype=np.complex128)
    th = 100
    S[:, (th + d.offsets) % n_az] = a_m
    out = O.sparse_azimuth(S, w_t, o_t)
    assert out[0, th] == pytest.approx(np.vdot(d.w, a_m), rel=1e-6)
