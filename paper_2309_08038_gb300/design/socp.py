"""Dense primal-dual interior-point solver for second-order cone programs.

    minimize    c^T x
    subject to  G x + s = h,   A x = b,   s in K = R_+^l x Q^{q_1} x ... x Q^{q_m},

with Q^q = {u in R^q : u_0 >= ||u_{1:}||_2}.  Dual: maximize -h^T z - b^T y subject to
G^T z + A^T y + c = 0, z in K.

Method: infeasible-start path following with Nesterov-Todd scaling and Mehrotra's
predictor-corrector, as published by Nesterov and Todd ("Self-scaled barriers and interior-point
methods for convex programming", 1997) and laid out for cone programs by Vandenberghe ("The CVXOPT
linear and quadratic cone program solvers", 2010).  Each Newton system is reduced to the dense
normal matrix (W^-1 G)^T (W^-1 G), factored by Cholesky; A is handled by a Schur complement.

Used offline (the weight design of the sparse aperture), never on the imaging path.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Cones:
    l: int                  # nonnegative orthant dimension
    q: tuple                # second-order cone dimensions (each >= 2), blocks laid out after the orthant

    def __post_init__(self):
        self.q = tuple(int(d) for d in self.q)
        groups = {}
        off = self.l
        for d in self.q:
            groups.setdefault(d, []).append(np.arange(off, off + d))
            off += d
        # blocks of equal dimension handled together: index arrays [n_blocks, d]
        self.groups = [np.array(v) for _, v in sorted(groups.items())]

    @property
    def size(self) -> int:
        return self.l + int(sum(self.q))

    @property
    def degree(self) -> int:
        return self.l + len(self.q)


@dataclass
class Result:
    x: np.ndarray
    s: np.ndarray
    z: np.ndarray
    y: np.ndarray
    status: str             # "optimal", "max_iterations" or "stalled"
    iterations: int
    primal_objective: float
    dual_objective: float
    gap: float
    residual: float


def identity(cones: Cones) -> np.ndarray:
    e = np.zeros(cones.size)
    e[:cones.l] = 1.0
    for idx in cones.groups:
        e[idx[:, 0]] = 1.0
    return e


def min_eig(u: np.ndarray, cones: Cones) -> float:
    """Smallest Jordan eigenvalue of u (u is interior iff this is positive)."""
    vals = [np.min(u[:cones.l])] if cones.l else []
    for idx in cones.groups:
        U = u[idx]
        vals.append(np.min(U[:, 0] - np.linalg.norm(U[:, 1:], axis=1)))
    return float(min(vals))


def jordan(u: np.ndarray, v: np.ndarray, cones: Cones) -> np.ndarray:
    """u o v: elementwise on the orthant, (u^T v, u_0 v_1 + v_0 u_1) on each second-order cone."""
    out = np.empty_like(u)
    out[:cones.l] = u[:cones.l] * v[:cones.l]
    for idx in cones.groups:
        U, V = u[idx], v[idx]
        out[idx[:, 0]] = np.sum(U * V, axis=1)
        out[idx[:, 1:]] = U[:, :1] * V[:, 1:] + V[:, :1] * U[:, 1:]
    return out


def jordan_solve(lam: np.ndarray, u: np.ndarray, cones: Cones) -> np.ndarray:
    """x with lam o x = u (lam interior): the inverse of the arrow matrix of lam applied to u."""
    out = np.empty_like(u)
    out[:cones.l] = u[:cones.l] / lam[:cones.l]
    for idx in cones.groups:
        Lm, U = lam[idx], u[idx]
        l0, l1 = Lm[:, 0], Lm[:, 1:]
        u0, u1 = U[:, 0], U[:, 1:]
        nl = np.linalg.norm(l1, axis=1)
        det = (l0 - nl) * (l0 + nl)
        lu = np.sum(l1 * u1, axis=1)
        out[idx[:, 0]] = (l0 * u0 - lu) / det
        out[idx[:, 1:]] = (-u0[:, None] * l1 + (det / l0)[:, None] * u1 + (lu / l0)[:, None] * l1) / det[:, None]
    return out


class Scaling:
    """Nesterov-Todd scaling W (symmetric) with W z = W^-1 s = lambda.

    Orthant: W = diag(sqrt(s/z)).  Second-order cone: W = beta (2 v v^T - J), J = diag(1, -1, ..., -1),
    beta = (s^T J s / z^T J z)^(1/4), v built from the normalised points s/sqrt(s^T J s), z/sqrt(z^T J z);
    W^-1 = (2 (Jv)(Jv)^T - J) / beta.
    """

    def __init__(self, s: np.ndarray, z: np.ndarray, cones: Cones):
        self.cones = cones
        self.d = np.sqrt(s[:cones.l] / z[:cones.l])
        self.soc = []
        for idx in cones.groups:
            Sb, Zb = s[idx], z[idx]
            ns, nz = np.linalg.norm(Sb[:, 1:], axis=1), np.linalg.norm(Zb[:, 1:], axis=1)
            sjs = (Sb[:, 0] - ns) * (Sb[:, 0] + ns)          # s^T J s without cancellation
            zjz = (Zb[:, 0] - nz) * (Zb[:, 0] + nz)
            sn, zn = Sb / np.sqrt(sjs)[:, None], Zb / np.sqrt(zjz)[:, None]
            gamma = np.sqrt(0.5 * (1.0 + np.sum(sn * zn, axis=1)))
            wb = sn.copy()
            wb[:, 0] += zn[:, 0]
            wb[:, 1:] -= zn[:, 1:]
            wb /= (2.0 * gamma)[:, None]
            v = wb.copy()
            v[:, 0] += 1.0
            v /= np.sqrt(2.0 * (wb[:, 0] + 1.0))[:, None]
            beta = (sjs / zjz) ** 0.25
            jv = -v
            jv[:, 0] = v[:, 0]
            self.soc.append((idx, beta, v, jv))

    def apply(self, u: np.ndarray, inverse: bool = False) -> np.ndarray:
        """W u (or W^-1 u); u may be a vector or a matrix with the cone index first."""
        out = np.empty_like(u)
        l = self.cones.l
        if u.ndim == 1:
            out[:l] = u[:l] / self.d if inverse else u[:l] * self.d
        else:
            out[:l] = u[:l] / self.d[:, None] if inverse else u[:l] * self.d[:, None]
        for idx, beta, v, jv in self.soc:
            Ub = u[idx]                                  # [nb, d] or [nb, d, n]
            vv = jv if inverse else v
            if Ub.ndim == 2:
                r = 2.0 * vv * np.sum(vv * Ub, axis=1)[:, None]
                r[:, 0] -= Ub[:, 0]
                r[:, 1:] += Ub[:, 1:]
                out[idx] = r / beta[:, None] if inverse else r * beta[:, None]
            else:
                r = 2.0 * vv[:, :, None] * np.einsum("bd,bdn->bn", vv, Ub)[:, None, :]
                r[:, 0] -= Ub[:, 0]
                r[:, 1:] += Ub[:, 1:]
                out[idx] = r / beta[:, None, None] if inverse else r * beta[:, None, None]
        return out


def max_step(u: np.ndarray, du: np.ndarray, cones: Cones) -> float:
    """Largest alpha >= 0 with u + alpha du in K (u interior); inf if the ray stays inside.

    On a second-order cone the boundary is a t^2 + 2 b t + c = 0 (a = d^T J d, b = u^T J d, c = u^T J u)
    with u_0 + t d_0 >= 0; its roots are taken in the cancellation-free forms q/a and c/q."""
    alpha = np.inf
    if cones.l:
        neg = du[:cones.l] < 0
        if np.any(neg):
            alpha = min(alpha, float(np.min(-u[:cones.l][neg] / du[:cones.l][neg])))
    for idx in cones.groups:
        U, D = u[idx], du[idx]
        u0, d0 = U[:, 0], D[:, 0]
        a = d0 * d0 - np.sum(D[:, 1:] ** 2, axis=1)
        b = u0 * d0 - np.sum(U[:, 1:] * D[:, 1:], axis=1)
        nu = np.linalg.norm(U[:, 1:], axis=1)
        c = (u0 - nu) * (u0 + nu)
        stays = (a >= 0) & (d0 >= 0) & ~((a == 0) & (b < 0))
        disc = np.maximum(b * b - a * c, 0.0)
        q = -(b + np.copysign(np.sqrt(disc), b))
        with np.errstate(divide="ignore", invalid="ignore"):
            r1 = np.where(a != 0, q / a, np.where(b < 0, -c / (2.0 * b), np.inf))
            r2 = np.where(q != 0, c / q, np.inf)
        r1 = np.where(r1 > 0, r1, np.inf)
        r2 = np.where(r2 > 0, r2, np.inf)
        t = np.where(stays, np.inf, np.minimum(r1, r2))
        if t.size:
            alpha = min(alpha, float(np.min(t)))
    return alpha


def _factor(Y: np.ndarray, A: np.ndarray | None):
    H = Y.T @ Y
    n = H.shape[0]
    reg = 1e-13 * max(1.0, float(np.max(np.abs(np.diag(H)))))
    H[np.diag_indices(n)] += reg
    Lh = np.linalg.cholesky(H)
    if A is None or A.shape[0] == 0:
        return Lh, None, None
    HA = _chol_solve(Lh, A.T)                 # H^-1 A^T
    Sc = A @ HA
    Sc[np.diag_indices(Sc.shape[0])] += reg
    return Lh, HA, np.linalg.cholesky(Sc)


def _chol_solve(L: np.ndarray, r: np.ndarray) -> np.ndarray:
    from scipy.linalg import solve_triangular
    return solve_triangular(L.T, solve_triangular(L, r, lower=True), lower=False)


def solve(c, G, h, cones: Cones, A=None, b=None, feastol=1e-8, abstol=1e-9, reltol=1e-8,
          max_iter=100) -> Result:
    """Solve the cone program above.  Returns the last iterate with status "optimal" when the scaled
    primal/dual residuals are below ``feastol`` and the duality gap below ``abstol`` or ``reltol``
    relative to the objective; "max_iterations" or "stalled" (an iterate reached the cone boundary in
    floating point before the tolerances were met) otherwise."""
    c = np.asarray(c, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n = c.shape[0]
    if A is None:
        A = np.zeros((0, n))
        b = np.zeros(0)
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p = A.shape[0]
    e = identity(cones)

    # start: the Newton point with identity scaling, both slacks pushed into the cone interior
    Lh, HA, Ls = _factor(G, A)
    rhs = -c + G.T @ h
    x, y = _kkt_solve(Lh, HA, Ls, A, rhs, b)
    z = G @ x - h
    s = -z
    for u in (s, z):
        m = min_eig(u, cones)
        if m <= 1e-8 * (1.0 + np.linalg.norm(u)):
            u += (1.0 - m) * e if m < 0 else (1.0) * e

    nc, nb, nh = 1.0 + np.linalg.norm(c), 1.0 + np.linalg.norm(b), 1.0 + np.linalg.norm(h)
    status = "max_iterations"
    it = 0
    for it in range(1, max_iter + 1):
        rx = c + G.T @ z + A.T @ y
        ry = A @ x - b
        rz = G @ x + s - h
        gap = float(s @ z)
        pobj, dobj = float(c @ x), float(-h @ z - b @ y)
        res = max(np.linalg.norm(rx) / nc, np.linalg.norm(ry) / nb if p else 0.0, np.linalg.norm(rz) / nh)
        if res < feastol and (gap < abstol or gap < reltol * max(abs(pobj), abs(dobj))):
            status = "optimal"
            break
        if min_eig(s, cones) <= 0.0 or min_eig(z, cones) <= 0.0:
            status = "stalled"
            break
        mu = gap / cones.degree
        W = Scaling(s, z, cones)
        lam = W.apply(z)
        Y = W.apply(G, inverse=True)
        Lh, HA, Ls = _factor(Y, A)

        def newton(ds):
            u = jordan_solve(lam, ds, cones)                    # lambda <> ds
            bz_s = W.apply(-rz, inverse=True) - u               # W^-1 bz - lambda <> ds
            dx, dy = _kkt_solve(Lh, HA, Ls, A, -rx + Y.T @ bz_s, -ry)
            dz = W.apply(Y @ dx - bz_s, inverse=True)           # W^-1 (W^-1 (G dx - bz) + lambda <> ds)
            dsv = W.apply(u - W.apply(dz))                      # W (lambda <> ds - W dz)
            return dx, dy, dsv, dz

        dx, dy, dsa, dza = newton(-jordan(lam, lam, cones))
        a_aff = min(1.0, max_step(s, dsa, cones), max_step(z, dza, cones))
        sigma = (float((s + a_aff * dsa) @ (z + a_aff * dza)) / gap) ** 3 if gap > 0 else 0.0
        corr = jordan(W.apply(dsa, inverse=True), W.apply(dza), cones)
        dx, dy, ds_, dz_ = newton(-jordan(lam, lam, cones) + sigma * mu * e - corr)
        alpha = min(1.0, 0.99 * min(max_step(s, ds_, cones), max_step(z, dz_, cones)))
        x = x + alpha * dx
        y = y + alpha * dy
        s = s + alpha * ds_
        z = z + alpha * dz_
    rx = c + G.T @ z + A.T @ y
    rz = G @ x + s - h
    ry = A @ x - b
    res = max(np.linalg.norm(rx) / nc, np.linalg.norm(ry) / nb if p else 0.0, np.linalg.norm(rz) / nh)
    return Result(x=x, s=s, z=z, y=y, status=status, iterations=it, primal_objective=float(c @ x),
                  dual_objective=float(-h @ z - b @ y), gap=float(s @ z), residual=float(res))


def _kkt_solve(Lh, HA, Ls, A, r1, r2):
    """[[H, A^T], [A, 0]] [x; y] = [r1; r2] with H = Lh Lh^T."""
    Hr = _chol_solve(Lh, r1)
    if Ls is None:
        return Hr, np.zeros(0)
    y = _chol_solve(Ls, A @ Hr - r2)
    return Hr - HA @ y, y
