"""FP64 reference interior point method (TEST INFRASTRUCTURE ONLY).

Follows, in order, the paper's problem statement and Algorithm 1:

* Eq. (1)  convex QP  min 1/2 x'Hx + p'x,  l <= Ax <= u,  Cx = b  (plus simple
  variable bounds, which section 3.1 treats separately);
* Eq. (2)  log-barrier on the slacks s_l, s_u and the penalty-barrier
  (1/2mu)||Cx-b||^2 for equalities;
* Eq. (3)  perturbed KKT conditions (residuals r_H, r_A, r_e, r_c);
* Eq. (7)  full Newton system in (dx, dlam, ds) with bounds separated;
* Eq. (8)  2x2 block reduction [Q -B'; B D];
* Eq. (9)  doubly augmented SPD system [Q+2B'D^-1B  B'; B  D];
* Eq. (10) ratio test with gamma = 0.99;
* section 3.2 mu rule: if ||r|| < mu then (return if mu < mu_tol, else mu/=10).

Readings of places where the paper is silent or inconsistent (the same
readings the GPU library implements, from this text, independently):

* r_c2 = lam_u * s_u - mu and r_uA = -Ax - s_u + u (the printed r_c2 uses lam_l
  and r_uA's slack sign differs from Eq. (2); the forms here are the ones
  Eq. (2) and the block "-A ... -I" row of Eq. (7) imply).
* The stationarity term of the equalities is -C' lam_e (Eq. (3)); the Jacobian
  entry is therefore -C', which is what B = [C; A; -A] with -B' in Eq. (8)
  gives.  The printed +C' in the top row of Eq. (7) is read as a sign typo.
* mu is kept as an exact power of ten 10^-k; the iteration returns when
  ||r||_2 < mu and mu < mu_tol (strict), so with mu_tol = 1e-6 the final mu
  is 1e-7.
* The residual norm ||r|| is the 2-norm of all ten blocks of the right-hand
  side of Eq. (7) evaluated with the current mu.
* Ratio test: alpha_x over all slack groups (s_lA, s_uA, s_lx, s_ux), alpha_lam
  over all sign-constrained multipliers (lam_lA, lam_uA, lam_lx, lam_ux); an
  empty set gives 1.  lam_e (free) is updated with alpha_lam.
* Initial point: x0 = midpoint of two finite bounds, l+1 / u-1 if one, 0 if
  none; each slack = max(its constraint value at x0, 1); inequality
  multipliers = 1; lam_e = 0; mu0 = 1.
* Scaling: objective scaled by sigma = 1/max(1, max_i H_ii, ||p||_inf); every
  A and C row (and its bounds / rhs) divided by its 2-norm.  No variable
  scaling.  Results are mapped back to original units.
* PCG stopping test (only used by :func:`pcg_reference`): relative
  unpreconditioned residual ||rhs - K z||_2 <= tol ||rhs||_2, z0 = 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


# ---------------------------------------------------------------------------
# Scaled problem
# ---------------------------------------------------------------------------
@dataclass
class Scaled:
    n: int
    hkind: str
    sigma: float
    p: np.ndarray
    H: Optional[np.ndarray] = None          # dense, scaled
    P: Optional[sp.csr_matrix] = None       # csr_lsq: float64 P
    w2: Optional[np.ndarray] = None         # csr_lsq: 2*sigma*w  (H = P' diag(w2) P)
    Z: Optional[np.ndarray] = None          # lowrank: sqrt(sigma) Z (float64)
    zw: Optional[np.ndarray] = None         # lowrank: column weights W (H = Z W Z' + H0)
    d0: Optional[np.ndarray] = None         # lowrank: sigma * diagonal H0
    A: object = None                        # scaled rows: dense ndarray or csr
    rhoA: Optional[np.ndarray] = None
    lA: Optional[np.ndarray] = None
    uA: Optional[np.ndarray] = None
    L: Optional[np.ndarray] = None          # rows with finite lower bound
    U: Optional[np.ndarray] = None          # rows with finite upper bound
    C: Optional[np.ndarray] = None          # scaled equality rows (dense)
    rhoC: Optional[np.ndarray] = None
    b: Optional[np.ndarray] = None
    lx: Optional[np.ndarray] = None
    ux: Optional[np.ndarray] = None
    Lx: Optional[np.ndarray] = None
    Ux: Optional[np.ndarray] = None
    _hband: object = field(default=None, repr=False)

    @property
    def m(self):
        return self.A.shape[0]

    @property
    def me(self):
        return self.C.shape[0]

    @property
    def NK(self):
        return self.n + self.me + len(self.L) + len(self.U)

    # H v from the operator's structure
    def Hv(self, v):
        if self.hkind == "dense":
            return self.H @ v
        if self.hkind == "csr_lsq":
            return self.P.T @ (self.w2 * (self.P @ v))
        return self.Z @ (self.zw * (self.Z.T @ v)) + self.d0 * v

    def Hdiag(self):
        if self.hkind == "dense":
            return np.diag(self.H).copy()
        if self.hkind == "csr_lsq":
            return np.asarray(self.P.multiply(self.P).T @ self.w2).ravel()
        return np.einsum("ij,ij,j->i", self.Z, self.Z, self.zw) + self.d0

    def Hmat(self):
        """Explicit scaled H (dense) for small problems."""
        if self.hkind == "dense":
            return self.H
        if self.hkind == "csr_lsq":
            return np.asarray((self.P.T @ sp.diags(self.w2) @ self.P).todense())
        return (self.Z * self.zw) @ self.Z.T + np.diag(self.d0)

    def Adense(self):
        return self.A.toarray() if sp.issparse(self.A) else np.asarray(self.A)


def _rownorm(M):
    if sp.issparse(M):
        r = np.sqrt(np.asarray(M.multiply(M).sum(axis=1)).ravel())
    else:
        r = np.sqrt(np.einsum("ij,ij->i", M, M)) if M.shape[0] else np.zeros(0)
    r = np.where(r > 0, r, 1.0)
    return r


def rbf_hessian(X, y, gamma):
    """Gaussian-kernel SVM Hessian (Eq. (6) with k(u, v) = exp(-gamma |u - v|^2)):
    H_ij = y_i y_j exp(-gamma sum_k (X_ik - X_jk)^2), the squared distance
    summed difference by difference (y = None: all labels 1)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    H = np.empty((n, n))
    for i0 in range(0, n, 128):
        D = X[i0:i0 + 128, None, :] - X[None, :, :]
        H[i0:i0 + 128] = np.exp(-gamma * np.einsum("ijk,ijk->ij", D, D))
    if y is not None:
        y = np.asarray(y, dtype=np.float64)
        H *= y[:, None] * y[None, :]
    return H


def scale(qp) -> Scaled:
    """Objective scaling by sigma and 2-norm row scaling of A and C."""
    n = qp.n
    if qp.hkind in ("dense", "rbf"):
        # an RBF-kernel H is an explicit dense matrix once formed
        H = qp.H_dense() if qp.hkind == "dense" else rbf_hessian(qp.X, qp.y, qp.gamma)
        hmax = float(np.max(np.diag(H))) if n else 0.0
    elif qp.hkind == "csr_lsq":
        P = qp.P.astype(np.float64)
        hmax = float(np.max(2.0 * (P.multiply(P).T @ qp.w)))
    else:
        Z = qp.Z.astype(np.float64)
        zw = np.ones(Z.shape[1]) if qp.zw is None else np.asarray(qp.zw, float)
        d0 = np.zeros(n) if qp.d0 is None else np.asarray(qp.d0, float)
        hmax = float(np.max(np.einsum("ij,ij,j->i", Z, Z, zw) + d0))
    pinf = float(np.max(np.abs(qp.p))) if n else 0.0
    sigma = 1.0 / max(1.0, hmax, pinf)
    hk = "dense" if qp.hkind == "rbf" else qp.hkind
    S = Scaled(n=n, hkind=hk, sigma=sigma, p=sigma * np.asarray(qp.p, float))
    if hk == "dense":
        S.H = sigma * H
    elif qp.hkind == "csr_lsq":
        S.P = P
        S.w2 = 2.0 * sigma * np.asarray(qp.w, float)
    else:
        S.Z = np.sqrt(sigma) * Z
        S.zw = zw
        S.d0 = sigma * d0
    # general rows
    A = qp.A_matrix()
    if sp.issparse(A):
        A = A.tocsr().astype(np.float64)
    m = A.shape[0]
    rho = 1.0 / _rownorm(A) if m else np.zeros(0)
    S.rhoA = rho
    S.A = (sp.diags(rho) @ A).tocsr() if sp.issparse(A) else A * rho[:, None]
    lA = np.asarray(qp.lA, float) if m else np.zeros(0)
    uA = np.asarray(qp.uA, float) if m else np.zeros(0)
    S.lA, S.uA = lA * rho, uA * rho
    S.L = np.nonzero(np.isfinite(lA))[0]
    S.U = np.nonzero(np.isfinite(uA))[0]
    # equality rows
    if qp.C is not None and qp.C.shape[0]:
        C = np.asarray(qp.C, float)
        rc = 1.0 / _rownorm(C)
        S.C, S.rhoC, S.b = C * rc[:, None], rc, np.asarray(qp.b, float) * rc
    else:
        S.C, S.rhoC, S.b = np.zeros((0, n)), np.zeros(0), np.zeros(0)
    S.lx = np.asarray(qp.lx, float)
    S.ux = np.asarray(qp.ux, float)
    S.Lx = np.nonzero(np.isfinite(S.lx))[0]
    S.Ux = np.nonzero(np.isfinite(S.ux))[0]
    return S


# ---------------------------------------------------------------------------
# Iterate
# ---------------------------------------------------------------------------
@dataclass
class State:
    x: np.ndarray
    s_lA: np.ndarray
    s_uA: np.ndarray
    s_lx: np.ndarray
    s_ux: np.ndarray
    lam_e: np.ndarray
    lam_lA: np.ndarray
    lam_uA: np.ndarray
    lam_lx: np.ndarray
    lam_ux: np.ndarray

    def copy(self):
        return State(*[getattr(self, f).copy() for f in self.__dataclass_fields__])


def initial_point(S: Scaled) -> State:
    n = S.n
    x = np.zeros(n)
    fl, fu = np.isfinite(S.lx), np.isfinite(S.ux)
    both = fl & fu
    x[both] = 0.5 * (S.lx[both] + S.ux[both])
    x[fl & ~fu] = S.lx[fl & ~fu] + 1.0
    x[~fl & fu] = S.ux[~fl & fu] - 1.0
    Ax = S.A @ x
    s_lA = np.maximum(Ax[S.L] - S.lA[S.L], 1.0)
    s_uA = np.maximum(S.uA[S.U] - Ax[S.U], 1.0)
    s_lx = np.maximum(x[S.Lx] - S.lx[S.Lx], 1.0)
    s_ux = np.maximum(S.ux[S.Ux] - x[S.Ux], 1.0)
    return State(x=x, s_lA=s_lA, s_uA=s_uA, s_lx=s_lx, s_ux=s_ux,
                 lam_e=np.zeros(S.me), lam_lA=np.ones(len(S.L)),
                 lam_uA=np.ones(len(S.U)), lam_lx=np.ones(len(S.Lx)),
                 lam_ux=np.ones(len(S.Ux)))


# ---------------------------------------------------------------------------
# Residuals, Eq. (3) with the bound blocks of Eq. (7)
# ---------------------------------------------------------------------------
def _ATy(S: Scaled, yL, yU):
    """A_L' yL - A_U' yU  (general-row multipliers mapped to x-space)."""
    y = np.zeros(S.m)
    y[S.L] += yL
    y[S.U] -= yU
    return S.A.T @ y


def residuals(S: Scaled, st: State, mu: float) -> dict:
    x = st.x
    Ax = S.A @ x
    g = S.Hv(x) + S.p - _ATy(S, st.lam_lA, st.lam_uA) - S.C.T @ st.lam_e
    g[S.Lx] -= st.lam_lx
    g[S.Ux] += st.lam_ux
    return {
        "r_H": g,
        "r_e": S.C @ x - S.b + mu * st.lam_e,
        "r_lA": Ax[S.L] - st.s_lA - S.lA[S.L],
        "r_uA": -Ax[S.U] - st.s_uA + S.uA[S.U],
        "r_lx": x[S.Lx] - st.s_lx - S.lx[S.Lx],
        "r_ux": -x[S.Ux] - st.s_ux + S.ux[S.Ux],
        "r_c1": st.lam_lA * st.s_lA - mu,
        "r_c2": st.lam_uA * st.s_uA - mu,
        "r_c3": st.lam_lx * st.s_lx - mu,
        "r_c4": st.lam_ux * st.s_ux - mu,
    }


RES_KEYS = ("r_H", "r_e", "r_lA", "r_uA", "r_lx", "r_ux", "r_c1", "r_c2", "r_c3", "r_c4")


def residual_norm(r: dict) -> float:
    """2-norm of the whole right-hand side of Eq. (7)."""
    return float(np.sqrt(sum(float(r[k] @ r[k]) for k in RES_KEYS)))


def infeasibilities(r: dict):
    """Primal, dual and complementarity infeasibility of section 5.2.  The
    equality residual r_e counts as primal, so the three norms split the
    residual norm of Eq. (7) exactly: prim^2 + dual^2 + comp^2 = ||r||^2."""
    prim = np.sqrt(sum(float(r[k] @ r[k]) for k in ("r_e", "r_lA", "r_uA", "r_lx", "r_ux")))
    dual = float(np.linalg.norm(r["r_H"]))
    comp = np.sqrt(sum(float(r[k] @ r[k]) for k in ("r_c1", "r_c2", "r_c3", "r_c4")))
    return prim, dual, comp


# ---------------------------------------------------------------------------
# Reduced 2x2 system, Eq. (8)
# ---------------------------------------------------------------------------
def reduced_system(S: Scaled, st: State, r: dict, mu: float):
    """Returns (dg, D, r1, r2): Q = H + diag(dg), D as a vector."""
    n = S.n
    dg = np.zeros(n)
    dg[S.Lx] += st.lam_lx / st.s_lx
    dg[S.Ux] += st.lam_ux / st.s_ux
    D = np.concatenate([np.full(S.me, mu), st.s_lA / st.lam_lA, st.s_uA / st.lam_uA])
    r1 = -r["r_H"].copy()
    r1[S.Lx] += -r["r_c3"] / st.s_lx - st.lam_lx / st.s_lx * r["r_lx"]
    r1[S.Ux] += r["r_c4"] / st.s_ux + st.lam_ux / st.s_ux * r["r_ux"]
    r2 = np.concatenate([-r["r_e"],
                         -r["r_lA"] - r["r_c1"] / st.lam_lA,
                         -r["r_uA"] - r["r_c2"] / st.lam_uA])
    return dg, D, r1, r2


def B_matrix(S: Scaled):
    """B = [C; A_L; -A_U] as a dense array (small problems only)."""
    Ad = S.Adense()
    return np.vstack([S.C, Ad[S.L], -Ad[S.U]])


def B_apply(S: Scaled, v):
    Av = S.A @ v
    return np.concatenate([S.C @ v, Av[S.L], -Av[S.U]])


def BT_apply(S: Scaled, y):
    me, nl = S.me, len(S.L)
    return S.C.T @ y[:me] + _ATy(S, y[me:me + nl], y[me + nl:])


def doubly_augmented_matrix(S: Scaled, dg, D):
    """Explicit K of Eq. (9): [Q + 2B'D^-1B, B'; B, D] (small problems)."""
    B = B_matrix(S)
    Q = S.Hmat() + np.diag(dg)
    top = Q + 2.0 * B.T @ (B / D[:, None])
    return np.block([[top, B.T], [B, np.diag(D)]])


def doubly_augmented_rhs(S: Scaled, D, r1, r2):
    return np.concatenate([r1 + 2.0 * BT_apply(S, r2 / D), r2])


def kkt_apply(S: Scaled, dg, D, v):
    """K v for the K of Eq. (9), matrix-free from H, B, B' and D."""
    n = S.n
    vx, vl = v[:n], v[n:]
    t = B_apply(S, vx)
    top = S.Hv(vx) + dg * vx + BT_apply(S, 2.0 * t / D + vl)
    return np.concatenate([top, t + D * vl])


def jacobi_diagonal(S: Scaled, dg, D):
    """diag(K) of Eq. (9): diag(H) + dg + 2 diag(B'D^-1B), then D."""
    me, nl = S.me, len(S.L)
    wrow = np.zeros(S.m)
    wrow[S.L] += 1.0 / D[me:me + nl]
    wrow[S.U] += 1.0 / D[me + nl:]
    if sp.issparse(S.A):
        a2 = S.A.multiply(S.A).T @ wrow
    else:
        a2 = (S.A * S.A).T @ wrow
    c2 = (S.C * S.C).T @ (1.0 / D[:me])
    dx = S.Hdiag() + dg + 2.0 * (np.asarray(a2).ravel() + c2)
    return np.concatenate([dx, D])


def jacobi_scaled_eigenvalues(K):
    """Eigenvalues (ascending) of diag(K)^-1/2 K diag(K)^-1/2: the operator
    Jacobi-preconditioned CG works with, whose condition number section 5.3
    reports next to that of K itself."""
    d = 1.0 / np.sqrt(np.diag(K))
    return np.linalg.eigvalsh(K * d[:, None] * d[None, :])


def full_newton_matrix(S: Scaled, st: State, mu: float):
    """Explicit Eq. (7) in the unknown order (dx, dlam_lA, dlam_uA, dlam_lx,
    dlam_ux, dlam_e, ds_lA, ds_uA, ds_lx, ds_ux) with the -C' reading; the
    right-hand side is -(r_H, r_e, r_lA, r_uA, r_lx, r_ux, r_c1..r_c4)."""
    n = S.n
    Ad = S.Adense()
    AL, AU = Ad[S.L], Ad[S.U]
    Ex_l = np.eye(n)[S.Lx]
    Ex_u = np.eye(n)[S.Ux]
    sizes = [n, len(S.L), len(S.U), len(S.Lx), len(S.Ux), S.me,
             len(S.L), len(S.U), len(S.Lx), len(S.Ux)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    N = off[-1]
    J = np.zeros((N, N))

    def put(bi, bj, M):
        J[off[bi]:off[bi + 1], off[bj]:off[bj + 1]] = M

    put(0, 0, S.Hmat())
    put(0, 1, -AL.T)
    put(0, 2, AU.T)
    put(0, 3, -Ex_l.T)
    put(0, 4, Ex_u.T)
    put(0, 5, -S.C.T)
    # r_e row
    put(5, 0, S.C)
    put(5, 5, mu * np.eye(S.me))
    # constraint rows (row block order in J follows the unknown order)
    put(1, 0, AL)
    put(1, 6, -np.eye(len(S.L)))
    put(2, 0, -AU)
    put(2, 7, -np.eye(len(S.U)))
    put(3, 0, Ex_l)
    put(3, 8, -np.eye(len(S.Lx)))
    put(4, 0, -Ex_u)
    put(4, 9, -np.eye(len(S.Ux)))
    # complementarity rows
    put(6, 1, np.diag(st.s_lA))
    put(6, 6, np.diag(st.lam_lA))
    put(7, 2, np.diag(st.s_uA))
    put(7, 7, np.diag(st.lam_uA))
    put(8, 3, np.diag(st.s_lx))
    put(8, 8, np.diag(st.lam_lx))
    put(9, 4, np.diag(st.s_ux))
    put(9, 9, np.diag(st.lam_ux))
    return J, off


def full_newton_rhs(r):
    return -np.concatenate([r["r_H"], r["r_lA"], r["r_uA"], r["r_lx"], r["r_ux"],
                            r["r_e"], r["r_c1"], r["r_c2"], r["r_c3"], r["r_c4"]])


# ---------------------------------------------------------------------------
# Direct Newton solve of Eq. (8)
# ---------------------------------------------------------------------------
def _banded_upper(M: sp.spmatrix, u: int):
    """Upper banded storage ab[u + i - j, j] = M[i, j] for j >= i."""
    Mc = sp.triu(M).tocoo()
    ab = np.zeros((u + 1, M.shape[0]))
    ab[u + Mc.row - Mc.col, Mc.col] = Mc.data
    return ab


def newton_direct(S: Scaled, dg, D, r1, r2, solver: str = "auto"):
    """Solve [Q -B'; B D][dx; dlam] = [r1; r2] directly.

    * ``ldl``:  the symmetric quasi-definite form [Q B'; B -D][dx; -dlam] =
      [r1; r2] with LAPACK's Bunch-Kaufman LDL^T (dense).
    * ``schur``: exact block elimination dlam = D^-1 (r2 - B dx) and the SPD
      system (Q + B'D^-1B) dx = r1 + B'D^-1 r2, by Cholesky: dense, banded
      (LAPACK pbsv) for the csr_lsq structure, or Woodbury on the capacitance
      matrix for the low-rank structure.
    """
    n = S.n
    NK = S.NK
    if solver == "auto":
        if NK <= 3000:
            solver = "ldl"
        elif S.hkind == "csr_lsq":
            solver = "schur_banded"
        elif S.hkind == "lowrank":
            solver = "schur_woodbury"
        else:
            solver = "schur_dense"
    if solver == "ldl":
        B = B_matrix(S)
        Q = S.Hmat() + np.diag(dg)
        M = np.block([[Q, B.T], [B, -np.diag(D)]])
        sol = sla.solve(M, np.concatenate([r1, r2]), assume_a="sym")
        return sol[:n], -sol[n:]
    rhs = r1 + BT_apply(S, r2 / D)
    if solver == "schur_dense":
        B = B_matrix(S)
        Smat = S.Hmat() + np.diag(dg) + B.T @ (B / D[:, None])
        c = sla.cho_factor(Smat, lower=False)
        dx = sla.cho_solve(c, rhs)
    elif solver == "schur_banded":
        me, nl = S.me, len(S.L)
        wrow = np.zeros(S.m)
        wrow[S.L] += 1.0 / D[me:me + nl]
        wrow[S.U] += 1.0 / D[me + nl:]
        if S._hband is None:
            Hs = (S.P.T @ sp.diags(S.w2) @ S.P).tocsr()
            S._hband = Hs
        Msp = S._hband + sp.diags(dg) + (S.A.T @ sp.diags(wrow) @ S.A)
        if me:
            Msp = Msp + sp.csr_matrix(S.C.T @ (S.C / D[:me, None]))
        Mc = Msp.tocoo()
        u = int(np.max(np.abs(Mc.row - Mc.col))) if Mc.nnz else 0
        if 4 * u > n:
            # wide band: plain dense Cholesky of the same Schur complement
            dx = sla.cho_solve(sla.cho_factor(Msp.toarray(), lower=False), rhs)
        else:
            ab = _banded_upper(Msp, u)
            dx = sla.solveh_banded(ab, rhs, lower=False)
    elif solver == "schur_woodbury":
        # Q + B'D^-1B = diag(dg + H0) + Z W Z' + B' D^-1 B with B = [C; A_L;
        # -A_U]: a diagonal plus U U', U = [Z W^1/2, (D^-1/2 B)'] (positive
        # weights W); capacitance matrix of size k + rows of B
        assert S.hkind == "lowrank" and np.all(S.zw > 0)
        B = B_matrix(S)
        U = np.hstack([S.Z * np.sqrt(S.zw), (B / np.sqrt(D)[:, None]).T])
        Dinv = 1.0 / (dg + S.d0)
        cap = np.eye(U.shape[1]) + U.T @ (U * Dinv[:, None])
        t = U.T @ (Dinv * rhs)
        dx = Dinv * rhs - Dinv * (U @ sla.solve(cap, t, assume_a="pos"))
    else:
        raise ValueError(solver)
    dlam = (r2 - B_apply(S, dx)) / D
    return dx, dlam


# ---------------------------------------------------------------------------
# Reference Jacobi PCG on Eq. (9) (textbook algorithm, float64)
# ---------------------------------------------------------------------------
def pcg_reference(Kmv, rhs, diag, tol=1e-7, maxit=5000):
    """Jacobi-preconditioned CG from z0 = 0; stops when the recursively
    updated residual satisfies ||r|| <= tol ||rhs||.  Returns (z, iters,
    true relative residual)."""
    z = np.zeros_like(rhs)
    r = rhs.copy()
    bn = float(np.linalg.norm(rhs))
    if bn == 0.0:
        return z, 0, 0.0
    y = r / diag
    p = y.copy()
    rho = float(r @ y)
    it = 0
    while it < maxit and float(np.linalg.norm(r)) > tol * bn:
        q = Kmv(p)
        alpha = rho / float(p @ q)
        z += alpha * p
        r -= alpha * q
        y = r / diag
        rho_new = float(r @ y)
        p = y + (rho_new / rho) * p
        rho = rho_new
        it += 1
    true = float(np.linalg.norm(rhs - Kmv(z))) / bn
    return z, it, true


# ---------------------------------------------------------------------------
# Step recovery and ratio test
# ---------------------------------------------------------------------------
def recover_step(S: Scaled, st: State, r: dict, dx, dlam):
    """Slack and bound-multiplier directions from the linearised Eq. (3)."""
    me, nl = S.me, len(S.L)
    Adx = S.A @ dx
    d = {
        "x": dx,
        "lam_e": dlam[:me],
        "lam_lA": dlam[me:me + nl],
        "lam_uA": dlam[me + nl:],
        "s_lA": Adx[S.L] + r["r_lA"],
        "s_uA": -Adx[S.U] + r["r_uA"],
        "s_lx": dx[S.Lx] + r["r_lx"],
        "s_ux": -dx[S.Ux] + r["r_ux"],
    }
    d["lam_lx"] = -(r["r_c3"] + st.lam_lx * d["s_lx"]) / st.s_lx
    d["lam_ux"] = -(r["r_c4"] + st.lam_ux * d["s_ux"]) / st.s_ux
    return d


def _max_step(v, dv):
    neg = dv < 0
    if not np.any(neg):
        return np.inf
    return float(np.min(-v[neg] / dv[neg]))


def ratio_test(st: State, d: dict, gamma: float = 0.99):
    """Eq. (10)."""
    sx = min(_max_step(getattr(st, k), d[k]) for k in ("s_lA", "s_uA", "s_lx", "s_ux"))
    sl = min(_max_step(getattr(st, k), d[k]) for k in ("lam_lA", "lam_uA", "lam_lx", "lam_ux"))
    return min(1.0, gamma * sx), min(1.0, gamma * sl)


def apply_step(st: State, d: dict, ax: float, al: float) -> State:
    out = st.copy()
    out.x += ax * d["x"]
    for k in ("s_lA", "s_uA", "s_lx", "s_ux"):
        setattr(out, k, getattr(out, k) + ax * d[k])
    for k in ("lam_e", "lam_lA", "lam_uA", "lam_lx", "lam_ux"):
        setattr(out, k, getattr(out, k) + al * d[k])
    return out


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------
@dataclass
class IpmResult:
    status: str
    iters: int
    mu: float
    x: np.ndarray
    lam: dict
    s: dict
    state: State
    scaled: Scaled
    log: list


def ipm_iterate(qp, gamma=0.99, mu_tol=1e-6, maxit=200, solver="auto",
                pcg_tol=1e-7, pcg_maxit=5000, max_iters=None, log=False):
    """Algorithm 1 as a generator: yields a dict after every IPM iteration
    (its number, mu, ||r||, step lengths, and the iterate so far); the last
    dict carries the final result under "result".  ipm_solve consumes it."""
    S = scale(qp)
    st = initial_point(S)
    k = 0                       # mu = 10^-k
    mu = 1.0
    hist = []
    status = "maxit"
    it = 0
    r = residuals(S, st, mu)
    limit = maxit if max_iters is None else min(maxit, max_iters)
    for it in range(1, limit + 1):
        dg, D, r1, r2 = reduced_system(S, st, r, mu)
        info = {}
        if solver == "pcg":
            rhs = doubly_augmented_rhs(S, D, r1, r2)
            diag = jacobi_diagonal(S, dg, D)
            z, nit, tres = pcg_reference(lambda v: kkt_apply(S, dg, D, v), rhs, diag,
                                         pcg_tol, pcg_maxit)
            dx, dlam = z[:S.n], z[S.n:]
            info = {"pcg_iters": nit, "pcg_res": tres}
        else:
            dx, dlam = newton_direct(S, dg, D, r1, r2, solver)
        d = recover_step(S, st, r, dx, dlam)
        ax, al = ratio_test(st, d, gamma)
        st = apply_step(st, d, ax, al)
        r = residuals(S, st, mu)
        rn = residual_norm(r)
        if log:
            pr, du, co = infeasibilities(r)
            hist.append(dict(it=it, mu=mu, res=rn, alpha_x=ax, alpha_lam=al,
                             primal=pr, dual=du, compl=co, **info))
        step = {"it": it, "mu": mu, "res": rn, "alpha_x": ax, "alpha_lam": al}
        done = False
        if rn < mu:
            if mu < mu_tol:
                status = "converged"
                done = True
            else:
                k += 1
                mu = 10.0 ** (-k)
                r = residuals(S, st, mu)
        if done or it == limit:
            x, lam, s = unscale_solution(S, st)
            step["result"] = IpmResult(status=status, iters=it, mu=mu, x=x, lam=lam, s=s,
                                       state=st, scaled=S, log=hist)
            yield step
            return
        yield step
    x, lam, s = unscale_solution(S, st)
    yield {"it": it, "mu": mu, "result": IpmResult(status=status, iters=it, mu=mu, x=x, lam=lam,
                                                   s=s, state=st, scaled=S, log=hist)}


def ipm_solve(qp, gamma=0.99, mu_tol=1e-6, maxit=200, solver="auto",
              pcg_tol=1e-7, pcg_maxit=5000, max_iters=None, log=False) -> IpmResult:
    """Algorithm 1 with a direct (default) or reference-PCG Newton solve."""
    last = None
    for last in ipm_iterate(qp, gamma, mu_tol, maxit, solver, pcg_tol, pcg_maxit, max_iters, log):
        pass
    return last["result"]


def unscale_solution(S: Scaled, st: State):
    """Map multipliers and slacks of the scaled problem to original units."""
    sg = S.sigma
    lam = {
        "lA": st.lam_lA * S.rhoA[S.L] / sg,
        "uA": st.lam_uA * S.rhoA[S.U] / sg,
        "lx": st.lam_lx / sg,
        "ux": st.lam_ux / sg,
        "e": st.lam_e * S.rhoC / sg,
    }
    s = {"lA": st.s_lA / S.rhoA[S.L], "uA": st.s_uA / S.rhoA[S.U],
         "lx": st.s_lx.copy(), "ux": st.s_ux.copy()}
    return st.x.copy(), lam, s


# ---------------------------------------------------------------------------
# Adjoint: d(g'x*)/d(p, lA, uA, b) at the converged iterate
# ---------------------------------------------------------------------------
def adjoint_solve(S: Scaled, st: State, mu: float, gbar, solver="auto"):
    """One solve with the converged Newton matrix.

    Differentiating the mu-fixed perturbed KKT conditions (Eq. (3)) gives the
    2x2 system of Eq. (8) with right-hand side [-dp; (db, dlA, -duA)].  For a
    loss with gradient gbar = dL/dx the transposed system is equivalent to
    K [v; w] = [gbar; 0] with the K of Eq. (9), so that

        dL/dp = -v,   dL/d(b, lA) = -w_(e, lA),   dL/duA = +w_(uA)

    in scaled units.  Returned in original units (chain rule through the
    sigma and row scalings).  Inactive (infinite) bounds get 0.
    """
    n = S.n
    r = residuals(S, st, mu)
    dg, D, _, _ = reduced_system(S, st, r, mu)
    # K [v; w] = [gbar; 0]  <=>  (Q + B'D^-1B) v = gbar,  w = -D^-1 B v
    rhs1 = np.asarray(gbar, float)
    zero2 = np.zeros(len(D))
    v, lam_neg = newton_direct(S, dg, D, rhs1, zero2, solver)
    # newton_direct solves [Q -B'; B D][a; c] = [gbar; 0]: a = v, c = -D^-1 B v = w
    w = lam_neg
    me, nl = S.me, len(S.L)
    g_p = -v * S.sigma
    g_lA = np.zeros(S.m)
    g_uA = np.zeros(S.m)
    g_lA[S.L] = -w[me:me + nl] * S.rhoA[S.L]
    g_uA[S.U] = w[me + nl:] * S.rhoA[S.U]
    g_b = -w[:me] * S.rhoC
    return {"p": g_p, "lA": g_lA, "uA": g_uA, "b": g_b, "v": v, "w": w}
