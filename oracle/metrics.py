"""Acceptance metrics in original units (TEST INFRASTRUCTURE ONLY).

The paper measures convergence by the primal, dual and complementarity
infeasibilities of section 5.2 (2-norms of the constraint residuals, of r_H and
of the complementarity residuals).  Those are unnormalised and depend on the
internal scaling; the checks here use the following size-independent reading,
evaluated in float64 from the original problem data and a candidate solution
(x, multipliers):

* primal_rel = max over constraints of the violation divided by the row's
  2-norm (distance to the violated hyperplane), over (1 + ||x||_inf);
* dual_rel   = ||H x + p - A'(lam_lA - lam_uA) - (lam_lx - lam_ux) - C' lam_e||_inf
               over 1 + max(||Hx||_inf, ||p||_inf, ||A'(lam_lA - lam_uA)||_inf,
               ||lam_lx - lam_ux||_inf, ||C' lam_e||_inf);
* compl_rel  = max_i |lam_i * shat_i| / ((1 + ||x||_inf) * G), shat the slack
               recomputed from x and G the dual normaliser above: the product
               of a multiplier relative to the gradient scale and a slack
               relative to the primal scale, so it is invariant to scaling the
               objective or the rows;
* gap        = sum of lam_i * shat_i + lam_e'(Cx - b): the primal-dual gap
               f(x) - g(lam) at a dual-feasible point (g the Lagrangian dual
               function); gap_rel = |gap| / (1 + |f|);
* kkt_rel    = max(primal_rel, dual_rel): the residuals the acceptance gate
               (1e-6) applies to.  Complementarity is set by the final barrier
               parameter through the method's internal scaling (lam*s = mu in
               scaled units), so it is reported, and compared between two
               solvers that follow the same mu path, but not gated.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def objective(qp, x):
    return qp.objective(np.asarray(x, float))


def _Hx(qp, x):
    if qp.hkind == "dense":
        return qp.H_dense() @ x
    if qp.hkind == "rbf":
        from .ipm import rbf_hessian
        return rbf_hessian(qp.X, qp.y, qp.gamma) @ x
    if qp.hkind == "csr_lsq":
        P = qp.P.astype(np.float64)
        return 2.0 * (P.T @ (qp.w * (P @ x)))
    Z = qp.Z.astype(np.float64)
    zw = np.ones(Z.shape[1]) if qp.zw is None else np.asarray(qp.zw, float)
    d0 = np.zeros(qp.n) if qp.d0 is None else np.asarray(qp.d0, float)
    return Z @ (zw * (Z.T @ x)) + d0 * x


def kkt_metrics(qp, x, lam_lA, lam_uA, lam_lx, lam_ux, lam_e):
    """lam_lA / lam_uA are length-m arrays (0 on rows without that bound),
    lam_lx / lam_ux length n (0 where unbounded), lam_e length me."""
    x = np.asarray(x, float)
    n = qp.n
    A = qp.A_matrix()
    m = A.shape[0]
    Ax = A @ x if m else np.zeros(0)
    if sp.issparse(A):
        rn = np.sqrt(np.asarray(A.multiply(A).sum(axis=1)).ravel())
    else:
        rn = np.sqrt(np.einsum("ij,ij->i", A, A)) if m else np.zeros(0)
    rn = np.where(rn > 0, rn, 1.0)
    viol = [0.0]
    if m:
        lA = np.asarray(qp.lA, float)
        uA = np.asarray(qp.uA, float)
        with np.errstate(invalid="ignore"):
            v = np.maximum(np.where(np.isfinite(lA), lA - Ax, 0.0),
                           np.where(np.isfinite(uA), Ax - uA, 0.0))
        viol.append(float(np.max(np.maximum(v, 0.0) / rn)))
    me = 0 if qp.C is None else qp.C.shape[0]
    if me:
        C = np.asarray(qp.C, float)
        cn = np.sqrt(np.einsum("ij,ij->i", C, C))
        viol.append(float(np.max(np.abs(C @ x - qp.b) / np.where(cn > 0, cn, 1.0))))
    lx, ux = np.asarray(qp.lx, float), np.asarray(qp.ux, float)
    with np.errstate(invalid="ignore"):
        vb = np.maximum(np.where(np.isfinite(lx), lx - x, 0.0),
                        np.where(np.isfinite(ux), x - ux, 0.0))
    viol.append(float(np.max(np.maximum(vb, 0.0))) if n else 0.0)
    primal = max(viol) / (1.0 + float(np.max(np.abs(x))))

    Hx = _Hx(qp, x)
    lam_A = np.asarray(lam_lA, float) - np.asarray(lam_uA, float) if m else np.zeros(0)
    ATl = A.T @ lam_A if m else np.zeros(n)
    ATl = np.asarray(ATl).ravel()
    lxx = np.asarray(lam_lx, float) - np.asarray(lam_ux, float)
    CTl = np.asarray(qp.C, float).T @ np.asarray(lam_e, float) if me else np.zeros(n)
    rH = Hx + qp.p - ATl - lxx - CTl
    scale = 1.0 + max(float(np.max(np.abs(Hx))), float(np.max(np.abs(qp.p))),
                      float(np.max(np.abs(ATl))) if m else 0.0,
                      float(np.max(np.abs(lxx))), float(np.max(np.abs(CTl))) if me else 0.0)
    dual = float(np.max(np.abs(rH))) / scale

    f = float(0.5 * x @ Hx + qp.p @ x)
    fscale = max(abs(0.5 * float(x @ Hx)), abs(float(qp.p @ x)))
    comp = [0.0]
    if m:
        with np.errstate(invalid="ignore"):
            sl = np.where(np.isfinite(lA), Ax - lA, 0.0)
            su = np.where(np.isfinite(uA), uA - Ax, 0.0)
        comp.append(float(np.max(np.abs(np.asarray(lam_lA) * sl))))
        comp.append(float(np.max(np.abs(np.asarray(lam_uA) * su))))
    with np.errstate(invalid="ignore"):
        slx = np.where(np.isfinite(lx), x - lx, 0.0)
        sux = np.where(np.isfinite(ux), ux - x, 0.0)
    comp.append(float(np.max(np.abs(np.asarray(lam_lx) * slx))))
    comp.append(float(np.max(np.abs(np.asarray(lam_ux) * sux))))
    compl = max(comp) / ((1.0 + float(np.max(np.abs(x)))) * scale)
    # duality gap: sum of multiplier x slack over every inequality (shat from x)
    # plus lam_e'(Cx - b); equals f(x) - g(lam) + x'r_H, g the Lagrangian dual
    # function, so at a dual-feasible point (r_H = 0) it is the primal-dual gap
    gap = 0.0
    if m:
        gap += float(np.sum(np.asarray(lam_lA) * sl) + np.sum(np.asarray(lam_uA) * su))
    gap += float(np.sum(np.asarray(lam_lx) * slx) + np.sum(np.asarray(lam_ux) * sux))
    if me:
        gap += float(np.asarray(lam_e, float) @ (C @ x - qp.b))
    return {"primal_rel": primal, "dual_rel": dual, "compl_rel": compl,
            "kkt_rel": max(primal, dual), "dual_scale": scale, "objective": f, "gap": gap,
            "gap_rel": abs(gap) / (1.0 + abs(f))}


def full_multipliers(res_or_S, lam: dict, qp):
    """Expand the oracle's compact multipliers to full-length arrays."""
    S = res_or_S
    m, n = qp.m, qp.n
    lA = np.zeros(m)
    uA = np.zeros(m)
    lx = np.zeros(n)
    ux = np.zeros(n)
    lA[S.L] = lam["lA"]
    uA[S.U] = lam["uA"]
    lx[S.Lx] = lam["lx"]
    ux[S.Ux] = lam["ux"]
    return lA, uA, lx, ux, lam["e"]
