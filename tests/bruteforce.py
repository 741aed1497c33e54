"""Brute-force active-set enumeration for tiny strictly convex QPs.

Independent of the oracle: enumerates every assignment of each inequality
(general row or variable bound) to {inactive, at lower, at upper}, solves the
resulting equality-constrained QP with its KKT matrix, and keeps the unique
assignment whose point is feasible and whose multipliers have the right sign
(Nocedal & Wright, Thm. 16.4 / 12.1: for strictly convex QPs the KKT point is
the unique minimiser).
"""
import itertools

import numpy as np


def solve_bruteforce(H, p, A=None, lA=None, uA=None, C=None, b=None, lx=None, ux=None,
                     tol=1e-9):
    n = len(p)
    rows = []   # (vector, lower, upper)
    if A is not None:
        for i in range(A.shape[0]):
            rows.append((A[i], lA[i], uA[i]))
    if lx is not None:
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            rows.append((e, lx[j], ux[j]))
    me = 0 if C is None else C.shape[0]
    choices = []
    for (_, lo, hi) in rows:
        c = [0]
        if np.isfinite(lo):
            c.append(1)
        if np.isfinite(hi):
            c.append(2)
        choices.append(c)
    best = None
    for assign in itertools.product(*choices):
        E, e, sgn = [], [], []
        for (a, lo, hi), s in zip(rows, assign):
            if s == 1:
                E.append(a), e.append(lo), sgn.append(1.0)
            elif s == 2:
                E.append(a), e.append(hi), sgn.append(-1.0)
        k = len(E)
        if k + me > n:
            continue
        G = np.array(E).reshape(k, n)
        if me:
            G = np.vstack([G, C])
            rhs_c = np.concatenate([np.array(e), b])
        else:
            rhs_c = np.array(e)
        K = np.block([[H, -G.T], [G, np.zeros((k + me, k + me))]])
        try:
            sol = np.linalg.solve(K, np.concatenate([-p, rhs_c]))
        except np.linalg.LinAlgError:
            continue
        x, nu = sol[:n], sol[n:]
        # multipliers: Hx + p = sum nu_i g_i  with g = +a (lower), -a (upper)
        # here nu is the multiplier of +a for both; sign-correct it.
        nu_ineq = nu[:k] * np.array(sgn) if k else np.zeros(0)
        if np.any(nu_ineq < -tol):
            continue
        ok = True
        for (a, lo, hi) in rows:
            v = a @ x
            if (np.isfinite(lo) and v < lo - 1e-9) or (np.isfinite(hi) and v > hi + 1e-9):
                ok = False
                break
        if not ok:
            continue
        f = 0.5 * x @ H @ x + p @ x
        if best is None or f < best[1] - 1e-12:
            best = (x, f)
    return best
