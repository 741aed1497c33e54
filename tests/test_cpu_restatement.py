"""The CPU restatement of the paper's Newton-step design (FP64, OpenMP,
matrix-free Eq. (9) and Jacobi-PCG) against the oracle: K v on a small dose
QP at a random interior iterate, and its PCG solution against the oracle's
direct Newton solve (no GPU)."""
import numpy as np
import pytest

import qpgen
from oracle import ipm as I

cr = pytest.importorskip("cpu_restatement")


def _system(seed=0):
    qp = qpgen.dose_qp(3000, 300, 30, 40, 150, seed=8)
    S = I.scale(qp)
    st = I.initial_point(S)
    rng = np.random.default_rng(seed)
    for k in ("s_lA", "s_uA", "s_lx", "lam_lA", "lam_uA", "lam_lx"):
        v = getattr(st, k)
        setattr(st, k, np.exp(rng.uniform(-2, 1, len(v))))
    st.x = rng.uniform(0.1, 1.0, S.n)
    r = I.residuals(S, st, 0.1)
    dg, D, r1, r2 = I.reduced_system(S, st, r, 0.1)
    sysc = cr.System(S.P, S.w2, S.A, S.L, S.U, dg, D)
    return S, dg, D, r1, r2, sysc


def test_apply_matches_oracle():
    S, dg, D, r1, r2, sysc = _system()
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.standard_normal(sysc.N)
        ref = I.kkt_apply(S, dg, D, v)
        got = sysc.apply(v)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_pcg_matches_direct_solve():
    S, dg, D, r1, r2, sysc = _system(2)
    rhs = I.doubly_augmented_rhs(S, D, r1, r2)
    diag = I.jacobi_diagonal(S, dg, D)
    sol, it, rel = sysc.pcg(diag, rhs, tol=1e-10, maxit=20000)
    assert rel <= 1e-10 and 0 < it < 20000
    res = rhs - I.kkt_apply(S, dg, D, sol)
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(rhs)
    dx, dl = I.newton_direct(S, dg, D, r1, r2)
    assert np.max(np.abs(sol[:S.n] - dx)) <= 1e-6 * (1 + np.max(np.abs(dx)))
    # tol = 0 runs exactly maxit iterations (the benchmark's fixed sample)
    _, it0, _ = sysc.pcg(diag, rhs, tol=0.0, maxit=7)
    assert it0 == 7
