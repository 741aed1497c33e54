"""GPU parity: every step of the CUDA path against the FP64 CPU oracle on the
same seeded inputs, through the C ABI.

Tolerances (derivation): the FP64 path evaluates the same sums as the oracle
in a different order, so single products agree to a few ulps of the largest
term, well below 1e-11 relative; the mixed path rounds the matrix-vector
product to FP32 (unit roundoff 6e-8) over at most a few hundred terms per
entry, so 1e-5 relative is a safe bound.  Solves are compared through their
FP64 residuals (a property that holds at any size) and, where the system is
well conditioned, against the direct solution.  IPM results use the gate of
the acceptance metrics: objective within 1e-6 relative and KKT_rel <= 1e-6.
"""
import numpy as np
import pytest

import oracle
import qpgen
from oracle import ipm as I
from tests.gpu_helpers import (from_padded, kkt_abs_apply, random_state, relerr, set_gpu_state,
                               to_padded)

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "dense_eq": lambda: qpgen.tiny_qp(37, 23, 5, me=2),
    "dense_onesided": lambda: qpgen.dense_qp(70, 45, seed=3),
    "csr": lambda: qpgen.dose_qp(3000, 300, 30, 40, 150, seed=8),
    "csr_multichunk": lambda: qpgen.dose_qp(60000, 3000, 100, 300, 3000, seed=10,
                                            unit_dose=True),
    "csr_irregular": lambda: qpgen.irregular_lsq_qp(),
    # rows of 0..128 nonzeros (empty rows, the longest rows of the
    # register-streamed operator, lengths that need padding), scattered columns
    "csr_short_irregular": lambda: qpgen.irregular_lsq_qp(max_len=128, long_rows=0, seed=13),
    "lowrank": lambda: qpgen.svm_qp(500, 16, seed=9),
    # general sparse A (CSR) and equality rows with every H structure (Eq. (1))
    "dense_csrA_eq": lambda: qpgen.dense_qp_general(),
    "csr_csrA_eq": lambda: qpgen.dose_qp_general(),
    "lowrank_csrA_eq": lambda: qpgen.svm_qp_general(),
    # quasi-Newton Hessian H0 + U W U' (section 2.1) with sparse dose-like rows
    "lowrank_bfgs": lambda: qpgen.bfgs_qp(800, 10, 60, 15, seed=43),
    # Gaussian-kernel SVM dual (Eq. (6)): H formed on the device from X, y, gamma
    # (n = 500 is not a multiple of the 32 x 32 build tile; d = 37 spans two
    # 32-feature slabs)
    "rbf_svm": lambda: qpgen.rbf_svm_qp(500, 37, seed=52),
    # bf16 H and f32 A (the batched QPs' storage): FP64 products in
    # double-float arithmetic; n = 700 >= 512 takes the column pass for A'
    "dense_bf16": lambda: qpgen.batch_qp(3, 300),
    "dense_bf16_colpass": lambda: qpgen.batch_qp(5, 700),
}


@pytest.fixture(scope="module")
def kq():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as m
    m.load()
    return m


def _setup(kq, name, seed=0, mu=0.01):
    qp = PROBLEMS[name]()
    S = I.scale(qp)
    st = random_state(S, seed)
    h = kq.create_from(qp)
    set_gpu_state(kq, h, S, st, mu)
    return qp, S, st, h


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_scaling_matches(kq, name):
    qp = PROBLEMS[name]()
    S = I.scale(qp)
    h = kq.create_from(qp)
    sigma, rhoA, rhoC = kq.qp_scaling(h)
    assert sigma == pytest.approx(S.sigma, rel=1e-13)
    assert relerr(rhoA, S.rhoA) <= 1e-13
    assert relerr(rhoC, S.rhoC) <= 1e-13


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_residuals_rhs_diag(kq, name):
    qp, S, st, h = _setup(kq, name)
    mu = 0.01
    n, m, me = S.n, S.m, S.me
    bufs = {k: np.zeros(n) for k in ("r_H", "r_lx", "r_ux", "r_c3", "r_c4")}
    bufs.update({k: np.zeros(m) for k in ("r_lA", "r_uA", "r_c1", "r_c2")})
    bufs["r_e"] = np.zeros(me)
    bufs["rhs"] = np.zeros(n + me + 2 * m)
    norm = kq.qp_residuals(h, **bufs)
    r = I.residuals(S, st, mu)
    assert relerr(bufs["r_H"], r["r_H"]) <= 1e-11
    assert relerr(bufs["r_lA"][S.L], r["r_lA"]) <= 1e-11
    assert relerr(bufs["r_uA"][S.U], r["r_uA"]) <= 1e-11
    assert relerr(bufs["r_c1"][S.L], r["r_c1"]) <= 1e-11
    assert relerr(bufs["r_lx"][S.Lx], r["r_lx"]) <= 1e-11
    assert relerr(bufs["r_c4"][S.Ux], r["r_c4"]) <= 1e-11
    assert relerr(bufs["r_e"], r["r_e"]) <= 1e-11
    assert norm == pytest.approx(I.residual_norm(r), rel=1e-11)
    dg, D, r1, r2 = I.reduced_system(S, st, r, mu)
    rhs = I.doubly_augmented_rhs(S, D, r1, r2)
    assert relerr(from_padded(S, bufs["rhs"]), rhs) <= 1e-11
    diag = np.zeros(n + me + 2 * m)
    kq.kkt_diag(h, diag)
    assert relerr(from_padded(S, diag), I.jacobi_diagonal(S, dg, D)) <= 1e-11


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)], ids=["f64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_kkt_apply(kq, name, prec, tol):
    qp, S, st, h = _setup(kq, name, seed=1)
    mu = 0.01
    r = I.residuals(S, st, mu)
    dg, D, _, _ = I.reduced_system(S, st, r, mu)
    v = np.random.default_rng(5).standard_normal(S.NK)
    ref = I.kkt_apply(S, dg, D, v)
    out = np.zeros(h.nkp)
    kq.kkt_apply(h, to_padded(S, v), out, prec)
    got = from_padded(S, out)
    assert relerr(got, ref) <= tol
    # every entry, against the magnitude of the terms summed into it (|K||v|):
    # FP64 sums of up to a few thousand terms in another order stay far below
    # 1e-10 of it; the FP32 products' rounding (unit 6e-8) far below 1e-4
    scale = kkt_abs_apply(S, dg, D, v)
    etol = 1e-10 if prec == 0 else 1e-4
    bad = np.abs(got - ref) > etol * scale + 1e-300
    assert not np.any(bad), (np.flatnonzero(bad)[:5], np.max(np.abs(got - ref) / (scale + 1e-300)))
    # padded rows of absent bounds stay exactly zero
    pad = np.ones(h.nkp, bool)
    pad[np.concatenate([np.arange(S.n + S.me), S.n + S.me + S.L, S.n + S.me + S.m + S.U])] = False
    assert np.all(out[pad] == 0.0)


@pytest.mark.parametrize("name", ["csr", "csr_multichunk", "csr_short_irregular"])
def test_kkt_apply_staged_operator(kq, name, monkeypatch):
    """FP32 products of short-row CSR problems normally run the
    register-streamed operator; KQ_STAGED=1 at create selects the staged
    shared-memory operator instead.  Both against the oracle."""
    monkeypatch.setenv("KQ_STAGED", "1")
    qp, S, st, h = _setup(kq, name, seed=1)
    monkeypatch.delenv("KQ_STAGED")
    mu = 0.01
    r = I.residuals(S, st, mu)
    dg, D, _, _ = I.reduced_system(S, st, r, mu)
    v = np.random.default_rng(5).standard_normal(S.NK)
    ref = I.kkt_apply(S, dg, D, v)
    out = np.zeros(h.nkp)
    kq.kkt_apply(h, to_padded(S, v), out, 1)
    got = from_padded(S, out)
    assert relerr(got, ref) <= 1e-5
    assert np.all(np.abs(got - ref) <= 1e-4 * kkt_abs_apply(S, dg, D, v))


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_kkt_pcg_solve(kq, name, prec):
    qp, S, st, h = _setup(kq, name, seed=2)
    mu = 0.01
    r = I.residuals(S, st, mu)
    dg, D, r1, r2 = I.reduced_system(S, st, r, mu)
    rhs = I.doubly_augmented_rhs(S, D, r1, r2)
    sol = np.zeros(h.nkp)
    opts = kq.default_pcg_opts(tol=1e-10, maxit=20000, precision=prec, refine_steps=3,
                               inner_tol=1e-5)
    rc, stt = kq.kkt_pcg_solve(h, to_padded(S, rhs), sol, opts)
    z = from_padded(S, sol)
    # FP64 residual of the returned solution, evaluated by the oracle
    res = np.linalg.norm(rhs - I.kkt_apply(S, dg, D, z)) / np.linalg.norm(rhs)
    assert res <= 1e-10 * 1.01, (res, stt.as_dict())
    dx, dl = I.newton_direct(S, dg, D, r1, r2)
    zs = np.concatenate([dx, dl])
    assert relerr(z, zs) <= 1e-6


_ORACLE = {}


def _oracle_result(name):
    if name not in _ORACLE:
        _ORACLE[name] = oracle.ipm_solve(PROBLEMS[name]())
    return _ORACLE[name]


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_ipm_matches_oracle(kq, name, prec):
    qp = PROBLEMS[name]()
    res = _oracle_result(name)
    assert res.status == "converged"
    opts = kq.default_ipm_opts(precision=prec)
    rc, st, out = kq.solve(qp, opts)
    f_gpu, f_ref = qp.objective(out["x"]), qp.objective(res.x)
    assert abs(f_gpu - f_ref) <= 1e-6 * (1 + abs(f_ref)), (f_gpu, f_ref, st.as_dict())
    met = oracle.kkt_metrics(qp, out["x"], out["lam_lA"], out["lam_uA"], out["lam_lx"],
                             out["lam_ux"], out["lam_e"])
    # Algorithm 1 stops once the residual norm of the scaled problem is below
    # mu (itself below mu_tol); the objective scaling sigma divides the dual
    # residual back out, so |r_H| in original units is below mu_final / sigma.
    # The gate is 1e-6 or that guarantee, whichever is looser.
    assert st.res_norm < st.mu_final, st.as_dict()
    sigma = I.scale(qp).sigma
    dual_bound = max(1e-6, 2.0 * st.mu_final / (sigma * met["dual_scale"]))
    assert met["primal_rel"] <= 1e-6 and met["dual_rel"] <= dual_bound, (met, dual_bound)
    # same mu path: complementarity of the same size as the oracle's
    from oracle.metrics import full_multipliers
    ref = oracle.kkt_metrics(qp, res.x, *full_multipliers(res.scaled, res.lam, qp))
    assert met["compl_rel"] <= 2.0 * ref["compl_rel"] + 1e-12, (met, ref)
    assert st.mu_final == pytest.approx(res.mu)


def test_config0(kq):
    """Tiny dense convex QP (n=200, 100 one-sided rows, box bounds)."""
    qp = qpgen.config0()
    res = oracle.ipm_solve(qp)
    for prec in (0, 1):
        rc, st, out = kq.solve(qp, kq.default_ipm_opts(precision=prec))
        f_gpu, f_ref = qp.objective(out["x"]), qp.objective(res.x)
        assert abs(f_gpu - f_ref) <= 1e-6 * (1 + abs(f_ref))
        met = oracle.kkt_metrics(qp, out["x"], out["lam_lA"], out["lam_uA"], out["lam_lx"],
                                 out["lam_ux"], out["lam_e"])
        assert met["kkt_rel"] <= 1e-6


def test_unconstrained_closed_form(kq):
    qp = qpgen.dense_qp(50, 1, seed=4)
    qp.akind, qp.A, qp.lA, qp.uA = "none", None, None, None
    qp.lx = np.full(qp.n, -np.inf)
    qp.ux = np.full(qp.n, np.inf)
    rc, st, out = kq.solve(qp)
    xs = -np.linalg.solve(qp.H_dense(), qp.p)
    assert relerr(out["x"], xs) <= 1e-9


def test_bad_arguments_are_rejected(kq):
    import ctypes
    H = kq.KqHop()
    H.kind = 7
    with pytest.raises(kq.KQError) as e:
        kq.qp_create(4, H, np.zeros(4))
    assert e.value.status == kq.KQ_ERR_ARG
    with pytest.raises(kq.KQError):
        kq.qp_create(0, kq.KqHop(), np.zeros(1))


def test_backward_before_solve_is_a_state_error(kq):
    h = kq.create_from(qpgen.dense_qp(10, 5, seed=1))
    with pytest.raises(kq.KQError) as e:
        kq.qp_backward(h, np.ones(10), np.zeros(10))
    assert e.value.status == kq.KQ_ERR_STATE


def test_residuals_worked_example(kq):
    """The library's residual blocks of Eq. (7) and ||r||_2 on the hand-worked
    example of the oracle pins (values computed by hand from Eq. (3), not by
    the oracle)."""
    from tests.test_oracle import WORKED_BLOCKS, WORKED_NORM2, _worked_qp, _worked_state
    qp = _worked_qp()
    S = I.scale(qp)
    h = kq.create_from(qp)
    set_gpu_state(kq, h, S, _worked_state(), 0.1)
    n, m, me = 2, 1, 1
    bufs = {k: np.zeros(n) for k in ("r_H", "r_lx", "r_ux", "r_c3", "r_c4")}
    bufs.update({k: np.zeros(m) for k in ("r_lA", "r_uA", "r_c1", "r_c2")})
    bufs["r_e"] = np.zeros(me)
    norm = kq.qp_residuals(h, **bufs)
    # the library stores bound blocks at full length n (0 where a bound is absent)
    assert np.allclose(bufs["r_H"], WORKED_BLOCKS["r_H"], rtol=0, atol=1e-13)
    assert np.allclose(bufs["r_lx"], WORKED_BLOCKS["r_lx"], rtol=0, atol=1e-13)
    assert np.allclose(bufs["r_ux"][:1], WORKED_BLOCKS["r_ux"], rtol=0, atol=1e-13)
    assert np.allclose(bufs["r_c3"], WORKED_BLOCKS["r_c3"], rtol=0, atol=1e-13)
    assert np.allclose(bufs["r_c4"][:1], WORKED_BLOCKS["r_c4"], rtol=0, atol=1e-13)
    for k in ("r_lA", "r_uA", "r_c1", "r_c2", "r_e"):
        assert np.allclose(bufs[k], WORKED_BLOCKS[k], rtol=0, atol=1e-13), k
    assert norm == pytest.approx(np.sqrt(WORKED_NORM2), rel=1e-13)
    kq.qp_destroy(h)


def test_initial_point_worked_example(kq):
    """The library's initial iterate (read back after create) equals the
    hand-worked R6 values of the oracle pin."""
    from tests.test_oracle import IP_EXPECT, _ip_qp
    qp = _ip_qp()
    h = kq.create_from(qp)
    n, m = 5, 3
    bufs = {k: np.zeros(n) for k in ("x", "s_lx", "s_ux", "lam_lx", "lam_ux")}
    bufs.update({k: np.zeros(m) for k in ("s_lA", "s_uA", "lam_lA", "lam_uA")})
    bufs["lam_e"] = np.zeros(1)
    mu = kq.qp_get_state(h, **bufs)
    assert mu == 1.0
    assert np.allclose(bufs["x"], IP_EXPECT["x"], rtol=0, atol=1e-14)
    L, U = [0, 1], [1, 2]              # rows with a finite lower / upper bound
    Lx, Ux = [0, 1, 4], [0, 2, 4]
    assert np.allclose(bufs["s_lA"][L], IP_EXPECT["s_lA"], rtol=0, atol=1e-13)
    assert np.allclose(bufs["s_uA"][U], IP_EXPECT["s_uA"], rtol=0, atol=1e-13)
    assert np.allclose(bufs["s_lx"][Lx], IP_EXPECT["s_lx"], rtol=0, atol=1e-14)
    assert np.allclose(bufs["s_ux"][Ux], IP_EXPECT["s_ux"], rtol=0, atol=1e-14)
    assert np.allclose(bufs["lam_lA"][L], 1.0) and np.allclose(bufs["lam_uA"][U], 1.0)
    assert np.allclose(bufs["lam_lx"][Lx], 1.0) and np.allclose(bufs["lam_ux"][Ux], 1.0)
    # absent bounds: multiplier 0
    assert bufs["lam_uA"][0] == 0.0 and bufs["lam_lA"][2] == 0.0
    assert bufs["lam_lx"][2] == 0.0 and bufs["lam_ux"][1] == 0.0
    assert np.allclose(bufs["lam_e"], 0.0)
    kq.qp_destroy(h)


@pytest.mark.parametrize("name", ["dense_eq", "csr", "lowrank_bfgs", "rbf_svm"])
def test_warm_start_matches_oracle(kq, name):
    """Warm-started Newton solves (opts.warm_start: each PCG starts from the
    previous Newton direction when that halves the FP64 residual) take the
    same IPM path to the same point: objective within 1e-6 of the oracle's,
    the same final mu, and the termination test met."""
    qp = PROBLEMS[name]()
    res = _oracle_result(name)
    rc, st, out = kq.solve(qp, kq.default_ipm_opts(warm_start=1))
    _, st0, _ = kq.solve(qp, kq.default_ipm_opts())
    print(name, "PCG iterations warm", st.pcg_iters, "cold", st0.pcg_iters)
    f_gpu, f_ref = qp.objective(out["x"]), qp.objective(res.x)
    assert abs(f_gpu - f_ref) <= 1e-6 * (1 + abs(f_ref)), (f_gpu, f_ref, st.as_dict())
    assert st.mu_final == pytest.approx(res.mu)
    assert st.res_norm < st.mu_final
