"""Failure detection through the C ABI (GPU).  Every failure is made on the
host side of the data or by a bounded wait that cannot complete; none faults,
traps or hangs the GPU.  Each test expects a status code and then checks that
the handle (or the context) still works.

* NaN in the linear term            -> KQ_ERR_NUMERIC at qp_create
* NaN planted in the iterate        -> KQ_ERR_NUMERIC from ipm_solve
* H = -I (not convex)               -> KQ_ERR_NOT_CONVEX (PCG meets p'Kp <= 0)
* pcg_maxit = 5                     -> KQ_WARN_PCG_MAXIT (kkt_pcg_solve), and
                                       ipm_solve counts the capped solves
* ipm_maxit = 3                     -> KQ_ERR_IPM_MAXIT with the third iterate
                                       returned (checked against the oracle's
                                       third iterate)
* grid barrier that cannot complete -> KQ_ERR_TIMEOUT (kq_barrier_selftest),
                                       then a normal solve on a live handle
* qp_backward before a solve        -> KQ_ERR_STATE
* column index out of range         -> KQ_ERR_ARG
"""
import numpy as np
import pytest

import oracle
import qpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kq():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as m
    m.load()
    return m


def _solve_ok(kq, qp, prec=0):
    rc, st, out = kq.solve(qp, kq.default_ipm_opts(precision=prec))
    res = oracle.ipm_solve(qp)
    f, fr = qp.objective(out["x"]), qp.objective(res.x)
    assert rc == kq.KQ_OK and abs(f - fr) <= 1e-6 * (1 + abs(fr))


def test_nan_in_data_rejected_at_create(kq):
    qp = qpgen.dense_qp(40, 20, seed=3)
    qp.p = qp.p.copy()
    qp.p[5] = np.nan
    with pytest.raises(kq.KQError) as e:
        kq.create_from(qp)
    assert e.value.status == kq.KQ_ERR_NUMERIC


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
def test_nan_in_iterate(kq, prec):
    qp = qpgen.dense_qp(40, 20, seed=3)
    h = kq.create_from(qp)
    x = np.zeros(qp.n)
    x[3] = np.nan
    kq.qp_set_state(h, 1.0, x=x)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(precision=prec), allow=(kq.KQ_ERR_NUMERIC,))
    assert rc == kq.KQ_ERR_NUMERIC
    # the same handle solves normally from its initial point afterwards
    out = np.zeros(qp.n)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(precision=prec), x=out)
    res = oracle.ipm_solve(qp)
    assert rc == kq.KQ_OK
    assert abs(qp.objective(out) - qp.objective(res.x)) <= 1e-6 * (1 + abs(qp.objective(res.x)))
    kq.qp_destroy(h)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
def test_not_convex(kq, prec):
    n = 32
    qp = qpgen.QPData(n=n, hkind="dense", p=np.linspace(-1, 1, n), H=-np.eye(n), akind="none",
                      lx=np.full(n, -np.inf), ux=np.full(n, np.inf))
    h = kq.create_from(qp)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(precision=prec), allow=(kq.KQ_ERR_NOT_CONVEX,))
    assert rc == kq.KQ_ERR_NOT_CONVEX
    assert "positive definite" in kq.load().qp_last_error(h.h).decode()
    kq.qp_destroy(h)
    _solve_ok(kq, qpgen.dense_qp(40, 20, seed=4), prec)


def test_pcg_iteration_cap(kq):
    qp = qpgen.config0()
    h = kq.create_from(qp)
    rhs = np.zeros(h.nkp)
    kq.qp_residuals(h, rhs=rhs)
    sol = np.zeros(h.nkp)
    rc, st = kq.kkt_pcg_solve(h, rhs, sol, kq.default_pcg_opts(maxit=5))
    assert rc == kq.KQ_WARN_PCG_MAXIT and st.iters == 5 and st.rel_res > 1e-7
    # inside the IPM a capped solve still takes its step and is counted
    rc, ist = kq.ipm_solve(h, kq.default_ipm_opts(pcg_maxit=5, ipm_maxit=4),
                           allow=(kq.KQ_ERR_IPM_MAXIT,))
    assert rc == kq.KQ_ERR_IPM_MAXIT and ist.pcg_maxit_hits == 4 and ist.ipm_iters == 4
    kq.qp_destroy(h)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
def test_ipm_iteration_cap_returns_last_iterate(kq, prec):
    qp = qpgen.config0()
    h = kq.create_from(qp)
    x = np.zeros(qp.n)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(precision=prec, ipm_maxit=3), x=x,
                          allow=(kq.KQ_ERR_IPM_MAXIT,))
    assert rc == kq.KQ_ERR_IPM_MAXIT and st.ipm_iters == 3
    ref = oracle.ipm_solve(qp, max_iters=3)
    assert ref.iters == 3 and ref.status == "maxit"
    # three Newton steps solved to 1e-7 relative: the iterates agree closely
    assert np.max(np.abs(x - ref.x)) <= 1e-5 * (1 + np.max(np.abs(ref.x)))
    xs = np.zeros(qp.n)
    kq.qp_get_state(h, x=xs)
    assert np.array_equal(xs, x)
    kq.qp_destroy(h)


def test_barrier_timeout_then_normal_solve(kq):
    qp = qpgen.config0()
    h = kq.create_from(qp)
    rc, gave_up, ms = kq.barrier_selftest(ctas=8, budget_s=0.05)
    assert rc == kq.KQ_ERR_TIMEOUT and gave_up == 8
    assert 40.0 <= ms <= 2000.0, ms
    # the context and an existing handle keep working
    x = np.zeros(qp.n)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(), x=x)
    res = oracle.ipm_solve(qp)
    assert rc == kq.KQ_OK
    assert abs(qp.objective(x) - qp.objective(res.x)) <= 1e-6 * (1 + abs(qp.objective(res.x)))
    kq.qp_destroy(h)


def test_backward_before_solve(kq):
    qp = qpgen.dense_qp(30, 10, seed=5)
    h = kq.create_from(qp)
    with pytest.raises(kq.KQError) as e:
        kq.qp_backward(h, np.ones(qp.n), grad_p=np.zeros(qp.n))
    assert e.value.status == kq.KQ_ERR_STATE
    kq.qp_destroy(h)


def test_bad_csr_rejected(kq):
    qp = qpgen.dose_qp(300, 40, 8, 10, 12, seed=12)
    qp.P = qp.P.copy()
    qp.P.indices = qp.P.indices.copy()
    qp.P.indices[17] = 40          # one past the last column
    with pytest.raises(kq.KQError) as e:
        kq.create_from(qp)
    assert e.value.status == kq.KQ_ERR_ARG
