"""Batched solve of many dense QPs of uneven size (one persistent PCG launch
per lock-step IPM iteration for all active QPs) against the oracle, per QP.

Small batch: every QP checked (objective within 1e-6 relative of the oracle's,
feasible).  Medium batch (128 QPs, n log-uniform in [64, 1024], H stored as
bf16, A as f32): all QPs converge; the smallest, the median and the largest QP
are checked against the oracle's full solve."""
import numpy as np
import pytest

import oracle
import qpgen
from oracle.metrics import full_multipliers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kq():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as m
    m.load()
    return m


def _check_against_oracle(qp, x, tag):
    res = oracle.ipm_solve(qp)
    assert res.status == "converged"
    f_ref = qp.objective(res.x)
    f = qp.objective(x)
    assert abs(f - f_ref) <= 1e-6 * (1 + abs(f_ref)), (tag, f, f_ref)
    # feasibility of x in original units (the batch API returns x only)
    A = qp.A_matrix()
    viol = max(0.0, float(np.max(qp.lA - A @ x)), float(np.max(np.abs(x)) - 1.0))
    assert viol <= 1e-6 * (1 + np.max(np.abs(x))), (tag, viol)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
def test_small_batch_against_oracle(kq, prec):
    sizes = qpgen.batch_sizes(16, 16, 400, size_seed=3)
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    b = kq.qp_create_batch(qps)
    xs = [np.zeros(qp.n) for qp in qps]
    rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=prec), xs)
    print("batch", st.as_dict())
    assert rc == kq.KQ_OK and all(s == kq.KQ_OK for s in status)
    for k, qp in enumerate(qps):
        _check_against_oracle(qp, xs[k], k)
    kq.qp_batch_destroy(b)


def test_batch_equals_single_solves(kq):
    sizes = [64, 300, 122, 900, 40, 2]
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    b = kq.qp_create_batch(qps)
    xs = [np.zeros(qp.n) for qp in qps]
    rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=1), xs)
    assert rc == kq.KQ_OK
    for k, qp in enumerate(qps):
        _, s1, out = kq.solve(qp, kq.default_ipm_opts(precision=1))
        f1, fb = qp.objective(out["x"]), qp.objective(xs[k])
        assert abs(f1 - fb) <= 1e-6 * (1 + abs(f1)), (k, f1, fb)


def test_medium_batch(kq):
    """128 QPs, n log-uniform in [64, 1024] (bf16 H, f32 A), mixed precision:
    all converge; smallest, median and largest QP checked against the oracle."""
    sizes = qpgen.batch_sizes(128, 64, 1024, size_seed=5)
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    b = kq.qp_create_batch(qps)
    xs = [np.zeros(qp.n) for qp in qps]
    rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=1), xs)
    print("medium batch", st.as_dict())
    assert rc == kq.KQ_OK and st.converged == len(qps)
    ns = np.array([qp.n for qp in qps])
    order = np.argsort(ns, kind="stable")
    for k in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        _check_against_oracle(qps[k], xs[k], (k, int(ns[k])))
    kq.qp_batch_destroy(b)
