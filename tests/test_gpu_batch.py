"""Batched solve of many dense QPs of uneven size (one persistent PCG launch
per lock-step IPM iteration for all active QPs) against the oracle, per QP.

Small batch: every QP checked (objective within 1e-6 relative of the oracle's,
KKT_rel <= 1e-6 with the batch's multipliers).  Medium batch (128 QPs, n log-uniform in [64, 1024], H stored as
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


def _check_solution(kq, b, k, qp, f_ref, compl_ref, tag):
    """QP k of the batch: x and its multipliers (qp_batch_solution) against
    the oracle's objective, KKT_rel <= 1e-6 by the oracle's metric code, and
    complementarity of the oracle's size (the same mu path)."""
    out = kq.qp_batch_solution(b, k, qp)
    met = oracle.kkt_metrics(qp, out["x"], out["lam_lA"], out["lam_uA"], out["lam_lx"],
                             out["lam_ux"], out["lam_e"])
    f = met["objective"]
    print(tag, "df %.2e kkt %.2e compl %.2e (oracle %.2e)" % (
        abs(f - f_ref) / (1 + abs(f_ref)), met["kkt_rel"], met["compl_rel"], compl_ref))
    assert abs(f - f_ref) <= 1e-6 * (1 + abs(f_ref)), (tag, f, f_ref)
    assert met["kkt_rel"] <= 1e-6, (tag, met)
    assert met["compl_rel"] <= 2.0 * compl_ref + 1e-12, (tag, met["compl_rel"], compl_ref)
    return out


def _check_against_oracle(kq, b, k, qp, x, tag):
    res = oracle.ipm_solve(qp)
    assert res.status == "converged"
    ref = oracle.kkt_metrics(qp, res.x, *full_multipliers(res.scaled, res.lam, qp))
    out = _check_solution(kq, b, k, qp, ref["objective"], ref["compl_rel"], tag)
    assert np.array_equal(out["x"], x)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
def test_small_batch_against_oracle(kq, prec, monkeypatch):
    # mixed: FP32 correction passes for every QP (by default only QPs whose
    # products read >= 128 MB take them; these are far smaller)
    monkeypatch.setenv("KQ_BATCH_F32_MIN_BYTES", "0")
    sizes = qpgen.batch_sizes(16, 16, 400, size_seed=3)
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    b = kq.qp_create_batch(qps)
    xs = [np.zeros(qp.n) for qp in qps]
    rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=prec), xs)
    print("batch", st.as_dict())
    assert rc == kq.KQ_OK and all(s == kq.KQ_OK for s in status)
    for k, qp in enumerate(qps):
        _check_against_oracle(kq, b, k, qp, xs[k], k)
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
        _check_against_oracle(kq, b, k, qps[k], xs[k], (k, int(ns[k])))
    kq.qp_batch_destroy(b)


@pytest.mark.parametrize("prec", [1, 0], ids=["mixed", "f64"])
def test_c3_largest_against_oracle(kq, prec):
    """The large end of the 512-QP batch workload: QPs 5, 9, 10, 12 and 26
    (n = 2850, 3126, 1904, 2264 and 4048, the largest QP of the batch; bf16
    H, f32 A) solved together, every QP against the oracle's stored solve
    (tests/golden/make_oracle_results.py): objective within 1e-6 relative,
    KKT_rel <= 1e-6 with the batch's multipliers, complementarity of the
    oracle's size."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_results.json")))["c3_subset"]
    sizes = qpgen.batch_sizes(512, 64, 4096)
    ids = sorted(int(k) for k in gold)
    qps = [qpgen.batch_qp(k, sizes[k]) for k in ids]
    assert [q.n for q in qps] == [gold[str(k)]["n"] for k in ids]
    b = kq.qp_create_batch(qps)
    xs = [np.zeros(q.n) for q in qps]
    rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=prec), xs)
    print("c3 subset", st.as_dict())
    assert rc == kq.KQ_OK and all(s_ == kq.KQ_OK for s_ in status)
    for j, k in enumerate(ids):
        g = gold[str(k)]
        assert g["status"] == "converged"
        out = _check_solution(kq, b, j, qps[j], g["objective"], g["compl_rel"], (k, qps[j].n))
        dx = np.max(np.abs(out["x"][g["x_idx"]] - np.array(g["x_at_idx"]))) / (1 + g["x_inf"])
        print("  x distance at sampled indices %.2e" % dx)
    kq.qp_batch_destroy(b)


@pytest.mark.parametrize("prec", [1, 0], ids=["mixed", "f64"])
def test_graph_replay_matches_host_driven(kq, prec, monkeypatch):
    """The lock-step IPM iteration captured once in a CUDA graph and
    replayed, every decision (pass precision, PCG stop, step lengths, mu
    rule, done) and the teams of every pass made on the device, gives the
    host-driven solver's solution and the oracle's; the graph is captured
    again only when QPs finish.  Mixed: FP32 passes for every QP."""
    monkeypatch.setenv("KQ_BATCH_F32_MIN_BYTES", "0")
    sizes = qpgen.batch_sizes(24, 16, 600, size_seed=11)
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    res = {}
    for graph in (1, 0):
        b = kq.qp_create_batch(qps)
        xs = [np.zeros(q.n) for q in qps]
        rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=prec, graph=graph), xs)
        print("graph", graph, st.as_dict())
        assert rc == kq.KQ_OK and all(s_ == kq.KQ_OK for s_ in status)
        if graph:
            assert 1 <= st.graph_captures <= len(qps) and st.graph_replays == st.ipm_iters_max
            for k in (0, len(qps) // 2, len(qps) - 1):
                _check_against_oracle(kq, b, k, qps[k], xs[k], ("graph", k))
        res[graph] = (xs, st)
        kq.qp_batch_destroy(b)
    for k, q in enumerate(qps):
        f1, f0 = q.objective(res[1][0][k]), q.objective(res[0][0][k])
        assert abs(f1 - f0) <= 1e-6 * (1 + abs(f0)), (k, f1, f0)
    # the same Algorithm 1 (the atomics' summation order may move a
    # borderline mu test by one iteration on a few QPs)
    assert abs(res[1][1].ipm_iters_total - res[0][1].ipm_iters_total) <= len(qps)
