"""Host-side helpers of bench.py (CPU): the roofline byte counts it reports and
the traffic record it trusts."""
import json
import os

import numpy as np
import pytest

import bench
import qpgen


def test_algorithmic_bytes_of_the_dose_qp():
    qp = qpgen.dose_qp(3000, 300, 30, 40, 150, seed=8)
    rows, nnz = qp.P.shape[0], qp.P.nnz
    # nnz x (4 B value + 4 B column) + (rows + 1) x 4 B pointer + rows x 4 B weight
    assert bench.algo_bytes(qp) == nnz * 8 + (rows + 1) * 4 + rows * 4
    # the benchmark workload: 161.6 MB per product
    assert abs((2e7 * 8 + 200_001 * 4 + 200_000 * 4) - 161.6e6) < 1e2


def test_stored_bytes_of_the_register_streamed_layout():
    qp = qpgen.irregular_lsq_qp(rows=200, cols=300, max_len=37, long_rows=0, ntarget=10, seed=2)
    ln = np.diff(qp.P.indptr)
    groups = (ln + 3) // 4
    assert bench.stored_bytes(qp) == float(np.sum(groups) * 4 * 6 + len(ln) * 16)


def test_traffic_record_is_well_formed():
    # bench.py uses the record only while its kernel hash equals the current
    # kernel sources' (otherwise it reports traffic as null)
    tr = json.load(open(bench.TRAFFIC_FILE))
    assert len(tr["kernel_hash"]) == len(bench.kernel_source_hash()) == 16
    assert tr["precision"] == "mixed"
    assert 0.5 * 123.2e6 < tr["dram_bytes_per_product"] < 1.5 * 161.6e6


def test_peak_source():
    peak, src = bench.read_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and peak > 1000
    else:
        assert src == "fallback" and peak == 6800.0


def test_dose_kkt_matches_the_oracle_metric():
    """The bench's restated acceptance measure for the dose QP equals the
    oracle's (the GPU arm of the bench does not call the oracle)."""
    import numpy as np
    import oracle
    import qpgen
    from oracle.metrics import full_multipliers
    qp = qpgen.dose_qp(3000, 300, 30, 40, 150, seed=8)
    res = oracle.ipm_solve(qp)
    lam = full_multipliers(res.scaled, res.lam, qp)
    ref = oracle.kkt_metrics(qp, res.x, *lam)
    got = bench.dose_kkt(qp, res.x, *lam[:4])
    for k in ("primal_rel", "dual_rel", "kkt_rel", "objective"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-300), k
    # a perturbed point: both measures move together
    x2 = res.x + 1e-3
    ref2 = oracle.kkt_metrics(qp, x2, *lam)
    got2 = bench.dose_kkt(qp, x2, *lam[:4])
    assert got2["kkt_rel"] == pytest.approx(ref2["kkt_rel"], rel=1e-12)


def test_oracle_solve_estimate_counts_the_setup_once():
    """A full oracle solve = the step that ran the set-up with the first
    IPM iteration + (iterations - 1) x the plain iteration time."""
    r = {"times": [10.0, 3.0, 3.0], "iters": [1, 2, 3], "warm_times": []}
    total, first, per = bench.oracle_solve_estimate(r, 29)
    assert (total, first, per) == (10.0 + 28 * 3.0, 10.0, 3.0)
    r = {"times": [3.0, 5.0], "iters": [4, 5], "warm_times": [12.0, 3.0, 3.0]}
    total, first, per = bench.oracle_solve_estimate(r, 29)
    assert (total, first, per) == (12.0 + 28 * 4.0, 12.0, 4.0)
