"""The seeded synthetic workloads have the shapes and structure the input
recipe states (CPU).  These are the inputs every GPU parity test and the
benchmark use, so their structure is pinned here: sizes, sparsity pattern,
value ranges, feasibility of the reference plans, determinism of the seeds."""
import numpy as np
import pytest

import qpgen


def test_config0_shapes_and_feasible_start():
    qp = qpgen.config0()
    assert qp.n == 200 and qp.A.shape == (100, 200)
    H = qp.H_dense()
    assert np.allclose(H, H.T)
    assert np.linalg.eigvalsh(H).min() >= 1e-2 - 1e-12          # Q'Q/300 + 1e-2 I
    assert np.all(np.isinf(qp.uA)) and np.all(qp.lx == -1.0) and np.all(qp.ux == 1.0)


def test_dose_qp_structure_small():
    rows, cols, k, hw, nt = 4000, 400, 30, 40, 200
    qp = qpgen.dose_qp(rows, cols, k, hw, nt, seed=8, unit_dose=True)
    P = qp.P
    assert P.shape == (rows, cols) and P.nnz == rows * k
    assert P.dtype == np.float32 and np.all(P.data > 0)
    ln = np.diff(P.indptr)
    assert np.all(ln == k)
    for r in range(0, rows, 97):
        c = P.indices[P.indptr[r]:P.indptr[r + 1]]
        centre = r * cols // rows
        assert np.all(np.diff(c) > 0)                              # sorted, distinct
        assert c.min() >= max(0, centre - hw) and c.max() <= min(cols - 1, centre + hw)
    assert np.all((qp.w >= 0.5) & (qp.w <= 2.0))
    T = qp.a_rows
    assert len(np.unique(T)) == nt and np.all(np.diff(T) > 0)
    xhat = qp.meta["xhat"]
    dose = P[T].astype(np.float64) @ xhat
    assert np.mean(dose) == pytest.approx(1.0, rel=1e-12)           # unit prescription dose
    assert np.all(qp.lA < dose) and np.all(dose < qp.uA)           # strictly feasible plan
    assert np.allclose(qp.lA, 0.95 * dose) and np.allclose(qp.uA, 1.05 * dose)
    assert np.all(qp.lx == 0.0) and np.all(np.isinf(qp.ux))


def test_dose_qp_is_deterministic():
    a = qpgen.dose_qp(2000, 200, 20, 30, 50, seed=3)
    b = qpgen.dose_qp(2000, 200, 20, 30, 50, seed=3)
    assert np.array_equal(a.P.indices, b.P.indices) and np.array_equal(a.P.data, b.P.data)
    assert np.array_equal(a.p, b.p) and np.array_equal(a.a_rows, b.a_rows)


def test_svm_qp_structure():
    qp = qpgen.svm_qp(2000, 16, seed=9)
    y = qp.meta["y"]
    assert qp.Z.shape == (2000, 16) and qp.Z.dtype == np.float32
    assert np.sum(y == 1) == np.sum(y == -1) == 1000
    assert np.array_equal(qp.C[0], y) and np.all(qp.b == 0)
    assert np.all(qp.p == -1.0) and np.all(qp.lx == 0.0) and np.all(qp.ux == 1.0)


def test_batch_sizes_distribution():
    s = np.array(qpgen.batch_sizes(512, 64, 4096, size_seed=0))
    assert len(s) == 512 and np.all(s % 2 == 0)
    assert s.min() >= 64 and s.max() <= 4096
    # log-uniform: about half the sizes below the geometric mean 512
    assert 0.4 < np.mean(s < 512) < 0.6


def test_batch_qp_storage_is_exact():
    qp = qpgen.batch_qp(3, 96, light=True)
    assert qp.H is None and qp.meta["H_bf16_bits"].shape == (96, 96)
    H = qp.H_dense()
    assert np.allclose(H, H.T)
    assert qp.A.dtype == np.float32 and qp.A.shape == (48, 96)
    # the stored bf16 H is the problem solved: rebuilding it twice gives the same matrix
    assert np.array_equal(H, qp.H_dense())


@pytest.mark.parametrize("maker", ["dense_qp_general", "dose_qp_general", "svm_qp_general"])
def test_general_rows_structure(maker):
    """General sparse rows: CSR A, reference point strictly inside every row
    bound, variable bound and on the equality rows."""
    import scipy.sparse as sp
    qp = getattr(qpgen, maker)()
    assert qp.akind == "csr" and sp.issparse(qp.A)
    A = qp.A.tocsr()
    assert A.shape == (qp.m, qp.n) and A.has_sorted_indices
    x = qp.meta["x_ref"]
    Ax = A.astype(np.float64) @ x
    assert np.all(Ax > qp.lA) and np.all(Ax < qp.uA)
    assert np.all(x > qp.lx) and np.all(x < qp.ux)
    if qp.me:
        assert np.allclose(qp.C @ x, qp.b)
