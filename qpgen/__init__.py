"""Seeded synthetic convex-QP generators.

This module only *builds problem data* (matrices, vectors, bounds) with numpy's
PCG64 generator.  It holds none of the interior point method's arithmetic and is
the one piece of code shared by the CPU oracle, the tests, the benchmark and the
GPU path.  Every problem is a convex QP in the form of Eq. (1) of the paper,

    min 1/2 x^T H x + p^T x   s.t.  lA <= A x <= uA,  C x = b,  lx <= x <= ux,

with absent bounds given as +-inf.  The H operator comes in one of three
structures:

* ``dense``   : H is an explicit symmetric n x n matrix;
* ``csr_lsq`` : H = 2 P^T W P with P a CSR matrix (rows x n) and W = diag(w),
                the least-squares dose objective sum_i w_i (P x - d)_i^2;
* ``lowrank`` : H = Z W Z^T + H0 with Z a dense n x k matrix, W = diag(zw)
                (default I) and H0 = diag(d0) (default 0): the linear-kernel SVM
                dual (Z Z^T), or a quasi-Newton (BFGS) Hessian of the form
                H0 + U W U^T;
* ``rbf``     : H_ij = y_i y_j exp(-gamma ||x_i - x_j||^2), the Gaussian-kernel
                SVM dual, given by its samples X (n x d), labels y and gamma.

A constraint matrix A is either dense, a CSR matrix, or a subset of the rows of
P (``a_rows``), which is how dose-limit constraints reuse the dose matrix.

Only the primitive draws ``random``, ``uniform``, ``standard_normal``,
``lognormal`` and ``permutation`` are used, in a fixed order per generator, so
that the same seed gives the same problem on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

INF = np.inf


@dataclass
class QPData:
    """One convex QP (Eq. (1)), in original (unscaled) units."""

    n: int
    hkind: str                      # 'dense' | 'csr_lsq' | 'lowrank' | 'rbf'
    p: np.ndarray                   # linear term, float64 (n,)
    H: Optional[np.ndarray] = None  # dense H (float64 values), n x n
    P: Optional[sp.csr_matrix] = None   # csr_lsq: float32 CSR, rows x n
    w: Optional[np.ndarray] = None      # csr_lsq: float64 row weights
    Z: Optional[np.ndarray] = None      # lowrank: float32 n x k
    zw: Optional[np.ndarray] = None     # lowrank: column weights W (None = 1)
    d0: Optional[np.ndarray] = None     # lowrank: diagonal H0 (None = 0)
    X: Optional[np.ndarray] = None      # rbf: samples, float64 n x d
    y: Optional[np.ndarray] = None      # rbf: labels (+-1), float64 n
    gamma: float = 0.0                  # rbf: kernel width
    akind: str = "none"             # 'none' | 'dense' | 'csr' | 'rows_of_p'
    A: object = None                # dense ndarray (float64) or csr (float32)
    a_rows: Optional[np.ndarray] = None  # rows_of_p: int32 row ids into P
    lA: Optional[np.ndarray] = None
    uA: Optional[np.ndarray] = None
    C: Optional[np.ndarray] = None  # dense me x n float64
    b: Optional[np.ndarray] = None
    lx: Optional[np.ndarray] = None
    ux: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    # ---- sizes -----------------------------------------------------------
    @property
    def m(self) -> int:
        if self.akind == "none":
            return 0
        if self.akind == "rows_of_p":
            return int(len(self.a_rows))
        return int(self.A.shape[0])

    @property
    def me(self) -> int:
        return 0 if self.C is None else int(self.C.shape[0])

    def A_matrix(self):
        """Constraint rows as a scipy CSR (float64 data) or dense ndarray."""
        if self.akind == "none":
            return sp.csr_matrix((0, self.n))
        if self.akind == "rows_of_p":
            return self.P[self.a_rows].astype(np.float64)
        if self.akind == "csr":
            return self.A.astype(np.float64)
        return np.asarray(self.A, dtype=np.float64)

    def H_dense(self) -> np.ndarray:
        """Explicit H in float64 (only for sizes where that is affordable)."""
        if self.hkind == "dense":
            if self.H is None:
                return from_bf16_bits(self.meta["H_bf16_bits"]).reshape(self.n, self.n)
            return np.asarray(self.H, dtype=np.float64)
        if self.hkind == "csr_lsq":
            P = self.P.astype(np.float64)
            return np.asarray((2.0 * (P.T @ sp.diags(self.w) @ P)).todense())
        if self.hkind == "rbf":
            return rbf_matrix(self.X, self.y, self.gamma)
        Z = self.Z.astype(np.float64)
        zw = np.ones(Z.shape[1]) if self.zw is None else np.asarray(self.zw, float)
        d0 = np.zeros(self.n) if self.d0 is None else np.asarray(self.d0, float)
        return (Z * zw) @ Z.T + np.diag(d0)

    def objective(self, x: np.ndarray) -> float:
        """1/2 x^T H x + p^T x, evaluated from the operator's structure."""
        if self.hkind in ("dense", "rbf"):
            Hx = self.H_dense() @ x
        elif self.hkind == "csr_lsq":
            P = self.P.astype(np.float64)
            Hx = 2.0 * (P.T @ (self.w * (P @ x)))
        else:
            Z = self.Z.astype(np.float64)
            zw = np.ones(Z.shape[1]) if self.zw is None else np.asarray(self.zw, float)
            d0 = np.zeros(self.n) if self.d0 is None else np.asarray(self.d0, float)
            Hx = Z @ (zw * (Z.T @ x)) + d0 * x
        return float(0.5 * x @ Hx + self.p @ x)


def _full(n, v):
    return np.full(n, v, dtype=np.float64)


# ---------------------------------------------------------------------------
# bf16 rounding of problem data (round to nearest even).  Used so that a QP
# whose Hessian is *stored* in bf16 is exactly the QP the oracle solves.
# ---------------------------------------------------------------------------
def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """float -> uint16 bf16 bit patterns, round-to-nearest-even."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)


def from_bf16_bits(bits: np.ndarray) -> np.ndarray:
    u = bits.astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Dense QP ("tiny dense convex QP"):  H = Q^T Q / q + 1e-2 I, Q q x n iid N(0,1),
# p ~ N(0,1), A m x n iid N(0,1), b = A x0 - u, x0 ~ U(-.5,.5), u ~ U(.1,1),
# constraints A x >= b, -1 <= x <= 1.  Draw order: Q, p, A, x0, u.
# ---------------------------------------------------------------------------
def dense_qp(n: int = 200, m: int = 100, q: Optional[int] = None, seed: int = 0,
             h_bf16: bool = False, a_f32: bool = False, light: bool = False) -> QPData:
    """``light`` (with h_bf16 and a_f32): keep only the bf16 bits of H and A in
    float32 (no float64 copies); H_dense() / A_matrix() rebuild them."""
    rng = np.random.default_rng(seed)
    q = int(round(1.5 * n)) if q is None else q
    Q = rng.standard_normal((q, n))
    p = rng.standard_normal(n)
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(-0.5, 0.5, n)
    u = rng.uniform(0.1, 1.0, m)
    H = Q.T @ Q / q + 1e-2 * np.eye(n)
    H = 0.5 * (H + H.T)
    del Q
    meta = {"seed": seed, "q": q, "a_f32": a_f32}
    if h_bf16:
        bits = to_bf16_bits(H).reshape(n, n)
        H = None if light else from_bf16_bits(bits).reshape(n, n)
        meta["H_bf16_bits"] = bits
    if a_f32:
        A = A.astype(np.float32)
        b = A.astype(np.float64) @ x0 - u
        if not light:
            A = A.astype(np.float64)
        return QPData(n=n, hkind="dense", p=p, H=H, akind="dense", A=A,
                      lA=b, uA=_full(m, INF), lx=_full(n, -1.0), ux=_full(n, 1.0), meta=meta)
    b = A @ x0 - u
    return QPData(n=n, hkind="dense", p=p, H=H, akind="dense", A=A,
                  lA=b, uA=_full(m, INF), lx=_full(n, -1.0), ux=_full(n, 1.0),
                  meta=meta)


def config0() -> QPData:
    """Tiny dense convex QP: n=200, Q 300x200, A 100x200, seed 0."""
    return dense_qp(200, 100, q=300, seed=0)


# ---------------------------------------------------------------------------
# Dose-shaped least-squares QP.  P rows x cols CSR, nnz_row nonzeros per row,
# row r's columns drawn without replacement from the window of +-halfwin
# columns around floor(r*cols/rows) (clamped), sorted; values lognormal(0,1) in
# float32.  w ~ U(0.5,2), d ~ U(0,1).  ntarget distinct target rows T; a
# reference plan xhat ~ U(0.5,1.5); dose limits 0.95 P_T xhat <= P_T x <=
# 1.05 P_T xhat; x >= 0.  Objective sum_i w_i (P x - d)_i^2 = x^T (P^T W P) x
# - 2 (P^T W d)^T x + const, i.e. H = 2 P^T W P, p = -2 P^T W d.
# Draw order: column keys (per chunk of rows), values, w, d, T, xhat.
# ---------------------------------------------------------------------------
def _banded_csr_pattern(rng, rows, cols, nnz_row, halfwin, chunk=4096):
    W = 2 * halfwin + 1
    indptr = np.arange(rows + 1, dtype=np.int64) * nnz_row
    indices = np.empty(rows * nnz_row, dtype=np.int32)
    for r0 in range(0, rows, chunk):
        r1 = min(rows, r0 + chunk)
        r = np.arange(r0, r1, dtype=np.int64)
        centre = (r * cols) // rows
        lo = np.maximum(0, centre - halfwin)
        hi = np.minimum(cols - 1, centre + halfwin)
        width = hi - lo + 1
        keys = rng.random((r1 - r0, W))
        keys[np.arange(W)[None, :] >= width[:, None]] = 2.0   # outside window
        pick = np.argpartition(keys, nnz_row - 1, axis=1)[:, :nnz_row]
        colsel = np.sort(pick, axis=1) + lo[:, None]
        indices[r0 * nnz_row:r1 * nnz_row] = colsel.ravel().astype(np.int32)
    return indptr, indices


def dose_qp(rows: int = 200_000, cols: int = 20_000, nnz_row: int = 100,
            halfwin: int = 1000, ntarget: int = 10_000, seed: int = 1,
            unit_dose: bool = False) -> QPData:
    """``unit_dose``: the reference plan is rescaled so that its mean target
    dose is 1, the units of d ~ U(0,1) (prescription dose 1)."""
    rng = np.random.default_rng(seed)
    assert nnz_row <= halfwin + 1, "window too narrow for nnz_row"
    indptr, indices = _banded_csr_pattern(rng, rows, cols, nnz_row, halfwin)
    vals = rng.lognormal(0.0, 1.0, rows * nnz_row).astype(np.float32)
    P = sp.csr_matrix((vals, indices, indptr), shape=(rows, cols))
    w = rng.uniform(0.5, 2.0, rows)
    d = rng.uniform(0.0, 1.0, rows)
    T = np.sort(rng.permutation(rows)[:ntarget]).astype(np.int32)
    xhat = rng.uniform(0.5, 1.5, cols)
    P64 = P.astype(np.float64)
    if unit_dose:
        xhat = xhat / float(np.mean(P64[T] @ xhat))
    p = -2.0 * (P64.T @ (w * d))
    dose_hat = P64[T] @ xhat
    return QPData(n=cols, hkind="csr_lsq", p=p, P=P, w=w, akind="rows_of_p",
                  a_rows=T, lA=0.95 * dose_hat, uA=1.05 * dose_hat,
                  lx=_full(cols, 0.0), ux=_full(cols, INF),
                  meta={"seed": seed, "rows": rows, "nnz_row": nnz_row,
                        "halfwin": halfwin, "d": d, "xhat": xhat})


def irregular_lsq_qp(rows: int = 3000, cols: int = 5000, max_len: int = 250,
                     long_rows: int = 2, long_len: int = 4500, ntarget: int = 300,
                     seed: int = 12) -> QPData:
    """Least-squares QP with an irregular P: row lengths U{0..max_len} with
    uniformly scattered columns, plus a few over-long rows; two-sided limits
    on ntarget rows around a feasible reference plan; 0 <= x <= 2."""
    rng = np.random.default_rng(seed)
    lens = np.floor(rng.random(rows) * (max_len + 1)).astype(np.int64)
    pos = np.sort(rng.permutation(rows)[:long_rows])
    lens[pos] = long_len
    indptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    indices = np.empty(indptr[-1], dtype=np.int32)
    for r in range(rows):
        keys = rng.random(cols)
        indices[indptr[r]:indptr[r + 1]] = np.sort(np.argpartition(keys, lens[r])[:lens[r]]) \
            if lens[r] < cols else np.arange(cols)
    vals = rng.lognormal(0.0, 1.0, indptr[-1]).astype(np.float32)
    P = sp.csr_matrix((vals, indices, indptr), shape=(rows, cols))
    w = rng.uniform(0.5, 2.0, rows)
    d = rng.uniform(0.0, 1.0, rows)
    nz = np.nonzero(lens > 0)[0]
    T = np.sort(nz[rng.permutation(len(nz))[:ntarget]]).astype(np.int32)
    xhat = rng.uniform(0.5, 1.5, cols)
    P64 = P.astype(np.float64)
    xhat = xhat / float(np.mean(P64[T] @ xhat))
    p = -2.0 * (P64.T @ (w * d))
    dose_hat = P64[T] @ xhat
    return QPData(n=cols, hkind="csr_lsq", p=p, P=P, w=w, akind="rows_of_p", a_rows=T,
                  lA=0.9 * dose_hat, uA=1.1 * dose_hat, lx=_full(cols, 0.0),
                  ux=_full(cols, 2.0 * float(np.max(xhat))), meta={"seed": seed})


def config1() -> QPData:
    """Dose-shaped QP: P 200k x 20k, 2e7 nnz, 10k target rows, seed 1."""
    return dose_qp(200_000, 20_000, 100, 1000, 10_000, seed=1, unit_dose=True)


def config4() -> QPData:
    """Dose-shaped QP at 1/4 size: P 50k x 5k, 5e6 nnz, 2.5k targets, seed 4."""
    return dose_qp(50_000, 5_000, 100, 1000, 2_500, seed=4, unit_dose=True)


def config4_directions(qp: QPData, ndir: int = 32, seed: int = 4):
    """Seeded loss weights gbar (n,) and ndir N(0,1) directions in (p, lA, uA).

    The draws come after the problem's own draws in a generator seeded the
    same way, so they are fixed by the seed alone.
    """
    rng = np.random.default_rng([seed, 1])
    gbar = rng.standard_normal(qp.n)
    dirs_p = rng.standard_normal((ndir, qp.n))
    dirs_l = rng.standard_normal((ndir, qp.m))
    dirs_u = rng.standard_normal((ndir, qp.m))
    return gbar, dirs_p, dirs_l, dirs_u


# ---------------------------------------------------------------------------
# Linear soft-margin SVM dual (Eq. (6) with a linear kernel):  N samples of
# dim features drawn from a two-Gaussian mixture with means +-0.5 (all
# features) and unit variance; labels y = +-1 in equal numbers.
#   min 1/2 a^T (Y X X^T Y) a - e^T a   s.t.  y^T a = 0,  0 <= a <= cbox.
# Z = Y X (float32) so H = Z Z^T.  Draw order: label permutation, X noise.
# ---------------------------------------------------------------------------
def svm_qp(N: int = 50_000, dim: int = 256, cbox: float = 1.0, seed: int = 2) -> QPData:
    rng = np.random.default_rng(seed)
    y = np.ones(N)
    y[rng.permutation(N)[: N // 2]] = -1.0
    X = (0.5 * y[:, None] + rng.standard_normal((N, dim))).astype(np.float32)
    Z = (y[:, None].astype(np.float32) * X).astype(np.float32)
    return QPData(n=N, hkind="lowrank", p=_full(N, -1.0), Z=Z, akind="none",
                  C=y[None, :].copy(), b=np.zeros(1), lx=_full(N, 0.0),
                  ux=_full(N, cbox), meta={"seed": seed, "y": y})


# ---------------------------------------------------------------------------
# Gaussian-kernel SVM dual (Eq. (6) with k(u, v) = exp(-gamma ||u - v||^2)):
# samples and labels as in svm_qp (two Gaussians, means +-0.5 in every
# feature), gamma = 1/dim by default.
#   min 1/2 a^T (Y K Y) a - e^T a   s.t.  y^T a = 0,  0 <= a <= cbox.
# Draw order: label permutation, X noise.
# ---------------------------------------------------------------------------
def rbf_matrix(X: np.ndarray, y: Optional[np.ndarray], gamma: float) -> np.ndarray:
    """H = diag(y) K diag(y), K_ij = exp(-gamma ||x_i - x_j||^2), float64."""
    X = np.asarray(X, dtype=np.float64)
    sq = np.einsum("ij,ij->i", X, X)
    d2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * (X @ X.T), 0.0)
    np.fill_diagonal(d2, 0.0)
    K = np.exp(-gamma * d2)
    if y is not None:
        K = K * np.outer(y, y)
    return K


def rbf_svm_qp(N: int = 600, dim: int = 10, cbox: float = 1.0, gamma: Optional[float] = None,
               seed: int = 51) -> QPData:
    rng = np.random.default_rng(seed)
    y = np.ones(N)
    y[rng.permutation(N)[: N // 2]] = -1.0
    X = 0.5 * y[:, None] + rng.standard_normal((N, dim))
    g = 1.0 / dim if gamma is None else float(gamma)
    return QPData(n=N, hkind="rbf", p=_full(N, -1.0), X=X, y=y, gamma=g, akind="none",
                  C=y[None, :].copy(), b=np.zeros(1), lx=_full(N, 0.0),
                  ux=_full(N, cbox), meta={"seed": seed, "y": y})


def config2() -> QPData:
    """Linear SVM dual: N=50k samples, 256 features, seed 2."""
    return svm_qp(50_000, 256, 1.0, seed=2)


# ---------------------------------------------------------------------------
# Batched dense QPs: sizes n_k = 2*round(exp(U(ln lo, ln hi))/2) drawn with
# seed `size_seed`; QP k is dense_qp(n_k, n_k/2, q=3n_k/2, seed=k+1) with its
# Hessian rounded to bf16 (exactly the stored data) and A rounded to float32.
# ---------------------------------------------------------------------------
def batch_sizes(nqp: int = 512, lo: int = 64, hi: int = 4096, size_seed: int = 0) -> List[int]:
    rng = np.random.default_rng(size_seed)
    u = rng.uniform(np.log(lo), np.log(hi), nqp)
    return [int(max(2, 2 * round(np.exp(v) / 2))) for v in u]


def batch_qp(k: int, n: int, light: bool = False) -> QPData:
    return dense_qp(n, n // 2, q=(3 * n) // 2, seed=k + 1, h_bf16=True, a_f32=True, light=light)


def config3(nqp: int = 512, lo: int = 64, hi: int = 4096, light: bool = True) -> List[QPData]:
    """512 dense QPs; ``light`` keeps H as bf16 bits and A as float32 only."""
    return [batch_qp(k, n, light) for k, n in enumerate(batch_sizes(nqp, lo, hi))]


def tiny_qp(n: int, m: int, seed: int, me: int = 0, two_sided: bool = True,
            bounds: bool = True) -> QPData:
    """Small random strictly convex QP with two-sided rows, optional
    equalities and variable bounds; used for brute-force checks."""
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((n + 2, n))
    H = Q.T @ Q / (n + 2) + 0.1 * np.eye(n)
    H = 0.5 * (H + H.T)
    p = rng.standard_normal(n)
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(-0.3, 0.3, n)
    lo = A @ x0 - rng.uniform(0.1, 0.6, m)
    hi = A @ x0 + rng.uniform(0.1, 0.6, m) if two_sided else _full(m, INF)
    C = rng.standard_normal((me, n)) if me else None
    b = C @ x0 if me else None
    lx = _full(n, -0.6) if bounds else _full(n, -INF)
    ux = _full(n, 0.6) if bounds else _full(n, INF)
    return QPData(n=n, hkind="dense", p=p, H=H, akind="dense" if m else "none",
                  A=A if m else None, lA=lo if m else None, uA=hi if m else None,
                  C=C, b=b, lx=lx, ux=ux, meta={"seed": seed, "x0": x0})


# ---------------------------------------------------------------------------
# General sparse rows (Eq. (1) with a CSR A): every H structure above can take
# a general constraint matrix A in CSR and equality rows C.  The rows are
# drawn around a reference point x_ref that is strictly inside every bound, so
# that the problem stays strictly feasible:
#   A: m rows with nnz_row distinct random columns each, values N(0,1) (or
#      lognormal(0,1), positive, for dose-like rows), float32 or float64;
#      lA = A x_ref - U(0.1,1) on every row, uA = A x_ref + U(0.1,1) on a
#      `two_sided` fraction of the rows (+inf on the others);
#   C: me dense rows N(0,1), b = C x_ref.
# Draw order: column keys, values, lower margins, upper margins, two-sided
# mask, C.
# ---------------------------------------------------------------------------
def _sparse_rows(rng, m, n, nnz_row, positive, dtype):
    indptr = np.arange(m + 1, dtype=np.int64) * nnz_row
    keys = rng.random((m, n))
    cols = np.sort(np.argpartition(keys, nnz_row - 1, axis=1)[:, :nnz_row], axis=1)
    vals = rng.lognormal(0.0, 1.0, m * nnz_row) if positive else rng.standard_normal(m * nnz_row)
    return sp.csr_matrix((vals.astype(dtype), cols.ravel().astype(np.int32), indptr), shape=(m, n))


def with_general_rows(qp: QPData, m: int, nnz_row: int, me: int, x_ref: np.ndarray, seed: int,
                      two_sided: float = 0.5, positive: bool = False,
                      dtype=np.float64) -> QPData:
    """Replace qp's constraint rows by [existing rows as CSR; m new sparse rows]
    (kind 'csr') and its equality rows by me new dense rows."""
    rng = np.random.default_rng(seed)
    n = qp.n
    R = _sparse_rows(rng, m, n, nnz_row, positive, dtype)
    Rx = R.astype(np.float64) @ x_ref
    lo = Rx - rng.uniform(0.1, 1.0, m)
    hi = Rx + rng.uniform(0.1, 1.0, m)
    hi[rng.random(m) >= two_sided] = INF
    old = qp.A_matrix() if qp.akind != "none" else None
    if old is not None and old.shape[0]:
        A = sp.vstack([sp.csr_matrix(old, dtype=np.float64).astype(dtype), R]).tocsr()
        lA = np.concatenate([np.asarray(qp.lA, float), lo])
        uA = np.concatenate([np.asarray(qp.uA, float), hi])
    else:
        A, lA, uA = R, lo, hi
    C = rng.standard_normal((me, n)) if me else None
    b = C @ x_ref if me else None
    meta = dict(qp.meta)
    meta.update({"general_rows_seed": seed, "x_ref": x_ref})
    return QPData(n=n, hkind=qp.hkind, p=qp.p, H=qp.H, P=qp.P, w=qp.w, Z=qp.Z, zw=qp.zw,
                  d0=qp.d0, akind="csr",
                  A=A, lA=lA, uA=uA, C=C, b=b, lx=qp.lx, ux=qp.ux, meta=meta)


def dense_qp_general(n: int = 120, m: int = 90, nnz_row: int = 7, me: int = 3,
                     seed: int = 31) -> QPData:
    """Dense H (as dense_qp) with a sparse general A and equality rows."""
    base = dense_qp(n, 1, seed=seed)
    base.akind, base.A, base.lA, base.uA = "none", None, None, None
    x_ref = np.random.default_rng([seed, 7]).uniform(-0.5, 0.5, n)
    return with_general_rows(base, m, nnz_row, me, x_ref, seed + 1)


def dose_qp_general(rows: int = 6000, cols: int = 600, nnz_row: int = 40, halfwin: int = 60,
                    ntarget: int = 300, extra: int = 200, extra_nnz: int = 30, me: int = 2,
                    seed: int = 33) -> QPData:
    """Dose-shaped least-squares QP whose dose-limit rows are given as a
    general CSR A (not as rows of P), plus `extra` sparse positive rows with
    limits around the reference plan, and me equality rows (the setting of
    the photon case of section 4: general linear constraints besides the
    objective's dose matrix)."""
    base = dose_qp(rows, cols, nnz_row, halfwin, ntarget, seed=seed, unit_dose=True)
    xhat = base.meta["xhat"]
    return with_general_rows(base, extra, extra_nnz, me, xhat, seed + 1, two_sided=1.0,
                             positive=True, dtype=np.float32)


def svm_qp_general(N: int = 400, dim: int = 12, m: int = 30, nnz_row: int = 25,
                   seed: int = 35) -> QPData:
    """Linear SVM dual (lowrank H, y'a = 0, box bounds) with extra sparse
    general rows around a = 1/2 (which meets y'a = 0 for balanced labels)."""
    base = svm_qp(N, dim, seed=seed)
    x_ref = np.full(N, 0.5)
    q = with_general_rows(base, m, nnz_row, 0, x_ref, seed + 1)
    q.C, q.b = base.C, base.b
    return q


# ---------------------------------------------------------------------------
# Quasi-Newton Hessian (section 2.1: the RT objectives are nonlinear and the
# QP subproblem's Hessian is a BFGS approximation H0 + U W U^T).  H0 =
# diag(d0), d0 ~ U(0.5, 2); U n x k with entries N(0,1)/sqrt(k) in float32;
# W = diag(w), w ~ U(0.1, 1); p ~ N(0,1); bounds 0 <= x <= 1 and, with
# `rows` > 0, sparse positive (dose-like) general rows with two-sided limits
# around x_ref = 1/2.  Draw order: d0, U, w, p, then the rows.
# ---------------------------------------------------------------------------
def bfgs_qp(n: int = 3000, k: int = 20, rows: int = 200, nnz_row: int = 40,
            seed: int = 41) -> QPData:
    rng = np.random.default_rng(seed)
    d0 = rng.uniform(0.5, 2.0, n)
    U = (rng.standard_normal((n, k)) / np.sqrt(k)).astype(np.float32)
    w = rng.uniform(0.1, 1.0, k)
    p = rng.standard_normal(n)
    qp = QPData(n=n, hkind="lowrank", p=p, Z=U, zw=w, d0=d0, akind="none",
                lx=_full(n, 0.0), ux=_full(n, 1.0), meta={"seed": seed})
    if rows:
        qp = with_general_rows(qp, rows, nnz_row, 0, np.full(n, 0.5), seed + 1, two_sided=1.0,
                               positive=True, dtype=np.float32)
    return qp
