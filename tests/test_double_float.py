"""The double-float arithmetic of the FP64-class products (float pairs on the
FP32 pipe), emulated step for step in NumPy float32 (no GPU): the two-sum and
the product residual are error-free, and a dot of bf16/f32 data with an FP64
vector stays within ~2^-48 per term of the exact sum, as the kernels assume.
The CUDA kernels themselves are checked against the oracle by the GPU parity
tests (dense bf16 problems and the CSR FP64 products)."""
from fractions import Fraction

import numpy as np

import qpgen

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    err = f32(f32(a - f32(s - bp)) + f32(b - bp))
    return s, err


def add_prod(h, l, m, vh, vl):
    """One term m * (vh + vl) into the pair (h, l), as DFAcc::add_prod."""
    p = f32(m * vh)
    e = f32(np.float64(m) * np.float64(vh) - np.float64(p))   # the FMA residual, exact
    q = f32(np.float64(m) * np.float64(vl) + np.float64(e))   # fma(m, vl, e)
    s, err = two_sum(h, p)
    return s, f32(l + f32(err + q))


def split(v):
    vh = f32(v)
    return vh, f32(v - np.float64(vh))


def test_two_sum_and_product_residual_are_exact():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = f32(rng.standard_normal() * 10.0 ** int(rng.integers(-8, 8))), f32(rng.standard_normal())
        s, err = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(err)) == Fraction(float(a)) + Fraction(float(b))
        m, v = f32(rng.standard_normal()), f32(rng.standard_normal())
        p = f32(m * v)
        e = f32(np.float64(m) * np.float64(v) - np.float64(p))
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(m)) * Fraction(float(v))


def test_dot_of_bf16_rows_within_2_to_48_per_term():
    qp = qpgen.batch_qp(3, 300)
    H = qp.H_dense()                       # bf16 values, exact in float32
    v = np.random.default_rng(5).standard_normal(qp.n)
    Hf = H.astype(f32)
    for i in range(0, qp.n, 37):
        h, l = f32(0), f32(0)
        for j in range(qp.n):
            vh, vl = split(v[j])
            h, l = add_prod(h, l, Hf[i, j], vh, vl)
        got = float(h) + float(l)
        exact = sum(Fraction(float(H[i, j])) * Fraction(float(v[j])) for j in range(qp.n))
        scale = float(np.abs(H[i]) @ np.abs(v))
        assert abs(Fraction(got) - exact) <= Fraction(qp.n * 2.0 ** -48 * scale)
        # and far inside it in practice
        assert abs(float(Fraction(got) - exact)) <= 1e-13 * scale
