"""Python binding of the GB300 Krylov interior point library (``libkktqp.so``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Buffers may be numpy arrays (host) or torch tensors (host or
device); they are passed to the C ABI as raw pointers.  There is no CPU
fallback: if the shared library is missing or fails to load, every call
raises.

Function names match the C ABI (``include/kktqp.h``):
``qp_create``, ``ipm_solve``, ``kkt_pcg_solve``, ``kkt_apply``, ``kkt_diag``,
``qp_backward``, ``qp_get_state``, ``qp_set_state``, ``qp_residuals``,
``qp_scaling``, ``qp_sizes``, ``qp_destroy``.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkktqp.so")

KQ_OK, KQ_ERR_ARG, KQ_ERR_CUDA, KQ_ERR_OOM, KQ_ERR_NOT_CONVEX = 0, 1, 2, 3, 4
KQ_WARN_PCG_MAXIT, KQ_ERR_IPM_MAXIT, KQ_ERR_TIMEOUT, KQ_ERR_NUMERIC, KQ_ERR_STATE = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_CONVEX",
                5: "WARN_PCG_MAXIT", 6: "ERR_IPM_MAXIT", 7: "ERR_TIMEOUT", 8: "ERR_NUMERIC",
                9: "ERR_STATE"}
KQ_H_DENSE, KQ_H_CSR_LSQ, KQ_H_LOWRANK, KQ_H_RBF = 0, 1, 2, 3
KQ_A_NONE, KQ_A_DENSE, KQ_A_CSR, KQ_A_ROWS_OF_P = 0, 1, 2, 3
KQ_F64, KQ_F32, KQ_BF16 = 0, 1, 2
KQ_PREC_F64, KQ_PREC_MIXED = 0, 1


class KqHop(C.Structure):
    _fields_ = [("kind", C.c_int), ("dtype", C.c_int), ("rows", C.c_int64), ("cols", C.c_int64),
                ("nnz", C.c_int64), ("val", C.c_void_p), ("col", C.c_void_p),
                ("rowptr", C.c_void_p), ("w", C.c_void_p), ("d0", C.c_void_p),
                ("gamma", C.c_double)]


class KqAmat(C.Structure):
    _fields_ = [("kind", C.c_int), ("dtype", C.c_int), ("m", C.c_int64), ("val", C.c_void_p),
                ("rows", C.c_void_p), ("nnz", C.c_int64), ("col", C.c_void_p),
                ("rowptr", C.c_void_p)]


class KqIpmOpts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu0", C.c_double), ("mu_tol", C.c_double),
                ("ipm_maxit", C.c_int), ("pcg_tol", C.c_double), ("pcg_maxit", C.c_int),
                ("precision", C.c_int), ("refine_steps", C.c_int), ("inner_tol", C.c_double),
                ("timeout_s", C.c_double), ("grid_ctas", C.c_int), ("verbose", C.c_int),
                ("record", C.c_int), ("graph", C.c_int), ("warm_start", C.c_int)]


class KqIpmIter(C.Structure):
    _fields_ = [("it", C.c_int), ("pcg_iters", C.c_int), ("pcg_iters_f64", C.c_int),
                ("lanczos_steps", C.c_int), ("mu", C.c_double), ("res_norm", C.c_double),
                ("primal_inf", C.c_double), ("dual_inf", C.c_double), ("compl_inf", C.c_double),
                ("alpha_x", C.c_double), ("alpha_lam", C.c_double), ("pcg_rel_res", C.c_double),
                ("pcg_ms", C.c_double), ("lanczos_min", C.c_double), ("lanczos_max", C.c_double),
                ("kappa_jacobi", C.c_double), ("diag_ratio", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KqIpmStats(C.Structure):
    _fields_ = [("status", C.c_int), ("ipm_iters", C.c_int), ("mu_final", C.c_double),
                ("res_norm", C.c_double), ("primal_inf", C.c_double), ("dual_inf", C.c_double),
                ("compl_inf", C.c_double), ("pcg_iters", C.c_longlong),
                ("pcg_maxit_hits", C.c_int), ("time_s", C.c_double), ("pcg_time_s", C.c_double),
                ("pcg_kernel_ms", C.c_double), ("pcg_launches", C.c_longlong),
                ("pcg_products", C.c_longlong), ("kernel_launches", C.c_longlong),
                ("pcg_iters_f64", C.c_longlong), ("pcg_products_f64", C.c_longlong),
                ("pcg_kernel_ms_f64", C.c_double), ("pcg_launches_f64", C.c_longlong),
                ("switched_to_f64", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KqPcgOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("precision", C.c_int),
                ("refine_steps", C.c_int), ("inner_tol", C.c_double)]


class KqPcgStats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("passes", C.c_int),
                ("rel_res", C.c_double), ("kernel_ms", C.c_double), ("iters_f64", C.c_int),
                ("products_f64", C.c_int), ("kernel_ms_f64", C.c_double),
                ("launches_f64", C.c_int), ("products", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

EXPORTS = ["kq_default_ipm_opts", "kq_default_pcg_opts", "qp_create", "ipm_solve",
           "kkt_pcg_solve", "kkt_apply", "kkt_diag", "qp_backward", "qp_get_state",
           "qp_set_state", "qp_residuals", "qp_scaling", "qp_sizes", "qp_last_error",
           "qp_destroy", "kq_global_error"]


def load(path: str = LIB_PATH):
    """Load libkktqp.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libkktqp.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I64, D, I = C.c_void_p, C.c_int64, C.c_double, C.c_int
    sig = {
        "kq_default_ipm_opts": (None, [C.POINTER(KqIpmOpts)]),
        "kq_default_pcg_opts": (None, [C.POINTER(KqPcgOpts)]),
        "qp_create": (I, [C.POINTER(P), I64, C.POINTER(KqHop), P, C.POINTER(KqAmat), P, P, I64, P,
                          P, P, P, P]),
        "ipm_solve": (I, [P, C.POINTER(KqIpmOpts), P, P, P, P, P, P, C.POINTER(KqIpmStats)]),
        "kkt_pcg_solve": (I, [P, P, P, C.POINTER(KqPcgOpts), C.POINTER(KqPcgStats)]),
        "kkt_apply": (I, [P, P, P, I]),
        "kkt_diag": (I, [P, P]),
        "qp_backward": (I, [P, P, P, P, P, P, C.POINTER(KqPcgOpts), C.POINTER(KqPcgStats)]),
        "qp_get_state": (I, [P] * 11 + [C.POINTER(D)]),
        "qp_set_state": (I, [P] * 11 + [D]),
        "qp_residuals": (I, [P] * 13),
        "qp_scaling": (I, [P, C.POINTER(D), P, P]),
        "qp_sizes": (I, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
        "qp_last_error": (C.c_char_p, [P]),
        "qp_destroy": (None, [P]),
        "kq_global_error": (C.c_char_p, []),
        "kkt_pcg_solve_static": (I, [I64, I64, P, P, P, P, P, P, P, D, I, P, C.POINTER(C.c_int),
                                     C.POINTER(D)]),
        "kq_barrier_selftest": (I, [I, D, C.POINTER(I), C.POINTER(D)]),
        "qp_update": (I, [P, P, P, P, P]),
        "qp_iteration_log": (I, [P, C.POINTER(KqIpmIter), I, C.POINTER(I)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class KQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported buffer type {type(a)}")


def default_ipm_opts(**kw) -> KqIpmOpts:
    o = KqIpmOpts()
    load().kq_default_ipm_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_pcg_opts(**kw) -> KqPcgOpts:
    o = KqPcgOpts()
    load().kq_default_pcg_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Handle:
    """Owns a kq_handle; keeps Python references to the input buffers alive
    until qp_create has copied them."""

    def __init__(self, h, n, m, me, nkp):
        self.h, self.n, self.m, self.me, self.nkp = h, n, m, me, nkp

    def check(self, st, allow=(KQ_OK,)):
        if st not in allow:
            raise KQError(st, load().qp_last_error(self.h).decode())
        return st

    def __del__(self):
        try:
            qp_destroy(self)
        except Exception:
            pass


def qp_create(n, H: KqHop, p, A: Optional[KqAmat] = None, lA=None, uA=None, me=0, Cm=None,
              b=None, lx=None, ux=None, stream=None, keep=()) -> Handle:
    lib = load()
    h = C.c_void_p()
    st = lib.qp_create(C.byref(h), int(n), C.byref(H), _ptr(p), C.byref(A) if A is not None else None,
                       _ptr(lA), _ptr(uA), int(me), _ptr(Cm), _ptr(b), _ptr(lx), _ptr(ux), stream)
    if st != KQ_OK:
        raise KQError(st, lib.kq_global_error().decode())
    n_, m_, me_, nkp_ = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    lib.qp_sizes(h, C.byref(n_), C.byref(m_), C.byref(me_), C.byref(nkp_))
    return Handle(h, n_.value, m_.value, me_.value, nkp_.value)


def qp_iteration_log(h: Handle):
    """Per-IPM-iteration records of the last ipm_solve run with record=1, as
    a list of dicts (see kq_ipm_iter in kktqp.h)."""
    lib = load()
    cnt = C.c_int()
    h.check(lib.qp_iteration_log(h.h, None, 0, C.byref(cnt)))
    buf = (KqIpmIter * max(1, cnt.value))()
    h.check(lib.qp_iteration_log(h.h, buf, cnt.value, C.byref(cnt)))
    return [buf[i].as_dict() for i in range(cnt.value)]


def qp_update(h: Handle, p=None, lA=None, uA=None, b=None):
    """Replace p, lA, uA and/or b (None keeps a value); see qp_update in kktqp.h."""
    h.check(load().qp_update(h.h, _ptr(p), _ptr(lA), _ptr(uA), _ptr(b)))


def qp_destroy(h: Handle):
    if h is not None and h.h:
        load().qp_destroy(h.h)
        h.h = None


def ipm_solve(h: Handle, opts: Optional[KqIpmOpts] = None, x=None, lam_lA=None, lam_uA=None,
              lam_lx=None, lam_ux=None, lam_e=None, allow=(KQ_OK,)):
    st = KqIpmStats()
    rc = load().ipm_solve(h.h, C.byref(opts) if opts is not None else None, _ptr(x), _ptr(lam_lA),
                          _ptr(lam_uA), _ptr(lam_lx), _ptr(lam_ux), _ptr(lam_e), C.byref(st))
    h.check(rc, allow)
    return rc, st


def kkt_pcg_solve(h: Handle, rhs, sol, opts: Optional[KqPcgOpts] = None,
                  allow=(KQ_OK, KQ_WARN_PCG_MAXIT)):
    st = KqPcgStats()
    rc = load().kkt_pcg_solve(h.h, _ptr(rhs), _ptr(sol), C.byref(opts) if opts else None, C.byref(st))
    h.check(rc, allow)
    return rc, st


def kkt_apply(h: Handle, v, out, precision=KQ_PREC_F64):
    h.check(load().kkt_apply(h.h, _ptr(v), _ptr(out), int(precision)))


def kkt_diag(h: Handle, out):
    h.check(load().kkt_diag(h.h, _ptr(out)))


def qp_backward(h: Handle, gbar, grad_p=None, grad_lA=None, grad_uA=None, grad_b=None,
                opts: Optional[KqPcgOpts] = None, allow=(KQ_OK, KQ_WARN_PCG_MAXIT)):
    st = KqPcgStats()
    rc = load().qp_backward(h.h, _ptr(gbar), _ptr(grad_p), _ptr(grad_lA), _ptr(grad_uA), _ptr(grad_b),
                            C.byref(opts) if opts else None, C.byref(st))
    h.check(rc, allow)
    return rc, st


def qp_get_state(h: Handle, **bufs):
    mu = C.c_double()
    keys = ["x", "s_lA", "s_uA", "s_lx", "s_ux", "lam_lA", "lam_uA", "lam_lx", "lam_ux", "lam_e"]
    h.check(load().qp_get_state(h.h, *[_ptr(bufs.get(k)) for k in keys], C.byref(mu)))
    return mu.value


def qp_set_state(h: Handle, mu, **bufs):
    keys = ["x", "s_lA", "s_uA", "s_lx", "s_ux", "lam_lA", "lam_uA", "lam_lx", "lam_ux", "lam_e"]
    h.check(load().qp_set_state(h.h, *[_ptr(bufs.get(k)) for k in keys], float(mu)))


def qp_residuals(h: Handle, **bufs):
    keys = ["r_H", "r_lA", "r_uA", "r_c1", "r_c2", "r_lx", "r_ux", "r_c3", "r_c4", "r_e", "rhs"]
    norm = C.c_double()
    h.check(load().qp_residuals(h.h, *[_ptr(bufs.get(k)) for k in keys], C.byref(norm)))
    return norm.value


def _dev_ptr(a, name):
    """Device pointer of a contiguous CUDA tensor (None passes as NULL); the
    allocation-free entry point takes device memory only, so host arrays are
    refused here rather than handed to its kernels."""
    if a is None:
        return None
    if not (hasattr(a, "is_cuda") and a.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    return _ptr(a)


def kkt_pcg_solve_static(n, m, H, A, Dl, Du, dg, rhs, sol, tol=1e-7, maxit=5000, stream=None,
                         allow=(KQ_OK, KQ_WARN_PCG_MAXIT)):
    """Allocation-free dense PCG solve; every buffer is a CUDA tensor (float64)."""
    it = C.c_int()
    rel = C.c_double()
    lib = load()
    n, m = int(n), int(m)
    if n <= 0 or n > 4096 or m < 0 or m > 4096:
        rc = lib.kkt_pcg_solve_static(n, m, None, None, None, None, None, None, None, float(tol),
                                      int(maxit), stream, C.byref(it), C.byref(rel))
        raise KQError(rc, lib.kq_global_error().decode())
    ptrs = [_dev_ptr(a, k) for a, k in ((H, "H"), (A, "A"), (Dl, "Dl"), (Du, "Du"), (dg, "dg"),
                                        (rhs, "rhs"), (sol, "sol"))]
    rc = lib.kkt_pcg_solve_static(n, m, *ptrs, float(tol), int(maxit), stream,
                                  C.byref(it), C.byref(rel))
    if rc not in allow:
        raise KQError(rc, lib.kq_global_error().decode())
    return rc, it.value, rel.value


def barrier_selftest(ctas=4, budget_s=0.05):
    """Bounded-wait self-test (kq_barrier_selftest): returns (status, CTAs
    that gave up, device ms).  The expected status is KQ_ERR_TIMEOUT."""
    gave = C.c_int()
    ms = C.c_double()
    rc = load().kq_barrier_selftest(int(ctas), float(budget_s), C.byref(gave), C.byref(ms))
    return rc, gave.value, ms.value


def qp_scaling(h: Handle):
    sigma = C.c_double()
    rhoA = np.zeros(h.m)
    rhoC = np.zeros(h.me)
    h.check(load().qp_scaling(h.h, C.byref(sigma), _ptr(rhoA), _ptr(rhoC)))
    return sigma.value, rhoA, rhoC


# ---------------------------------------------------------------- convenience
def _as(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def create_from(qp, device_tensors: bool = False, stream=None) -> Handle:
    """Marshal a problem object (attributes n, hkind, p, H/P/w/Z/X, akind, A,
    a_rows, lA, uA, C, b, lx, ux -- the layout of the seeded generators) into
    qp_create.  With ``device_tensors`` the buffers are first moved to the
    current CUDA device (torch), so that qp_create copies device to device."""
    keep = []

    def buf(a, dtype):
        if a is None:
            return None
        arr = _as(a, dtype)
        if device_tensors:
            import torch
            t = torch.from_numpy(arr).cuda()
            keep.append(t)
            return t
        keep.append(arr)
        return arr

    n = qp.n
    H = KqHop()
    if qp.hkind == "dense":
        bits = qp.meta.get("H_bf16_bits") if getattr(qp, "meta", None) else None
        H.kind, H.rows, H.cols = KQ_H_DENSE, n, n
        if bits is not None:
            H.dtype, H.val = KQ_BF16, _ptr(buf(bits, np.uint16))
        else:
            H.dtype, H.val = KQ_F64, _ptr(buf(qp.H, np.float64))
    elif qp.hkind == "csr_lsq":
        H.kind, H.dtype, H.rows, H.cols, H.nnz = KQ_H_CSR_LSQ, KQ_F32, qp.P.shape[0], n, qp.P.nnz
        H.val = _ptr(buf(qp.P.data, np.float32))
        H.col = _ptr(buf(qp.P.indices, np.int32))
        H.rowptr = _ptr(buf(qp.P.indptr, np.int64))
        H.w = _ptr(buf(qp.w, np.float64))
    elif qp.hkind == "rbf":
        # samples, labels and width; the library forms H (stored as `rbf_dtype`)
        H.kind, H.rows, H.cols = KQ_H_RBF, n, qp.X.shape[1]
        H.dtype = {"f64": KQ_F64, "f32": KQ_F32, "bf16": KQ_BF16}[qp.meta.get("rbf_dtype", "f64")]
        H.val = _ptr(buf(qp.X, np.float64))
        if getattr(qp, "y", None) is not None:
            H.w = _ptr(buf(qp.y, np.float64))
        H.gamma = float(qp.gamma)
    else:
        H.kind, H.dtype, H.rows, H.cols = KQ_H_LOWRANK, KQ_F32, n, qp.Z.shape[1]
        H.val = _ptr(buf(qp.Z, np.float32))
        if getattr(qp, "zw", None) is not None:
            H.w = _ptr(buf(qp.zw, np.float64))
        if getattr(qp, "d0", None) is not None:
            H.d0 = _ptr(buf(qp.d0, np.float64))
    A = None
    lA = uA = None
    if qp.akind != "none":
        A = KqAmat()
        if qp.akind == "rows_of_p":
            A.kind, A.m, A.rows = KQ_A_ROWS_OF_P, len(qp.a_rows), _ptr(buf(qp.a_rows, np.int32))
        elif qp.akind == "csr":
            Ac = qp.A.tocsr()
            A.kind, A.m, A.nnz = KQ_A_CSR, Ac.shape[0], Ac.nnz
            if Ac.dtype == np.float32:
                A.dtype, A.val = KQ_F32, _ptr(buf(Ac.data, np.float32))
            else:
                A.dtype, A.val = KQ_F64, _ptr(buf(Ac.data, np.float64))
            A.col = _ptr(buf(Ac.indices, np.int32))
            A.rowptr = _ptr(buf(Ac.indptr, np.int64))
        else:
            Am = np.asarray(qp.A)
            A.kind, A.m = KQ_A_DENSE, Am.shape[0]
            if Am.dtype == np.float32 or qp.meta.get("a_f32", False):
                A.dtype, A.val = KQ_F32, _ptr(buf(Am, np.float32))
            else:
                A.dtype, A.val = KQ_F64, _ptr(buf(Am, np.float64))
        lA, uA = buf(qp.lA, np.float64), buf(qp.uA, np.float64)
    me = 0 if qp.C is None else qp.C.shape[0]
    Cm = buf(qp.C, np.float64) if me else None
    b = buf(qp.b, np.float64) if me else None
    h = qp_create(n, H, buf(qp.p, np.float64), A, lA, uA, me, Cm, b,
                  buf(qp.lx, np.float64), buf(qp.ux, np.float64), stream)
    if device_tensors:
        import torch
        torch.cuda.synchronize()
    return h


class _HandlePool:
    """Handles of one problem structure (H, A, C, variable bounds), created
    once and reused: a forward takes a free handle (creating one only when all
    are in use, e.g. several forwards before their backwards), replaces p, lA,
    uA and b with qp_update, and keeps the handle until its backward has run
    (the converged K lives in it)."""

    def __init__(self, qp):
        self.qp = qp
        self.free = []
        self.created = 0

    def take(self):
        if self.free:
            return self.free.pop()
        self.created += 1
        return create_from(self.qp)

    def give(self, h):
        self.free.append(h)


_POOLS = {}


def _pool(qp):
    key = id(qp)
    pl = _POOLS.get(key)
    if pl is None or pl.qp is not qp:
        pl = _POOLS[key] = _HandlePool(qp)
    return pl


def _qp_torch_layer():
    """Build the torch.autograd.Function lazily (torch is optional for the
    plain C-ABI binding)."""
    import torch

    def _dev(t, n):
        if n == 0 or t is None:
            return None
        return t.detach().to(dtype=torch.float64).contiguous()

    class QPFunction(torch.autograd.Function):
        """x* = argmin of the QP with linear term p, row bounds lA/uA and
        equality right-hand side b (the structure H, A, C and the variable
        bounds come from ``qp``).  Forward: qp_update + ipm_solve on a pooled
        handle (the tensors are passed as device pointers, no host copy).
        Backward: qp_backward, one PCG solve with the converged KKT matrix
        (Eq. (9)); gradients in original units, zero for absent bounds."""

        @staticmethod
        def forward(ctx, p, lA, uA, b, qp, opts):
            pool = _pool(qp)
            h = pool.take()
            pt, lt, ut, bt = _dev(p, h.n), _dev(lA, h.m), _dev(uA, h.m), _dev(b, h.me)
            torch.cuda.current_stream().synchronize()
            qp_update(h, pt, lt, ut, bt)
            x = torch.zeros(h.n, dtype=torch.float64, device=p.device)
            ipm_solve(h, opts, x=x)
            ctx.h, ctx.pool, ctx.dev = h, pool, p.device
            return x

        @staticmethod
        def backward(ctx, gx):
            h, dev = ctx.h, ctx.dev
            g = gx.detach().double().contiguous().to(dev)
            gp = torch.zeros(h.n, dtype=torch.float64, device=dev)
            glA = torch.zeros(h.m, dtype=torch.float64, device=dev)
            guA = torch.zeros(h.m, dtype=torch.float64, device=dev)
            gb = torch.zeros(h.me, dtype=torch.float64, device=dev)
            torch.cuda.current_stream().synchronize()
            qp_backward(h, g, gp, glA if h.m else None, guA if h.m else None,
                        gb if h.me else None)
            ctx.pool.give(h)
            ctx.h = None
            return gp, glA, guA, gb, None, None

    return QPFunction


_QPF = None


def qp_layer(qp, p, lA, uA, b, opts: Optional[KqIpmOpts] = None):
    """Differentiable QP solution x*(p, lA, uA, b) (torch tensors on cuda).
    The structure (H, A, C, variable bounds) is taken from ``qp``; its device
    handles are built once per ``qp`` object and reused across calls."""
    global _QPF
    if _QPF is None:
        _QPF = _qp_torch_layer()
    return _QPF.apply(p, lA, uA, b, qp, opts)


def solve(qp, opts: Optional[KqIpmOpts] = None, allow=(KQ_OK,)):
    """Create, solve, destroy; returns (status, stats, out) with out a dict of
    host arrays x, lam_lA, lam_uA, lam_lx, lam_ux, lam_e (original units)."""
    h = create_from(qp)
    n, m, me = h.n, h.m, h.me
    out = {k: np.zeros(s) for k, s in (("x", n), ("lam_lA", m), ("lam_uA", m), ("lam_lx", n),
                                       ("lam_ux", n), ("lam_e", me))}
    rc, st = ipm_solve(h, opts, **out, allow=allow)
    qp_destroy(h)
    return rc, st, out


# ---------------------------------------------------------------- batched QPs
class KqQpDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("H", KqHop), ("p", C.c_void_p), ("A", KqAmat),
                ("lA", C.c_void_p), ("uA", C.c_void_p), ("me", C.c_int64), ("C", C.c_void_p),
                ("b", C.c_void_p), ("lx", C.c_void_p), ("ux", C.c_void_p)]


class KqBatchStats(C.Structure):
    _fields_ = [("converged", C.c_int), ("ipm_iters_max", C.c_int),
                ("ipm_iters_total", C.c_longlong), ("pcg_iters", C.c_longlong),
                ("pcg_maxit_hits", C.c_int), ("max_active", C.c_int),
                ("pcg_kernel_ms", C.c_double), ("pcg_launches", C.c_longlong),
                ("time_s", C.c_double), ("graph_captures", C.c_int), ("graph_replays", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Batch:
    def __init__(self, b, ns):
        self.b, self.ns = b, ns

    def __del__(self):
        try:
            qp_batch_destroy(self)
        except Exception:
            pass


def _batch_lib():
    lib = load()
    if not hasattr(lib, "_batch_sigs"):
        P = C.c_void_p
        lib.qp_create_batch.restype = C.c_int
        lib.qp_create_batch.argtypes = [C.POINTER(P), C.c_int, C.POINTER(KqQpDesc), P]
        lib.ipm_solve_batch.restype = C.c_int
        lib.ipm_solve_batch.argtypes = [P, C.POINTER(KqIpmOpts), C.POINTER(P), C.POINTER(C.c_int),
                                        C.POINTER(KqBatchStats)]
        lib.qp_batch_destroy.restype = None
        lib.qp_batch_destroy.argtypes = [P]
        lib.qp_batch_last_error.restype = C.c_char_p
        lib.qp_batch_last_error.argtypes = [P]
        lib.kq_batch_error.restype = C.c_char_p
        lib.kq_batch_error.argtypes = []
        lib.qp_batch_qp_stats.restype = C.c_int
        lib.qp_batch_qp_stats.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
        lib.qp_batch_solution.restype = C.c_int
        lib.qp_batch_solution.argtypes = [P, C.c_int] + [P] * 6
        lib._batch_sigs = True
    return lib


def qp_create_batch(qps, stream=None) -> Batch:
    """Create a batch from problem objects with a dense H (generator layout:
    H as bf16 bits in meta['H_bf16_bits'] or float64, A dense)."""
    lib = _batch_lib()
    keep = []

    def arr(a, dt):
        x = np.ascontiguousarray(np.asarray(a, dtype=dt))
        keep.append(x)
        return x.ctypes.data

    descs = (KqQpDesc * len(qps))()
    for i, qp in enumerate(qps):
        d = descs[i]
        d.n = qp.n
        bits = qp.meta.get("H_bf16_bits") if qp.meta else None
        d.H.kind, d.H.rows, d.H.cols = KQ_H_DENSE, qp.n, qp.n
        if bits is not None:
            d.H.dtype, d.H.val = KQ_BF16, arr(bits, np.uint16)
        else:
            d.H.dtype, d.H.val = KQ_F64, arr(qp.H, np.float64)
        d.p = arr(qp.p, np.float64)
        if qp.akind == "dense":
            Am = np.asarray(qp.A)
            d.A.kind, d.A.m = KQ_A_DENSE, Am.shape[0]
            if Am.dtype == np.float32 or (qp.meta or {}).get("a_f32", False):
                d.A.dtype, d.A.val = KQ_F32, arr(Am, np.float32)
            else:
                d.A.dtype, d.A.val = KQ_F64, arr(Am, np.float64)
            d.lA, d.uA = arr(qp.lA, np.float64), arr(qp.uA, np.float64)
        else:
            d.A.kind = KQ_A_NONE
        d.me = 0 if qp.C is None else qp.C.shape[0]
        if d.me:
            d.C, d.b = arr(qp.C, np.float64), arr(qp.b, np.float64)
        d.lx, d.ux = arr(qp.lx, np.float64), arr(qp.ux, np.float64)
    b = C.c_void_p()
    rc = lib.qp_create_batch(C.byref(b), len(qps), descs, stream)
    if rc != KQ_OK:
        raise KQError(rc, lib.kq_batch_error().decode())
    return Batch(b, [qp.n for qp in qps])


def ipm_solve_batch(batch: Batch, opts: Optional[KqIpmOpts] = None, xs=None,
                    allow=(KQ_OK, KQ_ERR_IPM_MAXIT)):
    lib = _batch_lib()
    nq = len(batch.ns)
    ptrs = (C.c_void_p * nq)()
    if xs is not None:
        for i, x in enumerate(xs):
            ptrs[i] = _ptr(x)
    status = (C.c_int * nq)()
    st = KqBatchStats()
    rc = lib.ipm_solve_batch(batch.b, C.byref(opts) if opts is not None else None, ptrs, status,
                             C.byref(st))
    if rc not in allow:
        raise KQError(rc, lib.qp_batch_last_error(batch.b).decode())
    return rc, list(status), st


def qp_batch_solution(batch: Batch, i: int, qp):
    """QP i's iterate in original units: dict of host arrays x, lam_lA,
    lam_uA, lam_lx, lam_ux, lam_e (the layout of ``solve``)."""
    lib = _batch_lib()
    n, m, me = qp.n, qp.m, qp.me
    out = {k: np.zeros(s) for k, s in (("x", n), ("lam_lA", m), ("lam_uA", m), ("lam_lx", n),
                                       ("lam_ux", n), ("lam_e", me))}
    rc = lib.qp_batch_solution(batch.b, int(i), *[_ptr(out[k]) for k in
                                                  ("x", "lam_lA", "lam_uA", "lam_lx", "lam_ux",
                                                   "lam_e")])
    if rc != KQ_OK:
        raise KQError(rc, lib.qp_batch_last_error(batch.b).decode())
    return out


def qp_batch_qp_stats(batch: Batch, i: int):
    """(IPM iterations, PCG iterations) of QP i in the last ipm_solve_batch."""
    lib = _batch_lib()
    a, b = C.c_int(), C.c_longlong()
    rc = lib.qp_batch_qp_stats(batch.b, int(i), C.byref(a), C.byref(b))
    if rc != KQ_OK:
        raise KQError(rc, lib.qp_batch_last_error(batch.b).decode())
    return a.value, b.value


def qp_batch_destroy(batch: Batch):
    if batch is not None and batch.b:
        _batch_lib().qp_batch_destroy(batch.b)
        batch.b = None
