"""Helpers shared by the GPU parity tests: map between the oracle's compact
multiplier layout and the library's padded layout, and set the same iterate
on both sides."""
import numpy as np

from oracle import ipm as I


def padded_index(S):
    """Indices of the oracle's compact KKT unknown inside the padded layout
    [x (n) | lam_e (me) | lam_lA (m) | lam_uA (m)]."""
    n, me, m = S.n, S.me, S.m
    return np.concatenate([np.arange(n), n + np.arange(me), n + me + S.L, n + me + m + S.U])


def to_padded(S, v):
    out = np.zeros(S.n + S.me + 2 * S.m)
    out[padded_index(S)] = v
    return out


def from_padded(S, v):
    return np.asarray(v)[padded_index(S)]


def random_state(S, seed, lo=-3.0, hi=1.5):
    rng = np.random.default_rng(seed)
    st = I.initial_point(S)
    st.x = rng.uniform(-0.4, 0.4, S.n)
    for k in ("s_lA", "s_uA", "s_lx", "s_ux", "lam_lA", "lam_uA", "lam_lx", "lam_ux"):
        v = getattr(st, k)
        setattr(st, k, np.exp(rng.uniform(lo, hi, len(v))))
    st.lam_e = rng.standard_normal(len(st.lam_e))
    return st


def set_gpu_state(kq, h, S, st, mu):
    n, m = S.n, S.m

    def full(idx, vals, size, fill):
        a = np.full(size, fill, dtype=np.float64)
        a[idx] = vals
        return a
    kq.qp_set_state(h, mu, x=np.ascontiguousarray(st.x),
                    s_lA=full(S.L, st.s_lA, m, 1.0), s_uA=full(S.U, st.s_uA, m, 1.0),
                    lam_lA=full(S.L, st.lam_lA, m, 0.0), lam_uA=full(S.U, st.lam_uA, m, 0.0),
                    s_lx=full(S.Lx, st.s_lx, n, 1.0), s_ux=full(S.Ux, st.s_ux, n, 1.0),
                    lam_lx=full(S.Lx, st.lam_lx, n, 0.0), lam_ux=full(S.Ux, st.lam_ux, n, 0.0),
                    lam_e=np.ascontiguousarray(st.lam_e))


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    d = np.max(np.abs(a - b)) if a.size else 0.0
    return d / (1e-300 + max(np.max(np.abs(b)) if b.size else 0.0, 1e-300))


def kkt_abs_apply(S, dg, D, v):
    """|K| |v| for the K of Eq. (9), matrix-free from |H|, |B| and D (every
    term of each entry's sum taken by its magnitude): the per-entry scale
    that rounding errors of K v are bounded by."""
    import scipy.sparse as sp
    n = S.n
    ax, al = np.abs(v[:n]), np.abs(v[n:])
    if S.hkind == "dense":
        hv = np.abs(S.H) @ ax
    elif S.hkind == "csr_lsq":
        Pa = abs(S.P)
        hv = Pa.T @ (np.abs(S.w2) * (Pa @ ax))
    else:
        Za = np.abs(S.Z)
        hv = Za @ (np.abs(S.zw) * (Za.T @ ax)) + np.abs(S.d0) * ax
    Aa = abs(S.A) if sp.issparse(S.A) else np.abs(S.A)
    Ca = np.abs(S.C)
    Av = Aa @ ax
    t = np.concatenate([Ca @ ax, Av[S.L], Av[S.U]])
    y = 2.0 * t / D + al
    me, nl = S.me, len(S.L)
    z = np.zeros(Aa.shape[0])
    np.add.at(z, S.L, y[me:me + nl])
    np.add.at(z, S.U, y[me + nl:])
    top = hv + np.abs(dg) * ax + Ca.T @ y[:me] + np.asarray(Aa.T @ z).ravel()
    return np.concatenate([top, t + D * al])
