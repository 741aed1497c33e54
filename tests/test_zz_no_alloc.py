"""kkt_pcg_solve_static: the allocation-free entry point, for callers that
cannot allocate device memory (a fixed memory budget reserved up front, or an
allocator that must not be bypassed).  Its solution must match the
handle-based kkt_pcg_solve on the same doubly augmented system (Eq. (9)), on
two calls in a row (the static work array keeps the previous call's
contents), and meet the tolerance on the FP64 residual evaluated by the
oracle's matrix-free product.  Also covered: the largest work-space carve
(n = m = 4096), no general rows (m = 0), a D entry that is not positive
(KQ_ERR_ARG), an iteration cap (KQ_WARN_PCG_MAXIT) and oversize requests.
Collected last on purpose."""
import numpy as np
import pytest

from oracle import ipm as I

pytestmark = pytest.mark.gpu


def _problem(n=300, m=150, seed=21, rank=None):
    """Dense QP whose internal scaling is the identity (max H_ii = 1,
    |p|_inf <= 1, unit-norm rows), so both entry points see the same K."""
    import qpgen
    rng = np.random.default_rng(seed)
    q = 3 * n if rank is None else rank
    Q = rng.standard_normal((q, n))
    H = Q.T @ Q / q + 0.05 * np.eye(n)
    H = 0.5 * (H + H.T)
    H = H / np.max(np.diag(H))
    p = rng.uniform(-1.0, 1.0, n)
    x0 = rng.uniform(-0.2, 0.2, n)
    if m:
        A = rng.standard_normal((m, n))
        A = A / np.linalg.norm(A, axis=1)[:, None]
        qp = qpgen.QPData(n=n, hkind="dense", p=p, H=H, akind="dense", A=A,
                          lA=A @ x0 - 1.0, uA=A @ x0 + 1.0, lx=np.full(n, -1.0),
                          ux=np.full(n, 1.0))
    else:
        qp = qpgen.QPData(n=n, hkind="dense", p=p, H=H, akind="none",
                          lx=np.full(n, -1.0), ux=np.full(n, 1.0))
    st = {k: np.exp(rng.uniform(-2.0, 1.0, m)) for k in ("s_lA", "s_uA", "lam_lA", "lam_uA")}
    st.update({k: np.exp(rng.uniform(-2.0, 1.0, n)) for k in ("s_lx", "s_ux", "lam_lx", "lam_ux")})
    st["x"] = rng.uniform(-0.3, 0.3, n)
    return qp, st


@pytest.fixture(scope="module")
def kq():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as m
    m.load()
    return m


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _blocks(qp, st):
    m = qp.m
    Dl = st["s_lA"] / st["lam_lA"] if m else np.zeros(0)
    Du = st["s_uA"] / st["lam_uA"] if m else np.zeros(0)
    dg = st["lam_lx"] / st["s_lx"] + st["lam_ux"] / st["s_ux"]
    return Dl, Du, dg


def _oracle_K(qp, st, mu):
    """The oracle's matrix-free K*v of Eq. (9) at the same iterate (compact
    layout = the padded one here: every row two-sided, no equalities)."""
    S = I.scale(qp)
    ost = I.initial_point(S)
    for k, v in st.items():
        setattr(ost, k, np.asarray(v, float))
    r = I.residuals(S, ost, mu)
    dg, D, _, _ = I.reduced_system(S, ost, r, mu)
    return lambda v: I.kkt_apply(S, dg, D, v)


def _compare(kq, qp, st, tol, maxit, calls=2, seed=3):
    import torch
    n, m = qp.n, qp.m
    h = kq.create_from(qp)
    sigma, rhoA, _ = kq.qp_scaling(h)
    assert sigma == 1.0 and (m == 0 or np.max(np.abs(rhoA - 1.0)) < 1e-14)
    mu = 0.1
    kq.qp_set_state(h, mu, **st)
    Kv = _oracle_K(qp, st, mu)
    Dl, Du, dg = _blocks(qp, st)
    H_d, dg_d = _dev(qp.H), _dev(dg)
    A_d = _dev(qp.A) if m else None
    Dl_d = _dev(Dl) if m else None
    Du_d = _dev(Du) if m else None
    rng = np.random.default_rng(seed)
    opts = kq.default_pcg_opts(tol=tol, maxit=maxit)
    for call in range(calls):
        rhs = rng.standard_normal(n + 2 * m)
        ref = np.zeros(n + 2 * m)
        kq.kkt_pcg_solve(h, rhs, ref, opts)
        sol = torch.zeros(n + 2 * m, dtype=torch.float64, device="cuda")
        rc, iters, rel = kq.kkt_pcg_solve_static(n, m, H_d, A_d, Dl_d, Du_d, dg_d, _dev(rhs), sol,
                                                 tol=tol, maxit=maxit)
        torch.cuda.synchronize()
        got = sol.cpu().numpy()
        assert rc == kq.KQ_OK and iters > 0, (call, rc, iters, rel)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 1e-8, (call, err)
        true_res = np.linalg.norm(rhs - Kv(got)) / np.linalg.norm(rhs)
        assert true_res <= 10 * tol, (call, true_res)
    kq.qp_destroy(h)


def test_static_entry_matches_kkt_pcg_solve(kq):
    qp, st = _problem()
    _compare(kq, qp, st, tol=1e-12, maxit=20000)


def test_static_entry_no_general_rows(kq):
    qp, st = _problem(n=257, m=0, seed=5)
    _compare(kq, qp, st, tol=1e-12, maxit=20000)


def test_static_entry_largest_carve(kq):
    """n = m = 4096: every carve of the static array at its maximum."""
    qp, st = _problem(n=4096, m=4096, seed=9, rank=2112)
    _compare(kq, qp, st, tol=1e-10, maxit=20000, calls=2, seed=4)


def test_static_entry_iteration_cap(kq):
    import torch
    qp, st = _problem(seed=31)
    n, m = qp.n, qp.m
    Dl, Du, dg = _blocks(qp, st)
    rhs = np.random.default_rng(1).standard_normal(n + 2 * m)
    sol = torch.zeros(n + 2 * m, dtype=torch.float64, device="cuda")
    rc, iters, rel = kq.kkt_pcg_solve_static(n, m, _dev(qp.H), _dev(qp.A), _dev(Dl), _dev(Du),
                                             _dev(dg), _dev(rhs), sol, tol=1e-12, maxit=3)
    assert rc == kq.KQ_WARN_PCG_MAXIT and iters == 3 and rel > 1e-12


def test_static_entry_rejects_bad_D(kq):
    import torch
    qp, st = _problem(seed=32)
    n, m = qp.n, qp.m
    Dl, Du, dg = _blocks(qp, st)
    Dl[7] = 0.0
    sol = torch.zeros(n + 2 * m, dtype=torch.float64, device="cuda")
    with pytest.raises(kq.KQError) as e:
        kq.kkt_pcg_solve_static(n, m, _dev(qp.H), _dev(qp.A), _dev(Dl), _dev(Du), _dev(dg),
                                _dev(np.ones(n + 2 * m)), sol)
    assert e.value.status == kq.KQ_ERR_ARG
    Du[3] = np.nan
    Dl[7] = 1.0
    with pytest.raises(kq.KQError) as e:
        kq.kkt_pcg_solve_static(n, m, _dev(qp.H), _dev(qp.A), _dev(Dl), _dev(Du), _dev(dg),
                                _dev(np.ones(n + 2 * m)), sol)
    assert e.value.status == kq.KQ_ERR_ARG


def test_static_entry_rejects_oversize_and_host_buffers(kq):
    with pytest.raises(kq.KQError) as e:
        kq.kkt_pcg_solve_static(5000, 10, 1, 1, 1, 1, 1, 1, 1)
    assert e.value.status == kq.KQ_ERR_ARG
    with pytest.raises(TypeError):
        kq.kkt_pcg_solve_static(4, 0, np.eye(4), None, None, None, np.ones(4), np.ones(4),
                                np.zeros(4))
