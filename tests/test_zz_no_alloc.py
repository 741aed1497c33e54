"""kkt_pcg_solve_static: the allocation-free entry point for callers that
cannot allocate device memory.  Its solution must match the handle-based
kkt_pcg_solve on the same doubly augmented system, on two calls in a row
(the static work array keeps the previous call's contents).  Collected last
on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _problem(n=300, m=150, seed=21):
    """Dense QP whose internal scaling is the identity (max H_ii = 1,
    |p|_inf <= 1, unit-norm rows), so both entry points see the same K."""
    import qpgen
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((3 * n, n))
    H = Q.T @ Q / (3 * n) + 0.05 * np.eye(n)
    H = 0.5 * (H + H.T)
    H = H / np.max(np.diag(H))
    p = rng.uniform(-1.0, 1.0, n)
    A = rng.standard_normal((m, n))
    A = A / np.linalg.norm(A, axis=1)[:, None]
    x0 = rng.uniform(-0.2, 0.2, n)
    qp = qpgen.QPData(n=n, hkind="dense", p=p, H=H, akind="dense", A=A,
                      lA=A @ x0 - 1.0, uA=A @ x0 + 1.0, lx=np.full(n, -1.0), ux=np.full(n, 1.0))
    st = {k: np.exp(rng.uniform(-2.0, 1.0, m)) for k in ("s_lA", "s_uA", "lam_lA", "lam_uA")}
    st.update({k: np.exp(rng.uniform(-2.0, 1.0, n)) for k in ("s_lx", "s_ux", "lam_lx", "lam_ux")})
    st["x"] = rng.uniform(-0.3, 0.3, n)
    return qp, st


def test_static_entry_matches_kkt_pcg_solve():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as kq
    qp, st = _problem()
    n, m = qp.n, qp.m
    h = kq.create_from(qp)
    sigma, rhoA, _ = kq.qp_scaling(h)
    assert sigma == 1.0 and np.max(np.abs(rhoA - 1.0)) < 1e-14
    mu = 0.1
    kq.qp_set_state(h, mu, **st)
    Dl = st["s_lA"] / st["lam_lA"]
    Du = st["s_uA"] / st["lam_uA"]
    dg = st["lam_lx"] / st["s_lx"] + st["lam_ux"] / st["s_ux"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    H_d, A_d, Dl_d, Du_d, dg_d = dev(qp.H), dev(qp.A), dev(Dl), dev(Du), dev(dg)
    rng = np.random.default_rng(3)
    opts = kq.default_pcg_opts(tol=1e-12, maxit=20000)
    for call in range(2):
        rhs = rng.standard_normal(n + 2 * m)
        ref = np.zeros(n + 2 * m)
        kq.kkt_pcg_solve(h, rhs, ref, opts)
        sol = torch.zeros(n + 2 * m, dtype=torch.float64, device="cuda")
        rc, iters, rel = kq.kkt_pcg_solve_static(n, m, H_d, A_d, Dl_d, Du_d, dg_d, dev(rhs), sol,
                                                 tol=1e-12, maxit=20000)
        torch.cuda.synchronize()
        got = sol.cpu().numpy()
        assert rc == kq.KQ_OK and iters > 0, (call, rc, iters, rel)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 1e-8, (call, err)
    kq.qp_destroy(h)


def test_static_entry_rejects_oversize():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as kq
    with pytest.raises(kq.KQError) as e:
        kq.kkt_pcg_solve_static(5000, 10, 1, 1, 1, 1, 1, 1, 1)
    assert e.value.status == kq.KQ_ERR_ARG
