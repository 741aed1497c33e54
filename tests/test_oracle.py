"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: a closed
form, brute-force enumeration, an independently assembled Newton system
(Eq. (7)), linear-algebra invariants (K symmetric positive definite, Eq. (9)),
finite differences, or the paper's printed settings.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import qpgen
from oracle import ipm as I
from oracle.metrics import full_multipliers
from tests.bruteforce import solve_bruteforce

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _random_interior_state(S, seed):
    rng = np.random.default_rng(seed)
    st = I.initial_point(S)
    st.x = rng.uniform(-0.4, 0.4, S.n)
    for k in ("s_lA", "s_uA", "s_lx", "s_ux", "lam_lA", "lam_uA", "lam_lx", "lam_ux"):
        v = getattr(st, k)
        setattr(st, k, np.exp(rng.uniform(-4, 2, len(v))))
    st.lam_e = rng.standard_normal(len(st.lam_e))
    return st


def _tiny_problems():
    out = []
    for seed in range(4):
        out.append(qpgen.tiny_qp(5, 3, seed, me=0))
        out.append(qpgen.tiny_qp(5, 2, 100 + seed, me=1))
        out.append(qpgen.tiny_qp(4, 3, 200 + seed, me=0, two_sided=False))
    return out


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("kind", ["dense", "csr_lsq"])
def test_unconstrained_closed_form(kind):
    """No A, C or bounds: x* = -H^{-1} p (section 2.1, Eq. (1) with no constraints)."""
    if kind == "dense":
        qp = qpgen.dense_qp(30, 1, seed=3)
        qp.akind, qp.A, qp.lA, qp.uA = "none", None, None, None
    else:
        qp = qpgen.dose_qp(400, 40, 10, 12, 1, seed=5)
        qp.akind, qp.a_rows, qp.lA, qp.uA = "none", None, None, None
    qp.lx = np.full(qp.n, -np.inf)
    qp.ux = np.full(qp.n, np.inf)
    res = oracle.ipm_solve(qp)
    H = qp.H_dense()
    xstar = -np.linalg.solve(H, qp.p)
    assert res.status == "converged"
    assert np.max(np.abs(res.x - xstar)) <= 1e-10 * (1 + np.max(np.abs(xstar)))


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("qp", _tiny_problems(), ids=lambda q: f"seed{q.meta['seed']}")
def test_bruteforce_active_set(qp):
    """IPM optimum equals the active-set enumeration optimum to O(mu_final)."""
    res = oracle.ipm_solve(qp)
    assert res.status == "converged"
    H = qp.H_dense()
    ref = solve_bruteforce(H, qp.p, qp.A, qp.lA, qp.uA, qp.C, qp.b, qp.lx, qp.ux)
    assert ref is not None
    xs, fs = ref
    ftol = 1e-6 * (1 + abs(fs))
    assert abs(qp.objective(res.x) - fs) <= ftol
    # strict convexity: f(x) - f* >= lam_min(H)/2 ||x - x*||^2 for feasible x,
    # so the objective gate bounds the distance (degenerate constraints make
    # the central path approach x* like sqrt(mu), not mu)
    lmin = np.min(np.linalg.eigvalsh(H))
    assert np.linalg.norm(res.x - xs) <= np.sqrt(2 * ftol / lmin)
    lA, uA, lx, ux, le = full_multipliers(res.scaled, res.lam, qp)
    met = oracle.kkt_metrics(qp, res.x, lA, uA, lx, ux, le)
    assert met["kkt_rel"] <= 1e-6


def test_bruteforce_catches_planted_sign_error(monkeypatch):
    """A planted mistake in the oracle (wrong sign of the A' lam term in r_H)
    must be caught by the brute-force pin."""
    qp = qpgen.tiny_qp(5, 3, 1, me=0)
    H = qp.H_dense()
    xs, _ = solve_bruteforce(H, qp.p, qp.A, qp.lA, qp.uA, qp.C, qp.b, qp.lx, qp.ux)
    orig = I._ATy

    def bad(S, yL, yU):
        return -orig(S, yL, yU)
    monkeypatch.setattr(I, "_ATy", bad)
    res = oracle.ipm_solve(qp, maxit=60)
    assert res.status != "converged" or np.max(np.abs(res.x - xs)) > 1e-4


# ---------------------------------------------------------------- reductions
@pytest.mark.parametrize("qp", _tiny_problems()[:6], ids=lambda q: f"seed{q.meta['seed']}")
def test_newton_formulations_agree(qp):
    """Eq. (7) (full, LU), Eq. (8) (LDL^T), Eq. (9) (Cholesky) and the Schur
    form give the same Newton direction at random interior iterates."""
    S = I.scale(qp)
    for seed in range(3):
        st = _random_interior_state(S, seed)
        mu = 10.0 ** -seed
        r = I.residuals(S, st, mu)
        J, off = I.full_newton_matrix(S, st, mu)
        sol = np.linalg.solve(J, I.full_newton_rhs(r))
        dx_full = sol[off[0]:off[1]]
        dl_full = np.concatenate([sol[off[5]:off[6]], sol[off[1]:off[2]], sol[off[2]:off[3]]])
        dg, D, r1, r2 = I.reduced_system(S, st, r, mu)
        dx1, dl1 = I.newton_direct(S, dg, D, r1, r2, "ldl")
        dx2, dl2 = I.newton_direct(S, dg, D, r1, r2, "schur_dense")
        K = I.doubly_augmented_matrix(S, dg, D)
        z = sla.cho_solve(sla.cho_factor(K), I.doubly_augmented_rhs(S, D, r1, r2))
        scale = 1 + np.max(np.abs(sol))
        for dx, dl in ((dx1, dl1), (dx2, dl2), (z[:S.n], z[S.n:])):
            assert np.max(np.abs(dx - dx_full)) <= 1e-9 * scale
            assert np.max(np.abs(dl - dl_full)) <= 1e-9 * scale
        # full-system slack / bound-multiplier parts equal the recovery formulas
        d = I.recover_step(S, st, r, dx1, dl1)
        for blk, key in ((6, "s_lA"), (7, "s_uA"), (8, "s_lx"), (9, "s_ux"),
                         (3, "lam_lx"), (4, "lam_ux")):
            assert np.max(np.abs(sol[off[blk]:off[blk + 1]] - d[key]), initial=0) <= 1e-8 * scale


def test_reduction_catches_planted_dropped_term(monkeypatch):
    """Dropping the S_lx^-1 r_c3 term of r1 (Eq. (8)) is caught by the
    comparison against the independently assembled Eq. (7)."""
    qp = qpgen.tiny_qp(5, 3, 2, me=0)
    S = I.scale(qp)
    st = _random_interior_state(S, 7)
    mu = 0.1
    r = I.residuals(S, st, mu)
    J, off = I.full_newton_matrix(S, st, mu)
    dx_full = np.linalg.solve(J, I.full_newton_rhs(r))[:S.n]
    orig = I.reduced_system

    def bad(S_, st_, r_, mu_):
        dg, D, r1, r2 = orig(S_, st_, r_, mu_)
        r1 = r1.copy()
        r1[S_.Lx] += r_["r_c3"] / st_.s_lx
        return dg, D, r1, r2
    monkeypatch.setattr(I, "reduced_system", bad)
    dg, D, r1, r2 = I.reduced_system(S, st, r, mu)
    dx, _ = I.newton_direct(S, dg, D, r1, r2, "ldl")
    assert np.max(np.abs(dx - dx_full)) > 1e-6


@pytest.mark.parametrize("seed", range(3))
def test_K_symmetric_positive_definite(seed):
    """Eq. (9) is SPD for convex problems (section 3.1)."""
    qp = qpgen.tiny_qp(6, 4, 300 + seed, me=1)
    S = I.scale(qp)
    st = _random_interior_state(S, seed)
    r = I.residuals(S, st, 1e-3)
    dg, D, _, _ = I.reduced_system(S, st, r, 1e-3)
    K = I.doubly_augmented_matrix(S, dg, D)
    assert np.allclose(K, K.T, atol=1e-13 * np.abs(K).max(), rtol=0)
    sla.cholesky(K)          # raises if not SPD
    assert np.min(np.linalg.eigvalsh(K)) > 0


@pytest.mark.parametrize("maker", [
    lambda: qpgen.tiny_qp(6, 4, 11, me=1),
    lambda: qpgen.dose_qp(300, 40, 8, 10, 12, seed=12),
    lambda: qpgen.svm_qp(60, 5, seed=13),
    lambda: qpgen.bfgs_qp(50, 6, 8, 7, seed=14),
], ids=["dense", "csr_lsq", "lowrank", "lowrank_weighted_diag"])
def test_matrix_free_apply_and_diag(maker):
    qp = maker()
    S = I.scale(qp)
    st = _random_interior_state(S, 3)
    r = I.residuals(S, st, 0.01)
    dg, D, _, _ = I.reduced_system(S, st, r, 0.01)
    K = I.doubly_augmented_matrix(S, dg, D)
    v = np.random.default_rng(0).standard_normal(K.shape[0])
    assert np.allclose(I.kkt_apply(S, dg, D, v), K @ v, rtol=1e-12, atol=1e-12 * np.abs(K).max())
    assert np.allclose(I.jacobi_diagonal(S, dg, D), np.diag(K), rtol=1e-12, atol=0)


@pytest.mark.parametrize("maker,solver", [
    (lambda: qpgen.dose_qp(600, 80, 12, 15, 30, seed=21), "schur_banded"),
    (lambda: qpgen.svm_qp(120, 6, seed=22), "schur_woodbury"),
    (lambda: qpgen.bfgs_qp(150, 7, 25, 9, seed=24), "schur_woodbury"),
    (lambda: qpgen.dense_qp(40, 20, seed=23), "schur_dense"),
])
def test_structured_direct_solvers(maker, solver):
    qp = maker()
    S = I.scale(qp)
    st = _random_interior_state(S, 5)
    r = I.residuals(S, st, 0.01)
    dg, D, r1, r2 = I.reduced_system(S, st, r, 0.01)
    dx0, dl0 = I.newton_direct(S, dg, D, r1, r2, "ldl")
    dx1, dl1 = I.newton_direct(S, dg, D, r1, r2, solver)
    sc = 1 + np.max(np.abs(np.concatenate([dx0, dl0])))
    assert np.max(np.abs(dx1 - dx0)) <= 1e-8 * sc
    assert np.max(np.abs(dl1 - dl0)) <= 1e-8 * sc


def test_pcg_reference_matches_direct():
    qp = qpgen.tiny_qp(6, 4, 31, me=1)
    S = I.scale(qp)
    st = _random_interior_state(S, 1)
    r = I.residuals(S, st, 0.1)
    dg, D, r1, r2 = I.reduced_system(S, st, r, 0.1)
    K = I.doubly_augmented_matrix(S, dg, D)
    rhs = I.doubly_augmented_rhs(S, D, r1, r2)
    z, it, tres = I.pcg_reference(lambda v: K @ v, rhs, np.diag(K), 1e-12, 500)
    zs = np.linalg.solve(K, rhs)
    assert tres <= 1e-11
    assert np.max(np.abs(z - zs)) <= 1e-9 * (1 + np.max(np.abs(zs)))


def test_ratio_test_closed_form():
    """Eq. (10) on hand-made values."""
    st = I.State(x=np.zeros(1), s_lA=np.array([1.0, 2.0]), s_uA=np.array([4.0]),
                 s_lx=np.zeros(0), s_ux=np.zeros(0), lam_e=np.zeros(0),
                 lam_lA=np.array([1.0, 1.0]), lam_uA=np.array([3.0]),
                 lam_lx=np.zeros(0), lam_ux=np.zeros(0))
    d = {"s_lA": np.array([-4.0, 1.0]), "s_uA": np.array([-2.0]), "s_lx": np.zeros(0),
         "s_ux": np.zeros(0), "lam_lA": np.array([0.5, 0.5]), "lam_uA": np.array([-1.0]),
         "lam_lx": np.zeros(0), "lam_ux": np.zeros(0)}
    ax, al = I.ratio_test(st, d, 0.99)
    assert ax == pytest.approx(0.99 * 0.25)
    assert al == 1.0        # 0.99 * 3 > 1
    d["s_lA"][:] = 1.0
    d["s_uA"][:] = 0.0
    ax, _ = I.ratio_test(st, d, 0.99)
    assert ax == 1.0        # empty set


# ---------------------------------------------------------------- adjoint
def test_adjoint_unconstrained_equals_minus_Hinv():
    qp = qpgen.dense_qp(20, 1, seed=41)
    qp.akind, qp.A, qp.lA, qp.uA = "none", None, None, None
    qp.lx = np.full(qp.n, -np.inf)
    qp.ux = np.full(qp.n, np.inf)
    res = oracle.ipm_solve(qp)
    g = np.random.default_rng(1).standard_normal(qp.n)
    adj = oracle.adjoint_solve(res.scaled, res.state, res.mu, g)
    ref = -np.linalg.solve(qp.H_dense(), g)
    assert np.max(np.abs(adj["p"] - ref)) <= 1e-9 * (1 + np.max(np.abs(ref)))


def test_adjoint_active_set_limit():
    """With a known active set the mu -> 0 derivative is -N (N'HN)^-1 N' g."""
    qp = qpgen.tiny_qp(5, 3, 2, me=0)
    res = oracle.ipm_solve(qp)
    H = qp.H_dense()
    x = res.x
    act = []
    for i in range(qp.m):
        v = qp.A[i] @ x
        if abs(v - qp.lA[i]) < 1e-5 or abs(v - qp.uA[i]) < 1e-5:
            act.append(qp.A[i])
    for j in range(qp.n):
        if abs(x[j] - qp.lx[j]) < 1e-5 or abs(x[j] - qp.ux[j]) < 1e-5:
            e = np.zeros(qp.n)
            e[j] = 1
            act.append(e)
    G = np.array(act).reshape(len(act), qp.n)
    N = sla.null_space(G) if len(act) else np.eye(qp.n)
    g = np.random.default_rng(3).standard_normal(qp.n)
    ref = -N @ np.linalg.solve(N.T @ H @ N, N.T @ g)
    adj = oracle.adjoint_solve(res.scaled, res.state, res.mu, g)
    assert np.max(np.abs(adj["p"] - ref)) <= 1e-4 * (1 + np.max(np.abs(ref)))


def test_adjoint_finite_differences():
    """dL/dp, dL/dlA, dL/duA against central differences of the IPM output."""
    qp = qpgen.tiny_qp(6, 3, 5, me=0)
    res = oracle.ipm_solve(qp)
    rng = np.random.default_rng(9)
    g = rng.standard_normal(qp.n)
    adj = oracle.adjoint_solve(res.scaled, res.state, res.mu, g)
    for _ in range(3):
        dp = rng.standard_normal(qp.n)
        dl = rng.standard_normal(qp.m)
        du = rng.standard_normal(qp.m)
        h = 1e-4
        vals = []
        for sgn in (1, -1):
            q2 = qpgen.tiny_qp(6, 3, 5, me=0)
            q2.p = qp.p + sgn * h * dp
            q2.lA = qp.lA + sgn * h * dl
            q2.uA = qp.uA + sgn * h * du
            vals.append(g @ oracle.ipm_solve(q2).x)
        fd = (vals[0] - vals[1]) / (2 * h)
        an = adj["p"] @ dp + adj["lA"] @ dl + adj["uA"] @ du
        assert abs(fd - an) <= 2e-3 * (1 + abs(an))


# ---------------------------------------------------------------- settings
def test_paper_settings_golden():
    gold = json.load(open(os.path.join(GOLD, "paper_settings.json")))
    import inspect
    sig = inspect.signature(oracle.ipm_solve)
    assert sig.parameters["gamma"].default == gold["gamma"]["value"]
    assert sig.parameters["mu_tol"].default == gold["mu_tol"]["value"]
    assert sig.parameters["pcg_tol"].default == gold["pcg_tol"]["value"]
    assert sig.parameters["pcg_maxit"].default == gold["pcg_maxit"]["value"]
    # Table 2 rows: parts add up to the total within the printed rounding
    for row in gold["profiling_seconds"]["rows"]:
        assert abs(sum(row[2:]) - row[1]) <= 0.01 * row[1] + 0.01


def test_config0_converges_and_mu_rule():
    """Config-0 run: converges, mu ends at 1e-7 (mu_tol 1e-6, strict test),
    PCG-mode oracle reaches the same objective, and CG iterations grow as mu
    decreases (section 5.1)."""
    qp = qpgen.config0()
    res = oracle.ipm_solve(qp, log=True)
    assert res.status == "converged" and res.mu == pytest.approx(1e-7)
    lA, uA, lx, ux, le = full_multipliers(res.scaled, res.lam, qp)
    assert oracle.kkt_metrics(qp, res.x, lA, uA, lx, ux, le)["kkt_rel"] <= 1e-6
    res2 = oracle.ipm_solve(qp, solver="pcg", log=True)
    assert res2.status == "converged"
    assert abs(qp.objective(res.x) - qp.objective(res2.x)) <= 1e-6 * (1 + abs(qp.objective(res.x)))
    its = [h["pcg_iters"] for h in res2.log]
    assert np.mean(its[-4:]) > 5 * np.mean(its[:4])


def test_metrics_flag_bad_solution():
    qp = qpgen.config0()
    res = oracle.ipm_solve(qp)
    lA, uA, lx, ux, le = full_multipliers(res.scaled, res.lam, qp)
    good = oracle.kkt_metrics(qp, res.x, lA, uA, lx, ux, le)
    bad = oracle.kkt_metrics(qp, res.x + 1e-3, lA, uA, lx, ux, le)
    assert good["kkt_rel"] <= 1e-6 < bad["kkt_rel"]


# ---------------------------------------------------------------- hand-computed worked examples
def _worked_qp():
    """n = 2, one two-sided general row (norm 5), one equality row (norm 2),
    x1 in [-1, 1], x2 >= 0.  max H_ii = 0.5 and |p|_inf = 0.5, so the
    objective scale sigma is 1; the rows are divided by 5 and by 2."""
    return qpgen.QPData(n=2, hkind="dense", p=np.array([0.5, -0.25]),
                        H=np.array([[0.5, 0.0], [0.0, 0.25]]), akind="dense",
                        A=np.array([[3.0, 4.0]]), lA=np.array([-5.0]), uA=np.array([10.0]),
                        C=np.array([[0.0, 2.0]]), b=np.array([2.0]),
                        lx=np.array([-1.0, 0.0]), ux=np.array([1.0, np.inf]))


def _worked_state():
    """Scaled units.  x = (0.5, 1); row slacks 1.5 / 0.5 with multipliers 2 / 1;
    bound slacks (1, 2) on the lower bounds of x1, x2 and 0.25 on the upper
    bound of x1, with multipliers (0.5, 0.25) and 4; lam_e = 0.5."""
    return I.State(x=np.array([0.5, 1.0]), s_lA=np.array([1.5]), s_uA=np.array([0.5]),
                   s_lx=np.array([1.0, 2.0]), s_ux=np.array([0.25]), lam_e=np.array([0.5]),
                   lam_lA=np.array([2.0]), lam_uA=np.array([1.0]),
                   lam_lx=np.array([0.5, 0.25]), lam_ux=np.array([4.0]))


# Every block of the right-hand side of Eq. (7) for the worked example at
# mu = 0.1, worked out by hand from Eq. (3) (readings R1: r_uA = -Ax - s_u + u,
# r_c2 = lam_u s_u - mu, stationarity term -C' lam_e):
#   scaled A x = 0.6*0.5 + 0.8*1 = 1.1;  H x + p = (0.75, 0);  A'(lam_l - lam_u) = (0.6, 0.8)
#   r_H  = (0.75 - 0.6 - 0 - 0.5 + 4,  0 - 0.8 - 0.5 - 0.25) = (3.65, -1.55)
#   r_e  = 1 - 1 + 0.1*0.5 = 0.05
#   r_lA = 1.1 - 1.5 + 1 = 0.6          r_uA = -1.1 - 0.5 + 2 = 0.4
#   r_lx = (0.5 - 1 + 1, 1 - 2 - 0) = (0.5, -1)     r_ux = -0.5 - 0.25 + 1 = 0.25
#   r_c1 = 2*1.5 - 0.1 = 2.9            r_c2 = 1*0.5 - 0.1 = 0.4
#   r_c3 = (0.5 - 0.1, 0.5 - 0.1)       r_c4 = 4*0.25 - 0.1 = 0.9
# sum of squares = 15.725 + 0.0025 + 0.36 + 0.16 + 1.25 + 0.0625 + 8.41 + 0.16 + 0.32 + 0.81
#                = 27.26
WORKED_BLOCKS = {"r_H": [3.65, -1.55], "r_e": [0.05], "r_lA": [0.6], "r_uA": [0.4],
                 "r_lx": [0.5, -1.0], "r_ux": [0.25], "r_c1": [2.9], "r_c2": [0.4],
                 "r_c3": [0.4, 0.4], "r_c4": [0.9]}
WORKED_NORM2 = 27.26


def _residual_norm_pinned(norm_fn, resid_fn):
    S = I.scale(_worked_qp())
    assert S.sigma == 1.0
    r = resid_fn(S, _worked_state(), 0.1)
    blocks_ok = all(np.allclose(r[k], v, rtol=0, atol=1e-14) for k, v in WORKED_BLOCKS.items())
    return blocks_ok and abs(norm_fn(r) - np.sqrt(WORKED_NORM2)) <= 1e-13


def test_residual_norm_worked_example():
    """R8: ||r||_2 over all ten blocks of Eq. (7) at the current mu, on a
    worked example computed by hand (including the row and equality scaling
    of R9)."""
    assert _residual_norm_pinned(I.residual_norm, I.residuals)


def test_residual_norm_pin_catches_planted_mistakes():
    """Plausible mistakes in the residual norm or in the blocks it sums are
    caught by the worked example: complementarity blocks dropped, mu left out
    of r_c, the penalty term mu*lam_e dropped from r_e, the r_uA slack sign of
    the printed Eq. (3)."""
    def drop_compl(r):
        return float(np.sqrt(sum(float(r[k] @ r[k]) for k in I.RES_KEYS[:6])))

    def resid_no_mu(S, st, mu):
        return I.residuals(S, st, 0.0)

    def resid_no_penalty(S, st, mu):
        r = I.residuals(S, st, mu)
        r["r_e"] = r["r_e"] - mu * st.lam_e
        return r

    def resid_printed_sign(S, st, mu):
        r = I.residuals(S, st, mu)
        r["r_uA"] = r["r_uA"] + 2.0 * st.s_uA
        return r
    assert not _residual_norm_pinned(drop_compl, I.residuals)
    for bad in (resid_no_mu, resid_no_penalty, resid_printed_sign):
        assert not _residual_norm_pinned(I.residual_norm, bad)


def _ip_qp():
    """Four variables with every bound pattern: [-1, 3] (midpoint 1), [2, inf)
    (2 + 1), (-inf, 5] (5 - 1), free (0), plus [-0.25, 0.25] (midpoint 0, gap
    below 2 so both slacks are clipped to 1).  Rows (original units):
    a1 = e1 with lA = -2; a2 = (0, 0, 3, 0, 4, ...) / norm 5 with lA = 10 (scaled 2)
    and uA = 50 (scaled 10); a3 = (0, 4, 0, 3, 0) norm 5 with uA = 14.5 (scaled 2.9).
    One equality row."""
    n = 5
    A = np.array([[1.0, 0, 0, 0, 0], [0, 0, 3.0, 0, 4.0], [0, 4.0, 0, 3.0, 0]])
    return qpgen.QPData(n=n, hkind="dense", p=np.zeros(n), H=np.eye(n), akind="dense", A=A,
                        lA=np.array([-2.0, 10.0, -np.inf]), uA=np.array([np.inf, 50.0, 14.5]),
                        C=np.array([[1.0, 1.0, 1.0, 1.0, 1.0]]), b=np.array([0.0]),
                        lx=np.array([-1.0, 2.0, -np.inf, -np.inf, -0.25]),
                        ux=np.array([3.0, np.inf, 5.0, np.inf, 0.25]))


# R6 by hand for _ip_qp: x0 = (1, 3, 4, 0, 0).  Scaled row values at x0:
#   a1: 1 (lower -2: slack max(3, 1) = 3)
#   a2: (3*4 + 4*0)/5 = 2.4 (lower 2: max(0.4, 1) = 1; upper 10: max(7.6, 1) = 7.6)
#   a3: (4*3 + 3*0)/5 = 2.4 (upper 2.9: max(0.5, 1) = 1)
# bound slacks: lower bounds of x1, x2, x5: max(2, 1), max(1, 1), max(0.25, 1);
# upper bounds of x1, x3, x5: max(2, 1), max(1, 1), max(0.25, 1)
IP_EXPECT = {"x": [1.0, 3.0, 4.0, 0.0, 0.0], "s_lA": [3.0, 1.0], "s_uA": [7.6, 1.0],
             "s_lx": [2.0, 1.0, 1.0], "s_ux": [2.0, 1.0, 1.0], "lam_lA": [1.0, 1.0],
             "lam_uA": [1.0, 1.0], "lam_lx": [1.0, 1.0, 1.0], "lam_ux": [1.0, 1.0, 1.0],
             "lam_e": [0.0]}


def _initial_point_pinned(fn):
    st = fn(I.scale(_ip_qp()))
    return all(np.shape(getattr(st, k)) == np.shape(v)
               and np.allclose(getattr(st, k), v, rtol=0, atol=1e-14) for k, v in IP_EXPECT.items())


def test_initial_point_worked_example():
    """R6 on a worked example with every bound pattern, computed by hand."""
    assert _initial_point_pinned(I.initial_point)


def test_initial_point_pin_catches_planted_mistakes():
    """A slack without the max(., 1) clip, l + 1 used for a two-sided bound,
    and unit multipliers on absent bounds all fail the worked example."""
    def no_clip(S):
        st = I.initial_point(S)
        Ax = S.A @ st.x
        st.s_lA = Ax[S.L] - S.lA[S.L]
        return st

    def lower_plus_one(S):
        st = I.initial_point(S)
        both = np.isfinite(S.lx) & np.isfinite(S.ux)
        st.x = st.x.copy()
        st.x[both] = S.lx[both] + 1.0
        return st

    def all_multipliers(S):
        st = I.initial_point(S)
        st.lam_lx = np.ones(S.n)
        return st
    for bad in (no_clip, lower_plus_one, all_multipliers):
        assert not _initial_point_pinned(bad)


def test_duality_gap_is_primal_minus_dual_objective():
    """The reported gap equals f(x) - g(lam) + x'r_H, with the Lagrangian dual
    function of Eq. (1) written out: g = -1/2 x'Hx + lam_lA'lA - lam_uA'uA +
    lam_lx'lx - lam_ux'ux + lam_e'b (at x satisfying stationarity up to r_H)."""
    qp = qpgen.tiny_qp(5, 3, 7, me=1)
    res = oracle.ipm_solve(qp)
    lA, uA, lx, ux, le = full_multipliers(res.scaled, res.lam, qp)
    x = res.x
    H = qp.H_dense()
    met = oracle.kkt_metrics(qp, x, lA, uA, lx, ux, le)
    rH = H @ x + qp.p - qp.A.T @ (lA - uA) - (lx - ux) - qp.C.T @ le
    f = 0.5 * x @ H @ x + qp.p @ x
    g = -0.5 * x @ H @ x + lA @ qp.lA - uA @ qp.uA + lx @ qp.lx - ux @ qp.ux + le @ qp.b
    assert met["gap"] == pytest.approx(f - g + x @ rH, rel=1e-10, abs=1e-12)
    # converged: the gap is of the order of the final barrier parameter
    assert 0.0 < met["gap"] < 1e-5


def test_jacobi_scaled_eigenvalues_closed_form():
    """[[4, 2], [2, 1 + 1e-2]] scaled by its diagonal is [[1, c], [c, 1]] with
    c = 2 / sqrt(4 (1.01)): eigenvalues 1 -+ c (section 5.3's conditioning of
    the Jacobi-preconditioned system)."""
    K = np.array([[4.0, 2.0], [2.0, 1.01]])
    c = 2.0 / np.sqrt(4.0 * 1.01)
    ev = I.jacobi_scaled_eigenvalues(K)
    assert np.allclose(ev, [1 - c, 1 + c], rtol=1e-13, atol=0)
    # a diagonal K is perfectly conditioned after Jacobi scaling
    assert np.allclose(I.jacobi_scaled_eigenvalues(np.diag([1e-8, 3.0, 1e9])), 1.0)


def test_weighted_lowrank_unconstrained_closed_form():
    """H = H0 + U W U' (section 2.1's quasi-Newton form), no constraints or
    bounds: x* = -H^-1 p with H assembled explicitly from its definition."""
    qp = qpgen.bfgs_qp(60, 5, 0, seed=15)
    qp.lx = np.full(qp.n, -np.inf)
    qp.ux = np.full(qp.n, np.inf)
    U = qp.Z.astype(np.float64)
    H = np.diag(qp.d0) + U @ np.diag(qp.zw) @ U.T
    res = oracle.ipm_solve(qp)
    xstar = -np.linalg.solve(H, qp.p)
    assert res.status == "converged"
    assert np.max(np.abs(res.x - xstar)) <= 1e-10 * (1 + np.max(np.abs(xstar)))


def test_infeasibilities_split_the_residual_norm():
    """Section 5.2's primal, dual and complementarity infeasibilities cover
    the ten blocks of Eq. (7) between them: on the hand-worked example,
    primal^2 = r_e^2 + r_lA^2 + r_uA^2 + r_lx^2 + r_ux^2 = 0.0025 + 0.36 +
    0.16 + 1.25 + 0.0625, dual^2 = |r_H|^2 = 15.725, compl^2 = 8.41 + 0.16 +
    0.32 + 0.81."""
    S = I.scale(_worked_qp())
    r = I.residuals(S, _worked_state(), 0.1)
    pr, du, co = I.infeasibilities(r)
    assert pr ** 2 == pytest.approx(1.835, rel=1e-13)
    assert du ** 2 == pytest.approx(15.725, rel=1e-13)
    assert co ** 2 == pytest.approx(9.7, rel=1e-13)
    assert pr ** 2 + du ** 2 + co ** 2 == pytest.approx(WORKED_NORM2, rel=1e-13)


def test_rbf_hessian_library_distances_and_invariants():
    """The Gaussian-kernel Hessian of the SVM dual (Eq. (6)): squared
    distances from scipy's cdist agree; a hand case (|x1 - x2|^2 = 25,
    gamma = 0.02, labels +-1) gives H12 = -exp(-0.5); H is symmetric positive
    semidefinite with unit diagonal (y_i^2 exp(0))."""
    from scipy.spatial.distance import cdist
    H2 = oracle.rbf_hessian(np.array([[0.0, 0.0], [3.0, 4.0]]), np.array([1.0, -1.0]), 0.02)
    assert H2[0, 1] == pytest.approx(-np.exp(-0.5), rel=1e-15)
    assert H2[1, 0] == H2[0, 1] and H2[0, 0] == 1.0 and H2[1, 1] == 1.0
    qp = qpgen.rbf_svm_qp(150, 7, seed=3)
    H = oracle.rbf_hessian(qp.X, qp.y, qp.gamma)
    Hl = np.exp(-qp.gamma * cdist(qp.X, qp.X, "sqeuclidean")) * np.outer(qp.y, qp.y)
    assert np.max(np.abs(H - Hl)) <= 1e-13
    assert np.array_equal(H, H.T) and np.all(np.diag(H) == 1.0)
    assert np.min(np.linalg.eigvalsh(H)) >= -1e-10
    # the generator's own Gram-form matrix (used for objectives) agrees too
    assert np.max(np.abs(H - qp.H_dense())) <= 1e-12


def test_rbf_svm_two_samples_closed_form():
    """Two samples of opposite labels at distance r: y'a = 0 forces
    a1 = a2 = a and the dual objective is a^2 (1 - k) - 2a with
    k = exp(-gamma r^2), so a* = 1 / (1 - k) while the box is inactive."""
    gamma, r = 1.0, 1.0
    y = np.array([1.0, -1.0])
    qp = qpgen.QPData(n=2, hkind="rbf", p=np.full(2, -1.0), X=np.array([[0.0], [r]]), y=y,
                      gamma=gamma, akind="none", C=y[None, :].copy(), b=np.zeros(1),
                      lx=np.zeros(2), ux=np.full(2, 10.0))
    res = oracle.ipm_solve(qp)
    astar = 1.0 / (1.0 - np.exp(-gamma * r * r))
    assert res.status == "converged"
    assert np.max(np.abs(res.x - astar)) <= 1e-5 * astar
    assert qp.objective(res.x) == pytest.approx(-astar, rel=1e-6)
