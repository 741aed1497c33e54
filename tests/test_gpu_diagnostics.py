"""Per-IPM-iteration records (opts.record = 1): CG iterations per Newton
solve (section 5.1), the primal / dual / complementarity infeasibilities
(section 5.2) and the conditioning of the Jacobi-preconditioned doubly
augmented system from the PCG coefficients (section 5.3), against the oracle
on the same iterate."""
import numpy as np
import pytest

import oracle
import qpgen
from oracle import ipm as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kq():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as m
    m.load()
    return m


def test_first_iteration_record_against_oracle(kq):
    qp = qpgen.tiny_qp(37, 23, 5, me=2)
    h = kq.create_from(qp)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(ipm_maxit=1, record=1, pcg_tol=1e-12,
                                                 pcg_maxit=20000),
                          allow=(kq.KQ_ERR_IPM_MAXIT,))
    log = kq.qp_iteration_log(h)
    assert len(log) == 1
    r0 = log[0]
    # the Newton system of the first iteration, from the oracle
    S = I.scale(qp)
    st0 = I.initial_point(S)
    res = I.residuals(S, st0, 1.0)
    dg, D, _, _ = I.reduced_system(S, st0, res, 1.0)
    K = I.doubly_augmented_matrix(S, dg, D)
    ev = I.jacobi_scaled_eigenvalues(K)
    d = np.diag(K)
    print(r0, "true extremes", ev[0], ev[-1])
    assert r0["diag_ratio"] == pytest.approx(d.max() / d.min(), rel=1e-12)
    # Ritz values lie inside the spectrum and, after a pass run to 1e-12, are
    # close to its ends
    assert ev[0] * (1 - 1e-9) <= r0["lanczos_min"] <= ev[0] * 1.05
    assert ev[-1] * (1 - 1e-4) <= r0["lanczos_max"] <= ev[-1] * (1 + 1e-9)
    assert r0["kappa_jacobi"] == pytest.approx(r0["lanczos_max"] / r0["lanczos_min"])
    # the oracle's first iteration: same step up to the PCG tolerance
    first = next(oracle.ipm_iterate(qp))
    assert r0["res_norm"] == pytest.approx(first["res"], rel=1e-6)
    assert r0["alpha_x"] == pytest.approx(first["alpha_x"], rel=1e-6)
    assert r0["alpha_lam"] == pytest.approx(first["alpha_lam"], rel=1e-6)
    # section 5.2 norms: the oracle's infeasibilities after its first step
    S2 = I.scale(qp)
    stx = I.initial_point(S2)
    r = I.residuals(S2, stx, 1.0)
    dg, D, r1, r2 = I.reduced_system(S2, stx, r, 1.0)
    dx, dl = I.newton_direct(S2, dg, D, r1, r2)
    dd = I.recover_step(S2, stx, r, dx, dl)
    ax, al = I.ratio_test(stx, dd)
    st1 = I.apply_step(stx, dd, ax, al)
    pr, du, co = I.infeasibilities(I.residuals(S2, st1, 1.0))
    assert r0["primal_inf"] == pytest.approx(pr, rel=1e-6)
    assert r0["dual_inf"] == pytest.approx(du, rel=1e-6, abs=1e-9)
    assert r0["compl_inf"] == pytest.approx(co, rel=1e-6)
    kq.qp_destroy(h)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "mixed"])
def test_full_solve_records(kq, prec):
    """One record per IPM iteration; their CG counts add up to the solve's;
    mu follows the rule of Algorithm 1; the Jacobi-scaled system gets worse
    conditioned as mu decreases (section 5.3)."""
    qp = qpgen.config0()
    h = kq.create_from(qp)
    rc, st = kq.ipm_solve(h, kq.default_ipm_opts(precision=prec, record=1))
    log = kq.qp_iteration_log(h)
    assert rc == kq.KQ_OK and len(log) == st.ipm_iters
    assert sum(r["pcg_iters"] for r in log) == st.pcg_iters
    mus = [r["mu"] for r in log]
    assert mus[0] == 1.0 and all(b <= a for a, b in zip(mus, mus[1:]))
    assert all(r["lanczos_steps"] > 0 and r["lanczos_min"] > 0 for r in log)
    assert log[-1]["kappa_jacobi"] > 10 * log[0]["kappa_jacobi"]
    assert log[-1]["pcg_iters"] > log[0]["pcg_iters"]
    kq.qp_destroy(h)
