"""Plain FP64 CPU oracle for the Krylov interior point method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library and
its Python binding) may import, call or link anything in this package; only
the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.

The oracle runs the same interior point iteration as the GPU library
(Algorithm 1 of Liu, Fredriksson and Markidis, "Krylov Solvers for Interior
Point Methods with Applications in Radiation Therapy and Support Vector
Machines", arXiv 2308.00637) but solves every Newton system *directly*
(LAPACK LDL^T / Cholesky), in float64, with no blocking or fusion beyond what
the equations state.  It shares no code with the GPU path.
"""
from .ipm import (  # noqa: F401
    Scaled, State, scale, initial_point, residuals, residual_norm, reduced_system,
    doubly_augmented_matrix, doubly_augmented_rhs, kkt_apply, jacobi_diagonal,
    full_newton_matrix, newton_direct, recover_step, ratio_test, ipm_solve, ipm_iterate,
    pcg_reference, adjoint_solve, unscale_solution, IpmResult, jacobi_scaled_eigenvalues,
    rbf_hessian,
)
from .metrics import kkt_metrics, objective, full_multipliers  # noqa: F401
