"""GB300 solver for the implicit Runge-Kutta stage system of P1 parabolic
problems, preconditioned by block Jacobi / Gauss-Seidel / optimised
Gauss-Seidel / the LDU-based P_DU and P_LD with one AMG V-cycle per
diagonal block (Rana, Howle, Long, Meek, Milestone, arXiv:2010.11377).

The compute path is libirk.so (hand-written CUDA for sm_103a behind the C ABI
of include/irk.h); this package is its Python binding."""

from .binding import (  # noqa: F401
    Batch, Context, irk_adjoint_run, irk_adjoint_step, irk_amg_aggregates, irk_amg_info,
    irk_amg_level_matrix, irk_apply_mass, irk_apply_operator, irk_apply_operator_f32, irk_apply_precond,
    irk_atilde, irk_batch_adjoint, irk_batch_create, irk_batch_destroy, irk_batch_run, irk_butcher_table,
    irk_default_options, irk_destroy, irk_fem_assemble, irk_fem_assemble_p2, irk_fem_assemble_supg,
    irk_fem_quad_points, irk_kernel_launches, irk_ldu, irk_profile, irk_residual_norm,
    irk_residual_norm_noalloc, irk_run, irk_set_kappa, irk_setup, irk_solve, irk_step, irk_vcycle,
)
