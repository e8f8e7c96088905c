/*
 * irk.h -- C ABI of the GB300 solver for the implicit Runge-Kutta stage system
 *
 *     (I_s (x) M + h_t A (x) F) k = r,        r = -(1_s (x) (F u_n + g))
 *
 * of a P1 finite-element parabolic problem (Section 3, Eq. block_coeff_mtx and
 * Section 4 of Rana, Howle, Long, Meek, Milestone, "A new block preconditioner
 * for implicit Runge-Kutta methods for parabolic PDE problems").  The system is
 * solved by right-preconditioned restarted flexible GMRES with the block
 * preconditioners P = I_s (x) M + h_t A~ (x) F of Eq. PrecForm (block Jacobi,
 * block Gauss-Seidel, optimised block Gauss-Seidel of Eq. GSLopt, and the LDU
 * based P_DU / P_LD of Eq. PLDandPDU), each diagonal-block subsolve being one
 * smoothed-aggregation AMG V-cycle (Section 4.2).
 *
 * Conventions for every entry point
 *  - Arguments named d_* are DEVICE pointers (CUDA global memory on the device
 *    that was current at irk_setup), caller-owned, FP64, contiguous.  Stage
 *    blocks are s x n, stage-major: entry (i, r) at [i*n + r], i.e. the block
 *    vector [K_1; ...; K_s] of the paper.  The library never frees them.
 *  - All other pointers are HOST memory, caller-owned, read during the call
 *    (or written, for outputs) and not retained.
 *  - The context owns all internal device memory; irk_destroy frees it.
 *  - Work is ordered after all prior work on the stream given to irk_setup and
 *    the call returns after its work is complete (it synchronises), except
 *    where stated.
 *  - No C++ exception crosses the ABI.  On failure an irk_status other than
 *    IRK_OK is returned and irk_last_error() describes it.  A NULL context
 *    pointer gives IRK_ERR_INVALID.
 */
#ifndef IRK_H
#define IRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IRK_OK = 0,
  IRK_ERR_INVALID = 1,       /* bad argument: sizes, NULL pointer, s out of range */
  IRK_ERR_NOMEM = 2,         /* device allocation failed */
  IRK_ERR_CUDA = 3,          /* CUDA runtime error */
  IRK_ERR_NOT_CONVERGED = 4, /* FGMRES reached max_it above rtol; outputs hold the last iterate */
  IRK_ERR_BREAKDOWN = 5,     /* Arnoldi breakdown above the tolerance */
  IRK_ERR_ZERO_PIVOT = 6,    /* LDU without pivoting met a zero leading minor, or a singular coarse matrix */
  IRK_ERR_NONFINITE = 7,     /* NaN or Inf in a residual norm */
  IRK_ERR_TIMEOUT = 8,       /* a bounded device-side wait expired */
  IRK_ERR_CAPACITY = 9       /* a fixed capacity was exceeded (stated in the message) */
} irk_status;

/* Preconditioner coefficient matrix A~ (Eq. PrecForm).                       */
enum {
  IRK_PC_J = 0,       /* diag(A): block Jacobi                                  */
  IRK_PC_GSL = 1,     /* tril(A): block Gauss-Seidel (forward substitution)     */
  IRK_PC_GSL_OPT = 2, /* optimised lower triangular A~ of Eq. GSLopt            */
  IRK_PC_DU = 3,      /* D U of A = L D U (Section 4.1): backward substitution  */
  IRK_PC_LD = 4,      /* L D of A = L D U: forward substitution (the paper's P_LD) */
  IRK_PC_CUSTOM = 5   /* caller-given A~: diagonal, lower or upper triangular   */
};

/* Arithmetic of the AMG hierarchies and V-cycles.  The FGMRES basis, the true
 * residual and the solution update are always FP64; the operator on FP32
 * preconditioner outputs runs in single-float pairs (irk_apply_operator_f32). */
enum { IRK_AMG_F64 = 64, IRK_AMG_F32 = 32, IRK_AMG_BF16 = 16 /* BF16 finest matrix, FP32 elsewhere */ };

enum { IRK_SMOOTH_L1JACOBI = 0, IRK_SMOOTH_CHEBYSHEV = 1 };
/* AMG cycle of one subsolve: the V-cycle (Section 4.2), or the same finest-level
 * visit with a W-cycle below it (every level l >= 1 whose next level is not the
 * coarsest corrects twice) */
enum { IRK_CYCLE_V = 0, IRK_CYCLE_W_COARSE = 1 };

enum { IRK_METHOD_RADAU_IIA = 0, IRK_METHOD_LOBATTO_IIIC = 1 };

typedef struct {
  int32_t n;             /* rows = columns */
  int64_t nnz;
  const int64_t* rowptr; /* n + 1 */
  const int32_t* col;    /* nnz, strictly increasing within each row */
  const double* val;     /* nnz */
} irk_csr;               /* host CSR, copied by the call that takes it */

typedef struct {
  int32_t s;             /* 1 <= s <= 8 */
  const double* A;       /* s*s row-major Butcher matrix */
  const double* b;       /* s */
  const double* c;       /* s */
} irk_butcher;

typedef struct {
  int32_t kind;          /* IRK_PC_* */
  const double* Atilde;  /* s*s row-major, required for IRK_PC_CUSTOM, else ignored */
  int32_t amg_prec;      /* IRK_AMG_F64 / _F32 / _BF16 */
  int32_t smoother;      /* IRK_SMOOTH_* */
  int32_t cheb_degree;   /* Chebyshev polynomial degree per sweep (1..16) */
  double cheb_lo;        /* lower end of the Chebyshev interval [lo, 1] of D_l1^{-1} A, 0 < lo < 1 */
  int32_t nu_pre, nu_post; /* V(nu_pre, nu_post) sweeps */
  double theta;          /* strength threshold, 0 <= theta <= 1 */
  int32_t coarse_max;    /* coarsest level has at most this many rows (<= 2048) */
  int32_t max_levels;    /* 1..16 */
  int32_t restart;       /* FGMRES restart length m (1..64) */
  double rtol;           /* stop when ||b - A k||_2 <= rtol ||b||_2 */
  int32_t max_it;        /* total inner iterations per solve */
  int32_t reorth;        /* 0: classical Gram-Schmidt with a second pass when the projected
                            norm drops below reorth_eta of its value; 1: always twice */
  double reorth_eta;     /* 0 <= reorth_eta < 1; 0: never a second pass.  Default 0.1: one
                            classical pass loses at most about eps/reorth_eta of orthogonality
                            per vector, so a second pass is taken only on heavy cancellation */
  int32_t side;          /* 0: right-preconditioned flexible GMRES, stop on the true residual
                            (default); 1: left-preconditioned GMRES on P^{-1} A k = P^{-1} b
                            (the left-preconditioned runs of Section 5), stop on the
                            preconditioned residual ||P^{-1}(b - A k)|| <= rtol ||P^{-1} b||.
                            Left preconditioning needs a fixed linear P^{-1}: use FP64 AMG for
                            rtol below the AMG precision.  Forward solves only: the adjoint
                            entry points and batches reject side = 1 */
  int32_t p_smooth;      /* damped-Jacobi steps smoothing the tentative prolongator on
                            every level, P = (I - omega D^{-1} A)^p_smooth P_t, 1, 2 or 3
                            (default 2); omega = 4/(3 rho), rho a 20-step power-iteration
                            estimate of the spectral radius of D^{-1} A */
  int32_t strength;      /* coupling measure of the strength test (c_ij + c_ji)/2 >= theta
                            sqrt(|a_ii a_jj|): 0 = |a_ij| (default), 1 = max(-a_ij, 0);
                            the negative-only measure helps P2 heat blocks but can leave a
                            convection-dominated block without strong couplings (no
                            coarsening) */
  int32_t cycle;         /* IRK_CYCLE_V (default): one V(nu_pre, nu_post) cycle per subsolve.
                            IRK_CYCLE_W_COARSE: the finest level is visited once, as in the
                            V-cycle; every coarser level l >= 1 whose next level is not the
                            coarsest applies the coarse-grid correction (residual,
                            restriction, recursion, prolongation) twice between its pre- and
                            post-smoothing.  It keeps the subsolve's contraction at the
                            two-grid rate on stiffness-dominated blocks (large h_t / h_x^2),
                            where the V-cycle's rate degrades with the number of levels; it
                            costs one more pass over levels 2.. per subsolve */
} irk_options;

typedef struct {
  int32_t iterations;      /* FGMRES inner iterations (summed over the steps of the call) */
  int32_t restarts;        /* restart cycles (summed) */
  int32_t max_step_iterations; /* largest per-step iteration count of the call */
  int32_t steps;           /* time steps taken by the call */
  double resid;            /* true relative residual ||b - A k|| / ||b|| of the last solve */
  double ms;               /* device time of the call's work (CUDA events) */
} irk_stats;

typedef struct irk_ctx irk_ctx;

/* ------------------------------------------------------------------------- *
 * Host-side tables (no device work).                                         *
 * ------------------------------------------------------------------------- */

/* Butcher table of an s-stage method (Section 2, Table 1).  Radau IIA: nodes
 * are the zeros of P_s(2x-1) - P_{s-1}(2x-1), a_ij = int_0^{c_i} l_j, b_j =
 * int_0^1 l_j (collocation).  Lobatto IIIC: Lobatto nodes, a_i1 = b_1 and the
 * simplifying conditions C(s-1).  A is written s*s row-major, b and c s each.
 * IRK_ERR_INVALID for s outside 1..8 (2..8 for Lobatto IIIC). */
irk_status irk_butcher_table(int32_t method, int32_t s, double* A, double* b, double* c);

/* A = L D U without pivoting (Section 4.1).  L, U s*s row-major unit
 * triangular, D the s pivots.  IRK_ERR_ZERO_PIVOT if a leading minor is 0. */
irk_status irk_ldu(int32_t s, const double* A, double* L, double* D, double* U);

/* The preconditioner coefficient matrix A~ of Eq. PrecForm for `kind`
 * (IRK_PC_J .. IRK_PC_LD), s*s row-major.  IRK_PC_GSL_OPT solves Eq. GSLopt
 * (minimum 2-norm condition number of A~^{-1} A over lower triangular A~ with
 * diag(A~) = diag(A)) by Nelder-Mead from tril(A); `kappa` (may be NULL)
 * receives kappa_2(A~^{-1} A). */
irk_status irk_atilde(int32_t kind, int32_t s, const double* A, double* Atilde, double* kappa);

/* Fill *opt with the defaults: P_LD, FP32 AMG, Chebyshev degree 4 on [0.1, 1],
 * V(1,1), theta 0.08, coarse_max 2048, 12 levels, FGMRES(30), rtol 1e-10,
 * max_it 1000, selective reorthogonalisation (reorth_eta 0.1), right preconditioning,
 * two prolongator smoothing steps, strength from |a_ij|, the V-cycle. */
void irk_default_options(irk_options* opt);

/* ------------------------------------------------------------------------- *
 * P1 / P2 finite elements (Sections 3 and 5), host side.                     *
 * ------------------------------------------------------------------------- */

/* Physical coordinates of the 6 quadrature points per triangle at which
 * irk_fem_assemble reads the wind (the symmetric degree-4 rule of Dunavant,
 * 1985).  xq: n_tri*6*2 doubles (x, y per point). */
irk_status irk_fem_quad_points(int32_t n_tri, const double* xy, const int32_t* tri, double* xq);

/* Assemble the interior-unknown matrices of one problem.
 *   M_kl = int phi_k phi_l
 *   F    = sum_e kappa_e K_e + C,   K_e[a,b] = |T| grad l_a . grad l_b,
 *          C_kl = int phi_k (w . grad phi_l)   (omitted when wind == NULL)
 * kappa: n_tri per-element diffusion (NULL = 1).  wind: n_tri*6*2 wind
 * values at the points of irk_fem_quad_points.  dof: n_nodes, interior index
 * 0..n-1 or -1 for a Dirichlet node.  ub: n_nodes Dirichlet values (NULL = 0).
 * Outputs: M and F share one pattern; call once with val arrays NULL to get
 * *nnz (rowptr/col then also NULL), then with arrays of that size.  g (n):
 * the lift F_IB u_B.  Triangles must be counter-clockwise. */
irk_status irk_fem_assemble(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri,
                            const int32_t* dof, int32_t n, const double* kappa, const double* wind,
                            const double* ub, int64_t* nnz, int64_t* rowptr, int32_t* col,
                            double* valM, double* valF, double* g);

/* Quadratic (6-node) triangles for the heat problem, the discretisation of
 * the paper's heat runs (Section 5): M_kl = int phi_k phi_l, F = sum_e
 * kappa_e K_e with K_e the P2 stiffness.  tri6: n_tri*6 node indices per
 * triangle, vertices counter-clockwise then the midpoints of edges ab, bc,
 * ca (the vertices give the affine map).  Other arguments, the size query
 * and the outputs as irk_fem_assemble (no wind). */
irk_status irk_fem_assemble_p2(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri6,
                               const int32_t* dof, int32_t n, const double* kappa, const double* ub, int64_t* nnz,
                               int64_t* rowptr, int32_t* col, double* valM, double* valF, double* g);

/* Double glazing with SUPG stabilisation and symmetric Nitsche boundary
 * conditions, the discretisation of the paper's advection-diffusion runs
 * (Section 5); every node is an unknown (n = n_nodes):
 *   M = M_gal + S_M, S_M[i,j] = delta_e (w_e . grad l_i) |T|/3
 *   F = eps K + C + S + N, S[i,j] = delta_e (w_e . grad l_i) (int_T w) . grad l_j
 *   N: -eps int_e (grad phi_j . n) phi_i - eps int_e (grad phi_i . n) phi_j
 *      + (gamma eps/|e|) int_e phi_i phi_j on every edge of only one triangle
 *   g = -(-eps int_e (grad phi_i . n) u_B + (gamma eps/|e|) int_e u_B phi_i)
 * delta_e = h_e/(2|w_e|)(1 - 1/P_e) when the Peclet number P_e = |w_e| h_e/(2 eps)
 * exceeds 1, else 0, with h_e = 2|w_e| / sum_a |w_e . grad l_a|.  wind: n_tri*6*2
 * values at irk_fem_quad_points; wind_c: n_tri*2 values at the centroids (the
 * mean of the three vertices); ub: n_nodes boundary values (u_B is linear
 * along each edge), NULL = 0; gamma > 0 the Nitsche penalty.  The wind must be
 * tangential on the boundary (no inflow term).  Size query and outputs as
 * irk_fem_assemble. */
irk_status irk_fem_assemble_supg(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri, double eps,
                                 const double* wind, const double* wind_c, const double* ub, double gamma,
                                 int64_t* nnz, int64_t* rowptr, int32_t* col, double* valM, double* valF,
                                 double* g);

/* Streamline-diffusion matrix of the coarse-level SUPG stabilisation, on the
 * pattern (rowptr, col: n_nodes rows, from irk_fem_assemble_supg) of the SUPG
 * matrices: valT[i,j] = sum over the triangles with mesh Peclet number
 * P_e = |w_e| h_e/(2 eps) > 1 of h_e/(2|w_e|) |T| (w_e . grad l_i)(w_e . grad l_j),
 * h_e = 2|w_e| / sum_a |w_e . grad l_a|, w_e = wind_c (n_tri*2, centroid wind).
 * (h_e/(2|w_e|) is the slope of the SUPG parameter in the element size at large
 * Peclet numbers.)  IRK_ERR_INVALID for a bad mesh, eps <= 0, or a triangle
 * entry missing from the pattern. */
irk_status irk_fem_assemble_streamline(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri,
                                       double eps, const double* wind_c, const int64_t* rowptr,
                                       const int32_t* col, double* valT);

/* ------------------------------------------------------------------------- *
 * Solver context.                                                            *
 * ------------------------------------------------------------------------- */

typedef struct {
  irk_csr M;             /* n x n interior mass matrix */
  irk_csr F;             /* n x n interior F; same pattern as M */
  const double* g;       /* n lift F_IB u_B, or NULL (zero) */
  /* Mesh, needed only by irk_set_kappa and the kappa gradient of
   * irk_adjoint_step (heat problems, F = sum_e kappa_e K_e); n_tri = 0 if absent. */
  int32_t n_nodes, n_tri;
  const double* xy;      /* n_nodes*2 */
  const int32_t* tri;    /* n_tri*3, counter-clockwise */
  const int32_t* dof;    /* n_nodes: interior index or -1 */
  /* Coarse-level SUPG stabilisation (Section 5: the SUPG discretisation is
   * stabilised on every coarse mesh of the AMG): nnz values, on the pattern of
   * M, of the streamline-diffusion matrix T (irk_fem_assemble_streamline), or
   * NULL.  With T, level l (n_l rows) of the hierarchy of the block M + c F is
   * A_l = P^T A_{l-1} P + c (f_l - f_{l-1}) T_l, T_l = P^T T_{l-1} P, T_0 = T,
   * f_l = sqrt(n_0 / n_l); it is stabilised before it is coarsened.  Copied. */
  const double* stab;
} irk_problem;

/* Build the solver for one problem, Butcher table and step h_t: the stage
 * system (I_s (x) M + h_t A (x) F) k = r of Section 4 (Eq. block_coeff_mtx)
 * with the preconditioner P = I_s (x) M + h_t A~ (x) F of Section 4.2
 * (Eq. PrecForm), one AMG V-cycle per diagonal-block subsolve (Sections 4.2
 * and 5).  Copies M, F,
 * g (and the mesh) to the device, forms A~ (opt->kind), and builds on the GPU
 * one AMG hierarchy per distinct diagonal block M + h_t A~_jj F.  `stream` is
 * a cudaStream_t (NULL = legacy default stream); the library also creates a
 * private stream ordered after it.  *out receives the context; on failure
 * *out is NULL.  Errors: IRK_ERR_INVALID (sizes, patterns of M and F differ,
 * s out of range), IRK_ERR_ZERO_PIVOT, IRK_ERR_NOMEM, IRK_ERR_CAPACITY,
 * IRK_ERR_CUDA. */
irk_status irk_setup(const irk_problem* prob, const irk_butcher* bt, double h_t,
                     const irk_options* opt, void* stream, irk_ctx** out);

/* One time step (Section 2): solves the stage system for k from u_n and
 * returns u_{n+1} = u_n + h_t sum_i b_i k_i.  d_u_n, d_u_np1: n (may alias).
 * d_k: s*n stage block out, or NULL.  stats may be NULL.  Returns
 * IRK_ERR_NOT_CONVERGED / _BREAKDOWN / _NONFINITE from the device solve. */
irk_status irk_step(irk_ctx* ctx, const double* d_u_n, double* d_u_np1, double* d_k,
                    irk_stats* stats);

/* Solve the stage system (I_s (x) M + h A (x) F) k = b (Eq. block_coeff_mtx)
 * for a given right-hand side with the context's preconditioner and Krylov
 * method (the manufactured-solution runs of Section 5 solve it for
 * b = A k* with a chosen k*).  d_b, d_k: s*n FP64 device vectors, stage-major
 * [K_1; ...; K_s], caller-owned; d_k receives the solution.  Statistics and
 * errors as irk_step (IRK_ERR_NOT_CONVERGED leaves the last iterate). */
irk_status irk_solve(irk_ctx* ctx, const double* d_b, double* d_k, irk_stats* stats);

/* nsteps steps from d_u0 (n) to d_u_out (n).  If d_ckpt is not NULL it
 * receives u at steps 0, ckpt_every, 2 ckpt_every, ... (row q = u_{q*ckpt_every},
 * ceil(nsteps/ckpt_every) rows of n).  Steps are launched back to back with no
 * host synchronisation between them. */
irk_status irk_run(irk_ctx* ctx, const double* d_u0, int32_t nsteps, double* d_u_out,
                   double* d_ckpt, int32_t ckpt_every, irk_stats* stats);

/* Backward through one step (discrete adjoint).  Given lambda_{n+1} = dL/du_{n+1},
 * solves the transposed stage system (I (x) M^T + h_t A^T (x) F^T) mu =
 * h_t (b (x) lambda_{n+1}) with FGMRES and the transposed preconditioner, and
 * returns lambda_n = lambda_{n+1} - F^T sum_i mu_i.  If d_grad_kappa (n_tri)
 * is not NULL, adds dL/dkappa_e = -sum_i mu_i[e]^T K_e U_i[e] with the stage
 * values U_i = u_n + h_t sum_j a_ij k_j (heat problems with a mesh; F must be
 * sum_e kappa_e K_e).  d_u_n (n) and d_k_n (s*n) are the forward step's input
 * and stages.  d_lambda_n may alias d_lambda_np1.  For nonsymmetric M or F the
 * first adjoint call builds M^T, F^T and the AMG hierarchies of the transposed
 * diagonal blocks (kept by the context).  The transposed system is solved with
 * right-preconditioned FGMRES whatever the side of the forward solves. */
irk_status irk_adjoint_step(irk_ctx* ctx, const double* d_lambda_np1, const double* d_u_n,
                            const double* d_k_n, double* d_lambda_n, double* d_grad_kappa,
                            irk_stats* stats);

/* Checkpointed reverse sweep over irk_run(nsteps, ckpt_every): recomputes each
 * segment forward from d_ckpt, then takes adjoint steps backwards.
 * d_lambda (n): in = dL/du_N, out = dL/du_0.  d_grad_kappa (n_tri) or NULL:
 * accumulated as in irk_adjoint_step. */
irk_status irk_adjoint_run(irk_ctx* ctx, const double* d_ckpt, int32_t nsteps, int32_t ckpt_every,
                           double* d_lambda, double* d_grad_kappa, irk_stats* stats);

/* Re-assemble F = sum_e kappa_e K_e on the GPU from d_kappa (n_tri, device)
 * and rebuild the hierarchies.  Needs the mesh in irk_setup. */
irk_status irk_set_kappa(irk_ctx* ctx, const double* d_kappa);

/* ------------------------------------------------------------------------- *
 * Batched instances: independent problems of different sizes advanced by one *
 * CUDA graph launch (each instance a concurrent chain of the graph, its time *
 * loop and FGMRES loop device-driven WHILE nodes).                           *
 * ------------------------------------------------------------------------- */
typedef struct irk_batch irk_batch;

/* Build the batch over `count` contexts (same device; they must outlive the
 * batch and must not be used concurrently with it).  Instance q runs nsteps
 * IRK steps from d_u0[q] (n_q) into d_uN[q] (n_q), storing u every
 * ckpt_every steps in d_ckpt[q] (ceil(nsteps/ckpt_every) x n_q).  If d_lambda
 * is not NULL the adjoint graph is built too: irk_batch_adjoint then runs the
 * checkpointed reverse sweep of every instance (as irk_adjoint_run), with
 * d_lambda[q] (n_q) holding dL/du_N on entry and dL/du_0 on exit, and adds
 * dL/dkappa into d_grad_kappa[q] (n_tri_q) when d_grad_kappa and its entry are
 * not NULL.  All buffers are caller-owned device memory bound at creation. */
irk_status irk_batch_create(irk_ctx* const* ctxs, int32_t count, int32_t nsteps, int32_t ckpt_every,
                            const double* const* d_u0, double* const* d_uN, double* const* d_ckpt,
                            double* const* d_lambda, double* const* d_grad_kappa, irk_batch** out);
/* One graph launch: every instance forward.  stats (count entries, may be NULL)
 * receive per-instance statistics; *ms (may be NULL) the device time. */
irk_status irk_batch_run(irk_batch* b, void* stream, irk_stats* stats, double* ms);
/* One graph launch: every instance's checkpointed adjoint sweep. */
irk_status irk_batch_adjoint(irk_batch* b, void* stream, irk_stats* stats, double* ms);
void irk_batch_destroy(irk_batch* b);

/* ------------------------------------------------------------------------- *
 * Single operations (each one kernel sequence; used by tests and callers     *
 * composing their own iterations).                                           *
 * ------------------------------------------------------------------------- */

/* d_w = (I (x) M + h_t A (x) F) d_z; transpose != 0 applies
 * I (x) M^T + h_t A^T (x) F^T (for nonsymmetric M or F with the transposed
 * matrices, built on first use).  s*n each. */
irk_status irk_apply_operator(irk_ctx* ctx, const double* d_z, double* d_w, int32_t transpose);

/* The same operator on an FP32 d_z (s*n floats), as FGMRES applies it to the
 * FP32/BF16 preconditioner outputs z_j = P^{-1} v_j (Section 4.2); d_w (s*n)
 * is FP64.  Single-float pair arithmetic: each FP64 entry of M, F and h_t A is
 * split into two floats, products are exact up to the split (2^-48 relative),
 * sums carry their rounding errors, so |w - A z| is about 2^-47 times the sum
 * of the absolute terms of each row (FP64: 2^-53).  When the context has FP64
 * AMG, the environment sets IRK_KRON_FF=0, or an entry of M, F or h_t A lies
 * outside [2^-64, 2^64], the product is taken in FP64 on the widened z instead.
 * transpose as for irk_apply_operator; both pointers device, caller-owned. */
irk_status irk_apply_operator_f32(irk_ctx* ctx, const float* d_z, double* d_w, int32_t transpose);

/* d_z = P^{-1} d_v by the substitutions of Section 4.2, one V-cycle per
 * diagonal block (transpose != 0: P^T).  s*n each; the result is rounded to
 * the AMG precision before it is returned in FP64. */
irk_status irk_apply_precond(irk_ctx* ctx, const double* d_v, double* d_z, int32_t transpose);

/* d_x = one V-cycle on diagonal block `stage` (0..s-1) applied to d_b (n). */
irk_status irk_vcycle(irk_ctx* ctx, int32_t stage, const double* d_b, double* d_x);

/* True residual norm of a stage block: *norm = ||d_b - (I (x) M + h_t A (x) F) d_k||_2
 * (d_k, d_b: s*n device).  The per-block partial sums go to the context's
 * scratch; the result is copied to the host double *norm. */
irk_status irk_residual_norm(irk_ctx* ctx, const double* d_k, const double* d_b, double* norm);

/* The same norm as irk_residual_norm, for callers that must not allocate:
 * the call makes no cudaMalloc, cudaFree or other allocation.  The paper has
 * no counterpart; this is a library facility.  d_norm is a DEVICE double that
 * receives the norm.  The partial sums use a fixed device array inside libirk
 * with one slot per 256 rows, so n (rows per stage) may be at most
 * IRK_NOALLOC_MAX_ROWS; larger n gives IRK_ERR_CAPACITY.  The array's device
 * address is looked up the first time the entry point runs on a device and
 * kept for the life of the process (a device reset is not supported); make
 * that first call outside any stream capture.  Under lazy module loading that
 * first call may load libirk's device code, which the driver allocates memory
 * for; later calls allocate nothing.  The norm is ready on the caller's stream
 * when the call returns (the host does not wait).  Every call shares the array
 * (its contents are those of the last call), so calls that overlap on the GPU,
 * from any context or thread, race: serialise them. */
#define IRK_NOALLOC_MAX_ROWS 1048576
irk_status irk_residual_norm_noalloc(irk_ctx* ctx, const double* d_k, const double* d_b, double* d_norm);

/* d_y = M d_x (n). */
irk_status irk_apply_mass(irk_ctx* ctx, const double* d_x, double* d_y);

/* The final-time misfit of the adjoint runs (the L2 misfit 1/2 (u - d)^T M (u - d)
 * whose gradient the discrete adjoint propagates, Section 2 with the adjoint of
 * the time loop): *d_value (a DEVICE double) = 1/2 (d_u - d_d)^T M (d_u - d_d),
 * summed in a fixed order; d_grad (n, or NULL) = M (d_u - d_d), the misfit's
 * gradient for symmetric M.  d_u, d_d: n. */
irk_status irk_misfit(irk_ctx* ctx, const double* d_u, const double* d_d, double* d_grad, double* d_value);

/* Hierarchy of diagonal block `stage`: *nlevels and, per level (up to 16),
 * rows[l] and nnz[l] (host arrays of 16). */
irk_status irk_amg_info(irk_ctx* ctx, int32_t stage, int32_t* nlevels, int32_t* rows, int64_t* nnz);

/* Aggregate index of every row of level `level` (< nlevels-1) of block
 * `stage` into agg (host, rows[level] int32). */
irk_status irk_amg_aggregates(irk_ctx* ctx, int32_t stage, int32_t level, int32_t* agg);

/* Level matrix (FP64 CSR as built) of block `stage`: rowptr (rows+1), col and
 * val (nnz) host arrays sized from irk_amg_info. */
irk_status irk_amg_level_matrix(irk_ctx* ctx, int32_t stage, int32_t level, int64_t* rowptr,
                                int32_t* col, double* val);

/* Timing of one piece of an FGMRES iteration, replayed `reps` times on the
 * context's stream between CUDA events after `warm` untimed launches, on the
 * buffers of the last solve (their contents are overwritten; call it between
 * solves).  which: IRK_PROF_KRON (w = A z_j, the operator apply as in the
 * loop), IRK_PROF_VCYCLE (one V-cycle on the first diagonal block),
 * IRK_PROF_PRECOND (the whole P^{-1} application), IRK_PROF_GS_DOTS and
 * IRK_PROF_GS_AXPY (the two Gram-Schmidt passes at basis index j),
 * IRK_PROF_SMOOTH0 (one finest-level Chebyshev step of the first block),
 * IRK_PROF_VCYCLE_FROM (the part of a V-cycle of the first block from level j
 * (>= 1) down: its smoothing, restrictions, coarsest solve and prolongations).
 * *ms receives the mean time per replay, *bytes the algorithmic DRAM bytes
 * of one replay and *flops its algorithmic floating-point operations. */
enum { IRK_PROF_KRON = 0, IRK_PROF_VCYCLE = 1, IRK_PROF_PRECOND = 2, IRK_PROF_GS_DOTS = 3,
       IRK_PROF_GS_AXPY = 4, IRK_PROF_SMOOTH0 = 5, IRK_PROF_VCYCLE_FROM = 6 };
irk_status irk_profile(irk_ctx* ctx, int32_t which, int32_t j, int32_t warm, int32_t reps, double* ms,
                       double* bytes, double* flops);

/* Number of kernels the library has launched through this context so far
 * (graph-launched kernels included). */
int64_t irk_kernel_launches(const irk_ctx* ctx);

void irk_destroy(irk_ctx* ctx);
const char* irk_last_error(const irk_ctx* ctx);   /* thread-local message if ctx is NULL */
const char* irk_status_string(irk_status st);

#ifdef __cplusplus
}
#endif
#endif /* IRK_H */
