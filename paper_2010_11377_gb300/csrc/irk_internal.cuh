// Internal declarations of the GB300 IRK stage-system solver (libirk).
//
// Data layout in HBM
//   * stage blocks: s x n FP64, stage-major ([K_1; ...; K_s]), so a stage
//     block row gather reads s coalesced streams of the same index pattern;
//   * matrices: SELL-32 (slices of 32 consecutive rows, column-major inside a
//     slice, rows kept in their original order), int32 column indices; M and F
//     share one index array; AMG level matrices carry values in the V-cycle
//     precision (FP64, FP32, or BF16 on the finest level);
//   * Krylov bases: V (m+1 vectors, FP64, stored unnormalised with a scale
//     sigma_i), Z (m vectors, in the AMG precision: the preconditioner outputs
//     are kept exactly, so the flexible Arnoldi relation is exact for them).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "irk.h"

namespace irk {

constexpr int SELL_C = 32;
constexpr int MAX_S = 8;
constexpr int MAX_M = 64;
constexpr int MAX_LEVELS = 16;
constexpr int MAX_COARSE = 2048;

struct Error {
  irk_status st;
  std::string msg;
};
[[noreturn]] void fail(irk_status st, const std::string& msg);
void set_global_error(const std::string& msg);   // message for irk_last_error(NULL)
void cuda_check(cudaError_t e, const char* what, const char* file, int line);
#define CK(x) ::irk::cuda_check((x), #x, __FILE__, __LINE__)
#define CK_LAUNCH() ::irk::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_k may begin
// while the previous kernel on the stream drains.  Every such kernel calls
// pdl_wait() before it touches global memory (the wait returns once the
// previous grid has completed and its writes are visible).  IRK_PDL=0
// disables the attribute.
// ---------------------------------------------------------------------------
bool pdl_enabled();

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// dependents launch when this grid's blocks exit (no early trigger: measured,
// an early trigger let waiting blocks crowd the tail of multi-wave grids)
__device__ __forceinline__ void pdl_trigger() {}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  CK(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// ---------------------------------------------------------------------------
// Device memory owned by a context (freed at irk_destroy).
// ---------------------------------------------------------------------------
struct DevPool {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  void* alloc(size_t nbytes);
  template <typename T>
  T* get(size_t count) { return static_cast<T*>(alloc(count * sizeof(T))); }
  void release(void* p);   // free one pointer early (setup temporaries)
  void free_all();
};

// Scratch allocation for setup steps, freed when it goes out of scope.
struct Tmp {
  std::vector<void*> ptrs;
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    size_t nb = count * sizeof(T);
    if (nb == 0) nb = 16;
    CK(cudaMalloc(&p, nb));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Tmp();
};

// ---------------------------------------------------------------------------
// Sparse matrices
// ---------------------------------------------------------------------------
struct CsrD {               // device CSR, FP64 values, int32 indices
  int n = 0, ncols = 0;
  int64_t nnz = 0;
  int* rowptr = nullptr;    // n + 1 (nnz < 2^31 is enforced)
  int* col = nullptr;
  double* val = nullptr;
};

constexpr int PAT_W = 8;    // widest shared slice pattern (one 16-byte slot per slice)
static_assert(PAT_W * sizeof(short) == 16, "one 16-byte slot per slice");

struct Sell {               // SELL: slices of 32 / tpr rows, tpr threads per row (1: SELL-32)
  int n = 0, ncols = 0, nslices = 0;
  int tpr = 1;
  int64_t nnz_pad = 0;
  int64_t* sptr = nullptr;  // nslices + 1, element offsets
  int* col = nullptr;       // nnz_pad (padding: column 0, value 0)
  // square matrices whose columns all lie within +-32767 of their row: the
  // same columns as 16-bit offsets from the row (padding: offset 0), read by
  // the bandwidth-bound kernels instead of col (2 bytes per entry less)
  short* dcol = nullptr;
  // SELL-32 with 16-bit offsets: slices whose 32 rows all have the same length
  // w <= PAT_W and the same offsets (the interior of a stencil in natural order)
  // keep one offset per chunk in a fixed 16-byte slot of the slice,
  // pdcol[PAT_W sl + k] (k < w, zero beyond), read once per warp instead of 32
  // times and without waiting for the slice base; suni[sl] = w marks them
  // (0: per-entry offsets).  nnz_nonuni counts the stored entries of the other
  // slices (whose per-entry offsets are read).
  unsigned char* suni = nullptr;
  short* pdcol = nullptr;
  int64_t nnz_nonuni = 0;
  double* v64 = nullptr;
  float* v32 = nullptr;
  __nv_bfloat16* v16 = nullptr;
};

template <typename V>
struct SellView {
  int n;
  const int64_t* __restrict__ sptr;
  const int* __restrict__ col;
  const V* __restrict__ val;
  const short* __restrict__ dcol;
  const unsigned char* __restrict__ suni;   // width of the slice's shared pattern (0: none), or null
  const short* __restrict__ pdcol;          // the patterns, PAT_W offsets per slice
};

// column of SELL entry idx of row r
__device__ __forceinline__ int sell_col(const int* __restrict__ col, const short* __restrict__ dcol, int64_t idx,
                                        int r) {
  return dcol ? r + static_cast<int>(dcol[idx]) : col[idx];
}

template <typename V> const V* sell_vals(const Sell& s);
template <> inline const double* sell_vals<double>(const Sell& s) { return s.v64; }
template <> inline const float* sell_vals<float>(const Sell& s) { return s.v32; }
template <> inline const __nv_bfloat16* sell_vals<__nv_bfloat16>(const Sell& s) { return s.v16; }

template <typename V>
inline SellView<V> view(const Sell& s) {
  return SellView<V>{s.n, s.sptr, s.col, sell_vals<V>(s), s.dcol, s.suni, s.pdcol};
}

// One operator of a V-cycle level in the V-cycle precision, in one of three
// layouts chosen per operator (row-length rule or the layout autotuner):
//   lanes ==  1  SELL-32, one thread per row;
//   lanes == -T  SELL with slices of 32/T rows and T threads per row (T = 2, 4, 8),
//                each warp load one contiguous run of 32 entries;
//   lanes ==  L  CSR with L consecutive threads per row (2..32) and a shuffle
//                reduction, so a coarse Galerkin row of a few hundred entries is
//                not walked by a single thread.
struct MatT {
  int n = 0, ncols = 0;
  int64_t nnz = 0;
  int lanes = 1;
  Sell sell;                 // lanes <= 1
  int* rowptr = nullptr;     // lanes > 1
  int* col = nullptr;
  short* dcol = nullptr;     // lanes > 1, square: 16-bit column offsets from the row, or null
  void* val = nullptr;       // CSR values (V-cycle precision, or BF16)
  bool uses_sell() const { return lanes <= 1; }
  int64_t stored() const { return uses_sell() ? sell.nnz_pad : nnz; }
  const short* offsets() const { return uses_sell() ? sell.dcol : dcol; }
  // threads of one launch over the operator
  int64_t threads() const { return lanes < 0 ? int64_t(sell.nslices) * SELL_C : int64_t(n) * lanes; }
};

template <typename V>
struct LMat {
  int n;
  const int64_t* __restrict__ sptr;
  const int* __restrict__ rowptr;
  const int* __restrict__ col;
  const V* __restrict__ val;
  const short* __restrict__ dcol;   // 16-bit column offsets from the row (SELL or CSR), or null
  const unsigned char* __restrict__ suni;   // SELL-32: width of the slice's shared pattern (0: none), or null
  const short* __restrict__ pdcol;          // the patterns, PAT_W offsets per slice
};

template <typename V>
inline LMat<V> lmat(const MatT& m) {
  if (m.uses_sell())
    return LMat<V>{m.n, m.sell.sptr, nullptr, m.sell.col, sell_vals<V>(m.sell), m.sell.dcol, m.sell.suni,
                   m.sell.pdcol};
  return LMat<V>{m.n, nullptr, m.rowptr, m.col, static_cast<const V*>(m.val), m.dcol, nullptr, nullptr};
}

// bytes of column information per stored entry that a product reads
inline double offset_bytes_per_entry(const Sell& s) {
  if (!s.dcol) return 4.0;
  if (!s.suni || s.nnz_pad == 0) return 2.0;
  return 2.0 * double(s.nnz_nonuni) / double(s.nnz_pad);
}

// ---------------------------------------------------------------------------
// AMG hierarchy (one per distinct diagonal block M + h A~_jj F)
// ---------------------------------------------------------------------------
struct Level {
  int n = 0;
  int64_t nnz = 0;
  CsrD A;                    // FP64 CSR as built (kept for export and rebuilds)
  MatT Am, Pm, Rm;           // level operator, prolongation n x nc, restriction nc x n
  int* agg = nullptr;        // aggregate of every row (not on the coarsest level)
  void* dinv = nullptr;      // 1 / sum_j |a_ij|, V-cycle precision
  void *b = nullptr, *x = nullptr, *y = nullptr, *r = nullptr, *d = nullptr;
};

struct Hier {
  DevPool pool;              // every device allocation of this hierarchy
  double coef = 0.0;         // c in M + c F
  int amg_prec = 32;         // 64, 32 or 16
  std::vector<Level> lv;
  void* cinv = nullptr;      // coarsest dense inverse, row-major, V-cycle precision
  int nc_dense = 0;
  bool coarse_smooth = false;  // stalled coarsest level: 4 smoothing sweeps instead
};

struct AmgParams {
  double theta = 0.08;
  int coarse_max = 2048;
  int max_levels = 12;
  int smoother = IRK_SMOOTH_CHEBYSHEV;
  int cheb_degree = 4;
  double cheb_lo = 0.1;
  int nu_pre = 1, nu_post = 1;
  int amg_prec = 32;
  int p_smooth = 2;        // damped-Jacobi steps on the tentative prolongator
  int strength_negative = 0;   // strength from max(-a_ij, 0) (else |a_ij|)
  int w_coarse = 0;        // W-cycle below the finest level (two coarse-grid corrections on levels >= 1)
};

// Chebyshev step coefficients: step i updates d_i = alpha_i d_{i-1} + beta_i D^{-1}(b - A x_i)
struct SmoothCoef {
  int steps = 1;
  double alpha[16];
  double beta[16];
};
SmoothCoef smooth_coefficients(const AmgParams& p);

// ---------------------------------------------------------------------------
// FGMRES state (device resident; every control decision is taken on the GPU)
// ---------------------------------------------------------------------------
struct GmresState {
  int j;           // current inner index
  int it;          // inner iterations of this solve
  int restarts;
  int done;        // 1: solve finished (converged or stopped)
  int cycle_end;   // 1: update x and restart or stop after this iteration
  int reorth;      // 1: reorthogonalise this iteration
  int status;      // irk_status from the device
  int m, max_it;
  unsigned int counter;   // last-block-done ticket
  int guard;              // loop-body executions of this solve (bounded)
  double bnorm, rtol;
  double bnorm_true;      // ||b|| (left preconditioning: bnorm is ||P^{-1} b||)
  double wnorm2;          // ||w||^2 before projection
  double eta2;            // second pass when ||w_proj||^2 < eta2 ||w||^2 (< 0: always)
  double resid;           // last true relative residual
  double H[MAX_M * (MAX_M + 1)];   // column-major, column j at H[j*(MAX_M+1)]
  double cs[MAX_M], sn[MAX_M];
  double g[MAX_M + 1];
  double sigma[MAX_M + 1];         // 1/||v_i|| of the stored basis vectors
  double h2[MAX_M + 1];            // reorthogonalisation coefficients
};

// per-step record kept on the device by irk_run
struct StepRecord {
  int it, restarts, status, pad_;
  double resid;
};

struct KronCoef {          // h A (or h A^T), row-major MAX_S x MAX_S
  double a[MAX_S * MAX_S];
};

struct KronCoefF {         // the same as single-float pairs: a = hi + lo (to 2^-48 |a|)
  float hi[MAX_S * MAX_S];
  float lo[MAX_S * MAX_S];
};

struct SweepPlan {         // substitution order and couplings of P^{-1}
  int s;
  int order[MAX_S];                // stage processed at position p
  int hier[MAX_S];                 // hierarchy index used by stage order[p]
  int nprev[MAX_S];                // couplings of the stage at position p
  int prev[MAX_S][MAX_S];          // stages k coupled into it
  double coef[MAX_S][MAX_S];       // h A~_jk for those k
};

// index-indirected device pointer: base + (*jp + add) * stride + off
template <typename T>
struct JPtr {
  T* base;
  const int* jp;
  int64_t stride;
  int add;
  int64_t off;
  __device__ __forceinline__ T* get() const {
    return base + (jp ? static_cast<int64_t>(*jp + add) * stride : static_cast<int64_t>(add) * stride) + off;
  }
};
template <typename T>
inline JPtr<T> jptr(T* base, const int* jp = nullptr, int64_t stride = 0, int add = 0, int64_t off = 0) {
  return JPtr<T>{base, jp, stride, add, off};
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct Graph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t body_kernels = 0;     // kernels per FGMRES iteration
  int64_t fixed_kernels = 0;    // kernels per launch outside the loop
  bool conditional = false;
};

struct Ctx {
  int device = 0;
  int n = 0, s = 0;
  double h = 0.0;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  DevPool pool;
  std::string err;

  // problem
  CsrD Mc, Fc;              // FP64 CSR, one pattern
  Sell Ms, Fs;              // SELL-32: Ms.v64 = M, Fs.v64 = F (FP64), Fs.v32 = F (FP32)
  float4* MFs = nullptr;    // SELL-32 {M hi, M lo, F hi, F lo} single-float pairs, or null
  double* g = nullptr;      // lift (n)
  double* Tval = nullptr;   // streamline matrix of the coarse-level SUPG stabilisation (pattern of Mc), or null
  bool symmetric = false;

  // mesh (optional)
  int n_nodes = 0, n_tri = 0;
  double* xy = nullptr;     // device
  int* tri = nullptr;       // device
  int* dof = nullptr;       // device
  int* asm_ptr = nullptr;   // F entry -> contribution list offsets (nnz + 1)
  int* asm_src = nullptr;   // contributions: element*9 + a*3 + b
  double* Ke = nullptr;     // unit-kappa element stiffness (n_tri * 9)

  // method
  double A[MAX_S * MAX_S], b[MAX_S], c[MAX_S], At[MAX_S * MAX_S];
  int kind = IRK_PC_LD;
  KronCoef K, KT;
  KronCoefF Kf, KTf;
  SweepPlan plan, planT;
  AmgParams amg;
  SmoothCoef sc;
  std::vector<Hier> hiers;
  // the transposed problem for the adjoint of nonsymmetric M and F (M^T, F^T on
  // one pattern, their pair copy and the hierarchies of the blocks (M + c F)^T),
  // built on first use and swapped in while adjoint work is launched
  struct Transposed {
    bool built = false;
    CsrD Mc, Fc;
    Sell Ms, Fs;
    float4* MFs = nullptr;
    std::vector<Hier> hiers;
  } tr;
  irk_options opt;

  // FGMRES storage
  int m = 30, max_it = 1000, reorth = 0;
  double reorth_eta = 0.1;
  double rtol = 1e-10;
  int64_t N = 0;            // s * n
  int side = 0;             // 0: right-preconditioned FGMRES; 1: left-preconditioned GMRES
  double* T = nullptr;      // N (left: A v_j, and the restart residual)
  double* V = nullptr;      // (m+1) * N
  void* Z = nullptr;        // m * N in the AMG precision
  double* x = nullptr;      // N
  double* bv = nullptr;     // N (right-hand side)
  int* rhs_given = nullptr; // device flag: the forward head takes bv as given (irk_solve)
  double* u = nullptr;      // n (current state)
  double* lam = nullptr;    // n (adjoint state)
  double* tmpn = nullptr;   // n
  GmresState* st = nullptr;
  double* partials = nullptr;
  int gs_grid = 0;
  StepRecord* rec = nullptr;
  int rec_cap = 0;
  int* step_counter = nullptr;
  double* kstore = nullptr; // adjoint recompute segment storage
  double* ustore = nullptr;
  int kstore_cap = 0;

  Graph graph[2];           // forward step, adjoint step
  int64_t launches = 0;
  bool host_loop = false;   // IRK_HOST_LOOP=1: host-driven FGMRES loop (same kernels, no graph)
  int* h_flag = nullptr;    // pinned host copy of GmresState::done
};

// ---------------------------------------------------------------------------
// Launch helpers implemented in the .cu files
// ---------------------------------------------------------------------------
int num_sms();
inline unsigned nblk(int64_t n, int bs = 256) { return static_cast<unsigned>((n + bs - 1) / bs); }

// scans (exclusive, out has n + 1 entries, out[n] = total)
void scan_exclusive(const int* in, int* out, int n, cudaStream_t st);
void scan_exclusive64(const int64_t* in, int64_t* out, int n, cudaStream_t st);

// sparse utilities
void csr_upload(const irk_csr& h, CsrD& d, DevPool& pool, cudaStream_t st);
void csr_alloc(CsrD& d, int n, int ncols, int64_t nnz, DevPool& pool);
void csr_to_sell(const CsrD& A, Sell& S, int want64, int want32, int want16, DevPool& pool,
                 cudaStream_t st, int tpr = 1);
void sell_share_pattern(const Sell& pat, const double* csr_vals, const CsrD& A, Sell& S, int want64,
                        int want32, DevPool& pool, cudaStream_t st);
// single-float pair copies of M, F and h A for the operator on FP32 vectors
// (MFs stays null when disabled or when an entry is outside [2^-64, 2^64])
void kron_split_build(Ctx& c);
void kron_apply_f32(Ctx& c, const float* z, double* w, bool transpose, cudaStream_t st);
void csr_transpose(const CsrD& A, CsrD& T, DevPool& pool, cudaStream_t st);
int choose_lanes(int64_t nnz, int n);
int autotune_lanes(const CsrD& A, int prec, cudaStream_t st);
void matT_spmv_launch(const MatT& m, int prec, const void* x, void* y, cudaStream_t st);
// V-cycle operator in precision prec (64, 32, 16 = BF16) from an FP64 CSR that
// stays alive (its index arrays are shared); force_lanes > 0 fixes the layout
void make_matT(const CsrD& A, MatT& m, int prec, DevPool& pool, cudaStream_t st, int force_lanes = 0);
void csr_spgemm(const CsrD& A, const CsrD& B, CsrD& C, DevPool& pool, cudaStream_t st);
void csr_axpby_same_pattern(const CsrD& X, const double* valX, const double* valY, double c,
                            double* out, cudaStream_t st);   // out = X + c Y (no FMA)
void csr_copy_to_host(const CsrD& A, std::vector<int>& rp, std::vector<int>& col,
                      std::vector<double>& val, cudaStream_t st);

// AMG setup
// T0: streamline matrix of the coarse-level SUPG stabilisation on the pattern
// of A0 (or null), c_stab: the block coefficient c of A0 = M + c F
void amg_build(Hier& H, const CsrD& A0, const AmgParams& p, DevPool& pool, cudaStream_t st,
               const CsrD* T0 = nullptr, double c_stab = 0.0);

// V-cycle on hierarchy H: rhs in H.lv[0].b, result written to out (level-0 size,
// V-cycle precision).  Returns the number of kernels launched.
int vcycle_launch(const Hier& H, const AmgParams& p, const SmoothCoef& sc, void* out_base,
                  const int* jp, int64_t jstride, int64_t off, cudaStream_t st, double* bytes = nullptr,
                  double* flops = nullptr);
int vcycle_launch_from(const Hier& H, const AmgParams& p, const SmoothCoef& sc, int l0, cudaStream_t st,
                       double* bytes = nullptr, double* flops = nullptr);
void smooth0_launch(const Hier& H, const AmgParams& p, const SmoothCoef& sc, cudaStream_t st, double* bytes,
                    double* flops);

// preconditioner z = P^{-1} (sigma_j V_j), stage by stage (Section 4.2)
struct PrecondArgs {
  const double* V;          // base of V (FP64)
  const int* jp;            // index j (device) or nullptr for 0
  int64_t ldv;              // stride between basis vectors
  const double* sigma;      // per-vector scale (indexed by j) or nullptr for 1
  void* Z;                  // base of Z (AMG precision)
  int64_t ldz;
  const int* skip;          // device flag: write zeros instead (nullptr: never)
  double* bytes = nullptr;  // accumulated algorithmic bytes / flops (optional)
  double* flops = nullptr;
};
int precond_launch(Ctx& c, const PrecondArgs& a, bool transpose, cudaStream_t st);

// FGMRES pieces (krylov.cu)
int fgmres_body_launch(Ctx& c, bool transpose, cudaStream_t st);   // one iteration after P^{-1}
// Left preconditioning (forward solves): after the right-hand side, P^{-1} b
// and the first basis vector; one iteration w = P^{-1} A v_j including the
// preconditioner; the true residual for the stats after the loop.
int left_head_launch(Ctx& c, cudaStream_t st);
int left_body_launch(Ctx& c, cudaStream_t st);
int left_tail_launch(Ctx& c, cudaStream_t st);
void set_loop_condition_launch(Ctx& c, cudaGraphConditionalHandle h, cudaStream_t st);
void rhs_forward_launch(Ctx& c, const double* u, cudaStream_t st);
void rhs_adjoint_launch(Ctx& c, const double* lam, cudaStream_t st);
void stage_update_launch(Ctx& c, double* u, cudaStream_t st);
void record_launch(Ctx& c, cudaStream_t st);
void kron_apply_plain(Ctx& c, const double* z, double* w, bool transpose, cudaStream_t st);
void mass_apply_launch(Ctx& c, const double* x, double* y, cudaStream_t st);
void misfit_launch(Ctx& c, const double* u, const double* d, double* grad, double* out, cudaStream_t st);
void adjoint_lambda_launch(Ctx& c, const double* lam_in, double* lam_out, cudaStream_t st);
void adjoint_grad_launch(Ctx& c, const double* u_n, const double* k_n, double* grad, cudaStream_t st);
void adjoint_grad_launch_at(Ctx& c, const double* u_base, const double* k_base, const int* step, double* grad,
                            cudaStream_t st);
void assemble_kappa_launch(Ctx& c, const double* kappa, double* Fval, cudaStream_t st);
void convert_launch(const void* in, int in_prec, void* out, int out_prec, int64_t n, cudaStream_t st);
void profile_kron_launch(Ctx& c, cudaStream_t st);
// the transposed problem of a nonsymmetric context (built on first use) and a
// scope that swaps it in while adjoint work is launched or captured
void ensure_transposed(Ctx& c);
void swap_transposed(Ctx& c);
struct AdjointView {
  Ctx& c;
  bool on;
  AdjointView(Ctx& c_, bool adjoint) : c(c_), on(adjoint && !c_.symmetric) {
    if (on) {
      ensure_transposed(c);
      swap_transposed(c);
    }
  }
  ~AdjointView() {
    if (on) swap_transposed(c);
  }
  AdjointView(const AdjointView&) = delete;
  AdjointView& operator=(const AdjointView&) = delete;
};

// threads (= rows per grid-stride pass) per block of the outer Krylov kernels
constexpr int OUTER_BLOCK = 256;
void residual_norm_launch(Ctx& c, const double* k, const double* b, double* partials, int grid, double* out,
                          cudaStream_t st);
void profile_gs_launch(Ctx& c, GmresState* scratch, bool axpy, cudaStream_t st);

}  // namespace irk

struct irk_ctx {
  irk::Ctx c;
};
