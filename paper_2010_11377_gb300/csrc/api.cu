// C ABI entry points of libirk: context set-up, the time step and run loops
// (one CUDA graph per step whose FGMRES loop is a device-driven WHILE node),
// the adjoint, and the single-operation entry points.
#include "irk_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <vector>

extern "C" irk_status irk_atilde(int32_t kind, int32_t s, const double* A, double* Atilde, double* kappa);

namespace {

thread_local std::string g_err;

irk_status set_err(irk_ctx* h, irk_status st, const std::string& msg) {
  if (h) h->c.err = msg;
  g_err = msg;
  return st;
}

template <typename F>
irk_status guarded(irk_ctx* h, F&& f) {
  try {
    f();
    return IRK_OK;
  } catch (const irk::Error& e) {
    return set_err(h, e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return set_err(h, IRK_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_err(h, IRK_ERR_INVALID, e.what());
  }
}

}  // namespace

namespace irk {

void set_global_error(const std::string& msg) { g_err = msg; }

static void begin_call(Ctx& c) {
  CK(cudaSetDevice(c.device));
  CK(cudaEventRecord(c.ev_a, c.user_stream));
  CK(cudaStreamWaitEvent(c.stream, c.ev_a, 0));
}

static void end_call(Ctx& c) {
  CK(cudaEventRecord(c.ev_b, c.stream));
  CK(cudaStreamWaitEvent(c.user_stream, c.ev_b, 0));
  CK(cudaStreamSynchronize(c.stream));
}

// sweep plan of P = I (x) M + h At (x) F; transpose uses At^T
static void make_plan(Ctx& c, const double* At, SweepPlan& P, std::vector<double>& coefs) {
  int s = c.s;
  bool lower = true, upper = true;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      double v = At[i * s + j];
      if (j > i && v != 0.0) lower = false;
      if (j < i && v != 0.0) upper = false;
    }
  if (!lower && !upper) fail(IRK_ERR_INVALID, "A~ must be diagonal, lower or upper triangular");
  bool backward = upper && !lower;   // diagonal A~: forward order, no couplings
  P.s = s;
  for (int p = 0; p < s; ++p) {
    int j = backward ? s - 1 - p : p;
    P.order[p] = j;
    double cj = c.h * At[j * s + j];
    if (cj != cj) fail(IRK_ERR_INVALID, "non-finite A~");
    auto it = std::find(coefs.begin(), coefs.end(), cj);
    int hidx;
    if (it == coefs.end()) {
      coefs.push_back(cj);
      hidx = static_cast<int>(coefs.size()) - 1;
    } else {
      hidx = static_cast<int>(it - coefs.begin());
    }
    P.hier[p] = hidx;
    int np = 0;
    for (int q = 0; q < p; ++q) {
      int k = P.order[q];
      double v = At[j * s + k];
      if (v != 0.0) {
        P.prev[p][np] = k;
        P.coef[p][np] = c.h * v;
        ++np;
      }
    }
    P.nprev[p] = np;
  }
}

static void alloc_solver_buffers(Ctx& c) {
  size_t es = (c.amg.amg_prec == 64) ? sizeof(double) : sizeof(float);
  c.N = int64_t(c.s) * c.n;
  c.V = c.pool.get<double>(size_t(c.m + 1) * c.N);
  c.Z = c.pool.alloc(es * size_t(c.m) * c.N);
  c.x = c.pool.get<double>(c.N);
  c.bv = c.pool.get<double>(c.N);
  c.T = c.side == 1 ? c.pool.get<double>(c.N) : nullptr;
  c.rhs_given = c.pool.get<int>(1);
  CK(cudaMemset(c.rhs_given, 0, sizeof(int)));
  c.u = c.pool.get<double>(c.n);
  c.lam = c.pool.get<double>(c.n);
  c.tmpn = c.pool.get<double>(c.n);
  c.st = c.pool.get<GmresState>(1);
  CK(cudaMemset(c.st, 0, sizeof(GmresState)));
  c.gs_grid = 4 * num_sms();
  c.partials = c.pool.get<double>(size_t(c.gs_grid) * (MAX_M + 2));
  c.rec_cap = 4096;
  c.rec = c.pool.get<StepRecord>(c.rec_cap);
  c.step_counter = c.pool.get<int>(1);
}

static void build_hierarchies(Ctx& c) {
  std::vector<double> coefs;
  make_plan(c, c.At, c.plan, coefs);
  double AtT[MAX_S * MAX_S];
  for (int i = 0; i < c.s; ++i)
    for (int j = 0; j < c.s; ++j) AtT[i * c.s + j] = c.At[j * c.s + i];
  make_plan(c, AtT, c.planT, coefs);
  for (auto& H : c.hiers) H.pool.free_all();
  c.hiers.clear();
  c.hiers.resize(coefs.size());
  for (size_t q = 0; q < coefs.size(); ++q) {
    Hier& H = c.hiers[q];
    H.coef = coefs[q];
    CsrD A0;
    A0.n = c.n;
    A0.ncols = c.n;
    A0.nnz = c.Mc.nnz;
    A0.rowptr = c.Mc.rowptr;
    A0.col = c.Mc.col;
    A0.val = H.pool.get<double>(c.Mc.nnz > 0 ? c.Mc.nnz : 1);
    csr_axpby_same_pattern(c.Mc, c.Mc.val, c.Fc.val, coefs[q], A0.val, c.stream);
    CsrD T0 = A0;
    T0.val = c.Tval;
    amg_build(H, A0, c.amg, H.pool, c.stream, c.Tval ? &T0 : nullptr, coefs[q]);
  }
}

static void destroy_graphs(Ctx& c) {
  for (auto& g : c.graph) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = Graph{};
  }
}

// adjoint work of a nonsymmetric problem runs on the transposed matrices and
// hierarchies: swap them in for the scope (graphs capture the pointers)
void swap_transposed(Ctx& c) {
  std::swap(c.Mc, c.tr.Mc);
  std::swap(c.Fc, c.tr.Fc);
  std::swap(c.Ms, c.tr.Ms);
  std::swap(c.Fs, c.tr.Fs);
  std::swap(c.MFs, c.tr.MFs);
  c.hiers.swap(c.tr.hiers);
}

void ensure_transposed(Ctx& c) {
  if (c.tr.built) return;
  CsrD Mt, Ft;
  csr_transpose(c.Mc, Mt, c.pool, c.stream);
  csr_transpose(c.Fc, Ft, c.pool, c.stream);   // the same pattern as Mt: M and F share one
  c.tr.Mc = Mt;
  c.tr.Fc = Ft;
  c.tr.Fc.rowptr = Mt.rowptr;
  c.tr.Fc.col = Mt.col;
  csr_to_sell(Mt, c.tr.Ms, 1, 0, 0, c.pool, c.stream);
  sell_share_pattern(c.tr.Ms, Ft.val, Ft, c.tr.Fs, 1, 1, c.pool, c.stream);
  swap_transposed(c);
  try {
    kron_split_build(c);
    build_hierarchies(c);
  } catch (...) {
    swap_transposed(c);
    throw;
  }
  swap_transposed(c);
  c.tr.built = true;
}

// One time-step graph (forward: rhs from c.u, update c.u; adjoint: rhs from
// c.lam, lambda update into c.tmpn).  The FGMRES loop is a WHILE node whose
// condition the last kernel of each iteration sets from the device state.
static void build_graph(Ctx& c, bool adjoint) {
  AdjointView av(c, adjoint);
  Graph& G = c.graph[adjoint ? 1 : 0];
  if (G.exec || c.host_loop) return;
  cudaStream_t st = c.stream;
  cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t graph;
  CK(cudaGraphCreate(&graph, 0));
  const bool left = !adjoint && c.side == 1;
  int64_t fixed = 3;
  // head
  CK(cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, mode));
  if (adjoint) rhs_adjoint_launch(c, c.lam, st);
  else rhs_forward_launch(c, c.u, st);
  if (left) fixed += left_head_launch(c, st);
  std::vector<cudaGraphNode_t> head;   // the captured nodes the loop follows
  {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
    head.assign(deps, deps + nd);
  }
  CK(cudaStreamEndCapture(st, &graph));
  // loop
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  CK(cudaGraphAddNode(&loop, graph, head.data(), nullptr, head.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  int64_t nb = 0;
  if (left) {
    nb += left_body_launch(c, st);
  } else {
    PrecondArgs pa{c.V, &c.st->j, c.N, c.st->sigma, c.Z, c.N, &c.st->done};
    nb += precond_launch(c, pa, adjoint, st);
    nb += fgmres_body_launch(c, adjoint, st);
  }
  set_loop_condition_launch(c, handle, st);
  nb += 1;
  CK(cudaStreamEndCapture(st, &body));
  // tail
  CK(cudaStreamBeginCaptureToGraph(st, graph, &loop, nullptr, 1, mode));
  if (left) fixed += left_tail_launch(c, st);
  if (adjoint) adjoint_lambda_launch(c, c.lam, c.tmpn, st);
  else stage_update_launch(c, c.u, st);
  record_launch(c, st);
  CK(cudaStreamEndCapture(st, &graph));
  CK(cudaGraphInstantiate(&G.exec, graph, 0));
  G.graph = graph;
  G.body_kernels = nb;
  G.fixed_kernels = fixed;
  G.conditional = true;
}

// One solve: the step graph, or (host loop) the same kernel sequence with the
// loop condition read back on the host after every iteration.
static void launch_solve(Ctx& c, bool adjoint) {
  AdjointView av(c, adjoint);
  Graph& G = c.graph[adjoint ? 1 : 0];
  if (!c.host_loop) {
    CK(cudaGraphLaunch(G.exec, c.stream));
    return;
  }
  cudaStream_t st = c.stream;
  const bool left = !adjoint && c.side == 1;
  if (adjoint) rhs_adjoint_launch(c, c.lam, st);
  else rhs_forward_launch(c, c.u, st);
  int64_t k = 1;
  if (left) k += left_head_launch(c, st);
  for (int it = 0; it < c.max_it + 8; ++it) {
    if (left) {
      k += left_body_launch(c, st);
    } else {
      PrecondArgs pa{c.V, &c.st->j, c.N, c.st->sigma, c.Z, c.N, &c.st->done};
      k += precond_launch(c, pa, adjoint, st);
      k += fgmres_body_launch(c, adjoint, st);
    }
    CK(cudaMemcpyAsync(c.h_flag, &c.st->done, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*c.h_flag) break;
  }
  if (left) k += left_tail_launch(c, st);
  if (adjoint) adjoint_lambda_launch(c, c.lam, c.tmpn, st);
  else stage_update_launch(c, c.u, st);
  record_launch(c, st);
  c.launches += k + 2;
}

static void reset_records(Ctx& c) { CK(cudaMemsetAsync(c.step_counter, 0, sizeof(int), c.stream)); }

static void collect_stats(Ctx& c, int nsteps, irk_stats* out, irk_status* dev_status, int graph_idx) {
  std::vector<StepRecord> rec(std::min(nsteps, c.rec_cap));
  if (!rec.empty())
    CK(cudaMemcpyAsync(rec.data(), c.rec, sizeof(StepRecord) * rec.size(), cudaMemcpyDeviceToHost, c.stream));
  float ms = 0.f;
  CK(cudaStreamSynchronize(c.stream));
  CK(cudaEventElapsedTime(&ms, c.ev_t0, c.ev_t1));
  irk_stats s{};
  s.steps = nsteps;
  s.ms = ms;
  *dev_status = IRK_OK;
  int64_t its = 0;
  for (const auto& r : rec) {
    s.iterations += r.it;
    s.restarts += r.restarts;
    s.max_step_iterations = std::max(s.max_step_iterations, r.it);
    s.resid = r.resid;
    its += std::max(r.it, 1);
    if (r.status != IRK_OK && *dev_status == IRK_OK) *dev_status = static_cast<irk_status>(r.status);
  }
  const Graph& G = c.graph[graph_idx];
  if (!c.host_loop) c.launches += G.fixed_kernels * nsteps + G.body_kernels * its;
  if (out) *out = s;
}

static irk_status run_steps(Ctx& c, const double* u0, int nsteps, double* uout, double* ckpt, int every,
                            double* kout, irk_stats* stats) {
  build_graph(c, false);
  begin_call(c);
  if (u0 != c.u) CK(cudaMemcpyAsync(c.u, u0, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  reset_records(c);
  CK(cudaEventRecord(c.ev_t0, c.stream));
  for (int t = 0; t < nsteps; ++t) {
    if (ckpt && every > 0 && t % every == 0)
      CK(cudaMemcpyAsync(ckpt + int64_t(t / every) * c.n, c.u, sizeof(double) * c.n, cudaMemcpyDeviceToDevice,
                         c.stream));
    launch_solve(c, false);
    if (kout) CK(cudaMemcpyAsync(kout + int64_t(t) * c.N, c.x, sizeof(double) * c.N, cudaMemcpyDeviceToDevice,
                                 c.stream));
  }
  CK(cudaEventRecord(c.ev_t1, c.stream));
  if (uout && uout != c.u)
    CK(cudaMemcpyAsync(uout, c.u, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  irk_status dev = IRK_OK;
  collect_stats(c, nsteps, stats, &dev, 0);
  end_call(c);
  return dev;
}

static irk_status adjoint_one(Ctx& c, const double* lam_in, const double* u_n, const double* k_n, double* lam_out,
                              double* grad, bool timed) {
  if (lam_in != c.lam)
    CK(cudaMemcpyAsync(c.lam, lam_in, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  launch_solve(c, true);
  if (grad) adjoint_grad_launch(c, u_n, k_n, grad, c.stream);
  CK(cudaMemcpyAsync(lam_out, c.tmpn, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  (void)timed;
  return IRK_OK;
}

static void check_adjoint_ok(Ctx& c, bool need_grad) {
  // the transposed stage systems are solved with right-preconditioned FGMRES for
  // either side of the forward solve (the adjoint needs their solutions only)
  if (need_grad && c.n_tri == 0) fail(IRK_ERR_INVALID, "kappa gradient needs the mesh in irk_setup");
}

// host-side symmetry check (to 1e-13 relative per entry pair)
static bool csr_symmetric(const irk_csr& A) {
  for (int i = 0; i < A.n; ++i)
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      int j = A.col[k];
      const int32_t* b = A.col + A.rowptr[j];
      const int32_t* e = A.col + A.rowptr[j + 1];
      const int32_t* p = std::lower_bound(b, e, i);
      if (p == e || *p != i) return false;
      double x = A.val[p - A.col], y = A.val[k];
      if (std::fabs(x - y) > 1e-13 * std::max(std::fabs(x), std::fabs(y))) return false;
    }
  return true;
}

// unit-kappa element stiffness and the F-entry <- element contribution map
static void setup_mesh(Ctx& c, const irk_problem& P, const std::vector<int>& rp, const std::vector<int>& col) {
  int nt = P.n_tri, nn = P.n_nodes;
  std::vector<double> Ke(size_t(nt) * 9);
  std::vector<std::vector<int>> contrib(c.Fc.nnz);
  for (int e = 0; e < nt; ++e) {
    const int* t = P.tri + 3 * e;
    double x0 = P.xy[2 * t[0]], y0 = P.xy[2 * t[0] + 1];
    double x1 = P.xy[2 * t[1]], y1 = P.xy[2 * t[1] + 1];
    double x2 = P.xy[2 * t[2]], y2 = P.xy[2 * t[2] + 1];
    double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    if (!(det > 0.0)) fail(IRK_ERR_INVALID, "mesh triangles must be counter-clockwise and non-degenerate");
    double area = 0.5 * det;
    double gx[3] = {(y1 - y2) / det, (y2 - y0) / det, (y0 - y1) / det};
    double gy[3] = {(x2 - x1) / det, (x0 - x2) / det, (x1 - x0) / det};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Ke[size_t(e) * 9 + a * 3 + b] = area * (gx[a] * gx[b] + gy[a] * gy[b]);
    for (int a = 0; a < 3; ++a) {
      int da = P.dof[t[a]];
      if (da < 0) continue;
      for (int b = 0; b < 3; ++b) {
        int db = P.dof[t[b]];
        if (db < 0) continue;
        auto beg = col.begin() + rp[da], end = col.begin() + rp[da + 1];
        auto it = std::lower_bound(beg, end, db);
        if (it == end || *it != db) fail(IRK_ERR_INVALID, "F pattern misses an element coupling");
        contrib[it - col.begin()].push_back(e * 9 + a * 3 + b);
      }
    }
  }
  std::vector<int> ptr(c.Fc.nnz + 1, 0), src;
  for (int64_t q = 0; q < c.Fc.nnz; ++q) {
    ptr[q + 1] = ptr[q] + static_cast<int>(contrib[q].size());
    for (int v : contrib[q]) src.push_back(v);
  }
  c.n_tri = nt;
  c.n_nodes = nn;
  c.xy = c.pool.get<double>(size_t(nn) * 2);
  c.tri = c.pool.get<int>(size_t(nt) * 3);
  c.dof = c.pool.get<int>(nn);
  c.Ke = c.pool.get<double>(Ke.size());
  c.asm_ptr = c.pool.get<int>(ptr.size());
  c.asm_src = c.pool.get<int>(src.size() + 1);
  CK(cudaMemcpy(c.xy, P.xy, sizeof(double) * nn * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.tri, P.tri, sizeof(int) * nt * 3, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.dof, P.dof, sizeof(int) * nn, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.Ke, Ke.data(), sizeof(double) * Ke.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.asm_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice));
  if (!src.empty()) CK(cudaMemcpy(c.asm_src, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice));
}

}  // namespace irk

using irk::Ctx;

extern "C" {

void irk_default_options(irk_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->kind = IRK_PC_LD;
  o->Atilde = nullptr;
  o->amg_prec = IRK_AMG_F32;
  o->smoother = IRK_SMOOTH_CHEBYSHEV;
  o->cheb_degree = 4;
  o->cheb_lo = 0.1;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->theta = 0.08;
  o->coarse_max = 2048;
  o->max_levels = 12;
  o->restart = 30;
  o->rtol = 1e-10;
  o->max_it = 1000;
  o->reorth = 0;
  o->reorth_eta = 0.1;
  o->side = 0;
  o->p_smooth = 2;
  o->strength = 0;
  o->cycle = IRK_CYCLE_V;
}

const char* irk_status_string(irk_status st) {
  switch (st) {
    case IRK_OK: return "ok";
    case IRK_ERR_INVALID: return "invalid argument";
    case IRK_ERR_NOMEM: return "out of device memory";
    case IRK_ERR_CUDA: return "CUDA error";
    case IRK_ERR_NOT_CONVERGED: return "not converged";
    case IRK_ERR_BREAKDOWN: return "breakdown";
    case IRK_ERR_ZERO_PIVOT: return "zero pivot";
    case IRK_ERR_NONFINITE: return "non-finite value";
    case IRK_ERR_TIMEOUT: return "device wait timed out";
    case IRK_ERR_CAPACITY: return "capacity exceeded";
  }
  return "unknown status";
}

const char* irk_last_error(const irk_ctx* h) { return h ? h->c.err.c_str() : g_err.c_str(); }

irk_status irk_setup(const irk_problem* prob, const irk_butcher* bt, double h_t, const irk_options* opt,
                     void* stream, irk_ctx** out) {
  if (out) *out = nullptr;
  if (!prob || !bt || !out) return set_err(nullptr, IRK_ERR_INVALID, "NULL argument");
  if (bt->s < 1 || bt->s > irk::MAX_S || !bt->A || !bt->b) return set_err(nullptr, IRK_ERR_INVALID, "s must be 1..8");
  if (!(h_t > 0.0) || !std::isfinite(h_t)) return set_err(nullptr, IRK_ERR_INVALID, "h_t must be positive");
  irk_options o;
  if (opt) o = *opt;
  else irk_default_options(&o);
  if (o.kind < IRK_PC_J || o.kind > IRK_PC_CUSTOM) return set_err(nullptr, IRK_ERR_INVALID, "unknown preconditioner kind");
  if (o.kind == IRK_PC_CUSTOM && !o.Atilde) return set_err(nullptr, IRK_ERR_INVALID, "IRK_PC_CUSTOM needs Atilde");
  if (o.smoother != IRK_SMOOTH_L1JACOBI && o.smoother != IRK_SMOOTH_CHEBYSHEV)
    return set_err(nullptr, IRK_ERR_INVALID, "unknown smoother");
  if (!(o.cheb_lo > 0.0 && o.cheb_lo < 1.0)) return set_err(nullptr, IRK_ERR_INVALID, "cheb_lo must lie in (0, 1)");
  if (!(o.theta >= 0.0 && o.theta <= 1.0)) return set_err(nullptr, IRK_ERR_INVALID, "theta must lie in [0, 1]");
  if (o.max_levels < 1 || o.max_levels > irk::MAX_LEVELS)
    return set_err(nullptr, IRK_ERR_INVALID, "max_levels must be 1..16");
  if (o.restart < 1 || o.restart > irk::MAX_M) return set_err(nullptr, IRK_ERR_INVALID, "restart must be 1..64");
  if (o.amg_prec != 64 && o.amg_prec != 32 && o.amg_prec != 16)
    return set_err(nullptr, IRK_ERR_INVALID, "amg_prec must be 64, 32 or 16");
  if (o.cheb_degree < 1 || o.cheb_degree > 16) return set_err(nullptr, IRK_ERR_INVALID, "cheb_degree must be 1..16");
  if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post == 0)
    return set_err(nullptr, IRK_ERR_INVALID, "need at least one smoothing sweep");
  if (!(o.rtol > 0.0) || o.max_it < 1) return set_err(nullptr, IRK_ERR_INVALID, "bad rtol/max_it");
  if (!(o.reorth_eta >= 0.0 && o.reorth_eta < 1.0) || o.reorth < 0 || o.reorth > 1)
    return set_err(nullptr, IRK_ERR_INVALID, "reorth must be 0 or 1 and 0 <= reorth_eta < 1");
  if (o.side != 0 && o.side != 1) return set_err(nullptr, IRK_ERR_INVALID, "side must be 0 (right) or 1 (left)");
  if (o.p_smooth < 1 || o.p_smooth > 3) return set_err(nullptr, IRK_ERR_INVALID, "p_smooth must be 1, 2 or 3");
  if (o.strength != 0 && o.strength != 1) return set_err(nullptr, IRK_ERR_INVALID, "strength must be 0 or 1");
  if (o.cycle != IRK_CYCLE_V && o.cycle != IRK_CYCLE_W_COARSE)
    return set_err(nullptr, IRK_ERR_INVALID, "cycle must be IRK_CYCLE_V or IRK_CYCLE_W_COARSE");
  if (o.coarse_max < 1 || o.coarse_max > irk::MAX_COARSE)
    return set_err(nullptr, IRK_ERR_INVALID, "coarse_max must be 1..2048");
  const irk_csr& M = prob->M;
  const irk_csr& F = prob->F;
  if (M.n != F.n || M.nnz != F.nnz || M.n < 1) return set_err(nullptr, IRK_ERR_INVALID, "M and F differ in size");
  if (!M.rowptr || !F.rowptr || M.nnz < 0 || (M.nnz > 0 && (!M.col || !F.col || !M.val || !F.val)))
    return set_err(nullptr, IRK_ERR_INVALID, "bad CSR matrix");
  if (M.rowptr[0] != 0 || M.rowptr[M.n] != M.nnz)
    return set_err(nullptr, IRK_ERR_INVALID, "CSR rowptr must start at 0 and end at nnz");
  for (int i = 0; i <= M.n; ++i) {
    if (M.rowptr[i] != F.rowptr[i]) return set_err(nullptr, IRK_ERR_INVALID, "M and F must share one pattern");
    if (i > 0 && M.rowptr[i] < M.rowptr[i - 1]) return set_err(nullptr, IRK_ERR_INVALID, "CSR rowptr not monotone");
  }
  for (int64_t k = 0; k < M.nnz; ++k) {
    if (M.col[k] != F.col[k]) return set_err(nullptr, IRK_ERR_INVALID, "M and F must share one pattern");
    if (M.col[k] < 0 || M.col[k] >= M.n) return set_err(nullptr, IRK_ERR_INVALID, "CSR column index out of range");
  }
  if (prob->n_tri > 0 && (!prob->xy || !prob->tri || !prob->dof || prob->n_nodes <= 0))
    return set_err(nullptr, IRK_ERR_INVALID, "incomplete mesh");

  irk_ctx* h = new irk_ctx();
  Ctx& c = h->c;
  irk_status st = guarded(h, [&] {
    CK(cudaGetDevice(&c.device));
    c.user_stream = static_cast<cudaStream_t>(stream);
    CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c.ev_a, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c.ev_b, cudaEventDisableTiming));
    CK(cudaEventCreate(&c.ev_t0));
    CK(cudaEventCreate(&c.ev_t1));
    irk::begin_call(c);
    c.opt = o;
    c.opt.Atilde = nullptr;
    c.n = M.n;
    c.s = bt->s;
    c.h = h_t;
    c.m = o.restart;
    c.max_it = o.max_it;
    c.rtol = o.rtol;
    c.reorth = o.reorth;
    c.reorth_eta = o.reorth_eta;
    c.side = o.side;
    c.kind = o.kind;
    c.amg.theta = o.theta;
    c.amg.coarse_max = o.coarse_max;
    c.amg.max_levels = o.max_levels;
    c.amg.smoother = o.smoother;
    c.amg.cheb_degree = o.cheb_degree;
    c.amg.cheb_lo = o.cheb_lo;
    c.amg.p_smooth = o.p_smooth;
    c.amg.strength_negative = o.strength;
    c.amg.w_coarse = o.cycle == IRK_CYCLE_W_COARSE ? 1 : 0;
    c.amg.nu_pre = o.nu_pre;
    c.amg.nu_post = o.nu_post;
    c.amg.amg_prec = o.amg_prec;
    c.sc = irk::smooth_coefficients(c.amg);
    int s = c.s;
    for (int i = 0; i < s * s; ++i) c.A[i] = bt->A[i];
    for (int i = 0; i < s; ++i) {
      c.b[i] = bt->b[i];
      c.c[i] = bt->c ? bt->c[i] : 0.0;
    }
    if (o.kind == IRK_PC_CUSTOM) {
      if (!o.Atilde) irk::fail(IRK_ERR_INVALID, "IRK_PC_CUSTOM needs Atilde");
      for (int i = 0; i < s * s; ++i) c.At[i] = o.Atilde[i];
    } else {
      irk_status a = irk_atilde(o.kind, s, bt->A, c.At, nullptr);
      if (a != IRK_OK) irk::fail(a, irk_last_error(nullptr));
    }
    for (int i = 0; i < irk::MAX_S * irk::MAX_S; ++i) {
      c.K.a[i] = 0.0;
      c.KT.a[i] = 0.0;
    }
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) {
        c.K.a[i * irk::MAX_S + j] = h_t * c.A[i * s + j];
        c.KT.a[i * irk::MAX_S + j] = h_t * c.A[j * s + i];
      }
    irk::csr_upload(M, c.Mc, c.pool, c.stream);
    irk::csr_upload(F, c.Fc, c.pool, c.stream);
    c.pool.release(c.Fc.rowptr);
    c.pool.release(c.Fc.col);
    c.Fc.rowptr = c.Mc.rowptr;
    c.Fc.col = c.Mc.col;
    irk::csr_to_sell(c.Mc, c.Ms, 1, 0, 0, c.pool, c.stream);
    irk::sell_share_pattern(c.Ms, c.Fc.val, c.Fc, c.Fs, 1, 1, c.pool, c.stream);
    irk::kron_split_build(c);
    if (prob->stab) {
      c.Tval = c.pool.get<double>(M.nnz > 0 ? M.nnz : 1);
      if (M.nnz) CK(cudaMemcpy(c.Tval, prob->stab, sizeof(double) * M.nnz, cudaMemcpyHostToDevice));
    }
    c.g = c.pool.get<double>(c.n);
    if (prob->g) CK(cudaMemcpy(c.g, prob->g, sizeof(double) * c.n, cudaMemcpyHostToDevice));
    else CK(cudaMemset(c.g, 0, sizeof(double) * c.n));
    c.symmetric = irk::csr_symmetric(M) && irk::csr_symmetric(F);
    if (prob->n_tri > 0) {
      std::vector<int> rp(M.n + 1), col(M.nnz);
      for (int i = 0; i <= M.n; ++i) rp[i] = static_cast<int>(M.rowptr[i]);
      for (int64_t k = 0; k < M.nnz; ++k) col[k] = M.col[k];
      irk::setup_mesh(c, *prob, rp, col);
    }
    const char* hl = std::getenv("IRK_HOST_LOOP");
    c.host_loop = hl && std::atoi(hl) != 0;
    CK(cudaMallocHost(&c.h_flag, sizeof(int)));
    irk::alloc_solver_buffers(c);
    irk::build_hierarchies(c);
    CK(cudaStreamSynchronize(c.stream));
  });
  if (st != IRK_OK) {
    std::string msg = c.err;
    irk_destroy(h);
    return set_err(nullptr, st, msg);
  }
  *out = h;
  return IRK_OK;
}

irk_status irk_step(irk_ctx* h, const double* d_u_n, double* d_u_np1, double* d_k, irk_stats* stats) {
  if (!h || !d_u_n || !d_u_np1) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  irk_status dev = IRK_OK;
  irk_status st = guarded(h, [&] {
    Ctx& c = h->c;
    irk::build_graph(c, false);
    irk::begin_call(c);
    CK(cudaMemcpyAsync(c.u, d_u_n, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
    irk::reset_records(c);
    CK(cudaEventRecord(c.ev_t0, c.stream));
    irk::launch_solve(c, false);
    CK(cudaEventRecord(c.ev_t1, c.stream));
    if (d_k) CK(cudaMemcpyAsync(d_k, c.x, sizeof(double) * c.N, cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaMemcpyAsync(d_u_np1, c.u, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
    irk::collect_stats(c, 1, stats, &dev, 0);
    irk::end_call(c);
  });
  if (st != IRK_OK) return st;
  if (dev != IRK_OK) return set_err(h, dev, std::string("device solve: ") + irk_status_string(dev));
  return IRK_OK;
}

irk_status irk_solve(irk_ctx* h, const double* d_b, double* d_k, irk_stats* stats) {
  if (!h || !d_b || !d_k) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  irk_status dev = IRK_OK;
  irk_status st = guarded(h, [&] {
    Ctx& c = h->c;
    irk::build_graph(c, false);
    irk::begin_call(c);
    CK(cudaMemcpyAsync(c.bv, d_b, sizeof(double) * c.N, cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaMemsetAsync(c.rhs_given, 0x01, 1, c.stream));
    irk::reset_records(c);
    CK(cudaEventRecord(c.ev_t0, c.stream));
    irk::launch_solve(c, false);
    CK(cudaEventRecord(c.ev_t1, c.stream));
    CK(cudaMemsetAsync(c.rhs_given, 0, sizeof(int), c.stream));
    CK(cudaMemcpyAsync(d_k, c.x, sizeof(double) * c.N, cudaMemcpyDeviceToDevice, c.stream));
    irk::collect_stats(c, 1, stats, &dev, 0);
    irk::end_call(c);
  });
  if (st != IRK_OK) return st;
  if (dev != IRK_OK) return set_err(h, dev, std::string("device solve: ") + irk_status_string(dev));
  return IRK_OK;
}

irk_status irk_run(irk_ctx* h, const double* d_u0, int32_t nsteps, double* d_u_out, double* d_ckpt,
                   int32_t ckpt_every, irk_stats* stats) {
  if (!h || !d_u0 || !d_u_out || nsteps < 0) return set_err(h, IRK_ERR_INVALID, "bad argument");
  if (d_ckpt && ckpt_every < 1) return set_err(h, IRK_ERR_INVALID, "ckpt_every must be >= 1");
  irk_status dev = IRK_OK;
  irk_status st = guarded(h, [&] { dev = irk::run_steps(h->c, d_u0, nsteps, d_u_out, d_ckpt, ckpt_every, nullptr, stats); });
  if (st != IRK_OK) return st;
  if (dev != IRK_OK) return set_err(h, dev, std::string("device solve: ") + irk_status_string(dev));
  return IRK_OK;
}

irk_status irk_adjoint_step(irk_ctx* h, const double* d_lambda_np1, const double* d_u_n, const double* d_k_n,
                            double* d_lambda_n, double* d_grad_kappa, irk_stats* stats) {
  if (!h || !d_lambda_np1 || !d_lambda_n) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  if (d_grad_kappa && (!d_u_n || !d_k_n)) return set_err(h, IRK_ERR_INVALID, "gradient needs u_n and k_n");
  irk_status dev = IRK_OK;
  irk_status st = guarded(h, [&] {
    Ctx& c = h->c;
    irk::check_adjoint_ok(c, d_grad_kappa != nullptr);
    irk::build_graph(c, true);
    irk::begin_call(c);
    irk::reset_records(c);
    CK(cudaEventRecord(c.ev_t0, c.stream));
    irk::adjoint_one(c, d_lambda_np1, d_u_n, d_k_n, d_lambda_n, d_grad_kappa, true);
    CK(cudaEventRecord(c.ev_t1, c.stream));
    irk::collect_stats(c, 1, stats, &dev, 1);
    irk::end_call(c);
  });
  if (st != IRK_OK) return st;
  if (dev != IRK_OK) return set_err(h, dev, std::string("device adjoint solve: ") + irk_status_string(dev));
  return IRK_OK;
}

irk_status irk_adjoint_run(irk_ctx* h, const double* d_ckpt, int32_t nsteps, int32_t every, double* d_lambda,
                           double* d_grad_kappa, irk_stats* stats) {
  if (!h || !d_ckpt || !d_lambda || nsteps < 0 || every < 1) return set_err(h, IRK_ERR_INVALID, "bad argument");
  irk_status dev = IRK_OK;
  irk_status st = guarded(h, [&] {
    Ctx& c = h->c;
    irk::check_adjoint_ok(c, d_grad_kappa != nullptr);
    irk::build_graph(c, false);
    irk::build_graph(c, true);
    if (c.kstore_cap < every) {
      c.pool.release(c.kstore);
      c.pool.release(c.ustore);
      c.kstore = c.pool.get<double>(size_t(every) * c.N);
      c.ustore = c.pool.get<double>(size_t(every) * c.n);
      c.kstore_cap = every;
    }
    irk::begin_call(c);
    CK(cudaEventRecord(c.ev_t0, c.stream));
    int nseg = (nsteps + every - 1) / every;
    int fwd_steps = 0, adj_steps = 0;
    std::vector<irk::StepRecord> all;
    CK(cudaMemcpyAsync(c.lam, d_lambda, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
    for (int q = nseg - 1; q >= 0; --q) {
      int s0 = q * every, s1 = std::min(nsteps, s0 + every);
      irk::reset_records(c);
      CK(cudaMemcpyAsync(c.u, d_ckpt + int64_t(q) * c.n, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
      for (int t = s0; t < s1; ++t) {
        CK(cudaMemcpyAsync(c.ustore + int64_t(t - s0) * c.n, c.u, sizeof(double) * c.n, cudaMemcpyDeviceToDevice,
                           c.stream));
        irk::launch_solve(c, false);
        CK(cudaMemcpyAsync(c.kstore + int64_t(t - s0) * c.N, c.x, sizeof(double) * c.N, cudaMemcpyDeviceToDevice,
                           c.stream));
      }
      for (int t = s1 - 1; t >= s0; --t) {
        irk::launch_solve(c, true);
        if (d_grad_kappa)
          irk::adjoint_grad_launch(c, c.ustore + int64_t(t - s0) * c.n, c.kstore + int64_t(t - s0) * c.N, d_grad_kappa,
                                   c.stream);
        CK(cudaMemcpyAsync(c.lam, c.tmpn, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
      }
      std::vector<irk::StepRecord> rec(2 * (s1 - s0));
      CK(cudaMemcpyAsync(rec.data(), c.rec, sizeof(irk::StepRecord) * rec.size(), cudaMemcpyDeviceToHost, c.stream));
      CK(cudaStreamSynchronize(c.stream));
      for (size_t i = 0; i < rec.size(); ++i) all.push_back(rec[i]);
      fwd_steps += s1 - s0;
      adj_steps += s1 - s0;
    }
    CK(cudaEventRecord(c.ev_t1, c.stream));
    CK(cudaMemcpyAsync(d_lambda, c.lam, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c.ev_t0, c.ev_t1));
    irk_stats s{};
    s.steps = nsteps;
    s.ms = ms;
    int64_t its_f = 0, its_a = 0;
    size_t idx = 0;
    for (int q = nseg - 1; q >= 0; --q) {
      int s0 = q * every, s1 = std::min(nsteps, s0 + every);
      for (int t = s0; t < s1; ++t, ++idx) its_f += std::max(all[idx].it, 1);
      for (int t = s0; t < s1; ++t, ++idx) {
        const auto& r = all[idx];
        s.iterations += r.it;
        s.restarts += r.restarts;
        s.max_step_iterations = std::max(s.max_step_iterations, r.it);
        s.resid = r.resid;
        its_a += std::max(r.it, 1);
        if (r.status != IRK_OK && dev == IRK_OK) dev = static_cast<irk_status>(r.status);
      }
    }
    if (!c.host_loop) {
      c.launches += c.graph[0].fixed_kernels * fwd_steps + c.graph[0].body_kernels * its_f;
      c.launches += c.graph[1].fixed_kernels * adj_steps + c.graph[1].body_kernels * its_a;
    }
    if (d_grad_kappa) c.launches += adj_steps;
    if (stats) *stats = s;
    irk::end_call(c);
  });
  if (st != IRK_OK) return st;
  if (dev != IRK_OK) return set_err(h, dev, std::string("device adjoint solve: ") + irk_status_string(dev));
  return IRK_OK;
}

irk_status irk_set_kappa(irk_ctx* h, const double* d_kappa) {
  if (!h || !d_kappa) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    if (c.n_tri == 0) irk::fail(IRK_ERR_INVALID, "irk_set_kappa needs the mesh in irk_setup");
    irk::begin_call(c);
    irk::assemble_kappa_launch(c, d_kappa, c.Fc.val, c.stream);
    c.launches += 1;
    // refresh the SELL copies of F and rebuild the hierarchies
    c.pool.release(c.Fs.v64);
    c.pool.release(c.Fs.v32);
    irk::sell_share_pattern(c.Ms, c.Fc.val, c.Fc, c.Fs, 1, 1, c.pool, c.stream);
    irk::kron_split_build(c);
    irk::destroy_graphs(c);
    irk::build_hierarchies(c);
    if (c.tr.built) {   // the transposed problem follows F
      for (auto& H : c.tr.hiers) H.pool.free_all();
      c.tr.hiers.clear();
      c.tr = irk::Ctx::Transposed{};
    }
    irk::end_call(c);
  });
}

irk_status irk_apply_operator(irk_ctx* h, const double* d_z, double* d_w, int32_t transpose) {
  if (!h || !d_z || !d_w) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    irk::AdjointView av(c, transpose != 0);
    irk::begin_call(c);
    irk::kron_apply_plain(c, d_z, d_w, transpose != 0, c.stream);
    c.launches += 1;
    irk::end_call(c);
  });
}

irk_status irk_apply_operator_f32(irk_ctx* h, const float* d_z, double* d_w, int32_t transpose) {
  if (!h || !d_z || !d_w) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    irk::AdjointView av(c, transpose != 0);
    irk::begin_call(c);
    irk::kron_apply_f32(c, d_z, d_w, transpose != 0, c.stream);
    c.launches += 1;
    irk::end_call(c);
  });
}

irk_status irk_apply_precond(irk_ctx* h, const double* d_v, double* d_z, int32_t transpose) {
  if (!h || !d_v || !d_z) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    irk::AdjointView av(c, transpose != 0);
    irk::begin_call(c);
    irk::PrecondArgs pa{d_v, nullptr, 0, nullptr, c.Z, 0, nullptr};
    c.launches += irk::precond_launch(c, pa, transpose != 0, c.stream);
    irk::convert_launch(c.Z, c.amg.amg_prec == 64 ? 64 : 32, d_z, 64, c.N, c.stream);
    c.launches += 1;
    irk::end_call(c);
  });
}

irk_status irk_vcycle(irk_ctx* h, int32_t stage, const double* d_b, double* d_x) {
  if (!h || !d_b || !d_x) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    if (stage < 0 || stage >= c.s) irk::fail(IRK_ERR_INVALID, "stage out of range");
    int pos = 0;
    while (c.plan.order[pos] != stage) ++pos;
    const irk::Hier& H = c.hiers[c.plan.hier[pos]];
    int prec = c.amg.amg_prec == 64 ? 64 : 32;
    irk::begin_call(c);
    irk::convert_launch(d_b, 64, H.lv[0].b, prec, c.n, c.stream);
    c.launches += 1 + irk::vcycle_launch(H, c.amg, c.sc, c.Z, nullptr, 0, 0, c.stream);
    irk::convert_launch(c.Z, prec, d_x, 64, c.n, c.stream);
    c.launches += 1;
    irk::end_call(c);
  });
}

irk_status irk_residual_norm(irk_ctx* h, const double* d_k, const double* d_b, double* norm) {
  if (!h || !d_k || !d_b || !norm) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    irk::begin_call(c);
    // scratch: the context's partial-sum buffer (gs_grid slots), result in tmpn[0]
    irk::residual_norm_launch(c, d_k, d_b, c.partials, c.gs_grid, c.tmpn, c.stream);
    c.launches += 2;
    CK(cudaMemcpyAsync(norm, c.tmpn, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    irk::end_call(c);
  });
}

irk_status irk_apply_mass(irk_ctx* h, const double* d_x, double* d_y) {
  if (!h || !d_x || !d_y) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    irk::begin_call(c);
    irk::mass_apply_launch(c, d_x, d_y, c.stream);
    c.launches += 1;
    irk::end_call(c);
  });
}

irk_status irk_misfit(irk_ctx* h, const double* d_u, const double* d_d, double* d_grad, double* d_value) {
  if (!h || !d_u || !d_d || !d_value) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    irk::begin_call(c);
    irk::misfit_launch(c, d_u, d_d, d_grad, d_value, c.stream);
    c.launches += 2;
    irk::end_call(c);
  });
}

static const irk::Hier* hier_of(Ctx& c, int stage) {
  if (stage < 0 || stage >= c.s) irk::fail(IRK_ERR_INVALID, "stage out of range");
  int pos = 0;
  while (c.plan.order[pos] != stage) ++pos;
  return &c.hiers[c.plan.hier[pos]];
}

irk_status irk_amg_info(irk_ctx* h, int32_t stage, int32_t* nlevels, int32_t* rows, int64_t* nnz) {
  if (!h || !nlevels) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    const irk::Hier* H = hier_of(h->c, stage);
    *nlevels = static_cast<int32_t>(H->lv.size());
    for (size_t l = 0; l < H->lv.size() && l < 16; ++l) {
      if (rows) rows[l] = H->lv[l].n;
      if (nnz) nnz[l] = H->lv[l].nnz;
    }
  });
}

irk_status irk_amg_aggregates(irk_ctx* h, int32_t stage, int32_t level, int32_t* agg) {
  if (!h || !agg) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    const irk::Hier* H = hier_of(h->c, stage);
    if (level < 0 || level + 1 >= static_cast<int>(H->lv.size())) irk::fail(IRK_ERR_INVALID, "level out of range");
    CK(cudaMemcpy(agg, H->lv[level].agg, sizeof(int) * H->lv[level].n, cudaMemcpyDeviceToHost));
  });
}

irk_status irk_amg_level_matrix(irk_ctx* h, int32_t stage, int32_t level, int64_t* rowptr, int32_t* col,
                                double* val) {
  if (!h || !rowptr || !col || !val) return set_err(h, IRK_ERR_INVALID, "NULL argument");
  return guarded(h, [&] {
    const irk::Hier* H = hier_of(h->c, stage);
    if (level < 0 || level >= static_cast<int>(H->lv.size())) irk::fail(IRK_ERR_INVALID, "level out of range");
    std::vector<int> rp, cl;
    std::vector<double> vl;
    irk::csr_copy_to_host(H->lv[level].A, rp, cl, vl, h->c.stream);
    for (size_t i = 0; i < rp.size(); ++i) rowptr[i] = rp[i];
    std::copy(cl.begin(), cl.end(), col);
    std::copy(vl.begin(), vl.end(), val);
  });
}

irk_status irk_profile(irk_ctx* h, int32_t which, int32_t j, int32_t warm, int32_t reps, double* ms, double* bytes,
                       double* flops) {
  if (!h || !ms || reps < 1 || warm < 0) return set_err(h, IRK_ERR_INVALID, "bad argument");
  return guarded(h, [&] {
    Ctx& c = h->c;
    double B = 0.0, Fl = 0.0;
    irk::GmresState* scratch = nullptr;
    irk::GmresState host_state;
    std::function<void()> prep = [] {};
    std::function<void()> launch;
    const irk::Hier& H0 = c.hiers[c.plan.hier[0]];
    switch (which) {
      case IRK_PROF_KRON: {
        launch = [&] { irk::profile_kron_launch(c, c.stream); };
        double zs = c.amg.amg_prec == 64 ? 8.0 : 4.0;
        const double idx = irk::offset_bytes_per_entry(c.Ms);
        // per nonzero: M and F (two FP64, or one float4 of single-float pairs) and its column
        B = double(c.Mc.nnz) * (16.0 + idx) + double(c.N) * (zs + 8.0);
        Fl = 2.0 * (2.0 * c.s * double(c.Mc.nnz) + double(c.s) * c.s * c.n);
        break;
      }
      case IRK_PROF_VCYCLE: {
        irk::vcycle_launch(H0, c.amg, c.sc, c.Z, nullptr, 0, 0, c.stream, &B, &Fl);   // accounting pass
        launch = [&] { irk::vcycle_launch(H0, c.amg, c.sc, c.Z, nullptr, 0, 0, c.stream); };
        break;
      }
      case IRK_PROF_PRECOND: {
        irk::PrecondArgs pa{c.V, nullptr, 0, nullptr, c.Z, 0, nullptr, &B, &Fl};
        irk::precond_launch(c, pa, false, c.stream);
        irk::PrecondArgs pb{c.V, nullptr, 0, nullptr, c.Z, 0, nullptr};
        launch = [&, pb] { irk::precond_launch(c, pb, false, c.stream); };
        break;
      }
      case IRK_PROF_GS_DOTS:
      case IRK_PROF_GS_AXPY: {
        if (j < 0 || j + 1 > c.m) irk::fail(IRK_ERR_INVALID, "j out of range");
        scratch = c.pool.get<irk::GmresState>(1);
        std::memset(&host_state, 0, sizeof(host_state));
        host_state.j = j;
        host_state.m = irk::MAX_M;
        host_state.max_it = 1 << 30;
        host_state.rtol = 0.0;
        host_state.bnorm = 1.0;
        host_state.wnorm2 = 0.0;   // never reorthogonalise
        for (int i = 0; i <= irk::MAX_M; ++i) host_state.sigma[i] = 1.0;
        for (int i = 0; i <= j; ++i) host_state.H[j * (irk::MAX_M + 1) + i] = 1e-3;
        host_state.g[0] = 1.0;
        bool axpy = which == IRK_PROF_GS_AXPY;
        prep = [&] {
          CK(cudaMemcpyAsync(scratch, &host_state, sizeof(host_state), cudaMemcpyHostToDevice, c.stream));
        };
        launch = [&, axpy] { irk::profile_gs_launch(c, scratch, axpy, c.stream); };
        double N = double(c.N);
        B = axpy ? (j + 3) * N * 8.0 : (j + 2) * N * 8.0;
        Fl = axpy ? 2.0 * (j + 2) * N : 2.0 * (j + 2) * N;
        break;
      }
      case IRK_PROF_VCYCLE_FROM: {
        // j = the first level (>= 1) of the partial V-cycle
        irk::vcycle_launch_from(H0, c.amg, c.sc, j, c.stream, &B, &Fl);
        launch = [&] { irk::vcycle_launch_from(H0, c.amg, c.sc, j, c.stream); };
        break;
      }
      case IRK_PROF_SMOOTH0: {
        irk::smooth0_launch(H0, c.amg, c.sc, c.stream, &B, &Fl);
        launch = [&] {
          double b2, f2;
          irk::smooth0_launch(H0, c.amg, c.sc, c.stream, &b2, &f2);
        };
        break;
      }
      default:
        irk::fail(IRK_ERR_INVALID, "unknown profile target");
    }
    irk::begin_call(c);
    for (int w = 0; w < warm; ++w) {
      prep();
      launch();
    }
    double total = 0.0;
    for (int r = 0; r < reps; ++r) {
      prep();
      CK(cudaEventRecord(c.ev_t0, c.stream));
      launch();
      CK(cudaEventRecord(c.ev_t1, c.stream));
      CK(cudaEventSynchronize(c.ev_t1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, c.ev_t0, c.ev_t1));
      total += t;
    }
    irk::end_call(c);
    if (scratch) c.pool.release(scratch);
    *ms = total / reps;
    if (bytes) *bytes = B;
    if (flops) *flops = Fl;
  });
}

int64_t irk_kernel_launches(const irk_ctx* h) { return h ? h->c.launches : 0; }

void irk_destroy(irk_ctx* h) {
  if (!h) return;
  Ctx& c = h->c;
  cudaSetDevice(c.device);
  if (c.stream) cudaStreamSynchronize(c.stream);
  irk::destroy_graphs(c);
  for (auto& H : c.hiers) H.pool.free_all();
  for (auto& H : c.tr.hiers) H.pool.free_all();
  c.pool.free_all();
  if (c.ev_a) cudaEventDestroy(c.ev_a);
  if (c.ev_b) cudaEventDestroy(c.ev_b);
  if (c.ev_t0) cudaEventDestroy(c.ev_t0);
  if (c.ev_t1) cudaEventDestroy(c.ev_t1);
  if (c.stream) cudaStreamDestroy(c.stream);
  if (c.h_flag) cudaFreeHost(c.h_flag);
  delete h;
}

}  // extern "C"
