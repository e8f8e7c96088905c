// Batched instances: one CUDA graph advances any number of independent
// problems (contexts of different sizes) through all their time steps, or
// through the whole checkpointed adjoint sweep, in a single graph launch.
//
// Each instance is an independent chain of the graph, so the GPU runs the
// instances concurrently.  Inside a chain, the time-step loop is a WHILE node
// whose body holds the step (right-hand side, the FGMRES WHILE node, update)
// and a control kernel that advances a device step counter; nothing returns to
// the host until every instance is done.
#include "irk_internal.cuh"

#include <algorithm>
#include <vector>

namespace irk {

// ---------------------------------------------------------------------------
// small control kernels
// ---------------------------------------------------------------------------
__global__ void k_set_int(int* p, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, v);
}

// step += delta; loop while lo <= step < hi
__global__ void k_step_ctrl(int* step, int delta, int lo, int hi, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int s = *step + delta;
    *step = s;
    cudaGraphSetConditional(h, (s >= lo && s < hi) ? 1u : 0u);
  }
}

// dst[(*step / every) * n + r] = src[r] when *step % every == 0
__global__ void k_ckpt_store(const int* step, int every, double* __restrict__ dst, const double* __restrict__ src,
                             int n) {
  int s = *step;
  if (s % every) return;
  double* d = dst + int64_t(s / every) * n;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) d[r] = src[r];
}

// dst[(*step) * len + i] = src[i]  (segment stores of u and k)
__global__ void k_store_at(const int* step, double* __restrict__ dst, const double* __restrict__ src, int64_t len) {
  double* d = dst + int64_t(*step) * len;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < len; i += int64_t(gridDim.x) * blockDim.x)
    d[i] = src[i];
}

__global__ void k_copy(double* __restrict__ dst, const double* __restrict__ src, int64_t len) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < len; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// graph construction helpers
// ---------------------------------------------------------------------------
struct Builder {
  cudaStream_t st;
  cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  int64_t kernels = 0;

  // capture fn into graph after deps; returns the sink nodes
  template <typename Fn>
  std::vector<cudaGraphNode_t> capture(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, Fn fn) {
    CK(cudaStreamBeginCaptureToGraph(st, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), mode));
    fn(st);
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(st, &status, nullptr, nullptr, &d, nullptr, &nd));
    std::vector<cudaGraphNode_t> sinks(d, d + nd);
    cudaGraph_t out;
    CK(cudaStreamEndCapture(st, &out));
    return sinks;
  }

  // WHILE node after deps; body graph returned, handle created on g
  std::vector<cudaGraphNode_t> add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                                         cudaGraphConditionalHandle* h, cudaGraph_t* body) {
    CK(cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = *h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
    *body = cp.conditional.phGraph_out[0];
    return {node};
  }

  // one stage solve (forward or adjoint) into graph g after deps:
  // [set inner condition] head -> WHILE(FGMRES iteration) -> tail
  std::vector<cudaGraphNode_t> solve(Ctx& c, bool adjoint, cudaGraph_t g, std::vector<cudaGraphNode_t> deps) {
    cudaGraphConditionalHandle hi;
    CK(cudaGraphConditionalHandleCreate(&hi, g, 1, cudaGraphCondAssignDefault));
    deps = capture(g, deps, [&](cudaStream_t s) {
      k_set_cond<<<1, 32, 0, s>>>(hi, 1u);
      if (adjoint) rhs_adjoint_launch(c, c.lam, s);
      else rhs_forward_launch(c, c.u, s);
    });
    kernels += 2;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hi;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    CK(cudaGraphAddNode(&loop, g, deps.data(), nullptr, deps.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    capture(body, {}, [&](cudaStream_t s) {
      PrecondArgs pa{c.V, &c.st->j, c.N, c.st->sigma, c.Z, c.N, &c.st->done};
      precond_launch(c, pa, adjoint, s);
      fgmres_body_launch(c, adjoint, s);
      set_loop_condition_launch(c, hi, s);
    });
    return capture(g, {loop}, [&](cudaStream_t s) {
      if (adjoint) adjoint_lambda_launch(c, c.lam, c.tmpn, s);
      else stage_update_launch(c, c.u, s);
      record_launch(c, s);
    });
  }
};

struct Instance {
  Ctx* c;
  int* step = nullptr;         // device step counter
  double* ustore = nullptr;    // every x n
  double* kstore = nullptr;    // every x s n
};

}  // namespace irk

struct irk_batch {
  std::vector<irk::Instance> inst;
  int nsteps = 0, every = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t fwd = nullptr, adj = nullptr;
  cudaGraph_t gfwd = nullptr, gadj = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  irk::DevPool pool;
  std::string err;
};

using irk::Builder;
using irk::Ctx;

static unsigned grid_n(int64_t n) { return static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4096)); }

extern "C" {

irk_status irk_batch_create(irk_ctx* const* ctxs, int32_t count, int32_t nsteps, int32_t ckpt_every,
                            const double* const* d_u0, double* const* d_uN, double* const* d_ckpt,
                            double* const* d_lambda, double* const* d_grad_kappa, irk_batch** out) {
  if (out) *out = nullptr;
  if (!ctxs || count < 1 || nsteps < 1 || ckpt_every < 1 || !d_u0 || !d_uN || !d_ckpt || !out) {
    irk::set_global_error("bad argument to irk_batch_create");
    return IRK_ERR_INVALID;
  }
  irk_batch* b = new irk_batch();
  b->nsteps = nsteps;
  b->every = ckpt_every;
  try {
    int dev = ctxs[0]->c.device;
    for (int q = 0; q < count; ++q) {
      if (!ctxs[q] || ctxs[q]->c.device != dev) irk::fail(IRK_ERR_INVALID, "all batch contexts must share one device");
      if (!d_u0[q] || !d_uN[q] || !d_ckpt[q]) irk::fail(IRK_ERR_INVALID, "NULL instance buffer");
      if (ctxs[q]->c.side != 0) irk::fail(IRK_ERR_INVALID, "batches run right-preconditioned contexts only");
      if (d_lambda && d_grad_kappa && d_grad_kappa[q] && ctxs[q]->c.n_tri == 0)
        irk::fail(IRK_ERR_INVALID, "kappa gradients of an instance need its mesh");
    }
    CK(cudaSetDevice(dev));
    CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&b->e0));
    CK(cudaEventCreate(&b->e1));
    Builder B{b->stream};
    // ---------------- forward: every instance through nsteps steps
    CK(cudaGraphCreate(&b->gfwd, 0));
    for (int q = 0; q < count; ++q) {
      Ctx& c = ctxs[q]->c;
      irk::Instance I{&c};
      I.step = b->pool.get<int>(1);
      if (d_lambda) {
        I.ustore = b->pool.get<double>(size_t(ckpt_every) * c.n);
        I.kstore = b->pool.get<double>(size_t(ckpt_every) * c.N);
      }
      b->inst.push_back(I);
      const double* u0 = d_u0[q];
      double* uN = d_uN[q];
      double* ck = d_ckpt[q];
      auto deps = B.capture(b->gfwd, {}, [&](cudaStream_t s) {
        CK(cudaMemcpyAsync(c.u, u0, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(c.step_counter, 0, sizeof(int), s));
        irk::k_set_int<<<1, 32, 0, s>>>(I.step, 0);
      });
      cudaGraphConditionalHandle hs;
      cudaGraph_t body;
      deps = B.add_while(b->gfwd, deps, &hs, &body);
      auto bd = B.capture(body, {}, [&](cudaStream_t s) {
        irk::k_ckpt_store<<<grid_n(c.n), 256, 0, s>>>(I.step, ckpt_every, ck, c.u, c.n);
      });
      bd = B.solve(c, false, body, bd);
      B.capture(body, bd, [&](cudaStream_t s) { irk::k_step_ctrl<<<1, 32, 0, s>>>(I.step, 1, 0, nsteps, hs); });
      B.capture(b->gfwd, deps, [&](cudaStream_t s) {
        CK(cudaMemcpyAsync(uN, c.u, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s));
      });
    }
    CK(cudaGraphInstantiate(&b->fwd, b->gfwd, 0));
    // ---------------- adjoint: checkpointed reverse sweep of every instance
    if (d_lambda) {
      CK(cudaGraphCreate(&b->gadj, 0));
      int nseg = (nsteps + ckpt_every - 1) / ckpt_every;
      for (int q = 0; q < count; ++q) {
        Ctx& c = ctxs[q]->c;
        irk::Instance& I = b->inst[q];
        double* lam_io = d_lambda[q];
        double* grad = d_grad_kappa ? d_grad_kappa[q] : nullptr;
        double* ck = d_ckpt[q];
        auto deps = B.capture(b->gadj, {}, [&](cudaStream_t s) {
          CK(cudaMemcpyAsync(c.lam, lam_io, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s));
          CK(cudaMemsetAsync(c.step_counter, 0, sizeof(int), s));
        });
        for (int sg = nseg - 1; sg >= 0; --sg) {
          int s0 = sg * ckpt_every, len = std::min(nsteps, s0 + ckpt_every) - s0;
          // recompute the segment from its checkpoint, storing u_t and k_t
          deps = B.capture(b->gadj, deps, [&](cudaStream_t s) {
            CK(cudaMemcpyAsync(c.u, ck + int64_t(sg) * c.n, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s));
            irk::k_set_int<<<1, 32, 0, s>>>(I.step, 0);
          });
          cudaGraphConditionalHandle hr;
          cudaGraph_t rbody;
          deps = B.add_while(b->gadj, deps, &hr, &rbody);
          auto rd = B.capture(rbody, {}, [&](cudaStream_t s) {
            irk::k_store_at<<<grid_n(c.n), 256, 0, s>>>(I.step, I.ustore, c.u, c.n);
          });
          rd = B.solve(c, false, rbody, rd);
          B.capture(rbody, rd, [&](cudaStream_t s) {
            irk::k_store_at<<<grid_n(c.N), 256, 0, s>>>(I.step, I.kstore, c.x, c.N);
            irk::k_step_ctrl<<<1, 32, 0, s>>>(I.step, 1, 0, len, hr);
          });
          // adjoint steps t = s0 + len - 1 .. s0
          deps = B.capture(b->gadj, deps, [&](cudaStream_t s) { irk::k_set_int<<<1, 32, 0, s>>>(I.step, len - 1); });
          cudaGraphConditionalHandle ha;
          cudaGraph_t abody;
          deps = B.add_while(b->gadj, deps, &ha, &abody);
          std::vector<cudaGraphNode_t> ad;
          {
            irk::AdjointView av(c, true);   // nonsymmetric instances: transposed matrices and hierarchies
            ad = B.solve(c, true, abody, {});
          }
          B.capture(abody, ad, [&](cudaStream_t s) {
            if (grad) irk::adjoint_grad_launch_at(c, I.ustore, I.kstore, I.step, grad, s);
            irk::k_copy<<<grid_n(c.n), 256, 0, s>>>(c.lam, c.tmpn, c.n);
            irk::k_step_ctrl<<<1, 32, 0, s>>>(I.step, -1, 0, len, ha);
          });
        }
        B.capture(b->gadj, deps, [&](cudaStream_t s) {
          CK(cudaMemcpyAsync(lam_io, c.lam, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s));
        });
      }
      CK(cudaGraphInstantiate(&b->adj, b->gadj, 0));
    }
  } catch (const irk::Error& e) {
    irk::set_global_error(e.msg);
    irk_batch_destroy(b);
    return e.st;
  }
  *out = b;
  return IRK_OK;
}

static irk_status batch_launch(irk_batch* b, cudaGraphExec_t exec, void* stream, irk_stats* stats, double* ms) {
  try {
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    CK(cudaEventRecord(b->e0, user));
    CK(cudaStreamWaitEvent(b->stream, b->e0, 0));
    CK(cudaEventRecord(b->e0, b->stream));
    CK(cudaGraphLaunch(exec, b->stream));
    CK(cudaEventRecord(b->e1, b->stream));
    CK(cudaStreamWaitEvent(user, b->e1, 0));
    CK(cudaStreamSynchronize(b->stream));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, b->e0, b->e1));
    if (ms) *ms = t;
    irk_status worst = IRK_OK;
    for (size_t q = 0; q < b->inst.size(); ++q) {
      Ctx& c = *b->inst[q].c;
      int nrec = 0;
      CK(cudaMemcpy(&nrec, c.step_counter, sizeof(int), cudaMemcpyDeviceToHost));
      nrec = std::min(nrec, c.rec_cap);
      std::vector<irk::StepRecord> rec(nrec);
      if (nrec) CK(cudaMemcpy(rec.data(), c.rec, sizeof(irk::StepRecord) * nrec, cudaMemcpyDeviceToHost));
      irk_stats s{};
      s.steps = nrec;
      s.ms = t;
      int64_t its = 0;
      for (auto& r : rec) {
        s.iterations += r.it;
        s.restarts += r.restarts;
        s.max_step_iterations = std::max(s.max_step_iterations, r.it);
        s.resid = r.resid;
        its += std::max(r.it, 1);
        if (r.status != IRK_OK && worst == IRK_OK) worst = static_cast<irk_status>(r.status);
      }
      c.launches += its * (c.graph[0].body_kernels > 0 ? c.graph[0].body_kernels : 1) + 6 * nrec;
      if (stats) stats[q] = s;
    }
    return worst;
  } catch (const irk::Error& e) {
    b->err = e.msg;
    irk::set_global_error(e.msg);
    return e.st;
  }
}

irk_status irk_batch_run(irk_batch* b, void* stream, irk_stats* stats, double* ms) {
  if (!b || !b->fwd) return IRK_ERR_INVALID;
  return batch_launch(b, b->fwd, stream, stats, ms);
}

irk_status irk_batch_adjoint(irk_batch* b, void* stream, irk_stats* stats, double* ms) {
  if (!b) return IRK_ERR_INVALID;
  if (!b->adj) {
    irk::set_global_error("batch created without adjoint buffers");
    return IRK_ERR_INVALID;
  }
  return batch_launch(b, b->adj, stream, stats, ms);
}

void irk_batch_destroy(irk_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->fwd) cudaGraphExecDestroy(b->fwd);
  if (b->adj) cudaGraphExecDestroy(b->adj);
  if (b->gfwd) cudaGraphDestroy(b->gfwd);
  if (b->gadj) cudaGraphDestroy(b->gadj);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->stream) cudaStreamDestroy(b->stream);
  b->pool.free_all();
  delete b;
}

}  // extern "C"
