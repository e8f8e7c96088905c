// irk_residual_norm_noalloc: the true-residual norm of irk_residual_norm for
// callers that must not allocate device memory during the call.  Such callers
// include code that runs while a memory pool owns the device (a caching
// allocator that would be bypassed or fragmented by cudaMalloc), code on a
// latency-critical path where cudaMalloc/cudaFree would synchronise the
// device, and code that needs a fixed, known memory footprint.
//
// The per-block partial sums live in a fixed array in device global memory,
// declared at file scope below; every GPU that loads libirk holds it until the
// process exits.  It has one slot per 256-row block, so the stage size n is
// limited to IRK_NOALLOC_MAX_ROWS rows.  Host code cannot use the array's
// name as a device address (it is a host-side stand-in), so its address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, the first time the entry point runs on it, and kept for the life
// of the process (a device reset that drops libirk's module is not supported).
// Under lazy module loading that first lookup may load the module, which the
// CUDA driver allocates memory for; later calls allocate nothing.
#include "irk_internal.cuh"

#include <exception>
#include <mutex>
#include <new>
#include <string>

namespace {

constexpr int kBlockRows = irk::OUTER_BLOCK;       // rows per block of the residual kernel
static_assert(kBlockRows == 256, "one scratch slot per 256-row block");
constexpr int kMaxBlocks = IRK_NOALLOC_MAX_ROWS / kBlockRows;

static __device__ __align__(256) double g_resid_scratch[kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

// device address of g_resid_scratch on the current device
irk_status scratch_address(int dev, double** out, std::string& err) {
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index out of range for the no-allocation scratch table";
    return IRK_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_resid_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress of the residual scratch failed: ") + cudaGetErrorString(e);
      return IRK_ERR_CUDA;
    }
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return IRK_OK;
}

irk_status fail_with(irk::Ctx* c, irk_status st, const std::string& msg) {
  irk::set_global_error(msg);
  if (c) c->err = msg;
  return st;
}

}  // namespace

extern "C" irk_status irk_residual_norm_noalloc(irk_ctx* h, const double* d_k, const double* d_b, double* d_norm) {
  if (!h || !d_k || !d_b || !d_norm) return fail_with(h ? &h->c : nullptr, IRK_ERR_INVALID, "NULL argument");
  irk::Ctx& c = h->c;
  try {
    if (c.n > IRK_NOALLOC_MAX_ROWS)
      return fail_with(&c, IRK_ERR_CAPACITY,
                       "irk_residual_norm_noalloc: n = " + std::to_string(c.n) +
                           " rows per stage exceeds the maximum of " + std::to_string(IRK_NOALLOC_MAX_ROWS));
    CK(cudaSetDevice(c.device));
    double* scratch = nullptr;
    std::string err;
    irk_status st = scratch_address(c.device, &scratch, err);
    if (st != IRK_OK) return fail_with(&c, st, err);
    CK(cudaEventRecord(c.ev_a, c.user_stream));
    CK(cudaStreamWaitEvent(c.stream, c.ev_a, 0));
    // every slot that the final sum reads is written by its block first: nothing
    // in the array has to start at zero
    int grid = (c.n + kBlockRows - 1) / kBlockRows;
    irk::residual_norm_launch(c, d_k, d_b, scratch, grid, d_norm, c.stream);
    c.launches += 2;
    // the caller's stream waits for the norm; the host does not
    CK(cudaEventRecord(c.ev_b, c.stream));
    CK(cudaStreamWaitEvent(c.user_stream, c.ev_b, 0));
  } catch (const irk::Error& e) {
    return fail_with(&c, e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail_with(&c, IRK_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail_with(&c, IRK_ERR_INVALID, e.what());
  }
  return IRK_OK;
}
