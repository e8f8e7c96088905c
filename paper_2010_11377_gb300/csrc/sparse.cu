// Sparse-matrix utilities of the AMG setup: exclusive scans, CSR upload,
// CSR -> SELL-32 conversion, transpose, and a deterministic row-wise SpGEMM
// (one warp per output row; products sorted by (column, generation order) in
// shared memory and summed in that order, so results do not depend on thread
// scheduling).
#include "irk_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

namespace irk {

// ---------------------------------------------------------------------------
// error handling and memory
// ---------------------------------------------------------------------------
void fail(irk_status st, const std::string& msg) { throw Error{st, msg}; }

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) throw Error{IRK_ERR_NOMEM, buf};
  throw Error{IRK_ERR_CUDA, buf};
}

void* DevPool::alloc(size_t nbytes) {
  void* p = nullptr;
  if (nbytes == 0) nbytes = 16;
  CK(cudaMalloc(&p, nbytes));
  ptrs.push_back(p);
  bytes += nbytes;
  return p;
}

void DevPool::release(void* p) {
  if (!p) return;
  auto it = std::find(ptrs.begin(), ptrs.end(), p);
  if (it != ptrs.end()) {
    cudaFree(p);
    ptrs.erase(it);
  }
}

void DevPool::free_all() {
  for (void* p : ptrs) cudaFree(p);
  ptrs.clear();
  bytes = 0;
}

Tmp::~Tmp() {
  for (void* p : ptrs) cudaFree(p);
}

bool pdl_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("IRK_PDL");
    on = (e && std::atoi(e) == 0) ? 0 : 1;
  }
  return on == 1;
}

// shared per-slice offset patterns in SELL-32 (IRK_SLICE_PATTERN=0 reads the
// per-entry offsets everywhere)
static bool slice_patterns_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("IRK_SLICE_PATTERN");
    on = (e && std::atoi(e) == 0) ? 0 : 1;
  }
  return on == 1;
}

// 16-bit column offsets in the SELL and CSR layouts of square operators
// (IRK_SELL16=0 keeps 32-bit columns everywhere)
static bool sell_offsets_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("IRK_SELL16");
    on = (e && std::atoi(e) == 0) ? 0 : 1;
  }
  return on == 1;
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ---------------------------------------------------------------------------
// exclusive scan: per-block inclusive scan, recursive scan of block sums, add
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 1024;

template <typename T>
__global__ void k_scan_block(const T* __restrict__ in, T* __restrict__ out, T* __restrict__ bsum,
                             int n) {
  __shared__ T sh[SCAN_BLOCK];
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  T v = (i < n) ? in[i] : T(0);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    T t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : T(0);
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;   // exclusive
  if (threadIdx.x == SCAN_BLOCK - 1) bsum[blockIdx.x] = sh[threadIdx.x];
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ boff, int n, T* total,
                           const T* __restrict__ in) {
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
  if (i == n - 1) *total = out[i] + in[i];
}

template <typename T>
static void scan_impl(const T* in, T* out, int n, cudaStream_t st) {
  if (n <= 0) {
    CK(cudaMemsetAsync(out, 0, sizeof(T), st));
    return;
  }
  int nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  T* bsum = nullptr;
  T* boff = nullptr;
  CK(cudaMallocAsync(&bsum, sizeof(T) * (nb + 1), st));
  CK(cudaMallocAsync(&boff, sizeof(T) * (nb + 1), st));
  k_scan_block<T><<<nb, SCAN_BLOCK, 0, st>>>(in, out, bsum, n);
  CK_LAUNCH();
  if (nb > 1) {
    scan_impl<T>(bsum, boff, nb, st);
  } else {
    CK(cudaMemsetAsync(boff, 0, sizeof(T), st));
  }
  k_scan_add<T><<<nb, SCAN_BLOCK, 0, st>>>(out, boff, n, out + n, in);
  CK_LAUNCH();
  CK(cudaFreeAsync(bsum, st));
  CK(cudaFreeAsync(boff, st));
}

void scan_exclusive(const int* in, int* out, int n, cudaStream_t st) { scan_impl<int>(in, out, n, st); }
void scan_exclusive64(const int64_t* in, int64_t* out, int n, cudaStream_t st) {
  scan_impl<int64_t>(in, out, n, st);
}

template <typename T>
static T read_scalar(const T* d, cudaStream_t st) {
  T h;
  CK(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

// ---------------------------------------------------------------------------
// CSR
// ---------------------------------------------------------------------------
void csr_alloc(CsrD& d, int n, int ncols, int64_t nnz, DevPool& pool) {
  if (nnz >= (int64_t(1) << 31)) fail(IRK_ERR_CAPACITY, "matrix has 2^31 or more nonzeros");
  d.n = n;
  d.ncols = ncols;
  d.nnz = nnz;
  d.rowptr = pool.get<int>(n + 1);
  d.col = pool.get<int>(nnz > 0 ? nnz : 1);
  d.val = pool.get<double>(nnz > 0 ? nnz : 1);
}

void csr_upload(const irk_csr& h, CsrD& d, DevPool& pool, cudaStream_t st) {
  if (h.n < 0 || h.nnz < 0 || !h.rowptr || (h.nnz > 0 && (!h.col || !h.val)))
    fail(IRK_ERR_INVALID, "bad CSR matrix");
  if (h.rowptr[0] != 0 || h.rowptr[h.n] != h.nnz) fail(IRK_ERR_INVALID, "CSR rowptr inconsistent with nnz");
  std::vector<int> rp(h.n + 1);
  for (int i = 0; i <= h.n; ++i) {
    if (i > 0 && h.rowptr[i] < h.rowptr[i - 1]) fail(IRK_ERR_INVALID, "CSR rowptr not monotone");
    rp[i] = static_cast<int>(h.rowptr[i]);
  }
  for (int i = 0; i < h.n; ++i)
    for (int64_t k = h.rowptr[i]; k < h.rowptr[i + 1]; ++k) {
      if (h.col[k] < 0 || h.col[k] >= h.n) fail(IRK_ERR_INVALID, "CSR column index out of range");
      if (k > h.rowptr[i] && h.col[k] <= h.col[k - 1])
        fail(IRK_ERR_INVALID, "CSR columns must be strictly increasing within a row");
    }
  csr_alloc(d, h.n, h.n, h.nnz, pool);
  CK(cudaMemcpyAsync(d.rowptr, rp.data(), sizeof(int) * (h.n + 1), cudaMemcpyHostToDevice, st));
  if (h.nnz > 0) {
    CK(cudaMemcpyAsync(d.col, h.col, sizeof(int) * h.nnz, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d.val, h.val, sizeof(double) * h.nnz, cudaMemcpyHostToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
}

void csr_copy_to_host(const CsrD& A, std::vector<int>& rp, std::vector<int>& col,
                      std::vector<double>& val, cudaStream_t st) {
  rp.resize(A.n + 1);
  col.resize(A.nnz);
  val.resize(A.nnz);
  CK(cudaMemcpyAsync(rp.data(), A.rowptr, sizeof(int) * (A.n + 1), cudaMemcpyDeviceToHost, st));
  if (A.nnz) {
    CK(cudaMemcpyAsync(col.data(), A.col, sizeof(int) * A.nnz, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(val.data(), A.val, sizeof(double) * A.nnz, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
}

__global__ void k_axpby_nofma(int64_t nnz, const double* __restrict__ x, const double* __restrict__ y,
                              double c, double* __restrict__ out) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < nnz) out[i] = __dadd_rn(x[i], __dmul_rn(c, y[i]));
}

void csr_axpby_same_pattern(const CsrD& X, const double* valX, const double* valY, double c,
                            double* out, cudaStream_t st) {
  if (X.nnz == 0) return;
  int64_t nb = (X.nnz + 255) / 256;
  k_axpby_nofma<<<static_cast<unsigned>(nb), 256, 0, st>>>(X.nnz, valX, valY, c, out);
  CK_LAUNCH();
}

// ---------------------------------------------------------------------------
// CSR -> SELL: slices of H = 32 / T rows, T threads per row (T = 1: SELL-32).
// Chunk k of a slice holds 32 entries; entry (row i of the slice, position p of
// the row) sits at base + (p / T) * 32 + (p % T) * H + i, so every warp load of
// a chunk is one contiguous run of 32 entries.  Padding: column 0 (offset 0),
// value 0.
// ---------------------------------------------------------------------------
__global__ void k_slice_width(int n, int nslices, int tpr, const int* __restrict__ rowptr, int64_t* __restrict__ w) {
  int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslices) return;
  const int H = SELL_C / tpr;
  int mx = 0;
  for (int l = 0; l < H; ++l) {
    int r = sl * H + l;
    if (r < n) mx = max(mx, rowptr[r + 1] - rowptr[r]);
  }
  w[sl] = int64_t((mx + tpr - 1) / tpr) * SELL_C;
}

// one thread per (slice, lane): lane = q * H + i serves positions q, q + T, ...
// of row i of the slice
__device__ __forceinline__ void sell_slot(int t, int tpr, int& sl, int& lane, int& r, int& q) {
  const int H = SELL_C / tpr;
  sl = t / SELL_C;
  lane = t % SELL_C;
  r = sl * H + lane % H;
  q = lane / H;
}

__global__ void k_sell_fill(int n, int nslices, int tpr, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, const int64_t* __restrict__ sptr,
                            int* __restrict__ scol, double* __restrict__ v64, float* __restrict__ v32,
                            __nv_bfloat16* __restrict__ v16) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslices * SELL_C) return;
  int sl, lane, r, q;
  sell_slot(t, tpr, sl, lane, r, q);
  int64_t base = sptr[sl];
  int w = static_cast<int>((sptr[sl + 1] - base) / SELL_C);
  int beg = 0, len = 0;
  if (r < n) {
    beg = rowptr[r];
    len = rowptr[r + 1] - beg;
  }
  for (int k = 0; k < w; ++k) {
    int64_t idx = base + int64_t(k) * SELL_C + lane;
    int p = k * tpr + q;
    int c = 0;
    double v = 0.0;
    if (p < len) {
      c = col[beg + p];
      v = val[beg + p];
    }
    scol[idx] = c;
    if (v64) v64[idx] = v;
    if (v32) v32[idx] = static_cast<float>(v);
    if (v16) v16[idx] = __double2bfloat16(v);
  }
}

__global__ void k_sell_fill_vals(int n, int nslices, const int* __restrict__ rowptr,
                                 const double* __restrict__ val, const int64_t* __restrict__ sptr,
                                 double* __restrict__ v64, float* __restrict__ v32) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslices * SELL_C) return;
  int sl = t / SELL_C, lane = t % SELL_C;
  int64_t base = sptr[sl];
  int w = static_cast<int>((sptr[sl + 1] - base) / SELL_C);
  int beg = 0, len = 0;
  if (t < n) {
    beg = rowptr[t];
    len = rowptr[t + 1] - beg;
  }
  for (int k = 0; k < w; ++k) {
    int64_t idx = base + int64_t(k) * SELL_C + lane;
    double v = (k < len) ? val[beg + k] : 0.0;
    if (v64) v64[idx] = v;
    if (v32) v32[idx] = static_cast<float>(v);
  }
}

// 16-bit column offsets from the row; flag set if one does not fit
__global__ void k_sell_offsets(int n, int nslices, int tpr, const int* __restrict__ rowptr,
                               const int64_t* __restrict__ sptr, const int* __restrict__ scol,
                               short* __restrict__ dcol, int* __restrict__ overflow) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslices * SELL_C) return;
  int sl, lane, r, q;
  sell_slot(t, tpr, sl, lane, r, q);
  int64_t base = sptr[sl];
  int w = static_cast<int>((sptr[sl + 1] - base) / SELL_C);
  int len = r < n ? rowptr[r + 1] - rowptr[r] : 0;
  bool bad = false;
  for (int k = 0; k < w; ++k) {
    int64_t idx = base + int64_t(k) * SELL_C + lane;
    int d = (k * tpr + q) < len ? scol[idx] - r : 0;
    if (d < -32767 || d > 32767) {
      bad = true;
      d = 0;
    }
    dcol[idx] = static_cast<short>(d);
  }
  if (bad) atomicOr(overflow, 1);
}

// one warp per SELL-32 slice: the slice shares one offset pattern when its 32
// rows are all real, all as long as the slice is wide (at most PAT_W), and agree
// chunk by chunk; the pattern goes to the slice's slot pdcol[PAT_W sl ..]
__global__ void k_sell_uniform(int n, int nslices, const int* __restrict__ rowptr, const int64_t* __restrict__ sptr,
                               const short* __restrict__ dcol, unsigned char* __restrict__ suni,
                               short* __restrict__ pdcol, unsigned long long* __restrict__ nonuni) {
  int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (sl >= nslices) return;
  int64_t base = sptr[sl];
  int w = static_cast<int>((sptr[sl + 1] - base) >> 5);
  int r = sl * SELL_C + lane;
  bool ok = r < n && (rowptr[r + 1] - rowptr[r]) == w;
  for (int k = 0; k < w; ++k) {
    short d = dcol[base + (int64_t(k) << 5) + lane];
    short d0 = __shfl_sync(0xffffffffu, d, 0);
    ok = ok && d == d0;
  }
  bool all = __all_sync(0xffffffffu, ok) && w >= 1 && w <= PAT_W;
  if (lane == 0) {
    suni[sl] = all ? static_cast<unsigned char>(w) : 0;
    if (!all) atomicAdd(nonuni, static_cast<unsigned long long>(w) * SELL_C);
  }
  if (lane < PAT_W)
    pdcol[int64_t(sl) * PAT_W + lane] = (all && lane < w) ? dcol[base + (int64_t(lane) << 5)] : short(0);
}

// the same for CSR (one thread per row)
__global__ void k_csr_offsets(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                              short* __restrict__ dcol, int* __restrict__ overflow) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  bool bad = false;
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    int d = col[k] - r;
    if (d < -32767 || d > 32767) {
      bad = true;
      d = 0;
    }
    dcol[k] = static_cast<short>(d);
  }
  if (bad) atomicOr(overflow, 1);
}

void csr_to_sell(const CsrD& A, Sell& S, int want64, int want32, int want16, DevPool& pool,
                 cudaStream_t st, int tpr) {
  if (tpr != 1 && tpr != 2 && tpr != 4 && tpr != 8) fail(IRK_ERR_INVALID, "SELL threads per row must be 1, 2, 4 or 8");
  const int H = SELL_C / tpr;
  S.n = A.n;
  S.ncols = A.ncols;
  S.tpr = tpr;
  S.nslices = (A.n + H - 1) / H;
  int ns = S.nslices;
  S.sptr = pool.get<int64_t>(ns + 1);
  {
    Tmp tmp;
    int64_t* w = tmp.get<int64_t>(ns > 0 ? ns : 1);
    if (ns > 0) {
      k_slice_width<<<(ns + 255) / 256, 256, 0, st>>>(A.n, ns, tpr, A.rowptr, w);
      CK_LAUNCH();
    }
    scan_exclusive64(w, S.sptr, ns, st);
    S.nnz_pad = read_scalar(S.sptr + ns, st);
  }
  int64_t np = S.nnz_pad > 0 ? S.nnz_pad : 1;
  S.col = pool.get<int>(np);
  S.v64 = want64 ? pool.get<double>(np) : nullptr;
  S.v32 = want32 ? pool.get<float>(np) : nullptr;
  S.v16 = want16 ? pool.get<__nv_bfloat16>(np) : nullptr;
  if (ns > 0) {
    int nt = ns * SELL_C;
    k_sell_fill<<<(nt + 255) / 256, 256, 0, st>>>(A.n, ns, tpr, A.rowptr, A.col, A.val, S.sptr, S.col, S.v64,
                                                  S.v32, S.v16);
    CK_LAUNCH();
  }
  S.dcol = nullptr;
  if (ns > 0 && A.ncols == A.n && sell_offsets_enabled()) {
    short* dc = pool.get<short>(np);
    Tmp tmp;
    int* ovf = tmp.get<int>(1);
    CK(cudaMemsetAsync(ovf, 0, sizeof(int), st));
    int nt = ns * SELL_C;
    k_sell_offsets<<<(nt + 255) / 256, 256, 0, st>>>(A.n, ns, tpr, A.rowptr, S.sptr, S.col, dc, ovf);
    CK_LAUNCH();
    if (read_scalar(ovf, st) == 0) S.dcol = dc;
  }
  S.suni = nullptr;
  S.pdcol = nullptr;
  S.nnz_nonuni = S.nnz_pad;
  if (S.dcol && tpr == 1 && sell_offsets_enabled() && slice_patterns_enabled()) {
    S.suni = pool.get<unsigned char>(ns);
    S.pdcol = pool.get<short>(size_t(ns) * PAT_W);
    Tmp tmp;
    unsigned long long* nonuni = tmp.get<unsigned long long>(1);
    CK(cudaMemsetAsync(nonuni, 0, sizeof(unsigned long long), st));
    k_sell_uniform<<<(ns * SELL_C + 255) / 256, 256, 0, st>>>(A.n, ns, A.rowptr, S.sptr, S.dcol, S.suni, S.pdcol,
                                                              nonuni);
    CK_LAUNCH();
    S.nnz_nonuni = static_cast<int64_t>(read_scalar(nonuni, st));
  }
  CK(cudaStreamSynchronize(st));
}

// A second value array on an existing SELL pattern (M and F share one pattern)
void sell_share_pattern(const Sell& pat, const double* csr_vals, const CsrD& A, Sell& S, int want64,
                        int want32, DevPool& pool, cudaStream_t st) {
  if (pat.tpr != 1) fail(IRK_ERR_INVALID, "shared SELL patterns have one thread per row");
  S = pat;
  S.v64 = nullptr;
  S.v32 = nullptr;
  S.v16 = nullptr;
  int64_t np = pat.nnz_pad > 0 ? pat.nnz_pad : 1;
  if (want64) S.v64 = pool.get<double>(np);
  if (want32) S.v32 = pool.get<float>(np);
  if (pat.nslices > 0) {
    int nt = pat.nslices * SELL_C;
    k_sell_fill_vals<<<(nt + 255) / 256, 256, 0, st>>>(A.n, pat.nslices, A.rowptr, csr_vals, pat.sptr,
                                                       S.v64, S.v32);
    CK_LAUNCH();
  }
  CK(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// V-cycle operator: SELL for short rows, CSR with lanes-per-row otherwise
// ---------------------------------------------------------------------------
__global__ void k_convert_vals(int64_t nnz, const double* __restrict__ in, double* __restrict__ v64,
                               float* __restrict__ v32, __nv_bfloat16* __restrict__ v16) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= nnz) return;
  double v = in[i];
  if (v64) v64[i] = v;
  if (v32) v32[i] = static_cast<float>(v);
  if (v16) v16[i] = __double2bfloat16(v);
}

// Row-length rule (the autotuner's starting point, and the layout when it is
// off): SELL-32 for short rows, sliced SELL for medium rows (measured at 1024^2
// on the Galerkin levels of the heat blocks: 2 threads per row at 26 entries,
// 4 at 40, 8 at 81, each 1.2-1.45x faster than CSR with 4 or 8 lanes), CSR
// with 16 or 32 lanes for long rows.
int choose_lanes(int64_t nnz, int n) {
  double avg = n > 0 ? double(nnz) / n : 0.0;
  if (avg <= 16.0) return 1;
  if (avg <= 32.0) return -2;
  if (avg <= 48.0) return -4;
  if (avg <= 96.0) return -8;
  if (avg <= 192.0) return 16;
  return 32;
}

// ---------------------------------------------------------------------------
// Layout autotuner: for an operator of a given shape class (log2 of the rows,
// log2 of the mean row length, precision, square or not) time y = A x with every candidate
// thread tile (SELL thread-per-row, sliced SELL with 2, 4 or 8 threads per row,
// or CSR with 2..32 lanes per row) and keep the fastest.  Decisions are cached for the process, so repeated set-ups
// (batches, kappa updates) reuse them.  IRK_AUTOTUNE=0 uses the row-length rule.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune;

int ilog2(double v) {
  int k = 0;
  while (v >= 2.0) {
    v *= 0.5;
    ++k;
  }
  return k;
}

bool autotune_enabled() {
  const char* e = std::getenv("IRK_AUTOTUNE");
  return !(e && std::atoi(e) == 0);
}
}  // namespace

static void build_layout(const CsrD& A, MatT& m, int prec, int lanes, DevPool& pool, cudaStream_t st);

// IRK_LAYOUT=<code> (1, -2, -4, -8, 2, 4, 8, 16, 32) puts every V-cycle operator
// in that layout (diagnosis and layout tests; every layout is exact for any row
// length, only its speed differs)
static int forced_layout() {
  const char* e = std::getenv("IRK_LAYOUT");
  if (!e) return 0;
  int v = std::atoi(e);
  for (int c : {1, -2, -4, -8, 2, 4, 8, 16, 32})
    if (v == c) return v;
  return 0;
}

int autotune_lanes(const CsrD& A, int prec, cudaStream_t st) {
  if (int f = forced_layout()) return f;
  int heuristic = choose_lanes(A.nnz, A.n);
  if (!autotune_enabled() || A.n < 64 || A.nnz == 0) return heuristic;
  double avg = double(A.nnz) / A.n;
  // square operators (level matrices, 16-bit offsets possible) and rectangular
  // ones (prolongation, restriction) are tuned separately
  auto key = std::make_tuple(ilog2(A.n), ilog2(avg * 2.0), prec, A.ncols == A.n ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  // SELL-32, sliced SELL with 2/4/8 threads per row, CSR with 2..32 lanes
  const int cand[] = {1, -2, -4, -8, 2, 4, 8, 16, 32};
  size_t es = prec == 64 ? 8 : 4;
  DevPool tmp;
  void* x = tmp.alloc(es * (A.ncols > 0 ? A.ncols : 1));
  void* y = tmp.alloc(es * A.n);
  CK(cudaMemsetAsync(x, 0, es * A.ncols, st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // each candidate: the fastest of 3 trials of 10 back-to-back products; a
  // candidate replaces the row-length rule only when it is more than 10%
  // faster, so timing noise (or a profiler's overhead) keeps the rule
  float t_rule = 1e30f;
  int best = heuristic;
  float best_t = 1e30f;
  for (int L : cand) {
    if (L != heuristic && L > 1 && avg < L / 2.0) continue;   // more lanes than half the row: idle lanes
    if (L != heuristic && L == 1 && avg > 48.0) continue;      // one thread walking a long row
    if (L < 0 && (avg < 2.0 * -L || avg > 96.0)) continue;     // sliced: at least 2 entries per thread, medium rows
    MatT m;
    DevPool mp;
    build_layout(A, m, prec, L, mp, st);
    for (int w = 0; w < 3; ++w) matT_spmv_launch(m, prec, x, y, st);
    float t = 1e30f;
    for (int trial = 0; trial < 3; ++trial) {
      CK(cudaEventRecord(e0, st));
      for (int r = 0; r < 10; ++r) matT_spmv_launch(m, prec, x, y, st);
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float tt = 0.f;
      CK(cudaEventElapsedTime(&tt, e0, e1));
      t = tt < t ? tt : t;
    }
    if (L == heuristic) t_rule = t;
    if (t < best_t) {
      best_t = t;
      best = L;
    }
    mp.free_all();
  }
  if (best != heuristic && !(best_t < 0.9f * t_rule)) best = heuristic;
  if (const char* v = std::getenv("IRK_VERBOSE"); v && std::atoi(v) > 0)
    std::fprintf(stderr, "irk autotune: %d rows, %.1f entries per row, prec %d: layout %d (rule %d: %.4f ms, best %.4f ms per 10)\n",
                 A.n, avg, prec, best, heuristic, double(t_rule), double(best_t));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tmp.free_all();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

void make_matT(const CsrD& A, MatT& m, int prec, DevPool& pool, cudaStream_t st, int force_lanes) {
  int lanes = force_lanes > 0 ? force_lanes : autotune_lanes(A, prec == 16 ? 32 : prec, st);
  build_layout(A, m, prec, lanes, pool, st);
}

static void build_layout(const CsrD& A, MatT& m, int prec, int lanes, DevPool& pool, cudaStream_t st) {
  m = MatT{};
  m.n = A.n;
  m.ncols = A.ncols;
  m.nnz = A.nnz;
  m.lanes = lanes;
  if (m.uses_sell()) {
    csr_to_sell(A, m.sell, prec == 64, prec == 32, prec == 16, pool, st, lanes < 0 ? -lanes : 1);
    return;
  }
  m.rowptr = A.rowptr;
  m.col = A.col;
  int64_t nn = A.nnz > 0 ? A.nnz : 1;
  double* v64 = nullptr;
  float* v32 = nullptr;
  __nv_bfloat16* v16 = nullptr;
  if (prec == 64) m.val = v64 = pool.get<double>(nn);
  else if (prec == 32) m.val = v32 = pool.get<float>(nn);
  else m.val = v16 = pool.get<__nv_bfloat16>(nn);
  if (A.nnz) {
    k_convert_vals<<<nblk(A.nnz), 256, 0, st>>>(A.nnz, A.val, v64, v32, v16);
    CK_LAUNCH();
  }
  m.dcol = nullptr;
  if (A.nnz > 0 && A.ncols == A.n && sell_offsets_enabled()) {
    short* dc = pool.get<short>(A.nnz);
    Tmp tmp;
    int* ovf = tmp.get<int>(1);
    CK(cudaMemsetAsync(ovf, 0, sizeof(int), st));
    k_csr_offsets<<<nblk(A.n), 256, 0, st>>>(A.n, A.rowptr, A.col, dc, ovf);
    CK_LAUNCH();
    if (read_scalar(ovf, st) == 0) m.dcol = dc;
  }
}

// ---------------------------------------------------------------------------
// transpose (counting sort, then each row sorted by column)
// ---------------------------------------------------------------------------
__global__ void k_count_cols(int64_t nnz, const int* __restrict__ col, int* __restrict__ cnt) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < nnz) atomicAdd(&cnt[col[i]], 1);
}

__global__ void k_transpose_fill(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, int* __restrict__ cursor,
                                 int* __restrict__ tcol, double* __restrict__ tval) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    int c = col[k];
    int pos = atomicAdd(&cursor[c], 1);
    tcol[pos] = r;
    tval[pos] = val[k];
  }
}

// insertion sort of each row by column index (rows of a transposed AMG
// operator are short); values follow their columns
__global__ void k_sort_rows(int n, const int* __restrict__ rowptr, int* __restrict__ col,
                            double* __restrict__ val) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int b = rowptr[r], e = rowptr[r + 1];
  for (int i = b + 1; i < e; ++i) {
    int c = col[i];
    double v = val[i];
    int k = i - 1;
    while (k >= b && col[k] > c) {
      col[k + 1] = col[k];
      val[k + 1] = val[k];
      --k;
    }
    col[k + 1] = c;
    val[k + 1] = v;
  }
}

void csr_transpose(const CsrD& A, CsrD& T, DevPool& pool, cudaStream_t st) {
  csr_alloc(T, A.ncols, A.n, A.nnz, pool);
  Tmp tmp;
  int* cnt = tmp.get<int>(A.ncols + 1);
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (A.ncols + 1), st));
  if (A.nnz) {
    k_count_cols<<<static_cast<unsigned>((A.nnz + 255) / 256), 256, 0, st>>>(A.nnz, A.col, cnt);
    CK_LAUNCH();
  }
  scan_exclusive(cnt, T.rowptr, A.ncols, st);
  int* cursor = tmp.get<int>(A.ncols + 1);
  CK(cudaMemcpyAsync(cursor, T.rowptr, sizeof(int) * (A.ncols + 1), cudaMemcpyDeviceToDevice, st));
  if (A.n) {
    k_transpose_fill<<<(A.n + 255) / 256, 256, 0, st>>>(A.n, A.rowptr, A.col, A.val, cursor, T.col, T.val);
    CK_LAUNCH();
  }
  if (T.n) {
    k_sort_rows<<<(T.n + 255) / 256, 256, 0, st>>>(T.n, T.rowptr, T.col, T.val);
    CK_LAUNCH();
  }
  CK(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// SpGEMM C = A B, one warp per row of C
// ---------------------------------------------------------------------------
constexpr int GEMM_CAP = 2048;        // products per row held in shared memory
constexpr int GEMM_WARPS = 2;          // warps per block

__global__ void k_gemm_rowcount(int n, const int* __restrict__ arp, const int* __restrict__ acol,
                                const int* __restrict__ brp, int64_t* __restrict__ ub) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int64_t s = 0;
  for (int k = arp[r]; k < arp[r + 1]; ++k) {
    int c = acol[k];
    s += brp[c + 1] - brp[c];
  }
  ub[r] = s;
}

// Products of row r: generation order g = (position in A row, position in B row).
// Sorted by key = (column << 32) | g, then summed sequentially per column, which
// is the order of the classical row-by-row accumulation.
__global__ void __launch_bounds__(GEMM_WARPS * 32)
k_gemm_numeric(int n, const int* __restrict__ arp, const int* __restrict__ acol,
               const double* __restrict__ aval, const int* __restrict__ brp,
               const int* __restrict__ bcol, const double* __restrict__ bval,
               const int64_t* __restrict__ off, int* __restrict__ tcol, double* __restrict__ tval,
               int* __restrict__ cnt, int* __restrict__ novf, int* __restrict__ ovf_rows) {
  extern __shared__ unsigned char smem[];
  int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem) + warp * GEMM_CAP;
  double* vals = reinterpret_cast<double*>(smem + sizeof(unsigned long long) * GEMM_CAP * GEMM_WARPS) +
                 warp * GEMM_CAP;
  int r = blockIdx.x * GEMM_WARPS + warp;
  if (r >= n) return;
  int total = 0;
  // pass over A row: products go to [pos, pos + nnz(B_k))
  int a0 = arp[r], a1 = arp[r + 1];
  for (int k = a0; k < a1; ++k) total += brp[acol[k] + 1] - brp[acol[k]];
  if (total > GEMM_CAP) {     // long row: left to k_gemm_merge
    if (lane == 0) ovf_rows[atomicAdd(novf, 1)] = r;
    return;
  }
  int pos = 0;
  for (int k = a0; k < a1; ++k) {
    int c = acol[k];
    double av = aval[k];
    int b0 = brp[c], len = brp[c + 1] - b0;
    for (int t = lane; t < len; t += 32) {
      int g = pos + t;
      key[g] = (static_cast<unsigned long long>(static_cast<unsigned>(bcol[b0 + t])) << 32) |
               static_cast<unsigned>(g);
      vals[g] = av * bval[b0 + t];
    }
    pos += len;
  }
  int np2 = 1;
  while (np2 < total) np2 <<= 1;
  for (int g = total + lane; g < np2; g += 32) {
    key[g] = ~0ull;
    vals[g] = 0.0;
  }
  __syncwarp();
  // bitonic sort (ascending) of np2 keys
  for (int kk = 2; kk <= np2; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int i = lane; i < np2; i += 32) {
        int ixj = i ^ jj;
        if (ixj > i) {
          bool up = (i & kk) == 0;
          unsigned long long ki = key[i], kj = key[ixj];
          if ((ki > kj) == up) {
            key[i] = kj;
            key[ixj] = ki;
            double t = vals[i];
            vals[i] = vals[ixj];
            vals[ixj] = t;
          }
        }
      }
      __syncwarp();
    }
  }
  // segmented sum in sorted order (lane 0: rows are short)
  if (lane == 0) {
    int64_t o = off[r];
    int u = 0;
    int i = 0;
    while (i < total) {
      unsigned c = static_cast<unsigned>(key[i] >> 32);
      double sum = vals[i];
      int k = i + 1;
      while (k < total && static_cast<unsigned>(key[k] >> 32) == c) {
        sum += vals[k];
        ++k;
      }
      tcol[o + u] = static_cast<int>(c);
      tval[o + u] = sum;
      ++u;
      i = k;
    }
    cnt[r] = u;
  }
}

// Long rows (more products than the shared-memory sort holds): one thread
// merges a_rk B_k into the running sorted row for k in A-row order, in global
// scratch.  Sums accumulate in the same generation order as the sorted path.
__global__ void k_gemm_merge(int nrows, const int* __restrict__ rows, const int* __restrict__ arp,
                             const int* __restrict__ acol, const double* __restrict__ aval,
                             const int* __restrict__ brp, const int* __restrict__ bcol,
                             const double* __restrict__ bval, const int64_t* __restrict__ off, int* __restrict__ tcol,
                             double* __restrict__ tval, int* __restrict__ tcol2, double* __restrict__ tval2,
                             int* __restrict__ cnt) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nrows) return;
  int r = rows[q];
  int64_t o = off[r];
  int* ca = tcol + o;
  double* va = tval + o;
  int* cb = tcol2 + o;
  double* vb = tval2 + o;
  int len = 0;
  for (int k = arp[r]; k < arp[r + 1]; ++k) {
    int c = acol[k];
    double av = aval[k];
    int b0 = brp[c], b1 = brp[c + 1];
    int i = 0, t = b0, u = 0;
    while (i < len || t < b1) {
      if (t >= b1 || (i < len && ca[i] < bcol[t])) {
        cb[u] = ca[i];
        vb[u] = va[i];
        ++i;
      } else if (i >= len || bcol[t] < ca[i]) {
        cb[u] = bcol[t];
        vb[u] = __dmul_rn(av, bval[t]);
        ++t;
      } else {
        cb[u] = ca[i];
        vb[u] = __dadd_rn(va[i], __dmul_rn(av, bval[t]));
        ++i;
        ++t;
      }
      ++u;
    }
    int* tc = ca; ca = cb; cb = tc;
    double* tv = va; va = vb; vb = tv;
    len = u;
  }
  if (ca != tcol + o) {
    for (int i = 0; i < len; ++i) {
      tcol[o + i] = ca[i];
      tval[o + i] = va[i];
    }
  }
  cnt[r] = len;
}

__global__ void k_gemm_compact(int n, const int64_t* __restrict__ off, const int* __restrict__ rp,
                               const int* __restrict__ tcol, const double* __restrict__ tval,
                               int* __restrict__ col, double* __restrict__ val) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int64_t o = off[r];
  int b = rp[r], e = rp[r + 1];
  for (int k = b; k < e; ++k) {
    col[k] = tcol[o + (k - b)];
    val[k] = tval[o + (k - b)];
  }
}

void csr_spgemm(const CsrD& A, const CsrD& B, CsrD& C, DevPool& pool, cudaStream_t st) {
  int n = A.n;
  Tmp tmp;
  int64_t* ub = tmp.get<int64_t>(n + 1);
  int64_t* off = tmp.get<int64_t>(n + 1);
  if (n) {
    k_gemm_rowcount<<<(n + 255) / 256, 256, 0, st>>>(n, A.rowptr, A.col, B.rowptr, ub);
    CK_LAUNCH();
  }
  scan_exclusive64(ub, off, n, st);
  int64_t total = read_scalar(off + n, st);
  // products are staged in device scratch (12 bytes each, twice for long rows)
  if (total > (int64_t(1) << 30))
    fail(IRK_ERR_CAPACITY, "Galerkin product has more than 2^30 partial products (AMG coarsening stalled); "
                           "lower theta");
  int* tcol = tmp.get<int>(total > 0 ? total : 1);
  double* tval = tmp.get<double>(total > 0 ? total : 1);
  int* cnt = tmp.get<int>(n + 1);
  int* novf = tmp.get<int>(1);
  int* ovf_rows = tmp.get<int>(n > 0 ? n : 1);
  CK(cudaMemsetAsync(novf, 0, sizeof(int), st));
  size_t shm = (sizeof(unsigned long long) + sizeof(double)) * GEMM_CAP * GEMM_WARPS;
  static bool attr = false;
  if (!attr) {
    CK(cudaFuncSetAttribute(k_gemm_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(shm)));
    attr = true;
  }
  if (n) {
    k_gemm_numeric<<<(n + GEMM_WARPS - 1) / GEMM_WARPS, GEMM_WARPS * 32, shm, st>>>(
        n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, off, tcol, tval, cnt, novf, ovf_rows);
    CK_LAUNCH();
  }
  int nlong = read_scalar(novf, st);
  if (nlong > 0) {
    int* tcol2 = tmp.get<int>(total > 0 ? total : 1);
    double* tval2 = tmp.get<double>(total > 0 ? total : 1);
    k_gemm_merge<<<(nlong + 63) / 64, 64, 0, st>>>(nlong, ovf_rows, A.rowptr, A.col, A.val, B.rowptr, B.col,
                                                   B.val, off, tcol, tval, tcol2, tval2, cnt);
    CK_LAUNCH();
  }
  int* rp = pool.get<int>(n + 1);
  scan_exclusive(cnt, rp, n, st);
  int nnz = read_scalar(rp + n, st);
  C.n = n;
  C.ncols = B.ncols;
  C.nnz = nnz;
  C.rowptr = rp;
  C.col = pool.get<int>(nnz > 0 ? nnz : 1);
  C.val = pool.get<double>(nnz > 0 ? nnz : 1);
  if (n) {
    k_gemm_compact<<<(n + 255) / 256, 256, 0, st>>>(n, off, rp, tcol, tval, C.col, C.val);
    CK_LAUNCH();
  }
  CK(cudaStreamSynchronize(st));
}

}  // namespace irk
