// One AMG V-cycle per diagonal-block subsolve, and the block substitutions of
// Section 4.2 that apply P = I_s (x) M + h A~ (x) F.
//
// V(nu1, nu2) cycle on a hierarchy built by amg_setup.cu; each smoothing sweep
// is a Chebyshev polynomial on the l1-scaled operator D_l1^{-1} A (or one
// l1-Jacobi step).  Kernels are one thread per row over SELL-32 matrices (each
// warp reads one slice: coalesced column/value loads), values in the V-cycle
// precision T (FP32 or FP64; BF16 finest-level values are widened to FP32).
// The first pre-smoothing step from a zero guess needs no matrix product; its
// iterate is recomputed from b where a neighbour needs it.
#include "irk_internal.cuh"

#include <cmath>

namespace irk {

template <typename T> __device__ __forceinline__ T widen(T v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

SmoothCoef smooth_coefficients(const AmgParams& p) {
  SmoothCoef c;
  if (p.smoother == IRK_SMOOTH_L1JACOBI) {
    c.steps = 1;
    c.alpha[0] = 0.0;
    c.beta[0] = 1.0;
    return c;
  }
  int k = p.cheb_degree < 1 ? 1 : (p.cheb_degree > 16 ? 16 : p.cheb_degree);
  double lo = p.cheb_lo;
  double theta = 0.5 * (1.0 + lo), delta = 0.5 * (1.0 - lo);
  double sigma = theta / delta;
  double rho = 1.0 / sigma;
  c.steps = k;
  c.alpha[0] = 0.0;
  c.beta[0] = 1.0 / theta;
  for (int i = 1; i < k; ++i) {
    double rn = 1.0 / (2.0 * sigma - rho);
    c.alpha[i] = rn * rho;
    c.beta[i] = 2.0 * rn / delta;
    rho = rn;
  }
  return c;
}

// x^(0) implicit: x1 = beta0 * dinv * b
enum { XM_EXPLICIT = 0, XM_IMPLICIT = 1, XM_ZERO = 2 };

// Thread -> (row, lane) of an operator layout (see MatT): L >= 1 gives L
// consecutive threads per row; L = -T gives the sliced SELL mapping, where the
// 32 threads of a warp serve the 32/T rows of one slice, T threads per row.
template <int L>
__device__ __forceinline__ void row_lane(int gid, int& r, int& lane) {
  if constexpr (L < 0) {
    constexpr int H = 32 / (-L);
    const int t = gid & 31;
    r = (gid >> 5) * H + (t % H);
    lane = t / H;
  } else {
    r = gid / L;
    lane = gid % L;
  }
}

// Row product sum_c a_rc x(c) of operator A at row r (r < 0: an idle thread
// that only takes part in the shuffles).  L == 1: SELL-32, one thread per row;
// L == -T: sliced SELL, T threads per row reduced by xor-shuffles across the
// slice; L > 1: CSR, L consecutive lanes per row, strided over the row, reduced
// by an xor-shuffle.  Every thread of a row's group ends with the sum.
template <int L, typename V, typename T, typename XF>
__device__ __forceinline__ T row_dot(const LMat<V>& A, int r, int lane, XF xf) {
  T acc = T(0);
  if constexpr (L == 1) {
    if (r >= 0) {
      int sl = r >> 5, ln = r & 31;
      int wu = 0;
      union {
        int4 v;
        short o[PAT_W];
      } pat;
      if (A.suni) {
        // the slice's shared pattern: its width and its 16-byte slot are loaded
        // alongside the slice base, so the gathers of x do not wait for the base
        wu = A.suni[sl];
        pat.v = reinterpret_cast<const int4*>(A.pdcol)[sl];
      }
      int64_t base = A.sptr[sl];
      if (wu) {
#pragma unroll
        for (int k = 0; k < PAT_W; ++k)
          if (k < wu)
            acc = fma(widen(A.val[base + (int64_t(k) << 5) + ln]), xf(r + static_cast<int>(pat.o[k])), acc);
        return acc;
      }
      int w = static_cast<int>((A.sptr[sl + 1] - base) >> 5);
      if (A.dcol) {
        for (int k = 0; k < w; ++k) {
          int64_t idx = base + (int64_t(k) << 5) + ln;
          acc = fma(widen(A.val[idx]), xf(r + static_cast<int>(A.dcol[idx])), acc);
        }
      } else {
        for (int k = 0; k < w; ++k) {
          int64_t idx = base + (int64_t(k) << 5) + ln;
          acc = fma(widen(A.val[idx]), xf(A.col[idx]), acc);
        }
      }
    }
  } else if constexpr (L < 0) {
    constexpr int H = 32 / (-L);
    if (r >= 0) {
      const int sl = r / H, i = r - sl * H;
      const int64_t base = A.sptr[sl];
      const int w = static_cast<int>((A.sptr[sl + 1] - base) >> 5);
      const int64_t off = base + lane * H + i;
      if (A.dcol) {
        for (int k = 0; k < w; ++k) {
          int64_t idx = off + (int64_t(k) << 5);
          acc = fma(widen(A.val[idx]), xf(r + static_cast<int>(A.dcol[idx])), acc);
        }
      } else {
        for (int k = 0; k < w; ++k) {
          int64_t idx = off + (int64_t(k) << 5);
          acc = fma(widen(A.val[idx]), xf(A.col[idx]), acc);
        }
      }
    }
#pragma unroll
    for (int o = 16; o >= H; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  } else {
    if (r >= 0) {
      int e = A.rowptr[r + 1];
      if (A.dcol) {
        for (int k = A.rowptr[r] + lane; k < e; k += L)
          acc = fma(widen(A.val[k]), xf(r + static_cast<int>(A.dcol[k])), acc);
      } else {
        for (int k = A.rowptr[r] + lane; k < e; k += L) acc = fma(widen(A.val[k]), xf(A.col[k]), acc);
      }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
  }
  return acc;
}

// One smoothing step: d = alpha d_prev + beta D^{-1}(b - A x); x_out = x + d.
// XM_IMPLICIT: x and d_prev are the implicit first step; XM_ZERO: x = 0, no product.
template <typename V, typename T, int L, int XM>
__global__ void __launch_bounds__(256)
k_smooth(LMat<V> A, const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ xin,
         const T* din, T* __restrict__ xout, T* dout, T alpha, T beta, T beta0, JPtr<T> out) {
  pdl_trigger();
  pdl_wait();
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int r, lane;
  row_lane<L>(gid, r, lane);
  bool valid = r < A.n;
  // the row's own vector entries are loaded first, so that they are in flight with the
  // row product's chain (slice base -> offsets and values -> gathered x)
  const bool owner = valid && lane == 0;
  T dr = T(0), br = T(0), xr = T(0), dprev = T(0);
  if (owner) {
    dr = dinv[r];
    br = b[r];
    if (XM == XM_EXPLICIT) {
      xr = xin[r];
      if (din) dprev = din[r];
    }
  }
  T ax = T(0);
  if (XM != XM_ZERO)
    ax = row_dot<L, V, T>(A, valid ? r : -1, lane, [&](int c) {
      return (XM == XM_IMPLICIT) ? beta0 * dinv[c] * b[c] : xin[c];
    });
  if (!owner) return;
  if (XM == XM_IMPLICIT) {
    xr = beta0 * dr * br;
    dprev = xr;
  }
  T res = dr * (br - ax);
  T d = alpha * dprev + beta * res;
  T xn = xr + d;
  if (out.base) out.get()[r] = xn;
  else xout[r] = xn;
  if (dout) dout[r] = d;
}

// r = b - A x  (x explicit or the implicit first step)
template <typename V, typename T, int L, int XM>
__global__ void __launch_bounds__(256)
k_resid(LMat<V> A, const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x, T beta0,
        T* __restrict__ r_out) {
  pdl_trigger();
  pdl_wait();
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int r, lane;
  row_lane<L>(gid, r, lane);
  bool valid = r < A.n;
  const bool owner = valid && lane == 0;
  const T br = owner ? b[r] : T(0);   // in flight with the row product
  T ax = row_dot<L, V, T>(A, valid ? r : -1, lane, [&](int c) {
    return (XM == XM_IMPLICIT) ? beta0 * dinv[c] * b[c] : x[c];
  });
  if (owner) r_out[r] = br - ax;
}

// y = R x (restriction)
template <typename T, int L>
__global__ void __launch_bounds__(256)
k_spmv(LMat<T> A, const T* __restrict__ x, T* __restrict__ y) {
  pdl_trigger();
  pdl_wait();
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int r, lane;
  row_lane<L>(gid, r, lane);
  bool valid = r < A.n;
  T s = row_dot<L, T, T>(A, valid ? r : -1, lane, [&](int c) { return x[c]; });
  if (valid && lane == 0) y[r] = s;
}

// x += P e (prolongation and correction); IMPLICIT: x starts as beta0 dinv b
template <typename T, int L, bool IMPLICIT>
__global__ void __launch_bounds__(256)
k_prolong(LMat<T> P, const T* __restrict__ e, T* x, const T* __restrict__ dinv, const T* __restrict__ b, T beta0) {
  pdl_trigger();
  pdl_wait();
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int r, lane;
  row_lane<L>(gid, r, lane);
  bool valid = r < P.n;
  const bool owner = valid && lane == 0;
  T x0 = T(0);   // in flight with the row product
  if (owner) x0 = IMPLICIT ? beta0 * dinv[r] * b[r] : x[r];
  T s = row_dot<L, T, T>(P, valid ? r : -1, lane, [&](int c) { return e[c]; });
  if (owner) x[r] = x0 + s;
}

// coarsest level: x = A^{-1} b with the stored dense inverse; one warp per row
template <typename T>
__global__ void __launch_bounds__(256)
k_dense_mv(int n, const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x, JPtr<T> out) {
  pdl_trigger();
  pdl_wait();
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const T* row = Ainv + size_t(warp) * n;
  T s = T(0);
  for (int c = lane; c < n; c += 32) s = fma(row[c], b[c], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    if (out.base) out.get()[warp] = s;
    else x[warp] = s;
  }
}

template <typename T>
__global__ void k_copy_out(int n, const T* __restrict__ src, JPtr<T> out) {
  pdl_trigger();
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out.get()[r] = src[r];
}

// dispatch on the lanes-per-row of an operator
#define IRK_DISPATCH_L(LANES, ...)                          \
  switch (LANES) {                                          \
    case -8: { constexpr int LN = -8; __VA_ARGS__; } break;  \
    case -4: { constexpr int LN = -4; __VA_ARGS__; } break;  \
    case -2: { constexpr int LN = -2; __VA_ARGS__; } break;  \
    case 1: { constexpr int LN = 1; __VA_ARGS__; } break;    \
    case 2: { constexpr int LN = 2; __VA_ARGS__; } break;    \
    case 4: { constexpr int LN = 4; __VA_ARGS__; } break;    \
    case 8: { constexpr int LN = 8; __VA_ARGS__; } break;    \
    case 16: { constexpr int LN = 16; __VA_ARGS__; } break;  \
    case 32: { constexpr int LN = 32; __VA_ARGS__; } break;  \
    default: fail(IRK_ERR_INVALID, "bad lanes per row");    \
  }

static inline unsigned grid_for(const MatT& m) { return nblk(m.threads()); }

// y = m x in the V-cycle precision (prec 64: FP64, else FP32 vectors); used by
// the layout autotuner
void matT_spmv_launch(const MatT& m, int prec, const void* x, void* y, cudaStream_t st) {
  if (prec == 64) {
    LMat<double> A = lmat<double>(m);
    IRK_DISPATCH_L(m.lanes, { launch_k(k_spmv<double, LN>, grid_for(m), 256, 0, st, A, static_cast<const double*>(x),
                                                                               static_cast<double*>(y)); });
  } else {
    LMat<float> A = lmat<float>(m);
    IRK_DISPATCH_L(m.lanes, { launch_k(k_spmv<float, LN>, grid_for(m), 256, 0, st, A, static_cast<const float*>(x),
                                                                              static_cast<float*>(y)); });
  }
  CK_LAUNCH();
}

// ---------------------------------------------------------------------------
// V-cycle driver (kernel sequence; captured into CUDA graphs by the caller)
// ---------------------------------------------------------------------------
// algorithmic DRAM bytes / flops of the kernels (each operand counted once)
struct Cost {
  double bytes = 0.0, flops = 0.0;
};

template <typename T, typename V0>
struct VCycle {
  const Hier& H;
  const AmgParams& p;
  const SmoothCoef& sc;
  cudaStream_t st;
  int launches = 0;
  Cost cost;

  template <typename V>
  void count_matvec(const Level& L, int vec_reads, int vec_writes) {
    const double idx_bytes = L.Am.uses_sell() ? offset_bytes_per_entry(L.Am.sell)
                                               : (L.Am.dcol ? 2.0 : 4.0);   // 16-bit / shared offsets
    cost.bytes += double(L.nnz) * (idx_bytes + sizeof(V)) + double(L.n) * sizeof(T) * (vec_reads + vec_writes);
    cost.flops += 2.0 * double(L.nnz) + 4.0 * L.n;
  }

  template <typename V, int XM>
  void smooth(const Level& L, const T* xin, const T* din, T* xout, T* dout, int step, JPtr<T> out) {
    LMat<V> A = lmat<V>(L.Am);
    IRK_DISPATCH_L(L.Am.lanes, {
      launch_k(k_smooth<V, T, LN, XM>, grid_for(L.Am), 256, 0, st, A, static_cast<const T*>(L.dinv),
                                                           static_cast<const T*>(L.b), xin, din, xout, dout,
                                                           T(sc.alpha[step]), T(sc.beta[step]), T(sc.beta[0]), out);
    });
    ++launches;
    // reads: x (or b, dinv for the implicit step), b, dinv, d_prev; writes x, d
    count_matvec<V>(L, XM == XM_EXPLICIT ? (din ? 4 : 3) : 2, dout ? 2 : 1);
  }

  // returns the buffer holding the level's result (or nullptr if written to out)
  template <typename V>
  T* level(int l, JPtr<T> out) {
    const Level& L = H.lv[l];
    T* b = static_cast<T*>(L.b);
    T* xb = static_cast<T*>(L.x);
    T* yb = static_cast<T*>(L.y);
    T* db = static_cast<T*>(L.d);
    T* rb = static_cast<T*>(L.r);
    JPtr<T> none = jptr<T>(nullptr);
    int last = static_cast<int>(H.lv.size()) - 1;
    if (l == last && H.coarse_smooth) {
      // stalled coarsest level: 4 smoothing sweeps from zero
      const int steps = sc.steps;
      bool implicit = false;
      T* cur = xb;
      T* oth = yb;
      int total = 4 * steps, q = 0;
      for (int sw = 0; sw < 4; ++sw) {
        for (int k = 0; k < steps; ++k, ++q) {
          bool final_step = (q == total - 1);
          JPtr<T> o = (final_step && out.base) ? out : none;
          if (sw == 0 && k == 0) {
            if (total == 1) {
              smooth<V, XM_ZERO>(L, nullptr, nullptr, cur, db, 0, o);
              break;
            }
            implicit = true;
            continue;
          }
          if (implicit) {
            smooth<V, XM_IMPLICIT>(L, nullptr, nullptr, cur, db, k, o);
            implicit = false;
          } else {
            smooth<V, XM_EXPLICIT>(L, cur, k == 0 ? nullptr : db, oth, db, k, o);
            T* t = cur;
            cur = oth;
            oth = t;
          }
        }
      }
      return out.base ? nullptr : cur;
    }
    if (l == last) {
      int nl = L.n;
      unsigned blocks = nblk(int64_t(nl) * 32);
      launch_k(k_dense_mv<T>, blocks, 256, 0, st, nl, static_cast<const T*>(H.cinv), b, xb, out);
      ++launches;
      cost.bytes += double(nl) * nl * sizeof(T) + 2.0 * nl * sizeof(T);
      cost.flops += 2.0 * double(nl) * nl;
      return out.base ? nullptr : xb;
    }
    const int steps = sc.steps;
    // ---- pre-smoothing from zero
    bool implicit = false;   // x = beta0 dinv b, d = x, not materialised
    T* cur = xb;
    T* oth = yb;
    for (int sw = 0; sw < p.nu_pre; ++sw) {
      for (int k = 0; k < steps; ++k) {
        if (sw == 0 && k == 0) {
          implicit = true;
          continue;
        }
        if (implicit) {
          smooth<V, XM_IMPLICIT>(L, nullptr, nullptr, cur, db, k, none);
          implicit = false;
        } else {
          smooth<V, XM_EXPLICIT>(L, cur, k == 0 ? nullptr : db, oth, db, k, none);
          T* t = cur;
          cur = oth;
          oth = t;
        }
      }
    }
    // ---- coarse-grid correction(s): once in the V-cycle; twice on levels l >= 1 of the
    // W-cycle below the finest level, unless the next level is the coarsest
    const T beta0 = T(sc.beta[0]);
    const int corrections = (p.w_coarse && l >= 1 && l + 2 <= last) ? 2 : 1;
    const Level& C = H.lv[l + 1];
    for (int corr = 0; corr < corrections; ++corr) {
      const bool first = corr == 0;
      const bool have_x = p.nu_pre > 0 || !first;   // else x = 0 and the residual is b
      // residual r = b - A x (x implicit after a first step from zero)
      if (have_x) {
        LMat<V> A = lmat<V>(L.Am);
        const T* dv = static_cast<const T*>(L.dinv);
        IRK_DISPATCH_L(L.Am.lanes, {
          if (first && implicit)
            launch_k(k_resid<V, T, LN, XM_IMPLICIT>, grid_for(L.Am), 256, 0, st, A, dv, b, nullptr, beta0, rb);
          else
            launch_k(k_resid<V, T, LN, XM_EXPLICIT>, grid_for(L.Am), 256, 0, st, A, dv, b, cur, beta0, rb);
        });
        ++launches;
        count_matvec<V>(L, 2, 1);
      }
      // restriction
      {
        LMat<T> R = lmat<T>(L.Rm);
        const T* src = have_x ? rb : b;
        IRK_DISPATCH_L(L.Rm.lanes, { launch_k(k_spmv<T, LN>, grid_for(L.Rm), 256, 0, st, R, src, static_cast<T*>(C.b)); });
      }
      ++launches;
      cost.bytes += double(L.Rm.nnz) * (sizeof(int) + sizeof(T)) + double(L.n + C.n) * sizeof(T);
      cost.flops += 2.0 * double(L.Rm.nnz);
      T* e = level<T>(l + 1, none);
      // prolongation and correction x += P e (x = beta0 D^-1 b + P e after an implicit step)
      {
        LMat<T> P = lmat<T>(L.Pm);
        const T* dv = static_cast<const T*>(L.dinv);
        if (!have_x) CK(cudaMemsetAsync(cur, 0, sizeof(T) * L.n, st));
        IRK_DISPATCH_L(L.Pm.lanes, {
          if (first && p.nu_pre > 0 && implicit)
            launch_k(k_prolong<T, LN, true>, grid_for(L.Pm), 256, 0, st, P, e, cur, dv, b, beta0);
          else
            launch_k(k_prolong<T, LN, false>, grid_for(L.Pm), 256, 0, st, P, e, cur, nullptr, nullptr, beta0);
        });
      }
      ++launches;
      cost.bytes += double(L.Pm.nnz) * (sizeof(int) + sizeof(T)) + double(2 * L.n + C.n) * sizeof(T);
      cost.flops += 2.0 * double(L.Pm.nnz);
    }
    // ---- post-smoothing
    int total = p.nu_post * steps;
    int q = 0;
    for (int sw = 0; sw < p.nu_post; ++sw) {
      for (int k = 0; k < steps; ++k, ++q) {
        bool final_step = (q == total - 1);
        JPtr<T> o = (final_step && out.base) ? out : none;
        smooth<V, XM_EXPLICIT>(L, cur, k == 0 ? nullptr : db, oth, db, k, o);
        T* t = cur;
        cur = oth;
        oth = t;
      }
    }
    if (total == 0 && out.base) {
      launch_k(k_copy_out<T>, nblk(L.n), 256, 0, st, L.n, cur, out);
      ++launches;
    }
    return out.base ? nullptr : cur;
  }
};

template <typename T, typename V0>
static int run_vcycle(const Hier& H, const AmgParams& p, const SmoothCoef& sc, JPtr<T> out,
                      cudaStream_t st, double* bytes, double* flops) {
  VCycle<T, V0> vc{H, p, sc, st, 0, Cost{}};
  vc.template level<V0>(0, out);
  CK_LAUNCH();
  if (bytes) *bytes += vc.cost.bytes;
  if (flops) *flops += vc.cost.flops;
  return vc.launches;
}

int vcycle_launch(const Hier& H, const AmgParams& p, const SmoothCoef& sc, void* out_base, const int* jp,
                  int64_t jstride, int64_t off, cudaStream_t st, double* bytes, double* flops) {
  if (H.amg_prec == 64) {
    JPtr<double> o = jptr<double>(static_cast<double*>(out_base), jp, jstride, 0, off);
    return run_vcycle<double, double>(H, p, sc, o, st, bytes, flops);
  }
  JPtr<float> o = jptr<float>(static_cast<float*>(out_base), jp, jstride, 0, off);
  if (H.amg_prec == 16) return run_vcycle<float, __nv_bfloat16>(H, p, sc, o, st, bytes, flops);
  return run_vcycle<float, float>(H, p, sc, o, st, bytes, flops);
}

// the part of one V-cycle from level l0 >= 1 down (on that level's buffers)
int vcycle_launch_from(const Hier& H, const AmgParams& p, const SmoothCoef& sc, int l0, cudaStream_t st,
                       double* bytes, double* flops) {
  if (l0 < 1 || l0 >= static_cast<int>(H.lv.size())) fail(IRK_ERR_INVALID, "start level out of range");
  int launches = 0;
  if (H.amg_prec == 64) {
    VCycle<double, double> vc{H, p, sc, st, 0, Cost{}};
    vc.template level<double>(l0, jptr<double>(nullptr));
    launches = vc.launches;
    if (bytes) *bytes += vc.cost.bytes;
    if (flops) *flops += vc.cost.flops;
  } else {
    VCycle<float, float> vc{H, p, sc, st, 0, Cost{}};
    vc.template level<float>(l0, jptr<float>(nullptr));
    launches = vc.launches;
    if (bytes) *bytes += vc.cost.bytes;
    if (flops) *flops += vc.cost.flops;
  }
  CK_LAUNCH();
  return launches;
}

// one explicit finest-level smoothing step (step index 1) of hierarchy H
void smooth0_launch(const Hier& H, const AmgParams& p, const SmoothCoef& sc, cudaStream_t st, double* bytes,
                    double* flops) {
  const Level& L = H.lv[0];
  JPtr<float> n32 = jptr<float>(nullptr);
  JPtr<double> n64 = jptr<double>(nullptr);
  int step = sc.steps > 1 ? 1 : 0;
  if (H.amg_prec == 64) {
    VCycle<double, double> vc{H, p, sc, st, 0, Cost{}};
    vc.template smooth<double, XM_EXPLICIT>(L, static_cast<double*>(L.x), static_cast<double*>(L.d),
                                            static_cast<double*>(L.y), static_cast<double*>(L.d), step, n64);
    *bytes = vc.cost.bytes;
    *flops = vc.cost.flops;
  } else if (H.amg_prec == 16) {
    VCycle<float, __nv_bfloat16> vc{H, p, sc, st, 0, Cost{}};
    vc.template smooth<__nv_bfloat16, XM_EXPLICIT>(L, static_cast<float*>(L.x), static_cast<float*>(L.d),
                                                   static_cast<float*>(L.y), static_cast<float*>(L.d), step, n32);
    *bytes = vc.cost.bytes;
    *flops = vc.cost.flops;
  } else {
    VCycle<float, float> vc{H, p, sc, st, 0, Cost{}};
    vc.template smooth<float, XM_EXPLICIT>(L, static_cast<float*>(L.x), static_cast<float*>(L.d),
                                           static_cast<float*>(L.y), static_cast<float*>(L.d), step, n32);
    *bytes = vc.cost.bytes;
    *flops = vc.cost.flops;
  }
  CK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Block substitution right-hand side (Section 4.2):
//   rhs_j = sigma_j v_j - sum_{k in prev(j)} h A~_jk F w_k
// one pass over F for all coupled stages; w_k are the already computed stage
// outputs in Z[j].
// ---------------------------------------------------------------------------
struct Couplings {
  int n;
  int idx[MAX_S];
  float c32[MAX_S];
  double c64[MAX_S];
};

template <typename T, int NP>
__global__ void __launch_bounds__(256)
k_sweep_rhs(SellView<T> F, const double* __restrict__ V, const int* __restrict__ jp, int64_t ldv,
            int64_t voff, const double* __restrict__ sigma, const T* __restrict__ Z, int64_t ldz,
            Couplings cp, const int* __restrict__ skip, T* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int n = F.n;
  if (r >= n) return;
  if (skip && *skip) {
    out[r] = T(0);
    return;
  }
  int j = jp ? *jp : 0;
  double sj = sigma ? sigma[j] : 1.0;
  T v = static_cast<T>(V[int64_t(j) * ldv + voff + r] * sj);
  if (NP == 0) {
    out[r] = v;
    return;
  }
  const T* zj = Z + int64_t(j) * ldz;
  T acc[NP > 0 ? NP : 1];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q] = T(0);
  auto entry = [&](int64_t idx, int c) {
    T f = F.val[idx];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q] = fma(f, zj[int64_t(cp.idx[q]) * n + c], acc[q]);
  };
  int sl = r >> 5, lane = r & 31;
  // a shared slice pattern (width and 16-byte slot) is loaded alongside the slice base
  int wu = 0;
  union {
    int4 v;
    short o[PAT_W];
  } pat;
  if (F.suni) {
    wu = F.suni[sl];
    pat.v = reinterpret_cast<const int4*>(F.pdcol)[sl];
  }
  int64_t base = F.sptr[sl];
  if (wu) {
#pragma unroll
    for (int k = 0; k < PAT_W; ++k)
      if (k < wu) entry(base + (int64_t(k) << 5) + lane, r + static_cast<int>(pat.o[k]));
  } else {
    int w = static_cast<int>((F.sptr[sl + 1] - base) >> 5);
    for (int k = 0; k < w; ++k) {
      int64_t idx = base + (int64_t(k) << 5) + lane;
      entry(idx, sell_col(F.col, F.dcol, idx, r));
    }
  }
  T res = v;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    T cq = sizeof(T) == 8 ? static_cast<T>(cp.c64[q]) : static_cast<T>(cp.c32[q]);
    res = fma(-cq, acc[q], res);
  }
  out[r] = res;
}

template <typename T>
static void launch_sweep_rhs(int np, SellView<T> F, const double* V, const int* jp, int64_t ldv, int64_t voff,
                             const double* sigma, const T* Z, int64_t ldz, const Couplings& cp, const int* skip,
                             T* out, cudaStream_t st) {
  unsigned g = nblk(F.n);
  switch (np) {
#define IRK_SW(NPV) \
  case NPV: launch_k(k_sweep_rhs<T, NPV>, g, 256, 0, st, F, V, jp, ldv, voff, sigma, Z, ldz, cp, skip, out); break;
    IRK_SW(0) IRK_SW(1) IRK_SW(2) IRK_SW(3) IRK_SW(4) IRK_SW(5) IRK_SW(6) IRK_SW(7)
#undef IRK_SW
    default: fail(IRK_ERR_INVALID, "too many stage couplings");
  }
}

int precond_launch(Ctx& c, const PrecondArgs& a, bool transpose, cudaStream_t st) {
  const SweepPlan& P = transpose ? c.planT : c.plan;
  int n = c.n;
  int launches = 0;
  bool f64 = c.amg.amg_prec == 64;
  for (int pos = 0; pos < P.s; ++pos) {
    int stage = P.order[pos];
    const Hier& H = c.hiers[P.hier[pos]];
    Couplings cp;
    cp.n = P.nprev[pos];
    for (int q = 0; q < MAX_S; ++q) {
      cp.idx[q] = q < cp.n ? P.prev[pos][q] : 0;
      cp.c64[q] = q < cp.n ? P.coef[pos][q] : 0.0;
      cp.c32[q] = static_cast<float>(cp.c64[q]);
    }
    if (f64) {
      launch_sweep_rhs<double>(cp.n, view<double>(c.Fs), a.V, a.jp, a.ldv, int64_t(stage) * n, a.sigma,
                               static_cast<const double*>(a.Z), a.ldz, cp, a.skip,
                               static_cast<double*>(H.lv[0].b), st);
    } else {
      launch_sweep_rhs<float>(cp.n, view<float>(c.Fs), a.V, a.jp, a.ldv, int64_t(stage) * n, a.sigma,
                              static_cast<const float*>(a.Z), a.ldz, cp, a.skip, static_cast<float*>(H.lv[0].b),
                              st);
    }
    CK_LAUNCH();
    ++launches;
    if (a.bytes) {
      const Sell& F = c.Fs;
      double sv = f64 ? 8.0 : 4.0;
      *a.bytes += double(c.Fc.nnz) * (offset_bytes_per_entry(F) + sv) * (cp.n > 0 ? 1 : 0) + double(n) * (8.0 + sv) +
                  double(n) * sv * cp.n;
      *a.flops += 2.0 * double(c.Fc.nnz) * cp.n + 2.0 * n * cp.n;
      (void)F;
    }
    launches += vcycle_launch(H, c.amg, c.sc, a.Z, a.jp, a.ldz, int64_t(stage) * n, st, a.bytes, a.flops);
  }
  return launches;
}

}  // namespace irk
