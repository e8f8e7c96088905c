// FP64 kernels of the outer solve: the Kronecker operator of Section 4,
// A z = (I_s (x) M + h A (x) F) z, the stage right-hand side of
// Eq. block_coeff_mtx, restarted right-preconditioned flexible GMRES with
// classical Gram-Schmidt (a second pass when the projected norm drops below
// eta of the original, eta = 0.1 by default), the IRK update u_{n+1} = u_n + h sum_i b_i k_i
// (Section 2), and the discrete adjoint kernels.
//
// All FGMRES control lives on the device (GmresState): the index j, the
// Hessenberg matrix, the Givens rotations and the convergence decision, so an
// iteration is a fixed kernel sequence that a CUDA graph replays.  Reductions
// are deterministic: per-block partial sums (fixed shuffle tree), then the
// last block to finish sums the partials in block order.
#include "irk_internal.cuh"

#include <cmath>
#include <cstdlib>

namespace irk {

constexpr int PL = MAX_M + 2;   // partial-sum slots per block
constexpr int BS = OUTER_BLOCK;   // threads per block of the outer kernels

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Exact FP32 -> FP64 widening by IEEE-754 field arithmetic on the integer
// pipe only (the conversion instruction shares the narrow FP64 pipe with the
// DFMAs of the operator).  Normal numbers: sign kept, exponent re-biased by
// 1023 - 127 = 896, the 23 fraction bits become the top of the 52.  Zero keeps
// its sign; a subnormal m 2^-149 is normalised (leading one of m at bit p gives
// exponent p - 149); infinities and NaNs keep their fraction bits.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  unsigned hi, lo;
  if (e == 0xffu) {
    hi = sign | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (e != 0u) {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {
    hi = sign;
    lo = 0u;
  } else {
    const int p = 31 - __clz(static_cast<int>(m));
    const unsigned long long f = (static_cast<unsigned long long>(m) << (52 - p)) & 0xfffffffffffffull;
    hi = sign | (static_cast<unsigned>(p - 149 + 1023) << 20) | static_cast<unsigned>(f >> 32);
    lo = static_cast<unsigned>(f);
  }
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// Sum C <= 16 per-thread values over the block; thread t < C writes slot t.
// Within a warp a transposing butterfly: at each of the first log2(P) xor
// steps (P = C rounded up to a power of two) a lane keeps one half of its
// values and adds the partner's copy of that half, so a lane performs P - 1
// adds (plus 5 - log2 P for the lanes that share an index) instead of 5 C.
// Lane l then holds value index (l >> (5 - log2 P)) & (P - 1).  The warps'
// results are added in warp order (deterministic).
template <int C>
__device__ __forceinline__ void block_sum_store_t(const double (&v)[C], double* __restrict__ out) {
  static_assert(C >= 1 && C <= 16, "1..16 values");
  constexpr int LP = C <= 1 ? 0 : C <= 2 ? 1 : C <= 4 ? 2 : C <= 8 ? 3 : 4;
  constexpr int P = 1 << LP;
  __shared__ double sm[BS / 32][P];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double a[P];
#pragma unroll
  for (int q = 0; q < P; ++q) a[q] = q < C ? v[q] : 0.0;
#pragma unroll
  for (int k = 0; k < LP; ++k) {
    const int half = P >> (k + 1);
    const int mbit = 16 >> k;
    const bool up = (lane & mbit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      double send = up ? a[i] : a[i + half];
      double keep = up ? a[i + half] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, mbit);
    }
  }
  double x = a[0];
#pragma unroll
  for (int mbit = 16 >> LP; mbit > 0; mbit >>= 1) x += __shfl_xor_sync(0xffffffffu, x, mbit);
  constexpr int SH = 5 - LP;
  if ((lane & ((1 << SH) - 1)) == 0) sm[warp][(lane >> SH) & (P - 1)] = x;
  __syncthreads();
  if (threadIdx.x < C) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < BS / 32; ++w) s += sm[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// sum NV per-thread values over the block; thread t < NV writes slot t
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* __restrict__ out, int cnt = NV) {
  __shared__ double sm[BS / 32][NV];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[q] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[warp][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV && threadIdx.x < cnt) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < BS / 32; ++w) s += sm[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ bool last_block(GmresState* st) {
  __shared__ bool am;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&st->counter, 1u);
    am = (t == gridDim.x - 1);
  }
  __syncthreads();
  return am;
}

// Sum of partial q over the grid's blocks, by one whole warp (every lane returns it): the
// lanes load strided partials, so the loads are in flight together, and meet in a shuffle
// tree.  Deterministic: the order depends only on the grid size.
__device__ __forceinline__ double warp_gather_partials(const double* partials, int q) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < static_cast<int>(gridDim.x); b += 32) s += ldcg(partials + int64_t(b) * PL + q);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// ---------------------------------------------------------------------------
// Givens update of Hessenberg column j and the convergence decision
// ---------------------------------------------------------------------------
__device__ void gmres_finish(GmresState* st, double hnext) {
  int j = st->j;
  double* Hc = st->H + j * (MAX_M + 1);
  Hc[j + 1] = hnext;
  st->sigma[j + 1] = (hnext != 0.0) ? 1.0 / hnext : 0.0;
  for (int i = 0; i < j; ++i) {
    double t = st->cs[i] * Hc[i] + st->sn[i] * Hc[i + 1];
    Hc[i + 1] = -st->sn[i] * Hc[i] + st->cs[i] * Hc[i + 1];
    Hc[i] = t;
  }
  double den = hypot(Hc[j], Hc[j + 1]);
  double c = den != 0.0 ? Hc[j] / den : 1.0;
  double s = den != 0.0 ? Hc[j + 1] / den : 0.0;
  st->cs[j] = c;
  st->sn[j] = s;
  Hc[j] = den;
  Hc[j + 1] = 0.0;
  st->g[j + 1] = -s * st->g[j];
  st->g[j] = c * st->g[j];
  st->it += 1;
  double est = fabs(st->g[j + 1]);
  bool bad = !isfinite(est) || !isfinite(den);
  if (bad) {
    st->status = IRK_ERR_NONFINITE;
    st->done = 1;
    return;
  }
  bool conv = est <= st->rtol * st->bnorm;
  if (conv || j + 1 >= st->m || st->it >= st->max_it || hnext == 0.0 || den == 0.0)
    st->cycle_end = 1;
  else
    st->j = j + 1;
}

// ---------------------------------------------------------------------------
// Kronecker operator, one thread per row (grid-stride), each nonzero of the
// shared M/F pattern read once for all s stages:
//   w_i = (M z_i) + sum_j (h a_ij) (F z_j)
// MODE 0: w = A z;  MODE 1: w = b - A z with the squared norm reduced and the
// restart decision taken by the last block (true residual of FGMRES).
// ---------------------------------------------------------------------------
template <int S, typename TZ, int MODE>
__global__ void __launch_bounds__(BS)
k_kron(int n, SellView<double> Mv, const double* __restrict__ Fval, JPtr<const TZ> zp, JPtr<double> wp,
       KronCoef K, const double* __restrict__ bsub, GmresState* st, double* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (st) {
    if (st->done) return;
    if (MODE == 1 && !st->cycle_end) return;
  }
  const TZ* __restrict__ z = zp.get();
  double* __restrict__ w = wp.get();
  double nrm = 0.0;
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    double mz[S], fz[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      mz[i] = 0.0;
      fz[i] = 0.0;
    }
    int sl = r >> 5, lane = r & 31;
    int64_t base = Mv.sptr[sl];
    int wdt = static_cast<int>((Mv.sptr[sl + 1] - base) >> 5);
    for (int k = 0; k < wdt; ++k) {
      int64_t idx = base + (int64_t(k) << 5) + lane;
      int c = sell_col(Mv.col, Mv.dcol, idx, r);
      double m = Mv.val[idx];
      double f = Fval[idx];
#pragma unroll
      for (int i = 0; i < S; ++i) {
        double zz = to_f64(z[int64_t(i) * n + c]);
        mz[i] = fma(m, zz, mz[i]);
        fz[i] = fma(f, zz, fz[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double wi = mz[i];
#pragma unroll
      for (int j = 0; j < S; ++j) wi = fma(K.a[i * MAX_S + j], fz[j], wi);
      if (MODE == 1) {
        wi = bsub[int64_t(i) * n + r] - wi;
        nrm = fma(wi, wi, nrm);
      }
      w[int64_t(i) * n + r] = wi;
    }
  }
  if (MODE == 1) {
    double v[1] = {nrm};
    block_sum_store<1>(v, partials + int64_t(blockIdx.x) * PL);
    if (last_block(st)) {
      double b2 = 0.0;
      if (threadIdx.x < 32) b2 = warp_gather_partials(partials, 0);
      if (threadIdx.x == 0) {
        double beta = sqrt(b2);
        st->resid = beta / st->bnorm;
        st->cycle_end = 0;
        if (!isfinite(beta)) {
          st->status = IRK_ERR_NONFINITE;
          st->done = 1;
        } else if (beta <= st->rtol * st->bnorm) {
          st->done = 1;
        } else if (st->it >= st->max_it) {
          st->status = IRK_ERR_NOT_CONVERGED;
          st->done = 1;
        } else {
          st->sigma[0] = 1.0 / beta;
          st->g[0] = beta;
          for (int i = 1; i <= MAX_M; ++i) st->g[i] = 0.0;
          st->j = 0;
          st->restarts += 1;
        }
        st->counter = 0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The operator on FP32 vectors (the FGMRES product on FP32 preconditioner
// outputs) in single-float pair arithmetic, off the narrow FP64 pipe.  An FP64
// entry m is held as hi + lo with hi = rn(m), lo = rn(m - hi), so that
// |m - hi - lo| <= 2^-48 |m|.  A product of hi with an FP32 z is exact as p + e
// (e the FMA residual, the error-free product of Ogita, Rump and Oishi 2005);
// a sum h + p is exact as s + t (Knuth's TwoSum).  The accumulator (h, l) keeps
// the rounded head in h and a float tail of the small terms in l, so a row sum
// is off by about 2^-47 of the sum of its absolute terms (FP64 2^-53), and the
// result h + l is formed in FP64 at the end.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ff_add(float& h, float& l, float p, float tail) {
  const float s = __fadd_rn(h, p);
  const float b = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, b)), __fsub_rn(p, b));
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, tail));
}

// (h, l) += (ah + al) z
__device__ __forceinline__ void ff_fma1(float& h, float& l, float ah, float al, float z) {
  const float p = __fmul_rn(ah, z);
  const float e = __fmaf_rn(ah, z, -p);
  ff_add(h, l, p, __fmaf_rn(al, z, e));
}

// (h, l) += (ah + al)(bh + bl), the al bl term dropped (2^-48 relative)
__device__ __forceinline__ void ff_fma2(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  ff_add(h, l, p, e);
}

// w = A z for FP32 z: one thread per row (grid-stride), {M hi, M lo, F hi,
// F lo} of each nonzero in one 16-byte load, all s stages per nonzero.
template <int S>
__global__ void __launch_bounds__(BS)
k_kron_ff(int n, SellView<double> Mv, const float4* __restrict__ mf, JPtr<const float> zp, JPtr<double> wp,
          KronCoefF K, GmresState* st) {
  pdl_trigger();
  pdl_wait();
  if (st && st->done) return;
  const float* __restrict__ z = zp.get();
  double* __restrict__ w = wp.get();
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    float mh[S], ml[S], fh[S], fl[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      mh[i] = 0.f;
      ml[i] = 0.f;
      fh[i] = 0.f;
      fl[i] = 0.f;
    }
    auto entry = [&](int64_t idx, int c) {
      const float4 q = mf[idx];
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const float zz = z[int64_t(i) * n + c];
        ff_fma1(mh[i], ml[i], q.x, q.y, zz);
        ff_fma1(fh[i], fl[i], q.z, q.w, zz);
      }
    };
    int sl = r >> 5, lane = r & 31;
    // a shared slice pattern (width and 16-byte slot) is loaded alongside the slice base
    int wu = 0;
    union {
      int4 v;
      short o[PAT_W];
    } pat;
    if (Mv.suni) {
      wu = Mv.suni[sl];
      pat.v = reinterpret_cast<const int4*>(Mv.pdcol)[sl];
    }
    int64_t base = Mv.sptr[sl];
    if (wu) {
#pragma unroll
      for (int k = 0; k < PAT_W; ++k)
        if (k < wu) entry(base + (int64_t(k) << 5) + lane, r + static_cast<int>(pat.o[k]));
    } else {
      int wdt = static_cast<int>((Mv.sptr[sl + 1] - base) >> 5);
      for (int k = 0; k < wdt; ++k) {
        int64_t idx = base + (int64_t(k) << 5) + lane;
        entry(idx, sell_col(Mv.col, Mv.dcol, idx, r));
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      float h = mh[i], l = ml[i];
#pragma unroll
      for (int j = 0; j < S; ++j) ff_fma2(h, l, K.hi[i * MAX_S + j], K.lo[i * MAX_S + j], fh[j], fl[j]);
      w[int64_t(i) * n + r] = to_f64(h) + to_f64(l);
    }
  }
}

// {M hi, M lo, F hi, F lo}; flag entries outside [2^-64, 2^64] (other than 0)
__global__ void k_split_ff(int64_t nnz, const double* __restrict__ m, const double* __restrict__ f,
                           float4* __restrict__ out, int* __restrict__ bad) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= nnz) return;
  const double a = m[i], b = f[i];
  const double big = 18446744073709551616.0, small = 1.0 / 18446744073709551616.0;   // 2^64, 2^-64
  const bool ok_a = a == 0.0 || (fabs(a) <= big && fabs(a) >= small);
  const bool ok_b = b == 0.0 || (fabs(b) <= big && fabs(b) >= small);
  if (!(ok_a && ok_b)) atomicOr(bad, 1);
  const float ah = __double2float_rn(a), bh = __double2float_rn(b);
  out[i] = make_float4(ah, __double2float_rn(a - static_cast<double>(ah)), bh,
                       __double2float_rn(b - static_cast<double>(bh)));
}

// ---------------------------------------------------------------------------
// Gram-Schmidt.  Basis vectors V_i are stored unnormalised; v_i = sigma_i V_i.
// dots:  h_i = sigma_i <w, V_i> (i <= j) and ||w||^2 (PASS 0), or the
//        reorthogonalisation coefficients (PASS 1, only when st->reorth).
// axpy:  w -= sum_i h_i sigma_i V_i and ||w||^2; the last block decides on
//        reorthogonalisation or finishes the iteration.
// ---------------------------------------------------------------------------
constexpr int CH = 16;

// C basis vectors starting at i0 against w: per-block partial sums into slots
// i0 .. i0 + C - 1 (exact count, so no predicated-off DFMAs)
template <int C>
__device__ __forceinline__ void dots_chunk(const double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                                           int64_t N, int i0, double* __restrict__ out) {
  double acc[C];
#pragma unroll
  for (int q = 0; q < C; ++q) acc[q] = 0.0;
  const double* __restrict__ Vb = V + int64_t(i0) * ldv;
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) {
    double we = w[e];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = fma(Vb[int64_t(q) * ldv + e], we, acc[q]);
  }
  block_sum_store_t<C>(acc, out + i0);
}

template <int PASS>
__global__ void __launch_bounds__(BS, 4)
k_gs_dots(GmresState* st, const double* __restrict__ V, int64_t ldv, int64_t N, double* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  if (PASS == 1 && !st->reorth) return;
  int j = st->j;
  const double* __restrict__ w = V + int64_t(j + 1) * ldv;
  int nvec = (PASS == 0) ? j + 2 : j + 1;   // PASS 0 also takes <w, w>
  // near-equal chunks of at most CH vectors
  int nch = (nvec + CH - 1) / CH;
  int base = nvec / nch, extra = nvec % nch;
  double* pb = partials + int64_t(blockIdx.x) * PL;
  for (int ch = 0, i0 = 0; ch < nch; ++ch) {
    int cnt = base + (ch < extra ? 1 : 0);
    switch (cnt) {
#define IRK_DC(K) case K: dots_chunk<K>(V, ldv, w, N, i0, pb); break;
      IRK_DC(1) IRK_DC(2) IRK_DC(3) IRK_DC(4) IRK_DC(5) IRK_DC(6) IRK_DC(7) IRK_DC(8)
      IRK_DC(9) IRK_DC(10) IRK_DC(11) IRK_DC(12) IRK_DC(13) IRK_DC(14) IRK_DC(15) IRK_DC(16)
#undef IRK_DC
      default: break;
    }
    i0 += cnt;
  }
  if (last_block(st)) {
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < nvec; i += BS / 32) {
      double d = warp_gather_partials(partials, i);
      if (lane != 0) continue;
      if (i <= j) {
        double h = st->sigma[i] * d;
        if (PASS == 0) st->H[j * (MAX_M + 1) + i] = h;
        else {
          st->h2[i] = h;
          st->H[j * (MAX_M + 1) + i] += h;
        }
      } else {
        st->wnorm2 = d;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) st->counter = 0;
  }
}

template <int PASS>
__global__ void __launch_bounds__(BS)
k_gs_axpy(GmresState* st, double* __restrict__ V, int64_t ldv, int64_t N, double* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  if (PASS == 1 && !st->reorth) return;
  __shared__ double coef[MAX_M + 1];
  int j = st->j;
  for (int i = threadIdx.x; i <= j; i += BS)
    coef[i] = (PASS == 0 ? st->H[j * (MAX_M + 1) + i] : st->h2[i]) * st->sigma[i];
  __syncthreads();
  double* __restrict__ w = V + int64_t(j + 1) * ldv;
  double nrm = 0.0;
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) {
    double we = w[e];
    int i = 0;
    for (; i + 4 <= j + 1; i += 4) {
      we = fma(-coef[i], V[int64_t(i) * ldv + e], we);
      we = fma(-coef[i + 1], V[int64_t(i + 1) * ldv + e], we);
      we = fma(-coef[i + 2], V[int64_t(i + 2) * ldv + e], we);
      we = fma(-coef[i + 3], V[int64_t(i + 3) * ldv + e], we);
    }
    for (; i <= j; ++i) we = fma(-coef[i], V[int64_t(i) * ldv + e], we);
    w[e] = we;
    nrm = fma(we, we, nrm);
  }
  double v[1] = {nrm};
  block_sum_store<1>(v, partials + int64_t(blockIdx.x) * PL);
  if (last_block(st)) {
    double n2 = 0.0;
    if (threadIdx.x < 32) n2 = warp_gather_partials(partials, 0);
    if (threadIdx.x == 0) {
      if (PASS == 0 && (st->eta2 < 0.0 || n2 < st->eta2 * st->wnorm2)) {
        st->reorth = 1;
      } else {
        st->reorth = 0;
        gmres_finish(st, sqrt(n2));
      }
      st->counter = 0;
    }
  }
}

// cycle end: y = H^{-1} g (upper triangular, k = j+1 columns; every block
// solves it redundantly), then x += sum_i y_i Z_i
template <typename TZ>
__global__ void __launch_bounds__(BS)
k_xupdate(GmresState* st, const TZ* __restrict__ Z, int64_t ldz, double* __restrict__ x, int64_t N) {
  pdl_trigger();
  pdl_wait();
  if (st->done || !st->cycle_end) return;
  __shared__ double y[MAX_M];
  int k = st->j + 1;
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = st->g[i];
      for (int q = i + 1; q < k; ++q) s -= st->H[q * (MAX_M + 1) + i] * y[q];
      y[i] = s / st->H[i * (MAX_M + 1) + i];
    }
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) {
    double xe = x[e];
    for (int i = 0; i < k; ++i) xe = fma(y[i], to_f64(Z[int64_t(i) * ldz + e]), xe);
    x[e] = xe;
  }
}

// WHILE-node condition: keep iterating until the solve is done.  The body
// count is bounded independently of the solver logic: past max_it + 8 bodies
// the solve stops with IRK_ERR_TIMEOUT.
__global__ void k_loop_ctrl(GmresState* st, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->guard += 1;
    if (!st->done && st->guard > st->max_it + 8) {
      st->done = 1;
      st->status = IRK_ERR_TIMEOUT;
    }
    cudaGraphSetConditional(h, st->done ? 0u : 1u);
  }
}

// ---------------------------------------------------------------------------
// Right-hand sides and FGMRES initialisation (x = 0, V_0 = b, sigma_0 = 1/||b||)
// ---------------------------------------------------------------------------
__device__ void gmres_init_last(GmresState* st, double* partials, int m, int max_it, double rtol, double eta2) {
  double b2 = 0.0;
  if (threadIdx.x < 32) b2 = warp_gather_partials(partials, 0);
  if (threadIdx.x == 0) {
    double beta = sqrt(b2);
    st->bnorm = beta;
    st->bnorm_true = beta;
    st->rtol = rtol;
    st->m = m;
    st->max_it = max_it;
    st->eta2 = eta2;
    st->j = 0;
    st->it = 0;
    st->restarts = 0;
    st->cycle_end = 0;
    st->reorth = 0;
    st->guard = 0;
    st->status = IRK_OK;
    st->resid = beta > 0.0 ? 1.0 : 0.0;
    st->done = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
    if (!isfinite(beta)) st->status = IRK_ERR_NONFINITE;
    st->sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    st->g[0] = beta;
    for (int i = 1; i <= MAX_M; ++i) st->g[i] = 0.0;
    st->counter = 0;
  }
}

// b_i = -(F u + g) for every stage (Eq. block_coeff_mtx); V_0 = b; x = 0
template <int S>
__global__ void __launch_bounds__(BS)
k_rhs_forward(int n, SellView<double> Fv, const double* __restrict__ u, const double* __restrict__ g,
              double* __restrict__ b, double* __restrict__ V0, double* __restrict__ x, GmresState* st,
              double* __restrict__ partials, int m, int max_it, double rtol, double eta2,
              const int* __restrict__ given) {
  pdl_trigger();
  pdl_wait();
  double nrm = 0.0;
  if (*given) {   // irk_solve: b was copied into place by the caller
    for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
#pragma unroll
      for (int i = 0; i < S; ++i) {
        double t = b[int64_t(i) * n + r];
        V0[int64_t(i) * n + r] = t;
        x[int64_t(i) * n + r] = 0.0;
        nrm = fma(t, t, nrm);
      }
    }
    double v[1] = {nrm};
    block_sum_store<1>(v, partials + int64_t(blockIdx.x) * PL);
    if (last_block(st)) gmres_init_last(st, partials, m, max_it, rtol, eta2);
    return;
  }
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    int sl = r >> 5, lane = r & 31;
    int64_t base = Fv.sptr[sl];
    int wdt = static_cast<int>((Fv.sptr[sl + 1] - base) >> 5);
    double t = 0.0;
    for (int k = 0; k < wdt; ++k) {
      int64_t idx = base + (int64_t(k) << 5) + lane;
      t = fma(Fv.val[idx], u[Fv.col[idx]], t);
    }
    t = -(t + (g ? g[r] : 0.0));
#pragma unroll
    for (int i = 0; i < S; ++i) {
      b[int64_t(i) * n + r] = t;
      V0[int64_t(i) * n + r] = t;
      x[int64_t(i) * n + r] = 0.0;
      nrm = fma(t, t, nrm);
    }
  }
  double v[1] = {nrm};
  block_sum_store<1>(v, partials + int64_t(blockIdx.x) * PL);
  if (last_block(st)) gmres_init_last(st, partials, m, max_it, rtol, eta2);
}

// adjoint: b_i = h b_i lambda (the right-hand side of A^T mu = h (b (x) lambda))
template <int S>
__global__ void __launch_bounds__(BS)
k_rhs_adjoint(int n, KronCoef hb, const double* __restrict__ lam, double* __restrict__ b,
              double* __restrict__ V0, double* __restrict__ x, GmresState* st, double* __restrict__ partials,
              int m, int max_it, double rtol, double eta2) {
  pdl_trigger();
  pdl_wait();
  double nrm = 0.0;
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    double l = lam[r];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double t = hb.a[i] * l;
      b[int64_t(i) * n + r] = t;
      V0[int64_t(i) * n + r] = t;
      x[int64_t(i) * n + r] = 0.0;
      nrm = fma(t, t, nrm);
    }
  }
  double v[1] = {nrm};
  block_sum_store<1>(v, partials + int64_t(blockIdx.x) * PL);
  if (last_block(st)) gmres_init_last(st, partials, m, max_it, rtol, eta2);
}

// u += sum_i (h b_i) k_i   (Section 2)
template <int S>
__global__ void __launch_bounds__(BS)
k_stage_update(int n, KronCoef hb, const double* __restrict__ k, double* __restrict__ u) {
  pdl_trigger();
  pdl_wait();
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    double s = u[r];
#pragma unroll
    for (int i = 0; i < S; ++i) s = fma(hb.a[i], k[int64_t(i) * n + r], s);
    u[r] = s;
  }
}

__global__ void k_record(const GmresState* st, StepRecord* rec, int* counter, int cap) {
  if (threadIdx.x || blockIdx.x) return;
  int q = *counter;
  if (q < cap) {
    rec[q].it = st->it;
    rec[q].restarts = st->restarts;
    rec[q].status = st->status;
    rec[q].resid = st->resid;
  }
  *counter = q + 1;
}

// y = M x
__global__ void __launch_bounds__(BS)
k_spmv64(int n, SellView<double> A, const double* __restrict__ x, double* __restrict__ y) {
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    int sl = r >> 5, lane = r & 31;
    int64_t base = A.sptr[sl];
    int wdt = static_cast<int>((A.sptr[sl + 1] - base) >> 5);
    double t = 0.0;
    for (int k = 0; k < wdt; ++k) {
      int64_t idx = base + (int64_t(k) << 5) + lane;
      t = fma(A.val[idx], x[A.col[idx]], t);
    }
    y[r] = t;
  }
}

// lambda_n = lambda_{n+1} - F^T sum_i mu_i   (Fv: F^T, or F when F is symmetric)
template <int S>
__global__ void __launch_bounds__(BS)
k_adj_lambda(int n, SellView<double> Fv, const double* __restrict__ mu, const double* __restrict__ lin,
             double* __restrict__ lout) {
  pdl_trigger();
  pdl_wait();
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    int sl = r >> 5, lane = r & 31;
    int64_t base = Fv.sptr[sl];
    int wdt = static_cast<int>((Fv.sptr[sl + 1] - base) >> 5);
    double t = 0.0;
    for (int k = 0; k < wdt; ++k) {
      int64_t idx = base + (int64_t(k) << 5) + lane;
      int c = Fv.col[idx];
      double ms = 0.0;
#pragma unroll
      for (int i = 0; i < S; ++i) ms += mu[int64_t(i) * n + c];
      t = fma(Fv.val[idx], ms, t);
    }
    lout[r] = lin[r] - t;
  }
}

// dL/dkappa_e += -sum_i mu_i[e]^T K_e U_i[e],  U_i = u + sum_j (h a_ij) k_j
template <int S>
__global__ void __launch_bounds__(BS)
k_adj_grad(int n_tri, const int* __restrict__ tri, const int* __restrict__ dof, const double* __restrict__ Ke,
           KronCoef K, int n, JPtr<const double> up, JPtr<const double> kp, const double* __restrict__ mu,
           double* __restrict__ grad) {
  const double* __restrict__ u = up.get();
  const double* __restrict__ kst = kp.get();
  for (int e = blockIdx.x * BS + threadIdx.x; e < n_tri; e += gridDim.x * BS) {
    int d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = dof[tri[3 * e + a]];
    double ke[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) ke[q] = Ke[int64_t(e) * 9 + q];
    double kv[S][3];
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a) kv[j][a] = d[a] >= 0 ? kst[int64_t(j) * n + d[a]] : 0.0;
    double ua[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ua[a] = d[a] >= 0 ? u[d[a]] : 0.0;
    double gsum = 0.0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double U[3], m3[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double t = ua[a];
#pragma unroll
        for (int j = 0; j < S; ++j) t = fma(K.a[i * MAX_S + j], kv[j][a], t);
        U[a] = t;
        m3[a] = d[a] >= 0 ? mu[int64_t(i) * n + d[a]] : 0.0;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) gsum = fma(m3[a] * ke[a * 3 + bb], U[bb], gsum);
    }
    grad[e] -= gsum;
  }
}

// F values = sum over contributions kappa_e K_e[a][b] (deterministic gather)
__global__ void __launch_bounds__(BS)
k_assemble_kappa(int64_t nnz, const int* __restrict__ ptr, const int* __restrict__ src,
                 const double* __restrict__ Ke, const double* __restrict__ kappa, double* __restrict__ Fval) {
  for (int64_t q = blockIdx.x * int64_t(BS) + threadIdx.x; q < nnz; q += int64_t(gridDim.x) * BS) {
    double s = 0.0;
    for (int t = ptr[q]; t < ptr[q + 1]; ++t) {
      int c = src[t];
      s += kappa[c / 9] * Ke[c];
    }
    Fval[q] = s;
  }
}

__global__ void k_convert(const void* in, int ip, void* out, int op, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  double v = ip == 64 ? static_cast<const double*>(in)[i] : static_cast<double>(static_cast<const float*>(in)[i]);
  if (op == 64) static_cast<double*>(out)[i] = v;
  else static_cast<float*>(out)[i] = static_cast<float>(v);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
#define IRK_DISPATCH_S(S_, ...)                              \
  switch (S_) {                                              \
    case 1: { constexpr int S = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int S = 2; __VA_ARGS__; } break;     \
    case 3: { constexpr int S = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int S = 4; __VA_ARGS__; } break;     \
    case 5: { constexpr int S = 5; __VA_ARGS__; } break;     \
    case 6: { constexpr int S = 6; __VA_ARGS__; } break;     \
    case 7: { constexpr int S = 7; __VA_ARGS__; } break;     \
    case 8: { constexpr int S = 8; __VA_ARGS__; } break;     \
    default: fail(IRK_ERR_INVALID, "s must be 1..8");        \
  }

static unsigned row_grid(const Ctx& c) { return static_cast<unsigned>(c.gs_grid); }

// the pair operator is latency-bound (gathers of z, no FP64 pipe limit): one
// row per thread, so the block scheduler keeps every SM at its register limit
static unsigned ff_grid(const Ctx& c) { return static_cast<unsigned>(c.n > 0 ? (c.n + BS - 1) / BS : 1); }

// One FGMRES iteration after the preconditioner: w = A z_j into V_{j+1},
// Gram-Schmidt, Givens, and at a cycle end x += Z y and the true residual.
int fgmres_body_launch(Ctx& c, bool transpose, cudaStream_t st) {
  const KronCoef& K = transpose ? c.KT : c.K;
  int n = c.n;
  int64_t N = c.N;
  int launches = 0;
  unsigned G = row_grid(c);
  const int* jp = &c.st->j;
  bool z32 = c.amg.amg_prec != 64;
  IRK_DISPATCH_S(c.s, {
    if (z32 && c.MFs)
      launch_k(k_kron_ff<S>, ff_grid(c), BS, 0, st, n, view<double>(c.Ms), static_cast<const float4*>(c.MFs),
                                      JPtr<const float>{static_cast<const float*>(c.Z), jp, N, 0, 0},
                                      JPtr<double>{c.V, jp, N, 1, 0}, transpose ? c.KTf : c.Kf, c.st);
    else if (z32)
      launch_k(k_kron<S, float, 0>, G, BS, 0, st, n, view<double>(c.Ms), c.Fs.v64,
                                            JPtr<const float>{static_cast<const float*>(c.Z), jp, N, 0, 0},
                                            JPtr<double>{c.V, jp, N, 1, 0}, K, nullptr, c.st, c.partials);
    else
      launch_k(k_kron<S, double, 0>, G, BS, 0, st, n, view<double>(c.Ms), c.Fs.v64,
                                             JPtr<const double>{static_cast<const double*>(c.Z), jp, N, 0, 0},
                                             JPtr<double>{c.V, jp, N, 1, 0}, K, nullptr, c.st, c.partials);
  });
  ++launches;
  launch_k(k_gs_dots<0>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launch_k(k_gs_axpy<0>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launch_k(k_gs_dots<1>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launch_k(k_gs_axpy<1>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launches += 4;
  if (z32)
    launch_k(k_xupdate<float>, G, BS, 0, st, c.st, static_cast<const float*>(c.Z), N, c.x, N);
  else
    launch_k(k_xupdate<double>, G, BS, 0, st, c.st, static_cast<const double*>(c.Z), N, c.x, N);
  ++launches;
  IRK_DISPATCH_S(c.s, {
    launch_k(k_kron<S, double, 1>, G, BS, 0, st, n, view<double>(c.Ms), c.Fs.v64, JPtr<const double>{c.x, nullptr, 0, 0, 0},
                                           JPtr<double>{c.V, nullptr, 0, 0, 0}, K, c.bv, c.st, c.partials);
  });
  ++launches;
  CK_LAUNCH();
  return launches;
}

// ---------------------------------------------------------------------------
// Left-preconditioned GMRES on P^{-1} A k = P^{-1} b (x0 = 0), stopping on the
// preconditioned residual.  The basis is built from w = P^{-1} A v_j; the
// preconditioner output (AMG precision) is widened into the next basis slot.
// A restart takes the residual P^{-1}(b - A x) = g_k V_{k+1} Q^T e_k from the
// Givens rotations instead of another operator and preconditioner application.
// ---------------------------------------------------------------------------

// V_{j+1} = sigma_j P^{-1}(A V_j)   (P^{-1} applied to the unscaled A V_j)
template <typename TZ>
__global__ void __launch_bounds__(BS)
k_left_widen(GmresState* st, const TZ* __restrict__ Zt, double* __restrict__ V, int64_t ldv, int64_t N) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  const int j = st->j;
  const double sj = st->sigma[j];
  double* __restrict__ w = V + int64_t(j + 1) * ldv;
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS)
    w[e] = sj * to_f64(Zt[e]);
}

// first basis vector: Zt = P^{-1}(b / ||b||) -> V_0, ||P^{-1} b|| = ||V_0|| ||b||
template <typename TZ>
__global__ void __launch_bounds__(BS)
k_left_start(GmresState* st, const TZ* __restrict__ Zt, double* __restrict__ V, int64_t N,
             double* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  double nrm = 0.0;
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) {
    double v = to_f64(Zt[e]);
    V[e] = v;
    nrm = fma(v, v, nrm);
  }
  double v1[1] = {nrm};
  block_sum_store<1>(v1, partials + int64_t(blockIdx.x) * PL);
  if (last_block(st)) {
    double n0sq = 0.0;
    if (threadIdx.x < 32) n0sq = warp_gather_partials(partials, 0);
    if (threadIdx.x == 0) {
      double n0 = sqrt(n0sq);
      double beta = n0 * st->bnorm;          // ||P^{-1} b||
      st->bnorm_true = st->bnorm;
      st->bnorm = beta;
      st->sigma[0] = n0 > 0.0 ? 1.0 / n0 : 0.0;
      st->g[0] = beta;
      for (int i = 1; i <= MAX_M; ++i) st->g[i] = 0.0;
      if (!(beta > 0.0) || !isfinite(beta)) {
        st->status = isfinite(beta) ? IRK_OK : IRK_ERR_NONFINITE;
        st->done = 1;
        st->resid = 0.0;
      }
      st->counter = 0;
    }
  }
}

// x += sum_i y_i sigma_i V_i at a cycle end (y from the triangular system)
__global__ void __launch_bounds__(BS)
k_left_xupdate(GmresState* st, const double* __restrict__ V, int64_t ldv, double* __restrict__ x, int64_t N) {
  pdl_trigger();
  pdl_wait();
  if (st->done || !st->cycle_end) return;
  __shared__ double y[MAX_M];
  int k = st->j + 1;
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = st->g[i];
      for (int q = i + 1; q < k; ++q) s -= st->H[q * (MAX_M + 1) + i] * y[q];
      y[i] = s / st->H[i * (MAX_M + 1) + i];
    }
    for (int i = 0; i < k; ++i) y[i] *= st->sigma[i];
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) {
    double xe = x[e];
    for (int i = 0; i < k; ++i) xe = fma(y[i], V[int64_t(i) * ldv + e], xe);
    x[e] = xe;
  }
}

// cycle end: stop on the estimate |g_k| (or the iteration cap), else restart
__global__ void k_left_decide(GmresState* st) {
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x || blockIdx.x) return;
  if (st->done || !st->cycle_end) return;
  int k = st->j + 1;
  double est = fabs(st->g[k]);
  st->resid = est / st->bnorm;
  if (est <= st->rtol * st->bnorm || est == 0.0) {
    st->done = 1;
  } else if (st->it >= st->max_it) {
    st->status = IRK_ERR_NOT_CONVERGED;
    st->done = 1;
  }
}

// restart residual r = g_k sum_i t_i sigma_i V_i with t = Q^T e_k, into T
__global__ void __launch_bounds__(BS)
k_left_residual(GmresState* st, const double* __restrict__ V, int64_t ldv, double* __restrict__ T, int64_t N,
                double* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (st->done || !st->cycle_end) return;
  __shared__ double t[MAX_M + 1];
  const int k = st->j + 1;
  if (threadIdx.x == 0) {
    for (int i = 0; i <= k; ++i) t[i] = (i == k) ? 1.0 : 0.0;
    for (int i = k - 1; i >= 0; --i) {   // t <- G_i^T t on rows (i, i+1)
      double c = st->cs[i], s = st->sn[i];
      double a = t[i], b = t[i + 1];
      t[i] = c * a - s * b;
      t[i + 1] = s * a + c * b;
    }
    double gk = st->g[k];
    for (int i = 0; i <= k; ++i) t[i] *= gk * st->sigma[i];
  }
  __syncthreads();
  double nrm = 0.0;
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) {
    double r = 0.0;
    for (int i = 0; i <= k; ++i) r = fma(t[i], V[int64_t(i) * ldv + e], r);
    T[e] = r;
    nrm = fma(r, r, nrm);
  }
  double v1[1] = {nrm};
  block_sum_store<1>(v1, partials + int64_t(blockIdx.x) * PL);
  if (last_block(st)) {
    double b2 = 0.0;
    if (threadIdx.x < 32) b2 = warp_gather_partials(partials, 0);
    if (threadIdx.x == 0) {
      double beta = sqrt(b2);
      st->wnorm2 = beta;   // handed to k_left_restart
      st->counter = 0;
    }
  }
}

// V_0 = T, sigma_0 = 1/||T||, g = ||T|| e_0, next cycle
__global__ void __launch_bounds__(BS)
k_left_restart(GmresState* st, const double* __restrict__ T, double* __restrict__ V, int64_t N) {
  pdl_trigger();
  pdl_wait();
  if (st->done || !st->cycle_end) return;
  for (int64_t e = blockIdx.x * int64_t(BS) + threadIdx.x; e < N; e += int64_t(gridDim.x) * BS) V[e] = T[e];
  if (last_block(st)) {
    if (threadIdx.x == 0) {
      double beta = st->wnorm2;
      st->sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
      st->g[0] = beta;
      for (int i = 1; i <= MAX_M; ++i) st->g[i] = 0.0;
      st->j = 0;
      st->restarts += 1;
      st->cycle_end = 0;
      st->reorth = 0;
      if (!(beta > 0.0)) st->done = 1;
      st->counter = 0;
    }
  }
}

// true relative residual ||b - A x|| / ||b|| for the stats (after the loop)
__global__ void k_left_final_resid(GmresState* st, const double* __restrict__ partials, int count) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int q = 0; q < count; ++q) s += partials[q];
  st->resid = st->bnorm_true > 0.0 ? sqrt(s) / st->bnorm_true : 0.0;
}

// ||b - A k||_2: per-block partial sums of the squared residual, then one
// block sums them in block order
template <int S>
__global__ void __launch_bounds__(BS)
k_resid_partials(int n, SellView<double> Mv, const double* __restrict__ Fval, const double* __restrict__ k,
                 const double* __restrict__ b, KronCoef K, double* __restrict__ partials) {
  double nrm = 0.0;
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    double mz[S], fz[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      mz[i] = 0.0;
      fz[i] = 0.0;
    }
    int sl = r >> 5, lane = r & 31;
    int64_t base = Mv.sptr[sl];
    int wdt = static_cast<int>((Mv.sptr[sl + 1] - base) >> 5);
    for (int q = 0; q < wdt; ++q) {
      int64_t idx = base + (int64_t(q) << 5) + lane;
      int c = sell_col(Mv.col, Mv.dcol, idx, r);
      double m = Mv.val[idx];
      double f = Fval[idx];
#pragma unroll
      for (int i = 0; i < S; ++i) {
        double zz = k[int64_t(i) * n + c];
        mz[i] = fma(m, zz, mz[i]);
        fz[i] = fma(f, zz, fz[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double wi = mz[i];
#pragma unroll
      for (int j = 0; j < S; ++j) wi = fma(K.a[i * MAX_S + j], fz[j], wi);
      wi = b[int64_t(i) * n + r] - wi;
      nrm = fma(wi, wi, nrm);
    }
  }
  double v[1] = {nrm};
  block_sum_store<1>(v, partials + blockIdx.x);
}

__global__ void k_sum_partials(const double* __restrict__ partials, int count, double* __restrict__ out) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int q = 0; q < count; ++q) s += partials[q];
  *out = sqrt(s);
}

// misfit 1/2 (u - d)^T M (u - d): per-block partial sums of (u - d)_r (M (u - d))_r
// (deterministic order), and M (u - d) when grad is given
__global__ void __launch_bounds__(BS)
k_misfit_partials(int n, SellView<double> Mv, const double* __restrict__ u, const double* __restrict__ d,
                  double* __restrict__ grad, double* __restrict__ partials) {
  double acc = 0.0;
  for (int r = blockIdx.x * BS + threadIdx.x; r < n; r += gridDim.x * BS) {
    int sl = r >> 5, lane = r & 31;
    int64_t base = Mv.sptr[sl];
    int wdt = static_cast<int>((Mv.sptr[sl + 1] - base) >> 5);
    double me = 0.0;
    for (int q = 0; q < wdt; ++q) {
      int64_t idx = base + (int64_t(q) << 5) + lane;
      int c = sell_col(Mv.col, Mv.dcol, idx, r);
      me = fma(Mv.val[idx], u[c] - d[c], me);
    }
    if (grad) grad[r] = me;
    acc = fma(u[r] - d[r], me, acc);
  }
  double v[1] = {acc};
  block_sum_store<1>(v, partials + blockIdx.x);
}

__global__ void k_half_sum(const double* __restrict__ partials, int count, double* __restrict__ out) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int q = 0; q < count; ++q) s += partials[q];
  *out = 0.5 * s;
}

void misfit_launch(Ctx& c, const double* u, const double* d, double* grad, double* out, cudaStream_t st) {
  k_misfit_partials<<<c.gs_grid, BS, 0, st>>>(c.n, view<double>(c.Ms), u, d, grad, c.partials);
  k_half_sum<<<1, 32, 0, st>>>(c.partials, c.gs_grid, out);
  CK_LAUNCH();
}

void residual_norm_launch(Ctx& c, const double* k, const double* b, double* partials, int grid, double* out,
                          cudaStream_t st) {
  IRK_DISPATCH_S(c.s, {
    k_resid_partials<S><<<grid, BS, 0, st>>>(c.n, view<double>(c.Ms), c.Fs.v64, k, b, c.K, partials);
  });
  k_sum_partials<<<1, 32, 0, st>>>(partials, grid, out);
  CK_LAUNCH();
}

// w = A z_0 with the same kernel, buffers and launch shape as the loop
void profile_kron_launch(Ctx& c, cudaStream_t st) {
  int n = c.n;
  int64_t N = c.N;
  unsigned G = row_grid(c);
  bool z32 = c.amg.amg_prec != 64;
  IRK_DISPATCH_S(c.s, {
    if (z32 && c.MFs)
      launch_k(k_kron_ff<S>, ff_grid(c), BS, 0, st, n, view<double>(c.Ms), static_cast<const float4*>(c.MFs),
                                      JPtr<const float>{static_cast<const float*>(c.Z), nullptr, N, 0, 0},
                                      JPtr<double>{c.V, nullptr, N, 1, 0}, c.Kf, nullptr);
    else if (z32)
      launch_k(k_kron<S, float, 0>, G, BS, 0, st, n, view<double>(c.Ms), c.Fs.v64,
                                            JPtr<const float>{static_cast<const float*>(c.Z), nullptr, N, 0, 0},
                                            JPtr<double>{c.V, nullptr, N, 1, 0}, c.K, nullptr, nullptr, nullptr);
    else
      launch_k(k_kron<S, double, 0>, G, BS, 0, st, n, view<double>(c.Ms), c.Fs.v64,
                                             JPtr<const double>{static_cast<const double*>(c.Z), nullptr, N, 0, 0},
                                             JPtr<double>{c.V, nullptr, N, 1, 0}, c.K, nullptr, nullptr, nullptr);
  });
  CK_LAUNCH();
}

// one Gram-Schmidt pass on a scratch state (axpy: also the Givens update)
void profile_gs_launch(Ctx& c, GmresState* scratch, bool axpy, cudaStream_t st) {
  unsigned G = row_grid(c);
  if (axpy) launch_k(k_gs_axpy<0>, G, BS, 0, st, scratch, c.V, c.N, c.N, c.partials);
  else launch_k(k_gs_dots<0>, G, BS, 0, st, scratch, c.V, c.N, c.N, c.partials);
  CK_LAUNCH();
}

void set_loop_condition_launch(Ctx& c, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_loop_ctrl<<<1, 32, 0, st>>>(c.st, h);
  CK_LAUNCH();
}

// the second-pass test of the Gram-Schmidt kernels: eta^2, or -1 for "always"
static double reorth_eta2(const Ctx& c) { return c.reorth == 1 ? -1.0 : c.reorth_eta * c.reorth_eta; }

void rhs_forward_launch(Ctx& c, const double* u, cudaStream_t st) {
  IRK_DISPATCH_S(c.s, {
    launch_k(k_rhs_forward<S>, row_grid(c), BS, 0, st, c.n, view<double>(c.Fs), u, c.g, c.bv, c.V, c.x, c.st, c.partials,
                                                 c.m, c.max_it, c.rtol, reorth_eta2(c), c.rhs_given);
  });
  CK_LAUNCH();
}

void rhs_adjoint_launch(Ctx& c, const double* lam, cudaStream_t st) {
  KronCoef hb;
  for (int i = 0; i < MAX_S * MAX_S; ++i) hb.a[i] = 0.0;
  for (int i = 0; i < c.s; ++i) hb.a[i] = c.h * c.b[i];
  IRK_DISPATCH_S(c.s, {
    launch_k(k_rhs_adjoint<S>, row_grid(c), BS, 0, st, c.n, hb, lam, c.bv, c.V, c.x, c.st, c.partials, c.m, c.max_it,
                                                 c.rtol, reorth_eta2(c));
  });
  CK_LAUNCH();
}

void stage_update_launch(Ctx& c, double* u, cudaStream_t st) {
  KronCoef hb;
  for (int i = 0; i < MAX_S * MAX_S; ++i) hb.a[i] = 0.0;
  for (int i = 0; i < c.s; ++i) hb.a[i] = c.h * c.b[i];
  IRK_DISPATCH_S(c.s, { launch_k(k_stage_update<S>, row_grid(c), BS, 0, st, c.n, hb, c.x, u); });
  CK_LAUNCH();
}

void record_launch(Ctx& c, cudaStream_t st) {
  k_record<<<1, 32, 0, st>>>(c.st, c.rec, c.step_counter, c.rec_cap);
  CK_LAUNCH();
}

void kron_apply_plain(Ctx& c, const double* z, double* w, bool transpose, cudaStream_t st) {
  const KronCoef& K = transpose ? c.KT : c.K;
  IRK_DISPATCH_S(c.s, {
    launch_k(k_kron<S, double, 0>, row_grid(c), BS, 0, st, c.n, view<double>(c.Ms), c.Fs.v64,
                                                     JPtr<const double>{z, nullptr, 0, 0, 0},
                                                     JPtr<double>{w, nullptr, 0, 0, 0}, K, nullptr, nullptr, nullptr);
  });
  CK_LAUNCH();
}

// single-float pair operator on (IRK_KRON_FF=0: FP64 products on widened z)
static bool kron_ff_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("IRK_KRON_FF");
    on = (e && std::atoi(e) == 0) ? 0 : 1;
  }
  return on == 1;
}

static bool split_coef(const KronCoef& K, KronCoefF& F) {
  bool ok = true;
  for (int i = 0; i < MAX_S * MAX_S; ++i) {
    const double a = K.a[i];
    F.hi[i] = static_cast<float>(a);
    F.lo[i] = static_cast<float>(a - static_cast<double>(F.hi[i]));
    if (a != 0.0 && !(std::fabs(a) <= 0x1p64 && std::fabs(a) >= 0x1p-64)) ok = false;
  }
  return ok;
}

void kron_split_build(Ctx& c) {
  if (c.MFs) {
    c.pool.release(c.MFs);
    c.MFs = nullptr;
  }
  bool ok = split_coef(c.K, c.Kf);
  ok = split_coef(c.KT, c.KTf) && ok;
  const int64_t np = c.Ms.nnz_pad;
  if (!ok || !kron_ff_enabled() || c.amg.amg_prec == 64 || np <= 0 || !c.Ms.v64 || !c.Fs.v64) return;
  float4* mf = c.pool.get<float4>(np);
  Tmp tmp;
  int* bad = tmp.get<int>(1);
  CK(cudaMemsetAsync(bad, 0, sizeof(int), c.stream));
  k_split_ff<<<static_cast<unsigned>((np + 255) / 256), 256, 0, c.stream>>>(np, c.Ms.v64, c.Fs.v64, mf, bad);
  CK_LAUNCH();
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, bad, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  if (flag) c.pool.release(mf);
  else c.MFs = mf;
}

void kron_apply_f32(Ctx& c, const float* z, double* w, bool transpose, cudaStream_t st) {
  IRK_DISPATCH_S(c.s, {
    if (c.MFs)
      launch_k(k_kron_ff<S>, ff_grid(c), BS, 0, st, c.n, view<double>(c.Ms), static_cast<const float4*>(c.MFs),
                                        JPtr<const float>{z, nullptr, 0, 0, 0}, JPtr<double>{w, nullptr, 0, 0, 0},
                                        transpose ? c.KTf : c.Kf, nullptr);
    else
      launch_k(k_kron<S, float, 0>, row_grid(c), BS, 0, st, c.n, view<double>(c.Ms), c.Fs.v64,
                                              JPtr<const float>{z, nullptr, 0, 0, 0}, JPtr<double>{w, nullptr, 0, 0, 0},
                                              transpose ? c.KT : c.K, nullptr, nullptr, nullptr);
  });
  CK_LAUNCH();
}

void mass_apply_launch(Ctx& c, const double* x, double* y, cudaStream_t st) {
  k_spmv64<<<row_grid(c), BS, 0, st>>>(c.n, view<double>(c.Ms), x, y);
  CK_LAUNCH();
}

void adjoint_lambda_launch(Ctx& c, const double* lam_in, double* lam_out, cudaStream_t st) {
  IRK_DISPATCH_S(c.s, { launch_k(k_adj_lambda<S>, row_grid(c), BS, 0, st, c.n, view<double>(c.Fs), c.x, lam_in, lam_out); });
  CK_LAUNCH();
}

void adjoint_grad_launch(Ctx& c, const double* u_n, const double* k_n, double* grad, cudaStream_t st) {
  adjoint_grad_launch_at(c, u_n, k_n, nullptr, grad, st);
}

// u_n and k_n at u_base + (*step) n and k_base + (*step) s n (step == nullptr: offset 0)
void adjoint_grad_launch_at(Ctx& c, const double* u_base, const double* k_base, const int* step, double* grad,
                            cudaStream_t st) {
  JPtr<const double> up{u_base, step, int64_t(c.n), 0, 0};
  JPtr<const double> kp{k_base, step, c.N, 0, 0};
  IRK_DISPATCH_S(c.s, {
    k_adj_grad<S><<<row_grid(c), BS, 0, st>>>(c.n_tri, c.tri, c.dof, c.Ke, c.K, c.n, up, kp, c.x, grad);
  });
  CK_LAUNCH();
}

void assemble_kappa_launch(Ctx& c, const double* kappa, double* Fval, cudaStream_t st) {
  k_assemble_kappa<<<row_grid(c), BS, 0, st>>>(c.Fc.nnz, c.asm_ptr, c.asm_src, c.Ke, kappa, Fval);
  CK_LAUNCH();
}

void convert_launch(const void* in, int in_prec, void* out, int out_prec, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_convert<<<nblk(n), 256, 0, st>>>(in, in_prec, out, out_prec, n);
  CK_LAUNCH();
}

}  // namespace irk

namespace irk {

int left_head_launch(Ctx& c, cudaStream_t st) {
  // P^{-1} (sigma_0 V_0) = P^{-1} b / ||b|| into Z, then V_0 and the norms
  PrecondArgs pa{c.V, &c.st->j, c.N, c.st->sigma, c.Z, 0, &c.st->done};
  int launches = precond_launch(c, pa, false, st);
  unsigned G = static_cast<unsigned>(c.gs_grid);
  if (c.amg.amg_prec == 64)
    launch_k(k_left_start<double>, G, BS, 0, st, c.st, static_cast<const double*>(c.Z), c.V, c.N, c.partials);
  else
    launch_k(k_left_start<float>, G, BS, 0, st, c.st, static_cast<const float*>(c.Z), c.V, c.N, c.partials);
  CK_LAUNCH();
  return launches + 1;
}

int left_body_launch(Ctx& c, cudaStream_t st) {
  int n = c.n;
  int64_t N = c.N;
  unsigned G = static_cast<unsigned>(c.gs_grid);
  const int* jp = &c.st->j;
  int launches = 0;
  // T = A V_j
  IRK_DISPATCH_S(c.s, {
    launch_k(k_kron<S, double, 0>, G, BS, 0, st, n, view<double>(c.Ms), c.Fs.v64,
             JPtr<const double>{c.V, jp, N, 0, 0}, JPtr<double>{c.T, nullptr, 0, 0, 0}, c.K, nullptr, c.st,
             c.partials);
  });
  ++launches;
  // Z = P^{-1} T; V_{j+1} = sigma_j Z
  PrecondArgs pa{c.T, nullptr, 0, nullptr, c.Z, 0, &c.st->done};
  launches += precond_launch(c, pa, false, st);
  if (c.amg.amg_prec == 64)
    launch_k(k_left_widen<double>, G, BS, 0, st, c.st, static_cast<const double*>(c.Z), c.V, N, N);
  else
    launch_k(k_left_widen<float>, G, BS, 0, st, c.st, static_cast<const float*>(c.Z), c.V, N, N);
  ++launches;
  launch_k(k_gs_dots<0>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launch_k(k_gs_axpy<0>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launch_k(k_gs_dots<1>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launch_k(k_gs_axpy<1>, G, BS, 0, st, c.st, c.V, N, N, c.partials);
  launches += 4;
  launch_k(k_left_xupdate, G, BS, 0, st, c.st, c.V, N, c.x, N);
  launch_k(k_left_decide, 1, 32, 0, st, c.st);
  launch_k(k_left_residual, G, BS, 0, st, c.st, c.V, N, c.T, N, c.partials);
  launch_k(k_left_restart, G, BS, 0, st, c.st, c.T, c.V, N);
  launches += 4;
  CK_LAUNCH();
  return launches;
}

int left_tail_launch(Ctx& c, cudaStream_t st) {
  int grid = c.gs_grid;
  IRK_DISPATCH_S(c.s, {
    k_resid_partials<S><<<grid, BS, 0, st>>>(c.n, view<double>(c.Ms), c.Fs.v64, c.x, c.bv, c.K, c.partials);
  });
  k_left_final_resid<<<1, 32, 0, st>>>(c.st, c.partials, grid);
  CK_LAUNCH();
  return 2;
}

}  // namespace irk
