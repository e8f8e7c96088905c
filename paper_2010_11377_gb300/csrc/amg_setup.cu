// Smoothed-aggregation AMG setup on the GPU, for the diagonal-block subsolves
// (M + h A~_jj F) w_j = v_j of Section 4.2 (one V-cycle each; the paper uses
// IFISS smoothed aggregation and fixes no further parameter).
//
// Per level:
//   strength   (c_ij + c_ji)/2 >= theta_l sqrt(|a_ii a_jj|), c_ij = |a_ij| (option: max(-a_ij, 0))
//              (or |a_ij|), a symmetric graph;
//              theta_l = theta, halved (at most 6 times) while more than a
//              quarter of the level's nodes have no strong coupling
//   roots      maximal distance-2 independent set chosen by fixed 64-bit
//              priorities (fmix32 hash of the index, salted by the level):
//              in each round an undecided node becomes a root when its key is
//              the largest among undecided nodes within distance 2, and a node
//              within distance 2 of a root drops out.  With fixed priorities
//              this yields exactly the set of the sequential greedy pass in
//              decreasing priority.
//   aggregates root + strong neighbours; every other node joins the
//              aggregate of its phase-1 strong neighbour of largest priority;
//              aggregates numbered by increasing root index
//   P          (I - omega D^{-1} A)^p P_tent (p = p_smooth on every level),
//              omega = 4/(3 rho), rho the estimate of rho(D^{-1} A) by 20 steps
//              of the power iteration on S = |D|^{-1/2} A |D|^{-1/2} from the
//              +-1 vector x_i = +1 iff fmix32(i ^ 0x68E31DA4) is odd:
//              x <- S x / ||x||, rho = ||S x_19|| / ||x_19|| (deterministic
//              block-tree reductions)
//   coarse     A_c = P^T A P by two deterministic SpGEMMs, until n <= coarse_max (2048)
//              or coarsening stalls (a level would keep > 90% of its rows);
//              the coarsest level is inverted densely (Gauss-Jordan, partial
//              pivoting, FP64).
#include "irk_internal.cuh"

#include <cmath>
#include <cstring>
#include <cstdio>

namespace irk {

__device__ __forceinline__ unsigned fmix32(unsigned x) {
  // MurmurHash3 32-bit finaliser
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ unsigned long long prio_key(int i, int level) {
  unsigned salt = 0x9E3779B9u * static_cast<unsigned>(level + 1);
  unsigned h = fmix32(static_cast<unsigned>(i) ^ salt);
  return (static_cast<unsigned long long>(h) << 32) | static_cast<unsigned>(i);
}

__device__ __forceinline__ double find_entry(const int* __restrict__ rp, const int* __restrict__ col,
                                             const double* __restrict__ val, int r, int c) {
  int lo = rp[r], hi = rp[r + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int cm = col[mid];
    if (cm == c) return val[mid];
    if (cm < c) lo = mid + 1;
    else hi = mid - 1;
  }
  return 0.0;
}

__global__ void k_diag(int n, const int* __restrict__ rp, const int* __restrict__ col,
                       const double* __restrict__ val, double* __restrict__ diag, double* __restrict__ dsq,
                       int* __restrict__ bad) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double d = 0.0;
  for (int k = rp[r]; k < rp[r + 1]; ++k)
    if (col[k] == r) d = val[k];
  diag[r] = d;
  dsq[r] = sqrt(fabs(d));
  if (d == 0.0) atomicExch(bad, 1);
}

// ---------------------------------------------------------------------------
// Power iteration for rho(D^{-1} A) on S = |D|^{-1/2} A |D|^{-1/2}
// ---------------------------------------------------------------------------
constexpr unsigned POWER_SALT = 0x68E31DA4u;
constexpr int POWER_STEPS = 20;
constexpr int POWER_BS = 256;

__global__ void k_power_init(int n, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (fmix32(static_cast<unsigned>(i) ^ POWER_SALT) & 1u) ? 1.0 : -1.0;
}

// y = S (x * scale), scale = 1/||x||; per-block partial sums of y_i^2 (fixed tree)
__global__ void __launch_bounds__(POWER_BS)
k_power_step(int n, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
             const double* __restrict__ dsq, const double* __restrict__ x, const double* __restrict__ scale,
             double* __restrict__ y, double* __restrict__ partials) {
  __shared__ double sh[POWER_BS];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  double yr = 0.0;
  if (r < n) {
    const double sc = *scale;
    double acc = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      int c = col[k];
      acc = fma(val[k], (x[c] * sc) / dsq[c], acc);
    }
    yr = acc / dsq[r];
    y[r] = yr;
  }
  sh[threadIdx.x] = yr * yr;
  __syncthreads();
  for (int o = POWER_BS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// one block: the norm from the partials in a fixed order; scale = 1/norm
__global__ void __launch_bounds__(1024)
k_power_norm(int nparts, const double* __restrict__ partials, double* __restrict__ norm,
             double* __restrict__ scale) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double nv = sqrt(sh[0]);
    *norm = nv;
    *scale = nv > 0.0 ? 1.0 / nv : 0.0;
  }
}

// strength flags per entry and strong count per row
__global__ void k_strength(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ diag,
                           double theta, int negative, unsigned char* __restrict__ strong,
                           int* __restrict__ cnt, int* __restrict__ niso) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int c0 = 0;
  double dr = fabs(diag[r]);
  for (int k = rp[r]; k < rp[r + 1]; ++k) {
    int c = col[k];
    unsigned char s = 0;
    if (c != r) {
      double aji = find_entry(rp, col, val, c, r);
      double cij = negative ? fmax(-val[k], 0.0) : fabs(val[k]);
      double cji = negative ? fmax(-aji, 0.0) : fabs(aji);
      double sij = (cij + cji) * 0.5;
      double thr = theta * sqrt(dr * fabs(diag[c]));
      s = (sij >= thr) ? 1 : 0;
    }
    strong[k] = s;
    c0 += s;
  }
  cnt[r] = c0;
  if (c0 == 0) atomicAdd(niso, 1);
}

__global__ void k_strength_fill(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const unsigned char* __restrict__ strong, const int* __restrict__ grp,
                                int* __restrict__ gcol) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int o = grp[r];
  for (int k = rp[r]; k < rp[r + 1]; ++k)
    if (strong[k]) gcol[o++] = col[k];
}

enum : unsigned char { UND = 0, ROOT = 1, OUTN = 2 };

// m1[i] = max key over undecided nodes of {i} u N(i); r1[i] = a root in {i} u N(i)
__global__ void k_mis_hop1(int n, int level, const int* __restrict__ grp, const int* __restrict__ gcol,
                           const unsigned char* __restrict__ state, unsigned long long* __restrict__ m1,
                           unsigned char* __restrict__ r1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = 0;
  unsigned char rr = 0;
  unsigned char si = state[i];
  if (si == UND) m = prio_key(i, level);
  if (si == ROOT) rr = 1;
  for (int k = grp[i]; k < grp[i + 1]; ++k) {
    int u = gcol[k];
    unsigned char su = state[u];
    if (su == UND) {
      unsigned long long ku = prio_key(u, level);
      m = ku > m ? ku : m;
    } else if (su == ROOT) {
      rr = 1;
    }
  }
  m1[i] = m;
  r1[i] = rr;
}

__global__ void k_mis_hop2(int n, int level, const int* __restrict__ grp, const int* __restrict__ gcol,
                           const unsigned char* __restrict__ state, const unsigned long long* __restrict__ m1,
                           const unsigned char* __restrict__ r1, unsigned char* __restrict__ nstate,
                           int* __restrict__ und_count) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  unsigned char sv = state[v];
  if (sv != UND) {
    nstate[v] = sv;
    return;
  }
  unsigned long long m = m1[v];
  unsigned char rr = r1[v];
  for (int k = grp[v]; k < grp[v + 1]; ++k) {
    int u = gcol[k];
    unsigned long long mu = m1[u];
    m = mu > m ? mu : m;
    rr |= r1[u];
  }
  unsigned char ns;
  if (rr) ns = OUTN;
  else if (m == prio_key(v, level)) ns = ROOT;
  else ns = UND;
  nstate[v] = ns;
  if (ns == UND) atomicAdd(und_count, 1);
}

__global__ void k_root_flag(int n, const unsigned char* __restrict__ state, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == ROOT ? 1 : 0;
}

__global__ void k_agg_phase1(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                             const unsigned char* __restrict__ state, const int* __restrict__ rootid,
                             int* __restrict__ agg1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = -1;
  if (state[i] == ROOT) {
    a = rootid[i];
  } else {
    for (int k = grp[i]; k < grp[i + 1]; ++k) {
      int u = gcol[k];
      if (state[u] == ROOT) {
        a = rootid[u];
        break;
      }
    }
  }
  agg1[i] = a;
}

__global__ void k_agg_phase2(int n, int level, const int* __restrict__ grp, const int* __restrict__ gcol,
                             const int* __restrict__ agg1, int* __restrict__ agg, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg1[i];
  if (a < 0) {
    unsigned long long best = 0;
    for (int k = grp[i]; k < grp[i + 1]; ++k) {
      int u = gcol[k];
      int au = agg1[u];
      if (au >= 0) {
        unsigned long long ku = prio_key(u, level);
        if (a < 0 || ku > best) {
          best = ku;
          a = au;
        }
      }
    }
    if (a < 0) atomicExch(bad, 1);
  }
  agg[i] = a;
}

// P row r: entries over aggregates J of the row's columns,
// P[r,J] = delta(agg(r)==J) - omega * ((1/a_rr) * sum_{c in row, agg(c)=J} a_rc)
// summed in increasing column order.  Row length is at most the row of A.
__global__ void k_prolong_count(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const int* __restrict__ agg, int* __restrict__ cnt) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int u = 0;
  for (int k = rp[r]; k < rp[r + 1]; ++k) {
    int J = agg[col[k]];
    bool seen = false;
    for (int q = rp[r]; q < k; ++q)
      if (agg[col[q]] == J) {
        seen = true;
        break;
      }
    if (!seen) ++u;
  }
  cnt[r] = u;
}

__global__ void k_prolong_fill(int n, const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ val, const double* __restrict__ diag,
                               const int* __restrict__ agg, double omega, const int* __restrict__ prp,
                               int* __restrict__ pcol, double* __restrict__ pval) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int o = prp[r];
  int u = prp[r + 1] - o;
  // distinct aggregates in increasing order
  int cnt = 0;
  int last = -1;
  for (int q = 0; q < u; ++q) {
    int best = 0x7fffffff;
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      int J = agg[col[k]];
      if (J > last && J < best) best = J;
    }
    pcol[o + cnt] = best;
    double t = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k)
      if (agg[col[k]] == best) t = __dadd_rn(t, val[k]);
    double sc = __dmul_rn(omega, __dmul_rn(1.0 / diag[r], t));
    double p = (best == agg[r]) ? __dadd_rn(1.0, -sc) : -sc;
    pval[o + cnt] = p;
    ++cnt;
    last = best;
  }
}

__global__ void k_l1_inverse(int n, const int* __restrict__ rp, const double* __restrict__ val,
                             double* __restrict__ d64, float* __restrict__ d32) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int k = rp[r]; k < rp[r + 1]; ++k) s += fabs(val[k]);
  double inv = 1.0 / s;
  if (d64) d64[r] = inv;
  if (d32) d32[r] = static_cast<float>(inv);
}

// dense Gauss-Jordan with partial pivoting on [A | I] (n <= MAX_COARSE), one
// launch per pivot column; the augmented matrix is row-major n x 2n
__global__ void k_dense_from_csr(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ aug) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double* row = aug + size_t(r) * 2 * n;
  for (int c = 0; c < 2 * n; ++c) row[c] = (c == n + r) ? 1.0 : 0.0;
  for (int k = rp[r]; k < rp[r + 1]; ++k) row[col[k]] = val[k];
}

__global__ void k_gj_pivot(int n, int k, double* __restrict__ aug, int* __restrict__ bad) {
  // single block: find pivot row, swap, scale
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int bidx = -1;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(aug[size_t(i) * 2 * n + k]);
    if (v > best || (v == best && i < bidx)) {
      best = v;
      bidx = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = bv[threadIdx.x + s];
      int oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi >= 0 && (bi[threadIdx.x] < 0 || oi < bi[threadIdx.x]))) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  int p = bi[0];
  if (p < 0 || bv[0] == 0.0) {
    if (threadIdx.x == 0) atomicExch(bad, 1);
    return;
  }
  double* rk = aug + size_t(k) * 2 * n;
  double* rp_ = aug + size_t(p) * 2 * n;
  if (p != k) {
    for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) {
      double t = rk[c];
      rk[c] = rp_[c];
      rp_[c] = t;
    }
  }
  __syncthreads();
  double piv = rk[k];
  __syncthreads();
  for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) rk[c] /= piv;
}

__global__ void k_gj_eliminate(int n, int k, double* __restrict__ aug) {
  int i = blockIdx.y;
  if (i == k) return;
  double* ri = aug + size_t(i) * 2 * n;
  const double* rk = aug + size_t(k) * 2 * n;
  double f = ri[k];
  if (f == 0.0) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * n; c += gridDim.x * blockDim.x)
    if (c != k) ri[c] -= f * rk[c];
  // column k itself is cleared after all other columns used f
}

__global__ void k_gj_clear(int n, int k, double* __restrict__ aug) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && i != k) aug[size_t(i) * 2 * n + k] = 0.0;
}

__global__ void k_gj_extract(int n, const double* __restrict__ aug, double* __restrict__ inv64,
                             float* __restrict__ inv32) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  int r = t / n, c = t % n;
  double v = aug[size_t(r) * 2 * n + n + c];
  if (inv64) inv64[t] = v;
  if (inv32) inv32[t] = static_cast<float>(v);
}

template <typename T>
static T rd(const T* d, cudaStream_t st) {
  T h;
  CK(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

static inline unsigned nb(int64_t n, int bs = 256) { return nblk(n, bs); }

// one coarsening step: fills lev.agg, lev.P (as CSR) and the coarse CSR Ac
// One more damped-Jacobi step on the prolongator, on the pattern of A P:
// out[r,J] = P[r,J] - omega ((1/a_rr) (A P)[r,J])  (P[r,J] = 0 off its pattern).
// The pattern of A P contains that of P (A has its diagonal); a P entry
// missing from it sets *bad.
__global__ void k_psmooth_merge(int n, const int* __restrict__ prp, const int* __restrict__ pcol,
                                const double* __restrict__ pval, const int* __restrict__ arp,
                                const int* __restrict__ acol, const double* __restrict__ aval,
                                const double* __restrict__ diag, double omega, double* __restrict__ out,
                                int* __restrict__ bad) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int q = prp[r];
  const int qe = prp[r + 1];
  const double dinv = 1.0 / diag[r];
  for (int k = arp[r]; k < arp[r + 1]; ++k) {
    double pv = 0.0;
    if (q < qe && pcol[q] == acol[k]) pv = pval[q++];
    else if (q < qe && pcol[q] < acol[k]) atomicOr(bad, 1);
    out[k] = __dsub_rn(pv, __dmul_rn(omega, __dmul_rn(dinv, aval[k])));
  }
  if (q != qe) atomicOr(bad, 1);
}

// rho(D^{-1} A) estimated by POWER_STEPS normalised power steps on S (see the
// file header); dsq = sqrt(|diag A|)
static double spectral_radius_estimate(const CsrD& A, const double* dsq, cudaStream_t st) {
  const int n = A.n;
  Tmp tmp;
  double* x = tmp.get<double>(n);
  double* y = tmp.get<double>(n);
  const unsigned nbk = nb(n, POWER_BS);
  double* partials = tmp.get<double>(nbk);
  double* norm = tmp.get<double>(1);
  double* scale = tmp.get<double>(1);
  k_power_init<<<nb(n), 256, 0, st>>>(n, x);
  const double s0 = 1.0 / std::sqrt(static_cast<double>(n));   // ||x_0|| = sqrt(n)
  CK(cudaMemcpyAsync(scale, &s0, sizeof(double), cudaMemcpyHostToDevice, st));
  for (int k = 0; k < POWER_STEPS; ++k) {
    k_power_step<<<nbk, POWER_BS, 0, st>>>(n, A.rowptr, A.col, A.val, dsq, x, scale, y, partials);
    k_power_norm<<<1, 1024, 0, st>>>(static_cast<int>(nbk), partials, norm, scale);
    std::swap(x, y);
  }
  CK_LAUNCH();
  return rd(norm, st);
}

static bool coarsen(Level& lev, int level, const AmgParams& p, CsrD& P, CsrD& R, CsrD& Ac, DevPool& pool,
                    cudaStream_t st) {
  const CsrD& A = lev.A;
  int n = A.n;
  Tmp tmp;
  double* diag = tmp.get<double>(n);
  double* dsq = tmp.get<double>(n);
  int* bad = tmp.get<int>(1);
  CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_diag<<<nb(n), 256, 0, st>>>(n, A.rowptr, A.col, A.val, diag, dsq, bad);
  CK_LAUNCH();
  if (rd(bad, st)) fail(IRK_ERR_ZERO_PIVOT, "AMG level matrix has a zero diagonal entry");
  const double rho = spectral_radius_estimate(A, dsq, st);
  if (!(rho > 0.0) || !std::isfinite(rho)) fail(IRK_ERR_NONFINITE, "AMG spectral radius estimate is not positive");
  double omega = 4.0 / (3.0 * rho);

  // strength graph (threshold halved while more than n/4 nodes are isolated)
  unsigned char* strong = tmp.get<unsigned char>(A.nnz > 0 ? A.nnz : 1);
  int* scnt = tmp.get<int>(n + 1);
  int* niso = tmp.get<int>(1);
  double theta_l = p.theta;
  for (int halving = 0;; ++halving) {
    CK(cudaMemsetAsync(niso, 0, sizeof(int), st));
    k_strength<<<nb(n), 256, 0, st>>>(n, A.rowptr, A.col, A.val, diag, theta_l, p.strength_negative, strong, scnt,
                                      niso);
    CK_LAUNCH();
    if (halving == 6 || 4 * int64_t(rd(niso, st)) <= int64_t(n)) break;
    theta_l *= 0.5;
  }
  int* grp = tmp.get<int>(n + 1);
  scan_exclusive(scnt, grp, n, st);
  int gnnz = rd(grp + n, st);
  int* gcol = tmp.get<int>(gnnz > 0 ? gnnz : 1);
  k_strength_fill<<<nb(n), 256, 0, st>>>(n, A.rowptr, A.col, strong, grp, gcol);
  CK_LAUNCH();

  // distance-2 independent set by fixed-priority rounds
  unsigned char* state = tmp.get<unsigned char>(n);
  unsigned char* nstate = tmp.get<unsigned char>(n);
  unsigned long long* m1 = tmp.get<unsigned long long>(n);
  unsigned char* r1 = tmp.get<unsigned char>(n);
  int* und = tmp.get<int>(1);
  CK(cudaMemsetAsync(state, UND, n, st));
  for (int round = 0;; ++round) {
    if (round > n + 2) fail(IRK_ERR_CUDA, "independent-set rounds did not terminate");
    CK(cudaMemsetAsync(und, 0, sizeof(int), st));
    k_mis_hop1<<<nb(n), 256, 0, st>>>(n, level, grp, gcol, state, m1, r1);
    CK_LAUNCH();
    k_mis_hop2<<<nb(n), 256, 0, st>>>(n, level, grp, gcol, state, m1, r1, nstate, und);
    CK_LAUNCH();
    std::swap(state, nstate);
    if (rd(und, st) == 0) break;
  }
  int* flag = tmp.get<int>(n + 1);
  int* rootid = tmp.get<int>(n + 1);
  k_root_flag<<<nb(n), 256, 0, st>>>(n, state, flag);
  CK_LAUNCH();
  scan_exclusive(flag, rootid, n, st);
  int nc = rd(rootid + n, st);
  // stop when coarsening stalls: the next level would keep more than 90% of the rows
  if (nc == 0 || 10 * int64_t(nc) > 9 * int64_t(n)) return false;

  int* agg1 = tmp.get<int>(n);
  lev.agg = pool.get<int>(n);
  k_agg_phase1<<<nb(n), 256, 0, st>>>(n, grp, gcol, state, rootid, agg1);
  CK_LAUNCH();
  CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_agg_phase2<<<nb(n), 256, 0, st>>>(n, level, grp, gcol, agg1, lev.agg, bad);
  CK_LAUNCH();
  if (rd(bad, st)) fail(IRK_ERR_CUDA, "aggregation left a node without an aggregate");

  // smoothed prolongator
  int* pcnt = tmp.get<int>(n + 1);
  k_prolong_count<<<nb(n), 256, 0, st>>>(n, A.rowptr, A.col, lev.agg, pcnt);
  CK_LAUNCH();
  P.n = n;
  P.ncols = nc;
  P.rowptr = pool.get<int>(n + 1);
  scan_exclusive(pcnt, P.rowptr, n, st);
  P.nnz = rd(P.rowptr + n, st);
  P.col = pool.get<int>(P.nnz);
  P.val = pool.get<double>(P.nnz);
  k_prolong_fill<<<nb(n), 256, 0, st>>>(n, A.rowptr, A.col, A.val, diag, lev.agg, omega, P.rowptr, P.col,
                                        P.val);
  // further Jacobi steps: P <- P - omega D^{-1} (A P)
  const int steps = p.p_smooth;
  for (int q = 1; q < steps; ++q) {
    CK_LAUNCH();
    CsrD AP1;
    csr_spgemm(A, P, AP1, pool, st);
    double* v2 = pool.get<double>(AP1.nnz > 0 ? AP1.nnz : 1);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_psmooth_merge<<<nb(n), 256, 0, st>>>(n, P.rowptr, P.col, P.val, AP1.rowptr, AP1.col, AP1.val, diag, omega,
                                           v2, bad);
    CK_LAUNCH();
    if (rd(bad, st)) fail(IRK_ERR_INVALID, "prolongator pattern not contained in that of A P");
    pool.release(P.rowptr);
    pool.release(P.col);
    pool.release(P.val);
    pool.release(AP1.val);
    P.rowptr = AP1.rowptr;
    P.col = AP1.col;
    P.val = v2;
    P.nnz = AP1.nnz;
  }
  CK_LAUNCH();
  csr_transpose(P, R, pool, st);
  CsrD AP;
  csr_spgemm(A, P, AP, pool, st);
  csr_spgemm(R, AP, Ac, pool, st);
  pool.release(AP.rowptr);
  pool.release(AP.col);
  pool.release(AP.val);
  return true;
}

// A += coef * T where the pattern of T lies inside that of A (both rows sorted);
// an entry of T missing from A sets *bad
__global__ void k_csr_add_subpattern(int n, const int* __restrict__ arp, const int* __restrict__ acol,
                                     double* __restrict__ aval, const int* __restrict__ trp,
                                     const int* __restrict__ tcol, const double* __restrict__ tval, double coef,
                                     int* __restrict__ bad) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int k = arp[r];
  const int ke = arp[r + 1];
  for (int q = trp[r]; q < trp[r + 1]; ++q) {
    const int c = tcol[q];
    while (k < ke && acol[k] < c) ++k;
    if (k == ke || acol[k] != c) {
      atomicOr(bad, 1);
      return;
    }
    aval[k] = __dadd_rn(aval[k], __dmul_rn(coef, tval[q]));
  }
}

static void alloc_level_vectors(Level& L, int prec, DevPool& pool) {
  size_t es = (prec == 64) ? sizeof(double) : sizeof(float);
  size_t n = L.n > 0 ? L.n : 1;
  L.b = pool.alloc(es * n);
  L.x = pool.alloc(es * n);
  L.y = pool.alloc(es * n);
  L.r = pool.alloc(es * n);
  L.d = pool.alloc(es * n);
}

void amg_build(Hier& H, const CsrD& A0, const AmgParams& p, DevPool& pool, cudaStream_t st, const CsrD* T0,
               double c_stab) {
  H.amg_prec = p.amg_prec;
  H.lv.clear();
  H.lv.emplace_back();
  H.lv[0].A = A0;
  H.lv[0].n = A0.n;
  H.lv[0].nnz = A0.nnz;
  int maxl = p.max_levels < MAX_LEVELS ? p.max_levels : MAX_LEVELS;
  int coarse_max = p.coarse_max < MAX_COARSE ? p.coarse_max : MAX_COARSE;
  // coarse-level SUPG stabilisation: the projected streamline matrix of the
  // current level and the mesh-size factor f of the level above
  CsrD T = T0 ? *T0 : CsrD{};
  double f_prev = 1.0;
  while (true) {
    Level& lev = H.lv.back();
    int l = static_cast<int>(H.lv.size()) - 1;
    if (lev.n <= coarse_max || static_cast<int>(H.lv.size()) >= maxl) break;
    CsrD P, R, Ac;
    if (!coarsen(lev, l, p, P, R, Ac, pool, st)) break;
    if (T0) {
      CsrD TP, Tc;
      csr_spgemm(T, P, TP, pool, st);
      csr_spgemm(R, TP, Tc, pool, st);
      pool.release(TP.rowptr);
      pool.release(TP.col);
      pool.release(TP.val);
      const double f = std::sqrt(double(A0.n) / double(Ac.n));
      const double coef = c_stab * (f - f_prev);
      Tmp tmp;
      int* bad = tmp.get<int>(1);
      CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
      k_csr_add_subpattern<<<nb(Ac.n), 256, 0, st>>>(Ac.n, Ac.rowptr, Ac.col, Ac.val, Tc.rowptr, Tc.col, Tc.val,
                                                     coef, bad);
      CK_LAUNCH();
      if (rd(bad, st)) fail(IRK_ERR_INVALID, "streamline matrix pattern not inside the Galerkin pattern");
      f_prev = f;
      T = Tc;
    }
    int pprec = p.amg_prec == 64 ? 64 : 32;
    make_matT(P, lev.Pm, pprec, pool, st);
    make_matT(R, lev.Rm, pprec, pool, st);
    Level nl;
    nl.A = Ac;
    nl.n = Ac.n;
    nl.nnz = Ac.nnz;
    H.lv.push_back(nl);
  }
  Level& last = H.lv.back();
  // a coarsest level above coarse_max (stalled coarsening) is smoothed, not inverted
  H.coarse_smooth = last.n > coarse_max;
  // per-level SELL matrices, l1 inverse diagonals, work vectors
  for (size_t l = 0; l < H.lv.size(); ++l) {
    Level& L = H.lv[l];
    int aprec = p.amg_prec == 64 ? 64 : ((p.amg_prec == 16 && l == 0) ? 16 : 32);
    make_matT(L.A, L.Am, aprec, pool, st);
    if (p.amg_prec == 64) {
      L.dinv = pool.get<double>(L.n > 0 ? L.n : 1);
      k_l1_inverse<<<nb(L.n), 256, 0, st>>>(L.n, L.A.rowptr, L.A.val, static_cast<double*>(L.dinv), nullptr);
    } else {
      L.dinv = pool.get<float>(L.n > 0 ? L.n : 1);
      k_l1_inverse<<<nb(L.n), 256, 0, st>>>(L.n, L.A.rowptr, L.A.val, nullptr, static_cast<float*>(L.dinv));
    }
    CK_LAUNCH();
    alloc_level_vectors(L, p.amg_prec == 64 ? 64 : 32, pool);
  }
  // coarsest dense inverse
  int nL = last.n;
  H.nc_dense = H.coarse_smooth ? 0 : nL;
  if (!H.coarse_smooth) {
    Tmp tmp;
    double* aug = tmp.get<double>(size_t(nL) * 2 * nL + 1);
    int* bad = tmp.get<int>(1);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_dense_from_csr<<<nb(nL), 256, 0, st>>>(nL, last.A.rowptr, last.A.col, last.A.val, aug);
    CK_LAUNCH();
    for (int k = 0; k < nL; ++k) {
      k_gj_pivot<<<1, 1024, 0, st>>>(nL, k, aug, bad);
      dim3 g((2 * nL + 255) / 256, nL);
      k_gj_eliminate<<<g, 256, 0, st>>>(nL, k, aug);
      k_gj_clear<<<nb(nL), 256, 0, st>>>(nL, k, aug);
    }
    CK_LAUNCH();
    if (rd(bad, st)) fail(IRK_ERR_ZERO_PIVOT, "coarsest AMG matrix is singular");
    if (p.amg_prec == 64) {
      H.cinv = pool.get<double>(size_t(nL) * nL + 1);
      k_gj_extract<<<nb(nL * nL), 256, 0, st>>>(nL, aug, static_cast<double*>(H.cinv), nullptr);
    } else {
      H.cinv = pool.get<float>(size_t(nL) * nL + 1);
      k_gj_extract<<<nb(nL * nL), 256, 0, st>>>(nL, aug, nullptr, static_cast<float*>(H.cinv));
    }
    CK_LAUNCH();
    CK(cudaStreamSynchronize(st));
  }
}

}  // namespace irk
