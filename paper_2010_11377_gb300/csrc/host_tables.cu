// Host-side tables of the method (no device work):
//  * Butcher tables (Section 2, Table 1).  Radau IIA: collocation at the zeros
//    of P_s(2x-1) - P_{s-1}(2x-1); Lobatto IIIC: Lobatto nodes, first column
//    equal to b_1 and the simplifying conditions C(s-1).  Nodes are found by
//    bracketing sign changes and bisection in long double; integrals of the
//    Lagrange basis by Gauss-Legendre quadrature (exact for degree s-1).
//  * A = L D U without pivoting (Section 4.1).
//  * the preconditioner coefficient matrices A~ of Eq. PrecForm, including the
//    optimised lower-triangular A~ of Eq. GSLopt, found here by Nelder-Mead
//    (adaptive coefficients of Gao and Han, 2012) on kappa_2(A~^{-1} A).
#include "irk_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

using ld = long double;

ld legendre(int k, ld x) {
  if (k == 0) return 1.0L;
  ld p0 = 1.0L, p1 = x;
  for (int q = 2; q <= k; ++q) {
    ld p2 = ((2 * q - 1) * x * p1 - (q - 1) * p0) / q;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// derivative of P_k by the identity (x^2 - 1) P'_k = k (x P_k - P_{k-1}), away from +-1
ld legendre_deriv(int k, ld x) {
  if (k == 0) return 0.0L;
  return k * (x * legendre(k, x) - legendre(k - 1, x)) / (x * x - 1.0L);
}

template <typename Fn>
std::vector<ld> roots_in(Fn f, ld a, ld b, int want) {
  const int NS = 20000;
  std::vector<ld> r;
  ld xa = a, fa = f(a);
  for (int i = 1; i <= NS; ++i) {
    ld xb = a + (b - a) * i / NS;
    ld fb = f(xb);
    if (fa == 0.0L) {
      r.push_back(xa);
    } else if ((fa < 0) != (fb < 0) && fb != 0.0L) {
      ld lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200; ++it) {
        ld mid = 0.5L * (lo + hi);
        ld fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      r.push_back(0.5L * (lo + hi));
    }
    xa = xb;
    fa = fb;
  }
  (void)want;
  return r;
}

// Gauss-Legendre nodes/weights on [-1, 1]
void gauss(int q, std::vector<ld>& x, std::vector<ld>& w) {
  x = roots_in([q](ld t) { return legendre(q, t); }, -1.0L, 1.0L, q);
  w.resize(x.size());
  for (size_t i = 0; i < x.size(); ++i) {
    ld d = legendre_deriv(q, x[i]);
    w[i] = 2.0L / ((1.0L - x[i] * x[i]) * d * d);
  }
}

// I[i][j] = int_0^{up[i]} l_j(tau) dtau
std::vector<ld> lagrange_integrals(const std::vector<ld>& c, const std::vector<ld>& up) {
  int s = static_cast<int>(c.size());
  std::vector<ld> gx, gw;
  gauss(std::max(s, 1), gx, gw);
  std::vector<ld> I(up.size() * s, 0.0L);
  for (size_t i = 0; i < up.size(); ++i)
    for (int j = 0; j < s; ++j) {
      ld acc = 0.0L;
      for (size_t q = 0; q < gx.size(); ++q) {
        ld tau = 0.5L * up[i] * (gx[q] + 1.0L);
        ld l = 1.0L;
        for (int m = 0; m < s; ++m)
          if (m != j) l *= (tau - c[m]) / (c[j] - c[m]);
        acc += 0.5L * up[i] * gw[q] * l;
      }
      I[i * s + j] = acc;
    }
  return I;
}

bool solve_ld(std::vector<ld> M, std::vector<ld> rhs, int n, std::vector<ld>& x) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(M[i * n + k]) > std::fabs(M[p * n + k])) p = i;
    if (M[p * n + k] == 0.0L) return false;
    if (p != k) {
      for (int c = 0; c < n; ++c) std::swap(M[k * n + c], M[p * n + c]);
      std::swap(rhs[k], rhs[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      ld f = M[i * n + k] / M[k * n + k];
      for (int c = k; c < n; ++c) M[i * n + c] -= f * M[k * n + c];
      rhs[i] -= f * rhs[k];
    }
  }
  x.assign(n, 0.0L);
  for (int i = n - 1; i >= 0; --i) {
    ld s = rhs[i];
    for (int c = i + 1; c < n; ++c) s -= M[i * n + c] * x[c];
    x[i] = s / M[i * n + i];
  }
  return true;
}

// 2-norm condition number of an s x s matrix via Jacobi eigenvalues of X^T X
double cond2(const double* X, int s) {
  double G[64];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      double t = 0.0;
      for (int k = 0; k < s; ++k) t += X[k * s + i] * X[k * s + j];
      G[i * s + j] = t;
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < s; ++p)
      for (int q = p + 1; q < s; ++q) off += G[p * s + q] * G[p * s + q];
    if (off < 1e-300) break;
    for (int p = 0; p < s; ++p)
      for (int q = p + 1; q < s; ++q) {
        double apq = G[p * s + q];
        if (apq == 0.0) continue;
        double tau = (G[q * s + q] - G[p * s + p]) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < s; ++k) {
          double gkp = G[k * s + p], gkq = G[k * s + q];
          G[k * s + p] = cs * gkp - sn * gkq;
          G[k * s + q] = sn * gkp + cs * gkq;
        }
        for (int k = 0; k < s; ++k) {
          double gpk = G[p * s + k], gqk = G[q * s + k];
          G[p * s + k] = cs * gpk - sn * gqk;
          G[q * s + k] = sn * gpk + cs * gqk;
        }
      }
  }
  double mx = 0.0, mn = 1e300;
  for (int i = 0; i < s; ++i) {
    mx = std::max(mx, G[i * s + i]);
    mn = std::min(mn, G[i * s + i]);
  }
  if (!(mn > 0.0)) return 1e300;
  return std::sqrt(mx / mn);
}

// kappa_2(At^{-1} A) for lower triangular At
double kappa_lower(const double* At, const double* A, int s) {
  double X[64];
  for (int c = 0; c < s; ++c)
    for (int i = 0; i < s; ++i) {
      double v = A[i * s + c];
      for (int k = 0; k < i; ++k) v -= At[i * s + k] * X[k * s + c];
      if (At[i * s + i] == 0.0) return 1e300;
      X[i * s + c] = v / At[i * s + i];
    }
  return cond2(X, s);
}

}  // namespace

extern "C" {

irk_status irk_butcher_table(int32_t method, int32_t s, double* A, double* b, double* c) {
  if (!A || !b || !c) {
    irk::set_global_error("NULL output array");
    return IRK_ERR_INVALID;
  }
  if (method == IRK_METHOD_RADAU_IIA) {
    if (s < 1 || s > irk::MAX_S) {
      irk::set_global_error("Radau IIA needs 1 <= s <= 8");
      return IRK_ERR_INVALID;
    }
    // zeros of P_s(t) - P_{s-1}(t): s-1 in (-1, 1) and t = 1
    std::vector<ld> t;
    if (s > 1) {
      t = roots_in([s](ld x) { return legendre(s, x) - legendre(s - 1, x); }, -1.0L, 1.0L - 1e-9L, s - 1);
    }
    t.push_back(1.0L);
    if (static_cast<int>(t.size()) != s) {
      irk::set_global_error("Radau node search failed");
      return IRK_ERR_INVALID;
    }
    std::vector<ld> cn(s);
    for (int i = 0; i < s; ++i) cn[i] = 0.5L * (t[i] + 1.0L);
    cn[s - 1] = 1.0L;
    std::vector<ld> Ai = lagrange_integrals(cn, cn);
    std::vector<ld> bi = lagrange_integrals(cn, std::vector<ld>{1.0L});
    for (int i = 0; i < s * s; ++i) A[i] = static_cast<double>(Ai[i]);
    for (int i = 0; i < s; ++i) {
      b[i] = static_cast<double>(bi[i]);
      c[i] = static_cast<double>(cn[i]);
    }
    return IRK_OK;
  }
  if (method == IRK_METHOD_LOBATTO_IIIC) {
    if (s < 2 || s > irk::MAX_S) {
      irk::set_global_error("Lobatto IIIC needs 2 <= s <= 8");
      return IRK_ERR_INVALID;
    }
    std::vector<ld> t{-1.0L};
    if (s > 2) {
      std::vector<ld> in = roots_in([s](ld x) { return legendre_deriv(s - 1, x); }, -1.0L + 1e-9L, 1.0L - 1e-9L, s - 2);
      t.insert(t.end(), in.begin(), in.end());
    }
    t.push_back(1.0L);
    if (static_cast<int>(t.size()) != s) {
      irk::set_global_error("Lobatto node search failed");
      return IRK_ERR_INVALID;
    }
    std::vector<ld> cn(s);
    for (int i = 0; i < s; ++i) cn[i] = 0.5L * (t[i] + 1.0L);
    std::vector<ld> bi = lagrange_integrals(cn, std::vector<ld>{1.0L});
    // rows: a_i1 = b_1, sum_{j>=2} a_ij c_j^{q-1} = c_i^q/q - b_1 c_1^{q-1}, q = 1..s-1
    int m = s - 1;
    std::vector<ld> V(m * m);
    for (int q = 1; q <= m; ++q)
      for (int j = 1; j < s; ++j) V[(q - 1) * m + (j - 1)] = std::pow(cn[j], static_cast<ld>(q - 1));
    for (int i = 0; i < s; ++i) {
      std::vector<ld> rhs(m), x;
      for (int q = 1; q <= m; ++q)
        rhs[q - 1] = std::pow(cn[i], static_cast<ld>(q)) / q - bi[0] * std::pow(cn[0], static_cast<ld>(q - 1));
      if (!solve_ld(V, rhs, m, x)) {
        irk::set_global_error("Lobatto system singular");
        return IRK_ERR_INVALID;
      }
      A[i * s] = static_cast<double>(bi[0]);
      for (int j = 1; j < s; ++j) A[i * s + j] = static_cast<double>(x[j - 1]);
    }
    for (int i = 0; i < s; ++i) {
      b[i] = static_cast<double>(bi[i]);
      c[i] = static_cast<double>(cn[i]);
    }
    return IRK_OK;
  }
  irk::set_global_error("unknown method");
  return IRK_ERR_INVALID;
}

irk_status irk_ldu(int32_t s, const double* A, double* L, double* D, double* U) {
  if (s < 1 || s > irk::MAX_S || !A || !L || !D || !U) {
    irk::set_global_error("bad argument to irk_ldu");
    return IRK_ERR_INVALID;
  }
  for (int i = 0; i < s * s; ++i) L[i] = U[i] = 0.0;
  for (int i = 0; i < s; ++i) L[i * s + i] = U[i * s + i] = 1.0;
  for (int k = 0; k < s; ++k) {
    double d = A[k * s + k];
    for (int m = 0; m < k; ++m) d -= L[k * s + m] * D[m] * U[m * s + k];
    if (d == 0.0) {
      irk::set_global_error("zero pivot in the LDU factorisation of the Butcher matrix");
      return IRK_ERR_ZERO_PIVOT;
    }
    D[k] = d;
    for (int i = k + 1; i < s; ++i) {
      double v = A[i * s + k];
      for (int m = 0; m < k; ++m) v -= L[i * s + m] * D[m] * U[m * s + k];
      L[i * s + k] = v / d;
    }
    for (int j = k + 1; j < s; ++j) {
      double v = A[k * s + j];
      for (int m = 0; m < k; ++m) v -= L[k * s + m] * D[m] * U[m * s + j];
      U[k * s + j] = v / d;
    }
  }
  return IRK_OK;
}

irk_status irk_atilde(int32_t kind, int32_t s, const double* A, double* At, double* kappa) {
  if (s < 1 || s > irk::MAX_S || !A || !At) {
    irk::set_global_error("bad argument to irk_atilde");
    return IRK_ERR_INVALID;
  }
  for (int i = 0; i < s * s; ++i) At[i] = 0.0;
  if (kind == IRK_PC_J) {
    for (int i = 0; i < s; ++i) At[i * s + i] = A[i * s + i];
  } else if (kind == IRK_PC_GSL) {
    for (int i = 0; i < s; ++i)
      for (int j = 0; j <= i; ++j) At[i * s + j] = A[i * s + j];
  } else if (kind == IRK_PC_DU || kind == IRK_PC_LD) {
    double L[64], D[8], U[64];
    irk_status st = irk_ldu(s, A, L, D, U);
    if (st != IRK_OK) return st;
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j)
        At[i * s + j] = (kind == IRK_PC_DU) ? D[i] * U[i * s + j] : L[i * s + j] * D[j];
  } else if (kind == IRK_PC_GSL_OPT) {
    // variables: strictly lower entries; Nelder-Mead from tril(A)
    std::vector<std::pair<int, int>> idx;
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < i; ++j) idx.push_back({i, j});
    int nv = static_cast<int>(idx.size());
    auto build = [&](const std::vector<double>& p, double* out) {
      for (int i = 0; i < s * s; ++i) out[i] = 0.0;
      for (int i = 0; i < s; ++i) out[i * s + i] = A[i * s + i];
      for (int q = 0; q < nv; ++q) out[idx[q].first * s + idx[q].second] = p[q];
    };
    auto f = [&](const std::vector<double>& p) {
      double T[64];
      build(p, T);
      return kappa_lower(T, A, s);
    };
    std::vector<double> p0(nv);
    for (int q = 0; q < nv; ++q) p0[q] = A[idx[q].first * s + idx[q].second];
    if (nv > 0) {
      double n = nv;
      double alpha = 1.0, gamma = 1.0 + 2.0 / n, rho = 0.75 - 1.0 / (2.0 * n), sigma = 1.0 - 1.0 / n;
      std::vector<std::vector<double>> X(nv + 1, p0);
      for (int q = 0; q < nv; ++q) X[q + 1][q] = p0[q] != 0.0 ? 1.05 * p0[q] : 0.00025;
      std::vector<double> fx(nv + 1);
      for (int q = 0; q <= nv; ++q) fx[q] = f(X[q]);
      for (int iter = 0; iter < 20000; ++iter) {
        std::vector<int> ord(nv + 1);
        for (int q = 0; q <= nv; ++q) ord[q] = q;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fx[a] < fx[b]; });
        std::vector<std::vector<double>> Xs(nv + 1);
        std::vector<double> fs(nv + 1);
        for (int q = 0; q <= nv; ++q) {
          Xs[q] = X[ord[q]];
          fs[q] = fx[ord[q]];
        }
        X = Xs;
        fx = fs;
        double xspread = 0.0;
        for (int q = 1; q <= nv; ++q)
          for (int k = 0; k < nv; ++k) xspread = std::max(xspread, std::fabs(X[q][k] - X[0][k]));
        if (xspread <= 1e-10 && fx[nv] - fx[0] <= 1e-12) break;
        std::vector<double> cen(nv, 0.0);
        for (int q = 0; q < nv; ++q)
          for (int k = 0; k < nv; ++k) cen[k] += X[q][k] / n;
        auto point = [&](double t) {
          std::vector<double> y(nv);
          for (int k = 0; k < nv; ++k) y[k] = cen[k] + t * (X[nv][k] - cen[k]);
          return y;
        };
        std::vector<double> xr = point(-alpha);
        double fr = f(xr);
        if (fr < fx[0]) {
          std::vector<double> xe = point(-alpha * gamma);
          double fe = f(xe);
          if (fe < fr) {
            X[nv] = xe;
            fx[nv] = fe;
          } else {
            X[nv] = xr;
            fx[nv] = fr;
          }
        } else if (fr < fx[nv - 1]) {
          X[nv] = xr;
          fx[nv] = fr;
        } else {
          bool shrink = false;
          if (fr < fx[nv]) {
            std::vector<double> xc = point(-alpha * rho);
            double fc = f(xc);
            if (fc <= fr) {
              X[nv] = xc;
              fx[nv] = fc;
            } else {
              shrink = true;
            }
          } else {
            std::vector<double> xc = point(rho);
            double fc = f(xc);
            if (fc < fx[nv]) {
              X[nv] = xc;
              fx[nv] = fc;
            } else {
              shrink = true;
            }
          }
          if (shrink) {
            for (int q = 1; q <= nv; ++q) {
              for (int k = 0; k < nv; ++k) X[q][k] = X[0][k] + sigma * (X[q][k] - X[0][k]);
              fx[q] = f(X[q]);
            }
          }
        }
      }
      int best = 0;
      for (int q = 1; q <= nv; ++q)
        if (fx[q] < fx[best]) best = q;
      p0 = X[best];
    }
    build(p0, At);
  } else {
    irk::set_global_error("unknown preconditioner kind");
    return IRK_ERR_INVALID;
  }
  if (kappa) {
    // kappa_2(A~^{-1} A) for the triangular or diagonal A~
    double X[64];
    bool upper = (kind == IRK_PC_DU);
    for (int c = 0; c < s; ++c) {
      if (!upper) {
        for (int i = 0; i < s; ++i) {
          double v = A[i * s + c];
          for (int k = 0; k < i; ++k) v -= At[i * s + k] * X[k * s + c];
          X[i * s + c] = v / At[i * s + i];
        }
      } else {
        for (int i = s - 1; i >= 0; --i) {
          double v = A[i * s + c];
          for (int k = i + 1; k < s; ++k) v -= At[i * s + k] * X[k * s + c];
          X[i * s + c] = v / At[i * s + i];
        }
      }
    }
    *kappa = cond2(X, s);
  }
  return IRK_OK;
}

}  // extern "C"
