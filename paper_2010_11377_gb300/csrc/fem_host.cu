// Host P1 (and, for the heat problem, P2) assembly of the interior-unknown
// matrices of Section 3:
//   M_kl = int phi_k phi_l,  F = sum_e kappa_e K_e + C,
//   K_e[a,b] = |T| grad l_a . grad l_b,  C_kl = int phi_k (w . grad phi_l),
// with strong Dirichlet elimination and the lift g = F_IB u_B.  The convection
// integrand (P1 times the sampled wind) uses the symmetric 6-point degree-4
// rule of Dunavant (1985); callers sample the wind at irk_fem_quad_points.
#include "irk_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

// barycentric coordinates and weights (weights sum to 1) of the degree-4 rule
const double kA1 = 0.445948490915965, kW1 = 0.223381589678011;
const double kA2 = 0.091576213509771, kW2 = 0.109951743655322;

void rule(double bary[6][3], double w[6]) {
  const double a[2] = {kA1, kA2}, ww[2] = {kW1, kW2};
  int q = 0;
  for (int g = 0; g < 2; ++g) {
    double x = a[g], y = 1.0 - 2.0 * a[g];
    double pts[3][3] = {{x, x, y}, {x, y, x}, {y, x, x}};
    for (int k = 0; k < 3; ++k, ++q) {
      bary[q][0] = pts[k][0];
      bary[q][1] = pts[k][1];
      bary[q][2] = pts[k][2];
      w[q] = ww[g];
    }
  }
}

struct Geo {
  double area;
  double gx[3], gy[3];
};

bool geometry(const double* xy, const int32_t* t, Geo& g) {
  double x0 = xy[2 * t[0]], y0 = xy[2 * t[0] + 1];
  double x1 = xy[2 * t[1]], y1 = xy[2 * t[1] + 1];
  double x2 = xy[2 * t[2]], y2 = xy[2 * t[2] + 1];
  double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
  if (!(det > 0.0)) return false;
  g.area = 0.5 * det;
  g.gx[0] = (y1 - y2) / det;
  g.gx[1] = (y2 - y0) / det;
  g.gx[2] = (y0 - y1) / det;
  g.gy[0] = (x2 - x1) / det;
  g.gy[1] = (x0 - x2) / det;
  g.gy[2] = (x1 - x0) / det;
  return true;
}

}  // namespace

extern "C" {

irk_status irk_fem_quad_points(int32_t n_tri, const double* xy, const int32_t* tri, double* xq) {
  if (n_tri < 0 || (n_tri > 0 && (!xy || !tri || !xq))) {
    irk::set_global_error("bad argument to irk_fem_quad_points");
    return IRK_ERR_INVALID;
  }
  double bary[6][3], w[6];
  rule(bary, w);
  for (int e = 0; e < n_tri; ++e) {
    const int32_t* t = tri + 3 * e;
    for (int q = 0; q < 6; ++q) {
      double x = 0.0, y = 0.0;
      for (int a = 0; a < 3; ++a) {
        x += bary[q][a] * xy[2 * t[a]];
        y += bary[q][a] * xy[2 * t[a] + 1];
      }
      xq[(size_t(e) * 6 + q) * 2] = x;
      xq[(size_t(e) * 6 + q) * 2 + 1] = y;
    }
  }
  return IRK_OK;
}

irk_status irk_fem_assemble(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri, const int32_t* dof,
                            int32_t n, const double* kappa, const double* wind, const double* ub, int64_t* nnz,
                            int64_t* rowptr, int32_t* col, double* valM, double* valF, double* g) {
  if (n_nodes <= 0 || n_tri <= 0 || n <= 0 || !xy || !tri || !dof || !nnz) {
    irk::set_global_error("bad argument to irk_fem_assemble");
    return IRK_ERR_INVALID;
  }
  for (int e = 0; e < 3 * n_tri; ++e)
    if (tri[e] < 0 || tri[e] >= n_nodes) {
      irk::set_global_error("triangle vertex out of range");
      return IRK_ERR_INVALID;
    }
  for (int v = 0; v < n_nodes; ++v)
    if (dof[v] >= n) {
      irk::set_global_error("dof index out of range");
      return IRK_ERR_INVALID;
    }
  // pattern: interior couplings of each element, sorted and unique per row
  std::vector<int64_t> cnt(n + 1, 0);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) {
      int da = dof[tri[3 * e + a]];
      if (da < 0) continue;
      for (int b = 0; b < 3; ++b)
        if (dof[tri[3 * e + b]] >= 0) ++cnt[da + 1];
    }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> raw(cnt[n]);
  std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) {
      int da = dof[tri[3 * e + a]];
      if (da < 0) continue;
      for (int b = 0; b < 3; ++b) {
        int db = dof[tri[3 * e + b]];
        if (db >= 0) raw[cur[da]++] = db;
      }
    }
  std::vector<int64_t> rp(n + 1, 0);
  std::vector<int> cl;
  cl.reserve(raw.size() / 2 + 1);
  for (int i = 0; i < n; ++i) {
    auto b = raw.begin() + cnt[i], e = raw.begin() + cnt[i + 1];
    std::sort(b, e);
    auto u = std::unique(b, e);
    cl.insert(cl.end(), b, u);
    rp[i + 1] = static_cast<int64_t>(cl.size());
  }
  *nnz = rp[n];
  if (!rowptr || !col || !valM || !valF) return IRK_OK;   // size query
  std::copy(rp.begin(), rp.end(), rowptr);
  std::copy(cl.begin(), cl.end(), col);
  std::fill(valM, valM + rp[n], 0.0);
  std::fill(valF, valF + rp[n], 0.0);
  if (g) std::fill(g, g + n, 0.0);
  double bary[6][3], w[6];
  rule(bary, w);
  for (int e = 0; e < n_tri; ++e) {
    const int32_t* t = tri + 3 * e;
    Geo geo;
    if (!geometry(xy, t, geo)) {
      irk::set_global_error("mesh triangles must be counter-clockwise and non-degenerate");
      return IRK_ERR_INVALID;
    }
    double ke = kappa ? kappa[e] : 1.0;
    double Me[3][3], Fe[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        Me[a][b] = geo.area / 12.0 * (a == b ? 2.0 : 1.0);
        Fe[a][b] = ke * geo.area * (geo.gx[a] * geo.gx[b] + geo.gy[a] * geo.gy[b]);
      }
    if (wind) {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double s = 0.0;
          for (int q = 0; q < 6; ++q) {
            double wx = wind[(size_t(e) * 6 + q) * 2], wy = wind[(size_t(e) * 6 + q) * 2 + 1];
            s += w[q] * bary[q][a] * (wx * geo.gx[b] + wy * geo.gy[b]);
          }
          Fe[a][b] += geo.area * s;
        }
    }
    for (int a = 0; a < 3; ++a) {
      int da = dof[t[a]];
      if (da < 0) continue;
      for (int b = 0; b < 3; ++b) {
        int db = dof[t[b]];
        if (db < 0) {
          if (g && ub) g[da] += Fe[a][b] * ub[t[b]];
          continue;
        }
        auto beg = cl.begin() + rp[da], end = cl.begin() + rp[da + 1];
        int64_t pos = std::lower_bound(beg, end, db) - cl.begin();
        valM[pos] += Me[a][b];
        valF[pos] += Fe[a][b];
      }
    }
  }
  return IRK_OK;
}

// Quadratic (6-node) triangles for the heat problem of the paper's runs
// (Section 5): M_e and K_e from the degree-4 rule (exact: the mass integrand
// has degree 4, the stiffness integrand degree 2).  Basis at barycentric l:
// vertex i: l_i (2 l_i - 1), edge (i, j): 4 l_i l_j, node order a, b, c, ab,
// bc, ca.
irk_status irk_fem_assemble_p2(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri6,
                               const int32_t* dof, int32_t n, const double* kappa, const double* ub, int64_t* nnz,
                               int64_t* rowptr, int32_t* col, double* valM, double* valF, double* g) {
  if (n_nodes <= 0 || n_tri <= 0 || n <= 0 || !xy || !tri6 || !dof || !nnz) {
    irk::set_global_error("bad argument to irk_fem_assemble_p2");
    return IRK_ERR_INVALID;
  }
  for (int64_t e = 0; e < 6 * int64_t(n_tri); ++e)
    if (tri6[e] < 0 || tri6[e] >= n_nodes) {
      irk::set_global_error("triangle node out of range");
      return IRK_ERR_INVALID;
    }
  for (int v = 0; v < n_nodes; ++v)
    if (dof[v] >= n) {
      irk::set_global_error("dof index out of range");
      return IRK_ERR_INVALID;
    }
  std::vector<int64_t> cnt(n + 1, 0);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 6; ++a) {
      int da = dof[tri6[6 * e + a]];
      if (da < 0) continue;
      for (int b = 0; b < 6; ++b)
        if (dof[tri6[6 * e + b]] >= 0) ++cnt[da + 1];
    }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> raw(cnt[n]);
  std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 6; ++a) {
      int da = dof[tri6[6 * e + a]];
      if (da < 0) continue;
      for (int b = 0; b < 6; ++b) {
        int db = dof[tri6[6 * e + b]];
        if (db >= 0) raw[cur[da]++] = db;
      }
    }
  std::vector<int64_t> rp(n + 1, 0);
  std::vector<int> cl;
  cl.reserve(raw.size() / 2 + 1);
  for (int i = 0; i < n; ++i) {
    auto b = raw.begin() + cnt[i], e = raw.begin() + cnt[i + 1];
    std::sort(b, e);
    auto u = std::unique(b, e);
    cl.insert(cl.end(), b, u);
    rp[i + 1] = static_cast<int64_t>(cl.size());
  }
  *nnz = rp[n];
  if (!rowptr || !col || !valM || !valF) return IRK_OK;   // size query
  std::copy(rp.begin(), rp.end(), rowptr);
  std::copy(cl.begin(), cl.end(), col);
  std::fill(valM, valM + rp[n], 0.0);
  std::fill(valF, valF + rp[n], 0.0);
  if (g) std::fill(g, g + n, 0.0);
  double bary[6][3], w[6];
  rule(bary, w);
  // basis values and barycentric-gradient coefficients at the rule's points
  double phi[6][6], dl[6][6][3];
  for (int q = 0; q < 6; ++q) {
    const double* l = bary[q];
    const int ea[3] = {0, 1, 2}, eb[3] = {1, 2, 0};
    for (int k = 0; k < 6; ++k)
      for (int i = 0; i < 3; ++i) dl[q][k][i] = 0.0;
    for (int i = 0; i < 3; ++i) {
      phi[q][i] = l[i] * (2.0 * l[i] - 1.0);
      dl[q][i][i] = 4.0 * l[i] - 1.0;
    }
    for (int k = 0; k < 3; ++k) {
      int i = ea[k], j = eb[k];
      phi[q][3 + k] = 4.0 * l[i] * l[j];
      dl[q][3 + k][i] = 4.0 * l[j];
      dl[q][3 + k][j] = 4.0 * l[i];
    }
  }
  for (int e = 0; e < n_tri; ++e) {
    const int32_t* t = tri6 + 6 * e;
    Geo geo;
    if (!geometry(xy, t, geo)) {
      irk::set_global_error("mesh triangles must be counter-clockwise and non-degenerate");
      return IRK_ERR_INVALID;
    }
    double ke = kappa ? kappa[e] : 1.0;
    double Me[6][6], Fe[6][6];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) {
        double sm = 0.0, sk = 0.0;
        for (int q = 0; q < 6; ++q) {
          double gax = 0.0, gay = 0.0, gbx = 0.0, gby = 0.0;
          for (int i = 0; i < 3; ++i) {
            gax += dl[q][a][i] * geo.gx[i];
            gay += dl[q][a][i] * geo.gy[i];
            gbx += dl[q][b][i] * geo.gx[i];
            gby += dl[q][b][i] * geo.gy[i];
          }
          sm += w[q] * phi[q][a] * phi[q][b];
          sk += w[q] * (gax * gbx + gay * gby);
        }
        Me[a][b] = geo.area * sm;
        Fe[a][b] = ke * geo.area * sk;
      }
    for (int a = 0; a < 6; ++a) {
      int da = dof[t[a]];
      if (da < 0) continue;
      for (int b = 0; b < 6; ++b) {
        int db = dof[t[b]];
        if (db < 0) {
          if (g && ub) g[da] += Fe[a][b] * ub[t[b]];
          continue;
        }
        auto beg = cl.begin() + rp[da], end = cl.begin() + rp[da + 1];
        int64_t pos = std::lower_bound(beg, end, db) - cl.begin();
        valM[pos] += Me[a][b];
        valF[pos] += Fe[a][b];
      }
    }
  }
  return IRK_OK;
}

// Double glazing with SUPG stabilisation and symmetric Nitsche boundary
// conditions (the discretisation of the paper's advection-diffusion runs,
// Section 5); every node is an unknown.
//   M = M_gal + S_M,  S_M[i,j] = delta_e (w_e . grad l_i) |T| / 3
//   F = eps K + C + S + N,  S[i,j] = delta_e (w_e . grad l_i) (int_T w) . grad l_j
//   N on each boundary edge (a triangle edge no other triangle shares):
//     -eps int_e (grad phi_j . n) phi_i - eps int_e (grad phi_i . n) phi_j
//     + (gamma eps / |e|) int_e phi_i phi_j
//   g = -G,  G_i = -eps int_e (grad phi_i . n) u_B + (gamma eps / |e|) int_e u_B phi_i
// delta_e: streamline length h_e = 2|w_e| / sum_a |w_e . grad l_a|, Peclet
// number P_e = |w_e| h_e / (2 eps), delta_e = h_e / (2 |w_e|) (1 - 1/P_e) for
// P_e > 1, else 0; w_e = the wind at the centroid.
irk_status irk_fem_assemble_supg(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri, double eps,
                                 const double* wind, const double* wind_c, const double* ub, double gamma,
                                 int64_t* nnz, int64_t* rowptr, int32_t* col, double* valM, double* valF,
                                 double* g) {
  if (n_nodes <= 0 || n_tri <= 0 || !xy || !tri || !wind || !wind_c || !nnz || !(eps > 0.0) || !(gamma > 0.0)) {
    irk::set_global_error("bad argument to irk_fem_assemble_supg");
    return IRK_ERR_INVALID;
  }
  for (int64_t e = 0; e < 3 * int64_t(n_tri); ++e)
    if (tri[e] < 0 || tri[e] >= n_nodes) {
      irk::set_global_error("triangle vertex out of range");
      return IRK_ERR_INVALID;
    }
  const int n = n_nodes;
  std::vector<int64_t> cnt(n + 1, 0);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) cnt[tri[3 * e + a] + 1] += 3;
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> raw(cnt[n]);
  std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) raw[cur[tri[3 * e + a]]++] = tri[3 * e + b];
  std::vector<int64_t> rp(n + 1, 0);
  std::vector<int> cl;
  cl.reserve(raw.size() / 2 + 1);
  for (int i = 0; i < n; ++i) {
    auto b = raw.begin() + cnt[i], e = raw.begin() + cnt[i + 1];
    std::sort(b, e);
    auto u = std::unique(b, e);
    cl.insert(cl.end(), b, u);
    rp[i + 1] = static_cast<int64_t>(cl.size());
  }
  *nnz = rp[n];
  if (!rowptr || !col || !valM || !valF) return IRK_OK;   // size query
  std::copy(rp.begin(), rp.end(), rowptr);
  std::copy(cl.begin(), cl.end(), col);
  std::fill(valM, valM + rp[n], 0.0);
  std::fill(valF, valF + rp[n], 0.0);
  if (g) std::fill(g, g + n, 0.0);
  auto at = [&](int i, int j) -> int64_t {
    auto beg = cl.begin() + rp[i], end = cl.begin() + rp[i + 1];
    return std::lower_bound(beg, end, j) - cl.begin();
  };
  // boundary edges: edges of exactly one triangle
  std::vector<std::pair<int64_t, int>> edges;   // (min*n + max, triangle*3 + local start vertex)
  edges.reserve(size_t(n_tri) * 3);
  for (int e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) {
      int p0 = tri[3 * e + a], p1 = tri[3 * e + (a + 1) % 3];
      int64_t key = int64_t(std::min(p0, p1)) * n + std::max(p0, p1);
      edges.push_back({key, 3 * e + a});
    }
  std::sort(edges.begin(), edges.end());
  std::vector<char> on_boundary(size_t(n_tri) * 3, 0);
  for (size_t q = 0; q < edges.size();) {
    size_t r = q + 1;
    while (r < edges.size() && edges[r].first == edges[q].first) ++r;
    if (r - q == 1) on_boundary[edges[q].second] = 1;
    q = r;
  }
  double bary[6][3], w[6];
  rule(bary, w);
  for (int e = 0; e < n_tri; ++e) {
    const int32_t* t = tri + 3 * e;
    Geo geo;
    if (!geometry(xy, t, geo)) {
      irk::set_global_error("mesh triangles must be counter-clockwise and non-degenerate");
      return IRK_ERR_INVALID;
    }
    double Me[3][3], Fe[3][3];
    double wi[2] = {0.0, 0.0};   // int_T w
    for (int q = 0; q < 6; ++q) {
      wi[0] += geo.area * w[q] * wind[(size_t(e) * 6 + q) * 2];
      wi[1] += geo.area * w[q] * wind[(size_t(e) * 6 + q) * 2 + 1];
    }
    const double wcx = wind_c[2 * e], wcy = wind_c[2 * e + 1];
    double wcg[3], sum = 0.0;
    for (int a = 0; a < 3; ++a) {
      wcg[a] = wcx * geo.gx[a] + wcy * geo.gy[a];
      sum += std::fabs(wcg[a]);
    }
    const double wn = std::sqrt(wcx * wcx + wcy * wcy);
    double delta = 0.0;
    if (sum > 0.0 && wn > 0.0) {
      double he = 2.0 * wn / sum;
      double pe = wn * he / (2.0 * eps);
      if (pe > 1.0) delta = he / (2.0 * wn) * (1.0 - 1.0 / pe);
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double conv = 0.0;
        for (int q = 0; q < 6; ++q) {
          double wx = wind[(size_t(e) * 6 + q) * 2], wy = wind[(size_t(e) * 6 + q) * 2 + 1];
          conv += w[q] * bary[q][a] * (wx * geo.gx[b] + wy * geo.gy[b]);
        }
        Me[a][b] = geo.area / 12.0 * (a == b ? 2.0 : 1.0) + delta * wcg[a] * geo.area / 3.0;
        Fe[a][b] = eps * geo.area * (geo.gx[a] * geo.gx[b] + geo.gy[a] * geo.gy[b]) + geo.area * conv +
                   delta * wcg[a] * (wi[0] * geo.gx[b] + wi[1] * geo.gy[b]);
      }
    // Nitsche terms of this triangle's boundary edges
    for (int a = 0; a < 3; ++a) {
      if (!on_boundary[3 * e + a]) continue;
      const int b = (a + 1) % 3;
      const int ia = t[a], ib = t[b];
      const double tx = xy[2 * ib] - xy[2 * ia], ty = xy[2 * ib + 1] - xy[2 * ia + 1];
      const double L = std::sqrt(tx * tx + ty * ty);
      const double nx = ty / L, ny = -tx / L;   // outward for a counter-clockwise triangle
      double gn[3];
      for (int k = 0; k < 3; ++k) gn[k] = geo.gx[k] * nx + geo.gy[k] * ny;
      const int loc[2] = {a, b};
      for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 2; ++m) {
          Fe[loc[m]][k] += -eps * gn[k] * L / 2.0;
          Fe[k][loc[m]] += -eps * gn[k] * L / 2.0;
        }
      for (int m = 0; m < 2; ++m)
        for (int r = 0; r < 2; ++r) Fe[loc[m]][loc[r]] += gamma * eps / 6.0 * (m == r ? 2.0 : 1.0);
      if (g) {
        const double ga = ub ? ub[ia] : 0.0, gb = ub ? ub[ib] : 0.0;
        for (int k = 0; k < 3; ++k) g[t[k]] -= -eps * gn[k] * L * (ga + gb) / 2.0;
        g[ia] -= gamma * eps / 6.0 * (2.0 * ga + gb);
        g[ib] -= gamma * eps / 6.0 * (2.0 * gb + ga);
      }
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        int64_t pos = at(t[a], t[b]);
        valM[pos] += Me[a][b];
        valF[pos] += Fe[a][b];
      }
  }
  return IRK_OK;
}

irk_status irk_fem_assemble_streamline(int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri,
                                       double eps, const double* wind_c, const int64_t* rowptr,
                                       const int32_t* col, double* valT) {
  if (n_nodes <= 0 || n_tri <= 0 || !xy || !tri || !wind_c || !rowptr || !col || !valT || !(eps > 0.0)) {
    irk::set_global_error("bad argument to irk_fem_assemble_streamline");
    return IRK_ERR_INVALID;
  }
  for (int64_t e = 0; e < 3 * int64_t(n_tri); ++e)
    if (tri[e] < 0 || tri[e] >= n_nodes) {
      irk::set_global_error("triangle vertex out of range");
      return IRK_ERR_INVALID;
    }
  std::fill(valT, valT + rowptr[n_nodes], 0.0);
  for (int e = 0; e < n_tri; ++e) {
    const int32_t* t = tri + 3 * e;
    Geo geo;
    if (!geometry(xy, t, geo)) {
      irk::set_global_error("mesh triangles must be counter-clockwise and non-degenerate");
      return IRK_ERR_INVALID;
    }
    const double wcx = wind_c[2 * e], wcy = wind_c[2 * e + 1];
    double wcg[3], sum = 0.0;
    for (int a = 0; a < 3; ++a) {
      wcg[a] = wcx * geo.gx[a] + wcy * geo.gy[a];
      sum += std::fabs(wcg[a]);
    }
    const double wn = std::sqrt(wcx * wcx + wcy * wcy);
    if (!(sum > 0.0 && wn > 0.0)) continue;
    const double he = 2.0 * wn / sum;
    if (!(wn * he / (2.0 * eps) > 1.0)) continue;   // Peclet number at most 1: no SUPG term
    const double slope = he / (2.0 * wn);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int i = t[a], j = t[b];
        const int32_t* beg = col + rowptr[i];
        const int32_t* end = col + rowptr[i + 1];
        const int32_t* it = std::lower_bound(beg, end, j);
        if (it == end || *it != j) {
          irk::set_global_error("triangle entry missing from the given pattern");
          return IRK_ERR_INVALID;
        }
        valT[it - col] += slope * geo.area * wcg[a] * wcg[b];
      }
  }
  return IRK_OK;
}

}  // extern "C"
