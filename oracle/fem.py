"""P1 and P2 finite-element matrices (oracle; test infrastructure only).

Section 3 of the paper: after the weak form, the stage system involves the
mass matrix M_kl = int phi_k phi_l and F, which is the stiffness
F_kl = int grad phi_k . grad phi_l for the heat problem (Eq. block_coeff_mtx)
and eps*K + C for the double-glazing problem (Eq. testProblemAD), with
C_kl = int phi_k (w . grad phi_l).

Element integrals are written out from the definitions:
  * M_e[a,b] = |T|/12 (1 + delta_ab)          (exact for P1)
  * K_e[a,b] = kappa_e |T| grad l_a . grad l_b (l = barycentric coordinates)
  * C_e[a,b] = int_T l_a (w . grad l_b), by a collapsed (Duffy) 3x3
    Gauss-Legendre rule, exact for the degree-4 integrand (w is cubic).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def element_geometry(xy, tri):
    """Per element: area |T| (nt,) and barycentric gradients G (nt, 3, 2),
    G[e, a] = grad l_a.  From B = [[1,1,1],[x0,x1,x2],[y0,y1,y2]],
    l = B^{-1} [1, x, y]^T, so grad l_a = rows of B^{-1}, columns 1..2."""
    p = xy[tri]                                    # (nt, 3, 2)
    B = np.ones((tri.shape[0], 3, 3))
    B[:, 1, :] = p[:, :, 0]
    B[:, 2, :] = p[:, :, 1]
    Binv = np.linalg.inv(B)
    G = Binv[:, :, 1:3]
    area = 0.5 * np.abs(np.linalg.det(B))
    return area, G


def _duffy_rule(k=3):
    """Points (xi, eta) and weights on the reference triangle
    {xi, eta >= 0, xi + eta <= 1} (weights sum to 1/2), from the square
    [0,1]^2 by xi = u, eta = v (1 - u)."""
    t, w = np.polynomial.legendre.leggauss(k)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    U, V = np.meshgrid(t, t, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    xi = U.ravel()
    eta = (V * (1.0 - U)).ravel()
    wt = (WU * WV * (1.0 - U)).ravel()
    return xi, eta, wt


def assemble(xy, tri, kappa=None, wind=None):
    """Global (all-node) CSR matrices M, K and, if ``wind`` (a callable
    (x, y) -> (..., 2)) is given, C.  ``kappa`` is a per-element diffusion
    coefficient (default 1)."""
    nn = xy.shape[0]
    nt = tri.shape[0]
    area, G = element_geometry(xy, tri)
    if kappa is None:
        kappa = np.ones(nt)
    Me = (area / 12.0)[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None]
    Ke = (kappa * area)[:, None, None] * np.einsum("eai,ebi->eab", G, G)
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(nn, nn))
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(nn, nn))
    M.sum_duplicates()
    K.sum_duplicates()
    out = {"M": M, "K": K}
    if wind is not None:
        xi, eta, wq = _duffy_rule(3)
        lam = np.stack([1.0 - xi - eta, xi, eta], axis=1)   # (nq, 3)
        p = xy[tri]                                         # (nt, 3, 2)
        X = np.einsum("qa,eai->eqi", lam, p)                # physical points
        W = wind(X[..., 0], X[..., 1])                      # (nt, nq, 2)
        wg = np.einsum("eqi,ebi->eqb", W, G)                # w . grad l_b
        # int_T f = 2 |T| sum_q wq f(q)
        Ce = 2.0 * area[:, None, None] * np.einsum("q,qa,eqb->eab", wq, lam, wg)
        C = sp.csr_matrix((Ce.ravel(), (rows, cols)), shape=(nn, nn))
        C.sum_duplicates()
        out["C"] = C
    return out


def p2_basis(lam):
    """Quadratic Lagrange basis at barycentric points lam (nq, 3), node order
    (a, b, c, ab, bc, ca): vertex l_i (2 l_i - 1), edge 4 l_i l_j.  Returns
    the values (nq, 6) and, per basis function, the coefficients of grad in
    terms of grad l_0..l_2: D (nq, 6, 3) with grad phi_k = sum_i D[q,k,i] grad l_i."""
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    nq = lam.shape[0]
    phi = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                    4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=1)
    D = np.zeros((nq, 6, 3))
    D[:, 0, 0] = 4 * l0 - 1
    D[:, 1, 1] = 4 * l1 - 1
    D[:, 2, 2] = 4 * l2 - 1
    D[:, 3, 0], D[:, 3, 1] = 4 * l1, 4 * l0
    D[:, 4, 1], D[:, 4, 2] = 4 * l2, 4 * l1
    D[:, 5, 2], D[:, 5, 0] = 4 * l0, 4 * l2
    return phi, D


def assemble_p2(xy, tri6, kappa=None):
    """Global CSR mass and stiffness of quadratic triangles (Section 5 runs
    the heat problem with P2 elements).  The vertex columns of tri6 give the
    affine map; integrals use the collapsed 3x3 Gauss rule (exact to degree
    5, the mass integrand has degree 4)."""
    nn = xy.shape[0]
    nt = tri6.shape[0]
    area, G = element_geometry(xy, tri6[:, :3])
    if kappa is None:
        kappa = np.ones(nt)
    xi, eta, wq = _duffy_rule(3)
    lam = np.stack([1.0 - xi - eta, xi, eta], axis=1)
    phi, D = p2_basis(lam)
    # int_T f = 2 |T| sum_q wq f(q)
    Mref = 2.0 * np.einsum("q,qa,qb->ab", wq, phi, phi)            # per unit area
    gradk = np.einsum("qki,eij->eqkj", D, G)                        # (nt, nq, 6, 2)
    Ke = 2.0 * (kappa * area)[:, None, None] * np.einsum("q,eqaj,eqbj->eab", wq, gradk, gradk)
    Me = area[:, None, None] * Mref[None]
    rows = np.repeat(tri6, 6, axis=1).ravel()
    cols = np.tile(tri6, (1, 6)).ravel()
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(nn, nn))
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(nn, nn))
    M.sum_duplicates()
    K.sum_duplicates()
    return {"M": M, "K": K}


def heat_problem_p2(mesh, kappa=None):
    """The heat problem of Section 3.1 with quadratic elements (Section 5)."""
    mats = assemble_p2(mesh.xy, mesh.tri, kappa=kappa)
    M = restrict(mats["M"], mesh.interior)
    F = restrict(mats["K"], mesh.interior)
    return Problem(M, F, np.zeros(mesh.n), mesh, kappa=kappa, kind="heat")


def element_stiffness_unit(xy, tri):
    """K_e for kappa_e = 1: (nt, 3, 3) = |T| G G^T (the derivative of the
    stiffness matrix with respect to kappa_e)."""
    area, G = element_geometry(xy, tri)
    return area[:, None, None] * np.einsum("eai,ebi->eab", G, G)


def restrict(A, interior, boundary_nodes=None):
    """Interior-interior block A_II and interior-boundary block A_IB."""
    A = A.tocsr()
    AI = A[interior]
    A_II = AI[:, interior].tocsr()
    A_II.sort_indices()
    if boundary_nodes is None:
        return A_II
    A_IB = AI[:, boundary_nodes].tocsr()
    return A_II, A_IB


class Problem:
    """Interior-unknown matrices of one test problem.

    M, F: CSR (n x n) over interior nodes; g: the boundary lift F_IB u_B that
    enters the stage right-hand side (zero for the heat problem)."""

    def __init__(self, M, F, g, mesh, kappa=None, eps=None, kind="heat"):
        self.M = M
        self.F = F
        self.g = g
        self.mesh = mesh
        self.kappa = kappa
        self.eps = eps
        self.kind = kind

    @property
    def n(self):
        return self.M.shape[0]


def heat_problem(mesh, kappa=None):
    """Heat equation u_t = div(kappa grad u), zero Dirichlet (Section 3.1);
    F = K (kappa-weighted when a per-element kappa is given)."""
    mats = assemble(mesh.xy, mesh.tri, kappa=kappa)
    M = restrict(mats["M"], mesh.interior)
    F = restrict(mats["K"], mesh.interior)
    return Problem(M, F, np.zeros(mesh.n), mesh, kappa=kappa, kind="heat")


def double_glazing_problem(mesh, eps, wind, ub):
    """Double glazing (Section 3.2): F = eps K + C, Dirichlet values ub
    (all nodes) eliminated, lift g = F_IB u_B."""
    mats = assemble(mesh.xy, mesh.tri, wind=wind)
    Ffull = (eps * mats["K"] + mats["C"]).tocsr()
    bnodes = np.flatnonzero(mesh.boundary)
    M = restrict(mats["M"], mesh.interior)
    F, F_IB = restrict(Ffull, mesh.interior, bnodes)
    g = F_IB @ ub[bnodes]
    return Problem(M, F, g, mesh, eps=eps, kind="double_glazing")


# ----------------------------------------------------------------------------
# Double glazing with SUPG stabilisation and Nitsche boundary conditions (the
# paper's discretisation of the advection-diffusion runs, Section 5)
# ----------------------------------------------------------------------------

def boundary_edges(mesh):
    """(tri index, local vertex a, local vertex b) of every boundary edge: both
    end nodes on the boundary and the edge on one of the four walls."""
    out = []
    xy, tri = mesh.xy, mesh.tri
    lo, hi = mesh.lo, mesh.hi
    for e in range(tri.shape[0]):
        for a in range(3):
            b = (a + 1) % 3
            pa, pb = xy[tri[e, a]], xy[tri[e, b]]
            for ax, val in ((0, lo[0]), (0, hi[0]), (1, lo[1]), (1, hi[1])):
                if pa[ax] == val and pb[ax] == val:
                    out.append((e, a, b))
    return out


def supg_parameter(area, G, w_c, eps):
    """Per element: the streamline length h_e = 2|w_e| / sum_a |w_e . grad l_a|
    (Tezduyar and Park), the mesh Peclet number P_e = |w_e| h_e / (2 eps) and
    delta_e = h_e / (2|w_e|) (1 - 1/P_e) when P_e > 1, else 0 (Elman,
    Silvester and Wathen, the reference of Section 3.2), w_e = the wind at the
    centroid."""
    wn = np.linalg.norm(w_c, axis=1)
    proj = np.abs(np.einsum("ei,eai->ea", w_c, G)).sum(axis=1)
    he = np.where(proj > 0, 2.0 * wn / np.where(proj > 0, proj, 1.0), 0.0)
    Pe = wn * he / (2.0 * eps)
    delta = np.where(Pe > 1.0, he / (2.0 * np.where(wn > 0, wn, 1.0)) * (1.0 - 1.0 / np.where(Pe > 0, Pe, 1.0)),
                     0.0)
    return delta


def streamline_matrix(mesh, eps, wind):
    """All-node streamline-diffusion matrix of the coarse-level SUPG
    stabilisation: T[i,j] = sum over elements with mesh Peclet number P_e > 1
    of h_e/(2|w_e|) |T| (w_e . grad l_i)(w_e . grad l_j), with h_e, P_e and the
    centroid wind w_e of supg_parameter (the large-Peclet slope of delta_e in
    the element size)."""
    xy, tri = mesh.xy, mesh.tri
    area, G = element_geometry(xy, tri)
    p = xy[tri]
    centroid = p.mean(axis=1)
    w_c = wind(centroid[:, 0], centroid[:, 1])
    wn = np.linalg.norm(w_c, axis=1)
    wcg = np.einsum("ei,eai->ea", w_c, G)
    proj = np.abs(wcg).sum(axis=1)
    he = np.where(proj > 0, 2.0 * wn / np.where(proj > 0, proj, 1.0), 0.0)
    Pe = wn * he / (2.0 * eps)
    slope = np.where(Pe > 1.0, he / (2.0 * np.where(wn > 0, wn, 1.0)), 0.0)
    Te = (slope * area)[:, None, None] * wcg[:, :, None] * wcg[:, None, :]
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    n = xy.shape[0]
    T = sp.csr_matrix((Te.ravel(), (rows, cols)), shape=(n, n))
    T.sum_duplicates()
    T.sort_indices()
    return T


def double_glazing_supg_nitsche(mesh, eps, wind, ub, gamma=10.0):
    """All-node matrices of
        (M + S_M) u' + (eps K + C + S + N) u = G
    on the P1 mesh: S_M[i,j] = delta_e int phi_j (w_e . grad phi_i),
    S[i,j] = delta_e int (w . grad phi_j)(w_e . grad phi_i) (the streamline
    residual of the Galerkin convection, tested along the centroid wind),
    Nitsche's symmetric terms on the boundary edges
        N[i,j] = -eps int_e (grad phi_j . n) phi_i - eps int_e (grad phi_i . n) phi_j
                 + (gamma eps / |e|) int_e phi_i phi_j,
    and the load G[i] = -eps int_e (grad phi_i . n) u_B + (gamma eps / |e|) int_e u_B phi_i
    with u_B linear along each edge from the nodal values ub.  The wind is
    tangential on the walls, so there is no inflow term.  Every node is an
    unknown; the stage right-hand side uses g = -G."""
    xy, tri = mesh.xy, mesh.tri
    nn = xy.shape[0]
    nt = tri.shape[0]
    area, G = element_geometry(xy, tri)
    base = assemble(xy, tri, wind=wind)
    p = xy[tri]
    centroid = p.mean(axis=1)
    w_c = wind(centroid[:, 0], centroid[:, 1])
    delta = supg_parameter(area, G, w_c, eps)
    xi, eta, wq = _duffy_rule(3)
    lam = np.stack([1.0 - xi - eta, xi, eta], axis=1)
    X = np.einsum("qa,eai->eqi", lam, p)
    W = wind(X[..., 0], X[..., 1])                      # (nt, nq, 2)
    Wint = 2.0 * area[:, None] * np.einsum("q,eqi->ei", wq, W)   # int_T w
    wcg = np.einsum("ei,eai->ea", w_c, G)               # w_e . grad l_i
    wig = np.einsum("ei,ebi->eb", Wint, G)              # (int_T w) . grad l_j
    Se = delta[:, None, None] * wcg[:, :, None] * wig[:, None, :]
    SMe = delta[:, None, None] * wcg[:, :, None] * (area / 3.0)[:, None, None] * np.ones((1, 1, 3))
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    S = sp.csr_matrix((Se.ravel(), (rows, cols)), shape=(nn, nn))
    SM = sp.csr_matrix((SMe.ravel(), (rows, cols)), shape=(nn, nn))
    nr, nc, nv = [], [], []
    load = np.zeros(nn)
    for (e, a, b) in boundary_edges(mesh):
        ia, ib = tri[e, a], tri[e, b]
        t = xy[ib] - xy[ia]
        L = np.hypot(t[0], t[1])
        n = np.array([t[1], -t[0]]) / L             # outward for counter-clockwise triangles
        gn = G[e] @ n                               # grad l_k . n, k = 0..2
        on = {ia: None, ib: None}
        for k in range(3):
            for (m, i_node) in ((0, ia), (1, ib)):
                # -eps int_e (grad phi_k . n) phi_i  and its transpose
                nr.append(i_node); nc.append(tri[e, k]); nv.append(-eps * gn[k] * L / 2.0)
                nr.append(tri[e, k]); nc.append(i_node); nv.append(-eps * gn[k] * L / 2.0)
        for i_node in (ia, ib):
            for j_node in (ia, ib):
                nr.append(i_node); nc.append(j_node)
                nv.append(gamma * eps / L * L / 6.0 * (2.0 if i_node == j_node else 1.0))
        ga, gb = ub[ia], ub[ib]
        for k in range(3):
            load[tri[e, k]] += -eps * gn[k] * L * (ga + gb) / 2.0
        load[ia] += gamma * eps / L * L / 6.0 * (2.0 * ga + gb)
        load[ib] += gamma * eps / L * L / 6.0 * (2.0 * gb + ga)
    Nmat = sp.csr_matrix((np.array(nv), (np.array(nr), np.array(nc))), shape=(nn, nn))
    M = (base["M"] + SM).tocsr()
    F = (eps * base["K"] + base["C"] + S + Nmat).tocsr()
    M.sum_duplicates()
    F.sum_duplicates()
    M.sort_indices()
    F.sort_indices()
    prob = Problem(M, F, -load, mesh, eps=eps, kind="double_glazing_supg")
    prob.T = streamline_matrix(mesh, eps, wind)
    return prob


def supg_load(mesh, eps, wind, f):
    """int f phi_i + delta_e int f (w_e . grad phi_i) for a source f(x, y)
    (tests only: the consistency pins of the stabilised discretisation).
    Collapsed 4x4 Gauss (exact to degree 7)."""
    xy, tri = mesh.xy, mesh.tri
    area, G = element_geometry(xy, tri)
    p = xy[tri]
    centroid = p.mean(axis=1)
    w_c = wind(centroid[:, 0], centroid[:, 1])
    delta = supg_parameter(area, G, w_c, eps)
    xi, eta, wq = _duffy_rule(4)
    lam = np.stack([1.0 - xi - eta, xi, eta], axis=1)
    X = np.einsum("qa,eai->eqi", lam, p)
    fq = f(X[..., 0], X[..., 1])                          # (nt, nq)
    wcg = np.einsum("ei,eai->ea", w_c, G)
    le = 2.0 * area[:, None] * (np.einsum("q,eq,qa->ea", wq, fq, lam)
                                + delta[:, None] * wcg * np.einsum("q,eq->e", wq, fq)[:, None])
    out = np.zeros(xy.shape[0])
    np.add.at(out, tri.ravel(), le.ravel())
    return out
