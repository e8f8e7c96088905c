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
