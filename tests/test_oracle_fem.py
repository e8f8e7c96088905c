"""Pins for oracle/fem.py: exact integrals of polynomials, null spaces and
skew-symmetry of the P1 matrices of Section 3."""
import numpy as np
import pytest

import synth
from oracle import fem


@pytest.mark.parametrize("N,domain", [(4, "unit"), (7, "box")])
def test_mass_and_stiffness_exact(N, domain):
    mesh = synth.structured_mesh(N, domain)
    mats = fem.assemble(mesh.xy, mesh.tri)
    M, K = mats["M"], mats["K"]
    area = (mesh.hi[0] - mesh.lo[0]) * (mesh.hi[1] - mesh.lo[1])
    one = np.ones(mesh.n_nodes)
    assert abs(one @ M @ one - area) < 1e-13 * area
    assert np.max(np.abs(K @ one)) < 1e-12
    assert abs(M - M.T).max() < 1e-16 and abs(K - K.T).max() < 1e-14
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    # linear u = 2x - 3y + 1: int |grad u|^2 = 13 * area; int u^2 exact (P1 interp exact)
    u = 2 * x - 3 * y + 1
    assert abs(u @ K @ u - 13.0 * area) < 1e-11
    (x0, y0), (x1, y1) = mesh.lo, mesh.hi
    # int (2x - 3y + 1)^2 over the rectangle, by hand
    def I(px, py):
        return (x1 ** (px + 1) - x0 ** (px + 1)) / (px + 1) * (y1 ** (py + 1) - y0 ** (py + 1)) / (py + 1)
    exact = 4 * I(2, 0) + 9 * I(0, 2) + I(0, 0) - 12 * I(1, 1) + 4 * I(1, 0) - 6 * I(0, 1)
    assert abs(u @ M @ u - exact) < 1e-12


def test_stiffness_stencil_uniform():
    # interior row of the uniform right-triangle mesh: 4 on the diagonal, -1 at
    # the four axis neighbours, 0 at the two diagonal neighbours
    mesh = synth.structured_mesh(6)
    K = fem.assemble(mesh.xy, mesh.tri)["K"].tocsr()
    i = 3 * 7 + 3
    row = dict(zip(K.indices[K.indptr[i]:K.indptr[i + 1]], K.data[K.indptr[i]:K.indptr[i + 1]]))
    assert abs(row[i] - 4) < 1e-14
    for j in (i - 1, i + 1, i - 7, i + 7):
        assert abs(row[j] + 1) < 1e-14
    for j in (i - 8, i + 8):
        assert abs(row[j]) < 1e-14
    assert len(row) == 7


def test_convection_double_glazing():
    """C_kl = int phi_k (w . grad phi_l) with w = (2y(1-x^2), -2x(1-y^2)):
    div w = 0 and w.n = 0 on the box boundary give C + C^T = 0; C 1 = 0; and
    v^T C u = int v (w . grad u) for linear u, v (exact with the rule):
    v = y, u = x -> 16/9;  v = x, u = y -> -16/9."""
    mesh = synth.structured_mesh(8, "box")
    C = fem.assemble(mesh.xy, mesh.tri, wind=synth.double_glazing_wind)["C"]
    assert abs(C + C.T).max() < 1e-15
    assert np.max(np.abs(C @ np.ones(mesh.n_nodes))) < 1e-15
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    assert abs(y @ C @ x - 16 / 9) < 1e-13
    assert abs(x @ C @ y + 16 / 9) < 1e-13


def test_kappa_linearity():
    mesh = synth.structured_mesh(5)
    rng = np.random.default_rng(3)
    kap = np.exp(rng.standard_normal(mesh.n_tri))
    K = fem.assemble(mesh.xy, mesh.tri, kappa=kap)["K"].toarray()
    Ke = fem.element_stiffness_unit(mesh.xy, mesh.tri)
    K2 = np.zeros_like(K)
    for e in range(mesh.n_tri):
        t = mesh.tri[e]
        K2[np.ix_(t, t)] += kap[e] * Ke[e]
    assert np.max(np.abs(K - K2)) < 1e-13


def test_problem_restriction():
    mesh = synth.structured_mesh(6, "box")
    ub = synth.double_glazing_boundary(mesh)
    prob = fem.double_glazing_problem(mesh, 0.005, synth.double_glazing_wind, ub)
    assert prob.M.shape == (25, 25) and prob.F.shape == (25, 25)
    # lift: F_full @ u_full restricted to interior rows equals F_II u_I + g
    mats = fem.assemble(mesh.xy, mesh.tri, wind=synth.double_glazing_wind)
    Ff = (0.005 * mats["K"] + mats["C"]).tocsr()
    uI = np.random.default_rng(0).standard_normal(mesh.n)
    full = ub.copy()
    full[mesh.interior] = uI
    assert np.allclose((Ff @ full)[mesh.interior], prob.F @ uI + prob.g, atol=1e-14)
    # hot east wall only
    east = mesh.xy[:, 0] == 1.0
    assert np.all(ub[east] == 1) and np.all(ub[~east] == 0)


# ---------------------------------------------------------------------------
# quadratic (P2) elements, the heat discretisation of the paper's runs
# ---------------------------------------------------------------------------
def test_p2_mesh_counts():
    """(2N-1)^2 unknowns per stage: 225 at N = 8 and 961 at N = 16 (the DOF
    column of the Radau IIA table divided by s: 450 / 2, 1922 / 2)."""
    for N, n in ((8, 225), (16, 961), (128, 65025)):
        m = synth.structured_mesh_p2(N)
        assert m.n == n and m.tri.shape == (2 * N * N, 6) and m.n_nodes == (2 * N + 1) ** 2


def test_p2_element_mass_closed_form():
    """P2 mass matrix of one triangle: |T|/180 [[6,-1,-1,0,-4,0], ...] (node
    order vertices, then midpoints of edges 01, 12, 20): the textbook closed
    form, against the quadrature-based assembly."""
    xy = np.array([[0.3, 0.1], [1.4, 0.5], [0.6, 1.2], [0.85, 0.3], [1.0, 0.85], [0.45, 0.65]])
    tri = np.array([[0, 1, 2, 3, 4, 5]])
    M = fem.assemble_p2(xy, tri)["M"].toarray()
    area = 0.5 * abs((xy[1, 0] - xy[0, 0]) * (xy[2, 1] - xy[0, 1]) - (xy[2, 0] - xy[0, 0]) * (xy[1, 1] - xy[0, 1]))
    ref = np.array([[6, -1, -1, 0, -4, 0], [-1, 6, -1, 0, 0, -4], [-1, -1, 6, -4, 0, 0],
                    [0, 0, -4, 32, 16, 16], [-4, 0, 0, 16, 32, 16], [0, -4, 0, 16, 16, 32]]) * area / 180.0
    assert np.abs(M - ref).max() <= 1e-14


def test_p2_reproduces_quadratics():
    """P2 Galerkin reproduces quadratic solutions exactly: -Lap u = f with
    u = x^2 + 3xy - 2y^2 + x (f = -2) and Dirichlet data u: the interior
    solution of K_II u_I = M_I f - K_IB u_B equals u at the nodes.  Checks the
    whole P2 stiffness and mass assembly, boundary coupling included."""
    mesh = synth.structured_mesh_p2(6)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    u = x * x + 3 * x * y - 2 * y * y + x
    f = -(2.0 - 4.0) * np.ones(mesh.n_nodes)
    mats = fem.assemble_p2(mesh.xy, mesh.tri)
    b = np.flatnonzero(mesh.boundary)
    K_II, K_IB = fem.restrict(mats["K"], mesh.interior, b)
    M_I = mats["M"].tocsr()[mesh.interior]
    rhs = M_I @ f - K_IB @ u[b]
    import scipy.sparse.linalg as spla
    uI = spla.spsolve(K_II.tocsc(), rhs)
    assert np.abs(uI - u[mesh.interior]).max() <= 1e-12
    assert abs(mats["M"].sum() - 1.0) <= 1e-14
    assert np.abs(mats["K"] @ np.ones(mesh.n_nodes)).max() <= 1e-12


# ---------------------------------------------------------------------------
# double glazing with SUPG and Nitsche boundary conditions (Section 5)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [0.04, 0.005])
def test_supg_nitsche_reproduces_linear_solutions(eps):
    """The stabilised discretisation is consistent, so a linear exact solution
    is reproduced exactly: steady -eps Lap u + w.grad u = f (f = w.grad u,
    Dirichlet data u through Nitsche's terms), and the semi-discrete
    (M + S_M) u' + F u = G for u = t phi at t = 1 (source phi + w.grad phi).
    Pins every term: Galerkin, streamline, SUPG mass, Nitsche matrix and load."""
    import scipy.sparse.linalg as spla
    mesh = synth.structured_mesh(12, "box")
    wind = synth.double_glazing_wind
    bx, cy = 0.7, -0.4
    phi = lambda x, y: 0.3 + bx * x + cy * y
    ub = phi(mesh.xy[:, 0], mesh.xy[:, 1])
    P = fem.double_glazing_supg_nitsche(mesh, eps, wind, ub)
    area, G = fem.element_geometry(mesh.xy, mesh.tri)
    wc = wind(*mesh.xy[mesh.tri].mean(axis=1).T)
    assert fem.supg_parameter(area, G, wc, eps).max() > 0.0     # stabilisation active
    f = lambda x, y: wind(x, y) @ np.array([bx, cy])
    uh = spla.spsolve(P.F.tocsc(), fem.supg_load(mesh, eps, wind, f) - P.g)
    assert np.abs(uh - ub).max() <= 1e-12
    f2 = lambda x, y: phi(x, y) + wind(x, y) @ np.array([bx, cy])
    res = P.M @ ub + P.F @ ub - (fem.supg_load(mesh, eps, wind, f2) - P.g)
    assert np.abs(res).max() <= 1e-13
    assert P.M.shape[0] == 13 * 13     # every node is an unknown


def test_nitsche_laplace_without_wind():
    """w = 0: no stabilisation; Nitsche's Laplace problem still reproduces a
    linear solution, and the matrix is symmetric."""
    import scipy.sparse.linalg as spla
    mesh = synth.structured_mesh(8, "box")
    zero = lambda x, y: np.zeros(np.broadcast(x, y).shape + (2,))
    ub = 1.0 + 2.0 * mesh.xy[:, 0] - mesh.xy[:, 1]
    P = fem.double_glazing_supg_nitsche(mesh, 0.1, zero, ub)
    assert abs(P.F - P.F.T).max() <= 1e-15
    uh = spla.spsolve(P.F.tocsc(), -P.g)
    assert np.abs(uh - ub).max() <= 1e-12
