"""Pins for oracle/amg.py: the hash, the distance-2 independent set, the
aggregation rule, the Galerkin product, and the V-cycle as a linear,
convergent operator."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import amg
from oracle import butcher as bt
from oracle import fem


def _block(N, c=0.05 * 0.4, domain="unit", eps=None):
    mesh = synth.structured_mesh(N, domain)
    if eps is None:
        prob = fem.heat_problem(mesh)
    else:
        prob = fem.double_glazing_problem(mesh, eps, synth.double_glazing_wind,
                                          synth.double_glazing_boundary(mesh))
    return (prob.M + c * prob.F).tocsr()


def test_fmix32_reference_values():
    # MurmurHash3 fmix32: fmix32(0) = 0, and the bijection is invertible
    assert amg.fmix32(0) == 0
    vals = [amg.fmix32(i) for i in range(1 << 12)]
    assert len(set(vals)) == len(vals)
    k = amg.priority_keys(5000, 2)
    assert np.all((k >> np.uint64(32)) == np.array([amg.fmix32(i ^ ((0x9E3779B9 * 3) & 0xFFFFFFFF))
                                                   for i in range(5000)], dtype=np.uint64))
    assert len(np.unique(k)) == 5000


def _dist2(G):
    G = G.astype(np.int32)
    I = sp.identity(G.shape[0], dtype=np.int32, format="csr")
    return ((I + G) @ (I + G)).tocsr()


@pytest.mark.parametrize("eps", [None, 0.005])
def test_mis2_independent_maximal(eps):
    A = _block(24, domain="unit" if eps is None else "box", eps=eps)
    G = amg.strength_graph(A, 0.08)
    assert abs(G - G.T).max() == 0
    root = amg.mis2_roots(G, 0)
    D2 = _dist2(G)
    r = np.flatnonzero(root)
    # independent: no two roots within distance 2
    sub = D2[r][:, r]
    assert sub.nnz == r.size
    # maximal: every node is within distance 2 of a root
    cover = D2[:, r].sum(axis=1).A.ravel()
    assert np.all(cover > 0)


def test_mis2_equals_parallel_rounds():
    """The greedy set equals the fixed-priority parallel rounds (select the
    undecided nodes whose key is the maximum over undecided nodes within
    distance 2; drop nodes within distance 2 of a root; repeat)."""
    A = _block(30)
    G = amg.strength_graph(A, 0.08)
    n = A.shape[0]
    key = amg.priority_keys(n, 1)
    D2 = _dist2(G)
    state = np.zeros(n, dtype=np.int8)   # 0 undecided, 1 root, 2 out
    while np.any(state == 0):
        und = state == 0
        kk = np.where(und, key, np.uint64(0))
        new = state.copy()
        for v in np.flatnonzero(und):
            nb = D2.indices[D2.indptr[v]:D2.indptr[v + 1]]
            if np.any(state[nb] == 1):
                new[v] = 2
            elif kk[nb].max() == key[v]:
                new[v] = 1
        state = new
    assert np.array_equal(state == 1, amg.mis2_roots(G, 1))


def test_aggregates_partition():
    A = _block(40)
    G = amg.strength_graph(A, 0.08)
    agg, root = amg.aggregate(G, 0)
    nc = agg.max() + 1
    assert agg.min() == 0 and np.unique(agg).size == nc == root.sum()
    # numbering by increasing root index
    assert np.array_equal(agg[np.flatnonzero(root)], np.arange(nc))
    # each aggregate is connected in the strength graph and contains its root
    for a in range(0, nc, 7):
        members = np.flatnonzero(agg == a)
        sub = G[members][:, members]
        ncomp, _ = sp.csgraph.connected_components(sub, directed=False)
        assert ncomp == 1
    sizes = np.bincount(agg)
    assert 4 <= sizes.mean() <= 16


def test_galerkin_and_hierarchy():
    A = _block(48)
    H = amg.Hierarchy(A, coarse_max=64)
    assert len(H.levels) >= 3
    for l in range(len(H.levels) - 1):
        lev, nxt = H.levels[l], H.levels[l + 1]
        Pd = lev.P.toarray()
        Ad = lev.A.toarray()
        assert np.allclose(nxt.A.toarray(), Pd.T @ Ad @ Pd, atol=1e-13 * np.abs(Ad).max())
        # P reproduces the smoothed constant: row sums of P_t are one
        assert np.allclose(np.asarray((lev.R.T - lev.P).sum()), 0)
    assert H.levels[-1].n <= 64


def test_vcycle_linear_and_convergent():
    A = _block(64)
    H = amg.Hierarchy(A)
    rng = np.random.default_rng(0)
    b1 = rng.standard_normal(A.shape[0])
    b2 = rng.standard_normal(A.shape[0])
    v = H.vcycle(2.0 * b1 - 3.0 * b2)
    assert np.allclose(v, 2.0 * H.vcycle(b1) - 3.0 * H.vcycle(b2), atol=1e-12)
    # stationary iteration x <- x + V(b - A x): contraction factor
    x = np.zeros_like(b1)
    r0 = np.linalg.norm(b1)
    for _ in range(8):
        x = x + H.vcycle(b1 - A @ x)
    rate = (np.linalg.norm(b1 - A @ x) / r0) ** (1 / 8)
    assert rate < 0.3, rate


def test_vcycle_nonsymmetric_block():
    # double-glazing block (eps = 1/200, h = 0.01 * d_jj): still a contraction
    A, _, _ = bt.radau_iia(3)
    _, D, _ = bt.ldu(A)
    Bk = _block(64, c=0.01 * D[0, 0], domain="box", eps=1 / 200)
    H = amg.Hierarchy(Bk)
    b = np.random.default_rng(2).standard_normal(Bk.shape[0])
    x = np.zeros_like(b)
    for _ in range(10):
        x = x + H.vcycle(b - Bk @ x)
    assert np.linalg.norm(b - Bk @ x) < 1e-2 * np.linalg.norm(b)


@pytest.mark.parametrize("steps", [1, 2])
def test_prolongator_is_jacobi_power(steps):
    """P = (I - omega D^{-1} A)^steps P_t against the dense matrix power, and
    the constant vector on the aggregates stays in range: P 1_c = S^steps 1."""
    mesh = synth.structured_mesh(9)
    prob = fem.heat_problem(mesh)
    A = (prob.M + 0.01 * prob.F).tocsr()
    G = amg.strength_graph(A, 0.08)
    agg, _ = amg.aggregate(G, 0)
    nc = int(agg.max()) + 1
    P, omega = amg.smoothed_prolongator(A, agg, nc, steps)
    Ad = A.toarray()
    S = np.eye(A.shape[0]) - omega * Ad / np.diag(Ad)[:, None]
    Pt = np.zeros((A.shape[0], nc))
    Pt[np.arange(A.shape[0]), agg] = 1.0
    ref = np.linalg.matrix_power(S, steps) @ Pt
    assert np.abs(P.toarray() - ref).max() <= 1e-14
    assert omega == 4.0 / (3.0 * amg.spectral_radius_estimate(A))
    # the estimate is a lower bound of rho(D^{-1} A) for this symmetric block,
    # within 3 % after 20 steps
    rho = np.max(np.abs(np.linalg.eigvals(Ad / np.diag(Ad)[:, None])))
    assert 0.97 * rho <= 4.0 / (3.0 * omega) <= rho * (1 + 1e-12)


def test_power_start_vector():
    """+-1 entries from the lowest bit of fmix32(i ^ 0x68E31DA4), balanced."""
    x = amg.power_start_vector(4096)
    assert set(np.unique(x)) == {-1.0, 1.0}
    ref = np.array([1.0 if amg.fmix32(i ^ 0x68E31DA4) & 1 else -1.0 for i in range(4096)])
    assert np.array_equal(x, ref)
    assert abs(x.sum()) < 4 * np.sqrt(4096)


def test_spectral_radius_estimate_closed_forms():
    """The power-iteration estimate of rho(D^{-1} A) against closed forms:
    the 1-D Laplacian tridiag(-1, 2, -1) of size n has rho(D^{-1} A) =
    1 + cos(pi/(n+1)); a scaled diagonal matrix has D^{-1} A = I; a 2x2 block
    with a large diagonal spread has rho = 1 + |b|/sqrt(a c), which the
    unscaled norm ratio ||D^{-1} A x|| / ||x|| overshoots and the symmetric
    scaling does not."""
    for n in (6, 12):
        T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
        rho = 1 + np.cos(np.pi / (n + 1))
        est = amg.spectral_radius_estimate(T)
        assert est <= rho * (1 + 1e-14)
        assert est >= rho * (1 - 1e-2)
        assert abs(amg.spectral_radius_estimate(T, steps=400) - rho) < 1e-12
    Dm = sp.diags(np.linspace(1.0, 50.0, 9)).tocsr()
    assert abs(amg.spectral_radius_estimate(Dm) - 1.0) < 1e-15
    a, bb, c = 100.0, -1.0, 0.01
    B = sp.csr_matrix(np.array([[a, bb], [bb, c]]))
    rho = 1 + abs(bb) / np.sqrt(a * c)
    assert abs(amg.spectral_radius_estimate(B, steps=60) - rho) < 1e-12
    x = np.array([1.0, 1.0])
    assert np.linalg.norm((B @ x) / B.diagonal()) / np.linalg.norm(x) > 1.5 * rho


@pytest.mark.parametrize("N", [64, 128])
@pytest.mark.parametrize("c", [0.05 * 0.4, (1 / 64) * 0.2628])
def test_vcycle_contraction_below_0_3(N, c):
    """Stationary contraction of the default V-cycle on heat blocks
    M + c K at two mesh sizes and two block coefficients (C1's and the
    s = 5 LD block of the C2 runs): below 0.3 in the energy norm, measured by
    the power iteration on the error propagator I - B A."""
    A = _block(N, c=c)
    H = amg.Hierarchy(A)
    e = np.random.default_rng(5).standard_normal(A.shape[0])
    rate = 0.0
    for _ in range(20):
        e2 = e - H.vcycle(A @ e)
        rate = np.sqrt(e2 @ (A @ e2) / (e @ (A @ e)))
        e = e2 / np.linalg.norm(e2)
    assert rate < 0.3, rate


def test_strength_on_negative_couplings():
    """The negative-coupling strength option counts only negative couplings: for a
    block with nonpositive off-diagonals it equals the |a_ij| graph; positive
    off-diagonal entries (as in quadratic elements) are never strong; a P2
    stiffness-dominated block has positive entries, so the two graphs differ."""
    A = _block(11)
    Ap = (A - sp.diags(A.diagonal())).tocsr()
    Ap.data = np.minimum(Ap.data, 0.0)            # an M-matrix with the same diagonal
    M = (Ap + sp.diags(A.diagonal())).tocsr()
    Gn = amg.strength_graph(M, 0.08, negative=True)
    Ga = amg.strength_graph(M, 0.08, negative=False)
    assert (Gn != Ga).nnz == 0
    Pos = (abs(Ap) + sp.diags(A.diagonal())).tocsr()  # the same magnitudes, all positive
    assert amg.strength_graph(Pos, 0.08, negative=True).nnz == 0
    assert amg.strength_graph(Pos, 0.08, negative=False).nnz == Ga.nnz
    mesh = synth.structured_mesh_p2(6)
    K = fem.heat_problem_p2(mesh).F
    assert (K > 0).sum() > K.shape[0]                # positive off-diagonals exist
    assert (amg.strength_graph(K, 0.08, True) != amg.strength_graph(K, 0.08, False)).nnz > 0


def test_streamline_matrix_closed_forms():
    """The streamline-diffusion matrix of the coarse-level SUPG stabilisation:
    symmetric, positive semidefinite, annihilates constants; for the uniform
    wind w = (1, 0) on the structured mesh with every element at Peclet > 1,
    h_e = h and the slope is h/2, so for u = x^2 at an interior node
    (T u)_i = (h/2) int 2x d(phi_i)/dx = -(h/2) 2 int phi_i = -h^3; with a
    large eps (every Peclet number below 1) T vanishes."""
    mesh = synth.structured_mesh(10)
    wind = lambda x, y: (np.ones_like(x), np.zeros_like(y))   # noqa: E731
    T = fem.streamline_matrix(mesh, 1e-4, lambda x, y: np.stack(wind(x, y), axis=-1))
    assert abs(T - T.T).max() <= 1e-15
    assert np.abs(T @ np.ones(T.shape[0])).max() <= 1e-15
    h = 1.0 / 10
    x = mesh.xy[:, 0]
    Tu = T @ (x ** 2)
    inner = np.flatnonzero(~mesh.boundary)
    assert np.allclose(Tu[inner], -h ** 3, rtol=1e-12, atol=0)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(T.shape[0])
    assert v @ (T @ v) >= 0.0
    T0 = fem.streamline_matrix(mesh, 10.0, lambda x, y: np.stack(wind(x, y), axis=-1))
    assert T0.nnz == 0 or abs(T0).max() == 0.0


def _dg_supg(N, eps):
    mesh = synth.structured_mesh(N, "box")
    return mesh, fem.double_glazing_supg_nitsche(mesh, eps, synth.double_glazing_wind,
                                                  synth.double_glazing_boundary(mesh))


def test_stabilised_hierarchy_adds_psd_streamline_diffusion():
    """Each stabilised coarse level differs from the Galerkin product of the
    level above by a positive semidefinite term (the projected streamline
    diffusion times c (f_l - f_{l-1}) > 0); without T the hierarchy is the
    plain one."""
    mesh, prob = _dg_supg(48, 0.005)
    c = 0.3
    Bk = (prob.M + c * prob.F).tocsr()
    Hs = amg.Hierarchy(Bk, coarse_max=64, p_smooth=1, stab=(prob.T, c))
    Hp = amg.Hierarchy(Bk, coarse_max=64, p_smooth=1)
    assert Hp.sizes()[0] == Hs.sizes()[0] and len(Hs.levels) >= 3
    rng = np.random.default_rng(2)
    for l in range(1, len(Hs.levels)):
        up, lev = Hs.levels[l - 1], Hs.levels[l]
        D = (lev.A - up.R @ up.A @ up.P).toarray()
        D = 0.5 * (D + D.T)
        assert np.linalg.eigvalsh(D).min() >= -1e-12 * np.abs(D).max()
        assert np.abs(D).max() > 0.0
    Hn = amg.Hierarchy(Bk, coarse_max=64, p_smooth=1, stab=None)
    for a, b in zip(Hn.levels, Hp.levels):
        assert abs(a.A - b.A).max() == 0.0


def test_stabilisation_restores_convergence_on_convection_dominated_blocks():
    """The paper's double-glazing time-step table (Table 13) at h_x^-1 = 128,
    eps = 0.005, s = 2, h_t = 1: the paper's preconditioned GMRES converges in
    11 iterations with its stabilised AMG; the oracle's left GMRES with P_LD and
    the stabilised V-cycle (Chebyshev degree 8 on [0.3, 1], V(2,2)) converges
    within 40, and the unstabilised V-cycle does not within 100."""
    from oracle import irk
    mesh, prob = _dg_supg(256, 0.005)
    A, b, _ = bt.radau_iia(2)
    opts = dict(cheb_lo=0.3, cheb_degree=8, nu_pre=2, nu_post=2, p_smooth=1)
    kstar = synth.random_stage_block(prob.n, 2, 2128)
    op = lambda z: irk.apply_operator(prob.M, prob.F, A, 1.0, z)   # noqa: E731
    rhs = op(kstar)
    pc = irk.BlockPreconditioner(prob.M, prob.F, A, 1.0, "LD", "amg", amg_opts=opts, stab=prob.T)
    res = irk.gmres_left(op, pc.apply, rhs, rtol=1e-8, max_it=40)
    assert res.converged, res.iterations
    assert np.linalg.norm(res.x - kstar) <= 1e-6 * np.linalg.norm(kstar)
    pc0 = irk.BlockPreconditioner(prob.M, prob.F, A, 1.0, "LD", "amg", amg_opts=opts)
    assert not irk.gmres_left(op, pc0.apply, rhs, rtol=1e-8, max_it=100).converged


def _energy_rate(A, solve, iters=30, seed=1):
    """Asymptotic energy-norm contraction of x <- x + B(b - A x): power
    iteration on the error propagator I - B A."""
    e = np.random.default_rng(seed).standard_normal(A.shape[0])
    rate = 0.0
    for _ in range(iters):
        e2 = e - solve(A @ e)
        rate = np.sqrt(e2 @ (A @ e2) / (e @ (A @ e)))
        e = e2 / np.linalg.norm(e2)
    return rate


def test_coarse_w_cycle_reduces_to_the_v_cycle_on_three_levels():
    """With three levels the only level below the finest has the coarsest as
    its next level, so the W-cycle below the finest level is the V-cycle,
    operation for operation."""
    A = _block(48, c=1.0)
    HV = amg.Hierarchy(A, coarse_max=64)
    HW = amg.Hierarchy(A, coarse_max=64, cycle="Wc")
    assert len(HV.sizes()) == 3, HV.sizes()
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    assert np.array_equal(HV.vcycle(b), HW.vcycle(b))
    with pytest.raises(ValueError):
        amg.Hierarchy(A, cycle="F")


def test_coarse_w_cycle_is_symmetric_positive_definite():
    """Pre- and post-smoothing by the same Chebyshev polynomial and a
    coarse-grid correction applied twice with a symmetric coarse cycle give a
    symmetric preconditioner, positive definite on an SPD block: the dense
    matrix of the cycle on a four-level hierarchy (built column by column)."""
    A = _block(24, c=1.0)
    H = amg.Hierarchy(A, coarse_max=8, cycle="Wc")
    assert len(H.sizes()) >= 4, H.sizes()
    n = A.shape[0]
    Bm = np.column_stack([H.vcycle(np.eye(n)[:, i]) for i in range(n)])
    assert np.max(np.abs(Bm - Bm.T)) <= 1e-12 * np.max(np.abs(Bm))
    assert np.min(np.linalg.eigvalsh(0.5 * (Bm + Bm.T))) > 0.0
    # the second correction changes the operator (the coarse cycle is inexact)
    HV = amg.Hierarchy(A, coarse_max=8)
    BV = np.column_stack([HV.vcycle(np.eye(n)[:, i]) for i in range(n)])
    assert np.max(np.abs(Bm - BV)) > 1e-6 * np.max(np.abs(BV))


def test_coarse_w_cycle_reaches_the_two_grid_rate():
    """On a stiffness-dominated heat block (M + K, 192^2, four levels) the
    V-cycle's energy contraction falls well short of the two-grid method's
    (level 1 solved exactly by sparse LU), and the W-cycle below the finest
    level comes within 5 % of the two-grid rate."""
    import scipy.sparse.linalg as spla
    A = _block(192, c=1.0)
    HV = amg.Hierarchy(A, coarse_max=128)
    HW = amg.Hierarchy(A, coarse_max=128, cycle="Wc")
    assert len(HV.sizes()) == 4, HV.sizes()
    lev = HV.levels[0]
    lu = spla.splu(HV.levels[1].A.tocsc())

    def two_grid(b):
        x = HV.smooth(lev, b, np.zeros_like(b))
        x = x + lev.P @ lu.solve(lev.R @ (b - lev.A @ x))
        return HV.smooth(lev, b, x)

    tg = _energy_rate(A, two_grid)
    v = _energy_rate(A, HV.vcycle)
    w = _energy_rate(A, HW.vcycle)
    assert v > 1.2 * tg, (v, tg)
    assert w < 1.05 * tg, (w, tg)
