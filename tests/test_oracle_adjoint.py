"""Pins for the oracle's discrete adjoint: the transpose identity and the
gradients against central finite differences."""
import numpy as np

import synth
from oracle import butcher as bt
from oracle import fem
from oracle import irk


def test_transpose_dot_product():
    mesh = synth.structured_mesh(6, "box")
    prob = fem.double_glazing_problem(mesh, 0.01, synth.double_glazing_wind,
                                      synth.double_glazing_boundary(mesh))
    A, b, _ = bt.radau_iia(3)
    sol = irk.IRKSolver(prob, A, b, 0.03, kind=None)
    x = synth.random_stage_block(prob.n, 3, 1)
    y = synth.random_stage_block(prob.n, 3, 2)
    lhs = np.sum(sol.op(x) * y)
    rhs = np.sum(x * sol.opT(y))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def _setup(N=6, s=3, nsteps=3, seed=0):
    mesh = synth.structured_mesh(N)
    logk = synth.grf_log_kappa(mesh, seed=seed)
    kap = np.exp(logk)
    A, b, _ = bt.radau_iia(s)
    u0 = synth.random_smooth_u0(mesh, seed=seed)
    d = 0.5 * u0
    return mesh, kap, A, b, u0, d


def _loss(mesh, kap, A, b, u0, d, h, nsteps):
    prob = fem.heat_problem(mesh, kappa=kap)
    sol = irk.IRKSolver(prob, A, b, h, kind=None)
    us, _ = sol.run(u0, nsteps, direct=True)
    return irk.misfit(prob.M, us[-1], d)


def test_gradients_vs_finite_differences():
    mesh, kap, A, b, u0, d = _setup()
    h, nsteps = 1 / 32, 3
    prob = fem.heat_problem(mesh, kappa=kap)
    sol = irk.IRKSolver(prob, A, b, h, kind="LD", subsolve="direct")
    Ke = fem.element_stiffness_unit(mesh.xy, mesh.tri)
    edofs = mesh.dof[mesh.tri]
    gu, gk, L = irk.adjoint_gradients(sol, Ke, edofs, u0, nsteps, d, direct=True)
    assert abs(L - _loss(mesh, kap, A, b, u0, d, h, nsteps)) < 1e-15 + 1e-12 * L
    rng = np.random.default_rng(5)
    # directional derivatives (central differences, relative step 1e-6)
    for _ in range(3):
        dk = rng.standard_normal(kap.size) * kap
        t = 1e-6
        fd = (_loss(mesh, kap + t * dk, A, b, u0, d, h, nsteps)
              - _loss(mesh, kap - t * dk, A, b, u0, d, h, nsteps)) / (2 * t)
        assert abs(fd - gk @ dk) <= 1e-6 * abs(fd), (fd, gk @ dk)
        du = rng.standard_normal(u0.size)
        fd = (_loss(mesh, kap, A, b, u0 + t * du, d, h, nsteps)
              - _loss(mesh, kap, A, b, u0 - t * du, d, h, nsteps)) / (2 * t)
        assert abs(fd - gu @ du) <= 1e-6 * abs(fd), (fd, gu @ du)


def test_adjoint_preconditioned_matches_direct():
    mesh, kap, A, b, u0, d = _setup(N=10)
    h, nsteps = 1 / 32, 2
    prob = fem.heat_problem(mesh, kappa=kap)
    Ke = fem.element_stiffness_unit(mesh.xy, mesh.tri)
    edofs = mesh.dof[mesh.tri]
    s1 = irk.IRKSolver(prob, A, b, h, kind="LD", subsolve="amg")
    gu1, gk1, _ = irk.adjoint_gradients(s1, Ke, edofs, u0, nsteps, d, direct=False)
    s2 = irk.IRKSolver(prob, A, b, h, kind="LD", subsolve="direct")
    gu2, gk2, _ = irk.adjoint_gradients(s2, Ke, edofs, u0, nsteps, d, direct=True)
    assert np.linalg.norm(gu1 - gu2) <= 1e-8 * np.linalg.norm(gu2)
    assert np.linalg.norm(gk1 - gk2) <= 1e-8 * np.linalg.norm(gk2)
