"""torch.autograd through the C ABI: dL/dlog(kappa) and dL/du0 of the
misfit 1/2 (u_N - d)^T M (u_N - d) against the oracle's discrete adjoint."""
import numpy as np
import pytest

import synth
from oracle import butcher as obt
from oracle import fem as ofem
from oracle import irk as oirk

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11377_gb300.build import build
    build()


def test_autograd_matches_oracle_adjoint():
    from paper_2010_11377_gb300 import binding as B
    from paper_2010_11377_gb300 import problems
    from paper_2010_11377_gb300.autograd import IRKTrajectory, MassMisfit, Solver
    N, s, h, nsteps, every = 24, 3, 1 / 32, 8, 4
    mesh = synth.structured_mesh(N)
    logk = synth.grf_log_kappa(mesh, seed=7)
    u0 = synth.random_smooth_u0(mesh, seed=7)
    d = 0.3 * u0
    # oracle: exact solves
    kap = np.exp(logk)
    prob = ofem.heat_problem(mesh, kappa=kap)
    A, b, _ = obt.radau_iia(s)
    sol = oirk.IRKSolver(prob, A, b, h, kind="LD", subsolve="direct")
    Ke = ofem.element_stiffness_unit(mesh.xy, mesh.tri)
    gu, gk, L = oirk.adjoint_gradients(sol, Ke, mesh.dof[mesh.tri], u0, nsteps, d, direct=True)
    # CUDA path through autograd (kappa = exp(logk) in torch)
    p = problems.heat(N)
    At, bt, ct = B.irk_butcher_table("radau_iia", s)
    ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (At, bt, ct), h, mesh=p["mesh_arrays"])
    solver = Solver(ctx)
    lk = torch.tensor(logk, dtype=torch.float64, device="cuda", requires_grad=True)
    x0 = torch.tensor(u0, dtype=torch.float64, device="cuda", requires_grad=True)
    uN = IRKTrajectory.apply(x0, torch.exp(lk), solver, nsteps, every)
    loss = MassMisfit.apply(uN - torch.tensor(d, device="cuda"), solver)
    loss.backward()
    assert abs(loss.item() - L) <= 1e-8 * L
    assert np.linalg.norm(x0.grad.cpu().numpy() - gu) <= 1e-8 * np.linalg.norm(gu)
    glog = gk * kap
    assert np.linalg.norm(lk.grad.cpu().numpy() - glog) <= 1e-8 * np.linalg.norm(glog)
    ctx.close()


def test_misfit_entry_point():
    """irk_misfit against the oracle's misfit 1/2 (u - d)^T M (u - d) (FP64
    sum-order rounding) and its gradient M (u - d)."""
    from paper_2010_11377_gb300 import binding as B
    from paper_2010_11377_gb300 import problems
    N = 37
    mesh = synth.structured_mesh(N)
    prob = ofem.heat_problem(mesh)
    p = problems.heat(N)
    At, bt, ct = B.irk_butcher_table("radau_iia", 2)
    ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (At, bt, ct), 0.05)
    u = synth.random_smooth_u0(mesh, seed=3)
    d = 0.5 * synth.random_smooth_u0(mesh, seed=4)
    ref = oirk.misfit(prob.M, u, d)
    value = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
    ud = torch.tensor(u, device="cuda")
    dd = torch.tensor(d, device="cuda")
    B.irk_misfit(ctx, ud, dd, value, grad=grad)
    assert abs(value.item() - ref) <= 1e-13 * abs(ref)
    assert np.abs(grad.cpu().numpy() - prob.M @ (u - d)).max() <= 1e-14 * np.abs(prob.M @ (u - d)).max()
    B.irk_misfit(ctx, ud, dd, value)           # without the gradient
    assert abs(value.item() - ref) <= 1e-13 * abs(ref)
    ctx.close()
