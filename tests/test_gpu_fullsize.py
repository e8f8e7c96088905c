"""Full-size parity in the benchmark's launch configuration (default options,
graph-launched step): the stage residual and the update are checked with the
oracle's own operator on every row, and the heat step's stages and update
against the oracle's exact stage solve (the Butcher matrix diagonalised: one
sparse LU per conjugate pair of eigenvalues)."""
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


@pytest.mark.parametrize("which,N,s,h", [("heat", 1024, 5, 1 / 64), ("dg", 512, 4, 0.01)])
def test_fullsize_residual_and_update(which, N, s, h):
    from paper_2010_11377_gb300 import binding as B
    from paper_2010_11377_gb300 import problems
    p = problems.heat(N) if which == "heat" else problems.double_glazing(N, 1 / 200)
    mesh = p["mesh"]
    A, b, c = B.irk_butcher_table("radau_iia", s)
    ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, g=p["g"])
    u0 = synth.heat_u0(mesh) if which == "heat" else np.zeros(mesh.n)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    k = torch.empty(s * mesh.n, dtype=torch.float64, device="cuda")
    st = B.irk_step(ctx, u, out, k)
    kk = k.cpu().numpy().reshape(s, -1)
    un = out.cpu().numpy()
    if which == "heat":
        prob = ofem.heat_problem(mesh)
    else:
        prob = ofem.double_glazing_problem(mesh, 1 / 200, synth.double_glazing_wind,
                                           synth.double_glazing_boundary(mesh))
    OA, Ob, _ = obt.radau_iia(s)
    rhs = oirk.stage_rhs(prob.F, prob.g, u0, s)
    r = rhs - oirk.apply_operator(prob.M, prob.F, OA, h, kk)
    rel = np.linalg.norm(r) / np.linalg.norm(rhs)
    assert rel <= 1.05e-10, rel
    assert st["resid"] <= 1e-10
    ref = u0 + h * (Ob @ kk)
    assert np.max(np.abs(un - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))
    ctx.close()


def test_fullsize_heat_step_against_exact_solve():
    """Heat 1024^2, Radau IIA s = 5, h_t = 1/64, P_LD with FP32 AMG (the
    benchmark's workload and options, graph-launched step): the stages k and
    the update u_1 within 1e-8 (relative L2) of the oracle's exact stage solve,
    at rtol 1e-10."""
    from paper_2010_11377_gb300 import binding as B
    from paper_2010_11377_gb300 import problems
    N, s, h = 1024, 5, 1 / 64
    p = problems.heat(N)
    mesh = p["mesh"]
    A, b, c = B.irk_butcher_table("radau_iia", s)
    ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, g=p["g"])
    u0 = synth.heat_u0(mesh)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    k = torch.empty(s * mesh.n, dtype=torch.float64, device="cuda")
    st = B.irk_step(ctx, u, out, k)
    kk = k.cpu().numpy().reshape(s, -1)
    un = out.cpu().numpy()
    ctx.close()
    assert st["resid"] <= 1e-10
    prob = ofem.heat_problem(mesh)
    OA, Ob, _ = obt.radau_iia(s)
    kex = oirk.solve_stages_eig(prob.M, prob.F, OA, h, oirk.stage_rhs(prob.F, prob.g, u0, s))
    uex = u0 + h * (Ob @ kex)
    ek = np.linalg.norm(kk - kex) / np.linalg.norm(kex)
    eu = np.linalg.norm(un - uex) / np.linalg.norm(uex)
    print(f"heat 1024^2 s=5 FP32 AMG: {st['iterations']} iterations, resid {st['resid']:.2e}, "
          f"error k {ek:.2e}, u {eu:.2e}")
    assert ek <= 1e-8 and eu <= 1e-8, (ek, eu)
