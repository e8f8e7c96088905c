"""Full-size parity in the benchmark's launch configuration (default options,
graph-launched step): the stage residual and the update are checked with the
oracle's own operator on every row (the oracle cannot solve these sizes in
test time, but the residual and the update fix the answer at any size)."""
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
