"""Every V-cycle operator layout (SELL-32, sliced SELL with 2, 4 and 8 threads
per row, CSR with 4 lanes per row) against the oracle's V-cycle and the exact
stage solve.  The layout autotuner picks one per operator shape at run time;
IRK_LAYOUT forces one for the whole process, so each layout runs in a child
process (``python tests/test_gpu_layouts.py`` prints its errors)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import amg as oamg  # noqa: E402
from oracle import butcher as obt  # noqa: E402
from oracle import fem as ofem  # noqa: E402
from oracle import irk as oirk  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def layout_errors():
    """FP64 V-cycles of both diagonal blocks of a 61^2 heat problem (s = 2,
    coarse_max 256: three levels, rows of 7 to ~80 entries) against the
    oracle's, and one FP32-AMG step against the exact stage solve."""
    from paper_2010_11377_gb300.build import build
    build()
    from paper_2010_11377_gb300 import binding as B
    mesh = synth.structured_mesh(61)
    prob = ofem.heat_problem(mesh)
    A, b, _ = obt.radau_iia(2)
    h = 0.05
    At = obt.atilde(A, "LD")
    M = prob.M.tocsr()
    M.sort_indices()
    coo = M.tocoo()
    Fv = np.asarray(prob.F.tocsr()[coo.row, coo.col]).ravel()
    opts = dict(theta=0.08, coarse_max=256, smoother="chebyshev", cheb_degree=4, cheb_lo=0.1)
    out = {"vcycle": [], "step": None, "levels": None}
    for prec in ("f64", "f32"):
        At_c = np.ascontiguousarray(At)
        o = B.irk_default_options(kind="CUSTOM", amg_prec=prec, **opts)
        o.Atilde = At_c.ctypes.data_as(B._abi.c_double_p)
        ctx = B.irk_setup(M.indptr.astype(np.int64), M.indices, M.data, Fv, (A, b, np.zeros(2)), h, options=o)
        if prec == "f64":
            rhs = synth.random_stage_block(prob.n, 1, 3)[0]
            for stage in range(2):
                Bk = (prob.M + (h * At[stage, stage]) * prob.F).tocsr()
                ref = oamg.Hierarchy(Bk, **opts).vcycle(rhs)
                x = torch.empty(prob.n, dtype=torch.float64, device="cuda")
                B.irk_vcycle(ctx, stage, torch.tensor(rhs, device="cuda"), x)
                out["vcycle"].append(float(np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)))
            out["levels"] = B.irk_amg_info(ctx, 0)[0]
        else:
            u0 = synth.heat_u0(mesh)
            ref = oirk.IRKSolver(prob, A, b, h, kind=None).step(u0, direct=True).u
            u = torch.tensor(u0, device="cuda")
            nxt = torch.empty_like(u)
            B.irk_step(ctx, u, nxt)
            out["step"] = float(np.linalg.norm(nxt.cpu().numpy() - ref) / np.linalg.norm(ref))
        ctx.close()
    return out


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("layout,pattern", [(1, "1"), (1, "0"), (-2, "1"), (-4, "1"), (-8, "1"), (4, "1")])
def test_layout_against_oracle(gpu, layout, pattern):
    """pattern "0": SELL-32 reads every entry's own column offset instead of the
    shared per-slice pattern (IRK_SLICE_PATTERN=0)."""
    env = dict(os.environ, IRK_LAYOUT=str(layout), IRK_SLICE_PATTERN=pattern)
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res["levels"]) >= 3, res
    assert max(res["vcycle"]) <= 1e-12, (layout, res)
    assert res["step"] <= 1e-8, (layout, res)


if __name__ == "__main__":
    print(json.dumps(layout_errors()))
