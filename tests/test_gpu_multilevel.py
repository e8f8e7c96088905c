"""GPU steps on hierarchies of three or more levels with the library's default
AMG options, against the oracle's exact stage solves: every precision of the
preconditioner (FP64, FP32, BF16 finest level) and the operator with and
without single-float pairs; and a batch of 8 uneven instances (64^2..256^2).

Run as a script (``python tests/test_gpu_multilevel.py N steps``) it prints
the per-precision errors against the oracle as one JSON line; the test of the
FP64-product operator runs it in a child process, since that operator is
selected once per process (environment variable IRK_KRON_FF=0)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import butcher as obt  # noqa: E402
from oracle import fem as ofem  # noqa: E402
from oracle import irk as oirk  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _build():
    from paper_2010_11377_gb300.build import build
    build()
    from paper_2010_11377_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _build()


def step_errors(B, N, nsteps, precs=("f64", "f32", "bf16"), s=5, h=1 / 64, kind="LD"):
    """Heat N^2, Radau IIA s, P_kind, default options (FP32/FP64/BF16 AMG):
    relative L2 error of every step's state against the oracle's exact stage
    solves, the iteration counts and the hierarchy sizes of the first block."""
    from paper_2010_11377_gb300 import problems
    mesh = synth.structured_mesh(N)
    prob = ofem.heat_problem(mesh)
    A, b, _ = obt.radau_iia(s)
    refs, _ = oirk.IRKSolver(prob, A, b, h, kind=None).run(synth.heat_u0(mesh), nsteps, direct=True)
    p = problems.heat(N)
    At, bt, ct = B.irk_butcher_table("radau_iia", s)
    out = {}
    for prec in precs:
        o = B.irk_default_options(kind=kind, amg_prec=prec)
        ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (At, bt, ct), h, options=o)
        u = torch.tensor(refs[0], dtype=torch.float64, device="cuda")
        errs, its = [], []
        for t in range(nsteps):
            nxt = torch.empty_like(u)
            st = B.irk_step(ctx, u, nxt)
            got = nxt.cpu().numpy()
            errs.append(float(np.linalg.norm(got - refs[t + 1]) / np.linalg.norm(refs[t + 1])))
            its.append(st["iterations"])
            u = nxt
        rows, _ = B.irk_amg_info(ctx, 0)
        out[prec] = {"errors": errs, "iterations": its, "levels": rows}
        ctx.close()
    return out


@pytest.mark.parametrize("N", [128])
def test_multilevel_steps_against_exact_solve(B, N):
    """128^2 heat, s = 5, LD, default options: the finest block coarsens over
    at least three levels, and every step in every preconditioner precision is
    within 1e-8 of the exact stage solve."""
    res = step_errors(B, N, 3)
    for prec, r in res.items():
        assert len(r["levels"]) >= 3, (prec, r["levels"])
        assert max(r["errors"]) <= 1e-8, (prec, r)
    # the oracle's FGMRES with the same AMG reading takes as many iterations
    mesh = synth.structured_mesh(N)
    prob = ofem.heat_problem(mesh)
    A, b, _ = obt.radau_iia(5)
    oits = oirk.IRKSolver(prob, A, b, 1 / 64, kind="LD", subsolve="amg").step(synth.heat_u0(mesh)).iterations
    got = res["f64"]["iterations"][0]
    assert abs(got - oits) <= max(1, int(np.ceil(0.1 * oits))), (got, oits)


def test_mesh_independent_counts_in_the_paper_time_step_scaling(B):
    """h_x-independence (Section 5.1, Table 5) from 256^2 to 1024^2 with the
    time step tied to the mesh as in the paper, h_t = h_x^((p+1)/(2s-1)) with
    p = 1 (P1), s = 5, rtol 1e-10, FP32 AMG.  These blocks are
    stiffness-dominated, and the V-cycle's contraction degrades with the
    number of levels: its LD count grows by more than 2.  With the W-cycle
    below the finest level (the two-grid rate) the LD count differs by at most
    2, GSL and DU by at most 10 %, and block Jacobi, whose 67+ iterations
    restart FGMRES(30) twice, grows by less than with the V-cycle.  At 256^2
    the LD count is within 10 % of the oracle's FGMRES with the same AMG
    reading."""
    from paper_2010_11377_gb300 import problems
    s = 5
    A, b, c = B.irk_butcher_table("radau_iia", s)
    counts = {}
    for N in (256, 1024):
        p = problems.heat(N)
        h = (1.0 / N) ** (2.0 / (2 * s - 1))
        u0 = torch.tensor(synth.heat_u0(p["mesh"]), dtype=torch.float64, device="cuda")
        for kind in ("J", "GSL", "DU", "LD"):
            for cyc in ("V", "Wc"):
                o = B.irk_default_options(kind=kind, cycle=cyc)
                ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, options=o, g=p["g"])
                out = torch.empty_like(u0)
                st = B.irk_step(ctx, u0, out)
                assert st["resid"] <= 1e-10
                counts[(N, kind, cyc)] = st["iterations"]
                ctx.close()

    def growth(kind, cyc):
        return counts[(1024, kind, cyc)] - counts[(256, kind, cyc)]

    assert abs(growth("LD", "Wc")) <= 2, counts
    for kind in ("GSL", "DU"):
        assert abs(growth(kind, "Wc")) <= max(2, int(np.ceil(0.1 * counts[(256, kind, "Wc")]))), (kind, counts)
    assert growth("LD", "V") > 2, counts
    assert growth("J", "Wc") < growth("J", "V"), counts
    mesh = synth.structured_mesh(256)
    prob = ofem.heat_problem(mesh)
    OA, Ob, _ = obt.radau_iia(s)
    h = (1.0 / 256) ** (2.0 / (2 * s - 1))
    oits = oirk.IRKSolver(prob, OA, Ob, h, kind="LD", subsolve="amg",
                          amg_opts=dict(cycle="Wc")).step(synth.heat_u0(mesh)).iterations
    got = counts[(256, "LD", "Wc")]
    assert abs(got - oits) <= max(1, int(np.ceil(0.1 * oits))), (got, oits)


def test_coarse_w_cycle_through_step_adjoint_and_batch(B):
    """The W-cycle below the finest level on the library's whole paths: heat
    97^2 with the coarsest level at most 16 rows (four or more levels),
    h_t = 4 (stiffness-dominated blocks), Radau IIA s = 3, P_LD, FP32 AMG.  A
    step within 1e-8 of the oracle's exact stage solve and its iteration count
    within 10 % of the oracle's FGMRES with the same cycle; an adjoint step
    within 1e-8 of the oracle's exact one; a batch of two instances (61^2 and
    97^2) equal to the per-instance runs."""
    from paper_2010_11377_gb300 import problems
    s, h, nsteps, every = 3, 4.0, 4, 2
    A, b, c = B.irk_butcher_table("radau_iia", s)
    OA, Ob, _ = obt.radau_iia(s)
    opts = dict(kind="LD", cycle="Wc", coarse_max=16)
    ctxs, meshes = [], []
    for N in (61, 97):
        p = problems.heat(N)
        ctxs.append(B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h,
                                options=B.irk_default_options(**opts), g=p["g"]))
        meshes.append(p["mesh"])
    ctx, mesh = ctxs[1], meshes[1]
    rows, _ = B.irk_amg_info(ctx, 0)
    assert len(rows) >= 4, rows
    prob = ofem.heat_problem(mesh)
    u0 = synth.heat_u0(mesh)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    st = B.irk_step(ctx, u, out)
    assert st["resid"] <= 1e-10
    ref = oirk.IRKSolver(prob, OA, Ob, h, kind=None).step(u0, direct=True).u
    assert np.linalg.norm(out.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    oits = oirk.IRKSolver(prob, OA, Ob, h, kind="LD", subsolve="amg",
                          amg_opts=dict(cycle="Wc", coarse_max=16)).step(u0).iterations
    assert abs(st["iterations"] - oits) <= max(1, int(np.ceil(0.1 * oits))), (st["iterations"], oits)
    lam1 = synth.random_smooth_u0(mesh, seed=3)
    lam = torch.empty_like(u)
    B.irk_adjoint_step(ctx, torch.tensor(lam1, dtype=torch.float64, device="cuda"), None, None, lam)
    ref_lam, _ = oirk.IRKSolver(prob, OA, Ob, h, kind=None).adjoint_step(lam1, direct=True)
    assert np.linalg.norm(lam.cpu().numpy() - ref_lam) <= 1e-8 * np.linalg.norm(ref_lam)
    u0s = [torch.tensor(synth.heat_u0(m), dtype=torch.float64, device="cuda") for m in meshes]
    uNs = [torch.empty_like(x) for x in u0s]
    cks = [torch.empty(nsteps // every, m.n, dtype=torch.float64, device="cuda") for m in meshes]
    batch = B.irk_batch_create(ctxs, nsteps, every, u0s, uNs, cks)
    stats, _ = B.irk_batch_run(batch)
    assert all(x["steps"] == nsteps and x["resid"] <= 1e-10 for x in stats)
    for q, cq in enumerate(ctxs):
        uN = torch.empty_like(uNs[q])
        B.irk_run(cq, u0s[q], nsteps, uN)
        assert torch.allclose(uN, uNs[q], rtol=0, atol=1e-14 * float(uN.abs().max()))
    batch.close()
    for cq in ctxs:
        cq.close()


def test_operator_without_pairs_child_process(B):
    """The FP32-AMG step with the operator in FP64 products (IRK_KRON_FF=0, a
    child process) is within 1e-8 of the exact solve, like the pair operator."""
    env = dict(os.environ, IRK_KRON_FF="0")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "96", "2", "f32"], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert max(res["f32"]["errors"]) <= 1e-8, res


def test_batch_of_eight_64_to_256(B):
    """8 uneven heat instances, 64^2..256^2, s = 3, h = 1/32, 8 steps,
    checkpoints every 4: one graph launch equals the per-instance runs bit for
    bit and the largest instance is within 1e-8 of the oracle's exact solves."""
    from paper_2010_11377_gb300 import problems
    s, h, nsteps, every = 3, 1 / 32, 8, 4
    sizes = synth.batch_instance_sizes(8, 64, 256)
    assert sizes[0] == 64 and sizes[-1] == 256
    A, b, c = B.irk_butcher_table("radau_iia", s)
    ctxs, u0s, uNs, cks, lams, grads, meta = [], [], [], [], [], [], []
    for i, N in enumerate(sizes):
        mesh = synth.structured_mesh(N)
        kap = np.exp(synth.grf_log_kappa(mesh, seed=i))
        p = problems.heat(N, kappa=kap)
        ctxs.append(B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, mesh=p["mesh_arrays"]))
        u0 = synth.random_smooth_u0(mesh, seed=i)
        u0s.append(torch.tensor(u0, dtype=torch.float64, device="cuda"))
        uNs.append(torch.empty(mesh.n, dtype=torch.float64, device="cuda"))
        cks.append(torch.empty(nsteps // every, mesh.n, dtype=torch.float64, device="cuda"))
        lams.append(torch.empty(mesh.n, dtype=torch.float64, device="cuda"))
        grads.append(torch.zeros(mesh.n_tri, dtype=torch.float64, device="cuda"))
        meta.append((mesh, kap, u0))
    batch = B.irk_batch_create(ctxs, nsteps, every, u0s, uNs, cks, lams, grads)
    stats, _ = B.irk_batch_run(batch)
    assert all(st["steps"] == nsteps and st["resid"] <= 1e-10 for st in stats)
    for q, ctx in enumerate(ctxs):
        uN = torch.empty_like(uNs[q])
        ck = torch.empty_like(cks[q])
        B.irk_run(ctx, u0s[q], nsteps, uN, ckpt=ck, ckpt_every=every)
        assert torch.equal(uN, uNs[q]) and torch.equal(ck, cks[q]), q
    mesh, kap, u0 = meta[-1]
    prob = ofem.heat_problem(mesh, kappa=kap)
    OA, Ob, _ = obt.radau_iia(s)
    refs, _ = oirk.IRKSolver(prob, OA, Ob, h, kind=None).run(u0, nsteps, direct=True)
    got = uNs[-1].cpu().numpy()
    assert np.linalg.norm(got - refs[-1]) <= 1e-8 * np.linalg.norm(refs[-1])
    batch.close()
    for ctx in ctxs:
        ctx.close()


if __name__ == "__main__":
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 256
    nsteps = int(sys.argv[2]) if len(sys.argv) > 2 else 3
    precs = tuple(sys.argv[3].split(",")) if len(sys.argv) > 3 else ("f64", "f32", "bf16")
    print(json.dumps(step_errors(_build(), N, nsteps, precs)))
