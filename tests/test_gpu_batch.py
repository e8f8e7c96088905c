"""Batched uneven instances in one graph launch (forward and checkpointed
adjoint) against per-instance runs and the oracle."""
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_batch_matches_single_and_oracle():
    from paper_2010_11377_gb300 import binding as B
    from paper_2010_11377_gb300 import problems
    s, h, nsteps, every = 3, 1 / 32, 6, 2
    sizes = [12, 20, 28, 37]
    A, b, c = B.irk_butcher_table("radau_iia", s)
    ctxs, u0s, uNs, cks, lams, grads, meta = [], [], [], [], [], [], []
    for i, N in enumerate(sizes):
        mesh = synth.structured_mesh(N)
        kap = np.exp(synth.grf_log_kappa(mesh, seed=i))
        p = problems.heat(N, kappa=kap)
        ctx = B.irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, mesh=p["mesh_arrays"])
        u0 = synth.random_smooth_u0(mesh, seed=i)
        ctxs.append(ctx)
        u0s.append(dev(u0))
        uNs.append(torch.empty(mesh.n, dtype=torch.float64, device="cuda"))
        cks.append(torch.empty(nsteps // every, mesh.n, dtype=torch.float64, device="cuda"))
        lams.append(torch.empty(mesh.n, dtype=torch.float64, device="cuda"))
        grads.append(torch.zeros(mesh.n_tri, dtype=torch.float64, device="cuda"))
        meta.append((mesh, kap, u0))
    batch = B.irk_batch_create(ctxs, nsteps, every, u0s, uNs, cks, lams, grads)
    stats, ms = B.irk_batch_run(batch)
    assert all(st["steps"] == nsteps and st["resid"] <= 1e-10 for st in stats)
    # per-instance runs give the same states and checkpoints
    for q, ctx in enumerate(ctxs):
        uN = torch.empty_like(uNs[q])
        ck = torch.empty_like(cks[q])
        B.irk_run(ctx, u0s[q], nsteps, uN, ckpt=ck, ckpt_every=every)
        assert torch.allclose(uN, uNs[q], rtol=0, atol=1e-14 * float(uN.abs().max()))
        assert torch.allclose(ck, cks[q], rtol=0, atol=1e-14 * float(ck.abs().max()))
    # oracle for the largest instance
    mesh, kap, u0 = meta[-1]
    prob = ofem.heat_problem(mesh, kappa=kap)
    OA, Ob, _ = obt.radau_iia(s)
    refs, _ = oirk.IRKSolver(prob, OA, Ob, h, kind=None).run(u0, nsteps, direct=True)
    got = uNs[-1].cpu().numpy()
    assert np.linalg.norm(got - refs[-1]) <= 1e-8 * np.linalg.norm(refs[-1])
    # adjoint of the misfit 1/2 (u_N - d)^T M (u_N - d), d = 0.5 u0
    seeds = []
    for q, ctx in enumerate(ctxs):
        d = 0.5 * u0s[q]
        Me = torch.empty_like(uNs[q])
        B.irk_apply_mass(ctx, (uNs[q] - d).contiguous(), Me)
        lams[q].copy_(Me)
        seeds.append(Me.clone())
    astats, ams = B.irk_batch_adjoint(batch)
    for q, ctx in enumerate(ctxs):
        lam = seeds[q].clone()
        g = torch.zeros_like(grads[q])
        B.irk_adjoint_run(ctx, cks[q], nsteps, every, lam, g)
        assert torch.allclose(lam, lams[q], rtol=0, atol=1e-13 * float(lam.abs().max()))
        assert torch.allclose(g, grads[q], rtol=0, atol=1e-13 * float(g.abs().max()))
    Ke = ofem.element_stiffness_unit(mesh.xy, mesh.tri)
    sol = oirk.IRKSolver(prob, OA, Ob, h, kind="LD", subsolve="direct")
    gu, gk, _ = oirk.adjoint_gradients(sol, Ke, mesh.dof[mesh.tri], u0, nsteps, 0.5 * u0, direct=True)
    assert np.linalg.norm(lams[-1].cpu().numpy() - gu) <= 1e-8 * np.linalg.norm(gu)
    assert np.linalg.norm(grads[-1].cpu().numpy() - gk) <= 1e-8 * np.linalg.norm(gk)
    batch.close()
    for ctx in ctxs:
        ctx.close()
