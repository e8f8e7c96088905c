"""GPU parity: libirk (through the C ABI) against the FP64 oracle on the same
seeded inputs.  Sizes span several 32-row slices with a ragged tail."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import amg as oamg
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


def B():
    from paper_2010_11377_gb300 import binding
    return binding


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def oracle_ctx(prob, A, kind, h, amg_prec="f64", mesh=None, b=None, **opt):
    """GPU context on the oracle's own matrices, Butcher table and A~ (so both
    sides start from bit-identical data)."""
    bnd = B()
    At = obt.atilde(A, kind)
    M = prob.M.tocsr()
    M.sort_indices()
    F = M.copy()
    coo = M.tocoo()
    # F on the pattern of M (scipy drops exact zeros from sums such as eps K + C)
    F.data = np.asarray(prob.F.tocsr()[coo.row, coo.col]).ravel()
    At_c = np.ascontiguousarray(At, dtype=np.float64)
    o = bnd.irk_default_options(kind="CUSTOM", amg_prec=amg_prec, **opt)
    o.Atilde = At_c.ctypes.data_as(bnd._abi.c_double_p)
    bw = A[-1].copy() if b is None else b
    # a SUPG problem's streamline matrix (coarse-level stabilisation) on the same pattern
    T = getattr(prob, "T", None)
    stab = None if T is None else np.asarray(T.tocsr()[coo.row, coo.col]).ravel()
    ctx = bnd.irk_setup(M.indptr.astype(np.int64), M.indices, M.data, F.data,
                        (A, bw, np.zeros(A.shape[0])), h, options=o, g=prob.g, mesh=mesh, stab=stab)
    ctx._keep = At_c
    return ctx, At


def heat(N, kappa=None):
    mesh = synth.structured_mesh(N)
    return mesh, ofem.heat_problem(mesh, kappa=kappa)


def dg(N, eps=1 / 200):
    mesh = synth.structured_mesh(N, "box")
    return mesh, ofem.double_glazing_problem(mesh, eps, synth.double_glazing_wind,
                                             synth.double_glazing_boundary(mesh))


AMG_OPTS = dict(theta=0.08, coarse_max=256, smoother="chebyshev", cheb_degree=3, cheb_lo=0.1)


def oracle_amg_opts():
    return dict(theta=0.08, coarse_max=256, smoother="chebyshev", cheb_degree=3, cheb_lo=0.1)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s", [1, 3, 7, 8])
def test_operator_parity(s):
    mesh, prob = heat(41)
    A, _, _ = obt.radau_iia(s)
    h = 1 / 64
    ctx, _ = oracle_ctx(prob, A, "LD" if s > 1 else "J", h)
    z = synth.random_stage_block(prob.n, s, 11)
    for tr in (False, True):
        w = torch.empty(s * prob.n, dtype=torch.float64, device="cuda")
        B().irk_apply_operator(ctx, dev(z.ravel()), w, transpose=tr)
        Am = A.T if tr else A
        ref = oirk.apply_operator(prob.M, prob.F, Am, h, z)
        err = np.max(np.abs(host(w).reshape(s, -1) - ref)) / np.max(np.abs(ref))
        assert err < 1e-14, err
    x = synth.random_stage_block(prob.n, 1, 3)[0]
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    B().irk_apply_mass(ctx, dev(x), y)
    assert np.max(np.abs(host(y) - prob.M @ x)) < 1e-15 * np.max(np.abs(x))


@pytest.mark.parametrize("s", [1, 3, 5, 8])
def test_operator_f32_parity(s):
    """The operator on FP32 vectors (the FGMRES product on FP32 preconditioner
    outputs), computed in single-float pairs: against the oracle in FP64 on the
    same (exactly widened) input.  Each term of a row carries at most 2^-47 of
    its size (split of the FP64 entry plus the rounded low product), and the
    float tail of the accumulator adds at most one 2^-24 rounding of itself per
    term; with at most 16 terms per row (nonzeros plus stages) the bound is
    16^2 2^-48 = 2^-40 of the row's sum of absolute terms."""
    mesh, prob = heat(41)
    A, _, _ = obt.radau_iia(s)
    h = 1 / 64
    ctx, _ = oracle_ctx(prob, A, "LD" if s > 1 else "J", h, amg_prec="f32")
    z32 = synth.random_stage_block(prob.n, s, 12).astype(np.float32)
    z = z32.astype(np.float64)
    zd = torch.tensor(z32.ravel(), device="cuda")
    for tr in (False, True):
        w = torch.empty(s * prob.n, dtype=torch.float64, device="cuda")
        B().irk_apply_operator_f32(ctx, zd, w, transpose=tr)
        Am = A.T if tr else A
        ref = oirk.apply_operator(prob.M, prob.F, Am, h, z)
        absref = oirk.apply_operator(abs(prob.M), abs(prob.F), np.abs(Am), h, np.abs(z))
        err = np.abs(host(w).reshape(s, -1) - ref)
        assert np.all(err <= 2.0 ** -40 * absref), (err / absref).max()
        w64 = torch.empty_like(w)
        B().irk_apply_operator(ctx, dev(z.ravel()), w64, transpose=tr)
        # the FP64 product on the same input, to the same bound
        assert np.all(np.abs(host(w) - host(w64)).reshape(s, -1) <= 2.0 ** -40 * absref)


def test_operator_f32_range_fallback():
    """Matrix entries below 2^-64 (here M and F scaled by 2^-80) keep the FP32
    input product in FP64: bit-identical to the FP64 operator on the widened
    input.  At unit scale the single-float pair product is the one that runs
    (it rounds differently somewhere, within the same bound)."""
    mesh, prob = heat(33)
    A, _, _ = obt.radau_iia(3)
    h = 1 / 64
    z32 = synth.random_stage_block(prob.n, 3, 13).astype(np.float32)
    zd = torch.tensor(z32.ravel(), device="cuda")
    z64 = dev(z32.astype(np.float64).ravel())
    for scale, same in ((2.0 ** -80, True), (1.0, False)):
        scaled = ofem.Problem((prob.M * scale).tocsr(), (prob.F * scale).tocsr(), prob.g, mesh)
        ctx, _ = oracle_ctx(scaled, A, "LD", h, amg_prec="f32")
        w32 = torch.empty(3 * prob.n, dtype=torch.float64, device="cuda")
        w64 = torch.empty_like(w32)
        B().irk_apply_operator_f32(ctx, zd, w32)
        B().irk_apply_operator(ctx, z64, w64)
        assert torch.equal(w32, w64) == same, scale
        ctx.close()


@pytest.mark.parametrize("which", ["heat", "dg"])
@pytest.mark.parametrize("p_smooth,strength", [(1, 0), (2, 1), (2, 0), (3, 0)])
def test_aggregates_and_galerkin_parity(which, p_smooth, strength):
    mesh, prob = heat(57) if which == "heat" else dg(57)
    A, _, _ = obt.radau_iia(3)
    h = 1 / 64 if which == "heat" else 0.01
    ctx, At = oracle_ctx(prob, A, "LD", h, p_smooth=p_smooth, strength=strength, **AMG_OPTS)
    for stage in range(3):
        Bk = (prob.M + (h * At[stage, stage]) * prob.F).tocsr()
        H = oamg.Hierarchy(Bk, p_smooth=p_smooth, strength_negative=bool(strength), **oracle_amg_opts())
        rows, nnz = B().irk_amg_info(ctx, stage)
        assert rows[0] == prob.n
        # level 0: bit-identical block, identical aggregates
        rp, col, val = B().irk_amg_level_matrix(ctx, stage, 0)
        L0 = sp.csr_matrix((val, col, rp), shape=(prob.n, prob.n))
        assert abs(L0 - H.levels[0].A).max() == 0.0
        # same level sizes, including where coarsening stops at once (the
        # negative-coupling measure on a convection-dominated block)
        assert rows == H.sizes()
        if len(rows) > 1:
            assert np.array_equal(B().irk_amg_aggregates(ctx, stage, 0), H.levels[0].agg)
        # Galerkin coarse matrices agree to rounding
        for l in range(1, len(rows)):
            rp, col, val = B().irk_amg_level_matrix(ctx, stage, l)
            Lg = sp.csr_matrix((val, col, rp), shape=(rows[l], rows[l]))
            Lo = H.levels[l].A
            assert abs(Lg - Lo).max() <= 1e-13 * abs(Lo).max()
            if l + 1 < len(rows):
                assert np.array_equal(B().irk_amg_aggregates(ctx, stage, l), H.levels[l].agg)


def bf16_round(x):
    """Round FP64 values to the nearest BF16 value (8 significant bits,
    ties to even), as __double2bfloat16 does."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0), e - 8)


def test_bf16_rounding_definition():
    assert bf16_round(1.0 + 2.0 ** -8) == 1.0                      # tie -> even
    assert bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie -> even
    assert bf16_round(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7          # representable
    assert bf16_round(-3.0) == -3.0 and bf16_round(0.0) == 0.0


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5), ("bf16", 2e-5)])
def test_vcycle_parity(prec, tol):
    """One V-cycle against the oracle's.  BF16 stores the finest-level values
    in BF16 (smoother and residual products); the oracle then runs the same
    V-cycle with those rounded finest values and everything else unchanged."""
    mesh, prob = heat(45)
    A, _, _ = obt.radau_iia(2)
    h = 0.05
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec=prec, **AMG_OPTS)
    rhs = synth.random_stage_block(prob.n, 1, 5)[0]
    for stage in range(2):
        Bk = (prob.M + (h * At[stage, stage]) * prob.F).tocsr()
        H = oamg.Hierarchy(Bk, **oracle_amg_opts())
        exact_ref = H.vcycle(rhs)
        if prec == "bf16":
            A0 = H.levels[0].A.copy()
            A0.data = bf16_round(A0.data)
            H.levels[0].A = A0
        ref = H.vcycle(rhs)
        x = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        B().irk_vcycle(ctx, stage, dev(rhs), x)
        err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
        assert err < tol, (prec, stage, err)
        if prec == "bf16":   # the rounded operator stays close to the FP64 one
            assert np.linalg.norm(host(x) - exact_ref) < 0.1 * np.linalg.norm(exact_ref)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_coarse_w_cycle_parity(prec, tol):
    """The W-cycle below the finest level (IRK_CYCLE_W_COARSE) against the
    oracle's on hierarchies of four or more levels (stiffness-dominated heat
    blocks, h_t = 4, 97^2 with a ragged tail, coarsest at most 16 rows): one
    cycle per stage through irk_vcycle, and the LD preconditioner (both
    directions) through irk_apply_precond."""
    mesh, prob = heat(97)
    A, _, _ = obt.radau_iia(2)
    h = 4.0
    opts = dict(AMG_OPTS, coarse_max=16)
    oopts = dict(oracle_amg_opts(), coarse_max=16)
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec=prec, cycle="Wc", **opts)
    rhs = synth.random_stage_block(prob.n, 1, 21)[0]
    for stage in range(2):
        Bk = (prob.M + (h * At[stage, stage]) * prob.F).tocsr()
        H = oamg.Hierarchy(Bk, cycle="Wc", **oopts)
        assert len(H.sizes()) >= 4, H.sizes()
        ref = H.vcycle(rhs)
        x = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        B().irk_vcycle(ctx, stage, dev(rhs), x)
        err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
        assert err < tol, (prec, stage, err)
        vref = oamg.Hierarchy(Bk, **oopts).vcycle(rhs)
        assert np.linalg.norm(vref - ref) > 100 * tol * np.linalg.norm(ref)
    v = synth.random_stage_block(prob.n, 2, 22)
    for tr in (False, True):
        pc = oirk.BlockPreconditioner(prob.M, prob.F, A, h, "LD", "amg", Atilde=At,
                                      amg_opts=dict(oopts, cycle="Wc"), transpose=tr)
        ref = pc.apply(v)
        z = torch.empty(2 * prob.n, dtype=torch.float64, device="cuda")
        B().irk_apply_precond(ctx, dev(v.ravel()), z, transpose=tr)
        err = np.linalg.norm(host(z).reshape(2, -1) - ref) / np.linalg.norm(ref)
        assert err < 2 * tol, (prec, tr, err)
    ctx.close()


@pytest.mark.parametrize("kind", ["J", "GSL", "GSL_OPT", "DU", "LD"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 5e-5)])
def test_precond_parity(kind, prec, tol):
    mesh, prob = heat(38)
    A, _, _ = obt.radau_iia(4)
    h = 1 / 64
    ctx, At = oracle_ctx(prob, A, kind, h, amg_prec=prec, **AMG_OPTS)
    v = synth.random_stage_block(prob.n, 4, 9)
    for tr in (False, True):
        pc = oirk.BlockPreconditioner(prob.M, prob.F, A, h, kind, "amg", Atilde=At, amg_opts=oracle_amg_opts(),
                                      transpose=tr)
        ref = pc.apply(v)
        z = torch.empty(4 * prob.n, dtype=torch.float64, device="cuda")
        B().irk_apply_precond(ctx, dev(v.ravel()), z, transpose=tr)
        err = np.linalg.norm(host(z).reshape(4, -1) - ref) / np.linalg.norm(ref)
        assert err < tol, (kind, prec, tr, err)


def _its_close(a, b):
    return abs(a - b) <= max(1, int(np.ceil(0.1 * b)))


@pytest.mark.parametrize("kind", ["J", "GSL", "DU", "LD"])
def test_heat_c1_run(kind):
    """32x32 heat, Radau IIA s=2, h_t=0.05, 20 steps: every step within 1e-8
    of the oracle's exact stage solve; FGMRES iteration counts within 10% of
    the oracle's FGMRES with the same AMG reading."""
    mesh, prob = heat(32)
    A, b, _ = obt.radau_iia(2)
    h, nsteps = 0.05, 20
    ctx, At = oracle_ctx(prob, A, kind, h, amg_prec="f32", b=b, **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    direct = oirk.IRKSolver(prob, A, b, h, kind=None)
    refs, _ = direct.run(u0, nsteps, direct=True)
    amg_sol = oirk.IRKSolver(prob, A, b, h, kind=kind, subsolve="amg", amg_opts=oracle_amg_opts(), Atilde=At)
    u = dev(u0)
    for t in range(nsteps):
        out = torch.empty_like(u)
        st = B().irk_step(ctx, u, out)
        got = host(out)
        err = np.linalg.norm(got - refs[t + 1]) / np.linalg.norm(refs[t + 1])
        assert err < 1e-8, (t, err)
        if t < 3:
            oit = amg_sol.step(refs[t]).iterations
            assert _its_close(st["iterations"], oit), (t, st["iterations"], oit)
        assert st["resid"] <= 1e-10
        u = out
    # the same through irk_run with checkpoints
    uN = torch.empty_like(u)
    ck = torch.empty((nsteps + 4) // 5, prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_run(ctx, dev(u0), nsteps, uN, ckpt=ck, ckpt_every=5)
    assert st["steps"] == nsteps
    assert np.linalg.norm(host(uN) - refs[-1]) <= 1e-8 * np.linalg.norm(refs[-1])
    for q in range(ck.shape[0]):
        assert np.linalg.norm(host(ck[q]) - refs[5 * q]) <= 1e-8 * np.linalg.norm(refs[5 * q])


def test_table5_small_sizes_through_irk_solve():
    """The paper's Radau IIA table (Table 5) at h_x^-1 = 8 and 16 through the
    library: P2 assembly, irk_solve with the default FP32 AMG (these blocks
    fall under the dense coarsest solve), manufactured right-hand side, rtol
    1e-8: every count within max(2, 10%) of the printed one."""
    import json
    import os
    from paper_2010_11377_gb300 import problems
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table5_radau_p2.json")) as f:
        ref = json.load(f)
    for N in (8, 16):
        p = problems.heat_p2(N)
        for s_ in range(2, 8):
            A, b, c = B().irk_butcher_table("radau_iia", s_)
            h = (1.0 / N) ** (3.0 / (2 * s_ - 1))
            kstar = dev(synth.random_stage_block(p["n"], s_, 1000 + N).ravel())
            for q, kind in enumerate(ref["columns"]):
                o = B().irk_default_options(kind=kind, rtol=1e-8)
                ctx = B().irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, options=o)
                rhs = torch.empty_like(kstar)
                B().irk_apply_operator(ctx, kstar, rhs)
                k = torch.empty_like(kstar)
                st = B().irk_solve(ctx, rhs, k)
                paper = ref["iterations"][str(N)][str(s_)][q]
                assert abs(st["iterations"] - paper) <= max(2, int(np.ceil(0.1 * paper))), (N, s_, kind)
                assert float((k - kstar).norm() / kstar.norm()) < 1e-5
                ctx.close()


def test_solve_scale_invariance():
    """Right-hand sides scaled by 2^-100, 1e-30, 1 and 1e30: the solution
    scales with them and the FGMRES iteration count stays the same (the
    preconditioner and the single-float pair operator only see the unit
    vectors sigma_j V_j), with exact zeros in the manufactured solution."""
    mesh, prob = heat(60)
    A, b, c = obt.radau_iia(3)
    h = 1 / 64
    ctx, _ = oracle_ctx(prob, A, "LD", h, amg_prec="f32", b=b, **AMG_OPTS)
    kstar = synth.random_stage_block(prob.n, 3, 21).ravel()
    kstar[::7] = 0.0
    rhs = torch.empty(kstar.size, dtype=torch.float64, device="cuda")
    B().irk_apply_operator(ctx, dev(kstar), rhs)
    k1 = torch.empty_like(rhs)
    st1 = B().irk_solve(ctx, rhs, k1)
    assert float((k1 - dev(kstar)).norm() / np.linalg.norm(kstar)) < 1e-6
    # a power of two scales every step exactly: the same iterates, scaled
    k = torch.empty_like(rhs)
    st = B().irk_solve(ctx, rhs * 2.0 ** -100, k)
    assert st["iterations"] == st1["iterations"]
    assert torch.equal(k * 2.0 ** 100, k1)
    for scale in (1e-30, 1e30):
        k = torch.empty_like(rhs)
        st = B().irk_solve(ctx, rhs * scale, k)
        assert abs(st["iterations"] - st1["iterations"]) <= 1, (scale, st["iterations"], st1["iterations"])
        assert st["resid"] <= 1e-10
        assert float((k / scale - k1).norm() / k1.norm()) < 1e-6, scale


def test_table6_lobatto_small_sizes_through_irk_solve():
    """The paper's Lobatto IIIC table (Table 6) at h_x^-1 = 8 and 16 through the
    library (P2, FP32 AMG = a dense solve here, manufactured right-hand side,
    rtol 1e-8): every count within max(3, 10%) of the printed one."""
    import json
    import os
    from paper_2010_11377_gb300 import problems
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table6_lobatto_p2.json")) as f:
        ref = json.load(f)
    for N in (8, 16):
        p = problems.heat_p2(N)
        for s_ in range(2, 6):
            A, b, c = B().irk_butcher_table("lobatto_iiic", s_)
            h = (1.0 / N) ** (3.0 / (2 * s_ - 2))
            kstar = dev(synth.random_stage_block(p["n"], s_, 1000 + N).ravel())
            for q, kind in enumerate(ref["columns"]):
                o = B().irk_default_options(kind=kind, rtol=1e-8)
                ctx = B().irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, options=o)
                rhs = torch.empty_like(kstar)
                B().irk_apply_operator(ctx, kstar, rhs)
                k = torch.empty_like(kstar)
                st = B().irk_solve(ctx, rhs, k)
                paper = ref["iterations"][str(N)][str(s_)][q]
                assert abs(st["iterations"] - paper) <= max(3, int(np.ceil(0.1 * paper))), (N, s_, kind)
                ctx.close()


def test_table8_small_sizes_left_through_irk_solve():
    """The paper's left-preconditioned table (Table 8) at h_x^-1 = 8 and 16
    through the library (left GMRES, FP64 AMG, which is a dense solve here):
    J, GSL, DU and LD counts within max(2, 10%) of the printed ones."""
    import json
    import os
    from paper_2010_11377_gb300 import problems
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table8_radau_p2_left.json")) as f:
        ref = json.load(f)
    for N in (8, 16):
        p = problems.heat_p2(N)
        for s_ in range(2, 7):
            A, b, c = B().irk_butcher_table("radau_iia", s_)
            h = (1.0 / N) ** (3.0 / (2 * s_ - 1))
            kstar = dev(synth.random_stage_block(p["n"], s_, 1000 + N).ravel())
            for q, kind in enumerate(ref["columns"]):
                if kind == "GSL_OPT":
                    continue
                o = B().irk_default_options(kind=kind, rtol=1e-8, side="left", amg_prec="f64")
                ctx = B().irk_setup(p["rowptr"], p["col"], p["valM"], p["valF"], (A, b, c), h, options=o)
                rhs = torch.empty_like(kstar)
                B().irk_apply_operator(ctx, kstar, rhs)
                k = torch.empty_like(kstar)
                st = B().irk_solve(ctx, rhs, k)
                paper = ref["iterations"][str(N)][str(s_)][q]
                assert abs(st["iterations"] - paper) <= max(2, int(np.ceil(0.1 * paper))), (N, s_, kind)
                ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["GSL", "LD"])
def test_supg_nitsche_steps(prec, kind):
    """Double glazing with SUPG and Nitsche terms (nonsymmetric M and F, every
    node an unknown): 3 steps within 1e-8 of the oracle's exact stage solves,
    iteration counts within 10% of the oracle's FGMRES on the same matrices."""
    N, eps = 24, 0.005
    mesh = synth.structured_mesh(N, "box")
    prob = ofem.double_glazing_supg_nitsche(mesh, eps, synth.double_glazing_wind, synth.double_glazing_boundary(mesh))
    A, b, _ = obt.radau_iia(3)
    h = 0.05
    ctx, At = oracle_ctx(prob, A, kind, h, amg_prec=prec, b=b, **AMG_OPTS)
    u0 = synth.double_glazing_boundary(mesh)
    refs, _ = oirk.IRKSolver(prob, A, b, h, kind=None).run(u0, 3, direct=True)
    amg_sol = oirk.IRKSolver(prob, A, b, h, kind=kind, subsolve="amg", amg_opts=oracle_amg_opts(), Atilde=At)
    u = dev(u0)
    for t in range(3):
        out = torch.empty_like(u)
        st = B().irk_step(ctx, u, out)
        err = np.linalg.norm(host(out) - refs[t + 1]) / np.linalg.norm(refs[t + 1])
        assert err < 1e-8, (t, err)
        if prec == "f64":
            assert _its_close(st["iterations"], amg_sol.step(refs[t]).iterations)
        u = out


def test_supg_stabilised_hierarchy_parity():
    """Coarse-level SUPG stabilisation: the library's hierarchy of a SUPG
    double-glazing block (level 0 bit-identical, aggregates identical on every
    level, stabilised coarse matrices within 1e-13 of the oracle's)."""
    N, eps = 80, 0.005
    mesh = synth.structured_mesh(N, "box")
    prob = ofem.double_glazing_supg_nitsche(mesh, eps, synth.double_glazing_wind, synth.double_glazing_boundary(mesh))
    A, _, _ = obt.radau_iia(2)
    h = 1.0
    opts = dict(theta=0.08, coarse_max=256, smoother="chebyshev", cheb_degree=4, cheb_lo=0.3)
    ctx, At = oracle_ctx(prob, A, "LD", h, p_smooth=1, **opts)
    for stage in range(2):
        c = h * At[stage, stage]
        Bk = (prob.M + c * prob.F).tocsr()
        H = oamg.Hierarchy(Bk, p_smooth=1, stab=(prob.T, c), **opts)
        Hplain = oamg.Hierarchy(Bk, p_smooth=1, **opts)
        rows, _ = B().irk_amg_info(ctx, stage)
        assert rows == H.sizes() and len(rows) >= 3
        for l in range(1, len(rows)):
            rp, col, val = B().irk_amg_level_matrix(ctx, stage, l)
            Lg = sp.csr_matrix((val, col, rp), shape=(rows[l], rows[l]))
            Lo = H.levels[l].A
            assert abs(Lg - Lo).max() <= 1e-13 * abs(Lo).max()
            if l + 1 < len(rows):
                assert np.array_equal(B().irk_amg_aggregates(ctx, stage, l), H.levels[l].agg)
        # the stabilisation changed the coarse operators
        assert abs(H.levels[1].A - Hplain.levels[1].A).max() > 0.0


def test_supg_convection_dominated_solve():
    """The paper's double-glazing time-step table (Table 13) at h_x^-1 = 128,
    eps = 0.005, s = 2, h_t = 1 (where the unstabilised V-cycle stops
    contracting): the library with the coarse-level stabilisation and the
    stronger smoother (Chebyshev degree 8 on [0.3, 1], V(2,2)) solves the
    manufactured system with left GMRES to 1e-8, k within 1e-6 of k*, in as many
    iterations as the oracle (within 10 %)."""
    mesh = synth.structured_mesh(256, "box")
    prob = ofem.double_glazing_supg_nitsche(mesh, 0.005, synth.double_glazing_wind,
                                            synth.double_glazing_boundary(mesh))
    A, b, _ = obt.radau_iia(2)
    h = 1.0
    opts = dict(cheb_lo=0.3, cheb_degree=8, nu_pre=2, nu_post=2, p_smooth=1)
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec="f64", b=b, side="left", rtol=1e-8, **opts)
    kstar = synth.random_stage_block(prob.n, 2, 2128)
    rhs = oirk.apply_operator(prob.M, prob.F, A, h, kstar)
    k = torch.empty(2 * prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_solve(ctx, dev(rhs.ravel()), k)
    assert np.linalg.norm(host(k).reshape(2, -1) - kstar) <= 1e-6 * np.linalg.norm(kstar)
    pc = oirk.BlockPreconditioner(prob.M, prob.F, A, h, "LD", "amg", Atilde=At, amg_opts=opts, stab=prob.T)
    ores = oirk.gmres_left(lambda z: oirk.apply_operator(prob.M, prob.F, A, h, z), pc.apply, rhs, rtol=1e-8)
    assert ores.converged
    assert _its_close(st["iterations"], ores.iterations), (st["iterations"], ores.iterations)
    ctx.close()


@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("kind", ["J", "LD"])
def test_p2_manufactured_solve(side, kind):
    """irk_solve on the P2 heat matrices (the paper's runs, Section 5) for a
    manufactured right-hand side b = A k* (random k*, Radau IIA s = 3,
    h_t = h_x^(3/5)): k within 1e-7 of k*, FP64 AMG, iteration counts within
    10% of the oracle's (F)GMRES with the same AMG reading on the same b."""
    N, s_ = 12, 3
    mesh = synth.structured_mesh_p2(N)
    prob = ofem.heat_problem_p2(mesh)
    A, b, _ = obt.radau_iia(s_)
    h = (1.0 / N) ** (3.0 / (2 * s_ - 1))
    ctx, At = oracle_ctx(prob, A, kind, h, amg_prec="f64", b=b, side=side, **AMG_OPTS)
    kstar = synth.random_stage_block(prob.n, s_, 7)
    rhs = oirk.apply_operator(prob.M, prob.F, A, h, kstar)
    k = torch.empty(s_ * prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_solve(ctx, dev(rhs.ravel()), k)
    got = host(k).reshape(s_, prob.n)
    assert np.linalg.norm(got - kstar) <= 1e-7 * np.linalg.norm(kstar)
    sol = oirk.IRKSolver(prob, A, b, h, kind=kind, subsolve="amg", amg_opts=oracle_amg_opts(), Atilde=At,
                         side=side)
    oit = sol.solve_stages(rhs).iterations
    assert _its_close(st["iterations"], oit), (st["iterations"], oit)


@pytest.mark.parametrize("kind", ["GSL", "LD"])
@pytest.mark.parametrize("s", [2, 5])
def test_left_preconditioned_steps(kind, s):
    """Left-preconditioned GMRES (FP64 AMG, so P^{-1} is a fixed linear map):
    3 steps within 1e-8 of the exact stage solves, iteration counts within 10%
    of the oracle's left GMRES with the same AMG reading, the reported true
    residual small, and the preconditioned stopping test met."""
    mesh, prob = heat(44)
    A, b, _ = obt.radau_iia(s)
    h = 1 / 16
    ctx, At = oracle_ctx(prob, A, kind, h, amg_prec="f64", b=b, side="left", **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    refs, _ = oirk.IRKSolver(prob, A, b, h, kind=None).run(u0, 3, direct=True)
    left = oirk.IRKSolver(prob, A, b, h, kind=kind, subsolve="amg", amg_opts=oracle_amg_opts(), Atilde=At,
                          side="left")
    u = dev(u0)
    for t in range(3):
        out = torch.empty_like(u)
        st = B().irk_step(ctx, u, out)
        err = np.linalg.norm(host(out) - refs[t + 1]) / np.linalg.norm(refs[t + 1])
        assert err < 1e-8, (t, err)
        o = left.step(refs[t])
        assert _its_close(st["iterations"], o.iterations), (t, st["iterations"], o.iterations)
        assert st["resid"] < 1e-8
        u = out


def test_left_preconditioning_fp32_amg_and_limits():
    """FP32 AMG with left preconditioning converges to a looser preconditioned
    tolerance; the same context runs adjoint steps (right-preconditioned on the
    transposed system)."""
    mesh, prob = heat(40)
    A, b, _ = obt.radau_iia(3)
    h = 1 / 16
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec="f32", b=b, side="left", rtol=1e-6, **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    ref = oirk.IRKSolver(prob, A, b, h, kind=None).step(u0, direct=True).u
    out = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_step(ctx, dev(u0), out)
    assert np.linalg.norm(host(out) - ref) <= 1e-5 * np.linalg.norm(ref)
    assert st["iterations"] > 0
    lam = dev(np.ones(prob.n))
    lam0 = torch.empty_like(lam)
    st = B().irk_adjoint_step(ctx, lam, None, None, lam0)
    assert st["iterations"] > 0 and bool(torch.isfinite(lam0).all())


@pytest.mark.parametrize("kind", ["GSL", "DU", "LD"])
@pytest.mark.parametrize("s", [2, 4])
def test_lobatto_iiic_steps(kind, s):
    """Lobatto IIIC through the same path (the library's own Butcher table):
    3 steps within 1e-8 of the oracle's exact stage solves, iteration counts
    within 10% of the oracle's FGMRES with the same AMG reading."""
    mesh, prob = heat(44)
    A, b, _ = obt.lobatto_iiic(s)
    Al, bl, cl = B().irk_butcher_table("lobatto_iiic", s)
    assert np.allclose(Al, A, atol=1e-14) and np.allclose(bl, b, atol=1e-14)
    h = 1 / 32
    ctx, At = oracle_ctx(prob, A, kind, h, amg_prec="f32", b=b, **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    refs, _ = oirk.IRKSolver(prob, A, b, h, kind=None).run(u0, 3, direct=True)
    amg_sol = oirk.IRKSolver(prob, A, b, h, kind=kind, subsolve="amg", amg_opts=oracle_amg_opts(), Atilde=At)
    u = dev(u0)
    for t in range(3):
        out = torch.empty_like(u)
        st = B().irk_step(ctx, u, out)
        err = np.linalg.norm(host(out) - refs[t + 1]) / np.linalg.norm(refs[t + 1])
        assert err < 1e-8, (t, err)
        assert _its_close(st["iterations"], amg_sol.step(refs[t]).iterations)
        u = out


@pytest.mark.parametrize("s,restart", [(8, 30), (3, 1), (3, 64)])
def test_limits_stage_count_and_restart(s, restart):
    """The largest stage count (s = 8) and the restart limits (FGMRES(1) and
    FGMRES(64)): a step within 1e-8 of the oracle's exact stage solve."""
    mesh, prob = heat(26)
    A, b, _ = obt.radau_iia(s)
    h = 1 / 32
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec="f32", b=b, restart=restart, **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    ref = oirk.IRKSolver(prob, A, b, h, kind=None).step(u0, direct=True).u
    out = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_step(ctx, dev(u0), out)
    assert np.linalg.norm(host(out) - ref) <= 1e-8 * np.linalg.norm(ref)
    assert st["resid"] <= 1e-10
    if restart == 1:
        assert st["restarts"] >= st["iterations"] - 1


@pytest.mark.parametrize("reorth,eta", [(1, 0.1), (0, 0.7071067811865476), (0, 0.1), (0, 0.0)])
def test_gram_schmidt_second_pass_threshold(reorth, eta):
    """The second Gram-Schmidt pass (always, 1/sqrt(2) rule, the default 0.1,
    never) leaves the step within 1e-8 of the oracle's exact stage solve and
    the FGMRES iteration counts within 10% of the oracle's MGS-FGMRES."""
    mesh, prob = heat(60)
    A, b, _ = obt.radau_iia(5)
    h = 1 / 64
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec="f32", b=b, reorth=reorth, reorth_eta=eta, **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    ref = oirk.IRKSolver(prob, A, b, h, kind=None).step(u0, direct=True).u
    oit = oirk.IRKSolver(prob, A, b, h, kind="LD", subsolve="amg", amg_opts=oracle_amg_opts(),
                         Atilde=At).step(u0).iterations
    out = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_step(ctx, dev(u0), out)
    assert np.linalg.norm(host(out) - ref) <= 1e-8 * np.linalg.norm(ref)
    assert st["resid"] <= 1e-10
    assert _its_close(st["iterations"], oit), (st["iterations"], oit)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_double_glazing_steps(prec):
    mesh, prob = dg(48)
    A, b, _ = obt.radau_iia(3)
    h = 0.01
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec=prec, **AMG_OPTS)
    u0 = np.zeros(prob.n)
    refs, _ = oirk.IRKSolver(prob, A, b, h, kind=None).run(u0, 3, direct=True)
    u = dev(u0)
    for t in range(3):
        out = torch.empty_like(u)
        B().irk_step(ctx, u, out)
        err = np.linalg.norm(host(out) - refs[t + 1]) / np.linalg.norm(refs[t + 1])
        assert err < 1e-8, (prec, t, err)
        u = out


def test_stage_output_and_residual():
    mesh, prob = heat(36)
    A, b, _ = obt.radau_iia(5)
    h = 1 / 64
    ctx, _ = oracle_ctx(prob, A, "LD", h, amg_prec="f32", **AMG_OPTS)
    u0 = synth.heat_u0(mesh)
    u = dev(u0)
    out = torch.empty_like(u)
    k = torch.empty(5 * prob.n, dtype=torch.float64, device="cuda")
    st = B().irk_step(ctx, u, out, k)
    kk = host(k).reshape(5, -1)
    rhs = oirk.stage_rhs(prob.F, prob.g, u0, 5)
    r = rhs - oirk.apply_operator(prob.M, prob.F, A, h, kk)
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(rhs)
    assert np.allclose(host(out), u0 + h * b @ kk, rtol=0, atol=1e-15 * np.abs(u0).max())
    assert st["resid"] <= 1e-10


def test_residual_norm():
    """||b - A k|| through the C ABI against the oracle's operator."""
    mesh, prob = heat(39)
    A, b, _ = obt.radau_iia(4)
    h = 1 / 64
    ctx, _ = oracle_ctx(prob, A, "LD", h)
    k = synth.random_stage_block(prob.n, 4, 21)
    rhs = synth.random_stage_block(prob.n, 4, 22)
    ref = np.linalg.norm(rhs - oirk.apply_operator(prob.M, prob.F, A, h, k))
    got = B().irk_residual_norm(ctx, dev(k.ravel()), dev(rhs.ravel()))
    assert abs(got - ref) <= 1e-13 * ref


def test_edge_cases():
    bnd = B()
    from paper_2010_11377_gb300._abi import IrkError
    # one unknown (N = 2), s = 1
    mesh, prob = heat(2)
    A, b, _ = obt.radau_iia(1)
    ctx, _ = oracle_ctx(prob, A, "J", 0.1)
    u = dev(np.array([1.0]))
    out = torch.empty_like(u)
    bnd.irk_step(ctx, u, out)
    ref = oirk.IRKSolver(prob, A, b, 0.1, kind=None).step(np.array([1.0]), direct=True).u
    assert abs(host(out)[0] - ref[0]) < 1e-12
    # zero state -> zero stages, no iterations
    mesh, prob = heat(20)
    A, b, _ = obt.radau_iia(3)
    ctx, _ = oracle_ctx(prob, A, "LD", 0.05)
    z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(z)
    st = bnd.irk_step(ctx, z, out)
    assert st["iterations"] == 0 and torch.count_nonzero(out) == 0
    # iteration cap: NOT_CONVERGED is reported, the iterate is returned
    ctx2, _ = oracle_ctx(prob, A, "J", 0.05, max_it=2)
    with pytest.raises(IrkError) as ei:
        bnd.irk_step(ctx2, dev(synth.heat_u0(mesh)), out)
    assert ei.value.status == 4
    # non-finite input
    bad = dev(np.full(prob.n, np.nan))
    with pytest.raises(IrkError) as ei:
        bnd.irk_step(ctx, bad, out)
    assert ei.value.status == 7
    # invalid: wrong dtype / stage index
    with pytest.raises(ValueError):
        bnd.irk_step(ctx, z.float(), out)
    with pytest.raises(IrkError):
        bnd.irk_vcycle(ctx, 9, z, out)


def test_adjoint_nonsymmetric():
    """Double glazing (F = eps K + C nonsymmetric): the transposed
    preconditioner against the oracle's P^T, one adjoint step against the
    oracle's exact transposed stage solve, and dL/du0 of the checkpointed
    reverse sweep against the oracle's discrete adjoint with exact solves."""
    mesh, prob = dg(24)
    A, b, _ = obt.radau_iia(3)
    h, nsteps, every = 0.05, 4, 2
    ctx, At = oracle_ctx(prob, A, "LD", h, amg_prec="f64", b=b, **AMG_OPTS)
    bnd = B()
    v = synth.random_stage_block(prob.n, 3, 11)
    pc = oirk.BlockPreconditioner(prob.M, prob.F, A, h, "LD", "amg", Atilde=At, amg_opts=oracle_amg_opts(),
                                  transpose=True)
    z = torch.empty(3 * prob.n, dtype=torch.float64, device="cuda")
    bnd.irk_apply_precond(ctx, dev(v.ravel()), z, transpose=True)
    ref = pc.apply(v)
    assert np.linalg.norm(host(z).reshape(3, -1) - ref) <= 1e-12 * np.linalg.norm(ref)
    sol = oirk.IRKSolver(prob, A, b, h, kind="LD", subsolve="direct")
    zt = synth.random_stage_block(prob.n, 3, 12)
    wt = torch.empty(3 * prob.n, dtype=torch.float64, device="cuda")
    bnd.irk_apply_operator(ctx, dev(zt.ravel()), wt, transpose=True)
    reft = sol.opT(zt)
    assert np.abs(host(wt).reshape(3, -1) - reft).max() <= 1e-14 * np.abs(reft).max()
    lam1 = synth.random_smooth_u0(mesh, seed=5)
    ref_lam, _ = sol.adjoint_step(lam1, direct=True)
    out = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    st = bnd.irk_adjoint_step(ctx, dev(lam1), None, None, out)
    assert st["resid"] <= 1e-10
    assert np.linalg.norm(host(out) - ref_lam) <= 1e-8 * np.linalg.norm(ref_lam)
    # checkpointed sweep: dL/du0 for L = 1/2 (u_N - d)^T M (u_N - d)
    u0 = synth.random_smooth_u0(mesh, seed=6)
    d = 0.5 * u0
    us, _ = sol.run(u0, nsteps, direct=True)
    lam = prob.M @ (us[-1] - d)
    for _ in range(nsteps):
        lam, _ = sol.adjoint_step(lam, direct=True)
    uN = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ck = torch.empty(nsteps // every, prob.n, dtype=torch.float64, device="cuda")
    bnd.irk_run(ctx, dev(u0), nsteps, uN, ckpt=ck, ckpt_every=every)
    g = torch.empty_like(uN)
    bnd.irk_apply_mass(ctx, uN - dev(d), g)
    bnd.irk_adjoint_run(ctx, ck, nsteps, every, g, None)
    assert np.linalg.norm(host(g) - lam) <= 1e-8 * np.linalg.norm(lam)
    # the same instance through a batch graph (forward and adjoint launches)
    u0d = dev(u0)
    uNb = torch.empty_like(uN)
    ckb = torch.empty_like(ck)
    lamb = torch.empty_like(uN)
    batch = bnd.irk_batch_create([ctx], nsteps, every, [u0d], [uNb], [ckb], [lamb], [None])
    bnd.irk_batch_run(batch)
    bnd.irk_apply_mass(ctx, uNb - dev(d), lamb)
    bnd.irk_batch_adjoint(batch)
    assert np.linalg.norm(host(lamb) - lam) <= 1e-8 * np.linalg.norm(lam)
    batch.close()
    ctx.close()


def test_adjoint_of_left_preconditioned_context():
    """A context whose forward solves are left-preconditioned runs its adjoint
    steps with right-preconditioned FGMRES on the transposed system: one
    adjoint step against the oracle's exact transposed solve."""
    mesh, prob = heat(20)
    A, b, _ = obt.radau_iia(3)
    h = 0.05
    ctx, _ = oracle_ctx(prob, A, "LD", h, amg_prec="f64", b=b, side="left", **AMG_OPTS)
    sol = oirk.IRKSolver(prob, A, b, h, kind="LD", subsolve="direct")
    lam1 = synth.random_smooth_u0(mesh, seed=8)
    ref, _ = sol.adjoint_step(lam1, direct=True)
    out = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    B().irk_adjoint_step(ctx, dev(lam1), None, None, out)
    assert np.linalg.norm(host(out) - ref) <= 1e-8 * np.linalg.norm(ref)
    ctx.close()


def test_adjoint_gradients():
    """Checkpointed adjoint (C ABI) vs the oracle's discrete adjoint with exact
    solves: dL/du0 and dL/dkappa to 1e-8."""
    N, s, h, nsteps, every = 20, 3, 1 / 32, 6, 2
    mesh = synth.structured_mesh(N)
    kap = np.exp(synth.grf_log_kappa(mesh, seed=4))
    prob = ofem.heat_problem(mesh, kappa=kap)
    A, b, _ = obt.radau_iia(s)
    meshd = dict(xy=mesh.xy, tri=mesh.tri, dof=mesh.dof)
    ctx, _ = oracle_ctx(prob, A, "LD", h, amg_prec="f32", mesh=meshd, **AMG_OPTS)
    u0 = synth.random_smooth_u0(mesh, seed=4)
    d = 0.5 * u0
    Ke = ofem.element_stiffness_unit(mesh.xy, mesh.tri)
    sol = oirk.IRKSolver(prob, A, b, h, kind="LD", subsolve="direct")
    gu, gk, L = oirk.adjoint_gradients(sol, Ke, mesh.dof[mesh.tri], u0, nsteps, d, direct=True)
    bnd = B()
    uN = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ck = torch.empty(nsteps // every, prob.n, dtype=torch.float64, device="cuda")
    bnd.irk_run(ctx, dev(u0), nsteps, uN, ckpt=ck, ckpt_every=every)
    lam = torch.empty_like(uN)
    bnd.irk_apply_mass(ctx, uN - dev(d), lam)
    grad = torch.zeros(mesh.n_tri, dtype=torch.float64, device="cuda")
    bnd.irk_adjoint_run(ctx, ck, nsteps, every, lam, grad)
    assert np.linalg.norm(host(lam) - gu) <= 1e-8 * np.linalg.norm(gu)
    assert np.linalg.norm(host(grad) - gk) <= 1e-8 * np.linalg.norm(gk)
    # set_kappa rebuilds F on the GPU: the forward run still matches
    ctx2, _ = oracle_ctx(ofem.heat_problem(mesh), A, "LD", h, amg_prec="f32", mesh=meshd, **AMG_OPTS)
    bnd.irk_set_kappa(ctx2, dev(kap))
    uN2 = torch.empty_like(uN)
    bnd.irk_run(ctx2, dev(u0), nsteps, uN2)
    assert np.linalg.norm(host(uN2) - host(uN)) <= 1e-9 * np.linalg.norm(host(uN))
