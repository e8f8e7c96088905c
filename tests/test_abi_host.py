"""CPU tests of libirk without a GPU: the library loads, exports every entry
point declared in include/irk.h, and its host-side tables and P1 assembly
match the oracle (no device work is done here)."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import butcher as obt
from oracle import fem as ofem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2010_11377_gb300.build import build
    build()
    from paper_2010_11377_gb300._abi import lib
    return lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "irk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(irk_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(L, nm), nm
    from paper_2010_11377_gb300._abi import SIGNATURES
    assert sorted(n for n, _, _ in SIGNATURES) == names


def test_missing_library_fails_loudly(monkeypatch):
    import paper_2010_11377_gb300._abi as abi
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "LIB", "/nonexistent/libirk.so")
    with pytest.raises(RuntimeError):
        abi.lib()


@pytest.mark.parametrize("s", range(1, 9))
def test_radau_table_matches_oracle(L, s):
    from paper_2010_11377_gb300 import binding as B
    A, b, c = B.irk_butcher_table("radau_iia", s)
    if s <= 7:
        OA, Ob, Oc = obt.radau_iia(s)
        assert np.max(np.abs(A - OA)) < 1e-14 and np.max(np.abs(b - Ob)) < 1e-14
        assert np.max(np.abs(c - Oc)) < 1e-15
    for q in range(1, 2 * s):
        assert abs(b @ c ** (q - 1) - 1.0 / q) < 1e-13


@pytest.mark.parametrize("s", range(2, 6))
def test_lobatto_table_matches_oracle(L, s):
    from paper_2010_11377_gb300 import binding as B
    A, b, c = B.irk_butcher_table("lobatto_iiic", s)
    OA, Ob, Oc = obt.lobatto_iiic(s)
    assert np.max(np.abs(A - OA)) < 1e-14 and np.max(np.abs(b - Ob)) < 1e-14


def test_ldu_and_atilde_match_oracle(L):
    from paper_2010_11377_gb300 import binding as B
    for s in range(2, 8):
        A, _, _ = obt.radau_iia(s)
        Lm, D, U = B.irk_ldu(A)
        OL, OD, OU = obt.ldu(A)
        assert np.allclose(Lm, OL, atol=1e-13) and np.allclose(D, np.diag(OD), atol=1e-15)
        assert np.allclose(U, OU, atol=1e-13)
        for kind in ("J", "GSL", "DU", "LD"):
            At, kap = B.irk_atilde(kind, A)
            assert np.allclose(At, obt.atilde(A, kind), atol=1e-14)
            ref = obt.kappa2(np.linalg.solve(obt.atilde(A, kind), A))
            assert abs(kap - ref) < 1e-9 * ref
    from paper_2010_11377_gb300._abi import IrkError
    with pytest.raises(IrkError):
        B.irk_ldu(np.array([[0.0, 1.0], [1.0, 0.0]]))


def test_gsl_opt_matches_oracle_optimum(L):
    """Eq. GSLopt solved by the library's own Nelder-Mead: the optimum is
    lower triangular with diag(A), and its kappa is within 2% of the oracle's."""
    from paper_2010_11377_gb300 import binding as B
    for s in range(2, 8):
        A, _, _ = obt.radau_iia(s)
        At, kap = B.irk_atilde("GSL_OPT", A)
        assert np.allclose(np.diag(At), np.diag(A)) and np.allclose(np.triu(At, 1), 0)
        ko = obt.kappa2(np.linalg.solve(obt.gsl_optimized(A), A))
        assert kap <= obt.kappa2(np.linalg.solve(np.tril(A), A)) + 1e-12
        assert kap <= 1.02 * ko, (s, kap, ko)


def _csr(rp, col, val, n):
    import scipy.sparse as sp
    return sp.csr_matrix((val, col, rp), shape=(n, n))


@pytest.mark.parametrize("N", [5, 16])
def test_fem_heat_matches_oracle(L, N):
    from paper_2010_11377_gb300 import binding as B
    mesh = synth.structured_mesh(N)
    kap = np.exp(synth.grf_log_kappa(mesh, seed=2))
    rp, col, vM, vF, g = B.irk_fem_assemble(mesh.xy, mesh.tri, mesh.dof, mesh.n, kappa=kap)
    prob = ofem.heat_problem(mesh, kappa=kap)
    assert abs(_csr(rp, col, vM, mesh.n) - prob.M).max() < 1e-15
    assert abs(_csr(rp, col, vF, mesh.n) - prob.F).max() < 1e-12 * abs(prob.F).max()
    assert np.all(g == 0)


def test_fem_double_glazing_matches_oracle(L):
    """Different exact quadrature rules on both sides (Dunavant degree 4 here,
    collapsed Gauss in the oracle) give the same convection matrix."""
    from paper_2010_11377_gb300 import problems
    p = problems.double_glazing(12, eps=0.005)
    mesh = p["mesh"]
    prob = ofem.double_glazing_problem(mesh, 0.005, synth.double_glazing_wind, synth.double_glazing_boundary(mesh))
    F = _csr(p["rowptr"], p["col"], p["valF"], mesh.n)
    assert abs(F - prob.F).max() < 1e-13 * abs(prob.F).max()
    assert np.max(np.abs(p["g"] - prob.g)) < 1e-13
    assert abs(_csr(p["rowptr"], p["col"], p["valM"], mesh.n) - prob.M).max() < 1e-16


def test_fem_quad_rule_exact_degree4(L):
    """The convection rule integrates every monomial of degree <= 4 exactly:
    with the wind w = (x^a y^b, 0) on one reference-like triangle, sum of the
    C row entries against linear data reproduces int x^a y^b dphi/dx."""
    from paper_2010_11377_gb300 import binding as B
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [2.0, 2.0]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    dof = np.array([0, 1, 2, -1], dtype=np.int32)
    from math import factorial
    for a in range(5):
        for bexp in range(5 - a):
            xq = B.irk_fem_quad_points(xy, tri)
            wind = np.zeros_like(xq)
            wind[..., 0] = xq[..., 0] ** a * xq[..., 1] ** bexp
            rp, col, vM, vF, g = B.irk_fem_assemble(xy, tri, dof, 3, kappa=np.zeros(1), wind=wind)
            C = _csr(rp, col, vF, 3).toarray()
            # sum_k C[k, l] = int w . grad phi_l ; for l = 1 (phi = x): int x^a y^b
            exact = factorial(a) * factorial(bexp) / factorial(a + bexp + 2)
            assert abs(C[:, 1].sum() - exact) < 1e-14, (a, bexp)


def _setup_one_unknown(L, o, null_rowptr=False):
    """irk_setup on a one-unknown problem; returns (status, context pointer)."""
    import ctypes as C
    from paper_2010_11377_gb300 import _abi as A
    rowptr = np.array([0, 1], dtype=np.int64)
    col = np.array([0], dtype=np.int32)
    val = np.array([1.0])
    Am, b, c = obt.radau_iia(2)
    Am, b, c = (np.ascontiguousarray(x, dtype=np.float64) for x in (Am, b, c))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    prob = A.IrkProblem()
    rp = None if null_rowptr else rowptr.ctypes.data_as(C.POINTER(C.c_int64))
    prob.M = A.IrkCsr(1, 1, rp, col.ctypes.data_as(C.POINTER(C.c_int32)), dp(val))
    prob.F = prob.M
    bt = A.IrkButcher(2, dp(Am), dp(b), dp(c))
    out = C.c_void_p()
    st = L.irk_setup(C.byref(prob), C.byref(bt), 0.1, C.byref(o), None, C.byref(out))
    return st, out


@pytest.mark.parametrize("field,value", [("reorth_eta", 1.0), ("reorth_eta", -0.1), ("reorth", 2),
                                         ("restart", 0), ("coarse_max", 4096), ("cheb_degree", 0), ("p_smooth", 0), ("p_smooth", 4), ("strength", 2),
                                         ("cycle", 2), ("cycle", -1),
                                         ("side", 2), ("kind", 6), ("kind", -1), ("smoother", 2),
                                         ("cheb_lo", 0.0), ("cheb_lo", 1.0), ("cheb_lo", float("nan")),
                                         ("theta", -0.1), ("theta", float("nan")), ("max_levels", 0),
                                         ("max_levels", 17), ("rtol", 0.0), ("max_it", 0)])
def test_setup_rejects_bad_options_before_device_work(L, field, value):
    """Option validation happens on the host, before any CUDA call: a bad
    option returns IRK_ERR_INVALID with a message and no context."""
    from paper_2010_11377_gb300.binding import irk_default_options
    o = irk_default_options()
    setattr(o, field, value)
    st, out = _setup_one_unknown(L, o)
    assert st == 1 and not out.value
    assert L.irk_last_error(None)


def test_setup_validation_other_cases(L):
    """A custom A~ without its matrix and a NULL row pointer are rejected on the
    host; the default options pass validation (without a GPU the call then
    fails in CUDA, with one it builds a context)."""
    from paper_2010_11377_gb300.binding import irk_default_options
    st, out = _setup_one_unknown(L, irk_default_options(kind="CUSTOM"))
    assert st == 1 and not out.value
    st, out = _setup_one_unknown(L, irk_default_options(), null_rowptr=True)
    assert st == 1 and not out.value
    st, out = _setup_one_unknown(L, irk_default_options())
    assert st != 1, L.irk_last_error(None)
    if out.value:
        L.irk_destroy(out)


def _setup_csr(L, n, nnz, rowptr, col):
    """irk_setup on a CSR structure given as Python lists (values all one)."""
    import ctypes as C
    from paper_2010_11377_gb300 import _abi as A
    from paper_2010_11377_gb300.binding import irk_default_options
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ones(max(len(col), 1))
    Am, b, c = (np.ascontiguousarray(x, dtype=np.float64) for x in obt.radau_iia(2))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    prob = A.IrkProblem()
    prob.M = A.IrkCsr(n, nnz, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                      cl.ctypes.data_as(C.POINTER(C.c_int32)), dp(val))
    prob.F = prob.M
    bt = A.IrkButcher(2, dp(Am), dp(b), dp(c))
    out = C.c_void_p()
    o = irk_default_options()
    st = L.irk_setup(C.byref(prob), C.byref(bt), 0.1, C.byref(o), None, C.byref(out))
    return st, out


@pytest.mark.parametrize("rowptr,col,why", [
    ([1, 2, 3], [0, 1, 1], "rowptr[0] != 0"),
    ([0, 2, 2], [0, 1, 1], "rowptr[n] != nnz"),
    ([0, 3, 2], [0, 1, 1], "rowptr decreasing"),
    ([0, 1, 3], [0, 0, 2], "column n"),
    ([0, 1, 3], [0, -1, 1], "negative column"),
])
def test_setup_rejects_malformed_csr_before_device_work(L, rowptr, col, why):
    """A CSR structure whose row pointer does not start at 0, end at nnz and
    rise monotonically, or whose columns leave [0, n), is rejected on the host
    with IRK_ERR_INVALID before any device work (no context is made)."""
    st, out = _setup_csr(L, 2, 3, rowptr, col)
    assert st == 1 and not out.value, why
    assert L.irk_last_error(None)


@pytest.mark.parametrize("N", [3, 10])
def test_fem_p2_heat_matches_oracle(L, N):
    """libirk's host P2 assembly (its own quadrature) against the oracle's."""
    from paper_2010_11377_gb300 import problems
    p = problems.heat_p2(N)
    mesh = synth.structured_mesh_p2(N)
    o = ofem.heat_problem_p2(mesh)
    import scipy.sparse as sp
    M = sp.csr_matrix((p["valM"], p["col"], p["rowptr"]), shape=(p["n"], p["n"]))
    F = sp.csr_matrix((p["valF"], p["col"], p["rowptr"]), shape=(p["n"], p["n"]))
    assert p["n"] == (2 * N - 1) ** 2
    assert abs(M - o.M).max() <= 1e-15 * max(1.0, abs(o.M).max()) + 1e-17
    assert abs(F - o.F).max() <= 1e-13


@pytest.mark.parametrize("eps", [0.04, 0.005])
def test_fem_supg_nitsche_matches_oracle(L, eps):
    """libirk's SUPG / Nitsche assembly (degree-4 rule, edge-count boundary
    detection) against the oracle's (collapsed Gauss, wall test)."""
    from paper_2010_11377_gb300 import problems
    import scipy.sparse as sp
    N = 14
    p = problems.double_glazing_supg(N, eps)
    mesh = synth.structured_mesh(N, "box")
    o = ofem.double_glazing_supg_nitsche(mesh, eps, synth.double_glazing_wind, synth.double_glazing_boundary(mesh))
    M = sp.csr_matrix((p["valM"], p["col"], p["rowptr"]), shape=(p["n"], p["n"]))
    F = sp.csr_matrix((p["valF"], p["col"], p["rowptr"]), shape=(p["n"], p["n"]))
    assert p["n"] == (N + 1) ** 2
    assert abs(M - o.M).max() <= 1e-15
    assert abs(F - o.F).max() <= 1e-14
    assert np.abs(p["g"] - o.g).max() <= 1e-14


def _header_structs():
    """Field names, in order, of every anonymous `typedef struct { ... } name;`
    in include/irk.h."""
    src = open(os.path.join(ROOT, "include", "irk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:   # "type a" or "type a, b"
                fields += [re.findall(r"(\w+)\s*$", part)[0] for part in decl.split(",")]
        out[name] = fields
    return out


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """The ctypes mirrors of the header's structs have the same fields in the
    same order, and the same offsets and sizes as the C compiler gives them."""
    import ctypes
    import shutil
    import subprocess
    from paper_2010_11377_gb300 import _abi
    mirrors = {"irk_csr": _abi.IrkCsr, "irk_butcher": _abi.IrkButcher, "irk_options": _abi.IrkOptions,
               "irk_stats": _abi.IrkStats, "irk_problem": _abi.IrkProblem}
    structs = _header_structs()
    assert set(mirrors) <= set(structs), sorted(structs)
    for name, cls in mirrors.items():
        assert [f for f, _ in cls._fields_] == structs[name], name
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "irk.h"', "int main(void) {"]
    for name, fields in structs.items():
        if name not in mirrors:
            continue
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    csrc = tmp_path / "layout.c"
    csrc.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(csrc), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    checked = 0
    for ln in got:
        if not ln:
            continue
        name, field, value = ln.split()
        cls = mirrors[name]
        if field == "sizeof":
            assert ctypes.sizeof(cls) == int(value), name
        else:
            assert getattr(cls, field).offset == int(value), (name, field)
        checked += 1
    assert checked > 30


def test_default_options_as_documented(L):
    """irk_default_options fills the values its declaration documents: P_LD, FP32
    AMG, Chebyshev degree 4 on [0.1, 1], V(1,1), theta 0.08, coarse_max 2048,
    12 levels, FGMRES(30), rtol 1e-10, max_it 1000, reorth_eta 0.1, right
    preconditioning, two prolongator smoothing steps, strength from |a_ij|."""
    import ctypes
    from paper_2010_11377_gb300 import _abi
    o = _abi.IrkOptions()
    L.irk_default_options(ctypes.byref(o))
    src = open(os.path.join(ROOT, "include", "irk.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"\b(IRK_[A-Z0-9_]+)\s*=\s*(-?\d+)", src))
    assert o.kind == enum["IRK_PC_LD"]
    assert o.amg_prec == enum["IRK_AMG_F32"]
    assert (o.cheb_degree, o.cheb_lo, o.nu_pre, o.nu_post) == (4, 0.1, 1, 1)
    assert (o.theta, o.coarse_max, o.max_levels) == (0.08, 2048, 12)
    assert (o.restart, o.rtol, o.max_it) == (30, 1e-10, 1000)
    assert (o.reorth, o.reorth_eta, o.side, o.p_smooth, o.strength, o.cycle) == (0, 0.1, 0, 2, 0, 0)
    assert o.cycle == enum["IRK_CYCLE_V"]
    from paper_2010_11377_gb300.binding import irk_default_options
    assert irk_default_options(cycle="Wc").cycle == enum["IRK_CYCLE_W_COARSE"]
