"""Python binding of the C ABI (include/irk.h), one function per entry point
with the same name.  Argument marshalling only: host arrays are numpy, device
arrays are contiguous FP64 torch CUDA tensors; every computation runs in
libirk's CUDA kernels (or, for the host tables, in libirk's C++)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import IrkButcher, IrkCsr, IrkOptions, IrkProblem, IrkStats, check, lib

PC_KINDS = {"J": 0, "GSL": 1, "GSL_OPT": 2, "DU": 3, "LD": 4, "CUSTOM": 5}
METHODS = {"radau_iia": 0, "lobatto_iiic": 1}
AMG_PREC = {"f64": 64, "f32": 32, "bf16": 16, 64: 64, 32: 32, 16: 16}
SMOOTHERS = {"l1jacobi": 0, "chebyshev": 1}
CYCLES = {"V": 0, "Wc": 1}


def _dp(a):
    return a.ctypes.data_as(_abi.c_double_p) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_abi.c_int32_p) if a is not None else None


def _lp(a):
    return a.ctypes.data_as(_abi.c_int64_p) if a is not None else None


def _dev(t):
    """Device pointer of a contiguous FP64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("device arguments must be contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# host tables
# ---------------------------------------------------------------------------
def irk_butcher_table(method: str, s: int):
    A = np.zeros(s * s)
    b = np.zeros(s)
    c = np.zeros(s)
    check(lib().irk_butcher_table(METHODS[method], s, _dp(A), _dp(b), _dp(c)))
    return A.reshape(s, s), b, c


def irk_ldu(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    s = A.shape[0]
    L = np.zeros(s * s)
    D = np.zeros(s)
    U = np.zeros(s * s)
    check(lib().irk_ldu(s, _dp(A), _dp(L), _dp(D), _dp(U)))
    return L.reshape(s, s), D, U.reshape(s, s)


def irk_atilde(kind: str, A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    s = A.shape[0]
    At = np.zeros(s * s)
    kap = C.c_double(0.0)
    check(lib().irk_atilde(PC_KINDS[kind.upper()], s, _dp(A), _dp(At), C.byref(kap)))
    return At.reshape(s, s), kap.value


def irk_default_options(**overrides) -> IrkOptions:
    """irk_options filled by the library's defaults, then any field overridden by keyword
    (the names of include/irk.h).  Symbolic values: kind "J", "GSL", "GSL_OPT", "DU", "LD",
    "CUSTOM"; amg_prec "f64", "f32", "bf16"; side "right", "left"; smoother "l1jacobi",
    "chebyshev"; cycle "V" (one V-cycle per subsolve) or "Wc" (the W-cycle below the finest
    level).  Values are checked by irk_setup, not here."""
    o = IrkOptions()
    lib().irk_default_options(C.byref(o))
    for k, v in overrides.items():
        if k == "kind":
            v = PC_KINDS[v.upper()] if isinstance(v, str) else v
        elif k == "amg_prec":
            v = AMG_PREC[v]
        elif k == "side":
            v = {"right": 0, "left": 1}[v] if isinstance(v, str) else v
        elif k == "smoother":
            v = SMOOTHERS[v] if isinstance(v, str) else v
        elif k == "cycle":
            v = CYCLES[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


def irk_fem_quad_points(xy, tri):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    out = np.zeros((tri.shape[0], 6, 2))
    check(lib().irk_fem_quad_points(tri.shape[0], _dp(xy), _ip(tri), _dp(out)))
    return out


def irk_fem_assemble(xy, tri, dof, n, kappa=None, wind=None, ub=None):
    """Interior CSR (rowptr, col, valM, valF) and the lift g."""
    L = lib()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    dof = np.ascontiguousarray(dof, dtype=np.int32)
    kappa = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64)
    wind = None if wind is None else np.ascontiguousarray(wind, dtype=np.float64)
    ub = None if ub is None else np.ascontiguousarray(ub, dtype=np.float64)
    nnz = C.c_int64(0)
    args = (xy.shape[0], _dp(xy), tri.shape[0], _ip(tri), _ip(dof), n, _dp(kappa), _dp(wind), _dp(ub))
    check(L.irk_fem_assemble(*args, C.byref(nnz), None, None, None, None, None))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz.value, dtype=np.int32)
    valM = np.zeros(nnz.value)
    valF = np.zeros(nnz.value)
    g = np.zeros(n)
    check(L.irk_fem_assemble(*args, C.byref(nnz), _lp(rowptr), _ip(col), _dp(valM), _dp(valF), _dp(g)))
    return rowptr, col, valM, valF, g


def irk_fem_assemble_p2(xy, tri6, dof, n, kappa=None, ub=None):
    """Interior CSR (rowptr, col, valM, valF) and the lift g of quadratic triangles."""
    L = lib()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri6 = np.ascontiguousarray(tri6, dtype=np.int32)
    dof = np.ascontiguousarray(dof, dtype=np.int32)
    kappa = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64)
    ub = None if ub is None else np.ascontiguousarray(ub, dtype=np.float64)
    nnz = C.c_int64(0)
    args = (xy.shape[0], _dp(xy), tri6.shape[0], _ip(tri6), _ip(dof), n, _dp(kappa), _dp(ub))
    check(L.irk_fem_assemble_p2(*args, C.byref(nnz), None, None, None, None, None))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz.value, dtype=np.int32)
    valM = np.zeros(nnz.value)
    valF = np.zeros(nnz.value)
    g = np.zeros(n)
    check(L.irk_fem_assemble_p2(*args, C.byref(nnz), _lp(rowptr), _ip(col), _dp(valM), _dp(valF), _dp(g)))
    return rowptr, col, valM, valF, g


def irk_fem_assemble_supg(xy, tri, eps, wind, wind_c, ub=None, gamma=10.0):
    """All-node CSR (rowptr, col, valM, valF) and lift g of the SUPG / Nitsche
    double-glazing discretisation."""
    L = lib()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    wind = np.ascontiguousarray(wind, dtype=np.float64)
    wind_c = np.ascontiguousarray(wind_c, dtype=np.float64)
    ub = None if ub is None else np.ascontiguousarray(ub, dtype=np.float64)
    n = xy.shape[0]
    nnz = C.c_int64(0)
    args = (n, _dp(xy), tri.shape[0], _ip(tri), float(eps), _dp(wind), _dp(wind_c), _dp(ub), float(gamma))
    check(L.irk_fem_assemble_supg(*args, C.byref(nnz), None, None, None, None, None))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz.value, dtype=np.int32)
    valM = np.zeros(nnz.value)
    valF = np.zeros(nnz.value)
    g = np.zeros(n)
    check(L.irk_fem_assemble_supg(*args, C.byref(nnz), _lp(rowptr), _ip(col), _dp(valM), _dp(valF), _dp(g)))
    return rowptr, col, valM, valF, g


def irk_fem_assemble_streamline(xy, tri, eps, wind_c, rowptr, col):
    """Streamline-diffusion matrix of the coarse-level SUPG stabilisation on the
    pattern (rowptr, col) of irk_fem_assemble_supg."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    wind_c = np.ascontiguousarray(wind_c, dtype=np.float64)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    valT = np.zeros(col.size)
    check(lib().irk_fem_assemble_streamline(xy.shape[0], _dp(xy), tri.shape[0], _ip(tri), float(eps), _dp(wind_c),
                                            _lp(rowptr), _ip(col), _dp(valT)))
    return valT


# ---------------------------------------------------------------------------
# context
# ---------------------------------------------------------------------------
class Context:
    """An irk_ctx plus the host arrays its set-up referenced."""

    def __init__(self, handle, n, s, n_tri):
        self.handle = handle
        self.n = n
        self.s = s
        self.n_tri = n_tri

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if getattr(self, "handle", None):
            lib().irk_destroy(self.handle)
            self.handle = None

    @property
    def ptr(self):
        if not self.handle:
            raise RuntimeError("context destroyed")
        return self.handle


def irk_setup(rowptr, col, valM, valF, butcher, h_t, options=None, g=None, mesh=None, stream=None,
              stab=None) -> Context:
    """butcher = (A, b, c); mesh = dict(xy, tri, dof) or None; stream = a
    torch.cuda.Stream (None: the current stream); stab = the streamline
    matrix's values on the pattern of M (coarse-level SUPG stabilisation) or None."""
    import torch
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    valM = np.ascontiguousarray(valM, dtype=np.float64)
    valF = np.ascontiguousarray(valF, dtype=np.float64)
    n = rowptr.size - 1
    A, b, c = (np.ascontiguousarray(x, dtype=np.float64) for x in butcher)
    s = A.shape[0]
    keep = [rowptr, col, valM, valF, A, b, c]
    prob = IrkProblem()
    prob.M = IrkCsr(n, col.size, _lp(rowptr), _ip(col), _dp(valM))
    prob.F = IrkCsr(n, col.size, _lp(rowptr), _ip(col), _dp(valF))
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float64)
        keep.append(g)
    prob.g = _dp(g)
    if stab is not None:
        stab = np.ascontiguousarray(stab, dtype=np.float64)
        if stab.size != col.size:
            raise ValueError("stab must hold one value per entry of the pattern of M")
        keep.append(stab)
    prob.stab = _dp(stab)
    n_tri = 0
    if mesh is not None:
        xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        dof = np.ascontiguousarray(mesh["dof"], dtype=np.int32)
        keep += [xy, tri, dof]
        prob.n_nodes = xy.shape[0]
        prob.n_tri = tri.shape[0]
        prob.xy, prob.tri, prob.dof = _dp(xy), _ip(tri), _ip(dof)
        n_tri = tri.shape[0]
    bt = IrkButcher(s, _dp(A), _dp(b), _dp(c))
    opts = options if options is not None else irk_default_options()
    At = None
    if opts.kind == PC_KINDS["CUSTOM"] and not opts.Atilde:
        raise ValueError("CUSTOM preconditioner needs Atilde")
    if stream is None:
        stream = torch.cuda.current_stream()
    out = C.c_void_p()
    check(lib().irk_setup(C.byref(prob), C.byref(bt), float(h_t), C.byref(opts), C.c_void_p(stream.cuda_stream),
                          C.byref(out)))
    del keep, At
    return Context(out, n, s, n_tri)


def irk_step(ctx: Context, u_n, u_np1, k=None) -> dict:
    st = IrkStats()
    check(lib().irk_step(ctx.ptr, _dev(u_n), _dev(u_np1), _dev(k), C.byref(st)), ctx.ptr)
    return st.as_dict()


def irk_solve(ctx: Context, b, k) -> dict:
    """Solve the stage system for the right-hand side b (s*n FP64, stage-major) into k."""
    st = IrkStats()
    check(lib().irk_solve(ctx.ptr, _dev(b), _dev(k), C.byref(st)), ctx.ptr)
    return st.as_dict()


def irk_run(ctx: Context, u0, nsteps, u_out, ckpt=None, ckpt_every=0) -> dict:
    st = IrkStats()
    check(lib().irk_run(ctx.ptr, _dev(u0), int(nsteps), _dev(u_out), _dev(ckpt), int(ckpt_every), C.byref(st)),
          ctx.ptr)
    return st.as_dict()


def irk_adjoint_step(ctx: Context, lam_np1, u_n, k_n, lam_n, grad_kappa=None) -> dict:
    st = IrkStats()
    check(lib().irk_adjoint_step(ctx.ptr, _dev(lam_np1), _dev(u_n), _dev(k_n), _dev(lam_n), _dev(grad_kappa),
                                 C.byref(st)), ctx.ptr)
    return st.as_dict()


def irk_adjoint_run(ctx: Context, ckpt, nsteps, ckpt_every, lam, grad_kappa=None) -> dict:
    st = IrkStats()
    check(lib().irk_adjoint_run(ctx.ptr, _dev(ckpt), int(nsteps), int(ckpt_every), _dev(lam), _dev(grad_kappa),
                                C.byref(st)), ctx.ptr)
    return st.as_dict()


class Batch:
    """An irk_batch and the tensors it is bound to."""

    def __init__(self, handle, ctxs, tensors):
        self.handle = handle
        self.ctxs = ctxs
        self.tensors = tensors

    def close(self):
        if getattr(self, "handle", None):
            lib().irk_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(ts):
    return (C.c_void_p * len(ts))(*[C.c_void_p(t.data_ptr()) if t is not None else None for t in ts])


def irk_batch_create(ctxs, nsteps, ckpt_every, u0s, uNs, ckpts, lambdas=None, grads=None) -> Batch:
    for t in list(u0s) + list(uNs) + list(ckpts) + list(lambdas or []) + [g for g in (grads or []) if g is not None]:
        _dev(t)
    n = len(ctxs)
    handles = (C.c_void_p * n)(*[c.ptr for c in ctxs])
    out = C.c_void_p()
    lam = _ptr_array(lambdas) if lambdas is not None else None
    gr = _ptr_array(grads) if grads is not None else None
    check(lib().irk_batch_create(handles, n, int(nsteps), int(ckpt_every), _ptr_array(u0s), _ptr_array(uNs),
                                 _ptr_array(ckpts), lam, gr, C.byref(out)))
    return Batch(out, list(ctxs), [u0s, uNs, ckpts, lambdas, grads])


def _batch_call(fn, b, stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    stats = (IrkStats * len(b.ctxs))()
    ms = C.c_double(0.0)
    check(fn(b.handle, C.c_void_p(stream.cuda_stream), stats, C.byref(ms)))
    return [s.as_dict() for s in stats], ms.value


def irk_batch_run(b: Batch, stream=None):
    return _batch_call(lib().irk_batch_run, b, stream)


def irk_batch_adjoint(b: Batch, stream=None):
    return _batch_call(lib().irk_batch_adjoint, b, stream)


def irk_batch_destroy(b: Batch):
    b.close()


def irk_set_kappa(ctx: Context, kappa):
    check(lib().irk_set_kappa(ctx.ptr, _dev(kappa)), ctx.ptr)


def irk_apply_operator(ctx: Context, z, w, transpose=False):
    check(lib().irk_apply_operator(ctx.ptr, _dev(z), _dev(w), int(bool(transpose))), ctx.ptr)


def irk_apply_operator_f32(ctx: Context, z, w, transpose=False):
    """w (FP64) = the stage operator applied to an FP32 z, as FGMRES applies it
    to FP32 preconditioner outputs."""
    import torch
    if not (z.is_cuda and z.dtype == torch.float32 and z.is_contiguous()):
        raise ValueError("z must be a contiguous float32 CUDA tensor")
    check(lib().irk_apply_operator_f32(ctx.ptr, C.c_void_p(z.data_ptr()), _dev(w), int(bool(transpose))), ctx.ptr)


def irk_apply_precond(ctx: Context, v, z, transpose=False):
    check(lib().irk_apply_precond(ctx.ptr, _dev(v), _dev(z), int(bool(transpose))), ctx.ptr)


def irk_vcycle(ctx: Context, stage, b, x):
    check(lib().irk_vcycle(ctx.ptr, int(stage), _dev(b), _dev(x)), ctx.ptr)


def irk_residual_norm(ctx: Context, k, b) -> float:
    out = C.c_double(0.0)
    check(lib().irk_residual_norm(ctx.ptr, _dev(k), _dev(b), C.byref(out)), ctx.ptr)
    return out.value


def irk_residual_norm_noalloc(ctx: Context, k, b, out):
    """Allocation-free variant: the norm is written to the one-element FP64
    CUDA tensor `out`."""
    check(lib().irk_residual_norm_noalloc(ctx.ptr, _dev(k), _dev(b), _dev(out)), ctx.ptr)


def irk_apply_mass(ctx: Context, x, y):
    check(lib().irk_apply_mass(ctx.ptr, _dev(x), _dev(y)), ctx.ptr)


def irk_misfit(ctx: Context, u, d, value, grad=None):
    """value (one-element FP64 CUDA tensor) = 1/2 (u - d)^T M (u - d); grad
    (n, or None) = M (u - d)."""
    check(lib().irk_misfit(ctx.ptr, _dev(u), _dev(d), _dev(grad), _dev(value)), ctx.ptr)


def irk_amg_info(ctx: Context, stage):
    nl = C.c_int32(0)
    rows = np.zeros(16, dtype=np.int32)
    nnz = np.zeros(16, dtype=np.int64)
    check(lib().irk_amg_info(ctx.ptr, int(stage), C.byref(nl), _ip(rows), _lp(nnz)), ctx.ptr)
    return rows[: nl.value].tolist(), nnz[: nl.value].tolist()


def irk_amg_aggregates(ctx: Context, stage, level):
    rows, _ = irk_amg_info(ctx, stage)
    agg = np.zeros(rows[level], dtype=np.int32)
    check(lib().irk_amg_aggregates(ctx.ptr, int(stage), int(level), _ip(agg)), ctx.ptr)
    return agg


def irk_amg_level_matrix(ctx: Context, stage, level):
    rows, nnz = irk_amg_info(ctx, stage)
    rp = np.zeros(rows[level] + 1, dtype=np.int64)
    col = np.zeros(nnz[level], dtype=np.int32)
    val = np.zeros(nnz[level])
    check(lib().irk_amg_level_matrix(ctx.ptr, int(stage), int(level), _lp(rp), _ip(col), _dp(val)), ctx.ptr)
    return rp, col, val


PROFILE_TARGETS = {"kron": 0, "vcycle": 1, "precond": 2, "gs_dots": 3, "gs_axpy": 4, "smooth0": 5,
                   "vcycle_from": 6}


def irk_profile(ctx: Context, which: str, j: int = 0, warm: int = 3, reps: int = 20) -> dict:
    ms = C.c_double(0.0)
    by = C.c_double(0.0)
    fl = C.c_double(0.0)
    check(lib().irk_profile(ctx.ptr, PROFILE_TARGETS[which], int(j), int(warm), int(reps), C.byref(ms), C.byref(by),
                            C.byref(fl)), ctx.ptr)
    return {"ms": ms.value, "bytes": by.value, "flops": fl.value}


def irk_kernel_launches(ctx: Context) -> int:
    return int(lib().irk_kernel_launches(ctx.ptr))


def irk_destroy(ctx: Context):
    ctx.close()
