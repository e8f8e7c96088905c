"""ctypes declarations of the C ABI in include/irk.h (argument marshalling
only).  Loading fails loudly when libirk.so has not been built."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

c_int32_p = C.POINTER(C.c_int32)
c_int64_p = C.POINTER(C.c_int64)
c_double_p = C.POINTER(C.c_double)


class IrkCsr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", c_int64_p),
                ("col", c_int32_p), ("val", c_double_p)]


class IrkButcher(C.Structure):
    _fields_ = [("s", C.c_int32), ("A", c_double_p), ("b", c_double_p), ("c", c_double_p)]


class IrkOptions(C.Structure):
    _fields_ = [("kind", C.c_int32), ("Atilde", c_double_p), ("amg_prec", C.c_int32),
                ("smoother", C.c_int32), ("cheb_degree", C.c_int32), ("cheb_lo", C.c_double),
                ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("theta", C.c_double),
                ("coarse_max", C.c_int32), ("max_levels", C.c_int32), ("restart", C.c_int32),
                ("rtol", C.c_double), ("max_it", C.c_int32), ("reorth", C.c_int32),
                ("reorth_eta", C.c_double), ("side", C.c_int32), ("p_smooth", C.c_int32),
                ("strength", C.c_int32), ("cycle", C.c_int32)]


class IrkStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32),
                ("max_step_iterations", C.c_int32), ("steps", C.c_int32),
                ("resid", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class IrkProblem(C.Structure):
    _fields_ = [("M", IrkCsr), ("F", IrkCsr), ("g", c_double_p), ("n_nodes", C.c_int32),
                ("n_tri", C.c_int32), ("xy", c_double_p), ("tri", c_int32_p), ("dof", c_int32_p),
                ("stab", c_double_p)]


# (name, restype, argtypes) for every entry point of include/irk.h
SIGNATURES = [
    ("irk_butcher_table", C.c_int, [C.c_int32, C.c_int32, c_double_p, c_double_p, c_double_p]),
    ("irk_ldu", C.c_int, [C.c_int32, c_double_p, c_double_p, c_double_p, c_double_p]),
    ("irk_atilde", C.c_int, [C.c_int32, C.c_int32, c_double_p, c_double_p, c_double_p]),
    ("irk_default_options", None, [C.POINTER(IrkOptions)]),
    ("irk_fem_quad_points", C.c_int, [C.c_int32, c_double_p, c_int32_p, c_double_p]),
    ("irk_fem_assemble", C.c_int, [C.c_int32, c_double_p, C.c_int32, c_int32_p, c_int32_p, C.c_int32,
                                   c_double_p, c_double_p, c_double_p, c_int64_p, c_int64_p, c_int32_p,
                                   c_double_p, c_double_p, c_double_p]),
    ("irk_fem_assemble_p2", C.c_int, [C.c_int32, c_double_p, C.c_int32, c_int32_p, c_int32_p, C.c_int32,
                                      c_double_p, c_double_p, c_int64_p, c_int64_p, c_int32_p,
                                      c_double_p, c_double_p, c_double_p]),
    ("irk_fem_assemble_supg", C.c_int, [C.c_int32, c_double_p, C.c_int32, c_int32_p, C.c_double, c_double_p,
                                        c_double_p, c_double_p, C.c_double, c_int64_p, c_int64_p, c_int32_p,
                                        c_double_p, c_double_p, c_double_p]),
    ("irk_misfit", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("irk_fem_assemble_streamline", C.c_int, [C.c_int32, c_double_p, C.c_int32, c_int32_p, C.c_double,
                                              c_double_p, c_int64_p, c_int32_p, c_double_p]),
    ("irk_setup", C.c_int, [C.POINTER(IrkProblem), C.POINTER(IrkButcher), C.c_double,
                            C.POINTER(IrkOptions), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("irk_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(IrkStats)]),
    ("irk_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(IrkStats)]),
    ("irk_run", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                          C.POINTER(IrkStats)]),
    ("irk_adjoint_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.POINTER(IrkStats)]),
    ("irk_adjoint_run", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.POINTER(IrkStats)]),
    ("irk_set_kappa", C.c_int, [C.c_void_p, C.c_void_p]),
    ("irk_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_int32,
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    ("irk_batch_run", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(IrkStats), c_double_p]),
    ("irk_batch_adjoint", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(IrkStats), c_double_p]),
    ("irk_batch_destroy", None, [C.c_void_p]),
    ("irk_apply_operator", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("irk_apply_operator_f32", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("irk_apply_precond", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("irk_vcycle", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("irk_residual_norm", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, c_double_p]),
    ("irk_residual_norm_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("irk_apply_mass", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("irk_amg_info", C.c_int, [C.c_void_p, C.c_int32, c_int32_p, c_int32_p, c_int64_p]),
    ("irk_amg_aggregates", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, c_int32_p]),
    ("irk_amg_level_matrix", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, c_int64_p, c_int32_p, c_double_p]),
    ("irk_profile", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, c_double_p, c_double_p,
                              c_double_p]),
    ("irk_kernel_launches", C.c_int64, [C.c_void_p]),
    ("irk_destroy", None, [C.c_void_p]),
    ("irk_last_error", C.c_char_p, [C.c_void_p]),
    ("irk_status_string", C.c_char_p, [C.c_int]),
]

_lib = None


def lib():
    """The loaded libirk (built in-tree by paper_2010_11377_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libirk.so is not built ({LIB}); run __graft_entry__.build() "
                               "or python -m paper_2010_11377_gb300.build")
        L = C.CDLL(LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class IrkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def check(status, ctx=None):
    if status != 0:
        L = lib()
        msg = L.irk_last_error(ctx)
        raise IrkError(status, (msg or b"").decode() or L.irk_status_string(status).decode())
