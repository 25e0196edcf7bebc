"""ctypes binding of the C ABI in include/mg.h and include/mg_ops.h.

Argument marshalling only: every step of the solve runs in the CUDA kernels
of ``libmgpu.so``.  Loading fails loudly when the library has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import buildlib as _build

_lock = threading.Lock()
_lib = None

c_int, c_double, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
c_int3 = ctypes.c_int * 3
c_int_p = ctypes.POINTER(ctypes.c_int)
c_ll_p = ctypes.POINTER(ctypes.c_longlong)

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_CUDA, MG_ERR_OOM = 0, 1, 2, 3
MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, MG_ERR_NONFINITE = 4, 5, 6
MG_ERR_TIMEOUT, MG_ERR_UNSUPPORTED = 7, 8
MG_FP64, MG_MIXED = 0, 1
MG_OPS_F64, MG_OPS_F32 = 0, 1
MG_MAX_BOTTOM = 1024
MG_MAX_HIST = 128
MG_ZERO_GUESS = 1

STATUS_NAMES = {
    MG_OK: "ok", MG_ERR_INVALID_ARG: "invalid_arg", MG_ERR_CUDA: "cuda", MG_ERR_OOM: "oom",
    MG_ERR_NOT_CONVERGED: "not_converged", MG_ERR_DIVERGED: "diverged",
    MG_ERR_NONFINITE: "nonfinite", MG_ERR_TIMEOUT: "timeout", MG_ERR_UNSUPPORTED: "unsupported",
}


DEV_ALLOC = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p)
DEV_FREE = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class mg_opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("nu1", c_int), ("nu2", c_int), ("max_cycles", c_int),
                ("use_graph", c_int), ("smoother", c_int), ("coarse_cells", c_int),
                ("inner_cycles", c_int), ("full_residual", c_int), ("tma", c_int),
                ("krylov", c_int), ("max_norm", c_int), ("wait_limit", c_int),
                ("persistent", c_int), ("sweep_zc", c_int), ("level_ctas", c_int),
                ("fp32_setup", c_int), ("reserved", c_int),
                ("dev_alloc", DEV_ALLOC), ("dev_free", DEV_FREE), ("alloc_user", c_void_p)]


class mg_stats(ctypes.Structure):
    _fields_ = [("cycles", c_int), ("status", c_int), ("norm_f", c_double),
                ("rel_resid0", c_double), ("rel_resid", c_double),
                ("hist", c_double * MG_MAX_HIST), ("t_setup_ms", ctypes.c_float),
                ("t_solve_ms", ctypes.c_float), ("rel_resid_max", c_double)]


MG_PROF_NKIND = 16
PROF_NAMES = ["sweep", "pass", "restrict", "prolong", "norm", "coarse", "refine", "krylov",
              "level", "sweep_prolong"]


class mg_profile(ctypes.Structure):
    _fields_ = [("ms", c_double * MG_PROF_NKIND), ("launches", c_ll * MG_PROF_NKIND),
                ("kernels", c_ll), ("cells", c_ll * MG_PROF_NKIND)]


_SIGS = {
    # mg.h
    "mg_default_opts": (None, [ctypes.POINTER(mg_opts)]),
    "mg_create": (c_int, [ctypes.POINTER(c_void_p), c_int3, c_double, c_int,
                          ctypes.POINTER(mg_opts)]),
    "mg_set_beta": (c_int, [c_void_p, c_void_p, c_void_p]),
    "mg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(mg_stats),
                         c_void_p]),
    "mg_solve_multi": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double,
                               ctypes.POINTER(mg_stats), c_void_p]),
    "mg_solve_ex": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int,
                            ctypes.POINTER(mg_stats), c_void_p]),
    "mg_adjoint": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_double,
                           ctypes.POINTER(mg_stats), c_void_p]),
    "mg_levels": (c_int, [c_void_p, c_int_p, c_int_p]),
    "mg_smoother_kind": (c_int, [c_void_p, c_int, c_int_p]),
    "mg_project_rhs": (c_int, [c_void_p] * 7),
    "mg_project_correct": (c_int, [c_void_p] * 6),
    "mg_bc_lift": (c_int, [c_void_p] * 5),
    "mg_level_create": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int, c_void_p]),
    "mg_level_set_beta": (c_int, [c_void_p] * 3),
    "mg_level_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p]),
    "mg_level_solve_ex": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p,
                                  c_void_p]),
    "mg_level_levels": (c_int, [c_void_p, c_void_p]),
    "mg_level_destroy": (None, [c_void_p]),
    "mg_level_intersections": (c_int, [c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                       c_int]),
    "mg_destroy": (None, [c_void_p]),
    "mg_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int_p,
                                ctypes.POINTER(c_double), c_int, ctypes.POINTER(mg_opts)]),
    "mg_batch_set_beta": (c_int, [c_void_p, c_void_p, c_void_p]),
    "mg_solve_batched": (c_int, [c_void_p, c_void_p, c_void_p, c_double,
                                 ctypes.POINTER(mg_stats), c_void_p]),
    "mg_solve_batched_ex": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int,
                                    ctypes.POINTER(mg_stats), c_void_p]),
    "mg_batch_destroy": (None, [c_void_p]),
    "mg_profile_enable": (c_int, [c_void_p, c_int]),
    "mg_profile_read": (c_int, [c_void_p, ctypes.POINTER(mg_profile), c_int]),
    "mg_batch_profile_enable": (c_int, [c_void_p, c_int]),
    "mg_batch_profile_read": (c_int, [c_void_p, ctypes.POINTER(mg_profile), c_int]),
    "mg_level_profile_enable": (c_int, [c_void_p, c_int]),
    "mg_level_profile_read": (c_int, [c_void_p, ctypes.POINTER(mg_profile), c_int]),
    "mg_slab_plan": (c_int, [c_int3, c_int, c_void_p, c_void_p]),
    "mg_slab_halo": (c_int, [c_int3, c_int, c_int, c_void_p, c_void_p, c_int]),
    "mg_slab_create": (c_int, [ctypes.POINTER(c_void_p), c_int3, c_double, c_int, c_void_p,
                               ctypes.POINTER(mg_opts)]),
    "mg_slab_set_beta": (c_int, [c_void_p, c_void_p]),
    "mg_slab_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int,
                              ctypes.POINTER(mg_stats)]),
    "mg_slab_destroy": (None, [c_void_p]),
    "mg_error_string": (ctypes.c_char_p, [c_int]),
    "mg_last_error": (ctypes.c_char_p, []),
    # mg_ops.h
    "mg_layout": (c_int, [c_int3, c_ll_p, c_ll_p, c_ll_p]),
    "mg_op_face_weights": (c_int, [c_int3, c_double, c_int, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p]),
    "mg_op_coarsen_weights": (c_int, [c_int3] + [c_void_p] * 7),
    "mg_op_inv_diag": (c_int, [c_int3] + [c_void_p] * 6),
    "mg_op_round_f32": (c_int, [c_int3] + [c_void_p] * 9),
    "mg_op_rbgs_pass": (c_int, [c_int, c_int3] + [c_void_p] * 6 + [c_int, c_void_p]),
    "mg_op_rbgs_sweep": (c_int, [c_int, c_int3] + [c_void_p] * 6 + [c_int, c_void_p]),
    "mg_op_rbgs_sweep_tma": (c_int, [c_int3] + [c_void_p] * 6 + [c_int, c_void_p]),
    "mg_op_rbgs_sweep_tma_prolong": (c_int, [c_int3] + [c_void_p] * 7 + [c_int, c_void_p]),
    "mg_op_residual": (c_int, [c_int, c_int3] + [c_void_p] * 8),
    "mg_op_residual_restrict": (c_int, [c_int, c_int3] + [c_void_p] * 9),
    "mg_op_residual_restrict_red": (c_int, [c_int, c_int3] + [c_void_p] * 9),
    "mg_op_prolong_add": (c_int, [c_int, c_int3, c_void_p, c_void_p, c_void_p]),
    "mg_op_bottom_inverse": (c_int, [c_int3, c_int] + [c_void_p] * 6),
    "mg_op_bottom_solve": (c_int, [c_int, c_int3] + [c_void_p] * 4),
    "mg_op_norm_scratch": (c_ll, [c_int3]),
    "mg_op_residual_norm": (c_int, [c_int, c_int3] + [c_void_p] * 9),
    "mg_op_residual_norm_noalloc": (c_int, [c_int, c_int3] + [c_void_p] * 8),
    "mg_op_refine": (c_int, [c_int3] + [c_void_p] * 13),
    "mg_op_beta_grad": (c_int, [c_int3, c_double, c_int] + [c_void_p] * 5),
}


def header_symbols():
    """Function names declared in include/*.h (parsed from the text)."""
    names = set()
    inc = os.path.join(_build.ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(inc, fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"\b(mg_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


def load(path: str | None = None):
    """Load libmgpu.so (building it first if sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            if path is None:
                if not _build.up_to_date():
                    _build.build()
                path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: run build() first")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return load().mg_last_error().decode(errors="replace")


class MGError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {last_error()}")


def check(status: int, where: str = "") -> int:
    if status != MG_OK:
        raise MGError(status, where)
    return status
