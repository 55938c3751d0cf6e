"""ctypes declarations of the libmstress C ABI (include/mstress.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Loading fails loudly when libmstress.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmstress.so")

MSTRESS_OK = 0
MSTRESS_EINVAL = -1
MSTRESS_ENOMEM = -2
MSTRESS_ENOT_CONVERGED = -3
MSTRESS_EDEVICE_TIMEOUT = -4
MSTRESS_ENUMERIC = -5
MSTRESS_ECUDA = -6

MSTRESS_FP64 = 0
MSTRESS_TF32 = 1
MSTRESS_BF16 = 2
MSTRESS_BF16X3 = 3

MSTRESS_BLOCK_KR = 0
MSTRESS_BLOCK_BR = 1
MSTRESS_BLOCK_S = 2
MSTRESS_BLOCK_F = 3
MSTRESS_BLOCK_SMEAN = 4
MSTRESS_BLOCK_SGRID = 5

MSTRESS_COEFF = 0
MSTRESS_VM_ELEM = 1
MSTRESS_SIGMA_GP = 2
MSTRESS_U_NODE = 3
MSTRESS_LATTICE = 4
MSTRESS_VM_GRID = 5

MSTRESS_RQ_QUEUED = 0
MSTRESS_RQ_RUNNING = 1
MSTRESS_RQ_DONE = 2
MSTRESS_RQ_FAILED = 3

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ENOT_CONVERGED", -4: "EDEVICE_TIMEOUT",
                -5: "ENUMERIC", -6: "ECUDA"}


class mstress_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("alpha", C.c_double)]


class mstress_block_mesh(C.Structure):
    _fields_ = [("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("ex", C.c_int), ("ey", C.c_int), ("ez", C.c_int),
                ("mat_id", C.POINTER(C.c_uint8))]


class mstress_tsv_geom(C.Structure):
    _fields_ = [("r_cu", C.c_double), ("t_liner", C.c_double)]


class mstress_layout(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("site_type", C.POINTER(C.c_uint8)),
                ("blocks", C.POINTER(C.c_void_p)), ("n_blocks", C.c_int)]


class mstress_bc(C.Structure):
    _fields_ = [("clamp_bottom", C.c_int), ("clamp_top", C.c_int),
                ("prescribed_dof", C.POINTER(C.c_int64)), ("prescribed_val", C.POINTER(C.c_double)),
                ("n_prescribed", C.c_size_t)]


class mstress_strip(C.Structure):
    _fields_ = [("j0", C.c_int), ("j1", C.c_int), ("y_own0", C.c_int), ("y_own1", C.c_int),
                ("y_send", C.c_int), ("y_recv", C.c_int), ("prev", C.c_int), ("next", C.c_int)]


class mstress_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int),
                ("inner_rtol", C.c_double), ("max_outer", C.c_int), ("hbm_budget", C.c_size_t),
                ("offline_max_iter", C.c_int), ("offline_rtol", C.c_double)]


P = C.c_void_p
I = C.c_int
PI = C.POINTER(C.c_int)
PD = C.POINTER(C.c_double)
PSZ = C.POINTER(C.c_size_t)

# name: (restype, argtypes) -- every function declared in include/mstress.h
SIGNATURES = {
    "mstress_opts_default": (I, [C.POINTER(mstress_opts)]),
    "mstress_create": (I, [C.POINTER(P), P, C.POINTER(mstress_opts)]),
    "mstress_set_opts": (I, [P, C.POINTER(mstress_opts)]),
    "mstress_get_opts": (I, [P, C.POINTER(mstress_opts)]),
    "mstress_free_ctx": (None, [P]),
    "mstress_last_error": (C.c_char_p, [P]),
    "mstress_mem_info": (I, [P, PSZ, PSZ]),
    "mstress_sync": (I, [P]),
    "mstress_build_block": (I, [P, C.POINTER(mstress_block_mesh), C.POINTER(mstress_tsv_geom),
                                C.POINTER(mstress_material), I, I, C.POINTER(P)]),
    "mstress_block_import": (I, [P, C.POINTER(mstress_block_mesh), I, PD, PD, PD, PD, C.POINTER(P)]),
    "mstress_block_export": (I, [P, I, PD, C.c_size_t]),
    "mstress_block_info": (I, [P, PI, PI, PI, PI]),
    "mstress_block_grid": (I, [P, I]),
    "mstress_free_block": (None, [P]),
    "mstress_solve": (I, [P, C.POINTER(mstress_layout), C.c_double, C.POINTER(mstress_bc), C.POINTER(P)]),
    "mstress_solve_batch": (I, [P, C.POINTER(mstress_layout), PD, C.POINTER(mstress_bc), I, C.POINTER(P)]),
    "mstress_recover_size": (I, [P, I, PSZ]),
    "mstress_recover": (I, [P, P, I, P, C.c_size_t, I]),
    "mstress_sol_info": (I, [P, I, PI, PI, PD, PI]),
    "mstress_sol_count": (I, [P, PI, C.POINTER(C.c_int64)]),
    "mstress_sol_tiling": (I, [P, PI, PI, PI]),
    "mstress_free_sol": (None, [P]),
    "mstress_apply": (I, [P, C.POINTER(mstress_layout), P, P, I]),
    "mstress_launch_count": (I, [C.POINTER(C.c_int64)]),
    "mstress_set_wait_limit": (I, [P, C.c_int64, I]),
    "mstress_strip_partition": (I, [I, I, I, I, C.POINTER(mstress_strip)]),
    "mstress_profile": (I, [P, P, I, I, PD]),
    "mstress_apply_noalloc": (I, [P, I, I, P, P, P]),
    "mstress_sol_phase_ms": (I, [P, PD]),
    "mstress_server_create": (I, [P, I, C.c_size_t, C.POINTER(P)]),
    "mstress_server_submit": (I, [P, C.POINTER(mstress_layout), C.c_double, C.POINTER(mstress_bc),
                                  C.POINTER(C.c_int64)]),
    "mstress_server_step": (I, [P, PI, PI, PI]),
    "mstress_server_poll": (I, [P, C.POINTER(C.c_int64)]),
    "mstress_server_info": (I, [P, C.c_int64, PI, PI, PI, PD, PD]),
    "mstress_server_result": (I, [P, C.c_int64, P, C.c_size_t, I]),
    "mstress_server_release": (I, [P, C.c_int64]),
    "mstress_free_server": (None, [P]),
}

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libmstress.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libmstress.so is not built ({path}); run paper_2411_12690_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
