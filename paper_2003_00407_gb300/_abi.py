"""ctypes mirror of include/dgdft.h (structures, status codes, prototypes)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgdft.so")

OK, INVALID_ARG, OUT_OF_MEMORY, NOT_CONVERGED, CHOLESKY_FAIL, BAD_INPUT, TIMEOUT, CUDA_ERROR, UNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "INVALID_ARG", "OUT_OF_MEMORY", "NOT_CONVERGED", "CHOLESKY_FAIL", "BAD_INPUT", "TIMEOUT",
                "CUDA_ERROR", "UNSUPPORTED"]
FP64, MIXED = 0, 1
CHEFSI, LOBPCG = 0, 1
HOST_BUFFERS = 1

PI = C.POINTER(C.c_int)
PD = C.POINTER(C.c_double)
PL = C.POINTER(C.c_int64)


class Problem(C.Structure):
    _fields_ = [("n_dom", C.c_int), ("dom_n", PI), ("dom_h", PD), ("dom_voff", PL), ("v_extra", C.c_void_p),
                ("n_elem", C.c_int), ("elem_dom", PI), ("elem_E0", PI), ("elem_En", PI), ("elem_Qn", PI),
                ("neighbors", PI), ("n_stencil", C.c_int), ("n_atoms", C.c_int), ("atom_dom", PI),
                ("atom_pos", PD), ("well_depth", PD), ("well_width", PD), ("n_proj_per_atom", C.c_int),
                ("proj_gamma", PD), ("proj_width", PD), ("r_cut", C.c_double)]


class AlbParams(C.Structure):
    _fields_ = [("n_eig", PI), ("n_alb", PI), ("n_blk", PI), ("cheb_degree", C.c_int), ("tol", C.c_double),
                ("tol_mixed", C.c_double), ("max_iter", C.c_int), ("lanczos_steps", C.c_int),
                ("precision", C.c_int), ("seed", C.c_uint64), ("flags", C.c_int), ("x0", C.c_void_p),
                ("solver", C.c_int)]


class AlbResult(C.Structure):
    _fields_ = [("eigval", C.c_void_p), ("resid", C.c_void_p), ("sing", C.c_void_p), ("coef", C.c_void_p),
                ("alb", C.c_void_p), ("eigvec", C.c_void_p), ("iters", C.c_void_p), ("status", C.c_void_p),
                ("history", C.c_void_p)]


class DGSolveParams(C.Structure):
    _fields_ = [("n_states", C.c_int), ("n_blk", C.c_int), ("cheb_degree", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("lanczos_steps", C.c_int), ("seed", C.c_uint64)]


FUNCTIONS = {
    "dgdft_alb_query_sizes": (C.c_int, [C.POINTER(Problem), C.POINTER(AlbParams), PL]),
    "dgdft_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "dgdft_ctx_destroy": (None, [C.c_void_p]),
    "dgdft_last_error": (C.c_char_p, [C.c_void_p]),
    "dgdft_kernel_launches": (C.c_int64, []),
    "dgdft_alb_generate": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.POINTER(AlbResult),
                                     C.c_void_p]),
    "dgdft_dg_assemble": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.POINTER(AlbResult),
                                    C.c_double, C.c_void_p, C.c_void_p]),
    "dgdft_alb_grad": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.POINTER(AlbResult),
                                 C.c_double, PD, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgdft_apply_hamiltonian": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
    "dgdft_chebyshev_filter": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), PD, C.c_void_p,
                                         C.c_void_p, C.c_void_p]),
    "dgdft_dg_query_layout": (C.c_int, [C.POINTER(Problem), C.POINTER(AlbParams), PL, PL]),
    "dgdft_dg_ingredients": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.POINTER(AlbResult),
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgdft_dg_blocks": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "dgdft_dg_eigensolve": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.c_void_p,
                                      C.POINTER(DGSolveParams), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "dgdft_dg_density": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.POINTER(AlbParams), C.POINTER(AlbResult),
                                   C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    "dgdft_stage_converged": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, PD, PI]),
    "dgdft_gram_fp32": (C.c_int, [C.c_void_p, C.c_int, PI, PI, PI, PD, C.c_void_p, PL, C.c_void_p, PL, C.c_void_p,
                                  C.c_int, C.c_void_p]),
    "dgdft_rotate_fp32": (C.c_int, [C.c_void_p, C.c_int, PI, PI, PI, C.c_void_p, PL, C.c_void_p, C.c_int, C.c_void_p,
                                    PL, C.c_void_p]),
    "dgdft_apply_hamiltonian_noalloc": (C.c_int, [C.POINTER(Problem), C.POINTER(AlbParams), C.c_void_p, C.c_void_p,
                                                  C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libdgdft.so (built in-tree by paper_2003_00407_gb300.build).  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdgdft.so not found at {path}: build it with "
                           "`python -m paper_2003_00407_gb300.build` (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in FUNCTIONS.items():
        if not hasattr(lib, name):
            continue  # reported by tests/test_abi.py
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
