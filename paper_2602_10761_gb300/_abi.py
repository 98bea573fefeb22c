"""ctypes declarations of the C ABI in include/tribo.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

TRIBO_OK = 0
TRIBO_ERR_ARG = 1
TRIBO_ERR_UNSUPPORTED = 2
TRIBO_ERR_CUDA = 3
TRIBO_ERR_OOM = 4
TRIBO_ERR_DEVICE = 5
TRIBO_ERR_CAPACITY = 6

TRIBO_DEV_ESCAPED = 0x1
TRIBO_DEV_NONFINITE = 0x2
TRIBO_DEV_OUTSIDE = 0x4
TRIBO_DEV_TIMEOUT = 0x8

TRIBO_FP64 = 0
TRIBO_MIXED = 1
TRIBO_DRAG_STOKES = 0
TRIBO_DRAG_SCHILLER_NAUMANN = 1
TRIBO_DRAG_OFF = 2
TRIBO_IMPACT_SPEED = 0
TRIBO_IMPACT_NORMAL = 1
TRIBO_NPHASES = 12


class tribo_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("lx", C.c_double), ("lz", C.c_double), ("y_faces", C.POINTER(C.c_double))]


class tribo_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mu_p", "E_p", "phi_p", "k_e", "mu_w", "E_w", "eps_w", "h", "eps", "eps0",
                 "nu", "rho", "rho_p", "U_c", "kappa_A")] + \
               [(n, C.c_int32) for n in
                ("drag_law", "impact_vel", "dq_t", "electrostatics", "precision", "sort_every", "coulomb", "collisions")]


class tribo_fluid(C.Structure):
    _fields_ = [("u", C.c_void_p), ("on_host", C.c_int32)]


class tribo_modes(C.Structure):
    _fields_ = [("n_modes", C.c_int32), ("nxi", C.c_void_p), ("nzi", C.c_void_p), ("ky", C.c_void_p),
                ("amp", C.c_void_p), ("phase", C.c_void_p), ("ubar", C.c_void_p), ("damp", C.c_void_p),
                ("t0", C.c_double)]


class tribo_ssm(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("r0", "un0", "mu0", "sigma0", "gamma0", "dq0_min", "c_sat")] + \
               [("seed", C.c_uint64)]


class tribo_particles(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(n, C.c_void_p) for n in ("x", "y", "z", "vx", "vy", "vz", "d")] + \
               [("q", C.c_void_p), ("q_wall", C.c_void_p), ("n_imp", C.c_void_p), ("id", C.c_void_p),
                ("cell", C.c_void_p), ("on_host", C.c_int32), ("site", C.c_void_p)]


_SIGS = {
    "tribo_init": (C.c_int32, [C.POINTER(C.c_void_p), C.POINTER(tribo_grid), C.POINTER(tribo_fluid),
                               C.POINTER(tribo_params), C.c_int64, C.c_void_p]),
    "tribo_set_fluid": (C.c_int32, [C.c_void_p, C.POINTER(tribo_fluid)]),
    "tribo_set_params": (C.c_int32, [C.c_void_p, C.POINTER(tribo_params)]),
    "tribo_set_modes": (C.c_int32, [C.c_void_p, C.POINTER(tribo_modes)]),
    "tribo_set_ssm": (C.c_int32, [C.c_void_p, C.POINTER(tribo_ssm)]),
    "tribo_set_momentum_source": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "tribo_set_adjoint_memory": (C.c_int32, [C.c_void_p, C.c_int64]),
    "tribo_transfer_bytes": (C.c_int32, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "tribo_eval_modes": (C.c_int32, [C.c_void_p, C.c_double, C.c_void_p]),
    "tribo_step": (C.c_int32, [C.c_void_p, C.POINTER(tribo_particles), C.c_double, C.c_int32]),
    "tribo_poisson": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tribo_adjoint": (C.c_int32, [C.c_void_p, C.POINTER(tribo_particles), C.c_double, C.c_int32, C.c_int32,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.c_void_p]),
    "tribo_poisson_noalloc": (C.c_int32, [C.POINTER(tribo_grid), C.c_double, C.c_int32, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "tribo_stats": (C.c_int32, [C.c_void_p, C.POINTER(tribo_particles), C.POINTER(C.c_double),
                                C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_int64)]),
    "tribo_reset_stats": (C.c_int32, [C.c_void_p]),
    "tribo_sync": (C.c_int32, [C.c_void_p]),
    "tribo_error_bits": (C.c_uint32, [C.c_void_p]),
    "tribo_clear_error": (C.c_int32, [C.c_void_p]),
    "tribo_test_pipeline_wait": (C.c_int32, [C.c_void_p, C.c_int32]),
    "tribo_launch_count": (C.c_int64, [C.c_void_p]),
    "tribo_timing_enable": (C.c_int32, [C.c_void_p, C.c_int32]),
    "tribo_timing_read": (C.c_int32, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "tribo_phase_name": (C.c_char_p, [C.c_int32]),
    "tribo_batch_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p), C.c_int32,
                                       C.c_void_p]),
    "tribo_batch_autotune": (C.c_int32, [C.c_void_p, C.POINTER(C.POINTER(tribo_particles)), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int32)]),
    "tribo_batch_step": (C.c_int32, [C.c_void_p, C.POINTER(C.POINTER(tribo_particles)), C.POINTER(C.c_double),
                                     C.c_int32]),
    "tribo_batch_sync": (C.c_int32, [C.c_void_p]),
    "tribo_batch_launch_count": (C.c_int64, [C.c_void_p]),
    "tribo_batch_timing": (C.c_int32, [C.c_void_p, C.c_int32]),
    "tribo_batch_kernel_time": (C.c_int32, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "tribo_batch_destroy": (None, [C.c_void_p]),
    "tribo_strerror": (C.c_char_p, [C.c_int32]),
    "tribo_last_error": (C.c_char_p, []),
    "tribo_destroy": (None, [C.c_void_p]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load libtribo.so (raises if it is not built; there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libtribo.so is not built ({path}); call paper_2602_10761_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_names() -> list:
    return sorted(_SIGS)


class TriboError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.tribo_strerror(status).decode()
        detail = lib.tribo_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def check(status: int, where: str) -> None:
    if status != TRIBO_OK:
        raise TriboError(status, where)
