"""ctypes declarations of include/goc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from .build import LIB, build

c_int, c_double, c_ll, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p
P = ctypes.POINTER


class GocGrid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("bc", c_int * 4), ("wall_u", c_double * 4),
                ("wall_b", (c_double * 2) * 4)]


class GocMap(ctypes.Structure):
    _fields_ = [("kind", c_int * 2), ("beta", c_double * 2), ("a", c_double * 2),
                ("gamma", c_double * 2), ("alpha", c_double * 2), ("mu", c_double * 2), ("yc", c_double * 2),
                ("r_inner", c_double), ("r_outer", c_double), ("sectors", c_double),
                ("table", c_void_p), ("wall_table", c_void_p)]


class GocFlow(ctypes.Structure):
    _fields_ = [("rho0", c_double), ("tau", c_double), ("nu", c_double), ("tau_zeta", c_double),
                ("omega_free", c_double), ("fext", c_double * 2), ("gi_correction", c_int)]


class GocMhd(ctypes.Structure):
    _fields_ = [("enabled", c_int), ("tau_m", c_double), ("eta", c_double), ("mu_m", c_double),
                ("b_init", c_double * 2)]


class GocExec(ctypes.Structure):
    _fields_ = [("storage", c_int), ("cuda_stream", c_void_p), ("device", c_int), ("check_every", c_int),
                ("rounding", c_int), ("scheme", c_int), ("fixed_launch", c_int), ("plateau_checks", c_int),
                ("reference_every", c_int), ("streaming", c_int)]


GOC_OK, GOC_EINVAL, GOC_ENOMEM, GOC_ECUDA, GOC_EDIVERGED, GOC_ETIMEOUT, GOC_EBUSY, GOC_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
MAPS = {"uniform": 0, "tanh2": 1, "sine": 2, "roberts": 3, "tanh1": 4, "sinh": 5, "annulus": 6, "table": 7}

# name -> (restype, argtypes); every entry point of include/goc.h
SIGNATURES = {
    "goc_metric_info": (c_int, [P(GocGrid), P(GocMap), P(c_double), P(c_double)]),
    "goc_create": (c_int, [P(GocGrid), P(GocMap), P(GocFlow), P(GocMhd), P(GocExec), P(c_void_p)]),
    "goc_init_fields": (c_int, [c_void_p] + [P(c_double)] * 5),
    "goc_destroy": (None, [c_void_p]),
    "goc_step": (c_int, [c_void_p, c_ll]),
    "goc_run_until": (c_int, [c_void_p, c_double, c_ll, P(c_ll), P(c_double)]),
    "goc_sync": (c_int, [c_void_p]),
    "goc_moments": (c_int, [c_void_p, c_int] + [P(c_double)] * 5),
    "goc_moments_device": (c_int, [c_void_p, c_void_p]),
    "goc_diagnostics": (c_int, [c_void_p, P(c_double), P(c_double), P(c_double)]),
    "goc_steps_done": (c_ll, [c_void_p]),
    "goc_footprint": (c_int, [c_void_p, P(c_ll), P(c_ll)]),
    "goc_bytes_per_node": (c_double, [c_void_p]),
    "goc_get_state": (c_int, [c_void_p, c_void_p, P(ctypes.c_size_t)]),
    "goc_set_state": (c_int, [c_void_p, c_void_p, ctypes.c_size_t]),
    "goc_batch_create": (c_int, [c_ll, c_int, P(GocExec), P(c_void_p)]),
    "goc_batch_destroy": (None, [c_void_p]),
    "goc_batch_add": (c_int, [c_void_p, P(GocGrid), P(GocMap), P(GocFlow), P(GocMhd), c_int, P(c_int)]),
    "goc_batch_remove": (c_int, [c_void_p, c_int]),
    "goc_batch_step": (c_int, [c_void_p, c_ll]),
    "goc_batch_lattice": (c_int, [c_void_p, c_int, P(c_void_p)]),
    "goc_batch_check": (c_int, [c_void_p, c_int, c_int]),
    "goc_batch_residual": (c_int, [c_void_p, c_int, P(c_double), P(c_double)]),
    "goc_batch_usage": (c_int, [c_void_p, P(c_ll), P(c_ll), P(c_int)]),
    "goc_mass_noalloc": (c_int, [c_void_p, P(c_double)]),
    "goc_selftest_bounded_wait": (c_int, [c_ll]),
    "goc_check_guards": (c_int, [c_void_p, P(c_ll)]),
    "goc_launch_config": (c_int, [c_void_p, P(c_int), P(c_int), P(c_int)]),
    "goc_set_launch_config": (c_int, [c_void_p, c_int, c_int]),
    "goc_launch_grid": (c_int, [c_void_p, P(c_int)]),
    "goc_set_launch_grid": (c_int, [c_void_p, c_int]),
    "goc_tile_height": (c_int, [c_void_p, P(c_int)]),
    "goc_set_tile_height": (c_int, [c_void_p, c_int]),
    "goc_create_slab": (c_int, [P(GocGrid), P(GocMap), P(GocFlow), P(GocMhd), P(GocExec), c_int, c_int,
                                P(c_void_p)]),
    "goc_slab_info": (c_int, [c_void_p] + [P(c_int)] * 4),
    "goc_slab_halo_bytes": (c_ll, [c_void_p]),
    "goc_slab_pack": (c_int, [c_void_p, c_void_p, c_void_p]),
    "goc_slab_unpack": (c_int, [c_void_p, c_void_p, c_void_p]),
    "goc_last_error": (ctypes.c_char_p, []),
}

_lib = None


class GocError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"goc status {status}: {msg}")
        self.status = status


def lib(build_if_missing: bool = True):
    """Load libgoc.so (building it first when sources are newer).  Raises if
    the library cannot be loaded: there is no fallback implementation."""
    global _lib
    if _lib is None:
        path = build() if build_if_missing else LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgoc.so not found at {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != GOC_OK:
        raise GocError(status, lib().goc_last_error().decode())
    return status
