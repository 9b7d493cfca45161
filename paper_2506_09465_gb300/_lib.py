"""ctypes binding of libiugkp.so (include/iugkp.h). Argument marshalling only: every step
of the solver runs in the CUDA library. There is no CPU fallback: if the library is
missing or cannot be loaded, loading raises."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libiugkp.so")

STATUS = {0: "IUGKP_OK", 1: "IUGKP_EINVAL", 2: "IUGKP_ENOMEM", 3: "IUGKP_ECUDA", 4: "IUGKP_ENOCONV",
          5: "IUGKP_EBUDGET", 6: "IUGKP_EDEVICE"}

TRACK_FP64, TRACK_FP32 = 0, 1
TALLY_FP64, TALLY_STAGED, TALLY_STAGED_K32 = 0, 1, 2
DRAWS_FRESH, DRAWS_FROZEN = 0, 1
SCHED_PLAIN, SCHED_PERSISTENT = 0, 1
FIELD_SOURCE, FIELD_WALL_T, FIELD_WALL_FACE_T, FIELD_TAU = 0, 1, 2, 3


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class Bands(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("C", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tally", ctypes.c_int), ("draws", ctypes.c_int),
                ("newton", ctypes.c_int), ("schedule", ctypes.c_int),
                ("particles_per_cell", ctypes.c_longlong), ("particles_per_wall_face", ctypes.c_longlong),
                ("seed", ctypes.c_ulonglong), ("epoch0", ctypes.c_uint), ("instance_base", ctypes.c_uint),
                ("cg_rtol", ctypes.c_double), ("cg_maxit", ctypes.c_int), ("step_budget", ctypes.c_longlong),
                ("block_threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("refill_lanes", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("warp_grab", ctypes.c_int), ("walk_k", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("refill_lanes", ctypes.c_int), ("warp_grab", ctypes.c_int), ("walk_k", ctypes.c_int),
                ("tally", ctypes.c_int), ("sweep_ms", ctypes.c_double), ("baseline_ms", ctypes.c_double)]


class Layout(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int), ("dim", ctypes.c_int), ("nb", ctypes.c_int),
                ("total_cells", ctypes.c_longlong), ("total_faces", ctypes.c_longlong),
                ("total_walls", ctypes.c_longlong), ("total_particles", ctypes.c_longlong),
                ("total_wall_faces", ctypes.c_longlong)]


# Every exported symbol of include/iugkp.h with its ctypes signature.
_vp, _i, _u, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_longlong
SIGNATURES = {
    "iugkp_default_options": (None, [ctypes.POINTER(Options)]),
    "iugkp_create": (_i, [ctypes.POINTER(Grid), _vp, ctypes.POINTER(Bands), _vp, _vp, ctypes.POINTER(Options),
                          ctypes.POINTER(_vp)]),
    "iugkp_create_batch": (_i, [_i, ctypes.POINTER(Grid), _vp, ctypes.POINTER(Bands), _vp, _vp,
                                ctypes.POINTER(Options), ctypes.POINTER(_vp)]),
    "iugkp_destroy": (None, [_vp]),
    "iugkp_last_error": (ctypes.c_char_p, [_vp]),
    "iugkp_get_layout": (_i, [_vp, ctypes.POINTER(Layout), _vp, _vp]),
    "iugkp_set_field": (_i, [_vp, _i, _vp, _i, _vp]),
    "iugkp_sweep": (_i, [_vp, _vp, _u, _vp, _vp, _vp, _vp, _vp, _vp]),
    "iugkp_macro": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "iugkp_newton_step": (_i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_i)]),
    "iugkp_residual": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "iugkp_autotune": (_i, [_vp, _vp, _u, _i, ctypes.POINTER(Tuning), _vp]),
    "iugkp_average": (_i, [_vp, _vp, _i, _u, _vp, _vp, _vp, _vp]),
    "iugkp_persistent_reset": (_i, [_vp, _vp]),
    "iugkp_persistent_step": (_i, [_vp, _vp, _u, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong), _vp]),
    "iugkp_solve_steady": (_i, [_vp, _vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d), _vp]),
    "iugkp_adjoint": (_i, [_vp, _vp, _vp, _d, _i, _vp, _vp, _vp, _vp]),
    "iugkp_replayed": (_i, [_vp, ctypes.POINTER(_ll), _vp]),
    "iugkp_check_fp32_walk": (_i, [ctypes.POINTER(_d)]),
    "iugkp_measure_atomics": (_i, [ctypes.POINTER(_d)]),
    "iugkp_diffusion_solve_noalloc": (_i, [ctypes.POINTER(Grid), _vp, _d, _vp, _vp, _d, _i, ctypes.POINTER(_i), _vp]),
}

_lib = None


class IugkpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Loads libiugkp.so (built by paper_2506_09465_gb300.build). Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2506_09465_gb300.build` "
                               "(the solver has no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, ctx=None):
    if status != 0:
        msg = load().iugkp_last_error(ctx)
        raise IugkpError(status, msg.decode() if msg else "")


def default_options(**kw) -> Options:
    o = Options()
    load().iugkp_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o
