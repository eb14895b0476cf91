"""ctypes binding of libdoctors (include/doctors.h): argument marshalling only.

Every function named like the C entry point forwards to it.  The library is
built in-tree (``paper_1811_12391_gb300/_build/libdoctors.so``); importing a
function when it is missing raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdoctors.so")

DOCTORS_OK = 0
DOCTORS_ERR_INVALID_ARG = 1
DOCTORS_ERR_OOM = 2
DOCTORS_ERR_CUDA = 3
DOCTORS_ERR_NOT_CONVERGED = 4
DOCTORS_ERR_TIMEOUT = 5
DOCTORS_ERR_STATE = 6

DOCTORS_MEM_HOST = 0
DOCTORS_MEM_DEVICE = 1

DOCTORS_SRC_POINT = 0
DOCTORS_SRC_FAN_CONE = 1
DOCTORS_SRC_VOLUME = 2

DOCTORS_FLUENCE_UNCOLLIDED = 0
DOCTORS_FLUENCE_COLLIDED = 1
DOCTORS_FLUENCE_TOTAL = 2
DOCTORS_FLUENCE_ADJOINT = 3
DOCTORS_DIFF_STEP = 0
DOCTORS_DIFF_DIAMOND = 1

ERROR_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "TIMEOUT",
               6: "STATE"}


class doctors_mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("origin", ctypes.c_double * 3)]


class doctors_options(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int), ("sn_order", ctypes.c_int), ("legendre", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int), ("tile_x", ctypes.c_int),
                ("tile_y", ctypes.c_int), ("angles_per_block", ctypes.c_int),
                ("sweep_kernel", ctypes.c_int), ("device_loop", ctypes.c_int),
                ("differencing", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class doctors_source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("pos", ctypes.c_double * 3), ("axis", ctypes.c_double * 3),
                ("fan_deg", ctypes.c_double), ("z_half_iso", ctypes.c_double),
                ("iso_dist", ctypes.c_double), ("weight", ctypes.c_double),
                ("spectrum", ctypes.POINTER(ctypes.c_double))]


class doctors_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("residual", ctypes.c_double), ("balance_rel", ctypes.c_double),
                ("tol_used", ctypes.c_double), ("cell_updates", ctypes.c_double),
                ("ms_raytrace", ctypes.c_double), ("ms_iterate", ctypes.c_double),
                ("ms_sweep", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class doctors_tuning(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("angles_per_block", ctypes.c_int),
                ("sweep_kernel", ctypes.c_int), ("ms_per_sweep", ctypes.c_double), ("candidates", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = ctypes.c_void_p
_int = ctypes.c_int
_P = ctypes.POINTER

# (name, restype, argtypes) of every entry point declared in include/doctors.h
SIGNATURES = [
    ("doctors_create_problem", _int, [_P(doctors_mesh), _P(doctors_options), _vp, _P(_vp)]),
    ("doctors_set_materials", _int, [_vp, _int, _vp, _vp, _P(ctypes.c_double), _P(ctypes.c_double), _int]),
    ("doctors_set_source", _int, [_vp, _int, _P(doctors_source)]),
    ("doctors_solve", _int, [_vp, _P(doctors_result)]),
    ("doctors_get_fluence", _int, [_vp, _int, _vp, _int]),
    ("doctors_dose", _int, [_vp, _P(ctypes.c_double), _vp, _int]),
    ("doctors_dose_noalloc", _int, [_vp, _P(ctypes.c_double), _vp]),
    ("doctors_adjoint_solve", _int, [_vp, _vp, _int, _vp, _vp, _vp, _P(doctors_result)]),
    ("doctors_roi_dose", _int, [_vp, _P(ctypes.c_double), _vp, _int, _P(ctypes.c_double), _vp]),
    ("doctors_roi_gradients", _int, [_vp, _P(ctypes.c_double), _vp, _int, _P(ctypes.c_double), _vp, _vp, _vp,
                                     _P(doctors_result)]),
    ("doctors_debug_withhold_faces", _int, [_vp, _int]),
    ("doctors_debug_ray_indices", _int, [_vp, _int, _int, _P(ctypes.c_int32), _P(ctypes.c_float), _int,
                                         _P(_int)]),
    ("doctors_quadrature", _int, [_int, _int, _P(ctypes.c_double), _P(ctypes.c_double),
                                  _P(ctypes.c_double), _P(_int)]),
    ("doctors_solve_batch", _int, [_P(_vp), _int, _P(doctors_result)]),
    ("doctors_ct_to_materials", _int, [_vp, ctypes.c_size_t, _int, _P(ctypes.c_float), _P(ctypes.c_uint8), _int,
                                       _P(ctypes.c_float), _P(ctypes.c_float), _vp, _vp, _int, _vp]),
    ("doctors_autotune", _int, [_vp, _P(doctors_tuning)]),
    ("doctors_destroy", None, [_vp]),
    ("doctors_last_error", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


class DoctorsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libdoctors.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdoctors.so is not built ({LIB_PATH}); run "
                                   "paper_1811_12391_gb300.build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().doctors_last_error().decode()


def check(rc, allow=()):
    if rc != DOCTORS_OK and rc not in allow:
        raise DoctorsError(rc, last_error())
    return rc


def _fwd(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    return f


doctors_create_problem = _fwd("doctors_create_problem")
doctors_set_materials = _fwd("doctors_set_materials")
doctors_set_source = _fwd("doctors_set_source")
doctors_solve = _fwd("doctors_solve")
doctors_get_fluence = _fwd("doctors_get_fluence")
doctors_dose = _fwd("doctors_dose")
doctors_dose_noalloc = _fwd("doctors_dose_noalloc")
doctors_adjoint_solve = _fwd("doctors_adjoint_solve")
doctors_roi_dose = _fwd("doctors_roi_dose")
doctors_roi_gradients = _fwd("doctors_roi_gradients")
doctors_debug_ray_indices = _fwd("doctors_debug_ray_indices")
doctors_debug_withhold_faces = _fwd("doctors_debug_withhold_faces")
doctors_quadrature = _fwd("doctors_quadrature")
doctors_solve_batch = _fwd("doctors_solve_batch")
doctors_ct_to_materials = _fwd("doctors_ct_to_materials")
doctors_autotune = _fwd("doctors_autotune")
doctors_destroy = _fwd("doctors_destroy")
doctors_last_error = _fwd("doctors_last_error")
