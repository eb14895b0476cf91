"""ctypes binding of the oracle's plain-C loops (transport.c).

Test infrastructure only (see the package docstring).  ``build()`` compiles
transport.c with gcc into oracle/_build/liboracle.so; ``lib()`` loads it,
building on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "transport.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile transport.c (no FMA contraction, IEEE operations as written),
    with OpenMP when the compiler offers it (the sweep's direction blocks and
    the ray trace's planes then run on all host cores; results do not depend
    on the thread count)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
        try:
            subprocess.check_call(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def threads() -> int:
    """Host threads of the oracle's OpenMP loops (1 without OpenMP)."""
    return int(lib().oracle_threads())


def set_threads(n: int) -> int:
    """Sets the oracle's host threads; returns the number in effect."""
    return int(lib().oracle_set_threads(int(n)))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_siddon_f32.argtypes = [_f, _int, _int, _int, _int, _int, _int, _f, _f, _i32, _f, _int]
            L.oracle_siddon_f32.restype = _int
            L.oracle_siddon_f64.argtypes = [_d, _int, _int, _int, _int, _int, _int, _d, _d, _i32, _d, _int]
            L.oracle_siddon_f64.restype = _int
            L.oracle_optical_depth.argtypes = [_int, _int, _int, _d, _d, _u8, _d, _int, _d, _d, _d, _d]
            L.oracle_optical_depth.restype = _int
            L.oracle_collimator_mask.argtypes = [_int, _int, _int, _f, _f, _f, _f, _f, _f,
                                                 ctypes.c_float, ctypes.c_float, _u8]
            L.oracle_collimator_mask.restype = None
            L.oracle_sweep.argtypes = [_int, _int, _int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _int, _d, _d, _int, _d, _d, _d, _d, _d,
                                       _d, _d, _int]
            L.oracle_sweep.restype = _int
            L.oracle_threads.argtypes = []
            L.oracle_threads.restype = _int
            L.oracle_set_threads.argtypes = [_int]
            L.oracle_set_threads.restype = _int
            L.oracle_backproject.argtypes = [_int, _int, _int, _d, _d, _u8, _int, _d, _d, _d]
            L.oracle_backproject.restype = _int
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ct)


def siddon_f32(S, voxel, dims, origin, spacing, cap=None):
    """FP32 index list and lengths of the ray from S to the centre of voxel."""
    nx, ny, nz = dims
    cap = cap or 4 * (nx + ny + nz) + 8
    S = np.ascontiguousarray(S, np.float32)
    o = np.ascontiguousarray(origin, np.float32)
    d = np.ascontiguousarray(spacing, np.float32)
    idx = np.zeros(cap, np.int32)
    ln = np.zeros(cap, np.float32)
    n = lib().oracle_siddon_f32(_p(S, _f), int(voxel[0]), int(voxel[1]), int(voxel[2]), nx, ny, nz,
                                _p(o, _f), _p(d, _f), _p(idx, _i32), _p(ln, _f), cap)
    if n < 0:
        raise RuntimeError("ray longer than the list capacity")
    return idx[:n].copy(), ln[:n].copy()


def siddon_f64(S, voxel, dims, origin, spacing, cap=None):
    nx, ny, nz = dims
    cap = cap or 4 * (nx + ny + nz) + 8
    S = np.ascontiguousarray(S, np.float64)
    o = np.ascontiguousarray(origin, np.float64)
    d = np.ascontiguousarray(spacing, np.float64)
    idx = np.zeros(cap, np.int32)
    ln = np.zeros(cap, np.float64)
    n = lib().oracle_siddon_f64(_p(S, _d), int(voxel[0]), int(voxel[1]), int(voxel[2]), nx, ny, nz,
                                _p(o, _d), _p(d, _d), _p(idx, _i32), _p(ln, _d), cap)
    if n < 0:
        raise RuntimeError("ray longer than the list capacity")
    return idx[:n].copy(), ln[:n].copy()


def optical_depth(dims, origin, spacing, mat, rho, sigt, S):
    nx, ny, nz = dims
    V = nx * ny * nz
    G = sigt.shape[1]
    tau = np.zeros((G, V))
    r2 = np.zeros(V)
    o = np.ascontiguousarray(origin, np.float64)
    d = np.ascontiguousarray(spacing, np.float64)
    mat = np.ascontiguousarray(mat, np.uint8)
    rho = np.ascontiguousarray(rho, np.float64)
    sigt = np.ascontiguousarray(sigt, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    rc = lib().oracle_optical_depth(nx, ny, nz, _p(o, _d), _p(d, _d), _p(mat, _u8), _p(rho, _d), G,
                                    _p(sigt, _d), _p(S, _d), _p(tau, _d), _p(r2, _d))
    if rc != 0:
        raise RuntimeError("ray overflow")
    return tau, r2


def collimator_mask(dims, origin, spacing, S, axis, perp, up, tan_half, z_slope):
    nx, ny, nz = dims
    W = np.zeros(nx * ny * nz, np.uint8)
    f32 = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
    o, d, S, axis, perp, up = map(f32, (origin, spacing, S, axis, perp, up))
    lib().oracle_collimator_mask(nx, ny, nz, _p(o, _f), _p(d, _f), _p(S, _f), _p(axis, _f),
                                 _p(perp, _f), _p(up, _f), ctypes.c_float(tan_half),
                                 ctypes.c_float(z_slope), _p(W, _u8))
    return W


def sweep(dims, spacing, dirs, w, Mop, Dop, sigt, src, store_psi=False, diamond=False):
    """One sweep of one group; returns (phi [M][V], leakage, psi [A][V] or None).
    diamond selects diamond differencing instead of step differencing."""
    nx, ny, nz = dims
    V = nx * ny * nz
    A = dirs.shape[0]
    M = Mop.shape[1]
    dirs = np.ascontiguousarray(dirs, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    Mop = np.ascontiguousarray(Mop, np.float64)
    Dop = np.ascontiguousarray(Dop, np.float64)
    sigt = np.ascontiguousarray(sigt, np.float64)
    src = np.ascontiguousarray(src, np.float64).reshape(M, V)
    phi = np.zeros((M, V))
    leak = np.zeros(1)
    psi = np.zeros((A, V)) if store_psi else None
    rc = lib().oracle_sweep(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]), A,
                            _p(dirs, _d), _p(w, _d), M, _p(Mop, _d), _p(Dop, _d), _p(sigt, _d),
                            _p(src, _d), _p(phi, _d), _p(leak, _d),
                            _p(psi, _d) if psi is not None else None, int(bool(diamond)))
    if rc != 0:
        raise MemoryError("oracle sweep: scratch allocation failed")
    return phi, float(leak[0]), psi


def backproject(dims, origin, spacing, mat, H, S, grad):
    nx, ny, nz = dims
    o = np.ascontiguousarray(origin, np.float64)
    d = np.ascontiguousarray(spacing, np.float64)
    mat = np.ascontiguousarray(mat, np.uint8)
    H = np.ascontiguousarray(H, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    assert grad.dtype == np.float64 and grad.flags.c_contiguous
    rc = lib().oracle_backproject(nx, ny, nz, _p(o, _d), _p(d, _d), _p(mat, _u8), H.shape[0],
                                  _p(H, _d), _p(S, _d), _p(grad, _d))
    if rc != 0:
        raise RuntimeError("ray overflow")
    return grad
