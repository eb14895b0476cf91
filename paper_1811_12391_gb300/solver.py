"""Thin object wrapper over the C-ABI: builds the argument structs from a
problem description and moves buffers with PyTorch (device memory and the
current CUDA stream).  Every step of the computation runs in libdoctors.

A problem description is any object with the attributes nx, ny, nz, dx, dy,
dz, origin[3], mat [V] uint8, density [V] float32, sigma_t [nmat][G],
sigma_s [nmat][L+1][G][G], sn, legendre, sources (each with kind, pos,
axis, fan_deg, z_half_iso, iso_dist, weight, spectrum) and optionally tol and
max_iters.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _lib as C


def _require_torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libdoctors needs a CUDA device")
    return torch


def _dptr(arr: np.ndarray, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def make_sources(sources, G: int):
    """doctors_source array plus the spectrum buffers it points into."""
    arr = (C.doctors_source * len(sources))()
    keep = []
    for q, s in enumerate(sources):
        spec = np.ascontiguousarray(np.asarray(s.spectrum, dtype=np.float64)[:G])
        keep.append(spec)
        d = arr[q]
        d.kind = int(s.kind)
        d.pos[:] = [float(x) for x in s.pos]
        d.axis[:] = [float(x) for x in s.axis]
        d.fan_deg = float(getattr(s, "fan_deg", 360.0))
        d.z_half_iso = float(getattr(s, "z_half_iso", 0.0))
        d.iso_dist = float(getattr(s, "iso_dist", 1.0))
        d.weight = float(s.weight)
        d.spectrum = _dptr(spec, ctypes.c_double)
    return arr, keep


class DoctorsProblem:
    """One problem on the current CUDA device, ordered on `stream`
    (default: torch's current stream)."""

    def __init__(self, prob, stream=None, tol: Optional[float] = None, max_iters: Optional[int] = None,
                 tile=(0, 0), angles_per_block: int = 0, sweep_kernel: int = 0, device_loop: int = 0):
        torch = _require_torch_cuda()
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.G = int(prob.sigma_t.shape[1])
        self.nmat = int(prob.sigma_t.shape[0])
        self.V = int(prob.nx * prob.ny * prob.nz)
        self.dims = (int(prob.nx), int(prob.ny), int(prob.nz))
        mesh = C.doctors_mesh(int(prob.nx), int(prob.ny), int(prob.nz), float(prob.dx), float(prob.dy),
                              float(prob.dz), (ctypes.c_double * 3)(*[float(x) for x in prob.origin]))
        opt = C.doctors_options()
        opt.groups = self.G
        opt.sn_order = int(prob.sn)
        opt.legendre = int(prob.legendre)
        opt.tol = float(tol if tol is not None else getattr(prob, "tol", 1e-6))
        opt.max_iters = int(max_iters if max_iters is not None else getattr(prob, "max_iters", 500))
        opt.tile_x, opt.tile_y = int(tile[0]), int(tile[1])
        opt.angles_per_block = int(angles_per_block)
        opt.sweep_kernel = int(sweep_kernel)
        opt.device_loop = int(device_loop)
        opt.differencing = int(getattr(prob, "differencing", 0))
        h = ctypes.c_void_p()
        C.check(C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt),
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.set_materials(prob.mat, prob.density, prob.sigma_t, prob.sigma_s)
        self.set_sources(prob.sources)
        self.result = None

    # ------------------------------------------------------------------
    def set_materials(self, mat, density, sigma_t, sigma_s):
        torch = self.torch
        st = np.ascontiguousarray(sigma_t, np.float64)
        ss = np.ascontiguousarray(sigma_s, np.float64)
        if isinstance(mat, torch.Tensor) and mat.is_cuda:
            m = mat.contiguous()
            d = density.contiguous() if density is not None else None
            C.check(C.doctors_set_materials(self.h, st.shape[0], ctypes.c_void_p(m.data_ptr()),
                                            ctypes.c_void_p(d.data_ptr()) if d is not None else None,
                                            _dptr(st, ctypes.c_double), _dptr(ss, ctypes.c_double),
                                            C.DOCTORS_MEM_DEVICE))
        else:
            m = np.ascontiguousarray(mat, np.uint8)
            d = np.ascontiguousarray(density, np.float32) if density is not None else None
            C.check(C.doctors_set_materials(self.h, st.shape[0], m.ctypes.data_as(ctypes.c_void_p),
                                            d.ctypes.data_as(ctypes.c_void_p) if d is not None else None,
                                            _dptr(st, ctypes.c_double), _dptr(ss, ctypes.c_double),
                                            C.DOCTORS_MEM_HOST))

    def set_sources(self, sources: Sequence):
        arr, keep = make_sources(sources, self.G)
        C.check(C.doctors_set_source(self.h, len(sources), arr))
        self.n_src = len(sources)
        del keep

    # ------------------------------------------------------------------
    def solve(self, allow_not_converged: bool = False) -> dict:
        r = C.doctors_result()
        allow = (C.DOCTORS_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        C.check(C.doctors_solve(self.h, ctypes.byref(r)), allow)
        self.result = r.as_dict()
        return self.result

    def fluence(self, which: int = C.DOCTORS_FLUENCE_TOTAL, out=None):
        """[G][V] float32 torch tensor on the device."""
        torch = self.torch
        if out is None:
            out = torch.empty((self.G, self.V), dtype=torch.float32, device="cuda")
        C.check(C.doctors_get_fluence(self.h, which, ctypes.c_void_p(out.data_ptr()), C.DOCTORS_MEM_DEVICE))
        return out

    def fluence_host(self, which: int = C.DOCTORS_FLUENCE_TOTAL, out: Optional[np.ndarray] = None) -> np.ndarray:
        """[G][V] float32 on the host (into `out` if given, e.g. a pinned buffer)."""
        if out is None:
            out = np.zeros((self.G, self.V), np.float32)
        elif out.dtype != np.float32 or out.size != self.G * self.V or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float32 array of G*V values")
        C.check(C.doctors_get_fluence(self.h, which, out.ctypes.data_as(ctypes.c_void_p), C.DOCTORS_MEM_HOST))
        return out

    def dose(self, k, out=None):
        """[V] float64 torch tensor on the device."""
        torch = self.torch
        kk = np.ascontiguousarray(k, np.float64)
        if out is None:
            out = torch.empty(self.V, dtype=torch.float64, device="cuda")
        C.check(C.doctors_dose(self.h, _dptr(kk, ctypes.c_double), ctypes.c_void_p(out.data_ptr()),
                               C.DOCTORS_MEM_DEVICE))
        return out

    def dose_host(self, k, out: Optional[np.ndarray] = None) -> np.ndarray:
        """[V] float64 on the host (into `out` if given)."""
        kk = np.ascontiguousarray(k, np.float64)
        if out is None:
            out = np.zeros(self.V, np.float64)
        elif out.dtype != np.float64 or out.size != self.V or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of V values")
        C.check(C.doctors_dose(self.h, _dptr(kk, ctypes.c_double), out.ctypes.data_as(ctypes.c_void_p),
                               C.DOCTORS_MEM_HOST))
        return out

    def adjoint(self, response, want=("weights", "spectrum", "density")) -> dict:
        """Gradients of J = sum response * phi (response: [G][V] float64 torch
        tensor on the device).  Returns device tensors."""
        torch = self.torch
        r = response.contiguous().to(torch.float64)
        outs = {
            "weights": torch.zeros(self.n_src, dtype=torch.float64, device="cuda") if "weights" in want else None,
            "spectrum": torch.zeros(self.G, dtype=torch.float64, device="cuda") if "spectrum" in want else None,
            "density": torch.zeros(self.V, dtype=torch.float64, device="cuda") if "density" in want else None,
        }
        res = C.doctors_result()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        C.check(C.doctors_adjoint_solve(self.h, ctypes.c_void_p(r.data_ptr()), C.DOCTORS_MEM_DEVICE,
                                        ptr(outs["weights"]), ptr(outs["spectrum"]), ptr(outs["density"]),
                                        ctypes.byref(res)))
        outs["result"] = res.as_dict()
        return outs

    def roi_dose(self, k, roi, want_dose: bool = False):
        """J = sum_v roi(v) D(v) (float) and, if want_dose, the dose [V]
        (float64 device tensor).  roi: [V] float64 device tensor."""
        torch = self.torch
        kk = np.ascontiguousarray(k, np.float64)
        r = roi.contiguous().to(torch.float64)
        J = ctypes.c_double()
        dose = torch.empty(self.V, dtype=torch.float64, device="cuda") if want_dose else None
        C.check(C.doctors_roi_dose(self.h, _dptr(kk, ctypes.c_double), ctypes.c_void_p(r.data_ptr()),
                                   C.DOCTORS_MEM_DEVICE, ctypes.byref(J),
                                   ctypes.c_void_p(dose.data_ptr()) if dose is not None else None))
        return (J.value, dose) if want_dose else J.value

    def roi_gradients(self, k, roi, want=("weights", "spectrum", "density")) -> dict:
        """J and its gradients with respect to the source weights, the shared
        spectrum and the densities (the density gradient includes the dose's
        own density factor).  roi: [V] float64 device tensor.  Returns device
        tensors and J (float)."""
        torch = self.torch
        kk = np.ascontiguousarray(k, np.float64)
        r = roi.contiguous().to(torch.float64)
        outs = {
            "weights": torch.zeros(self.n_src, dtype=torch.float64, device="cuda") if "weights" in want else None,
            "spectrum": torch.zeros(self.G, dtype=torch.float64, device="cuda") if "spectrum" in want else None,
            "density": torch.zeros(self.V, dtype=torch.float64, device="cuda") if "density" in want else None,
        }
        J = ctypes.c_double()
        res = C.doctors_result()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        C.check(C.doctors_roi_gradients(self.h, _dptr(kk, ctypes.c_double), ctypes.c_void_p(r.data_ptr()),
                                        C.DOCTORS_MEM_DEVICE, ctypes.byref(J), ptr(outs["weights"]),
                                        ptr(outs["spectrum"]), ptr(outs["density"]), ctypes.byref(res)))
        outs["J"] = J.value
        outs["result"] = res.as_dict()
        return outs

    def autotune(self) -> dict:
        t = C.doctors_tuning()
        C.check(C.doctors_autotune(self.h, ctypes.byref(t)))
        return t.as_dict()

    def ray_indices(self, src: int, voxel: int, cap: int = 4096):
        idx = (ctypes.c_int32 * cap)()
        ln = (ctypes.c_float * cap)()
        n = ctypes.c_int()
        C.check(C.doctors_debug_ray_indices(self.h, src, voxel, idx, ln, cap, ctypes.byref(n)))
        return (np.frombuffer(idx, np.int32)[:n.value].copy(), np.frombuffer(ln, np.float32)[:n.value].copy())

    def close(self):
        if getattr(self, "h", None):
            C.doctors_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def solve_batch(problems: Sequence["DoctorsProblem"]) -> list:
    """Solve several problems in one graph-captured device-side loop."""
    n = len(problems)
    arr = (ctypes.c_void_p * n)(*[p.h.value for p in problems])
    res = (C.doctors_result * n)()
    C.check(C.doctors_solve_batch(arr, n, res))
    out = [r.as_dict() for r in res]
    for p, r in zip(problems, out):
        p.result = r
    return out


def quadrature(sn_order: int, legendre: int):
    """(dirs [A,3], w [A], R [A,(L+1)^2]) as built by the library (host only)."""
    n = ctypes.c_int()
    C.check(C.doctors_quadrature(sn_order, legendre, None, None, None, ctypes.byref(n)))
    A = n.value
    M = (legendre + 1) ** 2
    dirs = np.zeros((A, 3))
    w = np.zeros(A)
    R = np.zeros((A, M))
    C.check(C.doctors_quadrature(sn_order, legendre, _dptr(dirs, ctypes.c_double), _dptr(w, ctypes.c_double),
                                 _dptr(R, ctypes.c_double), ctypes.byref(n)))
    return dirs, w, R


def ct_to_materials(hu, thresholds, bin_material, hu_knots, rho_knots, stream=None):
    """CT numbers -> (material ids uint8, densities float32) by the library's
    kernel (doctors_ct_to_materials).  `hu` is a float32 numpy array (host;
    numpy arrays are returned) or a float32 CUDA tensor (device; CUDA tensors
    are returned, stream-ordered on `stream` or the current torch stream)."""
    t = np.ascontiguousarray(thresholds, np.float32).ravel()
    bm = np.ascontiguousarray(bin_material, np.uint8).ravel()
    hk = np.ascontiguousarray(hu_knots, np.float32).ravel()
    rk = np.ascontiguousarray(rho_knots, np.float32).ravel()
    tp = _dptr(t, ctypes.c_float) if t.size else None
    if isinstance(hu, np.ndarray):
        h = np.ascontiguousarray(hu, np.float32).ravel()
        mat = np.zeros(h.size, np.uint8)
        rho = np.zeros(h.size, np.float32)
        C.check(C.doctors_ct_to_materials(h.ctypes.data_as(ctypes.c_void_p), h.size, t.size, tp,
                                          _dptr(bm, ctypes.c_uint8), hk.size, _dptr(hk, ctypes.c_float),
                                          _dptr(rk, ctypes.c_float), mat.ctypes.data_as(ctypes.c_void_p),
                                          rho.ctypes.data_as(ctypes.c_void_p), C.DOCTORS_MEM_HOST, None))
        return mat, rho
    torch = _require_torch_cuda()
    if hu.dtype != torch.float32 or not hu.is_cuda:
        raise ValueError("hu must be a float32 numpy array or a float32 CUDA tensor")
    h = hu.contiguous().view(-1)
    mat = torch.empty(h.numel(), dtype=torch.uint8, device=h.device)
    rho = torch.empty(h.numel(), dtype=torch.float32, device=h.device)
    s = stream if stream is not None else torch.cuda.current_stream(h.device)
    with torch.cuda.device(h.device):
        C.check(C.doctors_ct_to_materials(ctypes.c_void_p(h.data_ptr()), h.numel(), t.size, tp,
                                          _dptr(bm, ctypes.c_uint8), hk.size, _dptr(hk, ctypes.c_float),
                                          _dptr(rk, ctypes.c_float), ctypes.c_void_p(mat.data_ptr()),
                                          ctypes.c_void_p(rho.data_ptr()), C.DOCTORS_MEM_DEVICE,
                                          ctypes.c_void_p(s.cuda_stream)))
    return mat, rho
