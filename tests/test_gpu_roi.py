"""Region-of-interest dose and its gradients through the C-ABI
(doctors_roi_dose, doctors_roi_gradients): J and all three gradients against
the FP64 oracle, host and device memory, argument checks, and the
forward-adjoint reciprocity of the GPU's own solves."""
import ctypes
import math

import numpy as np
import pytest

from oracle import solver as osv
from synth import phantoms as ph
from tests.parity import DENSITY_GRAD_TOL, REL_TOL, max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1811_12391_gb300.build import build
    build()
    import torch
    from paper_1811_12391_gb300 import _lib as C
    from paper_1811_12391_gb300.solver import DoctorsProblem
    return torch, C, DoctorsProblem


def _problem(L=1, seed=3):
    p = ph.water_cylinder(seed=seed, nx=20, ny=18, nz=6, G=3, sn=4, L=L, dx=1.0, dy=1.0, dz=1.5,
                          diameter=16.0, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources = ph.axial_scan_sources(p, 2, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources[-1].weight = 0.7
    rng = np.random.default_rng(seed)
    p.density[:] = (p.density * rng.uniform(0.9, 1.1, size=p.V)).astype(np.float32)
    return p


def _roi(p):
    roi = np.zeros(p.V)
    roi.reshape(p.nz, p.ny, p.nx)[2:4, 7:11, 8:12] = 1.0 / 32.0
    return roi


@pytest.fixture(scope="module")
def ref_p1():
    p = _problem(L=1)
    roi = _roi(p)
    return p, roi, osv.gradients(p, roi, tol=1e-12)


@pytest.fixture(scope="module")
def ref_p3():
    p = _problem(L=3)
    roi = _roi(p)
    return p, roi, osv.gradients(p, roi, tol=1e-12)


@pytest.mark.parametrize("L,kernel", [(1, 0), (1, 1), (3, 0), (3, 3), (3, 4)])
def test_roi_gradients_match_oracle(env, ref_p1, ref_p3, L, kernel):
    torch, C, DoctorsProblem = env
    p, roi, ref = ref_p1 if L == 1 else ref_p3
    d = DoctorsProblem(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, angles_per_block=3)
    d.solve()
    g = d.roi_gradients(p.k_dep, torch.as_tensor(roi, device="cuda"))
    assert g["result"]["converged"] == 1
    assert abs(g["J"] - ref["J"]) <= REL_TOL * abs(ref["J"])
    assert max_rel(g["weights"].cpu().numpy(), ref["d_weights"]) <= REL_TOL
    assert max_rel(g["spectrum"].cpu().numpy(), ref["d_spectrum"]) <= REL_TOL
    # the full density gradient, the dose's own density factor included
    gd = g["density"].cpu().numpy()
    assert max_rel(gd, ref["d_density"], floor=1e-4) <= REL_TOL
    assert max_rel(gd, ref["d_density"], floor=1e-6) <= DENSITY_GRAD_TOL
    d.close()


def test_roi_dose_host_and_device_memory_agree(env, ref_p1):
    torch, C, DoctorsProblem = env
    p, roi, ref = ref_p1
    d = DoctorsProblem(p, tol=1e-6, max_iters=400)
    d.solve()
    J_dev, dose_dev = d.roi_dose(p.k_dep, torch.as_tensor(roi, device="cuda"), want_dose=True)
    k = np.ascontiguousarray(p.k_dep, np.float64)
    r = np.ascontiguousarray(roi)
    J = ctypes.c_double()
    dose = np.full(p.V, np.nan)
    C.check(C.doctors_roi_dose(d.h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               r.ctypes.data_as(ctypes.c_void_p), C.DOCTORS_MEM_HOST, ctypes.byref(J),
                               dose.ctypes.data_as(ctypes.c_void_p)))
    assert J.value == J_dev                       # fixed summation order: same bits
    assert np.array_equal(dose, dose_dev.cpu().numpy())
    assert np.array_equal(dose, d.dose_host(p.k_dep))
    assert abs(J.value - ref["J"]) <= REL_TOL * abs(ref["J"])
    # host-memory gradients equal the device-memory ones
    gw = np.full(len(p.sources), np.nan)
    gs = np.full(p.G, np.nan)
    gd = np.full(p.V, np.nan)
    Jg = ctypes.c_double()
    C.check(C.doctors_roi_gradients(d.h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    r.ctypes.data_as(ctypes.c_void_p), C.DOCTORS_MEM_HOST, ctypes.byref(Jg),
                                    gw.ctypes.data_as(ctypes.c_void_p), gs.ctypes.data_as(ctypes.c_void_p),
                                    gd.ctypes.data_as(ctypes.c_void_p), None))
    g = d.roi_gradients(p.k_dep, torch.as_tensor(roi, device="cuda"))
    # J is summed in a fixed order from the same forward solution: same bits.
    # Each call solves the adjoint again, and the sweep's FP32 moment sums are
    # atomic (their order varies from run to run), so the gradients of two
    # calls agree to about 1e-9, far inside the parity bar
    assert Jg.value == J_dev
    assert max_rel(gw, g["weights"].cpu().numpy(), floor=0.0) <= 1e-6
    assert max_rel(gs, g["spectrum"].cpu().numpy(), floor=0.0) <= 1e-6
    assert np.abs(gd - g["density"].cpu().numpy()).max() <= 1e-6 * np.abs(gd).max()
    d.close()


def test_roi_argument_errors_leave_outputs_untouched(env):
    torch, C, DoctorsProblem = env
    p = ph.tiny_cube(n=4)
    d = DoctorsProblem(p, tol=1e-6, max_iters=200)
    k = np.ascontiguousarray(p.k_dep, np.float64)
    kp = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    roi = torch.full((p.V,), 1.0 / p.V, dtype=torch.float64, device="cuda")
    rp = ctypes.c_void_p(roi.data_ptr())
    dose = torch.full((p.V,), float("nan"), dtype=torch.float64, device="cuda")
    dp = ctypes.c_void_p(dose.data_ptr())
    J = ctypes.c_double(float("nan"))
    # before a solve
    assert C.doctors_roi_dose(d.h, kp, rp, C.DOCTORS_MEM_DEVICE, ctypes.byref(J), dp) == C.DOCTORS_ERR_STATE
    assert C.doctors_roi_gradients(d.h, kp, rp, C.DOCTORS_MEM_DEVICE, ctypes.byref(J), None, None, dp,
                                   None) == C.DOCTORS_ERR_STATE
    d.solve()
    bad = k.copy()
    bad[0, 1] = np.inf
    cases = [
        (None, rp, C.DOCTORS_MEM_DEVICE, ctypes.byref(J)),
        (kp, None, C.DOCTORS_MEM_DEVICE, ctypes.byref(J)),
        (kp, rp, C.DOCTORS_MEM_DEVICE, None),
        (kp, rp, 7, ctypes.byref(J)),
        (bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rp, C.DOCTORS_MEM_DEVICE, ctypes.byref(J)),
    ]
    for kk, rr, mem, jj in cases:
        assert C.doctors_roi_dose(d.h, kk, rr, mem, jj, dp) == C.DOCTORS_ERR_INVALID_ARG
        assert C.doctors_roi_gradients(d.h, kk, rr, mem, jj, None, None, dp, None) == C.DOCTORS_ERR_INVALID_ARG
    host_roi = np.full(p.V, 1.0 / p.V)
    host_roi[3] = np.nan
    host_dose = np.full(p.V, np.nan)
    assert C.doctors_roi_dose(d.h, kp, host_roi.ctypes.data_as(ctypes.c_void_p), C.DOCTORS_MEM_HOST,
                              ctypes.byref(J), host_dose.ctypes.data_as(ctypes.c_void_p)) == \
        C.DOCTORS_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert math.isnan(J.value)
    assert torch.isnan(dose).all().item()
    assert np.isnan(host_dose).all()
    d.close()


def test_reciprocity_volume_source(env):
    """A uniform isotropic volumetric source q and a response r: the forward
    and adjoint GPU solves satisfy <r, phi> = sum_g q_g / (4 pi) sum_v Z_00[g](v)
    (the adjoint source is 4 pi r in the l = 0 moment), to 1e-5."""
    torch, C, DoctorsProblem = env
    p = ph.infinite_medium_cube(n=10, G=3, sn=4, L=1, sigma_t=0.8)
    rng = np.random.default_rng(12)
    r = rng.uniform(0.0, 1.0, size=(p.G, p.V))
    d = DoctorsProblem(p, tol=1e-7, max_iters=600)
    d.solve()
    phi = d.fluence_host(C.DOCTORS_FLUENCE_TOTAL).astype(np.float64)
    g = d.adjoint(torch.as_tensor(r, device="cuda"), want=())
    assert g["result"]["converged"] == 1
    z00 = d.fluence_host(C.DOCTORS_FLUENCE_ADJOINT).astype(np.float64)
    q = p.sources[0].weight * np.asarray(p.sources[0].spectrum, np.float64)
    lhs = float((r * phi).sum())
    rhs = float((q[:, None] / (4.0 * math.pi) * z00).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    d.close()


@pytest.mark.parametrize("L", [1, 3])
def test_reciprocity_point_sources(env, L):
    """Point sources: the ROI dose of the forward solve equals the adjoint's
    sum_s w_s dJ/dw_s (J is linear in the view weights, and dJ/dw_s is the
    inner product of the source's uncollided fluence with the adjoint
    importance r + first-collision adjoint), to 1e-5."""
    torch, C, DoctorsProblem = env
    p = _problem(L=L)
    p.sources = ph.axial_scan_sources(p, 3, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources[1].weight = 0.6
    p.sources[2].weight = 1.3
    roi = _roi(p)
    d = DoctorsProblem(p, tol=1e-7, max_iters=600)
    d.solve()
    g = d.roi_gradients(p.k_dep, torch.as_tensor(roi, device="cuda"), want=("weights",))
    w = np.array([s.weight for s in p.sources])
    assert abs(float(w @ g["weights"].cpu().numpy()) - g["J"]) <= 1e-5 * abs(g["J"])
    d.close()
