"""Adjoint and gradients on the GPU: the adjoint scalar fluence and the
gradients of an ROI dose against the FP64 oracle's adjoint, and the
autograd wrapper against central differences of GPU forward solves."""
import copy

import numpy as np
import pytest

from oracle import solver as osv
from synth import phantoms as ph
from tests.parity import DENSITY_GRAD_TOL, REL_TOL, TF32X3_DENSITY_FLOOR, max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1811_12391_gb300.build import build
    build()
    import torch
    from paper_1811_12391_gb300 import _lib as C
    from paper_1811_12391_gb300.solver import DoctorsProblem
    return torch, C, DoctorsProblem


def _problem(views=2, seed=3):
    p = ph.water_cylinder(seed=seed, nx=20, ny=18, nz=6, G=3, sn=4, L=1, dx=1.0, dy=1.0, dz=1.5,
                          diameter=16.0, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources = ph.axial_scan_sources(p, views, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources[-1].weight = 0.7
    rng = np.random.default_rng(seed)
    p.density[:] = (p.density * rng.uniform(0.9, 1.1, size=p.V)).astype(np.float32)
    return p


def _roi(p):
    roi = np.zeros(p.V)
    roi.reshape(p.nz, p.ny, p.nx)[2:4, 7:11, 8:12] = 1.0 / 32.0
    return roi


@pytest.fixture(scope="module")
def grad_ref():
    p = _problem()
    roi = _roi(p)
    return p, roi, osv.gradients(p, roi, tol=1e-12)


@pytest.mark.parametrize("L,kernel", [(1, 1), (1, 3), (1, 4), (1, 5), (1, 7), (3, 1), (3, 3), (3, 4),
                                      (3, 5), (3, 7), (3, 8)])
def test_adjoint_fluence_and_gradients_match_oracle(env, grad_ref, L, kernel):
    torch, C, DoctorsProblem = env
    if L == 1:
        p, roi, ref = grad_ref
    else:
        p = _problem()
        p = ph.water_cylinder(seed=3, nx=20, ny=18, nz=6, G=3, sn=4, L=3, dx=1.0, dy=1.0, dz=1.5,
                              diameter=16.0, sid=20.0, fan_deg=60.0, z_width=8.0)
        p.sources = ph.axial_scan_sources(p, 2, sid=20.0, fan_deg=60.0, z_width=8.0)
        p.sources[-1].weight = 0.7
        p.density[:] = _problem().density
        roi = _roi(p)
        ref = osv.gradients(p, roi, tol=1e-12)
    d = DoctorsProblem(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, angles_per_block=3)
    d.solve()
    r = osv.response_from_roi(p, roi)
    g = d.adjoint(torch.as_tensor(r, device="cuda"))
    assert g["result"]["converged"] == 1
    z00 = d.fluence_host(C.DOCTORS_FLUENCE_ADJOINT)
    assert max_rel(z00, ref["adjoint"].Z[:, 0, :]) <= REL_TOL
    gw = g["weights"].cpu().numpy()
    gs = g["spectrum"].cpu().numpy()
    np.testing.assert_allclose(gw, ref["d_weights"], rtol=REL_TOL)
    np.testing.assert_allclose(gs, ref["d_spectrum"], rtol=REL_TOL)
    # the library's density gradient is through the transport; the oracle's
    # also holds the explicit density factor of the dose
    explicit = (roi[None, :] * p.k_dep[p.mat].T * ref["forward"].phi).sum(axis=0)
    gd = g["density"].cpu().numpy() + explicit
    rd = ref["d_density"]
    # kernel 8 runs the split sweep's P3 transforms on the tensor cores as
    # 3xTF32 (about 2^-21 relative error per transform against 2^-24 in FP32):
    # its bar for 1e-4 starts at 1e-3 of the largest gradient
    floor = TF32X3_DENSITY_FLOOR if kernel == 8 else 1e-4
    assert max_rel(gd, rd, floor=floor) <= REL_TOL
    assert max_rel(gd, rd, floor=1e-6) <= DENSITY_GRAD_TOL
    d.close()


def test_adjoint_volume_source(env):
    torch, C, DoctorsProblem = env
    p = ph.infinite_medium_cube(n=8, G=2, sn=4, L=1, sigma_t=0.8)
    roi = np.zeros(p.V)
    roi[p.V // 2 + 3] = 1.0
    ref = osv.gradients(p, roi, tol=1e-12, density=False)
    d = DoctorsProblem(p, tol=1e-6, max_iters=400)
    d.solve()
    r = osv.response_from_roi(p, roi)
    g = d.adjoint(torch.as_tensor(r, device="cuda"), want=("weights", "spectrum"))
    np.testing.assert_allclose(g["weights"].cpu().numpy(), ref["d_weights"], rtol=REL_TOL)
    np.testing.assert_allclose(g["spectrum"].cpu().numpy(), ref["d_spectrum"], rtol=REL_TOL)
    d.close()


def test_autograd_roi_dose_matches_finite_differences(env):
    torch, C, _ = env
    from paper_1811_12391_gb300.autograd import DoseProblem, RoiDose
    p = _problem()
    roi = _roi(p)
    dp = DoseProblem(p, roi, tol=1e-6, max_iters=400)
    w = torch.tensor([s.weight for s in p.sources], dtype=torch.float64, requires_grad=True)
    chi = torch.tensor(p.sources[0].spectrum, dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(p.density, dtype=torch.float32, device="cuda", requires_grad=True)
    J = RoiDose.apply(w, chi, rho, dp)
    J.backward()
    ref = osv.roi_dose(p, roi, tol=1e-12)
    assert abs(J.item() - ref) <= REL_TOL * abs(ref)

    def J_of(wv, cv, rv):
        with torch.no_grad():
            return RoiDose.apply(wv, cv, rv, dp).item()

    h = 1e-3
    for s in range(len(p.sources)):
        e = torch.zeros_like(w)
        e[s] = h * w[s].item()
        fd = (J_of(w + e, chi, rho) - J_of(w - e, chi, rho)) / (2 * e[s].item())
        assert abs(fd - w.grad[s].item()) <= 1e-3 * abs(fd)
    for g in range(p.G):
        e = torch.zeros_like(chi)
        e[g] = h * chi[g].item()
        fd = (J_of(w, chi + e, rho) - J_of(w, chi - e, rho)) / (2 * e[g].item())
        assert abs(fd - chi.grad[g].item()) <= 1e-3 * abs(fd)
    # densities: larger steps, FP32 forward solves
    gr = rho.grad.double().cpu().numpy()
    scale = np.abs(gr).max()
    rng = np.random.default_rng(2)
    picks = list(rng.choice(p.V, size=12, replace=False)) + list(np.flatnonzero(roi)[:4])
    Jv = abs(J.item())
    for v in picks:
        e = torch.zeros_like(rho)
        e[v] = 2e-2 * rho[v].item()
        fd = (J_of(w, chi, rho + e) - J_of(w, chi, rho - e)) / (2 * e[v].item())
        # FD noise of FP32 solves converged to 1e-6 relative: ~1e-6 |J| / step
        noise = 4e-6 * Jv / (2 * e[v].item())
        assert abs(fd - gr[v]) <= 2e-2 * abs(fd) + noise, (v, fd, gr[v], noise)


@pytest.mark.parametrize("kernel", [1, 3, 4, 5, 7])
def test_gradients_satisfy_euler_identity(env, kernel):
    """J is linear in every view weight and in every spectrum entry, so
    sum_s w_s dJ/dw_s = J and sum_g chi_g dJ/dchi_g = J (Euler's identity for
    homogeneous functions of degree one): the adjoint gradients against the
    forward dose of the same GPU solve, with no oracle involved."""
    torch, C, DoctorsProblem = env
    p = ph.water_cylinder(seed=3, nx=20, ny=18, nz=6, G=3, sn=4, L=3, dx=1.0, dy=1.0, dz=1.5,
                          diameter=16.0, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources = ph.axial_scan_sources(p, 3, sid=20.0, fan_deg=60.0, z_width=8.0)
    p.sources[1].weight = 0.6
    p.sources[2].weight = 1.3
    roi = _roi(p)
    d = DoctorsProblem(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, angles_per_block=3)
    d.solve()
    J = float((roi * d.dose_host(p.k_dep)).sum())
    g = d.adjoint(torch.as_tensor(osv.response_from_roi(p, roi), device="cuda"), want=("weights", "spectrum"))
    w = np.array([s.weight for s in p.sources])
    chi = np.asarray(p.sources[0].spectrum, dtype=np.float64)
    assert abs(float(w @ g["weights"].cpu().numpy()) - J) <= 2 * REL_TOL * abs(J)
    assert abs(float(chi @ g["spectrum"].cpu().numpy()) - J) <= 2 * REL_TOL * abs(J)
    d.close()


@pytest.mark.parametrize("sn,kernel,ab", [(16, 0, 0), (16, 1, 12), (16, 3, 12), (16, 4, 12), (16, 7, 12),
                                           (16, 4, 36), (12, 0, 0), (12, 3, 7)])
def test_adjoint_gradients_s16_direction_blocks(env, sn, kernel, ab):
    """S16: the tile-stage and chained kernels (blocks of 12 directions) store
    and pair the angular fluence in 16-byte runs of a voxel's directions, the
    dataflow kernels in one record per (voxel, octant, block) of 12
    directions (one launch per block) or of the whole octant's 36 (the
    default); S12 whole octants (21 directions, records padded to 24) and the
    chained kernel's blocks of 7; adjoint fluence and all gradients against
    the oracle."""
    torch, C, DoctorsProblem = env
    p = ph.abdomen(nx=16, ny=14, nz=4, d=2.0, dz=2.0, G=2, sn=sn, L=1)
    rng = np.random.default_rng(7)
    p.density[:] = (p.density * rng.uniform(0.9, 1.1, size=p.V)).astype(np.float32)
    roi = np.zeros(p.V)
    roi.reshape(p.nz, p.ny, p.nx)[1:3, 5:9, 5:9] = 1.0 / 32.0
    ref = osv.gradients(p, roi, tol=1e-12)
    d = DoctorsProblem(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, angles_per_block=ab)
    d.solve()
    r = osv.response_from_roi(p, roi)
    g = d.adjoint(torch.as_tensor(r, device="cuda"))
    assert g["result"]["converged"] == 1
    assert max_rel(d.fluence_host(C.DOCTORS_FLUENCE_ADJOINT), ref["adjoint"].Z[:, 0, :]) <= REL_TOL
    np.testing.assert_allclose(g["weights"].cpu().numpy(), ref["d_weights"], rtol=REL_TOL)
    np.testing.assert_allclose(g["spectrum"].cpu().numpy(), ref["d_spectrum"], rtol=REL_TOL)
    explicit = (roi[None, :] * p.k_dep[p.mat].T * ref["forward"].phi).sum(axis=0)
    gd = g["density"].cpu().numpy() + explicit
    rd = ref["d_density"]
    assert max_rel(gd, rd, floor=1e-4) <= REL_TOL
    assert max_rel(gd, rd, floor=1e-6) <= DENSITY_GRAD_TOL
    d.close()
