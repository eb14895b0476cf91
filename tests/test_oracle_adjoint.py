"""Pins of the oracle's adjoint and gradients: forward-adjoint reciprocity and
central finite differences (the paper has no adjoint; these check that the
oracle's discrete adjoint is the transpose of its forward operator)."""
import copy
import math

import numpy as np
import pytest

from oracle import quadrature as quad
from oracle import solver as osv
from synth import phantoms as ph


def _small(seed=3, views=2):
    p = ph.water_cylinder(seed=seed, nx=6, ny=6, nz=4, G=3, sn=4, L=1, dx=2.0, dy=2.0, dz=2.0,
                          diameter=10.0, sid=20.0, fan_deg=60.0, z_width=6.0)
    p.sources = ph.axial_scan_sources(p, views, sid=20.0, fan_deg=60.0, z_width=6.0)
    p.sources[1].weight = 0.7 if views > 1 else 1.0
    rng = np.random.default_rng(seed)
    p.density[:] = (p.density * rng.uniform(0.9, 1.1, size=p.V)).astype(np.float32)
    return p


def _roi(p):
    roi = np.zeros(p.V)
    roi.reshape(p.nz, p.ny, p.nx)[1:3, 2:4, 2:4] = 1.0 / 8.0
    return roi


@pytest.mark.parametrize("differencing", [0, 1])
def test_reciprocity_collided_response(differencing):
    """<r, phi_c,00> = sum_{g,lm,v} (2l+1)/(4 pi) (S^T Z)[g][lm][v] U[g][lm][v],
    for step and diamond differencing."""
    p = _small()
    p.differencing = differencing
    roi = _roi(p)
    sol = osv.solve(p, tol=1e-13)
    r = osv.response_from_roi(p, roi)
    adj = osv.adjoint_solve(p, r, tol=1e-13)
    ls = quad.moment_degrees(p.legendre)
    C = (2 * ls + 1) / (4 * math.pi)
    lhs = float((r * sol.phi_c[:, 0, :]).sum())
    rhs = float((C[None, :, None] * adj.T * sol.U).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_reciprocity_volume_source():
    """With a uniform volumetric source q and response r:
    <r, phi_00> = <q_00 / (4 pi), Z_00>."""
    p = ph.infinite_medium_cube(n=5, G=2, sn=4, L=1, sigma_t=0.8)
    p.density[:] = np.linspace(0.8, 1.2, p.V).astype(np.float32)
    rng = np.random.default_rng(1)
    r = rng.uniform(0, 1, size=(p.G, p.V))
    sol = osv.solve(p, tol=1e-13)
    adj = osv.adjoint_solve(p, r, tol=1e-13)
    E = osv.external_moments(p)
    lhs = float((r * sol.phi_c[:, 0, :]).sum())
    rhs = float((E[:, 0, :] / (4 * math.pi) * adj.Z[:, 0, :]).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def _J(p, roi):
    return osv.roi_dose(p, roi, tol=1e-13)


@pytest.mark.parametrize("differencing", [0, 1])
def test_gradients_match_central_differences(differencing):
    """View-weight, spectrum and density gradients by the adjoint against
    central differences of the forward solve (step and diamond differencing:
    the density enters both schemes' cell balance only through sigma_t psi)."""
    p = _small()
    p.differencing = differencing
    roi = _roi(p)
    gr = osv.gradients(p, roi, tol=1e-13)
    assert abs(gr["J"] - _J(p, roi)) < 1e-12 * abs(gr["J"])
    rel = 1e-3
    # per-view weights (J is linear in them)
    for s in range(len(p.sources)):
        q1, q2 = copy.deepcopy(p), copy.deepcopy(p)
        h = rel * p.sources[s].weight
        q1.sources[s].weight += h
        q2.sources[s].weight -= h
        fd = (_J(q1, roi) - _J(q2, roi)) / (2 * h)
        assert abs(fd - gr["d_weights"][s]) <= 1e-8 * abs(fd)
    # spectrum weights (shared by all views)
    for g in range(p.G):
        q1, q2 = copy.deepcopy(p), copy.deepcopy(p)
        h = rel * p.sources[0].spectrum[g]
        for q, sg in ((q1, 1), (q2, -1)):
            for s in q.sources:
                s.spectrum = s.spectrum.copy()
                s.spectrum[g] += sg * h
        fd = (_J(q1, roi) - _J(q2, roi)) / (2 * h)
        assert abs(fd - gr["d_spectrum"][g]) <= 1e-8 * abs(fd)
    # voxel densities (20 seeded entries, some inside the ROI)
    rng = np.random.default_rng(5)
    picks = list(rng.choice(p.V, size=16, replace=False)) + list(np.flatnonzero(roi)[:4])
    scale = np.abs(gr["d_density"]).max()
    for v in picks:
        q1, q2 = copy.deepcopy(p), copy.deepcopy(p)
        q1.density[v] = np.float32(p.density[v] * (1 + rel))
        q2.density[v] = np.float32(p.density[v] * (1 - rel))
        fd = (_J(q1, roi) - _J(q2, roi)) / (float(q1.density[v]) - float(q2.density[v]))
        assert abs(fd - gr["d_density"][v]) <= 1e-5 * max(abs(fd), 1e-3 * scale), (v, fd, gr["d_density"][v])


def test_volume_source_gradients_match_central_differences():
    p = ph.infinite_medium_cube(n=5, G=2, sn=4, L=1, sigma_t=0.8)
    p.sources.append(ph.Source(kind=ph.SRC_POINT, pos=np.array([0.3, -0.2, -9.0]), axis=np.array([0, 0, 1.0]),
                               weight=2.0, spectrum=p.sources[0].spectrum.copy()))
    roi = np.zeros(p.V)
    roi[p.V // 2] = 1.0
    gr = osv.gradients(p, roi, tol=1e-13, density=False)
    for s in range(2):
        q1, q2 = copy.deepcopy(p), copy.deepcopy(p)
        h = 1e-3 * p.sources[s].weight
        q1.sources[s].weight += h
        q2.sources[s].weight -= h
        fd = (_J(q1, roi) - _J(q2, roi)) / (2 * h)
        assert abs(fd - gr["d_weights"][s]) <= 1e-8 * abs(fd)
    for g in range(p.G):
        q1, q2 = copy.deepcopy(p), copy.deepcopy(p)
        h = 1e-3 * p.sources[0].spectrum[g]
        for q, sg in ((q1, 1), (q2, -1)):
            for s in q.sources:
                s.spectrum = s.spectrum.copy()
                s.spectrum[g] += sg * h
        fd = (_J(q1, roi) - _J(q2, roi)) / (2 * h)
        assert abs(fd - gr["d_spectrum"][g]) <= 1e-8 * abs(fd)
