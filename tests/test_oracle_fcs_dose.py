"""Pins of the oracle's first-collision source direction and of its dose tally.

First-collision source (Sec. II.A, the kernel of Eq. 2): the uncollided
photons at a voxel all travel along the unit vector from the source to the
voxel centre, so their scattering source in direction Omega_n is the
angle-to-angle form
    q_n(v) = sum_l (2l+1)/(4 pi) rho sigma_s,l P_l(Omega_n . Omega_sv) phi_u(v).
The test writes Omega_sv and P_l out itself (scipy's Legendre polynomials), so
a reversed direction (voxel to source) flips every odd-l term and fails.  A
physical check pins the same sign through the whole solve: with forward-peaked
P1 scattering, more collided photons leave a thin slab downstream than
upstream, and backward-peaked scattering reverses that.

Dose (Sec. II.A, III.A): particle conservation fixes the absorbed total.  With
k = sigma_a (unit energy per absorbed photon), every photon that collides out
of the uncollided beam is either absorbed or leaks as a collided photon, so
    vol * sum_v D(v) = vol * sum_{g,v} rho sigma_t phi_u[g](v) - sum_g leak_g.
Plus a two-voxel, two-material case whose dose is worked out by hand.
"""
import math

import numpy as np
from scipy.special import eval_legendre

from oracle import quadrature as quad
from oracle import solver as osv
from synth import phantoms as ph


def _p3_problem():
    """A small heterogeneous P3 problem with a point source off every axis,
    so that a sign or component error in any coordinate of the direction
    shows."""
    p = ph.water_cylinder(nx=7, ny=6, nz=5, G=3, sn=8, L=3, dx=2.0, dy=2.0, dz=2.0,
                          diameter=11.0)
    rng = np.random.default_rng(41)
    p.density[:] = rng.uniform(0.6, 1.6, p.V).astype(np.float32)
    src = ph.Source(kind=ph.SRC_POINT, pos=np.array([-13.0, 17.0, -21.0]),
                    axis=np.array([0.0, 0.0, 1.0]), spectrum=np.array([0.5, 0.3, 0.2]))
    return p.with_sources([src])


def test_first_collision_source_equals_angle_to_angle_form():
    p = _p3_problem()
    src = p.sources[0]
    dirs, w, R, Mop, Dop = quad.angular_operators(p.sn, p.legendre)
    phi_u = osv.uncollided(p, src)
    U = osv.uncollided_moments(p, src, phi_u)
    X, Y, Z = p.centres()
    rho = p.density.astype(np.float64)
    rng = np.random.default_rng(3)
    voxels = rng.choice(p.V, size=12, replace=False)
    for g_from, g_to in ((0, 0), (0, 2), (1, 2)):
        q_moment = Mop @ osv.scatter(p, U[g_from], g_from, g_to)          # [A, V]
        for v in voxels:
            d = np.array([X[v], Y[v], Z[v]]) - src.pos                    # source -> voxel
            omega_sv = d / math.sqrt(float(d @ d))
            cos_nv = dirs @ omega_sv                                       # [A]
            m = p.mat[v]
            q = np.zeros(dirs.shape[0])
            for l in range(p.legendre + 1):
                q += ((2 * l + 1) / (4.0 * math.pi) * rho[v] * p.sigma_s[m, l, g_from, g_to]
                      * eval_legendre(l, cos_nv) * phi_u[g_from, v])
            scale = np.abs(q).max()
            assert scale > 0.0
            assert np.abs(q_moment[:, v] - q).max() <= 1e-12 * scale


def _slab(aniso):
    """One group, P1: a 1.5 cm scattering slab in the middle of a column of
    void cells, a point source 20 cm upstream on the -z side.  aniso is
    sigma_s,1 / sigma_s,0 (the phase function is proportional to
    1 + 3 aniso cos(theta))."""
    nx, ny, nz = 5, 5, 12
    V = nx * ny * nz
    mat = np.zeros(V, np.uint8)
    mat.reshape(nz, ny, nx)[4:7] = 1
    sigt = np.array([[0.0], [1.0]])
    sigs = np.zeros((2, 2, 1, 1))
    sigs[1, 0, 0, 0] = 0.9
    sigs[1, 1, 0, 0] = 0.9 * aniso
    origin = np.array([-5.0, -5.0, -3.0])
    src = ph.Source(kind=ph.SRC_POINT, pos=np.array([0.0, 0.0, -23.0]),
                    axis=np.array([0.0, 0.0, 1.0]), spectrum=np.array([1.0]))
    return ph.Problem(name="slab", seed=0, nx=nx, ny=ny, nz=nz, dx=2.0, dy=2.0, dz=0.5,
                      origin=origin, mat=mat, density=np.ones(V, np.float32), sigma_t=sigt,
                      sigma_s=sigs, sn=8, legendre=1, sources=[src],
                      k_dep=np.zeros((2, 1)), e_mid=np.array([50.0]))


def _downstream_over_upstream(aniso):
    p = _slab(aniso)
    sol = osv.solve(p, tol=1e-12)
    phi_c = sol.phi_c[0, 0].reshape(p.nz, p.ny, p.nx)
    upstream = phi_c[0:4].sum()      # void cells between the source and the slab
    downstream = phi_c[7:].sum()     # void cells behind the slab
    return downstream / upstream


def test_forward_peaked_scattering_lights_the_far_side():
    fwd = _downstream_over_upstream(0.3)
    iso = _downstream_over_upstream(0.0)
    bwd = _downstream_over_upstream(-0.3)
    assert fwd > 1.0 > bwd
    assert fwd > iso > bwd


def test_absorbed_photons_balance_collisions_of_the_uncollided_beam():
    p = ph.water_cylinder(nx=10, ny=10, nz=6, G=4, sn=4, L=1, dx=1.6, dy=1.6, dz=1.5,
                          diameter=14.0)
    rng = np.random.default_rng(17)
    p.density[:] = (p.density * rng.uniform(0.7, 1.4, p.V)).astype(np.float32)
    sol = osv.solve(p, tol=1e-13)
    sigma_a = p.sigma_t - p.sigma_s[:, 0].sum(axis=2)                     # [nmat, G]
    vol = p.dx * p.dy * p.dz
    absorbed = vol * osv.dose(p, sol.phi, sigma_a).sum()
    rho = p.density.astype(np.float64)
    collided_out_of_beam = vol * (rho[None, :] * p.sigma_t[p.mat].T * sol.phi_u).sum()
    expect = collided_out_of_beam - sol.leak.sum()
    assert abs(absorbed - expect) <= 1e-10 * expect
    # the pin separates the tally from its plausible mistakes
    assert abs(vol * osv.dose(p, sol.phi_c[:, 0], sigma_a).sum() - expect) > 1e-3 * expect
    no_rho = vol * (sigma_a[p.mat].T * sol.phi).sum()
    assert abs(no_rho - expect) > 1e-3 * expect


def test_two_voxel_dose_by_hand():
    """mat = (0, 1), rho = (2, 0.5), phi[g][v] = ((1, 2), (3, 4)),
    k[m][g] = ((1, 10), (100, 1000)):
    D(0) = 2 * (1*1 + 10*3) = 62,  D(1) = 0.5 * (100*2 + 1000*4) = 2100."""
    p = ph.Problem(name="two", seed=0, nx=2, ny=1, nz=1, dx=1.0, dy=1.0, dz=1.0,
                   origin=np.zeros(3), mat=np.array([0, 1], np.uint8),
                   density=np.array([2.0, 0.5], np.float32), sigma_t=np.ones((2, 2)),
                   sigma_s=np.zeros((2, 1, 2, 2)), sn=2, legendre=0, sources=[],
                   k_dep=np.array([[1.0, 10.0], [100.0, 1000.0]]), e_mid=np.array([60.0, 30.0]))
    phi = np.array([[1.0, 2.0], [3.0, 4.0]])
    assert np.array_equal(osv.dose(p, phi), np.array([62.0, 2100.0]))
