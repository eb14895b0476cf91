"""Pins of the oracle's collided solve (Eq. 2 with vacuum boundaries, step
differencing, Legendre scattering, source iteration) against closed forms,
conservation, symmetry and a brute-force dense solve."""
import math

import numpy as np
import pytest

from oracle import quadrature as quad
from oracle import solver as osv
from synth import phantoms as ph


def test_infinite_medium_lower_triangular_closed_form():
    """Centre of a thick cube with a uniform source: the multigroup
    infinite-medium fluence phi_g = (Q_g + sum_{g'<g} s0(g'->g) phi_g') /
    (sigma_t - s0(g->g)); the boundary deficit of the step scheme decays by
    about 0.04 per cell and is below 1e-11 eight cells in."""
    p = ph.infinite_medium_cube(n=16, G=3, sn=4, L=0)
    sol = osv.solve(p, tol=1e-13)
    Q = p.sources[0].weight * p.sources[0].spectrum
    s0 = p.sigma_s[0, 0]
    st = p.sigma_t[0]
    phi = np.zeros(p.G)
    for g in range(p.G):
        phi[g] = (Q[g] + sum(s0[gp, g] * phi[gp] for gp in range(g))) / (st[g] - s0[g, g])
    c = 8
    v = (c * p.ny + c) * p.nx + c
    np.testing.assert_allclose(sol.phi_c[:, 0, v], phi, rtol=1e-10)


def test_one_group_infinite_medium_is_S_over_sigma_a():
    p = ph.infinite_medium_cube(n=16, G=1, sn=4, L=0, seed=11)
    sol = osv.solve(p, tol=1e-13)
    v = (8 * 16 + 8) * 16 + 8
    expect = p.sources[0].weight * p.sources[0].spectrum[0] / (p.sigma_t[0, 0] - p.sigma_s[0, 0, 0, 0])
    assert abs(sol.phi_c[0, 0, v] / expect - 1) < 1e-10


def test_sweep_balance_per_group():
    """Step differencing conserves particles exactly on every sweep:
    volume * sum(s_00) = volume * sum(sigma_t phi_00) + boundary leakage."""
    p = ph.water_cylinder(nx=12, ny=12, nz=6, G=3, sn=4, L=1, dx=1.5, dy=1.5, dz=1.5, diameter=16)
    sol = osv.solve(p, tol=1e-11)
    assert np.all(sol.balance < 1e-12)
    assert np.all(sol.leak > 0)


def test_global_balance_at_convergence():
    """Summed over groups: first-collision source = absorption + leakage +
    loss below the lowest group (downscatter out of the last group)."""
    p = ph.tiny_cube(n=8, sn=4, L=1)
    sol = osv.solve(p, tol=1e-13)
    vol = p.dx * p.dy * p.dz
    rho = p.density.astype(float)
    G = p.G
    fcs = 0.0
    absorb = 0.0
    for g in range(G):
        for gp in range(G):
            fcs += vol * (rho * p.sigma_s[p.mat, 0, g, gp] * sol.U[g, 0]).sum()
        sig_out = p.sigma_s[p.mat, 0, g, :].sum(axis=1)
        sig_remove = p.sigma_t[p.mat, g] - sig_out       # absorption
        absorb += vol * (rho * sig_remove * sol.phi_c[g, 0]).sum()
        if g == G - 1:
            pass
    # the lowest group keeps only its within-group scatter; the rest of its
    # out-scatter left the group structure and is counted as absorption above
    # (sigma_t - sum_g' sigma_s(g->g') includes it)
    total = absorb + sol.leak.sum()
    assert abs(total - fcs) / fcs < 1e-10


def test_cylinder_mirror_symmetry():
    """Source on the -y axis at the axial centre of a z-aligned cylinder:
    the fluence is mirror symmetric in x and in z."""
    p = ph.water_cylinder(nx=16, ny=16, nz=8, G=3, sn=4, L=1, dx=1.2, dy=1.2, dz=1.0, diameter=18)
    sol = osv.solve(p, tol=1e-13)
    for arr in (sol.phi_u, sol.phi_c[:, 0, :], sol.phi):
        a = arr.reshape(p.G, p.nz, p.ny, p.nx)
        scale = np.abs(a).max()
        assert np.abs(a - a[:, :, :, ::-1]).max() <= 1e-12 * scale
        assert np.abs(a - a[:, ::-1, :, :]).max() <= 1e-12 * scale


def _dense_solution(p):
    """Assemble the full linear system of the step-differenced multigroup
    problem (unknowns psi[g][n][v]) and solve it with dense LU."""
    dirs, w, R, Mop, Dop = quad.angular_operators(p.sn, p.legendre)
    A_, M = dirs.shape[0], Mop.shape[1]
    G, V = p.G, p.V
    nx, ny, nz = p.nx, p.ny, p.nz
    ls = quad.moment_degrees(p.legendre)
    rho = p.density.astype(float)
    N = G * A_ * V
    Amat = np.zeros((N, N))
    b = np.zeros(N)
    # uncollided moments and external source
    U = np.zeros((G, M, V))
    for s in p.sources:
        if s.kind != osv.SRC_VOLUME:
            U += osv.uncollided_moments(p, s, osv.uncollided(p, s))
    E = osv.external_moments(p)
    idx = lambda g, n, v: (g * A_ + n) * V + v  # noqa: E731
    for g in range(G):
        for n in range(A_):
            c = np.abs(dirs[n]) / np.array([p.dx, p.dy, p.dz])
            sgn = np.sign(dirs[n]).astype(int)
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        v = (k * ny + j) * nx + i
                        r = idx(g, n, v)
                        Amat[r, r] += rho[v] * p.sigma_t[p.mat[v], g] + c.sum()
                        for q, (ii, jj, kk) in enumerate(((i - sgn[0], j, k), (i, j - sgn[1], k),
                                                          (i, j, k - sgn[2]))):
                            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                                Amat[r, idx(g, n, (kk * ny + jj) * nx + ii)] -= c[q]
                        # scattering from group gp, direction n2
                        for gp in range(g + 1):
                            sig = rho[v] * p.sigma_s[p.mat[v], :, gp, g][ls]   # [M]
                            coef = (Mop[n] * sig) @ Dop.T                      # [A]
                            for n2 in range(A_):
                                Amat[r, idx(gp, n2, v)] -= coef[n2]
                            b[r] += (Mop[n] * sig) @ U[gp, :, v]
                        b[r] += Mop[n] @ E[g, :, v]
    psi = np.linalg.solve(Amat, b).reshape(G, A_, V)
    return np.einsum("nm,gnv->gmv", Dop, psi)


@pytest.mark.parametrize("sn,L", [(2, 0), (4, 1)])
def test_source_iteration_equals_dense_lu(sn, L):
    p = ph.water_cylinder(nx=3, ny=3, nz=2, G=2, sn=sn, L=L, dx=4.0, dy=4.0, dz=3.0, diameter=10)
    p.density[:] = np.array([1.0, 1.1, 0.9, 1.3, 1.0, 0.7, 1.2, 0.8, 1.05] * 2, np.float32)
    p.mat[:] = 1
    p.sources.append(ph.Source(kind=ph.SRC_VOLUME, pos=np.zeros(3), axis=np.array([0, 0, 1.0]),
                               weight=1e-3, spectrum=np.array([0.3, 0.7])))
    sol = osv.solve(p, tol=1e-14)
    ref = _dense_solution(p)
    np.testing.assert_allclose(sol.phi_c, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


# ---------------------------------------------------------------------------
# diamond differencing (the sweep variant with differencing = 1)
# ---------------------------------------------------------------------------

def _slab(axis, n, h, sigma, S0, sn=4, diamond=True):
    """A row of n cells of width h along `axis`, the other two extents huge
    (their streaming coefficients |Omega| / d vanish), uniform sigma and
    isotropic source S0 (moment l = 0): per direction the sweep along the row
    is the one-dimensional scheme.  Returns (dirs, Mop, psi [A][n])."""
    dirs, w, R, Mop, Dop = quad.angular_operators(sn, 0)
    dims = [1, 1, 1]
    dims[axis] = n
    sp = [1e12, 1e12, 1e12]
    sp[axis] = h
    V = n
    _, _, psi = osv.tr.sweep(tuple(dims), tuple(sp), dirs, w, Mop, Dop, np.full(V, sigma),
                             np.full((1, V), S0), store_psi=True, diamond=diamond)
    return dirs, Mop, psi


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_diamond_slab_closed_form(axis):
    """One-dimensional diamond difference from vacuum inflow: the edge fluxes
    obey psi_{i+1/2} = a psi_{i-1/2} + b q with a = (c - sigma/2)/(c + sigma/2),
    b = 1/(c + sigma/2), c = |mu|/h, whose solution is the geometric sum
    psi_{i+1/2} = (q/sigma)(1 - a^i); cell i is the mean of its two edges,
    (q/sigma)(1 - (a^(i-1) + a^i)/2).  (For c < sigma/2, a < 0: the scheme's
    oscillation, no fixup.)"""
    n, h, sigma, S0 = 9, 0.7, 1.3, 2.0
    dirs, Mop, psi = _slab(axis, n, h, sigma, S0)
    for k in range(dirs.shape[0]):
        mu = dirs[k, axis]
        c = abs(mu) / h
        q = Mop[k, 0] * S0
        a = (c - sigma / 2) / (c + sigma / 2)
        i = np.arange(1, n + 1)                       # cells in sweep order
        expect = (q / sigma) * (1 - (a ** (i - 1) + a ** i) / 2)
        got = psi[k] if mu > 0 else psi[k][::-1]
        np.testing.assert_allclose(got, expect, rtol=1e-9, atol=1e-14)


def test_diamond_slab_second_order_step_first_order():
    """Against the exact slab solution psi(x) = (q/sigma)(1 - exp(-sigma x/|mu|))
    averaged over the last cell of a slab of fixed thickness, halving the cells
    divides the diamond-difference error by about 4 and the step error by
    about 2."""
    T, sigma, S0, axis = 3.0, 1.0, 1.0, 0
    errs = {True: [], False: []}
    for n in (16, 32, 64):
        h = T / n
        for dd in (True, False):
            dirs, Mop, psi = _slab(axis, n, h, sigma, S0, diamond=dd)
            e = 0.0
            for k in range(dirs.shape[0]):
                mu = abs(dirs[k, axis])
                q = Mop[k, 0] * S0
                x0, x1 = T - h, T
                exact = (q / sigma) * (1 - (mu / (sigma * h)) * (np.exp(-sigma * x0 / mu) - np.exp(-sigma * x1 / mu)))
                last = psi[k][-1] if dirs[k, axis] > 0 else psi[k][0]
                e = max(e, abs(last - exact) / exact)
            errs[dd].append(e)
    r_dd = [errs[True][i] / errs[True][i + 1] for i in range(2)]
    r_st = [errs[False][i] / errs[False][i + 1] for i in range(2)]
    assert all(3.5 < r < 4.5 for r in r_dd), r_dd
    assert all(1.7 < r < 2.3 for r in r_st), r_st


def test_diamond_sweep_balance_per_group():
    """Diamond differencing keeps each cell's balance exact: summed over the
    mesh, volume * sum(s_00) = volume * sum(sigma_t phi_00) + the current
    leaving through boundary faces, counted with the outgoing face fluxes
    (2 psi - psi_in), not the cell fluxes."""
    p = ph.water_cylinder(nx=12, ny=10, nz=6, G=3, sn=4, L=1, dx=1.5, dy=1.3, dz=1.1, diameter=16)
    p.differencing = 1
    sol = osv.solve(p, tol=1e-11)
    assert np.all(sol.balance < 1e-12)
    assert np.all(sol.leak > 0)


def test_diamond_reversed_sweep_is_transpose():
    """On a uniform mesh with varying sigma_t, the diamond-differenced sweep of
    -Omega is the transpose of the sweep of Omega (cell fluxes from cell
    sources): <r, T q> = <T' r, q> for every direction, which is what lets
    the adjoint solve reuse the sweep."""
    rng = np.random.default_rng(5)
    dims, sp = (4, 3, 5), (0.8, 0.6, 1.1)
    V = int(np.prod(dims))
    sig = rng.uniform(0.05, 3.0, V)
    dirs, w, R, Mop, Dop = quad.angular_operators(4, 0)
    one = np.ones((1, 1))
    for n in range(dirs.shape[0]):
        d = dirs[n:n + 1]
        q = rng.standard_normal(V)
        r = rng.standard_normal(V)
        Tq, _, _ = osv.tr.sweep(dims, sp, d, np.ones(1), one, one, sig, q[None, :], diamond=True)
        Tr, _, _ = osv.tr.sweep(dims, sp, -d, np.ones(1), one, one, sig, r[None, :], diamond=True)
        lhs, rhs = float(r @ Tq[0]), float(Tr[0] @ q)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))

