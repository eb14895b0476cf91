"""FP64 oracle: uncollided fluence, first-collision source, source iteration,
dose, adjoint and gradients.

Test infrastructure only (see the package docstring).  Follows the paper's
steps in order:

1. Uncollided fluence by ray tracing (Sec. II.A): for a point source S and a
   voxel centre T, phi_u[g](T) = I * chi_g * W(T) * exp(-tau_g) / (4 pi r^2),
   tau_g = sum over the ray's voxels of rho * sigma_t[g] * length (Siddon walk
   in transport.c), r = |T - S|, W the collimator mask.
2. First-collision source (Sec. II.A): the uncollided angular fluence is a
   delta in the direction Omega_sT, so its moments are phi_u * R_lm(Omega_sT);
   scattering them gives the source of the collided problem.
3. Collided discrete-ordinates problem (Eq. 2, vacuum boundaries), with the
   scattering kernel as a Legendre expansion: the moment source
   s_lm[g](v) = rho(v) sum_{g' <= g} sigma_s,l(g' -> g) (phi_c + phi_u)_lm[g'](v)
   is mapped to directions with (2l+1)/(4 pi) R_lm(Omega_n) and swept with
   step differencing (or, when the problem asks for it, diamond differencing
   without a negative-flux fixup); moments are summed with w_n R_lm(Omega_n)
   (Eq. 3).
   Reading of the unstated iteration: groups are solved from high to low
   energy (Gauss-Seidel); within a group, unaccelerated source iteration until
   the relative L2 change of the scalar fluence is below tol.
4. Dose (Sec. II.A, III.A): D(v) = sum_g k[mat, g] * rho(v) * phi[g](v),
   phi = phi_u + phi_c (k: energy-deposition weights standing in for the
   ICRP116 fluence-to-dose factors).
5. Adjoint of steps 2-4 (transposed scattering, reversed directions) and the
   gradients of a dose functional J = sum_v R(v) D(v).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import quadrature as quad
from . import transport as tr

SRC_POINT, SRC_FAN_CONE, SRC_VOLUME = 0, 1, 2


def collimator_frame(axis):
    """(perp, up) unit vectors of a source whose beam axis is `axis`:
    perp = (-a_y, a_x, 0)/|(a_x, a_y)| (in the transverse plane; (1, 0, 0)
    when the axis is along z), up = axis x perp."""
    ax, ay, az = (float(a) for a in axis)
    h = math.sqrt(ax * ax + ay * ay)
    if h == 0.0:
        px, py, pz = 1.0, 0.0, 0.0
    else:
        px, py, pz = -ay / h, ax / h, 0.0
    up = (ay * pz - az * py, az * px - ax * pz, ax * py - ay * px)
    return np.array([px, py, pz]), np.array(up)


def source_mask(p, src) -> np.ndarray:
    """Collimator mask W[V] in {0, 1}."""
    if src.kind == SRC_POINT:
        return np.ones(p.V, np.uint8)
    perp, up = collimator_frame(src.axis)
    tan_half = math.tan(0.5 * src.fan_deg * (math.pi / 180.0))
    z_slope = src.z_half_iso / src.iso_dist
    return tr.collimator_mask((p.nx, p.ny, p.nz), p.origin, (p.dx, p.dy, p.dz), src.pos,
                              src.axis, perp, up, np.float32(tan_half), np.float32(z_slope))


def unit_uncollided(p, src) -> np.ndarray:
    """Uncollided fluence per unit emitted photon in each group,
    u[g][v] = W(v) exp(-tau_g(v)) / (4 pi r(v)^2)  (FP64)."""
    rho = p.density.astype(np.float64)
    tau, r2 = tr.optical_depth((p.nx, p.ny, p.nz), p.origin, (p.dx, p.dy, p.dz), p.mat, rho,
                               p.sigma_t, src.pos)
    W = source_mask(p, src).astype(np.float64)
    return W[None, :] * np.exp(-tau) / (4.0 * math.pi * r2[None, :])


def uncollided(p, src) -> np.ndarray:
    """phi_u[g][v] of one source (zero for volumetric sources, which enter the
    collided problem directly)."""
    if src.kind == SRC_VOLUME:
        return np.zeros((p.G, p.V))
    return src.weight * src.spectrum[:, None] * unit_uncollided(p, src)


def source_directions(p, src) -> np.ndarray:
    """Unit direction of travel from the source to every voxel centre [V, 3]."""
    X, Y, Z = p.centres()
    d = np.stack([X - src.pos[0], Y - src.pos[1], Z - src.pos[2]], axis=1)
    return d / np.linalg.norm(d, axis=1)[:, None]


def uncollided_moments(p, src, phi_u: np.ndarray) -> np.ndarray:
    """U[g][lm][v] = phi_u[g][v] R_lm(Omega_sv)."""
    R = quad.real_harmonics(p.legendre, source_directions(p, src))   # [V, M]
    return phi_u[:, None, :] * R.T[None, :, :]


def scatter(p, X: np.ndarray, g_from: int, g_to: int, transpose: bool = False) -> np.ndarray:
    """rho(v) sigma_s,l(g_from -> g_to)[mat v] X[lm][v] (or the transposed
    matrix sigma_s,l(g_to -> g_from) when transpose)."""
    ls = quad.moment_degrees(p.legendre)
    if transpose:
        tab = p.sigma_s[:, :, g_to, g_from]          # [nmat, L+1]
    else:
        tab = p.sigma_s[:, :, g_from, g_to]
    coef = tab[p.mat][:, ls].T * p.density.astype(np.float64)[None, :]   # [M, V]
    return coef * X


@dataclass
class Solution:
    phi_u: np.ndarray                 # [G][V] total uncollided fluence
    U: np.ndarray                     # [G][M][V] uncollided moments
    phi_c: np.ndarray                 # [G][M][V] collided moments
    iters: List[int]
    leak: np.ndarray                  # [G] leakage of the last sweep
    balance: np.ndarray               # [G] relative sweep balance residual
    source: np.ndarray                # [G][M][V] moment source of the last sweep
    per_source_phi_u: List[np.ndarray] = field(default_factory=list)
    psi: Optional[np.ndarray] = None  # [G][A][V] angular collided fluence (if stored)

    @property
    def phi(self) -> np.ndarray:
        return self.phi_u + self.phi_c[:, 0, :]


def diamond(p) -> bool:
    """Whether the problem asks for diamond differencing (differencing = 1)."""
    return bool(getattr(p, "differencing", 0))


def external_moments(p) -> np.ndarray:
    """Moment source of volumetric sources: s_00[g] = weight * chi_g per cm^3."""
    E = np.zeros((p.G, quad.n_moments(p.legendre), p.V))
    for s in p.sources:
        if s.kind == SRC_VOLUME:
            E[:, 0, :] += s.weight * s.spectrum[:, None]
    return E


def _iterate(p, fixed: np.ndarray, self_op, dirs, w, Mop, Dop, sigt_v, tol, max_iters,
             store_psi=False):
    """Source iteration of one group: s = fixed + self_op(phi); phi = sweep(s)."""
    dims = (p.nx, p.ny, p.nz)
    sp = (p.dx, p.dy, p.dz)
    M = fixed.shape[0]
    phi = np.zeros((M, p.V))
    it = 0
    while True:
        s = fixed + self_op(phi)
        new, leak, psi = tr.sweep(dims, sp, dirs, w, Mop, Dop, sigt_v, s, store_psi, diamond(p))
        it += 1
        nrm = np.linalg.norm(new[0])
        eps = 0.0 if nrm == 0.0 else np.linalg.norm(new[0] - phi[0]) / nrm
        phi = new
        if eps < tol or it >= max_iters:
            break
    vol = p.dx * p.dy * p.dz
    gain = vol * s[0].sum()
    loss = vol * (sigt_v * phi[0]).sum() + leak
    bal = 0.0 if gain == 0.0 else abs(gain - loss) / abs(gain)
    return phi, it, leak, bal, s, psi


def solve(p, tol: float = 1e-10, max_iters: int = 100000, store_psi: bool = False) -> Solution:
    """Forward solve: uncollided ray trace, first-collision source, collided
    source iteration (groups high -> low energy)."""
    dirs, w, R, Mop, Dop = quad.angular_operators(p.sn, p.legendre)
    M = quad.n_moments(p.legendre)
    G, V = p.G, p.V
    rho = p.density.astype(np.float64)
    phi_u = np.zeros((G, V))
    U = np.zeros((G, M, V))
    per = []
    for s in p.sources:
        if s.kind == SRC_VOLUME:
            per.append(np.zeros((G, V)))
            continue
        pu = uncollided(p, s)
        per.append(pu)
        phi_u += pu
        U += uncollided_moments(p, s, pu)
    ext = external_moments(p)
    phi_c = np.zeros((G, M, V))
    iters, leaks, bals, srcs = [], np.zeros(G), np.zeros(G), np.zeros((G, M, V))
    psi_all = np.zeros((G, dirs.shape[0], V)) if store_psi else None
    for g in range(G):
        fixed = ext[g] + scatter(p, U[g], g, g)
        for gp in range(g):
            fixed = fixed + scatter(p, phi_c[gp] + U[gp], gp, g)
        sigt_v = rho * p.sigma_t[p.mat, g]
        phi, it, leak, bal, s, psi = _iterate(p, fixed, lambda X, g=g: scatter(p, X, g, g),
                                              dirs, w, Mop, Dop, sigt_v, tol, max_iters, store_psi)
        phi_c[g] = phi
        iters.append(it)
        leaks[g], bals[g], srcs[g] = leak, bal, s
        if store_psi:
            # one more sweep with the converged source to store the angular fluence
            _, _, psi = tr.sweep((p.nx, p.ny, p.nz), (p.dx, p.dy, p.dz), dirs, w, Mop, Dop,
                                 sigt_v, fixed + scatter(p, phi, g, g), True, diamond(p))
            psi_all[g] = psi
    return Solution(phi_u=phi_u, U=U, phi_c=phi_c, iters=iters, leak=leaks, balance=bals,
                    source=srcs, per_source_phi_u=per, psi=psi_all)


def dose(p, phi: np.ndarray, k: Optional[np.ndarray] = None) -> np.ndarray:
    """D(v) = sum_g k[mat v, g] rho(v) phi[g](v)."""
    k = p.k_dep if k is None else k
    return (k[p.mat].T * phi).sum(axis=0) * p.density.astype(np.float64)


@dataclass
class AdjointSolution:
    Z: np.ndarray          # [G][M][V] adjoint flux moments
    T: np.ndarray          # [G][M][V] transposed scattering of Z: (S^T Z)
    iters: List[int]
    psi: Optional[np.ndarray] = None   # [G][A][V] adjoint angular fluence (if stored)


def adjoint_solve(p, r: np.ndarray, tol: float = 1e-10, max_iters: int = 100000,
                  store_psi: bool = False) -> AdjointSolution:
    """Adjoint of the collided problem for the response r[g][v] on the scalar
    fluence.  The discrete adjoint of the sweep of direction n (step or
    diamond differenced, on a uniform mesh) is the same sweep along -Omega_n;
    the adjoint moment equation is
      Z = D L^-T M (4 pi r delta_{lm,00} + S^T Z),
    solved from low to high energy (S^T couples each group to lower-energy
    groups)."""
    dirs, w, R, Mop, Dop = quad.angular_operators(p.sn, p.legendre)
    rdirs = -dirs
    M = quad.n_moments(p.legendre)
    G, V = p.G, p.V
    rho = p.density.astype(np.float64)
    Z = np.zeros((G, M, V))
    iters = []
    psi_all = np.zeros((G, dirs.shape[0], V)) if store_psi else None
    for g in reversed(range(G)):
        fixed = np.zeros((M, V))
        fixed[0] = 4.0 * math.pi * r[g]
        for gpp in range(g + 1, G):
            fixed = fixed + scatter(p, Z[gpp], gpp, g, transpose=True)
        sigt_v = rho * p.sigma_t[p.mat, g]
        phi, it, _, _, _, _ = _iterate(p, fixed, lambda X, g=g: scatter(p, X, g, g, transpose=True),
                                       rdirs, w, Mop, Dop, sigt_v, tol, max_iters)
        Z[g] = phi
        iters.append(it)
        if store_psi:
            _, _, psi = tr.sweep((p.nx, p.ny, p.nz), (p.dx, p.dy, p.dz), rdirs, w, Mop, Dop,
                                 sigt_v, fixed + scatter(p, phi, g, g, transpose=True), True,
                                 diamond(p))
            psi_all[g] = psi
    T = np.zeros_like(Z)
    for g in range(G):
        for gpp in range(g, G):
            T[g] += scatter(p, Z[gpp], gpp, g, transpose=True)
    return AdjointSolution(Z=Z, T=T, iters=iters[::-1], psi=psi_all)


def response_from_roi(p, roi_weights: np.ndarray, k: Optional[np.ndarray] = None) -> np.ndarray:
    """Fluence response r[g][v] of J = sum_v roi(v) D(v)."""
    k = p.k_dep if k is None else k
    return k[p.mat].T * (p.density.astype(np.float64) * roi_weights)[None, :]


def roi_dose(p, roi_weights: np.ndarray, tol: float = 1e-12) -> float:
    sol = solve(p, tol=tol)
    return float((roi_weights * dose(p, sol.phi)).sum())


def gradients(p, roi_weights: np.ndarray, tol: float = 1e-12, density: bool = True) -> Dict:
    """Gradients of J = sum_v roi(v) D(v) with respect to the source weights,
    the (shared) spectrum chi_g and the voxel densities, by the adjoint.

    All point sources must share one spectrum chi (that is what d/d chi_g
    means); each source's weight is its per-view tube-current weight."""
    sol = solve(p, tol=tol, store_psi=density)
    r = response_from_roi(p, roi_weights)
    adj = adjoint_solve(p, r, tol=tol, store_psi=density)
    L = p.legendre
    ls = quad.moment_degrees(L)
    C = (2 * ls + 1) / (4.0 * math.pi)
    G, V = p.G, p.V
    d_w = np.zeros(len(p.sources))
    d_chi = np.zeros(G)
    d_rho = np.zeros(V)
    J = float((roi_weights * dose(p, sol.phi)).sum())
    for si, s in enumerate(p.sources):
        if s.kind == SRC_VOLUME:
            # J depends on a volume source through <q_00 / (4 pi), Z_00>
            z00 = adj.Z[:, 0, :].sum(axis=1) / (4.0 * math.pi)
            d_w[si] = float(s.spectrum @ z00)
            d_chi += s.weight * z00
            continue
        u = unit_uncollided(p, s)                                     # [G][V]
        Rs = quad.real_harmonics(L, source_directions(p, s))          # [V][M]
        imp = r + np.einsum("vm,gmv->gv", Rs * C[None, :], adj.T)     # dJ/dphi_u of this source
        d_w[si] = float((s.spectrum[:, None] * u * imp).sum())
        d_chi += s.weight * (u * imp).sum(axis=1)
        if density:
            pu = s.weight * s.spectrum[:, None] * u
            H = p.sigma_t @ (imp * pu)                                 # [nmat][V]
            tr.backproject((p.nx, p.ny, p.nz), p.origin, (p.dx, p.dy, p.dz), p.mat, H, s.pos, d_rho)
    if density:
        rho = p.density.astype(np.float64)
        # (a) explicit dependence of the dose on rho
        d_rho += (roi_weights[None, :] * p.k_dep[p.mat].T * sol.phi).sum(axis=0)
        # (b) collision term of the sweep: -sum_{n,g} w_n psi_adj sigma_t psi
        dirs, w, *_ = quad.angular_operators(p.sn, L)
        for g in range(G):
            prod = (w[:, None] * adj.psi[g] * sol.psi[g]).sum(axis=0)
            d_rho -= p.sigma_t[p.mat, g] * prod
        # (c) scattering: sum_{g,lm} C_l Z[g][lm] sum_g' sigma_s,l(g'->g) (phi_c + U)[g'][lm]
        X = sol.phi_c + sol.U
        for g in range(G):
            for gp in range(g + 1):
                coef = p.sigma_s[:, :, gp, g][p.mat][:, ls].T        # [M][V]
                d_rho += (C[:, None] * adj.Z[g] * coef * X[gp]).sum(axis=0)
        del rho
    return {"J": J, "d_weights": d_w, "d_spectrum": d_chi, "d_density": d_rho,
            "forward": sol, "adjoint": adj}
