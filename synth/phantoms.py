"""Seeded synthetic phantoms, cross sections, spectra and sources.

Everything here is input data for the deterministic CT dose method
(Norris & Liu, arXiv:1811.12391).  The paper's own phantom voxel data, the
ORNL 47-group ENDF/B-VII photon library and the ICRP116 conversion factors
are not available, so stand-ins are generated with the shapes the paper
describes (Sec. II.D: 35 cm water cylinder, abdomen at liver level, mean free
paths of water of 13.9 mm at 20 keV and 60.6 mm at 100 keV).

Conventions shared by both consumers (the FP64 oracle and the CUDA path):
  * voxel arrays are flat, x fastest: v = (k*ny + j)*nx + i;
  * voxel (i, j, k) spans origin + [i, i+1)*dx etc.; the isocentre is (0, 0, 0);
  * groups are ordered from high to low energy (group 0 = highest energy);
  * sigma_t[m, g] and sigma_s[m, l, g_from, g_to] are cm^-1 at unit density;
    a voxel's macroscopic value is density[v] * table[mat[v]];
  * sigma_s holds Legendre moments sigma_s,l of the group-to-group
    differential scattering cross section, downscatter only (g_to >= g_from);
  * a source emits weight * spectrum[g] photons per source particle,
    isotropically (per 4 pi), masked by its collimator.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Source kinds (mirrored by the C-ABI header's DOCTORS_SRC_* constants).
SRC_POINT = 0        # isotropic point source, no collimator
SRC_FAN_CONE = 1     # point source behind a rectangular fan x cone collimator
SRC_VOLUME = 2       # uniform isotropic volumetric source over the whole mesh

# Water-like attenuation fit: sigma_t(E) = pe * A * (20 keV / E)^3 + B  [cm^-1]
# A, B chosen so that the mean free path of water is 13.9 mm at 20 keV and
# 60.6 mm at 100 keV (the two values the paper quotes in Sec. II.D).
_B = (1.0 / 6.06 - (1.0 / 1.39) / 125.0) / (1.0 - 1.0 / 125.0)
_A = 1.0 / 1.39 - _B

CONFIG_NAMES = (
    "tiny_cube",               # 16^3 water cube, S4 P1, 4 groups
    "water_cylinder",          # 64x64x32 35 cm cylinder, S8 P3, 19 groups
    "abdomen",                 # 128x128x48 abdomen, S16 P3, 19 groups
    "axial_scan",              # 64 views on the cylinder + 16 extra cylinders
    "differentiable_abdomen",  # abdomen, S8 P3, 32 views, liver ROI
    "paper_water_coarse_sp",   # the paper's 64x64x16 water runs, S6 P0, 7 groups: one point source
    "paper_water_coarse_ct",   # ... 16 cone beams
    "paper_water_fine_sp",     # the paper's 256x256x64 water runs
    "paper_water_fine_ct",
)


@dataclasses.dataclass
class Source:
    kind: int
    pos: np.ndarray                  # (3,) cm
    axis: np.ndarray                 # (3,) unit vector from source toward isocentre
    fan_deg: float = 360.0           # full in-plane opening angle
    z_half_iso: float = 0.0          # beam half-height at the isocentre distance (cm)
    iso_dist: float = 1.0            # source-to-isocentre distance (cm)
    weight: float = 1.0              # photons per source particle (view weight)
    spectrum: Optional[np.ndarray] = None   # (G,) sums to 1


@dataclasses.dataclass
class Problem:
    name: str
    seed: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    origin: np.ndarray               # (3,) cm, corner of voxel (0,0,0)
    mat: np.ndarray                  # uint8 [V]
    density: np.ndarray              # float32 [V], g/cm^3 relative to table
    sigma_t: np.ndarray              # float64 [nmat, G]
    sigma_s: np.ndarray              # float64 [nmat, L+1, G, G] (from, to)
    sn: int
    legendre: int
    sources: List[Source]
    k_dep: np.ndarray                # float64 [nmat, G] energy-deposition weights
    e_mid: np.ndarray                # float64 [G] keV
    tol: float = 1e-8
    max_iters: int = 500
    roi: Optional[np.ndarray] = None  # bool [V]
    differencing: int = 0            # spatial scheme of the sweep: 0 step, 1 diamond

    @property
    def G(self) -> int:
        return int(self.sigma_t.shape[1])

    @property
    def nmat(self) -> int:
        return int(self.sigma_t.shape[0])

    @property
    def V(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_angles(self) -> int:
        return self.sn * (self.sn + 2)

    def centres(self):
        """Voxel-centre coordinates (x, y, z), each of shape [V]."""
        i = np.arange(self.nx)
        j = np.arange(self.ny)
        k = np.arange(self.nz)
        x = self.origin[0] + (i + 0.5) * self.dx
        y = self.origin[1] + (j + 0.5) * self.dy
        z = self.origin[2] + (k + 0.5) * self.dz
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X.ravel(), Y.ravel(), Z.ravel()

    def with_sources(self, sources: List[Source], name: Optional[str] = None) -> "Problem":
        p = dataclasses.replace(self, sources=list(sources))
        if name is not None:
            p.name = name
        return p


# ----------------------------------------------------------------------------
# groups, spectra, cross sections
# ----------------------------------------------------------------------------

def group_edges(G: int, e_hi: float = 120.0, e_lo: float = 10.0) -> np.ndarray:
    """Equal-width group edges from high to low energy (keV)."""
    return np.linspace(e_hi, e_lo, G + 1)


def kramers_spectrum(e_mid: np.ndarray, rng: np.random.Generator, kvp: float = 120.0) -> np.ndarray:
    """Bremsstrahlung-like spectrum: Kramers (E0-E)/E times a filter with 50%
    transmission at 30 keV (attenuation ~ E^-3), jittered +-5%, normalised."""
    e = np.asarray(e_mid, dtype=np.float64)
    shape = np.clip(kvp - e, 0.0, None) / e * np.power(2.0, -(30.0 / e) ** 3)
    shape = shape * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=e.shape))
    return shape / shape.sum()


def _downscatter(total_out: np.ndarray, rng: np.random.Generator, L: int,
                 within=(0.3, 0.6), aniso=(0.1, 0.4), decay=0.5) -> np.ndarray:
    """Group-to-group Legendre scattering moments [L+1, G, G] (from, to).

    total_out[g] is sum_{g'} sigma_s,0(g -> g').  A seeded fraction stays in
    group g; the rest goes to lower groups with geometric decay.  For the
    lowest group the remainder leaves the group structure (it is absorbed
    below the lowest edge).  sigma_s,l = sigma_s,0 * a_g^l."""
    G = total_out.shape[0]
    s0 = np.zeros((G, G))
    for g in range(G):
        f_in = rng.uniform(*within)
        s0[g, g] = f_in * total_out[g]
        lower = np.arange(g + 1, G)
        if lower.size:
            wts = decay ** (lower - g - 1.0)
            s0[g, lower] = (1.0 - f_in) * total_out[g] * wts / wts.sum()
    a = rng.uniform(*aniso, size=G)
    out = np.zeros((L + 1, G, G))
    for l in range(L + 1):
        out[l] = s0 * (a[:, None] ** l)
    return out


def _material_tables(e_mid: np.ndarray, pe_mult: List[float], rng: np.random.Generator, L: int):
    """Water-like tables per material: sigma_t = pe*A*(20/E)^3 + B and
    Compton-like out-scatter B*f, f in [0.9, 1.0]."""
    nmat = len(pe_mult)
    G = e_mid.shape[0]
    sigt = np.zeros((nmat, G))
    sigs = np.zeros((nmat, L + 1, G, G))
    for m, pe in enumerate(pe_mult):
        pe = pe * (1.0 + 0.05 * rng.uniform(-1.0, 1.0))
        sigt[m] = pe * _A * (20.0 / e_mid) ** 3 + _B
        total_out = _B * rng.uniform(0.9, 1.0, size=G)
        sigs[m] = _downscatter(total_out, rng, L)
    return sigt, sigs


def deposition_weights(sigma_t: np.ndarray, sigma_s: np.ndarray, e_mid: np.ndarray) -> np.ndarray:
    """Energy-deposition weights k[m, g] = E_g * sigma_a[m, g] (keV cm^-1 per
    unit fluence at unit density), sigma_a = sigma_t - sum_g' sigma_s,0(g->g').
    They stand in for the ICRP116 fluence-to-dose factors."""
    sig_a = sigma_t - sigma_s[:, 0].sum(axis=2)
    return e_mid[None, :] * sig_a


def _centred_origin(nx, ny, nz, dx, dy, dz):
    return -0.5 * np.array([nx * dx, ny * dy, nz * dz], dtype=np.float64)


def _ring_source(theta: float, dist: float, spectrum, fan_deg: float, z_half: float,
                 weight: float = 1.0) -> Source:
    """Collimated point source on a gantry circle at angle theta (theta = 0
    puts it on the -y axis), aimed at the isocentre."""
    pos = dist * np.array([math.sin(theta), -math.cos(theta), 0.0])
    axis = -pos / np.linalg.norm(pos)
    return Source(kind=SRC_FAN_CONE, pos=pos, axis=axis, fan_deg=fan_deg,
                  z_half_iso=z_half, iso_dist=dist, weight=weight,
                  spectrum=np.asarray(spectrum, dtype=np.float64).copy())


# ----------------------------------------------------------------------------
# phantoms
# ----------------------------------------------------------------------------

def tiny_cube(seed: int = 0, n: int = 16, sn: int = 4, L: int = 1) -> Problem:
    """16^3 water cube, 1 cm voxels, 4 groups with sigma_t = 0.50/0.30/0.22/0.18,
    downscatter P1 with per-group scattering ratio in [0.4, 0.9], point source
    10 cm outside the centre of the -z face, isotropic."""
    rng = np.random.default_rng(seed)
    sigt_w = np.array([0.50, 0.30, 0.22, 0.18])
    G = sigt_w.size
    c = rng.uniform(0.4, 0.9, size=G)
    sigs = _downscatter(c * sigt_w, rng, L)[None]
    sigt = sigt_w[None, :].copy()
    e_mid = np.array([85.0, 57.5, 37.5, 20.0])
    V = n ** 3
    origin = _centred_origin(n, n, n, 1.0, 1.0, 1.0)
    spec = rng.uniform(0.5, 1.5, size=G)
    spec /= spec.sum()
    src = Source(kind=SRC_POINT, pos=np.array([0.0, 0.0, origin[2] - 10.0]),
                 axis=np.array([0.0, 0.0, 1.0]), spectrum=spec,
                 iso_dist=10.0 + n / 2.0)
    return Problem(name="tiny_cube", seed=seed, nx=n, ny=n, nz=n, dx=1.0, dy=1.0, dz=1.0,
                   origin=origin, mat=np.zeros(V, np.uint8), density=np.ones(V, np.float32),
                   sigma_t=sigt, sigma_s=sigs, sn=sn, legendre=L, sources=[src],
                   k_dep=deposition_weights(sigt, sigs, e_mid), e_mid=e_mid, tol=1e-8)


def water_cylinder(seed: int = 1, nx: int = 64, ny: int = 64, nz: int = 32,
                   dx: float = 0.55, dy: float = 0.55, dz: float = 0.5,
                   diameter: float = 35.0, G: int = 19, sn: int = 8, L: int = 3,
                   sid: float = 54.0, fan_deg: float = 40.0, z_width: float = 4.0,
                   theta: float = 0.0) -> Problem:
    """Uniform water cylinder along z (air outside) on a voxel mesh centred on
    the isocentre; one fan x cone collimated source at sid cm on the gantry
    circle (theta = 0: on the -y axis), 120 kVp spectrum over 10-120 keV."""
    rng = np.random.default_rng(seed)
    edges = group_edges(G)
    e_mid = 0.5 * (edges[:-1] + edges[1:])
    # materials: 0 = air, 1 = water
    sigt, sigs = _material_tables(e_mid, [0.9, 1.0], rng, L)
    rho_mat = np.array([0.0012, 1.0]) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=2))
    origin = _centred_origin(nx, ny, nz, dx, dy, dz)
    p = Problem(name="water_cylinder", seed=seed, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                origin=origin, mat=np.zeros(nx * ny * nz, np.uint8),
                density=np.zeros(nx * ny * nz, np.float32), sigma_t=sigt, sigma_s=sigs,
                sn=sn, legendre=L, sources=[], k_dep=deposition_weights(sigt, sigs, e_mid),
                e_mid=e_mid, tol=1e-8)
    X, Y, _ = p.centres()
    inside = X * X + Y * Y <= (0.5 * diameter) ** 2
    p.mat[:] = np.where(inside, 1, 0).astype(np.uint8)
    p.density[:] = rho_mat[p.mat].astype(np.float32)
    spec = kramers_spectrum(e_mid, rng)
    p.sources = [_ring_source(theta, sid, spec, fan_deg, 0.5 * z_width)]
    return p


def abdomen(seed: int = 2, nx: int = 128, ny: int = 128, nz: int = 48, d: float = 0.25,
            dz: float = 0.25, G: int = 19, sn: int = 16, L: int = 3, sid: float = 54.0,
            fan_deg: float = 40.0, z_width: Optional[float] = None, n_views: int = 1) -> Problem:
    """Abdomen-like phantom at liver level.  Outer 32 x 24 cm ellipse with a
    1 cm fat rim around soft tissue, an elliptic bone spine (4 x 3 cm at
    (0, -8) cm), two air-filled bowel ellipses (5 x 3 cm at (+-5, +7) cm) and
    a liver ellipse (10 x 8 cm at (-6, 0) cm); air outside.  Materials:
    0 air, 1 fat, 2 soft tissue, 3 liver, 4 bone.  Cone-beam source(s) on the
    54 cm gantry circle covering the full axial extent unless z_width is set."""
    rng = np.random.default_rng(seed)
    edges = group_edges(G)
    e_mid = 0.5 * (edges[:-1] + edges[1:])
    pe = [0.9, 0.6, 1.0, 1.05, 6.0]
    sigt, sigs = _material_tables(e_mid, pe, rng, L)
    rho_mat = np.array([0.0012, 0.92, 1.03, 1.06, 1.85]) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=5))
    origin = _centred_origin(nx, ny, nz, d, d, dz)
    V = nx * ny * nz
    p = Problem(name="abdomen", seed=seed, nx=nx, ny=ny, nz=nz, dx=d, dy=d, dz=dz, origin=origin,
                mat=np.zeros(V, np.uint8), density=np.zeros(V, np.float32), sigma_t=sigt,
                sigma_s=sigs, sn=sn, legendre=L, sources=[],
                k_dep=deposition_weights(sigt, sigs, e_mid), e_mid=e_mid, tol=1e-8)
    X, Y, _ = p.centres()

    def ell(cx, cy, ax, ay):
        return ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 <= 1.0

    m = np.zeros(V, np.uint8)
    m[ell(0, 0, 16.0, 12.0)] = 1
    m[ell(0, 0, 15.0, 11.0)] = 2
    m[ell(-6.0, 0.0, 5.0, 4.0)] = 3
    m[ell(0.0, -8.0, 2.0, 1.5)] = 4
    m[ell(5.0, 7.0, 2.5, 1.5)] = 0
    m[ell(-5.0, 7.0, 2.5, 1.5)] = 0
    p.mat[:] = m
    p.density[:] = rho_mat[m].astype(np.float32)
    spec = kramers_spectrum(e_mid, rng)
    zw = nz * dz if z_width is None else z_width
    p.sources = [_ring_source(2.0 * math.pi * k / n_views, sid, spec, fan_deg, 0.5 * zw)
                 for k in range(n_views)]
    return p


# ----------------------------------------------------------------------------
# synthetic CT calibration (the paper's stoichiometric calibration is cited,
# not printed; Sec. II.B)
# ----------------------------------------------------------------------------

def ct_calibration() -> dict:
    """A synthetic CT-number calibration for the abdomen's five materials
    (0 air, 1 fat, 2 soft tissue, 3 liver, 4 bone): bin thresholds in HU and
    a piecewise-linear HU -> density curve (g/cm^3)."""
    return {
        "thresholds": np.array([-500.0, -30.0, 45.0, 150.0], np.float32),
        "bin_material": np.array([0, 1, 2, 3, 4], np.uint8),
        "hu_knots": np.array([-1000.0, -100.0, 20.0, 60.0, 1000.0], np.float32),
        "rho_knots": np.array([0.0012, 0.93, 1.03, 1.06, 1.85], np.float32),
    }


# per material: centre and half-width of the synthetic CT numbers (inside the
# material's bin of ct_calibration)
_CT_HU = {0: (-1000.0, 20.0), 1: (-100.0, 30.0), 2: (10.0, 25.0), 3: (60.0, 10.0), 4: (700.0, 200.0)}


def synthetic_ct(p: Problem, seed: int = 9) -> np.ndarray:
    """A seeded CT image (HU, float32 [V]) of a phantom with the abdomen's
    materials: each voxel's number drawn uniformly around its material's
    centre, inside that material's calibration bin."""
    rng = np.random.default_rng(seed)
    hu = np.zeros(p.V, np.float32)
    for m, (c, w) in _CT_HU.items():
        sel = p.mat == m
        hu[sel] = (c + w * rng.uniform(-1.0, 1.0, size=int(sel.sum()))).astype(np.float32)
    return hu


# the paper's seven group edges (keV, high to low; Sec. II.D)
PAPER_EDGES = np.array([100.0, 75.0, 70.0, 60.0, 45.0, 30.0, 20.0, 10.0])


def paper_water(seed: int = 6, fine: bool = False, ct: bool = False, sn: int = 6, L: int = 0,
                sid: float = 54.0) -> Problem:
    """The paper's water-phantom runs (Sec. II.D, III.D, Table 6): a 35 cm
    water cylinder in a 50 x 50 x 12.5 cm volume, on the fine 256 x 256 x 64
    mesh (1.95 mm voxels) or the coarse 64 x 64 x 16 mesh (7.81 mm), seven
    groups with the paper's edges 10-100 keV, S6 P0.  Single projection: an
    isotropic point source; CT scan: 16 cone beams with a 30 degree cone angle
    placed uniformly on the gantry circle.  The source distance is not given
    in the paper; the sources sit at sid cm from the isocentre."""
    rng = np.random.default_rng(seed)
    n, nzz = (256, 64) if fine else (64, 16)
    d = 50.0 / n
    e_mid = 0.5 * (PAPER_EDGES[:-1] + PAPER_EDGES[1:])
    sigt, sigs = _material_tables(e_mid, [0.9, 1.0], rng, L)
    rho_mat = np.array([0.0012, 1.0]) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=2))
    origin = _centred_origin(n, n, nzz, d, d, d)
    V = n * n * nzz
    name = f"paper_water_{'fine' if fine else 'coarse'}_{'ct' if ct else 'sp'}"
    p = Problem(name=name, seed=seed, nx=n, ny=n, nz=nzz, dx=d, dy=d, dz=d, origin=origin,
                mat=np.zeros(V, np.uint8), density=np.zeros(V, np.float32), sigma_t=sigt, sigma_s=sigs,
                sn=sn, legendre=L, sources=[], k_dep=deposition_weights(sigt, sigs, e_mid),
                e_mid=e_mid, tol=1e-8)
    X, Y, _ = p.centres()
    p.mat[:] = np.where(X * X + Y * Y <= 17.5 ** 2, 1, 0).astype(np.uint8)
    p.density[:] = rho_mat[p.mat].astype(np.float32)
    spec = kramers_spectrum(e_mid, rng, kvp=100.0)
    if ct:
        z_half = sid * math.tan(math.radians(15.0))
        p.sources = [_ring_source(2.0 * math.pi * k / 16, sid, spec, 30.0, z_half) for k in range(16)]
    else:
        p.sources = [Source(kind=SRC_POINT, pos=np.array([0.0, -sid, 0.0]), axis=np.array([0.0, 1.0, 0.0]),
                            spectrum=spec, iso_dist=sid)]
    return p


def liver_roi(p: Problem, size_cm: float = 4.0, centre=(-6.0, 0.0, 0.0)) -> np.ndarray:
    """Cubic region of interest (bool [V]) of about size_cm centred at centre."""
    X, Y, Z = p.centres()
    h = 0.5 * size_cm
    return ((np.abs(X - centre[0]) < h) & (np.abs(Y - centre[1]) < h) & (np.abs(Z - centre[2]) < h))


def axial_scan_sources(p: Problem, n_views: int, sid: float = 54.0, fan_deg: float = 40.0,
                       z_width: float = 4.0) -> List[Source]:
    """n_views collimated sources evenly spaced on the gantry circle."""
    spec = p.sources[0].spectrum
    return [_ring_source(2.0 * math.pi * k / n_views, sid, spec, fan_deg, 0.5 * z_width)
            for k in range(n_views)]


def extra_cylinders(seed: int = 3, G: int = 19, sn: int = 8, L: int = 3) -> List[Problem]:
    """The 16 extra instances of the batched axial scan: 6 x 48^3 meshes with a
    16 cm cylinder, 5 x 64x64x32 with 24 cm, 5 x 96x96x32 with 32 cm.  In-plane
    spacing 0.55 cm, axial extent 16 cm.  One view each, at 2 pi k / 16."""
    out = []
    specs = [(48, 48, 48, 16.0)] * 6 + [(64, 64, 32, 24.0)] * 5 + [(96, 96, 32, 32.0)] * 5
    for k, (nx, ny, nz, dia) in enumerate(specs):
        q = water_cylinder(seed=seed + k, nx=nx, ny=ny, nz=nz, dx=0.55, dy=0.55, dz=16.0 / nz,
                           diameter=dia, G=G, sn=sn, L=L, theta=2.0 * math.pi * k / 16.0)
        q.name = f"cylinder_{int(dia)}cm_{nx}x{ny}x{nz}"
        out.append(q)
    return out


def infinite_medium_cube(seed: int = 5, n: int = 16, G: int = 3, sigma_t: float = 40.0,
                         sn: int = 4, L: int = 0, q_total: float = 1.0) -> Problem:
    """Thick cube (1 cm voxels, sigma_t = 40 cm^-1 in every group) with a
    uniform isotropic volumetric source: far from the boundary the fluence is
    the infinite-medium value.  (With step differencing the boundary deficit
    decays by sum_q c_q / (sigma_t + sum_q c_q) per cell, about 0.04 here, so
    eight cells from the boundary it is below 1e-11.)"""
    rng = np.random.default_rng(seed)
    sigt = np.full((1, G), sigma_t)
    total_out = sigma_t * rng.uniform(0.4, 0.9, size=G)
    sigs = _downscatter(total_out, rng, L)[None]
    e_mid = np.linspace(100.0, 20.0, G)
    spec = rng.uniform(0.5, 1.5, size=G)
    spec /= spec.sum()
    V = n ** 3
    src = Source(kind=SRC_VOLUME, pos=np.zeros(3), axis=np.array([0.0, 0.0, 1.0]),
                 weight=q_total, spectrum=spec)
    return Problem(name="infinite_medium", seed=seed, nx=n, ny=n, nz=n, dx=1.0, dy=1.0, dz=1.0,
                   origin=_centred_origin(n, n, n, 1.0, 1.0, 1.0), mat=np.zeros(V, np.uint8),
                   density=np.ones(V, np.float32), sigma_t=sigt, sigma_s=sigs, sn=sn, legendre=L,
                   sources=[src], k_dep=deposition_weights(sigt, sigs, e_mid), e_mid=e_mid)


def config_problem(name: str, sn: Optional[int] = None, L: Optional[int] = None) -> Problem:
    """The named full-size workloads (single-problem forms); `sn` and `L`
    override the quadrature order and the Legendre order of the tiny cube,
    the water cylinder and the abdomen."""
    kw = {k: v for k, v in (("sn", sn), ("L", L)) if v is not None}
    if name == "tiny_cube":
        return tiny_cube(**kw)
    if name == "water_cylinder":
        return water_cylinder(**kw)
    if name == "abdomen":
        return abdomen(**kw)
    if kw:
        raise ValueError(f"sn and L overrides apply to tiny_cube, water_cylinder and abdomen, not {name}")
    if name == "axial_scan":
        p = water_cylinder()
        return p.with_sources(axial_scan_sources(p, 64), name="axial_scan")
    if name.startswith("paper_water_"):
        _, _, mesh, mode = name.split("_")
        return paper_water(fine=mesh == "fine", ct=mode == "ct")
    if name == "differentiable_abdomen":
        p = abdomen(sn=8, n_views=32)
        p.name = "differentiable_abdomen"
        p.roi = liver_roi(p)
        return p
    raise KeyError(name)
