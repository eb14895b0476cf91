"""Pins of the oracle's Siddon walk and uncollided fluence (Sec. II.A: the
uncollided fluence is computed by ray tracing and is independent of the S_N
and P_N orders, Sec. III.A)."""
import math

import numpy as np
import pytest

from oracle import solver as osv
from oracle import transport as tr
from synth import phantoms as ph


def _in_mesh_length(S, T, lo, hi):
    """Closed-form length of the part of segment S->T inside the box (T inside)."""
    S, T = np.asarray(S, float), np.asarray(T, float)
    d = T - S
    a_in = 0.0
    for q in range(3):
        if d[q] != 0:
            a0, a1 = (lo[q] - S[q]) / d[q], (hi[q] - S[q]) / d[q]
            a_in = max(a_in, min(a0, a1))
    return (1.0 - a_in) * np.linalg.norm(d)


def _ijk(v, nx, ny):
    return v % nx, (v // nx) % ny, v // (nx * ny)


def test_axis_parallel_ray():
    dims, o, d = (4, 2, 2), (0, 0, 0), (1, 1, 1)
    idx, ln = tr.siddon_f64((-10.0, 0.5, 0.5), (3, 0, 0), dims, o, d)
    assert [_ijk(v, 4, 2) for v in idx] == [(3, 0, 0), (2, 0, 0), (1, 0, 0), (0, 0, 0)]
    np.testing.assert_allclose(ln, [0.5, 1, 1, 1], rtol=1e-14)
    idx32, ln32 = tr.siddon_f32((-10.0, 0.5, 0.5), (3, 0, 0), dims, o, d)
    assert list(idx32) == list(idx)


def test_diagonal_ray_through_corners():
    """A 45 degree in-plane ray crosses x and y planes at the same parameter:
    the tie is broken x first and the zero-length corner voxels are dropped."""
    dims, o, d = (4, 4, 1), (0, 0, 0), (1, 1, 1)
    for f in (tr.siddon_f64, tr.siddon_f32):
        idx, ln = f((-10.0, -10.0, 0.5), (3, 3, 0), dims, o, d)
        assert [_ijk(v, 4, 4) for v in idx] == [(3, 3, 0), (2, 2, 0), (1, 1, 0), (0, 0, 0)]
        np.testing.assert_allclose(ln, np.array([0.5, 1, 1, 1]) * math.sqrt(2), rtol=1e-6)


def test_reverse_direction_ray():
    """Source on the +x side: the walk steps toward +x."""
    dims, o, d = (5, 1, 1), (-2.5, 0, 0), (1, 1, 1)
    idx, ln = tr.siddon_f64((30.0, 0.5, 0.5), (1, 0, 0), dims, o, d)
    assert [_ijk(v, 5, 1)[0] for v in idx] == [1, 2, 3, 4]
    np.testing.assert_allclose(ln, [0.5, 1, 1, 1])


def test_random_rays_sum_to_closed_form_and_are_connected():
    rng = np.random.default_rng(7)
    dims = (7, 5, 6)
    o = np.array([-1.3, 0.4, -2.0])
    d = np.array([0.55, 0.7, 0.5])
    lo, hi = o, o + np.array(dims) * d
    for _ in range(300):
        S = rng.uniform(-30, 30, size=3)
        if np.all((S > lo) & (S < hi)):
            continue
        vox = tuple(int(rng.integers(0, n)) for n in dims)
        T = o + (np.array(vox) + 0.5) * d
        idx, ln = tr.siddon_f64(S, vox, dims, o, d)
        assert ln.min() > 0
        assert abs(ln.sum() - _in_mesh_length(S, T, lo, hi)) < 1e-11
        assert _ijk(idx[0], dims[0], dims[1]) == vox
        cells = [np.array(_ijk(v, dims[0], dims[1])) for v in idx]
        for a, b in zip(cells[:-1], cells[1:]):
            step = np.abs(a - b)
            assert 1 <= step.sum() <= 3 and step.max() == 1
        # FP32 list equals the FP64 list up to segments shorter than 1e-5 voxel
        idx32, ln32 = tr.siddon_f32(S, vox, dims, o, d)
        keep64 = [v for v, l in zip(idx, ln) if l > 1e-5 * d.min()]
        keep32 = [v for v, l in zip(idx32, ln32) if l > 1e-5 * d.min()]
        assert keep64 == keep32
        assert abs(ln32.sum() - ln.sum()) < 1e-4 * ln.sum() + 1e-5


def test_homogeneous_uncollided_closed_form():
    """phi_u = chi_g exp(-sigma_g l_in) / (4 pi r^2) in a homogeneous mesh."""
    p = ph.tiny_cube(n=8)
    p.density[:] = 1.0
    src = p.sources[0]
    src.pos = np.array([-3.1, 12.7, -15.3])
    phi = osv.uncollided(p, src)
    X, Y, Z = p.centres()
    lo = p.origin
    hi = p.origin + np.array([p.nx * p.dx, p.ny * p.dy, p.nz * p.dz])
    for v in range(p.V):
        T = (X[v], Y[v], Z[v])
        l_in = _in_mesh_length(src.pos, T, lo, hi)
        r2 = float(np.sum((np.array(T) - src.pos) ** 2))
        exact = src.spectrum * np.exp(-p.sigma_t[0] * l_in) / (4 * math.pi * r2)
        np.testing.assert_allclose(phi[:, v], exact, rtol=1e-12)


def test_uncollided_independent_of_sn_and_pn():
    a = ph.tiny_cube(n=6, sn=4, L=1)
    b = ph.tiny_cube(n=6, sn=8, L=3)
    np.testing.assert_array_equal(osv.uncollided(a, a.sources[0]), osv.uncollided(b, b.sources[0]))


def test_collimator_mask_matches_angles():
    """Away from the collimator edges the FP32 mask equals the FP64 angular test."""
    p = ph.water_cylinder(nx=24, ny=24, nz=12, G=3, sn=4, L=1)
    src = p.sources[0]
    W = osv.source_mask(p, src)
    X, Y, Z = p.centres()
    u = np.stack([X, Y, Z], 1) - src.pos
    along = u @ src.axis
    perp, up = osv.collimator_frame(src.axis)
    fan = np.degrees(np.abs(np.arctan2(u @ perp, along)))
    cone = np.abs(u @ up) / along
    margin = (np.abs(fan - src.fan_deg / 2) > 1e-3) & (np.abs(cone - src.z_half_iso / src.iso_dist) > 1e-5)
    expect = (along > 0) & (fan <= src.fan_deg / 2) & (cone <= src.z_half_iso / src.iso_dist)
    assert np.array_equal(W[margin].astype(bool), expect[margin])
    assert 0 < W.sum() < p.V


def test_synthetic_water_matches_paper_mean_free_paths():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "water_mean_free_path.txt")) as f:
        rows = [list(map(float, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for e, mfp in rows:
        sig = ph._A * (20.0 / e) ** 3 + ph._B
        assert abs(1.0 / sig - mfp) < 1e-12
