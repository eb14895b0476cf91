"""Parity of the full forward solve (ray trace, first-collision source,
collided source iteration with octant wavefront sweeps, dose) against the
FP64 oracle, plus properties that hold at any size."""
import math

import numpy as np
import pytest

from oracle import solver as osv
from synth import phantoms as ph
from tests.parity import REL_TOL, max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    from paper_1811_12391_gb300.build import build
    build()
    from paper_1811_12391_gb300.solver import DoctorsProblem
    return DoctorsProblem


def _compare(d, p, sol, tag):
    d.solve()
    phi_u = d.fluence_host(0)
    phi_c = d.fluence_host(1)
    phi = d.fluence_host(2)
    dose = d.dose_host(p.k_dep)
    errs = {
        "phi_u": max_rel(phi_u, sol.phi_u),
        "phi_c": max_rel(phi_c, sol.phi_c[:, 0, :]),
        "phi": max_rel(phi, sol.phi),
        "dose": max_rel(dose, osv.dose(p, sol.phi)),
    }
    for k, e in errs.items():
        assert e <= REL_TOL, (tag, k, e, errs)
    assert d.result["balance_rel"] < 1e-5
    return errs


def test_tiny_cube_full(dp):
    """16^3 water cube, S4 P1, 4 groups (the oracle finishes in seconds)."""
    p = ph.tiny_cube()
    sol = osv.solve(p, tol=1e-11)
    d = dp(p, tol=1e-6, max_iters=400)
    _compare(d, p, sol, "tiny_cube")
    d.close()


@pytest.fixture(scope="module")
def cylinder_ref():
    p = ph.water_cylinder(nx=36, ny=28, nz=10, dx=1.0, dy=1.25, dz=1.1, diameter=30.0, G=5, sn=8, L=3)
    return p, osv.solve(p, tol=1e-11)


@pytest.mark.parametrize("tile,ab,kernel", [((16, 16), 0, 1), ((16, 16), 0, 3), ((8, 4), 5, 1),
                                            ((8, 4), 5, 3), ((5, 7), 2, 1), ((5, 7), 2, 3),
                                            ((32, 8), 10, 1), ((32, 8), 10, 3), ((8, 16), 10, 1), ((16, 2), 1, 3),
                                            ((16, 16), 10, 4), ((16, 8), 10, 4), ((5, 7), 10, 4), ((8, 4), 10, 4),
                                            ((8, 8), 10, 4), ((8, 8), 10, 0),
                                            ((8, 8), 10, 5), ((16, 8), 10, 5), ((5, 7), 10, 5),
                                            ((8, 8), 10, 7), ((16, 8), 10, 7), ((5, 7), 10, 7), ((32, 8), 10, 7),
                                            ((8, 8), 10, 8), ((5, 7), 10, 8)])
def test_ragged_multitile_cylinder(dp, cylinder_ref, tile, ab, kernel):
    """Several sweep tiles with ragged tails in x and y, S8 P3, with the
    CUDA-core (1), chained (3), dataflow (4), dataflow with split
    transforms (5), dataflow with a face warp (7; 5x7 leaves a partly used
    column warp, 32x8 gives the face warp 40 records) and split transforms on
    the tensor cores (8; 3xTF32) sweeps."""
    p, sol = cylinder_ref
    d = dp(p, tol=1e-6, max_iters=400, tile=tile, angles_per_block=ab, sweep_kernel=kernel)
    _compare(d, p, sol, f"cylinder tile={tile} ab={ab} kernel={kernel}")
    d.close()


@pytest.fixture(scope="module")
def s16_abdomen():
    p = ph.abdomen(nx=32, ny=32, nz=6, d=1.0, dz=2.0, G=3, sn=16, L=3)
    return p, osv.solve(p, tol=1e-11)


@pytest.mark.parametrize("kernel,tile,ab", [(1, (0, 0), 0), (3, (0, 0), 0), (0, (0, 0), 0), (4, (0, 0), 36),
                                            (7, (5, 7), 36), (7, (16, 8), 36), (4, (5, 7), 12), (7, (16, 8), 12)])
def test_abdomen_s16_multi_angle_block(dp, s16_abdomen, kernel, tile, ab):
    """Heterogeneous abdomen-like phantom, S16, P3, five materials: the stage
    and chained kernels (three blocks of 12 directions per octant), the
    dataflow kernels on whole octants (36 directions per cell step; the
    default) and as one launch per block of 12 directions, on ragged 5x7 and
    16x8 face-warp tiles."""
    p, sol = s16_abdomen
    d = dp(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, tile=tile, angles_per_block=ab)
    _compare(d, p, sol, f"abdomen S16 kernel={kernel} tile={tile} ab={ab}")
    d.close()


@pytest.fixture(scope="module")
def s12_cylinder():
    p = ph.water_cylinder(nx=20, ny=18, nz=5, dx=1.5, dy=1.5, dz=2.0, diameter=24.0, G=3, sn=12, L=3)
    return p, osv.solve(p, tol=1e-11)


@pytest.mark.parametrize("kernel,tile,ab", [(0, (0, 0), 0), (4, (5, 7), 21), (7, (8, 8), 21), (3, (0, 0), 7),
                                            (1, (0, 0), 7)])
def test_s12_whole_octants_and_blocks(dp, s12_cylinder, kernel, tile, ab):
    """S12 (21 directions per octant), P3: the dataflow kernels on whole
    octants (the default, a ragged 5x7 tile, the face warp) and the chained and
    stage kernels in blocks of 7, against the oracle."""
    p, sol = s12_cylinder
    d = dp(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, tile=tile, angles_per_block=ab)
    _compare(d, p, sol, f"cylinder S12 kernel={kernel} tile={tile} ab={ab}")
    d.close()


def test_s16_dataflow_block_checks(dp):
    """S16 reaches the dataflow kernels as whole octants or in blocks of 12
    directions: other blocks, whole octants on the stage and chained
    kernels, and the split-transform kernels (S2..S8 only) are rejected with
    DOCTORS_ERR_INVALID_ARG."""
    from paper_1811_12391_gb300 import _lib as C
    p = ph.abdomen(nx=8, ny=8, nz=2, d=1.0, dz=2.0, G=2, sn=16, L=1)
    for kernel, ab in ((4, 6), (7, 9), (5, 12), (8, 12), (5, 36), (1, 36), (3, 36)):
        with pytest.raises(C.DoctorsError) as e:
            dp(p, tol=1e-6, max_iters=10, sweep_kernel=kernel, angles_per_block=ab)
        assert e.value.code == C.DOCTORS_ERR_INVALID_ARG


def test_sweep_kernels_agree(dp):
    """Every sweep kernel gives the same fluence on the full-size water
    cylinder (one sweep from the first-collision source)."""
    p = ph.water_cylinder()
    outs = []
    for kernel in (1, 3, 4, 5, 7, 8):
        d = dp(p, tol=1e-6, max_iters=1, sweep_kernel=kernel, angles_per_block=10)
        d.solve(allow_not_converged=True)
        outs.append(d.fluence_host(1))
        d.close()
    for k in range(1, len(outs)):
        assert max_rel(outs[k], outs[0]) <= 2e-5


def test_p0_and_p2_moment_counts(dp):
    for L in (0, 2):
        p = ph.water_cylinder(nx=12, ny=12, nz=6, dx=1.5, dy=1.5, dz=1.5, diameter=16, G=3, sn=6, L=L)
        sol = osv.solve(p, tol=1e-11)
        d = dp(p, tol=1e-6, max_iters=400)
        _compare(d, p, sol, f"L={L}")
        d.close()


def test_infinite_medium_volume_source(dp):
    p = ph.infinite_medium_cube(n=16, G=3, sn=4, L=0)
    d = dp(p, tol=1e-6, max_iters=400)
    d.solve()
    phi = d.fluence_host(2)
    Q = p.sources[0].weight * p.sources[0].spectrum
    s0, st = p.sigma_s[0, 0], p.sigma_t[0]
    ref = np.zeros(p.G)
    for g in range(p.G):
        ref[g] = (Q[g] + sum(s0[gp, g] * ref[gp] for gp in range(g))) / (st[g] - s0[g, g])
    v = (8 * 16 + 8) * 16 + 8
    np.testing.assert_allclose(phi[:, v], ref, rtol=1e-5)
    d.close()


@pytest.mark.parametrize("kernel", [1, 3, 4, 5, 7])
def test_degenerate_meshes(dp, kernel):
    """Single voxel, single column and single plane meshes."""
    for dims in ((1, 1, 1), (1, 1, 7), (5, 1, 1), (4, 6, 1)):
        p = ph.tiny_cube(n=2)
        p.nx, p.ny, p.nz = dims
        V = p.V
        p.mat = np.zeros(V, np.uint8)
        p.density = np.ones(V, np.float32)
        p.origin = -0.5 * np.array(dims, float)
        sol = osv.solve(p, tol=1e-12)
        d = dp(p, tol=1e-6, max_iters=400, sweep_kernel=kernel, angles_per_block=3)
        _compare(d, p, sol, f"dims={dims} kernel={kernel}")
        d.close()


def test_zero_weight_source_gives_zero(dp):
    p = ph.tiny_cube(n=6)
    p.sources[0].weight = 0.0
    d = dp(p, tol=1e-6, max_iters=10)
    r = d.solve()
    assert r["converged"] == 1
    assert np.all(d.fluence_host(2) == 0)
    d.close()


def test_errors_are_reported(dp):
    from paper_1811_12391_gb300 import _lib as C
    p = ph.tiny_cube(n=4)
    d = dp(p, tol=1e-6, max_iters=10)
    with pytest.raises(C.DoctorsError) as e:
        d.dose_host(p.k_dep)          # before solve
    assert e.value.code == C.DOCTORS_ERR_STATE
    bad = ph.tiny_cube(n=4)
    bad.sources[0].pos = np.array([0.1, 0.2, 0.3])       # inside the mesh
    with pytest.raises(C.DoctorsError) as e:
        d.set_sources(bad.sources)
    assert e.value.code == C.DOCTORS_ERR_INVALID_ARG
    ss = p.sigma_s.copy()
    ss[0, 0, 2, 1] = 0.01                                   # upscatter
    with pytest.raises(C.DoctorsError) as e:
        d.set_materials(p.mat, p.density, p.sigma_t, ss)
    assert e.value.code == C.DOCTORS_ERR_INVALID_ARG
    m = p.mat.copy()
    m[3] = 7
    with pytest.raises(C.DoctorsError):
        d.set_materials(m, p.density, p.sigma_t, p.sigma_s)
    d.close()


def test_iteration_cap_reports_not_converged(dp):
    """A cap below the iterations the problem needs returns
    DOCTORS_ERR_NOT_CONVERGED with the partial results still readable (host
    loop and graph-captured device loop alike); a later solve with a larger
    cap on the same problem converges to the oracle."""
    from paper_1811_12391_gb300 import _lib as C
    p = ph.tiny_cube(n=8)
    ref = osv.solve(p, tol=1e-11)
    for device_loop, kernel in ((0, 0), (1, 0), (1, 4), (0, 5), (1, 5), (0, 7), (1, 7)):
        d = dp(p, tol=1e-6, max_iters=3, device_loop=device_loop, sweep_kernel=kernel, angles_per_block=3)
        with pytest.raises(C.DoctorsError) as e:
            d.solve()
        assert e.value.code == C.DOCTORS_ERR_NOT_CONVERGED
        r = d.solve(allow_not_converged=True)
        assert r["converged"] == 0 and r["iterations"] == 3
        phi = d.fluence_host(2)
        assert np.all(np.isfinite(phi)) and phi.max() > 0
        d.dose_host(p.k_dep)                                  # results kept
        d.close()
        d = dp(p, tol=1e-6, max_iters=300, device_loop=device_loop, sweep_kernel=kernel, angles_per_block=3)
        assert d.solve()["converged"] == 1
        assert max_rel(d.fluence_host(2), ref.phi) <= REL_TOL
        d.close()


@pytest.mark.parametrize("kernel", [4, 7])
def test_dataflow_wait_times_out_and_recovers(dp, kernel):
    """The dataflow sweep's waits are bounded: with one task withholding the
    faces it owes (test hook), the downstream waits give up (in the column
    threads of kernel 4, in the face warp of kernel 7), the solve returns
    DOCTORS_ERR_TIMEOUT, and after the hook is cleared the same problem
    solves to the oracle again."""
    import time
    from paper_1811_12391_gb300 import _lib as C
    p = ph.tiny_cube(n=8)
    ref = osv.solve(p, tol=1e-11)
    d = dp(p, tol=1e-6, max_iters=3, tile=(4, 4), sweep_kernel=kernel, angles_per_block=3)
    C.check(C.doctors_debug_withhold_faces(d.h, 0))
    t0 = time.time()
    with pytest.raises(C.DoctorsError) as e:
        d.solve(allow_not_converged=True)
    assert e.value.code == C.DOCTORS_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    C.check(C.doctors_debug_withhold_faces(d.h, -1))
    d.close()
    d = dp(p, tol=1e-6, max_iters=300, tile=(4, 4), sweep_kernel=kernel, angles_per_block=3)
    C.check(C.doctors_debug_withhold_faces(d.h, 5))
    with pytest.raises(C.DoctorsError):
        d.solve(allow_not_converged=True)
    C.check(C.doctors_debug_withhold_faces(d.h, -1))
    r = d.solve()
    assert r["converged"] == 1
    assert max_rel(d.fluence_host(2), ref.phi) <= REL_TOL
    d.close()
    q = dp(p, tol=1e-6, max_iters=10, sweep_kernel=3, angles_per_block=3)
    with pytest.raises(C.DoctorsError) as e:
        C.check(C.doctors_debug_withhold_faces(q.h, 0))
    assert e.value.code == C.DOCTORS_ERR_STATE
    q.close()


@pytest.mark.parametrize("name", ["paper_water_coarse_sp", "paper_water_coarse_ct"])
def test_paper_coarse_water_runs(dp, name):
    """The paper's coarse 64x64x16 water runs (S6 P0, 7 groups; one isotropic
    point source, or 16 cone beams of 30 degrees) against the FP64 oracle."""
    p = ph.config_problem(name)
    sol = osv.solve(p, tol=1e-10)
    d = dp(p, tol=1e-6, max_iters=500)
    _compare(d, p, sol, name)
    d.close()


def test_air_dose_zeroing(dp):
    """Setting the air row of the conversion table to zero (the paper's remedy
    for ray effects in air, Sec. IV) zeroes the dose in air voxels and leaves
    every other voxel's dose unchanged."""
    p = ph.water_cylinder(nx=24, ny=24, nz=8, dx=1.5, dy=1.5, dz=2.0, diameter=30.0, G=4, sn=4, L=1)
    d = dp(p, tol=1e-6, max_iters=300)
    d.solve()
    full = d.dose_host(p.k_dep)
    k = p.k_dep.copy()
    k[0] = 0.0                                   # material 0 is air
    zeroed = d.dose_host(k)
    air = p.mat == 0
    assert np.all(zeroed[air] == 0.0) and np.any(full[air] > 0.0)
    assert np.array_equal(zeroed[~air], full[~air])
    d.close()


def test_water_cylinder_full_size_properties(dp):
    """The 64x64x32 S8 P3 19-group cylinder at full size: converged,
    particle balance, and mirror symmetry in x and z of the collided and
    total fluence (source on the -y axis at the axial centre)."""
    p = ph.water_cylinder()
    d = dp(p, tol=1e-6, max_iters=500)
    r = d.solve()
    assert r["converged"] == 1 and r["balance_rel"] < 1e-5
    for which in (1, 2):
        a = d.fluence_host(which).reshape(p.G, p.nz, p.ny, p.nx).astype(np.float64)
        for g in range(p.G):
            m = np.abs(a[g]).max()
            sel = np.abs(a[g]) > 1e-6 * m
            for flip in (a[g][:, :, ::-1], a[g][::-1, :, :]):
                assert (np.abs(a[g] - flip)[sel] / np.abs(a[g])[sel]).max() < 2e-4
    d.close()


@pytest.mark.parametrize("name", ["water_cylinder", "abdomen"])
def test_full_size_against_stored_oracle_samples(dp, name):
    """Full-size workloads in the configuration the benchmark times: the
    fluences and dose at 600 seeded voxels, and every group's fluence summed
    over the mesh, against FP64 oracle values stored by
    tests/golden/make_full_size_samples.py."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"{name}_samples.npz")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    ref = np.load(path)
    p = ph.config_problem(name)
    d = dp(p, tol=1e-6, max_iters=500)
    d.autotune()
    r = d.solve()
    assert r["converged"] == 1
    idx = ref["voxels"]
    phi = d.fluence_host(2)
    assert max_rel(d.fluence_host(0)[:, idx], ref["phi_u"]) <= REL_TOL
    assert max_rel(d.fluence_host(1)[:, idx], ref["phi_c"]) <= REL_TOL
    assert max_rel(phi[:, idx], ref["phi"]) <= REL_TOL
    assert max_rel(d.dose_host(p.k_dep)[idx], ref["dose"]) <= REL_TOL
    np.testing.assert_allclose(phi.astype(np.float64).sum(axis=1), ref["phi_total"], rtol=REL_TOL)
    d.close()
