"""Batched and graph-captured solves and the autotuner: the device-side
iteration loop (one CUDA graph with a while node) gives the same results as
the oracle, a batch of uneven problems matches each problem solved alone,
and an autotuned schedule keeps parity."""
import numpy as np
import pytest

from oracle import solver as osv
from synth import phantoms as ph
from tests.parity import REL_TOL, max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1811_12391_gb300.build import build
    build()
    from paper_1811_12391_gb300 import solver
    return solver


def _cases():
    a = ph.tiny_cube(n=10)
    b = ph.water_cylinder(nx=28, ny=20, nz=8, dx=1.2, dy=1.5, dz=1.2, diameter=26.0, G=4, sn=8, L=3)
    c = ph.abdomen(nx=24, ny=20, nz=5, d=1.3, dz=2.0, G=3, sn=16, L=3)
    return [a, b, c]


@pytest.fixture(scope="module")
def refs():
    return [osv.solve(p, tol=1e-11) for p in _cases()]


def test_device_loop_matches_oracle(env, refs):
    for p, ref in zip(_cases(), refs):
        d = env.DoctorsProblem(p, tol=1e-6, max_iters=400, device_loop=1)
        r = d.solve()
        assert r["converged"] == 1 and r["balance_rel"] < 1e-5
        assert max_rel(d.fluence_host(2), ref.phi) <= REL_TOL
        assert max_rel(d.dose_host(p.k_dep), osv.dose(p, ref.phi)) <= REL_TOL
        d.close()


def test_batch_of_uneven_problems(env, refs):
    ps = _cases()
    ds = [env.DoctorsProblem(p, tol=1e-6, max_iters=400) for p in ps]
    res = env.solve_batch(ds)
    for p, d, r, ref in zip(ps, ds, res, refs):
        assert r["converged"] == 1, r
        assert max_rel(d.fluence_host(2), ref.phi) <= REL_TOL
        alone = env.DoctorsProblem(p, tol=1e-6, max_iters=400)
        ra = alone.solve()
        assert r["iterations"] == ra["iterations"]
        np.testing.assert_allclose(d.fluence_host(2), alone.fluence_host(2), rtol=2e-5, atol=0)
        alone.close()
    for d in ds:
        d.close()


def test_batch_of_views_superposes(env):
    """The views of an axial scan solved as a batch sum to the dose of the
    same views superposed in one problem (the problem is linear)."""
    base = ph.water_cylinder(nx=24, ny=24, nz=6, dx=1.5, dy=1.5, dz=1.5, diameter=30.0, G=3, sn=4, L=1)
    views = ph.axial_scan_sources(base, 4, z_width=6.0)
    ds = [env.DoctorsProblem(base.with_sources([v]), tol=1e-6, max_iters=400) for v in views]
    env.solve_batch(ds)
    summed = sum(d.dose_host(base.k_dep) for d in ds)
    sup = env.DoctorsProblem(base.with_sources(views), tol=1e-6, max_iters=400)
    sup.solve()
    assert max_rel(summed, sup.dose_host(base.k_dep)) <= 1e-4
    for d in ds + [sup]:
        d.close()


def test_autotune_keeps_parity(env, refs):
    p = _cases()[1]
    ref = refs[1]
    d = env.DoctorsProblem(p, tol=1e-6, max_iters=400)
    t = d.autotune()
    assert t["candidates"] > 1 and t["ms_per_sweep"] > 0
    assert t["tile_x"] * t["tile_y"] <= 256
    d.solve()
    assert max_rel(d.fluence_host(2), ref.phi) <= REL_TOL
    d2 = env.DoctorsProblem(p, tol=1e-6, max_iters=400)
    t2 = d2.autotune()
    assert t2["candidates"] == 0 and (t2["tile_x"], t2["tile_y"]) == (t["tile_x"], t["tile_y"])
    d.close()
    d2.close()
