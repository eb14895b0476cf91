"""doctors_dose_noalloc: the dose tally for callers that cannot call
cudaMalloc (for example code inside a framework whose caching allocator owns
the device memory, or real-time callers that forbid allocation after
start-up).  Its output must match doctors_dose bit for bit on two calls in a
row with factor tables that differ in every entry (a stale entry of the
shared array would show), agree with the oracle's dose, reject tables larger
than its fixed array, and reject bad calls without writing anything.  This
file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

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
    import torch
    from paper_1811_12391_gb300 import _lib as C
    from paper_1811_12391_gb300.solver import DoctorsProblem
    return torch, C, DoctorsProblem


def _call(C, d, k, out):
    kk = np.ascontiguousarray(k, np.float64)
    return C.doctors_dose_noalloc(d.h, kk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(out.data_ptr()) if out is not None else None)


def _noalloc(C, torch, d, k):
    out = torch.full((d.V,), float("nan"), dtype=torch.float64, device="cuda")
    C.check(_call(C, d, k, out))
    d.stream.synchronize()
    return out.cpu().numpy()


def test_matches_doctors_dose_twice(env):
    torch, C, DoctorsProblem = env
    p = ph.water_cylinder(nx=24, ny=20, nz=8, dx=1.5, dy=1.5, dz=1.5, diameter=28.0, G=5, sn=4, L=1)
    d = DoctorsProblem(p, tol=1e-6, max_iters=300)
    d.solve()
    ref_sol = osv.solve(p, tol=1e-11)
    rng = np.random.default_rng(4)
    for k in (p.k_dep, p.k_dep * rng.uniform(0.5, 2.0, size=p.k_dep.shape)):
        ref = d.dose(k).cpu().numpy()
        got = _noalloc(C, torch, d, k)
        assert np.array_equal(got, ref)          # the same kernel on the same factors
        assert max_rel(got, osv.dose(p, ref_sol.phi, k)) <= REL_TOL
    d.close()


def test_rejects_tables_beyond_the_fixed_array(env):
    torch, C, DoctorsProblem = env
    p = ph.tiny_cube(n=2)
    G = 40
    nmat = 8
    p.sigma_t = np.full((nmat, G), 0.3)
    p.sigma_s = np.zeros((nmat, 2, G, G))
    p.sources[0].spectrum = np.full(G, 1.0 / G)
    p.k_dep = np.ones((nmat, G))
    d = DoctorsProblem(p, tol=1e-6, max_iters=5)
    out = torch.zeros(p.V, dtype=torch.float64, device="cuda")
    rc = _call(C, d, np.ones(nmat * G), out)
    assert rc == C.DOCTORS_ERR_INVALID_ARG
    assert "exceeds" in C.last_error()
    d.close()


def test_bad_calls_write_nothing(env):
    """Before a solve, a null table or output, and a non-finite factor are
    rejected with their codes and leave the output untouched."""
    torch, C, DoctorsProblem = env
    p = ph.tiny_cube(n=4)
    d = DoctorsProblem(p, tol=1e-6, max_iters=200)
    out = torch.full((p.V,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(C, d, p.k_dep, out) == C.DOCTORS_ERR_STATE
    d.solve()
    kk = np.ascontiguousarray(p.k_dep, np.float64)
    assert C.doctors_dose_noalloc(d.h, None, ctypes.c_void_p(out.data_ptr())) == C.DOCTORS_ERR_INVALID_ARG
    assert _call(C, d, p.k_dep, None) == C.DOCTORS_ERR_INVALID_ARG
    bad = kk.copy()
    bad[0, 0] = np.nan
    assert _call(C, d, bad, out) == C.DOCTORS_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.isnan(out).all().item()
    d.close()
