"""doctors_dose_noalloc: the dose tally for callers that cannot call
cudaMalloc (for example code inside a framework whose caching allocator owns
the device memory, or real-time callers that forbid allocation after
start-up).  Its output must match doctors_dose on two calls in a row, with
different factor tables, and it must reject tables larger than its fixed
array.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

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


def _noalloc(C, torch, d, k):
    out = torch.full((d.V,), float("nan"), dtype=torch.float64, device="cuda")
    kk = np.ascontiguousarray(k, np.float64)
    C.check(C.doctors_dose_noalloc(d.h, kk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.c_void_p(out.data_ptr())))
    d.stream.synchronize()
    return out.cpu().numpy()


def test_matches_doctors_dose_twice(env):
    torch, C, DoctorsProblem = env
    p = ph.water_cylinder(nx=24, ny=20, nz=8, dx=1.5, dy=1.5, dz=1.5, diameter=28.0, G=5, sn=4, L=1)
    d = DoctorsProblem(p, tol=1e-6, max_iters=300)
    d.solve()
    rng = np.random.default_rng(4)
    for k in (p.k_dep, p.k_dep * rng.uniform(0.5, 2.0, size=p.k_dep.shape)):
        ref = d.dose(k).cpu().numpy()
        got = _noalloc(C, torch, d, k)
        assert np.all(np.isfinite(got))
        assert max_rel(got, ref) <= REL_TOL
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
    kk = np.ones(nmat * G)
    out = torch.zeros(p.V, dtype=torch.float64, device="cuda")
    rc = C.doctors_dose_noalloc(d.h, kk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.c_void_p(out.data_ptr()))
    assert rc == C.DOCTORS_ERR_INVALID_ARG
    assert "exceeds" in C.last_error()
    d.close()
