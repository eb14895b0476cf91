"""The paper's S_N x P_N scan (Table 2) on its coarse water workload
(64 x 64 x 16 voxels of 7.81 mm, seven groups with the paper's 10-100 keV
edges, one isotropic point source at 54 cm): the lowest and the highest
quadrature order with P0 and P1, full solves against the FP64 oracle."""
import os

import pytest

from oracle import solver as osv
from oracle import transport as tr
from synth import phantoms as ph
from tests.parity import REL_TOL, max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    from paper_1811_12391_gb300.build import build
    build()
    from paper_1811_12391_gb300.solver import DoctorsProblem
    return DoctorsProblem


@pytest.mark.parametrize("sn,L", [(2, 0), (2, 1), (8, 0), (8, 1)])
def test_paper_coarse_water_against_oracle(dp, sn, L):
    p = ph.paper_water(sn=sn, L=L)
    tr.set_threads(os.cpu_count() or 1)
    sol = osv.solve(p, tol=1e-11)
    d = dp(p, tol=1e-6, max_iters=500)
    r = d.solve()
    assert r["converged"] == 1
    errs = {"phi_u": max_rel(d.fluence_host(0), sol.phi_u),
            "phi_c": max_rel(d.fluence_host(1), sol.phi_c[:, 0, :]),
            "phi": max_rel(d.fluence_host(2), sol.phi),
            "dose": max_rel(d.dose_host(p.k_dep), osv.dose(p, sol.phi))}
    assert max(errs.values()) <= REL_TOL, errs
    assert r["balance_rel"] < 1e-5
    d.close()
