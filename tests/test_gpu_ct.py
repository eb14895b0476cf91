"""Parity of the CT-number conversion kernel (doctors_ct_to_materials,
Sec. II.B) with the oracle: materials and densities bit for bit, host and
device memory, ragged sizes and special values; and a solve of a phantom
built from its synthetic CT against the oracle.  (The table checks, made
before any device work, are in test_abi.py.)"""
import numpy as np
import pytest

from oracle import ct as oct_
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
    from paper_1811_12391_gb300 import solver as S
    return torch, C, S


def _cal_args(cal):
    return cal["thresholds"], cal["bin_material"], cal["hu_knots"], cal["rho_knots"]


def test_full_size_abdomen_ct_bit_exact(env):
    """The 128x128x48 abdomen's synthetic CT (786 432 voxels), device memory."""
    torch, C, S = env
    p = ph.abdomen()
    cal = ph.ct_calibration()
    hu = ph.synthetic_ct(p)
    m_ref, r_ref = oct_.ct_to_materials(hu, *_cal_args(cal))
    mat, rho = S.ct_to_materials(torch.as_tensor(hu, device="cuda"), *_cal_args(cal))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(mat.cpu().numpy(), m_ref)
    np.testing.assert_array_equal(rho.cpu().numpy().view(np.uint32), r_ref.view(np.uint32))
    np.testing.assert_array_equal(m_ref, p.mat)


@pytest.mark.parametrize("n", [1, 31, 255, 257, 100003])
def test_ragged_sizes_and_special_values_host_memory(env, n):
    torch, C, S = env
    cal = ph.ct_calibration()
    rng = np.random.default_rng(n)
    hu = rng.uniform(-1500.0, 1500.0, size=n).astype(np.float32)
    # thresholds, knots, their float neighbours and non-finite values
    special = np.concatenate([cal["thresholds"], cal["hu_knots"],
                              np.nextafter(cal["thresholds"], np.float32(-np.inf)),
                              np.array([np.nan, np.inf, -np.inf, 0.0, -0.0], np.float32)]).astype(np.float32)
    k = min(n, special.size)
    hu[:k] = special[:k]
    m_ref, r_ref = oct_.ct_to_materials(hu, *_cal_args(cal))
    mat, rho = S.ct_to_materials(hu, *_cal_args(cal))
    np.testing.assert_array_equal(mat, m_ref)
    np.testing.assert_array_equal(rho.view(np.uint32), r_ref.view(np.uint32))


def test_one_knot_no_thresholds(env):
    torch, C, S = env
    hu = np.array([-3.0, 0.0, 7.0, np.nan], np.float32)
    mat, rho = S.ct_to_materials(hu, [], [4], [0.0], [1.25])
    np.testing.assert_array_equal(mat, [4, 4, 4, 4])
    np.testing.assert_array_equal(rho, np.float32([1.25] * 4))


def test_solve_from_converted_ct_matches_oracle(env):
    """A small abdomen whose materials and densities come from its synthetic
    CT through the kernel: the solve matches the oracle's solve of the same
    converted phantom."""
    torch, C, S = env
    p = ph.abdomen(nx=32, ny=32, nz=4, d=1.0, dz=2.0, G=3, sn=4, L=1)
    cal = ph.ct_calibration()
    hu = ph.synthetic_ct(p)
    mat, rho = S.ct_to_materials(torch.as_tensor(hu, device="cuda"), *_cal_args(cal))
    p.mat = mat.cpu().numpy()
    p.density = rho.cpu().numpy()
    sol = osv.solve(p, tol=1e-11)
    d = S.DoctorsProblem(p, tol=1e-6, max_iters=400)
    d.solve()
    assert max_rel(d.fluence_host(2), sol.phi) <= REL_TOL
    assert max_rel(d.dose_host(p.k_dep), osv.dose(p, sol.phi)) <= REL_TOL
    d.close()
