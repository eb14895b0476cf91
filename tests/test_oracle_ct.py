"""Pins of the oracle's CT-number -> material and density conversion
(Sec. II.B) against its definition's fixed points, a library interpolation
and a round trip through the synthetic CT of the abdomen phantom."""
import numpy as np

from oracle import ct
from synth import phantoms as ph


def test_round_trip_recovers_the_abdomen_materials():
    """Every synthetic CT number lies inside its material's bin, so the
    conversion returns the phantom's material map exactly."""
    p = ph.abdomen(nx=64, ny=64, nz=4, d=0.5, dz=1.0, G=2, sn=4, L=0)
    cal = ph.ct_calibration()
    hu = ph.synthetic_ct(p)
    mat, rho = ct.ct_to_materials(hu, cal["thresholds"], cal["bin_material"], cal["hu_knots"], cal["rho_knots"])
    np.testing.assert_array_equal(mat, p.mat)
    assert rho.dtype == np.float32 and np.all(rho > 0)


def test_density_matches_library_interpolation():
    """Inside the knot range the density is numpy's piecewise-linear
    interpolation (FP64) to FP32 rounding; outside it is the end value."""
    cal = ph.ct_calibration()
    rng = np.random.default_rng(4)
    hu = rng.uniform(-1200.0, 1300.0, size=20000).astype(np.float32)
    _, rho = ct.ct_to_materials(hu, cal["thresholds"], cal["bin_material"], cal["hu_knots"], cal["rho_knots"])
    ref = np.interp(hu.astype(np.float64), cal["hu_knots"].astype(np.float64), cal["rho_knots"].astype(np.float64))
    assert np.abs(rho - ref).max() <= 4e-7 * np.abs(ref).max()


def test_knots_and_ends_are_exact():
    cal = ph.ct_calibration()
    hk, rk = cal["hu_knots"], cal["rho_knots"]
    _, rho = ct.ct_to_materials(hk, cal["thresholds"], cal["bin_material"], hk, rk)
    np.testing.assert_array_equal(rho, rk)
    _, r2 = ct.ct_to_materials(np.array([-5000.0, 5000.0, np.inf, -np.inf], np.float32), cal["thresholds"],
                               cal["bin_material"], hk, rk)
    np.testing.assert_array_equal(r2, np.array([rk[0], rk[-1], rk[-1], rk[0]], np.float32))


def test_threshold_boundaries_and_nan():
    """A number equal to a threshold falls in the upper bin, the next float
    below it in the lower one; NaN gives bin 0 and the first knot's density."""
    cal = ph.ct_calibration()
    t = cal["thresholds"]
    below = np.nextafter(t, np.float32(-np.inf)).astype(np.float32)
    hu = np.concatenate([t, below, np.array([np.nan], np.float32)])
    mat, rho = ct.ct_to_materials(hu, t, cal["bin_material"], cal["hu_knots"], cal["rho_knots"])
    nb = t.size
    np.testing.assert_array_equal(mat[:nb], cal["bin_material"][1:])
    np.testing.assert_array_equal(mat[nb:2 * nb], cal["bin_material"][:-1])
    assert mat[-1] == cal["bin_material"][0] and rho[-1] == cal["rho_knots"][0]


def test_one_knot_and_no_thresholds():
    mat, rho = ct.ct_to_materials(np.array([-3.0, 0.0, 7.0], np.float32), [], [4], [0.0], [1.25])
    np.testing.assert_array_equal(mat, [4, 4, 4])
    np.testing.assert_array_equal(rho, np.float32([1.25, 1.25, 1.25]))
