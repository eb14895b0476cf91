"""CT numbers -> materials and densities (Sec. II.B).

Test infrastructure only (see the package docstring).  The paper reads a
reconstructed CT image and converts its numbers into dosimetrically
equivalent materials by a stoichiometric calibration that it cites but does
not print.  This restates the piecewise form the library applies, step by
step, in plain FP32 numpy (each operation rounded to nearest, no fused
multiply-add), so that the comparison with the kernel is bit for bit:

  material: bin b = number of thresholds t_i with t_i <= hu (NaN: 0),
            material = bin_material[b];
  density:  k = number of knots with hu_knots[j] <= hu;
            k = 0 (below the first knot, or NaN): rho_knots[0];
            k = n_knots (at or beyond the last): rho_knots[-1];
            else s = k - 1 and
            t = (hu - hu_knots[s]) / (hu_knots[s+1] - hu_knots[s]),
            rho = rho_knots[s] + t * (rho_knots[s+1] - rho_knots[s]).
"""
from __future__ import annotations

import numpy as np


def ct_to_materials(hu, thresholds, bin_material, hu_knots, rho_knots):
    """Returns (material uint8 [n], density float32 [n]).  Array form of the
    steps above: every arithmetic operation is one float32 numpy operation."""
    h = np.asarray(hu, np.float32).ravel()
    t = np.asarray(thresholds, np.float32).ravel()
    bm = np.asarray(bin_material, np.uint8).ravel()
    hk = np.asarray(hu_knots, np.float32).ravel()
    rk = np.asarray(rho_knots, np.float32).ravel()
    # comparisons with NaN are false: NaN counts no threshold and no knot
    b = (t[None, :] <= h[:, None]).sum(axis=1) if t.size else np.zeros(h.size, np.int64)
    mat = bm[b]
    k = (hk[None, :] <= h[:, None]).sum(axis=1)
    if hk.size == 1:
        return mat, np.full(h.size, rk[0], np.float32)
    s = np.clip(k - 1, 0, hk.size - 2)
    with np.errstate(invalid="ignore", over="ignore"):
        num = h - hk[s]
        den = hk[s + 1] - hk[s]
        frac = num / den
        mid = rk[s] + frac * (rk[s + 1] - rk[s])
    rho = np.where(k == 0, rk[0], np.where(k == hk.size, rk[-1], mid)).astype(np.float32)
    return mat, rho
