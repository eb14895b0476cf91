"""Gradients at full size: the differentiable abdomen (128 x 128 x 48 voxels of
0.25 cm, S8, P3, 19 groups, 32 axial views), J = mean dose over the 4 cm liver
region of interest.  The GPU's J and its gradients with respect to the 32
view weights, the 19 spectrum weights and the voxel densities against FP64
oracle values stored by tests/golden/make_gradient_samples.py (the density
gradient at 6087 voxels: a seeded sample, the 200 largest and every ROI
voxel)."""
import os

import numpy as np
import pytest

from synth import phantoms as ph
from tests.parity import DENSITY_GRAD_TOL, REL_TOL, max_rel

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "differentiable_abdomen_gradients.npz")


def test_differentiable_abdomen_gradients_against_oracle():
    from paper_1811_12391_gb300.build import build
    build()
    import torch
    from paper_1811_12391_gb300.solver import DoctorsProblem
    ref = np.load(GOLD)
    p = ph.config_problem("differentiable_abdomen")
    roi = p.roi.astype(np.float64)
    roi /= roi.sum()
    d = DoctorsProblem(p, tol=1e-6, max_iters=500)
    assert d.solve()["converged"] == 1
    g = d.roi_gradients(p.k_dep, torch.as_tensor(roi, device="cuda"))
    assert g["result"]["converged"] == 1
    assert abs(g["J"] / float(ref["J"]) - 1.0) <= REL_TOL
    assert max_rel(g["weights"].cpu().numpy(), ref["d_weights"]) <= REL_TOL
    assert max_rel(g["spectrum"].cpu().numpy(), ref["d_spectrum"]) <= REL_TOL
    idx = ref["voxels"]
    got = g["density"].cpu().numpy()[idx]
    want = ref["d_density"]
    top = float(ref["d_density_max"])
    err = np.abs(got - want) / np.abs(want)
    assert err[np.abs(want) > 1e-4 * top].max() <= REL_TOL
    assert err[np.abs(want) > 1e-6 * top].max() <= DENSITY_GRAD_TOL
    d.close()
