"""Write FP64 oracle gradients of the differentiable abdomen to
tests/golden/differentiable_abdomen_gradients.npz for the full-size GPU
gradient test.

The workload: the 128x128x48 abdomen (0.25 cm voxels), S8, P3, 19 groups, 32
axial views; J = mean dose over the 4 cm liver region of interest.  Calls
only the oracle (and the seeded input generator).  Usage:
    python tests/golden/make_gradient_samples.py [n_samples]
Stored: J, dJ/d view weight [32], dJ/d spectrum [19], the largest |dJ/d
density| over the mesh, and dJ/d density at a seed-fixed voxel sample, at
the 200 voxels of largest |dJ/d density| and at every ROI voxel.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import solver as osv  # noqa: E402
from oracle import transport as tr  # noqa: E402
from synth import phantoms as ph  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 2000
    p = ph.config_problem("differentiable_abdomen")
    roi = p.roi.astype(np.float64)
    roi /= roi.sum()
    t0 = time.time()
    g = osv.gradients(p, roi, tol=1e-10)
    el = time.time() - t0
    dd = g["d_density"]
    rng = np.random.default_rng(54321)
    sample = rng.choice(p.V, size=n, replace=False)
    top = np.argsort(-np.abs(dd))[:200]
    idx = np.unique(np.concatenate([sample, top, np.flatnonzero(p.roi)]))
    np.savez_compressed(os.path.join(HERE, "differentiable_abdomen_gradients.npz"),
                        J=g["J"], d_weights=g["d_weights"], d_spectrum=g["d_spectrum"],
                        d_density_max=np.abs(dd).max(), voxels=idx, d_density=dd[idx],
                        iters=np.array(g["forward"].iters), adjoint_iters=np.array(g["adjoint"].iters),
                        tol=1e-10, seconds=el, threads=tr.threads())
    print(f"differentiable_abdomen: oracle gradients {el:.1f} s on {tr.threads()} threads; "
          f"forward iterations {g['forward'].iters}")


if __name__ == "__main__":
    main()
