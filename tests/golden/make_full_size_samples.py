"""Write sampled FP64 oracle results of a full-size workload to
tests/golden/<workload>_samples.npz for the full-size GPU parity tests.

Calls only the oracle (and the seeded input generator).  Usage:
    python tests/golden/make_full_size_samples.py water_cylinder [n_samples]
Stored: the seed-fixed voxel sample, phi_u, phi_c and phi at those voxels for
every group, the dose there, and per-group totals of phi over the mesh.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import solver as osv  # noqa: E402
from synth import phantoms as ph  # noqa: E402


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "water_cylinder"
    n = int(sys.argv[2]) if len(sys.argv) > 2 else 600
    p = ph.config_problem(name)
    t0 = time.time()
    sol = osv.solve(p, tol=1e-10)
    el = time.time() - t0
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(p.V, size=n, replace=False))
    dose = osv.dose(p, sol.phi)
    np.savez_compressed(os.path.join(HERE, f"{name}_samples.npz"), voxels=idx,
                        phi_u=sol.phi_u[:, idx], phi_c=sol.phi_c[:, 0, idx], phi=sol.phi[:, idx],
                        dose=dose[idx], phi_total=sol.phi.sum(axis=1), dose_total=dose.sum(),
                        iters=np.array(sol.iters), tol=1e-10, seconds=el)
    print(f"{name}: oracle solve {el:.1f} s, iterations per group {sol.iters}")


if __name__ == "__main__":
    main()
