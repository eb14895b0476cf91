"""Host-side helpers of bench.py: the ray-trace work count reported for the
abdomen (1 + grid planes crossed per ray) against the oracle's Siddon lists."""
import importlib.util
import os

import numpy as np

from oracle import transport as tr
from synth import phantoms as ph


def _bench():
    path = os.path.join(os.path.dirname(__file__), "..", "bench.py")
    spec = importlib.util.spec_from_file_location("bench_module", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_ray_visits_bounds_the_siddon_lists():
    """The count is an upper bound within a few per cent: a ray that crosses
    two planes at once (a tie) visits one voxel fewer than it counts."""
    b = _bench()
    p = ph.abdomen(nx=24, ny=20, nz=6, d=1.3, dz=2.0, G=2, sn=4, L=0)
    s = p.sources[0]
    total = 0
    for v in range(p.V):
        k, j, i = v // (p.nx * p.ny), (v // p.nx) % p.ny, v % p.nx
        idx, _ = tr.siddon_f64(np.asarray(s.pos, float), (i, j, k), (p.nx, p.ny, p.nz),
                               np.asarray(p.origin, float), (p.dx, p.dy, p.dz))
        total += len(idx)
    est = b.ray_visits(p, s)
    assert total <= est <= 1.04 * total, (total, est)
