"""Ray-trace parity: voxel index lists bit-exact against the oracle's FP32
walk, uncollided fluence within the FP32 tolerance of the oracle's FP64
value (Sec. II.A), on the tiny cube, the water cylinder and the abdomen at
full size."""
import numpy as np
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


CASES = {
    "tiny_cube": lambda: ph.tiny_cube(),
    "water_cylinder": lambda: ph.water_cylinder(),
    "abdomen": lambda: ph.abdomen(),
}


@pytest.mark.parametrize("name", list(CASES))
def test_index_lists_bit_exact(dp, name):
    p = CASES[name]()
    d = dp(p, max_iters=1)
    rng = np.random.default_rng(11)
    vox = list(rng.choice(p.V, size=400, replace=False)) + [0, p.V - 1, p.nx - 1, p.V // 2]
    src = p.sources[0]
    for v in vox:
        v = int(v)
        ijk = (v % p.nx, (v // p.nx) % p.ny, v // (p.nx * p.ny))
        gi, gl = d.ray_indices(0, v)
        oi, ol = tr.siddon_f32(src.pos, ijk, (p.nx, p.ny, p.nz), p.origin, (p.dx, p.dy, p.dz))
        assert np.array_equal(gi, oi), (name, v)
        assert np.array_equal(gl, ol), (name, v)
    d.close()


def test_diagonal_ties_bit_exact(dp):
    p = ph.tiny_cube(n=4)
    p.origin = np.zeros(3)
    p.sources[0].pos = np.array([-10.0, -10.0, 0.5])
    d = dp(p, max_iters=1)
    v = (0 * 4 + 3) * 4 + 3
    gi, gl = d.ray_indices(0, v)
    assert list(gi) == [15, 10, 5, 0]
    oi, ol = tr.siddon_f32(p.sources[0].pos, (3, 3, 0), (4, 4, 4), p.origin, (1, 1, 1))
    assert np.array_equal(gi, oi) and np.array_equal(gl, ol)
    d.close()


@pytest.mark.parametrize("name", list(CASES))
def test_uncollided_fluence_parity(dp, name):
    p = CASES[name]()
    d = dp(p, max_iters=1)
    d.solve(allow_not_converged=True)
    gpu = d.fluence_host(0)
    ref = osv.uncollided(p, p.sources[0])
    assert max_rel(gpu, ref) <= REL_TOL
    # voxels outside the collimated beam stay exactly dark
    assert np.all(gpu[ref == 0] == 0)
    assert np.all(gpu[ref > 1e-20 * ref.max()] > 0)
    d.close()
