"""Pins of the oracle's quadrature and harmonics against mathematics and the
paper (Sec. II.D direction counts, Eq. 3 weights)."""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import quadrature as q

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_direction_counts_match_paper():
    for N, count in _golden("quadrature_counts.txt"):
        dirs, w = q.level_symmetric(int(N))
        assert dirs.shape == (int(count), 3)
    assert q.level_symmetric(16)[0].shape[0] == 288


@pytest.mark.parametrize("N", [2, 4, 6, 8, 16])
def test_basic_moments(N):
    dirs, w = q.level_symmetric(N)
    assert np.all(w > 0)
    np.testing.assert_allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-6)
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    np.testing.assert_allclose(w @ dirs, 0.0, atol=1e-12)
    for d in range(3):
        assert abs(w @ dirs[:, d] ** 2 - 4 * math.pi / 3) < 1e-12


@pytest.mark.parametrize("N", [4, 6, 8, 16])
def test_even_monomials_exact_up_to_degree_N_minus_2(N):
    """Every even monomial of degree <= N-2 integrates exactly (and every odd
    one to zero), compared with the closed-form sphere integral."""
    dirs, w = q.level_symmetric(N)
    for a in range(N):
        for b in range(N - a):
            for c in range(N - a - b):
                val = w @ (dirs[:, 0] ** a * dirs[:, 1] ** b * dirs[:, 2] ** c)
                if a % 2 or b % 2 or c % 2:
                    exact = 0.0
                elif a + b + c > N - 2:
                    continue
                else:
                    g = math.gamma
                    exact = 2 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)
                assert abs(val - exact) < 1e-12, (a, b, c, val, exact)


def test_closed_form_weights_S2_S4():
    """S2: one direction per octant of weight pi/2; S4: three per octant of
    weight pi/6 (one symmetry class)."""
    _, w2 = q.level_symmetric(2)
    np.testing.assert_allclose(w2, math.pi / 2, rtol=1e-14)
    _, w4 = q.level_symmetric(4)
    np.testing.assert_allclose(w4, math.pi / 6, rtol=1e-14)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_cube_symmetry_invariance(N):
    """The set is invariant under the 48 symmetries of the cube."""
    dirs, w = q.level_symmetric(N)
    key = {tuple(np.round(d, 9)): wi for d, wi in zip(dirs, w)}
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            t = dirs[:, perm] * np.array(signs)
            for d, wi in zip(t, w):
                assert abs(key[tuple(np.round(d, 9))] - wi) < 1e-12


def test_harmonics_addition_theorem():
    """sum_m R_lm(a) R_lm(b) = P_l(a . b) against scipy's Legendre P_l."""
    rng = np.random.default_rng(0)
    a = rng.normal(size=(50, 3))
    b = rng.normal(size=(50, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b /= np.linalg.norm(b, axis=1)[:, None]
    L = 4
    Ra, Rb = q.real_harmonics(L, a), q.real_harmonics(L, b)
    cos = (a * b).sum(axis=1)
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) ** 2)
        np.testing.assert_allclose((Ra[:, sl] * Rb[:, sl]).sum(axis=1), special.eval_legendre(l, cos),
                                   atol=1e-12)


def test_harmonics_orthogonality_product_gauss():
    """int R_lm R_l'm' dOmega = 4 pi/(2l+1) delta, by a 40 x 80 product rule
    (Gauss-Legendre in mu, uniform in phi) that is exact for these degrees."""
    L = 3
    x, wx = special.roots_legendre(40)
    nphi = 80
    phi = 2 * math.pi * np.arange(nphi) / nphi
    MU, PHI = np.meshgrid(x, phi, indexing="ij")
    s = np.sqrt(1 - MU ** 2)
    dirs = np.stack([s * np.cos(PHI), s * np.sin(PHI), MU], axis=-1).reshape(-1, 3)
    W = (wx[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).ravel()
    R = q.real_harmonics(L, dirs)
    G = (R * W[:, None]).T @ R
    ls = q.moment_degrees(L)
    np.testing.assert_allclose(G, np.diag(4 * math.pi / (2 * ls + 1)), atol=1e-12)


@pytest.mark.parametrize("N,L", [(4, 1), (8, 3), (16, 3)])
def test_discrete_orthogonality_of_used_sets(N, L):
    """The sets used by the workloads integrate all products R_lm R_l'm'
    (l, l' <= L) exactly: S4/P1, S8/P3, S16/P3."""
    dirs, w = q.level_symmetric(N)
    R = q.real_harmonics(L, dirs)
    G = (R * w[:, None]).T @ R
    ls = q.moment_degrees(L)
    np.testing.assert_allclose(G, np.diag(4 * math.pi / (2 * ls + 1)), atol=1e-12)


def test_first_moment_operator_is_eq3():
    """Dop row for lm = 00 is w_n (R_00 = 1): the Eq. 3 scalar fluence."""
    dirs, w, R, Mop, Dop = q.angular_operators(8, 3)
    np.testing.assert_allclose(Dop[:, 0], w)
    np.testing.assert_allclose(Mop[:, 0], 1 / (4 * math.pi))
