"""Level-symmetric S_N quadrature and real spherical harmonics (FP64).

Test infrastructure only (see the package docstring).

Sec. II.A, Eq. 3 and Sec. II.D: the scalar fluence is the weighted sum of the
angular fluence over N(N+2) discrete directions (S2/S4/S6/S8 = 8/24/48/80).
The paper does not print the directions or weights.  Reading: the standard
level-symmetric LQ_N set.  In each octant the direction cosines take values
from N/2 levels mu_i with mu_i^2 = mu_1^2 + (i-1) * 2(1 - 3 mu_1^2)/(N-2);
the directions are the index triples (a, b, c) with a + b + c = N/2 + 2; the
point weights depend only on the permutation class of the triple and are the
unique solution of the even-moment conditions (exact integration of every
even monomial x^2i y^2j z^2k of total degree <= N-2 over the octant).  The
weights sum to 4 pi, so Eq. 3's sum is the scalar fluence.

Eq. 2 expresses the scattering kernel as a Legendre expansion; through the
addition theorem that becomes a sum over real spherical harmonics R_lm,
semi-normalised so that sum_m R_lm(a) R_lm(b) = P_l(a . b).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import special

# mu_1 of the usual LQ_N sets (the paper uses S2..S8; S16 is used for the
# abdomen workload).  mu_1 is a free parameter of the construction; the
# moment conditions below fix the weights for any mu_1.
MU1 = {2: 0.5773503, 4: 0.3500212, 6: 0.2666355, 8: 0.2182179,
       12: 0.1672126, 16: 0.1389568}


def octant_integral(i: int, j: int, k: int) -> float:
    """Exact integral of x^2i y^2j z^2k over one octant of the unit sphere."""
    g = math.gamma
    return 2.0 * g(i + 0.5) * g(j + 0.5) * g(k + 0.5) / g(i + j + k + 1.5) / 8.0


def levels(N: int) -> np.ndarray:
    """The N/2 direction-cosine levels mu_1 < ... < mu_{N/2}."""
    n = N // 2
    mu1 = MU1[N]
    if N == 2:
        return np.array([math.sqrt(1.0 / 3.0)])   # the only unit (mu, mu, mu)
    c = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2)
    return np.sqrt(mu1 * mu1 + c * np.arange(n))


def octant_points(N: int):
    """Index triples (a, b, c), 1-based, with a + b + c = N/2 + 2."""
    n = N // 2
    return [(a, b, c) for a in range(1, n + 1) for b in range(1, n + 1)
            for c in range(1, n + 1) if a + b + c == n + 2]


def class_weights(N: int):
    """Solve the even-moment conditions for the per-class weights.

    Returns (points, classes, weights_per_class, max_residual)."""
    mu = levels(N)
    pts = octant_points(N)
    classes = sorted(set(tuple(sorted(p)) for p in pts))
    rows, rhs = [], []
    for deg in range(0, N - 1, 2):
        h = deg // 2
        for i in range(h + 1):
            for j in range(h + 1 - i):
                k = h - i - j
                row = np.zeros(len(classes))
                for p in pts:
                    x, y, z = mu[p[0] - 1], mu[p[1] - 1], mu[p[2] - 1]
                    row[classes.index(tuple(sorted(p)))] += x ** (2 * i) * y ** (2 * j) * z ** (2 * k)
                rows.append(row)
                rhs.append(octant_integral(i, j, k))
    A = np.array(rows)
    b = np.array(rhs)
    w, *_ = np.linalg.lstsq(A, b, rcond=None)
    return pts, classes, w, float(np.abs(A @ w - b).max())


def level_symmetric(N: int):
    """Directions [N(N+2), 3] and weights [N(N+2)] of LQ_N, octant-major.

    Octant o has signs (-1 if o & 1 else +1, -1 if o & 2 else +1,
    -1 if o & 4 else +1) on (x, y, z)."""
    if N not in MU1:
        raise ValueError(f"no level-symmetric set for N={N}")
    mu = levels(N)
    pts, classes, w, resid = class_weights(N)
    if resid > 1e-12:
        raise ValueError(f"LQ_{N}: moment conditions inconsistent ({resid:g})")
    if np.any(w <= 0):
        raise ValueError(f"LQ_{N}: non-positive weight")
    dirs, wts = [], []
    for o in range(8):
        sgn = np.array([-1.0 if o & 1 else 1.0, -1.0 if o & 2 else 1.0, -1.0 if o & 4 else 1.0])
        for p in pts:
            dirs.append(sgn * np.array([mu[p[0] - 1], mu[p[1] - 1], mu[p[2] - 1]]))
            wts.append(w[classes.index(tuple(sorted(p)))])
    return np.array(dirs), np.array(wts)


def n_moments(L: int) -> int:
    return (L + 1) ** 2


def moment_index(l: int, m: int) -> int:
    """Flat index of (l, m), m = -l..l."""
    return l * l + l + m


def moment_degrees(L: int) -> np.ndarray:
    """Legendre order l of every flat moment index."""
    return np.array([l for l in range(L + 1) for _ in range(2 * l + 1)])


def real_harmonics(L: int, dirs: np.ndarray) -> np.ndarray:
    """R_lm(Omega) for l <= L, shape [n, (L+1)^2].

    mu = Omega_z, phi = atan2(Omega_y, Omega_x);
    R_l0 = P_l(mu); R_lm = sqrt(2 (l-m)!/(l+m)!) P_l^m(mu) cos(m phi) for m > 0
    and the same with sin(|m| phi) for m < 0."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    mu = dirs[:, 2]
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    out = np.zeros((dirs.shape[0], n_moments(L)))
    for l in range(L + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            plm = special.lpmv(am, l, mu)
            if m == 0:
                val = plm
            else:
                norm = math.sqrt(2.0 * math.factorial(l - am) / math.factorial(l + am))
                val = norm * plm * (np.cos(am * phi) if m > 0 else np.sin(am * phi))
            out[:, moment_index(l, m)] = val
    return out


def angular_operators(N: int, L: int):
    """Quadrature plus the moment<->direction maps of the sweep.

    Returns (dirs, w, R, Mop, Dop):
      R[n, lm]   = R_lm(Omega_n)
      Mop[n, lm] = (2l+1)/(4 pi) R_lm(Omega_n)   (moments -> angular source)
      Dop[n, lm] = w_n R_lm(Omega_n)             (angular -> moments, Eq. 3 for l=0)"""
    dirs, w = level_symmetric(N)
    R = real_harmonics(L, dirs)
    ls = moment_degrees(L)
    Mop = R * ((2 * ls + 1) / (4.0 * math.pi))[None, :]
    Dop = R * w[:, None]
    return dirs, w, R, Mop, Dop
