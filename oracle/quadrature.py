"""Angular and spatial quadrature for the CPU oracle (test infrastructure only).

Angular: the level-symmetric S_N set of the semi-discrete equations (Eq. sntransport,
Sec. 1), with the scalar flux phi = sum_d w_d psi_d and sum_d w_d = 4*pi, so that the
isotropic scattering term sigma_s/(4 pi) * sum_d w_d psi_d of Eq. (1) keeps its meaning.
In 2D only the directions with positive polar cosine are kept and their weights doubled
(the paper's "40 angles" for S8 in 2D, Sec. 4.1).

Construction (Lewis & Miller, "Computational Methods of Neutron Transport", 1984, ch. 4):
the N/2 distinct direction cosines satisfy mu_i^2 = mu_1^2 + (i-1) * 2(1 - 3 mu_1^2)/(N-2),
the points of one octant are (mu_i, mu_j, mu_k) with i + j + k = N/2 + 2 (1-based), and
points that are permutations of one another share a weight.  The weights are fixed by
requiring that one octant integrates mu_x^(2k) exactly for k = 0 and k = 2..(#classes)
(k = 1 holds automatically because every point lies on the unit sphere).

Spatial: Gauss-Legendre rules and Legendre polynomials from numpy.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as _leg

# first direction cosine of the LQ_N sets (Lewis & Miller, Table 4-1)
LS_MU1 = {4: 0.3500212, 6: 0.2666355, 8: 0.2182179}


def level_symmetric_octant(N: int):
    """Return (mu, points, weights) of one octant; weights sum to 1."""
    if N not in LS_MU1:
        raise ValueError(f"S_{N} not tabulated")
    n = N // 2
    m1 = LS_MU1[N]
    mu = np.sqrt(np.array([m1 * m1 + i * 2.0 * (1.0 - 3.0 * m1 * m1) / (N - 2) for i in range(n)]))
    pts = [(i, j, n - 1 - i - j) for i in range(n) for j in range(n - i)]
    classes = sorted({tuple(sorted(p)) for p in pts})
    ks = [0] + list(range(2, len(classes) + 1))
    A = np.zeros((len(classes), len(classes)))
    b = np.zeros(len(classes))
    for r, k in enumerate(ks):
        for p in pts:
            A[r, classes.index(tuple(sorted(p)))] += mu[p[0]] ** (2 * k)
        b[r] = 1.0 / (2 * k + 1)
    wc = np.linalg.solve(A, b)
    w = np.array([wc[classes.index(tuple(sorted(p)))] for p in pts])
    return mu, pts, w


def level_symmetric(N: int, dim: int):
    """Directions (n_dirs, 3) and weights (n_dirs,) with sum 4*pi.

    Order: octant o = 0..7 (3D) or 0..3 (2D); the x component is negative when
    bit 0 of o is set, y when bit 1 is set, z when bit 2 is set.  Inside an octant
    the points (i, j, k) run over i ascending, then j ascending.
    """
    mu, pts, w = level_symmetric_octant(N)
    n_oct = 8 if dim == 3 else 4
    dirs, wts = [], []
    for o in range(n_oct):
        s = np.array([-1.0 if (o >> a) & 1 else 1.0 for a in range(3)])
        for (i, j, k), wp in zip(pts, w):
            dirs.append(s * np.array([mu[i], mu[j], mu[k]]))
            wts.append(wp)
    wts = np.array(wts)
    wts *= 4.0 * np.pi / wts.sum()
    return np.array(dirs), wts


def gauss(npts: int):
    """Gauss-Legendre points and weights on [-1, 1]."""
    return _leg.leggauss(npts)


def legendre(m: int, x):
    """P_m(x) (standard normalisation P_m(1) = 1)."""
    c = np.zeros(m + 1)
    c[m] = 1.0
    return _leg.legval(x, c)


def dlegendre(m: int, x):
    """P_m'(x)."""
    c = np.zeros(m + 1)
    c[m] = 1.0
    return _leg.legval(x, _leg.legder(c))
