"""Seeded synthetic workloads for the heterogeneous-DSA transport path.

This module only produces inputs: vertex coordinates, per-element cross
sections, sources and masks.  It holds none of the method's arithmetic
(no quadrature, no DG matrices, no sweep) so that both the CPU oracle and
the CUDA library can consume the same arrays without sharing solver code.

Randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in its counter form:
output k of a stream with seed s is mix64(s + (k + 1) * GAMMA).

The workloads stand in for the paper's heterogeneous benchmarks (the crooked
pipe of Sec. 4.1 / Table 1 and the hohlraum of Sec. 4.2, whose geometries are
not available): thick, thin and void regions, scattering ratios close to one
and cross sections spread over several decades.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASTER_SEED = 2001_09196


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(master: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(master % (1 << 64)) + np.uint64(stream) * GAMMA
    return _mix64(np.array([s], dtype=np.uint64))[0]


def uniform(master: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream `stream` of seed `master`."""
    s = stream_seed(master, stream)
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(s + k * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Problem:
    """One transport problem on a structured mesh of the unit square/cube.

    Arrays are per element, elements numbered lexicographically with x fastest.
    `vertices` is None for a uniform grid, else ((ny+1)*(nx+1), 2) with x fastest.
    """

    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    p: int
    sn: int
    sigma_t: np.ndarray
    sigma_s: np.ndarray
    q: np.ndarray
    vertices: Optional[np.ndarray] = None
    psi_inc: float = 0.0
    thick_rule: str = "sigma_s"          # "sigma_s" (sigma_s >= eta) | "sigma_t_h" (sigma_t*h > eta)
    eta: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def n_nodes(self) -> int:
        return (self.p + 1) ** self.dim

    @property
    def n_dirs(self) -> int:
        return self.sn * (self.sn + 2) // (2 if self.dim == 2 else 1)


def _centroids_uniform(nx, ny):
    i = np.arange(nx)
    j = np.arange(ny)
    xc = (i + 0.5) / nx
    yc = (j + 0.5) / ny
    X, Y = np.meshgrid(xc, yc, indexing="xy")  # shape (ny, nx), x fastest when raveled
    return X.ravel(), Y.ravel()


def _in(a, lo, hi):
    return (a >= lo) & (a < hi)


def config1() -> Problem:
    """16x16 Q1 S4, background sigma_t=1/sigma_s=0.9, a thick block, a void block and a source block."""
    nx = ny = 16
    xc, yc = _centroids_uniform(nx, ny)
    st = np.ones(nx * ny)
    ss = np.full(nx * ny, 0.9)
    thick = _in(xc, 0.25, 0.5) & _in(yc, 0.25, 0.5)
    void = _in(xc, 0.6, 0.8) & _in(yc, 0.6, 0.8)
    st[thick], ss[thick] = 100.0, 99.9
    st[void], ss[void] = 0.0, 0.0
    q = np.where(_in(xc, 0.0, 0.2) & _in(yc, 0.0, 0.2), 1.0, 0.0)
    return Problem("c1_16x16_q1_s4", 2, nx, ny, 1, 1, 4, st, ss, q)


def jittered_vertices(nx: int, ny: int, frac: float, seed: int) -> np.ndarray:
    """Vertices of an nx x ny grid on [0,1]^2 moved by U[-frac*h, frac*h].

    Interior vertices move in both coordinates, boundary vertices only along
    their boundary edge, corners stay fixed.
    """
    hx, hy = 1.0 / nx, 1.0 / ny
    ux = uniform(seed, 0, (nx + 1) * (ny + 1)).reshape(ny + 1, nx + 1)
    uy = uniform(seed, 1, (nx + 1) * (ny + 1)).reshape(ny + 1, nx + 1)
    X, Y = np.meshgrid(np.arange(nx + 1) * hx, np.arange(ny + 1) * hy, indexing="xy")
    dx = (2.0 * ux - 1.0) * frac * hx
    dy = (2.0 * uy - 1.0) * frac * hy
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    on_x_bnd = (ii == 0) | (ii == nx)
    on_y_bnd = (jj == 0) | (jj == ny)
    dx = np.where(on_x_bnd, 0.0, dx)
    dy = np.where(on_y_bnd, 0.0, dy)
    V = np.stack([X + dx, Y + dy], axis=-1).reshape(-1, 2)
    return np.ascontiguousarray(V)


def config2(n: int = 256, block: int = 16, p: int = 2, sn: int = 8, jitter: float = 0.15,
            seed: int = MASTER_SEED + 1) -> Problem:
    """Jittered n x n quads, Q2, S8; (n/block)^2 blocks each thick, thin or void; q = 1."""
    assert n % block == 0
    nb = n // block
    mat = np.floor(3.0 * uniform(seed, 2, nb * nb)).astype(np.int64).reshape(nb, nb)
    i = np.arange(n) // block
    BJ, BI = np.meshgrid(i, i, indexing="ij")  # BJ row block (y), BI column block (x)
    m = mat[BJ, BI].ravel()
    st = np.choose(m, [1.0e3, 0.1, 0.0])
    c = np.choose(m, [0.9999, 0.5, 0.0])
    ss = st * c
    q = np.ones(n * n)
    V = jittered_vertices(n, n, jitter, seed) if jitter > 0 else None
    return Problem(f"c2_{n}x{n}_q{p}_s{sn}_jitter", 2, n, n, 1, p, sn, st, ss, q, vertices=V,
                   extra={"block_material": mat})


def random_fields(n_elem: int, seed: int):
    """sigma_t = 10^U[-2,3], c ~ U[0.5, 0.9999], 10% void (Bernoulli)."""
    st = 10.0 ** (-2.0 + 5.0 * uniform(seed, 10, n_elem))
    c = 0.5 + (0.9999 - 0.5) * uniform(seed, 11, n_elem)
    void = uniform(seed, 12, n_elem) < 0.1
    st = np.where(void, 0.0, st)
    ss = np.where(void, 0.0, st * c)
    return st, ss


def central_block(n: int, dim: int) -> np.ndarray:
    """Indicator of the central (n/8)^dim block of elements, start 7n/16."""
    lo, hi = 7 * n // 16, 7 * n // 16 + n // 8
    r = np.arange(n)
    ind = _in(r, lo, hi)
    if dim == 2:
        return (ind[:, None] & ind[None, :]).ravel().astype(np.float64)
    return (ind[:, None, None] & ind[None, :, None] & ind[None, None, :]).ravel().astype(np.float64)


def config3(n: int = 64, p: int = 1, sn: int = 8, seed: int = MASTER_SEED + 2) -> Problem:
    """n^3 unit cube, Q1, S8 (80 dirs); log-uniform sigma_t, thick where sigma_t*h > 1."""
    st, ss = random_fields(n ** 3, seed)
    q = central_block(n, 3)
    return Problem(f"c3_{n}^3_q{p}_s{sn}", 3, n, n, n, p, sn, st, ss, q, thick_rule="sigma_t_h")


def config2d_fields(n: int, p: int, sn: int, seed: int, name: str) -> Problem:
    st, ss = random_fields(n * n, seed)
    q = central_block(n, 2)
    return Problem(name, 2, n, n, 1, p, sn, st, ss, q, thick_rule="sigma_t_h")


def config4(count: int = 64, seed: int = MASTER_SEED + 3) -> list:
    """Batch of `count` 2D instances: N in {32,48,...,192}, p in {1,2,3}, S_N in {4,6,8}."""
    uN = uniform(seed, 20, count)
    up = uniform(seed, 21, count)
    us = uniform(seed, 22, count)
    out = []
    for k in range(count):
        N = 32 + 16 * int(np.floor(11 * uN[k]))
        p = 1 + int(np.floor(3 * up[k]))
        sn = (4, 6, 8)[int(np.floor(3 * us[k]))]
        out.append(config2d_fields(N, p, sn, seed * 1000 + k, f"c4_{k}_{N}x{N}_q{p}_s{sn}"))
    return out


def config5(n: int = 128, seed: int = MASTER_SEED + 4) -> Problem:
    """128^2 Q1 S8 with the random fields; detector = right-edge strip of 4 columns x 16 rows."""
    prob = config2d_fields(n, 1, 8, seed, f"c5_{n}x{n}_q1_s8")
    i = np.arange(n)
    cols = _in(i, n - 4, n)
    rows = _in(i, 7 * n // 16, 7 * n // 16 + n // 8)
    strip = (rows[:, None] & cols[None, :]).ravel()
    nonvoid = np.flatnonzero(prob.sigma_t > 0)
    u = uniform(seed, 30, 32)
    # 32 distinct non-void elements, drawn without replacement by ranking random keys
    keys = uniform(seed, 31, nonvoid.size)
    fd = np.sort(nonvoid[np.argsort(keys, kind="stable")[:32]])
    # a second seeded set inside the detector's neighbourhood (12 columns to its left, 32 rows)
    jj, ii = np.divmod(np.arange(n * n), n)
    near = nonvoid[(ii[nonvoid] >= n - 16) & (jj[nonvoid] >= 7 * n // 16 - 8) & (jj[nonvoid] < 7 * n // 16 + n // 8 + 8)]
    keys2 = uniform(seed, 32, near.size)
    fd_near = np.sort(near[np.argsort(keys2, kind="stable")[:32]])
    prob.extra.update({"detector": strip.astype(np.uint8), "fd_elements": fd, "fd_near": fd_near, "fd_u": u})
    return prob


# Materials of the hohlraum problem (Sec. 4.2, Table hohlraum_materials): opacity sigma and heat
# capacity C_v of gold wall, helium fill, capsule CH layer, hydrogen fuel; NIF units.
HOHLRAUM_SIGMA = (1.0e3, 1.0e-3, 1.0e2, 1.0)
HOHLRAUM_CV = (1.0e5, 1.0e-2, 1.0e3, 1.0)
HOHLRAUM_A_RAD = 137.199      # radiation constant a
HOHLRAUM_C_LIGHT = 2.9979e4   # speed of light c
HOHLRAUM_DT = 1.0e-3          # the paper's single long time step (microseconds)
HOHLRAUM_T_COLD, HOHLRAUM_T_HOT = 1.0e-3, 0.4  # keV: initial temperature; laser-heated gold


def hohlraum_like(n: int = 256, p: int = 2, sn: int = 8, jitter: float = 0.15,
                  seed: int = MASTER_SEED + 6) -> Problem:
    """A synthetic 2D hohlraum-like layout (the paper's curvilinear hohlraum mesh is not available).

    Materials by undeformed cell centre (x, y) in [0, 1]^2; left to right through the capsule:
    gold wall, helium, CH, hydrogen, CH, helium, gold wall (Fig. hohlraum_mesh's order).
      gold: a frame of width 1/16, open (helium) on the top and bottom walls where |x - 1/2| < 1/8
        (laser entrance holes);
      capsule centred at (1/2, 1/2): hydrogen for r < 0.15, CH for 0.15 <= r < 0.18, with a helium
        fill tube through the CH on the right (x > 1/2, |y - 1/2| < 0.01);
      helium everywhere else.
    Temperature T = 0.4 keV on the laser spots (gold of the left and right walls with
    1/8 <= y < 3/8 or 5/8 <= y < 7/8), 1e-3 keV elsewhere; time step 1e-3.
    The returned Problem carries the plain absorber (sigma_t = sigma, sigma_s = 0, q = 0); the
    pseudo-scattering coefficients of Eq. hohlraum_sigma / Eq. hohlraum_q are computed from
    extra = {material, sigma, cv, T, dt, a_rad, c_light} by the consumer.
    """
    xc, yc = _centroids_uniform(n, n)
    w = 1.0 / 16.0
    mat = np.full(n * n, 1, dtype=np.int64)                       # helium
    frame = (xc < w) | (xc >= 1 - w) | (yc < w) | (yc >= 1 - w)
    leh = ((yc < w) | (yc >= 1 - w)) & (np.abs(xc - 0.5) < 0.125)
    mat[frame & ~leh] = 0                                          # gold
    r = np.hypot(xc - 0.5, yc - 0.5)
    mat[r < 0.15] = 3                                              # hydrogen
    ch = (r >= 0.15) & (r < 0.18)
    tube = (xc > 0.5) & (np.abs(yc - 0.5) < 0.01)
    mat[ch & ~tube] = 2                                            # CH
    spot = (mat == 0) & ((xc < w) | (xc >= 1 - w)) & (_in(yc, 0.125, 0.375) | _in(yc, 0.625, 0.875))
    T = np.where(spot, HOHLRAUM_T_HOT, HOHLRAUM_T_COLD)
    sigma = np.choose(mat, HOHLRAUM_SIGMA).astype(np.float64)
    cv = np.choose(mat, HOHLRAUM_CV).astype(np.float64)
    V = jittered_vertices(n, n, jitter, seed) if jitter > 0 else None
    return Problem(f"hohlraum_like_{n}x{n}_q{p}_s{sn}", 2, n, n, 1, p, sn, sigma.copy(), np.zeros(n * n),
                   np.zeros(n * n), vertices=V,
                   extra={"material": mat, "sigma": sigma, "cv": cv, "T": T, "dt": HOHLRAUM_DT,
                          "a_rad": HOHLRAUM_A_RAD, "c_light": HOHLRAUM_C_LIGHT})


def uniform_problem(dim, n, p, sn, sigma_t, sigma_s, q, psi_inc=0.0, name="uniform") -> Problem:
    ne = n ** dim
    return Problem(name, dim, n, n, n if dim == 3 else 1, p, sn,
                   np.full(ne, float(sigma_t)), np.full(ne, float(sigma_s)), np.full(ne, float(q)),
                   psi_inc=psi_inc)


def random_phi(prob: Problem, seed: int, stream: int = 40) -> np.ndarray:
    """A seeded positive scalar-flux field in GL-nodal layout [elem][node]."""
    return 0.5 + uniform(seed, stream, prob.n_elem * prob.n_nodes).reshape(prob.n_elem, prob.n_nodes)
