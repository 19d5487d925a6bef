"""The seeded synthetic inputs follow the recipes stated for the five workloads (no GPU).

The generators hold none of the method's arithmetic; these checks pin what they produce to the
stated shapes, material values and distributions, and check that they are reproducible."""
import os

import numpy as np

from paper_2001_09196_gb300 import inputs


def _centroids(prob):
    j, i = np.divmod(np.arange(prob.nx * prob.ny), prob.nx)
    return (i + 0.5) / prob.nx, (j + 0.5) / prob.ny


def test_config1_regions():
    p = inputs.config1()
    assert (p.dim, p.nx, p.ny, p.p, p.sn) == (2, 16, 16, 1, 4)
    x, y = _centroids(p)
    thick = (x >= 0.25) & (x < 0.5) & (y >= 0.25) & (y < 0.5)
    void = (x >= 0.6) & (x < 0.8) & (y >= 0.6) & (y < 0.8)
    rest = ~(thick | void)
    assert np.all(p.sigma_t[thick] == 100.0) and np.all(p.sigma_s[thick] == 99.9)
    assert np.all(p.sigma_t[void] == 0.0) and np.all(p.sigma_s[void] == 0.0)
    assert np.all(p.sigma_t[rest] == 1.0) and np.all(p.sigma_s[rest] == 0.9)
    assert np.array_equal(p.q == 1.0, (x < 0.2) & (y < 0.2))
    assert np.all(p.q[(x >= 0.2) | (y >= 0.2)] == 0.0)


def test_config2_blocks_and_jitter():
    p = inputs.config2()
    n, h = 256, 1.0 / 256
    assert (p.dim, p.nx, p.ny, p.p, p.sn) == (2, n, n, 2, 8)
    assert np.all(p.q == 1.0)
    st = p.sigma_t.reshape(n, n)
    ss = p.sigma_s.reshape(n, n)
    # 16 x 16 blocks of 16 x 16 elements, each one material: thick, thin or void
    blocks = st.reshape(16, 16, 16, 16).transpose(0, 2, 1, 3).reshape(256, 256)
    assert np.all(blocks.min(axis=1) == blocks.max(axis=1))
    assert set(np.unique(st)) <= {1.0e3, 0.1, 0.0}
    assert np.allclose(ss[st == 1.0e3], 999.9) and np.allclose(ss[st == 0.1], 0.05) and np.all(ss[st == 0.0] == 0.0)
    counts = [np.sum(blocks[:, 0] == v) for v in (1.0e3, 0.1, 0.0)]
    assert min(counts) > 40  # all three materials present in about equal shares
    # vertices within +-0.15 h of the grid, boundary vertices only along the boundary, corners fixed
    V = p.vertices.reshape(n + 1, n + 1, 2)
    jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    dx, dy = V[..., 0] - ii * h, V[..., 1] - jj * h
    assert np.abs(dx).max() <= 0.15 * h + 1e-15 and np.abs(dy).max() <= 0.15 * h + 1e-15
    assert np.abs(dx).max() > 0.14 * h
    assert np.all(dx[:, 0] == 0) and np.all(dx[:, n] == 0) and np.all(dy[0, :] == 0) and np.all(dy[n, :] == 0)


def test_config3_fields():
    p = inputs.config3()
    n = 64
    assert (p.dim, p.nx, p.ny, p.nz, p.p, p.sn, p.thick_rule) == (3, n, n, n, 1, 8, "sigma_t_h")
    void = p.sigma_t == 0.0
    assert 0.09 < void.mean() < 0.11
    st = p.sigma_t[~void]
    assert st.min() >= 1e-2 and st.max() <= 1e3
    logs = np.log10(st)
    assert abs(logs.mean() - 0.5) < 0.05  # log-uniform on [-2, 3]
    c = p.sigma_s[~void] / st
    assert c.min() >= 0.5 - 1e-12 and c.max() <= 0.9999 + 1e-12
    q = p.q.reshape(n, n, n)
    assert q.sum() == 8 ** 3 and np.all(q[28:36, 28:36, 28:36] == 1.0)


def test_config4_batch():
    probs = inputs.config4()
    assert len(probs) == 64
    assert {p.nx for p in probs} <= set(range(32, 193, 16))
    assert {p.p for p in probs} == {1, 2, 3}
    assert {p.sn for p in probs} == {4, 6, 8}
    assert all(p.nx == p.ny and p.dim == 2 for p in probs)


def test_config5_detector_and_fd_sets():
    p = inputs.config5()
    n = 128
    assert (p.nx, p.p, p.sn) == (n, 1, 8)
    strip = p.extra["detector"].reshape(n, n).astype(bool)
    rows, cols = np.nonzero(strip)
    assert strip.sum() == 16 * 4 and cols.min() == n - 4 and cols.max() == n - 1
    assert rows.max() - rows.min() == 15
    for key in ("fd_elements", "fd_near"):
        e = p.extra[key]
        assert len(np.unique(e)) == 32 and np.all(p.sigma_t[e] > 0)


def test_generators_are_reproducible():
    a, b = inputs.config2(n=32, block=8), inputs.config2(n=32, block=8)
    assert np.array_equal(a.sigma_t, b.sigma_t) and np.array_equal(a.vertices, b.vertices)
    assert np.array_equal(inputs.random_phi(a, 3), inputs.random_phi(b, 3))
    c = inputs.config2(n=32, block=8, seed=inputs.MASTER_SEED + 99)
    assert not np.array_equal(a.vertices, c.vertices)


def test_hohlraum_constants_are_the_papers():
    """The hohlraum-like layout's materials and constants equal the values the paper prints
    (Sec. 4.2, Table hohlraum_materials; tests/golden/hohlraum_materials.txt)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hohlraum_materials.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    mats = {r[0]: (float(r[1]), float(r[2])) for r in rows if len(r) == 3}
    consts = {r[0]: float(r[1]) for r in rows if len(r) == 2}
    order = ("gold", "helium", "CH", "hydrogen")
    assert inputs.HOHLRAUM_SIGMA == tuple(mats[k][0] for k in order)
    assert inputs.HOHLRAUM_CV == tuple(mats[k][1] for k in order)
    assert (inputs.HOHLRAUM_A_RAD, inputs.HOHLRAUM_C_LIGHT, inputs.HOHLRAUM_DT) == (consts["a"], consts["c"],
                                                                                   consts["dt"])
