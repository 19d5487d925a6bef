"""GPU: the upwind level sets the device builds (Kahn's algorithm on the upwind graph, Sec. 1).

On a Cartesian mesh the level of element (i, j[, k]) for a direction with signs (sx, sy[, sz]) is
the index sum i' + j' (+ k') with i' = i where sx > 0 and nx - 1 - i where sx < 0 (closed form).
On a jittered mesh, where faces nearly parallel to a direction change the graph, the levels equal
the oracle's own Kahn levels element by element.
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09196_gb300 import build
    build.build()
    from paper_2001_09196_gb300 import sn as mod
    return mod


@pytest.mark.parametrize("dim,shape,order", [(2, (7, 5, 1), 8), (2, (1, 6, 1), 4), (3, (4, 3, 5), 4), (3, (2, 2, 2), 8)])
def test_cartesian_levels_are_index_sums(sn, dim, shape, order):
    nx, ny, nz = shape
    m = sn.Mesh(dim, nx, ny, nz, 1, order)
    dirs, _ = m.quadrature()
    e = np.arange(m.n_elem)
    ijk = [e % nx, (e // nx) % ny, e // (nx * ny)]
    for d in range(m.n_dirs):
        expect = np.zeros(m.n_elem, dtype=np.int64)
        for a, n_a in enumerate(shape[:dim]):
            expect += np.where(dirs[d, a] > 0, ijk[a], n_a - 1 - ijk[a])
        assert np.array_equal(m.levels(d), expect), d
    assert m.n_levels == sum(shape[:dim]) - dim + 1


def test_jittered_levels_equal_the_oracle_kahn_levels(sn):
    from oracle import Transport
    prob = inputs.config2(n=32, block=8)
    T = Transport(prob)
    m = sn.Mesh.from_problem(prob, materials=False)
    for d in range(T.nd):
        ref = np.empty(T.ne, dtype=np.int64)
        for lev, elems in enumerate(T.levels(d)):
            ref[elems] = lev
        assert np.array_equal(m.levels(d), ref), d


def test_levels_argument_errors(sn):
    m = sn.Mesh(2, 3, 3, 1, 1, 4)
    for d in (-1, m.n_dirs):
        with pytest.raises(sn.SnError) as e:
            m.levels(d)
        assert e.value.status == 1
