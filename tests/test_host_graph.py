"""CPU: the library's directed-graph helpers of the tiled schedule (csrc/sn_setup.cpp, through
tests/host_drivers/graph_dump.cpp, no GPU).

The tiled sweep groups each direction's elements into tasks, one per strongly connected component
of the tile-level upwind graph, and lists the tasks in a topological order of the component graph;
that order is what keeps its persistent kernel free of deadlock.  These tests check the two
helpers it rests on: the CSR construction (sorted, de-duplicated edges) and the strongly connected
components, against scipy's on hand-made and seeded random graphs, including a long chain (the
component search is iterative, not recursive) and graphs whose component graph must be acyclic."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2001_09196_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("host_drivers") / "graph_dump")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "host_drivers", "graph_dump.cpp"), os.path.join(CSRC, "sn_setup.cpp"),
                    "-o", exe], check=True)
    return exe


def run(driver, n, edges):
    text = f"{n} {len(edges)}\n" + "".join(f"{a} {b}\n" for a, b in edges)
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    ptr = np.array(out[0].split()[1:], dtype=np.int64)
    adj = np.array(out[1].split()[1:], dtype=np.int64)
    nc = int(out[2].split()[1])
    comp = np.array(out[3].split()[1:], dtype=np.int64)
    return ptr, adj, nc, comp


def canonical(labels):
    """Relabel a partition by order of first appearance, so that two labellings compare equal."""
    first = {}
    return np.array([first.setdefault(int(c), len(first)) for c in labels], dtype=np.int64)


def scipy_components(n, edges):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    if n == 0:
        return 0, np.zeros(0, dtype=np.int64)
    a = np.array(edges, dtype=np.int64).reshape(-1, 2)
    g = sp.csr_matrix((np.ones(len(a)), (a[:, 0], a[:, 1])), shape=(n, n))
    return connected_components(g, directed=True, connection="strong")


def check(driver, n, edges):
    ptr, adj, nc, comp = run(driver, n, edges)
    # CSR: the de-duplicated edges, sorted by source and then target
    want = sorted(set(map(tuple, edges)))
    assert ptr.shape == (n + 1,) and ptr[0] == 0 and np.all(np.diff(ptr) >= 0)
    got = [(s, int(t)) for s in range(n) for t in adj[ptr[s]:ptr[s + 1]]]
    assert got == want
    # components: the same partition as scipy's, labels 0 .. nc-1
    k, ref = scipy_components(n, edges)
    assert nc == k and comp.shape == (n,)
    assert n == 0 or (comp.min() == 0 and comp.max() == nc - 1)
    assert np.array_equal(canonical(comp), canonical(ref))
    # the component graph is acyclic: Kahn's order reaches every component
    cedges = {(int(comp[a]), int(comp[b])) for a, b in want if comp[a] != comp[b]}
    indeg = np.zeros(nc, dtype=np.int64)
    for _, b in cedges:
        indeg[b] += 1
    out = {c: [] for c in range(nc)}
    for a, b in cedges:
        out[a].append(b)
    order = [c for c in range(nc) if indeg[c] == 0]
    for c in order:
        for b in out[c]:
            indeg[b] -= 1
            if indeg[b] == 0:
                order.append(b)
    assert len(order) == nc
    return nc, comp


def test_small_graphs(driver):
    assert check(driver, 0, [])[0] == 0
    assert check(driver, 1, [])[0] == 1
    assert check(driver, 1, [(0, 0)])[0] == 1
    assert check(driver, 3, [(0, 1), (1, 2), (2, 0)])[0] == 1                       # one ring
    assert check(driver, 4, [(0, 1), (1, 2), (2, 3)])[0] == 4                       # a chain
    nc, comp = check(driver, 6, [(0, 1), (1, 0), (1, 2), (2, 3), (3, 4), (4, 2), (5, 5), (5, 0)])
    assert nc == 3 and comp[0] == comp[1] and comp[2] == comp[3] == comp[4] and len({comp[0], comp[2], comp[5]}) == 3
    assert check(driver, 3, [(0, 1), (0, 1), (1, 2), (1, 2)])[0] == 3               # duplicate edges


def test_tile_grid_with_a_reversed_face(driver):
    """A 4x4 grid of tiles with the upwind edges of one direction (+x, +y) is acyclic, every tile a
    task of its own; one tile face whose flux jitter reversed adds the opposite edge, and the two
    tiles on either side of it must become one task."""
    n = 4
    tid = lambda i, j: i + n * j  # noqa: E731
    edges = [(tid(i, j), tid(i + 1, j)) for j in range(n) for i in range(n - 1)]
    edges += [(tid(i, j), tid(i, j + 1)) for j in range(n - 1) for i in range(n)]
    assert check(driver, n * n, edges)[0] == n * n
    nc, comp = check(driver, n * n, edges + [(tid(2, 1), tid(1, 1))])
    assert nc == n * n - 1 and comp[tid(1, 1)] == comp[tid(2, 1)]


def test_long_chain_and_long_ring(driver):
    n = 200_000
    chain = [(k, k + 1) for k in range(n - 1)]
    _, _, nc, _ = run(driver, n, chain)
    assert nc == n
    _, _, nc, comp = run(driver, n, chain + [(n - 1, 0)])
    assert nc == 1 and np.all(comp == 0)


@pytest.mark.parametrize("seed", range(8))
def test_random_graphs_match_scipy(driver, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(5, 300))
    m = int(rng.integers(0, 3 * n))
    edges = [tuple(map(int, e)) for e in rng.integers(0, n, size=(m, 2))]
    check(driver, n, edges)
