"""GPU: the direction-sharded iteration through the C ABI (Eq. phi: the transport update is a sum
over directions).  Two processes on the one GPU each sweep half of the directions of every
transport update and a gloo all-reduce of the partial scalar fluxes completes it (host copies:
the two processes' kernels never wait on one another).  The DSA step, the Krylov work and the
convergence test run replicated.  Both ranks must hold bitwise the same iterates, equal to the
unsharded iteration up to the order of the float64 sum over directions.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle.dsa import thick_mask
from tolerances import dsa_iterate_tol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    return inputs.config2(n=32, block=8)


RUNS = {"si_k6": dict(dsa="thick", tol=0.0, max_iters=6, inner_tol=1e-14, inner_max_iters=1000),
        "fgmres": dict(dsa="thick", outer="fgmres", tol=1e-12, inner_tol=1e-10, max_iters=400),
        "triangular_k4": dict(dsa="triangular", tol=0.0, max_iters=4, inner_tol=1e-14, inner_max_iters=1000)}


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2001_09196_gb300 import build
    build.build()
    from paper_2001_09196_gb300 import sn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    prob = _problem()
    m = sn.Mesh.from_problem(prob)
    nd = m.n_dirs
    mine = (rank * nd // world, (rank + 1) * nd // world)
    ex = sn.torch_allreduce()
    for name, kw in RUNS.items():
        r = m.source_iterate(directions=mine, exchange=ex, **kw)
        np.save(os.path.join(out_dir, f"{name}_rank{rank}.npy"), r["phi"].cpu().numpy())
        np.save(os.path.join(out_dir, f"{name}_iters_rank{rank}.npy"), np.array([r["iters"], r["sweeps"]]))
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09196_gb300 import build
    build.build()
    from paper_2001_09196_gb300 import sn as mod
    return mod


def test_two_rank_direction_sharded_iterations_match_the_unsharded_ones(sn, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    prob = _problem()
    m = sn.Mesh.from_problem(prob)
    tol = dsa_iterate_tol(prob, thick_mask(prob))
    for name, kw in RUNS.items():
        a = np.load(tmp_path / f"{name}_rank0.npy")
        b = np.load(tmp_path / f"{name}_rank1.npy")
        assert np.array_equal(a, b), name
        ia, ib = np.load(tmp_path / f"{name}_iters_rank0.npy"), np.load(tmp_path / f"{name}_iters_rank1.npy")
        assert np.array_equal(ia, ib)
        ref = m.source_iterate(**kw)
        rel = np.abs(a - ref["phi"].cpu().numpy()).max() / np.abs(ref["phi"].cpu().numpy()).max()
        if name == "fgmres":
            assert ref["converged"] and abs(int(ia[0]) - ref["iters"]) <= 1
            assert rel < 1e-9, (name, rel)
        else:
            assert int(ia[0]) == ref["iters"] and rel <= tol, (name, rel)


def test_sharding_argument_errors(sn):
    prob = inputs.config1()
    m = sn.Mesh.from_problem(prob)
    ex = lambda t: None  # noqa: E731  (a one-process "sum")
    for rng in ((5, 3), (0, m.n_dirs + 1), (-1, 4)):
        with pytest.raises(sn.SnError) as e:
            m.source_iterate(directions=rng, exchange=ex, max_iters=2)
        assert e.value.status == 1
    with pytest.raises(ValueError):
        m.source_iterate(directions=(0, 4), max_iters=2)
    # a one-process "exchange" over all directions reproduces the plain iteration bit for bit (the
    # same element solves and the same order of the sum over directions)
    r1 = m.source_iterate(directions=(0, m.n_dirs), exchange=ex, dsa="thick", tol=0.0, max_iters=5)
    r0 = m.source_iterate(dsa="thick", tol=0.0, max_iters=5)
    assert torch.equal(r1["phi"], r0["phi"])
    # an exchange that fails ends the iteration with its status
    def bad(t):
        raise RuntimeError("peer lost")
    with pytest.raises(RuntimeError, match="peer lost"):
        m.source_iterate(directions=(0, m.n_dirs), exchange=bad, max_iters=3)
