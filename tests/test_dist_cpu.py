"""Multi-process (N > 1) paths on CPU ranks with the gloo backend.

The library runs one process per GPU and the GPU tests use one GPU, so the N > 1 logic is covered
here: the max-over-ranks timing and barrier used by `bench.py`, the reference arm launched by
torch.distributed.run with two ranks (rank 0 alone prints the JSON line), and the exchange step
of a direction-sharded transport update (each rank sums its own directions, one sum-reduction of
the scalar flux completes the update), run on the oracle.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.max_over_ranks(10.0 + rank * 3.5, world)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(got))
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_with_gloo(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert float(open(tmp_path / f"rank{r}.txt").read()) == 13.5


def test_reference_arm_under_two_ranks_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def _shard_main(rank, world, port, out_dir):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import Transport
    from paper_2001_09196_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = inputs.config2d_fields(6, 1, 4, 77, "shard")
    T = Transport(prob)
    phi = inputs.random_phi(prob, 9)
    mine = range(rank * T.nd // world, (rank + 1) * T.nd // world)   # this rank's directions
    part = torch.as_tensor(T.sweep(phi, directions=mine))
    dist.all_reduce(part, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(os.path.join(out_dir, "reduced.npy"), part.numpy())
        np.save(os.path.join(out_dir, "full.npy"), T.sweep(phi))
    dist.destroy_process_group()


def test_direction_sharded_update_with_gloo(tmp_path):
    """Ranks sweep disjoint direction ranges; the allreduce of their partial scalar fluxes equals the
    full transport update (Eq. phi: phi = sum over all directions of w_d psi_d)."""
    import numpy as np
    import torch.multiprocessing as mp
    mp.spawn(_shard_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got, ref = np.load(tmp_path / "reduced.npy"), np.load(tmp_path / "full.npy")
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def _exchange_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2001_09196_gb300 import sn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ex = sn.torch_allreduce()
    t = torch.arange(12, dtype=torch.float64).reshape(3, 4) * (rank + 1)
    ex(t)  # in place, as the library's exchange step expects
    torch.save(t, os.path.join(out_dir, f"ex{rank}.pt"))
    dist.destroy_process_group()


def test_exchange_function_sums_partial_updates_in_place(tmp_path):
    """The exchange the binding hands to a direction-sharded iteration replaces each rank's partial
    update by the sum over ranks, in place and identically on every rank."""
    import torch.multiprocessing as mp
    mp.spawn(_exchange_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    a, b = (torch.load(tmp_path / f"ex{r}.pt") for r in range(2))
    expect = torch.arange(12, dtype=torch.float64).reshape(3, 4) * 3
    assert torch.equal(a, expect) and torch.equal(b, expect)
