"""GPU: the sweep schedules (level graphs, dataflow, tiles) agree bit for bit, and the bounded
dependency waits report a timeout."""
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


CASES = {
    "c2_32": lambda: inputs.config2(n=32, block=8),
    "c3_8": lambda: inputs.config3(n=8),
    "q3": lambda: inputs.config2d_fields(12, 3, 6, 77, "q3"),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine"])
def test_schedules_agree_bitwise(sn, name, precision):
    prob = CASES[name]()
    m = sn.Mesh.from_problem(prob)
    phi = torch.as_tensor(inputs.random_phi(prob, 5), device="cuda")
    m.set_schedule("levels", 128)
    ref = m.sweep(phi, precision=precision)
    for sched, block, param in (("levels", 32, 4), ("levels", 64, 3), ("levels", 32, 1000), ("dataflow", 128, 0),
                                ("dataflow", 64, 0), ("dataflow", 32, 1), ("dataflow", 96, 2), ("tiles", 128, 4),
                                ("tiles", 256, 8), ("tiles", 64, 3), ("tiles", 32, 16), ("barrier", 256, 1),
                                ("barrier", 512, 1), ("barrier", 128, 3), ("static", 128, 0), ("static", 32, 0),
                                ("static", 64, 2)):
        if sched == "levels" and param > m.n_dirs:
            param = m.n_dirs  # one chain per direction
        m.set_schedule(sched, block, param)
        got = m.sweep(phi, precision=precision)
        assert torch.equal(got, ref), (sched, block, param)


@pytest.mark.parametrize("schedule", [("dataflow", 128, 0), ("static", 32, 0), ("tiles", 128, 8), ("barrier", 256, 1)])
def test_dependency_wait_timeout_is_reported_and_recoverable(sn, schedule):
    prob = CASES["c2_32"]()
    m = sn.Mesh.from_problem(prob)
    m.set_schedule(*schedule)
    phi = torch.as_tensor(inputs.random_phi(prob, 6), device="cuda")
    ref = m.sweep(phi)
    m.debug_stall_next_sweep(0.2)
    with pytest.raises(sn.SnError) as e:
        m.sweep(phi)
    assert e.value.status == 7
    assert torch.equal(m.sweep(phi), ref)
    r = m.source_iterate(dsa="thick", tol=1e-6, max_iters=50)
    assert r["converged"]


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_schedules_agree_bitwise(sn, name):
    prob = CASES[name]()
    m = sn.Mesh.from_problem(prob)
    mu = torch.as_tensor(inputs.random_phi(prob, 8) - 0.7, device="cuda")
    m.set_schedule("levels", 128)
    ref = m.adjoint_sweep(mu)
    for sched, block, param in (("levels", 32, 4), ("dataflow", 128, 0), ("dataflow", 32, 1), ("tiles", 128, 8),
                                ("static", 32, 0)):
        m.set_schedule(sched, block, param)
        assert torch.equal(m.adjoint_sweep(mu), ref), (sched, block, param)


CANDIDATES = {("levels", 32, 0), ("levels", 64, 0), ("levels", 128, 0), ("levels", 32, 4), ("levels", 32, 8),
              ("levels", 64, 8), ("levels", 32, 16), ("dataflow", 128, 0), ("dataflow", 128, 1),
              ("dataflow", 64, 2), ("dataflow", 32, 4), ("tiles", 128, 8), ("tiles", 128, 16), ("tiles", 256, 16),
              ("tiles", 256, 32), ("levels", 32, 2), ("tiles", 256, 16), ("barrier", 256, 1), ("barrier", 512, 1),
              ("barrier", 256, 2), ("barrier", 128, 4), ("static", 128, 0), ("static", 64, 0), ("static", 128, 4),
              ("static", 128, 2), ("static", 32, 0)}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_picks_a_candidate_and_keeps_results(sn, precision):
    prob = inputs.config2(n=48, block=8)
    m = sn.Mesh.from_problem(prob)
    phi = torch.as_tensor(inputs.random_phi(prob, 9), device="cuda")
    ref = m.sweep(phi, precision=precision)
    choice = m.autotune(precision)
    assert choice in CANDIDATES
    assert torch.equal(m.sweep(phi, precision=precision), ref)
    # a second mesh of the same shape takes the cached choice
    m2 = sn.Mesh.from_problem(prob)
    assert m2.autotune(precision) == choice
    assert torch.equal(m2.sweep(phi, precision=precision), ref)


def test_batch_autotune_keeps_results(sn):
    probs = [inputs.config2d_fields(16, 1, 4, 11, "a"), inputs.config2d_fields(20, 2, 6, 12, "b"), inputs.config3(n=6)]
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    phis = [torch.as_tensor(inputs.random_phi(p, 30 + k), device="cuda") for k, p in enumerate(probs)]
    ref = batch.sweep(phis)
    assert batch.autotune("fp64") in CANDIDATES
    for a, b in zip(batch.sweep(phis), ref):
        assert torch.equal(a, b)
