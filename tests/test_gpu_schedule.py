"""GPU: the sweep schedules agree bit for bit, and the bounded dependency waits report a timeout."""
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
    for block, cap in ((128, 0), (64, 0), (32, 1), (96, 2)):
        m.set_schedule("dataflow", block, cap)
        got = m.sweep(phi, precision=precision)
        assert torch.equal(got, ref), (block, cap)


def test_dependency_wait_timeout_is_reported_and_recoverable(sn):
    prob = CASES["c2_32"]()
    m = sn.Mesh.from_problem(prob)
    m.set_schedule("dataflow", 128, 0)
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
    for block, cap in ((128, 0), (32, 1)):
        m.set_schedule("dataflow", block, cap)
        assert torch.equal(m.adjoint_sweep(mu), ref), (block, cap)
