"""GPU: the operator cache (every A_e^{-1} formed once per material set, node-per-lane sweeps)
against the on-the-fly element solves and the CPU oracle, through the C ABI.

Tolerances as in the other parity tests: 1e-12 relative to max |oracle| for float64 sweeps,
1e-5 for the FP32 element-solve form.
"""
import dataclasses

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


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(got, ref):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def ragged_problem():
    nx, ny = 13, 7
    st, ss = inputs.random_fields(nx * ny, 4243)
    q = np.where(np.arange(nx * ny) % 3 == 0, 1.0, 0.2)
    return inputs.Problem("ragged_13x7_q2_s4", 2, nx, ny, 1, 2, 4, st, ss, q, psi_inc=0.7)


CASES = {
    "c1": inputs.config1,
    "c2_32": lambda: inputs.config2(n=32, block=8),
    "c3_8": lambda: inputs.config3(n=8),
    "q3_s6": lambda: inputs.config2d_fields(12, 3, 6, 78, "q3"),
    "ragged_q2": ragged_problem,
}


@pytest.fixture(scope="module")
def oracles():
    return {}


def _oracle(name, cache):
    from oracle import Transport
    if name not in cache:
        prob = CASES[name]()
        cache[name] = (prob, Transport(prob))
    return cache[name]


@pytest.mark.parametrize("schedule", ["levels", "dataflow", "tiles"])
@pytest.mark.parametrize("name", list(CASES))
def test_cached_sweeps_match_oracle(sn, oracles, name, schedule):
    from oracle import adjoint
    prob, T = _oracle(name, oracles)
    phi = inputs.random_phi(prob, 14)
    mu = inputs.random_phi(prob, 15) - 0.75
    ref, ref_adj = T.sweep(phi), adjoint.adjoint_sweep(T, mu)
    on = sn.Mesh.from_problem(prob)
    on.set_schedule(schedule)
    on.set_operator_cache("on")
    off = sn.Mesh.from_problem(prob)
    off.set_schedule(schedule)
    off.set_operator_cache("off")
    got_on, got_off = on.sweep(_t(phi)), off.sweep(_t(phi))
    assert _rel(got_on, ref) < 1e-12
    assert _rel(got_off, ref) < 1e-12
    assert _rel(on.sweep(_t(phi), precision="fp32"), ref) < 1e-5
    assert _rel(on.adjoint_sweep(_t(mu)), ref_adj) < 1e-12
    assert _rel(off.adjoint_sweep(_t(mu)), ref_adj) < 1e-12
    # a second sweep reuses the cache and gives the same bits
    assert torch.equal(on.sweep(_t(phi)), got_on)


def test_cache_follows_material_changes(sn):
    """set_materials invalidates the cached inverses: the next sweep uses the new sigma_t."""
    from oracle import Transport
    prob = inputs.config2d_fields(12, 2, 6, 91, "mat")
    phi = inputs.random_phi(prob, 16)
    m = sn.Mesh.from_problem(prob)
    m.set_operator_cache("on")
    assert _rel(m.sweep(_t(phi)), Transport(prob).sweep(phi)) < 1e-12
    prob2 = dataclasses.replace(prob, sigma_t=prob.sigma_t * 1.7 + 0.3, sigma_s=prob.sigma_s * 0.5,
                                q=prob.q + 0.25)
    m.set_materials(prob2.sigma_t, prob2.sigma_s, prob2.q)
    assert _rel(m.sweep(_t(phi)), Transport(prob2).sweep(phi)) < 1e-12
    assert _rel(m.sweep(_t(phi), precision="fp32"), Transport(prob2).sweep(phi)) < 1e-5


def test_cache_modes_switch_between_paths(sn):
    """on -> off -> auto on one mesh: every path gives the oracle's sweep."""
    from oracle import Transport
    prob = inputs.config2d_fields(10, 1, 8, 92, "modes")
    phi = inputs.random_phi(prob, 17)
    ref = Transport(prob).sweep(phi)
    m = sn.Mesh.from_problem(prob)
    for mode in ("on", "off", "auto", "off", "on"):
        m.set_operator_cache(mode)
        assert _rel(m.sweep(_t(phi)), ref) < 1e-12
    with pytest.raises(sn.SnError):
        m.set_operator_cache(7)


@pytest.mark.parametrize("schedule", [("levels", 64, 0), ("dataflow", 128, 0)])
def test_batched_cached_sweeps_equal_single_sweeps(sn, schedule):
    """Cached batched sweeps (node-per-lane) equal each instance's own cached sweep bit for bit,
    and an uncached batch agrees with them to rounding."""
    probs = [inputs.config2d_fields(16, 1, 4, 21, "a"), inputs.config2d_fields(20, 2, 8, 22, "b"),
             inputs.config2d_fields(12, 3, 6, 23, "c"), inputs.config3(n=6)]
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    batch.set_schedule(*schedule)
    phis = [_t(inputs.random_phi(p, 70 + k)) for k, p in enumerate(probs)]
    for prec in ("fp64", "fp32"):
        outs = batch.sweep(phis, precision=prec)
        for m, phi, out in zip(meshes, phis, outs):
            assert torch.equal(m.sweep(phi, precision=prec), out)
    fp64 = [o.clone() for o in batch.sweep(phis, precision="fp64")]
    for m in meshes:
        m.set_operator_cache("off")
    for a, b in zip(batch.sweep(phis, precision="fp64"), fp64):
        assert _rel(a, b.cpu().numpy()) < 1e-13
