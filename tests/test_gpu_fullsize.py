"""GPU parity at the workloads' full sizes, in the launch configuration the benchmark times.

The oracle cannot sweep every direction of these meshes in seconds, so it checks samples it can
compute one by one: whole directions of a sweep (every element), and the residual of the
converged solution under the oracle's own transport update.  Tolerances as in the other parity
tests (1e-12 relative for float64 sweeps, 1e-5 for the FP32 form).

Workloads: the 256x256 jittered Q2 S8 mesh (config 2, the benchmark's), the 64^3 Q1 S8 mesh
(config 3) and the 64-instance batch (config 4).
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


@pytest.fixture(scope="module")
def c2(sn):
    from oracle import Transport
    prob = inputs.config2()
    m = sn.Mesh.from_problem(prob)
    m.autotune("fp64")  # the benchmark's launch configuration
    return prob, m, Transport(prob)


def _rel(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _oracle_direction(T, phi_nodal, d):
    src = T.isotropic_source(T.to_modal(phi_nodal))
    return T.to_nodal(T.sweep_direction(d, src))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_config2_sweep_directions_match_the_oracle(c2, precision, tol):
    prob, m, T = c2
    phi = inputs.random_phi(prob, 101)
    m.sweep(torch.as_tensor(phi, device="cuda"), precision=precision)
    for d in (0, 13, 27, 39):  # one direction per quadrant of the 2D set
        got = m.angular_flux(d, precision=precision).cpu().numpy()
        assert _rel(got, _oracle_direction(T, phi, d)) < tol, d


def test_config2_solution_has_the_oracle_residual(c2):
    """The benchmark's solve (FP64 thick-DSA fGMRES to 1e-8): the oracle's transport update of the
    GPU solution reproduces it to the residual the solve claims."""
    prob, m, T = c2
    r = m.source_iterate(dsa="thick", thick_rule="sigma_s", tol=1e-8, inner_tol=1e-4, max_iters=500,
                         outer="fgmres", restart=30)
    assert r["converged"] and r["rel_residual"] <= 1e-8
    phi = r["phi"].cpu().numpy()
    res = np.linalg.norm(T.sweep(phi) - phi)
    r0 = np.linalg.norm(T.sweep(np.zeros_like(phi)))  # residual of phi = 0
    assert res / r0 < 2e-8


def test_config3_sweep_directions_match_the_oracle(sn):
    from oracle import Transport
    prob = inputs.config3()
    m = sn.Mesh.from_problem(prob)
    m.autotune("fp64")
    T = Transport(prob)
    phi = inputs.random_phi(prob, 102)
    m.sweep(torch.as_tensor(phi, device="cuda"))
    for d in (5, 62):  # two octants
        got = m.angular_flux(d).cpu().numpy()
        assert _rel(got, _oracle_direction(T, phi, d)) < 1e-12, d


def test_config4_batched_sweep(sn):
    """The 64-instance batch: the batched sweep equals every instance's own sweep bit for bit, and
    sampled directions of two instances (the largest and a Q3 one) match the oracle."""
    from oracle import Transport
    probs = inputs.config4()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    batch.autotune("fp64")
    phis = [torch.as_tensor(inputs.random_phi(p, 200 + k), device="cuda") for k, p in enumerate(probs)]
    outs = batch.sweep(phis)
    for m, phi, out in zip(meshes, phis, outs):
        assert torch.equal(m.sweep(phi), out)
    largest = max(range(len(probs)), key=lambda k: probs[k].n_elem * probs[k].n_nodes * probs[k].n_dirs)
    q3 = next(k for k, p in enumerate(probs) if p.p == 3)
    for k in (largest, q3):
        T = Transport(probs[k])
        meshes[k].sweep(phis[k])
        d = probs[k].n_dirs // 2
        got = meshes[k].angular_flux(d).cpu().numpy()
        assert _rel(got, _oracle_direction(T, phis[k].cpu().numpy(), d)) < 1e-12, (k, d)
