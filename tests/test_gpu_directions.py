"""GPU: partial transport updates over direction ranges (the decomposition behind sharding the
sweep by direction).  The partial updates of a partition of the directions sum to the full
update to 1e-13 relative (only the order of the float64 additions differs); the angular fluxes
of a range are bitwise those of the full sweep; a range matches the oracle's partial update to
1e-12 (FP64).
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


def _rel(got, ref):
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300))


CASES = {
    "c2_32": (lambda: inputs.config2(n=32, block=8), [0, 13, 27, 40]),
    "c3_8": (lambda: inputs.config3(n=8), [0, 40, 80]),
    "q3_s6": (lambda: inputs.config2d_fields(12, 3, 6, 79, "q3"), [0, 1, 24]),
}


@pytest.mark.parametrize("schedule", ["levels", "dataflow"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_direction_ranges_sum_to_the_full_sweep(sn, name, precision, schedule):
    make, cuts = CASES[name]
    prob = make()
    m = sn.Mesh.from_problem(prob)
    m.set_schedule(schedule)
    phi = torch.as_tensor(inputs.random_phi(prob, 51), device="cuda")
    full = m.sweep(phi, precision=precision).cpu().numpy()
    psi = {d: m.angular_flux(d, precision=precision).clone() for d in range(prob.n_dirs)}
    total = np.zeros_like(full)
    for d0, d1 in zip(cuts, cuts[1:]):
        part = m.sweep_directions(phi, d0, d1, precision=precision).cpu().numpy()
        total += part
        for d in (d0, (d0 + d1) // 2, d1 - 1):
            assert torch.equal(m.angular_flux(d, precision=precision), psi[d]), (d0, d1, d)
    assert _rel(total, full) < 1e-13


def test_a_direction_range_matches_the_oracle(sn):
    from oracle import Transport
    prob = inputs.config2(n=32, block=8)
    T = Transport(prob)
    m = sn.Mesh.from_problem(prob)
    phi = inputs.random_phi(prob, 52)
    got = m.sweep_directions(torch.as_tensor(phi, device="cuda"), 7, 19).cpu().numpy()
    assert _rel(got, T.sweep(phi, directions=range(7, 19))) < 1e-12


def test_direction_range_errors(sn):
    prob = inputs.config1()
    m = sn.Mesh.from_problem(prob)
    phi = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    for d0, d1 in ((-1, 3), (0, 13), (5, 5), (7, 3)):
        with pytest.raises(sn.SnError) as e:
            m.sweep_directions(phi, d0, d1)
        assert e.value.status == 1
