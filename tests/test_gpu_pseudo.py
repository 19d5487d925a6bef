"""GPU: the pseudo-scattering time step (Sec. 4.2, Eq. hohlraum_sigma / Eq. hohlraum_q) through the
C ABI against the CPU oracle, on the hohlraum-like layout.

Coefficients: sigma_t exact, sigma_s to 1e-14 relative; q to 1e-13 of the emission term
4 pi sigma a c T^4 (the oracle evaluates the printed difference of two terms, which loses digits
when sigma_s is close to sigma; the library evaluates the combined form).  Sweeps 1e-12 relative;
converged solutions 1e-9.
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle.dsa import thick_mask

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


def _set(mesh, x, device):
    args = [x["sigma"], x["cv"], x["T"]]
    if device:
        args = [torch.as_tensor(a, device="cuda") for a in args]
    mesh.set_pseudo_scattering(*args, x["dt"], x["a_rad"], x["c_light"])


@pytest.mark.parametrize("device", [False, True])
def test_coefficients_match_the_oracle(sn, device):
    from oracle.pseudo import pseudo_scattering
    prob = inputs.hohlraum_like(48, p=1, sn=4)
    x = prob.extra
    m = sn.Mesh.from_problem(prob)
    _set(m, x, device)
    st, ss, q = m.materials()
    rst, rss, rq = pseudo_scattering(x["sigma"], x["cv"], x["T"], x["dt"], x["a_rad"], x["c_light"])
    assert np.array_equal(st, rst)
    assert np.all(np.abs(ss - rss) <= 1e-14 * rss)
    emission = 4 * np.pi * x["sigma"] * x["a_rad"] * x["c_light"] * x["T"] ** 4
    assert np.all(np.abs(q - rq) <= 1e-13 * emission)
    assert np.array_equal(ss >= 1.0, x["T"] == inputs.HOHLRAUM_T_HOT)  # thick = laser-heated gold


def test_sweep_and_solution_match_the_oracle(sn):
    from oracle import Transport
    from oracle.dsa import DSA
    from oracle.pseudo import problem
    lay = inputs.hohlraum_like(32, p=1, sn=4)
    prob = problem(lay)
    T = Transport(prob)
    m = sn.Mesh.from_problem(lay)
    _set(m, lay.extra, False)
    phi = inputs.random_phi(prob, 41) * 1e5
    got = m.sweep(torch.as_tensor(phi, device="cuda")).cpu().numpy()
    assert _rel(got, T.sweep(phi)) < 1e-12
    # 1e-12: the source spans eleven decades (hot gold against cold helium), and the oracle's
    # float64 residual stalls just below that
    r = m.source_iterate(dsa="thick", outer="fgmres", tol=1e-12, inner_tol=1e-10, max_iters=400)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-12, max_iters=200)
    assert r["converged"] and ref["converged"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-9


def test_uniform_temperature_stays_in_equilibrium_on_the_gpu(sn):
    """Hot gold everywhere with the equilibrium intensity a c T^4 flowing in: phi = 4 pi a c T^4."""
    a, c, Tk = inputs.HOHLRAUM_A_RAD, inputs.HOHLRAUM_C_LIGHT, inputs.HOHLRAUM_T_HOT
    prob = inputs.uniform_problem(2, 8, 2, 4, 1.0, 0.0, 0.0, psi_inc=a * c * Tk ** 4)
    m = sn.Mesh.from_problem(prob)
    ne = prob.n_elem
    m.set_pseudo_scattering(np.full(ne, 1e3), np.full(ne, 1e5), np.full(ne, Tk), 1e-3, a, c)
    r = m.source_iterate(dsa="thick", outer="fgmres", tol=1e-13, inner_tol=1e-10, max_iters=400)
    assert r["converged"] and r["inner_iters"] > 0
    expect = 4 * np.pi * a * c * Tk ** 4
    assert np.abs(r["phi"].cpu().numpy() - expect).max() < 1e-11 * expect


def test_argument_errors(sn):
    prob = inputs.uniform_problem(2, 4, 1, 4, 1.0, 0.0, 0.0)
    m = sn.Mesh.from_problem(prob)
    ne = prob.n_elem
    one = np.ones(ne)
    for sigma, cv, T, dt in ((one, 0 * one, one, 1.0), (one, one, -one, 1.0), (-one, one, one, 1.0),
                             (one, one, one, 0.0), (one, one, one * np.nan, 1.0)):
        with pytest.raises(sn.SnError) as e:
            m.set_pseudo_scattering(sigma, cv, T, dt)
        assert e.value.status == 1
    st, ss, q = m.materials()  # a refused call leaves the materials alone
    assert np.all(st == 1.0) and np.all(ss == 0.0) and np.all(q == 0.0)


def test_vanishing_heat_capacity_term_and_overflow(sn):
    """C_v/dt underflowing to 0 is the long-step limit sigma_ps = sigma (Eq. hohlraum_sigma): it is
    accepted with sigma_s = sigma_t; a temperature whose sigma b overflows is refused by name."""
    prob = inputs.uniform_problem(2, 4, 1, 4, 1.0, 0.0, 0.0)
    m = sn.Mesh.from_problem(prob)
    ne = prob.n_elem
    sigma = np.linspace(0.5, 3e3, ne)
    m.set_pseudo_scattering(sigma, np.full(ne, 1e-300), np.full(ne, 0.4), 1e300)
    st, ss, q = m.materials()
    assert np.all(st == sigma) and np.all(ss <= st) and np.all(np.abs(ss - st) <= 2e-16 * st)
    assert np.all(q == 0.0)
    with pytest.raises(sn.SnError, match="overflows") as e:
        m.set_pseudo_scattering(np.ones(ne), np.ones(ne), np.full(ne, 1e120), 1.0)
    assert e.value.status == 1
    assert np.array_equal(m.materials()[0], st)
