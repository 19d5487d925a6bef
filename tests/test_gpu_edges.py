"""GPU parity on the degenerate cases of the method: a single element, one-element-wide strips,
all-void media (pure streaming, with and without boundary inflow), a DSA request with no thick
element, and 3D counterparts.  Tolerances as in the other parity tests."""
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
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _problem(dim, nx, ny, nz, p, sn_order, st, ss, q, psi_inc=0.0, name="edge"):
    ne = nx * ny * (nz if dim == 3 else 1)
    full = lambda v: np.full(ne, float(v)) if np.isscalar(v) else np.asarray(v, dtype=np.float64)
    return inputs.Problem(name, dim, nx, ny, nz if dim == 3 else 1, p, sn_order, full(st), full(ss), full(q),
                          psi_inc=psi_inc)


CASES = {
    "one_q1": lambda: _problem(2, 1, 1, 1, 1, 4, 2.0, 1.0, 1.0),
    "one_q3_inflow": lambda: _problem(2, 1, 1, 1, 3, 6, 0.5, 0.2, 0.0, psi_inc=0.8),
    "strip_x": lambda: _problem(2, 17, 1, 1, 2, 8, 1.5, 1.2, 1.0, psi_inc=0.1),
    "strip_y": lambda: _problem(2, 1, 11, 1, 2, 4, 3.0, 0.5, 2.0),
    "void": lambda: _problem(2, 9, 7, 1, 2, 6, 0.0, 0.0, 1.0),
    "void_inflow": lambda: _problem(2, 6, 6, 1, 1, 8, 0.0, 0.0, 0.0, psi_inc=1.0),
    "one_3d": lambda: _problem(3, 1, 1, 1, 1, 4, 1.0, 0.5, 1.0, psi_inc=0.3),
    "void_3d": lambda: _problem(3, 4, 3, 5, 1, 6, 0.0, 0.0, 1.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cache", ["on", "off"])
def test_degenerate_sweeps_match_the_oracle(sn, name, cache):
    from oracle import Transport
    prob = CASES[name]()
    T = Transport(prob)
    m = sn.Mesh.from_problem(prob)
    m.set_operator_cache(cache)
    phi = inputs.random_phi(prob, 300)
    ref = T.sweep(phi)
    assert _rel(m.sweep(torch.as_tensor(phi, device="cuda")), ref) < 1e-12
    assert _rel(m.sweep(torch.as_tensor(phi, device="cuda"), precision="fp32"), ref) < 1e-5


def test_void_streaming_is_exact(sn):
    """In a void (sigma_t = sigma_s = 0) with constant inflow psi_inc and no source, every angular
    flux equals psi_inc and phi = 4 pi psi_inc exactly representable: the sweep reproduces it."""
    prob = CASES["void_inflow"]()
    m = sn.Mesh.from_problem(prob)
    out = m.sweep(torch.zeros(m.shape, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.abs(out - 4 * np.pi * prob.psi_inc).max() < 1e-12 * 4 * np.pi


def test_dsa_without_thick_elements_is_plain_source_iteration(sn):
    prob = _problem(2, 8, 8, 1, 1, 4, 1.0, 0.5, 1.0)  # sigma_s < 1 everywhere: no thick element
    m = sn.Mesh.from_problem(prob)
    a = m.source_iterate(dsa="thick", tol=0.0, max_iters=6)
    b = m.source_iterate(dsa="none", tol=0.0, max_iters=6)
    assert a["thick_fraction"] == 0.0 and a["inner_iters"] == 0
    assert torch.equal(a["phi"], b["phi"])
    t = m.source_iterate(dsa="triangular", tol=0.0, max_iters=6)
    assert torch.equal(t["phi"], b["phi"])


def test_single_element_solution_matches_the_oracle(sn):
    from oracle import Transport
    from oracle.dsa import DSA
    prob = _problem(2, 1, 1, 1, 2, 8, 5.0, 4.5, 1.0)  # thick (sigma_s >= 1): DSA on one element
    T = Transport(prob)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", tol=1e-12, inner_tol=1e-13, max_iters=200)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-13, max_iters=400)
    assert r["converged"] and _rel(r["phi"], ref["phi"]) < 1e-10
