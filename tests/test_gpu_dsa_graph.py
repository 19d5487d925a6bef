"""GPU: the thick-DSA PCG recorded as a CUDA graph with a device-side convergence loop.

The solve must agree with a sparse direct solve of the oracle's D_ff, stop by the tolerance it
was recorded for (a new tolerance records a new graph), report its iterations, and leave a zero
right-hand side alone.
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
def case():
    import scipy.sparse.linalg as spla
    from oracle import Transport
    from oracle.dsa import DSA
    prob = inputs.config2(n=32, block=8)
    T = Transport(prob)
    op = DSA(T, prob.thick_mask())
    b = inputs.random_phi(prob, 23)
    ref = np.zeros_like(b)
    ref[op.thick] = spla.spsolve(op.nodal_matrix().tocsc(), b[op.thick].ravel()).reshape(-1, T.n)
    return prob, b, ref, op


def _rel(got, ref):
    return float(np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max())


def test_recorded_pcg_follows_its_tolerance(sn, case):
    prob, b, ref, _ = case
    m = sn.Mesh.from_problem(prob)
    bt = torch.as_tensor(b, device="cuda")
    x_loose, it_loose = m.dsa_solve(bt, thick_rule=prob.thick_rule, inner_tol=1e-4, inner_max_iters=500)
    x_tight, it_tight = m.dsa_solve(bt, thick_rule=prob.thick_rule, inner_tol=1e-12, inner_max_iters=500)
    x_again, it_again = m.dsa_solve(bt, thick_rule=prob.thick_rule, inner_tol=1e-4, inner_max_iters=500)
    assert 0 < it_loose < it_tight < 500
    assert it_again == it_loose and torch.equal(x_again, x_loose)
    assert _rel(x_tight, ref) < 1e-10
    assert 1e-12 < _rel(x_loose, ref) < 1e-2


def test_recorded_pcg_stops_at_max_iters(sn, case):
    prob, b, _, _ = case
    m = sn.Mesh.from_problem(prob)
    _, its = m.dsa_solve(torch.as_tensor(b, device="cuda"), thick_rule=prob.thick_rule, inner_tol=1e-300,
                         inner_max_iters=3)
    assert its == 3


def test_recorded_pcg_zero_rhs(sn, case):
    prob, b, _, _ = case
    m = sn.Mesh.from_problem(prob)
    x, its = m.dsa_solve(torch.zeros(b.shape, dtype=torch.float64, device="cuda"), thick_rule=prob.thick_rule)
    assert its == 0 and float(x.abs().max()) == 0.0


def test_iterations_report_inner_pcg_counts(sn, case):
    prob, _, _, _ = case
    m = sn.Mesh.from_problem(prob)
    for outer in ("si", "fgmres"):
        r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, tol=0.0, max_iters=4, outer=outer, inner_tol=1e-6)
        assert r["inner_iters"] >= 4 * 2  # four DSA solves, each more than one PCG iteration at 1e-6
        r0 = m.source_iterate(dsa="none", tol=0.0, max_iters=4, outer=outer)
        assert r0["inner_iters"] == 0
