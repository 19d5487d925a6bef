"""GPU: the thick-DSA PCG recorded as a CUDA graph with a device-side convergence loop.

The solve must agree with a sparse direct solve of the oracle's D_ff, stop by the tolerance it
was recorded for (a new tolerance records a new graph), report its iterations, and leave a zero
right-hand side alone.
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


@pytest.fixture(scope="module")
def case():
    import scipy.sparse.linalg as spla
    from oracle import Transport
    from oracle.dsa import DSA
    prob = inputs.config2(n=32, block=8)
    T = Transport(prob)
    op = DSA(T, thick_mask(prob))
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


def _true_residual(op, b, x):
    """||b_f - D_ff x_f|| / ||b_f|| with the oracle's operator in float64 on the host."""
    D = op.nodal_matrix()
    bf = b[op.thick].ravel()
    xf = x.cpu().numpy()[op.thick].ravel()
    return float(np.linalg.norm(bf - D @ xf) / np.linalg.norm(bf))


@pytest.mark.parametrize("operator", ["sip", "nip"])
def test_float32_vcycle_preconditions_to_tight_tolerances(sn, case, operator):
    """The float32 V-cycle is only the preconditioner: the float64 Krylov residual still reaches
    1e-11, in about as many iterations as with the float64 V-cycle."""
    import scipy.sparse.linalg as spla
    from oracle.dsa import DSA
    prob, b, ref, op = case
    if operator != "sip":
        op = DSA(op.T, thick_mask(prob), operator=operator)
        ref = np.zeros_like(b)
        ref[op.thick] = spla.spsolve(op.nodal_matrix().tocsc(), b[op.thick].ravel()).reshape(-1, op.T.n)
    m = sn.Mesh.from_problem(prob)
    bt = torch.as_tensor(b, device="cuda")
    kw = dict(thick_rule=prob.thick_rule, operator=operator, inner_tol=1e-11, inner_max_iters=500)
    x32, it32 = m.dsa_solve(bt, vcycle="fp32", **kw)
    x64, it64 = m.dsa_solve(bt, vcycle="fp64", **kw)
    assert it32 < 500 and it32 <= 1.5 * it64 + 2
    assert _true_residual(op, b, x32) < 2e-11 and _true_residual(op, b, x64) < 2e-11
    assert _rel(x32, ref) < 1e-8


def test_auto_vcycle_is_float32_for_loose_and_float64_for_tight_tolerances(sn, case):
    prob, b, _, _ = case
    m = sn.Mesh.from_problem(prob)
    bt = torch.as_tensor(b, device="cuda")
    kw = dict(thick_rule=prob.thick_rule, inner_max_iters=500)
    loose = {v: m.dsa_solve(bt, vcycle=v, inner_tol=1e-4, **kw)[0].clone() for v in ("auto", "fp32", "fp64")}
    assert torch.equal(loose["auto"], loose["fp32"]) and not torch.equal(loose["auto"], loose["fp64"])
    tight = {v: m.dsa_solve(bt, vcycle=v, inner_tol=1e-10, **kw)[0].clone() for v in ("auto", "fp32", "fp64")}
    assert torch.equal(tight["auto"], tight["fp64"]) and not torch.equal(tight["auto"], tight["fp32"])


def test_float32_vcycle_leaves_the_fixed_point_alone(sn):
    """With the paper's loose inner tolerance (float32 V-cycle) fGMRES reaches the oracle's solution."""
    from oracle import Transport
    from oracle.dsa import DSA
    prob = inputs.config1()
    T = Transport(prob)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", outer="fgmres", tol=1e-12, inner_tol=1e-4, max_iters=400)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-13, max_iters=400)
    assert r["converged"] and r["inner_iters"] > 0
    assert np.abs(r["phi"].cpu().numpy() - ref["phi"]).max() < 1e-9 * np.abs(ref["phi"]).max()


@pytest.mark.parametrize("outer", ["si", "fgmres"])
def test_solves_report_sweep_and_dsa_device_time(sn, outer):
    """sn_iter_stats splits a solve's device time into transport updates and DSA solves (host loop)."""
    prob = inputs.config1()
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", outer=outer, tol=1e-8, max_iters=300, host_loop=True)
    assert r["converged"] and r["ms_sweep"] > 0 and r["ms_dsa"] > 0
    assert r["ms_sweep"] + r["ms_dsa"] <= r["ms"] * 1.02 + 0.1
    n = m.source_iterate(dsa="none", outer=outer, tol=1e-3, max_iters=60, host_loop=True)
    assert n["ms_dsa"] == 0 and n["ms_sweep"] > 0
    g = torch.ones(m.shape, dtype=torch.float64, device="cuda")
    a = m.adjoint_iterate(g, dsa="thick", outer=outer, tol=1e-8, max_iters=300)
    assert a["converged"] and a["ms_sweep"] > 0 and a["ms_dsa"] > 0 and a["sweeps"] > 0
