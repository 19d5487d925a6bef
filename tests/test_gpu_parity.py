"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances (float64 path): 1e-12 relative to the largest |value| of the oracle's result, the
bar the method sets for the FP64 form; 1e-5 for the FP32 element-solve form.  DSA-accelerated
iterates use the derived tolerance of tests/tolerances.py (the bar, widened by the rounding
amplification c/(1-c) of the DSA step only where that exceeds it).
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle.dsa import thick_mask
from tolerances import BAR, dsa_iterate_tol, fp32_fixed_point_tol, FP32_BAR

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
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300))


def ragged_problem():
    nx, ny = 13, 7
    ne = nx * ny
    st, ss = inputs.random_fields(ne, 4242)
    q = np.where(np.arange(ne) % 5 == 0, 1.0, 0.25)
    return inputs.Problem("ragged_13x7_q1_s6", 2, nx, ny, 1, 1, 6, st, ss, q, psi_inc=0.3)


SWEEP_CASES = {
    "c1": inputs.config1,
    "c2_32": lambda: inputs.config2(n=32, block=8),
    "c3_8": lambda: inputs.config3(n=8),
    "q3_s6": lambda: inputs.config2d_fields(12, 3, 6, 77, "q3"),
    "ragged": ragged_problem,
}


@pytest.fixture(scope="module")
def oracle_cache():
    return {}


def _oracle(name, cache):
    from oracle import Transport
    if name not in cache:
        prob = SWEEP_CASES[name]()
        cache[name] = (prob, Transport(prob))
    return cache[name]


def test_quadrature_matches_oracle(sn):
    from oracle.quadrature import level_symmetric
    for dim in (2, 3):
        for N in (4, 6, 8):
            m = sn.Mesh(dim, 2, 2, 2, 1, N)
            d, w = m.quadrature()
            od, ow = level_symmetric(N, dim)
            assert np.abs(d - od).max() < 1e-15 and np.abs(w - ow).max() < 1e-14


@pytest.mark.parametrize("name", list(SWEEP_CASES))
def test_sweep_fp64_parity(sn, oracle_cache, name):
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    phi = inputs.random_phi(prob, 11)
    got = m.sweep(_t(phi)).cpu().numpy()
    ref = T.sweep(phi)
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_sweep_fp32_forms(sn, oracle_cache, name):
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    phi = inputs.random_phi(prob, 12)
    ref = T.sweep(phi)
    assert _rel(m.sweep(_t(phi), precision="fp32").cpu().numpy(), ref) < 1e-5
    assert _rel(m.sweep(_t(phi), precision="fp32_refine").cpu().numpy(), ref) < 1e-12


def test_angular_flux_satisfies_the_oracle_element_equations(sn, oracle_cache):
    """psi_d of one GPU sweep, converted to the oracle's modal basis, solves the oracle's own
    element systems with the GPU's upwind traces (checked for every element and direction)."""
    prob, T = _oracle("c2_32", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    phi = inputs.random_phi(prob, 13)
    m.sweep(_t(phi))
    src = T.isotropic_source(T.to_modal(phi))
    for d in range(0, T.nd, 7):
        psi = T.to_modal(m.angular_flux(d).cpu().numpy())
        fw = T.face_flux(d)
        A = T.element_matrices(d, fw)
        rhs = np.einsum("emn,en->em", T.M, src)
        for f in range(4):
            inflow = (fw[f].sum(axis=1) < 0) & (T.mesh.nbr[:, f] >= 0)
            E = np.flatnonzero(inflow)
            trace = psi[T.mesh.nbr[E, f]] @ T.BFo[f].T
            rhs[E] -= np.einsum("eq,qm,eq->em", fw[f][E], T.BF[f], trace)
        res = np.einsum("emn,en->em", A, psi) - rhs
        assert np.abs(res).max() < 1e-12 * np.abs(rhs).max()


def test_iterate_parity_no_dsa(sn, oracle_cache):
    prob, T = _oracle("c1", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    K = 15
    r = m.source_iterate(dsa="none", tol=0.0, max_iters=K)
    ref = T.source_iterate(tol=0.0, max_iters=K)
    assert r["iters"] == K and not r["converged"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-12


@pytest.mark.parametrize("name,dsa", [("c1", "thick"), ("c2_32", "thick"), ("c3_8", "thick")])
def test_iterate_parity_with_dsa(sn, oracle_cache, name, dsa):
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    rule = prob.thick_rule
    K = 6
    r = m.source_iterate(dsa=dsa, thick_rule=rule, tol=0.0, max_iters=K, inner_tol=1e-14, inner_max_iters=500)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=0.0, max_iters=K)
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) <= dsa_iterate_tol(prob, thick_mask(prob))


def _c2_with_thick_ratio(c):
    prob = inputs.config2(n=32, block=8)
    thick = prob.sigma_t == 1.0e3
    prob.sigma_s[thick] = c * prob.sigma_t[thick]
    return prob


def test_dsa_iterate_gap_is_rounding_amplification(sn, oracle_cache):
    """Reading of the iterate tolerance: on configuration 2 the gap between library and oracle
    iterates comes from the DSA step amplifying rounding differences by c/(1-c), not from the
    inexact inner solve.  (1) The inner solve itself matches a sparse direct solve to 1e-13.
    (2) The iterate gap does not shrink when the inner tolerance drops from 1e-12 to 1e-15.
    (3) With the thick blocks' c lowered from 0.9999 to 0.99 (c/(1-c) from 9999 to 99) the same
    iterates meet the 1e-12 bar."""
    import scipy.sparse.linalg as spla
    from oracle import Transport
    from oracle.dsa import DSA
    prob, T = _oracle("c2_32", oracle_cache)
    op = DSA(T, thick_mask(prob))
    m = sn.Mesh.from_problem(prob)
    b = inputs.random_phi(prob, 23)
    x, _ = m.dsa_solve(_t(b), thick_rule=prob.thick_rule, inner_tol=1e-15, inner_max_iters=2000, vcycle="fp64")
    ref = np.zeros_like(b)
    ref[op.thick] = spla.spsolve(op.nodal_matrix().tocsc(), b[op.thick].ravel()).reshape(-1, T.n)
    assert _rel(x.cpu().numpy(), ref) < 1e-13
    K = 6
    ref_k = T.source_iterate(dsa=op, tol=0.0, max_iters=K)["phi"]
    gaps = [_rel(m.source_iterate(dsa="thick", tol=0.0, max_iters=K, inner_tol=t, inner_max_iters=2000,
                                  vcycle="fp64")["phi"].cpu().numpy(), ref_k) for t in (1e-12, 1e-15)]
    assert gaps[1] > gaps[0] / 3.0
    low = _c2_with_thick_ratio(0.99)
    T2 = Transport(low)
    m2 = sn.Mesh.from_problem(low)
    r2 = m2.source_iterate(dsa="thick", tol=0.0, max_iters=K, inner_tol=1e-15, inner_max_iters=2000, vcycle="fp64")
    ref2 = T2.source_iterate(dsa=DSA(T2, thick_mask(low)), tol=0.0, max_iters=K)["phi"]
    assert dsa_iterate_tol(low, thick_mask(low)) == BAR
    assert _rel(r2["phi"].cpu().numpy(), ref2) <= BAR


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_fp32_refine_iterates(sn, oracle_cache, name):
    """FP32 element solves with float64 residual corrections: the DSA-accelerated iterates match
    the oracle's float64 iterates to the float64 tolerance."""
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    K = 6
    r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, tol=0.0, max_iters=K, inner_tol=1e-14,
                         inner_max_iters=500, precision="fp32_refine")
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=0.0, max_iters=K)
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) <= dsa_iterate_tol(prob, thick_mask(prob))


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_fp32_mixed_refinement_reaches_the_fp64_fixed_point(sn, oracle_cache, name):
    """SN_FP32_MIXED: float32 element solves in every Arnoldi step, a float64 true residual between
    restart cycles.  It converges to the float64 fixed point (same bound as float64 fGMRES to the
    same tolerance), which plain float32 solves cannot reach on configuration 2."""
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, outer="fgmres", restart=30, tol=1e-13,
                         inner_tol=1e-10, max_iters=600, precision="fp32_mixed")
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-14, max_iters=3000)
    assert r["converged"] and r["rel_residual"] <= 1e-13
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-9
    r64 = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, outer="fgmres", restart=30, tol=1e-13,
                           inner_tol=1e-10, max_iters=600)
    assert _rel(r["phi"].cpu().numpy(), r64["phi"].cpu().numpy()) < 1e-9


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_fp32_iteration_against_the_fp64_fixed_point(sn, oracle_cache, name):
    """The FP32 element-solve form (float64 flux, residual and DSA) iterated by fGMRES to the
    residual float32 solves can reach, against the oracle's float64 fixed point: within 1e-5 where
    the scattering ratio leaves the fixed point well conditioned (configurations 1 and 3); on
    configuration 2, whose c = 0.9999 blocks amplify the float32 perturbation by up to c/(1-c),
    within the derived bound (measured 4e-5, above the 1e-5 target)."""
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, outer="fgmres", tol=1e-6, inner_tol=1e-10,
                         max_iters=400, precision="fp32")
    fixed = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-14, max_iters=3000)["phi"]
    assert r["converged"]
    err = _rel(r["phi"].cpu().numpy(), fixed)
    assert err <= fp32_fixed_point_tol(prob)
    if name != "c2_32":
        assert err <= FP32_BAR


def test_converged_solution_c1(sn, oracle_cache):
    from oracle.dsa import DSA
    prob, T = _oracle("c1", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", tol=1e-8, inner_tol=1e-12)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-8)
    assert r["converged"] and r["iters"] == ref["iters"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) <= dsa_iterate_tol(prob, thick_mask(prob))


def test_full_dsa_rejects_voids(sn, oracle_cache):
    prob, _ = _oracle("c1", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    with pytest.raises(sn.SnError) as e:
        m.source_iterate(dsa="full", max_iters=2)
    assert e.value.status == 5


def test_full_dsa_parity_void_free(sn):
    from oracle import Transport
    from oracle.dsa import DSA
    prob = inputs.config1()
    v = prob.sigma_t == 0
    prob.sigma_t[v], prob.sigma_s[v] = 1.0, 0.9
    T = Transport(prob)
    m = sn.Mesh.from_problem(prob)
    K = 5
    r = m.source_iterate(dsa="full", tol=0.0, max_iters=K, inner_tol=1e-14, inner_max_iters=500)
    ref = T.source_iterate(dsa=DSA(T, np.ones(T.ne)), tol=0.0, max_iters=K)
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) <= dsa_iterate_tol(prob, np.ones(T.ne))


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_dsa_operator_parity(sn, oracle_cache, name):
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    mask = thick_mask(prob).astype(bool)
    op = DSA(T, mask)
    Dn = op.nodal_matrix()
    x = inputs.random_phi(prob, 21) - 1.0
    y = m.dsa_apply(_t(x), thick_rule=prob.thick_rule).cpu().numpy()
    ref = np.zeros_like(x)
    ref[op.thick] = (Dn @ x[op.thick].ravel()).reshape(-1, T.n)
    assert _rel(y, ref) < 1e-12


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_dsa_pcg_solve(sn, oracle_cache, name):
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    op = DSA(T, thick_mask(prob))
    b = inputs.random_phi(prob, 22)
    x, its = m.dsa_solve(_t(b), thick_rule=prob.thick_rule, inner_tol=1e-13, inner_max_iters=1000)
    ref = np.zeros_like(b)
    import scipy.sparse.linalg as spla
    ref[op.thick] = spla.spsolve(op.nodal_matrix().tocsc(), b[op.thick].ravel()).reshape(-1, T.n)
    assert its < 200
    assert _rel(x.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_adjoint_sweep_parity(sn, oracle_cache, name):
    from oracle import adjoint
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    mu = inputs.random_phi(prob, 31) - 0.75
    got = m.adjoint_sweep(_t(mu)).cpu().numpy()
    ref = adjoint.adjoint_sweep(T, mu)
    assert _rel(got, ref) < 1e-12


def test_adjoint_dot_product_on_gpu(sn, oracle_cache):
    prob, _ = _oracle("c2_32", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    x = _t(inputs.random_phi(prob, 41) - 1.0)
    y = _t(inputs.random_phi(prob, 42) - 1.0)
    zero = torch.zeros_like(x)
    Tx = m.sweep(x) - m.sweep(zero)
    Aty = m.adjoint_sweep(y)
    lhs, rhs = float((y * Tx).sum()), float((Aty * x).sum())
    assert abs(lhs - rhs) < 1e-12 * float(y.norm() * Tx.norm())


def test_gradients_parity(sn):
    from oracle import Transport, adjoint
    from oracle.dsa import DSA
    prob = inputs.config2d_fields(8, 1, 4, 5150, "grad")
    prob.q[:] = 1.0
    det = np.zeros(prob.n_elem, dtype=np.uint8)
    det[[6, 7, 14, 15]] = 1
    T = Transport(prob)
    ref_phi = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-15, max_iters=3000)["phi"]
    g_m = adjoint.detector_modal(T, det)
    mu_m, _, _ = adjoint.adjoint_iterate(T, g_m, dsa=DSA(T, thick_mask(prob)), tol=1e-15)
    gt, gs, gq = adjoint.gradients(T, ref_phi, mu_m)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", tol=1e-14, inner_tol=1e-13, inner_max_iters=500)
    # nodal detector g = M 1_strip; mu (nodal) satisfies mu_m = V^T mu_n
    g_n = np.linalg.solve(T.V.T, g_m.T).T
    a = m.adjoint_iterate(_t(g_n), dsa="thick", tol=1e-14, inner_tol=1e-13, inner_max_iters=500)
    assert np.abs(a["mu"].cpu().numpy() @ T.V - mu_m).max() < 1e-9 * np.abs(mu_m).max()
    Gt, Gs, Gq = (x.cpu().numpy() for x in m.gradients(r["phi"], a["mu"]))
    for got, ref in ((Gt, gt), (Gs, gs), (Gq, gq)):
        assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_fgmres_reaches_the_oracle_fixed_point(sn, oracle_cache, name):
    """fGMRES (the paper's outer solver) converges to the same discrete solution as source iteration."""
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, outer="fgmres", restart=30, tol=1e-13,
                         inner_tol=1e-10, max_iters=400)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-14, max_iters=2000)
    assert r["converged"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-9
    si = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, tol=1e-13, inner_tol=1e-10, max_iters=2000)
    assert r["iters"] <= si["iters"]


@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_8"])
def test_iterate_parity_triangular_dsa(sn, oracle_cache, name):
    """Algorithm 1 (triangular heterogeneous DSA) iterates match the oracle's."""
    from oracle.dsa import DSA, TriangularDSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    K = 5
    r = m.source_iterate(dsa="triangular", thick_rule=prob.thick_rule, tol=0.0, max_iters=K, inner_tol=1e-14,
                         inner_max_iters=500)
    ref = T.source_iterate(dsa=TriangularDSA(DSA(T, thick_mask(prob))), tol=0.0, max_iters=K)
    assert r["sweeps"] == 2 * K
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) <= dsa_iterate_tol(prob, thick_mask(prob))


@pytest.mark.parametrize("name", ["c1", "c2_32"])
def test_fgmres_triangular_dsa_reaches_the_oracle_fixed_point(sn, oracle_cache, name):
    from oracle.dsa import DSA
    prob, T = _oracle(name, oracle_cache)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="triangular", thick_rule=prob.thick_rule, outer="fgmres", restart=30, tol=1e-13,
                         inner_tol=1e-10, max_iters=400)
    ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-14, max_iters=2000)
    assert r["converged"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-9


def test_fgmres_with_boundary_inflow(sn, oracle_cache):
    """The Krylov operator is the linear part of the update (no fixed source, vacuum inflow): with
    nonzero boundary inflow fGMRES still reaches the fixed point of source iteration."""
    prob, T = _oracle("ragged", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="none", outer="fgmres", restart=20, tol=1e-13, max_iters=400)
    ref = T.source_iterate(tol=1e-14, max_iters=4000)
    assert r["converged"] and ref["converged"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-10


def test_triangular_dsa_is_rejected_where_unsupported(sn, oracle_cache):
    prob, _ = _oracle("c1", oracle_cache)
    m = sn.Mesh.from_problem(prob)
    g = torch.ones(m.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(sn.SnError) as e:
        m.adjoint_iterate(g, dsa="triangular", max_iters=2)
    assert e.value.status == 1
    b = sn.Batch([m])
    with pytest.raises(sn.SnError) as e:
        b.source_iterate(dsa="triangular", max_iters=2)
    assert e.value.status == 1
