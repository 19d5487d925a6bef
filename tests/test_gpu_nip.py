"""GPU parity of the nonsymmetric DSA operators (Sec. 3.1: Eq. NIP, and Eq. NIP with the penalty
of Eq. ModifiedF0) and their BiCGStab solves, through the C ABI, against the CPU oracle.

Tolerances as for the symmetric operator: 1e-12 relative for operator products, 1e-9 for solves
to a 1e-13 inner tolerance and for converged solutions, and for a fixed number of iterates with
1e-14 inner solves the derived tolerance of tests/tolerances.py (1e-12, widened by the DSA step's
rounding amplification c/(1-c) where that exceeds it).
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle.dsa import thick_mask
from tolerances import dsa_iterate_tol

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


def ragged_q2():
    nx, ny = 13, 7
    st, ss = inputs.random_fields(nx * ny, 4244)
    q = np.where(np.arange(nx * ny) % 4 == 0, 1.0, 0.3)
    return inputs.Problem("ragged_13x7_q2_s4", 2, nx, ny, 1, 2, 4, st, ss, q, psi_inc=0.4, thick_rule="sigma_t_h")


def void_free_c3():
    prob = inputs.config3(n=6)
    v = prob.sigma_t == 0
    prob.sigma_t[v], prob.sigma_s[v] = 1.0, 0.5
    prob.q[:] = 1.0  # the source block of the 64^3 layout is empty at this size
    return prob


CASES = {
    "c1": inputs.config1,
    "c2_32": lambda: inputs.config2(n=32, block=8),
    "c3_8": lambda: inputs.config3(n=8),
    "c3_6_void_free": void_free_c3,
    "ragged_q2": ragged_q2,
}


@pytest.fixture(scope="module")
def cache():
    return {}


def _case(name, cache):
    from oracle import Transport
    if name not in cache:
        prob = CASES[name]()
        cache[name] = (prob, Transport(prob), {})
    return cache[name]


def _dsa(name, cache, op):
    """The oracle's operator, or None where it is undefined (mNIP next to a void)."""
    from oracle.dsa import DSA
    prob, T, ops = _case(name, cache)
    if op not in ops:
        try:
            ops[op] = DSA(T, thick_mask(prob), operator=op)
        except ValueError:
            ops[op] = None
    return ops[op]


@pytest.mark.parametrize("op", ["nip", "mnip"])
@pytest.mark.parametrize("name", list(CASES))
def test_operator_parity(sn, cache, name, op):
    prob, T, _ = _case(name, cache)
    d = _dsa(name, cache, op)
    m = sn.Mesh.from_problem(prob)
    x = inputs.random_phi(prob, 31) - 1.0
    if d is None:  # Eq. ModifiedF0 is undefined next to a void element
        with pytest.raises(sn.SnError) as e:
            m.dsa_apply(_t(x), thick_rule=prob.thick_rule, operator=op)
        assert e.value.status == 5
        return
    y = m.dsa_apply(_t(x), thick_rule=prob.thick_rule, operator=op).cpu().numpy()
    ref = np.zeros_like(x)
    ref[d.thick] = (d.nodal_matrix() @ x[d.thick].ravel()).reshape(-1, T.n)
    assert _rel(y, ref) < 1e-12
    # the product differs from the symmetric operator's (the face terms are not the same)
    y_sip = m.dsa_apply(_t(x), thick_rule=prob.thick_rule, operator="sip").cpu().numpy()
    assert _rel(y_sip, ref) > 1e-6


@pytest.mark.parametrize("op", ["nip", "mnip"])
@pytest.mark.parametrize("name", list(CASES))
def test_bicgstab_solve(sn, cache, name, op):
    import scipy.sparse.linalg as spla
    prob, T, _ = _case(name, cache)
    d = _dsa(name, cache, op)
    if d is None:
        pytest.skip("operator undefined next to a void element")
    m = sn.Mesh.from_problem(prob)
    b = inputs.random_phi(prob, 32)
    x, its = m.dsa_solve(_t(b), thick_rule=prob.thick_rule, operator=op, inner_tol=1e-13, inner_max_iters=1000)
    ref = np.zeros_like(b)
    ref[d.thick] = spla.spsolve(d.nodal_matrix().tocsc(), b[d.thick].ravel()).reshape(-1, T.n)
    assert 0 < its < 200
    assert _rel(x.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("op", ["nip", "mnip"])
@pytest.mark.parametrize("name", ["c1", "c2_32", "c3_6_void_free", "ragged_q2"])
def test_iterate_parity(sn, cache, name, op):
    prob, T, _ = _case(name, cache)
    d = _dsa(name, cache, op)
    if d is None:
        pytest.skip("operator undefined next to a void element")
    m = sn.Mesh.from_problem(prob)
    K = 6
    r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, operator=op, tol=0.0, max_iters=K,
                         inner_tol=1e-14, inner_max_iters=1000)
    ref = T.source_iterate(dsa=d, tol=0.0, max_iters=K)
    assert r["iters"] == K and r["inner_iters"] > 0
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) <= dsa_iterate_tol(prob, thick_mask(prob))


@pytest.mark.parametrize("name", ["c1", "c3_8"])
def test_fgmres_with_nip_reaches_the_oracle_fixed_point(sn, cache, name):
    prob, T, _ = _case(name, cache)
    d = _dsa(name, cache, "nip")
    m = sn.Mesh.from_problem(prob)
    r = m.source_iterate(dsa="thick", thick_rule=prob.thick_rule, operator="nip", outer="fgmres", restart=30,
                         tol=1e-13, inner_tol=1e-10, max_iters=400)
    ref = T.source_iterate(dsa=d, tol=1e-14, max_iters=2000)
    assert r["converged"]
    assert _rel(r["phi"].cpu().numpy(), ref["phi"]) < 1e-9


@pytest.mark.parametrize("outer", ["si", "fgmres"])
def test_adjoint_with_nip_uses_the_transposed_operator(sn, outer):
    """K adjoint iterates with the transposed NIP step match the oracle's iterates (which use
    D_ff^{-T}); the converged adjoint matches the oracle's converged adjoint."""
    from oracle import Transport, adjoint
    from oracle.dsa import DSA
    prob = inputs.config2d_fields(8, 1, 4, 5150, "grad")
    prob.q[:] = 1.0
    det = np.zeros(prob.n_elem, dtype=np.uint8)
    det[[6, 7, 14, 15]] = 1
    T = Transport(prob)
    d = DSA(T, thick_mask(prob), operator="nip")
    assert d.thick.size
    g_m = adjoint.detector_modal(T, det)
    g_n = np.linalg.solve(T.V.T, g_m.T).T
    m = sn.Mesh.from_problem(prob)
    if outer == "si":
        K = 5
        mu_k, _, _ = adjoint.adjoint_iterate(T, g_m, dsa=d, tol=0.0, max_iters=K)
        a = m.adjoint_iterate(_t(g_n), dsa="thick", thick_rule=prob.thick_rule, operator="nip", tol=0.0,
                              max_iters=K, inner_tol=1e-14, inner_max_iters=1000)
        assert a["iters"] == K
        assert np.abs(a["mu"].cpu().numpy() @ T.V - mu_k).max() <= dsa_iterate_tol(prob, thick_mask(prob)) * np.abs(mu_k).max()
    mu_ref, _, _ = adjoint.adjoint_iterate(T, g_m, dsa=d, tol=1e-15)
    a = m.adjoint_iterate(_t(g_n), dsa="thick", thick_rule=prob.thick_rule, operator="nip", outer=outer,
                          tol=1e-14, inner_tol=1e-13, inner_max_iters=1000, max_iters=3000)
    assert a["converged"] and a["inner_iters"] > 0
    assert np.abs(a["mu"].cpu().numpy() @ T.V - mu_ref).max() < 1e-9 * np.abs(mu_ref).max()


def test_operator_switch_on_one_mesh(sn, cache):
    """sip -> nip -> mnip -> sip on one mesh: each solve uses the operator it asks for."""
    prob, T, _ = _case("c1", cache)
    m = sn.Mesh.from_problem(prob)
    b = inputs.random_phi(prob, 33)
    for op in ("sip", "nip", "mnip", "sip"):
        import scipy.sparse.linalg as spla
        d = _dsa("c1", cache, op)
        x, _ = m.dsa_solve(_t(b), operator=op, inner_tol=1e-13, inner_max_iters=1000)
        ref = np.zeros_like(b)
        ref[d.thick] = spla.spsolve(d.nodal_matrix().tocsc(), b[d.thick].ravel()).reshape(-1, T.n)
        assert _rel(x.cpu().numpy(), ref) < 1e-9, op


def test_batches_take_the_symmetric_operator_only(sn):
    probs = [inputs.config2d_fields(8, 1, 4, 61, "a"), inputs.config2d_fields(10, 2, 4, 62, "b")]
    batch = sn.Batch([sn.Mesh.from_problem(p) for p in probs])
    with pytest.raises(sn.SnError) as e:
        batch.source_iterate(dsa="thick", operator="nip", max_iters=2)
    assert e.value.status == 1
    with pytest.raises(sn.SnError):
        sn.Mesh.from_problem(probs[0]).source_iterate(dsa="thick", operator=7, max_iters=2)
