"""GPU: differentiable transport solve (torch.autograd.Function over libsn's adjoint).

Gradients of a detector functional J = sum over a strip of the integral of phi with respect to
per-element sigma_t, sigma_s and q are checked against the oracle's adjoint and, on the
128x128 Q1 S8 differentiation workload, against central finite differences with relative step
1e-6 on 32 seeded non-void elements.
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle.dsa import thick_mask

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09196_gb300 import build
    build.build()
    from paper_2001_09196_gb300 import autograd, sn
    return sn, autograd


def _detector_nodal(prob, strip):
    """g with g . phi = sum over strip elements of the integral of phi (uniform Cartesian mesh)."""
    x, w = np.polynomial.legendre.leggauss(prob.p + 1)
    W = np.outer(w, w).ravel()  # x fastest: W[a + Q b] = w_a w_b
    h = 1.0 / prob.nx
    g = np.zeros((prob.n_elem, prob.n_nodes))
    g[strip.astype(bool)] = W * (h / 2) ** 2
    return g


def test_autograd_matches_oracle_gradients(lib):
    sn, ag = lib
    from oracle import Transport, adjoint
    from oracle.dsa import DSA
    prob = inputs.config2d_fields(8, 1, 4, 5150, "grad")
    prob.q[:] = 1.0
    strip = np.zeros(prob.n_elem, dtype=np.uint8)
    strip[[6, 7, 14, 15]] = 1
    T = Transport(prob)
    phi_ref = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-15, max_iters=3000)["phi"]
    mu_m, _, _ = adjoint.adjoint_iterate(T, adjoint.detector_modal(T, strip), dsa=DSA(T, thick_mask(prob)), tol=1e-15)
    gt, gs, gq = adjoint.gradients(T, phi_ref, mu_m)
    mesh = sn.Mesh.from_problem(prob)
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    phi = ag.solve(mesh, st, ss, q, solve_opts=dict(thick_rule="sigma_t_h", tol=1e-14))
    g = torch.as_tensor(_detector_nodal(prob, strip), device="cuda")
    J = (g * phi).sum()
    J.backward()
    J_ref = float((T.to_modal(phi_ref) * adjoint.detector_modal(T, strip)).sum())
    assert abs(float(J) - J_ref) < 1e-12 * abs(J_ref)
    for got, ref in ((st.grad, gt), (ss.grad, gs), (q.grad, gq)):
        assert np.abs(got.cpu().numpy() - ref).max() < 1e-9 * np.abs(ref).max()


def test_source_iteration_checkpoints(lib):
    sn, ag = lib
    prob = inputs.config1()
    mesh = sn.Mesh.from_problem(prob)
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    phi = ag.solve(mesh, st, ss, q, solve_opts=dict(outer="si", tol=1e-10, max_iters=200), checkpoint_every=5)
    ck = ag.SnSolve.last_checkpoints
    assert ck is not None and ck.shape[0] >= 2
    # checkpoint k holds iterate 5(k+1): re-running that many iterations reproduces it exactly
    r = mesh.source_iterate(outer="si", dsa="thick", tol=0.0, max_iters=10, inner_tol=1e-10, inner_max_iters=500)
    assert torch.equal(r["phi"], ck[1])
    phi.sum().backward()
    assert torch.isfinite(st.grad).all() and torch.isfinite(q.grad).all()


def test_gradients_match_finite_differences_config5(lib):
    """Central differences (relative step 1e-6) of deterministic fixed-iteration solves.

    The finite-difference map is made smooth by fixing every iteration count (fGMRES iterations
    K, 40 PCG iterations per DSA solve), so J_K(p) is a differentiable function of the parameters.
    Each entry must satisfy |adjoint - FD(h)| <= 1e-6 |FD(h)| + 2 delta + nu + r, where
      * delta = |FD(h) - FD(2h)| measures the round-off noise of the difference (truncation of a
        central difference with relative step 1e-6 is ~1e-12 relative), and
      * nu = 1e-12 |J| / h is the resolution of a difference of an iteratively solved functional:
        a fixed-iteration Krylov map is not exactly linear in its data, so J differences below
        about 1e-13 |J| (observed) are artefacts of the solver, not of the discretisation, and
      * r = 1e-9 max_e |dJ/dp_e| is the resolution of the adjoint itself: mu is solved to a relative
        residual of 1e-14, i.e. accurately relative to its largest entries, not to tiny ones.
    Two seeded sets of 32 non-void elements are used: anywhere in the domain (there most
    sensitivities are 1e-14..1e-21 of J, far below nu, so FD only confirms they are tiny) and next
    to the detector.  There every q entry (relative sensitivity 1e2..1e4) is resolved
    (2 delta + nu + r <= 1e-6 |FD|) and so checked at 1e-6 relative, which is asserted; sigma
    entries (relative sensitivities 1e-5..1e-1) are resolved by a 1e-6 step only to ~1e-5.
    """
    sn, ag = lib
    prob = inputs.config5()
    strip = prob.extra["detector"]
    mask = thick_mask(prob)
    mesh = sn.Mesh.from_problem(prob)
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    tight = dict(mask=mask, tol=1e-14, inner_tol=1e-13, max_iters=400)
    phi = ag.solve(mesh, st, ss, q, solve_opts=tight, adjoint_opts=tight)
    g = torch.as_tensor(_detector_nodal(prob, strip), device="cuda")
    J0 = float((g * phi).sum().detach())
    (g * phi).sum().backward()
    mesh.set_materials(prob.sigma_t, prob.sigma_s, prob.q)
    probe = mesh.source_iterate(dsa="thick", mask=mask, outer="fgmres", tol=1e-14, inner_tol=1e-13, max_iters=400)
    K = probe["iters"] + 5

    def J_of(st_h, ss_h, q_h, k=K):
        mesh.set_materials(st_h, ss_h, q_h)
        r = mesh.source_iterate(dsa="thick", mask=mask, outer="fgmres", tol=0.0, max_iters=k, inner_tol=1e-300,
                                inner_max_iters=40)
        return float((g * r["phi"]).sum())

    base = [prob.sigma_t.copy(), prob.sigma_s.copy(), prob.q.copy()]
    JK = J_of(*base)
    assert abs(JK - J0) < 1e-8 * abs(J0)
    grads = [st.grad.cpu().numpy(), ss.grad.cpu().numpy(), q.grad.cpu().numpy()]

    def fd(e, idx, h):
        p = base[idx][e]
        plus = [a.copy() for a in base]
        plus[idx][e] += h
        if p - h >= 0:
            minus = [a.copy() for a in base]
            minus[idx][e] -= h
            return (J_of(*plus) - J_of(*minus)) / (2 * h)
        return (J_of(*plus) - JK) / h  # q = 0: J is linear in q, one-sided is exact up to round-off

    res = [1e-9 * np.abs(gr).max() for gr in grads]
    strict_q = 0
    for set_name in ("fd_elements", "fd_near"):
        for e in prob.extra[set_name]:
            for idx in range(3):
                p = base[idx][e]
                h = 1e-6 * abs(p) if p != 0 else 1e-6
                ga = grads[idx][e]
                nu = 1e-12 * abs(JK) / h
                f1 = fd(e, idx, h)
                floor = nu + res[idx]
                if abs(ga - f1) > 1e-6 * abs(f1) + floor or (set_name == "fd_near" and idx == 2):
                    f2 = fd(e, idx, 2 * h)  # the noise estimate is needed only when it matters
                    floor += 2 * abs(f1 - f2)
                assert abs(ga - f1) <= 1e-6 * abs(f1) + floor, (set_name, int(e), idx, ga, f1, floor)
                if set_name == "fd_near" and idx == 2:
                    strict_q += floor <= 1e-6 * abs(f1)
    mesh.set_materials(prob.sigma_t, prob.sigma_s, prob.q)
    assert strict_q == len(prob.extra["fd_near"]), strict_q


@pytest.mark.parametrize("case", ["jittered_q2", "q3"])
def test_gradients_match_the_oracle_adjoint_on_higher_order_meshes(lib, case):
    """Gradients of J = sum over a strip of the integral of phi with respect to per-element sigma_t,
    sigma_s and q (Sec. 1 transport system and its transpose): the library's autograd Function
    against the oracle's adjoint gradients, on a jittered Q2 mesh and on a Q3 mesh, both with the
    random per-element fields of configuration 3 (thick where sigma_t h > 1).  The detector in nodal coordinates is V^{-T} of the oracle's
    modal M 1_strip, so both sides differentiate the same discrete functional."""
    sn, ag = lib
    from oracle import Transport, adjoint
    from oracle.dsa import DSA
    if case == "jittered_q2":
        prob = inputs.config2d_fields(12, 2, 4, 5152, "grad_q2_jittered")
        prob.vertices = inputs.jittered_vertices(12, 12, 0.15, 5152)
    else:
        prob = inputs.config2d_fields(10, 3, 4, 5151, "grad_q3")
    prob.q[:] = np.maximum(prob.q, 0.5)
    opts = dict(thick_rule="sigma_t_h")
    strip = np.zeros(prob.n_elem, dtype=np.uint8)
    strip[np.arange(prob.n_elem) % prob.nx >= prob.nx - 2] = 1
    T = Transport(prob)
    d = DSA(T, thick_mask(prob))
    phi_ref = T.source_iterate(dsa=d, tol=1e-15, max_iters=4000)["phi"]
    g_m = adjoint.detector_modal(T, strip)
    mu_m, _, _ = adjoint.adjoint_iterate(T, g_m, dsa=d, tol=1e-15, max_iters=4000)
    gt, gs, gq = adjoint.gradients(T, phi_ref, mu_m)
    mesh = sn.Mesh.from_problem(prob)
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    tight = dict(opts, tol=1e-14, inner_tol=1e-13)
    phi = ag.solve(mesh, st, ss, q, solve_opts=tight, adjoint_opts=tight)
    g = torch.as_tensor(np.linalg.solve(T.V.T, g_m.T).T, device="cuda")
    J = (g * phi).sum()
    J.backward()
    J_ref = float((T.to_modal(phi_ref) * g_m).sum())
    assert abs(float(J.detach()) - J_ref) < 1e-11 * abs(J_ref)
    for got, ref in ((st.grad, gt), (ss.grad, gs), (q.grad, gq)):
        assert np.abs(got.cpu().numpy() - ref).max() < 1e-9 * np.abs(ref).max()
