"""GPU: differentiable transport solve (torch.autograd.Function over libsn's adjoint).

Gradients of a detector functional J = sum over a strip of the integral of phi with respect to
per-element sigma_t, sigma_s and q: at the converged solution against the oracle's adjoint; through
K unaccelerated transport updates (iterate checkpointing) against the oracle's chain rule, against
their own limit K -> infinity, and on the 128x128 Q1 S8 differentiation workload against
Richardson-extrapolated central finite differences on 32 seeded elements next to the detector.
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


def _unrolled_problem(nx, p, seed, jitter=0.15):
    """Random fields without voids and with c <= 0.9, jittered vertices."""
    n = nx * nx
    st = 0.5 + 2.0 * inputs.uniform(seed, 50, n)
    ss = (0.3 + 0.6 * inputs.uniform(seed, 51, n)) * st
    q = 0.5 + inputs.uniform(seed, 52, n)
    return inputs.Problem(f"unrolled_{nx}_{p}", 2, nx, nx, 1, p, 4, st, ss, q,
                          vertices=inputs.jittered_vertices(nx, nx, jitter, seed))


@pytest.mark.parametrize("nx,p,K", [(8, 1, 5), (10, 2, 4)])
def test_unrolled_gradients_match_the_oracle(lib, nx, p, K):
    """Gradients of J = g^T phi_K through K unaccelerated transport updates (sn_unrolled_gradients:
    reverse accumulation with iterate checkpoints) against the oracle's chain rule through the same
    K updates (pinned by finite differences of its K-update map)."""
    sn, ag = lib
    from oracle import Transport, adjoint
    prob = _unrolled_problem(nx, p, 7300 + nx + p)
    T = Transport(prob)
    strip = (np.arange(prob.n_elem) % nx >= nx - 2).astype(np.uint8)
    g_m = adjoint.detector_modal(T, strip)
    ref = adjoint.unrolled_gradients(T, np.zeros((prob.n_elem, prob.n_nodes)), K, g_m)
    mesh = sn.Mesh.from_problem(prob)
    g = torch.as_tensor(np.ascontiguousarray(np.linalg.solve(T.V.T, g_m.T).T), device="cuda")
    got = mesh.unrolled_gradients(g, K, 2)
    for a, b in zip(got, ref):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-10 * np.abs(b).max()


def test_unrolled_checkpoint_spacings_and_autograd_agree(lib):
    """Every checkpoint spacing recomputes the same iterates, so the gradients agree bit for bit,
    whether the call keeps its own checkpoints or reads those of the forward source iteration; the
    autograd Function's backward pass returns the same gradients, and its forward value is the
    K-th iterate of the unaccelerated iteration."""
    sn, ag = lib
    prob = _unrolled_problem(12, 1, 7400)
    mesh = sn.Mesh.from_problem(prob)
    K = 7
    g = torch.as_tensor(inputs.random_phi(prob, 11), device="cuda")
    ref = mesh.unrolled_gradients(g, K, 1)
    for every in (2, 3, 7, 20):
        got = mesh.unrolled_gradients(g, K, every)
        assert all(torch.equal(a, b) for a, b in zip(got, ref)), every
        ck = torch.zeros((max(K // every, 1),) + mesh.shape, dtype=torch.float64, device="cuda")
        r = mesh.source_iterate(dsa="none", tol=0.0, max_iters=K, checkpoint_every=every, checkpoints=ck)
        assert r["iters"] == K
        got = mesh.unrolled_gradients(g, K, every, checkpoints=ck)
        assert all(torch.equal(a, b) for a, b in zip(got, ref)), every
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    phi_K = ag.unrolled(mesh, st, ss, q, K, checkpoint_every=3)
    x = torch.zeros(mesh.shape, dtype=torch.float64, device="cuda")
    for _ in range(K):
        x = mesh.sweep(x)
    assert torch.equal(phi_K.detach(), x)
    (g * phi_K).sum().backward()
    for a, b in zip((st.grad, ss.grad, q.grad), ref):
        assert torch.equal(a, b)


def test_unrolled_gradients_approach_the_fixed_point_gradients(lib):
    """With c <= 0.9 the unaccelerated iteration contracts, so the gradients of J(phi_K) tend to the
    gradients of J at the fixed point (sn_adjoint_iterate + sn_gradients, themselves checked against
    the oracle) as K grows."""
    sn, ag = lib
    prob = _unrolled_problem(8, 1, 7500)
    prob.sigma_s[:] = np.minimum(prob.sigma_s, 0.5 * prob.sigma_t)
    mesh = sn.Mesh.from_problem(prob)
    g = torch.as_tensor(inputs.random_phi(prob, 12), device="cuda")
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    phi = ag.solve(mesh, st, ss, q, solve_opts=dict(thick_rule="sigma_t_h", tol=1e-14))
    (g * phi).sum().backward()
    mesh.set_materials(prob.sigma_t, prob.sigma_s, prob.q)
    got = mesh.unrolled_gradients(g, 120, 12)
    for a, b in zip(got, (st.grad, ss.grad, q.grad)):
        assert float((a - b).abs().max()) <= 1e-10 * float(b.abs().max())


def test_unrolled_gradients_match_finite_differences_config5(lib):
    """Configuration 5 (128^2 Q1 S8, random fields, right-edge detector): the gradients of
    J_K = g^T phi_K, phi_K after K = 20 unaccelerated transport updates, with checkpoints every 5
    updates, against Richardson-extrapolated central differences (relative step 1e-3, and 2e-3),
    on the 32 seeded non-void elements next to the detector, every one of sigma_t, sigma_s and q
    within 1e-6 relative (q by a forward difference: J_K is affine in q).  J_K has no solver tolerance in it (a fixed number of updates, each
    deterministic), so its differences are limited by float64 rounding alone (~1e-15 |J| / h), and
    the extrapolation leaves a truncation of O(h^4).  The step of sigma_s (and of sigma_t) is
    capped at a quarter of sigma_t - sigma_s so that every perturbed material stays valid."""
    sn, ag = lib
    prob = inputs.config5()
    strip = prob.extra["detector"]
    mesh = sn.Mesh.from_problem(prob)
    K, every = 20, 5
    g = torch.as_tensor(_detector_nodal(prob, strip), device="cuda")
    st, ss, q = (torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                 for a in (prob.sigma_t, prob.sigma_s, prob.q))
    phi_K = ag.unrolled(mesh, st, ss, q, K, checkpoint_every=every)
    (g * phi_K).sum().backward()
    grads = [st.grad.cpu().numpy(), ss.grad.cpu().numpy(), q.grad.cpu().numpy()]
    base = [prob.sigma_t.copy(), prob.sigma_s.copy(), prob.q.copy()]

    def J_of(params):
        mesh.set_materials(*params)
        r = mesh.source_iterate(dsa="none", tol=0.0, max_iters=K)
        return float((g * r["phi"]).sum())

    def central(e, idx, h):
        vals = []
        for sign in (1.0, -1.0):
            pert = [a.copy() for a in base]
            pert[idx][e] += sign * h
            vals.append(J_of(pert))
        return (vals[0] - vals[1]) / (2 * h)

    J0 = J_of(base)
    for e in prob.extra["fd_near"]:
        margin = base[0][e] - base[1][e]
        for idx in range(2):
            h = 1e-3 * base[idx][e]
            if margin > 0:
                h = min(h, 0.25 * margin / 2)
            fd = (4 * central(e, idx, h) - central(e, idx, 2 * h)) / 3
            assert abs(grads[idx][e] - fd) <= 1e-6 * abs(fd), (int(e), idx, grads[idx][e], fd)
        # J_K is affine in q (q enters every update linearly), so a forward difference is exact
        # up to rounding, also where q = 0
        h = 1e-3 * max(base[2][e], 1.0)
        pert = [a.copy() for a in base]
        pert[2][e] += h
        fd = (J_of(pert) - J0) / h
        assert abs(grads[2][e] - fd) <= 1e-6 * abs(fd), (int(e), 2, grads[2][e], fd)
    mesh.set_materials(prob.sigma_t, prob.sigma_s, prob.q)


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
