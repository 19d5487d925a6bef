"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook quadrature
tables, closed-form solutions, exact reproduction of manufactured solutions, convergence
rates, a dense direct solve of the block system (Eq. system), symmetry / definiteness /
consistency of the diffusion operator, the DSA fixed-point invariance (Eq. DSA_fp),
the adjoint dot-product identity and finite differences.
"""
import copy
import os

import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle import Transport
from oracle import adjoint, dense
from oracle.dsa import DSA, TriangularDSA
from oracle.quadrature import level_symmetric, level_symmetric_octant
from oracle.dsa import thick_mask

FOUR_PI = 4.0 * np.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature (Sec. 1, Sec. 4.1)
@pytest.mark.parametrize("N,dim,count", [(4, 2, 12), (6, 2, 24), (8, 2, 40), (4, 3, 24), (6, 3, 48), (8, 3, 80)])
def test_quadrature_counts(N, dim, count):
    d, w = level_symmetric(N, dim)
    assert len(w) == count == d.shape[0]
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)


def test_quadrature_textbook_weights():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "ls_quadrature_weights.txt")) if ln[0] != "#"]
    for N, cls, wref in rows:
        N = int(N)
        cls = tuple(int(c) for c in cls.split(","))
        _, pts, w = level_symmetric_octant(N)
        got = [wi for p, wi in zip(pts, w) if tuple(sorted(p)) == cls]
        assert got, (N, cls)
        assert np.allclose(got, float(wref), atol=6e-8)


@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("dim", [2, 3])
def test_quadrature_moments(N, dim):
    d, w = level_symmetric(N, dim)
    assert abs(w.sum() - FOUR_PI) < 1e-13
    first = (w[:, None] * d).sum(axis=0)[:dim]
    assert np.all(np.abs(first) < 1e-14)
    second = np.einsum("d,di,dj->ij", w, d, d)
    assert np.allclose(second, FOUR_PI / 3 * np.eye(3), atol=1e-14)


# ---------------------------------------------------------------- transport discretisation
def _mms(prob, psi, grad, st, ss, tol=1e-14):
    """Manufactured psi independent of Omega: q_d = Omega.grad psi + (sigma_t - sigma_s) psi."""
    T = Transport(prob)
    src = []
    for d in range(T.nd):
        Om = T.dirs[d][: prob.dim]
        src.append(T.project(lambda x: np.einsum("eqk,k->eq", grad(x), Om) + (st - ss) * psi(x)))
    r = T.source_iterate(tol=tol, max_iters=400, src_per_dir=src, psi_inc=lambda x, Om: psi(x))
    exact = T.to_nodal(T.project(lambda x: FOUR_PI * psi(x)))
    return np.abs(r["phi"] - exact).max() / np.abs(exact).max()


PSI_BL = (lambda x: 1 + 2 * x[..., 0] + 3 * x[..., 1] + 4 * x[..., 0] * x[..., 1],
          lambda x: np.stack([2 + 4 * x[..., 1], 3 + 4 * x[..., 0]], -1))
PSI_LIN = (lambda x: 1 + 2 * x[..., 0] + 3 * x[..., 1],
           lambda x: np.stack([2 + 0 * x[..., 1], 3 + 0 * x[..., 0]], -1))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_polynomial_reproduction_cartesian(p):
    prob = inputs.uniform_problem(2, 4, p, 4, 2.0, 1.0, 0.0)
    assert _mms(prob, *PSI_BL, 2.0, 1.0) < 1e-13


@pytest.mark.parametrize("p,psi", [(1, PSI_LIN), (2, PSI_BL), (2, PSI_LIN)])
def test_polynomial_reproduction_jittered(p, psi):
    prob = inputs.config2(n=16, block=8, p=p, sn=4)
    prob.sigma_t[:] = 2.0
    prob.sigma_s[:] = 1.0
    assert _mms(prob, *psi, 2.0, 1.0) < 1e-13


def test_void_reproduces_linear_field():
    prob = inputs.config2(n=16, block=8, p=2, sn=6)
    prob.sigma_t[:] = 0.0
    prob.sigma_s[:] = 0.0
    assert _mms(prob, *PSI_BL, 0.0, 0.0) < 1e-13


def test_polynomial_reproduction_3d():
    psi = lambda x: 1 + 2 * x[..., 0] + 3 * x[..., 1] - x[..., 2] + x[..., 0] * x[..., 1] * x[..., 2]
    grad = lambda x: np.stack([2 + x[..., 1] * x[..., 2], 3 + x[..., 0] * x[..., 2], -1 + x[..., 0] * x[..., 1]], -1)
    prob = inputs.uniform_problem(3, 3, 1, 4, 2.0, 1.0, 0.0)
    assert _mms(prob, psi, grad, 2.0, 1.0) < 1e-13


@pytest.mark.parametrize("dim,p,use_dsa", [(2, 1, False), (2, 2, True), (3, 1, True)])
def test_infinite_medium(dim, p, use_dsa):
    """Homogeneous medium with isotropic inflow q/(4 pi sigma_a): phi = q/(sigma_t - sigma_s)."""
    st, ss, q = 3.0, 2.4, 1.5
    prob = inputs.uniform_problem(dim, 4, p, 4, st, ss, q, psi_inc=q / (FOUR_PI * (st - ss)))
    T = Transport(prob)
    dsa = DSA(T, np.ones(T.ne)) if use_dsa else None
    r = T.source_iterate(dsa=dsa, tol=1e-14, max_iters=400)
    assert np.abs(r["phi"] - q / (st - ss)).max() < 1e-12 * q / (st - ss)


@pytest.mark.parametrize("p,rate", [(1, 1.8), (2, 2.7)])
def test_pure_absorber_convergence_rate(p, rate):
    """sigma_s = 0, no source: psi_d = exp(-sigma_t (Omega.x)/|Omega|^2) exactly; L2 rate ~ p+1."""
    st = 2.0
    errs = []
    for n in (4, 8, 16):
        prob = inputs.uniform_problem(2, n, p, 4, st, 0.0, 0.0)
        T = Transport(prob)

        def exact_d(x, Om):
            o = Om[:2]
            return np.exp(-st * (x[..., :2] @ o) / (o @ o))

        phi = np.zeros((T.ne, T.n))
        for d in range(T.nd):
            phi += T.w[d] * T.sweep_direction(d, np.zeros((T.ne, T.n)), psi_inc=exact_d)
        exact_phi = lambda x: sum(T.w[d] * exact_d(x, T.dirs[d]) for d in range(T.nd))
        errs.append(T.l2_error(phi, exact_phi))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates >= rate), rates


def test_cartesian_levels_are_index_sums():
    prob = inputs.uniform_problem(3, 4, 1, 4, 1.0, 0.5, 1.0)
    T = Transport(prob)
    for d in range(T.nd):
        lev = np.empty(T.ne, dtype=np.int64)
        for L, E in enumerate(T.levels(d)):
            lev[E] = L
        s = np.where(T.dirs[d][:3] > 0, T.mesh.ijk, 3 - T.mesh.ijk)
        assert np.array_equal(lev, s.sum(axis=1))


def test_cyclic_upwind_graph_is_refused():
    """Kahn's order exists only for an acyclic upwind graph (the sweep of Sec. 1 needs one).  No
    direction on a mesh of convex elements makes a cycle, so the face fluxes are handed in: on a 2x2
    mesh a flow circulating 0 -> 1 -> 3 -> 2 -> 0 has no element without upwind neighbours and must
    raise; reversing the edge 2 -> 0 leaves the chain 0 -> 1 -> 3 -> 2 (with 0 -> 2), levels
    [0], [1], [3], [2]."""
    from oracle.transport import CycleError
    prob = inputs.uniform_problem(2, 2, 1, 4, 1.0, 0.5, 1.0)
    T = Transport(prob)
    shape = T.face_flux(0)[0].shape   # (ne, face points); face 2a + side, side 1 = positive axis

    def flows(edges):
        fw = [np.zeros(shape) for _ in range(4)]
        for e, f, sign in edges:
            fw[f][e] = sign
        return fw
    # (element, face, +1 outflow / -1 inflow); elements 0 (0,0), 1 (1,0), 2 (0,1), 3 (1,1)
    ring = [(0, 1, 1), (1, 0, -1),    # 0 -> 1 across x
            (1, 3, 1), (3, 2, -1),    # 1 -> 3 across y
            (3, 0, 1), (2, 1, -1),    # 3 -> 2 across x
            (2, 2, 1), (0, 3, -1)]    # 2 -> 0 across y
    assert np.array_equal(T.mesh.nbr[[0, 1, 3, 2]][:, [1, 3, 0, 2]].diagonal(), [1, 3, 2, 0])
    with pytest.raises(CycleError):
        T.levels(0, fw=flows(ring))
    broken = ring[:6] + [(2, 2, -1), (0, 3, 1)]   # 0 -> 2 instead of 2 -> 0
    assert [list(L) for L in T.levels(0, fw=flows(broken))] == [[0], [1], [3], [2]]


# ---------------------------------------------------------------- block system (Eq. system / schur)
@pytest.mark.parametrize("n,p", [(4, 1), (3, 2)])
def test_dense_direct_solve_matches_source_iteration(n, p):
    prob = inputs.config2d_fields(n, p, 4, 123 + p, "tiny")
    prob.q[:] = 1.0
    T = Transport(prob)
    direct = dense.solve_block_system(T)
    schur, _ = dense.solve_schur(T)
    si = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-15, max_iters=3000)["phi"]
    scale = np.abs(direct).max()
    assert np.abs(schur - direct).max() < 1e-12 * scale
    assert np.abs(si - direct).max() < 1e-12 * scale


# ---------------------------------------------------------------- DSA (Sec. 2.2, Algorithm 2, Sec. 3)
def _void_free_c1():
    prob = inputs.config1()
    v = prob.sigma_t == 0
    prob.sigma_t[v], prob.sigma_s[v] = 1.0, 0.9
    return prob


@pytest.mark.parametrize("operator", ["sip", "nip", "mnip"])
def test_dsa_fixed_point_invariance(operator):
    """DSA is a preconditioner only: none / thick / full reach the same phi (Eq. DSA_fp), with each
    interior-penalty operator of Sec. 3.1."""
    prob = inputs.config2d_fields(6, 1, 4, 99, "inv")
    prob.q[:] = 1.0
    prob.sigma_t[prob.sigma_t == 0] = 0.5
    prob.sigma_s[prob.sigma_s == 0] = 0.25
    T = Transport(prob)
    ref = dense.solve_block_system(T)
    for mask in (thick_mask(prob), np.ones(T.ne)):
        r = T.source_iterate(dsa=DSA(T, mask, operator=operator), tol=1e-15, max_iters=3000)
        assert np.abs(r["phi"] - ref).max() < 1e-11 * np.abs(ref).max()


def test_dsa_accelerates_config1():
    prob = inputs.config1()
    T = Transport(prob)
    r = T.source_iterate(dsa=DSA(T, thick_mask(prob)), tol=1e-8, max_iters=200)
    assert r["converged"] and r["iters"] < 40
    r0 = T.source_iterate(tol=1e-8, max_iters=60)
    assert not r0["converged"]


def _vacuum_thin(prob):
    """sigma_s = 0 on every element outside the thick set (the case of Eq. Stri)."""
    thick = thick_mask(prob).astype(bool)
    prob.sigma_s[~thick] = 0.0
    return prob


@pytest.mark.parametrize("prob_fn", [lambda: inputs.config1(), lambda: inputs.config2(n=16, block=4, p=1, sn=4)])
def test_triangular_dsa_makes_the_thin_block_the_identity(prob_fn):
    """Eq. Stri: with Sigma_s = 0 on the thin region S is block upper triangular, and Algorithm 1's
    preconditioner P (Eq. approxS) makes the thin rows of S P the identity, whatever D_ff is:
    (S P v)_s = v_s.  S v = v - T v with T the zero-source, vacuum-inflow transport update."""
    prob = _vacuum_thin(prob_fn())
    T = Transport(prob)
    tri = TriangularDSA(DSA(T, thick_mask(prob)))
    rng = np.random.default_rng(7)
    v = rng.standard_normal((T.ne, T.n))
    Pv = v + tri.correction(v)
    SPv = Pv - tri.homogeneous_update(Pv)
    thin = ~thick_mask(prob).astype(bool)
    assert thin.any() and (~thin).any()
    assert np.abs(SPv[thin] - v[thin]).max() < 1e-13 * np.abs(v).max()
    # the thick rows are not the identity (D_ff only approximates the thick block)
    assert np.abs(SPv[~thin] - v[~thin]).max() > 1e-6


def test_triangular_dsa_fixed_point_and_acceleration():
    """Algorithm 1 is a preconditioner: same fixed point as the dense solve of Eq. system, and with
    a nearly vacuum thin region it takes no more iterations than Algorithm 2."""
    prob = inputs.config2d_fields(8, 1, 4, 98, "tri")
    prob.q[:] = 1.0
    prob.sigma_t[prob.sigma_t == 0] = 0.5
    thick = thick_mask(prob).astype(bool)
    prob.sigma_s[~thick] = 1e-3 * prob.sigma_t[~thick]
    T = Transport(prob)
    ref = dense.solve_block_system(T)
    diag = DSA(T, thick_mask(prob))
    r_tri = T.source_iterate(dsa=TriangularDSA(diag), tol=1e-14, max_iters=3000)
    assert np.abs(r_tri["phi"] - ref).max() < 1e-11 * np.abs(ref).max()
    r_diag = T.source_iterate(dsa=diag, tol=1e-14, max_iters=3000)
    assert r_tri["iters"] <= r_diag["iters"]


@pytest.mark.parametrize("prob_fn", [inputs.config1, lambda: inputs.config2(n=16, block=4, p=1, sn=4),
                                     lambda: inputs.config2d_fields(8, 1, 4, 98, "tri")])
def test_thick_dsa_beats_full_dsa_with_scattering_free_thin_regions(prob_fn):
    """Sec. 2.3: with Sigma_s = 0 outside the thick region S is block upper triangular, so DSA on the
    thick block alone is the right preconditioner; the paper's tables show heterogeneous DSA needing
    no more iterations than full DSA.  Thin regions keep sigma_t > 0 so that full DSA is defined."""
    prob = prob_fn()
    thick = thick_mask(prob).astype(bool)
    prob.sigma_t[prob.sigma_t == 0] = 0.5
    prob.sigma_s[~thick] = 0.0
    T = Transport(prob)
    het = T.source_iterate(dsa=DSA(T, thick), tol=1e-10, max_iters=200)
    full = T.source_iterate(dsa=DSA(T, np.ones(T.ne)), tol=1e-10, max_iters=200)
    plain = T.source_iterate(tol=1e-10, max_iters=200)
    assert het["converged"] and het["iters"] <= full["iters"]
    assert 3 * het["iters"] < plain["iters"]


def test_full_dsa_rejects_voids():
    prob = inputs.config1()
    T = Transport(prob)
    with pytest.raises(ValueError):
        DSA(T, np.ones(T.ne))


@pytest.mark.parametrize("prob_fn", [_void_free_c1, lambda: inputs.config2(n=32, block=8, p=2, sn=4)])
def test_dsa_operator_spd(prob_fn):
    prob = prob_fn()
    T = Transport(prob)
    mask = np.ones(T.ne) if np.all(prob.sigma_t > 0) else thick_mask(prob)
    D = DSA(T, mask).D.toarray()
    assert np.abs(D - D.T).max() <= 1e-15 * np.abs(D).max()
    np.linalg.cholesky(D)


@pytest.mark.parametrize("operator", ["sip", "nip", "mnip"])
def test_dsa_operator_consistency_q2(operator):
    """u = x(1-x)y(1-y) in Q2: a(u,v) = (f,v) + 1/2 <D du/dn, v>_boundary exactly (consistency of
    the interior-penalty forms in the interior; the half-flux boundary term of the zero-exterior
    reading on the boundary).  u is continuous and zero on the boundary, so the penalty and the
    symmetrising term vanish and the three operators of Sec. 3.1 share this identity."""
    n, st, ss = 4, 2.0, 1.5
    prob = inputs.uniform_problem(2, n, 2, 4, st, ss, 0.0)
    T = Transport(prob)
    op = DSA(T, np.ones(T.ne), operator=operator)
    Dc, sa = 1.0 / (3 * st), st - ss
    u = lambda x: x[..., 0] * (1 - x[..., 0]) * x[..., 1] * (1 - x[..., 1])
    f = lambda x: Dc * (2 * x[..., 1] * (1 - x[..., 1]) + 2 * x[..., 0] * (1 - x[..., 0])) + sa * u(x)
    uc = T.project(u)
    F = np.einsum("emn,en->em", T.M, T.project(f)).ravel()
    # boundary term 1/2 <D du/dn, v> on the domain boundary, Gauss rule exact for its degree
    from oracle.dg import face_points, tensor_rule
    tf, wf = tensor_rule(4, 1)
    Bt = np.zeros((T.ne, T.n))
    for fidx in range(4):
        a, side = divmod(fidx, 2)
        xi = face_points(tf, a, side)
        B, _ = T.basis.eval(xi)
        x, _ = T.mesh.map(xi)
        h = 1.0 / n
        nrm = np.zeros(2)
        nrm[a] = 1.0 if side else -1.0
        gu = np.stack([(1 - 2 * x[..., 0]) * x[..., 1] * (1 - x[..., 1]),
                       x[..., 0] * (1 - x[..., 0]) * (1 - 2 * x[..., 1])], -1)
        dudn = gu @ nrm
        bnd = T.mesh.nbr[:, fidx] < 0
        Bt[bnd] += 0.5 * Dc * np.einsum("q,eq,qm->em", wf * h / 2, dudn[bnd], B)
    res = op.D @ uc.ravel() - F - Bt.ravel()
    assert np.abs(res).max() < 1e-13 * np.abs(F).max()


def test_dsa_penalty_on_piecewise_constant():
    """a(1_K, 1_K) = sigma_a |K| + sum_F kappa_F |F| with the max-floored penalty."""
    from oracle.dsa import C_IP
    prob = inputs.uniform_problem(2, 4, 1, 4, 2.0, 1.0, 0.0)
    prob.sigma_t[5] = 0.01  # changes D on one element: penalty = floor 1/4 there for small D/h
    prob.sigma_s[5] = 0.005
    prob.sigma_t[10] = 100.0  # small D/h: the 1/4 floor is active on its faces
    prob.sigma_s[10] = 50.0
    T = Transport(prob)
    op = DSA(T, np.ones(T.ne))
    h = 0.25
    cp = C_IP * 1 * 2
    for e in (5, 10, 0):
        u = np.zeros((T.ne, T.n))
        u[e, 0] = 1.0
        val = u.ravel() @ (op.D @ u.ravel())
        De = 1 / (3 * prob.sigma_t[e])
        expect = (prob.sigma_t[e] - prob.sigma_s[e]) * h * h
        for fidx in range(4):
            o = T.mesh.nbr[e, fidx]
            if o < 0:
                kap = max(0.25, cp * De / h)
            else:
                kap = max(0.25, cp * 0.5 * (De / h + 1 / (3 * prob.sigma_t[o]) / h))
            expect += kap * h
        assert abs(val - expect) < 1e-13 * abs(expect)


# ---------------------------------------------------------------- adjoint (transpose of Eq. schur)
@pytest.mark.parametrize("prob_fn", [
    lambda: inputs.config2d_fields(5, 1, 4, 5, "a"),
    lambda: inputs.config2(n=16, block=8, p=2, sn=4),
    lambda: inputs.config3(n=3),
])
def test_adjoint_dot_product(prob_fn):
    prob = prob_fn()
    T = Transport(prob)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((T.ne, T.n))
    y = rng.standard_normal((T.ne, T.n))
    Tx = T.sweep(x) - T.sweep(np.zeros_like(x))
    Aty = adjoint.adjoint_sweep(T, y)
    lhs, rhs = (y * Tx).sum(), (Aty * x).sum()
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(y) * np.linalg.norm(Tx)


def test_adjoint_gradients_match_finite_differences():
    prob = inputs.config2d_fields(6, 1, 4, 7, "fd")
    prob.q[:] = 1.0
    det = np.zeros(prob.n_elem, dtype=np.uint8)
    det[[5, 11, 17]] = 1

    def J(pr):
        T = Transport(pr)
        r = T.source_iterate(dsa=DSA(T, thick_mask(pr)), tol=1e-15, max_iters=3000)
        return (T.to_modal(r["phi"]) * adjoint.detector_modal(T, det)).sum(), r["phi"], T

    _, phi, T = J(prob)
    mu, _, _ = adjoint.adjoint_iterate(T, adjoint.detector_modal(T, det), dsa=DSA(T, thick_mask(prob)), tol=1e-15)
    gt, gs, gq = adjoint.gradients(T, phi, mu)
    nonvoid = np.flatnonzero(prob.sigma_t > 0)[:3]
    for e in nonvoid:
        for arr, g in (("sigma_t", gt), ("sigma_s", gs), ("q", gq)):
            h = 1e-5 * abs(getattr(prob, arr)[e])
            pp, pm = copy.deepcopy(prob), copy.deepcopy(prob)
            getattr(pp, arr)[e] += h
            getattr(pm, arr)[e] -= h
            fd = (J(pp)[0] - J(pm)[0]) / (2 * h)
            assert abs(g[e] - fd) < 2e-5 * abs(fd), (e, arr, g[e], fd)
