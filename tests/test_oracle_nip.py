"""Pins of the oracle's nonsymmetric DSA operators (Sec. 3.1: Eq. NIP and the modified penalty
of Eq. ModifiedF0) and of the transposed DSA step of the adjoint iteration.

Eq. NIP is Eq. SIP without the symmetrising face term G^T Sigma_t^{-1} F_1 and with the plain
penalty F_0.  The pins fix, from those definitions: which face term is dropped (it acts on the
jump of the trial function, so it vanishes on continuous functions, and the kept term is its
transpose), the penalty as the angular integral that defines F_0 and its modification, the
restriction of Eq. ModifiedF0 to void-free neighbourhoods, the preconditioner property (same
fixed point, fewer iterations) and the adjoint identity of the transposed correction.
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle import Transport, adjoint, dense
from oracle.dsa import C_M, DSA
from oracle.dsa import thick_mask


def _thick_uniform(p):
    # sigma_t large enough that the SIP penalty is at its 1/4 floor on every face
    return inputs.uniform_problem(2, 4, p, 4, 100.0, 99.0, 0.0)


@pytest.mark.parametrize("p", [1, 2])
def test_nip_drops_exactly_the_symmetrising_term(p):
    prob = _thick_uniform(p)
    T = Transport(prob)
    full = np.ones(T.ne)
    sip, nip = DSA(T, full, operator="sip").D.toarray(), DSA(T, full, operator="nip").D.toarray()
    S = sip - nip                                   # the dropped term (the penalties agree here)
    assert np.abs(S).max() > 1e-3 * np.abs(sip).max()
    # it acts on the jump of the trial function: zero on a continuous hat vanishing on the boundary
    hat = lambda x: (np.maximum(0, 1 - np.abs(x[..., 0] - 0.5) / 0.25)
                     * np.maximum(0, 1 - np.abs(x[..., 1] - 0.5) / 0.25))
    u = T.project(hat).ravel()
    assert np.abs(S @ u).max() < 1e-13 * np.abs(sip).max()
    assert np.abs(S.T @ u).max() > 1e-3 * np.abs(sip @ u).max()
    # the face-derivative term that stays is its transpose: NIP - NIP^T = S^T - S
    assert np.abs((nip - nip.T) - (S.T - S)).max() < 1e-14 * np.abs(sip).max()


def _kappa_from_angular_integral(sig_minus, h_minus, sig_plus, h_plus, c, modified):
    """(1/8 pi) int_{S^2} max(c/(sigma_t^up h^up), 1) |Omega.n| dOmega with the polar axis along n:
    mu = Omega.n > 0 flows from the - side (upwind) to the + side.  Gauss-Legendre in mu on each
    half, where the integrand is smooth; the azimuth integrates to 2 pi."""
    x, w = np.polynomial.legendre.leggauss(12)
    mu, wm = 0.5 * (x + 1), 0.5 * w
    f = (lambda s, h: max(c / (s * h), 1.0)) if modified else (lambda s, h: 1.0)
    return (2 * np.pi / (8 * np.pi)) * (f(sig_minus, h_minus) * np.sum(wm * mu) + f(sig_plus, h_plus) * np.sum(wm * mu))


@pytest.mark.parametrize("operator", ["nip", "mnip"])
def test_penalty_is_the_angular_integral_of_eq_modified_f0(operator):
    """Piecewise constants see only sigma_a and the penalty: a(1_K, 1_K) = sigma_a |K| + sum_F kappa_F |F|
    and a(1_K, 1_L) = -kappa_F |F| on the face between K and L; kappa_F from the definition."""
    p, n = 1, 4
    prob = inputs.uniform_problem(2, n, p, 4, 2.0, 1.0, 0.0)
    prob.sigma_t[5], prob.sigma_s[5] = 0.5, 0.25   # c/(sigma_t h) = 1.6: the max() takes it
    prob.sigma_t[6], prob.sigma_s[6] = 100.0, 50.0
    T = Transport(prob)
    op = DSA(T, np.ones(T.ne), operator=operator)
    h, c = 1.0 / n, C_M * p * (p + 1)
    modified = operator == "mnip"
    ones = lambda e: np.eye(T.ne)[e][:, None] * np.eye(T.n)[0][None, :]  # modal constant 1 on K
    for e in (5, 6, 0, 9):
        ue = ones(e).ravel()
        expect = (prob.sigma_t[e] - prob.sigma_s[e]) * h * h
        for f in range(4):
            o = T.mesh.nbr[e, f]
            so, ho = (prob.sigma_t[o], h) if o >= 0 else (prob.sigma_t[e], h)  # boundary: own value
            kap = _kappa_from_angular_integral(prob.sigma_t[e], h, so, ho, c, modified)
            expect += kap * h
            if o >= 0:
                off = ones(o).ravel() @ (op.D @ ue)
                assert abs(off + kap * h) < 1e-13 * kap * h, (e, f)
        assert abs(ue @ (op.D @ ue) - expect) < 1e-13 * expect, e


def test_mnip_rejects_void_neighbours():
    prob = inputs.config1()
    T = Transport(prob)
    mask = thick_mask(prob).copy()
    void = np.flatnonzero(prob.sigma_t == 0)
    e = next(int(u) for v in void for u in T.mesh.nbr[v] if u >= 0 and prob.sigma_t[u] > 0)
    mask[e] = 1                                     # a thick element next to a void one
    DSA(T, mask, operator="nip")                    # the unmodified penalty is defined there
    with pytest.raises(ValueError):
        DSA(T, mask, operator="mnip")


@pytest.mark.parametrize("operator", ["nip", "mnip"])
def test_nonsymmetric_dsa_accelerates_config1(operator):
    prob = inputs.config1()
    T = Transport(prob)
    r = T.source_iterate(dsa=DSA(T, thick_mask(prob), operator=operator), tol=1e-8, max_iters=200)
    assert r["converged"] and r["iters"] < 40
    assert not T.source_iterate(tol=1e-8, max_iters=60)["converged"]


@pytest.mark.parametrize("operator", ["sip", "nip", "mnip"])
def test_transposed_correction_is_the_adjoint(operator):
    """<y, C x> = <C^T y, x> for the Algorithm 2 correction C and the adjoint iteration's step."""
    prob = inputs.config2(n=16, block=4, p=1, sn=4)
    T = Transport(prob)
    dsa = DSA(T, thick_mask(prob), operator=operator)
    assert dsa.thick.size
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((T.ne, T.n)), rng.standard_normal((T.ne, T.n))
    lhs, rhs = (y * dsa.correction(x)).sum(), (dsa.correction_transposed(y) * x).sum()
    assert abs(lhs - rhs) < 1e-12 * np.abs(y).sum() * np.abs(dsa.correction(x)).max()


def test_adjoint_iteration_with_nip_reaches_the_dense_adjoint():
    """S^T mu = g (S from the dense Schur complement) by the adjoint iteration with NIP thick DSA."""
    prob = inputs.config2d_fields(5, 1, 4, 5, "a")
    T = Transport(prob)
    _, S = dense.solve_schur(T)
    g = np.random.default_rng(4).standard_normal((T.ne, T.n))
    mu_ref = np.linalg.solve(S.T, g.ravel()).reshape(T.ne, T.n)
    dsa = DSA(T, thick_mask(prob), operator="nip")
    mu, it, rel = adjoint.adjoint_iterate(T, g, dsa=dsa, tol=1e-14, max_iters=3000)
    assert rel <= 1e-14
    assert np.abs(mu - mu_ref).max() < 1e-11 * np.abs(mu_ref).max()
