"""Pins of the oracle's unrolled gradients: the chain rule through K transport updates without
acceleration (Eq. source0, phi_{k+1} = T phi_k + b), taken backwards with the adjoint sweep, against
central finite differences of the oracle's own K-update map.  The K-update map has no solver
tolerance in it, so a difference with relative step 1e-4 is accurate to about 1e-8 and a wrong
iterate index, a missing term or a transposed coupling shows up far above that."""
import numpy as np
import pytest

from oracle import Transport, adjoint
from paper_2001_09196_gb300 import inputs


def _problem(nx, p, sn, seed):
    n = nx * nx
    st = 0.5 + 2.0 * inputs.uniform(seed, 50, n)
    ss = (0.3 + 0.6 * inputs.uniform(seed, 51, n)) * st
    q = 0.5 + inputs.uniform(seed, 52, n)
    return inputs.Problem(f"unrolled_{nx}_{p}", 2, nx, nx, 1, p, sn, st, ss, q,
                          vertices=inputs.jittered_vertices(nx, nx, 0.15, seed))


def _J(prob, K, g_m):
    T = Transport(prob)
    phi = np.zeros((prob.n_elem, prob.n_nodes))
    for _ in range(K):
        phi = T.sweep(phi)
    return float((T.to_modal(phi) * g_m).sum())


@pytest.mark.parametrize("nx,p,K", [(4, 1, 3), (3, 2, 2)])
def test_unrolled_gradients_match_finite_differences(nx, p, K):
    prob = _problem(nx, p, 4, 7100 + nx + p)
    T = Transport(prob)
    strip = (np.arange(prob.n_elem) % nx == nx - 1).astype(np.uint8)
    g_m = adjoint.detector_modal(T, strip)
    grads = adjoint.unrolled_gradients(T, np.zeros((prob.n_elem, prob.n_nodes)), K, g_m)
    params = [prob.sigma_t, prob.sigma_s, prob.q]
    for idx, grad in enumerate(grads):
        scale = np.abs(grad).max()
        assert scale > 0
        for e in range(prob.n_elem):
            base = params[idx][e]
            h = 1e-4 * base
            vals = []
            for sign in (1.0, -1.0):
                params[idx][e] = base + sign * h
                vals.append(_J(prob, K, g_m))
            params[idx][e] = base
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(grad[e] - fd) <= 1e-6 * abs(fd) + 1e-10 * scale, (idx, e, grad[e], fd)


def test_one_update_is_the_single_step_contraction():
    """K = 1: the sum has one term, the contraction at (phi_0, g)."""
    prob = _problem(4, 1, 4, 7200)
    T = Transport(prob)
    g_m = adjoint.detector_modal(T, np.ones(prob.n_elem, dtype=np.uint8))
    phi0 = inputs.random_phi(prob, 3)
    got = adjoint.unrolled_gradients(T, phi0, 1, g_m)
    ref = adjoint.gradients(T, phi0, g_m)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
