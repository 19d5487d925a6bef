"""CPU: the C++ oracle (oracle/sweep_ref.cpp: the transport update, the thick-subdomain SIP DSA
operator and source iteration with and without Algorithm 2) against the pinned numpy oracle and
against closed forms.

The C++ code restates the same steps (Sec. 1, Eq. psi and Eq. phi; upwind DG of Sec. 3.1) in a second
implementation; it serves as the timed CPU baseline, so it is pinned here: element by element equal
to oracle.Transport.sweep (1e-13 relative) on Cartesian, jittered, Q3, 3D and inflow cases and on a
partial direction range; the same bits for any number of threads; and an infinite medium with the
equilibrium inflow psi_inc = q/(4 pi sigma_a) is a fixed point, phi = q/(sigma_t - sigma_s).  Its D_ff
(Eq. SIP on the thick elements, Sec. 3.2) equals oracle.dsa.DSA's entry by entry; its source
iteration reproduces the numpy oracle's iterates (unaccelerated to 1e-13; with the Algorithm 2 step,
where the numpy oracle factorises D_ff and the C++ code runs conjugate gradients, within the iterate
tolerance of the rounding-amplification reading) and its converged solutions.
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle import Transport, sweep_cpp


def _ragged():
    nx, ny = 13, 7
    st, ss = inputs.random_fields(nx * ny, 4242)
    q = np.where(np.arange(nx * ny) % 5 == 0, 1.0, 0.25)
    return inputs.Problem("ragged", 2, nx, ny, 1, 1, 6, st, ss, q, psi_inc=0.3)


CASES = {"c1": inputs.config1, "c2_32_jittered_q2": lambda: inputs.config2(n=32, block=8),
         "c3_8": lambda: inputs.config3(n=8), "q3_s6": lambda: inputs.config2d_fields(12, 3, 6, 77, "q3"),
         "ragged_inflow": _ragged}


@pytest.mark.parametrize("name", list(CASES))
def test_cpp_sweep_equals_the_numpy_oracle(name):
    prob = CASES[name]()
    T = Transport(prob)
    phi = inputs.random_phi(prob, 11)
    ref = T.sweep(phi)
    got = sweep_cpp.sweep(prob, phi, threads=1)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    part = range(T.nd // 3, 2 * T.nd // 3)
    refp = T.sweep(phi, directions=part)
    gotp = sweep_cpp.sweep(prob, phi, directions=part, threads=2)
    assert np.abs(gotp - refp).max() <= 1e-13 * np.abs(refp).max()


def test_cpp_sweep_is_independent_of_the_thread_count():
    prob = inputs.config2(n=32, block=8)
    phi = inputs.random_phi(prob, 5)
    a = sweep_cpp.sweep(prob, phi, threads=1)
    for t in (2, 3, max(1, sweep_cpp.max_threads())):
        assert np.array_equal(a, sweep_cpp.sweep(prob, phi, threads=t))


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_cpp_sweep_infinite_medium_fixed_point(dim, p):
    st, ss, q = 2.0, 1.5, 3.0
    prob = inputs.uniform_problem(dim, 4, p, 4, st, ss, q, psi_inc=q / (4 * np.pi * (st - ss)))
    phi = np.full((prob.n_elem, prob.n_nodes), q / (st - ss))
    got = sweep_cpp.sweep(prob, phi, threads=2)
    assert np.abs(got - phi).max() <= 1e-13 * phi.max()


DSA_CASES = {"c1": inputs.config1, "c2_16": lambda: inputs.config2(n=16, block=4),
             "c3_8": lambda: inputs.config3(n=8), "q3": lambda: inputs.config2d_fields(6, 3, 4, 78, "q3")}


def _jittered_q2():
    prob = inputs.config2d_fields(8, 2, 4, 77, "q2j")
    prob.vertices = inputs.jittered_vertices(8, 8, 0.15, 77)
    return prob


DSA_CASES["jittered_q2"] = _jittered_q2


@pytest.mark.parametrize("name", list(DSA_CASES))
def test_cpp_dsa_operator_equals_the_numpy_oracle(name):
    from oracle.dsa import DSA, thick_mask
    prob = DSA_CASES[name]()
    mask = thick_mask(prob)
    assert mask.sum() > 0
    ref = DSA(Transport(prob), mask).D.toarray()
    got = sweep_cpp.dsa_matrix(prob, mask)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(DSA_CASES))
def test_cpp_source_iteration_equals_the_numpy_oracle(name):
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from tolerances import dsa_iterate_tol
    from oracle.dsa import DSA, thick_mask
    prob = DSA_CASES[name]()
    T = Transport(prob)
    mask = thick_mask(prob)
    ref = T.source_iterate(dsa=None, tol=0.0, max_iters=5)["phi"]
    got = sweep_cpp.source_iterate(prob, None, tol=0.0, max_iters=5)["phi"]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    d = DSA(T, mask)
    ref = T.source_iterate(dsa=d, tol=0.0, max_iters=4)["phi"]
    got = sweep_cpp.source_iterate(prob, mask, tol=0.0, max_iters=4)["phi"]
    assert np.abs(got - ref).max() <= dsa_iterate_tol(prob, mask) * np.abs(ref).max()
    ref = T.source_iterate(dsa=d, tol=1e-12, max_iters=3000)
    got = sweep_cpp.source_iterate(prob, mask, tol=1e-12, max_iters=3000)
    assert got["iters"] == ref["iters"]
    assert np.abs(got["phi"] - ref["phi"]).max() <= 1e-10 * np.abs(ref["phi"]).max()


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_cpp_source_iteration_reaches_the_infinite_medium_solution(dim, p):
    """An optically thick infinite medium (sigma_t h = 5, c = 0.99, equilibrium inflow) converges to
    phi = q/(sigma_t - sigma_s) with the Algorithm 2 step on every element in a few tens of
    iterations, where plain source iteration needs about a thousand (measured 20-32 against
    826-1071): pins the C++ DSA step independently of the numpy oracle (a wrong sign or scale of the
    correction would stall or diverge)."""
    st, ss, q = 20.0, 19.8, 3.0
    prob = inputs.uniform_problem(dim, 4, p, 4, st, ss, q, psi_inc=q / (4 * np.pi * (st - ss)))
    exact = q / (st - ss)
    full = np.ones(prob.n_elem, dtype=np.uint8)
    acc = sweep_cpp.source_iterate(prob, full, tol=1e-12, max_iters=3000, threads=2)
    assert np.abs(acc["phi"] - exact).max() <= 1e-11 * exact
    assert acc["iters"] <= 50
    plain = sweep_cpp.source_iterate(prob, None, tol=1e-12, max_iters=3000, threads=2)
    assert plain["iters"] >= 10 * acc["iters"]
