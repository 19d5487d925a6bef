"""CPU: the C++ oracle of the transport update (oracle/sweep_ref.cpp) against the pinned numpy oracle
and against closed forms.

The C++ code restates the same steps (Sec. 1, Eq. psi and Eq. phi; upwind DG of Sec. 3.1) in a second
implementation; it serves as the timed CPU baseline, so it is pinned here: element by element equal
to oracle.Transport.sweep (1e-13 relative) on Cartesian, jittered, Q3, 3D and inflow cases and on a
partial direction range; the same bits for any number of threads; and an infinite medium with the
equilibrium inflow psi_inc = q/(4 pi sigma_a) is a fixed point, phi = q/(sigma_t - sigma_s).
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
