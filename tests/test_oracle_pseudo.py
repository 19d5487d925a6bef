"""Pins of the oracle's pseudo-scattering coefficients (Sec. 4.2, Eq. hohlraum_sigma and
Eq. hohlraum_q) and checks of the hohlraum-like input layout.

The coefficients are the linearisation of one implicit time step of gray radiative transfer, so
they are fixed by what that step must do: an infinite medium at uniform temperature T stays in
equilibrium (intensity a c T^4 in every direction, phi = 4 pi a c T^4) whatever sigma, C_v and dt
are; an infinitely long step turns absorption into scattering (sigma_ps -> sigma, q_ps -> 0); a
vanishing step leaves pure absorption and emission (sigma_ps -> 0, q_ps -> sigma a c T^4).
"""
import dataclasses

import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle import Transport
from oracle.dsa import DSA
from oracle.pseudo import problem, pseudo_scattering
from oracle.dsa import thick_mask

A, C = inputs.HOHLRAUM_A_RAD, inputs.HOHLRAUM_C_LIGHT


@pytest.mark.parametrize("sigma,cv,dt,T", [(2.0, 3.0, 0.5, 0.1), (1.0e3, 1.0e5, 1.0e-3, 0.4),
                                           (1.0e2, 1.0e3, 1.0e-3, 0.05), (0.5, 1.0e-2, 10.0, 0.02)])
def test_uniform_temperature_stays_in_equilibrium(sigma, cv, dt, T):
    """Homogeneous box with the equilibrium intensity a c T^4 flowing in: phi = 4 pi a c T^4."""
    st, ss, q = pseudo_scattering([sigma], [cv], [T], dt, A, C)
    prob = inputs.uniform_problem(2, 4, 1, 4, st[0], ss[0], q[0], psi_inc=A * C * T ** 4)
    Tr = Transport(prob)
    r = Tr.source_iterate(dsa=DSA(Tr, np.ones(Tr.ne)), tol=1e-14, max_iters=3000)
    expect = 4 * np.pi * A * C * T ** 4
    assert np.abs(r["phi"] - expect).max() < 1e-11 * expect


@pytest.mark.parametrize("sigma,cv,T", [(1.0e3, 1.0e5, 0.4), (1.0, 1.0, 1e-3), (1.0e-3, 1.0e-2, 0.4)])
def test_long_and_short_time_step_limits(sigma, cv, T):
    emission = 4 * np.pi * sigma * A * C * T ** 4
    _, ss, q = pseudo_scattering([sigma], [cv], [T], 1e30, A, C)   # dt -> infinity: pure scattering
    assert abs(ss[0] - sigma) <= 1e-12 * sigma and abs(q[0]) <= 1e-10 * emission
    _, ss, q = pseudo_scattering([sigma], [cv], [T], 1e-30, A, C)  # dt -> 0: absorber + emission
    assert ss[0] <= 1e-12 * sigma and abs(q[0] - emission) <= 1e-12 * emission


def test_scattering_ratio_grows_with_time_step_and_opacity():
    """Sec. 4.2: iterations slow down when the time step or sigma is large, i.e. c = sigma_ps / sigma
    grows with both; it stays in [0, 1) and the source stays non-negative."""
    dts = np.logspace(-6, 3, 10)
    sig = np.logspace(-3, 3, 7)
    for T in (1e-3, 0.1, 0.4):
        c_dt = [pseudo_scattering([10.0], [10.0], [T], dt, A, C)[1][0] / 10.0 for dt in dts]
        c_sig = [pseudo_scattering([s_], [10.0], [T], 1e-3, A, C)[1][0] / s_ for s_ in sig]
        for c in (c_dt, c_sig):
            assert np.all(np.diff(c) > 0) and 0 <= c[0] and c[-1] < 1
        q = [pseudo_scattering([10.0], [10.0], [T], dt, A, C)[2][0] for dt in dts]
        assert min(q) >= 0


def test_hohlraum_like_layout_and_thick_set():
    prob = inputs.hohlraum_like(64, jitter=0.0)
    mat = prob.extra["material"].reshape(64, 64)
    row = mat[int(0.45 * 64)]                      # a row through the capsule below the fill tube
    runs = [int(v) for k, v in enumerate(row) if k == 0 or v != row[k - 1]]
    assert runs == [0, 1, 2, 3, 2, 1, 0]           # gold, helium, CH, hydrogen, CH, helium, gold
    tp = problem(prob)
    hot = prob.extra["T"] == inputs.HOHLRAUM_T_HOT
    assert hot.any() and np.all(mat.ravel()[hot] == 0)
    # the paper's thick rule (sigma_s >= 1) selects exactly the laser-heated gold
    assert np.array_equal(tp.sigma_s >= 1.0, hot)
    assert np.all(tp.sigma_s <= tp.sigma_t) and np.all(tp.q >= 0)
    assert thick_mask(dataclasses.replace(tp)).sum() == hot.sum()


def test_heat_capacity_term_underflow_limit():
    """C_v/dt = 0 exactly (underflow): sigma_ps = sigma^2 b / (sigma b) = sigma and q_ps = 0 up to
    rounding (Eq. hohlraum_sigma, Eq. hohlraum_q with the C_v/dt term gone)."""
    for sigma in (0.5, 7.0, 3e3):
        _, ss, q = pseudo_scattering([sigma], [1e-300], [0.4], 1e300, A, C)
        emission = 4 * np.pi * sigma * A * C * 0.4 ** 4
        assert abs(ss[0] - sigma) <= 4e-16 * sigma and abs(q[0]) <= 1e-15 * emission
