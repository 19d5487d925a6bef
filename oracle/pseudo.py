"""Pseudo-scattering coefficients of one implicit time step of gray thermal radiative transfer
(CPU oracle, test infrastructure only).

Paper Sec. 4.2, Eq. hohlraum_sigma and Eq. hohlraum_q: with b = 16 pi a c T^3,
    sigma_ps = sigma^2 b / (C_v/dt + sigma b),
    q_ps     = sigma_a a c T^4 - sigma^2 b a c T^4 / (C_v/dt + sigma b),
and the steady transport problem of the time step takes sigma_t = sigma, sigma_s = sigma_ps and
the per-direction source q_d = q_ps.
Readings: sigma_a = sigma (the table lists the opacities sigma_a, and the text says the
coefficients are functions of sigma); the library's q is the total isotropic emission with
q_d = q / (4 pi), so q = 4 pi q_ps.  Both formulas are evaluated as printed, term by term.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def pseudo_scattering(sigma, cv, T, dt, a_rad, c_light):
    """(sigma_t, sigma_s, q) per element from Eq. hohlraum_sigma and Eq. hohlraum_q."""
    sigma, cv, T = (np.asarray(x, dtype=np.float64) for x in (sigma, cv, T))
    b = 16.0 * np.pi * a_rad * c_light * T ** 3
    den = cv / dt + sigma * b
    sigma_ps = sigma ** 2 * b / den
    q_ps = sigma * a_rad * c_light * T ** 4 - sigma ** 2 * 16.0 * np.pi * a_rad ** 2 * c_light ** 2 * T ** 7 / den
    return sigma.copy(), sigma_ps, 4.0 * np.pi * q_ps


def problem(prob):
    """The transport problem of the time step for a layout carrying extra = {sigma, cv, T, dt, ...}."""
    x = prob.extra
    st, ss, q = pseudo_scattering(x["sigma"], x["cv"], x["T"], x["dt"], x["a_rad"], x["c_light"])
    return dataclasses.replace(prob, sigma_t=st, sigma_s=ss, q=q)
