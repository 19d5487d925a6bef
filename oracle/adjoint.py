"""Adjoint sweep, adjoint source iteration and gradients (CPU oracle, test infrastructure only).

The forward problem is the block system of Eq. (system):
    L_d psi_d - Sigma_s phi = q_d (all d),   -sum_d w_d psi_d + phi = 0,
whose Schur complement on phi is S = I - sum_d w_d L_d^{-1} Sigma_s (Eq. schur).  For a
functional J = g^T phi the adjoint solves S^T mu = g, i.e.
    mu = g + Sigma_s^T sum_d w_d L_d^{-T} mu ,
and with psi_d = L_d^{-1}(q_d + Sigma_s phi) and lambda_d = w_d L_d^{-T} mu,
    dJ/dp = mu^T (d b/dp + dT/dp phi) = sum_d lambda_d^T (d q_d/dp + d Sigma_s/dp phi - d L_d/dp psi_d).
Per element e with mass matrix M_e this gives
    dJ/dsigma_t,e = -sum_d lambda_d,e^T M_e psi_d,e
    dJ/dsigma_s,e =  sum_d lambda_d,e^T M_e phi_e / (4 pi)
    dJ/dq_e       =  sum_d lambda_d,e^T M_e 1 / (4 pi).
L_d^T is solved element by element in reverse upwind order with transposed element and
face-coupling blocks.  The DSA step of the adjoint iteration uses the transposed
Algorithm 2 preconditioner, I + E_f Sigma_f D_ff^{-T} E_f^T (D_ff^{-T} = D_ff^{-1} for the
symmetric operator, a transposed solve for the nonsymmetric ones of Eq. NIP); like any
convergent preconditioner it leaves mu unchanged.
"""
from __future__ import annotations

import numpy as np

from .transport import FOUR_PI


def adjoint_sweep_direction(T, d, rhs_modal):
    """Solve L_d^T lam = rhs (modal) by a reverse upwind sweep."""
    fw = T.face_flux(d)
    A = T.element_matrices(d, fw)
    lam = np.zeros((T.ne, T.n))
    nbr = T.mesh.nbr
    for E in reversed(T.levels(d, fw)):
        r = rhs_modal[E].copy()
        for f in range(2 * T.dim):
            out = (fw[f][E].sum(axis=1) > 0) & (nbr[E, f] >= 0)
            if not np.any(out):
                continue
            Eo = E[out]
            dn = nbr[Eo, f]
            fo = f ^ 1   # the same face seen from the downwind element, where it is an inflow face
            # C(dn <- e)[m, k] = sum_q fw_fo[dn, q] BF_fo[q, m] BFo_fo[q, k]; we need C^T lam_dn
            t = lam[dn] @ T.BF[fo].T                      # (.., qf)
            r[out] -= np.einsum("eq,qk,eq->ek", fw[fo][dn], T.BFo[fo], t)
        lam[E] = np.linalg.solve(np.transpose(A[E], (0, 2, 1)), r[..., None])[..., 0]
    return lam


def adjoint_sweep_modal(T, mu_modal, keep_lambda=False):
    """T^T mu = sum_d w_d Sigma_s L_d^{-T} mu with Sigma_s = sigma_s M / (4 pi) (modal)."""
    acc = np.zeros((T.ne, T.n))
    lams = [] if keep_lambda else None
    for d in range(T.nd):
        lam = T.w[d] * adjoint_sweep_direction(T, d, mu_modal)
        acc += lam
        if keep_lambda:
            lams.append(lam)
    out = np.einsum("e,emn,en->em", T.sigma_s / FOUR_PI, T.M, acc)
    return (out, lams) if keep_lambda else out


def adjoint_sweep(T, mu_nodal):
    """Transpose of the nodal transport update's linear part: V^{-T} T_m^T V^T mu."""
    mu_m = np.asarray(mu_nodal).reshape(T.ne, T.n) @ T.V
    return adjoint_sweep_modal(T, mu_m) @ T.Vinv


def adjoint_iterate(T, g_modal, dsa=None, tol=1e-12, max_iters=2000):
    """Adjoint source iteration mu = g + T^T mu with the transposed DSA step (modal)."""
    mu = np.zeros((T.ne, T.n))
    r0 = None
    it = 0
    rel = np.inf
    while it < max_iters:
        half = g_modal + adjoint_sweep_modal(T, mu)
        r = half - mu
        rn = np.linalg.norm(r)
        r0 = r0 if r0 is not None else (rn if rn > 0 else 1.0)
        rel = rn / r0
        if dsa is not None and dsa.thick.size:
            half = half + dsa.correction_transposed(r)  # transposed Algorithm 2
        mu = half
        it += 1
        if rel <= tol:
            break
    return mu, it, rel


def detector_modal(T, indicator):
    """g with g^T phi = sum over marked elements of the integral of phi (modal)."""
    g = np.zeros((T.ne, T.n))
    ind = np.asarray(indicator).astype(bool)
    g[ind] = T.M[ind][:, :, 0]
    return g


def gradients(T, phi_nodal, mu_modal):
    """dJ/dsigma_t, dJ/dsigma_s, dJ/dq per element from converged phi and adjoint mu."""
    phi_m = T.to_modal(phi_nodal)
    _, psis = T.sweep_modal(phi_m, keep_psi=True)
    gt = np.zeros(T.ne)
    gs = np.zeros(T.ne)
    gq = np.zeros(T.ne)
    Mphi = np.einsum("emn,en->em", T.M, phi_m)
    M1 = T.M[:, :, 0]
    for d in range(T.nd):
        lam = T.w[d] * adjoint_sweep_direction(T, d, mu_modal)
        gt -= np.einsum("em,emn,en->e", lam, T.M, psis[d])
        gs += np.einsum("em,em->e", lam, Mphi) / FOUR_PI
        gq += np.einsum("em,em->e", lam, M1) / FOUR_PI
    return gt, gs, gq


def unrolled_gradients(T, phi0_nodal, K, g_modal):
    """dJ/dsigma_t, dJ/dsigma_s, dJ/dq of J = g^T phi_K, phi_K the K-th iterate of source iteration
    without acceleration from phi_0 (phi_{k+1} = T phi_k + b, Eq. source0): the chain rule through
    the K updates, taken backwards.  Update k maps phi_k to phi_{k+1} with the data p entering as in
    the converged case, so with mu_K = g and mu_k = T^T mu_{k+1},
        dJ/dp = sum_{k=0}^{K-1} mu_{k+1}^T (d b/dp + dT/dp phi_k),
    each term the contraction `gradients` forms at (phi_k, mu_{k+1}).  Every iterate is kept."""
    phis = [np.asarray(phi0_nodal, dtype=float)]
    for _ in range(K - 1):
        phis.append(T.sweep(phis[-1]))
    mu = np.array(g_modal, dtype=float)
    gt = np.zeros(T.ne)
    gs = np.zeros(T.ne)
    gq = np.zeros(T.ne)
    for k in range(K - 1, -1, -1):
        a, b, c = gradients(T, phis[k], mu)
        gt += a
        gs += b
        gq += c
        if k > 0:
            mu = adjoint_sweep_modal(T, mu)
    return gt, gs, gq
