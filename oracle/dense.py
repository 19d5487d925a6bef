"""Direct solves of the discrete transport system on tiny meshes (CPU oracle, tests only).

Eq. (system): the S_N transport equations as one block matrix
    [ L_1          -Sigma_s ] [psi_1]   [q_1]
    [      ...       ...    ] [ ... ] = [...]
    [         L_n  -Sigma_s ] [psi_n]   [q_n]
    [-w_1 I .. -w_n I    I  ] [ phi ]   [ 0 ]
and Eq. (schur): S = I - sum_d w_d L_d^{-1} Sigma_s with b = sum_d w_d L_d^{-1} q_d.
These pin the sweep and the source iteration, whose fixed point is the phi of this system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .transport import FOUR_PI


def global_L(T, d):
    """Global modal matrix of L_d: element blocks A_e plus upwind face couplings."""
    fw = T.face_flux(d)
    A = T.element_matrices(d, fw)
    n, ne = T.n, T.ne
    rows, cols, vals = [], [], []
    e = np.arange(ne)
    ri = (e[:, None] * n + np.arange(n))[:, :, None]
    ci = (e[:, None] * n + np.arange(n))[:, None, :]
    rows.append(np.broadcast_to(ri, A.shape).ravel())
    cols.append(np.broadcast_to(ci, A.shape).ravel())
    vals.append(A.ravel())
    for f in range(2 * T.dim):
        inflow = (fw[f].sum(axis=1) < 0) & (T.mesh.nbr[:, f] >= 0)
        E = np.flatnonzero(inflow)
        U = T.mesh.nbr[E, f]
        C = np.einsum("eq,qm,qk->emk", fw[f][E], T.BF[f], T.BFo[f])
        ri = (E[:, None] * n + np.arange(n))[:, :, None]
        ci = (U[:, None] * n + np.arange(n))[:, None, :]
        rows.append(np.broadcast_to(ri, C.shape).ravel())
        cols.append(np.broadcast_to(ci, C.shape).ravel())
        vals.append(C.ravel())
    N = ne * n
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def scatter_matrix(T):
    """Sigma_s: mass matrix with coefficient sigma_s / (4 pi) (modal, block diagonal)."""
    return sp.block_diag([sp.csr_matrix(T.sigma_s[e] / FOUR_PI * T.M[e]) for e in range(T.ne)], format="csr")


def source_vector(T):
    """q_d (isotropic): mass matrix applied to q/(4 pi)."""
    S = np.zeros((T.ne, T.n))
    S[:, 0] = T.q / FOUR_PI
    return np.einsum("emn,en->em", T.M, S).ravel()


def solve_block_system(T):
    """Dense solve of Eq. (system) with vacuum (or the problem's constant) inflow; nodal phi."""
    if T.prob.psi_inc != 0.0:
        raise ValueError("dense system is assembled for vacuum inflow")
    N = T.ne * T.n
    nd = T.nd
    Ms = scatter_matrix(T).toarray()
    q = source_vector(T)
    K = np.zeros(((nd + 1) * N, (nd + 1) * N))
    rhs = np.zeros((nd + 1) * N)
    for d in range(nd):
        K[d * N:(d + 1) * N, d * N:(d + 1) * N] = global_L(T, d).toarray()
        K[d * N:(d + 1) * N, nd * N:] = -Ms
        K[nd * N:, d * N:(d + 1) * N] = -T.w[d] * np.eye(N)
        rhs[d * N:(d + 1) * N] = q
    K[nd * N:, nd * N:] = np.eye(N)
    x = np.linalg.solve(K, rhs)
    return T.to_nodal(x[nd * N:].reshape(T.ne, T.n))


def solve_schur(T):
    """Assemble S = I - sum_d w_d L_d^{-1} Sigma_s and b densely; solve S phi = b; nodal phi."""
    N = T.ne * T.n
    Ms = scatter_matrix(T).toarray()
    q = source_vector(T)
    S = np.eye(N)
    b = np.zeros(N)
    for d in range(T.nd):
        Linv = np.linalg.inv(global_L(T, d).toarray())
        S -= T.w[d] * Linv @ Ms
        b += T.w[d] * Linv @ q
    return T.to_nodal(np.linalg.solve(S, b).reshape(T.ne, T.n)), S
