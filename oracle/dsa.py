"""Diffusion synthetic acceleration restricted to the thick subdomain (CPU oracle, tests only).

Paper: Sec. 2.2 (Eq. dsa_prec, Eq. DSA_fp and the additive form D^{-1} = I + D^{-1} Sigma),
Sec. 2.3 (Algorithm 2, diagonal heterogeneous DSA: phi_f <- phi_f + D_ff^{-1} Sigma_f r_f; and
Algorithm 1, triangular heterogeneous DSA, the same step followed by a zero-source transport
update of the thick correction whose result is added on the thin DOFs only),
Sec. 3.1 (interior-penalty DSA operators: Eq. SIP, Eq. NIP and the modified penalty of
Eq. ModifiedF0) and Sec. 3.2 (the heterogeneous operator is the principal submatrix on the
thick elements, thick where sigma_s >= eta).

Three operators, all with D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s and the same volume form
sum_K (D grad u, grad v)_K + (sigma_a u, v)_K; they differ on the faces.  A face whose neighbour
is not thick (thin, void or outside the domain) is treated as a face to a zero exterior state:
jump = u, average = half the interior value.  This is what the principal submatrix of a global
interior-penalty matrix gives on such a face.
  * "sip" (default; the conjugate-gradient path needs an SPD operator):
        <kappa [u],[v]> - <{D grad u.n},[v]> - <{D grad v.n},[u]>,
    kappa_F = max(1/4, c(p) (D^-/h^- + D^+/h^+)/2) on interior faces and max(1/4, c(p) D/h) on
    boundary faces, c(p) = C_IP p (p+1), h = |K|/|F|.  1/4 is the angular integral of the paper's
    F_0 = (1/4 pi) sum_d w_d |Omega_d.n|/2; the max() floor is the idea of Eq. ModifiedF0 in the
    form of the modified interior penalty method.  Only thick-element data enter (Sec. 3.2).
  * "nip" (Eq. NIP): drops the symmetrising term G^T Sigma_t^{-1} F_1, which is the face term
    -<{D grad v.n},[u]>; keeps -<{D grad u.n},[v]> (the term F_1^T Sigma_t^{-1} G) and the plain
    penalty F_0, kappa_F = 1/4.  Nonsymmetric.
  * "mnip" (Eq. NIP with Eq. ModifiedF0): the face terms of "nip" with the modified penalty
        kappa_F = 1/8 [max(c(p)/(sigma_t^- h^-), 1) + max(c(p)/(sigma_t^+ h^+), 1)],
    c(p) = C_M p (p+1), C_M = 0.1 (Sec. 3.1.1).  Reading: each side is the upwind side for the
    directions leaving it, and (1/4 pi) times the angular integral of |Omega.n| over either half
    of the sphere is 1/4, so the (1/8 pi) sum over directions splits into 1/8 per side.  The
    neighbour is any element, thin ones included (Sec. 3.2 notes that heterogeneous mNIP brings
    thin data into the thick submatrix); on the domain boundary the element's own value stands
    for the missing side.  A void neighbour (sigma_t = 0) makes the penalty infinite: the paper
    states that Eq. ModifiedF0 is not compatible with voids, so this is an error.
All integrals use (p+1)-point Gauss rules per direction (volume and faces), so that a nodal
implementation on the same points evaluates the identical bilinear form.  Right-hand side mass
matrix Sigma: sigma_s (default) or sigma_t (footnote of Sec. 2.2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dg import adjugate, face_points, tensor_rule

C_IP = 2.0
C_M = 0.1  # the constant of c(p) in Eq. ModifiedF0 (Sec. 3.1.1)
OPERATORS = ("sip", "nip", "mnip")


class DSA:
    """Assembles D_ff in the oracle's modal basis and applies the Algorithm 2 correction."""

    def __init__(self, T, mask, sigma="sigma_s", c_ip=C_IP, allow_void=False, operator="sip"):
        self.T = T
        if operator not in OPERATORS:
            raise ValueError(f"unknown DSA operator {operator!r}")
        self.operator = operator
        mask = np.asarray(mask).astype(bool).ravel()
        if not allow_void and np.any(T.sigma_t[mask] <= 0):
            raise ValueError("DSA on an element with sigma_t = 0 (full DSA is incompatible with voids)")
        if operator == "mnip":
            nb = T.mesh.nbr[mask]
            if np.any((nb >= 0) & (T.sigma_t[np.maximum(nb, 0)] <= 0)):
                raise ValueError("mNIP penalty next to a void element (Eq. ModifiedF0 is not compatible with voids)")
        self.mask = mask
        self.thick = np.flatnonzero(mask)
        self.local = -np.ones(T.ne, dtype=np.int64)
        self.local[self.thick] = np.arange(self.thick.size)
        self.c_ip = c_ip
        self.sig = T.sigma_s if sigma == "sigma_s" else T.sigma_t
        self.D = self.assemble()
        self.lu = spla.splu(self.D.tocsc()) if self.thick.size else None

    def assemble(self):
        T = self.T
        dim, p, n = T.dim, T.p, T.n
        nt = self.thick.size
        if nt == 0:
            return sp.csr_matrix((0, 0))
        th = self.thick
        Dc = 1.0 / (3.0 * T.sigma_t[th])
        sa = T.sigma_t[th] - T.sigma_s[th]
        cp = self.c_ip * p * (p + 1)
        pts, wts = tensor_rule(p + 1, dim)
        B, dB = T.basis.eval(pts)
        _, J = T.mesh.map(pts)
        J = J[th]
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        # physical gradients: grad u = J^{-T} grad_ref u
        gB = np.einsum("eqkr,qmk->eqmr", Jinv, dB)
        K = (np.einsum("e,q,eq,eqmr,eqnr->emn", Dc, wts, detJ, gB, gB)
             + np.einsum("e,q,eq,qm,qn->emn", sa, wts, detJ, B, B))
        vol = np.einsum("q,eq->e", wts, detJ)
        _, Jall = T.mesh.map(pts)
        vol_all = np.einsum("q,eq->e", wts, np.linalg.det(Jall))   # every element (mNIP neighbours)
        op = self.operator
        cm = C_M * p * (p + 1)
        sym = 1.0 if op == "sip" else 0.0            # weight of the symmetrising face term
        rows, cols, vals = [], [], []

        def add(re, ce, blk):
            ri = (re[:, None] * n + np.arange(n))[:, :, None]
            ci = (ce[:, None] * n + np.arange(n))[:, None, :]
            rows.append(np.broadcast_to(ri, blk.shape).ravel())
            cols.append(np.broadcast_to(ci, blk.shape).ravel())
            vals.append(blk.ravel())

        loc = np.arange(nt)
        add(loc, loc, K)
        tf, wf = tensor_rule(p + 1, dim - 1)
        nbr = T.mesh.nbr[th]
        for f in range(2 * dim):
            a, side = divmod(f, 2)
            s = 1.0 if side else -1.0
            xi = face_points(tf, a, side)
            xo = face_points(tf, a, 1 - side)
            Bf, dBf = T.basis.eval(xi)
            Bo, dBo = T.basis.eval(xo)
            _, Jf = T.mesh.map(xi)
            Jf = Jf[th]
            N = s * adjugate(Jf)[:, :, a, :]            # n dS / dt  (ne_t, qf, dim)
            dS = np.linalg.norm(N, axis=-1) * wf[None, :]
            nrm = N / np.linalg.norm(N, axis=-1)[..., None]
            area = dS.sum(axis=1)
            h = vol / area
            gBf = np.einsum("eqkr,qmk->eqmr", np.linalg.inv(Jf), dBf)
            dn = np.einsum("eqmr,eqr->eqm", gBf, nrm)         # grad(basis).n on this side
            u = nbr[:, f]
            ut = np.where(u >= 0, self.local[np.maximum(u, 0)], -1)
            inter = ut >= 0
            bnd = ~inter
            # boundary-type faces: <kappa u, v> - 1/2 <D du/dn, v> - 1/2 <D dv/dn, u>
            if np.any(bnd):
                e = np.flatnonzero(bnd)
                if op == "sip":
                    kap = np.maximum(0.25, cp * Dc[e] / h[e])
                elif op == "nip":
                    kap = np.full(e.size, 0.25)
                else:
                    st_e = T.sigma_t[th[e]]
                    own = np.maximum(cm / (st_e * h[e]), 1.0)
                    u_all = u[e]
                    has = u_all >= 0
                    ug = np.maximum(u_all, 0)
                    h_o = vol_all[ug] / area[e]
                    other = np.where(has, np.maximum(cm / (np.where(has, T.sigma_t[ug], 1.0) * h_o), 1.0), own)
                    kap = 0.125 * (own + other)
                blk = (np.einsum("e,eq,qm,qn->emn", kap, dS[e], Bf, Bf)
                       - 0.5 * np.einsum("e,eq,eqn,qm->emn", Dc[e], dS[e], dn[e], Bf)
                       - sym * 0.5 * np.einsum("e,eq,eqm,qn->emn", Dc[e], dS[e], dn[e], Bf))
                add(e, e, blk)
            # interior thick-thick faces, assembled once from the side with side == 1
            if side == 1 and np.any(inter):
                e = np.flatnonzero(inter)
                o = ut[e]
                _, Jo = T.mesh.map(xo)
                Jo = Jo[th][o]
                gBo = np.einsum("eqkr,qmk->eqmr", np.linalg.inv(Jo), dBo)
                dno = np.einsum("eqmr,eqr->eqm", gBo, nrm[e])       # neighbour gradient . n (n from e to o)
                ho = vol[o] / area[e]              # conforming faces: same |F| from both sides
                if op == "sip":
                    kap = np.maximum(0.25, cp * 0.5 * (Dc[e] / h[e] + Dc[o] / ho))
                elif op == "nip":
                    kap = np.full(e.size, 0.25)
                else:
                    kap = 0.125 * (np.maximum(cm / (T.sigma_t[th[e]] * h[e]), 1.0)
                                   + np.maximum(cm / (T.sigma_t[th[o]] * ho), 1.0))
                sides = [(e, Bf, dn[e], Dc[e], 1.0), (o, Bo, dno, Dc[o], -1.0)]
                for (ra, Ba, dna, Da, sa_) in sides:
                    for (cb, Bb, dnb, Db, sb_) in sides:
                        # row ra (test v), column cb (trial u): penalty, -{D du/dn}[v], -{D dv/dn}[u]
                        blk = (np.einsum("e,eq,qm,qn->emn", kap * sa_ * sb_, dS[e], Ba, Bb)
                               - 0.5 * np.einsum("e,eq,eqn,qm->emn", Db * sa_, dS[e], dnb, Ba)
                               - sym * 0.5 * np.einsum("e,eq,eqm,qn->emn", Da * sb_, dS[e], dna, Bb))
                        add(ra, cb, blk)
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(nt * n, nt * n))

    def rhs(self, r_modal):
        """Sigma_f r_f: (sigma r, v) on thick elements, flattened."""
        th = self.thick
        return np.einsum("e,emn,en->em", self.sig[th], self.T.M[th], r_modal[th]).ravel()

    def correction(self, r_modal):
        """E_f D_ff^{-1} Sigma_f r_f (Algorithm 2), modal, full-size array."""
        out = np.zeros_like(r_modal)
        if self.thick.size:
            out[self.thick] = self.lu.solve(self.rhs(r_modal)).reshape(-1, self.T.n)
        return out

    def correction_transposed(self, r_modal):
        """Transpose of correction(): E_f Sigma_f D_ff^{-T} E_f^T r (the adjoint iteration's step)."""
        out = np.zeros_like(r_modal)
        th = self.thick
        if th.size:
            z = self.lu.solve(r_modal[th].ravel(), trans="T").reshape(-1, self.T.n)
            out[th] = np.einsum("e,emn,en->em", self.sig[th], self.T.M[th], z)
        return out

    # nodal view of the operator, for comparisons with a nodal implementation
    def nodal_matrix(self):
        """D_ff in GL-nodal coordinates: V^{-T} D V^{-1} (block-diagonal V per element)."""
        nt = self.thick.size
        Vi = sp.block_diag([sp.csr_matrix(self.T.Vinv)] * nt, format="csr") if nt else sp.csr_matrix((0, 0))
        return (Vi.T @ self.D @ Vi).tocsr()


class TriangularDSA:
    """Algorithm 1 (triangular heterogeneous DSA) as the source-iteration correction.

    The preconditioner of Eq. approxS acts on a residual r in two steps:
      1. on the thick region, r_f <- r_f + D_ff^{-1} Sigma_f r_f (the DSA step of Algorithm 2);
      2. with phibar = [0; r_f] (the thin part set to zero, the thick part from step 1), every
         direction adds [w_d L_d^{-1} Sigma_s phibar]_s to the thin part: a transport update with
         zero fixed source and vacuum inflow whose result is kept on the thin DOFs only.
    As a correction of source iteration (phi^{i+1} = phi^i + P r^i = phi_half^i + (P r^i - r^i)) this
    is E_f D_ff^{-1} Sigma_f r_f plus, on the thin DOFs, the accumulated update of step 2.
    """

    def __init__(self, dsa):
        self.dsa = dsa
        self.T = dsa.T

    def homogeneous_update(self, x_modal):
        """sum_d w_d L_d^{-1} Sigma_s x / (4 pi) with no fixed source and vacuum inflow."""
        T = self.T
        zero = np.zeros((T.nd, T.ne, T.n))
        return T.sweep_modal(x_modal, src_per_dir=zero, psi_inc=0.0)

    def correction(self, r_modal):
        c = self.dsa.correction(r_modal)                      # step 1 (thick DOFs)
        phibar = np.zeros_like(r_modal)
        th = self.dsa.thick
        phibar[th] = r_modal[th] + c[th]
        y = self.homogeneous_update(phibar)                   # step 2, accumulated over directions
        thin = ~self.dsa.mask
        out = c.copy()
        out[thin] += y[thin]
        return out


def thick_mask(prob):
    """Thick/thin split of the problem's elements (uint8 per element).

    Rule "sigma_s" (the paper's, Sec. 2.3 and Sec. 3.2 with eta = 1 in Sec. 4.1): thick where
    sigma_s >= eta.  Rule "sigma_t_h": thick where sigma_t h > eta with h the element width 1/nx (an
    optically thick cell).  A void element (sigma_t = 0) is never thick under either rule.
    """
    st = np.asarray(prob.sigma_t, dtype=np.float64)
    ss = np.asarray(prob.sigma_s, dtype=np.float64)
    if prob.thick_rule == "sigma_s":
        return ((ss >= prob.eta) & (st > 0)).astype(np.uint8)
    if prob.thick_rule == "sigma_t_h":
        return (st * (1.0 / prob.nx) > prob.eta).astype(np.uint8)
    raise ValueError(f"unknown thick rule {prob.thick_rule!r}")
