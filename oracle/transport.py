"""Upwind DG S_N transport: sweep and source iteration (CPU oracle, test infrastructure only).

What is computed (paper references are to sections / equations):
  * Eq. (sntransport): for every direction d,
        Omega_d . grad psi_d + sigma_t psi_d = q_d + sigma_s/(4 pi) sum_d' w_d' psi_d',
    psi_d = psi_inc on inflow boundary faces, phi = sum_d w_d psi_d, sum_d w_d = 4 pi.
    The isotropic source q (total emission per unit volume) gives q_d = q/(4 pi).
  * Upwind DG in space (Sec. 3.1, Eq. Tmat1): on element K with test function v,
        -(psi, Omega.grad v)_K + (sigma_t psi, v)_K + sum_{F outflow} <(Omega.n) psi, v>_F
          = (S, v)_K - sum_{F inflow} <(Omega.n) psi_up, v>_F ,
    psi_up the upwind neighbour's trace, or psi_inc on the domain boundary.  (The
    printed q_inc form has a garbled sign; the standard upwind boundary term is used.)
  * The transport update inverts L_d for all d (Sec. 1): a forward block solve of the
    element systems in an upwind (topological) order of the mesh, built here with
    Kahn's algorithm from the sign of Omega.n on each face.
  * Source iteration (Eq. psi / phi, Eq. source0) with the DSA fixed point Eq. DSA_fp:
        phi_half^i = sum_d w_d L_d^{-1}(q_d + Sigma_s phi^i),   r^i = phi_half^i - phi^i,
        phi^{i+1}  = phi_half^i + E_f D_ff^{-1} Sigma_f r^i_f          (Algorithm 2),
    stopping after the iteration in which ||r^i|| <= tol ||r^0|| (Euclidean norm of the
    GL-nodal values), phi^0 = 0 unless a warm start is given.

All arithmetic is float64.  The element systems are formed in a modal Legendre basis with
exact (p+2)-point Gauss integration and solved with numpy.linalg.solve.
"""
from __future__ import annotations

import numpy as np

from .dg import Mesh, ModalBasis, adjugate, face_points, nodal_matrix, tensor_rule
from .quadrature import gauss, level_symmetric

FOUR_PI = 4.0 * np.pi


class CycleError(RuntimeError):
    pass


class Transport:
    """Oracle discretisation of one problem (see module docstring)."""

    def __init__(self, prob, n_exact=None):
        self.prob = prob
        self.dim, self.p = prob.dim, prob.p
        dim, p = self.dim, self.p
        self.mesh = Mesh(dim, prob.nx, prob.ny, prob.nz, prob.vertices)
        self.ne = self.mesh.n_elem
        self.dirs, self.w = level_symmetric(prob.sn, dim)
        self.nd = len(self.w)
        self.basis = ModalBasis(p, dim)
        self.n = self.basis.n
        self.V = nodal_matrix(p, dim)            # nodal values = V @ modal coefficients
        self.Vinv = np.linalg.inv(self.V)
        self.sigma_t = np.asarray(prob.sigma_t, dtype=np.float64)
        self.sigma_s = np.asarray(prob.sigma_s, dtype=np.float64)
        self.q = np.asarray(prob.q, dtype=np.float64)
        nq = n_exact if n_exact is not None else p + 2
        # volume: mass and the advection pieces G_l with Adv = sum_l Omega_l G_l
        pts, wts = tensor_rule(nq, dim)
        B, dB = self.basis.eval(pts)
        x, J = self.mesh.map(pts)
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("mesh has an inverted element")
        adj = adjugate(J)                         # (ne, q, dim, dim)
        self.M = np.einsum("q,eq,qm,qn->emn", wts, detJ, B, B)
        # -(psi, Omega . grad v): test m, trial n; Omega.grad v detJ = (adj(J) Omega) . grad_ref v
        self.G = -np.einsum("q,qn,eqkl,qmk->lemn", wts, B, adj, dB)
        self.volume = np.einsum("q,eq->e", wts, detJ)
        # faces
        tf, wf = tensor_rule(nq, dim - 1) if dim > 1 else (np.zeros((1, 0)), np.ones(1))
        self.face_w = wf
        self.BF, self.BFo, self.FN, self.face_x = [], [], [], []
        for f in range(2 * dim):
            a, side = divmod(f, 2)
            s = 1.0 if side else -1.0
            xi = face_points(tf, a, side)
            xio = face_points(tf, a, 1 - side)
            Bf, _ = self.basis.eval(xi)
            Bo, _ = self.basis.eval(xio)
            xf, Jf = self.mesh.map(xi)
            adjf = adjugate(Jf)
            # Nanson: n dS = detJ J^{-T} (s e_a) dt  =>  Omega.n dS = s (adj(J) Omega)_a dt
            self.FN.append(s * adjf[:, :, a, :] * wf[None, :, None])  # (ne, qf, dim)
            self.BF.append(Bf)
            self.BFo.append(Bo)
            self.face_x.append(xf)

    # ----- conversions -------------------------------------------------------------
    def project(self, f):
        """L2 projection onto Q_p of f(x (ne, q, dim)) -> (ne, q) values; modal (ne, n)."""
        pts, wts = tensor_rule(self.p + 2, self.dim)
        B, _ = self.basis.eval(pts)
        x, J = self.mesh.map(pts)
        detJ = np.linalg.det(J)
        rhs = np.einsum("q,eq,qm,eq->em", wts, detJ, B, f(x))
        return np.linalg.solve(self.M, rhs[..., None])[..., 0]

    def l2_error(self, modal, f, extra=3):
        """|| u_h - f ||_L2 with a (p+1+extra)-point tensor Gauss rule."""
        pts, wts = tensor_rule(self.p + 1 + extra, self.dim)
        B, _ = self.basis.eval(pts)
        x, J = self.mesh.map(pts)
        detJ = np.linalg.det(J)
        err = modal @ B.T - f(x)
        return float(np.sqrt(np.einsum("q,eq,eq->", wts, detJ, err * err)))

    def to_modal(self, nodal):
        return np.asarray(nodal, dtype=np.float64).reshape(self.ne, self.n) @ self.Vinv.T

    def to_nodal(self, modal):
        return modal @ self.V.T

    def isotropic_source(self, phi_modal):
        """Modal coefficients of S = (q + sigma_s phi)/(4 pi) on each element."""
        S = (self.sigma_s[:, None] * phi_modal) / FOUR_PI
        S[:, 0] += self.q / FOUR_PI  # P_0 = 1
        return S

    # ----- one direction -------------------------------------------------------------
    def face_flux(self, d):
        """Per face f: Omega.n dS weights at face points (ne, qf)."""
        Om = self.dirs[d][: self.dim]
        return [fn @ Om for fn in self.FN]

    def levels(self, d, fw=None):
        """Kahn levels of the upwind graph of direction d (list of element arrays)."""
        fw = fw if fw is not None else self.face_flux(d)
        ne, nbr = self.ne, self.mesh.nbr
        fsum = np.stack([x.sum(axis=1) for x in fw], axis=1)  # (ne, 2 dim)
        for f, x in enumerate(fw):
            mixed = (x.max(axis=1) > 0) & (x.min(axis=1) < 0)
            if np.any(mixed):
                raise ValueError("face with both inflow and outflow points")
        inflow_interior = (fsum < 0) & (nbr >= 0)
        indeg = inflow_interior.sum(axis=1)
        out = []
        frontier = np.flatnonzero(indeg == 0)
        done = 0
        while frontier.size:
            out.append(frontier)
            done += frontier.size
            nxt = []
            for f in range(2 * self.dim):
                src = frontier[(fsum[frontier, f] > 0) & (nbr[frontier, f] >= 0)]
                dst = nbr[src, f]
                np.subtract.at(indeg, dst, 1)
                nxt.append(dst)
            cand = np.unique(np.concatenate(nxt)) if nxt else np.zeros(0, dtype=np.int64)
            frontier = cand[indeg[cand] == 0]
        if done != ne:
            raise CycleError(f"direction {d}: upwind graph has a cycle")
        return out

    def element_matrices(self, d, fw=None):
        """A_e = sigma_t M + Adv + sum_{outflow F} face matrix, for all elements (ne, n, n)."""
        fw = fw if fw is not None else self.face_flux(d)
        Om = self.dirs[d][: self.dim]
        A = self.sigma_t[:, None, None] * self.M + np.einsum("l,lemn->emn", Om, self.G)
        for f in range(2 * self.dim):
            out = fw[f].sum(axis=1) > 0
            A[out] += np.einsum("eq,qm,qn->emn", fw[f][out], self.BF[f], self.BF[f])
        return A

    def sweep_direction(self, d, src_modal, psi_inc=None):
        """Solve L_d psi = M src + inflow terms; returns modal psi (ne, n).

        psi_inc: None -> the problem's constant; float; or callable(x (.., dim), Omega) -> values.
        """
        fw = self.face_flux(d)
        A = self.element_matrices(d, fw)
        rhs = np.einsum("emn,en->em", self.M, src_modal)
        psi = np.zeros((self.ne, self.n))
        inc = self.prob.psi_inc if psi_inc is None else psi_inc
        Om = self.dirs[d]
        for E in self.levels(d, fw):
            r = rhs[E].copy()
            for f in range(2 * self.dim):
                inflow = fw[f][E].sum(axis=1) < 0
                if not np.any(inflow):
                    continue
                Ein = E[inflow]
                u = self.mesh.nbr[Ein, f]
                trace = np.empty((Ein.size, self.face_w.size))
                interior = u >= 0
                trace[interior] = psi[u[interior]] @ self.BFo[f].T
                if np.any(~interior):
                    if callable(inc):
                        trace[~interior] = inc(self.face_x[f][Ein[~interior]], Om)
                    else:
                        trace[~interior] = float(inc)
                r[inflow] -= np.einsum("eq,qm,eq->em", fw[f][Ein], self.BF[f], trace)
            psi[E] = np.linalg.solve(A[E], r[..., None])[..., 0]
        return psi

    # ----- full transport update ---------------------------------------------------------
    def sweep_modal(self, phi_modal, src_per_dir=None, psi_inc=None, keep_psi=False, directions=None):
        """phi_half = sum_d w_d L_d^{-1}(q_d + Sigma_s phi) in modal coefficients (Eq. phi); with
        `directions` the sum runs over those directions only (a partial transport update)."""
        out = np.zeros((self.ne, self.n))
        psis = [] if keep_psi else None
        scatter = (self.sigma_s[:, None] * phi_modal) / FOUR_PI
        iso = self.isotropic_source(np.zeros_like(phi_modal))
        for d in (range(self.nd) if directions is None else directions):
            # src_per_dir (modal, per direction) replaces the isotropic q/(4 pi) when given
            src = scatter + (iso if src_per_dir is None else src_per_dir[d])
            psi = self.sweep_direction(d, src, psi_inc)
            out += self.w[d] * psi
            if keep_psi:
                psis.append(psi)
        return (out, psis) if keep_psi else out

    def sweep(self, phi_nodal, directions=None):
        """One transport update on GL-nodal data [elem][node] (Eq. source0), or its partial sum over
        `directions`."""
        return self.to_nodal(self.sweep_modal(self.to_modal(phi_nodal), directions=directions))

    # ----- source iteration -------------------------------------------------------------
    def source_iterate(self, dsa=None, tol=1e-8, max_iters=1000, phi0_nodal=None,
                       history=False, src_per_dir=None, psi_inc=None, checkpoint_every=0):
        """Source iteration with an optional DSA correction object (see dsa.py).

        Returns dict(phi=nodal phi, iters, rel_residual, converged, history, checkpoints).
        """
        phi = np.zeros((self.ne, self.n)) if phi0_nodal is None else self.to_modal(phi0_nodal)
        r0 = None
        hist, ckpts = [], []
        it = 0
        converged = False
        rel = np.inf
        while it < max_iters:
            half = self.sweep_modal(phi, src_per_dir=src_per_dir, psi_inc=psi_inc)
            r = half - phi
            rn = np.linalg.norm(self.to_nodal(r))
            if r0 is None:
                r0 = rn if rn > 0 else 1.0
            rel = rn / r0
            hist.append(rel)
            phi = half if dsa is None else half + dsa.correction(r)
            it += 1
            if checkpoint_every and it % checkpoint_every == 0:
                ckpts.append(self.to_nodal(phi))
            if rel <= tol:
                converged = True
                break
        return {"phi": self.to_nodal(phi), "iters": it, "rel_residual": rel, "converged": converged,
                "history": hist if history else None, "checkpoints": ckpts}
