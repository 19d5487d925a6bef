"""Differentiable transport solves: torch.autograd.Functions over the libsn C ABI.

phi = SnSolve.apply(sigma_t, sigma_s, q, mesh, solve_opts, adjoint_opts) solves the DG S_N system
(Eq. system) for per-element cross sections and source.  For any scalar loss L(phi) the backward
pass receives g = dL/dphi (nodal values) and returns dL/dsigma_t, dL/dsigma_s and dL/dq:

  * the adjoint solve S^T mu = g (sn_adjoint_iterate: reverse sweeps with the transposed DSA
    step as the preconditioner of flexible GMRES),
  * one forward sweep from the saved phi to regenerate psi_d and one adjoint sweep from mu for
    lambda_d = w_d L_d^{-T} mu, and the per-element contractions of sn_gradients.
The forward pass keeps only the converged scalar flux phi (n_elem x n_nodes values), never the
angular fluxes (n_dirs times larger); the backward recomputes them from phi.

phi_K = SnUnrolled.apply(sigma_t, sigma_s, q, mesh, K, checkpoint_every) is the K-th iterate of
source iteration without acceleration from phi_0 = 0 (Eq. source0: phi_{k+1} = T phi_k + b), a
deterministic function of the data with no solver tolerance in it.  Its forward pass keeps every
checkpoint_every-th iterate (sn_source_iterate's checkpoints); the backward pass
(sn_unrolled_gradients) runs the adjoint recursion mu_k = T^T mu_{k+1} from mu_K = g in reverse,
recomputing each segment of iterates from its checkpoint, and sums every update's gradient
contractions.
All numerical work runs in libsn; this module only moves tensors and chains the calls.
"""
from __future__ import annotations

import torch

from . import sn as _sn


class SnSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, q, mesh, solve_opts=None, adjoint_opts=None):
        solve_opts = dict(solve_opts or {})
        adjoint_opts = dict(adjoint_opts or {})
        st, ss, qq = (x.detach().contiguous().to(torch.float64) for x in (sigma_t, sigma_s, q))
        mesh.set_materials(st, ss, qq)
        r = mesh.source_iterate(**solve_opts)
        if not r["converged"]:
            raise RuntimeError(f"forward transport solve did not converge (rel. residual {r['rel_residual']:.3e})")
        phi = r["phi"]
        ctx.mesh = mesh
        ctx.adjoint_opts = adjoint_opts
        ctx.save_for_backward(st, ss, qq, phi)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        st, ss, qq, phi = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_materials(st, ss, qq)  # the mesh may have been re-used since the forward pass
        a = mesh.adjoint_iterate(grad_phi.contiguous().to(torch.float64), **ctx.adjoint_opts)
        if not a["converged"]:
            raise RuntimeError(f"adjoint solve did not converge (rel. residual {a['rel_residual']:.3e})")
        gt, gs, gq = mesh.gradients(phi, a["mu"])
        return gt, gs, gq, None, None, None


class SnUnrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, q, mesh, K, checkpoint_every=1):
        st, ss, qq = (x.detach().contiguous().to(torch.float64) for x in (sigma_t, sigma_s, q))
        mesh.set_materials(st, ss, qq)
        n_ck = max(K // checkpoint_every, 1)
        ck = torch.empty((n_ck,) + mesh.shape, dtype=torch.float64, device=st.device)
        r = mesh.source_iterate(dsa="none", tol=0.0, max_iters=K, checkpoint_every=checkpoint_every, checkpoints=ck)
        if r["iters"] != K:
            raise RuntimeError(f"the unaccelerated iteration stopped after {r['iters']} of {K} updates")
        ctx.mesh = mesh
        ctx.K, ctx.every = K, checkpoint_every
        ctx.save_for_backward(st, ss, qq, ck)
        return r["phi"]

    @staticmethod
    def backward(ctx, grad_phi):
        st, ss, qq, ck = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_materials(st, ss, qq)  # the mesh may have been re-used since the forward pass
        g = grad_phi.contiguous().to(torch.float64)
        gt, gs, gq = mesh.unrolled_gradients(g, ctx.K, ctx.every, checkpoints=ck)
        return gt, gs, gq, None, None, None


DEFAULT_SOLVE = dict(dsa="thick", outer="fgmres", restart=30, tol=1e-12, inner_tol=1e-10, max_iters=600,
                     inner_max_iters=500)


def solve(mesh, sigma_t, sigma_s, q, solve_opts=None, adjoint_opts=None):
    """Differentiable phi(sigma_t, sigma_s, q) on `mesh` (a paper_2001_09196_gb300.sn.Mesh)."""
    so = dict(DEFAULT_SOLVE, **(solve_opts or {}))
    ao = dict(DEFAULT_SOLVE, **(adjoint_opts or {}))
    ao.pop("precision", None)
    # the adjoint's DSA step is the transpose of the forward one: same thick set, operator and Sigma
    for k in ("thick_rule", "eta", "mask", "operator", "dsa_sigma"):
        if k in so and k not in ao:
            ao[k] = so[k]
    return SnSolve.apply(sigma_t, sigma_s, q, mesh, so, ao)


def unrolled(mesh, sigma_t, sigma_s, q, K, checkpoint_every=1):
    """Differentiable phi_K(sigma_t, sigma_s, q): K unaccelerated transport updates from phi = 0."""
    return SnUnrolled.apply(sigma_t, sigma_s, q, mesh, int(K), int(checkpoint_every))
