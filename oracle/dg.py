"""Mesh, modal basis and geometry for the CPU oracle (test infrastructure only).

The oracle works in a *modal* tensor-Legendre basis of Q_p and integrates with
p+2 Gauss points per direction, which is exact for every integral of the upwind
DG transport operator on bilinear (2D) and affine (3D) elements.  Results are
converted to values at the (p+1)^d tensor Gauss-Legendre nodes only for
comparison, so that the oracle and a nodal implementation reach the same discrete
function along different routes.

Conventions (shared with the library only as a documented data layout):
  * elements: structured nx x ny (x nz), lexicographic with x fastest;
  * element corners: corner c has reference coordinate xi_a = +1 if bit a of c is
    set, else -1; it is vertex (i + bit0, j + bit1, k + bit2);
  * faces: f = 2*a + side, side 0 at xi_a = -1, side 1 at xi_a = +1;
  * GL nodes inside an element: lexicographic with x fastest.
"""
from __future__ import annotations

import itertools

import numpy as np

from .quadrature import dlegendre, gauss, legendre


class Mesh:
    def __init__(self, dim, nx, ny, nz=1, vertices=None):
        self.dim = dim
        self.nx, self.ny, self.nz = nx, ny, (nz if dim == 3 else 1)
        shape = (self.nx, self.ny, self.nz)[:dim]
        nv = [s + 1 for s in shape]
        if vertices is None:
            axes = [np.linspace(0.0, 1.0, s + 1) for s in shape]
            grids = np.meshgrid(*axes, indexing="ij")  # grids[a][i, j, k]
            V = np.stack([g.transpose(list(range(dim))[::-1]).ravel() for g in grids], axis=-1)
        else:
            V = np.asarray(vertices, dtype=np.float64).reshape(-1, dim)
            assert V.shape[0] == int(np.prod(nv))
        self.vertices = V
        self.n_elem = int(np.prod(shape))
        idx = np.array(list(itertools.product(*[range(s) for s in shape[::-1]])))[:, ::-1]
        self.ijk = idx  # (ne, dim), element e -> (i, j[, k]); x fastest
        strides = np.cumprod([1] + nv[:-1])
        corners = []
        for c in range(2 ** dim):
            off = np.array([(c >> a) & 1 for a in range(dim)])
            corners.append(((idx + off) * strides).sum(axis=1))
        self.corners = np.stack(corners, axis=1)  # (ne, 2^dim) vertex ids
        estrides = np.cumprod([1] + list(shape[:-1]))
        nbr = -np.ones((self.n_elem, 2 * dim), dtype=np.int64)
        for a in range(dim):
            for side in (0, 1):
                d = -1 if side == 0 else 1
                j = idx.copy()
                j[:, a] += d
                ok = (j[:, a] >= 0) & (j[:, a] < shape[a])
                nbr[ok, 2 * a + side] = (j[ok] * estrides).sum(axis=1)
        self.nbr = nbr
        self.shape = shape

    def map(self, xi):
        """Physical points, Jacobians for reference points xi (npts, dim).

        Returns x (ne, npts, dim) and J (ne, npts, dim, dim) with J[.., r, c] = dx_r/dxi_c.
        """
        dim = self.dim
        xi = np.atleast_2d(xi)
        N = np.ones((xi.shape[0], 2 ** dim))
        dN = np.ones((xi.shape[0], 2 ** dim, dim))
        for c in range(2 ** dim):
            s = np.array([1.0 if (c >> a) & 1 else -1.0 for a in range(dim)])
            fac = 0.5 * (1.0 + s[None, :] * xi)  # (npts, dim)
            N[:, c] = np.prod(fac, axis=1)
            for a in range(dim):
                others = np.prod(np.delete(fac, a, axis=1), axis=1) if dim > 1 else 1.0
                dN[:, c, a] = 0.5 * s[a] * others
        X = self.vertices[self.corners]  # (ne, 2^dim, dim)
        x = np.einsum("qc,ecr->eqr", N, X)
        J = np.einsum("qca,ecr->eqra", dN, X)
        return x, J


def adjugate(J):
    """adj(J) = det(J) J^{-1} for stacks of 2x2 or 3x3 matrices."""
    if J.shape[-1] == 2:
        A = np.empty_like(J)
        A[..., 0, 0] = J[..., 1, 1]
        A[..., 0, 1] = -J[..., 0, 1]
        A[..., 1, 0] = -J[..., 1, 0]
        A[..., 1, 1] = J[..., 0, 0]
        return A
    det = np.linalg.det(J)
    return det[..., None, None] * np.linalg.inv(J)


class ModalBasis:
    """Tensor Legendre basis of Q_p; mode m = (m_0, .., m_{d-1}) lexicographic, x fastest."""

    def __init__(self, p, dim):
        self.p, self.dim = p, dim
        self.modes = [tuple(t[::-1]) for t in itertools.product(range(p + 1), repeat=dim)]
        self.n = len(self.modes)

    def eval(self, xi):
        """Values (npts, n) and reference gradients (npts, n, dim) at points xi (npts, dim)."""
        xi = np.atleast_2d(xi)
        P = np.stack([legendre(m, xi) for m in range(self.p + 1)], axis=-1)   # (npts, dim, p+1)
        dP = np.stack([dlegendre(m, xi) for m in range(self.p + 1)], axis=-1)
        B = np.ones((xi.shape[0], self.n))
        dB = np.ones((xi.shape[0], self.n, self.dim))
        for k, mode in enumerate(self.modes):
            for a in range(self.dim):
                B[:, k] *= P[:, a, mode[a]]
                for b in range(self.dim):
                    dB[:, k, b] *= (dP if a == b else P)[:, a, mode[a]]
        return B, dB


def tensor_rule(npts, dim):
    """Tensor Gauss rule on [-1,1]^dim: points (npts^dim, dim) x fastest, weights."""
    x, w = gauss(npts)
    pts = np.array([t[::-1] for t in itertools.product(x, repeat=dim)])
    wts = np.array([np.prod(t) for t in itertools.product(w, repeat=dim)])
    return pts, wts


def face_points(t, a, side):
    """Insert xi_a = +-1 into face coordinates t (npts, dim-1)."""
    t = np.atleast_2d(t)
    return np.insert(t, a, 1.0 if side else -1.0, axis=1)


def nodal_matrix(p, dim):
    """V (n_nodes, n_modes): values of the modal basis at the (p+1)^dim GL nodes."""
    pts, _ = tensor_rule(p + 1, dim)
    B, _ = ModalBasis(p, dim).eval(pts)
    return B
