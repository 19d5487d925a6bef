"""ctypes front of the C++ oracle (sweep_ref.cpp): the transport update, the thick-subdomain DSA
operator (SIP) and source iteration with or without the Algorithm 2 correction.

Test infrastructure and timed CPU baseline only: the CUDA library never loads it.  The C++ code
restates the steps of oracle/transport.py and oracle/dsa.py (modal Legendre basis, (p+2)-point
Gauss rules for transport and (p+1)-point rules for the DSA integrals, element systems by Gaussian
elimination, Kahn order of the upwind graph; D_ff solved by block-Jacobi conjugate gradients where
the numpy oracle factorises it) with OpenMP over directions; its inputs are the problem arrays, the
oracle's own direction set and numpy's Gauss rules.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from .quadrature import gauss, level_symmetric

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sweep_ref.cpp")
_LIB = os.path.join(_HERE, "_build", "libsweep_ref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles sweep_ref.cpp with g++ (-O2, OpenMP) into oracle/_build/."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed on sweep_ref.cpp:\n{r.stderr}")
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        i = C.c_int
        lib.sno_sweep.argtypes = [i, i, i, i, i, d, i, d, d, d, d, d, C.c_double, d, d, d, d, d, i, i, i]
        lib.sno_sweep.restype = i
        u8 = C.POINTER(C.c_ubyte)
        lib.sno_dsa_matrix.argtypes = [i, i, i, i, i, d, d, d, u8, d, d, d, d, d, d]
        lib.sno_dsa_matrix.restype = i
        lib.sno_source_iterate.argtypes = [i, i, i, i, i, d, i, d, d, d, d, d, C.c_double, d, d, d, d, d, u8,
                                           C.c_double, i, C.c_double, d, C.POINTER(i), C.POINTER(C.c_double), i]
        lib.sno_source_iterate.restype = i
        lib.sno_max_threads.restype = i
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().sno_max_threads())


def sweep(prob, phi_nodal, directions=None, threads=1):
    """One transport update (Eq. phi) of nodal phi [elem][node] over `directions` (a range, default
    all), as oracle.Transport.sweep computes it."""
    lib = _load()
    dirs, w = level_symmetric(prob.sn, prob.dim)
    nd = len(w)
    d0, d1 = (0, nd) if directions is None else (directions.start, directions.stop)
    gx, gw = gauss(prob.p + 2)
    glx, _ = gauss(prob.p + 1)
    arr = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in
           (dirs, w, prob.sigma_t, prob.sigma_s, prob.q, gx, gw, glx, phi_nodal)]
    verts = None if prob.vertices is None else np.ascontiguousarray(np.asarray(prob.vertices, dtype=np.float64))
    out = np.empty((prob.n_elem, prob.n_nodes))
    ptr = lambda a: None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    st = lib.sno_sweep(prob.dim, prob.nx, prob.ny, prob.nz if prob.dim == 3 else 1, prob.p, ptr(verts), nd,
                       *[ptr(a) for a in arr[:5]], float(prob.psi_inc), *[ptr(a) for a in arr[5:]], ptr(out),
                       d0, d1, int(threads))
    if st != 0:
        raise RuntimeError("an upwind graph has a cycle")
    return out


def _common(prob):
    dirs, w = level_symmetric(prob.sn, prob.dim)
    gx, gw = gauss(prob.p + 2)
    glx, _ = gauss(prob.p + 1)
    gx1, gw1 = gauss(prob.p + 1)
    f64 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64))  # noqa: E731
    verts = None if prob.vertices is None else f64(prob.vertices)
    return dict(dirs=f64(dirs), w=f64(w), st=f64(prob.sigma_t), ss=f64(prob.sigma_s), q=f64(prob.q), gx=f64(gx),
                gw=f64(gw), glx=f64(glx), gx1=f64(gx1), gw1=f64(gw1), verts=verts)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def dsa_matrix(prob, mask):
    """The SIP thick-subdomain operator D_ff in the modal basis (dense, thick elements in order)."""
    lib = _load()
    c = _common(prob)
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
    nt = int(m.astype(bool).sum())
    N = nt * prob.n_nodes
    out = np.empty((N, N))
    lib.sno_dsa_matrix(prob.dim, prob.nx, prob.ny, prob.nz if prob.dim == 3 else 1, prob.p, _p(c["verts"]),
                       _p(c["st"]), _p(c["ss"]), m.ctypes.data_as(C.POINTER(C.c_ubyte)), _p(c["gx"]), _p(c["gw"]),
                       _p(c["glx"]), _p(c["gx1"]), _p(c["gw1"]), _p(out))
    return out


def source_iterate(prob, mask=None, tol=1e-8, max_iters=1000, cg_tol=1e-15, threads=1):
    """Source iteration from phi = 0 (Eq. DSA_fp), with the Algorithm 2 correction on the elements of
    `mask` (SIP operator, Sigma = sigma_s) or unaccelerated (mask None).  Returns dict(phi=nodal phi,
    iters, rel_residual)."""
    lib = _load()
    c = _common(prob)
    m = None if mask is None else np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
    out = np.empty((prob.n_elem, prob.n_nodes))
    it = C.c_int(0)
    rel = C.c_double(0.0)
    st = lib.sno_source_iterate(prob.dim, prob.nx, prob.ny, prob.nz if prob.dim == 3 else 1, prob.p,
                                _p(c["verts"]), len(c["w"]), _p(c["dirs"]), _p(c["w"]), _p(c["st"]), _p(c["ss"]),
                                _p(c["q"]), float(prob.psi_inc), _p(c["gx"]), _p(c["gw"]), _p(c["glx"]),
                                _p(c["gx1"]), _p(c["gw1"]),
                                None if m is None else m.ctypes.data_as(C.POINTER(C.c_ubyte)), float(tol),
                                int(max_iters), float(cg_tol), _p(out), C.byref(it), C.byref(rel), int(threads))
    if st != 0:
        raise RuntimeError("an upwind graph has a cycle")
    return {"phi": out, "iters": it.value, "rel_residual": rel.value}
