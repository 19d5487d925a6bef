"""ctypes front of the C++ oracle of the transport update (sweep_ref.cpp).

Test infrastructure and timed CPU baseline only: the CUDA library never loads it.  The C++ code
restates the steps of oracle/transport.py (modal Legendre basis, (p+2)-point Gauss rules, element
systems by Gaussian elimination, Kahn order of the upwind graph) with OpenMP over directions; its
inputs are the problem arrays, the oracle's own direction set and numpy's Gauss rules.
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
