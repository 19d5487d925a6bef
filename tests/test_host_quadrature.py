"""CPU: the library's quadrature data from its host setup code (tests/host_drivers/quad_dump.cpp,
no GPU) against the oracle's level-symmetric sets (themselves pinned to the textbook tables) and
against numpy's Gauss-Legendre rule and Lagrange basis.

The library and the oracle compute their level-symmetric sets independently; the transport
parity tests rely on both using the same directions and weights (Sec. 4.1, S8 = 40 angles in 2D).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2001_09196_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("host_drivers") / "quad_dump")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "host_drivers", "quad_dump.cpp"), os.path.join(CSRC, "sn_setup.cpp"),
                    "-o", exe], check=True)
    return exe


def _run(driver, *args):
    out = subprocess.run([driver, *map(str, args)], capture_output=True, text=True, check=True).stdout
    return np.array([[float(v) for v in line.split()] for line in out.strip().splitlines()])


@pytest.mark.parametrize("N,dim", [(4, 2), (6, 2), (8, 2), (4, 3), (6, 3), (8, 3)])
def test_level_symmetric_sets_match_the_oracle(driver, N, dim):
    from oracle.quadrature import level_symmetric
    got = _run(driver, "ls", N, dim)
    d, w = level_symmetric(N, dim)
    ref = np.hstack([np.asarray(d), np.asarray(w)[:, None]])
    assert got.shape == ref.shape
    key = lambda a: np.lexsort(np.round(a[:, :3], 12).T[::-1])
    assert np.abs(got[key(got)] - ref[key(ref)]).max() < 1e-14
    assert abs(got[:, 3].sum() - 4 * np.pi) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_gauss_legendre_nodal_data(driver, p):
    got = _run(driver, "gl", p)
    x, w = np.polynomial.legendre.leggauss(p + 1)
    assert np.abs(got[:, 0] - x).max() < 1e-14 and np.abs(got[:, 1] - w).max() < 1e-14
    # Lagrange basis l_k through the nodes: monomial coefficients from the Vandermonde system
    V = np.vander(x, p + 1, increasing=True)
    C = np.linalg.solve(V, np.eye(p + 1))          # column k: coefficients of l_k
    val = lambda t: np.array([np.polynomial.polynomial.polyval(t, C[:, k]) for k in range(p + 1)])
    der = lambda t: np.array([np.polynomial.polynomial.polyval(t, np.polynomial.polynomial.polyder(C[:, k]))
                              for k in range(p + 1)])
    assert np.abs(got[:, 2] - val(-1.0)).max() < 1e-12 and np.abs(got[:, 3] - val(1.0)).max() < 1e-12
    D = np.array([der(xa) for xa in x])            # D[a, k] = l_k'(x_a)
    assert np.abs(got[:, 4:] - D).max() < 1e-11
