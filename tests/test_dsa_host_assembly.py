"""CPU: the library's host assembly of the thick-subdomain DSA operator (sn::dsa_build, Sec. 3.1-3.2:
Eq. SIP, Eq. NIP and Eq. NIP with the penalty of Eq. ModifiedF0, and the transposed operator the
adjoint solves with) against the oracle's operator, element block by element block.

The library assembles in the nodal Gauss-Legendre basis, the oracle in a modal Legendre basis; both
use the (p+1)-point Gauss rule, so the nodal view of the oracle's matrix, V^{-T} D V^{-1}, must
equal the library's to rounding (1e-12 relative to the largest entry).  A small driver
(tests/host_drivers/dsa_dump.cpp) links the library's host setup sources and needs no GPU.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs
from oracle.dsa import thick_mask

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2001_09196_gb300", "csrc")
OPS = {"sip": 0, "nip": 1, "mnip": 2}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("host_drivers") / "dsa_dump")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "host_drivers", "dsa_dump.cpp"), os.path.join(CSRC, "sn_dsa_setup.cpp"),
                    os.path.join(CSRC, "sn_setup.cpp"), "-lpthread", "-o", exe], check=True)
    return exe


def _assemble(driver, tmp_path, prob, mask, op, transposed, levels=False):
    inp, out, lev = tmp_path / "in.bin", tmp_path / "out.bin", tmp_path / "levels.bin"
    has_v = prob.dim == 2 and prob.vertices is not None
    with open(inp, "wb") as f:
        f.write(struct.pack("8i", prob.dim, prob.nx, prob.ny, prob.nz, prob.p, OPS[op], int(transposed), int(has_v)))
        f.write(np.ascontiguousarray(prob.sigma_t, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(prob.sigma_s, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(mask, dtype=np.uint8).tobytes())
        if has_v:
            f.write(np.ascontiguousarray(prob.vertices, dtype=np.float64).tobytes())
    subprocess.run([driver, str(inp), str(out)] + ([str(lev)] if levels else []), check=True, capture_output=True)
    raw = open(out, "rb").read()
    status, nt, n, nnzb = struct.unpack_from("4i", raw, 0)
    if status:
        return None, bool(nt)
    off = 16
    thick = np.frombuffer(raw, np.int32, nt, off); off += 4 * nt
    ptr = np.frombuffer(raw, np.int32, nt + 1, off); off += 4 * (nt + 1)
    col = np.frombuffer(raw, np.int32, nnzb, off); off += 4 * nnzb
    val = np.frombuffer(raw, np.float64, nnzb * n * n, off).reshape(nnzb, n, n)
    D = np.zeros((nt * n, nt * n))
    for r in range(nt):
        for k in range(ptr[r], ptr[r + 1]):
            D[r * n:(r + 1) * n, col[k] * n:(col[k] + 1) * n] = val[k]
    if levels:
        return (thick, D, _read_levels(open(lev, "rb").read())), False
    return (thick, D), False


def _read_levels(raw):
    import scipy.sparse as sp
    (count,) = struct.unpack_from("i", raw, 0)
    off, out = 4, []
    for _ in range(count):
        rows, prow, annz, pnnz, dense = struct.unpack_from("5i", raw, off)
        off += 20

        def take(dtype, k):
            nonlocal off
            a = np.frombuffer(raw, dtype, k, off)
            off += a.nbytes
            return a
        ap, ac, av = take(np.int32, rows + 1), take(np.int32, annz), take(np.float64, annz)
        pp, pc, pv = take(np.int32, prow + 1), take(np.int32, pnnz), take(np.float64, pnnz)
        rp, rc, rv = take(np.int32, rows + 1), take(np.int32, pnnz), take(np.float64, pnnz)
        A = sp.csr_matrix((av, ac, ap), shape=(rows, rows)).toarray()
        P = sp.csr_matrix((pv, pc, pp), shape=(prow, rows)).toarray()
        R = sp.csr_matrix((rv, rc, rp), shape=(rows, prow)).toarray()
        assert np.all(np.diff(rp) >= 0) and all(np.all(np.diff(rc[rp[i]:rp[i + 1]]) > 0) for i in range(rows))
        inv = take(np.float64, rows * rows).reshape(rows, rows) if dense else None
        out.append((A, P, R, inv))
    return out


def _void_free_c1():
    prob = inputs.config1()
    v = prob.sigma_t == 0
    prob.sigma_t[v], prob.sigma_s[v] = 1.0, 0.9
    return prob


CASES = {
    "c1": inputs.config1,
    "c1_full": _void_free_c1,
    "c2_jittered_q2": lambda: inputs.config2(n=16, block=4, p=2, sn=4),
    "q3": lambda: inputs.config2d_fields(6, 3, 4, 81, "q3"),
    "c3_q1": lambda: inputs.config3(n=4),
    "c3_q2": lambda: inputs.config3(n=3, p=2),
}


@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("op", ["sip", "nip", "mnip"])
@pytest.mark.parametrize("name", list(CASES))
def test_host_assembly_matches_the_oracle(driver, tmp_path, name, op, transposed):
    from oracle import Transport
    from oracle.dsa import DSA
    prob = CASES[name]()
    T = Transport(prob)
    mask = np.ones(T.ne, dtype=np.uint8) if name == "c1_full" else thick_mask(prob).astype(np.uint8)
    try:
        ref = DSA(T, mask, operator=op)
    except ValueError:  # mNIP next to a void: the library must refuse it too, as a void conflict
        got, void_conflict = _assemble(driver, tmp_path, prob, mask, op, transposed)
        assert got is None and void_conflict
        return
    got, _ = _assemble(driver, tmp_path, prob, mask, op, transposed)
    assert got is not None
    thick, D = got
    assert np.array_equal(thick, ref.thick)
    Dn = ref.nodal_matrix().toarray()
    if transposed and op != "sip":
        Dn = Dn.T
    assert np.abs(D - Dn).max() <= 1e-12 * np.abs(Dn).max()
    if op != "sip":
        assert np.abs(Dn - Dn.T).max() > 1e-6 * np.abs(Dn).max()  # and the nonsymmetric ones are so


@pytest.mark.parametrize("op", ["sip", "nip"])
@pytest.mark.parametrize("name", ["c1_full", "c2_jittered_q2", "c3_q1"])
def test_multigrid_hierarchy_is_galerkin(driver, tmp_path, name, op):
    """The hierarchy behind the V-cycle: every continuous level's operator is P^T A P of the level
    above, every prolongation row is an interpolation (weights summing to 1), and the coarsest
    level holds the inverse of its operator."""
    prob = CASES[name]()
    mask = np.ones(prob.n_elem, dtype=np.uint8) if name == "c1_full" else thick_mask(prob).astype(np.uint8)
    got, _ = _assemble(driver, tmp_path, prob, mask, op, False, levels=True)
    _, D, levels = got
    assert levels and levels[-1][3] is not None
    fine = D
    for A, P, R, inv in levels:
        assert P.shape == (fine.shape[0], A.shape[0])
        assert np.array_equal(R, P.T)                # the restriction is exactly P^T, columns ascending
        assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-12
        G = P.T @ fine @ P
        assert np.abs(A - G).max() <= 1e-11 * np.abs(G).max()
        fine = A
    A, _, _, inv = levels[-1]
    assert np.abs(inv @ A - np.eye(A.shape[0])).max() < 1e-8
