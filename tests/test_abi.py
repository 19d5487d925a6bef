"""CPU-side checks of the C-ABI library: it builds, loads and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sn.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sn_status|void|const char\*)\s+(sn_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2001_09196_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for required in ("sn_mesh_create", "sn_sweep", "sn_source_iterate", "sn_adjoint_sweep", "sn_gradients",
                     "sn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    import ctypes
    lib = ctypes.CDLL(libpath)
    lib.sn_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sn_version()
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_loads_and_defaults(libpath):
    from paper_2001_09196_gb300 import sn
    o = sn.make_opts()
    assert o.dsa == sn.DSA_THICK and o.tol == 1e-8 and o.inner_tol == 1e-4 and o.eta == 1.0


def test_invalid_descriptor_is_rejected_without_touching_the_gpu(libpath):
    """Argument checks run before any CUDA call."""
    from paper_2001_09196_gb300 import sn
    with pytest.raises(sn.SnError) as e:
        sn.Mesh(4, 8, 8, p=1, sn=4)
    assert e.value.status == 1
    with pytest.raises(sn.SnError):
        sn.Mesh(3, 4, 4, 4, p=2, sn=4)
    with pytest.raises(sn.SnError):
        sn.Mesh(2, 4, 4, p=1, sn=5)


def test_every_descriptor_refusal_comes_before_the_gpu(libpath):
    """Each refusal of sn_mesh_create that depends only on the descriptor: element counts, order,
    dimension, inflow value, the element-count ceiling, and the vertices (finite, no inverted or
    degenerate quadrilateral, none in 3D).  All run before the first CUDA call, so they hold here."""
    import numpy as np
    from paper_2001_09196_gb300 import sn

    def verts(nx, ny):
        x, y = np.meshgrid(np.linspace(0, 1, nx + 1), np.linspace(0, 1, ny + 1))
        return np.stack([x, y], axis=-1).reshape(-1, 2).copy()

    inverted = verts(2, 2)
    inverted[[4, 5]] = inverted[[5, 4]]          # swap two vertices of the middle row
    flat = verts(1, 1)
    flat[3] = flat[1]                             # a triangle: zero Jacobian at one corner
    nan = verts(2, 2)
    nan[4, 0] = np.nan
    cases = [
        ("element counts", lambda: sn.Mesh(2, 0, 4, p=1, sn=4)),
        ("element counts", lambda: sn.Mesh(3, 4, 4, 0, p=1, sn=4)),
        ("2D supports", lambda: sn.Mesh(2, 4, 4, p=4, sn=4)),
        ("2D supports", lambda: sn.Mesh(2, 4, 4, p=0, sn=4)),
        ("psi_inc", lambda: sn.Mesh(2, 4, 4, p=1, sn=4, psi_inc=-1.0)),
        ("psi_inc", lambda: sn.Mesh(2, 4, 4, p=1, sn=4, psi_inc=float("inf"))),
        ("too many elements", lambda: sn.Mesh(2, 65536, 65536, p=1, sn=4)),
        ("too many elements", lambda: sn.Mesh(3, 1025, 1024, 1024, p=1, sn=4)),
        ("sn_order", lambda: sn.Mesh(3, 2, 2, 2, p=1, sn=10)),
        ("inverted", lambda: sn.Mesh(2, 2, 2, p=1, sn=4, vertices=inverted)),
        ("inverted or degenerate", lambda: sn.Mesh(2, 1, 1, p=2, sn=4, vertices=flat)),
        ("non-finite", lambda: sn.Mesh(2, 2, 2, p=1, sn=4, vertices=nan)),
        ("vertices must be NULL", lambda: sn.Mesh(3, 1, 1, 1, p=1, sn=4, vertices=verts(1, 1))),
    ]
    for what, call in cases:
        with pytest.raises(sn.SnError, match=what) as e:
            call()
        assert e.value.status == 1, what


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every field of the ctypes mirrors sits at the C compiler's offset, and the sizes agree."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    from paper_2001_09196_gb300 import sn
    pairs = {"sn_mesh_desc": sn.MeshDesc, "sn_mesh_info": sn.MeshInfo, "sn_iter_opts": sn.IterOpts,
             "sn_iter_stats": sn.IterStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sn.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        struct, field, value = line.split()
        got[(struct, field)] = int(value)
    import ctypes
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_noalloc_binding_checks_run_before_the_library(libpath):
    """The no-allocation flux binding refuses bad sizes and aliasing before any pointer reaches the
    library (CPU tensors here: every check fires before the binding asks for a device pointer)."""
    import torch
    from paper_2001_09196_gb300 import sn
    f64 = dict(dtype=torch.float64)
    psi = torch.zeros(3, 10, **f64)
    w = torch.ones(3, **f64)
    with pytest.raises(ValueError, match="n_dirs"):
        sn.scalar_flux_noalloc(torch.zeros(30, **f64), w)
    with pytest.raises(ValueError, match="weights"):
        sn.scalar_flux_noalloc(psi, torch.ones(2, **f64))
    with pytest.raises(ValueError, match="phi_prev"):
        sn.scalar_flux_noalloc(psi, w, phi_prev=torch.zeros(9, **f64))
    with pytest.raises(ValueError, match="phi_out"):
        sn.scalar_flux_noalloc(psi, w, phi_out=torch.zeros(11, **f64))
    with pytest.raises(ValueError, match="resid_norm2"):
        sn.scalar_flux_noalloc(psi, w, phi_out=torch.zeros(10, **f64), resid_norm2=torch.zeros(0, **f64))
    prev = torch.zeros(10, **f64)
    with pytest.raises(ValueError, match="share storage"):
        sn.scalar_flux_noalloc(psi, w, phi_prev=prev, phi_out=prev)
    with pytest.raises(ValueError, match="share storage"):
        sn.scalar_flux_noalloc(psi, w, phi_out=psi[0])
    buf = torch.zeros(11, **f64)
    with pytest.raises(ValueError, match="overlap"):
        sn.scalar_flux_noalloc(psi, w, phi_out=buf[:10], resid_norm2=buf[9:])


def test_mesh_and_batch_bindings_check_buffer_sizes_before_the_library(libpath):
    """Every Mesh / Batch method that hands the library a caller's buffer refuses a buffer of the
    wrong size before any pointer reaches the library (the library trusts the sizes it is given).
    The meshes here are stand-ins with only their sizes set: no GPU and no library handle."""
    import torch
    from paper_2001_09196_gb300 import sn
    f64 = dict(dtype=torch.float64)

    def fake_mesh(n_elem, n_nodes):
        m = object.__new__(sn.Mesh)
        m._h = None
        m.n_elem, m.n_nodes, m.n_dirs, m.n_levels, m.dim, m.p = n_elem, n_nodes, 12, 1, 2, 1
        return m

    m = fake_mesh(16, 4)
    bad = torch.zeros(63, **f64)
    good = torch.zeros(16, 4, **f64)
    cases = [
        ("phi_in", lambda: m.sweep(bad)),
        ("phi_out", lambda: m.sweep(good, phi_out=bad)),
        ("phi_in", lambda: m.sweep_directions(bad, 0, 3)),
        ("phi_out", lambda: m.sweep_directions(good, 0, 3, phi_out=bad)),
        ("phi", lambda: m.source_iterate(phi=bad)),
        ("checkpoints", lambda: m.source_iterate(phi=good, checkpoint_every=2, checkpoints=torch.zeros(65, **f64))),
        ("checkpoints", lambda: m.source_iterate(phi=good, checkpoint_every=2, checkpoints=torch.zeros(32, **f64))),
        ("mu", lambda: m.adjoint_sweep(bad)),
        ("out", lambda: m.adjoint_sweep(good, out=bad)),
        ("g", lambda: m.adjoint_iterate(bad)),
        ("mu", lambda: m.adjoint_iterate(good, mu=bad)),
        ("phi", lambda: m.gradients(bad, good)),
        ("mu", lambda: m.gradients(good, bad)),
        ("g and phi0", lambda: m.unrolled_gradients(bad, 3)),
        ("checkpoints", lambda: m.unrolled_gradients(good, 5, 2, checkpoints=torch.zeros(64, **f64))),
        ("x", lambda: m.dsa_apply(bad)),
        ("b", lambda: m.dsa_solve(bad)),
    ]
    for name, call in cases:
        with pytest.raises(ValueError, match=name):
            call()
    if torch.cuda.is_available():
        return  # the material checks below rely on CPU tensors taking the host path
    with pytest.raises(ValueError, match="one value per element"):
        m.set_materials(torch.ones(15, **f64), torch.ones(16, **f64), torch.ones(16, **f64))
    with pytest.raises(ValueError, match="one value per element"):
        m.set_pseudo_scattering(torch.ones(16, **f64), torch.ones(17, **f64), torch.ones(16, **f64), 1.0)

    b = object.__new__(sn.Batch)
    b._h = None
    b.meshes = [fake_mesh(16, 4), fake_mesh(9, 9)]
    with pytest.raises(ValueError, match="one tensor per instance"):
        b.sweep([good])
    with pytest.raises(ValueError, match="instance 1"):
        b.sweep([good, torch.zeros(80, **f64)])
    with pytest.raises(ValueError, match="instance 0"):
        b.source_iterate([bad, torch.zeros(81, **f64)])
