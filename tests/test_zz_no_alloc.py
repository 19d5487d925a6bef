"""GPU: the scalar-flux reduction that allocates nothing matches the flux that sn_sweep returns.

sn_scalar_flux_noalloc serves callers that cannot call cudaMalloc: frameworks whose caching
allocator owns the device memory, loops that cannot take cudaMalloc's device synchronisation, and
hosts with a device memory budget fixed at start-up.  It keeps its block partial sums in a fixed
device array inside the library.  This file is collected
last so that a failure here leaves every other test already run; it passes alone and after them.
"""
import numpy as np
import pytest

from paper_2001_09196_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09196_gb300 import build
    build.build()
    from paper_2001_09196_gb300 import sn as mod
    return mod


def _angular_fluxes(mesh, prob, seed):
    """One sweep through the C ABI: its phi_out, its psi_d for all d, the weights and phi_in."""
    phi_in = torch.as_tensor(inputs.random_phi(prob, seed), device="cuda")
    phi_out = mesh.sweep(phi_in)
    psi = torch.stack([mesh.angular_flux(d) for d in range(mesh.n_dirs)]).contiguous()
    _, w = mesh.quadrature()
    return phi_in, phi_out, psi, torch.as_tensor(w, device="cuda")


def test_noalloc_flux_matches_sweep_on_consecutive_calls(sn):
    # two different problems back to back: the second call reuses the shared device array
    cases = [inputs.config2(n=32, block=8), inputs.config1()]
    for seed, prob in enumerate(cases):
        mesh = sn.Mesh.from_problem(prob)
        phi_in, phi_ref, psi, w = _angular_fluxes(mesh, prob, 50 + seed)
        phi = torch.empty(psi[0].numel(), dtype=torch.float64, device="cuda")
        rr = torch.empty(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        sn.scalar_flux_noalloc(psi, w, phi_prev=phi_in, phi_out=phi, resid_norm2=rr)
        torch.cuda.synchronize()
        if seed > 0:  # after the first call's one-time set-up the device's free memory stays put
            assert torch.cuda.mem_get_info()[0] == free_before
        ref = phi_ref.reshape(-1)
        assert torch.max(torch.abs(phi - ref)).item() <= 1e-12 * torch.max(torch.abs(ref)).item()
        expect = float(torch.sum((ref - phi_in.reshape(-1)) ** 2))
        assert abs(float(rr.item()) - expect) <= 1e-12 * expect


def test_noalloc_rejects_sizes_beyond_its_limit(sn):
    big = 2_097_152 + 1
    psi = torch.zeros(1, dtype=torch.float64, device="cuda")
    w = torch.ones(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    C = sn.C
    status = sn.lib().sn_scalar_flux_noalloc(C.c_void_p(psi.data_ptr()), C.c_void_p(w.data_ptr()), 1, big,
                                             None, C.c_void_p(out.data_ptr()), None, None)
    assert status == 1
    assert b"2097152" in sn.lib().sn_last_error()
