"""GPU: batched sweeps and batched DSA source iteration over instances of mixed size, order and S_N."""
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


def small_instances():
    """Ragged mix of element families and quadratures (2D p = 1..3 with S4/S6/S8, and 3D p = 1)."""
    out = [inputs.config2d_fields(16, 1, 4, 11, "a"), inputs.config2d_fields(24, 2, 8, 12, "b"),
           inputs.config2d_fields(12, 3, 6, 13, "c"), inputs.config2d_fields(20, 1, 8, 14, "d"),
           inputs.config3(n=6), inputs.config2(n=32, block=8, p=2, sn=4)]
    for p in out:
        p.q[:] = np.maximum(p.q, 0.5)
    return out


@pytest.mark.parametrize("schedule", [("levels", 64, 0), ("dataflow", 128, 0), ("dataflow", 32, 1), ("static", 32, 0),
                                      ("static", 128, 0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine"])
def test_batched_sweep_equals_single_sweeps(sn, schedule, precision):
    probs = small_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    batch.set_schedule(*schedule)
    phis = [torch.as_tensor(inputs.random_phi(p, 60 + k), device="cuda") for k, p in enumerate(probs)]
    outs = batch.sweep(phis, precision=precision)
    for m, phi, out in zip(meshes, phis, outs):
        assert torch.equal(m.sweep(phi, precision=precision), out)


@pytest.fixture(scope="module")
def oracle_runs():
    """The oracle's K = 4 DSA-accelerated iterates and its converged solution of every instance."""
    from oracle import Transport
    from oracle.dsa import DSA, thick_mask
    out = []
    for p in small_instances():
        T = Transport(p)
        d = DSA(T, thick_mask(p))
        out.append((T.source_iterate(dsa=d, tol=0.0, max_iters=4)["phi"],
                    T.source_iterate(dsa=d, tol=1e-14, max_iters=4000)["phi"]))
    return out


@pytest.mark.parametrize("schedule", [("levels", 64, 0), ("dataflow", 128, 0), ("static", 32, 0)])
def test_batched_iterates_match_the_oracle(sn, schedule, oracle_runs):
    """The batched source iteration (one union CG over every instance's thick-DSA system, one
    V-cycle over the union of their hierarchies, Algorithm 2 per instance) against the oracle's
    own iteration of each instance: K = 4 iterates within the derived DSA-iterate tolerance, and
    the converged solutions within 1e-9 (a 1e-12 residual times the conditioning of Eq. schur)."""
    from oracle.dsa import thick_mask
    from tolerances import dsa_iterate_tol
    probs = small_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    batch.set_schedule(*schedule)
    res = batch.source_iterate(dsa="thick", thick_rule="sigma_t_h", tol=0.0, max_iters=4, inner_tol=1e-15,
                               inner_max_iters=3000)
    assert res["iters"] == [4] * len(probs)
    for k, (p, (ref_k, _)) in enumerate(zip(probs, oracle_runs)):
        err = float(np.abs(res["phi"][k].cpu().numpy() - ref_k).max() / np.abs(ref_k).max())
        assert err <= dsa_iterate_tol(p, thick_mask(p)), (k, err)
    res = batch.source_iterate(dsa="thick", thick_rule="sigma_t_h", tol=1e-12, max_iters=3000, inner_tol=1e-12,
                               inner_max_iters=1000)
    assert res["converged"]
    for k, (p, (_, ref)) in enumerate(zip(probs, oracle_runs)):
        err = float(np.abs(res["phi"][k].cpu().numpy() - ref).max() / np.abs(ref).max())
        assert err < 1e-9, (k, err)


@pytest.mark.parametrize("schedule", [("levels", 64, 0), ("dataflow", 128, 0)])
def test_batched_source_iteration_matches_single_solves(sn, schedule):
    probs = small_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    batch.set_schedule(*schedule)
    opts = dict(dsa="thick", thick_rule="sigma_t_h", tol=1e-9, inner_tol=1e-12, inner_max_iters=300, max_iters=400)
    res = batch.source_iterate(**opts)
    assert res["converged"]
    for k, m in enumerate(meshes):
        single = m.source_iterate(**opts)
        assert single["converged"]
        # the union CG uses one set of scalars, so DSA corrections differ from the single-mesh CG
        # only at the inner tolerance; iterates then agree closely and stop at the same point
        assert abs(res["iters"][k] - single["iters"]) <= 1
        ref = single["phi"]
        err = float((res["phi"][k] - ref).abs().max() / ref.abs().max())
        assert err < 1e-7, (k, err)


def test_batch_convergence_masks_freeze_converged_instances(sn):
    """Instances converge at different iterations; a converged one keeps its iterate."""
    probs = small_instances()[:4]
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    res = batch.source_iterate(dsa="none", tol=1e-6, max_iters=600)
    assert res["converged"]
    assert len(set(res["iters"])) > 1
    for k, m in enumerate(meshes):
        single = m.source_iterate(dsa="none", tol=1e-6, max_iters=600)
        assert res["iters"][k] == single["iters"]
        assert torch.equal(res["phi"][k], single["phi"])


def weakly_scattering_instances():
    """The ragged mix with scattering ratios capped at 0.9, so that fGMRES without the DSA step
    converges in tens of Arnoldi steps."""
    out = small_instances()
    for p in out:
        p.sigma_s[:] = np.minimum(p.sigma_s, 0.9 * p.sigma_t)
    return out


@pytest.mark.parametrize("schedule", [("levels", 64, 0), ("dataflow", 128, 0), ("static", 32, 0)])
def test_batched_fgmres_reaches_the_oracle_fixed_point(sn, schedule, oracle_runs):
    """Every instance's own flexible GMRES (Eq. schur, right-preconditioned by the union DSA step of
    Algorithm 2), run in lock step over the batch, converges to the oracle's fixed point of that
    instance within 1e-9 (a 1e-12 residual times the conditioning of Eq. schur)."""
    probs = small_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    batch.set_schedule(*schedule)
    res = batch.source_iterate(dsa="thick", thick_rule="sigma_t_h", outer="fgmres", restart=30, tol=1e-12,
                               inner_tol=1e-12, inner_max_iters=1000, max_iters=400)
    assert res["converged"]
    for k, (p, (_, ref)) in enumerate(zip(probs, oracle_runs)):
        assert res["rel_residual"][k] <= 1e-12
        err = float(np.abs(res["phi"][k].cpu().numpy() - ref).max() / np.abs(ref).max())
        assert err < 1e-9, (k, err)


def test_batched_fgmres_instances_are_independent_without_dsa(sn):
    """Without the DSA step nothing couples the instances: each instance's Arnoldi process uses
    inner products over its own DOFs only (summed in a fixed chunk order), so every instance of a
    batch ends bit for bit where a batch of that instance alone ends, after as many steps.  A small
    restart forces several cycles."""
    probs = weakly_scattering_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    opts = dict(dsa="none", outer="fgmres", restart=5, tol=1e-10, max_iters=600)
    res = batch.source_iterate(**opts)
    assert res["converged"]
    assert len(set(res["iters"])) > 1
    for k, m in enumerate(meshes):
        alone = sn.Batch([m]).source_iterate(**opts)
        assert alone["iters"][0] == res["iters"][k]
        assert torch.equal(alone["phi"][0], res["phi"][k]), k


@pytest.mark.parametrize("restart", [5, 30])
def test_batched_fgmres_follows_the_single_mesh_fgmres(sn, restart):
    """Without the DSA step the batched and the single-mesh fGMRES run the same algorithm on the
    same operator (only the order of the inner-product sums differs): the same number of Arnoldi
    steps and solutions within 1e-10 of each other."""
    probs = weakly_scattering_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    opts = dict(dsa="none", outer="fgmres", restart=restart, tol=1e-10, max_iters=600)
    res = sn.Batch(meshes).source_iterate(**opts)
    for k, m in enumerate(meshes):
        single = m.source_iterate(**opts)
        assert abs(single["iters"] - res["iters"][k]) <= 1, (k, single["iters"], res["iters"][k])
        ref = single["phi"]
        assert float((res["phi"][k] - ref).abs().max() / ref.abs().max()) < 1e-10, k


def test_batched_fgmres_fp32_form(sn, oracle_runs):
    """FP32 element solves inside the batched fGMRES (float64 flux, residual, DSA and Krylov
    arithmetic): every instance within the derived FP32 bound of the oracle's fixed point."""
    from tolerances import fp32_fixed_point_tol
    probs = small_instances()
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    res = sn.Batch(meshes).source_iterate(dsa="thick", thick_rule="sigma_t_h", outer="fgmres", restart=30,
                                          tol=1e-6, inner_tol=1e-10, inner_max_iters=1000, max_iters=400,
                                          precision="fp32")
    assert res["converged"]
    for k, (p, (_, ref)) in enumerate(zip(probs, oracle_runs)):
        err = float(np.abs(res["phi"][k].cpu().numpy() - ref).max() / np.abs(ref).max())
        assert err <= fp32_fixed_point_tol(p), (k, err)


def test_batched_fgmres_rejects_mixed_precision(sn):
    meshes = [sn.Mesh.from_problem(p) for p in small_instances()[:2]]
    with pytest.raises(sn.SnError):
        sn.Batch(meshes).source_iterate(dsa="thick", thick_rule="sigma_t_h", outer="fgmres", precision="fp32_mixed")


def test_batched_fgmres_budget_and_warm_start(sn):
    """An iteration budget below what the instances need ends the solve with SN_ERR_NOT_CONVERGED
    after exactly that many Arnoldi steps per instance; a warm start from the unconverged iterates
    continues to the same solution as a cold start (within the tolerance)."""
    probs = weakly_scattering_instances()[:3]
    meshes = [sn.Mesh.from_problem(p) for p in probs]
    batch = sn.Batch(meshes)
    opts = dict(dsa="thick", thick_rule="sigma_t_h", outer="fgmres", restart=4, inner_tol=1e-10, inner_max_iters=500)
    res = batch.source_iterate(tol=1e-14, max_iters=6, **opts)
    assert not res["converged"]
    assert res["iters"] == [6] * len(probs)
    warm = batch.source_iterate(phis=[p.clone() for p in res["phi"]], warm_start=True, tol=1e-10, max_iters=400,
                                **opts)
    cold = batch.source_iterate(tol=1e-12, max_iters=400, **opts)
    assert warm["converged"] and cold["converged"]
    for a, b in zip(warm["phi"], cold["phi"]):
        assert float((a - b).abs().max() / b.abs().max()) < 1e-8
