"""GPU: the recorded outer iterations (one CUDA graph per solve, loop control on the device).

Source iteration (Eq. DSA_fp with Algorithm 2 or 1) and flexible GMRES (Sec. 4) recorded as WHILE
conditional nodes run the same device operations in the same order as the host loops.  Source
iteration keeps every scalar on the device in both forms, so its iterates, iteration counts,
residual histories and checkpoints must be bitwise equal.  The host loop of fGMRES does its Givens
rotations and triangular solve on the CPU, the recorded one on the GPU; those few scalar operations
may round differently (contraction into fused multiply-adds, hypot), so the recorded fGMRES must
reach the same solution within its tolerance with at most one iteration more or fewer.
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


CASES = {"c1": inputs.config1, "c2_32": lambda: inputs.config2(n=32, block=8), "c3_8": lambda: inputs.config3(n=8)}
RUNS = [dict(outer="si", dsa="thick", tol=1e-8, inner_tol=1e-4, max_iters=300),
        dict(outer="si", dsa="none", tol=1e-3, max_iters=40),
        dict(outer="si", dsa="triangular", tol=1e-8, inner_tol=1e-6, max_iters=300),
        dict(outer="fgmres", dsa="thick", tol=1e-10, inner_tol=1e-4, max_iters=300, restart=8),
        dict(outer="fgmres", dsa="thick", tol=1e-10, inner_tol=1e-10, max_iters=300),
        dict(outer="fgmres", dsa="triangular", tol=1e-9, inner_tol=1e-6, max_iters=300, restart=5),
        dict(outer="fgmres", dsa="thick", tol=1e-10, inner_tol=1e-4, max_iters=300, precision="fp32_mixed"),
        dict(outer="fgmres", dsa="thick", tol=1e-12, inner_tol=1e-4, max_iters=7)]   # stops at max_iters


@pytest.mark.parametrize("schedule", [("levels", 32, 2), ("static", 32, 0), ("dataflow", 128, 0)],
                         ids=["levels", "static", "dataflow"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("k", range(len(RUNS)))
def test_recorded_iteration_equals_the_host_loop(sn, case, k, schedule):
    prob = CASES[case]()
    m = sn.Mesh.from_problem(prob)
    m.set_schedule(*schedule)
    kw = dict(RUNS[k], thick_rule=prob.thick_rule)
    hist = 400
    a = m.source_iterate(history=hist, **kw)                       # recorded (level schedule)
    b = m.source_iterate(history=hist, host_loop=True, **kw)       # host loop
    assert a["converged"] == b["converged"]
    if kw["outer"] == "si":
        assert torch.equal(a["phi"], b["phi"])
        for key in ("iters", "sweeps", "inner_iters", "rel_residual"):
            assert a[key] == b[key], key
        assert np.array_equal(a["history"], b["history"])
    else:
        # SN_FP32_MIXED restarts a cycle when the estimate crosses refine_drop, so a rounding
        # difference may move a restart by a step
        slack = 2 if kw.get("precision") == "fp32_mixed" else 1
        assert abs(a["iters"] - b["iters"]) <= slack
        scale = float(b["phi"].abs().max())
        assert float((a["phi"] - b["phi"]).abs().max()) <= max(1e-11, 100 * kw["tol"]) * scale
        n = min(a["iters"], b["iters"], 8)  # the first estimates, before rounding differences grow
        rtol = 1e-4 if slack == 2 else 1e-6    # float32 sweeps carry rounding differences further
        assert np.allclose(a["history"][: n + 1], b["history"][: n + 1], rtol=rtol, atol=1e-13)
    c = m.source_iterate(history=hist, **kw)                        # the graph is reused
    assert torch.equal(a["phi"], c["phi"]) and a["iters"] == c["iters"]


def test_recorded_source_iteration_checkpoints(sn):
    prob = inputs.config1()
    m = sn.Mesh.from_problem(prob)
    out = []
    for host in (False, True):
        ck = torch.zeros((6,) + m.shape, dtype=torch.float64, device="cuda")
        r = m.source_iterate(dsa="thick", tol=1e-8, max_iters=300, checkpoint_every=4, checkpoints=ck, host_loop=host)
        out.append((r, ck))
    (a, ca), (b, cb) = out
    assert a["n_checkpoints"] == b["n_checkpoints"] == min(6, a["iters"] // 4)
    assert torch.equal(ca, cb)


def test_one_synchronisation_per_recorded_solve(sn, monkeypatch):
    """The recorded fGMRES solve of configuration 2 (32^2) launches one graph: the library's kernel
    counter grows by the iteration's kernels, while the solve takes one host round trip; the
    warm call (graph reused) is not slower than the host loop."""
    import time
    prob = inputs.config2(n=32, block=8)
    m = sn.Mesh.from_problem(prob)
    kw = dict(dsa="thick", outer="fgmres", tol=1e-8, inner_tol=1e-4, max_iters=300)
    m.source_iterate(**kw)
    m.source_iterate(host_loop=True, **kw)
    ts = {}
    for host in (False, True):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            r = m.source_iterate(host_loop=host, **kw)
        torch.cuda.synchronize()
        ts[host] = time.perf_counter() - t0
        assert r["converged"]
    assert ts[False] <= ts[True] * 1.10
