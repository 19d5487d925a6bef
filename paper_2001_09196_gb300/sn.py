"""Thin Python binding of libsn (include/sn.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts torch tensors and
numpy arrays to the C ABI's pointers and raises on a non-OK status.  Importing it loads
libsn.so from paper_2001_09196_gb300/lib and fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsn.so")

FP64, FP32, FP32_REFINE, FP32_MIXED = 0, 1, 2, 3
DSA_NONE, DSA_FULL, DSA_THICK, DSA_TRIANGULAR = 0, 1, 2, 3
THICK_SIGMA_S, THICK_SIGMA_T_H, THICK_MASK = 0, 1, 2
DSA_SIGMA_S, DSA_SIGMA_T = 0, 1
DSA_OP_SIP, DSA_OP_NIP, DSA_OP_MNIP = 0, 1, 2
_DSA_OP = {"sip": DSA_OP_SIP, "nip": DSA_OP_NIP, "mnip": DSA_OP_MNIP}
_PREC = {"fp64": FP64, "fp32": FP32, "fp32_refine": FP32_REFINE, "fp32_mixed": FP32_MIXED}
_DSA = {"none": DSA_NONE, "full": DSA_FULL, "thick": DSA_THICK, "triangular": DSA_TRIANGULAR}
_RULE = {"sigma_s": THICK_SIGMA_S, "sigma_t_h": THICK_SIGMA_T_H, "mask": THICK_MASK}
SCHEDULES = ("levels", "dataflow", "tiles", "barrier", "static")

STATUS = {0: "SN_OK", 1: "SN_ERR_ARG", 2: "SN_ERR_CUDA", 3: "SN_ERR_OOM", 4: "SN_ERR_CYCLE",
          5: "SN_ERR_VOID_FULL_DSA", 6: "SN_ERR_NOT_CONVERGED", 7: "SN_ERR_TIMEOUT",
          8: "SN_ERR_INNER_NOT_CONVERGED"}


class SnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("p", C.c_int),
                ("sn_order", C.c_int), ("vertices", C.POINTER(C.c_double)), ("psi_inc", C.c_double)]


class MeshInfo(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("n_nodes", C.c_int), ("n_dirs", C.c_int), ("n_levels", C.c_int),
                ("n_items", C.c_longlong)]


class IterOpts(C.Structure):
    _fields_ = [("dsa", C.c_int), ("thick_rule", C.c_int), ("eta", C.c_double),
                ("mask", C.POINTER(C.c_ubyte)), ("dsa_sigma", C.c_int), ("tol", C.c_double),
                ("inner_tol", C.c_double), ("max_iters", C.c_int), ("inner_max_iters", C.c_int),
                ("precision", C.c_int), ("checkpoint_every", C.c_int), ("checkpoints", C.c_void_p),
                ("max_checkpoints", C.c_int), ("warm_start", C.c_int), ("outer", C.c_int), ("restart", C.c_int),
                ("dsa_operator", C.c_int), ("dsa_vcycle", C.c_int), ("dir_begin", C.c_int), ("dir_end", C.c_int),
                ("exchange", C.c_void_p), ("exchange_ctx", C.c_void_p), ("exchange_buf", C.c_void_p),
                ("refine_drop", C.c_double), ("host_loop", C.c_int)]


# sn_exchange_fn: sn_status (*)(double* phi_partial, long long n, void* stream, void* ctx)
EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p)


class IterStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_residual", C.c_double), ("inner_iters_total", C.c_int),
                ("thick_fraction", C.c_double), ("residual_history", C.POINTER(C.c_double)),
                ("history_len", C.c_int), ("n_checkpoints", C.c_int), ("ms_total", C.c_double),
                ("n_sweeps", C.c_int), ("ms_sweep", C.c_double), ("ms_dsa", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsn.so not built ({LIB_PATH}); run paper_2001_09196_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "sn_mesh_create": [C.POINTER(MeshDesc), C.POINTER(vp)],
        "sn_mesh_destroy": [vp],
        "sn_mesh_get_info": [vp, C.POINTER(MeshInfo)],
        "sn_mesh_quadrature": [vp, vp, vp],
        "sn_set_materials": [vp, vp, vp, vp, i, vp],
        "sn_set_pseudo_scattering": [vp, vp, vp, vp, d, d, d, i, vp],
        "sn_get_materials": [vp, vp, vp, vp],
        "sn_sweep": [vp, vp, vp, i, vp],
        "sn_sweep_directions": [vp, vp, vp, i, i, i, vp],
        "sn_source_iterate": [vp, C.POINTER(IterOpts), vp, C.POINTER(IterStats), vp],
        "sn_adjoint_sweep": [vp, vp, vp, i, vp],
        "sn_adjoint_iterate": [vp, C.POINTER(IterOpts), vp, vp, C.POINTER(IterStats), vp],
        "sn_gradients": [vp, vp, vp, vp, vp, vp, vp],
        "sn_unrolled_gradients": [vp, vp, i, i, vp, vp, vp, vp, vp, vp],
        "sn_dsa_apply": [vp, C.POINTER(IterOpts), vp, vp, vp],
        "sn_dsa_solve": [vp, C.POINTER(IterOpts), vp, vp, C.POINTER(C.c_int), vp],
        "sn_get_angular_flux": [vp, i, i, i, vp, vp],
        "sn_get_levels": [vp, i, vp],
        "sn_mesh_set_schedule": [vp, i, i, i],
        "sn_mesh_set_operator_cache": [vp, i],
        "sn_debug_stall_next_sweep": [vp, d],
        "sn_scalar_flux_noalloc": [vp, vp, i, C.c_longlong, vp, vp, vp, vp],
        "sn_batch_create": [vp, i, C.POINTER(vp)],
        "sn_batch_destroy": [vp],
        "sn_batch_set_schedule": [vp, i, i, i],
        "sn_batch_sweep": [vp, vp, vp, i, vp],
        "sn_batch_source_iterate": [vp, C.POINTER(IterOpts), vp, vp, vp],
        "sn_mesh_autotune": [vp, i, vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "sn_batch_autotune": [vp, i, vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.sn_last_error.restype = C.c_char_p
    lib.sn_version.restype = C.c_char_p
    lib.sn_launch_count.restype = C.c_longlong
    lib.sn_launch_count.argtypes = []
    lib.sn_iter_opts_default.argtypes = [C.POINTER(IterOpts)]
    lib.sn_iter_opts_default.restype = None
    return lib


_lib = _load()


def lib():
    return _lib


def launch_count():
    """Kernels launched by libsn so far in this process."""
    return int(_lib.sn_launch_count())


def _check(status):
    if status != 0:
        raise SnError(status, _lib.sn_last_error().decode())


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _need(n, **tensors):
    """Raise unless every given tensor (None = not given) holds exactly n values: the library reads
    and writes n values through each pointer, so a shorter buffer would be overrun on the device."""
    for name, t in tensors.items():
        if t is not None and t.numel() != n:
            raise ValueError(f"{name} needs exactly {n} values, got {t.numel()}")


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_opts(dsa="thick", thick_rule="sigma_s", eta=1.0, mask=None, dsa_sigma="sigma_s", tol=1e-8,
              inner_tol=1e-4, max_iters=1000, inner_max_iters=200, precision="fp64", checkpoint_every=0,
              checkpoints=None, warm_start=False, outer="si", restart=30, operator="sip", vcycle="auto",
              refine_drop=0.0, host_loop=False):
    """Options of sn_source_iterate / sn_adjoint_iterate.  operator: the DSA operator D_ff,
    "sip" (symmetric, conjugate gradients), "nip" (Eq. NIP) or "mnip" (Eq. NIP with the penalty
    of Eq. ModifiedF0); the nonsymmetric two are solved by BiCGStab.  vcycle: arithmetic of the
    multigrid preconditioner, "auto" (float32 when inner_tol >= 1e-8), "fp64" or "fp32".
    precision: "fp64", "fp32", "fp32_refine" or "fp32_mixed" (fGMRES with float32 sweeps inside
    each restart cycle and a float64 true residual between cycles; a cycle ends when its residual
    estimate fell by refine_drop, 0 = 1e-4).  host_loop: run the outer iteration as a host loop
    (one synchronisation per iteration, device time split into ms_sweep / ms_dsa) instead of one
    recorded graph launch."""
    o = IterOpts()
    _lib.sn_iter_opts_default(C.byref(o))
    o.dsa = _DSA[dsa] if isinstance(dsa, str) else int(dsa)
    o.thick_rule = _RULE[thick_rule] if isinstance(thick_rule, str) else int(thick_rule)
    o.eta = float(eta)
    keep = []
    if mask is not None:
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        keep.append(m)
        o.mask = m.ctypes.data_as(C.POINTER(C.c_ubyte))
        o.thick_rule = THICK_MASK
    o.dsa_sigma = DSA_SIGMA_S if dsa_sigma == "sigma_s" else DSA_SIGMA_T
    o.tol, o.inner_tol = float(tol), float(inner_tol)
    o.max_iters, o.inner_max_iters = int(max_iters), int(inner_max_iters)
    o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    o.checkpoint_every = int(checkpoint_every)
    if checkpoints is not None:
        o.checkpoints = _ptr(checkpoints)
        o.max_checkpoints = int(checkpoints.shape[0])
    o.warm_start = int(bool(warm_start))
    o.outer = {"si": 0, "fgmres": 1}[outer] if isinstance(outer, str) else int(outer)
    o.restart = int(restart)
    o.dsa_operator = _DSA_OP[operator] if isinstance(operator, str) else int(operator)
    o.dsa_vcycle = {"auto": 0, "fp64": 1, "fp32": 2}[vcycle] if isinstance(vcycle, str) else int(vcycle)
    o.refine_drop = float(refine_drop)
    o.host_loop = int(bool(host_loop))
    o._keep = keep
    return o


def torch_allreduce(group=None):
    """An exchange for Mesh.source_iterate(directions=..., exchange=...): the sum over the processes
    of a torch.distributed group.  NCCL reduces the CUDA tensor in place on the current stream; a
    CPU backend (gloo) reduces a host copy and writes the sum back."""
    import torch.distributed as dist

    def exchange(t):
        if dist.get_backend(group) == "nccl" or not t.is_cuda:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
            t.copy_(h)
    return exchange


def scalar_flux_noalloc(psi, weights, phi_prev=None, phi_out=None, resid_norm2=None, stream=None):
    """phi_out = sum_d w_d psi_d and ||phi_out - phi_prev||^2 without device allocation in libsn.

    psi: (n_dirs, ...) float64 CUDA tensor, n_values = the size of one direction's block; weights:
    (n_dirs,) float64 CUDA tensor on the same
    device; phi_prev (optional) and phi_out: n_values elements; resid_norm2: at least one element.
    Outputs are caller-provided (allocated here by torch only when not given).  Every size, device
    and aliasing rule is checked here, before anything reaches the GPU; the call runs with psi's
    device current, so the library resolves its scratch array on that device.
    """
    import torch
    if not isinstance(psi, torch.Tensor) or psi.dim() < 2 or psi.shape[0] < 1:
        raise ValueError("psi must have shape (n_dirs, ...) with n_dirs >= 1 and at least 2 dimensions")
    nd, m = int(psi.shape[0]), int(psi[0].numel())
    if weights is None or weights.numel() != nd:
        raise ValueError(f"weights needs exactly n_dirs = {nd} elements")
    if phi_prev is not None and phi_prev.numel() != m:
        raise ValueError(f"phi_prev needs exactly n_values = {m} elements")
    if phi_out is not None and phi_out.numel() != m:
        raise ValueError(f"phi_out needs exactly n_values = {m} elements")
    if resid_norm2 is not None and resid_norm2.numel() < 1:
        raise ValueError("resid_norm2 needs at least one element")

    def _overlap(a, b):
        if a is None or b is None:
            return False
        a0, b0 = a.data_ptr(), b.data_ptr()
        return a0 < b0 + b.numel() * b.element_size() and b0 < a0 + a.numel() * a.element_size()

    for out in (phi_out, resid_norm2):
        for other in (psi, weights, phi_prev):
            if _overlap(out, other):
                raise ValueError("outputs must not share storage with psi, weights or phi_prev")
    if _overlap(phi_out, resid_norm2):
        raise ValueError("phi_out and resid_norm2 must not overlap")
    for t in (psi, weights, phi_prev, phi_out, resid_norm2):
        if t is not None and t.device != psi.device:
            raise ValueError("every tensor must be on psi's device")
    with torch.cuda.device(psi.device):
        if phi_out is None:
            phi_out = torch.empty(m, dtype=torch.float64, device=psi.device)
        if resid_norm2 is None:
            resid_norm2 = torch.empty(1, dtype=torch.float64, device=psi.device)
        _check(_lib.sn_scalar_flux_noalloc(_ptr(psi), _ptr(weights), nd, m, _ptr(phi_prev), _ptr(phi_out),
                                           _ptr(resid_norm2), _stream(stream)))
    return phi_out, resid_norm2


class Mesh:
    """A structured mesh with its S_N quadrature and upwind level sets on the current GPU."""

    def __init__(self, dim, nx, ny, nz=1, p=1, sn=8, vertices=None, psi_inc=0.0):
        desc = MeshDesc(dim, nx, ny, nz if dim == 3 else 1, p, sn, None, float(psi_inc))
        self._verts = None
        if vertices is not None:
            self._verts = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64))
            desc.vertices = self._verts.ctypes.data_as(C.POINTER(C.c_double))
        h = C.c_void_p()
        _check(_lib.sn_mesh_create(C.byref(desc), C.byref(h)))
        self._h = h
        info = MeshInfo()
        _check(_lib.sn_mesh_get_info(h, C.byref(info)))
        self.n_elem, self.n_nodes, self.n_dirs, self.n_levels = info.n_elem, info.n_nodes, info.n_dirs, info.n_levels
        self.dim, self.p = dim, p

    @classmethod
    def from_problem(cls, prob, materials=True):
        m = cls(prob.dim, prob.nx, prob.ny, prob.nz, prob.p, prob.sn, prob.vertices, prob.psi_inc)
        if materials:
            m.set_materials(prob.sigma_t, prob.sigma_s, prob.q)
        return m

    def close(self):
        if getattr(self, "_h", None):
            _lib.sn_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.n_elem, self.n_nodes)

    def set_schedule(self, schedule="dataflow", block=128, param=0):
        """schedule "levels" | "dataflow" | "tiles" | "barrier" | "static"; param: direction groups
        (levels), per-SM block cap (dataflow, static), tile edge (tiles) or CTAs per SM (barrier)."""
        sched = SCHEDULES.index(schedule) if isinstance(schedule, str) else int(schedule)
        _check(_lib.sn_mesh_set_schedule(self._h, sched, int(block), int(param)))

    def set_operator_cache(self, mode="auto"):
        """Cache every element operator's inverse between sweeps: "off", "on" or "auto"."""
        m = {"off": 0, "on": 1, "auto": 2}[mode] if isinstance(mode, str) else int(mode)
        _check(_lib.sn_mesh_set_operator_cache(self._h, m))

    def debug_stall_next_sweep(self, timeout_s=0.2):
        _check(_lib.sn_debug_stall_next_sweep(self._h, float(timeout_s)))

    def autotune(self, precision="fp64", stream=None):
        """Pick the fastest sweep schedule for this mesh and precision; returns (schedule, block, cap)."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(_lib.sn_mesh_autotune(self._h, _PREC.get(precision, precision), _stream(stream), C.byref(a),
                                     C.byref(b), C.byref(c)))
        return SCHEDULES[a.value], b.value, c.value

    def quadrature(self):
        dirs = np.zeros((self.n_dirs, 3))
        w = np.zeros(self.n_dirs)
        _check(_lib.sn_mesh_quadrature(self._h, dirs.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)))
        return dirs, w

    def set_materials(self, sigma_t, sigma_s, q, stream=None):
        import torch
        if isinstance(sigma_t, torch.Tensor) and sigma_t.is_cuda:
            _need(self.n_elem, sigma_t=sigma_t, sigma_s=sigma_s, q=q)
            args = [_ptr(sigma_t.contiguous()), _ptr(sigma_s.contiguous()), _ptr(q.contiguous())]
            _check(_lib.sn_set_materials(self._h, *args, 1, _stream(stream)))
            return
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (sigma_t, sigma_s, q)]
        for a in arrs:
            if a.size != self.n_elem:
                raise ValueError("material arrays need one value per element")
        _check(_lib.sn_set_materials(self._h, *[a.ctypes.data_as(C.c_void_p) for a in arrs], 0, _stream(stream)))

    def sweep_directions(self, phi_in, d_begin, d_end, phi_out=None, precision="fp64", stream=None):
        """The contribution of directions d_begin <= d < d_end to one transport update."""
        import torch
        _need(self.n_elem * self.n_nodes, phi_in=phi_in, phi_out=phi_out)
        if phi_out is None:
            phi_out = torch.empty(self.shape, dtype=torch.float64, device=phi_in.device if phi_in is not None else "cuda")
        _check(_lib.sn_sweep_directions(self._h, _ptr(phi_in), _ptr(phi_out), int(d_begin), int(d_end),
                                        _PREC.get(precision, precision), _stream(stream)))
        return phi_out

    def set_pseudo_scattering(self, sigma, cv, T, dt, a_rad=137.199, c_light=2.9979e4, stream=None):
        """Materials of one pseudo-scattering time step (Sec. 4.2, Eq. hohlraum_sigma / hohlraum_q),
        formed on the device from per-element opacity, heat capacity and temperature; the default
        constants are the paper's NIF-unit a and c."""
        import torch
        if isinstance(sigma, torch.Tensor) and sigma.is_cuda:
            _need(self.n_elem, sigma=sigma, cv=cv, T=T)
            args = [_ptr(x.contiguous()) for x in (sigma, cv, T)]
            _check(_lib.sn_set_pseudo_scattering(self._h, *args, float(dt), float(a_rad), float(c_light), 1,
                                                 _stream(stream)))
            return
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (sigma, cv, T)]
        for a in arrs:
            if a.size != self.n_elem:
                raise ValueError("material arrays need one value per element")
        _check(_lib.sn_set_pseudo_scattering(self._h, *[a.ctypes.data_as(C.c_void_p) for a in arrs], float(dt),
                                             float(a_rad), float(c_light), 0, _stream(stream)))

    def materials(self):
        """(sigma_t, sigma_s, q) as the mesh holds them (host copies)."""
        out = [np.empty(self.n_elem) for _ in range(3)]
        _check(_lib.sn_get_materials(self._h, *[a.ctypes.data_as(C.c_void_p) for a in out]))
        return tuple(out)

    def sweep(self, phi_in, phi_out=None, precision="fp64", stream=None):
        import torch
        _need(self.n_elem * self.n_nodes, phi_in=phi_in, phi_out=phi_out)
        if phi_out is None:
            phi_out = torch.empty(self.shape, dtype=torch.float64, device=phi_in.device if phi_in is not None else "cuda")
        _check(_lib.sn_sweep(self._h, _ptr(phi_in), _ptr(phi_out), _PREC.get(precision, precision), _stream(stream)))
        return phi_out

    def source_iterate(self, phi=None, stream=None, history=0, directions=None, exchange=None, **kw):
        """Eq. DSA_fp (source iteration) or fGMRES with the DSA preconditioner; see make_opts.

        directions = (d_begin, d_end) with exchange: a direction-sharded iteration.  This process
        sweeps only its directions; exchange(t) receives each partial update as a float64 CUDA tensor
        of shape (n_elem, n_nodes) and must replace it in place by the sum over all processes
        (torch_allreduce builds one from a torch.distributed process group)."""
        import torch
        M = self.n_elem * self.n_nodes
        _need(M, phi=phi)
        ck = kw.get("checkpoints")
        if ck is not None and (ck.numel() < M or ck.numel() % M):
            raise ValueError(f"checkpoints need a whole number (>= 1) of n_elem * n_nodes = {M} value vectors")
        if phi is None:
            phi = torch.zeros(self.shape, dtype=torch.float64, device="cuda")
        if "warm_start" not in kw:
            kw["warm_start"] = False
        o = make_opts(**kw)
        if ck is not None:
            o.max_checkpoints = ck.numel() // M
        failure = []
        if directions is not None or exchange is not None:
            if directions is None or exchange is None:
                raise ValueError("a direction-sharded iteration needs both directions and exchange")
            buf = torch.empty(self.shape, dtype=torch.float64, device=phi.device)

            def _cb(ptr, n, strm, ctx):
                try:
                    exchange(buf)
                    return 0
                except Exception as e:  # reported after the call returns
                    failure.append(e)
                    return 1
            cb = EXCHANGE_FN(_cb)
            o.dir_begin, o.dir_end = int(directions[0]), int(directions[1])
            o.exchange = C.cast(cb, C.c_void_p)
            o.exchange_buf = buf.data_ptr()
            o._keep.extend([cb, buf])
        st = IterStats()
        hist = np.zeros(max(history, 0))
        if history:
            st.residual_history = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.history_len = history
        status = _lib.sn_source_iterate(self._h, C.byref(o), _ptr(phi), C.byref(st), _stream(stream))
        if failure:
            raise failure[0]
        out = {"phi": phi, "iters": st.iters, "rel_residual": st.rel_residual, "inner_iters": st.inner_iters_total,
               "thick_fraction": st.thick_fraction, "ms": st.ms_total, "converged": status == 0,
               "n_checkpoints": st.n_checkpoints, "sweeps": st.n_sweeps, "ms_sweep": st.ms_sweep, "ms_dsa": st.ms_dsa,
               "history": hist[: st.iters + 1] if history else None}
        if status not in (0, 6):
            _check(status)
        return out

    def adjoint_sweep(self, mu, out=None, stream=None):
        import torch
        _need(self.n_elem * self.n_nodes, mu=mu, out=out)
        out = torch.empty_like(mu) if out is None else out
        _check(_lib.sn_adjoint_sweep(self._h, _ptr(mu), _ptr(out), FP64, _stream(stream)))
        return out

    def adjoint_iterate(self, g, mu=None, stream=None, **kw):
        import torch
        _need(self.n_elem * self.n_nodes, g=g, mu=mu)
        mu = torch.zeros_like(g) if mu is None else mu
        kw.setdefault("warm_start", False)
        o = make_opts(**kw)
        st = IterStats()
        status = _lib.sn_adjoint_iterate(self._h, C.byref(o), _ptr(g), _ptr(mu), C.byref(st), _stream(stream))
        if status not in (0, 6):
            _check(status)
        return {"mu": mu, "iters": st.iters, "rel_residual": st.rel_residual, "converged": status == 0,
                "inner_iters": st.inner_iters_total, "sweeps": st.n_sweeps, "ms_sweep": st.ms_sweep,
                "ms_dsa": st.ms_dsa}

    def gradients(self, phi, mu, stream=None):
        import torch
        _need(self.n_elem * self.n_nodes, phi=phi, mu=mu)
        gt, gs, gq = (torch.empty(self.n_elem, dtype=torch.float64, device=phi.device) for _ in range(3))
        _check(_lib.sn_gradients(self._h, _ptr(phi), _ptr(mu), _ptr(gt), _ptr(gs), _ptr(gq), _stream(stream)))
        return gt, gs, gq

    def unrolled_gradients(self, g, K, checkpoint_every=1, phi0=None, checkpoints=None, stream=None):
        """Gradients of g . phi_K for the K-th unaccelerated source iterate (sn_unrolled_gradients):
        (d_sigma_t, d_sigma_s, d_q).  checkpoints: None, or the buffer source_iterate filled with
        dsa="none", max_iters=K and the same checkpoint_every."""
        import torch
        m = self.n_elem * self.n_nodes
        if int(K) < 1 or int(checkpoint_every) < 1:
            raise ValueError("K and checkpoint_every must be >= 1")
        if g.numel() != m or (phi0 is not None and phi0.numel() != m):
            raise ValueError(f"g and phi0 need exactly n_elem * n_nodes = {m} values")
        need = (-(-int(K) // int(checkpoint_every)) - 1) * m
        if checkpoints is not None and checkpoints.numel() < need:
            raise ValueError(f"checkpoints need at least {need} values")
        gt, gs, gq = (torch.empty(self.n_elem, dtype=torch.float64, device=g.device) for _ in range(3))
        _check(_lib.sn_unrolled_gradients(self._h, None if phi0 is None else _ptr(phi0), int(K), int(checkpoint_every),
                                          None if checkpoints is None else _ptr(checkpoints), _ptr(g), _ptr(gt),
                                          _ptr(gs), _ptr(gq), _stream(stream)))
        return gt, gs, gq

    def levels(self, d):
        """Upwind level of every element for direction d (the device's Kahn pass), host int array."""
        out = np.empty(self.n_elem, dtype=np.int32)
        _check(_lib.sn_get_levels(self._h, int(d), out.ctypes.data_as(C.c_void_p)))
        return out

    def angular_flux(self, d, adjoint=False, precision="fp64", stream=None):
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        _check(_lib.sn_get_angular_flux(self._h, int(d), int(adjoint), _PREC.get(precision, precision), _ptr(out),
                                        _stream(stream)))
        return out

    def dsa_apply(self, x, stream=None, **kw):
        import torch
        _need(self.n_elem * self.n_nodes, x=x)
        y = torch.empty_like(x)
        o = make_opts(**kw)
        _check(_lib.sn_dsa_apply(self._h, C.byref(o), _ptr(x), _ptr(y), _stream(stream)))
        return y

    def dsa_solve(self, b, stream=None, **kw):
        import torch
        _need(self.n_elem * self.n_nodes, b=b)
        x = torch.empty_like(b)
        o = make_opts(**kw)
        its = C.c_int(0)
        _check(_lib.sn_dsa_solve(self._h, C.byref(o), _ptr(b), _ptr(x), C.byref(its), _stream(stream)))
        return x, its.value


class Batch:
    """Many meshes swept and iterated together (one launch per sweep for all instances)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (C.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        h = C.c_void_p()
        _check(_lib.sn_batch_create(arr, len(self.meshes), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.sn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, schedule="levels", block=64, max_blocks_per_sm=0):
        sched = SCHEDULES.index(schedule) if isinstance(schedule, str) else int(schedule)
        _check(_lib.sn_batch_set_schedule(self._h, sched, int(block), int(max_blocks_per_sm)))

    def autotune(self, precision="fp64", stream=None):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(_lib.sn_batch_autotune(self._h, _PREC.get(precision, precision), _stream(stream), C.byref(a),
                                      C.byref(b), C.byref(c)))
        return SCHEDULES[a.value], b.value, c.value

    def _ptrs(self, tensors):
        """One pointer per instance; each tensor must hold its instance's n_elem * n_nodes values."""
        tensors = list(tensors)
        if len(tensors) != len(self.meshes):
            raise ValueError(f"need one tensor per instance ({len(self.meshes)}), got {len(tensors)}")
        for i, (t, m) in enumerate(zip(tensors, self.meshes)):
            _need(m.n_elem * m.n_nodes, **{f"instance {i}": t})
        return (C.c_void_p * len(tensors))(*[None if t is None else _ptr(t).value for t in tensors])

    def sweep(self, phis_in=None, precision="fp64", stream=None):
        import torch
        ins = self._ptrs(phis_in) if phis_in is not None else None
        outs = [torch.empty(m.shape, dtype=torch.float64, device="cuda") for m in self.meshes]
        _check(_lib.sn_batch_sweep(self._h, ins, self._ptrs(outs), _PREC.get(precision, precision), _stream(stream)))
        return outs

    def source_iterate(self, phis=None, stream=None, **kw):
        import torch
        if phis is None:
            phis = [torch.zeros(m.shape, dtype=torch.float64, device="cuda") for m in self.meshes]
        kw.setdefault("warm_start", False)
        kw.setdefault("outer", "si")
        o = make_opts(**kw)
        stats = (IterStats * len(self.meshes))()
        status = _lib.sn_batch_source_iterate(self._h, C.byref(o), self._ptrs(phis), stats, _stream(stream))
        if status not in (0, 6):
            _check(status)
        return {"phi": phis, "iters": [st.iters for st in stats], "rel_residual": [st.rel_residual for st in stats],
                "converged": status == 0, "ms": stats[0].ms_total if len(stats) else 0.0}
