"""GB300-native manufactured-solution PIC + DSMC hot path.

``Pic`` wraps one ``pic_ctx`` of the C ABI (``include/pic.h``); every step
of the method runs in the library's CUDA kernels. This module only
marshals arguments: numpy arrays (host) or torch tensors (host or CUDA) go
in as pointers, results come back as numpy arrays or torch CUDA tensors.
Device memory of the context is drawn from torch's caching allocator.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib, workloads
from ._lib import PicConfig, PicError, check, load

__all__ = ["Pic", "Batch", "PicConfig", "PicError", "PicObjective", "make_config", "workloads", "load"]


def make_config(p: dict) -> PicConfig:
    """pic_config from a workload dict (see ``workloads``).

    Keys are the pic_config fields of ``include/pic.h``: ``n``, ``K``,
    ``n_particles`` and ``dt`` are required; ``qm``, ``q``, ``eps0``,
    ``n_phys``, ``sigma0``, ``g_max``, ``fx_amp``, ``fx_speed``, ``v_mean``,
    ``v_sigma``, ``phi_amp``, ``phi_T``, ``phi_shift``, ``couple_qm_zero``,
    ``couple_q_zero``, ``precision`` (0 FP64, 1 the precision form),
    ``max_ppc``, ``seed``, ``cg_tol``, ``cg_maxit``, ``verify``
    (PIC_VERIFY_* bits), ``dist`` (PIC_DIST_*), ``n_sigma`` and ``sigma_n``
    (odd-power cross section), ``v_bar`` and ``t_ref`` (the paper's problem)
    are optional and default to the library's defaults."""
    L = load()
    c = PicConfig()
    check(L.pic_config_default(ctypes.byref(c)), "pic_config_default")
    c.n = int(p["n"])
    c.K = int(p["K"])
    c.n_particles = int(p["n_particles"])
    c.dt = float(p["dt"])
    for name in ("qm", "q", "eps0", "sigma0", "fx_amp", "fx_speed", "v_sigma", "phi_amp", "phi_T", "cg_tol"):
        if name in p:
            setattr(c, name, float(p[name]))
    if "n_phys" in p:
        c.n_phys = float(p["n_phys"])
    if "g_max" in p:
        c.g_max = float(p["g_max"])
    for d in range(3):
        if "v_mean" in p:
            c.v_mean[d] = float(p["v_mean"][d])
        if "phi_shift" in p:
            c.phi_shift[d] = float(p["phi_shift"][d])
    c.couple_qm_zero = int(p.get("couple_qm_zero", 0))
    c.couple_q_zero = int(p.get("couple_q_zero", 0))
    c.max_ppc = int(p.get("max_ppc", 0))
    c.precision = int(p.get("precision", 0))
    c.seed = int(p.get("seed", 0))
    c.cg_maxit = int(p.get("cg_maxit", c.cg_maxit))
    c.verify = int(p.get("verify", 0))
    c.dist = int(p.get("dist", _lib.PIC_DIST_CONFIG))
    c.n_sigma = int(p.get("n_sigma", 0))
    for k in range(3):
        c.sigma_n[k] = float(p.get("sigma_n", (0.0, 0.0, 0.0))[k])
    c.v_bar = float(p.get("v_bar", 0.0))
    c.t_ref = float(p.get("t_ref", 1.0))
    return c


class _TorchAllocator:
    """pic_allocator backed by torch's CUDA caching allocator."""

    def __init__(self):
        import torch

        self.torch = torch
        self.live = {}
        self._a = _lib.ALLOC_FN(self._alloc)
        self._f = _lib.FREE_FN(self._free)
        self.struct = _lib.PicAllocator(self._a, self._f, None)

    def _alloc(self, user, nbytes):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        except Exception:
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        return ptr

    def _free(self, user, ptr):
        self.live.pop(ptr, None)


def _ptr(a, count=None, dtype=np.float64):
    """(pointer, keepalive) for a C-contiguous numpy array or torch tensor of
    ``dtype`` with exactly ``count`` elements (any count when None); anything
    else raises ValueError, so the library never reads or writes past it."""
    if a is None:
        return None, None
    want = np.dtype(dtype)
    if isinstance(a, np.ndarray):
        ok, n, dt = a.flags.c_contiguous and a.dtype == want, a.size, a.dtype
    else:
        import torch

        tdt = {np.dtype(np.float64): torch.float64, np.dtype(np.int32): torch.int32}[want]
        ok, n, dt = a.is_contiguous() and a.dtype == tdt, a.numel(), a.dtype
    if not ok or (count is not None and n != count):
        raise ValueError(f"expected a contiguous {want} buffer of {count} elements, got {dt} with {n}")
    return (a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()), a


class Pic:
    """One simulation context on the current CUDA device."""

    def __init__(self, params: dict | PicConfig, stream=None, torch_allocator: bool = True):
        import torch

        L = load()
        self.L = L
        self.cfg = params if isinstance(params, PicConfig) else make_config(params)
        self.np = int(self.cfg.n_particles)
        self.n = int(self.cfg.n)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self._alloc = _TorchAllocator() if torch_allocator else None
        ctx = ctypes.c_void_p()
        check(L.pic_create(ctypes.byref(self.cfg), ctypes.c_void_p(handle),
                           ctypes.byref(self._alloc.struct) if self._alloc else None, ctypes.byref(ctx)),
              "pic_create")
        self.ctx = ctx

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.L.pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the method -------------------------------------------------------
    def sample_mms(self, t0: float = 0.0, allow=()):
        return check(self.L.pic_sample_mms(self.ctx, float(t0)), "pic_sample_mms", allow)

    def step(self, nsteps: int = 1, allow=()):
        return check(self.L.pic_step(self.ctx, int(nsteps)), "pic_step", allow)

    def collide_avg(self, phase: int, out=None):
        """(<dv>, <dv^M>) [N_p, 3] pid-indexed; numpy unless ``out`` tensors given."""
        if out is None:
            out = (np.zeros((self.np, 3)), np.zeros((self.np, 3)))
        pa, ka = _ptr(out[0], 3 * self.np)
        pb, kb = _ptr(out[1], 3 * self.np)
        check(self.L.pic_collide_avg(self.ctx, int(phase), pa, pb), "pic_collide_avg")
        return out

    def mms_error(self) -> dict:
        e = _lib.PicErrors()
        check(self.L.pic_mms_error(self.ctx, ctypes.byref(e)), "pic_mms_error", allow=(_lib.PIC_ENOCONV,))
        names = ["x", "y", "z", "u", "v", "w", "phi"]
        return {"eps2": dict(zip(names, list(e.eps2))), "epsinf": dict(zip(names, list(e.epsinf))),
                "array": np.array(list(e.eps2) + list(e.epsinf))}

    # -- state and test hooks ---------------------------------------------
    def get_state(self, out=None):
        if out is None:
            out = (np.zeros((self.np, 3)), np.zeros((self.np, 3)))
        pa, ka = _ptr(out[0], 3 * self.np)
        pb, kb = _ptr(out[1], 3 * self.np)
        check(self.L.pic_get_state(self.ctx, pa, pb), "pic_get_state")
        return out

    def set_state(self, x, v, t0: float = 0.0, step: int = 0, allow=()):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
            v = np.ascontiguousarray(v, dtype=np.float64)
        pa, ka = _ptr(x, 3 * self.np)
        pb, kb = _ptr(v, 3 * self.np)
        return check(self.L.pic_set_state(self.ctx, pa, pb, float(t0), int(step)), "pic_set_state", allow)

    def inject_barrier_stall(self):
        """Make the next Poisson solve's bounded barrier wait run out
        (pic_inject_barrier_stall): that call then returns PIC_ETIMEOUT."""
        check(self.L.pic_inject_barrier_stall(self.ctx), "pic_inject_barrier_stall")

    def get_field(self):
        nc = self.n ** 3
        rho, phi, E = np.zeros(nc), np.zeros(nc), np.zeros((nc, 3))
        check(self.L.pic_get_field(self.ctx, rho.ctypes.data, phi.ctypes.data, E.ctypes.data), "pic_get_field")
        return rho, phi, E

    def get_sort(self):
        nc = self.n ** 3
        cell = np.zeros(self.np, np.int32)
        count = np.zeros(nc, np.int32)
        start = np.zeros(nc + 1, np.int32)
        perm = np.zeros(self.np, np.int32)
        check(self.L.pic_get_sort(self.ctx, cell.ctypes.data, count.ctypes.data, start.ctypes.data,
                                  perm.ctypes.data), "pic_get_sort")
        return cell, count, start, perm

    def stats(self, allow=(_lib.PIC_ENOCONV,)) -> dict:
        s = _lib.PicStats()
        check(self.L.pic_get_stats(self.ctx, ctypes.byref(s)), "pic_get_stats", allow)
        return {f: getattr(s, f) for f, _ in _lib.PicStats._fields_}

    def reset_stats(self):
        check(self.L.pic_reset_stats(self.ctx), "pic_reset_stats")

    def step_history(self) -> np.ndarray:
        """[steps, 4] int64 per step since the last reset/sampling: CG
        iterations, candidate pairs, collisions, candidates with g > g_max."""
        out = np.zeros((4096, 4), np.int64)
        n = ctypes.c_int64()
        check(self.L.pic_get_step_history(self.ctx, out.ctypes.data, 4096, ctypes.byref(n)), "pic_get_step_history")
        return out[:n.value].copy()

    def set_decision_log(self, mode: int, capacity: int = 1 << 20):
        """Log the collision calls' decisions (pic_set_decision_log):
        mode 0 off, 1 flagged FP32 decisions only, 2 every N_pairs draw and
        candidate pair."""
        check(self.L.pic_set_decision_log(self.ctx, int(mode), int(capacity)), "pic_set_decision_log")
        self._dlog_cap = int(capacity)

    def decision_log(self) -> np.ndarray:
        """The logged records [n, 8] int32 (c0, cell, outcome, slot, p, q,
        result, kind) and clear the log; raises if records were dropped."""
        cap = getattr(self, "_dlog_cap", 0)
        out = np.zeros((max(cap, 1), 8), np.int32)
        n = ctypes.c_int64()
        check(self.L.pic_get_decision_log(self.ctx, out.ctypes.data, cap, ctypes.byref(n)), "pic_get_decision_log")
        if n.value > cap:
            raise RuntimeError(f"decision log overflow: {n.value} records, capacity {cap}")
        return out[:n.value].copy()

    def adjoint_gradient(self, nsteps: int, every: int = 20, E_app=(0.1, 0.1, 0.1), v0=None, grad: bool = True):
        """Objective J = J_field + J_vel at t_N and, with ``grad``, its
        pathwise gradient (dJ/dE_app [3], dJ/dv0 [N_p, 3]) by the library's
        adjoint (pic_adjoint_gradient). v0: [N_p, 3] pid order (numpy or a
        CUDA tensor), None for v^M(0)."""
        J = (ctypes.c_double * 3)()
        ea = (ctypes.c_double * 3)(*[float(x) for x in E_app])
        dE = (ctypes.c_double * 3)() if grad else None
        dv = np.zeros((self.np, 3)) if grad else None
        if v0 is not None and isinstance(v0, np.ndarray):
            v0 = np.ascontiguousarray(v0, dtype=np.float64)
        pv, kv = _ptr(v0, 3 * self.np)
        pd, kd = _ptr(dv, 3 * self.np)
        check(self.L.pic_adjoint_gradient(self.ctx, int(nsteps), int(every), ea, pv, J, dE, pd),
              "pic_adjoint_gradient")
        out = {"J": J[0], "J_field": J[1], "J_vel": J[2]}
        if grad:
            out["dJ_dEapp"] = np.array(list(dE))
            out["dJ_dv0"] = dv
        return out

    def angle_stats(self) -> dict:
        """Scattering-angle CDF errors of the recorded collisions (needs
        ``verify`` with PIC_VERIFY_ANGLES)."""
        a = _lib.PicAngleStats()
        check(self.L.pic_get_angle_stats(self.ctx, ctypes.byref(a)), "pic_get_angle_stats")
        return {"n_coll": a.n_coll, "max_bin": (a.max_bin[0], a.max_bin[1]), "eps2_chi": a.eps2_chi,
                "epsinf_chi": a.epsinf_chi, "eps2_eps": a.eps2_eps, "epsinf_eps": a.epsinf_eps}

    def set_profiling(self, on: bool):
        check(self.L.pic_set_profiling(self.ctx, 1 if on else 0), "pic_set_profiling")

    def kernel_times(self) -> dict:
        k = _lib.PicKernelTimes()
        check(self.L.pic_get_kernel_times(self.ctx, ctypes.byref(k)), "pic_get_kernel_times")
        return {name: {"ms": k.ms[i], "launches": k.launches[i]} for i, name in enumerate(_lib.KERNEL_CLASSES)}


class Batch(Pic):
    """Independent replicates advanced together (pic_create_batch)."""

    def __init__(self, params_list, stream=None, torch_allocator: bool = True):
        import torch

        L = load()
        self.L = L
        cfgs = (PicConfig * len(params_list))(*[make_config(p) for p in params_list])
        self.cfgs = cfgs
        self.nrep = len(params_list)
        self.np_rep = [int(p["n_particles"]) for p in params_list]
        self.np = sum(self.np_rep)
        self.n = None
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self._alloc = _TorchAllocator() if torch_allocator else None
        ctx = ctypes.c_void_p()
        check(L.pic_create_batch(cfgs, len(params_list), ctypes.c_void_p(handle),
                                 ctypes.byref(self._alloc.struct) if self._alloc else None, ctypes.byref(ctx)),
              "pic_create_batch")
        self.ctx = ctx

    def mms_error(self):
        out = (_lib.PicErrors * self.nrep)()
        check(self.L.pic_batch_mms_error(self.ctx, out), "pic_batch_mms_error", allow=(_lib.PIC_ENOCONV,))
        return np.array([list(e.eps2) + list(e.epsinf) for e in out])

    def get_state(self, rep: int, out=None):
        n = self.np_rep[rep]
        if out is None:
            out = (np.zeros((n, 3)), np.zeros((n, 3)))
        pa, ka = _ptr(out[0], 3 * n)
        pb, kb = _ptr(out[1], 3 * n)
        check(self.L.pic_batch_get_state(self.ctx, int(rep), pa, pb), "pic_batch_get_state")
        return out

    def cg_iters(self):
        it = (ctypes.c_int32 * self.nrep)()
        check(self.L.pic_batch_info(self.ctx, None, None, it), "pic_batch_info")
        return list(it)


def measure_alu_peaks(stream=None) -> dict:
    """Measured issue rates of the current GPU (pic_measure_alu_peaks), per
    second: INT32 multiply-add, 3-input logic, FP32 FMA, FP64 FMA and
    Philox4x32-10 blocks."""
    L = load()
    out = (ctypes.c_double * 5)()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    check(L.pic_measure_alu_peaks(ctypes.c_void_p(handle), out), "pic_measure_alu_peaks")
    return dict(zip(["imad", "lop3", "ffma", "dfma", "philox_blocks"], list(out)))


def measure_link(host, stream=None) -> dict:
    """Rate of the host link each way (pic_measure_link), bytes per second:
    DMA copies between the pinned host tensor ``host`` and a device buffer
    of its size."""
    L = load()
    out = (ctypes.c_double * 2)()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    nbytes = host.numel() * host.element_size()
    check(L.pic_measure_link(ctypes.c_void_p(host.data_ptr()), ctypes.c_uint64(nbytes), ctypes.c_void_p(handle), out),
          "pic_measure_link")
    return {"h2d": out[0], "d2h": out[1], "bytes": nbytes}


def derived(params: dict) -> dict:
    """Host-only derived constants (no GPU needed)."""
    L = load()
    c = make_config(params)
    out = (ctypes.c_double * 5)()
    check(L.pic_derived(ctypes.byref(c), out), "pic_derived")
    return {"w": out[0], "dV": out[1], "pmax": out[2], "ppc": out[3], "inv_pmax": out[4]}



try:
    import torch as _torch
except ImportError:  # pragma: no cover - the library needs torch for its allocator
    _torch = None

if _torch is not None:

    class PicObjective(_torch.autograd.Function):
        """J(E_app, v0) of ``Pic.adjoint_gradient`` as an autograd function:
        forward runs the library's simulation with checkpoints and its
        hand-written pathwise adjoint; backward scales the stored gradient.
        Call as ``PicObjective.apply(E_app, v0, sim, nsteps, every)``."""

        @staticmethod
        def forward(ctx, E_app, v0, sim, nsteps, every):
            e = [float(x) for x in E_app.detach().cpu().tolist()]
            v = v0.detach().to(_torch.float64).contiguous()
            r = sim.adjoint_gradient(nsteps, every, e, v if v.is_cuda else v.numpy(), grad=True)
            ctx.save_for_backward(_torch.as_tensor(r["dJ_dEapp"], dtype=E_app.dtype, device=E_app.device),
                                  _torch.as_tensor(r["dJ_dv0"], dtype=v0.dtype, device=v0.device))
            return _torch.tensor(r["J"], dtype=_torch.float64, device=E_app.device)

        @staticmethod
        def backward(ctx, g):
            dE, dv = ctx.saved_tensors
            return g * dE, g * dv, None, None, None
else:  # pragma: no cover
    PicObjective = None
