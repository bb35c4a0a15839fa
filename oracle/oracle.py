"""Python handle on the plain FP64 CPU oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It never imports the
CUDA package, and the CUDA package never imports it.

Layouts on this side are the oracle's own: particles are indexed by pid and
stored ``[N_p, 3]``; mesh arrays are ``[n^3]`` (x fastest) or ``[n^3, 3]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pic_oracle.c"
_LIB = _HERE / "liboracle.so"

# -ffp-contract=off: no fused multiply-adds, so x86 and Arm builds agree bit
# for bit (gcc contracts by default on aarch64).
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc into ``oracle/liboracle.so``, with OpenMP
    where the compiler has it (threads only over independent cells and
    particles; see ``orc_set_threads``), else serial."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.{os.getpid()}.tmp")
        r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", str(_SRC), "-o", str(tmp), "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.run(["gcc", *CFLAGS, str(_SRC), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Host threads of the oracle's independent loops (1 = serial, the
    default); returns the count in effect (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("np", ctypes.c_int64),
        ("K", ctypes.c_int64),
        ("cg_maxit", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("couple_qm_zero", ctypes.c_int64),
        ("couple_q_zero", ctypes.c_int64),
        ("dt", ctypes.c_double),
        ("qm", ctypes.c_double),
        ("q", ctypes.c_double),
        ("eps0", ctypes.c_double),
        ("nphys", ctypes.c_double),
        ("sigma0", ctypes.c_double),
        ("gmax", ctypes.c_double),
        ("fx_amp", ctypes.c_double),
        ("fx_speed", ctypes.c_double),
        ("vmean", ctypes.c_double * 3),
        ("vsig", ctypes.c_double),
        ("phi_amp", ctypes.c_double),
        ("phi_T", ctypes.c_double),
        ("phi_shift", ctypes.c_double * 3),
        ("cg_tol", ctypes.c_double),
        ("verify", ctypes.c_int64),
        ("E_app", ctypes.c_double * 3),
        ("dist", ctypes.c_int64),
        ("n_sigma", ctypes.c_int64),
        ("sigma_n", ctypes.c_double * 3),
        ("vbar", ctypes.c_double),
        ("t_ref", ctypes.c_double),
    ]


# verification switches (bit flags of ``verify``), Sec. 5.4
ISOLATE = 1
ERROR1 = 2
ERROR2 = 4
ANGLES = 8
ANISO = 16

# manufactured-distribution forms (``dist``)
DIST_CONFIG = 0   # travelling-wave f_x, Gaussian f_v
DIST_PAPER = 1    # the paper's own problem of Sec. 5.2 on the unit cube


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_CFG = ctypes.POINTER(OrcCfg)

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        sig = {
            "orc_philox": (None, [_U32, _U32, _U32]),
            "orc_u52": (ctypes.c_double, [ctypes.c_uint32, ctypes.c_uint32]),
            "orc_u32": (ctypes.c_double, [ctypes.c_uint32]),
            "orc_index": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32]),
            "orc_fxd": (ctypes.c_double, [_CFG, ctypes.c_double, ctypes.c_double]),
            "orc_Fxd": (ctypes.c_double, [_CFG, ctypes.c_double, ctypes.c_double]),
            "orc_xM": (ctypes.c_double, [_CFG, ctypes.c_double, ctypes.c_double]),
            "orc_xMdot": (ctypes.c_double, [_CFG, ctypes.c_double, ctypes.c_double]),
            "orc_vM": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double]),
            "orc_phiM": (ctypes.c_double, [_CFG, _D, ctypes.c_double]),
            "orc_EM": (None, [_CFG, _D, ctypes.c_double, _D]),
            "orc_lap_phiM": (ctypes.c_double, [_CFG, _D, ctypes.c_double]),
            "orc_rhoM": (ctypes.c_double, [_CFG, ctypes.c_double, _D, ctypes.c_double]),
            "orc_hs_R": (ctypes.c_double, [ctypes.c_double]),
            "orc_pmax": (ctypes.c_double, [_CFG]),
            "orc_hs_source": (None, [_CFG, _D, ctypes.c_int64, _D]),
            "orc_sample_xi": (None, [_CFG, ctypes.c_int64, _D]),
            "orc_create": (ctypes.c_void_p, [_CFG]),
            "orc_destroy": (None, [ctypes.c_void_p]),
            "orc_cell_of": (ctypes.c_int32, [_CFG, _D]),
            "orc_sort": (None, [ctypes.c_void_p]),
            "orc_deposit": (None, [ctypes.c_void_p]),
            "orc_gather": (None, [_CFG, _D, _D, _D]),
            "orc_rhs": (None, [ctypes.c_void_p, ctypes.c_double, _D]),
            "orc_neg_lap": (None, [ctypes.c_int64, _D, _D]),
            "orc_cg": (ctypes.c_int64, [ctypes.c_int64, _D, _D, ctypes.c_double, ctypes.c_int64, _D]),
            "orc_efield": (None, [ctypes.c_int64, _D, _D]),
            "orc_field": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_double]),
            "orc_dsmc_avg": (None, [ctypes.c_void_p, _D, ctypes.c_uint32, _D]),
            "orc_sample": (None, [ctypes.c_void_p, ctypes.c_double]),
            "orc_set_state": (None, [ctypes.c_void_p, _D, _D, ctypes.c_double, ctypes.c_int64]),
            "orc_wrap": (ctypes.c_double, [ctypes.c_double]),
            "orc_step": (None, [ctypes.c_void_p, ctypes.c_int64]),
            "orc_collide_avg": (None, [ctypes.c_void_p, ctypes.c_int64, _D, _D]),
            "orc_errors": (None, [ctypes.c_void_p, _D]),
            "orc_get_state": (None, [ctypes.c_void_p, _D, _D]),
            "orc_get_xi": (None, [ctypes.c_void_p, _D]),
            "orc_get_field": (None, [ctypes.c_void_p, _D, _D, _D]),
            "orc_get_sort": (None, [ctypes.c_void_p, _I32, _I32, _I32, _I32]),
            "orc_get_stats": (None, [ctypes.c_void_p, _I64, _D]),
            "orc_reset_stats": (None, [ctypes.c_void_p]),
            "orc_set_phi": (None, [ctypes.c_void_p, _D]),
            "orc_ntc_cell": (ctypes.c_int64, [_CFG, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_int64, _D]),
            "orc_angle_count": (ctypes.c_int64, [ctypes.c_void_p]),
            "orc_set_pair_log": (None, [ctypes.c_void_p, ctypes.c_int]),
            "orc_set_threads": (ctypes.c_int, [ctypes.c_int]),
            "orc_pair_log": (ctypes.c_int64, [ctypes.c_void_p, _I32, ctypes.c_int64]),
            "orc_pair_log_peek": (ctypes.c_int64, [ctypes.c_void_p, _I32, ctypes.c_int64]),
            "orc_aniso_F": (ctypes.c_double, [ctypes.c_double]),
            "orc_objective": (None, [ctypes.c_void_p, _D]),
            "orc_aniso_u": (ctypes.c_double, [ctypes.c_double]),
            "orc_get_angles": (None, [ctypes.c_void_p, _D]),
            "orc_fx_terms": (None, [_CFG, ctypes.c_int, ctypes.c_double, _D]),
            "orc_fx": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_Fx": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_xM_d": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_xMdot_d": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_vhat": (None, [_CFG, ctypes.c_double, _D, _D]),
            "orc_fv_paper": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_Fv_paper": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_vM_t": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_vMdot": (ctypes.c_double, [_CFG, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_fn": (None, [_CFG, ctypes.c_int, _D, ctypes.c_double, _D]),
            "orc_sigma_g": (ctypes.c_double, [_CFG, ctypes.c_double]),
            "orc_sg_max": (ctypes.c_double, [_CFG]),
            "orc_odd_source": (None, [_CFG, _D, ctypes.c_int64, ctypes.c_double, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        L.orc_set_threads(1)
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


def make_cfg(p: dict) -> OrcCfg:
    """Build the oracle's config from a plain parameter dict (see
    ``paper_2602_15130_gb300.workloads`` for the recipes)."""
    c = OrcCfg()
    c.n = int(p["n"])
    c.np = int(p["n_particles"])
    c.K = int(p["K"])
    c.cg_maxit = int(p.get("cg_maxit", 20000))
    c.seed = int(p.get("seed", 0))
    c.couple_qm_zero = int(p.get("couple_qm_zero", 0))
    c.couple_q_zero = int(p.get("couple_q_zero", 0))
    c.dt = float(p["dt"])
    c.qm = float(p.get("qm", 1.0))
    c.q = float(p.get("q", 1.0))
    c.eps0 = float(p.get("eps0", 1.0))
    c.nphys = float(p.get("n_phys", 1.0))
    c.sigma0 = float(p.get("sigma0", 0.0))
    c.gmax = float(p.get("g_max", 10.0 * np.sqrt(3.0)))
    c.fx_amp = float(p.get("fx_amp", 0.3))
    c.fx_speed = float(p.get("fx_speed", 0.1))
    for d in range(3):
        c.vmean[d] = float(p.get("v_mean", (0.2, 0.2, 0.2))[d])
        c.phi_shift[d] = float(p.get("phi_shift", (1 / 7, 1 / 5, 1 / 3))[d])
    c.vsig = float(p.get("v_sigma", 1.0))
    c.phi_amp = float(p.get("phi_amp", 0.1))
    c.phi_T = float(p.get("phi_T", 1.0))
    c.cg_tol = float(p.get("cg_tol", 1e-13))
    c.verify = int(p.get("verify", 0))
    for d in range(3):
        c.E_app[d] = float(p.get("E_app", (0.0, 0.0, 0.0))[d])
    c.dist = int(p.get("dist", DIST_CONFIG))
    c.n_sigma = int(p.get("n_sigma", 0))
    for k in range(3):
        c.sigma_n[k] = float(p.get("sigma_n", (0.0, 0.0, 0.0))[k])
    c.vbar = float(p.get("v_bar", 0.0))
    c.t_ref = float(p.get("t_ref", 1.0))
    return c


def philox(ctr, key):
    L = lib()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    L.orc_philox(c, k, o)
    return [int(o[i]) for i in range(4)]


class Oracle:
    """One oracle simulation state (pid-indexed, AoS)."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self.cfg = make_cfg(params)
        self.L = lib()
        self.h = self.L.orc_create(ctypes.byref(self.cfg))
        if not self.h:
            raise MemoryError("oracle allocation failed")
        self.np = self.cfg.np
        self.n = self.cfg.n

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- driving -------------------------------------------------------
    def sample(self, t0: float = 0.0):
        self.L.orc_sample(self.h, t0)

    def set_state(self, x: np.ndarray, v: np.ndarray, t0: float = 0.0, step: int = 0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        assert x.shape == (self.np, 3) and v.shape == (self.np, 3)
        self.L.orc_set_state(self.h, _dp(x), _dp(v), t0, step)

    def step(self, nsteps: int = 1):
        self.L.orc_step(self.h, nsteps)

    def collide_avg(self, phase: int):
        dv = np.zeros((self.np, 3))
        dvM = np.zeros((self.np, 3))
        self.L.orc_collide_avg(self.h, phase, _dp(dv), _dp(dvM))
        return dv, dvM

    def errors(self) -> np.ndarray:
        out = np.zeros(14)
        self.L.orc_errors(self.h, _dp(out))
        return out

    # --- reading -------------------------------------------------------
    def state(self):
        x = np.zeros((self.np, 3))
        v = np.zeros((self.np, 3))
        self.L.orc_get_state(self.h, _dp(x), _dp(v))
        return x, v

    def xi(self) -> np.ndarray:
        out = np.zeros((self.np, 6))
        self.L.orc_get_xi(self.h, _dp(out))
        return out

    def field(self):
        nc = self.n ** 3
        rho, phi, E = np.zeros(nc), np.zeros(nc), np.zeros((nc, 3))
        self.L.orc_get_field(self.h, _dp(rho), _dp(phi), _dp(E))
        return rho, phi, E

    def sort(self):
        nc = self.n ** 3
        cell = np.zeros(self.np, np.int32)
        count = np.zeros(nc, np.int32)
        start = np.zeros(nc + 1, np.int32)
        perm = np.zeros(self.np, np.int32)
        self.L.orc_get_sort(self.h, _ip(cell), _ip(count), _ip(start), _ip(perm))
        return cell, count, start, perm

    def stats(self) -> dict:
        out = (ctypes.c_int64 * 6)()
        res = ctypes.c_double()
        self.L.orc_get_stats(self.h, out, ctypes.byref(res))
        return dict(n_cand=out[0], n_coll=out[1], n_gmax_exceed=out[2], n_near_ties=out[3],
                    cg_iters=out[4], step=out[5], cg_res=res.value)

    def reset_stats(self):
        self.L.orc_reset_stats(self.h)

    def objective(self) -> np.ndarray:
        """(J, J_field, J_vel) at the current state."""
        out = np.zeros(3)
        self.L.orc_objective(self.h, _dp(out))
        return out

    def set_pair_log(self, on: bool = True):
        """Record the pair list of every collision call from now on (and
        clear what was recorded), or stop recording."""
        self.L.orc_set_pair_log(self.h, 1 if on else 0)

    def pair_log(self) -> np.ndarray:
        """The recorded pair list, ``[n, 8]`` int32 rows (c0, cell, outcome,
        slot, p, q, result, kind) in draw order; clears the log. slot = -1
        rows carry N_pairs in ``result`` (kind 4); candidate rows carry the
        in-cell indices p, q and 1/0 for accepted/rejected, kind 1 marking a
        near tie |U - sigma g/(sigma g)_max| < 1e-12."""
        cap = 1 << 16
        while True:
            out = np.zeros((cap, 8), np.int32)
            n = int(self.L.orc_pair_log_peek(self.h, _ip(out), cap))
            if n <= cap:
                self.L.orc_pair_log(self.h, None, 0)
                return out[:n].copy()
            cap = n

    def angles(self) -> np.ndarray:
        """(chi, eps) of every recorded collision, ``[N_coll, 2]``."""
        n = int(self.L.orc_angle_count(self.h))
        out = np.zeros((n, 2))
        if n:
            self.L.orc_get_angles(self.h, _dp(out))
        return out


# ---- scalar helpers used by the pins ---------------------------------------
def fxd(cfg, x, t):
    return lib().orc_fxd(ctypes.byref(cfg), x, t)


def Fxd(cfg, x, t):
    return lib().orc_Fxd(ctypes.byref(cfg), x, t)


def xM(cfg, xi, t):
    return lib().orc_xM(ctypes.byref(cfg), xi, t)


def xMdot(cfg, xm, t):
    return lib().orc_xMdot(ctypes.byref(cfg), xm, t)


def vM(cfg, d, xi):
    return lib().orc_vM(ctypes.byref(cfg), d, xi)


def fx_terms(cfg, d, t):
    out = np.zeros(4)
    lib().orc_fx_terms(ctypes.byref(cfg), d, t, _dp(out))
    return out


def fx(cfg, d, x, t):
    return lib().orc_fx(ctypes.byref(cfg), d, x, t)


def Fx(cfg, d, x, t):
    return lib().orc_Fx(ctypes.byref(cfg), d, x, t)


def xM_d(cfg, d, xi, t):
    return lib().orc_xM_d(ctypes.byref(cfg), d, xi, t)


def xMdot_d(cfg, d, xm, t):
    return lib().orc_xMdot_d(ctypes.byref(cfg), d, xm, t)


def vhat(cfg, t):
    vh, dvh = np.zeros(3), np.zeros(3)
    lib().orc_vhat(ctypes.byref(cfg), t, _dp(vh), _dp(dvh))
    return vh, dvh


def fv_paper(cfg, d, v, t):
    return lib().orc_fv_paper(ctypes.byref(cfg), d, v, t)


def Fv_paper(cfg, d, v, t):
    return lib().orc_Fv_paper(ctypes.byref(cfg), d, v, t)


def vM_t(cfg, d, xi, t):
    return lib().orc_vM_t(ctypes.byref(cfg), d, xi, t)


def vMdot(cfg, d, vm, t):
    return lib().orc_vMdot(ctypes.byref(cfg), d, vm, t)


def fn(cfg, k, vp, t):
    a = np.ascontiguousarray(vp, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_fn(ctypes.byref(cfg), k, _dp(a), t, _dp(out))
    return out


def sigma_g(cfg, g2):
    return lib().orc_sigma_g(ctypes.byref(cfg), g2)


def sg_max(cfg):
    return lib().orc_sg_max(ctypes.byref(cfg))


def odd_source(cfg, vp, ccell, t):
    a = np.ascontiguousarray(vp, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_odd_source(ctypes.byref(cfg), _dp(a), ccell, t, _dp(out))
    return out


def phiM(cfg, x, t):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_phiM(ctypes.byref(cfg), _dp(a), t)


def EM(cfg, x, t):
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_EM(ctypes.byref(cfg), _dp(a), t, _dp(out))
    return out


def lap_phiM(cfg, x, t):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_lap_phiM(ctypes.byref(cfg), _dp(a), t)


def rhoM(cfg, q, x, t):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_rhoM(ctypes.byref(cfg), q, _dp(a), t)


def pmax(cfg):
    return lib().orc_pmax(ctypes.byref(cfg))


def hs_R(a):
    return lib().orc_hs_R(a)


def hs_source(cfg, vp, ccell):
    a = np.ascontiguousarray(vp, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_hs_source(ctypes.byref(cfg), _dp(a), ccell, _dp(out))
    return out


def sample_xi(cfg, pid):
    out = np.zeros(6)
    lib().orc_sample_xi(ctypes.byref(cfg), pid, _dp(out))
    return out


def cg(n, b, phi0, tol, maxit):
    b = np.ascontiguousarray(b, dtype=np.float64)
    phi = np.ascontiguousarray(phi0, dtype=np.float64).copy()
    res = ctypes.c_double()
    it = lib().orc_cg(n, _dp(b), _dp(phi), tol, maxit, ctypes.byref(res))
    return phi, it, res.value


def neg_lap(n, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    lib().orc_neg_lap(n, _dp(x), _dp(y))
    return y


def efield(n, phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    E = np.zeros((n ** 3, 3))
    lib().orc_efield(n, _dp(phi), _dp(E))
    return E


def gather(cfg, E, x):
    E = np.ascontiguousarray(E, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_gather(ctypes.byref(cfg), _dp(E), _dp(xx), _dp(out))
    return out


def ntc_cell(cfg, c0, cell, outcome, v):
    """Run one NTC outcome (Algorithm 1) on velocities v[c,3]; returns
    (updated velocities, number of collisions)."""
    vv = np.ascontiguousarray(v, dtype=np.float64).copy()
    ncoll = lib().orc_ntc_cell(ctypes.byref(cfg), c0, cell, outcome, vv.shape[0], _dp(vv))
    return vv, ncoll


def F_chi_iso(chi):
    """Analytic CDF of the isotropic polar angle, (1 - cos chi)/2 (Eq. Fp_chi
    with the isotropic p(chi) = sin(chi)/2)."""
    return 0.5 * (1.0 - np.cos(chi))


def F_chi_aniso(chi):
    """Analytic CDF of the manufactured anisotropic polar angle (Sec. 5.1):
    sin^2(chi/2) - (3 + 5 cos 2 chi) sin^2(chi) / 58."""
    chi = np.asarray(chi)
    return np.sin(chi / 2) ** 2 - (3.0 + 5.0 * np.cos(2 * chi)) * np.sin(chi) ** 2 / 58.0


def F_eps(eps):
    """Analytic CDF of the azimuth, eps/(2 pi) (Eq. Fp_eps)."""
    return np.asarray(eps) / (2.0 * np.pi)


def angle_cdf_errors(alpha: np.ndarray, F) -> tuple[float, float]:
    """Sec. 4.4: e_r = F_emp(alpha_r) - F^M(alpha_r) for every recorded angle,
    with the empirical CDF F_emp(a) = (1/N) sum_s theta(a - alpha_s) and
    theta(0) = 1 (the CDF is right-continuous). Returns (eps_2, eps_inf)."""
    a = np.asarray(alpha, dtype=np.float64)
    N = a.size
    if N == 0:
        return 0.0, 0.0
    srt = np.sort(a)
    Femp = np.searchsorted(srt, a, side="right") / N
    e = Femp - F(a)
    return float(np.sqrt(np.mean(e * e))), float(np.max(np.abs(e)))


def wrap(x):
    return lib().orc_wrap(x)


def time_steps(params: dict, nsteps: int, t0: float = 0.0) -> dict:
    """Time the oracle as it stands: sample, then ``nsteps`` steps; returns
    particle-steps/s over the stepping only (single host thread)."""
    o = Oracle(params)
    o.sample(t0)
    t = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t
    o.close()
    return {"seconds": dt, "particle_steps_per_s": params["n_particles"] * nsteps / dt}
