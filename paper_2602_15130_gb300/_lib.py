"""ctypes declarations of the C ABI in ``include/pic.h``.

The shared library ``libpic_gb300.so`` is built in-tree by
``paper_2602_15130_gb300._build`` (``__graft_entry__.build()``). There is
no fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "libpic_gb300.so"
HEADER = PKG.parent / "include" / "pic.h"

STATUS = {
    0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_ECUDA", 4: "PIC_ENOCONV",
    5: "PIC_ETIMEOUT", 6: "PIC_ESTATE", 7: "PIC_ECAPACITY",
}
PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ENOCONV, PIC_ETIMEOUT, PIC_ESTATE, PIC_ECAPACITY = range(8)
PIC_FP64 = 0
PIC_MIXED = 1
# verification switches (pic_config.verify bits)
PIC_VERIFY_ISOLATE, PIC_VERIFY_ERROR1, PIC_VERIFY_ERROR2, PIC_VERIFY_ANGLES, PIC_VERIFY_ANISO = 1, 2, 4, 8, 16
PIC_ANGLE_BINS = 4194304
PIC_DIST_CONFIG, PIC_DIST_PAPER = 0, 1
NUM_KERNEL_CLASSES = 9
KERNEL_CLASSES = ["sample", "sort", "sort_gather_deposit", "rhs", "cg_efield", "dsmc", "kick_drift",
                  "error_norms", "other"]


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("n_particles", ctypes.c_int64),
        ("dt", ctypes.c_double),
        ("qm", ctypes.c_double),
        ("q", ctypes.c_double),
        ("eps0", ctypes.c_double),
        ("n_phys", ctypes.c_double),
        ("sigma0", ctypes.c_double),
        ("g_max", ctypes.c_double),
        ("fx_amp", ctypes.c_double),
        ("fx_speed", ctypes.c_double),
        ("v_mean", ctypes.c_double * 3),
        ("v_sigma", ctypes.c_double),
        ("phi_amp", ctypes.c_double),
        ("phi_T", ctypes.c_double),
        ("phi_shift", ctypes.c_double * 3),
        ("couple_qm_zero", ctypes.c_int32),
        ("couple_q_zero", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("max_ppc", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("cg_tol", ctypes.c_double),
        ("cg_maxit", ctypes.c_int32),
        ("verify", ctypes.c_int32),
        ("dist", ctypes.c_int32),
        ("n_sigma", ctypes.c_int32),
        ("sigma_n", ctypes.c_double * 3),
        ("v_bar", ctypes.c_double),
        ("t_ref", ctypes.c_double),
    ]


class PicErrors(ctypes.Structure):
    _fields_ = [("eps2", ctypes.c_double * 7), ("epsinf", ctypes.c_double * 7)]


class PicStats(ctypes.Structure):
    _fields_ = [
        ("n_cand", ctypes.c_int64),
        ("n_coll", ctypes.c_int64),
        ("n_gmax_exceed", ctypes.c_int64),
        ("n_near_ties", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("step", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("cg_iters_last", ctypes.c_int32),
        ("cg_iters_max", ctypes.c_int32),
        ("cg_res_last", ctypes.c_double),
        ("graph_replays", ctypes.c_int64),
        ("tuned_block", ctypes.c_int32),
        ("tuned_tile", ctypes.c_int32),
        ("n_floor_ties", ctypes.c_int64),
        ("binned_loads", ctypes.c_int64),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class PicAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class PicAngleStats(ctypes.Structure):
    _fields_ = [
        ("n_coll", ctypes.c_int64),
        ("max_bin", ctypes.c_int64 * 2),
        ("eps2_chi", ctypes.c_double),
        ("epsinf_chi", ctypes.c_double),
        ("eps2_eps", ctypes.c_double),
        ("epsinf_eps", ctypes.c_double),
    ]


class PicKernelTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NUM_KERNEL_CLASSES), ("launches", ctypes.c_int64 * NUM_KERNEL_CLASSES)]


_V = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_S = ctypes.c_int
SIGNATURES = {
    "pic_config_default": (_S, [ctypes.POINTER(PicConfig)]),
    "pic_validate_config": (_S, [ctypes.POINTER(PicConfig)]),
    "pic_derived": (_S, [ctypes.POINTER(PicConfig), _D]),
    "pic_create": (_S, [ctypes.POINTER(PicConfig), _V, ctypes.POINTER(PicAllocator), ctypes.POINTER(_V)]),
    "pic_sample_mms": (_S, [_V, ctypes.c_double]),
    "pic_step": (_S, [_V, ctypes.c_int32]),
    "pic_collide_avg": (_S, [_V, ctypes.c_int32, _V, _V]),
    "pic_mms_error": (_S, [_V, ctypes.POINTER(PicErrors)]),
    "pic_get_state": (_S, [_V, _V, _V]),
    "pic_set_state": (_S, [_V, _V, _V, ctypes.c_double, ctypes.c_int64]),
    "pic_get_field": (_S, [_V, _V, _V, _V]),
    "pic_get_sort": (_S, [_V, _V, _V, _V, _V]),
    "pic_get_stats": (_S, [_V, ctypes.POINTER(PicStats)]),
    "pic_reset_stats": (_S, [_V]),
    "pic_get_angle_stats": (_S, [_V, ctypes.POINTER(PicAngleStats)]),
    "pic_adjoint_gradient": (_S, [_V, ctypes.c_int32, ctypes.c_int32, _D, _V, _D, _D, _V]),
    "pic_set_profiling": (_S, [_V, ctypes.c_int32]),
    "pic_get_kernel_times": (_S, [_V, ctypes.POINTER(PicKernelTimes)]),
    "pic_destroy": (None, [_V]),
    "pic_status_string": (ctypes.c_char_p, [_S]),
    "pic_create_batch": (_S, [ctypes.POINTER(PicConfig), ctypes.c_int32, _V, ctypes.POINTER(PicAllocator),
                              ctypes.POINTER(_V)]),
    "pic_batch_mms_error": (_S, [_V, ctypes.POINTER(PicErrors)]),
    "pic_batch_get_state": (_S, [_V, ctypes.c_int32, _V, _V]),
    "pic_batch_info": (_S, [_V, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int32)]),
    "pic_inject_barrier_stall": (_S, [_V]),
    "pic_get_step_history": (_S, [_V, _V, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "pic_set_decision_log": (_S, [_V, ctypes.c_int32, ctypes.c_int64]),
    "pic_get_decision_log": (_S, [_V, _V, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "pic_measure_alu_peaks": (_S, [_V, _D]),
    "pic_measure_link": (_S, [_V, ctypes.c_uint64, _V, _D]),
    "pic_poisson_solve_noalloc": (_S, [ctypes.c_int32, _V, _V, _V, ctypes.c_double, ctypes.c_int32, _V,
                                      ctypes.POINTER(ctypes.c_int32), _D]),
}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/pic.h."""
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", text)))


def load() -> ctypes.CDLL:
    """Load the in-tree CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'). There is no CPU fallback.")
    L = ctypes.CDLL(str(LIB_PATH))
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class PicError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().pic_status_string(status).decode()
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


def check(status: int, where: str, allow=()):
    if status != PIC_OK and status not in allow:
        raise PicError(status, where)
    return status
