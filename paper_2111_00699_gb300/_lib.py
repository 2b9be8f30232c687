"""ctypes declarations of the libmpm C ABI (include/mpm.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of libmpm.so.  Loading fails loudly when the library is missing --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
# MPM_LIBRARY=ieee selects the build without fast-math intrinsics (the
# fast-math ablation); the default is the fast-math build
LIB_PATH = os.path.join(HERE, "libmpm_ieee.so" if os.environ.get("MPM_LIBRARY") == "ieee" else "libmpm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mpm.h")

MPM_OK, MPM_EINVAL, MPM_ENOMEM, MPM_ECAPACITY, MPM_EDOMAIN, MPM_ENONFINITE, MPM_ETIMEOUT, MPM_ECUDA, MPM_ENOTSUP = range(9)
STATUS_NAMES = ["MPM_OK", "MPM_EINVAL", "MPM_ENOMEM", "MPM_ECAPACITY", "MPM_EDOMAIN", "MPM_ENONFINITE",
                "MPM_ETIMEOUT", "MPM_ECUDA", "MPM_ENOTSUP"]
ELASTIC, FLUID, SNOW, SAND, NACC, NHSAND = 0, 1, 2, 3, 4, 5
STICKY, SLIP = 0, 1
APIC, ASFLIP = 0, 1
PHASES = 4
SORT_NOALLOC_MAX_KEYS = 1 << 20
P2G_VARIANTS = ("direct", "strided", "tile", "chunk4", "chunk8", "stage4", "stage8", "sacc4", "slab4", "warp",
                "warprun", "wtile8", "wxpose", "chunk8x2", "node", "chunk8s")
G2P_VARIANTS = ("direct", "chunk4", "chunk8", "tile", "occ", "stage", "occ10", "occsw")


class Material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("E", ctypes.c_float), ("nu", ctypes.c_float), ("rho", ctypes.c_float),
                ("gamma", ctypes.c_float), ("theta_c", ctypes.c_float), ("theta_s", ctypes.c_float),
                ("hardening", ctypes.c_float), ("friction_deg", ctypes.c_float),
                ("friction_M", ctypes.c_float), ("cohesion", ctypes.c_float), ("alpha0", ctypes.c_float)]


class Config(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int32 * 3), ("dx", ctypes.c_float), ("boundary", ctypes.c_int32),
                ("wall", ctypes.c_int32), ("gravity", ctypes.c_float * 3), ("max_particles", ctypes.c_int64),
                ("use_g2p2g", ctypes.c_int32), ("p2g_variant", ctypes.c_int32), ("g2p_variant", ctypes.c_int32),
                ("no_sort", ctypes.c_int32), ("resort_interval", ctypes.c_int32), ("transfer", ctypes.c_int32),
                ("flip_alpha", ctypes.c_float), ("flip_beta_min", ctypes.c_float), ("flip_beta_max", ctypes.c_float),
                ("flip_compress_margin", ctypes.c_float), ("reserved", ctypes.c_int32 * 1)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int32 * 3), ("dx", ctypes.c_float), ("boundary", ctypes.c_int32),
                ("wall", ctypes.c_int32), ("gravity", ctypes.c_float * 3), ("material", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("substeps", ctypes.c_int64), ("rebuilds", ctypes.c_int64), ("n_pblocks", ctypes.c_int64),
                ("grid_capacity", ctypes.c_int64), ("particle_capacity", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64)]


P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
F = ctypes.c_float

_PROTOS = {
    "mpm_create": (I, [P, P, I, P, P, P]),
    "mpm_add_particles": (I, [P, I64, P, P, P, I, I]),
    "mpm_emit_particles": (I, [P, I64, P, P, P, I, I]),
    "mpm_substep": (I, [P, F]),
    "mpm_advance": (I, [P, ctypes.c_double, F, F, I64, P, P]),
    "mpm_read_state": (I, [P, P, P, P, P, P, I]),
    "mpm_write_state": (I, [P, P, P, P, P, P, I]),
    "mpm_sync": (I, [P]),
    "mpm_rebuild": (I, [P]),
    "mpm_num_particles": (I64, [P]),
    "mpm_last_error": (ctypes.c_char_p, [P]),
    "mpm_destroy": (None, [P]),
    "mpm_get_stats": (I, [P, P]),
    "mpm_read_order": (I, [P, P, P, I]),
    "mpm_read_blocks": (I, [P, P, I64, P]),
    "mpm_debug_p2g": (I, [P, F, P, I]),
    "mpm_set_p2g_variant": (I, [P, I]),
    "mpm_set_cta_warps": (I, [P, I]),
    "mpm_set_resort_interval": (I, [P, I]),
    "mpm_set_layout": (I, [P, I]),
    "mpm_set_g2p_variant": (I, [P, I]),
    "mpm_set_g2p2g": (I, [P, I]),
    "mpm_use_graphs": (I, [P, I]),
    "mpm_debug_wait_timeout": (I, [I]),
    "mpm_debug_red_rate": (I, [P, I64, I64, I, I, P]),
    "mpm_graph_launches": (I64, [P]),
    "mpm_profile_enable": (I, [P, I]),
    "mpm_profile_read": (I, [P, P, P, I]),
    "mpm_radix_sort_pairs": (I, [P, P, P, P, I64, I, P, P, P]),
    "mpm_radix_sort_pairs_noalloc": (I, [P, P, P, P, I64, I, P]),
    "mpm_batch_create": (I, [I, P, P, I, P, P, P]),
    "mpm_batch_add_particles": (I, [P, I, I64, P, P, P]),
    "mpm_batch_substep": (I, [P, P]),
    "mpm_batch_use_graphs": (I, [P, I]),
    "mpm_batch_set_p2g_chunk": (I, [P, I]),
    "mpm_batch_set_cta_warps": (I, [P, I]),
    "mpm_batch_set_persistent": (I, [P, I]),
    "mpm_batch_read_state": (I, [P, I, P, P, P, P, P]),
    "mpm_batch_sync": (I, [P]),
    "mpm_batch_get_stats": (I, [P, P]),
    "mpm_batch_num_particles": (I64, [P, I]),
    "mpm_batch_last_error": (ctypes.c_char_p, [P]),
    "mpm_batch_destroy": (None, [P]),
    "mpm_diff_create": (I, [P, F, F, I64, P, P, P, P]),
    "mpm_diff_forward": (I, [P, F, P, P, P]),
    "mpm_diff_adjoint": (I, [P, F, P, P, P, P, P]),
    "mpm_diff_sync": (I, [P]),
    "mpm_diff_destroy": (None, [P]),
    "mpm_debug_svd": (I, [P, P, P, P, I64]),
    "mpm_debug_stress": (I, [P, P, P, P, I64]),
    "mpm_debug_plasticity": (I, [P, P, P, I64]),
}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/mpm.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_[a-z0-9_]+)\s*\(", text)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmpm.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2111_00699_gb300.build); there is no CPU fallback")
        try:
            import torch  # noqa: F401  -- load torch's CUDA runtime first, so one copy serves both
        except ImportError:
            pass
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class MpmError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s%s" % (name, (": " + msg) if msg else ""))


def material(kind=ELASTIC, E=1e4, nu=0.2, rho=1.0, gamma=7.0, theta_c=2.5e-2, theta_s=7.5e-3,
             hardening=10.0, friction_deg=30.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01) -> Material:
    return Material(int(kind), E, nu, rho, gamma, theta_c, theta_s, hardening, friction_deg, friction_M, cohesion,
                    alpha0)
