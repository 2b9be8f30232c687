"""FP64 CPU oracle for one explicit MLS-MPM substep (ctypes binding).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never loads it and the two share no code.

The C sources next to this file implement the method of "Principles towards
Real-Time Simulation of Material Point Method on Modern GPUs" (Sec. 4 phase
list; Sec. 4.2 keys, sort and physical blocks) with the MLS-MPM transfers and
constitutive models of the literature the paper cites; each C file's header
names the passage and the formula it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = ["bspline.c", "svd.c", "material.c", "transfer.c", "keys.c", "adjoint.c"]

ELASTIC, FLUID, SNOW, SAND, NACC, NHSAND = 0, 1, 2, 3, 4, 5
STICKY, SLIP = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into liboracle.so with gcc (no FMA contraction, so
    x86 and Arm hosts round identically)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class Material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho", ctypes.c_double), ("gamma", ctypes.c_double),
                ("theta_c", ctypes.c_double), ("theta_s", ctypes.c_double),
                ("hardening", ctypes.c_double), ("friction_deg", ctypes.c_double),
                ("friction_M", ctypes.c_double), ("cohesion", ctypes.c_double), ("alpha0", ctypes.c_double)]


APIC, ASFLIP = 0, 1


class Config(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int32 * 3), ("dx", ctypes.c_double),
                ("boundary", ctypes.c_int32), ("wall", ctypes.c_int32),
                ("gravity", ctypes.c_double * 3),
                ("transfer", ctypes.c_int32), ("flip_alpha", ctypes.c_double),
                ("flip_beta_min", ctypes.c_double), ("flip_beta_max", ctypes.c_double),
                ("flip_compress_margin", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int32 * 3), ("dim", ctypes.c_int32 * 3),
                ("m", ctypes.POINTER(ctypes.c_double)), ("p", ctypes.POINTER(ctypes.c_double)),
                ("v0", ctypes.POINTER(ctypes.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.orc_bspline_weights.argtypes = [ctypes.c_double, P]
        L.orc_svd3.argtypes = [P, P, P, P]
        L.orc_lame.argtypes = [ctypes.c_double, ctypes.c_double, P, P]
        L.orc_kirchhoff.argtypes = [P, P, ctypes.c_double, P]
        L.orc_wave_speed.argtypes = [P]
        L.orc_wave_speed.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_plasticity.argtypes = [P, P, P]
        L.orc_grid_bounds.argtypes = [i64, P, ctypes.c_double, P, P]
        L.orc_p2g.argtypes = [P, P, i64, P, P, P, P, P, P, P, ctypes.c_double, P]
        L.orc_p2g.restype = ctypes.c_int
        L.orc_grid_update.argtypes = [P, ctypes.c_double, P]
        L.orc_g2p.argtypes = [P, P, i64, P, P, P, P, P, P, ctypes.c_double, P]
        L.orc_g2p.restype = ctypes.c_int
        L.orc_substep.argtypes = [P, P, i64, P, P, P, P, P, P, P, ctypes.c_double]
        L.orc_substep.restype = ctypes.c_int
        L.orc_p2g_node.argtypes = [P, P, i64, P, P, P, P, P, P, P, ctypes.c_double, P, P]
        L.orc_particle_keys.argtypes = [i64, P, ctypes.c_float, ctypes.c_int32, P]
        L.orc_particle_keys.restype = ctypes.c_int
        L.orc_stable_sort.argtypes = [i64, P, P]
        L.orc_pblocks.argtypes = [i64, P, ctypes.c_int32, P]
        L.orc_pblocks.restype = i64
        L.orc_diff_forward.argtypes = [P, ctypes.c_double, ctypes.c_double, i64, P, P, ctypes.c_double, P, P]
        L.orc_diff_forward.restype = ctypes.c_int
        L.orc_diff_adjoint.argtypes = [P, ctypes.c_double, ctypes.c_double, i64, P, P, ctypes.c_double, P, P, P, P]
        L.orc_diff_adjoint.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def material(kind, E=1e4, nu=0.2, rho=1.0, gamma=7.0, theta_c=2.5e-2, theta_s=7.5e-3,
             hardening=10.0, friction_deg=30.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01) -> Material:
    return Material(int(kind), E, nu, rho, gamma, theta_c, theta_s, hardening, friction_deg, friction_M, cohesion,
                    alpha0)


def config(res, dx, boundary=STICKY, wall=3, gravity=(0.0, -9.8, 0.0), transfer=APIC, flip_alpha=0.0,
           flip_beta_min=0.0, flip_beta_max=0.0, flip_compress_margin=0.0) -> Config:
    r = (ctypes.c_int32 * 3)(*[int(v) for v in (res if hasattr(res, "__len__") else (res,) * 3)])
    return Config(r, float(dx), int(boundary), int(wall), (ctypes.c_double * 3)(*gravity), int(transfer),
                  float(flip_alpha), float(flip_beta_min), float(flip_beta_max), float(flip_compress_margin))


def _mats(mats):
    if isinstance(mats, Material):
        mats = [mats]
    arr = (Material * len(mats))(*mats)
    return arr


class State:
    """Particle state in FP64 (AoS row-major), as the oracle reads and writes it."""

    def __init__(self, x, v=None, C=None, F=None, Jp=None, vol=None, mat=None):
        n = len(x)
        self.x = _f64(x, (n, 3)).copy()
        self.v = _f64(np.zeros((n, 3)) if v is None else v, (n, 3)).copy()
        self.C = _f64(np.zeros((n, 3, 3)) if C is None else C, (n, 3, 3)).copy()
        self.F = _f64(np.tile(np.eye(3), (n, 1, 1)) if F is None else F, (n, 3, 3)).copy()
        self.Jp = _f64(np.ones(n) if Jp is None else Jp, (n,)).copy()
        self.vol = _f64(np.ones(n) if vol is None else (np.full(n, vol) if np.isscalar(vol) else vol), (n,)).copy()
        self.mat = np.ascontiguousarray(np.zeros(n) if mat is None else (np.full(n, mat) if np.isscalar(mat) else mat),
                                        dtype=np.int32).copy()

    @property
    def n(self):
        return len(self.x)

    def copy(self):
        return State(self.x, self.v, self.C, self.F, self.Jp, self.vol, self.mat)


def bspline_weights(f: float) -> np.ndarray:
    w = np.zeros(3)
    lib().orc_bspline_weights(float(f), _p(w))
    return w


def svd3(F):
    F = _f64(F, (3, 3))
    U, s, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    lib().orc_svd3(_p(F), _p(U), _p(s), _p(V))
    return U, s, V


def lame(E, nu):
    mu, la = ctypes.c_double(), ctypes.c_double()
    lib().orc_lame(E, nu, ctypes.byref(mu), ctypes.byref(la))
    return mu.value, la.value


def wave_speed(mat: Material) -> float:
    return lib().orc_wave_speed(ctypes.byref(mat))


def cfl_dt(cfg: Config, mats, v_bound: float, cfl: float, dt_max: float) -> float:
    ma = _mats(mats)
    return lib().orc_cfl_dt(ctypes.byref(cfg), ma, len(ma), float(v_bound), float(cfl), float(dt_max))


def kirchhoff(mat: Material, F, Jp=1.0) -> np.ndarray:
    F = _f64(F, (3, 3))
    tau = np.zeros((3, 3))
    lib().orc_kirchhoff(ctypes.byref(mat), _p(F), float(Jp), _p(tau))
    return tau


def plasticity(mat: Material, F, Jp=1.0):
    F = _f64(F, (3, 3)).copy()
    j = ctypes.c_double(Jp)
    lib().orc_plasticity(ctypes.byref(mat), _p(F), ctypes.byref(j))
    return F, j.value


class DenseGrid:
    """Dense box of nodes: m[k, j, i], p[k, j, i, 3] for global node lo + (i, j, k)."""

    def __init__(self, lo, dim):
        self.lo = np.array(lo, dtype=np.int32)
        self.dim = np.array(dim, dtype=np.int32)
        self.m = np.zeros(int(np.prod(dim)))
        self.p = np.zeros(3 * int(np.prod(dim)))
        self.v0 = np.zeros(3 * int(np.prod(dim)))   # grid velocity before forces (ASFLIP)

    def cstruct(self) -> Grid:
        return Grid((ctypes.c_int32 * 3)(*self.lo), (ctypes.c_int32 * 3)(*self.dim),
                    self.m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    self.p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    self.v0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    def mass(self):
        d = self.dim
        return self.m.reshape(d[2], d[1], d[0])

    def mom(self):
        d = self.dim
        return self.p.reshape(d[2], d[1], d[0], 3)

    def node_positions(self, dx):
        d = self.dim
        k, j, i = np.meshgrid(np.arange(d[2]), np.arange(d[1]), np.arange(d[0]), indexing="ij")
        return np.stack([i + self.lo[0], j + self.lo[1], k + self.lo[2]], axis=-1) * dx


def grid_bounds(x, dx, pad=0):
    x = _f64(x)
    lo = np.zeros(3, dtype=np.int32)
    dim = np.zeros(3, dtype=np.int32)
    lib().orc_grid_bounds(len(x), _p(x), float(dx), _p(lo), _p(dim))
    return lo - pad, dim + 2 * pad


def p2g(cfg: Config, mats, s: State, dt: float, grid: DenseGrid | None = None):
    if grid is None:
        lo, dim = grid_bounds(s.x, cfg.dx)
        grid = DenseGrid(lo, dim)
    ma = _mats(mats)
    g = grid.cstruct()
    st = lib().orc_p2g(ctypes.byref(cfg), ma, s.n, _p(s.x), _p(s.v), _p(s.C), _p(s.F), _p(s.Jp),
                       _p(s.vol), _p(s.mat), float(dt), ctypes.byref(g))
    return grid, st


def grid_update(cfg: Config, dt: float, grid: DenseGrid):
    g = grid.cstruct()
    lib().orc_grid_update(ctypes.byref(cfg), float(dt), ctypes.byref(g))
    return grid


def g2p(cfg: Config, mats, s: State, dt: float, grid: DenseGrid):
    ma = _mats(mats)
    g = grid.cstruct()
    return lib().orc_g2p(ctypes.byref(cfg), ma, s.n, _p(s.x), _p(s.v), _p(s.C), _p(s.F), _p(s.Jp),
                         _p(s.mat), float(dt), ctypes.byref(g))


def substep(cfg: Config, mats, s: State, dt: float) -> int:
    """Advance s in place by one substep; returns the oracle status (0 = ok)."""
    ma = _mats(mats)
    return lib().orc_substep(ctypes.byref(cfg), ma, s.n, _p(s.x), _p(s.v), _p(s.C), _p(s.F),
                             _p(s.Jp), _p(s.vol), _p(s.mat), float(dt))


def p2g_node(cfg: Config, mats, s: State, dt: float, node) -> np.ndarray:
    ma = _mats(mats)
    nd = np.ascontiguousarray(node, dtype=np.int32)
    out = np.zeros(4)
    lib().orc_p2g_node(ctypes.byref(cfg), ma, s.n, _p(s.x), _p(s.v), _p(s.C), _p(s.F), _p(s.Jp),
                       _p(s.vol), _p(s.mat), float(dt), _p(nd), _p(out))
    return out


def particle_keys(x_f32, inv_dx: float, L: int):
    x = np.ascontiguousarray(x_f32, dtype=np.float32).reshape(-1, 3)
    keys = np.zeros(len(x), dtype=np.uint32)
    st = lib().orc_particle_keys(len(x), _p(x), float(inv_dx), int(L), _p(keys))
    return keys, st


def stable_sort(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    perm = np.zeros(len(keys), dtype=np.int32)
    lib().orc_stable_sort(len(keys), _p(keys), _p(perm))
    return perm


def pblocks(keys, L: int):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    n = lib().orc_pblocks(len(keys), _p(keys), int(L), None)
    out = np.zeros(max(n, 1), dtype=np.int32)
    lib().orc_pblocks(len(keys), _p(keys), int(L), _p(out))
    return out[:n]


def pack_state(x, v, C, F):
    """(n, 24) FP64 state rows x, v, C, F."""
    n = len(x)
    return np.ascontiguousarray(np.concatenate([np.reshape(x, (n, 3)), np.reshape(v, (n, 3)), np.reshape(C, (n, 9)),
                                                np.reshape(F, (n, 9))], axis=1), dtype=np.float64)


def diff_forward(cfg: Config, nu, rho, vol, E, dt, s_in):
    s_in = _f64(s_in)
    n = len(s_in)
    vol = _f64(np.broadcast_to(vol, (n,)))
    E = _f64(E)
    out = np.zeros_like(s_in)
    st = lib().orc_diff_forward(ctypes.byref(cfg), float(nu), float(rho), n, _p(vol), _p(E), float(dt), _p(s_in),
                                _p(out))
    return out, st


def diff_adjoint(cfg: Config, nu, rho, vol, E, dt, s_in, g_out):
    s_in = _f64(s_in)
    n = len(s_in)
    vol = _f64(np.broadcast_to(vol, (n,)))
    E = _f64(E)
    g_out = _f64(g_out)
    g_in = np.zeros_like(s_in)
    gE = np.zeros(n)
    st = lib().orc_diff_adjoint(ctypes.byref(cfg), float(nu), float(rho), n, _p(vol), _p(E), float(dt), _p(s_in),
                                _p(g_out), _p(g_in), _p(gE))
    return g_in, gE, st
