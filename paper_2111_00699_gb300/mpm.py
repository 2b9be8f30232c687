"""Python binding of libmpm with the same names as the C ABI.

PyTorch provides device memory (its caching allocator, handed to the library
as an mpm_allocator) and the CUDA stream; every step of the substep runs in
the library's kernels.  Tensors passed in may live on the GPU (used in place)
or on the host (copied by the library); numpy arrays are host buffers.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import MpmError, load, material  # noqa: F401

ELASTIC, FLUID, SNOW, SAND, NACC, NHSAND = _lib.ELASTIC, _lib.FLUID, _lib.SNOW, _lib.SAND, _lib.NACC, _lib.NHSAND
STICKY, SLIP = _lib.STICKY, _lib.SLIP
APIC, ASFLIP = _lib.APIC, _lib.ASFLIP


def _check(st: int, ctx=None):
    if st != _lib.MPM_OK:
        msg = ""
        if ctx:
            raw = load().mpm_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise MpmError(st, msg)


def _buf(a, dtype, shape=None):
    """(pointer, on_device, keepalive) for a tensor or array argument."""
    if a is None:
        return None, 0, None
    if isinstance(a, torch.Tensor):
        t = a.detach().to(dtype).contiguous()
        if shape is not None:
            t = t.reshape(shape)
        return ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, t
    np_dtype = {torch.float32: np.float32, torch.int32: np.int32, torch.uint32: np.uint32}[dtype]
    arr = np.ascontiguousarray(a, dtype=np_dtype)
    if shape is not None:
        arr = arr.reshape(shape)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


class Simulator:
    """One MLS-MPM scene on one GPU (mpm_create ... mpm_destroy)."""

    def __init__(self, res, dx, materials, boundary=STICKY, wall=3, gravity=(0.0, -9.8, 0.0),
                 max_particles=0, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True,
                 device=None, p2g_variant: int = 3, g2p_variant: int = 0, g2p2g: bool = False,
                 no_sort: bool = False, graphs: bool = False, resort_interval: int = 0, transfer: int = 0,
                 flip_alpha: float = 0.0, flip_beta_min: float = 0.0, flip_beta_max: float = 0.0,
                 flip_compress_margin: float = 0.0):
        lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if isinstance(materials, _lib.Material):
            materials = [materials]
        self.materials = list(materials)
        res = [int(r) for r in (res if hasattr(res, "__len__") else (res,) * 3)]
        self.res = res
        self.dx = float(dx)
        cfg = _lib.Config()
        cfg.res = (ctypes.c_int32 * 3)(*res)
        cfg.dx = self.dx
        cfg.boundary = int(boundary)
        cfg.wall = int(wall)
        cfg.gravity = (ctypes.c_float * 3)(*gravity)
        cfg.max_particles = int(max_particles)
        cfg.use_g2p2g = 1 if g2p2g else 0
        cfg.p2g_variant = int(p2g_variant)
        cfg.g2p_variant = int(g2p_variant)
        cfg.no_sort = 1 if no_sort else 0
        cfg.resort_interval = int(resort_interval)
        cfg.transfer = int(transfer)
        cfg.flip_alpha = float(flip_alpha)
        cfg.flip_beta_min = float(flip_beta_min)
        cfg.flip_beta_max = float(flip_beta_max)
        cfg.flip_compress_margin = float(flip_compress_margin)
        mats = (_lib.Material * len(self.materials))(*self.materials)
        self._alloc = None
        if torch_allocator:
            dev = self.device.index

            def _a(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
                except Exception:  # an exception may not cross the C boundary
                    return None

            def _f(ptr, nbytes, stream, user):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            self._alloc_fns = (_lib.ALLOC_FN(_a), _lib.FREE_FN(_f))
            self._alloc = _lib.Allocator(self._alloc_fns[0], self._alloc_fns[1], None)
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = lib.mpm_create(ctypes.byref(cfg), mats, len(self.materials),
                                ctypes.byref(self._alloc) if self._alloc is not None else None,
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._ctx))
        _check(st)
        if graphs:
            self.use_graphs(True)

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            load().mpm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the C calls -------------------------------------------------------
    @property
    def n(self) -> int:
        return int(load().mpm_num_particles(self._ctx))

    def add_particles(self, x, v=None, vol=None, material: int = 0):
        n = len(x)
        px, dx_, kx = _buf(x, torch.float32, (n, 3))
        pv, dv, kv = _buf(v, torch.float32, (n, 3))
        pw, dw, kw = _buf(vol, torch.float32, (n,))
        flags = {f for f, p in ((dx_, px), (dv, pv), (dw, pw)) if p is not None}
        if len(flags) != 1:
            raise ValueError("x, v and vol must all be on the same side (host or device)")
        _check(load().mpm_add_particles(self._ctx, n, px, pv, pw, int(material), flags.pop()), self._ctx)

    def emit_particles(self, x, v=None, vol=None, material: int = 0):
        """Asynchronous particle source between substeps (mpm_emit_particles)."""
        n = len(x)
        px, dx_, kx = _buf(x, torch.float32, (n, 3))
        pv, dv, kv = _buf(v, torch.float32, (n, 3))
        pw, dw, kw = _buf(vol, torch.float32, (n,))
        flags = {f for f, p in ((dx_, px), (dv, pv), (dw, pw)) if p is not None}
        if len(flags) != 1:
            raise ValueError("x, v and vol must all be on the same side (host or device)")
        _check(load().mpm_emit_particles(self._ctx, n, px, pv, pw, int(material), flags.pop()), self._ctx)

    def substep(self, dt: float):
        _check(load().mpm_substep(self._ctx, float(dt)), self._ctx)

    def run(self, steps: int, dt: float):
        fn = load().mpm_substep
        for _ in range(steps):
            st = fn(self._ctx, float(dt))
            if st:
                _check(st, self._ctx)

    def advance(self, duration: float, cfl: float = 0.5, dt_max: float = 1e-3, max_substeps: int = 1 << 20):
        """Advance by `duration` seconds in adaptive substeps (mpm_advance);
        returns the dt of each substep as a numpy array."""
        dts = np.zeros(int(max_substeps), dtype=np.float32)
        k = ctypes.c_int64(0)
        st = load().mpm_advance(self._ctx, float(duration), float(cfl), float(dt_max), int(max_substeps),
                                dts.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k))
        _check(st, self._ctx)
        return dts[:k.value].copy()

    def sync(self):
        _check(load().mpm_sync(self._ctx), self._ctx)

    def rebuild(self):
        _check(load().mpm_rebuild(self._ctx), self._ctx)

    def read_state(self, fields=("x", "v", "C", "F", "Jp"), device: bool = True) -> dict:
        n = self.n
        shapes = {"x": (n, 3), "v": (n, 3), "C": (n, 3, 3), "F": (n, 3, 3), "Jp": (n,)}
        out = {}
        for f in fields:
            out[f] = torch.empty(shapes[f], dtype=torch.float32, device=self.device if device else "cpu",
                                 pin_memory=False)
        self.read_state_into(**out)
        return out

    def read_state_into(self, x=None, v=None, C=None, F=None, Jp=None):
        ptrs = []
        side = set()
        for t in (x, v, C, F, Jp):
            if t is None:
                ptrs.append(None)
                continue
            assert t.is_contiguous() and t.dtype == torch.float32
            ptrs.append(ctypes.c_void_p(t.data_ptr()))
            side.add(1 if t.is_cuda else 0)
        if len(side) > 1:
            raise ValueError("outputs must all be on the host or all on the device")
        _check(load().mpm_read_state(self._ctx, *ptrs, side.pop() if side else 1), self._ctx)

    def write_state(self, x=None, v=None, C=None, F=None, Jp=None):
        n = self.n
        bufs = [_buf(a, torch.float32, s) for a, s in ((x, (n, 3)), (v, (n, 3)), (C, (n, 9)), (F, (n, 9)), (Jp, (n,)))]
        side = {b[1] for b in bufs if b[0] is not None}
        if len(side) > 1:
            raise ValueError("inputs must all be on the host or all on the device")
        _check(load().mpm_write_state(self._ctx, *[b[0] for b in bufs], side.pop() if side else 1), self._ctx)

    def stats(self) -> dict:
        s = _lib.Stats()
        _check(load().mpm_get_stats(self._ctx, ctypes.byref(s)), self._ctx)
        return {k: int(getattr(s, k)) for k, _ in _lib.Stats._fields_}

    def read_order(self):
        n = self.n
        keys = np.zeros(n, dtype=np.uint32)
        ids = np.zeros(n, dtype=np.int32)
        _check(load().mpm_read_order(self._ctx, keys.ctypes.data_as(ctypes.c_void_p),
                                     ids.ctypes.data_as(ctypes.c_void_p), 0), self._ctx)
        return keys, ids

    def read_blocks(self):
        cnt = ctypes.c_int64()
        _check(load().mpm_read_blocks(self._ctx, None, 0, ctypes.byref(cnt)), self._ctx)
        out = np.zeros(max(cnt.value, 1), dtype=np.int32)
        _check(load().mpm_read_blocks(self._ctx, out.ctypes.data_as(ctypes.c_void_p), cnt.value,
                                      ctypes.byref(cnt)), self._ctx)
        return out[:cnt.value]

    def debug_p2g(self, dt: float) -> torch.Tensor:
        """P2G of the current state into a dense (res2, res1, res0, 4) grid of (m, p)."""
        r = self.res
        g = torch.empty((r[2], r[1], r[0], 4), dtype=torch.float32, device=self.device)
        _check(load().mpm_debug_p2g(self._ctx, float(dt), ctypes.c_void_p(g.data_ptr()), 1), self._ctx)
        return g

    def set_p2g_variant(self, variant: int):
        _check(load().mpm_set_p2g_variant(self._ctx, int(variant)), self._ctx)

    def set_cta_warps(self, warps: int):
        """Warps per CTA (2, 4 or 8) of the register-run P2G and the 64-register G2P."""
        _check(load().mpm_set_cta_warps(self._ctx, int(warps)), self._ctx)

    def set_resort_interval(self, interval: int):
        """Window re-sort every `interval` substeps between rebuilds (0: off)."""
        _check(load().mpm_set_resort_interval(self._ctx, int(interval)), self._ctx)

    def set_layout(self, aosoa: bool):
        """Particle store layout: False SoA (default), True AoSoA in packets of 32."""
        _check(load().mpm_set_layout(self._ctx, 1 if aosoa else 0), self._ctx)

    def set_g2p2g(self, on: bool):
        _check(load().mpm_set_g2p2g(self._ctx, 1 if on else 0), self._ctx)

    def use_graphs(self, on: bool = True):
        """Replay the separate substep from CUDA graphs (needs a non-default stream)."""
        _check(load().mpm_use_graphs(self._ctx, 1 if on else 0), self._ctx)

    @property
    def graph_launches(self) -> int:
        return int(load().mpm_graph_launches(self._ctx))

    def set_g2p_variant(self, variant: int):
        _check(load().mpm_set_g2p_variant(self._ctx, int(variant)), self._ctx)

    def profile_enable(self, on: bool = True):
        _check(load().mpm_profile_enable(self._ctx, 1 if on else 0), self._ctx)

    def profile_read(self):
        ms = (ctypes.c_double * _lib.PHASES)()
        la = (ctypes.c_int64 * _lib.PHASES)()
        _check(load().mpm_profile_read(self._ctx, ms, la, _lib.PHASES), self._ctx)
        names = ("rebuild", "p2g", "grid", "g2p")
        return {names[i]: (float(ms[i]), int(la[i])) for i in range(_lib.PHASES)}


class BatchSimulator:
    """Many small independent scenes advanced together (mpm_batch_*)."""

    def __init__(self, scenes, materials, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True,
                 graphs: bool = True, p2g_chunk: int = 4):
        lib = load()
        # graph capture needs a stream other than the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.materials = [materials] if isinstance(materials, _lib.Material) else list(materials)
        descs = (_lib.SceneDesc * len(scenes))()
        for d, sc in zip(descs, scenes):
            res = sc["res"] if hasattr(sc["res"], "__len__") else (sc["res"],) * 3
            d.res = (ctypes.c_int32 * 3)(*[int(r) for r in res])
            d.dx = float(sc.get("dx", 1.0 / res[0]))
            d.boundary = int(sc.get("boundary", SLIP))
            d.wall = int(sc.get("wall", 3))
            d.gravity = (ctypes.c_float * 3)(*sc.get("gravity", (0.0, -9.8, 0.0)))
            d.material = int(sc.get("material", 0))
        self.n_scenes = len(scenes)
        mats = (_lib.Material * len(self.materials))(*self.materials)
        self._alloc = None
        if torch_allocator:
            dev = torch.cuda.current_device()

            def _a(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
                except Exception:
                    return None

            def _f(ptr, nbytes, stream, user):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            self._alloc_fns = (_lib.ALLOC_FN(_a), _lib.FREE_FN(_f))
            self._alloc = _lib.Allocator(self._alloc_fns[0], self._alloc_fns[1], None)
        self._b = ctypes.c_void_p()
        _check(lib.mpm_batch_create(self.n_scenes, descs, mats, len(self.materials),
                                    ctypes.byref(self._alloc) if self._alloc is not None else None,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._b)))
        self.use_graphs(graphs)
        self.set_p2g_chunk(p2g_chunk)

    def _err(self, st):
        if st:
            raw = load().mpm_batch_last_error(self._b)
            raise MpmError(st, raw.decode() if raw else "")

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            load().mpm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_particles(self, scene: int, x, v=None, vol=None):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
        n = len(x)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float32).reshape(n, 3)
        vol = None if vol is None else np.ascontiguousarray(vol, dtype=np.float32).reshape(n)
        P = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        self._err(load().mpm_batch_add_particles(self._b, int(scene), n, P(x), P(v), P(vol)))

    def substep(self, dt):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float32), (self.n_scenes,)))
        self._dt_keep = d
        self._err(load().mpm_batch_substep(self._b, d.ctypes.data_as(ctypes.c_void_p)))

    def run(self, steps: int, dt):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float32), (self.n_scenes,)))
        ptr = d.ctypes.data_as(ctypes.c_void_p)
        fn = load().mpm_batch_substep
        for _ in range(steps):
            st = fn(self._b, ptr)
            if st:
                self._err(st)

    def use_graphs(self, on: bool = True):
        self._err(load().mpm_batch_use_graphs(self._b, 1 if on else 0))

    def set_p2g_chunk(self, k: int):
        self._err(load().mpm_batch_set_p2g_chunk(self._b, int(k)))

    def set_cta_warps(self, warps: int):
        """Warps per CTA (2, 4 or 8) of the per-phase P2G and G2P launches."""
        self._err(load().mpm_batch_set_cta_warps(self._b, int(warps)))

    def set_persistent(self, on: bool = True):
        """One cooperative launch per substep (grid barriers between the phases)."""
        self._err(load().mpm_batch_set_persistent(self._b, 1 if on else 0))

    def sync(self):
        self._err(load().mpm_batch_sync(self._b))

    def n_particles(self, scene: int = -1) -> int:
        return int(load().mpm_batch_num_particles(self._b, int(scene)))

    def read_state(self, scene: int) -> dict:
        n = self.n_particles(scene)
        out = {"x": np.zeros((n, 3), np.float32), "v": np.zeros((n, 3), np.float32),
               "C": np.zeros((n, 3, 3), np.float32), "F": np.zeros((n, 3, 3), np.float32),
               "Jp": np.zeros(n, np.float32)}
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self._err(load().mpm_batch_read_state(self._b, int(scene), P(out["x"]), P(out["v"]), P(out["C"]),
                                              P(out["F"]), P(out["Jp"])))
        return out

    def stats(self) -> dict:
        a = (ctypes.c_int64 * 4)()
        self._err(load().mpm_batch_get_stats(self._b, a))
        return {"substeps": a[0], "remaps": a[1], "kernel_launches": a[2], "graph_launches": a[3]}


# ---- stand-alone kernels ----------------------------------------------------

def radix_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, stream=None):
    """Stable sort of (key, value) pairs on the GPU; returns new tensors."""
    lib = load()
    assert keys.is_cuda and vals.is_cuda and keys.numel() == vals.numel()
    n = keys.numel()
    kin = keys.contiguous().view(torch.int32)
    vin = vals.to(torch.int32).contiguous()
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    nbytes = ctypes.c_size_t()
    _check(lib.mpm_radix_sort_pairs(None, None, None, None, n, key_bits, None, ctypes.byref(nbytes), None))
    scratch = torch.empty(max(int(nbytes.value), 1), dtype=torch.uint8, device=keys.device)
    s = stream if stream is not None else torch.cuda.current_stream(keys.device)
    _check(lib.mpm_radix_sort_pairs(ctypes.c_void_p(kin.data_ptr()), ctypes.c_void_p(vin.data_ptr()),
                                    ctypes.c_void_p(kout.data_ptr()), ctypes.c_void_p(vout.data_ptr()), n, key_bits,
                                    ctypes.c_void_p(scratch.data_ptr()), ctypes.byref(nbytes),
                                    ctypes.c_void_p(s.cuda_stream)))
    return kout.view(keys.dtype), vout


def debug_svd(F: torch.Tensor):
    F = F.reshape(-1, 9).contiguous().float()
    n = F.shape[0]
    U = torch.empty((n, 9), device=F.device)
    S = torch.empty((n, 3), device=F.device)
    V = torch.empty((n, 9), device=F.device)
    torch.cuda.synchronize(F.device)
    _check(load().mpm_debug_svd(ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(V.data_ptr()), n))
    return U.reshape(n, 3, 3), S, V.reshape(n, 3, 3)


def debug_stress(mat, F: torch.Tensor, Jp: torch.Tensor | None = None):
    F = F.reshape(-1, 9).contiguous().float()
    n = F.shape[0]
    tau = torch.empty((n, 9), device=F.device)
    jp = None if Jp is None else Jp.contiguous().float()
    torch.cuda.synchronize(F.device)
    _check(load().mpm_debug_stress(ctypes.byref(mat), ctypes.c_void_p(F.data_ptr()),
                                   None if jp is None else ctypes.c_void_p(jp.data_ptr()),
                                   ctypes.c_void_p(tau.data_ptr()), n))
    return tau.reshape(n, 3, 3)


def debug_plasticity(mat, F: torch.Tensor, Jp: torch.Tensor):
    F = F.reshape(-1, 9).contiguous().float().clone()
    Jp = Jp.contiguous().float().clone()
    torch.cuda.synchronize(F.device)
    _check(load().mpm_debug_plasticity(ctypes.byref(mat), ctypes.c_void_p(F.data_ptr()),
                                       ctypes.c_void_p(Jp.data_ptr()), F.shape[0]))
    return F.reshape(-1, 3, 3), Jp


def debug_wait_timeout(max_iter: int = 1000) -> int:
    """Run the bounded-wait check (mpm_debug_wait_timeout); returns the status
    (MPM_ETIMEOUT when the wait gave up, as it should)."""
    return int(load().mpm_debug_wait_timeout(int(max_iter)))


def radix_sort_pairs_noalloc(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32,
                             out: tuple | None = None, stream=None):
    """Stable sort of (key, value) pairs with the library's fixed scratch array
    (mpm_radix_sort_pairs_noalloc): no device memory is allocated by the call.
    Pass preallocated output tensors in `out` to allocate nothing at all."""
    lib = load()
    assert keys.is_cuda and vals.is_cuda and keys.numel() == vals.numel()
    n = keys.numel()
    kin = keys.contiguous().view(torch.int32)
    vin = vals.contiguous()
    assert vin.dtype == torch.int32
    kout, vout = out if out is not None else (torch.empty_like(kin), torch.empty_like(vin))
    s = stream if stream is not None else torch.cuda.current_stream(keys.device)
    _check(lib.mpm_radix_sort_pairs_noalloc(ctypes.c_void_p(kin.data_ptr()), ctypes.c_void_p(vin.data_ptr()),
                                            ctypes.c_void_p(kout.data_ptr()), ctypes.c_void_p(vout.data_ptr()),
                                            n, key_bits, ctypes.c_void_p(s.cuda_stream)))
    return kout.view(keys.dtype), vout


def debug_red_rate(grid: torch.Tensor, threads: int, reds_per_thread: int, pattern: int = 0,
                   stream: torch.cuda.Stream | None = None) -> None:
    """Launch the L2 float4-reduction rate probe (mpm_debug_red_rate) on
    `grid`, a float32 CUDA tensor of shape (nodes, 4); asynchronous on
    `stream` (default: the current stream)."""
    if grid.dtype != torch.float32 or not grid.is_cuda or grid.dim() != 2 or grid.shape[1] != 4 \
            or not grid.is_contiguous():
        raise ValueError("grid must be a contiguous float32 CUDA tensor of shape (nodes, 4)")
    s = stream if stream is not None else torch.cuda.current_stream(grid.device)
    _check(load().mpm_debug_red_rate(ctypes.c_void_p(grid.data_ptr()), int(grid.shape[0]), int(threads),
                                     int(reds_per_thread), int(pattern), ctypes.c_void_p(s.cuda_stream)), None)
