"""Differentiable rollouts of the elastic MLS-MPM substep.

`DiffSim` wraps the C ABI's mpm_diff_* calls (forward and hand-written
adjoint of one substep, device memory from PyTorch).  A state row is x, v, C
and H = F - I (the displacement gradient), 24 floats.  `rollout` is a
torch.autograd.Function: its forward runs `steps` substeps keeping a
checkpoint of the particle state every `k` substeps; its backward walks the
segments in reverse, recomputes each segment's states from its checkpoint,
and chains the per-substep adjoints.  Gradients flow to the initial
positions, the initial velocities and the per-particle Young's moduli.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .mpm import _check, load


class DiffSim:
    def __init__(self, res, dx, n, nu=0.2, rho=1.0, boundary=_lib.STICKY, wall=3, gravity=(0.0, -9.8, 0.0),
                 vol=None, stream: torch.cuda.Stream | None = None):
        lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        res = [int(r) for r in (res if hasattr(res, "__len__") else (res,) * 3)]
        cfg = _lib.Config()
        cfg.res = (ctypes.c_int32 * 3)(*res)
        cfg.dx = float(dx)
        cfg.boundary = int(boundary)
        cfg.wall = int(wall)
        cfg.gravity = (ctypes.c_float * 3)(*gravity)
        self.n = int(n)
        self._vol = None if vol is None else torch.as_tensor(vol, dtype=torch.float32, device="cuda").contiguous()
        self._d = ctypes.c_void_p()
        _check(lib.mpm_diff_create(ctypes.byref(cfg), float(nu), float(rho), self.n,
                                   None if self._vol is None else ctypes.c_void_p(self._vol.data_ptr()), None,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._d)))

    def close(self):
        if getattr(self, "_d", None) and self._d.value:
            load().mpm_diff_destroy(self._d)
            self._d = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, dt: float, E: torch.Tensor, s: torch.Tensor) -> torch.Tensor:
        out = torch.empty_like(s)
        _check(load().mpm_diff_forward(self._d, float(dt), ctypes.c_void_p(E.data_ptr()),
                                       ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    def adjoint(self, dt: float, E: torch.Tensor, s: torch.Tensor, g_out: torch.Tensor, gE: torch.Tensor):
        g_in = torch.empty_like(s)
        _check(load().mpm_diff_adjoint(self._d, float(dt), ctypes.c_void_p(E.data_ptr()),
                                       ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(g_out.data_ptr()),
                                       ctypes.c_void_p(g_in.data_ptr()), ctypes.c_void_p(gE.data_ptr())))
        return g_in

    def sync(self):
        _check(load().mpm_diff_sync(self._d))


def pack_state(x: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """(n, 24) state x, v, C = 0, H = F - I = 0 (rest shape)."""
    n = x.shape[0]
    s = torch.zeros((n, 24), dtype=torch.float32, device=x.device)
    s[:, 0:3] = x
    s[:, 3:6] = v
    return s


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, E, sim, steps, k, dt):
        E = E.detach().contiguous().float()
        s = pack_state(x0.detach().float(), v0.detach().float())
        ckpts = [s]
        with torch.cuda.stream(sim.stream):
            for t in range(steps):
                s = sim.forward(dt, E, s)
                if (t + 1) % k == 0 and t + 1 < steps:
                    ckpts.append(s)
        ctx.sim, ctx.steps, ctx.k, ctx.dt = sim, steps, k, dt
        ctx.ckpts = ckpts
        ctx.save_for_backward(E)
        return s.clone()

    @staticmethod
    def backward(ctx, g_final):
        (E,) = ctx.saved_tensors
        sim, steps, k, dt = ctx.sim, ctx.steps, ctx.k, ctx.dt
        g = g_final.contiguous().float().clone()
        gE = torch.zeros_like(E)
        n_seg = len(ctx.ckpts)
        with torch.cuda.stream(sim.stream):
            for seg in range(n_seg - 1, -1, -1):
                start = seg * k
                length = min(k, steps - start)
                states = [ctx.ckpts[seg]]
                for _ in range(length - 1):
                    states.append(sim.forward(dt, E, states[-1]))
                for t in range(length - 1, -1, -1):
                    g = sim.adjoint(dt, E, states[t], g, gE)
        return g[:, 0:3], g[:, 3:6], gE, None, None, None, None


def rollout(x0: torch.Tensor, v0: torch.Tensor, E: torch.Tensor, sim: DiffSim, steps: int, k: int = 20,
            dt: float = 1e-4) -> torch.Tensor:
    """Final (n, 24) state after `steps` substeps; differentiable in x0, v0, E."""
    return _Rollout.apply(x0, v0, E, sim, steps, k, dt)


def center_of_mass_loss(state: torch.Tensor, vol: torch.Tensor, target) -> torch.Tensor:
    """Squared distance of the mass-weighted mean position to a target point."""
    w = vol / vol.sum()
    com = (state[:, 0:3] * w[:, None]).sum(0)
    t = torch.as_tensor(target, dtype=state.dtype, device=state.device)
    return ((com - t) ** 2).sum()
