"""Autotuner for the launch-shape knobs of the substep.

Times each P2G scatter variant (direct float4 atomics, cell-strided lanes,
shared-memory node tile) on the caller's own scene with CUDA events on the
simulator's stream, and leaves the fastest one selected.  The simulation
advances while it is tuned (every variant computes the same substep).
"""
from __future__ import annotations

from . import _lib


def tune_p2g(sim, dt: float, steps: int = 50, rounds: int = 2) -> dict:
    """Return {"best": variant, "ms": {name: ms per P2G launch}}; sim keeps `best`."""
    ms = {name: [] for name in _lib.P2G_VARIANTS}
    sim.profile_enable(True)
    sim.profile_read()
    for _ in range(rounds):
        for v, name in enumerate(_lib.P2G_VARIANTS):
            sim.set_p2g_variant(v)
            sim.run(steps, dt)
            ph = sim.profile_read()
            t, k = ph["p2g"]
            if k:
                ms[name].append(t / k)
    sim.profile_enable(False)
    avg = {name: (min(v) if v else float("inf")) for name, v in ms.items()}
    best = min(range(len(_lib.P2G_VARIANTS)), key=lambda v: avg[_lib.P2G_VARIANTS[v]])
    sim.set_p2g_variant(best)
    return {"best": best, "best_name": _lib.P2G_VARIANTS[best], "ms": avg}
