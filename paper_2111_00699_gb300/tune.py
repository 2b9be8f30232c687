"""Autotuner for the launch-shape knobs of the substep.

Times each P2G scatter variant (direct float4 atomics, cell-strided lanes,
shared-memory node tile, register accumulation over runs of 4 or 8
particles) and each G2P gather variant (per particle, node velocities
cached over runs of 4 or 8) on the caller's own scene, with CUDA events on
the simulator's stream, and leaves the fastest of each selected.  The
simulation advances while it is tuned (every variant computes the same
substep, up to float summation order).
"""
from __future__ import annotations

from . import _lib


def _tune(sim, dt, names, setter, phase, steps, rounds):
    ms = {name: [] for name in names}
    sim.profile_enable(True)
    sim.profile_read()
    for _ in range(rounds):
        for v, name in enumerate(names):
            setter(v)
            sim.run(steps, dt)
            t, k = sim.profile_read()[phase]
            if k:
                ms[name].append(t / k)
    sim.profile_enable(False)
    avg = {name: (min(v) if v else float("inf")) for name, v in ms.items()}
    best = min(range(len(names)), key=lambda v: avg[names[v]])
    setter(best)
    return {"best": best, "best_name": names[best], "ms": avg}


def tune_p2g(sim, dt: float, steps: int = 50, rounds: int = 2) -> dict:
    """Return {"best": variant, "best_name", "ms": {name: ms per P2G launch}}; sim keeps `best`."""
    return _tune(sim, dt, _lib.P2G_VARIANTS, sim.set_p2g_variant, "p2g", steps, rounds)


def tune_g2p(sim, dt: float, steps: int = 50, rounds: int = 2) -> dict:
    """Same for the G2P gather variants."""
    return _tune(sim, dt, _lib.G2P_VARIANTS, sim.set_g2p_variant, "g2p", steps, rounds)
