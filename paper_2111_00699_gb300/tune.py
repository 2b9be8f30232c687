"""Autotuner for the launch-shape knobs of the substep.

Times each P2G scatter variant (direct float4 atomics, cell-strided lanes,
shared-memory node tile, register accumulation over runs of 4 or 8
particles) and each G2P gather variant (per particle, node velocities
cached over runs of 4 or 8) on the caller's own scene, with CUDA events on
the simulator's stream, and leaves the fastest of each selected.  The
simulation advances while it is tuned (every variant computes the same
substep, up to float summation order).

Variants whose times lie within a few per cent can rank differently once
the particle order has drifted from the last sort; ``refine_top`` re-times
the best few after ``drift`` further substeps, with longer runs, and keeps
the fastest of those.
"""
from __future__ import annotations

from . import _lib


def _time(sim, dt, names, setter, phase, steps, rounds, candidates):
    ms = {names[v]: [] for v in candidates}
    sim.profile_enable(True)
    sim.profile_read()
    for _ in range(rounds):
        for v in candidates:
            setter(v)
            sim.run(steps, dt)
            t, k = sim.profile_read()[phase]
            if k:
                ms[names[v]].append(t / k)
    sim.profile_enable(False)
    return {name: (min(v) if v else float("inf")) for name, v in ms.items()}


def _tune(sim, dt, names, setter, phase, steps, rounds, refine_top=0, refine_steps=100, drift=0):
    avg = _time(sim, dt, names, setter, phase, steps, rounds, range(len(names)))
    best = min(range(len(names)), key=lambda v: avg[names[v]])
    out = {"ms": avg}
    if refine_top > 1:
        top = sorted(range(len(names)), key=lambda v: avg[names[v]])[:refine_top]
        setter(best)
        sim.run(drift, dt)
        refined = _time(sim, dt, names, setter, phase, refine_steps, rounds, top)
        best = min(top, key=lambda v: refined[names[v]])
        out["refined_ms"] = refined
    setter(best)
    out.update({"best": best, "best_name": names[best]})
    return out


def tune_p2g(sim, dt: float, steps: int = 50, rounds: int = 2, refine_top: int = 0, refine_steps: int = 100,
             drift: int = 0) -> dict:
    """Return {"best": variant, "best_name", "ms": {name: ms per P2G launch}, and with refine_top > 1
    "refined_ms" for the re-timed candidates}; sim keeps `best`."""
    return _tune(sim, dt, _lib.P2G_VARIANTS, sim.set_p2g_variant, "p2g", steps, rounds, refine_top, refine_steps, drift)


def tune_g2p(sim, dt: float, steps: int = 50, rounds: int = 2) -> dict:
    """Same for the G2P gather variants."""
    return _tune(sim, dt, _lib.G2P_VARIANTS, sim.set_g2p_variant, "g2p", steps, rounds)


def tune_cta_warps(sim, dt: float, steps: int = 50, rounds: int = 2) -> dict:
    """Time P2G + G2P per substep in CTAs of 2, 4 and 8 warps (the register-run
    P2G and the 64-register G2P take the setting) and keep the fastest.
    Returns {"best": warps, "ms": {warps: ms of P2G + G2P per substep}}."""
    ms = {w: float("inf") for w in (2, 4, 8)}
    sim.profile_enable(True)
    for _ in range(rounds):
        for w in ms:
            sim.set_cta_warps(w)
            sim.run(2, dt)
            sim.profile_read()
            sim.run(steps, dt)
            ph = sim.profile_read()
            t = sum(ph[k][0] for k in ("p2g", "g2p")) / max(1, ph["p2g"][1])
            ms[w] = min(ms[w], t)
    sim.profile_enable(False)
    best = min(ms, key=ms.get)
    sim.set_cta_warps(best)
    return {"best": best, "ms": ms}


def _p2g_g2p_ms(sim, dt, steps):
    sim.run(2, dt)
    sim.profile_read()
    sim.run(steps, dt)
    ph = sim.profile_read()
    return sum(ph[k][0] for k in ("p2g", "g2p")) / max(1, ph["p2g"][1])


def tune_layout(sim, dt: float, warps: int, steps: int = 50, rounds: int = 2) -> dict:
    """SoA (at `warps` warps per CTA) against the AoSoA store at 2 and at 4
    warps per CTA (the warp counts it runs), timing P2G + G2P per substep;
    keeps the fastest.  Needs the register-run P2G (variant 3, 4, 14 or 15) and the
    64-register G2P (4 or 7) already selected; otherwise the store stays SoA.
    Returns {"best": "soa" | "aosoa", "ms": {...}, "cta_warps": the warps kept}."""
    ms = {"soa": float("inf"), "aosoa_2": float("inf"), "aosoa_4": float("inf")}
    sim.profile_enable(True)
    try:
        for _ in range(rounds):
            sim.set_layout(False)
            sim.set_cta_warps(warps)
            ms["soa"] = min(ms["soa"], _p2g_g2p_ms(sim, dt, steps))
            for w in (2, 4):
                sim.set_cta_warps(w)
                sim.set_layout(True)
                ms["aosoa_%d" % w] = min(ms["aosoa_%d" % w], _p2g_g2p_ms(sim, dt, steps))
                sim.set_layout(False)
    except Exception as exc:   # the selected variants have no AoSoA form
        sim.profile_enable(False)
        sim.set_layout(False)
        sim.set_cta_warps(warps)
        return {"best": "soa", "ms": ms, "cta_warps": warps, "skipped": str(exc)}
    sim.profile_enable(False)
    best = min(ms, key=ms.get)
    if best == "soa":
        sim.set_cta_warps(warps)
        return {"best": "soa", "ms": ms, "cta_warps": warps}
    w = int(best.split("_")[1])
    sim.set_cta_warps(w)
    sim.set_layout(True)
    # the G2P forms of the AoSoA store, re-timed on it (64 registers with the weights in
    # registers or in shared memory, 48 registers): their spills differ from SoA's
    g2p_ms = _time(sim, dt, _lib.G2P_VARIANTS, sim.set_g2p_variant, "g2p", steps, rounds, (4, 6, 7))
    g2p_best = min((4, 6, 7), key=lambda v: g2p_ms[_lib.G2P_VARIANTS[v]])
    sim.set_g2p_variant(g2p_best)
    return {"best": "aosoa", "ms": ms, "cta_warps": w, "aosoa_g2p_ms": g2p_ms,
            "aosoa_g2p": _lib.G2P_VARIANTS[g2p_best], "aosoa_g2p_variant": g2p_best}


def _substep_ms(sim, dt, steps):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sim.sync()
    e0.record(sim.stream)
    sim.run(steps, dt)
    e1.record(sim.stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_order(sim, dt: float, candidates, slice_steps: int = 256, rounds: int = 2) -> dict:
    """Whole-substep time of each (P2G variant, window re-sort interval) pair
    in `candidates`, and keep the fastest.  The re-sort restores P2G's runs of
    equal cells between rebuilds at a cost of its own, and the variants differ
    in how they suffer from the drift it undoes, so the pair is timed on whole
    substeps over slices longer than the intervals.  The slices run in the
    order A B C ... then ... C B A, so that every pair's slices sit at the same
    mean time of the run and the scene's evolution favours none.
    Returns {"best": (variant, interval), "best_name", "ms": {name: ms per substep}}."""
    def name(c):
        return "%s, re-sort every %d" % (_lib.P2G_VARIANTS[c[0]], c[1]) if c[1] else \
            "%s, no re-sort" % _lib.P2G_VARIANTS[c[0]]
    cands = list(dict.fromkeys(candidates))
    seq = []
    for r in range(rounds):
        seq += cands if r % 2 == 0 else cands[::-1]
    ms = {c: [] for c in cands}
    for c in seq:
        sim.set_p2g_variant(c[0])
        sim.set_resort_interval(c[1])
        ms[c].append(_substep_ms(sim, dt, slice_steps))
    avg = {c: sum(v) / len(v) for c, v in ms.items()}
    best = min(cands, key=avg.get)
    sim.set_p2g_variant(best[0])
    sim.set_resort_interval(best[1])
    return {"best": best, "best_name": name(best), "ms": {name(c): avg[c] for c in cands}}
