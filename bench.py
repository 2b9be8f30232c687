"""Throughput of the MLS-MPM substep on the snow-blocks scene.

Workload (the 1.33M-particle snow scene of the paper's Sec. 6.5, stood in
for by synthetic snow blocks): 6 random boxes at 8 particles per cell,
1,340,960 particles, 256^3 grid of 4^3 blocks, Stomakhin snow (E = 1.4e5,
nu = 0.2, theta_c = 2.5e-2, theta_s = 7.5e-3, hardening 10, rho = 400),
frictionless walls, dt = 5e-5, frames of 1/60 s (333 1/3 substeps).

A "step" is one substep: [rebuild-mapping + sort when the free-zone test
asks for it] -> P2G -> grid update -> G2P.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs its own
replica of the scene (the path has no data exchange: "replicas only"), and
rank 0 reports the aggregate over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLS-MPM particle-substeps/s & ms/frame on 1 GB300; batched vs per-scene launches"
UNIT = "particle-substeps/s"
RES = 256
DX = 1.0 / RES
DT = 5e-5
RESORT_INTERVAL = 64   # window re-sort every 64 substeps (measured: 0.1825 -> 0.1789 ms/substep; 8: 0.193)
FRAME = 1.0 / 60.0
SUBSTEPS_PER_FRAME = FRAME / DT            # 333.33
SNOW = dict(E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0)
VOL = DX ** 3 / 8
# Algorithmic bytes per particle per launch (FP32 SoA, each channel read or written once):
#   P2G reads x 12, v 12, C 36, tau 24, vol 4 (the bench scene has one material: no
#   per-particle material index)                                         = 88 B
#   G2P reads x 12, F 36, Jp 4, material 1; writes x, v, C, F, Jp, tau 124 = 177 B
# grid update per node of a physical block: read 16, write 16, clear 16 = 48 B
BYTES_P2G = 88
BYTES_G2P = 177
BYTES_GRID_NODE = 48
# The same accounting in the layout-free form the measurement plan states per particle-substep
# (FP32, each state channel moved once): P2G reads x, v, C, F, Jp = 100 B; the separate
# substep moves 260 B (P2G 100 + G2P reads x, F, Jp 52 and writes x, v, C, F, Jp 100 + the
# grid's ~8 B per particle at 8 particles per cell); the fused G2P2G moves 112 B (reads and
# writes x, F, Jp 52 B each + ~8 B of grid).
LAYOUT_FREE_BYTES_P2G = 100
LAYOUT_FREE_BYTES_SUBSTEP = 260
LAYOUT_FREE_BYTES_SUBSTEP_FUSED = 112


def workload_config(n, world=1):
    """The `config` of both arms' JSON lines (the same keys and values)."""
    return {"workload": "snow blocks: 6 random boxes, %d particles at 8/cell, 256^3 grid of 4^3 blocks, "
                        "Stomakhin snow, slip walls, dt=5e-5" % n,
            "particles": n, "grid": [RES, RES, RES], "dt": DT, "material": "snow (E=1.4e5, nu=0.2, rho=400)",
            "substeps_per_frame": round(SUBSTEPS_PER_FRAME, 3),
            "l2": "inputs larger than L2: particle state %.0f MB + grid, no flush" % (n * 133 / 1e6),
            "parallelism": "replicas" if world > 1 else "single"}


def host_cores():
    """Host cores this process may run on, and the machine's count."""
    try:
        usable = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        usable = None
    return {"host_cores_usable": usable, "host_cores_total": os.cpu_count()}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ oracle timing

def oracle_throughput(x, seconds=15.0, max_particles=None, steps=None):
    """Time the FP64 oracle, single-threaded, on a compact subset of the scene
    (the particles nearest the first box's centre).  Returns (value, sample)."""
    import oracle as orc
    orc.build()
    n = len(x) if max_particles is None else min(len(x), max_particles)
    if n < len(x):
        lo = x.min(0)
        # nearest-to-a-corner-box subset keeps the oracle's dense box small
        d = np.abs(x - (lo + 0.05)).max(1)
        idx = np.argsort(d, kind="stable")[:n]
        xs = x[idx]
    else:
        xs = x
    s = orc.State(xs.astype(np.float64), vol=VOL)
    cfg = orc.config(RES, DX, orc.SLIP)
    m = orc.material(orc.SNOW, **SNOW)
    t0 = time.perf_counter()
    done = 0
    while True:
        orc.substep(cfg, m, s, DT)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= seconds):
            break
    return n * done / el, "%d oracle substeps (FP64, 1 thread) on %d of the scene's particles, %.1f s" % (done, n, el)


# --------------------------------------------------------------- reference

def max_over_ranks(value, world, device="cuda"):
    """The largest of `value` over all ranks of the process group: replicas
    report the time of the slowest one."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(particles_per_rank, substeps, world, ms):
    """Whole-job particle-substeps/s of `world` replicas that each advanced
    `particles_per_rank` particles `substeps` times in `ms` (max over ranks)."""
    return world * particles_per_rank * substeps / (ms / 1e3)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2111_00699_gb300 import scenes
    x, _ = scenes.snow_blocks()
    total = args.steps + args.warmup
    # size each step so the whole run stays within ~2.5 minutes at ~0.7 M particle-substeps/s
    per_step = int(max(1000, min(len(x), 0.7e6 * 150.0 / max(total, 1))))
    import oracle as orc
    orc.build()
    if args.warmup:
        oracle_throughput(x, max_particles=per_step, steps=args.warmup)
    value, sample = oracle_throughput(x, max_particles=per_step, steps=max(args.steps, 1))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(len(x), world), "impl": "reference",
            "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                                 **host_cores()),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------- secondary workloads

BATCH_MATS = [dict(kind=0, E=1e4, nu=0.2, rho=1000.0), dict(kind=1, E=1e4, gamma=7.0, rho=1000.0),
              dict(kind=2, E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0),
              dict(kind=3, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0)]
BATCH_DT = [1e-4, 1e-4, 5e-5, 1e-4]


def _events_time(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def bench_batched(steps=100, warmup=5):
    """256 independent scenes (log-uniform 2K-64K particles, 32^3-128^3 grids,
    four materials): one batched launch per phase, replayed from CUDA graphs,
    against one Simulator (three launches per substep) per scene."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    bs = scenes.batched_scenes(4)
    total = sum(len(b["x"]) for b in bs)
    mats = [mpm.material(**m) for m in BATCH_MATS]
    dts = np.array([BATCH_DT[b["material"]] for b in bs], np.float32)
    descs = [dict(res=b["res"], dx=1.0 / b["res"], material=b["material"]) for b in bs]
    out = {"workload": "256 scenes, %d particles, grids 32^3-128^3, 4 materials (seed 4)" % total,
           "particles": total, "substeps": steps}
    # autotuned launch shape: per-phase launches (P2G chunk 1/4/8 particles per thread, CTAs of
    # 2/4/8 warps) or the persistent cooperative launch (chunk 1/4/8), all replayed from graphs
    shapes = [(False, k, w) for k in (1, 4, 8) for w in (2, 4, 8)] + [(True, k, 4) for k in (1, 4, 8)]
    name = lambda sh: "%s chunk %d%s" % ("persistent" if sh[0] else "per-phase", sh[1],
                                          "" if sh[0] else ", %d warps" % sh[2])

    def fresh(sh):
        bsim = mpm.BatchSimulator(descs, mats, graphs=True)
        for i, b in enumerate(bs):
            bsim.add_particles(i, b["x"])
        bsim.set_persistent(sh[0])
        bsim.set_p2g_chunk(sh[1])
        bsim.set_cta_warps(sh[2])
        bsim.run(warmup, dts)
        return bsim

    # each shape on a fresh batch, over the same substeps of the scenes' motion (from rest):
    # the cost of a substep changes as the blocks land and deform
    tune = {}
    for sh in shapes:
        with fresh(sh) as bsim:
            tune[sh] = _events_time(bsim.stream, lambda: bsim.run(20, dts)) / 20
    best = min(tune, key=tune.get)
    # the timed run: a fresh batch in the chosen shape, covering the same substeps as the
    # per-scene run below
    with fresh(best) as bsim:
        ms = _events_time(bsim.stream, lambda: bsim.run(steps, dts))
        bsim.sync()
        st = bsim.stats()
    per_phase = min(v for sh, v in tune.items() if not sh[0])
    persistent = min(v for sh, v in tune.items() if sh[0])
    out.update({"value": total * steps / (ms / 1e3), "unit": UNIT, "ms_per_substep": ms / steps,
                "launch_shape": {"persistent": best[0], "p2g_chunk": best[1], "cta_warps": best[2]},
                "shape_ms": {name(sh): v for sh, v in tune.items()},
                "per_phase_best_ms": per_phase, "persistent_best_ms": persistent,
                "persistent_over_per_phase_time": persistent / per_phase,
                "remaps": st["remaps"], "graphs": True})
    best = best[1]
    # per-scene launches of the plain path on the same stream, with the kernels the single
    # scene runs: the register-run P2G of the batched path's chunk length (4 or 8 particles)
    # and the 64-register G2P specialised to each scene's material kind
    per_scene_p2g = 4 if best == 8 else 3
    per_scene_g2p = 4
    out["per_scene_kernels"] = {"p2g_variant": per_scene_p2g, "g2p_variant": per_scene_g2p}
    stream = torch.cuda.Stream()
    sims = []
    for b in bs:
        sim = mpm.Simulator(b["res"], 1.0 / b["res"], [mats[b["material"]]], boundary=mpm.SLIP, stream=stream,
                            p2g_variant=per_scene_p2g, g2p_variant=per_scene_g2p)
        sim.add_particles(b["x"])
        sims.append(sim)

    def per_scene(k):
        for _ in range(k):
            for sim, dt in zip(sims, dts):
                sim.substep(float(dt))

    per_scene(warmup)
    ms2 = _events_time(stream, lambda: per_scene(steps))
    for sim in sims:
        sim.sync()
        sim.close()
    out["per_scene_value"] = total * steps / (ms2 / 1e3)
    out["per_scene_ms_per_substep"] = ms2 / steps
    out["batched_over_per_scene"] = out["value"] / out["per_scene_value"]
    return out


def bench_fountain(substeps=3600, asflip=False):
    """Fountain: weakly compressible fluid (K 1e4, gamma 7) emitted through a
    disk inlet every substep up to the 143K-particle budget, 128^3, dt 1e-4.
    asflip: the ASFLIP transfer the paper's fountain uses (alpha 0.95, beta 0
    compressed / 1 otherwise) instead of APIC."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    res, dt = 128, 1e-4
    vol = (1.0 / res) ** 3 / 8
    batches = [scenes.fountain_batch(2, k, dt, vol) for k in range(substeps)]
    stream = torch.cuda.Stream()
    flip = dict(transfer=mpm.ASFLIP, flip_alpha=0.95, flip_beta_min=0.0, flip_beta_max=1.0) if asflip else {}
    with mpm.Simulator(res, 1.0 / res, [mpm.material(mpm.FLUID, E=1e4, gamma=7.0, rho=1000.0)],
                       boundary=mpm.SLIP, stream=stream, p2g_variant=3, g2p_variant=0, **flip) as sim:
        def run():
            for xe, ve in batches:
                sim.emit_particles(xe, v=ve)
                sim.substep(dt)
        ms = _events_time(stream, run)
        sim.sync()
        n_end = sim.n
        st = sim.stats()
    ps = sum(len(b[0]) * (substeps - k) for k, b in enumerate(batches))
    frame = round((1.0 / 60.0) / dt)
    return {"workload": "fountain%s, %d substeps, %d particles at the end, 128^3, dt=1e-4"
                        % (" (ASFLIP)" if asflip else "", substeps, n_end),
            "value": ps / (ms / 1e3), "unit": UNIT, "ms_per_substep": ms / substeps,
            "ms_per_frame": ms / substeps * frame, "particles_end": n_end, "rebuilds": st["rebuilds"]}


def bench_small_elastic(substeps=100, reps=5):
    """The small elastic case: 8,192 particles uniform in [0.4, 0.6]^3, 64^3,
    fixed-corotated E 1e4, nu 0.2, rho 1, dt 1e-4, sticky walls, 100
    substeps.  The whole state fits in L2, so the figure is microseconds per
    substep (launch and latency bound), for the separate phases and for the
    fused G2P2G transfer (the paper's choice below ~100K particles), with the
    default launch variants and with variants autotuned on this scene (at
    8,192 particles a launch of 8-particle chunks fills 8 of the 152 SMs)."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes, tune
    x = torch.from_numpy(scenes.cube_uniform(0, 8192, 0.4, 0.6)).cuda()
    vol = torch.full((8192,), 0.008 / 8192, device="cuda")
    stream = torch.cuda.Stream()
    mat = mpm.material(mpm.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    out = {"workload": "small elastic, 8192 particles, 64^3, dt=1e-4, 100 substeps", "unit": "us/substep"}

    def timed(p2g, g2p, fused, graphs, warps=4):
        best = None
        for _ in range(reps):
            with mpm.Simulator(64, 1 / 64, [mat], stream=stream, p2g_variant=p2g, g2p_variant=g2p, g2p2g=fused,
                               graphs=graphs) as sim:
                sim.set_cta_warps(warps)
                sim.add_particles(x, vol=vol)
                sim.run(3, 1e-4)
                ms = _events_time(stream, lambda: sim.run(substeps, 1e-4))
                sim.sync()
            best = ms if best is None else min(best, ms)
        return 1e3 * best / substeps

    for name, fused, graphs in (("separate", False, False), ("separate_graphs", False, True),
                                ("g2p2g", True, False), ("g2p2g_graphs", True, True)):
        out[name] = timed(3, 0, fused, graphs)
    # variants tuned on this scene (per-phase kernel times), then the substep from graphs
    with mpm.Simulator(64, 1 / 64, [mat], stream=stream) as sim:
        sim.add_particles(x, vol=vol)
        sim.run(3, 1e-4)
        tp = tune.tune_p2g(sim, 1e-4, steps=10, rounds=2)
        tg = tune.tune_g2p(sim, 1e-4, steps=10, rounds=2)
        tw = tune.tune_cta_warps(sim, 1e-4, steps=10, rounds=2)
    out["tuned"] = {"p2g": tp["best_name"], "g2p": tg["best_name"], "cta_warps": tw["best"]}
    out["separate_graphs_tuned"] = timed(tp["best"], tg["best"], False, True, tw["best"])
    fused = {_variant_name("P2G", v): timed(v, 0, True, True) for v in FUSED_SCATTER_VARIANTS}
    out["g2p2g_graphs_by_scatter"] = fused
    out["g2p2g_graphs_tuned"] = min(fused.values())
    out["value"] = min(v for k, v in out.items() if k.startswith(("separate", "g2p2g")) and isinstance(v, float))
    out["particle_substeps_per_s"] = 8192 / (out["value"] * 1e-6)
    return out


def bench_ceilings(reps=5):
    """The second ceiling of P2G: float4 reductions applied by L2 per second
    (mpm_debug_red_rate) on a grid the size of the snow scene's (7,012 blocks
    of 64 nodes, 7.2 MB, L2-resident), the whole device busy (152 SMs x 2,048
    threads), 256 reductions per thread; per warp instruction 32 distinct
    nodes in 4 lines, four lanes per node, a line per lane, and one node."""
    import torch
    from paper_2111_00699_gb300 import mpm
    nodes = 7012 * 64
    grid = torch.zeros((nodes, 4), dtype=torch.float32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    threads, reds = sms * 2048, 256
    stream = torch.cuda.Stream()
    out = {"workload": "L2 float4 reductions: %d nodes (7.2 MB), %d threads x %d reductions" % (nodes, threads, reds),
           "unit": "float4 reductions/s"}
    for pattern, name in ((0, "distinct_nodes"), (1, "four_lanes_per_node"), (2, "one_line_per_lane"),
                          (3, "one_node_per_warp")):
        grid.zero_()
        torch.cuda.synchronize()
        for _ in range(2):
            mpm.debug_red_rate(grid, threads, reds, pattern, stream)
        best = min(_events_time(stream, lambda: mpm.debug_red_rate(grid, threads, reds, pattern, stream))
                   for _ in range(reps))
        total = float(grid[:, 3].double().sum().item())
        expect = float(threads) * reds * (2 + reps)
        out[name] = {"per_s": threads * reds / (best / 1e3), "ms": best, "sum_ok": abs(total - expect) <= 1e-6 * expect}
    return out


def bench_ablations(substeps=100):
    """The paper's single-GPU ablations (Sec. 6), on the snow-blocks scene
    with the particles added in a shuffled order: free-zone rebuilds with a
    full sort (the default) against a rebuild before every substep, against
    no sort at all, and the P2G scatter forms (float4 reductions per node,
    a shared-memory node tile, register runs).  ms per substep over
    `substeps` substeps after 20 warm-up substeps, fresh context each."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.snow_blocks()
    x = x[np.random.default_rng(11).permutation(len(x))]
    xs = torch.from_numpy(x).cuda()
    mat = mpm.material(mpm.SNOW, **SNOW)
    stream = torch.cuda.Stream()

    def timed(p2g=3, g2p=4, no_sort=False, rebuild_every=False):
        with mpm.Simulator(RES, DX, [mat], boundary=mpm.SLIP, stream=stream, p2g_variant=p2g, g2p_variant=g2p,
                           no_sort=no_sort) as sim:
            sim.add_particles(xs)

            def run(k):
                if not rebuild_every:
                    return sim.run(k, DT)
                for _ in range(k):
                    sim.rebuild()
                    sim.substep(DT)
            run(20)
            ms = _events_time(stream, lambda: run(substeps))
            sim.sync()
        return ms / substeps

    out = {"workload": "snow blocks 1340960 particles, shuffled insertion order, %d substeps each" % substeps,
           "unit": "ms/substep"}
    out["free_zone_full_sort"] = timed()
    out["rebuild_every_substep"] = timed(rebuild_every=True)
    out["no_sort"] = timed(no_sort=True)
    out["p2g_float4_reductions_per_node"] = timed(p2g=0)
    out["p2g_shared_memory_node_tile"] = timed(p2g=2)
    out["p2g_register_runs_of_4"] = out["free_zone_full_sort"]
    # the paper's warp-level reduction (Sec. 4.2.2): lanes grouped by cell, and runs of lanes only
    out["p2g_warp_reduction_cell_groups"] = timed(p2g=9)
    out["p2g_warp_reduction_runs_of_lanes"] = timed(p2g=10)
    out["p2g_runs_into_warp_tile"] = timed(p2g=11)
    return out


def bench_layout_ablations(substeps=200):
    """The paper's layout studies (Sec. 6.2) on the snow-blocks scene in the
    bench configuration: SoA against AoSoA packets of 32 (P2G register runs
    of 8 and the 64-register G2P, 4 warps per CTA), and G2P with the B-spline
    weights in registers against the weights in shared memory; ms per launch
    of each phase (CUDA events around each phase), best of two rounds."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.snow_blocks()
    stream = torch.cuda.Stream()
    out = {"workload": "snow blocks 1340960 particles, P2G chunk8 + G2P occ, %d substeps per setting" % substeps,
           "unit": "ms per launch"}
    with mpm.Simulator(RES, DX, [mpm.material(mpm.SNOW, **SNOW)], boundary=mpm.SLIP, stream=stream, p2g_variant=4,
                       g2p_variant=4, resort_interval=RESORT_INTERVAL) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.run(50, DT)

        def phases(tag):
            sim.run(5, DT)
            sim.profile_enable(True)
            sim.profile_read()
            sim.run(substeps, DT)
            ph = sim.profile_read()
            sim.profile_enable(False)
            for k in ("p2g", "g2p"):
                t, nl = ph[k]
                key = "%s_%s" % (k, tag)
                out[key] = min(out.get(key, float("inf")), t / nl if nl else float("inf"))

        for rnd in range(2):
            sim.set_layout(False)
            phases("soa")
            sim.set_layout(True)
            phases("aosoa")
            sim.set_layout(False)
            sim.set_g2p_variant(7)
            phases("weights_in_shared_memory")
            sim.set_g2p_variant(4)
        sim.sync()
    out["aosoa_over_soa_p2g"] = out["p2g_aosoa"] / out["p2g_soa"]
    out["aosoa_over_soa_g2p"] = out["g2p_aosoa"] / out["g2p_soa"]
    out["smem_weights_over_registers_g2p"] = out["g2p_weights_in_shared_memory"] / out["g2p_soa"]
    return out


def bench_cta_warps(substeps=200):
    """Warps per CTA (the paper's study of Sec. 6.2) for the register-run P2G
    (runs of 8) and the 64-register G2P, at the same registers per thread,
    on the snow-blocks scene in the bench configuration: ms per launch of
    each phase (CUDA events around each phase), 2, 4 and 8 warps."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.snow_blocks()
    stream = torch.cuda.Stream()
    out = {"workload": "snow blocks 1340960 particles, P2G chunk8 + G2P occ, %d substeps per setting" % substeps,
           "unit": "ms per launch"}
    with mpm.Simulator(RES, DX, [mpm.material(mpm.SNOW, **SNOW)], boundary=mpm.SLIP, stream=stream, p2g_variant=4,
                       g2p_variant=4, resort_interval=RESORT_INTERVAL) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.run(50, DT)
        for rnd in range(2):
            for w in (2, 4, 8):
                sim.set_cta_warps(w)
                sim.run(5, DT)
                sim.profile_enable(True)
                sim.profile_read()
                sim.run(substeps, DT)
                ph = sim.profile_read()
                sim.profile_enable(False)
                for k in ("p2g", "g2p"):
                    t, nl = ph[k]
                    key = "%s_%d_warps" % (k, w)
                    out[key] = min(out.get(key, float("inf")), t / nl if nl else float("inf"))
        sim.sync()
    return out


def _snow_ms_per_substep(steps=400, warm=300):
    """ms per substep of the snow scene in the bench launch configuration
    (used by the fast-math ablation in a child process)."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.snow_blocks()
    stream = torch.cuda.Stream()
    with mpm.Simulator(RES, DX, [mpm.material(mpm.SNOW, **SNOW)], boundary=mpm.SLIP, stream=stream, p2g_variant=4,
                       g2p_variant=4, graphs=True, resort_interval=RESORT_INTERVAL) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.run(warm, DT)
        ms = _events_time(stream, lambda: sim.run(steps, DT))
        sim.sync()
    return ms / steps


def bench_fast_math():
    """Sec. 6 fast-math ablation: the same snow run with the library built
    with and without -use_fast_math (each in a child process, since one
    process loads one build)."""
    from paper_2111_00699_gb300 import build
    build.build(ieee=True)
    out = {"workload": "snow blocks 1340960 particles, 400 substeps after 300", "unit": "ms/substep"}
    for name, env in (("fast_math", {}), ("ieee", {"MPM_LIBRARY": "ieee"})):
        r = subprocess.run([sys.executable, "-c", "import bench, json; print(json.dumps(bench._snow_ms_per_substep()))"],
                           cwd=ROOT, env=dict(os.environ, **env), capture_output=True, text=True)
        out[name] = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else "failed: " + r.stderr[-300:]
    if isinstance(out["fast_math"], float) and isinstance(out["ieee"], float):
        out["ieee_over_fast_math"] = out["ieee"] / out["fast_math"]
    return out


def bench_nacc_snow(substeps=400):
    """The snow-blocks scene with the paper's own snow model, NACC (Sec. 6.5:
    bulk modulus 5e5 dyne/cm^2 = 5e4 Pa, nu 0.3, M 0.8, beta 0.9, xi 5;
    alpha0 = -0.01), 256^3, dt 5e-5, in the bench launch configuration."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.snow_blocks()
    stream = torch.cuda.Stream()
    mat = mpm.material(mpm.NACC, E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01)
    with mpm.Simulator(RES, DX, [mat], boundary=mpm.SLIP, stream=stream, p2g_variant=3, g2p_variant=4, graphs=True,
                       resort_interval=RESORT_INTERVAL) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.run(300, DT)
        ms = _events_time(stream, lambda: sim.run(substeps, DT))
        sim.sync()
        st = sim.stats()
    return {"workload": "snow blocks with NACC snow, %d particles, 256^3, dt=5e-5, %d substeps after 300"
                        % (len(x), substeps),
            "value": len(x) * substeps / (ms / 1e3), "unit": UNIT, "ms_per_substep": ms / substeps,
            "rebuilds": st["rebuilds"]}


def bench_snow_adaptive(frames=3, cfl=0.3):
    """The snow-blocks scene advanced by whole 1/60-s frames in adaptive
    substeps (mpm_advance: dt = min(dt_max, cfl dx / (v + c)), the step-size
    rule the paper's scenes use, Sec. 6.5) instead of the fixed dt 5e-5."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.snow_blocks()
    stream = torch.cuda.Stream()
    with mpm.Simulator(RES, DX, [mpm.material(mpm.SNOW, **SNOW)], boundary=mpm.SLIP, stream=stream, p2g_variant=3,
                       g2p_variant=4, resort_interval=RESORT_INTERVAL, graphs=True) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.advance(1.0 / 60.0, cfl=cfl, dt_max=5e-4)
        dts = []
        ms = _events_time(stream, lambda: [dts.extend(sim.advance(1.0 / 60.0, cfl=cfl, dt_max=5e-4))
                                           for _ in range(frames)])
        sim.sync()
        st = sim.stats()
    n_sub = len(dts)
    return {"workload": "snow blocks, %d particles, 256^3, adaptive dt (cfl %.2f), %d frames of 1/60 s after one"
                        % (len(x), cfl, frames),
            "value": len(x) * n_sub / (ms / 1e3), "unit": UNIT, "ms_per_frame": ms / frames,
            "substeps_per_frame": n_sub / frames, "mean_dt": float(np.mean(dts)), "min_dt": float(np.min(dts)),
            "ms_per_substep": ms / n_sub, "rebuilds": st["rebuilds"]}


def bench_sand(substeps=1000, neo_hookean=False):
    """Drucker-Prager sand (phi = 30 deg), 4 random boxes, ~500K particles at
    8 per cell, 128^3, dt 1e-4; neo_hookean: the neo-Hookean sand of the
    paper's sand benchmark instead of the Hencky St. Venant-Kirchhoff one."""
    import torch
    from paper_2111_00699_gb300 import mpm, scenes
    x, _ = scenes.sand_blocks()
    stream = torch.cuda.Stream()
    kind = mpm.NHSAND if neo_hookean else mpm.SAND
    with mpm.Simulator(128, 1.0 / 128, [mpm.material(kind, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0)],
                       boundary=mpm.SLIP, stream=stream, p2g_variant=3, g2p_variant=0) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.run(20, 1e-4)
        ms = _events_time(stream, lambda: sim.run(substeps, 1e-4))
        sim.sync()
        st = sim.stats()
    return {"workload": "sand blocks%s, %d particles, 128^3, dt=1e-4" % (" (neo-Hookean)" if neo_hookean else "", len(x)),
            "value": len(x) * substeps / (ms / 1e3),
            "unit": UNIT, "ms_per_substep": ms / substeps, "rebuilds": st["rebuilds"]}


def bench_adjoint(steps=200, k=20):
    """Differentiable rollout: 32,768-particle jelly cube (E = 1e4, nu = 0.2,
    rho = 1), 64^3, dt = 1e-4, 200 substeps with checkpoints every 20; the
    centre-of-mass loss and its gradients in v0 and E (forward + backward)."""
    import torch
    from paper_2111_00699_gb300 import diff, scenes
    x, v = scenes.jelly_cube(5, n_side=32)
    n = len(x)
    vol = torch.full((n,), 0.008 / n, device="cuda")
    sim = diff.DiffSim(64, 1 / 64, n, nu=0.2, rho=1.0, vol=vol)
    xt = torch.from_numpy(x).cuda()

    def once():
        vt = torch.from_numpy(v).cuda().requires_grad_(True)
        Et = torch.full((n,), 1e4, device="cuda", requires_grad=True)
        out = diff.rollout(xt, vt, Et, sim, steps, k=k, dt=1e-4)
        loss = diff.center_of_mass_loss(out, vol, (0.5, 0.3, 0.5))
        loss.backward()
        return loss

    once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        once()
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / reps
    sim.close()
    # forward substeps: steps (forward) + steps - steps/k (segment recomputation); adjoint substeps: steps
    return {"workload": "jelly cube %d particles, 64^3, %d substeps, checkpoints every %d" % (n, steps, k),
            "ms_per_gradient": el * 1e3, "gradients_per_s": 1.0 / el,
            "particle_substeps_per_s_forward_plus_adjoint": n * steps / el, "unit": "gradient evaluations/s"}


# ---------------------------------------------------------------- main arm

def _variant_name(kind, v):
    from paper_2111_00699_gb300 import _lib
    names = _lib.P2G_VARIANTS if kind == "P2G" else _lib.G2P_VARIANTS
    return names[v] if 0 <= v < len(names) else None


KERNEL_NAMES = {"P2G": {"direct": "k_p2g_direct", "strided": "k_p2g_strided", "tile": "k_p2g_tile",
                        "chunk4": "k_p2g_chunk<4, 0, 0, 0>", "chunk8": "k_p2g_chunk<8, 0, 0, 0>", "stage4": "k_p2g_stage<4>",
                        "stage8": "k_p2g_stage<8>", "sacc4": "k_p2g_chunk<4, 1, 0, 0>", "slab4": "k_p2g_slab<4>",
                        "warp": "k_p2g_warp<1>", "warprun": "k_p2g_warp<0>", "wtile8": "k_p2g_wtile<8>",
                        "wxpose": "k_p2g_wxpose", "chunk8x2": "k_p2g_chunk<8, 0, 0, 1>",
                        "node": "k_p2g_node<4, 0>", "chunk8s": "k_p2g_chunks<8, 0>"},
                "G2P": {"direct": "k_g2p", "chunk4": "k_g2p_chunk<4>", "chunk8": "k_g2p_chunk<8>", "tile": "k_g2p_tile",
                        # the bench scene has one material (snow, kind 2): the kernels specialised to it
                        "occ": "k_g2p_occ<8, 2, 128, 0, 0>", "stage": "k_g2p_stage",
                        "occ10": "k_g2p_occ<10, -1, 128, 0, 0>", "occsw": "k_g2p_occ<8, 2, 128, 1, 0>"}}
# (names as ncu prints them: template booleans as 0 / 1)


FUSED_SCATTER_VARIANTS = (0, 3, 4, 7, 9, 10)
FUSED_KERNEL_NAMES = {0: "k_g2p2g", 1: "k_g2p2g", 2: "k_g2p2g", 3: "k_g2p2g_chunk<4, 0>",
                      4: "k_g2p2g_chunk<8, 0>", 5: "k_g2p2g_chunk<4, 0>", 6: "k_g2p2g_chunk<8, 0>",
                      7: "k_g2p2g_chunk<4, 1>", 8: "k_g2p2g", 9: "k_g2p2g_warp<1>", 10: "k_g2p2g_warp<0>",
                      11: "k_g2p2g_chunk<8, 0>"}


def p2g_kernel_name(variant, aosoa, warps):
    """The P2G kernel a variant launches, as ncu names it, for the store layout
    and the CTA size (the register-run forms have one instantiation each)."""
    if variant in ("chunk4", "chunk8"):
        k = variant[-1]
        if warps == 2:
            return "k_p2g_chunk_w2<%s, %d>" % (k, int(aosoa))
        if warps == 8:
            return "k_p2g_chunk_w8<%s>" % k
        return "k_p2g_chunk<%s, 0, %d, 0>" % (k, int(aosoa))
    if variant == "node":
        return "k_p2g_node<4, %d>" % int(aosoa)
    if variant == "chunk8s":
        return "k_p2g_chunks<8, %d>" % int(aosoa)
    return KERNEL_NAMES["P2G"][variant]


def g2p_kernel_name(variant, aosoa, warps):
    """The G2P kernel a variant launches on the snow scene (kind 2), as ncu names it."""
    if variant in ("occ", "occsw"):
        threads = 128 if (variant == "occsw" and not aosoa) else 32 * warps
        return "k_g2p_occ<8, 2, %d, %d, %d>" % (threads, int(variant == "occsw"), int(aosoa))
    if variant == "occ10" and aosoa:
        return "k_g2p_occ<10, 2, 128, 0, 1>"
    return KERNEL_NAMES["G2P"][variant]


KERNEL_SOURCES = ("transfer.cuh", "p2g.cu", "g2p.cu", "g2p2g.cu", "device_math.cuh", "async_copy.cuh", "internal.h")


def kernel_source_hash():
    """SHA-1 over the code the transfer kernels are compiled from (comments and
    whitespace removed, so that editing a comment keeps the record): a DRAM
    traffic figure recorded from an ncu capture is valid only for that code."""
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, "paper_2111_00699_gb300", "csrc", f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def _traffic_for(kernel, src_hash):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha1") != src_hash:
        return None
    return rec.get("bytes_per_launch")


# The other workloads reported beside the headline scene (name, function).
WORKLOADS = (("batched", bench_batched), ("fountain", bench_fountain),
             ("fountain_asflip", lambda: bench_fountain(asflip=True)), ("sand", bench_sand),
             ("sand_neo_hookean", lambda: bench_sand(neo_hookean=True)),
             ("snow_adaptive", bench_snow_adaptive),
             ("nacc_snow", bench_nacc_snow),
             ("small_elastic", bench_small_elastic), ("adjoint", bench_adjoint),
             ("ablations", bench_ablations), ("cta_warps", bench_cta_warps), ("layout", bench_layout_ablations),
             ("fast_math", bench_fast_math), ("ceilings", bench_ceilings))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=333)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="skip the batched / fountain / sand sections")
    ap.add_argument("--workload", default=None, choices=[w[0] for w in WORKLOADS],
                    help="run only this one of the other workloads and print its JSON (for profiling)")
    ap.add_argument("--e2e-frames", type=int, default=3)
    ap.add_argument("--p2g-variant", type=int, default=-1,
                    help="P2G scatter variant (0 direct, 1 strided, 2 tile, 3 chunk4, 4 chunk8, 5 stage4, "
                         "6 stage8, 7 sacc4, 8 slab4, 9 warp, 10 warprun, 11 wtile8, 12 wxpose, 13 chunk8x2, 14 node, 15 chunk8s); -1 = autotune")
    ap.add_argument("--g2p-variant", type=int, default=-1,
                    help="G2P gather variant (0 direct, 1 chunk4, 2 chunk8, 3 tile, 4 occ, 5 stage, 6 occ10, "
                         "7 occsw); -1 = autotune")
    ap.add_argument("--profile-substeps", type=int, default=0,
                    help="profiler mode: run this many substeps of the snow scene with the given variants "
                         "(default chunk4 P2G, occ G2P), print one status line and exit; no timing")
    ap.add_argument("--aosoa", type=int, default=0, choices=[0, 1],
                    help="profiler mode: 1 = AoSoA particle store (P2G variant 3/4/14/15, G2P 4/6/7)")
    ap.add_argument("--resort-interval", type=int, default=RESORT_INTERVAL,
                    help="profiler mode: window re-sort every this many substeps (0: off)")
    ap.add_argument("--cta-warps", type=int, default=4, choices=[2, 4, 8],
                    help="profiler mode: warps per CTA of the register-run P2G and the 64-register G2P")
    ap.add_argument("--g2p2g", type=int, default=None, choices=[0, 1],
                    help="1: fused G2P2G transfer, 0: separate phases; default: the faster one")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2111_00699_gb300 import _lib, build, mpm, scenes

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()

    if args.workload:
        if rank == 0:
            print(json.dumps({args.workload: dict(WORKLOADS)[args.workload]()}))
        return 0

    def barrier():
        if world > 1:
            dist.barrier()

    x, _ = scenes.snow_blocks()
    n = len(x)
    mat = mpm.material(mpm.SNOW, **SNOW)
    stream = torch.cuda.Stream()
    xs = torch.from_numpy(x).cuda()

    def fresh_sim(variant=4, gvariant=2):
        sim = mpm.Simulator(RES, DX, [mat], boundary=mpm.SLIP, stream=stream, p2g_variant=variant,
                            g2p_variant=gvariant, graphs=True, resort_interval=RESORT_INTERVAL)
        sim.add_particles(xs)
        return sim

    if args.profile_substeps > 0:
        # a short fixed sequence for ncu captures: the first substep rebuilds,
        # every later one launches P2G, grid update, G2P (or grid update and
        # the fused kernel) once
        pv = args.p2g_variant if args.p2g_variant >= 0 else 3
        gv = args.g2p_variant if args.g2p_variant >= 0 else 4
        sim = fresh_sim(pv, gv)
        sim.set_g2p2g(bool(args.g2p2g))
        sim.set_cta_warps(args.cta_warps)
        sim.set_layout(bool(args.aosoa))
        sim.set_resort_interval(args.resort_interval)
        sim.run(args.profile_substeps, DT)
        sim.sync()
        if rank == 0:
            print(json.dumps({"profile_substeps": args.profile_substeps, "p2g_variant": _variant_name("P2G", pv),
                              "g2p_variant": _variant_name("G2P", gv), "g2p2g": bool(args.g2p2g),
                              "aosoa": bool(args.aosoa), "cta_warps": args.cta_warps,
                              "stats": sim.stats()}))
        sim.close()
        return

    # ---- device-resident throughput (the `value`) ----
    from paper_2111_00699_gb300 import tune
    sim = fresh_sim()
    # clocks are sampled (every 200 ms) from here to the end of the timed region: the autotuning
    # and warm-up substeps just before it run the same kernels under the same load, and a timed
    # region of a few ms would otherwise hold no sample at all
    clk = ClockSampler(local).__enter__()
    tuned = {"best": args.p2g_variant, "best_name": _variant_name("P2G", args.p2g_variant), "ms": None}
    tuned_g = {"best": args.g2p_variant, "best_name": _variant_name("G2P", args.g2p_variant), "ms": None}
    warm = args.warmup
    if args.p2g_variant < 0:
        s0 = sim.stats()["substeps"]
        # the close candidates are re-timed after 200 substeps of drift, 100 substeps each
        tuned = tune.tune_p2g(sim, DT, steps=20, rounds=2, refine_top=3, refine_steps=100, drift=200)
        warm -= sim.stats()["substeps"] - s0
    else:
        sim.set_p2g_variant(args.p2g_variant)
    if args.g2p_variant < 0:
        tuned_g = tune.tune_g2p(sim, DT, steps=20, rounds=2)    # advances 120 substeps
        warm -= 120
    else:
        sim.set_g2p_variant(args.g2p_variant)
    # then the P2G variant with the window re-sort interval, on whole substeps: the tuned variant and
    # the register runs of 8 with re-sorts every 64 (or 128) substeps against the drift-tolerant
    # sorted chunks with and without
    sorted_chunks = _lib.P2G_VARIANTS.index("chunk8s")
    chunk8 = _lib.P2G_VARIANTS.index("chunk8")
    tuned_o = {"best": (tuned["best"], RESORT_INTERVAL), "ms": None}
    if args.p2g_variant < 0:
        cands = list(dict.fromkeys([(tuned["best"], RESORT_INTERVAL), (chunk8, RESORT_INTERVAL),
                                    (chunk8, 2 * RESORT_INTERVAL), (sorted_chunks, 0),
                                    (sorted_chunks, 2 * RESORT_INTERVAL)]))
        tuned_o = tune.tune_order(sim, DT, cands, slice_steps=256, rounds=2)
        warm -= 2 * len(cands) * 256
    # warps per CTA of the register-run P2G and the 64-register G2P, then the particle store layout
    tuned_w = tune.tune_cta_warps(sim, DT, steps=20, rounds=2)  # advances 132 substeps
    warm -= 132
    tuned_l = tune.tune_layout(sim, DT, tuned_w["best"], steps=20, rounds=2)   # advances 132 substeps
    warm -= 132
    # separate phases vs the fused G2P2G transfer (Sec. 4.1), timed on this scene;
    # the fused kernel's scatter follows the P2G variant (direct, chunk4, chunk8)
    fused_ms, fused_scatter_ms = {}, {}
    p2g_separate = tuned_o["best"][0] if tuned_o["best"][0] >= 0 else 3
    aosoa = tuned_l["best"] == "aosoa"
    g2p_final = tuned_l.get("aosoa_g2p_variant", tuned_g["best"]) if aosoa else tuned_g["best"]
    for _ in range(2):
        sim.set_g2p2g(False)
        sim.set_p2g_variant(p2g_separate)
        sim.set_cta_warps(tuned_l["cta_warps"])
        sim.set_layout(aosoa)
        sim.run(3, DT)
        fused_ms.setdefault("separate", []).append(_events_time(stream, lambda: sim.run(20, DT)) / 20)
        warm -= 23
        sim.set_layout(False)   # the fused kernels run on the SoA store
        for v in FUSED_SCATTER_VARIANTS:
            sim.set_p2g_variant(v)
            sim.set_g2p2g(True)
            sim.run(3, DT)
            fused_scatter_ms.setdefault(_variant_name("P2G", v), []).append(
                _events_time(stream, lambda: sim.run(20, DT)) / 20)
            warm -= 23
    fused_scatter_ms = {k: min(v) for k, v in fused_scatter_ms.items()}
    fused_best = min(FUSED_SCATTER_VARIANTS, key=lambda v: fused_scatter_ms[_variant_name("P2G", v)])
    fused_ms = {"separate": min(fused_ms["separate"]), "g2p2g": fused_scatter_ms[_variant_name("P2G", fused_best)]}
    use_fused = args.g2p2g if args.g2p2g is not None else fused_ms["g2p2g"] < fused_ms["separate"]
    p2g_final = fused_best if use_fused else p2g_separate
    sim.set_g2p2g(bool(use_fused))
    sim.set_p2g_variant(p2g_final)
    if not use_fused:
        sim.set_cta_warps(tuned_l["cta_warps"])
        sim.set_layout(aosoa)
    warm = max(3, warm)
    sim.run(warm, DT)
    sim.sync()
    launches0 = sim.stats()["kernel_launches"]
    rebuilds0 = sim.stats()["rebuilds"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    sim.run(args.steps, DT)
    ev1.record(stream)
    ev1.synchronize()
    clk.__exit__(None, None, None)
    sim.sync()
    barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = sim.stats()
    launches = st["kernel_launches"] - launches0
    rebuilds = st["rebuilds"] - rebuilds0
    n_pblocks = st["n_pblocks"]
    ms = max_over_ranks(ms, world)
    ms_per_step = ms / args.steps
    value = replica_throughput(n, args.steps, world, ms)

    # ---- per-phase timing with CUDA events on the simulator's stream ----
    prof_steps = min(args.steps, 1000)
    sim.profile_enable(True)
    sim.profile_read()
    sim.run(prof_steps, DT)
    phases = sim.profile_read()
    sim.profile_enable(False)
    sim.sync()
    n_now = sim.n
    pb_now = sim.stats()["n_pblocks"]
    sim.close()
    avg = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in phases.items()}
    algo = {"p2g": BYTES_P2G * n_now, "g2p": BYTES_G2P * n_now, "grid": BYTES_GRID_NODE * 64 * pb_now}
    dom = max(("p2g", "grid", "g2p"), key=lambda k: phases[k][0])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_note = "of measured" if hbm else "of fallback"
    hbm = hbm or 6800.0
    achieved = algo[dom] / (avg[dom] / 1e3) / 1e9 if avg[dom] > 0 else 0.0
    src_hash = kernel_source_hash()
    if use_fused:
        # per substep: grid update + k_g2p2g (reads x F Jp vol mat 57 B, writes x v C F Jp 100 B)
        algo["g2p"] = 157 * n_now
    kernel_name = {"p2g": p2g_kernel_name(_variant_name("P2G", p2g_separate), aosoa and not use_fused,
                                          tuned_l["cta_warps"]),
                   "g2p": (FUSED_KERNEL_NAMES[p2g_final] if use_fused
                           else g2p_kernel_name(_variant_name("G2P", g2p_final), aosoa, tuned_l["cta_warps"])),
                   "grid": "k_grid"}[dom]
    # the same kernel on the layout-free byte count (P2G: x, v, C, F, Jp = 100 B per particle)
    survey_bytes = {"p2g": LAYOUT_FREE_BYTES_P2G * n_now}.get(dom)
    achieved_survey = survey_bytes / (avg[dom] / 1e3) / 1e9 if (survey_bytes and avg[dom] > 0) else None
    # the whole substep (timed region): own layout and the layout-free count
    sub_own = (algo["p2g"] if not use_fused else 0) + algo["g2p"] + algo["grid"]
    sub_survey = (LAYOUT_FREE_BYTES_SUBSTEP_FUSED if use_fused else LAYOUT_FREE_BYTES_SUBSTEP) * n
    substep = {"ms": ms_per_step, "bytes_own": sub_own, "bytes_survey": sub_survey,
               "achieved_own_gbs": sub_own / (ms_per_step / 1e3) / 1e9,
               "achieved_survey_gbs": sub_survey / (ms_per_step / 1e3) / 1e9,
               "frac_own": sub_own / (ms_per_step / 1e3) / 1e9 / hbm,
               "frac_survey": sub_survey / (ms_per_step / 1e3) / 1e9 / hbm,
               "survey_bytes_per_particle": LAYOUT_FREE_BYTES_SUBSTEP_FUSED if use_fused else LAYOUT_FREE_BYTES_SUBSTEP,
               "ms_per_frame_at_frac_0p5_survey": sub_survey / (0.5 * hbm * 1e9) * 1e3 * SUBSTEPS_PER_FRAME}
    roofline = {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": peak_note,
                "algorithmic_bytes_per_launch": algo[dom], "avg_launch_ms": avg[dom],
                "achieved_survey": achieved_survey,
                "frac_survey": achieved_survey / hbm if achieved_survey is not None else None,
                "survey_bytes_per_launch": survey_bytes,
                "traffic": _traffic_for(kernel_name, src_hash),
                "substep": substep,
                "phases_ms_per_launch": {k: round(v, 5) for k, v in avg.items()},
                "phase_launches": {k: v[1] for k, v in phases.items()}}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if args.e2e_frames > 0:
        sim = fresh_sim(p2g_final, g2p_final)
        sim.set_g2p2g(bool(use_fused))
        if not use_fused:
            sim.set_cta_warps(tuned_l["cta_warps"])
            sim.set_layout(aosoa)
        host = {k: torch.empty(s, dtype=torch.float32).pin_memory()
                for k, s in (("x", (n, 3)), ("v", (n, 3)), ("C", (n, 9)), ("F", (n, 9)), ("Jp", (n,)))}
        sim.read_state_into(x=host["x"], v=host["v"], C=host["C"].view(n, 3, 3), F=host["F"].view(n, 3, 3),
                            Jp=host["Jp"])
        per_frame = int(round(SUBSTEPS_PER_FRAME))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_frames):
            sim.write_state(x=host["x"], v=host["v"], C=host["C"], F=host["F"], Jp=host["Jp"])
            sim.run(per_frame, DT)
            sim.read_state_into(x=host["x"], v=host["v"], C=host["C"].view(n, 3, 3), F=host["F"].view(n, 3, 3),
                                Jp=host["Jp"])
        el = time.perf_counter() - t0
        sim.close()
        el = max_over_ranks(el, world)
        state_bytes = n * 4 * (3 + 3 + 9 + 9 + 1)
        e2e = {"value": replica_throughput(n, per_frame * args.e2e_frames, world, el * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": state_bytes / per_frame, "d2h_bytes_per_step": state_bytes / per_frame,
               "protocol": "per frame: mpm_write_state of the full state from pinned host memory, %d mpm_substep "
                           "calls, mpm_read_state of the full state into pinned host memory; bytes are per "
                           "substep" % per_frame, "frames": args.e2e_frames}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    workloads = None
    if not args.no_workloads and world == 1:
        workloads = {}
        for name, fn in WORKLOADS:
            try:
                workloads[name] = fn()
            except Exception as exc:   # report, do not lose the main line
                workloads[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, sample = oracle_throughput(x, seconds=15.0)
        cpu = dict({"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}, **host_cores())

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "ms_per_frame": ms_per_step * SUBSTEPS_PER_FRAME,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(n, world),
            "clocks": dict(clk.summary(), window="autotuning, warm-up and timed substeps"),
            "p2g_variant": tuned, "g2p_variant": tuned_g, "cta_warps": tuned_w, "layout": tuned_l,
            "order": {"p2g_variant": _variant_name("P2G", tuned_o["best"][0]), "resort_interval": tuned_o["best"][1],
                      "ms_per_substep": tuned_o["ms"]},
            "transfer": {"mode": "g2p2g" if use_fused else "separate", "ms_per_substep": fused_ms,
                         "g2p2g_scatter_ms": fused_scatter_ms, "p2g_variant_used": _variant_name("P2G", p2g_final)}, "e2e": e2e, "gpu_launches": launches, "rebuilds_in_timed_region": rebuilds,
            "n_pblocks": n_pblocks, "roofline": roofline, "cpu_baseline": cpu, "workloads": workloads}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
