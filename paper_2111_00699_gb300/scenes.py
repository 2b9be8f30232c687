"""Seeded synthetic scenes shaped like the paper's workloads.

This module only draws particle positions and velocities: it holds none of
the method's arithmetic, so tests can feed the same inputs to the CUDA path
and to the oracle.  Every generator is deterministic in its seed.

Scenes (paper Sec. 6):
  * ``cube_uniform``  -- i.i.d. uniform particles in a cube (small elastic case).
  * ``blocks``        -- axis-aligned boxes of random sizes sampled at 8
    particles per cell with stratified jitter (one random point in each of a
    cell's 2x2x2 sub-cells), the sampling of the Sand Blocks setting (Sec. 6);
    used for the snow blocks and sand blocks scenes.
  * ``jelly_cube``    -- a jittered lattice cube with random initial velocity.
  * ``fountain_batch`` -- the particles a disk inlet emits in one substep,
    drawn from a counter-based generator (splitmix64) keyed by
    (seed, substep), standing in for the Fountain's particle source (Sec. 6.4).
  * ``batched_scenes`` -- many small independent scenes of log-uniform size.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea and Flood 2014) applied to an
    array of 64-bit counters."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _MASK
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK
        return z ^ (z >> np.uint64(31))


def _uniform01(counter: np.ndarray) -> np.ndarray:
    return (splitmix64(counter) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def cube_uniform(seed: int, n: int, lo: float = 0.4, hi: float = 0.6) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)


def _stratified_box(rng, lo_cell, n_cells, dx, ppc_side=2):
    """One particle uniformly inside each of ppc_side^3 sub-cells of every cell."""
    sub = dx / ppc_side
    ix = [np.arange(n_cells[a] * ppc_side) for a in range(3)]
    gz, gy, gx = np.meshgrid(ix[2], ix[1], ix[0], indexing="ij")
    idx = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64)
    jit = rng.uniform(0.0, 1.0, size=idx.shape)
    return np.asarray(lo_cell, dtype=np.float64) * dx + (idx + jit) * sub


def blocks(seed: int, target: int, res: int, n_boxes: int, edge_range=(0.08, 0.2),
           ppc_side: int = 2, y_range=(0.15, 0.95), wall: int = 3, gap_cells: int = 2,
           max_tries: int = 100000):
    """Non-overlapping axis-aligned boxes of random sizes, whole cells only,
    sampled at ppc_side^3 particles per cell.  Edge lengths are drawn in
    edge_range (fraction of the domain), then scaled by a common factor so the
    total particle count lands within 1% of target.  Returns (x float32 (n,3),
    list of (lo_cell, n_cells))."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    ppc = ppc_side ** 3
    edges = rng.uniform(edge_range[0], edge_range[1], size=(n_boxes, 3))
    cells_f = edges * res
    scale = (target / (ppc * np.prod(cells_f, axis=1).sum())) ** (1.0 / 3.0)
    n_cells = np.maximum(1, np.round(cells_f * scale)).astype(np.int64)
    # nudge the largest box until the count is within 1%
    for _ in range(1000):
        total = int(ppc * np.prod(n_cells, axis=1).sum())
        if abs(total - target) <= 0.01 * target:
            break
        b = int(np.argmax(np.prod(n_cells, axis=1)))
        a = int(rng.integers(0, 3))
        n_cells[b, a] += 1 if total < target else -1
    lo_min = wall + 1
    placed = []
    for b in range(n_boxes):
        for _ in range(max_tries):
            lo = np.empty(3, dtype=np.int64)
            for a in range(3):
                lo_a = lo_min if a != 1 else max(lo_min, int(y_range[0] * res))
                hi_a = (res - wall - 2 if a != 1 else int(y_range[1] * res)) - n_cells[b, a]
                if hi_a < lo_a:
                    raise ValueError("box does not fit in the domain")
                lo[a] = rng.integers(lo_a, hi_a + 1)
            ok = True
            for (plo, pn) in placed:
                if all(lo[a] < plo[a] + pn[a] + gap_cells and plo[a] < lo[a] + n_cells[b, a] + gap_cells
                       for a in range(3)):
                    ok = False
                    break
            if ok:
                placed.append((lo, n_cells[b].copy()))
                break
        else:
            raise ValueError("could not place box %d without overlap" % b)
    xs = [_stratified_box(rng, lo, n, dx, ppc_side) for (lo, n) in placed]
    return np.concatenate(xs).astype(np.float32), placed


def snow_blocks(seed: int = 1, target: int = 1_330_000, res: int = 256, n_boxes: int = 6):
    """Snow blocks scene: 6 random boxes at 8 particles per cell, about 1.33M
    particles, on a 256^3 grid (stands in for the 1.33M-particle snow scene
    of Sec. 6.5, whose animated character is not available)."""
    return blocks(seed, target, res, n_boxes)


def sand_blocks(seed: int = 3, target: int = 500_000, res: int = 128, n_boxes: int = 4):
    """Sand blocks scene: 4 random boxes at 8 particles per cell (Sec. 6,
    Sand Blocks setting)."""
    return blocks(seed, target, res, n_boxes)


def jelly_cube(seed: int = 5, n_side: int = 32, lo: float = 0.4, hi: float = 0.6,
               v_mean=(1.0, 0.5, 0.0), v_std: float = 0.1):
    """A jittered n_side^3 lattice filling [lo, hi]^3 with initial velocity
    v_mean + N(0, v_std^2) per particle and component."""
    rng = np.random.default_rng(seed)
    h = (hi - lo) / n_side
    i = np.arange(n_side)
    gz, gy, gx = np.meshgrid(i, i, i, indexing="ij")
    idx = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64)
    x = lo + (idx + rng.uniform(0.0, 1.0, idx.shape)) * h
    v = np.asarray(v_mean)[None, :] + v_std * rng.normal(size=x.shape)
    return x.astype(np.float32), v.astype(np.float32)


def fountain_count(dt: float, vol: float, radius: float = 0.05, speed: float = 3.0) -> int:
    """Particles the inlet emits per substep: the volume of the slab
    pi r^2 * speed * dt divided by the particle volume."""
    return int(round(math.pi * radius * radius * speed * dt / vol))


def fountain_batch(seed: int, substep: int, dt: float, vol: float, center=(0.5, 0.1, 0.5),
                   radius: float = 0.05, speed: float = 3.0):
    """Particles emitted at one substep: uniform in the disk (normal +y) times
    a slab of height speed*dt, all moving at (0, speed, 0).  Draws come from
    splitmix64 on the counter (seed << 40) + (substep << 16) + 3*i + k."""
    m = fountain_count(dt, vol, radius, speed)
    i = np.arange(m, dtype=np.uint64)
    base = (np.uint64(seed) << np.uint64(40)) + (np.uint64(substep) << np.uint64(16))
    u = [_uniform01(base + np.uint64(3) * i + np.uint64(k)) for k in range(3)]
    r = radius * np.sqrt(u[0])
    th = 2.0 * math.pi * u[1]
    x = np.stack([center[0] + r * np.cos(th), center[1] + speed * dt * u[2], center[2] + r * np.sin(th)], axis=1)
    v = np.tile(np.array([0.0, speed, 0.0]), (m, 1))
    return x.astype(np.float32), v.astype(np.float32)


def batched_scenes(seed: int = 4, n_scenes: int = 256, n_min: int = 2048, n_max: int = 65536,
                   grids=(32, 64, 128), n_materials: int = 4):
    """Independent small scenes: particle count log-uniform in [n_min, n_max],
    grid size uniform over `grids`, material uniform over n_materials, one
    random box per scene sampled at 8 particles per cell (rounded to whole
    cells).  Returns a list of dicts with x (float32), res, material."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        res = int(rng.choice(grids))
        mat = int(rng.integers(0, n_materials))
        cells = max(1.0, n / 8.0)
        side = max(2, int(round(cells ** (1.0 / 3.0))))
        side = min(side, res - 12)
        lo = [int(rng.integers(4, res - 4 - side + 1)) if a != 1 else int(rng.integers(max(4, res // 4), res - 4 - side + 1))
              for a in range(3)]
        x = _stratified_box(rng, lo, [side] * 3, 1.0 / res)
        out.append({"x": x.astype(np.float32), "res": res, "material": mat, "seed": int(rng.integers(0, 2**31))})
    return out
