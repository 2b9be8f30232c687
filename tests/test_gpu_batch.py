"""GPU parity of the batched substep: every scene of a batch must match the
FP64 oracle run on that scene alone (x within 1e-4 of the unit domain, v
within 1e-4 of max|v|, after 10 substeps), with and without CUDA graphs, and
per-scene remapping must keep parity."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2111_00699_gb300 import scenes

pytestmark = pytest.mark.gpu

MATS = [dict(kind=0, E=1e4, nu=0.2, rho=1000.0), dict(kind=1, E=1e4, gamma=7.0, rho=1000.0),
        dict(kind=2, E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0),
        dict(kind=3, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0)]
DT = [1e-4, 1e-4, 5e-5, 1e-4]


@pytest.fixture(scope="module")
def M():
    from paper_2111_00699_gb300 import build, mpm
    build.build()
    assert torch.cuda.is_available()
    orc.build()
    return mpm


def _mats(M):
    g = [M.material(**m) for m in MATS]
    o = [orc.material(**m) for m in MATS]
    return g, o


def _oracle_run(sc, x, v, om, dt, steps):
    res = sc["res"]
    s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=(1.0 / res) ** 3 / 8)
    cfg = orc.config(res, 1.0 / res, orc.SLIP)
    for _ in range(steps):
        assert orc.substep(cfg, om, s, dt) == 0
    return s


def _batch_case(n_scenes=8, seed=40, n_max=6000, v_scale=0.3):
    bs = scenes.batched_scenes(seed, n_scenes=n_scenes, n_min=1500, n_max=n_max, grids=(32, 64), n_materials=4)
    rng = np.random.default_rng(seed)
    vs = [(v_scale * rng.normal(size=(len(b["x"]), 3))).astype(np.float32) for b in bs]
    return bs, vs


def _run_batch(M, bs, vs, steps, graphs, chunk=4, persistent=False, warps=4):
    gm, _ = _mats(M)
    descs = [dict(res=b["res"], dx=1.0 / b["res"], material=b["material"]) for b in bs]
    dts = np.array([DT[b["material"]] for b in bs], np.float32)
    with M.BatchSimulator(descs, gm, graphs=graphs, p2g_chunk=chunk) as bsim:
        for i, (b, v) in enumerate(zip(bs, vs)):
            bsim.add_particles(i, b["x"], v)
        bsim.set_persistent(persistent)
        bsim.set_cta_warps(warps)
        bsim.run(steps, dts)
        out = [bsim.read_state(i) for i in range(len(bs))]
        st = bsim.stats()
    return out, st, dts


@pytest.mark.parametrize("graphs,chunk,persistent,warps", [(False, 4, False, 4), (True, 4, False, 4),
                                                            (True, 1, False, 4), (True, 8, False, 4),
                                                            (True, 4, False, 2), (True, 8, False, 8),
                                                            (False, 4, True, 4), (True, 1, True, 4),
                                                            (True, 4, True, 4), (True, 8, True, 4)])
def test_batched_scenes_match_oracle(M, graphs, chunk, persistent, warps):
    """Per-phase launches in CTAs of 2, 4 or 8 warps, and the persistent form
    (one cooperative launch per substep with grid barriers), each with P2G
    register runs of 1, 4 or 8 particles."""
    bs, vs = _batch_case()
    out, st, dts = _run_batch(M, bs, vs, 10, graphs, chunk, persistent, warps)
    _, om = _mats(M)
    assert st["substeps"] == 10
    if graphs:
        assert st["graph_launches"] == 10     # every substep replays a captured graph
    for i, b in enumerate(bs):
        s = _oracle_run(b, b["x"], vs[i], om[b["material"]], float(dts[i]), 10)
        g = out[i]
        assert np.abs(g["x"] - s.x).max() <= 1e-4, i
        assert np.abs(g["v"] - s.v).max() <= 1e-4 * np.abs(s.v).max(), i
        assert np.abs(g["Jp"] - s.Jp).max() <= 1e-4, i


@pytest.mark.parametrize("persistent", [False, True])
def test_batched_per_scene_remap(M, persistent):
    """One fast scene must remap repeatedly while a resting scene does not,
    and both must keep parity."""
    gm, om = _mats(M)
    xa = scenes.cube_uniform(1, 3000, 0.3, 0.4)
    xb = scenes.cube_uniform(2, 3000, 0.45, 0.55)
    va = np.tile(np.array([25.0, 15.0, 5.0], np.float32), (3000, 1))
    vb = np.zeros((3000, 3), np.float32)
    descs = [dict(res=64, dx=1 / 64, material=0), dict(res=64, dx=1 / 64, material=0)]
    with M.BatchSimulator(descs, gm) as bsim:
        bsim.add_particles(0, xa, va)
        bsim.add_particles(1, xb, vb)
        bsim.set_persistent(persistent)
        bsim.run(60, 1e-4)
        ga, gb = bsim.read_state(0), bsim.read_state(1)
        st = bsim.stats()
    assert st["remaps"] >= 3, st
    for g, x, v in ((ga, xa, va), (gb, xb, vb)):
        s = _oracle_run(dict(res=64), x, v, om[0], 1e-4, 60)
        assert np.abs(g["x"] - s.x).max() <= 1e-4
        assert np.abs(g["v"] - s.v).max() <= 1e-4 * np.abs(s.v).max()


def test_batched_rejects_bad_input(M):
    gm, _ = _mats(M)
    with pytest.raises(M.MpmError):
        M.BatchSimulator([dict(res=4, dx=0.25, material=0)], gm)
    with M.BatchSimulator([dict(res=32, dx=1 / 32, material=0)], gm) as bsim:
        bsim.add_particles(0, np.array([[0.001, 0.5, 0.5]], np.float32))
        with pytest.raises(M.MpmError) as e:
            bsim.substep(1e-4)
        assert e.value.status == 4


@pytest.mark.parametrize("persistent", [False, True])
def test_batched_full_size_sampled_scenes(M, persistent):
    """The full batched workload as bench.py times it (256 scenes, 4.8M
    particles, seed 4, CUDA graphs, P2G runs of 8), 10 substeps from rest,
    per-phase launches or the persistent launch; two scenes per material
    (the smallest and the largest) are compared with the oracle run on that
    scene alone."""
    bs = scenes.batched_scenes(4)
    assert len(bs) == 256
    vs = [np.zeros((len(b["x"]), 3), np.float32) for b in bs]
    out, st, dts = _run_batch(M, bs, vs, 10, True, 8, persistent)
    assert st["graph_launches"] == 10
    _, om = _mats(M)
    picks = []
    for mat in range(4):
        ids = [i for i, b in enumerate(bs) if b["material"] == mat]
        ids.sort(key=lambda i: len(bs[i]["x"]))
        picks += [ids[0], ids[-1]]
    for i in picks:
        b = bs[i]
        s = _oracle_run(b, b["x"], vs[i], om[b["material"]], float(dts[i]), 10)
        g = out[i]
        assert np.abs(g["x"] - s.x).max() <= 1e-4, i
        assert np.abs(g["v"] - s.v).max() <= 1e-4 * np.abs(s.v).max(), i
        assert np.abs(g["Jp"] - s.Jp).max() <= 1e-4, i


def test_batched_paper_materials(M):
    """The paper's own materials in one batch: an NACC snow scene and a
    neo-Hookean sand scene, each against the oracle run alone (10 substeps,
    random velocities so that both return maps act)."""
    kw = [dict(kind=M.NACC, E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01),
          dict(kind=M.NHSAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0)]
    gm = [M.material(**m) for m in kw]
    om = [orc.material(**m) for m in kw]
    rng = np.random.default_rng(44)
    xs = [scenes.cube_uniform(3, 4000, 0.3, 0.5), scenes.cube_uniform(4, 4000, 0.4, 0.6)]
    vs = [(0.5 * rng.normal(size=(4000, 3))).astype(np.float32) for _ in range(2)]
    descs = [dict(res=64, dx=1 / 64, material=0), dict(res=32, dx=1 / 32, material=1)]
    with M.BatchSimulator(descs, gm) as bsim:
        for i in range(2):
            bsim.add_particles(i, xs[i], vs[i])
        bsim.run(10, 5e-5)
        got = [bsim.read_state(i) for i in range(2)]
    for i, res in enumerate((64, 32)):
        s = _oracle_run(dict(res=res), xs[i], vs[i], om[i], 5e-5, 10)
        assert np.abs(got[i]["x"] - s.x).max() <= 1e-4
        assert np.abs(got[i]["v"] - s.v).max() <= 1e-4 * np.abs(s.v).max()
