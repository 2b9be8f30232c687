"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (stated per check):
  * keys, permutation, physical-block list: bit-exact;
  * grid mass and momentum after P2G: |gpu - oracle|_inf <= 1e-5 |oracle|_inf
    (per field);
  * x after 10 substeps: |dx|_inf <= 1e-4 (domain length 1); v after 10
    substeps: |dv|_inf <= 1e-4 |v|_inf;
  * total grid mass vs total particle mass: 1e-6 relative.
"""
import os

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2111_00699_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2111_00699_gb300 import build, mpm
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    orc.build()
    return mpm


def linf(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).max())


def mats_pair(M, kind, **kw):
    return M.material(kind, **kw), orc.material(kind, **kw)


def oracle_state_from(sim_state, vol, mat_ids=None):
    st = {k: v.detach().cpu().numpy().astype(np.float64) for k, v in sim_state.items()}
    return orc.State(st["x"], st["v"], st["C"], st["F"], st["Jp"], vol, 0 if mat_ids is None else mat_ids)


def L_of(res):
    L = 0
    while (4 << L) < res:
        L += 1
    return L


# ---------------------------------------------------------------- device math

def _rand_rot(rng, n):
    q, r = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    q = q * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    d = np.linalg.det(q)
    q[d < 0, :, 0] *= -1
    return q


def test_svd_matches_numpy(M):
    rng = np.random.default_rng(0)
    n = 4096
    F = np.concatenate([np.eye(3) + 0.1 * rng.normal(size=(n // 2, 3, 3)),
                        rng.normal(size=(n // 4, 3, 3)),
                        np.einsum("nab,nb,ncb->nac", _rand_rot(rng, n // 4),
                                  np.tile([1.2, 1.2, 0.7], (n // 4, 1)), _rand_rot(rng, n // 4))])
    F[-8:] = np.diag([1.0, 1.0, -1.0]) @ F[-8:]               # inverted
    Ft = torch.tensor(F, dtype=torch.float32, device="cuda")
    U, S, V = (t.double().cpu().numpy() for t in M.debug_svd(Ft))
    F32 = Ft.double().cpu().numpy()
    scale = np.abs(F32).reshape(n, -1).max(1)
    rec = np.einsum("nab,nb,ncb->nac", U, S, V)
    assert (np.abs(rec - F32).reshape(n, -1).max(1) / scale).max() < 2e-5
    I = np.eye(3)
    assert np.abs(np.einsum("nba,nbc->nac", U, U) - I).max() < 2e-5
    assert np.abs(np.einsum("nba,nbc->nac", V, V) - I).max() < 2e-5
    assert np.abs(np.linalg.det(U) - 1).max() < 2e-5 and np.abs(np.linalg.det(V) - 1).max() < 2e-5
    ref = np.linalg.svd(F32, compute_uv=False)
    assert (np.abs(np.abs(S) - ref).max(1) / ref[:, 0]).max() < 2e-5
    assert np.all(S[:, 0] >= S[:, 1] - 1e-5 * ref[:, 0]) and np.all(S[:, 1] >= np.abs(S[:, 2]) - 1e-5 * ref[:, 0])
    d = np.linalg.det(F32)
    big = np.abs(d) > 1e-3
    assert np.all(np.sign(S[big, 2]) == np.sign(d[big]))


@pytest.mark.parametrize("scale", [0.05, 0.01])
@pytest.mark.parametrize("kind", ["elastic", "snow", "fluid", "sand", "nacc", "nhsand"])
def test_stress_matches_oracle(M, kind, scale):
    """Stress of stored states, on the SVD path (5 % strain) and on the
    small-strain series path (1 %)."""
    rng = np.random.default_rng(1)
    n = 2048
    kw = dict(elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2), snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, hardening=10.0),
              fluid=dict(kind=M.FLUID, E=1e4, gamma=7.0), sand=dict(kind=M.SAND, E=3.5e5, nu=0.3),
              nacc=dict(kind=M.NACC, E=5e4, nu=0.3, hardening=5.0),
              nhsand=dict(kind=M.NHSAND, E=3.5e5, nu=0.3))[kind]
    k = kw.pop("kind")
    gm, om = M.material(k, **kw), orc.material(k, **kw)
    F = (np.eye(3) + scale * rng.normal(size=(n, 3, 3))).astype(np.float32)
    Jp = rng.uniform(0.95, 1.05, n).astype(np.float32)
    tau = M.debug_stress(gm, torch.from_numpy(F).cuda(), torch.from_numpy(Jp).cuda()).double().cpu().numpy()
    ref = np.stack([orc.kirchhoff(om, F[i].astype(np.float64), float(Jp[i])) for i in range(n)])
    assert linf(tau, ref) <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["elastic", "snow", "sand", "nhsand"])
def test_stress_small_strain_matches_oracle(M, kind):
    """Strains of 1e-4: the stress is proportional to sigma - 1, which an SVD
    of F itself resolves only to ~1e-7 / 1e-4 = 1e-3 relative.  The kernels
    hold H = F - I and get sigma - 1 from F^T F - I = H + H^T + H^T H, so
    they must match the oracle to 1e-4 here too (both sides see the same
    FP32-rounded F, for which F - I is exact)."""
    rng = np.random.default_rng(11)
    n = 2048
    kw = dict(elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2), snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, hardening=10.0),
              sand=dict(kind=M.SAND, E=3.5e5, nu=0.3), nhsand=dict(kind=M.NHSAND, E=3.5e5, nu=0.3))[kind]
    k = kw.pop("kind")
    gm, om = M.material(k, **kw), orc.material(k, **kw)
    F = (np.eye(3) + 1e-4 * rng.normal(size=(n, 3, 3))).astype(np.float32)
    Jp = np.ones(n, np.float32)
    tau = M.debug_stress(gm, torch.from_numpy(F).cuda(), torch.from_numpy(Jp).cuda()).double().cpu().numpy()
    ref = np.stack([orc.kirchhoff(om, F[i].astype(np.float64), 1.0) for i in range(n)])
    assert linf(tau, ref) <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("scale", [0.04, 0.01])
def test_plasticity_matches_oracle(M, scale):
    """Return maps on trial states.  At 4 % strain almost every particle takes
    the SVD path; at 1 % almost every one takes the small-strain series path
    (|F F^T - I|_F <= 0.1), including snow states inside the clamp, and sand
    states in each of the three Drucker-Prager cases."""
    rng = np.random.default_rng(2)
    n = 1024
    for kind, kw in ((M.SNOW, dict(E=1.4e5, nu=0.2, theta_c=2.5e-2, theta_s=7.5e-3)),
                     (M.SAND, dict(E=3.5e5, nu=0.3, friction_deg=30.0)),
                     (M.NHSAND, dict(E=3.5e5, nu=0.3, friction_deg=30.0)),
                     (M.NACC, dict(E=5e4, nu=0.3, hardening=5.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01))):
        gm, om = M.material(kind, **kw), orc.material(kind, **kw)
        F = (np.eye(3) + scale * rng.normal(size=(n, 3, 3))).astype(np.float32)
        Jp = rng.uniform(0.9, 1.1, n).astype(np.float32)
        Fg, Jg = M.debug_plasticity(gm, torch.from_numpy(F).cuda(), torch.from_numpy(Jp).cuda())
        Fg, Jg = Fg.double().cpu().numpy(), Jg.double().cpu().numpy()
        for i in range(n):
            Fo, Jo = orc.plasticity(om, F[i].astype(np.float64), float(Jp[i]))
            assert linf(Fg[i], Fo) <= 2e-5, (kind, i)
            assert abs(Jg[i] - Jo) <= 2e-5 * abs(Jo), (kind, i)


# ---------------------------------------------------------------------- sort

@pytest.mark.parametrize("n,bits", [(1, 8), (2047, 18), (2048, 24), (2049, 24), (100_003, 32), (1 << 20, 24)])
def test_radix_sort_bit_exact(M, n, bits):
    rng = np.random.default_rng(n + bits)
    mod = 1 << bits
    distinct = max(2, n // 4)                      # force runs of equal keys
    raw = rng.integers(0, min(mod, distinct), size=n, dtype=np.uint64)
    keys = ((raw * np.uint64(2654435761)) % np.uint64(mod)).astype(np.uint32)
    vals = np.arange(n, dtype=np.int32)
    ks, vs = M.radix_sort_pairs(torch.from_numpy(keys.view(np.int32)).cuda(), torch.from_numpy(vals).cuda(), bits)
    perm = orc.stable_sort(keys)
    np.testing.assert_array_equal(vs.cpu().numpy(), perm)
    np.testing.assert_array_equal(ks.cpu().numpy().view(np.uint32), keys[perm])


def _check_order_and_blocks(sim, x, res):
    L = L_of(res)
    keys, st = orc.particle_keys(x, float(res), L)
    assert st == 0
    perm = orc.stable_sort(keys)
    gk, gid = sim.read_order()
    np.testing.assert_array_equal(gk, keys[perm])
    np.testing.assert_array_equal(gid, perm)
    np.testing.assert_array_equal(sim.read_blocks(), orc.pblocks(keys, L))


def test_keys_order_blocks_small(M):
    x = scenes.cube_uniform(0, 8192, 0.4, 0.6)
    with M.Simulator(64, 1 / 64, [M.material(M.ELASTIC)]) as sim:
        sim.add_particles(x)
        sim.rebuild()
        _check_order_and_blocks(sim, x, 64)


def test_keys_order_blocks_snow_full_size(M):
    x, _ = scenes.snow_blocks()
    with M.Simulator(256, 1 / 256, [M.material(M.SNOW, E=1.4e5, nu=0.2, rho=400.0)], boundary=M.SLIP) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        sim.rebuild()
        _check_order_and_blocks(sim, x, 256)


# ------------------------------------------------------------------ P2G grid

def _perturbed_state(rng, n, v_scale=0.5, C_scale=5.0, F_scale=0.02):
    v = (v_scale * rng.normal(size=(n, 3))).astype(np.float32)
    C = (C_scale * rng.normal(size=(n, 3, 3))).astype(np.float32)
    F = (np.eye(3) + F_scale * rng.normal(size=(n, 3, 3))).astype(np.float32)
    return v, C, F


def _p2g_parity(M, sim, gm_list, om_list, x, vol, dt, res, mat_ids=None, tol=1e-5):
    rng = np.random.default_rng(7)
    n = len(x)
    v, C, F = _perturbed_state(rng, n)
    sim.write_state(v=torch.from_numpy(v).cuda(), C=torch.from_numpy(C).cuda(), F=torch.from_numpy(F).cuda())
    g = sim.debug_p2g(dt).double().cpu().numpy()            # (z, y, x, 4)
    s = oracle_state_from(sim.read_state(), vol, mat_ids)
    cfg = orc.config(res, 1.0 / res)
    og, st = orc.p2g(cfg, om_list, s, dt)
    assert st == 0
    lo, dim = og.lo, og.dim
    ref_m = np.zeros((res, res, res))
    ref_p = np.zeros((res, res, res, 3))
    ref_m[lo[2]:lo[2] + dim[2], lo[1]:lo[1] + dim[1], lo[0]:lo[0] + dim[0]] = og.mass()
    ref_p[lo[2]:lo[2] + dim[2], lo[1]:lo[1] + dim[1], lo[0]:lo[0] + dim[0]] = og.mom()
    assert linf(g[..., 0], ref_m) <= tol * np.abs(ref_m).max()
    assert linf(g[..., 1:], ref_p) <= tol * np.abs(ref_p).max()
    rho = np.array([m.rho for m in om_list])
    mass_p = float((rho[s.mat] * s.vol).sum())
    assert abs(g[..., 0].sum() - mass_p) <= 1e-6 * mass_p


@pytest.mark.parametrize("variant", list(range(16)))
def test_p2g_grid_small_elastic(M, variant):
    x = scenes.cube_uniform(0, 8192, 0.4, 0.6)
    vol = 0.008 / 8192
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    with M.Simulator(64, 1 / 64, [gm], p2g_variant=variant) as sim:
        sim.add_particles(x, vol=np.full(len(x), vol, np.float32))
        _p2g_parity(M, sim, [gm], [om], x, vol, 1e-4, 64)


@pytest.mark.parametrize("variant", list(range(16)))
def test_p2g_grid_ragged_tail(M, variant):
    """A particle count that is no multiple of a chunk (4, 8), a warp, a
    batch of the node-parallel form or a CTA: the last thread's, warp's and
    CTA's ranges end early."""
    n = 8192 - 3
    x = scenes.cube_uniform(3, n, 0.4, 0.6)
    vol = 0.008 / n
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    with M.Simulator(64, 1 / 64, [gm], p2g_variant=variant) as sim:
        sim.add_particles(x, vol=np.full(len(x), vol, np.float32))
        _p2g_parity(M, sim, [gm], [om], x, vol, 1e-4, 64)


@pytest.mark.parametrize("kind", ["snow", "fluid", "sand"])
def test_p2g_grid_materials(M, kind):
    kw = dict(snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, rho=400.0), fluid=dict(kind=M.FLUID, E=1e4, rho=1000.0),
              sand=dict(kind=M.SAND, E=3.5e5, nu=0.3, rho=2200.0))[kind]
    k = kw.pop("kind")
    gm, om = mats_pair(M, k, **kw)
    x, _ = scenes.blocks(11, 20000, 64, 2)
    vol = (1 / 64) ** 3 / 8
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP) as sim:
        sim.add_particles(x)
        if k == M.FLUID:
            sim.write_state(Jp=torch.full((len(x),), 0.97, device="cuda"))
        _p2g_parity(M, sim, [gm], [om], x, vol, 1e-4, 64)


@pytest.mark.parametrize("variant", list(range(16)))
def test_p2g_grid_snow_full_size(M, variant):
    x, _ = scenes.snow_blocks()
    vol = (1 / 256) ** 3 / 8
    gm, om = mats_pair(M, M.SNOW, E=1.4e5, nu=0.2, rho=400.0)
    with M.Simulator(256, 1 / 256, [gm], boundary=M.SLIP, p2g_variant=variant) as sim:
        sim.add_particles(torch.from_numpy(x).cuda())
        _p2g_parity(M, sim, [gm], [om], x, vol, 5e-5, 256)


# ------------------------------------------------------------- whole substeps

def _run_both(M, sim, om_list, s, steps, dt, cfg):
    sim.run(steps, dt)
    for _ in range(steps):
        assert orc.substep(cfg, om_list, s, dt) == 0
    return {k: v.double().cpu().numpy() for k, v in sim.read_state().items()}


def test_substeps_small_elastic(M):
    """The small elastic case: 8,192 particles, 64^3, E=1e4, nu=0.2, rho=1,
    dt=1e-4, sticky walls; 10 substeps within the stated tolerances, then the
    remaining 90 of its 100 substeps."""
    x = scenes.cube_uniform(0, 8192, 0.4, 0.6)
    vol = 0.008 / 8192
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.STICKY) as sim:
        sim.add_particles(x, vol=np.full(len(x), vol, np.float32))
        s = orc.State(x.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        g = _run_both(M, sim, [om], s, 90, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-3 * np.abs(s.v).max()


@pytest.mark.parametrize("kind", ["elastic", "snow", "fluid", "sand", "nacc", "nhsand"])
def test_substeps_materials(M, kind):
    kw = dict(elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2, rho=1000.0),
              snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0),
              fluid=dict(kind=M.FLUID, E=1e4, gamma=7.0, rho=1000.0),
              sand=dict(kind=M.SAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0),
              nacc=dict(kind=M.NACC, E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01),
              nhsand=dict(kind=M.NHSAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0))[kind]
    k = kw.pop("kind")
    gm, om = mats_pair(M, k, **kw)
    dt = 5e-5 if k == M.SNOW else 1e-4
    x, _ = scenes.blocks(13, 20000, 64, 2)
    vol = (1 / 64) ** 3 / 8
    rng = np.random.default_rng(3)
    n = len(x)
    v = (0.3 * rng.normal(size=(n, 3))).astype(np.float32)
    F = (np.eye(3) + 0.01 * rng.normal(size=(n, 3, 3))).astype(np.float32)
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP) as sim:
        sim.add_particles(x, v=v)
        if k != M.FLUID:
            sim.write_state(F=torch.from_numpy(F).cuda())
        s = oracle_state_from(sim.read_state(), vol)
        g = _run_both(M, sim, [om], s, 10, dt, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    if k != M.FLUID:
        assert linf(g["F"], s.F) <= 1e-4
    assert linf(g["Jp"], s.Jp) <= 1e-4


@pytest.mark.parametrize("kind", ["elastic", "snow", "fluid", "sand", "nacc", "nhsand"])
def test_asflip_substeps_match_oracle(M, kind):
    """ASFLIP transfer (alpha 0.95, beta 0 compressed / 1 otherwise, the
    usual weights) against the oracle over 10 substeps, random velocities and
    strains so that both beta branches occur; then 20 more substeps from CUDA
    graphs, where v is held to 1e-3 relative: the particle velocity carries
    alpha of its own past, FP32 rounding included, so the error grows with the
    substep count faster than under APIC (the fluid case reached 1.05e-4
    relative after 30).  The compressed-state test is the plain J < 1
    (margin 0) for elastic, snow and fluid.  The two sands and NACC snow run
    at a stated margin of 1e-4: their return maps leave particles at J = 1
    exactly (the sands every particle in tension, NACC every particle whose
    yield surface has shrunk to the origin, p0 = 0), on the plain test's
    threshold, where the rounding of det F decides in FP64 as in FP32 (at
    margin 0 NACC's positions differed by 2.4e-4 after 10 substeps)."""
    kw = dict(elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2, rho=1000.0),
              snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0),
              fluid=dict(kind=M.FLUID, E=1e4, gamma=7.0, rho=1000.0),
              sand=dict(kind=M.SAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0),
              nacc=dict(kind=M.NACC, E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9,
                        alpha0=-0.01),
              nhsand=dict(kind=M.NHSAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0))[kind]
    k = kw.pop("kind")
    gm, om = mats_pair(M, k, **kw)
    dt = 5e-5 if k == M.SNOW else 1e-4
    x, _ = scenes.blocks(14, 20000, 64, 2)
    vol = (1 / 64) ** 3 / 8
    rng = np.random.default_rng(4)
    n = len(x)
    v = (0.3 * rng.normal(size=(n, 3))).astype(np.float32)
    F = (np.eye(3) + 0.01 * rng.normal(size=(n, 3, 3))).astype(np.float32)
    margin = 1e-4 if k in (M.SAND, M.NHSAND, M.NACC) else 0.0
    flip = dict(flip_alpha=0.95, flip_beta_min=0.0, flip_beta_max=1.0, flip_compress_margin=margin)
    cfg = orc.config(64, 1 / 64, orc.SLIP, transfer=orc.ASFLIP, **flip)
    stream = torch.cuda.Stream()
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, transfer=M.ASFLIP, stream=stream, **flip) as sim:
        sim.add_particles(x, v=v)
        if k != M.FLUID:
            sim.write_state(F=torch.from_numpy(F).cuda())
        else:
            sim.write_state(Jp=torch.from_numpy(rng.uniform(0.99, 1.01, n).astype(np.float32)).cuda())
        s = oracle_state_from(sim.read_state(), vol)
        J = s.Jp if k == M.FLUID else np.linalg.det(s.F)
        assert (J < 1 - margin).mean() > 0.2 and (J >= 1 - margin).mean() > 0.2
        g = _run_both(M, sim, [om], s, 10, dt, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        if k != M.FLUID:
            assert linf(g["F"], s.F) <= 1e-4
        assert linf(g["Jp"], s.Jp) <= 1e-4
        sim.use_graphs(True)
        g = _run_both(M, sim, [om], s, 20, dt, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-3 * np.abs(s.v).max()
        assert sim.graph_launches > 0
        with pytest.raises(RuntimeError):
            sim.set_g2p2g(True)


def _expected_dt(om_list, cfg, starts, dts, reset, q, rem, cfl, dt_max, g=9.8):
    """The step rule of mpm_advance for global substep q, evaluated on the
    oracle's states (starts[k] = state at the start of substep k, dts[k] its
    step).  Speeds were last forgotten (context creation, an addition) before
    substep `reset`, where one reduction measured them.  The bound is the
    largest |v| at the start of substep q - 1 (what the G2P of q - 2
    reduced), grown by g dt_{q-1}, once q - 2 >= reset; before that it is the
    reduction's value grown by g dt_{q-1} per substep of age.  The remaining
    interval is then cut into equal steps."""
    if q - 2 >= reset:
        vb = np.linalg.norm(starts[q - 1].v, axis=1).max() + g * dts[q - 1]
    else:
        vb = np.linalg.norm(starts[reset].v, axis=1).max() + (q - reset) * g * (dts[q - 1] if q > reset else 0.0)
    dt = orc.cfl_dt(cfg, om_list, vb, cfl, dt_max)
    return rem if dt >= rem else rem / np.ceil(rem / dt)


@pytest.mark.parametrize("kind,fused,graphs,asflip", [("elastic", False, False, False), ("fluid", False, True, False),
                                                      ("elastic", True, True, False), ("fluid", False, True, True)])
def test_adaptive_dt_matches_oracle(M, kind, fused, graphs, asflip):
    """mpm_advance: the substep sizes follow the rule (within FP32 rounding of
    the speeds), each interval is covered exactly, and the state matches the
    oracle run with the same steps -- over three calls: a fresh context, a
    call that carries the speed bound over, and one after an addition (which
    forces a fresh reduction)."""
    kw = dict(elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2, rho=1000.0),
              fluid=dict(kind=M.FLUID, E=1e4, gamma=7.0, rho=1000.0))[kind]
    k = kw.pop("kind")
    gm, om = mats_pair(M, k, **kw)
    x, _ = scenes.blocks(15, 15000, 64, 2)
    rng = np.random.default_rng(5)
    v = (0.5 * rng.normal(size=(len(x), 3))).astype(np.float32)
    vol = (1 / 64) ** 3 / 8
    # two positional weights at the plain compressed-state test J < 1 (margin 0).  The
    # fluid's J crosses 1 continuously, so a particle within rounding of 1 may take the
    # other branch in FP32 than in FP64; that moves it by dt alpha |beta_max - beta_min|
    # |v - v0| and its neighbours' velocities by about |C| times that.  At these steps
    # (~7e-4 s, |C| ~ 10/s) weights 0.01 apart keep one such difference inside the
    # tolerance, while swapping the two branches, or one weight for all particles,
    # moves the velocities after the first call by 9.6e-4 / 4.8e-4 against a tolerance
    # of 1.1e-4 (measured with the oracle), so the decision is still checked.
    flip = dict(flip_alpha=0.95, flip_beta_min=0.49, flip_beta_max=0.5, flip_compress_margin=0.0) if asflip else {}
    cfg = orc.config(64, 1 / 64, orc.SLIP, transfer=orc.ASFLIP if asflip else orc.APIC, **flip)
    cfl, dt_max = 0.5, 5e-3
    starts, steps, reset, compressed = [], [], 0, []
    stream = torch.cuda.Stream()
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, g2p2g=fused, graphs=graphs, stream=stream,
                     transfer=M.ASFLIP if asflip else M.APIC, **flip) as sim:
        sim.add_particles(x, v=v)
        s = oracle_state_from(sim.read_state(), vol)
        for call, duration in enumerate((0.01, 0.0075, 0.0125)):
            if call == 2:
                x2 = scenes.cube_uniform(6, 400, 0.45, 0.55)
                v2 = np.tile(np.array([0.0, 2.0, 0.0], np.float32), (400, 1))
                sim.add_particles(x2, v=v2)
                s = orc.State(np.concatenate([s.x, x2]), np.concatenate([s.v, v2]),
                              np.concatenate([s.C, np.zeros((400, 3, 3))]),
                              np.concatenate([s.F, np.tile(np.eye(3), (400, 1, 1))]),
                              np.concatenate([s.Jp, np.ones(400)]), np.concatenate([s.vol, np.full(400, vol)]),
                              np.concatenate([s.mat, np.zeros(400, s.mat.dtype)]))
                reset = len(steps)
            dts = sim.advance(duration, cfl=cfl, dt_max=dt_max)
            assert len(dts) >= 4
            assert abs(float(np.sum(dts.astype(np.float64))) - duration) <= 1e-6 * duration
            t = 0.0
            for dt in dts:
                q = len(steps)
                starts.append(s.copy())
                want = _expected_dt([om], cfg, starts, steps, reset, q, duration - t, cfl, dt_max)
                assert abs(float(dt) - want) <= 1e-4 * want, (call, q, float(dt), want)
                compressed.append((s.Jp < 1.0).mean())
                steps.append(float(dt))
                t += float(dt)
                assert orc.substep(cfg, om, s, float(dt)) == 0
            assert dts.max() < dt_max      # the speed bound, not the cap, set the steps
            g = {key: val.double().cpu().numpy() for key, val in sim.read_state().items()}
            assert linf(g["x"], s.x) <= 1e-4
            assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        if graphs:   # steps of new sizes update the captured graphs instead of dropping them
            assert sim.graph_launches >= 10
        if asflip and kind == "fluid":   # both branches of the compressed-state test were taken
            assert max(compressed) > 0.2 and min(compressed) < 0.05


@pytest.mark.parametrize("g2p", [0, 4])
def test_mixed_materials_match_oracle(M, g2p):
    """One scene with all six material kinds, one per block of particles (the
    generic kernels, which read each particle's material index), against the
    oracle over 10 substeps."""
    specs = [(M.ELASTIC, dict(E=1e4, nu=0.2, rho=1000.0)),
             (M.SNOW, dict(E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0)),
             (M.FLUID, dict(E=1e4, gamma=7.0, rho=1000.0)),
             (M.SAND, dict(E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0)),
             (M.NACC, dict(E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9, alpha0=-0.01)),
             (M.NHSAND, dict(E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0))]
    gms = [M.material(k, **kw) for k, kw in specs]
    oms = [orc.material(k, **kw) for k, kw in specs]
    rng = np.random.default_rng(8)
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    xs, vs, ms = [], [], []
    with M.Simulator(64, 1 / 64, gms, boundary=M.SLIP, g2p_variant=g2p) as sim:
        for i in range(len(specs)):
            lo = np.array([0.1 + 0.13 * i, 0.2, 0.3])
            x = (lo + 0.1 * rng.random((1500, 3))).astype(np.float32)
            v = (0.3 * rng.normal(size=(1500, 3))).astype(np.float32)
            sim.add_particles(x, v=v, material=i)
            xs.append(x), vs.append(v), ms.append(np.full(1500, i, np.int32))
        n = sim.n
        F = (np.eye(3) + 0.01 * rng.normal(size=(n, 3, 3))).astype(np.float32)
        F[np.concatenate(ms) == 2] = np.eye(3)            # the fluid tracks J, not F
        sim.write_state(F=torch.from_numpy(F).cuda())
        s = oracle_state_from(sim.read_state(), vol, np.concatenate(ms))
        g = _run_both(M, sim, oms, s, 10, 5e-5, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["F"], s.F) <= 1e-4
    assert linf(g["Jp"], s.Jp) <= 1e-4


@pytest.mark.parametrize("p2g,g2p,aosoa,warps,resort", [(3, 4, False, 4, 0), (15, 7, True, 4, 0), (4, 7, True, 2, 4)])
def test_ten_substeps_snow_full_size_bench_configuration(M, p2g, g2p, aosoa, warps, resort):
    """The 1.34M-particle snow scene in the launch configurations bench.py's
    autotuner ends on (register runs in storage or base-cell order, the
    64-register G2P with the weights in registers or shared memory, SoA or
    AoSoA store, 2 or 4 warps per CTA, window re-sorts or none; CUDA-graph
    replay on a side stream): x and v after 10 substeps within 1e-4 of the
    FP64 oracle."""
    x, _ = scenes.snow_blocks()
    vol = (1 / 256) ** 3 / 8
    gm, om = mats_pair(M, M.SNOW, E=1.4e5, nu=0.2, rho=400.0)
    cfg = orc.config(256, 1 / 256, orc.SLIP)
    rng = np.random.default_rng(9)
    v = (0.2 * rng.normal(size=(len(x), 3))).astype(np.float32)
    stream = torch.cuda.Stream()
    with M.Simulator(256, 1 / 256, [gm], boundary=M.SLIP, stream=stream, p2g_variant=p2g, g2p_variant=g2p,
                     graphs=True, resort_interval=resort) as sim:
        sim.set_cta_warps(warps)
        sim.set_layout(aosoa)
        sim.add_particles(torch.from_numpy(x).cuda(), v=torch.from_numpy(v).cuda())
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 5e-5, cfg)
        assert sim.graph_launches >= 8
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["C"], s.C) <= 1e-4 * np.abs(s.C).max()
    assert linf(g["F"], s.F) <= 1e-5
    assert linf(g["Jp"], s.Jp) <= 1e-5


def test_rebuild_is_triggered_and_parity_holds(M):
    """A fast block crosses several cells: the free-zone test must request
    rebuilds, and the result still matches the oracle."""
    x = scenes.cube_uniform(4, 3000, 0.3, 0.4)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    v = np.tile(np.array([30.0, 20.0, 10.0], np.float32), (len(x), 1))
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP) as sim:
        sim.add_particles(x, v=v)
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 60, 1e-4, cfg)
        stats = sim.stats()
    assert stats["rebuilds"] >= 3, stats
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()


# ---------------------------------------------------------------- edge cases

def test_empty_and_ragged_sizes(M):
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    with M.Simulator(32, 1 / 32, [gm]) as sim:
        sim.run(3, 1e-4)                          # no particles: a no-op
        assert sim.n == 0
        assert sim.read_state()["x"].shape == (0, 3)
    cfg = orc.config(32, 1 / 32, orc.STICKY)
    for n in (1, 31, 127, 129, 2049):
        x = scenes.cube_uniform(n, n, 0.35, 0.65)
        with M.Simulator(32, 1 / 32, [gm]) as sim:
            sim.add_particles(x, vol=np.full(n, 1e-6, np.float32))
            s = orc.State(x.astype(np.float64), vol=1e-6)
            g = _run_both(M, sim, [om], s, 5, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4, n
        assert linf(g["v"], s.v) <= 1e-4 * max(np.abs(s.v).max(), 1e-12), n


@pytest.mark.parametrize("res", [(1024, 1024, 1024), (1024, 16, 512)])
def test_maximum_grid_far_corner(M, res):
    """The largest grid the key layout allows (1024 nodes per axis: 8 Morton
    bits per axis, 30-bit keys) and a flat, non-cubic one, with a cluster
    against the far corner's walls moving into them: parity with the oracle
    over 10 substeps."""
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    dx = 1 / 1024
    hi = np.array(res) * dx
    rng = np.random.default_rng(21)
    x = (hi - 0.012 + 0.008 * rng.random((3000, 3))).astype(np.float32)
    v = np.tile(np.array([0.5, 0.5, 0.5], np.float32), (3000, 1))
    vol = dx ** 3 / 8
    cfg = orc.config(list(res), dx, orc.STICKY)
    with M.Simulator(list(res), dx, [gm], boundary=M.STICKY) as sim:
        sim.add_particles(x, v=v, vol=np.full(3000, vol, np.float32))
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()


def test_growth_insertion_order_and_capacity(M):
    gm = M.material(M.ELASTIC)
    xs = [scenes.cube_uniform(i, m, 0.3, 0.7) for i, m in enumerate((100, 1000, 5000))]
    with M.Simulator(64, 1 / 64, [gm]) as sim:
        sim.add_particles(xs[0])
        sim.rebuild()
        sim.add_particles(torch.from_numpy(xs[1]).cuda())
        sim.rebuild()
        sim.add_particles(xs[2])
        caps = sim.stats()["particle_capacity"]
        assert caps >= 4 * 6100 - 256
        out = sim.read_state(("x",))["x"].cpu().numpy()
        np.testing.assert_array_equal(out, np.concatenate(xs))
        sim.rebuild()
        np.testing.assert_array_equal(sim.read_state(("x",))["x"].cpu().numpy(), np.concatenate(xs))
    with M.Simulator(64, 1 / 64, [gm], max_particles=500) as sim:
        sim.add_particles(xs[0])
        with pytest.raises(M.MpmError) as e:
            sim.add_particles(xs[1])
        assert e.value.status == 3                 # MPM_ECAPACITY


def test_domain_and_nonfinite_errors(M):
    gm = M.material(M.ELASTIC)
    with M.Simulator(32, 1 / 32, [gm]) as sim:
        sim.add_particles(np.array([[0.001, 0.5, 0.5], [0.5, 0.5, 0.5]], np.float32))
        sim.substep(1e-4)
        with pytest.raises(M.MpmError) as e:
            sim.sync()
        assert e.value.status == 4                 # MPM_EDOMAIN
    with M.Simulator(32, 1 / 32, [gm]) as sim:
        sim.add_particles(np.array([[0.5, 0.5, 0.5]], np.float32), v=np.array([[np.nan, 0, 0]], np.float32))
        sim.run(2, 1e-4)
        with pytest.raises(M.MpmError) as e:
            sim.sync()
        assert e.value.status == 5                 # MPM_ENONFINITE


def test_advance_reports_a_nan_velocity_before_stepping(M):
    """One NaN velocity among finite ones: the speed reduction behind
    mpm_advance carries the NaN to the host (a plain float max would drop it
    and size the step from the other particles), so the call fails with
    MPM_ENONFINITE before it runs a substep."""
    gm = M.material(M.ELASTIC)
    x = scenes.cube_uniform(9, 2000, 0.4, 0.6)
    v = np.zeros((len(x), 3), np.float32)
    v[1234, 1] = np.nan
    with M.Simulator(64, 1 / 64, [gm]) as sim:
        sim.add_particles(x, v=v)
        with pytest.raises(M.MpmError) as e:
            sim.advance(1e-3, cfl=0.5, dt_max=1e-4)
        assert e.value.status == 5                 # MPM_ENONFINITE
        assert sim.stats()["substeps"] == 0


def test_host_buffers_and_side_stream(M):
    x = scenes.cube_uniform(3, 4000, 0.4, 0.6)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with M.Simulator(64, 1 / 64, [gm], stream=stream) as sim:
            sim.add_particles(x, vol=np.full(len(x), 1e-6, np.float32))
            sim.run(5, 1e-4)
            host = {k: torch.empty(s, dtype=torch.float32).pin_memory()
                    for k, s in (("x", (len(x), 3)), ("v", (len(x), 3)))}
            sim.read_state_into(x=host["x"], v=host["v"])
    s = orc.State(x.astype(np.float64), vol=1e-6)
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    for _ in range(5):
        orc.substep(cfg, om, s, 1e-4)
    assert linf(host["x"].numpy(), s.x) <= 1e-4
    assert linf(host["v"].numpy(), s.v) <= 1e-4 * np.abs(s.v).max()


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 9, 10, 11, 12, 13, 14, 15])
def test_p2g_sparse_cloud_tile_fallback(M, variant):
    """Particles spread over the whole domain: each 256-particle tile's box is
    far larger than the shared-memory tile, so the tile variants take their
    direct-atomics fallback (and the warp-level reduction finds no groups);
    results must not change."""
    x = scenes.cube_uniform(21, 5000, 0.1, 0.9)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    vol = (1 / 64) ** 3 / 8
    with M.Simulator(64, 1 / 64, [gm], p2g_variant=variant) as sim:
        sim.add_particles(x)
        _p2g_parity(M, sim, [gm], [om], x, vol, 1e-4, 64)


def test_autotuner_picks_a_variant_and_keeps_parity(M):
    from paper_2111_00699_gb300 import _lib, tune
    x = scenes.cube_uniform(0, 8192, 0.4, 0.6)
    vol = 0.008 / 8192
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    with M.Simulator(64, 1 / 64, [gm]) as sim:
        sim.add_particles(x, vol=np.full(len(x), vol, np.float32))
        res = tune.tune_p2g(sim, 1e-4, steps=2, rounds=1, refine_top=2, refine_steps=3, drift=2)
        assert res["best"] in range(len(_lib.P2G_VARIANTS)) and len(res["ms"]) == len(_lib.P2G_VARIANTS)
        assert len(res["refined_ms"]) == 2 and _lib.P2G_VARIANTS[res["best"]] in res["refined_ms"]
        assert all(v > 0 for v in res["ms"].values())
        res = tune.tune_g2p(sim, 1e-4, steps=2, rounds=1)
        assert res["best"] in range(len(_lib.G2P_VARIANTS)) and len(res["ms"]) == len(_lib.G2P_VARIANTS)
        assert all(v > 0 for v in res["ms"].values())
        res = tune.tune_order(sim, 1e-4, [(4, 2), (15, 0), (4, 2)], slice_steps=3, rounds=2)
        assert res["best"] in ((4, 2), (15, 0)) and len(res["ms"]) == 2
        assert all(v > 0 for v in res["ms"].values())
        ran = sim.stats()["substeps"]
        s = orc.State(x.astype(np.float64), vol=vol)
        for _ in range(ran):
            orc.substep(cfg, om, s, 1e-4)
        g = {k: v.double().cpu().numpy() for k, v in sim.read_state().items()}
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()


@pytest.mark.parametrize("p2g,g2p", [(0, 0), (1, 1), (2, 2), (3, 1), (4, 2), (4, 0), (3, 3), (4, 4), (5, 0), (6, 4), (3, 5),
                                     (5, 5), (7, 4), (3, 6), (8, 4), (9, 4), (10, 0), (11, 4), (4, 7), (12, 7), (13, 4), (14, 4), (15, 7)])
def test_substeps_variant_combinations(M, p2g, g2p):
    """Every P2G / G2P launch variant computes the same substep (10 substeps
    of a moving, deforming elastic block against the oracle)."""
    x, _ = scenes.blocks(17, 12000, 64, 2)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    rng = np.random.default_rng(5)
    v = (0.5 * rng.normal(size=(len(x), 3))).astype(np.float32)
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, p2g_variant=p2g, g2p_variant=g2p) as sim:
        sim.add_particles(x, v=v)
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["C"], s.C) <= 1e-4 * np.abs(s.C).max()


@pytest.mark.parametrize("warps", [2, 8])
def test_cta_warps_keep_parity(M, warps):
    """The register-run P2G (runs of 8, then 4) and the 64-register G2P in
    CTAs of 2 or 8 warps compute the same substeps (10 + 10 against the
    oracle); other warp counts are refused."""
    x, _ = scenes.blocks(17, 12000, 64, 2)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    rng = np.random.default_rng(5)
    v = (0.5 * rng.normal(size=(len(x), 3))).astype(np.float32)
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, p2g_variant=4, g2p_variant=4) as sim:
        sim.add_particles(x, v=v)
        with pytest.raises(M.MpmError):
            sim.set_cta_warps(3)
        sim.set_cta_warps(warps)
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        sim.set_p2g_variant(3)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        assert linf(g["C"], s.C) <= 1e-4 * np.abs(s.C).max()


def test_aosoa_layout_keeps_parity(M):
    """The AoSoA particle store (packets of 32): converted from SoA mid-run,
    10 substeps against the oracle, particles added under AoSoA (capacity
    growth and a rebuild), 10 more, converted back, 10 more; the state reads
    back in insertion order throughout (the node-parallel P2G for 5 of the
    substeps).  Forms AoSoA lacks are refused."""
    x, _ = scenes.blocks(17, 12000, 64, 2)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    rng = np.random.default_rng(6)
    v = (0.5 * rng.normal(size=(len(x), 3))).astype(np.float32)
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, p2g_variant=4, g2p_variant=4) as sim:
        sim.add_particles(x, v=v)
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 3, 1e-4, cfg)
        sim.set_layout(True)
        for bad in (lambda: sim.set_p2g_variant(0), lambda: sim.set_g2p_variant(0), lambda: sim.set_g2p2g(True),
                    lambda: sim.set_cta_warps(8)):
            with pytest.raises(M.MpmError):
                bad()
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        x2 = scenes.cube_uniform(7, 30000, 0.3, 0.5)
        sim.add_particles(x2)
        s = orc.State(np.concatenate([s.x, x2]), np.concatenate([s.v, np.zeros((len(x2), 3))]),
                      np.concatenate([s.C, np.zeros((len(x2), 3, 3))]),
                      np.concatenate([s.F, np.tile(np.eye(3), (len(x2), 1, 1))]),
                      np.concatenate([s.Jp, np.ones(len(x2))]), vol)
        sim.set_p2g_variant(3)
        sim.set_cta_warps(2)   # the AoSoA kernels in CTAs of 2 warps
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        sim.set_cta_warps(4)
        sim.set_p2g_variant(14)   # the node-parallel runs on the AoSoA store
        g = _run_both(M, sim, [om], s, 5, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        sim.set_layout(False)
        sim.set_p2g_variant(0)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        assert linf(g["C"], s.C) <= 1e-4 * np.abs(s.C).max()


@pytest.mark.parametrize("kind,g2p", [("snow", 7), ("fluid", 7), ("sand", 7), ("nacc", 7), ("snow", 6), ("elastic", 4)])
def test_aosoa_material_kinds(M, kind, g2p):
    """The AoSoA store with the kernels specialised to one material kind (G2P
    at 64 registers with the weights in shared memory or in registers, or at
    48 registers; P2G register runs of 4): 10 substeps against the oracle,
    random velocities and strains so that the return maps act."""
    kw = dict(snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, rho=400.0, theta_c=2.5e-2, theta_s=7.5e-3, hardening=10.0),
              fluid=dict(kind=M.FLUID, E=1e4, gamma=7.0, rho=1000.0),
              sand=dict(kind=M.SAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0),
              nacc=dict(kind=M.NACC, E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9,
                        alpha0=-0.01),
              elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2, rho=1000.0))[kind]
    k = kw.pop("kind")
    gm, om = mats_pair(M, k, **kw)
    dt = 5e-5 if k == M.SNOW else 1e-4
    x, _ = scenes.blocks(23, 15000, 64, 2)
    vol = (1 / 64) ** 3 / 8
    rng = np.random.default_rng(9)
    n = len(x)
    v = (0.3 * rng.normal(size=(n, 3))).astype(np.float32)
    F = (np.eye(3) + 0.01 * rng.normal(size=(n, 3, 3))).astype(np.float32)
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, p2g_variant=3, g2p_variant=g2p) as sim:
        sim.add_particles(x, v=v)
        if k != M.FLUID:
            sim.write_state(F=torch.from_numpy(F).cuda())
        sim.set_layout(True)
        s = oracle_state_from(sim.read_state(), vol)
        g = _run_both(M, sim, [om], s, 10, dt, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    if k != M.FLUID:
        assert linf(g["F"], s.F) <= 1e-4
    assert linf(g["Jp"], s.Jp) <= 1e-4


# ------------------------------------------------------------- emission (a7)

@pytest.mark.parametrize("asflip", [False, True])
def test_fountain_emission_parity(M, asflip):
    """Fountain: weakly compressible fluid (K = 1e4, gamma = 7, rho = 1000)
    emitted through a disk inlet (r = 0.05, 3 m/s up) every substep on a 128^3
    grid, dt = 1e-4, with APIC or with the ASFLIP transfer the paper's
    fountain uses.  The oracle gets the same particles appended before each
    substep.  Emission must not force a rebuild every substep."""
    res, dt, steps = 128, 1e-4, 200
    vol = (1 / res) ** 3 / 8
    gm, om = mats_pair(M, M.FLUID, E=1e4, gamma=7.0, rho=1000.0)
    flip = dict(flip_alpha=0.95, flip_beta_min=0.0, flip_beta_max=1.0) if asflip else {}
    cfg = orc.config(res, 1 / res, orc.SLIP, transfer=orc.ASFLIP if asflip else orc.APIC, **flip)
    s = None
    with M.Simulator(res, 1 / res, [gm], boundary=M.SLIP, transfer=M.ASFLIP if asflip else M.APIC, **flip) as sim:
        for k in range(steps):
            xe, ve = scenes.fountain_batch(2, k, dt, vol)
            sim.emit_particles(xe, v=ve)
            ne = len(xe)
            add = orc.State(xe.astype(np.float64), ve.astype(np.float64), vol=vol)
            if s is None:
                s = add
            else:
                s = orc.State(np.concatenate([s.x, add.x]), np.concatenate([s.v, add.v]),
                              np.concatenate([s.C, add.C]), np.concatenate([s.F, add.F]),
                              np.concatenate([s.Jp, add.Jp]), np.concatenate([s.vol, add.vol]),
                              np.concatenate([s.mat, add.mat]))
            sim.substep(dt)
            assert orc.substep(cfg, om, s, dt) == 0
        g = {k: v.double().cpu().numpy() for k, v in sim.read_state().items()}
        stats = sim.stats()
    assert g["x"].shape == s.x.shape and ne == 40
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["Jp"], s.Jp) <= 1e-4
    assert stats["rebuilds"] <= steps // 4, stats


def test_fountain_full_budget_properties(M):
    """The whole fountain run bench.py times (3,600 emitting substeps up to
    144,000 particles, 128^3): too long for the oracle, so properties that
    hold at any size -- every emitted particle is there, in insertion order,
    finite and inside the walls, and P2G of the final state conserves mass
    to 1e-6."""
    res, dt, steps = 128, 1e-4, 3600
    vol = (1 / res) ** 3 / 8
    gm = M.material(M.FLUID, E=1e4, gamma=7.0, rho=1000.0)
    first = None
    total = 0
    stream = torch.cuda.Stream()
    with M.Simulator(res, 1 / res, [gm], boundary=M.SLIP, stream=stream) as sim:
        for k in range(steps):
            xe, ve = scenes.fountain_batch(2, k, dt, vol)
            if first is None:
                first = xe.copy()
            total += len(xe)
            sim.emit_particles(xe, v=ve)
            sim.substep(dt)
        st = sim.read_state()
        g = sim.debug_p2g(dt).double()
        n = sim.n
    assert n == total == 144000
    x = st["x"].double().cpu().numpy()
    assert np.isfinite(x).all() and np.isfinite(st["v"].cpu().numpy()).all()
    assert x.min() > 3 / res and x.max() < 1 - 3 / res
    # insertion order: the first batch rose from the inlet, still above it
    assert np.abs(x[: len(first), [0, 2]] - 0.5).max() < 0.45
    mass = 1000.0 * vol * n
    assert abs(float(g[..., 0].sum()) - mass) <= 1e-6 * mass


def test_sand_blocks_full_size_parity(M):
    """Drucker-Prager sand (phi = 30 deg, E = 3.5e5, nu = 0.3, rho = 2200), 4
    boxes, ~500K particles at 8 per cell on 128^3, dt = 1e-4, 10 substeps."""
    x, _ = scenes.sand_blocks()
    res = 128
    vol = (1 / res) ** 3 / 8
    gm, om = mats_pair(M, M.SAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0)
    cfg = orc.config(res, 1 / res, orc.SLIP)
    rng = np.random.default_rng(31)
    v = (0.5 * rng.normal(size=(len(x), 3))).astype(np.float32)
    with M.Simulator(res, 1 / res, [gm], boundary=M.SLIP) as sim:
        sim.add_particles(torch.from_numpy(x).cuda(), v=torch.from_numpy(v).cuda())
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["F"], s.F) <= 1e-4


# ------------------------------------------------------------ fused G2P2G (a6')

def test_graph_replay_matches_oracle(M):
    """Separate substeps replayed from CUDA graphs: parity through rebuilds
    (a fast block crosses many cells), a dt change and a particle addition,
    each of which drops the graphs; replays actually happen."""
    x = scenes.cube_uniform(4, 3000, 0.3, 0.4)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    v = np.tile(np.array([30.0, 20.0, 10.0], np.float32), (len(x), 1))
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    stream = torch.cuda.Stream()
    s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, stream=stream, graphs=True) as sim:
        sim.add_particles(x, v=v)
        for steps, dt in ((30, 1e-4), (20, 7e-5)):
            g = _run_both(M, sim, [om], s, steps, dt, cfg)
            assert linf(g["x"], s.x) <= 1e-4
            assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        x2 = scenes.cube_uniform(5, 500, 0.6, 0.65)
        sim.add_particles(x2)
        s = orc.State(np.concatenate([s.x, x2.astype(np.float64)]), np.concatenate([s.v, np.zeros((500, 3))]),
                      np.concatenate([s.C, np.zeros((500, 3, 3))]), np.concatenate([s.F, np.tile(np.eye(3), (500, 1, 1))]),
                      np.concatenate([s.Jp, np.ones(500)]), np.concatenate([s.vol, np.full(500, vol)]),
                      np.concatenate([s.mat, np.zeros(500, s.mat.dtype)]))
        g = _run_both(M, sim, [om], s, 20, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        assert sim.graph_launches >= 50
        assert sim.stats()["rebuilds"] >= 3
    with pytest.raises(RuntimeError):
        M.Simulator(64, 1 / 64, [gm], stream=torch.cuda.default_stream(), graphs=True)


@pytest.mark.parametrize("graphs", [False, True])
def test_window_resort_matches_oracle(M, graphs):
    """Window re-sorts every 2 substeps, then none, then every 3 (with and
    without graph replay, whose graphs are keyed by the particle buffer a
    re-sort switches to): the substeps match the oracle, the state reads back
    in insertion order, and rebuilds still happen when a fast block leaves its
    mapped blocks."""
    x = scenes.cube_uniform(4, 3000, 0.3, 0.4)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    rng = np.random.default_rng(13)
    v = (np.array([30.0, 20.0, 10.0]) + 3.0 * rng.normal(size=(len(x), 3))).astype(np.float32)
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, stream=torch.cuda.Stream(), graphs=graphs,
                     resort_interval=2) as sim:
        sim.add_particles(x, v=v)
        g = _run_both(M, sim, [om], s, 20, 1e-4, cfg)
        assert linf(g["x"], s.x) <= 1e-4
        sim.set_resort_interval(0)   # off, then every 3 substeps
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        sim.set_resort_interval(3)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        with pytest.raises(M.MpmError):
            sim.set_resort_interval(-1)
        stats = sim.stats()
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["F"], s.F) <= 1e-4
    assert stats["rebuilds"] >= 2


@pytest.mark.parametrize("pattern", [0, 1, 2, 3])
def test_red_rate_probe_applies_every_reduction(M, pattern):
    """The L2 reduction-rate probe: every one of threads x reductions float4
    additions of (1, 1, 1, 1) lands in the grid (all four components sum to
    the count), spread over the spans its sequence picks; four lanes per node
    touch nodes 0-7 of a span, one node per lane or per warp only node 0."""
    nodes, threads, reds = 32 * 1024, 32 * 300, 7
    grid = torch.zeros((nodes, 4), dtype=torch.float32, device="cuda")
    M.debug_red_rate(grid, threads, reds, pattern)
    torch.cuda.synchronize()
    g = grid.double().cpu().numpy()
    for c in range(4):
        assert g[:, c].sum() == threads * reds
    assert np.all(g[:, 0] == g[:, 3])
    touched = (g[:, 3] > 0).reshape(-1, 32)
    if pattern == 1:
        assert not touched[:, 8:].any()          # lanes l / 4: nodes 0-7 of a span
    if pattern >= 2:
        assert not touched[:, 1:].any()          # node 0 of a span only
    assert touched.any(axis=1).sum() > 100       # many spans
    with pytest.raises(ValueError):
        M.debug_red_rate(grid[:, :3], threads, reds, pattern)


def test_bounded_wait_times_out_and_device_stays_usable(M):
    """Failure detection without a fault: a device wait on an mbarrier that no
    copy completes gives up after its iteration limit and reports
    MPM_ETIMEOUT; the device then runs a normal substep."""
    from paper_2111_00699_gb300 import _lib
    assert M.debug_wait_timeout(1000) == _lib.MPM_ETIMEOUT
    assert M.debug_wait_timeout(0) == _lib.MPM_EINVAL
    x = scenes.cube_uniform(0, 2048, 0.4, 0.6)
    with M.Simulator(64, 1 / 64, [M.material(M.ELASTIC, E=1e4, nu=0.2, rho=1.0)]) as sim:
        sim.add_particles(x)
        sim.run(3, 1e-4)
        sim.sync()
        assert np.isfinite(sim.read_state()["x"].cpu().numpy()).all()


def test_no_sort_ablation_matches_oracle(M):
    """With no_sort = 1 the rebuild maps blocks but leaves the particles in
    their (here shuffled) storage order: the substeps are the same up to
    summation order, and the state still reads back in insertion order."""
    rng = np.random.default_rng(12)
    x = scenes.cube_uniform(0, 8192, 0.4, 0.6)
    x = x[rng.permutation(len(x))]
    vol = 0.008 / 8192
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1.0)
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    with M.Simulator(64, 1 / 64, [gm], no_sort=True) as sim:
        sim.add_particles(x, vol=np.full(len(x), vol, np.float32))
        s = orc.State(x.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, 1e-4, cfg)
        with pytest.raises(RuntimeError):
            sim.read_order()
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()


@pytest.mark.parametrize("scatter", [0, 3, 4, 7, 9, 10])
@pytest.mark.parametrize("kind", ["elastic", "snow", "fluid", "sand", "nacc", "nhsand"])
def test_g2p2g_matches_oracle(M, kind, scatter):
    """The fused transfer computes the same substeps as the separate phases,
    with each scatter form (thread per particle; register runs of 4 and 8;
    runs of 4 in shared memory; the warp-level reduction over cell groups
    and over runs of lanes)."""
    kw = dict(elastic=dict(kind=M.ELASTIC, E=1e4, nu=0.2, rho=1000.0),
              snow=dict(kind=M.SNOW, E=1.4e5, nu=0.2, rho=400.0),
              fluid=dict(kind=M.FLUID, E=1e4, gamma=7.0, rho=1000.0),
              sand=dict(kind=M.SAND, E=3.5e5, nu=0.3, rho=2200.0),
              nacc=dict(kind=M.NACC, E=5e4, nu=0.3, rho=400.0, hardening=5.0, friction_M=0.8, cohesion=0.9,
                        alpha0=-0.01),
              nhsand=dict(kind=M.NHSAND, E=3.5e5, nu=0.3, rho=2200.0, friction_deg=30.0))[kind]
    k = kw.pop("kind")
    gm, om = mats_pair(M, k, **kw)
    dt = 5e-5 if k == M.SNOW else 1e-4
    x, _ = scenes.blocks(19, 15000, 64, 2)
    vol = (1 / 64) ** 3 / 8
    rng = np.random.default_rng(8)
    v = (0.3 * rng.normal(size=(len(x), 3))).astype(np.float32)
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, g2p2g=True, p2g_variant=scatter) as sim:
        sim.add_particles(x, v=v)
        s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
        g = _run_both(M, sim, [om], s, 10, dt, cfg)
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
    assert linf(g["C"], s.C) <= 1e-4 * np.abs(s.C).max()
    assert linf(g["Jp"], s.Jp) <= 1e-4


@pytest.mark.parametrize("graphs", [False, True])
def test_g2p2g_rebuilds_switches_and_reads(M, graphs):
    """Fused mode with a fast block (rebuilds through the two-cell margin),
    switching to separate phases and back mid-run, and reading the state in
    between: every segment matches the oracle, with and without graph replay
    of both modes."""
    x = scenes.cube_uniform(4, 3000, 0.3, 0.4)
    gm, om = mats_pair(M, M.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    v = np.tile(np.array([30.0, 20.0, 10.0], np.float32), (len(x), 1))
    vol = (1 / 64) ** 3 / 8
    cfg = orc.config(64, 1 / 64, orc.SLIP)
    s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=vol)
    with M.Simulator(64, 1 / 64, [gm], boundary=M.SLIP, g2p2g=True, stream=torch.cuda.Stream(), graphs=graphs) as sim:
        sim.add_particles(x, v=v)
        for fused, steps in ((True, 25), (False, 10), (True, 25)):
            sim.set_g2p2g(fused)
            g = _run_both(M, sim, [om], s, steps, 1e-4, cfg)
            assert linf(g["x"], s.x) <= 1e-4
            assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()
        stats = sim.stats()
    assert stats["rebuilds"] >= 3, stats


def test_g2p2g_with_emission(M):
    """Emission between substeps in fused mode re-primes the momentum."""
    res, dt, steps = 128, 1e-4, 60
    vol = (1 / res) ** 3 / 8
    gm, om = mats_pair(M, M.FLUID, E=1e4, gamma=7.0, rho=1000.0)
    cfg = orc.config(res, 1 / res, orc.SLIP)
    s = None
    with M.Simulator(res, 1 / res, [gm], boundary=M.SLIP, g2p2g=True) as sim:
        for k in range(steps):
            xe, ve = scenes.fountain_batch(2, k, dt, vol)
            sim.emit_particles(xe, v=ve)
            add = orc.State(xe.astype(np.float64), ve.astype(np.float64), vol=vol)
            s = add if s is None else orc.State(np.concatenate([s.x, add.x]), np.concatenate([s.v, add.v]),
                                                np.concatenate([s.C, add.C]), np.concatenate([s.F, add.F]),
                                                np.concatenate([s.Jp, add.Jp]), np.concatenate([s.vol, add.vol]),
                                                np.concatenate([s.mat, add.mat]))
            sim.substep(dt)
            assert orc.substep(cfg, om, s, dt) == 0
        g = {k: v.double().cpu().numpy() for k, v in sim.read_state().items()}
    assert linf(g["x"], s.x) <= 1e-4
    assert linf(g["v"], s.v) <= 1e-4 * np.abs(s.v).max()


def test_ieee_build_matches_oracle():
    """The library built without fast-math intrinsics (the fast-math ablation)
    computes the same substeps: the small elastic and a snow case, in a child
    process that loads that build."""
    import subprocess
    import sys
    from paper_2111_00699_gb300 import build
    build.build(ieee=True)
    code = r"""
import numpy as np, torch, oracle as orc
from paper_2111_00699_gb300 import mpm, scenes, _lib
assert _lib.LIB_PATH.endswith("libmpm_ieee.so")
orc.build()
x = scenes.cube_uniform(0, 8192, 0.4, 0.6)
for kind, kw, dt in ((mpm.ELASTIC, dict(E=1e4, nu=0.2, rho=1.0), 1e-4),
                     (mpm.SNOW, dict(E=1.4e5, nu=0.2, rho=400.0), 5e-5)):
    rng = np.random.default_rng(3)
    v = (0.3 * rng.normal(size=x.shape)).astype(np.float32)
    with mpm.Simulator(64, 1 / 64, [mpm.material(kind, **kw)]) as sim:
        sim.add_particles(x, v=v, vol=np.full(len(x), 0.008 / 8192, np.float32))
        sim.run(10, dt)
        g = {k: t.double().cpu().numpy() for k, t in sim.read_state().items()}
    s = orc.State(x.astype(np.float64), v.astype(np.float64), vol=0.008 / 8192)
    for _ in range(10):
        assert orc.substep(orc.config(64, 1 / 64, orc.STICKY), [orc.material(kind, **kw)], s, dt) == 0
    assert np.abs(g["x"] - s.x).max() <= 1e-4
    assert np.abs(g["v"] - s.v).max() <= 1e-4 * np.abs(s.v).max()
print("ok")
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=dict(os.environ, MPM_LIBRARY="ieee"),
                       capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]


def test_fast_math_stress_error_against_ieee_and_oracle(M):
    """Fast-math acceptance in the paper's style (Sec. 4.3): the infinity norm
    of the stacked n x 3 x 3 Kirchhoff stresses of the fast-math build against
    the build without fast-math intrinsics and against the FP64 oracle, for
    random states on both constitutive paths (5 % and 1 % strain)."""
    import json
    import subprocess
    import sys
    import tempfile
    from paper_2111_00699_gb300 import build
    build.build(ieee=True)
    rng = np.random.default_rng(12)
    n = 4096
    kinds = {"elastic": dict(kind=M.ELASTIC, E=1e4, nu=0.2), "snow": dict(kind=M.SNOW, E=1.4e5, nu=0.2, hardening=10.0),
             "sand": dict(kind=M.SAND, E=3.5e5, nu=0.3), "nacc": dict(kind=M.NACC, E=5e4, nu=0.3, hardening=5.0),
             "nhsand": dict(kind=M.NHSAND, E=3.5e5, nu=0.3)}
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for scale in (0.05, 0.01):
        F = (np.eye(3) + scale * rng.normal(size=(n, 3, 3))).astype(np.float32)
        Jp = rng.uniform(0.95, 1.05, n).astype(np.float32)
        code = r"""
import json, sys, numpy as np, torch
from paper_2111_00699_gb300 import mpm, _lib
assert _lib.LIB_PATH.endswith("libmpm_ieee.so")
kinds = json.loads(%r)
F = torch.from_numpy(np.load(sys.argv[1])).cuda()
J = torch.from_numpy(np.load(sys.argv[2])).cuda()
out = {}
for name, kw in kinds.items():
    kw = dict(kw); k = kw.pop("kind")
    out[name] = mpm.debug_stress(mpm.material(k, **kw), F, J).double().cpu().numpy().tolist()
print(json.dumps(out))
""" % json.dumps(kinds)
        with tempfile.TemporaryDirectory() as tmp:
            fp, jp = os.path.join(tmp, "F.npy"), os.path.join(tmp, "J.npy")
            np.save(fp, F)
            np.save(jp, Jp)
            r = subprocess.run([sys.executable, "-c", code, fp, jp], cwd=root, env=dict(os.environ, MPM_LIBRARY="ieee"),
                               capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        ieee = json.loads(r.stdout.strip().splitlines()[-1])
        for name, kw in kinds.items():
            kw = dict(kw)
            k = kw.pop("kind")
            fast = M.debug_stress(M.material(k, **kw), torch.from_numpy(F).cuda(),
                                  torch.from_numpy(Jp).cuda()).double().cpu().numpy()
            ref = np.stack([orc.kirchhoff(orc.material(k, **kw), F[i].astype(np.float64), float(Jp[i]))
                            for i in range(n)])
            scale_ref = np.abs(ref).max()
            e_fast_ieee = linf(fast, np.array(ieee[name])) / scale_ref
            e_fast = linf(fast, ref) / scale_ref
            e_ieee = linf(np.array(ieee[name]), ref) / scale_ref
            print("stress %-7s strain %.2f  |fast-ieee|/|tau| %.2e  |fast-oracle| %.2e  |ieee-oracle| %.2e"
                  % (name, scale, e_fast_ieee, e_fast, e_ieee))
            assert e_fast <= 1e-4 and e_ieee <= 1e-4 and e_fast_ieee <= 1e-4
