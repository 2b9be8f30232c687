"""Differentiable rollout: the hand-written adjoint against the FP64 oracle's
adjoint and against FP64 finite differences (1e-3 relative)."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2111_00699_gb300 import scenes

pytestmark = pytest.mark.gpu

NU, RHO = 0.2, 1.0
TARGET = (0.5, 0.3, 0.5)


@pytest.fixture(scope="module")
def D():
    from paper_2111_00699_gb300 import build, diff
    build.build()
    assert torch.cuda.is_available()
    orc.build()
    return diff


def _jelly(n_side=32, seed=5):
    x, v = scenes.jelly_cube(seed, n_side=n_side)
    return x, v


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def test_diff_forward_matches_oracle(D):
    x, v = _jelly(12)
    n = len(x)
    rng = np.random.default_rng(1)
    E = rng.uniform(5e3, 2e4, n).astype(np.float32)
    vol = np.full(n, (1 / 64) ** 3 / 8)
    sim = D.DiffSim(64, 1 / 64, n, nu=NU, rho=RHO)
    s = D.pack_state(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda())
    Et = torch.from_numpy(E).cuda()
    so = orc.pack_state(x.astype(np.float64), v.astype(np.float64), np.zeros((n, 9)), np.tile(np.eye(3).reshape(9), (n, 1)))
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    for _ in range(10):
        s = sim.forward(1e-4, Et, s)
        so, st = orc.diff_forward(cfg, NU, RHO, vol, E.astype(np.float64), 1e-4, so)
        assert st == 0
    sim.sync()
    g = s.double().cpu().numpy()
    assert np.abs(g[:, 0:3] - so[:, 0:3]).max() <= 1e-4
    assert _rel(g[:, 3:6], so[:, 3:6]) <= 1e-4
    H_oracle = so[:, 15:] - np.eye(3).reshape(1, 9)        # the GPU state holds H = F - I
    assert np.abs(g[:, 15:] - H_oracle).max() <= 1e-4
    sim.close()


def test_diff_adjoint_matches_oracle_adjoint(D):
    x, v = _jelly(12, seed=6)
    n = len(x)
    rng = np.random.default_rng(2)
    E = rng.uniform(5e3, 2e4, n).astype(np.float32)
    C = (2.0 * rng.normal(size=(n, 9))).astype(np.float32)
    F = (np.eye(3) + 0.05 * rng.normal(size=(n, 3, 3))).reshape(n, 9).astype(np.float32)
    s64 = orc.pack_state(x.astype(np.float64), v.astype(np.float64), C.astype(np.float64), F.astype(np.float64))
    s_gpu = s64.copy()
    s_gpu[:, 15:] -= np.eye(3).reshape(1, 9)                 # GPU state: H = F - I
    s32 = torch.from_numpy(s_gpu.astype(np.float32)).cuda()
    s64[:, 15:] = s32[:, 15:].double().cpu().numpy() + np.eye(3).reshape(1, 9)   # same rounded input for both
    g_out = rng.normal(size=s64.shape)
    vol = np.full(n, (1 / 64) ** 3 / 8)
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    sim = D.DiffSim(64, 1 / 64, n, nu=NU, rho=RHO)
    gE = torch.zeros(n, device="cuda")
    g_in = sim.adjoint(1e-4, torch.from_numpy(E).cuda(), s32, torch.from_numpy(g_out.astype(np.float32)).cuda(), gE)
    sim.sync()
    gi = g_in.double().cpu().numpy()
    ge = gE.double().cpu().numpy()
    ri, re, st = orc.diff_adjoint(cfg, NU, RHO, vol, E.astype(np.float64), 1e-4, s64, g_out)
    assert st == 0
    for name, sl in (("x", slice(0, 3)), ("v", slice(3, 6)), ("C", slice(6, 15)), ("F", slice(15, 24))):
        assert _rel(gi[:, sl], ri[:, sl]) <= 1e-3, name
    assert _rel(ge, re) <= 1e-3
    sim.close()


def _oracle_final(x, v, E, vol, steps, dt):
    n = len(x)
    s = orc.pack_state(x, v, np.zeros((n, 9)), np.tile(np.eye(3).reshape(9), (n, 1)))
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    for _ in range(steps):
        s, st = orc.diff_forward(cfg, NU, RHO, vol, E, dt, s)
        assert st == 0
    return s


def _com_loss(s, vol):
    w = vol / vol.sum()
    com = (s[:, 0:3] * w[:, None]).sum(0)
    return float(((com - np.array(TARGET)) ** 2).sum())


def test_rollout_gradient_jelly_full_size(D):
    """The differentiable-rollout case: 32,768 particles (32^3 jittered
    lattice), E = 1e4, nu = 0.2, rho = 1, 64^3 grid, dt = 1e-4, 200 substeps,
    checkpoints every 20.  Two losses: the squared distance of the centre of
    mass to (0.5, 0.3, 0.5) -- which MLS-MPM's exact momentum conservation
    makes independent of E, so dL/dE must vanish -- and a random weighted sum
    of final positions, which depends on both v0 and E.  Directional
    derivatives against FP64 central differences of the oracle rollout."""
    x, v = _jelly(32)
    n = len(x)
    steps, dt = 200, 1e-4
    E0 = np.full(n, 1e4, np.float32)
    vol = np.full(n, 0.008 / n)
    rng = np.random.default_rng(9)
    Wpos = rng.normal(size=(n, 3))
    sim = D.DiffSim(64, 1 / 64, n, nu=NU, rho=RHO, vol=vol.astype(np.float32))
    xt = torch.from_numpy(x).cuda()
    grads = {}
    for name in ("com", "weighted"):
        vt = torch.from_numpy(v).cuda().requires_grad_(True)
        Et = torch.from_numpy(E0).cuda().requires_grad_(True)
        out = D.rollout(xt, vt, Et, sim, steps, k=20, dt=dt)
        if name == "com":
            loss = D.center_of_mass_loss(out, torch.from_numpy(vol.astype(np.float32)).cuda(), TARGET)
        else:
            loss = (out[:, 0:3] * torch.from_numpy(Wpos.astype(np.float32)).cuda()).sum()
        loss.backward()
        grads[name] = (vt.grad.double().cpu().numpy(), Et.grad.double().cpu().numpy())
    sim.close()
    dv = rng.normal(size=v.shape)
    # A stiffness field, not a random-sign one: along random signs the
    # per-particle terms of the directional derivative cancel to 1/375 of
    # their absolute sum, so FP32 rounding of each term (~3e-6) would already
    # reach the 1e-3 tolerance; along a positive field the ratio is ~1/17.
    dE = rng.uniform(0.5, 1.5, size=n) * 1e4
    eps = 1e-3
    x64, v64, E64 = x.astype(np.float64), v.astype(np.float64), E0.astype(np.float64)
    runs = {}
    for key, (vv, ee) in {"v+": (v64 + eps * dv, E64), "v-": (v64 - eps * dv, E64),
                          "E+": (v64, E64 + eps * dE), "E-": (v64, E64 - eps * dE),
                          "E+h": (v64, E64 + 0.5 * eps * dE), "E-h": (v64, E64 - 0.5 * eps * dE)}.items():
        runs[key] = _oracle_final(x64, vv, ee, vol, steps, dt)

    def central(loss, k, suffix="", h=eps):
        return (loss(runs[k + "+" + suffix]) - loss(runs[k + "-" + suffix])) / (2 * h)

    losses = {"com": lambda r: _com_loss(r, vol), "weighted": lambda r: float((r[:, 0:3] * Wpos).sum())}
    # The final positions oscillate with the stiffness (about ten elastic
    # wave crossings in 200 substeps), so the O(eps^2) truncation error of a
    # central difference in E is ~1.5e-3 relative at eps = 1e-3.  Richardson
    # extrapolation from eps and eps/2 cancels that term.
    fd = {name: {"v": central(lf, "v"),
                 "E": (4.0 * central(lf, "E", "h", 0.5 * eps) - central(lf, "E")) / 3.0}
          for name, lf in losses.items()}
    for name in ("com", "weighted"):
        gv, gE = grads[name]
        an_v = float((gv * dv).sum())
        an_E = float((gE * dE).sum())
        assert abs(fd[name]["v"] - an_v) <= 1e-3 * max(abs(fd[name]["v"]), abs(an_v)), (name, fd[name]["v"], an_v)
        if name == "com":
            # E cannot move the centre of mass: both sides ~0 on the scale of dL/dv0
            assert abs(an_E) <= 1e-3 * abs(an_v) and abs(fd[name]["E"]) <= 1e-3 * abs(fd[name]["v"])
        else:
            assert abs(fd[name]["E"] - an_E) <= 1e-3 * max(abs(fd[name]["E"]), abs(an_E)), (fd[name]["E"], an_E)


def test_rollout_gradient_matches_chained_oracle_adjoints(D):
    """Reduced case (1,728 particles, 20 substeps, checkpoints every 5, a
    random weighted sum of final positions as the loss): the autograd
    gradients equal the FP64 oracle's adjoints chained by hand."""
    x, v = _jelly(12, seed=8)
    n = len(x)
    steps, dt = 20, 1e-4
    rng = np.random.default_rng(4)
    E = rng.uniform(8e3, 1.2e4, n)
    vol = np.full(n, 0.008 / n)
    sim = D.DiffSim(64, 1 / 64, n, nu=NU, rho=RHO, vol=vol.astype(np.float32))
    Wpos = rng.normal(size=(n, 3))
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    Et = torch.from_numpy(E.astype(np.float32)).cuda().requires_grad_(True)
    out = D.rollout(torch.from_numpy(x).cuda(), vt, Et, sim, steps, k=5, dt=dt)
    loss = (out[:, 0:3] * torch.from_numpy(Wpos.astype(np.float32)).cuda()).sum()
    loss.backward()
    cfg = orc.config(64, 1 / 64, orc.STICKY)
    s = orc.pack_state(x.astype(np.float64), v.astype(np.float64), np.zeros((n, 9)), np.tile(np.eye(3).reshape(9), (n, 1)))
    states = [s]
    for _ in range(steps):
        states.append(orc.diff_forward(cfg, NU, RHO, vol, E, dt, states[-1])[0])
    g = np.zeros_like(s)
    g[:, 0:3] = Wpos
    gE = np.zeros(n)
    for t in range(steps - 1, -1, -1):
        g, e, st = orc.diff_adjoint(cfg, NU, RHO, vol, E, dt, states[t], g)
        gE += e
    assert _rel(vt.grad.double().cpu().numpy(), g[:, 3:6]) <= 1e-3
    assert _rel(Et.grad.double().cpu().numpy(), gE) <= 1e-3
    sim.close()
