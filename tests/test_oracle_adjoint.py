"""Pins for the oracle's adjoint: central finite differences of the FP64
forward substep along random directions, one state block at a time (so a
wrong term in any block fails), and a whole-rollout check."""
import numpy as np
import pytest


def _case(orc, seed, n=24, res=16):
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    x = rng.uniform(0.35, 0.65, (n, 3))
    v = 0.5 * rng.normal(size=(n, 3))
    C = 2.0 * rng.normal(size=(n, 9))
    F = (np.eye(3) + 0.05 * rng.normal(size=(n, 3, 3))).reshape(n, 9)
    s = orc.pack_state(x, v, C, F)
    E = rng.uniform(5e3, 2e4, n)
    vol = np.full(n, dx ** 3 / 8)
    return s, E, vol, orc.config(res, dx, orc.SLIP)


@pytest.mark.parametrize("block", ["x", "v", "C", "F", "E"])
def test_adjoint_matches_finite_differences(orc, block):
    nu, rho, dt = 0.2, 1000.0, 1e-3
    s, E, vol, cfg = _case(orc, 3)
    rng = np.random.default_rng(7)
    g_out = rng.normal(size=s.shape)
    g_in, gE, st = orc.diff_adjoint(cfg, nu, rho, vol, E, dt, s, g_out)
    assert st == 0
    ds = np.zeros_like(s)
    dE = np.zeros_like(E)
    sl = {"x": slice(0, 3), "v": slice(3, 6), "C": slice(6, 15), "F": slice(15, 24)}
    if block == "E":
        dE = rng.normal(size=E.shape) * E
    else:
        ds[:, sl[block]] = rng.normal(size=(len(s), sl[block].stop - sl[block].start))
    eps = 1e-6 if block != "E" else 1e-7

    def L(t):
        out, st2 = orc.diff_forward(cfg, nu, rho, vol, E + t * dE, dt, s + t * ds)
        assert st2 == 0
        return float((g_out * out).sum())

    fd = (L(eps) - L(-eps)) / (2 * eps)
    an = float((g_in * ds).sum() + (gE * dE).sum())
    assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 1e-9, (block, fd, an)


def test_adjoint_rollout_matches_finite_differences(orc):
    """Five chained substeps: the composed adjoints agree with central
    differences of the composed forward."""
    nu, rho, dt = 0.2, 1000.0, 1e-3
    s0, E, vol, cfg = _case(orc, 11, n=40)
    rng = np.random.default_rng(12)
    states = [s0]
    for _ in range(5):
        states.append(orc.diff_forward(cfg, nu, rho, vol, E, dt, states[-1])[0])
    g = rng.normal(size=s0.shape)
    gE = np.zeros_like(E)
    for k in range(5, 0, -1):
        g, e, st = orc.diff_adjoint(cfg, nu, rho, vol, E, dt, states[k - 1], g if k < 5 else g)
        gE += e
    ds = rng.normal(size=s0.shape)
    dE = rng.normal(size=E.shape) * E
    g_final = np.random.default_rng(12).normal(size=s0.shape)

    def L(t):
        s = s0 + t * ds
        for _ in range(5):
            s = orc.diff_forward(cfg, nu, rho, vol, E + t * dE, dt, s)[0]
        return float((g_final * s).sum())

    eps = 1e-7
    fd = (L(eps) - L(-eps)) / (2 * eps)
    an = float((g * ds).sum() + (gE * dE).sum())
    assert abs(fd - an) <= 1e-5 * max(abs(fd), abs(an)), (fd, an)


def test_diff_forward_is_the_plain_substep(orc):
    """With a common E the differentiable forward equals orc_substep."""
    nu, rho, dt = 0.2, 1000.0, 1e-3
    s, E, vol, cfg = _case(orc, 5)
    E[:] = 1e4
    out, st = orc.diff_forward(cfg, nu, rho, vol, E, dt, s)
    st_ = orc.State(s[:, 0:3], s[:, 3:6], s[:, 6:15].reshape(-1, 3, 3), s[:, 15:24].reshape(-1, 3, 3), None, vol, 0)
    orc.substep(cfg, orc.material(orc.ELASTIC, E=1e4, nu=nu, rho=rho), st_, dt)
    np.testing.assert_allclose(out, orc.pack_state(st_.x, st_.v, st_.C, st_.F), rtol=0, atol=1e-13)
