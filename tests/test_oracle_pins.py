"""Pins for the FP64 oracle: each check compares it with something other than
itself -- a closed form, an invariant of the method, a library routine
(numpy's SVD), or brute force on tiny inputs.  A dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one test.
"""
import numpy as np
import pytest

RNG = np.random.default_rng(12345)


def N_quad(u):
    """Quadratic B-spline kernel, piecewise definition (independent of the
    base/fraction form the oracle uses)."""
    u = np.abs(u)
    return np.where(u < 0.5, 0.75 - u * u, np.where(u < 1.5, 0.5 * (1.5 - u) ** 2, 0.0))


# ----------------------------------------------------------------- weights

@pytest.mark.parametrize("f", list(RNG.uniform(0.5, 1.5, 16)) + [0.5, 1.0, 1.4999999])
def test_bspline_moments_and_kernel(orc, f):
    w = orc.bspline_weights(f)
    off = np.arange(3) - f           # (x_i - x_p)/dx for the three nodes
    assert abs(w.sum() - 1.0) < 1e-14                  # partition of unity
    assert abs((w * off).sum()) < 1e-14                # zero first moment
    assert abs((w * off * off).sum() - 0.25) < 1e-14   # second moment = 1/4 (dx^2/4)
    np.testing.assert_allclose(w, N_quad(off), rtol=0, atol=1e-15)


# --------------------------------------------------------------------- SVD

def _rand_rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _svd_cases():
    rng = np.random.default_rng(7)
    cases = [np.eye(3), np.diag([2.0, 0.5, 1.0]), np.diag([1.0, 1.0, -1.0]),
             np.zeros((3, 3)), np.diag([3.0, 0.0, 0.0])]
    for _ in range(40):
        cases.append(rng.normal(size=(3, 3)))
    for _ in range(10):
        cases.append(np.eye(3) + 1e-3 * rng.normal(size=(3, 3)))
    for _ in range(10):                       # repeated singular values
        R1, R2 = _rand_rot(rng), _rand_rot(rng)
        cases.append(R1 @ np.diag([1.2, 1.2, 0.7]) @ R2.T)
    for _ in range(5):                        # inverted
        R1, R2 = _rand_rot(rng), _rand_rot(rng)
        cases.append(R1 @ np.diag([1.3, 0.9, -0.2]) @ R2.T)
    return cases


@pytest.mark.parametrize("F", _svd_cases())
def test_svd_against_numpy(orc, F):
    U, s, V = orc.svd3(F)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, F, atol=1e-12 * max(1.0, np.abs(F).max()))
    np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-12)
    assert abs(np.linalg.det(U) - 1) < 1e-12 and abs(np.linalg.det(V) - 1) < 1e-12
    ref = np.linalg.svd(F, compute_uv=False)          # library routine, descending
    np.testing.assert_allclose(np.abs(s), ref, atol=1e-12 * max(1.0, ref[0]))
    assert s[0] >= s[1] >= abs(s[2]) - 1e-12
    d = np.linalg.det(F)
    if abs(d) > 1e-9:
        assert np.sign(s[2]) == np.sign(d)


# ------------------------------------------------------------------ stress

def _psi_fixed_corotated(F, mu, la):
    s = np.linalg.svd(F, compute_uv=False)
    if np.linalg.det(F) < 0:
        s[2] = -s[2]
    J = np.linalg.det(F)
    return mu * ((s - 1) ** 2).sum() + 0.5 * la * (J - 1) ** 2


def _psi_hencky(F, mu, la):
    s = np.linalg.svd(F, compute_uv=False)
    e = np.log(s)
    return mu * (e * e).sum() + 0.5 * la * e.sum() ** 2


def _fd_first_pk(psi, F, h=1e-6):
    P = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            P[i, j] = (psi(F + E) - psi(F - E)) / (2 * h)
    return P


def test_fixed_corotated_is_energy_derivative(orc):
    """tau = P F^T with P the derivative of the fixed-corotated energy
    psi = mu sum (s_i - 1)^2 + la/2 (J - 1)^2 (Stomakhin et al. 2012)."""
    rng = np.random.default_rng(3)
    E, nu = 1e4, 0.2
    mu, la = orc.lame(E, nu)
    mat = orc.material(orc.ELASTIC, E=E, nu=nu)
    for _ in range(10):
        F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        P = _fd_first_pk(lambda G: _psi_fixed_corotated(G, mu, la), F)
        np.testing.assert_allclose(orc.kirchhoff(mat, F), P @ F.T, rtol=0, atol=1e-4 * E)


def test_fixed_corotated_special_cases(orc):
    E, nu = 1e4, 0.2
    mu, la = orc.lame(E, nu)
    assert abs(mu - E / 2.4) < 1e-9 and abs(la - E * 0.2 / (1.2 * 0.6)) < 1e-9
    mat = orc.material(orc.ELASTIC, E=E, nu=nu)
    R = _rand_rot(np.random.default_rng(1))
    np.testing.assert_allclose(orc.kirchhoff(mat, R), 0, atol=1e-9)      # rotation: no stress
    for s in (0.8, 1.0, 1.25):                                             # uniform dilation
        tau = orc.kirchhoff(mat, s * np.eye(3))
        expect = 2 * mu * (s - 1) * s + la * s ** 3 * (s ** 3 - 1)
        np.testing.assert_allclose(tau, expect * np.eye(3), atol=1e-9 * E)
    eps = 1e-6 * np.array([[1.0, 0.3, -0.2], [0.3, -0.5, 0.1], [-0.2, 0.1, 0.7]])
    lin = 2 * mu * eps + la * np.trace(eps) * np.eye(3)                    # small-strain limit
    np.testing.assert_allclose(orc.kirchhoff(mat, np.eye(3) + eps), lin, rtol=0, atol=1e-8 * E)
    F = np.eye(3) + 0.2 * np.random.default_rng(5).normal(size=(3, 3))
    tau, Q = orc.kirchhoff(mat, F), _rand_rot(np.random.default_rng(6))
    np.testing.assert_allclose(orc.kirchhoff(mat, Q @ F), Q @ tau @ Q.T, atol=1e-9 * E)   # objectivity
    np.testing.assert_allclose(tau, tau.T, atol=1e-9 * E)


def test_snow_hardening_and_fluid_and_sand_stress(orc):
    F = np.eye(3) + 0.05 * np.random.default_rng(8).normal(size=(3, 3))
    el = orc.material(orc.ELASTIC, E=1.4e5, nu=0.2)
    sn = orc.material(orc.SNOW, E=1.4e5, nu=0.2, hardening=10.0)
    for Jp in (1.0, 0.97, 1.02):
        np.testing.assert_allclose(orc.kirchhoff(sn, F, Jp), np.exp(10.0 * (1 - Jp)) * orc.kirchhoff(el, F),
                                   rtol=1e-12, atol=1e-9)
    fl = orc.material(orc.FLUID, E=1e4, gamma=7.0)
    np.testing.assert_allclose(orc.kirchhoff(fl, np.eye(3), 1.0), 0, atol=1e-12)
    for J in (0.9, 1.1):
        p = 1e4 * (J ** -7 - 1)
        np.testing.assert_allclose(orc.kirchhoff(fl, np.eye(3), J), -p * J * np.eye(3), rtol=1e-12)
    # sand: Hencky St. Venant-Kirchhoff, tau = P F^T of psi = mu |eps|^2 + la/2 tr(eps)^2
    sa = orc.material(orc.SAND, E=3.5e5, nu=0.3)
    mu, la = orc.lame(3.5e5, 0.3)
    rng = np.random.default_rng(9)
    for _ in range(6):
        G = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
        if np.linalg.det(G) < 0.3:
            continue
        P = _fd_first_pk(lambda H: _psi_hencky(H, mu, la), G, h=1e-7)
        np.testing.assert_allclose(orc.kirchhoff(sa, G), P @ G.T, rtol=0, atol=2e-4 * 3.5e5 * 1e-2)


# -------------------------------------------------------------- plasticity

def test_snow_clamp(orc):
    sn = orc.material(orc.SNOW, E=1.4e5, nu=0.2, theta_c=2.5e-2, theta_s=7.5e-3)
    rng = np.random.default_rng(11)
    R1, R2 = _rand_rot(rng), _rand_rot(rng)
    F_in = R1 @ np.diag([1.005, 0.99, 0.98]) @ R2.T          # inside [0.975, 1.0075]
    F2, J2 = orc.plasticity(sn, F_in, 1.0)
    np.testing.assert_allclose(F2, F_in, atol=1e-13)
    assert abs(J2 - 1.0) < 1e-13
    F_out = R1 @ np.diag([1.05, 1.0, 0.9]) @ R2.T
    F3, J3 = orc.plasticity(sn, F_out, 0.95)
    np.testing.assert_allclose(np.linalg.svd(F3, compute_uv=False), [1.0075, 1.0, 0.975], atol=1e-12)
    # total deformation det(F_E) Jp is conserved by the return map
    assert abs(np.linalg.det(F3) * J3 - np.linalg.det(F_out) * 0.95) < 1e-12
    np.testing.assert_allclose(F3, R1 @ np.diag([1.0075, 1.0, 0.975]) @ R2.T, atol=1e-12)


def test_drucker_prager_cases(orc):
    E, nu, phi = 3.5e5, 0.3, 30.0
    sa = orc.material(orc.SAND, E=E, nu=nu, friction_deg=phi)
    mu, la = orc.lame(E, nu)
    sphi = np.sin(np.radians(phi))
    alpha = np.sqrt(2 / 3) * 2 * sphi / (3 - sphi)
    rng = np.random.default_rng(13)
    R1, R2 = _rand_rot(rng), _rand_rot(rng)
    # case II: volume expansion -> cone tip, sigma = 1
    F, _ = orc.plasticity(sa, R1 @ np.diag([1.05, 1.01, 0.99]) @ R2.T)
    np.testing.assert_allclose(F, R1 @ R2.T, atol=1e-12)
    # case I: compression with little shear stays
    Fi = R1 @ np.diag([0.999, 0.998, 0.997]) @ R2.T
    F, _ = orc.plasticity(sa, Fi)
    np.testing.assert_allclose(F, Fi, atol=1e-13)
    # case III: sheared compression is returned onto the cone surface
    Fo = R1 @ np.diag([1.03, 0.99, 0.95]) @ R2.T
    eps = np.log([1.03, 0.99, 0.95])
    assert eps.sum() < 0
    F, _ = orc.plasticity(sa, Fo)
    s = np.linalg.svd(F, compute_uv=False)
    e2 = np.log(s)
    dev2 = e2 - e2.mean()
    assert abs(e2.sum() - eps.sum()) < 1e-12                       # trace preserved
    yield_fn = np.linalg.norm(dev2) + (3 * la + 2 * mu) / (2 * mu) * e2.sum() * alpha
    assert abs(yield_fn) < 1e-12                                   # on the cone
    dev = eps - eps.mean()
    np.testing.assert_allclose(dev2 / np.linalg.norm(dev2), np.sort(dev)[::-1] / np.linalg.norm(dev), atol=1e-9)


def _psi_neo_hookean(F, mu, la):
    """Compressible neo-Hookean energy mu/2 (tr F^T F - 3) - mu ln J + la/2 (ln J)^2."""
    lnJ = np.log(np.linalg.det(F))
    return 0.5 * mu * (np.sum(F * F) - 3.0) - mu * lnJ + 0.5 * la * lnJ * lnJ


def test_neo_hookean_sand_stress_and_return_map(orc):
    """Neo-Hookean sand: tau = P F^T with P the derivative of the neo-Hookean
    energy (finite differences of the energy); rotations carry no stress;
    the small-strain limit is linear elasticity, the Hencky sand stress to
    first order; the return map is the sand's (cases I-III pinned above)."""
    rng = np.random.default_rng(17)
    E, nu = 3.5e5, 0.3
    mu, la = orc.lame(E, nu)
    nh = orc.material(orc.NHSAND, E=E, nu=nu, friction_deg=30.0)
    sa = orc.material(orc.SAND, E=E, nu=nu, friction_deg=30.0)
    for _ in range(10):
        F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        P = _fd_first_pk(lambda G: _psi_neo_hookean(G, mu, la), F)
        np.testing.assert_allclose(orc.kirchhoff(nh, F), P @ F.T, rtol=0, atol=1e-4 * E)
    np.testing.assert_allclose(orc.kirchhoff(nh, _rand_rot(rng)), 0, atol=1e-9 * E)
    eps = 1e-6 * np.array([[1.0, 0.3, -0.2], [0.3, -0.5, 0.1], [-0.2, 0.1, 0.7]])
    lin = 2 * mu * eps + la * np.trace(eps) * np.eye(3)
    np.testing.assert_allclose(orc.kirchhoff(nh, np.eye(3) + eps), lin, rtol=0, atol=1e-8 * E)
    np.testing.assert_allclose(orc.kirchhoff(nh, np.eye(3) + eps), orc.kirchhoff(sa, np.eye(3) + eps), rtol=0,
                               atol=1e-8 * E)
    for _ in range(20):
        F = _rand_rot(rng) @ np.diag(rng.uniform(0.9, 1.1, 3)) @ _rand_rot(rng).T
        a, ja = orc.plasticity(nh, F)
        b, jb = orc.plasticity(sa, F)
        np.testing.assert_array_equal(a, b)
        assert ja == jb


def _nacc_pq(F, kappa, nu):
    """p = -tr(tau)/3 and q = sqrt(3/2)|dev tau| of the Hencky St. Venant-
    Kirchhoff stress of F, from numpy's SVD (independent of the oracle)."""
    mu = 3 * kappa * (1 - 2 * nu) / (2 * (1 + nu))
    e = np.log(np.linalg.svd(F, compute_uv=False))
    dev = e - e.mean()
    return -kappa * e.sum(), np.sqrt(1.5) * 2 * mu * np.linalg.norm(dev), e, dev


def test_nacc_cam_clay_return_map(orc):
    """NACC (Cam-Clay, non-associative): inside the ellipse nothing changes;
    beyond it q shrinks onto the surface at the same p with the deviatoric
    direction kept; beyond the tips the state moves to (p0, 0) or
    (-beta p0, 0) and Jp absorbs the removed volume; the stress is Hencky
    St. Venant-Kirchhoff with the bulk modulus kappa."""
    kappa, nu, M, beta, xi, a0 = 5e5, 0.3, 0.8, 0.9, 5.0, -0.01
    mat = orc.material(orc.NACC, E=kappa, nu=nu, hardening=xi, friction_M=M, cohesion=beta, alpha0=a0)
    mu = 3 * kappa * (1 - 2 * nu) / (2 * (1 + nu))
    la = kappa - 2 * mu / 3
    p0 = kappa * np.sinh(xi * 0.01)                   # Jp = 1: alpha = alpha0
    y = lambda p, q: (1 + 2 * beta) * q * q + M * M * (p + beta * p0) * (p - p0)
    rng = np.random.default_rng(21)
    R1, R2 = _rand_rot(rng), _rand_rot(rng)
    # stress
    Fs = R1 @ np.diag([1.01, 0.995, 0.98]) @ R2.T
    tau = orc.kirchhoff(mat, Fs, 1.0)
    e = np.log([1.01, 0.995, 0.98])
    ref = R1 @ np.diag(2 * mu * e + la * e.sum()) @ R1.T
    np.testing.assert_allclose(tau, ref, atol=1e-9 * np.abs(ref).max())
    assert abs(np.trace(tau) - 3 * kappa * e.sum()) < 1e-9 * kappa
    # inside: mild compression, little shear
    Fi = R1 @ np.diag([0.9999, 0.9998, 0.9997]) @ R2.T
    p, q, _, _ = _nacc_pq(Fi, kappa, nu)
    assert 0 < p < p0 and y(p, q) < 0
    F, Jp = orc.plasticity(mat, Fi, 1.0)
    np.testing.assert_allclose(F, Fi, atol=1e-13)
    assert Jp == 1.0
    # sheared: projected onto the ellipse at the same p, direction kept, no volume change
    Fo = R1 @ np.diag([1.03, 0.997, 0.975]) @ R2.T
    p, q, e, dev = _nacc_pq(Fo, kappa, nu)
    assert -beta * p0 < p < p0 and y(p, q) > 0
    F, Jp = orc.plasticity(mat, Fo, 1.0)
    p2, q2, e2, dev2 = _nacc_pq(F, kappa, nu)
    assert abs(p2 - p) < 1e-9 * kappa and abs(y(p2, q2)) < 1e-9 * (M * p0) ** 2
    np.testing.assert_allclose(dev2 / np.linalg.norm(dev2), np.sort(dev)[::-1] / np.linalg.norm(dev), atol=1e-9)
    assert abs(Jp - 1.0) < 1e-12
    # compressed past the cap: to (p0, 0); Jp takes the removed volume
    Fc = R1 @ np.diag([0.985, 0.98, 0.975]) @ R2.T
    p, q, e, _ = _nacc_pq(Fc, kappa, nu)
    assert p > p0
    F, Jp = orc.plasticity(mat, Fc, 1.0)
    p2, q2, e2, _ = _nacc_pq(F, kappa, nu)
    assert abs(p2 - p0) < 1e-9 * kappa and q2 < 1e-6 * kappa
    assert abs(Jp * np.linalg.det(F) - np.linalg.det(Fc)) < 1e-12
    # stretched past the cohesion tip: to (-beta p0, 0)
    Ft = R1 @ np.diag([1.016, 1.018, 1.015]) @ R2.T
    p, q, _, _ = _nacc_pq(Ft, kappa, nu)
    assert p < -beta * p0
    F, Jp = orc.plasticity(mat, Ft, 1.0)
    p2, q2, _, _ = _nacc_pq(F, kappa, nu)
    assert abs(p2 + beta * p0) < 1e-9 * kappa and q2 < 1e-6 * kappa
    assert abs(Jp * np.linalg.det(F) - np.linalg.det(Ft)) < 1e-12
    # no hardening (alpha >= 0): p0 = 0, every state returns to the stress-free one
    soft = orc.material(orc.NACC, E=kappa, nu=nu, hardening=xi, friction_M=M, cohesion=beta, alpha0=0.0)
    F, Jp = orc.plasticity(soft, Fo, 1.0)
    np.testing.assert_allclose(np.linalg.svd(F, compute_uv=False), 1.0, atol=1e-12)
    np.testing.assert_allclose(orc.kirchhoff(soft, F, Jp), 0.0, atol=1e-6)
    # hardening: compaction (Jp < 1, alpha = -0.03) raises p0 to kappa sinh(0.15), so the
    # state that was past the cap is now inside the ellipse and stays
    p, q, _, _ = _nacc_pq(Fc, kappa, nu)
    p0h = kappa * np.sinh(xi * 0.03)
    assert p < p0h and (1 + 2 * beta) * q * q + M * M * (p + beta * p0h) * (p - p0h) < 0
    F, Jp = orc.plasticity(mat, Fc, np.exp(-0.02))
    np.testing.assert_allclose(F, Fc, atol=1e-13)
    assert Jp == np.exp(-0.02)


# --------------------------------------------------------------- transfers

def _random_state(orc, rng, n, lo, hi, dx, F_noise=0.05, C_scale=1.0, v_scale=1.0):
    x = rng.uniform(lo, hi, size=(n, 3))
    v = v_scale * rng.normal(size=(n, 3))
    C = C_scale * rng.normal(size=(n, 3, 3))
    F = np.eye(3) + F_noise * rng.normal(size=(n, 3, 3))
    vol = rng.uniform(0.5, 1.5, n) * dx ** 3 / 8
    return orc.State(x, v, C, F, None, vol, 0)


def test_p2g_conservation(orc):
    rng = np.random.default_rng(21)
    dx = 1 / 64
    cfg = orc.config(64, dx)
    mat = orc.material(orc.ELASTIC, E=1e4, nu=0.2, rho=3.0)
    s = _random_state(orc, rng, 300, 0.3, 0.7, dx)
    dt = 1e-4
    g, st = orc.p2g(cfg, mat, s, dt)
    assert st == 0
    mp = 3.0 * s.vol
    assert abs(g.m.sum() - mp.sum()) <= 1e-13 * mp.sum()
    P = g.p.reshape(-1, 3).sum(0)
    np.testing.assert_allclose(P, (mp[:, None] * s.v).sum(0), rtol=1e-12, atol=1e-13)
    # angular momentum: sum_i x_i x p_i = sum_p x_p x m v + m (dx^2/4) eps_abc C_cb
    xi = g.node_positions(dx).reshape(-1, 3)
    L_grid = np.cross(xi, g.p.reshape(-1, 3)).sum(0)
    C = s.C
    spin = np.stack([C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0], C[:, 1, 0] - C[:, 0, 1]], axis=1)
    L_part = (np.cross(s.x, mp[:, None] * s.v) + mp[:, None] * dx * dx / 4 * spin).sum(0)
    np.testing.assert_allclose(L_grid, L_part, rtol=1e-10, atol=1e-14)


def test_p2g_brute_force_tiny(orc):
    """Tiny case against a naive loop over every node of an 8^3 grid with the
    piecewise kernel, the stress from the closed form of a uniform dilation."""
    dx = 1 / 8
    cfg = orc.config(8, dx)
    E, nu = 2e3, 0.25
    mat = orc.material(orc.ELASTIC, E=E, nu=nu, rho=2.0)
    mu, la = orc.lame(E, nu)
    rng = np.random.default_rng(4)
    n = 6
    x = rng.uniform(0.35, 0.65, size=(n, 3))
    v = rng.normal(size=(n, 3))
    C = rng.normal(size=(n, 3, 3))
    sc = rng.uniform(0.9, 1.1, n)
    F = sc[:, None, None] * np.eye(3)[None]
    vol = np.full(n, 1e-3)
    s = orc.State(x, v, C, F, None, vol, 0)
    dt = 1e-3
    g, st = orc.p2g(cfg, mat, s, dt, orc.DenseGrid([0, 0, 0], [8, 8, 8]))
    assert st == 0
    m_ref = np.zeros((8, 8, 8))
    p_ref = np.zeros((8, 8, 8, 3))
    for q in range(n):
        J = sc[q] ** 3
        tau = (2 * mu * (sc[q] - 1) * sc[q] + la * J * (J - 1)) * np.eye(3)
        mq = 2.0 * vol[q]
        A = mq * C[q] - 4 * dt * vol[q] / dx ** 2 * tau
        for k in range(8):
            for j in range(8):
                for i in range(8):
                    xi = np.array([i, j, k]) * dx
                    w = N_quad(x[q, 0] / dx - i) * N_quad(x[q, 1] / dx - j) * N_quad(x[q, 2] / dx - k)
                    m_ref[k, j, i] += w * mq
                    p_ref[k, j, i] += w * (mq * v[q] + A @ (xi - x[q]))
    np.testing.assert_allclose(g.mass(), m_ref, atol=1e-15)
    np.testing.assert_allclose(g.mom(), p_ref, atol=1e-12)


def test_p2g_node_matches_dense(orc):
    rng = np.random.default_rng(22)
    dx = 1 / 32
    cfg = orc.config(32, dx)
    mat = orc.material(orc.ELASTIC)
    s = _random_state(orc, rng, 200, 0.3, 0.7, dx)
    g, _ = orc.p2g(cfg, mat, s, 1e-4)
    m = g.mass()
    idx = np.argwhere(m > 0)
    for kk in idx[rng.choice(len(idx), 10, replace=False)]:
        node = np.array([kk[2], kk[1], kk[0]]) + g.lo
        out = orc.p2g_node(cfg, mat, s, 1e-4, node)
        assert abs(out[0] - m[tuple(kk)]) < 1e-15
        np.testing.assert_allclose(out[1:], g.mom()[tuple(kk)], atol=1e-13)


def test_grid_update_boundaries(orc):
    dx = 1 / 16
    dt = 1e-2
    g = orc.DenseGrid([0, 0, 0], [16, 16, 16])
    m, p = g.mass(), g.mom()
    m[8, 8, 8] = 2.0; p[8, 8, 8] = [2.0, 4.0, -6.0]          # interior
    m[8, 1, 8] = 1.0; p[8, 1, 8] = [1.0, -3.0, 0.5]          # y wall layer (low), moving into the wall
    m[8, 14, 8] = 1.0; p[8, 14, 8] = [1.0, 3.0, 0.5]         # y wall layer (high), moving into the wall
    m[8, 12, 2] = 1.0; p[8, 12, 2] = [0.5, 0.5, 0.5]         # x low wall, moving away
    p[5, 5, 5] = [1.0, 1.0, 1.0]                             # massless node carries no velocity
    gs = orc.DenseGrid(g.lo, g.dim); gs.m[:] = g.m; gs.p[:] = g.p
    gr = 9.8
    orc.grid_update(orc.config(16, dx, orc.SLIP, 3), dt, g)
    V = g.mom()
    np.testing.assert_allclose(V[8, 8, 8], [1.0, 2.0 - gr * dt, -3.0], atol=1e-14)
    np.testing.assert_allclose(V[8, 1, 8], [1.0, 0.0, 0.5], atol=1e-14)
    np.testing.assert_allclose(V[8, 14, 8], [1.0, 0.0, 0.5], atol=1e-14)
    np.testing.assert_allclose(V[8, 12, 2], [0.5, 0.5 - gr * dt, 0.5], atol=1e-14)
    np.testing.assert_allclose(V[5, 5, 5], 0, atol=0)
    orc.grid_update(orc.config(16, dx, orc.STICKY, 3), dt, gs)
    V = gs.mom()
    np.testing.assert_allclose(V[8, 8, 8], [1.0, 2.0 - gr * dt, -3.0], atol=1e-14)
    for c in ([8, 1, 8], [8, 14, 8], [8, 12, 2]):
        np.testing.assert_allclose(V[tuple(c)], 0, atol=0)


def test_g2p_affine_reproduction(orc):
    """Grid velocity a + B x_i is reproduced exactly: v_p = a + B x_p, C_p = B."""
    rng = np.random.default_rng(31)
    dx = 1 / 32
    cfg = orc.config(32, dx)
    mat = orc.material(orc.ELASTIC)
    n = 50
    F0 = np.eye(3) + 0.1 * rng.normal(size=(n, 3, 3))
    s = orc.State(rng.uniform(0.3, 0.7, (n, 3)), F=F0)
    a = rng.normal(size=3)
    B = rng.normal(size=(3, 3))
    lo, dim = orc.grid_bounds(s.x, dx)
    g = orc.DenseGrid(lo, dim)
    g.p[:] = (a + g.node_positions(dx).reshape(-1, 3) @ B.T).reshape(-1)
    x0 = s.x.copy()
    dt = 1e-3
    assert orc.g2p(cfg, mat, s, dt, g) == 0
    vp = a + x0 @ B.T
    np.testing.assert_allclose(s.v, vp, atol=1e-12)
    np.testing.assert_allclose(s.C, np.broadcast_to(B, (n, 3, 3)), atol=1e-10)
    np.testing.assert_allclose(s.x, x0 + dt * vp, atol=1e-14)
    np.testing.assert_allclose(s.F, np.einsum("ab,pbc->pac", np.eye(3) + dt * B, F0), atol=1e-12)
    # fluid: J <- (1 + dt tr C) J, F untouched
    sf = orc.State(x0, Jp=np.full(n, 0.9))
    fl = orc.material(orc.FLUID, E=1e4)
    orc.g2p(cfg, fl, sf, dt, g)
    np.testing.assert_allclose(sf.Jp, 0.9 * (1 + dt * np.trace(B)), rtol=1e-12)
    np.testing.assert_allclose(sf.F, np.broadcast_to(np.eye(3), (n, 3, 3)), atol=0)


def test_free_fall_closed_form(orc):
    """F = I, C = 0, uniform v0, no wall reached: each substep adds dt g, so
    x_n = x0 + n dt v0 + g dt^2 n (n + 1) / 2 (symplectic Euler)."""
    rng = np.random.default_rng(41)
    dx = 1 / 64
    cfg = orc.config(64, dx, orc.STICKY)
    mat = orc.material(orc.ELASTIC, E=1e4, nu=0.2)
    n = 400
    x0 = rng.uniform(0.4, 0.6, (n, 3))
    v0 = np.array([0.3, 0.1, -0.2])
    s = orc.State(x0, np.tile(v0, (n, 1)), vol=1e-6)
    dt, steps = 1e-3, 25
    for _ in range(steps):
        assert orc.substep(cfg, mat, s, dt) == 0
    g = np.array([0, -9.8, 0])
    expect = x0 + steps * dt * v0 + g * dt * dt * steps * (steps + 1) / 2
    np.testing.assert_allclose(s.x, expect, atol=1e-12)
    np.testing.assert_allclose(s.v, np.tile(v0 + steps * dt * g, (n, 1)), atol=1e-11)
    np.testing.assert_allclose(s.C, 0, atol=1e-9)
    np.testing.assert_allclose(s.F, np.broadcast_to(np.eye(3), (n, 3, 3)), atol=1e-12)


def test_substep_is_phase_composition(orc):
    rng = np.random.default_rng(51)
    dx = 1 / 32
    cfg = orc.config(32, dx, orc.SLIP)
    mats = [orc.material(orc.ELASTIC), orc.material(orc.SNOW, E=1.4e5, rho=400.0),
            orc.material(orc.FLUID, E=1e4, rho=1000.0), orc.material(orc.SAND, E=3.5e5, nu=0.3, rho=2200.0)]
    s = _random_state(orc, rng, 120, 0.3, 0.7, dx, F_noise=0.01, C_scale=0.1, v_scale=0.1)
    s.mat[:] = rng.integers(0, 4, s.n)
    s.Jp[:] = 1.0
    a, b = s.copy(), s.copy()
    dt = 1e-4
    orc.substep(cfg, mats, a, dt)
    g, _ = orc.p2g(cfg, mats, b, dt)
    orc.grid_update(cfg, dt, g)
    orc.g2p(cfg, mats, b, dt, g)
    for f in ("x", "v", "C", "F", "Jp"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


# ------------------------------------------------------------------ ASFLIP

@pytest.mark.parametrize("margin", [0.0, 1e-4])
@pytest.mark.parametrize("J_F", [1.0, 0.9, 1.1, 0.99995, 0.9998])
def test_asflip_two_coincident_particles_closed_form(orc, J_F, margin):
    """Two particles at one point, zero stress (E = 0), no gravity, no wall:
    every node of their common stencil carries their mean velocity vbar,
    before and after the grid update, so APIC would give both vbar.  ASFLIP
    (Fei et al. 2021) keeps alpha times each particle's deviation v - vbar in
    its velocity and beta alpha times it in its motion, beta = beta_min when
    the particle is compressed, J = det F < 1 - margin, and beta_max otherwise
    (three distinct weights, so that a swapped or dropped one fails).  With
    the default margin 0 the test is J < 1: J = 1 exactly is not compressed,
    J = 0.99995 is; a margin of 1e-4 moves J = 0.99995 to the other branch
    and leaves J = 0.9998 compressed."""
    dx = 1 / 32
    alpha, bmin, bmax = 0.9, 0.3, 0.7
    cfg = orc.config(32, dx, gravity=(0.0, 0.0, 0.0), transfer=orc.ASFLIP, flip_alpha=alpha,
                     flip_beta_min=bmin, flip_beta_max=bmax, flip_compress_margin=margin)
    mat = orc.material(orc.ELASTIC, E=0.0)
    xp = np.array([0.503, 0.49, 0.51])
    v = np.array([[0.3, -0.1, 0.2], [-0.1, 0.25, 0.0]])
    F = np.diag([J_F, 1.0, 1.0])
    s = orc.State(np.tile(xp, (2, 1)), v, F=np.tile(F, (2, 1, 1)), vol=1e-5)
    dt = 1e-3
    assert orc.substep(cfg, mat, s, dt) == 0
    vbar = v.mean(0)
    compressed = {(1.0, 0.0): False, (0.9, 0.0): True, (1.1, 0.0): False, (0.99995, 0.0): True,
                  (0.9998, 0.0): True, (1.0, 1e-4): False, (0.9, 1e-4): True, (1.1, 1e-4): False,
                  (0.99995, 1e-4): False, (0.9998, 1e-4): True}[(J_F, margin)]
    beta = bmin if compressed else bmax
    np.testing.assert_allclose(s.v, vbar + alpha * (v - vbar), atol=1e-13)
    np.testing.assert_allclose(s.x, xp + dt * (vbar + beta * alpha * (v - vbar)), atol=1e-15)
    np.testing.assert_allclose(s.C, 0, atol=1e-10)
    np.testing.assert_allclose(s.F, np.tile(F, (2, 1, 1)), atol=1e-12)


def test_asflip_with_zero_weights_is_apic(orc):
    """alpha = beta = 0 reduces ASFLIP to APIC exactly, all materials."""
    rng = np.random.default_rng(61)
    dx = 1 / 32
    mats = [orc.material(orc.ELASTIC), orc.material(orc.SNOW, E=1.4e5, rho=400.0),
            orc.material(orc.FLUID, E=1e4, rho=1000.0), orc.material(orc.SAND, E=3.5e5, nu=0.3, rho=2200.0)]
    s = _random_state(orc, rng, 120, 0.3, 0.7, dx, F_noise=0.01, C_scale=0.1, v_scale=0.1)
    s.mat[:] = rng.integers(0, 4, s.n)
    s.Jp[:] = 1.0
    a, b = s.copy(), s.copy()
    orc.substep(orc.config(32, dx, orc.SLIP), mats, a, 1e-4)
    orc.substep(orc.config(32, dx, orc.SLIP, transfer=orc.ASFLIP, flip_beta_max=0.0), mats, b, 1e-4)
    for f in ("x", "v", "C", "F", "Jp"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_asflip_keeps_the_momentum_and_centre_of_mass_of_apic(orc):
    """v0_i = p_i / m_i after P2G, so sum_p m_p v0_p = sum_i p_i = sum_p m_p
    v_p (the moments of the weights vanish): the blended-in deviations carry
    no net momentum.  Hence for any alpha the total particle momentum after
    G2P equals APIC's, and with one beta for all particles so does the mass
    centre.  A v0 taken after gravity or the walls breaks both (gravity on,
    sticky walls reached by some stencils)."""
    rng = np.random.default_rng(62)
    dx = 1 / 32
    mat = orc.material(orc.ELASTIC, E=1e4, nu=0.2, rho=1000.0)
    s = _random_state(orc, rng, 300, 0.08, 0.5, dx, F_noise=0.02, C_scale=0.5, v_scale=0.5)
    a, b = s.copy(), s.copy()
    dt = 1e-4
    orc.substep(orc.config(32, dx, orc.STICKY), mat, a, dt)
    orc.substep(orc.config(32, dx, orc.STICKY, transfer=orc.ASFLIP, flip_alpha=0.8, flip_beta_min=0.6,
                           flip_beta_max=0.6), mat, b, dt)
    m = s.vol[:, None] * 1000.0
    pa, pb = (m * a.v).sum(0), (m * b.v).sum(0)
    assert np.abs(pb - pa).max() <= 1e-12 * np.abs(m * s.v).sum()
    assert np.abs(b.v - a.v).max() > 1e-3            # the blend did change the particles
    np.testing.assert_allclose((m * b.x).sum(0), (m * a.x).sum(0), rtol=1e-13)
    np.testing.assert_array_equal(a.C, b.C)
    np.testing.assert_array_equal(a.F, b.F)


# ------------------------------------------------------------- adaptive dt

@pytest.mark.parametrize("kind", ["elastic", "snow", "sand"])
def test_wave_speed_is_the_p_wave_speed(orc, kind):
    """c^2 = E (1 - nu) / (rho (1 + nu)(1 - 2 nu)), the textbook P-wave
    modulus from E and nu (not the Lame form the oracle uses)."""
    E, nu, rho = 3.5e5, 0.3, 2200.0
    mat = orc.material(getattr(orc, kind.upper()), E=E, nu=nu, rho=rho)
    assert abs(orc.wave_speed(mat) ** 2 - E * (1 - nu) / (rho * (1 + nu) * (1 - 2 * nu))) <= 1e-12 * E / rho


def test_wave_speed_nacc_from_bulk_modulus(orc):
    """NACC takes kappa: the P-wave modulus is 3 kappa (1 - nu) / (1 + nu)."""
    k, nu, rho = 5e4, 0.3, 400.0
    c = orc.wave_speed(orc.material(orc.NACC, E=k, nu=nu, rho=rho))
    assert abs(c * c - 3 * k * (1 - nu) / ((1 + nu) * rho)) <= 1e-12 * k / rho


def test_wave_speed_fluid_from_the_stress(orc):
    """Fluid: c^2 = (bulk modulus) / rho with the bulk modulus -J dp/dJ at
    J = 1 differentiated numerically from the oracle's own stress
    (tau = -p J I)."""
    K, gamma, rho = 1e4, 7.0, 1000.0
    mat = orc.material(orc.FLUID, E=K, gamma=gamma, rho=rho)
    h = 1e-5

    def p(J):
        return -orc.kirchhoff(mat, np.eye(3), J)[0, 0] / J

    kb = -(p(1 + h) - p(1 - h)) / (2 * h)
    assert abs(orc.wave_speed(mat) ** 2 - kb / rho) <= 1e-7 * kb / rho


def test_cfl_dt_cases(orc):
    """The step takes the fastest material and the speed bound, and dt_max
    caps it: a particle moving at the wave speed halves the rest step."""
    cfg = orc.config(64, 1 / 64)
    soft = orc.material(orc.ELASTIC, E=1e3, nu=0.2, rho=1000.0)
    stiff = orc.material(orc.ELASTIC, E=1e5, nu=0.2, rho=1000.0)
    c = orc.wave_speed(stiff)
    rest = orc.cfl_dt(cfg, [soft, stiff], 0.0, 0.5, 1.0)
    assert abs(rest - 0.5 / 64 / c) <= 1e-15
    assert orc.cfl_dt(cfg, [stiff, soft], 0.0, 0.5, 1.0) == rest
    assert abs(orc.cfl_dt(cfg, [soft, stiff], c, 0.5, 1.0) - rest / 2) <= 1e-15
    assert orc.cfl_dt(cfg, [soft, stiff], 0.0, 0.5, 1e-6) == 1e-6


# -------------------------------------------------------- keys, sort, pblocks

def _morton(c, bits):
    code = 0
    for i in range(bits):
        for a in range(3):
            code |= ((int(c[a]) >> i) & 1) << (3 * i + a)
    return code


def test_keys_sort_pblocks_brute_force(orc):
    rng = np.random.default_rng(61)
    L, inv_dx = 3, 32.0          # 32^3 nodes, 8^3 blocks
    x = rng.uniform(0.05, 0.95, (500, 3)).astype(np.float32)
    x[:50] = x[50:100]           # duplicate positions -> equal keys
    keys, st = orc.particle_keys(x, inv_dx, L)
    assert st == 0
    ref = []
    for p in range(len(x)):
        b = [int(np.floor(np.float32(np.float32(x[p, a]) * np.float32(inv_dx)) - np.float32(0.5))) for a in range(3)]
        ref.append((_morton([c >> 2 for c in b], L) << 6) | _morton([c & 3 for c in b], 2))
    np.testing.assert_array_equal(keys, np.array(ref, dtype=np.uint32))
    perm = orc.stable_sort(keys)
    expect = sorted(range(len(x)), key=lambda i: (ref[i], i))
    np.testing.assert_array_equal(perm, expect)
    blocks = orc.pblocks(keys, L)
    want = set()
    for k in ref:
        code = k >> 6
        b = [sum(((code >> (3 * i + a)) & 1) << i for i in range(L)) for a in range(3)]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dxx in (-1, 0, 1):
                    c = (b[0] + dxx, b[1] + dy, b[2] + dz)
                    if min(c) >= 0 and max(c) < (1 << L):
                        want.add(_morton(c, L))
    np.testing.assert_array_equal(blocks, np.array(sorted(want), dtype=np.int32))


def test_keys_domain_error(orc):
    keys, st = orc.particle_keys(np.array([[0.001, 0.5, 0.5]], dtype=np.float32), 64.0, 4)
    assert st == 4 and keys[0] == 0xFFFFFFFF
