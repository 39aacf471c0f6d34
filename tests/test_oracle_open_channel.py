"""Pins of the oracle's open channel (Sec. 3.1: an open channel of height h,
free slip at the top): the Neumann top row of the Helmholtz solve, the
free-slip v problem, the half-Poiseuille laminar state held steady at
constant flow rate with its reward, and the sensing node in wall units of
the open channel.  Manufactured solutions and profiles are built with numpy's
polynomial routines, not the oracle's matrices.  No GPU."""

import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

import golden_util
from oracle import channel


def _params(**kw):
    base = dict(nx=4, ny=65, nz=4, lx=2 * np.pi, lz=np.pi, top_bc=1)
    base.update(kw)
    return channel.Params(**base)


def _pad(c, n1):
    out = np.zeros(n1, dtype=np.result_type(c, float))
    out[: len(c)] = c
    return out


@pytest.mark.parametrize("ny", [17, 65])
def test_helmholtz_neumann_top_manufactured(ny):
    ops = channel.Operators(_params(ny=ny))
    N = ops.N
    rng = np.random.default_rng(ny)
    P = 4
    lam = np.array([0.5, 30.0, 1e4, 3.4e6])
    f = (rng.standard_normal((P, N + 1)) + 1j * rng.standard_normal((P, N + 1))) * 0.7 ** np.arange(N + 1)
    r = np.array([_pad(npc.chebder(fi, 2), N + 1) - li * fi for fi, li in zip(f, lam)])
    top = np.array([npc.chebval(1.0, npc.chebder(fi)) for fi in f])   # f'(+1)
    bot = npc.chebval(-1.0, f.T)
    sol = channel.tau_dirichlet(ops, lam, r, top, bot, top_neumann=True)
    assert np.max(np.abs(sol - f)) / np.max(np.abs(f)) < 1e-11


def _free_slip_shape(p_coef):
    """s = (1+y)^2 (1-y) p + c (1-y^2)^2 with s(-1) = s'(-1) = s(1) = s''(1) = 0."""
    g = npc.chebmul(npc.chebmul([1.0, 1.0], [1.0, 1.0]), [1.0, -1.0])
    s = npc.chebmul(g, p_coef)
    h = npc.chebmul([0.5, 0, -0.5], [0.5, 0, -0.5])          # (1 - y^2)^2, h''(1) = 8
    c = -npc.chebval(1.0, npc.chebder(s, 2)) / npc.chebval(1.0, npc.chebder(h, 2))
    return npc.chebadd(s, c * h)


def _free_slip_lift():
    """Cubic q with q(-1) = 1, q'(-1) = 0, q(1) = 0, q''(1) = 0 (power basis solve)."""
    A = np.array([[1, -1, 1, -1], [0, 1, -2, 3], [1, 1, 1, 1], [0, 0, 2, 6]], float)
    a = np.linalg.solve(A, [1.0, 0.0, 0.0, 0.0])
    return npc.poly2cheb(a)


@pytest.mark.parametrize("ny", [17, 65])
def test_free_slip_v_manufactured(ny):
    ops = channel.Operators(_params(ny=ny))
    N = ops.N
    rng = np.random.default_rng(ny + 5)
    P = 4
    k2 = np.array([1.0, 7.3, 50.0, 400.0])
    lam = k2 + np.array([2.0, 1e4, 3.4e6, 10.0])
    vw = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    q = _free_slip_lift()
    v = np.zeros((P, N + 1), complex)
    r = np.zeros((P, N + 1), complex)
    for i in range(P):
        pc = (rng.standard_normal(N - 4) + 1j * rng.standard_normal(N - 4)) * 0.8 ** np.arange(N - 4)
        vi = _pad(_free_slip_shape(pc), N + 1) + vw[i] * _pad(q, N + 1)
        phi = _pad(npc.chebder(vi, 2), N + 1) - k2[i] * vi
        v[i] = vi
        r[i] = _pad(npc.chebder(phi, 2), N + 1) - lam[i] * phi
    sol = channel.coupled_v(ops, lam, k2, r, vw)
    assert np.max(np.abs(sol - v)) / np.max(np.abs(v)) < 1e-11
    # the four conditions: v(1) = 0, v(-1) = vw, D^2 v(1) = 0, Dv(-1) = 0
    assert np.allclose(npc.chebval(1.0, sol.T), 0, atol=1e-10)
    assert np.allclose(npc.chebval(-1.0, sol.T), vw, atol=1e-10)
    for i in range(P):
        assert abs(npc.chebval(1.0, npc.chebder(sol[i], 2))) < 1e-6
        assert abs(npc.chebval(-1.0, npc.chebder(sol[i]))) < 1e-8


def _half_poiseuille(N):
    """U = 1.5 (2 s - s^2), s = (1 + y) / 2: no slip at y = -1, DU(1) = 0, int U dy = 2."""
    a = np.array([1.5 * (1.0 - 0.25), 1.5 * (1.0 - 0.5), -1.5 * 0.25])  # power-basis coefficients
    return _pad(npc.poly2cheb(a), N + 1)


def test_half_poiseuille_steady_at_constant_flow_rate_and_laminar_reward():
    p = _params()
    ops = channel.Operators(p)
    N = ops.N
    U = _half_poiseuille(N)
    assert abs(npc.chebval(1.0, npc.chebder(U))) < 1e-15
    assert abs(npc.chebval(1, npc.chebint(U)) - npc.chebval(-1, npc.chebint(U)) - 2.0) < 1e-14
    ny, nz, nxh = p.ny, p.nz, p.nx // 2
    zero3 = np.zeros((ny, nz, nxh), complex)
    st = channel.new_state({"v": zero3, "g": zero3, "U": U, "W": np.zeros(ny)}, p)
    zero = np.zeros((p.nz, p.nx))
    for _ in range(50):
        obs, tau, reward = channel.env_step(st, ops, zero)
    assert np.abs(st["U"] - U).max() < 1e-12
    # nu D^2 U + f = 0 with D^2 U = -0.75
    assert abs(st["fx"] - 0.75 * p.nu) < 1e-9 * 0.75 * p.nu
    # nu = 2 / Re_b (Re_b on the height h = 2): tau_lam = 1.5 nu = 3 / Re_b, the
    # closed channel's value, so the laminar bound is the same closed form
    assert abs(p.nu - 2.0 / p.re_bulk) < 1e-18
    assert abs(tau - 3.0 / p.re_bulk) < 1e-13
    bound = golden_util.load("laminar_drag_bound.txt")
    assert abs(reward - bound["closed_form"]) < 1e-9
    ys = math.cos(math.pi * ops.js / ops.N)
    s = (1 + ys) / 2
    assert np.allclose(obs[0], 1.5 * (2 * s - s * s), atol=1e-13)
    assert np.abs(obs[1]).max() < 1e-15


def test_open_channel_sensing_node_in_wall_units():
    # y+ = (1 + y) Re_tau / 2 over the open channel; Ny = 65, Re_tau = 180
    p = _params(ny=65, re_tau=180.0, y_sense_plus=15.0)
    ops = channel.Operators(p)
    yplus = lambda j: (1.0 + math.cos(math.pi * j / ops.N)) * 90.0
    assert yplus(ops.js) >= 15.0 > yplus(ops.js + 1)
    assert abs(yplus(ops.js) - 90.0 * (1.0 - math.cos(12 * math.pi / 64))) < 1e-12  # 15.17
    assert abs(yplus(ops.js) - 15.17) < 0.01
    # the closed channel puts the same request at y+ = 17.28 (node 9 from the wall)
    closed = channel.Operators(channel.Params(nx=4, ny=65, nz=4, lx=1.0, lz=1.0))
    assert abs((1.0 + math.cos(math.pi * closed.js / 64)) * 180.0 - 17.28) < 0.01


def test_free_slip_diffusion_modes_decay_at_the_scheme_rate():
    """A mean-only flow has H = (0, W DW + U DU, 0), so W diffuses freely; with
    W(-1) = 0 and DW(1) = 0 its slowest mode sin(pi (1 + y) / 4) has the
    eigenvalue -pi^2/16.  Under the half-Poiseuille U and W = 0, a small
    kx = 0 omega_y mode with the same profile diffuses too (no advection along
    z, and its products are second order), with -(pi^2/16 + kz^2).  After n
    steps each has been multiplied by the scheme's amplification
    prod_k (1 + alpha_k dt nu mu) / (1 - beta_k dt nu mu)."""
    p = _params(ny=65, dt=0.005)
    ops = channel.Operators(p)
    N, ny, nz, nxh = ops.N, p.ny, p.nz, p.nx // 2
    prof = npc.chebinterpolate(lambda y: np.sin(np.pi * (1 + y) / 4), N)
    n = 20
    zero = np.zeros((p.nz, p.nx))

    def amp(mu):
        a = 1.0
        for al, be in zip(channel.ALPHA, channel.BETA):
            a *= (1 + al * p.dt * p.nu * mu) / (1 - be * p.dt * p.nu * mu)
        return a ** n

    muW = -np.pi ** 2 / 16
    zero3 = np.zeros((ny, nz, nxh), complex)
    st = channel.new_state({"v": zero3, "g": zero3, "U": _half_poiseuille(N), "W": prof.copy()}, p)
    for _ in range(n):
        channel.env_step(st, ops, zero)
    assert np.max(np.abs(st["W"] - amp(muW) * prof)) < 1e-12
    # the decay (4.4e-5 of the profile) is far above that tolerance
    assert np.max(np.abs(st["W"] - prof)) > 1e-5

    g = np.zeros((ny, nz, nxh), complex)
    eps = 1e-7
    g[:, 1, 0] = eps * prof          # kz index 1 and its conjugate partner (real field)
    g[:, nz - 1, 0] = eps * prof
    st = channel.new_state({"v": zero3, "g": g, "U": _half_poiseuille(N), "W": np.zeros(ny)}, p)
    for _ in range(n):
        channel.env_step(st, ops, zero)
    kz = 2 * np.pi / p.lz
    gn = channel.from_pencils(st["g"])[:, 1, 0]
    assert np.max(np.abs(gn - amp(muW - kz * kz) * eps * prof)) < 1e-9 * eps
