"""Pins of the oracle's Chebyshev-tau solvers with manufactured solutions.

The right-hand sides are built with numpy's Chebyshev-series routines
(``chebder``, ``chebmul``), not with the oracle's own matrices, so a wrong
row, sign or boundary row in the oracle fails here.
"""

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import channel


def _ops(ny=65, nx=4, nz=4, **kw):
    return channel.Operators(channel.Params(nx=nx, ny=ny, nz=nz, lx=2 * np.pi, lz=np.pi, **kw))


def _pad(c, n1):
    out = np.zeros(n1, dtype=np.result_type(c, float))
    out[: len(c)] = c
    return out


@pytest.mark.parametrize("ny", [9, 65, 129])
def test_helmholtz_dirichlet_manufactured(ny):
    ops = _ops(ny)
    N = ops.N
    rng = np.random.default_rng(ny)
    P = 5
    lam = np.array([0.5, 3.0, 1e3, 3.4e6, 12.0])
    f = rng.standard_normal((P, N + 1)) + 1j * rng.standard_normal((P, N + 1))
    r = np.array([_pad(npc.chebder(fi, 2), N + 1) - li * fi for fi, li in zip(f, lam)])
    top = npc.chebval(1.0, f.T)
    bot = npc.chebval(-1.0, f.T)
    sol = channel.tau_dirichlet(ops, lam, r, top, bot)
    err = np.max(np.abs(sol - f)) / np.max(np.abs(f))
    # random coefficients up to T_N: the tau system's conditioning grows like N^4
    assert err < 1e-17 * N ** 4 + 1e-13, err


def _quartic_shape(N):
    """(1 - y^2)^2 as Chebyshev coefficients via numpy."""
    return npc.chebmul(npc.chebmul([0.5, 0, -0.5], [0.5, 0, -0.5]), [1.0])


@pytest.mark.parametrize("ny", [17, 65])
def test_coupled_v_manufactured(ny):
    """v = (1-y^2)^2 p(y) + vw q(y) with q(-1)=1, q(1)=0, q'(+-1)=0 is recovered."""
    ops = _ops(ny)
    N = ops.N
    rng = np.random.default_rng(ny + 1)
    P = 4
    k2 = np.array([1.0, 7.3, 50.0, 400.0])
    lam = k2 + np.array([2.0, 1e4, 3.4e6, 10.0])
    vw = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    # q = (1-y)^2 (2+y) / 4
    q = npc.chebmul(npc.chebmul([1.0, -1.0], [1.0, -1.0]), [2.0, 1.0]) / 4.0
    assert abs(npc.chebval(-1.0, q) - 1) < 1e-15 and abs(npc.chebval(1.0, q)) < 1e-15
    sh = _quartic_shape(N)
    v = np.zeros((P, N + 1), complex)
    r = np.zeros((P, N + 1), complex)
    for i in range(P):
        # smooth profile: geometrically decaying Chebyshev coefficients
        p = (rng.standard_normal(N - 3) + 1j * rng.standard_normal(N - 3)) * 0.8 ** np.arange(N - 3)
        vi = _pad(npc.chebmul(sh, p), N + 1) + vw[i] * _pad(q, N + 1)
        phi = _pad(npc.chebder(vi, 2), N + 1) - k2[i] * vi
        ri = _pad(npc.chebder(phi, 2), N + 1) - lam[i] * phi
        v[i], r[i] = vi, ri
    sol = channel.coupled_v(ops, lam, k2, r, vw)
    err = np.max(np.abs(sol - v)) / np.max(np.abs(v))
    assert err < 1e-11, err
    # the four wall conditions hold to roundoff
    assert np.allclose(npc.chebval(1.0, sol.T), 0, atol=1e-10)
    assert np.allclose(npc.chebval(-1.0, sol.T), vw, atol=1e-10)
    for i in range(P):
        d = npc.chebder(sol[i])
        assert abs(npc.chebval(1.0, d)) < 1e-8 and abs(npc.chebval(-1.0, d)) < 1e-8


def test_coupled_v_random_rhs_satisfies_wall_conditions():
    ops = _ops(65)
    N = ops.N
    rng = np.random.default_rng(3)
    P = 6
    k2 = rng.uniform(0.5, 500, P)
    lam = k2 + 1.0 / (1.0 / 6.0 * 0.005 / 2800.0)
    r = rng.standard_normal((P, N + 1)) + 1j * rng.standard_normal((P, N + 1))
    vw = rng.standard_normal(P) * 1e-2 + 0j
    sol = channel.coupled_v(ops, lam, k2, r, vw)
    scale = np.max(np.abs(sol))
    assert np.allclose(npc.chebval(1.0, sol.T), 0, atol=1e-12 * scale + 1e-14)
    assert np.allclose(npc.chebval(-1.0, sol.T), vw, atol=1e-12 * scale + 1e-14)
    for i in range(P):
        d = npc.chebder(sol[i])
        assert abs(npc.chebval(1.0, d)) < 1e-9 * scale * N * N
        assert abs(npc.chebval(-1.0, d)) < 1e-9 * scale * N * N


def test_mean_cfr_fixed_point_is_poiseuille():
    """U = 1.5 (1 - y^2) with forcing 3 nu solves the CFR mean problem of any stage."""
    ops = _ops(65)
    nu, dt = ops.p.nu, ops.p.dt
    U = np.zeros(ops.N + 1)
    U[0], U[2] = 0.75, -0.75
    for k in range(3):
        a, b = channel.ALPHA[k], channel.BETA[k]
        bdn = b * dt * nu
        rU = -(U + a * dt * nu * _pad(npc.chebder(U, 2), ops.N + 1)) / bdn
        Un, fx = channel.mean_cfr(ops, 1.0 / bdn, (a + b) / (b * nu), rU)
        assert np.max(np.abs(Un - U)) < 1e-12
        assert abs(fx - 3.0 * nu) < 1e-9 * 3.0 * nu
        # flow rate fixed: int U = 2
        assert abs(npc.chebval(1, npc.chebint(Un)) - npc.chebval(-1, npc.chebint(Un)) - 2.0) < 1e-13
