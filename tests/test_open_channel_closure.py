"""The closures a parity-split tau solver needs for the free-slip top, checked
against the oracle's dense tau systems.  No GPU.

The library's tau solves split every wall-normal problem by parity: for
n >= 2 the tau rows, integrated twice, are quasi-tridiagonal in the
coefficients of one parity, so elimination leaves each parity affine in its
lowest coefficient, f = P + x Q.  Under two no-slip walls each parity is
closed by its own wall sum.  Under a free-slip top the wall rows couple the
parities, and these tests pin the closures that replace the per-parity
ones (Sec. 3.1, the open channel):

* omega_y: f(-1) = sum_e f - sum_o f and Df(+1) = sum_e n^2 f + sum_o n^2 f
  give a 2 x 2 system in (x_even, x_odd);
* v: phi = D^2 v - k^2 v has both wall values unknown; with phi_1, phi_2 the
  responses to unit values at y = +1 and y = -1 (and v_1, v_2 their v), two
  influence coefficients fixed by D^2 v(+1) = 0 and Dv(-1) = 0 reproduce the
  dense system's rows exactly;
* mean U at constant flow rate: U(-1) = 0, DU(+1) = 0 and the flux row give a
  3 x 3 system in (x_even, x_odd, forcing).
"""

import numpy as np
import pytest

from oracle import channel


def _ops(ny):
    return channel.Operators(channel.Params(nx=4, ny=ny, nz=4, lx=2 * np.pi, lz=np.pi, top_bc=1))


def _split_solve(N, lam, r, sig):
    """Parity sig of (D^2 - lam) f = r by the quasi-tridiagonal rows
    -lam cA_n f_{n-2} + (1 + lam cB_n) f_n - lam cC_n f_{n+2}
        = cA_n r_{n-2} - cB_n r_n + cC_n r_{n+2}   (n = 2i + sig >= 2),
    eliminated from the top: f_i = a_i + beta_i f_{i-1}.  Returns (P, Q) with
    f_i = P_i + Q_i f_0 and the parity's degrees n_i."""
    M = (N - sig) // 2 + 1
    n = 2 * np.arange(M) + sig
    c = lambda k: 2.0 if k == 0 else 1.0
    a = np.zeros(M, complex)
    beta = np.zeros(M)
    anext, bnext = 0.0, 0.0
    for i in range(M - 1, 0, -1):
        ni = n[i]
        cA = c(ni - 2) / (4.0 * ni * (ni - 1))
        cB = (1.0 if ni <= N - 2 else 0.0) / (2.0 * (ni * ni - 1))
        cC = (1.0 if ni + 2 <= N - 2 else 0.0) / (4.0 * ni * (ni + 1))
        R = cA * r[ni - 2] - cB * r[ni] + (cC * r[ni + 2] if ni + 2 <= N else 0.0)
        L, D, U = -lam * cA, 1.0 + lam * cB, -lam * cC
        den = D + U * bnext
        a[i] = (R - U * anext) / den
        beta[i] = -L / den
        anext, bnext = a[i], beta[i]
    P = np.zeros(M, complex)
    Q = np.zeros(M)
    Q[0] = 1.0
    for i in range(1, M):
        P[i] = a[i] + beta[i] * P[i - 1]
        Q[i] = beta[i] * Q[i - 1]
    return P, Q, n


def _assemble(N, parts):
    f = np.zeros(N + 1, complex)
    for (P, Q, n), x in parts:
        f[n] = P + x * Q
    return f


@pytest.mark.parametrize("ny", [17, 65])
def test_parity_split_with_wall_sums_is_the_dense_dirichlet_solve(ny):
    """The recurrences themselves: two no-slip walls, one closure per parity."""
    ops = _ops(ny)
    N = ops.N
    rng = np.random.default_rng(ny)
    for lam in (0.7, 3e2, 3.4e6):
        r = rng.standard_normal(N + 1) + 1j * rng.standard_normal(N + 1)
        top, bot = 0.3 - 0.1j, -0.2 + 0.5j
        parts = []
        for sig, s in ((0, (top + bot) / 2), (1, (top - bot) / 2)):
            P, Q, n = _split_solve(N, lam, r, sig)
            parts.append(((P, Q, n), (s - P.sum()) / Q.sum()))
        f = _assemble(N, parts)
        want = channel.tau_dirichlet(ops, np.array([lam]), r[None], np.array([top]), np.array([bot]))[0]
        assert np.max(np.abs(f - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("ny", [17, 65])
def test_coupled_parity_closure_for_a_neumann_top(ny):
    ops = _ops(ny)
    N = ops.N
    rng = np.random.default_rng(ny + 1)
    for lam in (0.7, 3e2, 3.4e6):
        r = rng.standard_normal(N + 1) + 1j * rng.standard_normal(N + 1)
        top, bot = 0.0, 0.0   # Df(+1) = 0, f(-1) = 0: omega_y under a free-slip top
        (Pe, Qe, ne), (Po, Qo, no) = _split_solve(N, lam, r, 0), _split_solve(N, lam, r, 1)
        S = lambda v: v.sum()
        T = lambda v, n: (n * n * v).sum()
        A = np.array([[S(Qe), -S(Qo)], [T(Qe, ne), T(Qo, no)]])
        b = np.array([bot - S(Pe) + S(Po), top - T(Pe, ne) - T(Po, no)])
        xe, xo = np.linalg.solve(A.astype(complex), b)
        f = _assemble(N, [((Pe, Qe, ne), xe), ((Po, Qo, no), xo)])
        want = channel.tau_dirichlet(ops, np.array([lam]), r[None], np.array([top]), np.array([bot]),
                                     top_neumann=True)[0]
        assert np.max(np.abs(f - want)) <= 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("ny", [17, 65])
def test_two_influence_coefficients_close_the_free_slip_v_problem(ny):
    ops = _ops(ny)
    N = ops.N
    rng = np.random.default_rng(ny + 2)
    d2top = ops.d2Tp          # T_n''(+1)
    dbot = ops.dTm            # T_n'(-1)
    for k2, lam_extra in ((1.0, 2.0), (50.0, 1e4), (400.0, 3.4e6)):
        lam = k2 + lam_extra
        r = rng.standard_normal(N + 1) + 1j * rng.standard_normal(N + 1)
        vw = 0.3 + 0.2j
        L = np.array([lam])
        K = np.array([k2])
        zero, one = np.zeros(1), np.ones(1)
        # particular part: phi_p(+-1) = 0, v_p(+1) = 0, v_p(-1) = vw
        phi_p = channel.tau_dirichlet(ops, L, r[None], zero, zero)[0]
        v_p = channel.tau_dirichlet(ops, K, phi_p[None], zero, np.array([vw]))[0]
        # responses to unit phi at the top and at the bottom, v zero at both walls
        phi_1 = channel.tau_dirichlet(ops, L, np.zeros((1, N + 1)), one, zero)[0]
        v_1 = channel.tau_dirichlet(ops, K, phi_1[None], zero, zero)[0]
        phi_2 = channel.tau_dirichlet(ops, L, np.zeros((1, N + 1)), zero, one)[0]
        v_2 = channel.tau_dirichlet(ops, K, phi_2[None], zero, zero)[0]
        A = np.array([[d2top @ v_1, d2top @ v_2], [dbot @ v_1, dbot @ v_2]])
        c1, c2 = np.linalg.solve(A.astype(complex), -np.array([d2top @ v_p, dbot @ v_p]))
        v = v_p + c1 * v_1 + c2 * v_2
        want = channel.coupled_v(ops, L, K, r[None], np.array([vw]))[0]
        assert np.max(np.abs(v - want)) <= 1e-10 * np.max(np.abs(want)), (k2, lam)


@pytest.mark.parametrize("ny", [17, 65])
def test_three_unknown_closure_for_the_mean_flow_at_constant_flow_rate(ny):
    """Mean U under a free-slip top: the parity-split parts, the response to the
    forcing (it enters the n = 0 tau row, so only the even parity), and the
    3 x 3 closure U(-1) = 0, DU(+1) = 0, int U dy = flux in (x_even, x_odd, f)."""
    ops = _ops(ny)
    N = ops.N
    rng = np.random.default_rng(ny + 3)
    w = ops.wint                                    # int_{-1}^{1} T_n dy
    for lam0, cforce in ((5.0, 3.0), (4.8e5, 2.2e6)):
        r = rng.standard_normal(N + 1)
        rF = np.zeros(N + 1)
        rF[0] = -cforce                             # the forcing term moved to the right-hand side
        (Pe, Qe, ne), (Po, Qo, no) = _split_solve(N, lam0, r, 0), _split_solve(N, lam0, r, 1)
        PF = _split_solve(N, lam0, rF, 0)[0]
        S = lambda v: v.sum()
        T = lambda v, n: (n * n * v).sum()
        I = lambda v, n: (w[n] * v).sum()
        A = np.array([[S(Qe), -S(Qo), S(PF)],
                      [T(Qe, ne), T(Qo, no), T(PF, ne)],
                      [I(Qe, ne), 0.0, I(PF, ne)]]).real
        b = np.array([-S(Pe) + S(Po), -T(Pe, ne) - T(Po, no), 2.0 - I(Pe, ne)]).real
        xe, xo, f = np.linalg.solve(A, b)
        U = np.zeros(N + 1)
        U[ne] = (Pe + f * PF + xe * Qe).real
        U[no] = (Po + xo * Qo).real
        want_U, want_f = channel.mean_cfr(ops, lam0, cforce, r)
        assert np.max(np.abs(U - want_U)) <= 1e-11 * np.max(np.abs(want_U))
        assert abs(f - want_f) <= 1e-10 * abs(want_f)
