"""The algebra behind the per-thread no-slip solves, checked on the CPU
against the FP64 oracle's dense operators (no CUDA path involved).

The tau rows n >= 2 of (D^2 - lam) f = r, integrated twice, read
    -lam cA_n f_{n-2} + (1 + lam cB_n) f_n - lam cC_n f_{n+2}
        = cA_n r_{n-2} - cB_n r_n + cC_n r_{n+2},
with cA_n = c_{n-2} / (4 n (n - 1)), cB_n = [n <= N-2] / (2 (n^2 - 1)),
cC_n = [n + 2 <= N-2] / (4 n (n + 1)) (paper Sec. 3.1: Chebyshev-tau in y).
Per parity the rows are tridiagonal in i = (n - parity) / 2, and the wall row
sum_i f_i = s closes them.  The solves eliminate from the top,
a_i = e_i R_i - h_i a_{i+1}, and
  1. take the wall sum of the particular solution P_i = a_i + b_i P_{i-1}
     (P_0 = 0) as sum_i W_i a_i, W_{M-1} = 1, W_i = 1 + b_{i+1} W_{i+1};
  2. then f_0 = (s - sum P) / sum Q (Q_i = prod_{m <= i} b_m) and
     f_i = a_i + b_i f_{i-1} in one pass;
and the phi solve of v uses that the stencil of D^2 v is v itself (n >= 2).
"""

import numpy as np
import pytest

from oracle import channel, spectral


def c_a(n):
    return (2.0 if n == 2 else 1.0) / (4.0 * n * (n - 1))


def c_b(n, N):
    return 1.0 / (2.0 * (n * n - 1.0)) if n <= N - 2 else 0.0


def c_c(n, N):
    return 1.0 / (4.0 * n * (n + 1)) if n + 2 <= N - 2 else 0.0


def folded_parity_solve(N, sig, lam, r, s):
    """One parity of (D^2 - lam) f = r with sum_i f_i = s, by the folded rows
    (eA, eB, eC = e cA, e cB, e cC), the W-weighted wall sum and one back
    substitution; r, f indexed by i (n = 2 i + sig)."""
    M = (N - sig) // 2 + 1
    e, h, b = np.zeros(M), np.zeros(M), np.zeros(M)
    bnext = 0.0
    for i in range(M - 1, 0, -1):
        n = 2 * i + sig
        U = -lam * c_c(n, N) if i + 1 < M else 0.0
        den = 1.0 + lam * c_b(n, N) + U * bnext
        e[i], h[i], b[i] = 1.0 / den, U / den, lam * c_a(n) / den
        bnext = b[i]
    W = np.zeros(M)
    w = 1.0
    for i in range(M - 1, 0, -1):
        if i < M - 1:
            w = 1.0 + b[i + 1] * w
        W[i] = w
    Q = np.cumprod(np.concatenate([[1.0], b[1:]]))
    a = np.zeros(M)
    anext, sumP = 0.0, 0.0
    for i in range(M - 1, 0, -1):
        n = 2 * i + sig
        R = (e[i] * c_a(n)) * r[i - 1] - (e[i] * c_b(n, N)) * r[i]
        if i + 1 < M:
            R += (e[i] * c_c(n, N)) * r[i + 1]
        a[i] = R - h[i] * anext
        anext = a[i]
        sumP += W[i] * a[i]
    f = np.zeros(M)
    f[0] = (s - sumP) / Q.sum()
    for i in range(1, M):
        f[i] = a[i] + b[i] * f[i - 1]
    return f


@pytest.mark.parametrize("ny", [17, 33, 65])
@pytest.mark.parametrize("lam", [0.0, 3.7, 250.0, 4.0e4])
def test_folded_rows_match_the_dense_tau_solve(ny, lam):
    N = ny - 1
    ops = channel.Operators(channel.Params(nx=4, ny=ny, nz=4, lx=1.0, lz=1.0, re_tau=180.0, re_bulk=2800.0,
                                           dt=0.005))
    rng = np.random.default_rng(ny + int(lam))
    r = rng.standard_normal(N + 1)
    top, bottom = rng.standard_normal(2)
    ref = channel.tau_dirichlet(ops, np.array([lam]), r[None, :].astype(np.complex128), np.array([top + 0j]),
                                np.array([bottom + 0j])).real[0]
    f = np.zeros(N + 1)
    for sig in (0, 1):
        s = 0.5 * (top + bottom) if sig == 0 else 0.5 * (top - bottom)  # sum over the parity's coefficients
        f[sig::2] = folded_parity_solve(N, sig, lam, r[sig::2], s)
    assert np.linalg.norm(f - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref))


@pytest.mark.parametrize("M", [3, 9, 33])
def test_wall_weights_sum_the_particular_solution(M):
    """sum_i P_i = sum_i W_i a_i for any a and b, and a_i + b_i f_{i-1} from
    f_0 reproduces P_i + Q_i f_0."""
    rng = np.random.default_rng(M)
    a, b = rng.standard_normal(M), rng.uniform(-0.5, 0.5, M)
    a[0] = b[0] = 0.0
    P = np.zeros(M)
    for i in range(1, M):
        P[i] = a[i] + b[i] * P[i - 1]
    W = np.zeros(M)
    w = 1.0
    for i in range(M - 1, 0, -1):
        if i < M - 1:
            w = 1.0 + b[i + 1] * w
        W[i] = w
    assert abs(P.sum() - (W * a).sum()) <= 1e-13 * max(1.0, np.abs(P).sum())
    f0 = 0.7
    Q = np.cumprod(np.concatenate([[1.0], b[1:]]))
    f = np.zeros(M)
    f[0] = f0
    for i in range(1, M):
        f[i] = a[i] + b[i] * f[i - 1]
    assert np.allclose(f, P + Q * f0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("ny", [9, 33, 65, 129])
def test_row_stencil_of_d2_is_the_field(ny):
    """cA_n (D^2 v)_{n-2} - cB_n (D^2 v)_n + cC_n (D^2 v)_{n+2} = v_n for n >= 2,
    with D^2 the oracle's coefficient-space second derivative."""
    N = ny - 1
    v = np.random.default_rng(ny).standard_normal(N + 1)
    D = spectral.cheb_diff(N)
    d2 = D @ D @ v
    for n in range(2, N + 1):
        terms = [c_a(n) * d2[n - 2], -c_b(n, N) * d2[n], c_c(n, N) * d2[n + 2] if n + 2 <= N else 0.0]
        # the D^2 v coefficients grow like n^4: the sum cancels terms up to 1e7
        # at 129 nodes, so the rounding scales with their size, while a wrong
        # constant or index leaves an error of the size of v
        assert abs(sum(terms) - v[n]) <= 1e-13 * (sum(abs(t) for t in terms) + abs(v[n])), n
