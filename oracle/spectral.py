"""Chebyshev and Fourier operators of the oracle (TEST INFRASTRUCTURE ONLY).

Sec. 3.1 of the paper: Fourier modes in the streamwise (x) and spanwise (z)
directions, Chebyshev polynomials in the wall-normal direction (y).  All
operators are dense matrices written from their textbook definitions.

Conventions
-----------
* Chebyshev Gauss-Lobatto nodes ``y_j = cos(pi j / N)``, ``j = 0..N``,
  ``N = ny - 1``; ``j = 0`` is the upper wall ``y = +1``, ``j = N`` the lower
  wall ``y = -1``.
* A wall-normal profile is stored as its Chebyshev coefficients ``a_n``,
  ``f(y) = sum_n a_n T_n(y)``.
* Fourier: ``f(x, z) = sum_k f_k exp(i (kx x + kz z))`` with the kept
  half-spectrum ``kx index 0..nx/2-1`` and ``kz index -(nz/2-1)..nz/2-1``
  stored in FFT row order; the ``-nz/2`` (Nyquist) row is zero.
"""

from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# Chebyshev (y)
# --------------------------------------------------------------------------

def cheb_nodes(N: int) -> np.ndarray:
    """Gauss-Lobatto nodes y_j = cos(pi j / N)."""
    return np.cos(np.pi * np.arange(N + 1) / N)


def _cos_pi_over(N: int) -> np.ndarray:
    """C[j, n] = cos(pi j n / N), the integer argument j n reduced mod 2N first."""
    j = np.arange(N + 1)
    return np.cos(np.pi * (np.outer(j, j) % (2 * N)) / N)


def cheb_synthesis(N: int) -> np.ndarray:
    """S[j, n] = T_n(y_j) = cos(pi n j / N): coefficients -> node values."""
    return _cos_pi_over(N)


def cheb_analysis(N: int) -> np.ndarray:
    """A[n, j]: node values -> coefficients of the interpolating polynomial.

    a_n = 2 / (N cbar_n) * sum_j f_j cos(pi n j / N) / cbar_j with
    cbar_0 = cbar_N = 2 and cbar = 1 otherwise (discrete Chebyshev transform
    at the Gauss-Lobatto nodes).
    """
    cbar = np.ones(N + 1)
    cbar[0] = cbar[N] = 2.0
    return 2.0 / N * _cos_pi_over(N) / np.outer(cbar, cbar)


def cheb_diff(N: int) -> np.ndarray:
    """Coefficient-space first derivative: (D a)_m = (2 / c_m) sum_{n>m, n+m odd} n a_n.

    c_0 = 2, c_m = 1 for m >= 1.
    """
    D = np.zeros((N + 1, N + 1))
    for m in range(N + 1):
        cm = 2.0 if m == 0 else 1.0
        for n in range(m + 1, N + 1):
            if (n + m) % 2 == 1:
                D[m, n] = 2.0 * n / cm
    return D


def cheb_at_plus1(N: int) -> np.ndarray:
    """T_n(+1) = 1."""
    return np.ones(N + 1)


def cheb_at_minus1(N: int) -> np.ndarray:
    """T_n(-1) = (-1)^n."""
    return (-1.0) ** np.arange(N + 1)


def cheb_integral(N: int) -> np.ndarray:
    """w_n = int_{-1}^{1} T_n dy = 2 / (1 - n^2) for even n, 0 for odd n."""
    n = np.arange(N + 1)
    w = np.zeros(N + 1)
    even = n % 2 == 0
    w[even] = 2.0 / (1.0 - n[even] ** 2)
    return w


# --------------------------------------------------------------------------
# Fourier (x, z)
# --------------------------------------------------------------------------

def kz_index(nz: int) -> np.ndarray:
    """Integer kz index of each storage row (FFT order)."""
    return np.concatenate([np.arange(0, nz // 2), np.arange(-nz // 2, 0)])


def wavenumbers(nx: int, nz: int, lx: float, lz: float):
    """kx[i] = 2 pi i / Lx (i < nx/2), kz[row] = 2 pi m / Lz; mask of kept rows."""
    kx = 2.0 * np.pi / lx * np.arange(nx // 2)
    m = kz_index(nz)
    kz = 2.0 * np.pi / lz * m
    kept = m != -nz // 2
    return kx, kz, kept


def _dft_mats(nx: int, nz: int, mx: int, mz: int):
    """Ex[a, i] = exp(2 pi i i a / mx), Ez[b, row] = exp(2 pi i m(row) b / mz)."""
    a = np.arange(mx)
    i = np.arange(nx // 2)
    Ex = np.exp(2j * np.pi * (np.outer(a, i) % mx) / mx)
    b = np.arange(mz)
    m = kz_index(nz)
    Ez = np.exp(2j * np.pi * (np.outer(b, m) % mz) / mz)
    return Ex, Ez


def to_physical(F: np.ndarray, nx: int, nz: int, mx: int, mz: int) -> np.ndarray:
    """Evaluate half-spectrum fields on an mz x mx grid.

    ``F[..., nz, nx/2]`` -> ``f[..., mz, mx]`` with
    ``f(x_a, z_b) = Re sum_{kz} F[kz, 0] e^{i kz z_b}
                    + 2 Re sum_{kx>0, kz} F[kz, kx] e^{i (kx x_a + kz z_b)}``,
    ``x_a = a Lx / mx``, ``z_b = b Lz / mz``.  With ``mx = 3 nx / 2`` and
    ``mz = 3 nz / 2`` this is the 3/2-padded grid of the dealiased product.
    The Nyquist row is skipped (zero by convention).
    """
    Ex, Ez = _dft_mats(nx, nz, mx, mz)
    kept = kz_index(nz) != -nz // 2
    w = np.full(nx // 2, 2.0)
    w[0] = 1.0
    Fk = F * w * kept[:, None]
    # sum over kz, then over kx: Ez @ Fk @ Ex^T
    return np.real(np.matmul(np.matmul(Ez, Fk), Ex.T))


def to_spectral(f: np.ndarray, nx: int, nz: int, mx: int, mz: int) -> np.ndarray:
    """Fourier coefficients of the kept modes of a real ``[..., mz, mx]`` grid field.

    ``F[kz, kx] = 1/(mx mz) sum_{a,b} f(x_a, z_b) e^{-i (kx x_a + kz z_b)}``;
    the Nyquist row is set to zero (truncation after the dealiased product).
    """
    Ex, Ez = _dft_mats(nx, nz, mx, mz)
    kept = kz_index(nz) != -nz // 2
    F = np.matmul(np.matmul(np.conj(Ez).T, f), np.conj(Ex)) / (mx * mz)
    return F * kept[:, None]
