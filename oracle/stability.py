"""Orr-Sommerfeld eigenvalue problem of plane Poiseuille flow (TEST INFRASTRUCTURE ONLY).

Used to pin the linear dynamics of the time step: a small Tollmien-Schlichting
wave of the laminar profile ``U = 1 - y^2`` (centre-line units) at Re = 10^4
and streamwise wavenumber alpha = 1 grows at the amplitude rate
``alpha c_i = 0.00373967``.  The eigenproblem is solved independently of the
time stepper: Chebyshev-tau in coefficient space, generalised eigenvalues by
``scipy.linalg.eig``.

    (U - c)(D^2 - a^2) v - U'' v = (D^2 - a^2)^2 v / (i a Re),
    v(+-1) = Dv(+-1) = 0.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg

from . import spectral as sp


def mult_y(N: int) -> np.ndarray:
    """Coefficient-space multiplication by y: y T_0 = T_1, y T_n = (T_{n+1} + T_{n-1}) / 2."""
    Y = np.zeros((N + 1, N + 1))
    for n in range(N + 1):
        if n == 0:
            if N >= 1:
                Y[1, 0] = 1.0
            continue
        Y[n - 1, n] += 0.5
        if n + 1 <= N:
            Y[n + 1, n] += 0.5
    return Y


def orr_sommerfeld(N: int, alpha: float, re: float):
    """All finite eigenvalues c and eigenvectors (Chebyshev coefficients of v)."""
    D = sp.cheb_diff(N)
    I = np.eye(N + 1)
    D2 = D @ D
    Y = mult_y(N)
    Umat = I - Y @ Y                  # multiplication by 1 - y^2
    Upp = -2.0 * I                    # U'' = -2
    L = D2 - alpha ** 2 * I
    A = Umat @ L - Upp - (L @ L) / (1j * alpha * re)
    B = L.astype(complex)
    A = A.astype(complex)
    rows = N - 3                      # tau rows 0..N-4
    A[rows:] = 0.0
    B[rows:] = 0.0
    A[rows] = sp.cheb_at_plus1(N)
    A[rows + 1] = sp.cheb_at_minus1(N)
    A[rows + 2] = sp.cheb_at_plus1(N) @ D
    A[rows + 3] = sp.cheb_at_minus1(N) @ D
    c, V = scipy.linalg.eig(A, B)
    finite = np.isfinite(c)
    return c[finite], V[:, finite]


def most_unstable(N: int, alpha: float = 1.0, re: float = 1.0e4):
    """Eigenvalue with the largest imaginary part and its eigenvector (max-normalised)."""
    c, V = orr_sommerfeld(N, alpha, re)
    # spurious large eigenvalues of the tau method are discarded
    ok = np.abs(c) < 10.0
    c, V = c[ok], V[:, ok]
    i = int(np.argmax(c.imag))
    v = V[:, i]
    v = v / v[np.argmax(np.abs(v))]
    return c[i], v
