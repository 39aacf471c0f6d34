"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the time step itself: it only draws random
numbers and lays them out as an initial flow state or as a wall action field.
Both sides of every parity test (the CPU oracle and the CUDA library) receive
exactly these arrays.

Random numbers
--------------
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) turned into 53-bit uniforms and then into normals by
the Box-Muller transform.  The library's host code implements the same
generator for ``env_reset``; a CPU test checks that the two agree.

State layout (the library's serialised state uses the same order)
----------------------------------------------------------------
* ``v``, ``g``: complex128 ``[ny][nz][nx//2]`` Chebyshev coefficients of the
  wall-normal velocity and the wall-normal vorticity, per Fourier mode
  (``kz`` in FFT storage order 0..nz/2-1, -nz/2..-1; the ``-nz/2`` row is the
  Nyquist row and stays zero; ``kx`` index 0..nx/2-1).
* ``U``, ``W``: float64 ``[ny]`` Chebyshev coefficients of the mean
  streamwise and spanwise velocity.

Perturbation recipe (divergence-free by construction, wall conditions exact)
------------------------------------------------------------------------------
For every excited mode (kx index ``i``, kz index ``m``; ``i <= kmax``,
``|m| <= kmax``, not (0,0), not Nyquist) four normals ``a, b, c, d`` are
drawn in storage order (kz row, then kx column)::

    v_hat(y) = s (a + i b) (1 - y^2)^2 ,   g_hat(y) = s (c + i d) (1 - y^2)

with ``s = amplitude / sqrt(number of excited modes)``.  ``v`` then vanishes
with its y-derivative at both walls and ``g`` vanishes at both walls.  On the
``kx = 0`` column only ``m > 0`` is drawn; ``m < 0`` takes the complex
conjugate so that the physical field is real.  The mean flow is laminar
Poiseuille ``U = 1.5 (1 - y^2)`` (bulk velocity 1), ``W = 0``.

Open channel (``top_bc = 1``: free slip at ``y = +1``): the same draws with
the shapes ``v: (1 + y)^2 (1 - y) (2 - y) / 2`` (v = Dv = 0 at ``y = -1``,
v = D^2 v = 0 at ``y = +1``) and ``g: (1 + y) (3 - y) / 4`` (g = 0 at
``y = -1``, Dg = 0 at ``y = +1``), and the half-Poiseuille mean flow
``U = 1.5 (2 s - s^2)``, ``s = (1 + y) / 2`` (bulk velocity 1 over the height).
"""

from __future__ import annotations

import math

import numpy as np

_MASK64 = (1 << 64) - 1

# Chebyshev coefficients of the fixed wall-normal shapes (exact rationals):
#   (1 - y^2)   = 1/2 T0 - 1/2 T2
#   (1 - y^2)^2 = 3/8 T0 - 1/2 T2 + 1/8 T4
SHAPE_G = {0: 0.5, 2: -0.5}
SHAPE_V = {0: 0.375, 2: -0.5, 4: 0.125}
POISEUILLE_U = {0: 0.75, 2: -0.75}
# open channel:
#   (1 + y)^2 (1 - y) (2 - y) / 2 = (2 + y - 3 y^2 - y^3 + y^4) / 2
#                                 = 7/16 T0 + 1/8 T1 - 1/2 T2 - 1/8 T3 + 1/16 T4
#   (1 + y) (3 - y) / 4           = 5/8 T0 + 1/2 T1 - 1/8 T2
#   1.5 (2 s - s^2), s = (1+y)/2  = 15/16 T0 + 3/4 T1 - 3/16 T2
SHAPE_V_OPEN = {0: 0.4375, 1: 0.125, 2: -0.5, 3: -0.125, 4: 0.0625}
SHAPE_G_OPEN = {0: 0.625, 1: 0.5, 2: -0.125}
HALF_POISEUILLE_U = {0: 0.9375, 1: 0.75, 2: -0.1875}


class SplitMix64:
    """SplitMix64 stream; ``next_u64`` follows the published definition."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal_pair(self) -> tuple[float, float]:
        """Two independent standard normals (Box-Muller, u1 in (0, 1])."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        t = 2.0 * math.pi * u2
        return r * math.cos(t), r * math.sin(t)

    def normals(self, n: int) -> list[float]:
        out: list[float] = []
        while len(out) < n:
            out.extend(self.normal_pair())
        return out[:n]


def kz_index(nz: int) -> np.ndarray:
    """Integer spanwise wavenumber index of each storage row (FFT order)."""
    return np.concatenate([np.arange(0, nz // 2), np.arange(-nz // 2, 0)])


def excited_modes(nx: int, nz: int, kmax: int) -> list[tuple[int, int]]:
    """(row, column) storage positions that receive random draws, in draw order."""
    modes = []
    kzi = kz_index(nz)
    for row in range(nz):
        m = int(kzi[row])
        if m == -nz // 2:
            continue
        for i in range(nx // 2):
            if i > kmax or abs(m) > kmax or (i == 0 and m == 0):
                continue
            if i == 0 and m < 0:
                continue  # conjugate of the m > 0 draw
            modes.append((row, i))
    return modes


def perturbed_poiseuille(nx: int, ny: int, nz: int, seed: int,
                         amplitude: float = 0.1, kmax: int = 4, top_bc: int = 0) -> dict:
    """Laminar Poiseuille flow plus the seeded perturbation described above
    (``top_bc = 1``: the open-channel shapes and the half-Poiseuille profile)."""
    if nx % 2 or nz % 2 or ny < 5:
        raise ValueError("nx, nz must be even and ny >= 5")
    nxh = nx // 2
    v = np.zeros((ny, nz, nxh), np.complex128)
    g = np.zeros((ny, nz, nxh), np.complex128)
    modes = excited_modes(nx, nz, kmax)
    rng = SplitMix64(seed)
    n_exc = len(modes) + sum(1 for (r, i) in modes if i == 0)
    s = amplitude / math.sqrt(n_exc) if n_exc else 0.0
    kzi = kz_index(nz)
    shape_v, shape_g, mean_u = ((SHAPE_V_OPEN, SHAPE_G_OPEN, HALF_POISEUILLE_U) if top_bc == 1 else
                                (SHAPE_V, SHAPE_G, POISEUILLE_U))
    for (row, i) in modes:
        a, b, c, d = rng.normals(4)
        cv = s * complex(a, b)
        cg = s * complex(c, d)
        for n, coef in shape_v.items():
            v[n, row, i] = cv * coef
        for n, coef in shape_g.items():
            g[n, row, i] = cg * coef
        if i == 0:
            mrow = int(np.nonzero(kzi == -kzi[row])[0][0])
            v[:, mrow, 0] = np.conj(v[:, row, 0])
            g[:, mrow, 0] = np.conj(g[:, row, 0])
    U = np.zeros(ny)
    for n, coef in mean_u.items():
        U[n] = coef
    W = np.zeros(ny)
    return {"v": v, "g": g, "U": U, "W": W}


def wall_action(nx: int, nz: int, seed: int, std: float) -> np.ndarray:
    """Seeded Gaussian wall-normal velocity field ``[nz][nx]`` with its plane mean removed."""
    rng = SplitMix64(seed)
    a = np.array(rng.normals(nx * nz), dtype=np.float64).reshape(nz, nx) * std
    return a - a.mean()


def action_sequence(nx: int, nz: int, seed: int, std: float, count: int) -> np.ndarray:
    """``count`` actions; action ``t`` uses seed ``seed * 1000003 + t``."""
    return np.stack([wall_action(nx, nz, seed * 1000003 + t, std) for t in range(count)])
