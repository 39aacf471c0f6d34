"""Pins of the oracle's Chebyshev and Fourier operators against independent routes.

Each operator is checked against something other than itself: numpy's own
Chebyshev-series routines, closed forms of T_n at the walls, brute-force
pure-Python DFT sums on tiny grids, and the exactness of the 3/2 rule for
quadratic products (truncated convolution computed by brute force).
"""

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import spectral as sp

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("N", [4, 16, 64, 128])
def test_synthesis_matches_numpy_chebval(N):
    rng = np.random.default_rng(N)
    a = rng.standard_normal(N + 1)
    y = sp.cheb_nodes(N)
    ref = npc.chebval(y, a)
    assert np.allclose(sp.cheb_synthesis(N) @ a, ref, rtol=0, atol=1e-12 * np.abs(a).sum())


@pytest.mark.parametrize("N", [4, 16, 64, 192])
def test_analysis_inverts_synthesis(N):
    rng = np.random.default_rng(N + 1)
    a = rng.standard_normal(N + 1)
    back = sp.cheb_analysis(N) @ (sp.cheb_synthesis(N) @ a)
    assert np.max(np.abs(back - a)) < 1e-13 * np.sqrt(N)


@pytest.mark.parametrize("N", [4, 17, 64])
def test_derivative_matches_numpy_chebder(N):
    rng = np.random.default_rng(N + 2)
    a = rng.standard_normal(N + 1)
    ref = np.zeros(N + 1)
    ref[:N] = npc.chebder(a)
    assert np.allclose(sp.cheb_diff(N) @ a, ref, rtol=1e-13, atol=1e-12 * N * N)


def test_derivative_of_polynomials_exact():
    # d/dy of y^3 - 2y = 3y^2 - 2 ; in Chebyshev: y^3 = (3T1 + T3)/4
    N = 8
    a = np.zeros(N + 1)
    a[1] = 0.75 - 2.0
    a[3] = 0.25
    d = sp.cheb_diff(N) @ a
    y = np.linspace(-1, 1, 11)
    assert np.allclose(npc.chebval(y, d), 3 * y ** 2 - 2, atol=1e-14)


@pytest.mark.parametrize("N", [8, 64])
def test_wall_values_closed_form(N):
    n = np.arange(N + 1)
    D = sp.cheb_diff(N)
    assert np.array_equal(sp.cheb_at_plus1(N), np.ones(N + 1))
    assert np.array_equal(sp.cheb_at_minus1(N), (-1.0) ** n)
    # T_n'(1) = n^2, T_n'(-1) = (-1)^(n+1) n^2
    assert np.allclose(sp.cheb_at_plus1(N) @ D, n ** 2, rtol=0, atol=1e-9)
    assert np.allclose(sp.cheb_at_minus1(N) @ D, (-1.0) ** (n + 1) * n ** 2, rtol=0, atol=1e-9)


@pytest.mark.parametrize("N", [8, 64])
def test_integral_weights_match_chebint(N):
    rng = np.random.default_rng(N + 3)
    a = rng.standard_normal(N + 1)
    prim = npc.chebint(a)
    ref = npc.chebval(1.0, prim) - npc.chebval(-1.0, prim)
    assert abs(sp.cheb_integral(N) @ a - ref) < 1e-12


def _brute_physical(F, nx, nz, mx, mz, lx=1.0, lz=1.0):
    """Real field from the full Hermitian spectrum, by pure-Python sums."""
    kzi = sp.kz_index(nz)
    f = np.zeros((mz, mx))
    for b in range(mz):
        for a in range(mx):
            x = a * lx / mx
            z = b * lz / mz
            s = 0.0 + 0.0j
            for row in range(nz):
                m = kzi[row]
                if m == -nz // 2:
                    continue
                for i in range(nx // 2):
                    ph = np.exp(2j * np.pi * (i * x / lx + m * z / lz))
                    s += F[row, i] * ph
                    if i > 0:  # the conjugate mode (-i, -m)
                        s += np.conj(F[row, i] * ph)
            f[b, a] = s.real
    return f


def _hermitian_random(nx, nz, rng):
    F = rng.standard_normal((nz, nx // 2)) + 1j * rng.standard_normal((nz, nx // 2))
    kzi = sp.kz_index(nz)
    F[kzi == -nz // 2] = 0.0
    F[0, 0] = F[0, 0].real
    for row in range(nz):
        m = kzi[row]
        if m < 0 and m != -nz // 2:
            F[row, 0] = np.conj(F[int(np.nonzero(kzi == -m)[0][0]), 0])
    return F


@pytest.mark.parametrize("nx,nz", [(4, 4), (6, 8), (8, 4)])
def test_to_physical_matches_brute_force(nx, nz):
    rng = np.random.default_rng(nx * 10 + nz)
    F = _hermitian_random(nx, nz, rng)
    for (mx, mz) in [(nx, nz), (3 * nx // 2, 3 * nz // 2)]:
        f = sp.to_physical(F, nx, nz, mx, mz)
        ref = _brute_physical(F, nx, nz, mx, mz)
        assert np.max(np.abs(f - ref)) < 1e-12


@pytest.mark.parametrize("nx,nz", [(4, 4), (8, 6), (16, 16), (64, 64)])
def test_spectral_roundtrip_and_numpy_fft(nx, nz):
    rng = np.random.default_rng(nx + nz)
    F = _hermitian_random(nx, nz, rng)
    for (mx, mz) in [(nx, nz), (3 * nx // 2, 3 * nz // 2)]:
        f = sp.to_physical(F, nx, nz, mx, mz)
        back = sp.to_spectral(f, nx, nz, mx, mz)
        assert np.max(np.abs(back - F)) < 1e-12
        # independent route: numpy's FFT of the same grid values
        ref = np.fft.fft2(f) / (mx * mz)
        kzi = sp.kz_index(nz)
        for row in range(nz):
            if kzi[row] == -nz // 2:
                continue
            assert np.allclose(back[row], ref[kzi[row] % mz, : nx // 2], atol=1e-12)


def _full_spectrum(F, nx, nz):
    """dict (m, i) -> coefficient over the full Hermitian spectrum."""
    kzi = sp.kz_index(nz)
    out = {}
    for row in range(nz):
        m = int(kzi[row])
        if m == -nz // 2:
            continue
        for i in range(nx // 2):
            out[(m, i)] = out.get((m, i), 0) + F[row, i]
            if i > 0:
                out[(-m, -i)] = out.get((-m, -i), 0) + np.conj(F[row, i])
    return out


@pytest.mark.parametrize("nx,nz", [(4, 4), (8, 8), (6, 10)])
def test_dealiased_product_is_truncated_convolution(nx, nz):
    """3/2 rule: the padded-grid product of two band-limited fields, truncated,
    equals the exact convolution restricted to the kept modes."""
    rng = np.random.default_rng(7 * nx + nz)
    A = _hermitian_random(nx, nz, rng)
    B = _hermitian_random(nx, nz, rng)
    mx, mz = 3 * nx // 2, 3 * nz // 2
    prod = sp.to_physical(A, nx, nz, mx, mz) * sp.to_physical(B, nx, nz, mx, mz)
    C = sp.to_spectral(prod, nx, nz, mx, mz)
    fa, fb = _full_spectrum(A, nx, nz), _full_spectrum(B, nx, nz)
    kzi = sp.kz_index(nz)
    for row in range(nz):
        m = int(kzi[row])
        for i in range(nx // 2):
            if m == -nz // 2:
                assert C[row, i] == 0
                continue
            s = 0.0
            for (m1, i1), a in fa.items():
                b = fb.get((m - m1, i - i1))
                if b is not None:
                    s += a * b
            assert abs(C[row, i] - s) < 1e-12, (row, i)
