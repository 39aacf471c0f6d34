"""The seeded input generator: SplitMix64 reference outputs and the recipe's invariants."""

import numpy as np
import numpy.polynomial.chebyshev as npc

import seeded_inputs as si


def test_splitmix64_reference_outputs():
    # First five outputs of the published SplitMix64 reference code for seed 1234567.
    r = si.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_normals_moments():
    r = si.SplitMix64(42)
    x = np.array(r.normals(200000))
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01


def test_shape_tables_are_the_stated_polynomials():
    y = np.linspace(-1, 1, 7)
    tv = np.zeros(5)
    for n, c in si.SHAPE_V.items():
        tv[n] = c
    tg = np.zeros(3)
    for n, c in si.SHAPE_G.items():
        tg[n] = c
    assert np.allclose(npc.chebval(y, tv), (1 - y * y) ** 2, atol=1e-15)
    assert np.allclose(npc.chebval(y, tg), 1 - y * y, atol=1e-15)


def test_perturbation_invariants():
    nx, ny, nz = 16, 33, 16
    f = si.perturbed_poiseuille(nx, ny, nz, seed=3, amplitude=0.1, kmax=4)
    v, g = f["v"], f["g"]
    kzi = si.kz_index(nz)
    # Nyquist row and mean mode empty
    assert np.all(v[:, kzi == -nz // 2] == 0) and np.all(v[:, 0, 0] == 0)
    # Hermitian kx = 0 column
    for row in range(nz):
        m = kzi[row]
        if m > 0:
            neg = int(np.nonzero(kzi == -m)[0][0])
            assert np.array_equal(v[:, neg, 0], np.conj(v[:, row, 0]))
    # wall conditions: v = Dv = 0, g = 0 at both walls
    vc = np.moveaxis(v, 0, -1).reshape(-1, ny)
    gc = np.moveaxis(g, 0, -1).reshape(-1, ny)
    for a in vc:
        assert abs(npc.chebval(1, a)) < 1e-16 and abs(npc.chebval(-1, a)) < 1e-16
        d = npc.chebder(a)
        assert abs(npc.chebval(1, d)) < 1e-15 and abs(npc.chebval(-1, d)) < 1e-15
    for a in gc:
        assert abs(npc.chebval(1, a)) < 1e-16 and abs(npc.chebval(-1, a)) < 1e-16
    # only |k index| <= kmax excited
    nz_rows = np.nonzero(np.abs(v).sum(axis=(0, 2)))[0]
    assert np.all(np.abs(kzi[nz_rows]) <= 4)
    # determinism
    f2 = si.perturbed_poiseuille(nx, ny, nz, seed=3, amplitude=0.1, kmax=4)
    assert np.array_equal(f2["v"], v) and np.array_equal(f2["g"], g)


def test_wall_action_zero_mean():
    a = si.wall_action(16, 16, 5, 0.05 * 180 / 2800)
    assert a.shape == (16, 16) and abs(a.mean()) < 1e-18
    assert 0.5 * 0.05 * 180 / 2800 < a.std() < 2 * 0.05 * 180 / 2800


def test_open_channel_shapes_are_the_stated_polynomials():
    y = np.linspace(-1, 1, 9)
    tv = np.zeros(5)
    for n, c in si.SHAPE_V_OPEN.items():
        tv[n] = c
    tg = np.zeros(3)
    for n, c in si.SHAPE_G_OPEN.items():
        tg[n] = c
    tu = np.zeros(3)
    for n, c in si.HALF_POISEUILLE_U.items():
        tu[n] = c
    sy = (1 + y) / 2
    assert np.allclose(npc.chebval(y, tv), (1 + y) ** 2 * (1 - y) * (2 - y) / 2, atol=1e-15)
    assert np.allclose(npc.chebval(y, tg), (1 + y) * (3 - y) / 4, atol=1e-15)
    assert np.allclose(npc.chebval(y, tu), 1.5 * (2 * sy - sy * sy), atol=1e-15)


def test_open_channel_perturbation_meets_the_free_slip_conditions():
    nx, ny, nz = 16, 33, 16
    f = si.perturbed_poiseuille(nx, ny, nz, seed=5, amplitude=0.2, kmax=4, top_bc=1)
    vc = np.moveaxis(f["v"], 0, -1).reshape(-1, ny)
    gc = np.moveaxis(f["g"], 0, -1).reshape(-1, ny)
    assert np.abs(vc).max() > 0 and np.abs(gc).max() > 0
    for a in vc:   # v = Dv = 0 at y = -1; v = D^2 v = 0 at y = +1
        assert abs(npc.chebval(-1, a)) < 1e-16 and abs(npc.chebval(1, a)) < 1e-16
        assert abs(npc.chebval(-1, npc.chebder(a))) < 1e-15
        assert abs(npc.chebval(1, npc.chebder(a, 2))) < 1e-14
    for a in gc:   # g = 0 at y = -1; Dg = 0 at y = +1
        assert abs(npc.chebval(-1, a)) < 1e-16 and abs(npc.chebval(1, npc.chebder(a))) < 1e-15
    U = f["U"]
    assert abs(npc.chebval(-1, U)) < 1e-16 and abs(npc.chebval(1, npc.chebder(U))) < 1e-15
    iU = npc.chebint(U)
    assert abs(npc.chebval(1, iU) - npc.chebval(-1, iU) - 2.0) < 1e-15
    # same draws as the closed channel: the random factors agree mode by mode
    fc = si.perturbed_poiseuille(nx, ny, nz, seed=5, amplitude=0.2, kmax=4)
    ratio = f["v"][4] / np.where(fc["v"][4] == 0, 1, fc["v"][4])
    assert np.allclose(ratio[fc["v"][4] != 0], si.SHAPE_V_OPEN[4] / si.SHAPE_V[4])
