"""Pins of the oracle's agent policy (Sec. 3.2): the observation window layout,
the opposition law as a linear policy (Sec. 4.1), a hand-evaluated network and
the translation invariance of a shared local policy.  No GPU."""

import math

import numpy as np
import pytest

from oracle import policy
from paper_2301_09889_gb300 import native


def _plane(B=2, nz=6, nx=8, seed=0):
    return np.random.default_rng(seed).standard_normal((B, 2, nz, nx))


@pytest.mark.parametrize("wz,wx", [(1, 1), (3, 5), (5, 3)])
def test_one_hot_first_layer_reads_the_documented_window_point(wz, wx):
    plane = _plane()
    K = 2 * wz * wx
    for k in range(K):
        c, q = divmod(k, wz * wx)
        dz, dx = divmod(q, wx)
        w = np.zeros(K + 1)
        w[k] = 1.0
        a = policy.actions(plane, w, wz, wx, (), out_tanh=False)
        # agent (iz, ix) sees row iz + dz - wz//2 and column ix + dx - wx//2
        want = np.roll(plane[:, c], shift=(-(dz - wz // 2), -(dx - wx // 2)), axis=(1, 2))
        assert np.array_equal(a, want), (k, c, dz, dx)


def test_linear_policy_is_the_opposition_law_without_the_mean():
    plane = _plane(seed=4)
    alpha = 0.7
    a = policy.actions(plane, np.array([0.0, -alpha, 0.0]), 1, 1, (), out_tanh=False)
    assert np.array_equal(a, -alpha * plane[:, 1])


def test_hand_evaluated_network():
    plane = np.array([1.5, -0.5]).reshape(1, 2, 1, 1)   # u = 1.5, v = -0.5
    W0 = [1.0, 2.0, -1.0, 1.0]                          # rows: (1, 2), (-1, 1)
    b0 = [0.5, -3.0]                                    # pre-activations 1.0 and -5.0
    Wo, bo = [2.0, 7.0], [0.25]                         # y = 2 * 1.0 + 7 * 0 + 0.25
    w = np.array(W0 + b0 + Wo + bo)
    assert policy.actions(plane, w, 1, 1, (2,), out_tanh=False)[0, 0, 0] == 2.25
    assert policy.actions(plane, w, 1, 1, (2,), out_tanh=True, u_tau=0.1)[0, 0, 0] == pytest.approx(
        0.1 * math.tanh(2.25), rel=1e-15)
    # a second hidden layer of width 1 with unit weight and zero bias leaves y unchanged
    w2 = np.array(W0 + b0 + [2.0, 7.0] + [0.25] + [1.0] + [0.0])
    assert policy.weight_count(1, 1, (2, 1)) == w2.size
    assert policy.actions(plane, w2, 1, 1, (2, 1), out_tanh=False)[0, 0, 0] == 2.25


def test_shared_local_policy_commutes_with_wall_translations():
    rng = np.random.default_rng(7)
    wz, wx, hidden = 3, 5, (6, 4)
    w = rng.standard_normal(policy.weight_count(wz, wx, hidden))
    plane = _plane(seed=9)
    a = policy.actions(plane, w, wz, wx, hidden, u_tau=0.05)
    shifted = np.roll(plane, shift=(2, -3), axis=(2, 3))
    assert np.allclose(policy.actions(shifted, w, wz, wx, hidden, u_tau=0.05),
                       np.roll(a, shift=(2, -3), axis=(1, 2)), rtol=0, atol=1e-15)
    assert np.all(np.abs(a) <= 0.05)


def test_weight_counts_agree_with_the_binding():
    for wz, wx, hidden in [(1, 1, ()), (3, 3, (32,)), (3, 5, (64, 16)), (7, 7, (64, 64))]:
        assert native.policy_weight_count(native.policy(wz, wx, hidden)) == policy.weight_count(wz, wx, hidden)
    with pytest.raises(ValueError):
        policy.unpack(np.zeros(5), 1, 1, ())


def test_bench_policy_weights_fit_the_layout():
    import bench
    for name, (wz, wx, hidden, tanh_out, seed) in bench.POLICIES.items():
        w = bench.policy_weights(wz, wx, hidden, seed)
        assert w.size == policy.weight_count(wz, wx, hidden)
        assert np.array_equal(w, bench.policy_weights(wz, wx, hidden, seed))  # seeded
        assert bench.WORKLOADS[name][0]["control"] == 2
