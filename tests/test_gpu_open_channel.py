"""The open channel of the paper (Sec. 3.1: height h, no slip at the actuated
wall, free slip at the top) through the C ABI against the oracle's top_bc = 1
step, on the same seeded inputs.

Reading: y in [-1, 1] is the whole open channel, so Re_b and Re_tau are based
on its height 2 (nu = 2 / Re_b, y+ = (1 + y) Re_tau / 2); the top rows are
v = 0, D^2 v = 0, D omega_y = 0, DU = DW = 0.  The library closes the
parity-split tau solves with the coupled wall rows (2 x 2 for omega_y and W,
two influence coefficients for v, 3 x 3 for U at constant flow rate), in both
forms of the implicit half.  Bars: relative L2 1e-11 (all FP64) and 1e-4
(mixed) for the state and the observation; the wall shear and the reward at
1e-9 (FP64, the n^2-weighted wall derivative) and 1e-4 (mixed).
"""

import math

import numpy as np
import pytest

import golden_util
import seeded_inputs as si
from gpu_util import rel_l2, run_batch_pair, run_pair

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 1e-4}
TAU_TOL = {0: 1e-9, 1: 1e-4}
OPEN_MINIMAL = dict(nx=16, ny=65, nz=16, lx=2.67, lz=0.8, re_tau=180.0, re_bulk=2800.0, dt=0.005, top_bc=1)
OPEN_LARGER = dict(nx=64, ny=65, nz=64, lx=2 * math.pi, lz=math.pi, re_tau=180.0, re_bulk=2800.0, dt=0.005,
                   top_bc=1)


def _errors(lo, oo, ls, os_, kw):
    err = {k: rel_l2(ls[k], os_[k]) for k in ("v", "g", "U")}
    err["W"] = float(np.linalg.norm(ls["W"] - os_["W"]) / np.linalg.norm(os_["U"]))
    err["obs"] = max(rel_l2(a[0], b[0]) for a, b in zip(lo, oo))
    err["wall_shear"] = max(abs(a[1] - b[1]) / abs(b[1]) for a, b in zip(lo, oo))
    u_tau = kw["re_tau"] / kw["re_bulk"]
    err["reward"] = max(abs(a[2] - b[2]) / max(abs(b[2]), abs(b[1]) / u_tau ** 2) for a, b in zip(lo, oo))
    return err


def _check(name, lo, oo, ls, os_, kw):
    prec = kw.get("precision", 0)
    err = _errors(lo, oo, ls, os_, kw)
    print(f"\n{name}: " + ", ".join(f"{k} {v:.2e}" for k, v in err.items()))
    for k in ("v", "g", "U", "W", "obs"):
        assert err[k] <= TOL[prec], (k, err)
    for k in ("wall_shear", "reward"):
        assert err[k] <= TAU_TOL[prec], (k, err)
    return err


@pytest.mark.parametrize("precision", [0, 1])
def test_open_channel_single_step(native_gpu, precision):
    kw = dict(OPEN_MINIMAL, precision=precision)
    lo, oo, ls, os_ = run_pair(native_gpu, kw, 1, seed=2, amp=0.2, kmax=99)
    _check(f"open minimal, precision {precision}, 1 step", lo, oo, ls, os_, kw)


@pytest.mark.parametrize("precision", [0, 1])
def test_open_channel_ten_step_window(native_gpu, precision):
    kw = dict(OPEN_MINIMAL, precision=precision)
    lo, oo, ls, os_ = run_pair(native_gpu, kw, 10, seed=3, amp=0.3, kmax=99)
    _check(f"open minimal, precision {precision}, 10 steps", lo, oo, ls, os_, kw)


def test_open_channel_ramp_with_clip(native_gpu):
    kw = dict(OPEN_MINIMAL, steps_per_action=3)
    lo, oo, ls, os_ = run_pair(native_gpu, kw, 2, seed=1, amp=0.2, kmax=4, action_std=1.5)
    _check("open minimal, ramp over 3 steps, clip active", lo, oo, ls, os_, kw)


@pytest.mark.parametrize("precision", [0, 1])
def test_open_channel_opposition_larger(native_gpu, precision):
    """Opposition control sensing at the node above y+ = 15 of the open
    channel (y+ = 15.17, the paper's plane)."""
    kw = dict(OPEN_LARGER, control=1, alpha=1.0, precision=precision)
    lo, oo, ls, os_ = run_pair(native_gpu, kw, 2, seed=4, amp=0.1, kmax=99)
    _check(f"open larger, opposition, precision {precision}, 2 steps", lo, oo, ls, os_, kw)
    assert rel_l2(ls["vw"], os_["vw"]) <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_open_channel_batched_implicit_half(native_gpu, precision):
    """80 open channels, the implicit half in its batched form (pinned)."""
    kw = dict(OPEN_MINIMAL, precision=precision)
    info, res = run_batch_pair(native_gpu, kw, 80, (0, 79), 2, tiles=(8, 16, 1))
    assert info.post_batched == 1
    for e, (lo, oo, ls, os_) in res.items():
        _check(f"open minimal x80 batched, precision {precision}, slot {e}", lo, oo, ls, os_, kw)


@pytest.mark.parametrize("precision", [0, 1])
def test_open_channel_tile_shapes_give_identical_results(native_gpu, precision):
    native = native_gpu
    B = 3
    kw = dict(OPEN_MINIMAL, precision=precision, autotune=0)
    acts = np.stack([si.wall_action(16, 16, 700 + e, 0.5 * 180 / 2800) for e in range(B)])
    ref = None
    for pre, post, bat in [(8, 8, 0), (4, 3, 0), (2, 1, 0), (8, 16, 1), (4, 8, 1), (2, 2, 1)]:
        env = native.env_create(native.params(**kw, batch=B))
        try:
            native.env_set_tiles(env, pre, post, bat)
            for e in range(B):
                native.env_set_state(env, e, native.pack_state(
                    si.perturbed_poiseuille(16, 65, 16, 60 + e, 0.2, 99, top_bc=1), 16, 65, 16))
            obs, tau, rew = np.zeros((B, 2, 16, 16)), np.zeros(B), np.zeros(B)
            for _ in range(2):
                assert native.env_step(env, acts, obs, tau, rew) == 0
            got = (np.concatenate([native.env_get_state(env, e) for e in range(B)]), obs.copy(), tau.copy())
        finally:
            native.env_destroy(env)
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(a, b) for a, b in zip(ref, got)), (pre, post, bat)


def test_open_channel_laminar_steady_and_reward(native_gpu):
    """The half-Poiseuille profile is a fixed point at constant flow rate;
    its wall shear is 1.5 nu = 3 / Re_b and the reward is the laminar bound
    1 - 3 Re_b / Re_tau^2 (the paper's 73.9 %, Sec. 3.2)."""
    native = native_gpu
    env = native.env_create(native.params(**OPEN_MINIMAL))
    try:
        info = native.env_info(env)
        assert abs(info.y_plus_sense - 15.17) < 0.01
        assert abs(info.nu - 2.0 / 2800.0) < 1e-18
        obs, tau, rew = np.zeros((2, 16, 16)), np.zeros(1), np.zeros(1)
        zero = np.zeros((16, 16))
        for _ in range(100):
            assert native.env_step(env, zero, obs, tau, rew) == 0
        st = native.unpack_state(native.env_get_state(env), 16, 65, 16)
    finally:
        native.env_destroy(env)
    U0 = np.zeros(65)
    U0[0], U0[1], U0[2] = 0.9375, 0.75, -0.1875
    assert np.abs(st["U"] - U0).max() < 1e-12
    assert np.abs(st["v"]).max() == 0 and np.abs(st["g"]).max() == 0
    assert abs(tau[0] - 3.0 / 2800.0) < 1e-13
    bound = golden_util.load("laminar_drag_bound.txt")
    assert abs(rew[0] - bound["closed_form"]) < 1e-9
