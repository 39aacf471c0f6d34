"""On-device policy (control = 2): the shared agent policy of Sec. 3.2
evaluated by the library before every step.

* Its actions are the oracle's perceptron (FP64) evaluated on the observation
  the previous step returned, within the FP32 evaluation error.
* The linear 1 x 1 policy (0, -alpha) is the opposition law of Sec. 4.1 once
  the library removes the plane mean, so its trajectory matches the library's
  opposition-control mode (which forms the same wall spectrum directly) to
  rounding while no action reaches the clip.
* Bad descriptors, counts and handles are rejected.
"""

import numpy as np
import pytest

from gpu_util import rel_l2
from oracle import policy as opol

pytestmark = pytest.mark.gpu

MINIMAL = dict(nx=16, ny=65, nz=16, lx=2.67, lz=0.8, re_tau=180.0, re_bulk=2800.0, dt=0.005)


def _weights(wz, wx, hidden, seed, scale=1.0):
    """Seeded weights ~ N(0, scale^2 / fan_in) per layer, biases ~ N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    out = []
    for o, i in opol.layer_shapes(wz, wx, hidden):
        out.append(rng.standard_normal(o * i) * scale / np.sqrt(i))
        out.append(rng.standard_normal(o) * 0.1)
    return np.concatenate(out)


@pytest.mark.parametrize("wz,wx,hidden,out_tanh,precision", [
    (3, 3, (32, 16), True, 0),
    (1, 3, (8,), False, 0),
    (5, 5, (64, 64), True, 1),
])
def test_policy_actions_match_oracle(native_gpu, wz, wx, hidden, out_tanh, precision):
    native = native_gpu
    B = 2
    env = native.env_create(native.params(**MINIMAL, batch=B, control=2, precision=precision))
    try:
        info = native.env_info(env)
        pol = native.policy(wz, wx, hidden, out_tanh)
        # u ~ 1 and v ~ 0.05 on the sensing plane: scale the weights so that the
        # pre-activations are O(1)
        w = _weights(wz, wx, hidden, seed=11 + wz, scale=2.0)
        native.env_set_policy(env, pol, w)
        native.env_reset(env, 5, 0.3, 4)
        obs, tau, rew = np.zeros((B, 2, 16, 16)), np.zeros(B), np.zeros(B)
        act = np.zeros((B, 16, 16))
        for _ in range(3):
            prev = obs.copy()
            assert native.env_step(env, None, obs, tau, rew) == 0
        native.env_get_action(env, act)
        want = opol.actions(prev, w, wz, wx, hidden, out_tanh, info.u_tau)
        scale = np.abs(want).max()
        assert scale > 1e-3
        err = np.abs(act - want).max()
        print(f"policy {wz}x{wx} {hidden} tanh={out_tanh}: max |a - a_oracle| = {err:.3e} (max |a| {scale:.3e})")
        assert err <= 2e-5 * max(scale, info.u_tau)
        assert np.all(np.isfinite(obs)) and np.all(np.isfinite(tau))
    finally:
        native.env_destroy(env)


def test_linear_policy_follows_opposition_control(native_gpu):
    native = native_gpu
    alpha = 0.1
    kw = dict(MINIMAL, alpha=alpha)
    pol_env = native.env_create(native.params(**kw, control=2))
    opp_env = native.env_create(native.params(**kw, control=1))
    try:
        native.env_set_policy(pol_env, native.policy(1, 1, (), out_tanh=False), np.array([0.0, -alpha, 0.0]))
        u_tau = native.env_info(pol_env).u_tau
        for env in (pol_env, opp_env):
            native.env_reset(env, 8, 0.3, 4)
        o1, o2 = np.zeros((1, 2, 16, 16)), np.zeros((1, 2, 16, 16))
        t1, t2, r1, r2 = np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(1)
        act = np.zeros((1, 16, 16))
        for _ in range(5):
            assert native.env_step(pol_env, None, o1, t1, r1) == 0
            assert native.env_step(opp_env, None, o2, t2, r2) == 0
            native.env_get_action(pol_env, act)
            assert np.abs(act).max() < u_tau  # no clipping: the two laws coincide
        s1, s2 = native.env_get_state(pol_env, 0), native.env_get_state(opp_env, 0)
        e_state, e_obs = rel_l2(s1, s2), rel_l2(o1, o2)
        print(f"linear policy vs opposition, 5 steps: state {e_state:.2e}, obs {e_obs:.2e}, "
              f"tau {abs(t1[0] - t2[0]) / abs(t2[0]):.2e}")
        assert e_state < 1e-6 and e_obs < 1e-6 and abs(t1[0] - t2[0]) < 1e-6 * abs(t2[0])
        assert np.abs(act).max() > 1e-4  # the action is not trivially zero
    finally:
        native.env_destroy(pol_env)
        native.env_destroy(opp_env)


def test_policy_errors(native_gpu):
    native = native_gpu
    ext = native.env_create(native.params(**MINIMAL, control=0))
    pol = native.env_create(native.params(**MINIMAL, control=2))
    try:
        lin = native.policy(1, 1, ())
        with pytest.raises(native.ChannelError) as e:
            native.env_set_policy(ext, lin, np.zeros(3))
        assert e.value.code == native.CH_ERR_STATE
        obs, tau, rew = np.zeros((1, 2, 16, 16)), np.zeros(1), np.zeros(1)
        with pytest.raises(native.ChannelError) as e:
            native.env_step(pol, None, obs, tau, rew)
        assert e.value.code == native.CH_ERR_STATE
        bad = [(native.policy(2, 1, ()), 5), (native.policy(9, 1, ()), 19), (native.policy(1, 1, (65,)), 1),
               (native.policy(1, 1, ()), 4), (native.policy(1, 1, (0,)), 3)]
        for p, n in bad:
            with pytest.raises(native.ChannelError) as e:
                native.env_set_policy(pol, p, np.zeros(n))
            assert e.value.code == native.CH_ERR_ARG
        with pytest.raises(native.ChannelError):
            native.env_set_policy(pol, lin, np.array([0.0, np.nan, 0.0]))
        native.env_set_policy(pol, lin, np.array([0.0, -0.5, 0.0]))
        assert native.env_step(pol, None, obs, tau, rew) == 0
        assert native.env_info(pol).launches_per_step == 5 + 10 + 3
        srv = native.srv_create(1 << 30, 4)
        try:
            with pytest.raises(native.ChannelError) as e:
                native.srv_admit(srv, native.params(**MINIMAL, control=2), 1)
            assert e.value.code == native.CH_ERR_UNSUPPORTED
        finally:
            native.srv_destroy(srv)
    finally:
        native.env_destroy(ext)
        native.env_destroy(pol)


def test_get_action_reports_a_device_action_in_both_launch_modes(native_gpu):
    """env_get_action returns the caller's action after env_step_device, whether
    the step is replayed from the captured graph or launched kernel by kernel."""
    import torch

    import seeded_inputs as si
    native = native_gpu
    B = 2
    acts = np.stack([si.wall_action(16, 16, 500 + e, 0.5 * 180 / 2800) for e in range(B)])
    d_act = torch.from_numpy(acts).to("cuda")
    d_out = torch.zeros(B * (2 * 16 * 16 + 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for profile in (False, True):
        env = native.env_create(native.params(**MINIMAL, batch=B))
        try:
            native.env_profile(env, profile)
            native.env_reset(env, 3, 0.1, 4)
            native.env_step_device(env, d_act.data_ptr(), d_out.data_ptr())
            got = np.zeros((B, 16, 16))
            native.env_get_action(env, got)
            assert np.array_equal(got, acts), profile
        finally:
            native.env_destroy(env)
