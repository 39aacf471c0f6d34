"""The multi-agent interface (Sec. 3.2-3.3) on the GPU: it adds nothing to the
physics, so its observations and rewards are bit-identical to the C ABI
driven by the same requests, every episode starts from the same flow, and the
per-agent dictionary and the array forms agree.  env_observe (STATE without a
step) returns the plane a step returns."""

import numpy as np
import pytest

from paper_2301_09889_gb300 import marl

pytestmark = pytest.mark.gpu

MINIMAL = dict(nx=16, ny=65, nz=16, lx=2.67, lz=0.8, re_tau=180.0, re_bulk=2800.0, dt=0.005, steps_per_action=2)


def test_wrapper_matches_the_c_abi(native_gpu):
    native = native_gpu
    B = 2
    env = marl.ChannelMARL(MINIMAL, batch=B, window=(3, 3), seed=5, amplitude=0.3)
    raw = native.env_create(native.params(**MINIMAL, batch=B, control=0))
    try:
        native.env_reset(raw, 5, 0.3, 4)
        init = [native.env_get_state(raw, b) for b in range(B)]
        for b in range(B):
            native.env_set_state(raw, b, init[b])
        obs = np.zeros((B, 2, 16, 16))
        tau, rew = np.zeros(B), np.zeros(B)
        w = env.reset_arrays()
        native.env_observe(raw, obs)
        assert np.array_equal(env.state(), obs)
        assert np.array_equal(w[:, :, :, :, 1, 1], obs.transpose(0, 2, 3, 1))
        for _ in range(3):
            act = marl.opposition_action(env.state())
            w, r, ws, term, trunc = env.step_arrays(act)
            assert native.env_step(raw, act, obs, tau, rew) == 0
            assert np.array_equal(env.state(), obs) and np.array_equal(r, rew) and np.array_equal(ws, tau)
            # STATE without a step returns the same plane the step returned
            again = np.zeros_like(obs)
            native.env_observe(raw, again)
            assert np.array_equal(again, obs)
            assert not term and not trunc
            assert np.all(np.isfinite(w))
    finally:
        env.close()
        native.env_destroy(raw)


def test_episodes_restart_from_the_same_flow_and_dict_form_agrees(native_gpu):
    a = marl.ChannelMARL(MINIMAL, seed=9, amplitude=0.3, max_cycles=2)
    b = marl.ChannelMARL(MINIMAL, seed=9, amplitude=0.3, max_cycles=2)
    try:
        first, _ = a.reset()
        wb = b.reset_arrays()
        for _ in range(2):
            plane = a.state()
            act = marl.opposition_action(plane)
            obs, rew, term, trunc, info = a.step({n: act[0, int(n.split("_")[1]), int(n.split("_")[2])]
                                                  for n in a.possible_agents})
            wb, rb, tb, termb, truncb = b.step_arrays(act)
            assert all(np.array_equal(obs[f"agent_{iz}_{ix}"], wb[0, iz, ix]) for iz in range(16) for ix in range(16))
            assert len(set(rew.values())) == 1 and next(iter(rew.values())) == rb[0]
        assert all(trunc.values()) and a.agents == []
        again, _ = a.reset()
        assert all(np.array_equal(first[n], again[n]) for n in first)
    finally:
        a.close()
        b.close()
