"""Host logic of the multi-agent interface (Sec. 3.2-3.3) against a host fake
of the binding: observation windows, action assembly, the shared reward,
episode bookkeeping and the STATE/CNTRL/EVOLVE/TERMN mapping.  No GPU."""

from types import SimpleNamespace

import numpy as np
import pytest

from paper_2301_09889_gb300 import marl, native


class FakeBinding:
    """Stands in for the C ABI: the sensing plane after step s is
    obs[b, c, iz, ix] = 1e4 s + 1000 b + 100 c + 10 iz + ix (a value that names
    its own position), the reward is 0.5 - 0.01 s - 0.1 b."""

    def __init__(self, diverge_at=None):
        self.calls = []
        self.actions = []
        self.diverge_at = diverge_at

    def params(self, **kw):
        p = SimpleNamespace(nx=16, nz=16)
        p.__dict__.update(kw)
        return p

    def env_create(self, p):
        self.p = p
        self.state = [np.zeros(4) for _ in range(p.batch)]
        self.step = 0
        self.calls.append("create")
        return object()

    def env_info(self, env):
        return SimpleNamespace(u_tau=180.0 / 2800.0, tau_ref=(180.0 / 2800.0) ** 2, y_plus_sense=15.17)

    def env_reset(self, env, seed, amplitude, kmax):
        self.calls.append(("reset", seed))
        self.state = [np.full(4, float(seed + b)) for b in range(self.p.batch)]

    def env_get_state(self, env, b):
        return self.state[b].copy()

    def env_set_state(self, env, b, buf):
        self.calls.append(("set_state", b, float(buf[0])))
        self.state[b] = np.array(buf, dtype=float)

    def env_observe(self, env, obs):
        self.calls.append("observe")
        B, _, nz, nx = obs.shape
        b, c, iz, ix = np.meshgrid(np.arange(B), np.arange(2), np.arange(nz), np.arange(nx), indexing="ij")
        obs[...] = 1e4 * self.step + 1000 * b + 100 * c + 10 * iz + ix

    def env_step(self, env, action, obs, wall_shear, reward):
        self.step += 1
        self.actions.append(np.array(action))
        self.env_observe(env, obs)
        self.calls.pop()
        reward[...] = 0.5 - 0.01 * self.step - 0.1 * np.arange(obs.shape[0])
        wall_shear[...] = 1.0 - reward
        if self.diverge_at == self.step:
            wall_shear[0] = np.nan
            return native.CH_ERR_DIVERGED
        return native.CH_OK

    def env_destroy(self, env):
        self.calls.append("destroy")


def make(batch=1, window=(1, 1), **kw):
    fake = FakeBinding(kw.pop("diverge_at", None))
    env = marl.ChannelMARL(dict(nx=16, nz=16), batch=batch, window=window, seed=7, backend=fake, **kw)
    return env, fake


def test_windows_wrap_periodically_around_each_agent():
    env, _ = make(batch=2, window=(3, 5))
    obs = env.reset_arrays()
    plane = env.state()
    assert obs.shape == (2, 16, 16, 2, 3, 5) and env.observation_shape() == (2, 3, 5)
    for b in range(2):
        for iz in (0, 7, 15):
            for ix in (0, 1, 15):
                for c in range(2):
                    for dz in range(3):
                        for dx in range(5):
                            want = plane[b, c, (iz + dz - 1) % 16, (ix + dx - 2) % 16]
                            assert obs[b, iz, ix, c, dz, dx] == want
    # the centre of the window is the point above the actuator
    assert np.array_equal(obs[:, :, :, :, 1, 2], plane.transpose(0, 2, 3, 1))


def test_single_point_window_is_the_plane_itself():
    env, _ = make()
    obs = env.reset_arrays()
    assert np.array_equal(obs[0, :, :, :, 0, 0], env.state()[0].transpose(1, 2, 0))


def test_dict_actions_land_on_their_grid_points_and_reward_is_shared():
    env, fake = make(batch=2)
    obs, infos = env.reset()
    assert len(obs) == 2 * 16 * 16 == len(env.agents) and set(obs) == set(env.possible_agents)
    acts = {"env0_agent_3_4": 0.01, "env1_agent_15_0": -0.02, "env1_agent_0_15": 0.005}
    o, r, term, trunc, info = env.step(acts)
    a = fake.actions[-1]
    want = np.zeros((2, 16, 16))
    want[0, 3, 4], want[1, 15, 0], want[1, 0, 15] = 0.01, -0.02, 0.005
    assert np.array_equal(a, want)
    assert len(set(r[n] for n in r if n.startswith("env0"))) == 1
    # reset takes no step, so this is step 1
    assert r["env0_agent_0_0"] == pytest.approx(0.5 - 0.01) and r["env1_agent_9_9"] == pytest.approx(0.5 - 0.01 - 0.1)
    assert info["env1_agent_2_2"]["wall_shear"] == pytest.approx(1 - r["env1_agent_2_2"])
    assert not any(term.values()) and not any(trunc.values())
    assert np.array_equal(o["env1_agent_5_6"], env.observe_arrays()[1, 5, 6])
    with pytest.raises(KeyError):
        env.step({"env2_agent_0_0": 0.0})


def test_single_environment_names_and_truncation():
    env, _ = make(max_cycles=3)
    obs, _ = env.reset()
    assert "agent_0_0" in obs and "agent_15_15" in obs
    for k in range(3):
        _, _, term, trunc, _ = env.step({"agent_1_1": 0.0})
        assert not term["agent_1_1"] and trunc["agent_1_1"] == (k == 2)
    assert env.agents == []


def test_divergence_terminates_every_agent():
    env, _ = make(diverge_at=2)
    env.reset()
    _, _, term, _, _ = env.step({})
    assert not any(term.values())
    _, _, term, _, _ = env.step({})
    assert all(term.values()) and env.agents == []


def test_reset_restores_the_same_initial_condition_unless_reseeded():
    env, fake = make(batch=2)
    assert ("reset", 7) in fake.calls
    env.reset()
    sets = [c for c in fake.calls if c[0] == "set_state"]
    assert sets == [("set_state", 0, 7.0), ("set_state", 1, 8.0)]
    env.reset(seed=11)
    assert ("reset", 11) in fake.calls
    fake.calls.clear()
    env.reset()
    assert [c for c in fake.calls if c[0] == "set_state"] == [("set_state", 0, 11.0), ("set_state", 1, 12.0)]
    # a reset observes the restored flow (STATE) without stepping it
    n_steps = len(fake.actions)
    obs = env.reset_arrays()
    assert len(fake.actions) == n_steps and fake.calls[-1] == "observe"
    assert obs[0, 0, 0, 0, 0, 0] == 1e4 * fake.step


def test_requests_map_and_termn_releases():
    env, fake = make()
    env.reset_arrays()
    env.cntrl(np.full((16, 16), 0.003))
    tau = env.evolve()
    assert np.array_equal(fake.actions[-1], np.full((1, 16, 16), 0.003)) and tau.shape == (1,)
    with pytest.raises(ValueError):
        env.cntrl(np.full((16, 16), np.inf))
    env.close()
    assert fake.calls[-1] == "destroy"
    with pytest.raises(RuntimeError):
        env.evolve()
    env.close()  # idempotent
    assert fake.calls.count("destroy") == 1


def test_window_validation():
    for w in ((2, 1), (1, 0), (17, 1), (1, 19)):
        with pytest.raises(ValueError):
            make(window=w)


def test_actuation_interval_and_opposition_policy():
    # Sec. 3.2: dt+ = 0.6 at dt = 0.005, Re_tau 180, Re_b 2800 (dt+ per step 0.0579)
    assert marl.steps_for_interval(0.6, 0.005, 180.0, 2800.0) == 10
    assert marl.steps_for_interval(0.01, 0.005, 180.0, 2800.0) == 1
    rng = np.random.default_rng(3)
    plane = rng.standard_normal((2, 2, 8, 8))
    a = marl.opposition_action(plane, alpha=0.5)
    assert np.allclose(a.mean(axis=(1, 2)), 0.0)
    v = plane[:, 1]
    assert np.allclose(a, -0.5 * (v - v.mean(axis=(1, 2), keepdims=True)))
