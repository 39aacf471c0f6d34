"""Host logic of the opposition-control validation run against a fake binding:
the drag reduction of the channels that were turbulent when the copies
branched, the laminar bound, and the sensing-plane quadrant statistics.  No GPU."""

from types import SimpleNamespace

import numpy as np
import pytest

from paper_2301_09889_gb300 import native, validate


class FakeBinding:
    """Channel b has wall shear tau_b (uncontrolled) and 0.75 tau_b under
    opposition control; channel 1 is laminar (3 / Re_b).  The sensing plane
    holds u' = +-1, v' = +-2 in a fixed quadrant pattern."""

    CH_OK = native.CH_OK
    taus = np.array([0.0041, 3.0 / 2800.0, 0.0045])

    def __init__(self):
        self.handles = []

    def params(self, **kw):
        return SimpleNamespace(**kw)

    def env_create(self, p):
        h = SimpleNamespace(p=p, state=None)
        self.handles.append(h)
        return h

    def env_reset(self, env, seed, amplitude, kmax):
        env.state = ["seeded"] * env.p.batch

    def env_get_state(self, env, b):
        return env.state[b]

    def env_set_state(self, env, b, buf):
        if env.state is None:
            env.state = [None] * env.p.batch
        env.state[b] = buf

    def env_info(self, env):
        return SimpleNamespace(j_sense=55, y_plus_sense=17.28)

    def env_step(self, env, act, obs, tau, rew):
        assert (act is None) == (env.p.control == 1)
        tau[:] = self.taus * (0.75 if env.p.control == 1 else 1.0)
        nz, nx = obs.shape[2:]
        iz, ix = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        # quadrants by (iz + ix) % 4: Q1, Q2, Q3, Q4
        q = (iz + ix) % 4
        obs[:, 0] = 5.0 + np.where((q == 0) | (q == 3), 1.0, -1.0)
        obs[:, 1] = 0.1 + np.where(q <= 1, 2.0, -2.0)
        return self.CH_OK

    def ch_strerror(self, rc):
        return str(rc)

    def env_destroy(self, env):
        pass


def test_drag_reduction_over_turbulent_channels(monkeypatch):
    fake = FakeBinding()
    monkeypatch.setattr(validate, "native", fake)
    out = validate.run("minimal", batch=3, t_spin=1.0, t_trans=0.2, t_avg=1.0, spa=10)
    assert out["turbulent_at_branch"] == 2
    assert out["drag_reduction"] == pytest.approx(0.25) and out["drag_reduction_spread"] == pytest.approx(0.0, abs=1e-15)
    tu = (0.0041 + 0.0045) / 2
    assert out["tau_w_uncontrolled"] == pytest.approx(tu)
    assert out["laminar_bound"] == pytest.approx(1 - (3 / 2800) / tu)
    assert out["re_tau_uncontrolled"] == pytest.approx(np.sqrt(tu) * 2800)
    pu = out["plane_uncontrolled"]
    assert pu["quadrants_Q1_Q2_Q3_Q4"] == [0.25, 0.25, 0.25, 0.25]
    u_tau0 = np.sqrt(tu)
    assert pu["u_rms_plus"] == pytest.approx(1.0 / u_tau0) and pu["v_rms_plus"] == pytest.approx(2.0 / u_tau0)
    # Q1 and Q3 give +2, Q2 and Q4 give -2: zero mean product
    assert pu["uv_plus"] == pytest.approx(0.0, abs=1e-12)
    assert len(fake.handles) == 2 and fake.handles[1].state == ["seeded"] * 3


def test_quadrant_fractions_and_fluctuation_removal():
    st = validate.PlaneStats(1)
    obs = np.zeros((1, 2, 2, 2))
    obs[0, 0] = [[3.0, 1.0], [1.0, 3.0]]       # u' = +1, -1, -1, +1 about the mean 2
    obs[0, 1] = [[-1.0, -1.0], [1.0, 1.0]]     # v' = -1, -1, +1, +1 about 0
    st.add(np.array([1.0]), obs, np.array([True]))
    # (u', v') = (+,-) Q4, (-,-) Q3, (-,+) Q2, (+,+) Q1
    assert st.summary(1.0)["quadrants_Q1_Q2_Q3_Q4"] == [0.25, 0.25, 0.25, 0.25]
    assert st.summary(1.0)["uv_plus"] == pytest.approx(0.0)
    obs[0, 1] = [[1.0, -1.0], [-1.0, 1.0]]     # v' follows u': Q1 and Q3 only
    st2 = validate.PlaneStats(1)
    st2.add(np.array([1.0]), obs, np.array([True]))
    assert st2.summary(1.0)["quadrants_Q1_Q2_Q3_Q4"] == [0.5, 0.0, 0.5, 0.0]
    assert st2.summary(2.0)["uv_plus"] == pytest.approx(1.0 / 4.0)


def test_open_channel_run_uses_the_papers_box_and_transient(monkeypatch):
    """top_bc = 1: the boxes are given in units of the channel height, which
    is 2 in units of y, so the lengths double; the default transient is
    t+ = 500 with nu = 2 / Re_b."""
    fake = FakeBinding()
    monkeypatch.setattr(validate, "native", fake)
    out = validate.run("minimal", batch=3, t_spin=1.0, t_avg=1.0, spa=10, top_bc=1)
    p = fake.handles[0].p
    assert p.top_bc == 1 and fake.handles[1].p.top_bc == 1
    assert p.lx == pytest.approx(2 * 2.67) and p.lz == pytest.approx(2 * 0.8)
    assert out["lx_lz"] == [pytest.approx(5.34), pytest.approx(1.6)]
    assert out["t_transient"] == pytest.approx(500 * (2 / 2800) / (180 / 2800) ** 2)
    assert out["geometry"] == "open channel, free-slip top"
