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


def test_fluctuation_densities_skewness_and_flatness():
    """The densities integrate to one over wall units and put their mass
    where the samples are; skewness and flatness follow from the moments."""
    scale, u_tau0 = 0.05, 0.064
    st = validate.PlaneStats(1, scale)
    obs = np.zeros((1, 2, 4, 4))
    rng = np.random.default_rng(3)
    for _ in range(200):
        obs[0, 0] = 2.0 + scale * rng.standard_normal((4, 4))
        obs[0, 1] = np.where(rng.random((4, 4)) < 0.25, 3.0, -1.0) * scale   # skewed two-point law
        st.add(np.array([1.0]), obs, np.array([True]))
    s = st.summary(u_tau0)
    for key in ("pdf_u", "pdf_v"):
        c, d = np.array(s[key]["bin_centers_plus"]), np.array(s[key]["density"])
        assert s[key]["outside"] == pytest.approx(0.0, abs=1e-3)
        assert float((d * np.gradient(c)).sum()) == pytest.approx(1.0, rel=2e-3)
    # the centred Gaussian u' (about each plane's mean): symmetric, flatness near 3
    assert abs(s["u_skewness"]) < 0.2 and s["u_flatness"] == pytest.approx(3.0, abs=0.4)
    # v' about each plane's mean of a +3 / -1 law with weights 1/4, 3/4: skewed
    # positive, so the density has more mass above zero at large |v'|
    assert s["v_skewness"] > 0.5
    cv, dv = np.array(s["pdf_v"]["bin_centers_plus"]), np.array(s["pdf_v"]["density"])
    assert dv[cv > 1.5 * scale / u_tau0].sum() > dv[cv < -1.5 * scale / u_tau0].sum()
    # exact moments of a two-point law: +-1 in equal numbers has skewness 0, flatness 1
    st2 = validate.PlaneStats(1, 1.0)
    obs2 = np.zeros((1, 2, 2, 2))
    obs2[0, 0] = [[1.0, -1.0], [-1.0, 1.0]]
    obs2[0, 1] = [[2.0, -2.0], [2.0, -2.0]]
    st2.add(np.array([1.0]), obs2, np.array([True]))
    s2 = st2.summary(1.0)
    assert s2["u_skewness"] == pytest.approx(0.0) and s2["u_flatness"] == pytest.approx(1.0)
    assert s2["v_flatness"] == pytest.approx(1.0)
