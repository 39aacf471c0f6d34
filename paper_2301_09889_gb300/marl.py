"""Multi-agent interface in the shape of a PettingZoo parallel environment.

The control problem of Sec. 3.2: a grid of Nx x Nz agents covers the lower
wall, one per grid point, all sharing one policy.  Agent (iz, ix) observes the
sensing plane (u and v at the Gauss-Lobatto node nearest y+_s) above its
actuator, here a periodic window of wz x wx points centred on it (1 x 1 =
only the point above the actuator), and sets the wall-normal velocity of its
grid point.  The library limits every action to [-u_tau, u_tau], removes the
plane mean (zero net mass flux) and ramps it linearly from the previous one
over the actuation interval.  Every agent receives the same reward, the
relative reduction of the wall-shear stress against the uncontrolled value,
averaged over the interval.  An episode restarts from the same initial
condition unless `reset` is given a new seed (Sec. 3.3).

The four requests of the paper's solver interface (Sec. 3.3) map to
`state` (STATE), `cntrl` (CNTRL), `evolve` (EVOLVE) and `close` (TERMN);
`reset` / `step` are the dictionary interface of a parallel multi-agent
environment built from them, and `reset_arrays` / `step_arrays` the same with
one array per quantity, the form a shared-policy learner batches over.

Every step runs through :mod:`paper_2301_09889_gb300.native` (the C ABI);
this module only slices observations and assembles actions on the host.
"""

from __future__ import annotations

import numpy as np

from . import native as _native


def steps_for_interval(dt_plus: float, dt: float, re_tau: float, re_bulk: float) -> int:
    """RK3 steps per action for an actuation interval of `dt_plus` viscous time
    units: t+ = t u_tau^2 / nu with u_tau = Re_tau / Re_b and nu = 1 / Re_b in
    bulk units (Sec. 3.2 uses dt+ = 0.6)."""
    u_tau = re_tau / re_bulk
    nu = 1.0 / re_bulk
    return max(1, int(round(dt_plus * nu / (u_tau * u_tau) / dt)))


class ChannelMARL:
    """B channels (one C-ABI handle), Nx x Nz agents each.

    params: keyword arguments of ``native.params`` (grid, box, Reynolds numbers,
    dt, steps_per_action, y_sense_plus, precision); `control` is forced to the
    external-action mode.  window: (wz, wx) odd window of the sensing plane
    each agent observes.  seed, amplitude, kmax: the seeded initial condition
    (environment b uses seed + b); initial_state: optional [B][state] arrays
    that replace it.  max_cycles: actions per episode before truncation.
    backend: the binding (tests substitute a host fake).
    """

    components = ("u", "v")

    def __init__(self, params: dict | None = None, *, batch: int = 1, window: tuple[int, int] = (1, 1),
                 seed: int = 0, amplitude: float = 0.1, kmax: int = 4, initial_state=None,
                 max_cycles: int = 1000, backend=None):
        self._nat = backend if backend is not None else _native
        kw = dict(params or {})
        kw["control"] = 0
        kw["batch"] = batch
        wz, wx = window
        if wz < 1 or wx < 1 or wz % 2 == 0 or wx % 2 == 0:
            raise ValueError("observation window sides must be odd and positive")
        self._p = self._nat.params(**kw)
        self.B, self.nx, self.nz = batch, self._p.nx, self._p.nz
        if wz > self.nz or wx > self.nx:
            raise ValueError("observation window larger than the wall grid")
        self.window = (wz, wx)
        self.max_cycles = max_cycles
        self._env = self._nat.env_create(self._p)
        try:
            info = self._nat.env_info(self._env)
            self.u_tau = float(info.u_tau)
            self.tau_ref = float(info.tau_ref)
            self.y_plus_sense = float(info.y_plus_sense)
            if initial_state is None:
                self._nat.env_reset(self._env, seed, amplitude, kmax)
            else:
                for b in range(batch):
                    self._nat.env_set_state(self._env, b, initial_state[b])
            self._init = [self._nat.env_get_state(self._env, b) for b in range(batch)]
        except Exception:
            self._nat.env_destroy(self._env)
            self._env = None
            raise
        # periodic window offsets, centred on the agent
        self._iz = (np.arange(self.nz)[:, None] + np.arange(wz)[None, :] - wz // 2) % self.nz
        self._ix = (np.arange(self.nx)[:, None] + np.arange(wx)[None, :] - wx // 2) % self.nx
        self.possible_agents = [self._name(b, iz, ix) for b in range(batch) for iz in range(self.nz)
                                for ix in range(self.nx)]
        self.agents: list[str] = []
        self._plane = np.zeros((batch, 2, self.nz, self.nx))
        self._action = np.zeros((batch, self.nz, self.nx))
        self._wall_shear = np.zeros(batch)
        self._reward = np.zeros(batch)
        self._cycles = 0
        self._diverged = False

    # ---- naming and spaces
    def _name(self, b: int, iz: int, ix: int) -> str:
        return f"agent_{iz}_{ix}" if self.B == 1 else f"env{b}_agent_{iz}_{ix}"

    def observation_shape(self) -> tuple[int, int, int]:
        """Per agent: (component, z, x) window of u and v."""
        return (2,) + self.window

    def action_bounds(self) -> tuple[float, float]:
        return -self.u_tau, self.u_tau

    # ---- the paper's requests
    def state(self) -> np.ndarray:
        """STATE: the sensing plane [B][2][nz][nx] (u, v) after the last interval."""
        return self._plane.copy()

    def cntrl(self, action) -> None:
        """CNTRL: set the wall-normal velocity [B][nz][nx] (or [nz][nx] for B = 1)
        applied over the next interval."""
        a = np.asarray(action, dtype=np.float64).reshape(self.B, self.nz, self.nx)
        if not np.all(np.isfinite(a)):
            raise ValueError("non-finite action")
        self._action[...] = a

    def evolve(self) -> np.ndarray:
        """EVOLVE: advance steps_per_action RK3 steps under the action set by
        `cntrl`; returns the wall shear [B] averaged over them."""
        self._require_open()
        rc = self._nat.env_step(self._env, self._action, self._plane, self._wall_shear, self._reward)
        self._diverged = rc == _native.CH_ERR_DIVERGED
        self._cycles += 1
        return self._wall_shear.copy()

    def close(self) -> None:
        """TERMN: release the device state."""
        if self._env is not None:
            self._nat.env_destroy(self._env)
            self._env = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _require_open(self):
        if self._env is None:
            raise RuntimeError("environment closed")

    # ---- array interface
    def observe_arrays(self) -> np.ndarray:
        """Per-agent windows [B][nz][nx][2][wz][wx] of the current sensing plane."""
        w = self._plane[:, :, self._iz[:, None, :, None], self._ix[None, :, None, :]]  # [B][2][nz][nx][wz][wx]
        return np.ascontiguousarray(w.transpose(0, 2, 3, 1, 4, 5))

    def reset_arrays(self, seed: int | None = None, amplitude: float = 0.1, kmax: int = 4) -> np.ndarray:
        """Restore the initial condition (or seed a new one, which then becomes
        the stored one) and return the windows of its sensing plane (STATE:
        no step is taken).  The restored state carries its wall action, zero
        for a seeded one, from which the first interval ramps."""
        self._require_open()
        if seed is None:
            for b in range(self.B):
                self._nat.env_set_state(self._env, b, self._init[b])
        else:
            self._nat.env_reset(self._env, seed, amplitude, kmax)
            self._init = [self._nat.env_get_state(self._env, b) for b in range(self.B)]
        self._action[...] = 0.0
        self._nat.env_observe(self._env, self._plane)
        self._cycles = 0
        self._diverged = False
        return self.observe_arrays()

    def step_arrays(self, action) -> tuple[np.ndarray, np.ndarray, np.ndarray, bool, bool]:
        """One interval: returns (windows [B][nz][nx][2][wz][wx], reward [B],
        wall shear [B], terminated, truncated).  `terminated` is set when a wall
        shear is not finite (the flow diverged)."""
        self.cntrl(action)
        self.evolve()
        truncated = self._cycles >= self.max_cycles
        return self.observe_arrays(), self._reward.copy(), self._wall_shear.copy(), self._diverged, truncated

    # ---- dictionary interface (parallel multi-agent environment)
    def reset(self, seed: int | None = None, options: dict | None = None):
        opts = options or {}
        obs = self.reset_arrays(seed, opts.get("amplitude", 0.1), opts.get("kmax", 4))
        self.agents = list(self.possible_agents)
        return self._to_dict(obs), {a: {} for a in self.agents}

    def step(self, actions: dict):
        a = np.zeros((self.B, self.nz, self.nx))
        for name, val in actions.items():
            b, iz, ix = self._index(name)
            a[b, iz, ix] = float(val)
        obs, rew, tau, term, trunc = self.step_arrays(a)
        od = self._to_dict(obs)
        rd, td, trd, info = {}, {}, {}, {}
        for b in range(self.B):
            for iz in range(self.nz):
                for ix in range(self.nx):
                    n = self._name(b, iz, ix)
                    rd[n] = float(rew[b])
                    td[n] = term
                    trd[n] = trunc
                    info[n] = {"wall_shear": float(tau[b])}
        if term or trunc:
            self.agents = []
        return od, rd, td, trd, info

    def _index(self, name: str) -> tuple[int, int, int]:
        parts = name.split("_")
        b = 0 if self.B == 1 else int(parts[0][3:])
        iz, ix = int(parts[-2]), int(parts[-1])
        if not (0 <= b < self.B and 0 <= iz < self.nz and 0 <= ix < self.nx):
            raise KeyError(name)
        return b, iz, ix

    def _to_dict(self, obs: np.ndarray) -> dict:
        return {self._name(b, iz, ix): obs[b, iz, ix] for b in range(self.B) for iz in range(self.nz)
                for ix in range(self.nx)}


def opposition_action(plane: np.ndarray, alpha: float = 1.0) -> np.ndarray:
    """Opposition control of Sec. 4.1 as an agent policy: v_w = -alpha (v_s - <v_s>)
    from the sensing plane [B][2][nz][nx] (v is component 1)."""
    v = plane[:, 1]
    return -alpha * (v - v.mean(axis=(1, 2), keepdims=True))


__all__ = ["ChannelMARL", "steps_for_interval", "opposition_action"]
