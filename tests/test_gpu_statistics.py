"""Long-window statistics of the GPU trajectory against the oracle's.

The mean streamwise profile U(y) and the Reynolds stresses <u'u'>, <v'v'>,
<w'w'>, <u'v'>, averaged over the wall-parallel planes and over every step of
a 200-step window of the minimal channel (seeded perturbed Poiseuille flow,
seeded zero-net-mass-flux wall actions), are computed the same way from the
library's states and from the oracle's states on the same inputs.  The all-FP64
path must agree to 1e-8 (its states agree to about 1e-11); the mixed path,
whose nonlinear term is FP32, within 1 %.
"""

import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import oracle_params
from oracle import channel

pytestmark = pytest.mark.gpu

MINIMAL = dict(nx=16, ny=65, nz=16, lx=2.67, lz=0.8, re_tau=180.0, re_bulk=2800.0, dt=0.005)
STEPS = 200
SEED, AMP = 9, 0.3


def _plane_stats(fields: dict, op, ops) -> np.ndarray:
    """[5][ny]: U, <u'u'>, <v'v'>, <w'w'>, <u'v'> at the Gauss-Lobatto nodes of
    one state (plane averages by Parseval; kx > 0 modes count twice)."""
    st = channel.new_state(fields, op)
    f = channel.velocity_vorticity(st, ops)          # [nz][nx/2][ny] coefficients
    S = ops.S
    u, v, w = (f[k] @ S.T for k in ("u", "v", "w"))  # values at the nodes
    wt = np.full((op.nz, op.nx // 2, 1), 2.0)
    wt[:, 0, 0] = 1.0
    wt[0, 0, 0] = 0.0                                # the (0,0) mode is the mean
    mean = S @ st["U"]
    uu = (wt * np.abs(u) ** 2).sum(axis=(0, 1))
    vv = (wt * np.abs(v) ** 2).sum(axis=(0, 1))
    ww = (wt * np.abs(w) ** 2).sum(axis=(0, 1))
    uv = (wt * (u * np.conj(v)).real).sum(axis=(0, 1))
    return np.stack([mean, uu, vv, ww, uv])


def _actions(op):
    return [si.wall_action(op.nx, op.nz, 9100 + t, 0.05 * op.u_tau) for t in range(STEPS)]


@pytest.fixture(scope="module")
def oracle_window():
    op = oracle_params(**MINIMAL)
    ops = channel.Operators(op)
    fields = si.perturbed_poiseuille(op.nx, op.ny, op.nz, SEED, AMP, 99)
    st = channel.new_state(fields, op)
    acc = np.zeros((5, op.ny))
    for a in _actions(op):
        channel.env_step(st, ops, a)
        acc += _plane_stats(channel.canonical(st), op, ops)
    return acc / STEPS


def _gpu_window(native, precision):
    op = oracle_params(**MINIMAL)
    ops = channel.Operators(op)
    env = native.env_create(native.params(**MINIMAL, precision=precision))
    try:
        fields = si.perturbed_poiseuille(op.nx, op.ny, op.nz, SEED, AMP, 99)
        native.env_set_state(env, 0, native.pack_state(fields, op.nx, op.ny, op.nz))
        obs, tau, rew = np.zeros((2, op.nz, op.nx)), np.zeros(1), np.zeros(1)
        acc = np.zeros((5, op.ny))
        for a in _actions(op):
            assert native.env_step(env, np.ascontiguousarray(a), obs, tau, rew) == 0
            acc += _plane_stats(native.unpack_state(native.env_get_state(env, 0), op.nx, op.ny, op.nz), op, ops)
    finally:
        native.env_destroy(env)
    return acc / STEPS


def _errors(gpu, ora):
    """Per statistic: max over y of the difference, relative to the max over y
    of the oracle's profile."""
    names = ("U", "uu", "vv", "ww", "uv")
    return {n: float(np.abs(g - o).max() / np.abs(o).max()) for n, g, o in zip(names, gpu, ora)}


def test_fp64_window_statistics(native_gpu, oracle_window):
    err = _errors(_gpu_window(native_gpu, 0), oracle_window)
    assert all(e < 1e-8 for e in err.values()), err
    # the window is not degenerate: the fluctuations carry energy
    assert np.abs(oracle_window[1]).max() > 1e-4


def test_mixed_window_statistics(native_gpu, oracle_window):
    err = _errors(_gpu_window(native_gpu, 1), oracle_window)
    print("\nmixed-precision 200-step statistics, relative error:", {k: f"{v:.1e}" for k, v in err.items()})
    assert all(e < 1e-2 for e in err.values()), err
