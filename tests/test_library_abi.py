"""The C-ABI library loads without a GPU, exports every declared symbol, and
its host-only entry points agree with the shared seeded-input generator."""

import ctypes
import os
import re

import numpy as np
import pytest

import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "channel_dns.h")


@pytest.fixture(scope="module")
def native():
    from paper_2301_09889_gb300 import build, native
    build.build()
    native.load()
    return native


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"^(?:int|size_t|const char\*)\s+(\w+)\s*\(", text, flags=re.M)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for n in ("env_create", "env_reset", "env_step", "env_destroy", "env_step_device",
              "env_get_state", "env_set_state", "ch_nonlinear", "ch_tau_helmholtz"):
        assert n in names


def test_every_declared_symbol_is_exported(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(native.EXPORTS)


def test_defaults_and_strerror(native):
    p = native.ch_default_params()
    assert (p.nx, p.ny, p.nz) == (16, 65, 16)
    assert p.re_tau == 180.0 and p.re_bulk == 2800.0 and p.dt == 0.005
    assert native.ch_strerror(native.CH_ERR_DIVERGED).startswith("flow diverged")
    assert native.ch_state_bytes(p) == 8 * (4 * 65 * 128 + 2 * 65 + 2 * 128 + 2)


@pytest.mark.parametrize("nx,ny,nz,seed,kmax", [(16, 65, 16, 0, 4), (12, 33, 24, 7, 99), (64, 65, 64, 3, 4)])
def test_seed_state_matches_python_generator(native, nx, ny, nz, seed, kmax):
    p = native.params(nx=nx, ny=ny, nz=nz)
    buf = native.ch_seed_state(p, seed, 0.1, kmax)
    st = native.unpack_state(buf, nx, ny, nz)
    ref = si.perturbed_poiseuille(nx, ny, nz, seed, 0.1, kmax)
    for k in ("v", "g", "U", "W"):
        assert np.array_equal(st[k], ref[k]), k
    assert np.all(st["vw"] == 0) and st["t"] == 0 and st["steps"] == 0


@pytest.mark.parametrize("nx,ny,nz,seed,kmax", [(16, 65, 16, 2, 4), (12, 33, 24, 9, 99)])
def test_open_channel_seed_state_matches_python_generator(native, nx, ny, nz, seed, kmax):
    p = native.params(nx=nx, ny=ny, nz=nz, top_bc=1)
    st = native.unpack_state(native.ch_seed_state(p, seed, 0.2, kmax), nx, ny, nz)
    ref = si.perturbed_poiseuille(nx, ny, nz, seed, 0.2, kmax, top_bc=1)
    for k in ("v", "g", "U", "W"):
        assert np.array_equal(st[k], ref[k]), k


def test_host_argument_checks(native):
    p = native.params(nx=15)
    with pytest.raises(native.ChannelError):
        native.ch_seed_state(p, 0, 0.1, 4)


def test_env_create_rejects_unsupported_parameters_before_any_device_work(native):
    """Parameter checks run before env_create touches the device, so they hold
    on a machine without a GPU: the free-slip top (top_bc = 1) is built for up
    to 65 nodes, other wall conditions do not exist, and malformed grids or
    modes are argument errors."""
    cases = [(dict(top_bc=1, ny=129), native.CH_ERR_UNSUPPORTED), (dict(top_bc=2), native.CH_ERR_ARG),
             (dict(precision=2), native.CH_ERR_UNSUPPORTED),
             (dict(control=3), native.CH_ERR_ARG), (dict(nx=15), native.CH_ERR_ARG),
             (dict(ny=5), native.CH_ERR_ARG), (dict(steps_per_action=0), native.CH_ERR_ARG),
             (dict(dt=0.0), native.CH_ERR_ARG)]
    for kw, code in cases:
        with pytest.raises(native.ChannelError) as e:
            native.env_create(native.params(**kw))
        assert e.value.code == code, kw
