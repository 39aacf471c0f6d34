"""The allocation-free tau entry point against the FP64 oracle and the regular
entry point.

``ch_tau_helmholtz_noalloc`` exists for callers that cannot let anything
allocate device memory (real-time control loops, processes whose memory is
owned by another allocator, hosts that only lend their own buffers).  It keeps
its work vectors in a static array inside the library instead of per-thread
local memory.  This file runs last so that a failure here leaves every other
test already run; it also passes on its own in a fresh process, where its
first call performs the one-time lookup of that array's device address.
"""

import numpy as np
import pytest

from gpu_util import oracle_params
from oracle import channel

pytestmark = pytest.mark.gpu

TOL = 1e-12   # per problem, relative L2: the tolerance of the tau tests in test_gpu_kernels.py
TOL_201 = 1e-11   # 201 nodes: the all-FP64 bar (the tau operator's conditioning grows like N^4)


def _capacity(ny):
    """Largest M the 2^21-double array holds: 2 M 8 mpad <= 2^21, mpad = ny/2 + 1 rounded up to even."""
    mpad = ((ny // 2 + 1) + 1) & ~1
    return (1 << 21) // (16 * mpad)


def _problem(ny, M, seed):
    rng = np.random.default_rng(seed)
    lam = np.concatenate([[0.0, 1.0, 3.4e6], rng.uniform(0, 5e4, M - 3)])
    r = (rng.standard_normal((M, ny)) + 1j * rng.standard_normal((M, ny))) * 0.9 ** np.arange(ny)
    top = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    bot = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    return lam, r, top, bot


def _run(native, fn, ny, M, lam, r, top, bot, raises=False):
    import torch
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_lam, d_r = t(lam), t(r.view(np.float64))
    d_top, d_bot = t(top.view(np.float64)), t(bot.view(np.float64))
    d_f = torch.full((M, ny, 2), float("nan"), dtype=torch.float64, device=dev)
    args = (ny, M, d_lam.data_ptr(), d_r.data_ptr(), d_top.data_ptr(), d_bot.data_ptr(), d_f.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    if raises:
        with pytest.raises(native.ChannelError) as exc:
            fn(*args)
        torch.cuda.synchronize()
        return exc.value.code, d_f.cpu().numpy()
    fn(*args)
    torch.cuda.synchronize()
    return d_f.cpu().numpy().view(np.complex128).reshape(M, ny)


def _oracle(ny, lam, r, top, bot):
    ops = channel.Operators(oracle_params(nx=4, ny=ny, nz=4, lx=6.28, lz=3.14))
    return channel.tau_dirichlet(ops, lam, r, top, bot)


def _per_problem_error(got, ref):
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("ny,M", [(65, 300), (129, 41), (201, 64)])
def test_noalloc_matches_oracle_on_two_calls_in_a_row(native_gpu, ny, M):
    native = native_gpu
    tol = TOL_201 if ny > 129 else TOL
    for call, seed in enumerate((ny, ny + 1)):    # two calls in a row share the static array
        lam, r, top, bot = _problem(ny, M, seed)
        got = _run(native, native.ch_tau_helmholtz_noalloc, ny, M, lam, r, top, bot)
        assert np.all(np.isfinite(got)), call
        err = _per_problem_error(got, _oracle(ny, lam, r, top, bot))
        assert err.max() <= tol, (call, err.max(), int(err.argmax()))
        # and the regular entry point, which keeps the same vectors in local memory
        ref = _run(native, native.ch_tau_helmholtz, ny, M, lam, r, top, bot)
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), call


@pytest.mark.parametrize("ny", [65, 201])
def test_noalloc_capacity_edge(native_gpu, ny):
    """The largest request the array holds runs and matches the oracle; one
    more problem is refused with CH_ERR_ARG before anything is launched (the
    output buffer keeps its contents)."""
    native = native_gpu
    cap = _capacity(ny)
    assert cap == {65: 3855, 201: 1285}[ny]
    lam, r, top, bot = _problem(ny, cap, 7 * ny)
    got = _run(native, native.ch_tau_helmholtz_noalloc, ny, cap, lam, r, top, bot)
    err = _per_problem_error(got, _oracle(ny, lam, r, top, bot))
    assert err.max() <= (TOL_201 if ny > 129 else TOL), (err.max(), int(err.argmax()))
    lam, r, top, bot = _problem(ny, cap + 1, 7 * ny + 1)
    code, out = _run(native, native.ch_tau_helmholtz_noalloc, ny, cap + 1, lam, r, top, bot, raises=True)
    assert code == native.CH_ERR_ARG
    assert np.isnan(out).all()


def test_noalloc_rejects_requests_far_beyond_its_array(native_gpu):
    native = native_gpu
    with pytest.raises(native.ChannelError) as exc:
        native.ch_tau_helmholtz_noalloc(65, 100000, 1, 1, 1, 1, 1, None)
    assert exc.value.code == native.CH_ERR_ARG
