"""The allocation-free tau entry point gives the same answers as the regular one.

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

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the tolerance of the tau tests in test_gpu_kernels.py


def _problem(ny, M, seed):
    rng = np.random.default_rng(seed)
    lam = np.concatenate([[0.0, 1.0, 3.4e6], rng.uniform(0, 5e4, M - 3)])
    r = (rng.standard_normal((M, ny)) + 1j * rng.standard_normal((M, ny))) * 0.9 ** np.arange(ny)
    top = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    bot = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    return lam, r, top, bot


def _run(native, fn, ny, M, lam, r, top, bot):
    import torch
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_lam, d_r = t(lam), t(r.view(np.float64))
    d_top, d_bot = t(top.view(np.float64)), t(bot.view(np.float64))
    d_f = torch.full((M, ny, 2), float("nan"), dtype=torch.float64, device=dev)
    fn(ny, M, d_lam.data_ptr(), d_r.data_ptr(), d_top.data_ptr(), d_bot.data_ptr(), d_f.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return d_f.cpu().numpy().view(np.complex128).reshape(M, ny)


@pytest.mark.parametrize("ny,M", [(65, 300), (129, 41)])
def test_noalloc_matches_regular_entry_point_twice(native_gpu, ny, M):
    native = native_gpu
    for call, seed in enumerate((ny, ny + 1)):    # two calls in a row share the static array
        lam, r, top, bot = _problem(ny, M, seed)
        ref = _run(native, native.ch_tau_helmholtz, ny, M, lam, r, top, bot)
        got = _run(native, native.ch_tau_helmholtz_noalloc, ny, M, lam, r, top, bot)
        assert np.all(np.isfinite(got)), call
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL, (call, err)


def test_noalloc_rejects_requests_beyond_its_array(native_gpu):
    native = native_gpu
    # 65 nodes: mpad = 34, capacity 2^21 doubles -> at most 3855 problems
    with pytest.raises(native.ChannelError) as exc:
        native.ch_tau_helmholtz_noalloc(65, 100000, 1, 1, 1, 1, 1, None)
    assert exc.value.code == native.CH_ERR_ARG
