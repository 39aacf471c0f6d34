"""Unit parity of single stages through the C ABI: the tau Helmholtz solver
and the dealiased nonlinear plane kernel against the FP64 oracle."""

import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import oracle_params, rel_l2
from oracle import channel

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.mark.parametrize("ny", [9, 33, 65, 129])
def test_tau_helmholtz_matches_dense_oracle(native_gpu, ny):
    import torch
    native = native_gpu
    op = oracle_params(nx=4, ny=ny, nz=4, lx=6.28, lz=3.14)
    ops = channel.Operators(op)
    rng = np.random.default_rng(ny)
    M = 37
    lam = np.concatenate([[0.0, 0.5, 1.0, 3.4e6, 2e5], rng.uniform(0, 5e4, M - 5)])
    r = (rng.standard_normal((M, ny)) + 1j * rng.standard_normal((M, ny))) * 0.9 ** np.arange(ny)
    top = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    bot = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    ref = channel.tau_dirichlet(ops, lam, r, top, bot)
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_lam, d_r, d_top, d_bot = t(lam), t(r.view(np.float64)), t(top.view(np.float64)), t(bot.view(np.float64))
    d_f = torch.zeros(M, ny, 2, dtype=torch.float64, device=dev)
    native.ch_tau_helmholtz(ny, M, d_lam.data_ptr(), d_r.data_ptr(), d_top.data_ptr(), d_bot.data_ptr(),
                            d_f.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    f = d_f.cpu().numpy().view(np.complex128).reshape(M, ny)
    for m in range(M):
        assert rel_l2(f[m], ref[m]) < 1e-12, (m, lam[m], rel_l2(f[m], ref[m]))


# (256, 17, 256): FP64 planes of 256 x 256 modes run in three passes through
# global memory (no cluster holds their padded slabs)
@pytest.mark.parametrize("nx,ny,nz", [(16, 65, 16), (12, 17, 24), (64, 9, 64), (4, 9, 4), (128, 129, 128),
                                      (256, 17, 256)])
def test_nonlinear_plane_kernel(native_gpu, nx, ny, nz):
    import torch
    native = native_gpu
    op = oracle_params(nx=nx, ny=ny, nz=nz, lx=2 * np.pi, lz=np.pi)
    ops = channel.Operators(op)
    st = channel.new_state(si.perturbed_poiseuille(nx, ny, nz, 5, 0.3, 99), op)
    rng = np.random.default_rng(1)
    st["v"] = st["v"] + 0.01 * rng.standard_normal(st["v"].shape) * (st["v"] != 0)
    f = channel.velocity_vorticity(st, ops)
    nodes = {k: channel.from_pencils(f[k] @ ops.S.T) for k in channel.NODE_FIELDS}
    ref = channel.nonlinear_nodes(nodes, ops)
    q = np.stack([nodes[k] for k in channel.NODE_FIELDS])[None]          # [1][6][ny][nz][nxh]
    env = native.env_create(native.params(nx=nx, ny=ny, nz=nz, lx=2 * np.pi, lz=np.pi))
    try:
        dev = torch.device("cuda")
        d_q = torch.from_numpy(np.ascontiguousarray(q).view(np.float64)).to(dev)
        d_h = torch.full((1, 3, ny, nz, nx // 2, 2), float("nan"), dtype=torch.float64, device=dev)
        native.ch_nonlinear(env, d_q.data_ptr(), d_h.data_ptr())
        torch.cuda.synchronize()
        h = d_h.cpu().numpy().reshape(1, 3, ny, nz, nx // 2 * 2).view(np.complex128)[0]
    finally:
        native.env_destroy(env)
    for ci, c in enumerate("xyz"):
        e = rel_l2(h[ci], ref[c])
        assert e < TOL, (c, e)
