"""Helpers shared by the GPU parity tests (library side vs oracle side)."""

from __future__ import annotations

import numpy as np

import seeded_inputs as si
from oracle import channel


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_params(**kw) -> channel.Params:
    keys = ("nx", "ny", "nz", "lx", "lz", "re_tau", "re_bulk", "dt", "steps_per_action",
            "y_sense_plus", "control", "alpha", "tau_ref", "top_bc")
    return channel.Params(**{k: kw[k] for k in keys if k in kw})


def lib_params(native, **kw):
    p = native.params(**{k: v for k, v in kw.items()})
    return p


def run_pair(native, kw: dict, nsteps: int, seed: int = 0, amp: float = 0.1, kmax: int = 4,
             action_std: float | None = 0.05, action_seed: int = 11):
    """Run the library and the oracle side by side from the same seeded state.

    Returns (lib_results, oracle_results, final lib state dict, final oracle state dict).
    """
    p = native.params(**kw)
    op = oracle_params(**kw)
    ops = channel.Operators(op)
    env = native.env_create(p)
    try:
        fields = si.perturbed_poiseuille(op.nx, op.ny, op.nz, seed, amp, kmax, top_bc=op.top_bc)
        native.env_set_state(env, 0, native.pack_state(fields, op.nx, op.ny, op.nz))
        ost = channel.new_state(fields, op)
        lib_out, ora_out = [], []
        for t in range(nsteps):
            act = None
            if op.control == 0:
                std = (action_std or 0.0) * op.u_tau
                act = si.wall_action(op.nx, op.nz, action_seed * 1000003 + t, std)
            obs = np.zeros((2, op.nz, op.nx))
            tau = np.zeros(1)
            rew = np.zeros(1)
            rc = native.env_step(env, None if act is None else np.ascontiguousarray(act), obs, tau, rew)
            assert rc == 0
            lib_out.append((obs, tau[0], rew[0]))
            ora_out.append(channel.env_step(ost, ops, act))
        lst = native.unpack_state(native.env_get_state(env, 0), op.nx, op.ny, op.nz)
    finally:
        native.env_destroy(env)
    return lib_out, ora_out, lst, channel.canonical(ost)


def compare_states(lst: dict, ost: dict, tol: float):
    errs = {k: rel_l2(lst[k], ost[k]) for k in ("v", "g", "U", "W")}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"state mismatch {errs}"
    return errs


def run_batch_pair(native, kw: dict, B: int, slots, nsteps: int, seed0: int = 300, amp: float = 0.2,
                   kmax: int = 99, action_std: float = 0.05, action_seed0: int = 5000, tiles=None):
    """One batched handle of B environments (seed0 + e) stepped with per-slot
    seeded actions; the oracle replays the sampled `slots` one by one.
    `tiles` = (ppc_pre, ppc_post, post_batched) pins the stage-kernel shapes.

    Returns (info, {slot: (lib_results, oracle_results, lib state, oracle state)})."""
    op = oracle_params(**kw)
    ops = channel.Operators(op)
    nx, ny, nz = op.nx, op.ny, op.nz
    env = native.env_create(native.params(**kw, batch=B))
    try:
        if tiles is not None:
            native.env_set_tiles(env, *tiles)
        info = native.env_info(env)
        fields = [si.perturbed_poiseuille(nx, ny, nz, seed0 + e, amp, kmax, top_bc=op.top_bc) for e in range(B)]
        for e in range(B):
            native.env_set_state(env, e, native.pack_state(fields[e], nx, ny, nz))
        acts = []
        outs = []
        obs, tau, rew = np.zeros((B, 2, nz, nx)), np.zeros(B), np.zeros(B)
        for t in range(nsteps):
            a = None
            if op.control == 0:
                a = np.stack([si.wall_action(nx, nz, action_seed0 + 7919 * t + e, action_std * op.u_tau)
                              for e in range(B)])
            acts.append(a)
            assert native.env_step(env, a, obs, tau, rew) == 0
            outs.append((obs.copy(), tau.copy(), rew.copy()))
        lib_states = {e: native.unpack_state(native.env_get_state(env, e), nx, ny, nz) for e in slots}
    finally:
        native.env_destroy(env)
    res = {}
    for e in slots:
        ost = channel.new_state(fields[e], op)
        ora = [channel.env_step(ost, ops, None if acts[t] is None else acts[t][e]) for t in range(nsteps)]
        lib = [(o[e], tt[e], rr[e]) for o, tt, rr in outs]
        res[e] = (lib, ora, lib_states[e], channel.canonical(ost))
    return info, res
