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
            "y_sense_plus", "control", "alpha", "tau_ref")
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
        fields = si.perturbed_poiseuille(op.nx, op.ny, op.nz, seed, amp, kmax)
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


def wall_shear_tol(U: np.ndarray, nu: float, tol: float) -> float:
    """Error bound of tau_w = nu sum_n (-1)^(n+1) n^2 U_n implied by a relative
    L2 error `tol` on the coefficients U (Cauchy-Schwarz): nu ||n^2||_2 tol ||U||_2."""
    n = np.arange(U.size, dtype=np.float64)
    return nu * float(np.linalg.norm(n * n)) * tol * float(np.linalg.norm(U))


def compare_states(lst: dict, ost: dict, tol: float):
    errs = {k: rel_l2(lst[k], ost[k]) for k in ("v", "g", "U", "W")}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"state mismatch {errs}"
    return errs
