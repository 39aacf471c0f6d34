"""ctypes binding of the C ABI in ``include/channel_dns.h``.

Argument marshalling only: every computation runs in ``libchannel_dns.so``.
Function names follow the C ABI.  Errors raise :class:`ChannelError` with the
library's status code.  Importing this module does not need a GPU; calling
anything that touches device memory does.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchannel_dns.so")

CH_OK = 0
CH_ERR_ARG = -1
CH_ERR_OOM = -2
CH_ERR_BUDGET = -3
CH_ERR_DIVERGED = -4
CH_ERR_TIMEOUT = -5
CH_ERR_STATE = -6
CH_ERR_CUDA = -7
CH_ERR_UNSUPPORTED = -8

# every symbol the header declares
EXPORTS = (
    "ch_default_params", "env_create", "env_set_stream", "env_reset", "env_step",
    "env_step_device", "env_get_state", "env_set_state", "env_info", "env_destroy",
    "ch_strerror", "ch_seed_state", "ch_state_bytes", "ch_nonlinear", "ch_tau_helmholtz",
    "env_profile", "env_profile_read", "ch_tau_helmholtz_noalloc", "env_set_tiles",
    "srv_create", "srv_admit", "srv_evict", "srv_submit", "srv_poll", "srv_wait", "srv_get_state",
    "srv_set_state", "srv_stats", "srv_destroy", "env_set_policy", "env_get_action", "env_observe",
    "srv_set_linger", "srv_submit_many", "srv_wait_many",
)
CH_PENDING = 1


class ChParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("lz", ctypes.c_double),
        ("re_tau", ctypes.c_double), ("re_bulk", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("steps_per_action", ctypes.c_int),
        ("y_sense_plus", ctypes.c_double),
        ("top_bc", ctypes.c_int), ("precision", ctypes.c_int), ("control", ctypes.c_int),
        ("alpha", ctypes.c_double), ("tau_ref", ctypes.c_double),
        ("batch", ctypes.c_int),
        ("autotune", ctypes.c_int),
    ]


class ChInfo(ctypes.Structure):
    _fields_ = [
        ("j_sense", ctypes.c_int),
        ("y_plus_sense", ctypes.c_double),
        ("nu", ctypes.c_double), ("u_tau", ctypes.c_double), ("tau_ref", ctypes.c_double),
        ("state_bytes", ctypes.c_size_t),
        ("device_bytes", ctypes.c_size_t),
        ("plane_cluster", ctypes.c_int),
        ("launches_per_step", ctypes.c_int),
        ("post_batched", ctypes.c_int),
        ("ppc_pre", ctypes.c_int), ("ppc_post", ctypes.c_int),
        ("tuned", ctypes.c_int),
        ("tune_ms", ctypes.c_double),
        ("plane_team", ctypes.c_int),
    ]


class ChPolicy(ctypes.Structure):
    _fields_ = [
        ("wz", ctypes.c_int), ("wx", ctypes.c_int),
        ("n_hidden", ctypes.c_int),
        ("width", ctypes.c_int * 2),
        ("out_tanh", ctypes.c_int),
    ]


class ChSrvStats(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_uint64),
        ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
        ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
        ("env_steps_per_s", ctypes.c_double),
        ("classes", ctypes.c_int), ("envs", ctypes.c_int), ("pending", ctypes.c_int),
        ("hbm_used", ctypes.c_size_t), ("hbm_budget", ctypes.c_size_t),
        ("worker_status", ctypes.c_int),
    ]


class ChannelError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ch_strerror(code)} ({code})")


_lib = None


def load() -> ctypes.CDLL:
    """Load the shared library; fails loudly when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    dp = P(ctypes.c_double)
    sig = {
        "ch_default_params": (ctypes.c_int, [P(ChParams)]),
        "env_create": (ctypes.c_int, [P(ChParams), P(vp)]),
        "env_set_stream": (ctypes.c_int, [vp, vp]),
        "env_reset": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_int]),
        "env_step": (ctypes.c_int, [vp, dp, dp, dp, dp]),
        "env_step_device": (ctypes.c_int, [vp, vp, vp]),
        "env_get_state": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_size_t]),
        "env_set_state": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_size_t]),
        "env_info": (ctypes.c_int, [vp, P(ChInfo)]),
        "env_destroy": (ctypes.c_int, [vp]),
        "ch_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "ch_seed_state": (ctypes.c_int, [P(ChParams), ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                         vp, ctypes.c_size_t]),
        "ch_state_bytes": (ctypes.c_size_t, [P(ChParams)]),
        "ch_nonlinear": (ctypes.c_int, [vp, vp, vp]),
        "ch_tau_helmholtz": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp]),
        "ch_tau_helmholtz_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp]),
        "env_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "env_set_tiles": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "srv_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, P(vp)]),
        "srv_set_linger": (ctypes.c_int, [vp, ctypes.c_int]),
        "srv_submit_many": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int), dp, P(ctypes.c_uint64)]),
        "srv_wait_many": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_uint64), ctypes.c_int, dp, dp, dp,
                                         P(ctypes.c_int)]),
        "srv_admit": (ctypes.c_int, [vp, P(ChParams), ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                     P(ctypes.c_int)]),
        "srv_evict": (ctypes.c_int, [vp, ctypes.c_int]),
        "srv_submit": (ctypes.c_int, [vp, ctypes.c_int, dp, P(ctypes.c_uint64)]),
        "srv_poll": (ctypes.c_int, [vp, ctypes.c_uint64, dp, dp, dp, dp]),
        "srv_wait": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_int, dp, dp, dp, dp]),
        "srv_get_state": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_size_t]),
        "srv_set_state": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_size_t]),
        "srv_stats": (ctypes.c_int, [vp, P(ChSrvStats), ctypes.c_int]),
        "srv_destroy": (ctypes.c_int, [vp]),
        "env_profile_read": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int)]),
        "env_set_policy": (ctypes.c_int, [vp, P(ChPolicy), vp, ctypes.c_size_t]),
        "env_get_action": (ctypes.c_int, [vp, dp]),
        "env_observe": (ctypes.c_int, [vp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != CH_OK:
        raise ChannelError(rc, what)


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------

def ch_default_params() -> ChParams:
    p = ChParams()
    _check(load().ch_default_params(ctypes.byref(p)), "ch_default_params")
    return p


def params(**kw) -> ChParams:
    """Defaults of ``ch_default_params`` overridden by keyword arguments."""
    p = ch_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def ch_strerror(code: int) -> str:
    return load().ch_strerror(code).decode()


def ch_state_bytes(p: ChParams) -> int:
    return int(load().ch_state_bytes(ctypes.byref(p)))


def ch_seed_state(p: ChParams, seed: int, amplitude: float, kmax: int) -> np.ndarray:
    buf = np.zeros(ch_state_bytes(p) // 8)
    _check(load().ch_seed_state(ctypes.byref(p), seed, amplitude, kmax, buf.ctypes.data, buf.nbytes),
           "ch_seed_state")
    return buf


# --------------------------------------------------------------------------
# environment handle
# --------------------------------------------------------------------------

def env_create(p: ChParams) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().env_create(ctypes.byref(p), ctypes.byref(h)), "env_create")
    return h


def env_set_stream(env, stream: int | None):
    _check(load().env_set_stream(env, ctypes.c_void_p(stream or 0)), "env_set_stream")


def env_reset(env, seed: int, amplitude: float = 0.1, kmax: int = 4):
    _check(load().env_reset(env, seed, amplitude, kmax), "env_reset")


def env_step(env, action: np.ndarray | None, obs: np.ndarray, wall_shear: np.ndarray,
             reward: np.ndarray) -> int:
    """Host-buffer step; returns the status (CH_ERR_DIVERGED is returned, not raised)."""
    rc = load().env_step(env, _dptr(action), _dptr(obs), _dptr(wall_shear), _dptr(reward))
    if rc not in (CH_OK, CH_ERR_DIVERGED):
        _check(rc, "env_step")
    return rc


def env_step_device(env, d_action: int | None, d_out: int):
    _check(load().env_step_device(env, ctypes.c_void_p(d_action or 0), ctypes.c_void_p(d_out)),
           "env_step_device")


def env_set_tiles(env, ppc_pre: int, ppc_post: int, post_batched: int):
    _check(load().env_set_tiles(env, ppc_pre, ppc_post, post_batched), "env_set_tiles")


def policy(wz: int = 1, wx: int = 1, hidden: tuple = (), out_tanh: bool = True) -> ChPolicy:
    """Policy descriptor: odd window (wz, wx), up to two hidden widths."""
    pol = ChPolicy()
    pol.wz, pol.wx, pol.n_hidden = wz, wx, len(hidden)
    for i, h in enumerate(hidden[:2]):
        pol.width[i] = h
    pol.out_tanh = 1 if out_tanh else 0
    return pol


def policy_weight_count(pol: ChPolicy) -> int:
    k = 2 * pol.wz * pol.wx
    if pol.n_hidden == 0:
        return k + 1
    h1 = pol.width[0]
    if pol.n_hidden == 1:
        return h1 * k + h1 + h1 + 1
    h2 = pol.width[1]
    return h1 * k + h1 + h2 * h1 + h2 + h2 + 1


def env_set_policy(env, pol: ChPolicy, weights: np.ndarray):
    w = np.ascontiguousarray(weights, dtype=np.float64).ravel()
    _check(load().env_set_policy(env, ctypes.byref(pol), w.ctypes.data, w.size), "env_set_policy")


def env_observe(env, obs: np.ndarray):
    """Sensing plane [B][2][nz][nx] of the current flow into `obs` (float64)."""
    _check(load().env_observe(env, _dptr(obs)), "env_observe")


def env_get_action(env, action: np.ndarray):
    """Copy the last step's wall action [B][nz][nx] into `action` (float64)."""
    _check(load().env_get_action(env, _dptr(action)), "env_get_action")


def env_info(env) -> ChInfo:
    info = ChInfo()
    _check(load().env_info(env, ctypes.byref(info)), "env_info")
    return info


def env_get_state(env, e: int = 0) -> np.ndarray:
    n = env_info(env).state_bytes
    buf = np.zeros(n // 8)
    _check(load().env_get_state(env, e, buf.ctypes.data, buf.nbytes), "env_get_state")
    return buf


def env_set_state(env, e: int, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, dtype=np.float64)
    _check(load().env_set_state(env, e, buf.ctypes.data, buf.nbytes), "env_set_state")


def env_destroy(env):
    _check(load().env_destroy(env), "env_destroy")


def env_profile(env, enable: bool):
    _check(load().env_profile(env, 1 if enable else 0), "env_profile")


def env_profile_read(env, cls: int) -> tuple[float, int]:
    ms = ctypes.c_double()
    n = ctypes.c_int()
    _check(load().env_profile_read(env, cls, ctypes.byref(ms), ctypes.byref(n)), "env_profile_read")
    return ms.value, n.value


def ch_nonlinear(env, d_q: int, d_h: int):
    _check(load().ch_nonlinear(env, ctypes.c_void_p(d_q), ctypes.c_void_p(d_h)), "ch_nonlinear")


def ch_tau_helmholtz(ny: int, M: int, d_lam: int, d_r: int, d_top: int, d_bot: int, d_f: int,
                     stream: int | None = None):
    _check(load().ch_tau_helmholtz(ny, M, ctypes.c_void_p(d_lam), ctypes.c_void_p(d_r),
                                   ctypes.c_void_p(d_top), ctypes.c_void_p(d_bot), ctypes.c_void_p(d_f),
                                   ctypes.c_void_p(stream or 0)), "ch_tau_helmholtz")


# --------------------------------------------------------------------------
# serialised-state layout (see env_get_state in the header)
# --------------------------------------------------------------------------

def unpack_state(buf: np.ndarray, nx: int, ny: int, nz: int) -> dict:
    nxh = nx // 2
    P = nz * nxh
    o = 0
    v = buf[o:o + 2 * ny * P].view(np.complex128).reshape(ny, nz, nxh); o += 2 * ny * P
    g = buf[o:o + 2 * ny * P].view(np.complex128).reshape(ny, nz, nxh); o += 2 * ny * P
    U = buf[o:o + ny]; o += ny
    W = buf[o:o + ny]; o += ny
    vw = buf[o:o + 2 * P].view(np.complex128).reshape(nz, nxh); o += 2 * P
    return {"v": v.copy(), "g": g.copy(), "U": U.copy(), "W": W.copy(), "vw": vw.copy(),
            "t": float(buf[o]), "steps": float(buf[o + 1])}


def pack_state(st: dict, nx: int, ny: int, nz: int) -> np.ndarray:
    nxh = nx // 2
    P = nz * nxh
    parts = [
        np.ascontiguousarray(st["v"], np.complex128).reshape(-1).view(np.float64),
        np.ascontiguousarray(st["g"], np.complex128).reshape(-1).view(np.float64),
        np.asarray(st["U"], np.float64).reshape(ny),
        np.asarray(st["W"], np.float64).reshape(ny),
        np.ascontiguousarray(st.get("vw", np.zeros((nz, nxh))), np.complex128).reshape(-1).view(np.float64),
        np.array([st.get("t", 0.0), st.get("steps", 0.0)]),
    ]
    out = np.concatenate(parts)
    assert out.size == 4 * ny * P + 2 * ny + 2 * P + 2
    return out


def ch_tau_helmholtz_noalloc(ny: int, M: int, d_lam: int, d_r: int, d_top: int, d_bot: int, d_f: int,
                             stream: int | None = None):
    """ch_tau_helmholtz without any device allocation (work vectors in the
    library's static 16 MiB array); for callers that cannot allocate."""
    _check(load().ch_tau_helmholtz_noalloc(ny, M, ctypes.c_void_p(d_lam), ctypes.c_void_p(d_r),
                                           ctypes.c_void_p(d_top), ctypes.c_void_p(d_bot),
                                           ctypes.c_void_p(d_f), ctypes.c_void_p(stream or 0)),
           "ch_tau_helmholtz_noalloc")


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

def srv_create(hbm_budget_bytes: int, slots_per_class: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().srv_create(hbm_budget_bytes, slots_per_class, ctypes.byref(h)), "srv_create")
    return h


def srv_set_linger(srv, linger_us: int):
    _check(load().srv_set_linger(srv, linger_us), "srv_set_linger")


def srv_admit(srv, p: ChParams, seed: int, amplitude: float = 0.1, kmax: int = 4) -> int:
    eid = ctypes.c_int()
    _check(load().srv_admit(srv, ctypes.byref(p), seed, amplitude, kmax, ctypes.byref(eid)), "srv_admit")
    return eid.value


def srv_evict(srv, env_id: int):
    _check(load().srv_evict(srv, env_id), "srv_evict")


def srv_submit(srv, env_id: int, action: np.ndarray | None) -> int:
    rid = ctypes.c_uint64()
    a = None if action is None else np.ascontiguousarray(action, dtype=np.float64)
    _check(load().srv_submit(srv, env_id, _dptr(a), ctypes.byref(rid)), "srv_submit")
    return rid.value


def _result_bufs(obs_shape):
    return (np.zeros(obs_shape), ctypes.c_double(), ctypes.c_double(), ctypes.c_double())


def srv_poll(srv, req_id: int, obs: np.ndarray):
    """(status, wall_shear, reward, latency_us); status CH_PENDING while running."""
    tau, rew, lat = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = load().srv_poll(srv, req_id, _dptr(obs), ctypes.byref(tau), ctypes.byref(rew), ctypes.byref(lat))
    return rc, tau.value, rew.value, lat.value


def srv_wait(srv, req_id: int, timeout_ms: int, obs: np.ndarray):
    """(status, wall_shear, reward, latency_us); CH_ERR_TIMEOUT if still running."""
    tau, rew, lat = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = load().srv_wait(srv, req_id, timeout_ms, _dptr(obs), ctypes.byref(tau), ctypes.byref(rew),
                         ctypes.byref(lat))
    return rc, tau.value, rew.value, lat.value


def srv_submit_many(srv, env_ids, actions: np.ndarray | None) -> np.ndarray:
    """Queue one request per environment of env_ids (actions [n][nz][nx] in
    the same order, or None); returns the request ids."""
    ids = np.ascontiguousarray(env_ids, dtype=np.int32)
    out = np.zeros(len(ids), dtype=np.uint64)
    act = None if actions is None else np.ascontiguousarray(actions, dtype=np.float64)
    _check(load().srv_submit_many(srv, len(ids), ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  None if act is None else _dptr(act), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
           "srv_submit_many")
    return out


def srv_wait_many(srv, req_ids: np.ndarray, timeout_ms: int, obs: np.ndarray):
    """(rc, wall_shear [n], reward [n], status [n]); obs [n][2][nz][nx] is filled."""
    ids = np.ascontiguousarray(req_ids, dtype=np.uint64)
    n = len(ids)
    tau, rew, st = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
    rc = load().srv_wait_many(srv, n, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), timeout_ms, _dptr(obs), _dptr(tau),
                              _dptr(rew), st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return rc, tau, rew, st


def srv_get_state(srv, env_id: int, nbytes: int) -> np.ndarray:
    buf = np.zeros(nbytes // 8)
    _check(load().srv_get_state(srv, env_id, buf.ctypes.data, buf.nbytes), "srv_get_state")
    return buf


def srv_set_state(srv, env_id: int, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, dtype=np.float64)
    _check(load().srv_set_state(srv, env_id, buf.ctypes.data, buf.nbytes), "srv_set_state")


def srv_stats(srv, reset: bool = False) -> ChSrvStats:
    st = ChSrvStats()
    _check(load().srv_stats(srv, ctypes.byref(st), 1 if reset else 0), "srv_stats")
    return st


def srv_destroy(srv):
    _check(load().srv_destroy(srv), "srv_destroy")
