"""Serving: continuous batching of environment steps from many actors.

* an environment steps identically alone and in a mix with other
  environments of its class and of another class, submitted concurrently
  from several actor threads;
* admission is refused beyond the HBM budget and succeeds after eviction;
* queued requests of an evicted environment complete with CH_ERR_STATE;
* bounded waits time out instead of hanging; poisoned actions are refused;
* latency percentiles and throughput are reported.
"""

import threading

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

MINIMAL = dict(nx=16, ny=65, nz=16, lx=2.67, lz=0.8, re_tau=180.0, re_bulk=2800.0, dt=0.005)
SMALL = dict(nx=16, ny=33, nz=16, lx=3.0, lz=1.2, re_tau=180.0, re_bulk=2800.0, dt=0.004, precision=1)
GB = 1 << 30


def _actions(seed, n, nx=16, nz=16):
    return [si.wall_action(nx, nz, seed * 1000 + t, 0.05 * 180 / 2800) for t in range(n)]


def _drive(native, srv, eid, acts, nz=16, nx=16):
    outs = []
    for a in acts:
        rid = native.srv_submit(srv, eid, a)
        obs = np.zeros((2, nz, nx))
        rc, tau, rew, lat = native.srv_wait(srv, rid, 60000, obs)
        assert rc == native.CH_OK, rc
        outs.append((obs, tau, rew))
    return outs


def test_alone_equals_in_mix(native_gpu):
    native = native_gpu
    acts = _actions(3, 6)
    # alone
    srv = native.srv_create(8 * GB, 4)
    try:
        eid = native.srv_admit(srv, native.params(**MINIMAL), seed=5, amplitude=0.2, kmax=99)
        alone = _drive(native, srv, eid, acts)
        nbytes = native.ch_state_bytes(native.params(**MINIMAL))
        st_alone = native.srv_get_state(srv, eid, nbytes)
    finally:
        native.srv_destroy(srv)
    # in a mix: two neighbours in the same class, two environments of another class,
    # all driven concurrently by actor threads
    srv = native.srv_create(8 * GB, 4)
    try:
        eid = native.srv_admit(srv, native.params(**MINIMAL), seed=5, amplitude=0.2, kmax=99)
        others = [native.srv_admit(srv, native.params(**MINIMAL), seed=50 + k, amplitude=0.3, kmax=99)
                  for k in range(2)]
        others += [native.srv_admit(srv, native.params(**SMALL), seed=70 + k, amplitude=0.2, kmax=99)
                   for k in range(2)]
        errors = []

        def actor(e, seed):
            try:
                _drive(native, srv, e, _actions(seed, 8))
            except Exception as exc:  # noqa: BLE001
                errors.append(exc)

        threads = [threading.Thread(target=actor, args=(e, 90 + i)) for i, e in enumerate(others)]
        for t in threads:
            t.start()
        mixed = _drive(native, srv, eid, acts)
        for t in threads:
            t.join()
        assert not errors, errors
        st_mixed = native.srv_get_state(srv, eid, nbytes)
        stats = native.srv_stats(srv)
        assert stats.completed == 6 + 4 * 8 and stats.classes == 2 and stats.envs == 5
        assert stats.p99_us >= stats.p50_us > 0
    finally:
        native.srv_destroy(srv)
    for (o1, t1, r1), (o2, t2, r2) in zip(alone, mixed):
        assert np.array_equal(o1, o2) and t1 == t2 and r1 == r2
    assert np.array_equal(st_alone, st_mixed)


def test_served_matches_env_api(native_gpu):
    """A served environment equals the same environment stepped through env_step
    on a handle of the same capacity."""
    native = native_gpu
    acts = _actions(4, 3)
    srv = native.srv_create(8 * GB, 2)
    try:
        eid = native.srv_admit(srv, native.params(**MINIMAL), seed=9, amplitude=0.2, kmax=99)
        served = _drive(native, srv, eid, acts)
    finally:
        native.srv_destroy(srv)
    env = native.env_create(native.params(**MINIMAL, batch=2))
    try:
        buf = native.ch_seed_state(native.params(**MINIMAL), 9, 0.2, 99)
        native.env_set_state(env, 0, buf)
        native.env_set_state(env, 1, buf)
        for a, (o_s, t_s, r_s) in zip(acts, served):
            obs, tau, rew = np.zeros((2, 2, 16, 16)), np.zeros(2), np.zeros(2)
            native.env_step(env, np.ascontiguousarray(np.stack([a, a])), obs, tau, rew)
            assert np.array_equal(obs[0], o_s) and tau[0] == t_s and rew[0] == r_s
    finally:
        native.env_destroy(env)


def test_admission_by_hbm_budget(native_gpu):
    native = native_gpu
    p1 = native.params(**MINIMAL)
    srv = native.srv_create(8 * GB, 2)
    try:
        e1 = native.srv_admit(srv, p1, seed=1)
        used = native.srv_stats(srv).hbm_used
    finally:
        native.srv_destroy(srv)
    # the admission estimate bounds what the class handle really holds
    env = native.env_create(native.params(**MINIMAL, batch=2))
    try:
        real = native.env_info(env).device_bytes
    finally:
        native.env_destroy(env)
    assert real <= used <= real + (8 << 20), (real, used)
    # a budget that holds one class but not two
    srv = native.srv_create(used + used // 2, 2)
    try:
        e1 = native.srv_admit(srv, p1, seed=1)
        e2 = native.srv_admit(srv, p1, seed=2)               # same class: a free slot
        with pytest.raises(native.ChannelError) as exc:
            native.srv_admit(srv, p1, seed=3)                # class full, a second handle does not fit
        assert exc.value.code == native.CH_ERR_BUDGET
        with pytest.raises(native.ChannelError) as exc:
            native.srv_admit(srv, native.params(**SMALL), seed=4)
        assert exc.value.code == native.CH_ERR_BUDGET
        native.srv_evict(srv, e1)
        native.srv_evict(srv, e2)                             # class released
        assert native.srv_stats(srv).hbm_used == 0
        e3 = native.srv_admit(srv, native.params(**SMALL), seed=4)
        assert native.srv_stats(srv).classes == 1
        out = _drive(native, srv, e3, _actions(5, 1))
        assert np.isfinite(out[0][1])
    finally:
        native.srv_destroy(srv)


def test_faults_are_reported_not_hung(native_gpu):
    native = native_gpu
    srv = native.srv_create(8 * GB, 2)
    try:
        eid = native.srv_admit(srv, native.params(**MINIMAL), seed=1)
        bad = np.full((16, 16), np.nan)
        with pytest.raises(native.ChannelError) as exc:
            native.srv_submit(srv, eid, bad)                  # poisoned action refused
        assert exc.value.code == native.CH_ERR_ARG
        rids = [native.srv_submit(srv, eid, a) for a in _actions(6, 40)]
        obs = np.zeros((2, 16, 16))
        rc, *_ = native.srv_wait(srv, rids[-1], 0, obs)       # bounded wait runs out
        assert rc in (native.CH_ERR_TIMEOUT, native.CH_OK)
        rc, *_ = native.srv_wait(srv, rids[0], 60000, obs)
        assert rc == native.CH_OK
        native.srv_evict(srv, eid)                           # the rest of the queue is cancelled
        states = [native.srv_wait(srv, r, 60000, obs)[0] for r in rids[1:]]
        assert all(s in (native.CH_OK, native.CH_ERR_STATE) for s in states)
        assert native.CH_ERR_STATE in states or len(states) == 0
        with pytest.raises(native.ChannelError):
            native.srv_submit(srv, eid, _actions(7, 1)[0])   # evicted id
    finally:
        native.srv_destroy(srv)


def test_batching_window_fills_ticks_and_keeps_results(native_gpu):
    """With a batching window the server holds a class's tick until all of its
    environments have a request (or the window ends): the first request of
    the first of four staggered actors waits for the last one, and every
    result is the same as without a window.  Out-of-range windows are
    refused."""
    import time
    native = native_gpu
    acts = [_actions(20 + k, 4) for k in range(4)]

    def run(linger_us):
        srv = native.srv_create(8 * GB, 4)
        try:
            for bad in (-1, 2_000_000):
                with pytest.raises(native.ChannelError):
                    native.srv_set_linger(srv, bad)
            native.srv_set_linger(srv, linger_us)
            eids = [native.srv_admit(srv, native.params(**MINIMAL), seed=90 + k, amplitude=0.2, kmax=99)
                    for k in range(4)]
            outs, lats = [None] * 4, [None] * 4

            def actor(k):
                time.sleep(0.05 * k)
                res, lat = [], []
                for a in acts[k]:
                    rid = native.srv_submit(srv, eids[k], a)
                    obs = np.zeros((2, 16, 16))
                    rc, tau, rew, us = native.srv_wait(srv, rid, 60000, obs)
                    assert rc == native.CH_OK, rc
                    res.append((obs, tau, rew))
                    lat.append(us)
                outs[k], lats[k] = res, lat

            threads = [threading.Thread(target=actor, args=(k,)) for k in range(4)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            return outs, lats, native.srv_stats(srv)
        finally:
            native.srv_destroy(srv)

    plain, lat0, _ = run(0)
    held, lat1, st = run(500_000)
    assert st.completed == 16 and st.worker_status == native.CH_OK
    for a, b in zip(plain, held):
        for (oa, ta, ra), (ob, tb, rb) in zip(a, b):
            assert np.array_equal(oa, ob) and ta == tb and ra == rb
    # the last actor starts 150 ms after the first: held, the first request
    # waits for it; without a window it runs at once
    assert lat1[0][0] > 100_000, lat1[0][0]
    assert lat0[0][0] < 100_000, lat0[0][0]


def test_submit_many_and_wait_many(native_gpu):
    """Requests queued and collected in batches give the same results as one
    at a time; a batch with an unknown environment or a poisoned action is
    refused whole, queueing nothing."""
    native = native_gpu
    acts = [_actions(40 + k, 3) for k in range(3)]

    def one_at_a_time():
        srv = native.srv_create(8 * GB, 4)
        try:
            eids = [native.srv_admit(srv, native.params(**MINIMAL), seed=95 + k, amplitude=0.2, kmax=99)
                    for k in range(3)]
            return [_drive(native, srv, eids[k], acts[k]) for k in range(3)]
        finally:
            native.srv_destroy(srv)

    ref = one_at_a_time()
    srv = native.srv_create(8 * GB, 4)
    try:
        eids = [native.srv_admit(srv, native.params(**MINIMAL), seed=95 + k, amplitude=0.2, kmax=99)
                for k in range(3)]
        bad = np.stack([acts[k][0] for k in range(3)])
        bad[1, 2, 3] = np.nan
        with pytest.raises(native.ChannelError):
            native.srv_submit_many(srv, eids, bad)
        with pytest.raises(native.ChannelError):
            native.srv_submit_many(srv, [eids[0], 9999], np.stack([acts[0][0], acts[1][0]]))
        assert native.srv_stats(srv).pending == 0
        obs = np.zeros((3, 2, 16, 16))
        for t in range(3):
            rids = native.srv_submit_many(srv, eids, np.stack([acts[k][t] for k in range(3)]))
            rc, tau, rew, st = native.srv_wait_many(srv, rids, 60000, obs)
            assert rc == native.CH_OK and (st == native.CH_OK).all()
            for k in range(3):
                o, ta, ra = ref[k][t]
                assert np.array_equal(obs[k], o) and tau[k] == ta and rew[k] == ra
    finally:
        native.srv_destroy(srv)
