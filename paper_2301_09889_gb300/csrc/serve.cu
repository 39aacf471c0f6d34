// Serving layer: continuous batching of environment steps from many actors.
//
// Environments are grouped into classes by their parameters (grid, box,
// Reynolds numbers, time step, control).  Each class owns one batched handle
// with a fixed number of slots and its own CUDA stream.  A worker thread runs
// ticks: for every class with a free tick it gathers the oldest pending
// request of each environment not already in a running tick, launches one
// masked batched step for exactly those slots, and moves on to the next
// class, so ticks of different classes overlap on the device.  A class keeps
// up to two ticks in flight, the second queued behind the first on its
// stream, so the GPU does not wait for the host between them.  A new
// environment is admitted into a free slot of its class; a new class is
// created only if its device footprint fits the HBM budget.
//
// Ticks of a large class fill every SM; blocks of a small class launched
// meanwhile would wait for them.  Each class's stream therefore gets a CUDA
// priority by the cost of one of its env-steps (shortest job first): the
// block scheduler dispatches pending blocks of a cheaper class before the
// remaining blocks of a more expensive one, so small environments keep their
// own latency next to large ones.
//
// A slot's result does not depend on which other slots are active (no
// cross-slot arithmetic, the launch shape depends on the class capacity
// only), so an environment steps identically alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/channel_dns.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  int env_id;
  std::vector<double> action;
  Clock::time_point submit;
  Clock::time_point done_at;
  int state = 0;  // 0 queued, 1 running, 2 done
  int status = CH_OK;
  std::vector<double> obs;
  double tau = 0.0, reward = 0.0;
};

// Host side of one tick.  Its copies read the actions and the mask and write
// the outputs when they execute, so a class alternates two sets: the next
// tick is gathered and enqueued while the previous one still runs.
struct Tick {
  double* h_act = nullptr;        // pinned [slots][nz][nx]
  double* h_out = nullptr;        // pinned [slots][out_stride]
  int* h_active = nullptr;        // pinned [slots]
  cudaEvent_t ev = nullptr;
  bool busy = false;
  std::vector<uint64_t> running;  // request per slot in this tick (0 none)
};

struct Class {
  ch_params_t key;  // parameters with batch = 0
  ch_env_t* env = nullptr;
  int slots = 0;
  int nx = 0, nz = 0;
  size_t out_stride = 0;
  size_t footprint = 0;
  std::vector<int> slot_env;  // env id per slot, -1 free
  int* d_active = nullptr;    // device mask, rewritten by each tick in stream order
  cudaStream_t stream = nullptr;  // prioritised stream the class's ticks run on
  Tick tick[2];
  int next_tick = 0;            // the set the class's next tick uses
  std::vector<char> in_flight;  // slot has a request in a tick not yet completed
  bool stuck = false;   // its stream did not drain after a failed enqueue: no further ticks
  bool busy() const { return tick[0].busy || tick[1].busy; }
};

struct Env {
  int cls;
  int slot;
  std::deque<uint64_t> queue;
};

bool same_key(const ch_params_t& a, const ch_params_t& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

// Stream priority of a class: one level lower for every factor 4 in grid
// points x solver steps per env-step above the 16x65x16 minimal channel.
int class_priority(const ch_params_t& p) {
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
  double cost = (double)p.nx * p.ny * p.nz * std::max(1, p.steps_per_action) / (16.0 * 65.0 * 16.0);
  int rank = 0;
  while (cost >= 4.0 && greatest + rank < least) {
    cost /= 4.0;
    ++rank;
  }
  return greatest + rank;
}

}  // namespace

struct ch_server {
  std::mutex mu;
  std::condition_variable cv_work;  // new requests / admissions
  std::condition_variable cv_done;  // completed requests / idle classes
  std::thread worker;
  bool stop = false;
  size_t budget = 0, used = 0;
  int slots_per_class = 0;
  // bounded batching window: a class with some but not all of its
  // environments pending waits up to this long after its oldest pending
  // request before it launches (0: launch with whatever is pending)
  std::chrono::microseconds linger{0};
  std::vector<std::unique_ptr<Class>> classes;
  std::unordered_map<int, Env> envs;
  std::map<uint64_t, Request> reqs;
  int next_env = 1;
  uint64_t next_req = 1;
  // submit-to-completion latencies of the last kLatencyWindow completed
  // requests since creation or the last srv_stats reset (a ring buffer)
  static constexpr size_t kLatencyWindow = (size_t)1 << 20;
  std::vector<double> latencies_us;
  size_t latency_next = 0;
  void record_latency(double us) {
    if (latencies_us.size() < kLatencyWindow) {
      latencies_us.push_back(us);
    } else {
      latencies_us[latency_next] = us;
      latency_next = (latency_next + 1) % kLatencyWindow;
    }
  }
  Clock::time_point t0 = Clock::now();
  uint64_t completed = 0;
  int worker_error = CH_OK;
  int device = 0;

  void run();
  int make_class(const ch_params_t& key, int* cls);
  void free_class(int c);
};

namespace {

ch_params_t key_of(const ch_params_t& p) {
  ch_params_t k;
  std::memset(&k, 0, sizeof(k));
  k.nx = p.nx; k.ny = p.ny; k.nz = p.nz; k.lx = p.lx; k.lz = p.lz;
  k.re_tau = p.re_tau; k.re_bulk = p.re_bulk; k.dt = p.dt; k.steps_per_action = p.steps_per_action;
  k.y_sense_plus = p.y_sense_plus; k.top_bc = p.top_bc; k.precision = p.precision; k.control = p.control;
  k.alpha = p.alpha; k.tau_ref = p.tau_ref; k.batch = 0; k.autotune = p.autotune;
  return k;
}

}  // namespace

int ch_server::make_class(const ch_params_t& key, int* cls) {
  ch_params_t p = key;
  p.batch = slots_per_class;
  const size_t fp = chdns::env_footprint(&p);
  if (used + fp > budget) return CH_ERR_BUDGET;
  std::unique_ptr<Class> c(new Class());
  c->key = key;
  c->slots = slots_per_class;
  c->nx = p.nx;
  c->nz = p.nz;
  int rc = env_create(&p, &c->env);
  if (rc != CH_OK) return rc;
  if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, class_priority(p)) != cudaSuccess) {
    env_destroy(c->env);
    return CH_ERR_CUDA;
  }
  if ((rc = env_set_stream(c->env, c->stream)) != CH_OK) {
    env_destroy(c->env);
    cudaStreamDestroy(c->stream);
    return rc;
  }
  c->out_stride = chdns::env_out_stride(c->env);
  c->footprint = fp;
  c->slot_env.assign(c->slots, -1);
  c->in_flight.assign(c->slots, 0);
  const size_t S = c->slots;
  bool ok = cudaMalloc(&c->d_active, S * sizeof(int)) == cudaSuccess;
  for (Tick& t : c->tick) {
    t.running.assign(c->slots, 0);
    ok = ok && cudaMallocHost(&t.h_act, S * p.nz * p.nx * sizeof(double)) == cudaSuccess &&
         cudaMallocHost(&t.h_out, S * c->out_stride * sizeof(double)) == cudaSuccess &&
         cudaMallocHost(&t.h_active, S * sizeof(int)) == cudaSuccess &&
         cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) std::memset(t.h_act, 0, S * p.nz * p.nx * sizeof(double));
  }
  if (!ok) {
    for (Tick& t : c->tick) {
      if (t.h_act) cudaFreeHost(t.h_act);
      if (t.h_out) cudaFreeHost(t.h_out);
      if (t.h_active) cudaFreeHost(t.h_active);
      if (t.ev) cudaEventDestroy(t.ev);
    }
    if (c->d_active) cudaFree(c->d_active);
    env_destroy(c->env);
    cudaStreamDestroy(c->stream);
    return CH_ERR_OOM;
  }
  used += fp;
  for (size_t i = 0; i < classes.size(); ++i)
    if (!classes[i]) {
      classes[i] = std::move(c);
      *cls = (int)i;
      return CH_OK;
    }
  classes.push_back(std::move(c));
  *cls = (int)classes.size() - 1;
  return CH_OK;
}

void ch_server::free_class(int ci) {
  Class* c = classes[ci].get();
  if (!c) return;
  env_destroy(c->env);  // synchronises the class stream first
  cudaStreamDestroy(c->stream);
  for (Tick& t : c->tick) {
    cudaFreeHost(t.h_act);
    cudaFreeHost(t.h_out);
    cudaFreeHost(t.h_active);
    cudaEventDestroy(t.ev);
  }
  cudaFree(c->d_active);
  used -= c->footprint;
  classes[ci].reset();
}

void ch_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    bool launched = false, any_busy = false;
    Clock::time_point wake = Clock::time_point::max();  // earliest end of a batching window
    // launch a tick on every class with a free tick set and pending requests
    // of environments not already in a running tick
    for (size_t ci = 0; ci < classes.size(); ++ci) {
      Class* c = classes[ci].get();
      if (!c || c->stuck) continue;
      Tick& T = c->tick[c->next_tick];
      if (T.busy) continue;
      int nenv = 0, nready = 0;
      Clock::time_point oldest = Clock::time_point::max();
      for (int sl = 0; sl < c->slots; ++sl) {
        const int eid = c->slot_env[sl];
        if (eid < 0 || c->in_flight[sl]) continue;
        ++nenv;
        const Env& e = envs[eid];
        if (e.queue.empty()) continue;
        ++nready;
        oldest = std::min(oldest, reqs[e.queue.front()].submit);
      }
      if (nready == 0) continue;
      // bounded batching window: hold the tick while some eligible
      // environments have no request yet and the oldest pending one is
      // younger than the window
      if (linger.count() > 0 && nready < nenv && Clock::now() < oldest + linger) {
        wake = std::min(wake, oldest + linger);
        continue;
      }
      const size_t plane = (size_t)c->nz * c->nx;
      for (int sl = 0; sl < c->slots; ++sl) {
        T.h_active[sl] = 0;
        T.running[sl] = 0;
        const int eid = c->slot_env[sl];
        if (eid < 0 || c->in_flight[sl]) continue;
        Env& e = envs[eid];
        if (e.queue.empty()) continue;
        Request& r = reqs[e.queue.front()];
        e.queue.pop_front();
        r.state = 1;
        T.running[sl] = r.id;
        T.h_active[sl] = 1;
        c->in_flight[sl] = 1;
        if (!r.action.empty()) std::memcpy(T.h_act + sl * plane, r.action.data(), plane * sizeof(double));
      }
      T.busy = true;
      c->next_tick ^= 1;
      launched = true;
      lk.unlock();
      // the copies and the step run in stream order after any earlier tick
      // of the class, so the device mask, action and output buffers are
      // rewritten only once that tick is done with them
      cudaStream_t st = chdns::env_stream(c->env);
      int rc = CH_OK;
      if (cudaMemcpyAsync(c->d_active, T.h_active, c->slots * sizeof(int), cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(chdns::env_dact(c->env), T.h_act, c->slots * plane * sizeof(double),
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = CH_ERR_CUDA;
      if (rc == CH_OK) rc = chdns::step_masked(c->env, chdns::env_dact(c->env), c->d_active, T.h_active);
      if (rc == CH_OK && cudaMemcpyAsync(T.h_out, chdns::env_dout(c->env), c->slots * c->out_stride * sizeof(double),
                                         cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = CH_ERR_CUDA;
      if (rc == CH_OK && cudaEventRecord(T.ev, st) != cudaSuccess) rc = CH_ERR_CUDA;
      bool drained = true;
      if (rc != CH_OK) {
        // copies and kernels queued before the failure may still read the
        // pinned action and mask buffers: wait (bounded, about 5 s) for the
        // class stream before a later tick may rewrite them
        drained = false;
        for (int it = 0; it < 100000 && !drained; ++it) {
          if (cudaStreamQuery(st) != cudaErrorNotReady) drained = true;
          else std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
      }
      lk.lock();
      if (rc != CH_OK) {
        worker_error = drained ? rc : CH_ERR_TIMEOUT;
        for (int sl = 0; sl < c->slots; ++sl)
          if (T.running[sl]) {
            Request& r = reqs[T.running[sl]];
            r.state = 2;
            r.status = rc;
            r.done_at = Clock::now();
            T.running[sl] = 0;
            c->in_flight[sl] = 0;
          }
        T.busy = !drained;
        c->stuck = !drained;
        cv_done.notify_all();
      }
    }
    // complete finished ticks, oldest first (a class's ticks finish in order)
    for (size_t ci = 0; ci < classes.size(); ++ci) {
      Class* c = classes[ci].get();
      if (!c || c->stuck) continue;
      for (int k = 0; k < 2; ++k) {
        Tick& T = c->tick[c->next_tick ^ (k == 0 ? 0 : 1)];
        if (!T.busy) continue;
        const cudaError_t q = cudaEventQuery(T.ev);
        if (q == cudaErrorNotReady) {
          any_busy = true;
          continue;
        }
        const auto now = Clock::now();
        const size_t plane = (size_t)c->nz * c->nx;
        for (int sl = 0; sl < c->slots; ++sl) {
          if (!T.running[sl]) continue;
          Request& r = reqs[T.running[sl]];
          const double* o = T.h_out + sl * c->out_stride;
          r.obs.assign(o, o + 2 * plane);
          r.tau = o[2 * plane];
          r.reward = o[2 * plane + 1];
          r.status = (q != cudaSuccess) ? CH_ERR_CUDA : (std::isfinite(r.tau) ? CH_OK : CH_ERR_DIVERGED);
          r.state = 2;
          r.done_at = now;
          record_latency(std::chrono::duration<double, std::micro>(now - r.submit).count());
          ++completed;
          T.running[sl] = 0;
          c->in_flight[sl] = 0;
        }
        T.busy = false;
        cv_done.notify_all();
      }
    }
    if (!launched && !any_busy) {
      // new requests wake the worker; so does the end of a batching window
      if (wake != Clock::time_point::max()) cv_work.wait_until(lk, wake);
      else cv_work.wait_for(lk, std::chrono::milliseconds(50));
    } else if (!launched && any_busy) {
      // ticks in flight: poll their events again shortly
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

namespace {

// wait (bounded) until class `ci` has no tick in flight
bool wait_idle(ch_server* s, std::unique_lock<std::mutex>& lk, int ci) {
  return s->cv_done.wait_for(lk, std::chrono::seconds(30), [&] {
    return !s->classes[ci] || !s->classes[ci]->busy();
  });
}

}  // namespace

extern "C" {

int srv_create(size_t hbm_budget_bytes, int slots_per_class, ch_server_t** out) {
  if (!out || slots_per_class < 1 || hbm_budget_bytes == 0) return CH_ERR_ARG;
  ch_server* s = new (std::nothrow) ch_server();
  if (!s) return CH_ERR_OOM;
  s->budget = hbm_budget_bytes;
  s->slots_per_class = slots_per_class;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return CH_ERR_CUDA;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return CH_OK;
}

int srv_set_linger(ch_server_t* s, int linger_us) {
  if (!s || linger_us < 0 || linger_us > 1000000) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  s->linger = std::chrono::microseconds(linger_us);
  s->cv_work.notify_all();
  return CH_OK;
}

int srv_admit(ch_server_t* s, const ch_params_t* p, uint64_t seed, double amplitude, int kmax, int* env_id) {
  if (!s || !p || !env_id) return CH_ERR_ARG;
  if (p->control == 2) return CH_ERR_UNSUPPORTED;  // no policy can be set through the server
  std::unique_lock<std::mutex> lk(s->mu);
  const ch_params_t key = key_of(*p);
  int ci = -1, slot = -1;
  for (size_t i = 0; i < s->classes.size() && slot < 0; ++i) {
    Class* c = s->classes[i].get();
    if (!c || !same_key(c->key, key)) continue;
    for (int sl = 0; sl < c->slots; ++sl)
      if (c->slot_env[sl] < 0) {
        ci = (int)i;
        slot = sl;
        break;
      }
  }
  if (slot < 0) {
    const int rc = s->make_class(key, &ci);
    if (rc != CH_OK) return rc;
    slot = 0;
  }
  if (!wait_idle(s, lk, ci)) return CH_ERR_TIMEOUT;
  Class* c = s->classes[ci].get();
  const int rc = chdns::env_slot_seed(c->env, slot, seed, amplitude, kmax);
  if (rc != CH_OK) return rc;
  const int id = s->next_env++;
  c->slot_env[slot] = id;
  s->envs[id] = Env{ci, slot, {}};
  *env_id = id;
  return CH_OK;
}

int srv_set_state(ch_server_t* s, int env_id, const void* buf, size_t nbytes) {
  if (!s || !buf) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->envs.find(env_id);
  if (it == s->envs.end()) return CH_ERR_ARG;
  if (!it->second.queue.empty()) return CH_ERR_STATE;
  if (!wait_idle(s, lk, it->second.cls)) return CH_ERR_TIMEOUT;
  return env_set_state(s->classes[it->second.cls]->env, it->second.slot, buf, nbytes);
}

int srv_get_state(ch_server_t* s, int env_id, void* buf, size_t nbytes) {
  if (!s || !buf) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->envs.find(env_id);
  if (it == s->envs.end()) return CH_ERR_ARG;
  if (!wait_idle(s, lk, it->second.cls)) return CH_ERR_TIMEOUT;
  return env_get_state(s->classes[it->second.cls]->env, it->second.slot, buf, nbytes);
}

int srv_evict(ch_server_t* s, int env_id) {
  if (!s) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->envs.find(env_id);
  if (it == s->envs.end()) return CH_ERR_ARG;
  const int ci = it->second.cls;
  if (!wait_idle(s, lk, ci)) return CH_ERR_TIMEOUT;
  for (uint64_t rid : it->second.queue) {
    Request& r = s->reqs[rid];
    r.state = 2;
    r.status = CH_ERR_STATE;
    r.done_at = Clock::now();
  }
  Class* c = s->classes[ci].get();
  c->slot_env[it->second.slot] = -1;
  s->envs.erase(it);
  if (std::all_of(c->slot_env.begin(), c->slot_env.end(), [](int e) { return e < 0; })) s->free_class(ci);
  s->cv_done.notify_all();
  return CH_OK;
}

int srv_submit(ch_server_t* s, int env_id, const double* action, uint64_t* req_id) {
  if (!s || !req_id) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->envs.find(env_id);
  if (it == s->envs.end()) return CH_ERR_ARG;
  Class* c = s->classes[it->second.cls].get();
  Request r;
  r.id = s->next_req++;
  r.env_id = env_id;
  r.submit = Clock::now();
  if (c->key.control == 0) {
    if (!action) return CH_ERR_ARG;
    const size_t n = (size_t)c->nz * c->nx;
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(action[i])) return CH_ERR_ARG;  // poisoned action
    r.action.assign(action, action + n);
  }
  it->second.queue.push_back(r.id);
  *req_id = r.id;
  s->reqs.emplace(r.id, std::move(r));
  s->cv_work.notify_one();
  return CH_OK;
}

int srv_submit_many(ch_server_t* s, int n, const int* env_ids, const double* actions, uint64_t* req_ids) {
  if (!s || n < 0 || (n > 0 && (!env_ids || !req_ids))) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  // check every request first: a refused batch queues nothing
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    auto it = s->envs.find(env_ids[i]);
    if (it == s->envs.end()) return CH_ERR_ARG;
    const Class* c = s->classes[it->second.cls].get();
    if (c->key.control != 0) continue;
    if (!actions) return CH_ERR_ARG;
    const size_t m = (size_t)c->nz * c->nx;
    for (size_t k = 0; k < m; ++k)
      if (!std::isfinite(actions[off + k])) return CH_ERR_ARG;  // poisoned action
    off += m;
  }
  off = 0;
  const auto now = Clock::now();
  for (int i = 0; i < n; ++i) {
    Env& e = s->envs[env_ids[i]];
    const Class* c = s->classes[e.cls].get();
    Request r;
    r.id = s->next_req++;
    r.env_id = env_ids[i];
    r.submit = now;
    if (c->key.control == 0) {
      const size_t m = (size_t)c->nz * c->nx;
      r.action.assign(actions + off, actions + off + m);
      off += m;
    }
    e.queue.push_back(r.id);
    req_ids[i] = r.id;
    s->reqs.emplace(r.id, std::move(r));
  }
  if (n > 0) s->cv_work.notify_one();
  return CH_OK;
}

static int take_result(ch_server* s, std::map<uint64_t, Request>::iterator it, double* obs, double* wall_shear,
                       double* reward, double* latency_us) {
  Request& r = it->second;
  if (obs && !r.obs.empty()) std::memcpy(obs, r.obs.data(), r.obs.size() * sizeof(double));
  if (wall_shear) *wall_shear = r.tau;
  if (reward) *reward = r.reward;
  if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r.done_at - r.submit).count();
  const int status = r.status;
  s->reqs.erase(it);
  return status;
}

int srv_poll(ch_server_t* s, uint64_t req_id, double* obs, double* wall_shear, double* reward, double* latency_us) {
  if (!s) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return CH_ERR_ARG;
  if (it->second.state != 2) return CH_PENDING;
  return take_result(s, it, obs, wall_shear, reward, latency_us);
}

int srv_wait(ch_server_t* s, uint64_t req_id, int timeout_ms, double* obs, double* wall_shear, double* reward,
             double* latency_us) {
  if (!s || timeout_ms < 0) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return CH_ERR_ARG;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    auto jt = s->reqs.find(req_id);
    return jt == s->reqs.end() || jt->second.state == 2;
  });
  if (!ok) return CH_ERR_TIMEOUT;
  it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return CH_ERR_ARG;
  return take_result(s, it, obs, wall_shear, reward, latency_us);
}

int srv_wait_many(ch_server_t* s, int n, const uint64_t* req_ids, int timeout_ms, double* obs, double* wall_shear,
                  double* reward, int* status) {
  if (!s || n < 0 || timeout_ms < 0 || (n > 0 && (!req_ids || !status))) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  for (int i = 0; i < n; ++i)
    if (s->reqs.find(req_ids[i]) == s->reqs.end()) return CH_ERR_ARG;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    for (int i = 0; i < n; ++i) {
      auto jt = s->reqs.find(req_ids[i]);
      if (jt != s->reqs.end() && jt->second.state != 2) return false;
    }
    return true;
  });
  if (!ok) return CH_ERR_TIMEOUT;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    auto it = s->reqs.find(req_ids[i]);
    if (it == s->reqs.end()) {  // taken meanwhile by another caller
      status[i] = CH_ERR_ARG;
      continue;
    }
    const size_t m = it->second.obs.size();
    status[i] = take_result(s, it, obs ? obs + off : nullptr, wall_shear ? wall_shear + i : nullptr,
                            reward ? reward + i : nullptr, nullptr);
    off += m;
  }
  return CH_OK;
}

int srv_stats(ch_server_t* s, ch_srv_stats_t* st, int reset) {
  if (!s || !st) return CH_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  std::vector<double> l = s->latencies_us;
  std::sort(l.begin(), l.end());
  st->completed = s->completed;
  if (!l.empty()) {
    st->p50_us = l[l.size() / 2];
    st->p99_us = l[std::min(l.size() - 1, (size_t)(0.99 * l.size()))];
    st->max_us = l.back();
    double sum = 0.0;
    for (double v : l) sum += v;
    st->mean_us = sum / l.size();
  }
  const double secs = std::chrono::duration<double>(Clock::now() - s->t0).count();
  st->env_steps_per_s = secs > 0 ? s->completed / secs : 0.0;
  for (auto& c : s->classes) st->classes += c ? 1 : 0;
  st->envs = (int)s->envs.size();
  for (auto& kv : s->envs) st->pending += (int)kv.second.queue.size();
  st->hbm_used = s->used;
  st->hbm_budget = s->budget;
  st->worker_status = s->worker_error;
  if (reset) {
    s->latencies_us.clear();
    s->latency_next = 0;
    s->completed = 0;
    s->t0 = Clock::now();
  }
  return CH_OK;
}

int srv_destroy(ch_server_t* s) {
  if (!s) return CH_ERR_ARG;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  s->worker.join();
  for (size_t i = 0; i < s->classes.size(); ++i) {
    if (s->classes[i]) {
      for (Tick& t : s->classes[i]->tick) cudaEventSynchronize(t.ev);
      s->free_class((int)i);
    }
  }
  delete s;
  return CH_OK;
}

}  // extern "C"
