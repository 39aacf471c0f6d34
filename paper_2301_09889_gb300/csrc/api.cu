// Host side of the C ABI declared in include/channel_dns.h: parameter checks,
// per-grid tables (tau factorisations, influence-matrix solutions, twiddles),
// the environment step driver and state serialisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/channel_dns.h"
#include "common.cuh"
#include "internal.h"

using namespace chdns;

namespace {

// Low-storage RK3 (third-order Runge-Kutta for the nonlinear term,
// Crank-Nicolson for the viscous term; paper Sec. 3.1).
const double kGamma[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
const double kZeta[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
const double kCEnd[3] = {8.0 / 15.0, 2.0 / 3.0, 1.0};
inline double rk_alpha(int k) { return 0.5 * (kGamma[k] + kZeta[k]); }
inline double rk_beta(int k) { return 0.5 * (kGamma[k] + kZeta[k]); }

// ---- host tau factorisation (same recurrences as the device solver) ------
inline double cA(int n) { return (n == 2 ? 2.0 : 1.0) / (4.0 * n * (n - 1)); }
inline double cB(int n, int N) { return n <= N - 2 ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0; }
inline double cC(int n, int N) { return n + 2 <= N - 2 ? 1.0 / (4.0 * n * (n + 1)) : 0.0; }

struct Factor {
  std::vector<double> e, h, b, Q;
  double isq = 0.0;
};

Factor host_factor(int N, int sig, double lam) {
  const int M = (N - sig) / 2 + 1;
  Factor F;
  F.e.assign(M, 0.0);
  F.h.assign(M, 0.0);
  F.b.assign(M, 0.0);
  F.Q.assign(M, 0.0);
  double bnext = 0.0;
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    const double L = -lam * cA(n);
    const double Dg = 1.0 + lam * cB(n, N);
    const double U = (i + 1 < M) ? -lam * cC(n, N) : 0.0;
    const double den = Dg + U * bnext;
    F.e[i] = 1.0 / den;
    F.h[i] = U / den;
    F.b[i] = -L / den;
    bnext = F.b[i];
  }
  F.Q[0] = 1.0;
  double sq = 1.0;
  for (int i = 1; i < M; ++i) {
    F.Q[i] = F.b[i] * F.Q[i - 1];
    sq += F.Q[i];
  }
  F.isq = 1.0 / sq;
  return F;
}

// real right-hand side r[i] = r_{2i+sig}; returns f[i]
std::vector<double> host_solve(int N, int sig, const std::vector<double>& r, const Factor& F, double s) {
  const int M = (N - sig) / 2 + 1;
  std::vector<double> f(M, 0.0);
  double anext = 0.0;
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    double R = cA(n) * r[i - 1] - cB(n, N) * r[i];
    if (i + 1 < M) R += cC(n, N) * r[i + 1];
    const double a = F.e[i] * R - F.h[i] * anext;
    f[i] = a;
    anext = a;
  }
  double Pp = 0.0, sum = 0.0;
  for (int i = 1; i < M; ++i) {
    Pp = f[i] + F.b[i] * Pp;
    f[i] = Pp;
    sum += Pp;
  }
  const double f0 = F.isq * (s - sum);
  f[0] = f0;
  for (int i = 1; i < M; ++i) f[i] += F.Q[i] * f0;
  return f;
}

// the tau rows n >= 2 only: f_i = P_i with the lowest coefficient f_0 = 0
std::vector<double> host_affine(int N, int sig, const std::vector<double>& r, const Factor& F) {
  const int M = (N - sig) / 2 + 1;
  std::vector<double> f(M, 0.0);
  double anext = 0.0;
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    double R = cA(n) * r[i - 1] - cB(n, N) * r[i];
    if (i + 1 < M) R += cC(n, N) * r[i + 1];
    const double a = F.e[i] * R - F.h[i] * anext;
    f[i] = a;
    anext = a;
  }
  double Pp = 0.0;
  for (int i = 1; i < M; ++i) {
    Pp = f[i] + F.b[i] * Pp;
    f[i] = Pp;
  }
  return f;
}

bool fft_plan(int n, FftPlan* pl) {
  pl->n = n;
  pl->nst = 0;
  int m = n;
  while (m % 4 == 0 && pl->nst < kMaxRadixStages) { pl->radix[pl->nst++] = 4; m /= 4; }
  while (m % 2 == 0 && pl->nst < kMaxRadixStages) { pl->radix[pl->nst++] = 2; m /= 2; }
  while (m % 3 == 0 && pl->nst < kMaxRadixStages) { pl->radix[pl->nst++] = 3; m /= 3; }
  return m == 1;
}

// e^{2 pi i k / n}; exact at multiples of a quarter turn, so that sums of
// twiddles that cancel in exact arithmetic also cancel in floating point
std::vector<double2> twiddles(int n) {
  std::vector<double2> t(n);
  const double qc[4] = {1.0, 0.0, -1.0, 0.0}, qs[4] = {0.0, 1.0, 0.0, -1.0};
  for (int k = 0; k < n; ++k) {
    if ((4L * k) % n == 0) {
      const int q = (int)((4L * k) / n);
      t[k] = make_double2(qc[q], qs[q]);
    } else {
      const double a = 2.0 * M_PI * (double)k / (double)n;
      t[k] = make_double2(std::cos(a), std::sin(a));
    }
  }
  return t;
}

// Re_b and Re_tau are based on the half height 1 of the closed channel and on
// the whole height 2 of the open channel (free-slip top): y+ = (1 + y) Re_tau / height
double channel_height(const ch_params_t* p) { return p->top_bc == 1 ? 2.0 : 1.0; }

int sensing_node(int N, double re_tau, double y_plus, double height) {
  for (int j = N; j >= 0; --j) {
    const double yj = std::cos(M_PI * j / N);
    if ((1.0 + yj) * re_tau / height >= y_plus) return j;
  }
  return 0;
}

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  void normal_pair(double* a, double* b) {
    const double u1 = 1.0 - uniform();
    const double u2 = uniform();
    const double r = std::sqrt(-2.0 * std::log(u1));
    const double t = 2.0 * M_PI * u2;
    *a = r * std::cos(t);
    *b = r * std::sin(t);
  }
};

int check_params(const ch_params_t* p) {
  if (!p) return CH_ERR_ARG;
  if (p->nx < 4 || p->nz < 4 || (p->nx & 1) || (p->nz & 1)) return CH_ERR_ARG;
  if (p->ny < 9 || p->ny > kMaxNy) return CH_ERR_ARG;
  if (!(p->lx > 0) || !(p->lz > 0) || !(p->re_bulk > 0) || !(p->re_tau > 0) || !(p->dt > 0)) return CH_ERR_ARG;
  if (p->steps_per_action < 1) return CH_ERR_ARG;
  if (p->control < 0 || p->control > 2) return CH_ERR_ARG;
  if (p->autotune != 0 && p->autotune != 1) return CH_ERR_ARG;
  if (p->top_bc != 0 && p->top_bc != 1) return CH_ERR_ARG;
  if (p->precision != 0 && p->precision != 1) return CH_ERR_UNSUPPORTED;
  // the free-slip top's stage kernels are built for ny <= 65 (one parity <= 33 unknowns)
  if (p->top_bc == 1 && p->ny > 65) return CH_ERR_UNSUPPORTED;
  FftPlan a, b;
  if (!fft_plan(3 * p->nx / 2, &a) || !fft_plan(3 * p->nz / 2, &b)) return CH_ERR_UNSUPPORTED;
  if ((3 * p->nx / 2) % 2 || (3 * p->nz / 2) % 2) return CH_ERR_UNSUPPORTED;
  return CH_OK;
}

}  // namespace

struct ch_env {
  ch_params_t prm;
  Grid g;
  int B = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  PencilBufs pb{};
  DevTables tab{};
  PlaneArgs<double> plane{};
  size_t plane_smem = 0;
  PlaneArgs<float> plane_f{};   // FP32 nonlinear term (precision 1)
  size_t plane_f_smem = 0;
  double* d_act = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;
  size_t out_stride = 0;
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  std::vector<double> t, steps;  // per slot
  int js = 0;
  double nu = 0, u_tau = 0, tau_ref = 0;
  int launches_per_step = 0;
  int ppc_pre = 8, ppc_post = 8;  // modes per CTA of the fused stage kernels
  bool post_batched = false;      // batched form of stage_post (one thread per mode, class, component)
  bool tuned = false;             // tile shapes chosen by timing at env_create
  double tune_ms = 0.0;
  // kernel timing (env_profile)
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
  int ev_used[4] = {0, 0, 0, 0};
  // The step's launch sequence is fixed for a handle: it is captured once into
  // a CUDA graph on the internal action/output buffers and replayed (one
  // launch instead of 14-15).  [0]: every slot; [1]: slots masked by
  // graph_mask (serving ticks).  Profiling launches the same kernels directly.
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  const int* graph_mask = nullptr;
  // on-device policy (control 2): FP32 weights, its input planes [B][2][nz][nx]
  float* d_pol_w = nullptr;
  double* d_pol_in = nullptr;
  PolicyDesc pol{};
  bool pol_set = false;
  char err[256] = {0};
};

namespace {

template <typename T>
int dalloc(ch_env* env, T** ptr, size_t count) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&p, bytes) != cudaSuccess) return CH_ERR_OOM;
  env->allocs.push_back(p);
  env->device_bytes += bytes;
  *ptr = static_cast<T*>(p);
  return CH_OK;
}

template <typename T>
int dupload(ch_env* env, const T** ptr, const std::vector<T>& host) {
  T* d = nullptr;
  int rc = dalloc(env, &d, host.size());
  if (rc) return rc;
  if (cudaMemcpy(d, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return CH_ERR_CUDA;
  *ptr = d;
  return CH_OK;
}

void free_env(ch_env* env) {
  if (!env) return;
  if (env->stream) cudaStreamSynchronize(env->stream);
  for (cudaGraphExec_t& x : env->graph)
    if (x) cudaGraphExecDestroy(x);
  for (auto& v : env->ev)
    for (auto& pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (void* p : env->allocs) cudaFree(p);
  if (env->h_out) cudaFreeHost(env->h_out);
  if (env->own_stream) cudaStreamDestroy(env->own_stream);
  delete env;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return CH_ERR_CUDA;     \
  } while (0)

#define RC(call)                 \
  do {                           \
    int r_ = (call);             \
    if (r_ != CH_OK) return r_;  \
  } while (0)

// nonlinear plane kernel: smallest cluster whose z-slab fits shared memory
template <typename R>
int setup_plane(ch_env* env, PlaneArgs<R>* a, size_t* smem) {
  using C = typename cpx<R>::T;
  const Grid& g = env->g;
  a->nxh = g.nxh; a->nz = g.nz; a->ny = g.ny; a->mx = g.mx; a->mz = g.mz; a->P = g.P;
  a->S = 0;
  const size_t csz = sizeof(C);
  // cluster size: the smallest feasible S whose ny * B * S CTAs fill the SMs
  // once; without one, the largest feasible S.  Handles of the same grid and
  // batch capacity give bit-identical results; other capacities may split the
  // planes differently and agree to rounding.
  int nsm = 152;
  {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      nsm = v;
  }
  int feasible[5], nf = 0;
  for (int S = 1; S <= 8; S *= 2) {
    if (g.mz % S || (g.mz / S) % 2) continue;
    if ((size_t)6 * (g.mz / S) * g.nxh * csz > 160 * 1024) continue;
    feasible[nf++] = S;
  }
  // three passes through a global scratch array: planes of 256 x 256 modes,
  // whose padded z-slab fits no portable cluster in either precision (the
  // traffic costs less than serialising 16-CTA clusters, of which the device
  // holds few), and the FP64 planes of 64 x 64 and 128 x 128 modes; only in
  // the precision the handle steps in (the other plane keeps a cluster, for
  // ch_nonlinear, where one fits)
  const bool stepping = (sizeof(R) == 8) == (env->prm.precision == 0);
  if (stepping && two_pass_chosen(g.mx, g.mz, g.nxh, sizeof(R) == 8)) {
    a->two_pass = 1;
    a->S = 1;
    a->Lz = g.mz;
    a->NP = 0;
    *smem = 0;
    C* y = nullptr;
    RC(dalloc(env, &y, (size_t)env->B * g.ny * 6 * g.mz * g.nxh));
    a->y = y;
    if (!fft_plan(g.mx, &a->px) || !fft_plan(g.mz, &a->pz)) return CH_ERR_UNSUPPORTED;
    auto cast2 = [](const std::vector<double2>& v) {
      std::vector<C> o(v.size());
      for (size_t i = 0; i < v.size(); ++i) o[i] = mk((R)v[i].x, (R)v[i].y);
      return o;
    };
    RC(dupload(env, &a->tw_x, cast2(twiddles(g.mx))));
    RC(dupload(env, &a->tw_z, cast2(twiddles(g.mz))));
    RC(dupload(env, &a->tw_mz, cast2(twiddles(g.mz))));
    a->scale = (R)(1.0 / ((double)g.mx * g.mz));
    return CH_OK;
  }
  // a 16-CTA cluster (non-portable opt-in) only where no portable size fits
  if (!nf && g.mz % 16 == 0 && (g.mz / 16) % 2 == 0 && (size_t)6 * (g.mz / 16) * g.nxh * csz <= 160 * 1024)
    feasible[nf++] = 16;
  if (!nf) return CH_ERR_UNSUPPORTED;
  int S = feasible[nf - 1];
  for (int k = 0; k < nf; ++k)
    if ((long)g.ny * env->B * feasible[k] >= nsm) { S = feasible[k]; break; }
  const int Lz = g.mz / S;
  const size_t zb = (size_t)6 * Lz * g.nxh * csz;
  const int npairs = Lz / 2;
  int np = 0;
  // row pairs per batch: keep two CTAs per SM (<= 100 KB) when possible
  for (size_t lim : {(size_t)100 * 1024, (size_t)220 * 1024}) {
    for (int d = std::min(npairs, 16); d >= 1 && !np; --d)
      if (npairs % d == 0 && zb + (size_t)6 * d * g.mx * csz <= lim) np = d;
    if (np) break;
  }
  if (np) {
    a->S = S; a->Lz = Lz; a->NP = np;
    *smem = zb + (size_t)6 * np * g.mx * csz;
  }
  if (!a->S) return CH_ERR_UNSUPPORTED;
  // planes of 16 x 16 modes run one plane per team of threads with the line
  // transforms in registers once the batch supplies enough planes to fill
  // the SMs (four per SM, two per CTA); fewer planes keep the cluster split,
  // which spreads each plane over S CTAs
  a->team16 = 0;
  if (plane16_shape(g.mx, g.mz, g.nxh, g.nz) && (long)g.ny * env->B >= 4L * nsm) {
    a->team16 = 1;
    a->S = 1;
    a->Lz = g.mz;
  }
  if (!fft_plan(g.mx, &a->px) || !fft_plan(a->Lz, &a->pz)) return CH_ERR_UNSUPPORTED;
  if (a->S > 8) {
    int clusters = 0;
    if (plane_max_clusters<R>(*a, *smem, &clusters) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      a->S = 0;
      return CH_ERR_UNSUPPORTED;
    }
  }
  auto cast = [](const std::vector<double2>& v) {
    std::vector<C> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = mk((R)v[i].x, (R)v[i].y);
    return o;
  };
  RC(dupload(env, &a->tw_x, cast(twiddles(g.mx))));
  RC(dupload(env, &a->tw_z, cast(twiddles(a->Lz))));
  RC(dupload(env, &a->tw_mz, cast(twiddles(g.mz))));
  a->scale = (R)(1.0 / ((double)g.mx * g.mz));
  return CH_OK;
}

int build_tables(ch_env* env) {
  const Grid& g = env->g;
  const int N = g.N, P = g.P, ny = g.ny;
  const int Mh = N / 2 + 1;
  const ch_params_t& p = env->prm;
  std::vector<double> kx(g.nxh), kz(g.nz);
  for (int i = 0; i < g.nxh; ++i) kx[i] = 2.0 * M_PI / p.lx * i;
  for (int r = 0; r < g.nz; ++r) {
    const int m = r < g.nz / 2 ? r : r - g.nz;
    kz[r] = (r == g.nz / 2) ? 0.0 : 2.0 * M_PI / p.lz * m;
  }
  std::vector<double> cheb((size_t)ny * ny);
  for (int j = 0; j < ny; ++j)
    for (int n = 0; n < ny; ++n) cheb[(size_t)j * ny + n] = std::cos(M_PI * (double)((j * n) % (2 * N)) / N);

  // tau tables, mode index fastest: [stage][parity][e, h, b, Q][Mh][P]
  std::vector<double> helm((size_t)3 * 2 * 4 * Mh * P, 0.0), helm_isq((size_t)3 * 2 * P, 0.0);
  std::vector<double> pois((size_t)2 * 4 * Mh * P, 0.0), pois_isq((size_t)2 * P, 0.0);
  std::vector<double> vh((size_t)3 * 2 * Mh * P, 0.0), vh_idv((size_t)3 * 2 * P, 0.0);
  std::vector<double> u1((size_t)3 * Mh, 0.0), u1_iflux(3, 0.0);
  // free-slip top: sum Q, sum n^2 Q per parity; A, B of vh per parity
  std::vector<double> helm_top((size_t)3 * 2 * 2 * P, 0.0), vh_top((size_t)3 * 2 * 2 * P, 0.0);
  const bool top = p.top_bc == 1;
  // no-slip top: the folded tables of the per-thread solves, [..][eA, eB, eC, h, b, W (, E1)][Mh][P];
  // e1 > 0 adds E1 = e1 e (the Helmholtz tables, e1 = 1 + alpha/beta of the stage)
  std::vector<double> helm_f(top ? 0 : (size_t)3 * 2 * 7 * Mh * P, 0.0);
  std::vector<double> pois_f(top ? 0 : (size_t)2 * 6 * Mh * P, 0.0);
  auto put_f = [&](std::vector<double>& tab, size_t base, const Factor& F, int M, int pp, int sig, double e1) {
    double w = 1.0;  // W_{M-1}
    for (int i = M - 1; i >= 1; --i) {
      const int n = 2 * i + sig;
      if (i < M - 1) w = 1.0 + F.b[i + 1] * w;
      tab[base + ((size_t)0 * Mh + i) * P + pp] = F.e[i] * cA(n);
      tab[base + ((size_t)1 * Mh + i) * P + pp] = F.e[i] * cB(n, N);
      tab[base + ((size_t)2 * Mh + i) * P + pp] = F.e[i] * cC(n, N);
      tab[base + ((size_t)3 * Mh + i) * P + pp] = F.h[i];
      tab[base + ((size_t)4 * Mh + i) * P + pp] = F.b[i];
      tab[base + ((size_t)5 * Mh + i) * P + pp] = w;
      if (e1 > 0.0) tab[base + ((size_t)6 * Mh + i) * P + pp] = e1 * F.e[i];
    }
  };
  auto put = [&](std::vector<double>& tab, size_t base, const Factor& F, int M, int pp) {
    for (int i = 0; i < M; ++i) {
      tab[base + ((size_t)0 * Mh + i) * P + pp] = F.e[i];
      tab[base + ((size_t)1 * Mh + i) * P + pp] = F.h[i];
      tab[base + ((size_t)2 * Mh + i) * P + pp] = F.b[i];
      tab[base + ((size_t)3 * Mh + i) * P + pp] = F.Q[i];
    }
  };
  for (int pp = 0; pp < P; ++pp) {
    const int row = pp / g.nxh, ix = pp % g.nxh;
    const double k2 = kx[ix] * kx[ix] + kz[row] * kz[row];
    for (int sig = 0; sig < 2; ++sig) {
      const int M = (N - sig) / 2 + 1;
      const Factor Fp = host_factor(N, sig, k2);
      put(pois, (size_t)sig * 4 * Mh * P, Fp, M, pp);
      if (!top) put_f(pois_f, (size_t)sig * 6 * Mh * P, Fp, M, pp, sig, 0.0);
      pois_isq[(size_t)sig * P + pp] = Fp.isq;
      for (int k = 0; k < 3; ++k) {
        const double ibdn = 1.0 / (rk_beta(k) * p.dt * env->nu);
        const Factor Fh = host_factor(N, sig, k2 + ibdn);
        const size_t slot = (size_t)(k * 2 + sig);
        // every Helmholtz right-hand side of the stage carries the factor
        // -1/(beta dt nu); the solve is linear in it, so the device tables take
        // it in the elimination factor e and the kernels leave it out
        Factor Fs = Fh;
        for (double& e : Fs.e) e *= -ibdn;
        put(helm, slot * 4 * Mh * P, Fs, M, pp);
        if (!top) put_f(helm_f, slot * 7 * Mh * P, Fs, M, pp, sig, 1.0 + rk_alpha(k) / rk_beta(k));
        helm_isq[slot * P + pp] = Fh.isq;
        {
          double sq = 0.0, sq2 = 0.0;
          for (int i = 0; i < M; ++i) {
            const double n = 2 * i + sig;
            sq += Fh.Q[i];
            sq2 += n * n * Fh.Q[i];
          }
          helm_top[(slot * 2 + 0) * P + pp] = sq;
          helm_top[(slot * 2 + 1) * P + pp] = sq2;
        }
        // homogeneous solution of this parity: phi_h = 1 on the wall row, r = 0
        const std::vector<double> zero(M, 0.0);
        const std::vector<double> phih = host_solve(N, sig, zero, Fh, 1.0);
        const std::vector<double> vhp = host_solve(N, sig, phih, Fp, 0.0);
        double d = 0.0, a2 = 0.0;
        for (int i = 0; i < M; ++i) {
          const int n = 2 * i + sig;
          const double nn = (double)n * n;
          vh[(slot * Mh + i) * P + pp] = vhp[i];
          d += nn * vhp[i];
          a2 += nn * (nn - 1.0) / 3.0 * vhp[i];   // T_n''(+1) = n^2 (n^2 - 1) / 3
        }
        vh_idv[slot * P + pp] = (d != 0.0 && std::isfinite(d)) ? 1.0 / d : 0.0;
        vh_top[(slot * 2 + 0) * P + pp] = a2;
        vh_top[(slot * 2 + 1) * P + pp] = d;
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    const double a = rk_alpha(k), b = rk_beta(k);
    const double ibdn = 1.0 / (b * p.dt * env->nu);
    const Factor F = host_factor(N, 0, ibdn);
    const int M = N / 2 + 1;
    std::vector<double> r(M, 0.0);
    r[0] = 1.0;
    // no-slip: the response with zero wall values; free-slip top: the affine
    // particular response (lowest coefficient 0), closed on the device
    const std::vector<double> uu = top ? host_affine(N, 0, r, F) : host_solve(N, 0, r, F, 0.0);
    const double cforce = (a + b) / (b * env->nu);
    double flux = 0.0;
    for (int i = 0; i < M; ++i) {
      const int n = 2 * i;
      const double v = -cforce * uu[i];
      u1[(size_t)k * Mh + i] = v;
      flux += 2.0 / (1.0 - (double)n * n) * v;
    }
    u1_iflux[k] = top ? 0.0 : 1.0 / flux;
  }
  // tau row constants per n
  std::vector<double> rowc((size_t)3 * ny, 0.0);
  for (int n = 2; n <= N; ++n) {
    rowc[n] = cA(n);
    rowc[ny + n] = cB(n, N);
    rowc[2 * ny + n] = cC(n, N);
  }
  RC(dupload(env, &env->tab.tau.rowc, rowc));
  // T_n'(y_js) = n sin(n theta) / sin(theta), theta = pi js / N (T_n'(+1) = n^2)
  std::vector<double> dts(ny, 0.0);
  for (int n = 0; n < ny; ++n) {
    if (env->js == 0) {
      dts[n] = (double)n * n;
    } else {
      dts[n] = n * std::sin(M_PI * (double)((n * env->js) % (2 * N)) / N) / std::sin(M_PI * (double)env->js / N);
    }
  }
  RC(dupload(env, &env->tab.dts, dts));
  RC(dupload(env, &env->tab.kx, kx));
  RC(dupload(env, &env->tab.kz, kz));
  RC(dupload(env, &env->tab.cheb, cheb));
  {
    std::vector<float> chf(cheb.size());
    for (size_t i = 0; i < cheb.size(); ++i) chf[i] = (float)cheb[i];
    RC(dupload(env, &env->tab.cheb_f, chf));
  }
  RC(dupload(env, &env->tab.tau.helm, helm));
  RC(dupload(env, &env->tab.tau.helm_isq, helm_isq));
  RC(dupload(env, &env->tab.tau.pois, pois));
  RC(dupload(env, &env->tab.tau.pois_isq, pois_isq));
  if (!top) {
    RC(dupload(env, &env->tab.tau.helm_f, helm_f));
    RC(dupload(env, &env->tab.tau.pois_f, pois_f));
  }
  RC(dupload(env, &env->tab.tau.vh, vh));
  RC(dupload(env, &env->tab.tau.vh_idv, vh_idv));
  RC(dupload(env, &env->tab.tau.u1, u1));
  RC(dupload(env, &env->tab.tau.u1_iflux, u1_iflux));
  RC(dupload(env, &env->tab.tau.helm_top, helm_top));
  RC(dupload(env, &env->tab.tau.vh_top, vh_top));
  env->tab.tau.Mh = Mh;
  env->tab.tau.top_bc = top ? 1 : 0;
  RC(dupload(env, &env->tab.tw_nx, twiddles(g.nx)));
  RC(dupload(env, &env->tab.tw_nz, twiddles(g.nz)));
  RC(dupload(env, &env->tab.tw_cheb, twiddles(g.N)));

  // the plane of the handle's precision is required; the other one serves
  // ch_nonlinear (FP64) and is skipped where its slab does not fit
  const int r64 = setup_plane(env, &env->plane, &env->plane_smem);
  const int r32 = setup_plane(env, &env->plane_f, &env->plane_f_smem);
  if (env->prm.precision == 1 ? r32 != CH_OK : r64 != CH_OK) return env->prm.precision == 1 ? r32 : r64;
  if (r64 != CH_OK) env->plane.S = 0;
  if (r32 != CH_OK) env->plane_f.S = 0;
  return CH_OK;
}

void fill_seed_state(const ch_params_t* p, uint64_t seed, double amplitude, int kmax, double* buf) {
  const int nx = p->nx, ny = p->ny, nz = p->nz, nxh = nx / 2, P = nz * nxh;
  double* v = buf;
  double* g = v + (size_t)2 * ny * P;
  double* U = g + (size_t)2 * ny * P;
  double* W = U + ny;
  double* vw = W + ny;
  double* tail = vw + 2 * P;
  std::memset(buf, 0, ch_state_bytes(p));
  struct Mode { int row, i; };
  std::vector<Mode> modes;
  int nexc = 0;
  for (int row = 0; row < nz; ++row) {
    const int m = row < nz / 2 ? row : row - nz;
    if (m == -nz / 2) continue;
    for (int i = 0; i < nxh; ++i) {
      if (i > kmax || std::abs(m) > kmax || (i == 0 && m == 0)) continue;
      if (i == 0 && m < 0) continue;
      modes.push_back({row, i});
      nexc += (i == 0) ? 2 : 1;
    }
  }
  const double s = nexc ? amplitude / std::sqrt((double)nexc) : 0.0;
  // wall-normal shapes (Chebyshev coefficients): closed channel (1 - y^2)^2 and
  // 1 - y^2; open channel (free-slip top) (1+y)^2 (1-y) (2-y) / 2 and
  // (1+y) (3-y) / 4
  const bool open = p->top_bc == 1;
  const double shape_v_closed[5] = {0.375, 0.0, -0.5, 0.0, 0.125};
  const double shape_g_closed[3] = {0.5, 0.0, -0.5};
  const double shape_v_open[5] = {0.4375, 0.125, -0.5, -0.125, 0.0625};
  const double shape_g_open[3] = {0.625, 0.5, -0.125};
  const double* shape_v = open ? shape_v_open : shape_v_closed;
  const double* shape_g = open ? shape_g_open : shape_g_closed;
  SplitMix64 rng{seed};
  for (const Mode& md : modes) {
    double a, b, c, d;
    rng.normal_pair(&a, &b);
    rng.normal_pair(&c, &d);
    const double cvr = s * a, cvi = s * b, cgr = s * c, cgi = s * d;
    const int m = md.row < nz / 2 ? md.row : md.row - nz;
    const int mrow = (-m + nz) % nz;
    for (int n = 0; n < 5; ++n) {
      if (shape_v[n] == 0.0) continue;
      const size_t o = ((size_t)n * P + md.row * nxh + md.i) * 2;
      v[o] = cvr * shape_v[n];
      v[o + 1] = cvi * shape_v[n];
      if (md.i == 0) {
        const size_t o2 = ((size_t)n * P + mrow * nxh) * 2;
        v[o2] = v[o];
        v[o2 + 1] = -v[o + 1];
      }
    }
    for (int n = 0; n < 3; ++n) {
      if (shape_g[n] == 0.0) continue;
      const size_t o = ((size_t)n * P + md.row * nxh + md.i) * 2;
      g[o] = cgr * shape_g[n];
      g[o + 1] = cgi * shape_g[n];
      if (md.i == 0) {
        const size_t o2 = ((size_t)n * P + mrow * nxh) * 2;
        g[o2] = g[o];
        g[o2 + 1] = -g[o + 1];
      }
    }
  }
  if (open) {  // half-Poiseuille 1.5 (2 s - s^2), s = (1 + y) / 2
    U[0] = 0.9375;
    U[1] = 0.75;
    U[2] = -0.1875;
  } else {
    U[0] = 0.75;
    U[2] = -0.75;
  }
  (void)W;
  tail[0] = tail[1] = 0.0;
}

int set_state_dev(ch_env* env, int e, const double* buf) {
  const Grid& g = env->g;
  const size_t P = g.P, ny = g.ny;
  const double* v = buf;
  const double* gg = v + 2 * ny * P;
  const double* U = gg + 2 * ny * P;
  const double* W = U + ny;
  const double* vw = W + ny;
  const double* tail = vw + 2 * P;
  cudaStream_t st = env->stream;
  CK(cudaMemcpyAsync(env->pb.V + (size_t)e * ny * P, v, ny * P * sizeof(double2), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(env->pb.G + (size_t)e * ny * P, gg, ny * P * sizeof(double2), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(env->pb.UM + (size_t)e * ny, U, ny * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(env->pb.WM + (size_t)e * ny, W, ny * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(env->pb.vw_new + (size_t)e * P, vw, P * sizeof(double2), cudaMemcpyHostToDevice, st));
  // previous right-hand sides: complex values in the node precision, [B][ny][P]
  const size_t hsz = env->prm.precision == 1 ? sizeof(float2) : sizeof(double2);
  CK(cudaMemsetAsync(reinterpret_cast<char*>(env->pb.HVP) + (size_t)e * ny * P * hsz, 0, ny * P * hsz, st));
  CK(cudaMemsetAsync(reinterpret_cast<char*>(env->pb.HGP) + (size_t)e * ny * P * hsz, 0, ny * P * hsz, st));
  CK(cudaMemsetAsync(env->pb.HXP + (size_t)e * ny, 0, ny * sizeof(double), st));
  CK(cudaMemsetAsync(env->pb.HZP + (size_t)e * ny, 0, ny * sizeof(double), st));
  CK(cudaStreamSynchronize(st));
  env->t[e] = tail[0];
  env->steps[e] = tail[1];
  return CH_OK;
}

// event pair around one launch of class `cls` (no-op unless profiling)
cudaError_t prof_mark(ch_env* env, int cls, bool begin) {
  if (!env->prof) return cudaSuccess;
  auto& v = env->ev[cls];
  int& used = env->ev_used[cls];
  if (begin) {
    if (used == (int)v.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> pr;
      cudaError_t e = cudaEventCreate(&pr.first);
      if (e != cudaSuccess) return e;
      e = cudaEventCreate(&pr.second);
      if (e != cudaSuccess) return e;
      v.push_back(pr);
    }
    return cudaEventRecord(v[used].first, env->stream);
  }
  cudaError_t e = cudaEventRecord(v[used].second, env->stream);
  ++used;
  return e;
}

#define LAUNCH(cls, call)                   \
  do {                                      \
    CK(prof_mark(env, (cls), true));        \
    CK(call);                               \
    CK(prof_mark(env, (cls), false));       \
  } while (0)

// Coefficients of RK stage k (C3) with the wall-velocity ramp at theta (C4).
StageCoef stage_coef(const ch_env* env, int k, double theta) {
  StageCoef sc;
  sc.alpha = rk_alpha(k);
  sc.beta = rk_beta(k);
  sc.gamma = kGamma[k];
  sc.zeta = kZeta[k];
  sc.dt = env->prm.dt;
  sc.nu = env->nu;
  sc.theta = theta;
  sc.flux = 2.0;
  sc.k = k;
  return sc;
}

int run_stage(ch_env* env, int k, double theta) {
  const Grid& g = env->g;
  const int B = env->B;
  cudaStream_t st = env->stream;
  const bool mixed = env->prm.precision == 1;
  if (mixed) {
    float2* q = reinterpret_cast<float2*>(env->pb.Q);
    LAUNCH(0, launch_stage_pre<float>(g, B, env->pb, env->tab, q, env->ppc_pre, st));
    PlaneArgs<float> a = env->plane_f;
    a.q = q;
    a.h = reinterpret_cast<float2*>(env->pb.R);
    LAUNCH(1, launch_plane<float>(a, B, env->plane_f_smem, st));
  } else {
    LAUNCH(0, launch_stage_pre<double>(g, B, env->pb, env->tab, env->pb.Q, env->ppc_pre, st));
    PlaneArgs<double> a = env->plane;
    a.q = env->pb.Q;
    a.h = env->pb.R;
    LAUNCH(1, launch_plane<double>(a, B, env->plane_smem, st));
  }
  const StageCoef sc = stage_coef(env, k, theta);
  if (mixed)
    LAUNCH(2, launch_stage_post<float>(g, B, env->pb, env->tab, reinterpret_cast<const float2*>(env->pb.R), sc,
                                       env->ppc_post, env->post_batched, st));
  else
    LAUNCH(2, launch_stage_post<double>(g, B, env->pb, env->tab, env->pb.R, sc, env->ppc_post, env->post_batched,
                                        st));
  return CH_OK;
}

// kernels of one env_step: the action or control kernels, per RK step three
// stages of (stage_pre, nonlinear term, implicit half) and the wall shear,
// then the outputs; the nonlinear term takes three launches where it runs in
// passes, the implicit half two in its wide form
static void set_launch_count(ch_env* env) {
  const ch_params_t* p = &env->prm;
  const bool passes = p->precision == 1 ? env->plane_f.two_pass : env->plane.two_pass;
  const int stage = 1 + (passes ? 3 : 1) + stage_post_launches(env->g, p->top_bc, env->post_batched);
  env->launches_per_step = (p->control == 0 ? 2 : p->control == 1 ? 1 : 5) + p->steps_per_action * (3 * stage + 1) + 3;
}

// The kernels of one environment step, in stream order.
int launch_step(ch_env* env, const double* d_action, double* d_out, const int* d_active) {
  const Grid& g = env->g;
  const int B = env->B;
  cudaStream_t st = env->stream;
  env->pb.active = d_active;
  env->plane.active = d_active;
  env->plane_f.active = d_active;
  struct Reset {
    ch_env* e;
    ~Reset() { e->pb.active = nullptr; e->plane.active = nullptr; e->plane_f.active = nullptr; }
  } reset{env};
  if (env->prm.control == 1) {
    LAUNCH(3, launch_sense(g, B, env->pb, env->tab, env->js, env->prm.alpha, 1, st));
  } else if (env->prm.control == 2) {
    // the policy sees the sensing plane of the current flow, the same values
    // the previous step returned as its observation
    const size_t pstride = (size_t)2 * g.nz * g.nx;
    LAUNCH(3, launch_sense(g, B, env->pb, env->tab, env->js, env->prm.alpha, 0, st));
    LAUNCH(3, launch_obs(g, B, env->pb.planes, env->tab, env->d_pol_in, pstride, d_active, st));
    LAUNCH(3, launch_policy(g.nx, g.nz, B, env->pol, env->d_pol_w, env->d_pol_in, env->d_act, env->u_tau, d_active,
                            st));
    LAUNCH(3, launch_action(g, B, env->d_act, env->u_tau, env->tab, env->pb, st));
  } else {
    LAUNCH(3, launch_action(g, B, d_action, env->u_tau, env->tab, env->pb, st));
  }
  const int spa = env->prm.steps_per_action;
  for (int s = 0; s < spa; ++s) {
    for (int k = 0; k < 3; ++k) RC(run_stage(env, k, (s + kCEnd[k]) / spa));
    LAUNCH(3, launch_wall_shear(g, B, env->pb.UM, env->nu, env->pb.tau_acc, d_active, st));
  }
  LAUNCH(3, launch_sense(g, B, env->pb, env->tab, env->js, env->prm.alpha, 0, st));
  LAUNCH(3, launch_obs(g, B, env->pb.planes, env->tab, d_out, env->out_stride, d_active, st));
  LAUNCH(3, launch_finalize(B, env->pb.tau_acc, 1.0 / spa, env->tau_ref, d_out, env->out_stride,
                            (size_t)2 * g.nz * g.nx, d_active, st));
  return CH_OK;
}

// Capture launch_step on the internal buffers into graph[gi].
int capture_step(ch_env* env, int gi, const int* d_active) {
  cudaStream_t st = env->stream;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  const int rc = launch_step(env, env->d_act, env->d_out, d_active);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc != CH_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc != CH_OK ? rc : CH_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&env->graph[gi], graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    env->graph[gi] = nullptr;
    return CH_ERR_CUDA;
  }
  return CH_OK;
}

// ---------------------------------------------------------------------------
// Tile shapes of the stage kernels.  Within a form of the implicit half every
// candidate performs the same floating-point operations per output (each
// mode's recurrences and sums run in one fixed order whatever the number of
// modes per CTA), so the widths change speed only, never results.  The
// autotuner keeps the form the size rule chose.
// ---------------------------------------------------------------------------
bool tiles_valid(const ch_env* env, int smem_max, int ppc_pre, int ppc_post, int post_batched) {
  const Grid& g = env->g;
  const size_t node = env->prm.precision == 1 ? sizeof(float2) : sizeof(double2);
  auto pow2 = [](int v, int hi) { return v >= 1 && v <= hi && (v & (v - 1)) == 0; };
  if (!pow2(ppc_pre, 8) || stage_pre_smem(g, ppc_pre, node) > (size_t)smem_max) return false;
  const int top = env->prm.top_bc;
  if (post_batched == 1) return pow2(ppc_post, 16) && stage_post_batched_smem(g, ppc_post, top, node) <= (size_t)smem_max;
  if (post_batched != 0) return false;
  // the per-tile form runs 8 ppc threads and any tile width up to 8 (widths
  // that are not powers of two fill the resident CTA slots more evenly)
  return ppc_post >= 1 && ppc_post <= 8 && stage_post_smem(g, env->tab.tau.Mh, ppc_post, top) <= (size_t)smem_max;
}

int drop_graphs(ch_env* env) {
  for (cudaGraphExec_t& x : env->graph) {
    if (x) CK(cudaGraphExecDestroy(x));
    x = nullptr;
  }
  env->graph_mask = nullptr;
  return CH_OK;
}

// Median device time of `reps` launches after one warm-up launch.
template <class F>
int time_launches(cudaStream_t st, int reps, F&& launch, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return CH_ERR_CUDA;
  }
  std::vector<float> t;
  int rc = launch();
  for (int i = 0; i < reps && rc == CH_OK; ++i) {
    float x = 0.f;
    if (cudaEventRecord(a, st) != cudaSuccess || (rc = launch()) != CH_OK || cudaEventRecord(b, st) != cudaSuccess ||
        cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&x, a, b) != cudaSuccess) {
      rc = rc != CH_OK ? rc : CH_ERR_CUDA;
      break;
    }
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != CH_OK) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return CH_OK;
}

// Time the candidate shapes of both stage kernels on this handle's buffers,
// before its initial state is written (the kernels run on zeroed fields), and
// keep the fastest of each.  Repeated launches of one kernel may overlap (an
// FP32-node stage kernel starts its prologue while the previous launch
// drains); the fields they touch are scratch here and are all rewritten when
// the initial state is set.
int autotune_tiles(ch_env* env, int smem_max) {
  const auto t0 = std::chrono::steady_clock::now();
  const Grid& g = env->g;
  const int B = env->B;
  const size_t Bs = B, P = g.P, ny = g.ny;
  cudaStream_t st = env->stream;
  PencilBufs& pb = env->pb;
  CK(cudaMemsetAsync(pb.V, 0, Bs * ny * P * sizeof(double2), st));
  CK(cudaMemsetAsync(pb.G, 0, Bs * ny * P * sizeof(double2), st));
  CK(cudaMemsetAsync(pb.HVP, 0, Bs * ny * P * sizeof(double2), st));
  CK(cudaMemsetAsync(pb.HGP, 0, Bs * ny * P * sizeof(double2), st));
  CK(cudaMemsetAsync(pb.R, 0, Bs * 3 * ny * P * sizeof(double2), st));
  CK(cudaMemsetAsync(pb.vw_old, 0, Bs * P * sizeof(double2), st));
  CK(cudaMemsetAsync(pb.vw_new, 0, Bs * P * sizeof(double2), st));
  for (double* x : {pb.UM, pb.WM, pb.HXP, pb.HZP}) CK(cudaMemsetAsync(x, 0, Bs * ny * sizeof(double), st));
  const bool mixed = env->prm.precision == 1;
  const StageCoef sc = stage_coef(env, 0, 1.0);
  auto pre = [&](int ppc) {
    const cudaError_t e = mixed ? launch_stage_pre<float>(g, B, pb, env->tab, reinterpret_cast<float2*>(pb.Q), ppc, st)
                                : launch_stage_pre<double>(g, B, pb, env->tab, pb.Q, ppc, st);
    return e == cudaSuccess ? CH_OK : CH_ERR_CUDA;
  };
  auto post = [&](int ppc, bool batched) {
    const cudaError_t e =
        mixed ? launch_stage_post<float>(g, B, pb, env->tab, reinterpret_cast<const float2*>(pb.R), sc, ppc, batched, st)
              : launch_stage_post<double>(g, B, pb, env->tab, pb.R, sc, ppc, batched, st);
    return e == cudaSuccess ? CH_OK : CH_ERR_CUDA;
  };
  constexpr int kReps = 3;
  float best = 0.f;
  bool have = false;
  for (int ppc : {8, 4, 2}) {
    if (!tiles_valid(env, smem_max, ppc, env->ppc_post, env->post_batched ? 1 : 0)) continue;
    float ms = 0.f;
    RC(time_launches(st, kReps, [&] { return pre(ppc); }, &ms));
    if (!have || ms < best) {
      best = ms;
      env->ppc_pre = ppc;
      have = true;
    }
  }
  have = false;
  // widths of the form the size rule chose: the per-tile and batched forms of
  // the no-slip solves sum in different orders (four-lane scans against one
  // thread per system), so timing never switches between them
  const int form = env->post_batched ? 1 : 0;
  const std::pair<int, int> cands[] = {{0, 8}, {0, 7}, {0, 6}, {0, 5}, {0, 4}, {0, 3}, {0, 2}, {0, 1}, {1, 16}, {1, 8}};
  for (const auto& c : cands) {
    if (c.first != form || !tiles_valid(env, smem_max, env->ppc_pre, c.second, c.first)) continue;
    float ms = 0.f;
    RC(time_launches(st, kReps, [&] { return post(c.second, c.first == 1); }, &ms));
    if (!have || ms < best) {
      best = ms;
      env->post_batched = c.first == 1;
      env->ppc_post = c.second;
      have = true;
    }
  }
  env->tuned = true;
  env->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return CH_OK;
}

// One environment step of every slot flagged in `h_active` (nullptr: all);
// `d_active` is the same mask on the device.
int run_step(ch_env* env, const double* d_action, double* d_out, const int* d_active = nullptr,
             const int* h_active = nullptr) {
  const int B = env->B;
  if (env->prm.control == 2 && !env->pol_set) return CH_ERR_STATE;
  if (env->prof) {
    // the action goes through the internal buffer as in the captured graph,
    // so env_get_action reports it in both modes
    const size_t plane = (size_t)env->g.nz * env->g.nx;
    if (env->prm.control == 0 && d_action != env->d_act)
      CK(cudaMemcpyAsync(env->d_act, d_action, B * plane * sizeof(double), cudaMemcpyDeviceToDevice, env->stream));
    RC(launch_step(env, env->d_act, d_out, d_active));
  } else {
    cudaStream_t st = env->stream;
    const int gi = d_active ? 1 : 0;
    if (d_active && env->graph_mask != d_active) {
      if (env->graph[1]) CK(cudaGraphExecDestroy(env->graph[1]));
      env->graph[1] = nullptr;
      env->graph_mask = d_active;
    }
    if (!env->graph[gi]) RC(capture_step(env, gi, d_active));
    const size_t plane = (size_t)env->g.nz * env->g.nx;
    if (env->prm.control == 0 && d_action != env->d_act)
      CK(cudaMemcpyAsync(env->d_act, d_action, B * plane * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaGraphLaunch(env->graph[gi], st));
    if (d_out != env->d_out)
      CK(cudaMemcpyAsync(d_out, env->d_out, B * env->out_stride * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  const int spa = env->prm.steps_per_action;
  for (int b = 0; b < B; ++b) {
    if (h_active && !h_active[b]) continue;
    env->t[b] += spa * env->prm.dt;
    env->steps[b] += spa;
  }
  return CH_OK;
}

}  // namespace

namespace chdns {
// internal entry points used by the serving layer (serve.cu)
int step_masked(ch_env* env, const double* d_action, const int* d_active, const int* h_active) {
  return run_step(env, d_action, env->d_out, d_active, h_active);
}
double* env_dout(ch_env* env) { return env->d_out; }
double* env_dact(ch_env* env) { return env->d_act; }
size_t env_out_stride(const ch_env* env) { return env->out_stride; }
cudaStream_t env_stream(const ch_env* env) { return env->stream; }
int env_slot_seed(ch_env* env, int e, uint64_t seed, double amplitude, int kmax) {
  std::vector<double> st(ch_state_bytes(&env->prm) / sizeof(double));
  fill_seed_state(&env->prm, seed, amplitude, kmax, st.data());
  return set_state_dev(env, e, st.data());
}
// device bytes env_create allocates for these parameters (tables and buffers)
size_t env_footprint(const ch_params_t* p) {
  const size_t B = p->batch > 0 ? p->batch : 1;
  const size_t nxh = p->nx / 2, P = nxh * p->nz, ny = p->ny, Mh = (ny - 1) / 2 + 1;
  const size_t state = B * (4 * ny * P * 16 + 4 * ny * 8 + 9 * ny * P * 16 + 3 * P * 16 + 8 +
                            (size_t)p->nz * p->nx * 8 + (2 * (size_t)p->nz * p->nx + 2) * 8);
  const size_t folded = p->top_bc == 0 ? (3 * 2 * 7 * Mh * P + 2 * 6 * Mh * P) * 8 : 0;
  const size_t tables = (3 * 2 * 4 * Mh * P + 3 * 2 * P + 2 * 4 * Mh * P + 2 * P + 3 * 2 * Mh * P + 3 * 2 * P +
                         3 * Mh + 3 + 3 * ny + ny + 2 * 3 * 2 * 2 * P) * 8 + ny * ny * 12 + (nxh + p->nz) * 8 +
                        folded;
  // the scratch of the three-pass nonlinear term, where it runs in passes
  // (complex values of the plane's precision)
  const size_t mx = 3 * (size_t)p->nx / 2, mz = 3 * (size_t)p->nz / 2;
  const size_t two_pass = two_pass_chosen((int)mx, (int)mz, (int)nxh, p->precision == 0)
                              ? B * ny * 6 * mz * nxh * (p->precision == 0 ? 16 : 8) : 0;
  return state + tables + two_pass + ((size_t)4 << 20);  // plus twiddles and rounding slack
}
}  // namespace chdns

extern "C" {

size_t ch_state_bytes(const ch_params_t* p) {
  if (!p) return 0;
  const size_t P = (size_t)p->nz * (p->nx / 2), ny = p->ny;
  return sizeof(double) * (4 * ny * P + 2 * ny + 2 * P + 2);
}

int ch_default_params(ch_params_t* p) {
  if (!p) return CH_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->nx = 16; p->ny = 65; p->nz = 16;
  p->lx = 2.67; p->lz = 0.8;
  p->re_tau = 180.0; p->re_bulk = 2800.0;
  p->dt = 0.005;
  p->steps_per_action = 1;
  p->y_sense_plus = 15.0;
  p->top_bc = 0; p->precision = 0; p->control = 0;
  p->alpha = 1.0; p->tau_ref = 0.0; p->batch = 1;
  p->autotune = 1;
  return CH_OK;
}

const char* ch_strerror(int code) {
  switch (code) {
    case CH_OK: return "ok";
    case CH_ERR_ARG: return "invalid argument";
    case CH_ERR_OOM: return "out of memory";
    case CH_ERR_BUDGET: return "memory budget exceeded";
    case CH_ERR_DIVERGED: return "flow diverged (non-finite wall shear)";
    case CH_ERR_TIMEOUT: return "bounded wait timed out";
    case CH_ERR_STATE: return "call not valid in this state";
    case CH_ERR_CUDA: return "CUDA runtime error";
    case CH_ERR_UNSUPPORTED: return "unsupported parameter combination";
    default: return "unknown error";
  }
}

int env_create(const ch_params_t* p, ch_env_t** out) {
  if (!out) return CH_ERR_ARG;
  *out = nullptr;
  RC(check_params(p));
  ch_env* env = new (std::nothrow) ch_env();
  if (!env) return CH_ERR_OOM;
  env->prm = *p;
  env->B = p->batch > 0 ? p->batch : 1;
  env->prm.batch = env->B;
  Grid& g = env->g;
  g.nx = p->nx; g.ny = p->ny; g.nz = p->nz; g.nxh = p->nx / 2; g.P = g.nz * g.nxh; g.N = p->ny - 1;
  g.mx = 3 * p->nx / 2; g.mz = 3 * p->nz / 2;
  env->nu = channel_height(p) / p->re_bulk;
  env->u_tau = p->re_tau / p->re_bulk;
  env->tau_ref = p->tau_ref > 0 ? p->tau_ref : env->u_tau * env->u_tau;
  env->js = sensing_node(g.N, p->re_tau, p->y_sense_plus, channel_height(p));
  env->t.assign(env->B, 0.0);
  env->steps.assign(env->B, 0.0);
  int rc = CH_OK;
  auto fail = [&](int code) { free_env(env); return code; };
  if (cudaStreamCreateWithFlags(&env->own_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(CH_ERR_CUDA);
  env->stream = env->own_stream;
  const size_t B = env->B, P = g.P, ny = g.ny;
  PencilBufs& pb = env->pb;
  if ((rc = dalloc(env, &pb.V, B * ny * P)) || (rc = dalloc(env, &pb.G, B * ny * P)) ||
      (rc = dalloc(env, &pb.HVP, B * ny * P)) || (rc = dalloc(env, &pb.HGP, B * ny * P)) ||
      (rc = dalloc(env, &pb.UM, B * ny)) || (rc = dalloc(env, &pb.WM, B * ny)) ||
      (rc = dalloc(env, &pb.HXP, B * ny)) || (rc = dalloc(env, &pb.HZP, B * ny)) ||
      (rc = dalloc(env, &pb.Q, B * 6 * ny * P)) || (rc = dalloc(env, &pb.R, B * 3 * ny * P)) ||
      (rc = dalloc(env, &pb.vw_old, B * P)) || (rc = dalloc(env, &pb.vw_new, B * P)) ||
      (rc = dalloc(env, &pb.planes, B * 2 * P)) || (rc = dalloc(env, &pb.tau_acc, B)))
    return fail(rc);
  env->out_stride = (size_t)2 * g.nz * g.nx + 2;
  if ((rc = dalloc(env, &env->d_act, B * g.nz * g.nx)) || (rc = dalloc(env, &env->d_out, B * env->out_stride)))
    return fail(rc);
  if (p->control == 2 && ((rc = dalloc(env, &env->d_pol_w, (size_t)kPolicyMaxWeights)) ||
                          (rc = dalloc(env, &env->d_pol_in, B * 2 * g.nz * g.nx))))
    return fail(rc);
  if (cudaMallocHost(&env->h_out, B * env->out_stride * sizeof(double)) != cudaSuccess) return fail(CH_ERR_OOM);
  if ((rc = build_tables(env))) return fail(rc);
  {
    int smem_max = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return fail(CH_ERR_CUDA);
    // per-tile width: 8 modes per CTA, fewer while that leaves fewer CTAs
    // than SMs (a single small channel) or exceeds the shared memory
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    env->ppc_post = 8;
    while (env->ppc_post > 1 && ((size_t)B * P + env->ppc_post - 1) / env->ppc_post < (size_t)nsm)
      env->ppc_post /= 2;
    while (env->ppc_post > 1 && stage_post_smem(g, env->tab.tau.Mh, env->ppc_post, p->top_bc) > (size_t)smem_max)
      env->ppc_post /= 2;
    env->ppc_pre = 8;
    while (env->ppc_pre > 1 && stage_pre_smem(g, env->ppc_pre, sizeof(double2)) > (size_t)smem_max) env->ppc_pre /= 2;
    if (stage_post_smem(g, env->tab.tau.Mh, env->ppc_post, p->top_bc) > (size_t)smem_max) return fail(CH_ERR_UNSUPPORTED);
    // The batched form of stage_post runs four threads per mode, each with
    // the same work; it pays once the batch supplies at least two such warps
    // per SM sub-partition (B P / 8 >= 2 x 4 x SMs).
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return fail(CH_ERR_CUDA);
    const size_t node = p->precision == 1 ? sizeof(float2) : sizeof(double2);
    if ((size_t)B * P >= (size_t)64 * sms && stage_post_batched_smem(g, 8, p->top_bc, node) <= (size_t)smem_max) {
      env->post_batched = true;
      env->ppc_post = 16;  // 64 threads; 8 when the tile would leave fewer than 3 CTAs per SM
      if (stage_post_batched_smem(g, 16, p->top_bc, node) > (size_t)76 * 1024) env->ppc_post = 8;
    }
    if (p->autotune && (rc = autotune_tiles(env, smem_max))) return fail(rc);
  }
  // laminar Poiseuille (the half-Poiseuille profile under a free-slip top), zero wall action
  std::vector<double> st(ch_state_bytes(p) / sizeof(double), 0.0);
  fill_seed_state(p, 0, 0.0, 0, st.data());
  for (int e = 0; e < env->B; ++e)
    if ((rc = set_state_dev(env, e, st.data()))) return fail(rc);
  if (cudaMemset(pb.vw_old, 0, B * P * sizeof(double2)) != cudaSuccess) return fail(CH_ERR_CUDA);
  if (cudaMemset(pb.tau_acc, 0, B * sizeof(double)) != cudaSuccess) return fail(CH_ERR_CUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(CH_ERR_CUDA);
  set_launch_count(env);
  *out = env;
  return CH_OK;
}

int env_set_stream(ch_env_t* env, void* stream) {
  if (!env) return CH_ERR_ARG;
  if (cudaStreamSynchronize(env->stream) != cudaSuccess) return CH_ERR_CUDA;
  env->stream = stream ? static_cast<cudaStream_t>(stream) : env->own_stream;
  return CH_OK;
}

int ch_seed_state(const ch_params_t* p, uint64_t seed, double amplitude, int kmax, void* buf, size_t nbytes) {
  if (!p || !buf) return CH_ERR_ARG;
  if (p->nx < 4 || p->nz < 4 || (p->nx & 1) || (p->nz & 1) || p->ny < 5) return CH_ERR_ARG;
  if (nbytes < ch_state_bytes(p)) return CH_ERR_ARG;
  fill_seed_state(p, seed, amplitude, kmax, static_cast<double*>(buf));
  return CH_OK;
}

int env_reset(ch_env_t* env, uint64_t seed, double amplitude, int kmax) {
  if (!env) return CH_ERR_ARG;
  std::vector<double> st(ch_state_bytes(&env->prm) / sizeof(double));
  for (int e = 0; e < env->B; ++e) {
    fill_seed_state(&env->prm, seed + (uint64_t)e, amplitude, kmax, st.data());
    RC(set_state_dev(env, e, st.data()));
  }
  return CH_OK;
}

int env_get_state(ch_env_t* env, int e, void* buf, size_t nbytes) {
  if (!env || !buf || e < 0 || e >= env->B) return CH_ERR_ARG;
  if (nbytes < ch_state_bytes(&env->prm)) return CH_ERR_ARG;
  const Grid& g = env->g;
  const size_t P = g.P, ny = g.ny;
  double* v = static_cast<double*>(buf);
  double* gg = v + 2 * ny * P;
  double* U = gg + 2 * ny * P;
  double* W = U + ny;
  double* vw = W + ny;
  double* tail = vw + 2 * P;
  cudaStream_t st = env->stream;
  CK(cudaMemcpyAsync(v, env->pb.V + (size_t)e * ny * P, ny * P * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(gg, env->pb.G + (size_t)e * ny * P, ny * P * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(U, env->pb.UM + (size_t)e * ny, ny * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(W, env->pb.WM + (size_t)e * ny, ny * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(vw, env->pb.vw_new + (size_t)e * P, P * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  tail[0] = env->t[e];
  tail[1] = env->steps[e];
  return CH_OK;
}

int env_set_state(ch_env_t* env, int e, const void* buf, size_t nbytes) {
  if (!env || !buf || e < 0 || e >= env->B) return CH_ERR_ARG;
  if (nbytes < ch_state_bytes(&env->prm)) return CH_ERR_ARG;
  return set_state_dev(env, e, static_cast<const double*>(buf));
}

int env_step_device(ch_env_t* env, const double* d_action, double* d_out) {
  if (!env || !d_out) return CH_ERR_ARG;
  if (env->prm.control == 0 && !d_action) return CH_ERR_ARG;
  return run_step(env, d_action, d_out);
}

// true iff no value is an infinity or a NaN (exponent field all ones); one
// branch-free pass over the encodings
static bool all_finite(const double* a, size_t n) {
  constexpr uint64_t kExp = 0x7ff0000000000000ull;
  uint64_t bad = 0;
  for (size_t i = 0; i < n; ++i) {
    uint64_t u;
    std::memcpy(&u, a + i, sizeof(u));
    bad |= (uint64_t)((u & kExp) == kExp);
  }
  return bad == 0;
}

// The observation rows of d_out go straight to the caller's array (one
// pitched copy); the wall shear and reward of every environment, adjacent in
// each row, come back as pairs into the pinned h_out and are scattered.
static cudaError_t fetch_outputs(ch_env* env, double* obs) {
  const size_t B = env->B, plane = (size_t)env->g.nz * env->g.nx, pitch = env->out_stride * sizeof(double);
  cudaStream_t st = env->stream;
  cudaError_t e = cudaSuccess;
  if (obs) e = cudaMemcpy2DAsync(obs, 2 * plane * sizeof(double), env->d_out, pitch, 2 * plane * sizeof(double), B,
                                 cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(env->h_out, 2 * sizeof(double), env->d_out + 2 * plane, pitch, 2 * sizeof(double), B,
                          cudaMemcpyDeviceToHost, st);
  return e;
}

int env_step(ch_env_t* env, const double* action, double* obs, double* wall_shear, double* reward) {
  if (!env) return CH_ERR_ARG;
  if (env->prm.control == 0 && !action) return CH_ERR_ARG;
  const Grid& g = env->g;
  const size_t B = env->B, plane = (size_t)g.nz * g.nx;
  cudaStream_t st = env->stream;
  if (env->prm.control == 0) {
    if (!all_finite(action, B * plane)) return CH_ERR_ARG;  // poisoned action: reject before any work
    CK(cudaMemcpyAsync(env->d_act, action, B * plane * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  RC(run_step(env, env->d_act, env->d_out));
  CK(fetch_outputs(env, obs));
  CK(cudaStreamSynchronize(st));
  int rc = CH_OK;
  for (size_t b = 0; b < B; ++b) {
    const double tau = env->h_out[2 * b], rew = env->h_out[2 * b + 1];
    if (wall_shear) wall_shear[b] = tau;
    if (reward) reward[b] = rew;
    if (!std::isfinite(tau)) rc = CH_ERR_DIVERGED;
  }
  return rc;
}

int env_info(const ch_env_t* env, ch_info_t* info) {
  if (!env || !info) return CH_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  info->j_sense = env->js;
  info->y_plus_sense = (1.0 + std::cos(M_PI * env->js / env->g.N)) * env->prm.re_tau / channel_height(&env->prm);
  info->nu = env->nu;
  info->u_tau = env->u_tau;
  info->tau_ref = env->tau_ref;
  info->state_bytes = ch_state_bytes(&env->prm);
  info->device_bytes = env->device_bytes;
  info->plane_cluster = env->prm.precision == 1 ? (env->plane_f.two_pass ? 0 : env->plane_f.S)
                                               : (env->plane.two_pass ? 0 : env->plane.S);
  info->launches_per_step = env->launches_per_step;
  info->post_batched = env->post_batched ? 1 : 0;
  info->ppc_pre = env->ppc_pre;
  info->ppc_post = env->ppc_post;
  info->tuned = env->tuned ? 1 : 0;
  info->tune_ms = env->tune_ms;
  info->plane_team = env->prm.precision == 1 ? env->plane_f.team16 : env->plane.team16;
  return CH_OK;
}

int env_set_tiles(ch_env_t* env, int ppc_pre, int ppc_post, int post_batched) {
  if (!env) return CH_ERR_ARG;
  int smem_max = 0, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (!tiles_valid(env, smem_max, ppc_pre, ppc_post, post_batched)) return CH_ERR_ARG;
  CK(cudaStreamSynchronize(env->stream));
  RC(drop_graphs(env));
  env->ppc_pre = ppc_pre;
  env->ppc_post = ppc_post;
  env->post_batched = post_batched == 1;
  env->tuned = false;
  set_launch_count(env);
  return CH_OK;
}

int env_set_policy(ch_env_t* env, const ch_policy_t* pol, const double* weights, size_t n_weights) {
  if (!env || !pol || !weights) return CH_ERR_ARG;
  if (env->prm.control != 2) return CH_ERR_STATE;
  const Grid& g = env->g;
  auto odd_side = [](int w, int n) { return w >= 1 && w <= kPolicyMaxWindow && (w & 1) && w <= n; };
  auto width = [](int h) { return h >= 1 && h <= kPolicyMaxWidth; };
  if (!odd_side(pol->wz, g.nz) || !odd_side(pol->wx, g.nx)) return CH_ERR_ARG;
  if (pol->n_hidden < 0 || pol->n_hidden > 2 || (pol->out_tanh != 0 && pol->out_tanh != 1)) return CH_ERR_ARG;
  if (pol->n_hidden >= 1 && !width(pol->width[0])) return CH_ERR_ARG;
  if (pol->n_hidden == 2 && !width(pol->width[1])) return CH_ERR_ARG;
  PolicyDesc d{};
  d.wz = pol->wz;
  d.wx = pol->wx;
  d.n_hidden = pol->n_hidden;
  d.h1 = pol->n_hidden >= 1 ? pol->width[0] : 0;
  d.h2 = pol->n_hidden == 2 ? pol->width[1] : 0;
  d.out_tanh = pol->out_tanh;
  d.n_weights = policy_weight_count(d);
  if (n_weights != (size_t)d.n_weights || d.n_weights > kPolicyMaxWeights) return CH_ERR_ARG;
  std::vector<float> w(n_weights);
  for (size_t i = 0; i < n_weights; ++i) {
    if (!std::isfinite(weights[i])) return CH_ERR_ARG;
    w[i] = (float)weights[i];
  }
  CK(cudaStreamSynchronize(env->stream));
  CK(cudaMemcpy(env->d_pol_w, w.data(), n_weights * sizeof(float), cudaMemcpyHostToDevice));
  RC(drop_graphs(env));  // the captured launches hold the previous descriptor
  env->pol = d;
  env->pol_set = true;
  return CH_OK;
}

int env_observe(ch_env_t* env, double* obs) {
  if (!env || !obs) return CH_ERR_ARG;
  const Grid& g = env->g;
  const size_t plane = (size_t)g.nz * g.nx;
  cudaStream_t st = env->stream;
  // the same kernels and buffers as the end of a step: the sensing-plane
  // spectra, then the observation planes into the output rows
  CK(launch_sense(g, env->B, env->pb, env->tab, env->js, env->prm.alpha, 0, st));
  CK(launch_obs(g, env->B, env->pb.planes, env->tab, env->d_out, env->out_stride, nullptr, st));
  CK(cudaMemcpy2DAsync(obs, 2 * plane * sizeof(double), env->d_out, env->out_stride * sizeof(double),
                       2 * plane * sizeof(double), env->B, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return CH_OK;
}

int env_get_action(ch_env_t* env, double* action) {
  if (!env || !action) return CH_ERR_ARG;
  if (env->prm.control == 1) return CH_ERR_STATE;
  const size_t n = (size_t)env->B * env->g.nz * env->g.nx;
  CK(cudaMemcpyAsync(action, env->d_act, n * sizeof(double), cudaMemcpyDeviceToHost, env->stream));
  CK(cudaStreamSynchronize(env->stream));
  return CH_OK;
}

int env_profile(ch_env_t* env, int enable) {
  if (!env) return CH_ERR_ARG;
  env->prof = enable != 0;
  for (int c = 0; c < 4; ++c) env->ev_used[c] = 0;
  return CH_OK;
}

int env_profile_read(ch_env_t* env, int cls, double* total_ms, int* launches) {
  if (!env || cls < 0 || cls > 3) return CH_ERR_ARG;
  if (cudaStreamSynchronize(env->stream) != cudaSuccess) return CH_ERR_CUDA;
  double tot = 0.0;
  for (int i = 0; i < env->ev_used[cls]; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, env->ev[cls][i].first, env->ev[cls][i].second) != cudaSuccess) return CH_ERR_CUDA;
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = env->ev_used[cls];
  return CH_OK;
}

int env_destroy(ch_env_t* env) {
  if (!env) return CH_ERR_ARG;
  free_env(env);
  return CH_OK;
}

int ch_nonlinear(ch_env_t* env, const double* d_q, double* d_h) {
  if (!env || !d_q || !d_h) return CH_ERR_ARG;
  if (env->plane.S == 0) return CH_ERR_UNSUPPORTED;
  PlaneArgs<double> a = env->plane;
  a.q = reinterpret_cast<const double2*>(d_q);
  a.h = reinterpret_cast<double2*>(d_h);
  CK(launch_plane<double>(a, env->B, env->plane_smem, env->stream));
  return CH_OK;
}

int ch_tau_helmholtz(int ny, int M, const double* d_lam, const double* d_r, const double* d_top,
                     const double* d_bot, double* d_f, void* stream) {
  if (ny < 5 || ny > kMaxNy || M < 0) return CH_ERR_ARG;
  if (M == 0) return CH_OK;
  if (!d_lam || !d_r || !d_top || !d_bot || !d_f) return CH_ERR_ARG;
  CK(launch_tau_helmholtz(ny, M, d_lam, reinterpret_cast<const double2*>(d_r),
                          reinterpret_cast<const double2*>(d_top), reinterpret_cast<const double2*>(d_bot),
                          reinterpret_cast<double2*>(d_f), static_cast<cudaStream_t>(stream)));
  return CH_OK;
}

}  // extern "C"
