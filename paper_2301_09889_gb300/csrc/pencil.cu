// The small kernels of the environment step (action, observation, wall shear,
// reward) and the stateless Chebyshev-tau entry points.  The Runge-Kutta stage
// itself lives in stage_kernels.cuh (wall-normal work) and plane.cu (nonlinear term).
//
// Chebyshev conventions: f(y) = sum_n a_n T_n(y), nodes y_j = cos(pi j / N).
// Derivative recurrence (coefficient space): c_m b_m = b_{m+2} + 2 (m+1) a_{m+1}
// with c_0 = 2, c_m = 1 otherwise, walked from m = N down to 0.
#include <algorithm>
#include <mutex>

#include "../../include/channel_dns.h"
#include "common.cuh"
#include "internal.h"

namespace chdns {

// ---------------------------------------------------------------------------
// Chebyshev-tau Dirichlet problem (D^2 - lam) f = r, split by parity.
//
// For n >= 2 the tau rows are equivalent to the quasi-tridiagonal rows
//   -lam c_{n-2}/(4n(n-1)) f_{n-2} + (1 + lam b_n/(2(n^2-1))) f_n
//   - lam b_{n+2}/(4n(n+1)) f_{n+2}
//     = c_{n-2}/(4n(n-1)) r_{n-2} - b_n/(2(n^2-1)) r_n + b_{n+2}/(4n(n+1)) r_{n+2}
// (b_m = 1 for m <= N-2, else 0: the two highest rows of r are dropped), obtained
// by integrating D^2 f = r + lam f twice.  With parity index i (n = 2i + sig) the
// rows i >= 1 are tridiagonal; the wall row sum_i f_i = s closes the system.
// Elimination from the bottom gives f_i = a_i + b_i f_{i-1}; all f_i are then
// affine in f_0, which the wall row fixes.  The lam-dependent factors
// e_i = 1/den_i, h_i = U_i/den_i, b_i = -L_i/den_i, Q_i = prod b and 1/sum Q
// are precomputed per mode and stage.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tau_cA(int n) { return (n == 2 ? 2.0 : 1.0) / (4.0 * n * (n - 1)); }
__device__ __forceinline__ double tau_cB(int n, int N) { return n <= N - 2 ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0; }
__device__ __forceinline__ double tau_cC(int n, int N) { return n + 2 <= N - 2 ? 1.0 / (4.0 * n * (n + 1)) : 0.0; }

struct TabGlobal {
  const double* base;  // element (field f, index i) at base[(f * Mh + i) * P]
  int Mh, P;
  __device__ double e(int i) const { return base[(size_t)(0 * Mh + i) * P]; }
  __device__ double h(int i) const { return base[(size_t)(1 * Mh + i) * P]; }
  __device__ double b(int i) const { return base[(size_t)(2 * Mh + i) * P]; }
  __device__ double Q(int i) const { return base[(size_t)(3 * Mh + i) * P]; }
};

struct TabLocal {
  const double *pe, *ph, *pb, *pQ;
  __device__ double e(int i) const { return pe[i]; }
  __device__ double h(int i) const { return ph[i]; }
  __device__ double b(int i) const { return pb[i]; }
  __device__ double Q(int i) const { return pQ[i]; }
};

// r[i] = r_{2i+sig}; f[i] receives f_{2i+sig}.  r and f must not alias.
template <class Tab>
__device__ void tau_solve(int N, int sig, const double2* r, double2* f, const Tab& T, double isq, double2 s) {
  const int M = (N - sig) / 2 + 1;
  double2 anext = mk(0.0, 0.0);
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    double2 R = tau_cA(n) * r[i - 1] - tau_cB(n, N) * r[i];
    if (i + 1 < M) R = R + tau_cC(n, N) * r[i + 1];
    const double2 a = T.e(i) * R - T.h(i) * anext;
    f[i] = a;
    anext = a;
  }
  double2 Pp = mk(0.0, 0.0), sum = mk(0.0, 0.0);
  for (int i = 1; i < M; ++i) {
    Pp = f[i] + T.b(i) * Pp;
    f[i] = Pp;
    sum = sum + Pp;
  }
  const double2 f0 = isq * (s - sum);
  f[0] = f0;
  for (int i = 1; i < M; ++i) f[i] = f[i] + T.Q(i) * f0;
}

// on-the-fly factorisation of one parity (for the stateless entry point)
__device__ void tau_factor(int N, int sig, double lam, double* e, double* h, double* b, double* Q, double* isq) {
  const int M = (N - sig) / 2 + 1;
  double bnext = 0.0;
  e[0] = h[0] = b[0] = 0.0;
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    const double L = -lam * tau_cA(n);
    const double Dg = 1.0 + lam * tau_cB(n, N);
    const double U = (i + 1 < M) ? -lam * tau_cC(n, N) : 0.0;
    const double den = Dg + U * bnext;
    e[i] = 1.0 / den;
    h[i] = U / den;
    b[i] = -L / den;
    bnext = b[i];
  }
  Q[0] = 1.0;
  double sq = 1.0;
  for (int i = 1; i < M; ++i) {
    Q[i] = b[i] * Q[i - 1];
    sq += Q[i];
  }
  *isq = 1.0 / sq;
}

// ---------------------------------------------------------------------------
// wall shear of the lower wall: tau_w = nu sum_n U_n T_n'(-1), T_n'(-1) = (-1)^(n+1) n^2
// one warp per environment, fixed summation order
// ---------------------------------------------------------------------------
__global__ void wall_shear_kernel(int ny, int B, const double* UM, double nu, double* acc, const int* active) {
  const int b = blockIdx.x;
  if (b >= B || (active && !active[b])) return;
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int n = lane; n < ny; n += 32) {
    const double d = (double)n * n * ((n & 1) ? 1.0 : -1.0);
    s += d * UM[(size_t)b * ny + n];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) acc[b] += nu * s;
}

// ---------------------------------------------------------------------------
// sensing plane: Fourier coefficients of u and v at node js (and, for
// opposition control, the wall spectrum -alpha v(y_s) with the mean removed,
// paper Sec. 4.1).  One warp per mode: v(y_s) = sum_n v_n T_n(y_s),
// Dv(y_s) = sum_n v_n T_n'(y_s), omega_y(y_s) likewise.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) sense_kernel(Grid g, int B, PencilBufs pb, DevTables t, int js, double alpha,
                                                    int opposition) {
  // 8 lanes per mode (4 modes per warp): the sums over the ny coefficients are
  // split over the lanes and combined by shuffles within the 8-lane group
  constexpr int L = 8;
  const int P = g.P, ny = g.ny;
  const int lane = threadIdx.x & (L - 1);
  const long wid = (blockIdx.x * (long)blockDim.x + threadIdx.x) / L;
  const bool live = wid < (long)P * B;
  const int p = live ? (int)(wid % P) : 0;
  const int b = live ? (int)(wid / P) : 0;
  const bool act = live && !(pb.active && !pb.active[b]);
  auto gsum = [](double v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, L);
    return v;
  };
  auto gsum2 = [&](double2 v) { return mk(gsum(v.x), gsum(v.y)); };
  const int row = p / g.nxh, ix = p % g.nxh;
  const double* cj = t.cheb + (size_t)js * ny;
  // partial sums (only the loads are conditional; every lane of the warp then
  // takes part in the same shuffles)
  double su = 0.0;
  double2 vs = mk(0.0, 0.0), gs = mk(0.0, 0.0), dvs = mk(0.0, 0.0);
  if (act && row != g.nz / 2) {
    if (p == 0) {
      for (int n = lane; n < ny; n += L) su += cj[n] * pb.UM[(size_t)b * ny + n];
    } else {
      const size_t fo = (size_t)b * ny * P + p;
#pragma unroll 8
      for (int n = lane; n < ny; n += L) {
        const double2 vn = pb.V[fo + (size_t)n * P];
        const double2 gn = pb.G[fo + (size_t)n * P];
        vs = vs + cj[n] * vn;
        gs = gs + cj[n] * gn;
        dvs = dvs + t.dts[n] * vn;
      }
    }
  }
  su = gsum(su);
  vs = gsum2(vs);
  gs = gsum2(gs);
  dvs = gsum2(dvs);
  double2 us = mk(0.0, 0.0);
  if (p == 0) {
    us = mk(su, 0.0);
  } else if (row != g.nz / 2) {
    const double kx = t.kx[ix], kz = t.kz[row];
    const double ik2 = 1.0 / (kx * kx + kz * kz);
    us = ik2 * (imul(kx, dvs) - imul(kz, gs));
  }
  if (!act) return;
  if (lane != 0) return;
  if (opposition) {
    // new action: the previous one becomes the start of the ramp, the wall
    // shear average restarts
    const size_t o = (size_t)b * P + p;
    pb.vw_old[o] = pb.vw_new[o];
    pb.vw_new[o] = (p == 0) ? mk(0.0, 0.0) : (-alpha) * vs;
    if (p == 0) pb.tau_acc[b] = 0.0;
  } else {
    pb.planes[((size_t)b * 2 + 0) * P + p] = us;
    pb.planes[((size_t)b * 2 + 1) * P + p] = vs;
  }
}

// ---------------------------------------------------------------------------
// observation planes: unpadded inverse transform of the two sensing-plane
// spectra, f(x_a, z_b) = Re sum_kz F[kz,0] e^{i kz z} + 2 Re sum_{kx>0} F e^{i(kx x + kz z)}.
// One CTA per (block of zblk output rows, field, environment); each row has
// nt / zblk threads.  The z sums t[z_b][kx] are split over nq parts (rows
// q, q + nq, ...) and the x sums of every output over nr parts (kx = 1 + q,
// 1 + q + nr, ...); the parts are added in ascending order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) obs_kernel(int nx, int nz, int nxh, int zblk, const double2* planes,
                                                  const double2* tw_nx, const double2* tw_nz, double* out,
                                                  size_t out_stride, const int* active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tpr = nt / zblk;                 // threads per output row
  const int nq = max(1, tpr / nxh), nr = max(1, tpr / nx);
  double2* part = reinterpret_cast<double2*>(smem_raw);  // [zblk][nq][nxh] z partial sums
  double2* tmp = part + (size_t)zblk * nq * nxh;         // [zblk][nxh]
  double* pr = reinterpret_cast<double*>(tmp + (size_t)zblk * nxh);  // [zblk][nr][nx] x partial sums
  const int z0 = blockIdx.x * zblk, f = blockIdx.y, b = blockIdx.z;
  if (active && !active[b]) return;
  const int P = nz * nxh;
  const double2* F = planes + ((size_t)b * 2 + f) * P;
  for (int w = tid; w < zblk * nq * nxh; w += nt) {
    const int zl = w / (nq * nxh), q = (w / nxh) % nq, i = w % nxh, zb = min(z0 + zl, nz - 1);
    double2 acc = mk(0.0, 0.0);
    int e = (q * zb) % nz;  // (row zb) mod nz; m = row - nz for row > nz/2 gives the same index
    const int step = (nq * zb) % nz;
#pragma unroll 4
    for (int row = q; row < nz; row += nq) {
      if (row != nz / 2) acc = acc + cmul(F[row * nxh + i], tw_nz[e]);
      e += step;
      if (e >= nz) e -= nz;
    }
    part[w] = acc;
  }
  __syncthreads();
  for (int w = tid; w < zblk * nxh; w += nt) {
    const int zl = w / nxh, i = w % nxh;
    const double2* pz = part + (size_t)zl * nq * nxh + i;
    double2 acc = pz[0];
    for (int q = 1; q < nq; ++q) acc = acc + pz[q * nxh];
    tmp[w] = acc;
  }
  __syncthreads();
  for (int w = tid; w < zblk * nr * nx; w += nt) {
    const int zl = w / (nr * nx), q = (w / nx) % nr, xa = w % nx;
    const double2* t = tmp + (size_t)zl * nxh;
    double s = 0.0;
    int e = ((1 + q) * xa) % nx;  // (kx xa) mod nx
    const int step = (nr * xa) % nx;
    for (int i = 1 + q; i < nxh; i += nr) {
      const double2 tw = tw_nx[e];
      const double2 v = t[i];
      s += v.x * tw.x - v.y * tw.y;
      e += step;
      if (e >= nx) e -= nx;
    }
    pr[w] = s;
  }
  __syncthreads();
  for (int w = tid; w < zblk * nx; w += nt) {
    const int zl = w / nx, xa = w % nx, zb = z0 + zl;
    if (zb >= nz) continue;
    const double* px = pr + (size_t)zl * nr * nx + xa;
    double s = 0.0;
    for (int q = 0; q < nr; ++q) s += px[q * nx];
    out[(size_t)b * out_stride + (size_t)f * nz * nx + (size_t)zb * nx + xa] = tmp[zl * nxh].x + 2.0 * s;
  }
}

// ---------------------------------------------------------------------------
// wall action -> wall spectrum: clip to [-u_tau, u_tau] (paper Sec. 3.2),
// forward transform of the kept modes; the mean mode (zero net mass flux,
// Sec. 4.1) and the Nyquist row are zero.  Removing the plane mean before the
// transform changes only the mean mode, which is set to zero, so it is not
// computed.  Two passes through a scratch plane tx[b][z][kx], one thread per
// output coefficient, each sum in ascending order:
//   action_x_kernel: x transform of the clipped rows; also starts the new
//                    action (the previous spectrum becomes the start of the
//                    ramp, the wall-shear average restarts);
//   action_z_kernel: z transform.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) action_x_kernel(int nx, int nz, int nxh, int B, const double* act,
                                                       double u_tau, const double2* tw_nx, double2* tx,
                                                       double2* vw_old, const double2* vw, double* acc,
                                                       const int* active) {
  const int P = nz * nxh;
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;  // (b, z, kx), kx fastest
  if (w >= (long)B * P) return;
  const int b = (int)(w / P), o = (int)(w % P), zb = o / nxh, i = o % nxh;
  if (active && !active[b]) return;
  const size_t bo = (size_t)b * P + o;
  vw_old[bo] = vw[bo];
  if (o == 0) acc[b] = 0.0;
  const double* src = act + ((size_t)b * nz + zb) * nx;
  double2 s = mk(0.0, 0.0);
  int e = 0;  // (i xa) mod nx
#pragma unroll 8
  for (int xa = 0; xa < nx; ++xa) {
    s = s + fmin(fmax(src[xa], -u_tau), u_tau) * cconj(tw_nx[e]);
    e += i;
    if (e >= nx) e -= nx;
  }
  tx[bo] = s;
}

__global__ void __launch_bounds__(128) action_z_kernel(int nx, int nz, int nxh, int B, const double2* tx,
                                                       const double2* tw_nz, double2* vw, const int* active) {
  const int P = nz * nxh;
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;  // (b, kz row, kx), kx fastest
  if (w >= (long)B * P) return;
  const int b = (int)(w / P), o = (int)(w % P), row = o / nxh, i = o % nxh;
  if (active && !active[b]) return;
  const double sc = 1.0 / ((double)nx * nz);
  double2 s = mk(0.0, 0.0);
  if (row != nz / 2 && !(row == 0 && i == 0)) {
    const int m = row < nz / 2 ? row : row - nz;
    const int step = m < 0 ? m + nz : m;  // (m zb) mod nz advances by m mod nz
    int e = 0;
#pragma unroll 8
    for (int zb = 0; zb < nz; ++zb) {
      s = s + cmul(tx[(size_t)b * P + (size_t)zb * nxh + i], cconj(tw_nz[e]));
      e += step;
      if (e >= nz) e -= nz;
    }
    s = sc * s;
  }
  vw[(size_t)b * P + o] = s;
}

__global__ void finalize_kernel(int B, const double* acc, double inv_steps, double tau_ref, double* out,
                                size_t out_stride, size_t out_offset, const int* active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  const double tau = acc[b] * inv_steps;
  out[(size_t)b * out_stride + out_offset] = tau;
  out[(size_t)b * out_stride + out_offset + 1] = 1.0 - tau / tau_ref;
}

// stateless tau problems: one thread per (problem, parity)
__global__ void tau_helmholtz_kernel(int ny, int M, const double* lam, const double2* r, const double2* top,
                                     const double2* bot, double2* f) {
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * M) return;
  const int m = (int)(tid / 2), sig = (int)(tid % 2);
  const int N = ny - 1;
  double e[kMaxHalf], h[kMaxHalf], bb[kMaxHalf], Q[kMaxHalf], isq;
  tau_factor(N, sig, lam[m], e, h, bb, Q, &isq);
  const int Mp = (N - sig) / 2 + 1;
  double2 rr[kMaxHalf], ff[kMaxHalf];
  for (int i = 0; i < Mp; ++i) rr[i] = r[(size_t)m * ny + 2 * i + sig];
  const double2 s = sig == 0 ? 0.5 * (top[m] + bot[m]) : 0.5 * (top[m] - bot[m]);
  tau_solve(N, sig, rr, ff, TabLocal{e, h, bb, Q}, isq, s);
  for (int i = 0; i < Mp; ++i) f[(size_t)m * ny + 2 * i + sig] = ff[i];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_wall_shear(const Grid& g, int B, const double* UM, double nu, double* acc, const int* active,
                              cudaStream_t st) {
  wall_shear_kernel<<<B, 32, 0, st>>>(g.ny, B, UM, nu, acc, active);
  return cudaGetLastError();
}

cudaError_t launch_sense(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, int js, double alpha,
                         int opposition, cudaStream_t st) {
  const long threads = (long)g.P * B * 8;  // 8 lanes per mode
  sense_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(g, B, pb, t, js, alpha, opposition);
  return cudaGetLastError();
}

cudaError_t launch_obs(const Grid& g, int B, const double2* planes, const DevTables& t, double* out,
                       size_t out_stride, const int* active, cudaStream_t st) {
  // several output rows per CTA once the batch alone gives 128 or more
  // (environment, field) CTAs; otherwise one row per CTA, its sums split over
  // the CTA's threads
  const int zblk = B >= 64 ? std::max(1, std::min(g.nz, 128 / g.nxh)) : 1;
  const int tpr = 128 / zblk;
  const int nq = std::max(1, tpr / g.nxh), nr = std::max(1, tpr / g.nx);
  const size_t smem = (size_t)zblk * ((nq + 1) * g.nxh * sizeof(double2) + (size_t)nr * g.nx * sizeof(double));
  obs_kernel<<<dim3((g.nz + zblk - 1) / zblk, 2, B), 128, smem, st>>>(g.nx, g.nz, g.nxh, zblk, planes, t.tw_nx,
                                                                       t.tw_nz, out, out_stride, active);
  return cudaGetLastError();
}

cudaError_t launch_action(const Grid& g, int B, const double* act, double u_tau, const DevTables& t,
                          const PencilBufs& pb, cudaStream_t st) {
  // the sensing-plane buffer is free at this point of the step: it is the scratch plane
  double2* tx = pb.planes;
  const long n = (long)B * g.nz * g.nxh;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  action_x_kernel<<<blocks, 128, 0, st>>>(g.nx, g.nz, g.nxh, B, act, u_tau, t.tw_nx, tx, pb.vw_old, pb.vw_new,
                                          pb.tau_acc, pb.active);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  action_z_kernel<<<blocks, 128, 0, st>>>(g.nx, g.nz, g.nxh, B, tx, t.tw_nz, pb.vw_new, pb.active);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int B, const double* acc, double inv_steps, double tau_ref, double* out,
                            size_t out_stride, size_t out_offset, const int* active, cudaStream_t st) {
  finalize_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, acc, inv_steps, tau_ref, out, out_stride, out_offset, active);
  return cudaGetLastError();
}

cudaError_t launch_tau_helmholtz(int ny, int M, const double* lam, const double2* r, const double2* top,
                                 const double2* bot, double2* f, cudaStream_t st) {
  const long n = 2L * M;
  tau_helmholtz_kernel<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(ny, M, lam, r, top, bot, f);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the stateless tau entry point.
//
// tau_helmholtz_kernel above keeps each problem's factorisation and work
// vectors (about 6.5 KB per thread) in local memory, which the CUDA driver
// allocates and may have to grow at launch time.  Some callers cannot let
// anything allocate device memory: a control loop with a fixed real-time
// budget (cudaMalloc and a driver-side resize can block for milliseconds and
// synchronise the device), a process whose device memory is already fully
// handed to another allocator's pool, or a host framework that only lends out
// buffers it owns.  For them the work vectors live in one file-scope array
// below, sized once when the library is loaded.
// ---------------------------------------------------------------------------
}  // namespace chdns

// 16 MiB of doubles, held by every GPU that loads the library until the
// process exits.  Shared by all calls; a call writes every slot it reads, so
// nothing has to start at zero.
constexpr size_t kNoAllocScratchDoubles = (size_t)2 << 20;
static __device__ __align__(256) double g_tau_noalloc_scratch[kNoAllocScratchDoubles];

namespace chdns {

__global__ void tau_helmholtz_noalloc_kernel(int ny, int M, int mpad, const double* lam, const double2* r,
                                             const double2* top, const double2* bot, double2* f,
                                             double* scratch) {
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * M) return;
  const int m = (int)(tid / 2), sig = (int)(tid % 2);
  const int N = ny - 1;
  // slot layout: e, h, b, Q (mpad doubles each), then r and f (mpad complex each)
  double* base = scratch + (size_t)tid * 8 * mpad;
  double* e = base;
  double* h = base + mpad;
  double* bb = base + 2 * mpad;
  double* Q = base + 3 * mpad;
  double2* rr = reinterpret_cast<double2*>(base + 4 * mpad);
  double2* ff = reinterpret_cast<double2*>(base + 6 * mpad);
  double isq;
  tau_factor(N, sig, lam[m], e, h, bb, Q, &isq);
  const int Mp = (N - sig) / 2 + 1;
  for (int i = 0; i < Mp; ++i) rr[i] = r[(size_t)m * ny + 2 * i + sig];
  const double2 s = sig == 0 ? 0.5 * (top[m] + bot[m]) : 0.5 * (top[m] - bot[m]);
  tau_solve(N, sig, rr, ff, TabLocal{e, h, bb, Q}, isq, s);
  for (int i = 0; i < Mp; ++i) f[(size_t)m * ny + 2 * i + sig] = ff[i];
}

}  // namespace chdns

namespace {

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CH_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tau_noalloc_scratch) != cudaSuccess || !p) return CH_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return CH_OK;
}

}  // namespace

extern "C" int ch_tau_helmholtz_noalloc(int ny, int M, const double* d_lam, const double* d_r,
                                        const double* d_top, const double* d_bot, double* d_f, void* stream) {
  if (ny < 5 || ny > chdns::kMaxNy || M < 0) return CH_ERR_ARG;
  if (M == 0) return CH_OK;
  if (!d_lam || !d_r || !d_top || !d_bot || !d_f) return CH_ERR_ARG;
  const int mpad = ((ny / 2 + 1) + 1) & ~1;  // even, keeps the complex work vectors 16-byte aligned
  if ((size_t)2 * M * 8 * mpad > kNoAllocScratchDoubles) return CH_ERR_ARG;
  double* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc != CH_OK) return rc;
  const long n = 2L * M;
  chdns::tau_helmholtz_noalloc_kernel<<<(unsigned)((n + 63) / 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(
      ny, M, mpad, d_lam, reinterpret_cast<const double2*>(d_r), reinterpret_cast<const double2*>(d_top),
      reinterpret_cast<const double2*>(d_bot), reinterpret_cast<double2*>(d_f), scratch);
  return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}
