// Warp-cooperative wall-normal operations on one Fourier mode.
//
// A warp owns one (mode, symmetry class).  The coefficients of one parity
// (n = 2i + sig) are spread cyclically over the lanes: lane l holds the parity
// indices i = 32 k + l for k < K.  Sequential recurrences of the
// coefficient-space algorithms become warp scans:
//   - the Chebyshev derivative b_m = sum_{n > m, n + m odd} 2 n a_n (b_0 halved)
//     is a suffix sum over the parity chain;
//   - the two elimination sweeps of the quasi-tridiagonal tau system are
//     compositions of affine maps x -> alpha + beta x, i.e. a suffix scan
//     (bottom-up sweep) and a prefix scan (top-down sweep);
//   - sums over coefficients (wall row, influence matrix, flow rate) are
//     butterfly reductions.
// Every lane of the warp must call these functions together.
#pragma once

#include "common.cuh"

namespace chdns {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double2 shfl_down2(double2 v, int off) {
  return mk(__shfl_down_sync(kFull, v.x, off), __shfl_down_sync(kFull, v.y, off));
}
__device__ __forceinline__ double2 shfl_up2(double2 v, int off) {
  return mk(__shfl_up_sync(kFull, v.x, off), __shfl_up_sync(kFull, v.y, off));
}
__device__ __forceinline__ double2 shfl_idx2(double2 v, int src) {
  return mk(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + shfl_idx2(v, (threadIdx.x & 31) ^ o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// number of coefficients of parity sig among n = 0..N
__device__ __forceinline__ int par_count(int N, int sig) { return (N - sig) / 2 + 1; }

// ---- loads / stores of one parity of a y-major array (element n at base[n * stride])
template <int K>
__device__ __forceinline__ void load_par(double2 (&x)[K], const double2* base, size_t stride, int sig, int M,
                                         int lane) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    x[k] = (i < M) ? base[(size_t)(2 * i + sig) * stride] : mk(0.0, 0.0);
  }
}
template <int K>
__device__ __forceinline__ void store_par(double2* base, size_t stride, int sig, int M, int lane,
                                          const double2 (&x)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    if (i < M) base[(size_t)(2 * i + sig) * stride] = x[k];
  }
}
template <int K>
__device__ __forceinline__ void load_par_real(double2 (&x)[K], const double* base, int sig, int M, int lane) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    x[k] = mk((i < M) ? base[2 * i + sig] : 0.0, 0.0);
  }
}
template <int K>
__device__ __forceinline__ void store_par_real(double* base, int sig, int M, int lane, const double2 (&x)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    if (i < M) base[2 * i + sig] = x[k].x;
  }
}

// ---- coefficient-space derivative: a has parity sig (Msrc entries), d gets
// parity 1 - sig (Mdst entries).  d_j = sum_{i >= j + 1 - sig} 2 (2i + sig) a_i,
// halved at n = 0.
template <int K>
__device__ __forceinline__ void deriv(const double2 (&a)[K], double2 (&d)[K], int sig, int Msrc, int Mdst,
                                      int lane) {
  double2 S[K];
  double2 carry = mk(0.0, 0.0);
#pragma unroll
  for (int k = K - 1; k >= 0; --k) {
    const int i = 32 * k + lane;
    double2 x = (i < Msrc) ? (2.0 * (2 * i + sig)) * a[k] : mk(0.0, 0.0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double2 t = shfl_down2(x, off);
      if (lane + off < 32) x = x + t;
    }
    S[k] = x + carry;
    carry = carry + shfl_idx2(x, 0);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = 32 * k + lane;
    double2 v = S[k];
    if (sig == 0) {  // d_j = S_{j+1}
      const double2 dn = shfl_down2(S[k], 1);
      double2 nx = mk(0.0, 0.0);
      if (k + 1 < K) nx = shfl_idx2(S[k + 1 < K ? k + 1 : k], 0);
      v = (lane < 31) ? dn : nx;
    }
    if (j >= Mdst) v = mk(0.0, 0.0);
    if (sig == 1 && j == 0) v = 0.5 * v;
    d[k] = v;
  }
}

// ---- affine maps x -> a + b x (a complex, b real)
struct Aff {
  double2 a;
  double b;
};
__device__ __forceinline__ Aff compose(const Aff& f, const Aff& g) {  // f(g(x))
  return Aff{f.a + f.b * g.a, f.b * g.b};
}
__device__ __forceinline__ Aff shfl_down_aff(const Aff& v, int off) {
  return Aff{shfl_down2(v.a, off), __shfl_down_sync(kFull, v.b, off)};
}
__device__ __forceinline__ Aff shfl_up_aff(const Aff& v, int off) {
  return Aff{shfl_up2(v.a, off), __shfl_up_sync(kFull, v.b, off)};
}
__device__ __forceinline__ Aff shfl_idx_aff(const Aff& v, int src) {
  return Aff{shfl_idx2(v.a, src), __shfl_sync(kFull, v.b, src)};
}

__device__ __forceinline__ double tau_ca(int n) { return (n == 2 ? 2.0 : 1.0) / (4.0 * n * (n - 1)); }
__device__ __forceinline__ double tau_cb(int n, int N) { return n <= N - 2 ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0; }
__device__ __forceinline__ double tau_cc(int n, int N) { return n + 2 <= N - 2 ? 1.0 / (4.0 * n * (n + 1)) : 0.0; }

// Tau factor tables of one (mode, parity), pencil-major: e, h, b, Q blocks of Mh.
struct TabP {
  const double* base;
  int Mh;
  __device__ double e(int i) const { return base[i]; }
  __device__ double h(int i) const { return base[Mh + i]; }
  __device__ double b(int i) const { return base[2 * Mh + i]; }
  __device__ double Q(int i) const { return base[3 * Mh + i]; }
};

// Quasi-tridiagonal Chebyshev-tau Dirichlet solve of one parity (see the
// sequential version in pencil.cu for the rows): r, f in parity layout,
// s = the wall-row sum.
template <int K>
__device__ void tau_solve_warp(int N, int sig, const double2 (&r)[K], double2 (&f)[K], const TabP& T, double isq,
                               double2 s, int lane) {
  const int M = par_count(N, sig);
  double2 R[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    const int n = 2 * i + sig;
    const double2 up = shfl_up2(r[k], 1);
    double2 prev = mk(0.0, 0.0);
    if (k > 0) prev = shfl_idx2(r[k > 0 ? k - 1 : 0], 31);
    const double2 rm = (lane > 0) ? up : prev;
    const double2 dn = shfl_down2(r[k], 1);
    double2 next = mk(0.0, 0.0);
    if (k + 1 < K) next = shfl_idx2(r[k + 1 < K ? k + 1 : k], 0);
    const double2 rp = (lane < 31) ? dn : next;
    double2 v = mk(0.0, 0.0);
    if (i >= 1 && i < M) {
      v = tau_ca(n) * rm - tau_cb(n, N) * r[k];
      if (i + 1 < M) v = v + tau_cc(n, N) * rp;
    }
    R[k] = v;
  }
  // bottom-up sweep a_i = e_i R_i - h_i a_{i+1}: suffix composition
  double2 a[K];
  Aff C{mk(0.0, 0.0), 1.0};
#pragma unroll
  for (int k = K - 1; k >= 0; --k) {
    const int i = 32 * k + lane;
    Aff x = (i >= 1 && i < M) ? Aff{T.e(i) * R[k], -T.h(i)} : Aff{mk(0.0, 0.0), 1.0};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const Aff t = shfl_down_aff(x, off);
      if (lane + off < 32) x = compose(x, t);
    }
    a[k] = compose(x, C).a;
    C = compose(shfl_idx_aff(x, 0), C);
  }
  // top-down sweep P_i = a_i + b_i P_{i-1}: prefix composition
  double2 Pv[K];
  double2 sum = mk(0.0, 0.0);
  C = Aff{mk(0.0, 0.0), 1.0};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    const bool act = (i >= 1 && i < M);
    Aff x = act ? Aff{a[k], T.b(i)} : Aff{mk(0.0, 0.0), 1.0};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const Aff t = shfl_up_aff(x, off);
      if (lane >= off) x = compose(x, t);
    }
    Pv[k] = compose(x, C).a;
    if (act) sum = sum + Pv[k];
    C = compose(shfl_idx_aff(x, 31), C);
  }
  sum = warp_sum2(sum);
  const double2 f0 = isq * (s - sum);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = 32 * k + lane;
    f[k] = (i == 0) ? f0 : ((i < M) ? Pv[k] + T.Q(i) * f0 : mk(0.0, 0.0));
  }
}

}  // namespace chdns
