// Dealiased nonlinear term H = u x omega for planes of 16 x 16 Fourier modes
// (the minimal channel of the paper's first domain; 3/2 rule, padded 24 x 24).
//
// The same transforms as plane.cu, with every 24-point line transformed in
// registers by one thread: 24 = 8 x 3, three 8-point DFTs of the samples
// 3m + j, the twiddles w^{j k} (w = e^{2 pi i / 24}, from the handle's table
// staged once per CTA) and eight 3-point DFTs, natural order in and out.  A
// team of 96 threads owns one plane:
//   1. z inverse: 48 lines (6 fields x 8 kx columns), the kz spectrum
//      zero-padded to 24 points;
//   2. x inverse: 72 lines (6 fields x 12 pairs of z rows), two real rows of a
//      field packed into one complex line and Hermitian-extended to 24 points;
//   3. the three products at the 288 points of every row pair;
//   4. x forward: 36 lines (3 fields x 12 pairs), unpacked into the two rows;
//   5. z forward: 24 lines (3 fields x 8 columns), truncated to |kz| < 8 and
//      scaled by 1/(mx mz).
// Five barriers per plane, no index arithmetic inside the transforms.
#include "common.cuh"
#include "internal.h"

namespace chdns {

namespace {

constexpr int kNxh = 8, kNz = 16, kM = 24, kPairs = 12, kTeam = 96;

// X[k' + 8 q] = sum_j (w^{j k'} A_j[k']) e^{SIGN 2 pi i j q / 3}, A_j the
// 8-point DFT of x[3 m + j]; tw[k] = e^{+2 pi i k / 24}
template <int SIGN, typename C, typename R>
__device__ __forceinline__ void fft24(C (&x)[kM], const C* tw) {
  C A[3][8];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int m = 0; m < 8; ++m) A[j][m] = x[3 * m + j];
    small_dft_ct<SIGN, 8, C, R>(A[j]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    C t[3] = {A[0][k], A[1][k], A[2][k]};
    if (k > 0) {
      t[1] = cmul(t[1], twiddle<SIGN>(tw, k));
      t[2] = cmul(t[2], twiddle<SIGN>(tw, 2 * k));
    }
    small_dft_ct<SIGN, 3, C, R>(t);
    x[k] = t[0];
    x[k + 8] = t[1];
    x[k + 16] = t[2];
  }
}

}  // namespace

template <typename R, int PPB>
__global__ void __launch_bounds__(kTeam * PPB) plane16_kernel(PlaneArgs<R> a) {
  using C = typename cpx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);  // [24]
  const int team = threadIdx.x / kTeam, lt = threadIdx.x % kTeam;
  C* Zs = tw + kM + (size_t)team * (6 * kM * kNxh + 6 * kPairs * kM);  // [6][24 z][8 kx]
  C* Xs = Zs + 6 * kM * kNxh;                                          // [6][12 pairs][24 x]
  const int j = blockIdx.x * PPB + team;  // Gauss-Lobatto plane of this team
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;  // whole CTA (same b) returns together
  pdl_wait_then_release();               // the node values come from stage_pre
  for (int w = threadIdx.x; w < kM; w += blockDim.x) tw[w] = a.tw_x[w];
  __syncthreads();
  const bool live = j < a.ny;
  const size_t plane = (size_t)a.P;

  // 1. z inverse
  if (live && lt < 6 * kNxh) {
    const int f = lt / kNxh, i = lt % kNxh;
    const C* qf = a.q + ((size_t)b * 6 + f) * a.ny * plane + (size_t)j * plane;
    C x[kM];
#pragma unroll
    for (int u = 0; u < kM; ++u) {
      // kz = u (u < 8) or u - 24 (u > 16, row 16 + kz); the rest is padding and
      // the Nyquist row
      const int row = u < kNz / 2 ? u : (u > kM - kNz / 2 ? u - (kM - kNz) : -1);
      x[u] = row >= 0 ? qf[row * kNxh + i] : czero<C>();
    }
    fft24<+1, C, R>(x, tw);
#pragma unroll
    for (int z = 0; z < kM; ++z) Zs[(f * kM + z) * kNxh + i] = x[z];
  }
  __syncthreads();

  // 2. x inverse on pairs of rows
  if (live && lt < 6 * kPairs) {
    const int f = lt / kPairs, m = lt % kPairs;
    const C* A = Zs + (f * kM + 2 * m) * kNxh;
    const C* Bv = A + kNxh;
    C x[kM];
    x[0] = mk(A[0].x, Bv[0].x);
#pragma unroll
    for (int k = 1; k < kNxh; ++k) x[k] = mk(A[k].x - Bv[k].y, A[k].y + Bv[k].x);
#pragma unroll
    for (int k = kNxh; k <= kM - kNxh; ++k) x[k] = czero<C>();
#pragma unroll
    for (int k = kM - kNxh + 1; k < kM; ++k) {
      const int kk = kM - k;
      x[k] = mk(A[kk].x + Bv[kk].y, Bv[kk].x - A[kk].y);
    }
    fft24<+1, C, R>(x, tw);
#pragma unroll
    for (int k = 0; k < kM; ++k) Xs[(f * kPairs + m) * kM + k] = x[k];
  }
  __syncthreads();

  // 3. products: real parts are the first row of a pair, imaginary parts the second
  if (live) {
    constexpr int fs = kPairs * kM;
    for (int w = lt; w < fs; w += kTeam) {
      C* L0 = Xs + w;
      const C u = L0[0], v = L0[fs], ww = L0[2 * fs];
      const C ox = L0[3 * fs], oy = L0[4 * fs], oz = L0[5 * fs];
      L0[0] = mk(v.x * oz.x - ww.x * oy.x, v.y * oz.y - ww.y * oy.y);
      L0[fs] = mk(ww.x * ox.x - u.x * oz.x, ww.y * ox.y - u.y * oz.y);
      L0[2 * fs] = mk(u.x * oy.x - v.x * ox.x, u.y * oy.y - v.y * ox.y);
    }
  }
  __syncthreads();

  // 4. x forward, unpacked into the two rows of each pair
  if (live && lt < 3 * kPairs) {
    const int f = lt / kPairs, m = lt % kPairs;
    C x[kM];
#pragma unroll
    for (int k = 0; k < kM; ++k) x[k] = Xs[(f * kPairs + m) * kM + k];
    fft24<-1, C, R>(x, tw);
    C* r1 = Zs + (f * kM + 2 * m) * kNxh;
#pragma unroll
    for (int i = 0; i < kNxh; ++i) {
      const C zk = x[i], zm = x[(kM - i) % kM];
      r1[i] = mk((zk.x + zm.x) * (R)0.5, (zk.y - zm.y) * (R)0.5);
      r1[kNxh + i] = mk((zk.y + zm.y) * (R)0.5, (zm.x - zk.x) * (R)0.5);
    }
  }
  __syncthreads();

  // 5. z forward, truncation and scaling
  if (live && lt < 3 * kNxh) {
    const int f = lt / kNxh, i = lt % kNxh;
    C x[kM];
#pragma unroll
    for (int z = 0; z < kM; ++z) x[z] = Zs[(f * kM + z) * kNxh + i];
    fft24<-1, C, R>(x, tw);
    C* hf = a.h + ((size_t)b * 3 + f) * a.ny * plane + (size_t)j * plane;
#pragma unroll
    for (int row = 0; row < kNz; ++row) {
      C out = czero<C>();
      if (row != kNz / 2) {
        const int kz = row < kNz / 2 ? row : row - kNz;
        out = a.scale * x[kz >= 0 ? kz : kM + kz];
      }
      hf[row * kNxh + i] = out;
    }
  }
}

bool plane16_shape(int mx, int mz, int nxh, int nz) { return mx == kM && mz == kM && nxh == kNxh && nz == kNz; }

template <typename R>
cudaError_t launch_plane16(const PlaneArgs<R>& a, int B, cudaStream_t st) {
  using C = typename cpx<R>::T;
  // two planes per CTA: 46 KB (FP32) or 92 KB (FP64) of shared memory
  constexpr int PPB = 2;
  const size_t smem = ((size_t)kM + (size_t)PPB * (6 * kM * kNxh + 6 * kPairs * kM)) * sizeof(C);
  static SmemLimit lim;
  const cudaError_t e = raise_smem_limit(plane16_kernel<R, PPB>, &lim, smem);
  if (e != cudaSuccess) return e;
  return launch_pdl_if<sizeof(R) == 4>(plane16_kernel<R, PPB>, dim3((a.ny + PPB - 1) / PPB, B), dim3(kTeam * PPB),
                                       smem, st, a);
}

template cudaError_t launch_plane16<double>(const PlaneArgs<double>&, int, cudaStream_t);
template cudaError_t launch_plane16<float>(const PlaneArgs<float>&, int, cudaStream_t);

}  // namespace chdns
