// Dealiased nonlinear term H = u x omega for planes whose padded z-slabs fit no
// portable cluster's shared memory: the plane of 256 x 256 modes takes 295 KB
// per CTA in FP64 even split over 16 CTAs, and 147 KB in FP32 over a 16-CTA
// cluster, of which the device holds only a few at once.  The same 3/2-rule
// transforms as plane.cu, in three passes through a global scratch array
// y[B][ny][6][mz][nxh]:
//   1. z inverse: per tile of CW kx columns of one field, zero-pad the kz
//      spectrum to mz points and transform along z (DIF, digit-reversed rows);
//   2. x pass: per pair of physical z rows, pack the two real rows of each
//      field into one complex line, Hermitian-extend to mx points, inverse
//      FFT (DIF), the three products, forward FFT (DIT), unpack the two rows
//      of H_x, H_y, H_z over fields 0..2 of the same rows;
//   3. z forward: per column tile of H, transform back (DIT, consuming the
//      digit-reversed rows) and keep the rows |kz| < nz/2, scaled by 1/(mx mz).
// Rows stay in the order the DIF leaves them: the products are pointwise in
// z, and the DIT of pass 3 takes that order back to natural.
#include "common.cuh"
#include "internal.h"

namespace chdns {

template <typename R, int MZ, int NXH, int CW, int NT>
__global__ void __launch_bounds__(NT) zpass_inverse_kernel(PlaneArgs<R> a) {
  using C = typename cpx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Z = reinterpret_cast<C*>(smem_raw);  // [MZ][CW]
  const int i0 = blockIdx.x * CW;
  const int f = blockIdx.y % 6, j = blockIdx.y / 6;
  const int b = blockIdx.z;
  if (a.active && !a.active[b]) return;
  pdl_wait_then_release();  // the node values come from stage_pre
  const int nz = a.nz;
  const C* qf = a.q + (((size_t)b * 6 + f) * a.ny + j) * a.P;
  for (int w = threadIdx.x; w < MZ * CW; w += NT) {
    const int c = w % CW, u = w / CW;
    C val = czero<C>();
    int row = -1;
    if (u < nz / 2) row = u;
    else if (u > MZ - nz / 2) row = nz + (u - MZ);
    if (row >= 0) val = qf[(size_t)row * NXH + i0 + c];
    Z[w] = val;
  }
  __syncthreads();
  fft_dif_ct<+1, R, MZ, CW, CW, false, NT>(Z, a.tw_mz);
  C* yf = a.y + (((size_t)b * a.ny + j) * 6 + f) * MZ * NXH;
  for (int w = threadIdx.x; w < MZ * CW; w += NT) {
    const int c = w % CW, u = w / CW;
    yf[(size_t)u * NXH + i0 + c] = Z[w];
  }
}

template <typename R, int MX, int MZ, int NXH, int NPR, int NT>
__global__ void __launch_bounds__(NT) xpass_kernel(PlaneArgs<R> a) {
  using C = typename cpx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);  // [6][NPR][MX]
  const int pr0 = blockIdx.x * NPR;       // first row pair of this CTA
  const int j = blockIdx.y, b = blockIdx.z;
  if (a.active && !a.active[b]) return;
  pdl_wait_then_release();
  C* yb = a.y + ((size_t)b * a.ny + j) * 6 * MZ * NXH;
  // every read of this CTA's rows happens before the first barrier; the rows
  // of H are written over fields 0..2 of the same rows at the end
  for (int w = threadIdx.x; w < 6 * NPR * MX; w += NT) {
    const int k = w % MX;
    const int t = w / MX;
    const int pp = t % NPR;
    const int f = t / NPR;
    const int r1 = 2 * (pr0 + pp);
    const C* A = yb + ((size_t)f * MZ + r1) * NXH;
    const C* Bv = A + NXH;
    C val;
    if (k == 0) {
      val = mk(A[0].x, Bv[0].x);
    } else if (k < NXH) {
      const C av = A[k], bv = Bv[k];
      val = mk(av.x - bv.y, av.y + bv.x);
    } else if (k > MX - NXH) {
      const int kk = MX - k;
      const C av = A[kk], bv = Bv[kk];
      val = mk(av.x + bv.y, bv.x - av.y);
    } else {
      val = czero<C>();
    }
    X[(f * NPR + pp) * MX + k] = val;
  }
  __syncthreads();
  fft_dif_ct<+1, R, MX, 6 * NPR, 1, true, NT>(X, a.tw_x);
  for (int w = threadIdx.x; w < NPR * MX; w += NT) {
    const int x = w % MX;
    const int pp = w / MX;
    C* L0 = X + pp * MX;
    constexpr int fs = NPR * MX;
    const C u = L0[x], v = L0[fs + x], ww = L0[2 * fs + x];
    const C ox = L0[3 * fs + x], oy = L0[4 * fs + x], oz = L0[5 * fs + x];
    // real parts: first row of the pair, imaginary parts: second row
    L0[x] = mk(v.x * oz.x - ww.x * oy.x, v.y * oz.y - ww.y * oy.y);
    L0[fs + x] = mk(ww.x * ox.x - u.x * oz.x, ww.y * ox.y - u.y * oz.y);
    L0[2 * fs + x] = mk(u.x * oy.x - v.x * ox.x, u.y * oy.y - v.y * ox.y);
  }
  __syncthreads();
  fft_dit_ct<-1, R, MX, 3 * NPR, 1, true, NT>(X, a.tw_x);
  for (int w = threadIdx.x; w < 3 * NPR * NXH; w += NT) {
    const int i = w % NXH;
    const int t = w / NXH;
    const int pp = t % NPR;
    const int f = t / NPR;
    const C* line = X + (f * NPR + pp) * MX;
    const C zk = line[i];
    const C zm = line[(MX - i) % MX];
    const int r1 = 2 * (pr0 + pp);
    C* dst = yb + ((size_t)f * MZ + r1) * NXH;
    dst[i] = mk((zk.x + zm.x) * (R)0.5, (zk.y - zm.y) * (R)0.5);
    dst[NXH + i] = mk((zk.y + zm.y) * (R)0.5, (zm.x - zk.x) * (R)0.5);
  }
}

template <typename R, int MZ, int NXH, int CW, int NT>
__global__ void __launch_bounds__(NT) zpass_forward_kernel(PlaneArgs<R> a) {
  using C = typename cpx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Z = reinterpret_cast<C*>(smem_raw);  // [MZ][CW]
  const int i0 = blockIdx.x * CW;
  const int f = blockIdx.y % 3, j = blockIdx.y / 3;
  const int b = blockIdx.z;
  if (a.active && !a.active[b]) return;
  pdl_wait_then_release();
  const int nz = a.nz;
  const C* yf = a.y + (((size_t)b * a.ny + j) * 6 + f) * MZ * NXH;
  for (int w = threadIdx.x; w < MZ * CW; w += NT) {
    const int c = w % CW, u = w / CW;
    Z[w] = yf[(size_t)u * NXH + i0 + c];
  }
  __syncthreads();
  fft_dit_ct<-1, R, MZ, CW, CW, false, NT>(Z, a.tw_mz);
  C* hf = a.h + (((size_t)b * 3 + f) * a.ny + j) * a.P;
  for (int w = threadIdx.x; w < nz * CW; w += NT) {
    const int c = w % CW, row = w / CW;
    C out = czero<C>();
    if (row != nz / 2) {
      const int kz = row < nz / 2 ? row : row - nz;
      const int u = kz >= 0 ? kz : MZ + kz;
      out = a.scale * Z[u * CW + c];
    }
    hf[(size_t)row * NXH + i0 + c] = out;
  }
}

// shapes of the passes: CW kx columns per z-pass CTA, NPR row pairs per x-pass CTA
constexpr int kTwoPassCW = 8;
constexpr int kTwoPassNPR = 2;
constexpr int kTwoPassNT = 256;

template <typename R, int MX, int MZ, int NXH>
static cudaError_t launch_two_pass_ct(const PlaneArgs<R>& a, int B, cudaStream_t st) {
  using C = typename cpx<R>::T;
  static SmemLimit lim_a, lim_b, lim_c;
  const size_t sz = (size_t)MZ * kTwoPassCW * sizeof(C);
  const size_t sx = (size_t)6 * kTwoPassNPR * MX * sizeof(C);
  auto ka = zpass_inverse_kernel<R, MZ, NXH, kTwoPassCW, kTwoPassNT>;
  auto kb = xpass_kernel<R, MX, MZ, NXH, kTwoPassNPR, kTwoPassNT>;
  auto kc = zpass_forward_kernel<R, MZ, NXH, kTwoPassCW, kTwoPassNT>;
  cudaError_t e;
  if ((e = raise_smem_limit(ka, &lim_a, sz)) != cudaSuccess) return e;
  if ((e = raise_smem_limit(kb, &lim_b, sx)) != cudaSuccess) return e;
  if ((e = raise_smem_limit(kc, &lim_c, sz)) != cudaSuccess) return e;
  constexpr bool pdl = sizeof(R) == 4;
  e = launch_pdl_if<pdl>(ka, dim3(NXH / kTwoPassCW, 6 * a.ny, B), dim3(kTwoPassNT), sz, st, a);
  if (e != cudaSuccess) return e;
  e = launch_pdl_if<pdl>(kb, dim3(MZ / 2 / kTwoPassNPR, a.ny, B), dim3(kTwoPassNT), sx, st, a);
  if (e != cudaSuccess) return e;
  return launch_pdl_if<pdl>(kc, dim3(NXH / kTwoPassCW, 3 * a.ny, B), dim3(kTwoPassNT), sz, st, a);
}

// The grids built in passes: 256 x 256 modes (mx = mz = 384) in both
// precisions, whose planes fit no portable cluster; in FP64 also 64 x 64 and
// 128 x 128 modes, where a cluster per plane leaves the last wave of SMs
// part-empty and the passes keep every SM on FP64 work.
bool two_pass_shape_ok(int mx, int mz, int nxh) {
  return (mx == 384 && mz == 384 && nxh == 128) || (mx == 96 && mz == 96 && nxh == 32) ||
         (mx == 192 && mz == 192 && nxh == 64);
}
bool two_pass_chosen(int mx, int mz, int nxh, bool fp64) {
  if (mx == 384 && mz == 384 && nxh == 128) return true;
  return fp64 && two_pass_shape_ok(mx, mz, nxh);
}

template <typename R>
cudaError_t launch_plane_two_pass(const PlaneArgs<R>& a, int B, cudaStream_t st) {
  if (a.mx == 384 && a.mz == 384 && a.nxh == 128) return launch_two_pass_ct<R, 384, 384, 128>(a, B, st);
  if constexpr (sizeof(R) == 8) {
    if (a.mx == 96 && a.mz == 96 && a.nxh == 32) return launch_two_pass_ct<R, 96, 96, 32>(a, B, st);
    if (a.mx == 192 && a.mz == 192 && a.nxh == 64) return launch_two_pass_ct<R, 192, 192, 64>(a, B, st);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_plane_two_pass<double>(const PlaneArgs<double>&, int, cudaStream_t);
template cudaError_t launch_plane_two_pass<float>(const PlaneArgs<float>&, int, cudaStream_t);

}  // namespace chdns
