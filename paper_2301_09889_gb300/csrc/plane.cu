// Dealiased nonlinear term H = u x omega on one Gauss-Lobatto plane per
// cluster of S CTAs (3/2 rule; paper Sec. 3.1 pseudo-spectral method).
//
// Input: Fourier coefficients (kept half spectrum) of u, v, w, omega_x,
// omega_y, omega_z at node j.  Output: kept Fourier coefficients of
// H_x, H_y, H_z at node j, scaled by 1/(mx mz).
//
// A plane never leaves shared memory between the inverse and the forward
// transforms.  CTA `r` of a cluster owns the physical rows z = S m + r of the
// padded mz x mx grid:
//   1. gather: fold the kz spectrum onto Lz = mz/S points with the pre-twiddle
//      e^{2 pi i kz r / mz}, then an Lz-point inverse FFT (DIF) along z;
//   2. per pair of rows: pack the two real rows of each field into one complex
//      line, Hermitian-extend to mx points, inverse FFT (DIF) along x, form the
//      three products pointwise, forward FFT (DIT) and unpack the two rows;
//   3. forward Lz-point FFT (DIT) along z; the S partial spectra are combined
//      through distributed shared memory with the twiddles e^{-2 pi i kz r / mz}.
// DIF leaves digit-reversed order and DIT consumes it, so no permutation pass
// is needed: the products are pointwise and do not care about the order.
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace chdns {

// v e^{2 pi i e / S} for 0 <= e < S (w = e^{2 pi i / mz}, mz = S Lz, table
// tw_mz[k] = w^k).  Multiples of a quarter turn are exact component swaps;
// other angles multiply by w^{e Lz}.
template <typename C>
__device__ __forceinline__ C turn(C v, int e, int S, int Lz, const C* tw_mz) {
  if (e == 0) return v;
  if ((4 * e) % S == 0) {
    const int k = 4 * e / S;
    if (k == 1) return mk(-v.y, v.x);
    if (k == 2) return mk(-v.x, -v.y);
    return mk(v.y, -v.x);
  }
  return cmul(v, tw_mz[e * Lz]);
}

// The cluster split of the z transforms.  CTA r owns the rows z = S m + r; the
// inverse transform at those rows is an Lz-point transform of the folded
// spectrum  sum_q X[u] w^{u r}  over u = m + q Lz (kz = u mod mz), and
// w^{u r} = w^{m r} e^{2 pi i q r / S}: the terms take turns by S-th roots of
// unity (exact quarter turns for S = 4) and the sum takes one table twiddle.
// The forward direction mirrors it: output kz = u + q Lz of the forward
// transform is  sum_r Z_r[u] w^{-u r} e^{-2 pi i q r / S},  and the factor
// w^{-u r} depends on u alone, so CTA r applies it to its own Z_r before the
// exchange.

template <typename R>
__global__ void __launch_bounds__(256) plane_kernel(PlaneArgs<R> a) {
  using C = typename cpx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Z = reinterpret_cast<C*>(smem_raw);          // [6][Lz][nxh]
  C* X = Z + 6 * a.Lz * a.nxh;                    // [6][NP][mx]
  const int nxh = a.nxh, nz = a.nz, Lz = a.Lz, mx = a.mx, mz = a.mz, S = a.S, NP = a.NP;
  const int tid = threadIdx.x, nt = blockDim.x;
  int rank = 0;
  if (S > 1) rank = (int)cg::this_cluster().block_rank();
  const int j = blockIdx.y;
  const int b = blockIdx.z;
  if (a.active && !a.active[b]) return;  // whole cluster (same b) returns together
  pdl_wait_then_release();               // the node values come from stage_pre
  const size_t plane = (size_t)a.P;
  const C* qb = a.q + (size_t)b * 6 * a.ny * plane + (size_t)j * plane;
  C* hb = a.h + (size_t)b * 3 * a.ny * plane + (size_t)j * plane;

  // 1. gather + fold + pre-twiddle
  for (int w = tid; w < 6 * Lz * nxh; w += nt) {
    const int i = w % nxh;
    const int t = w / nxh;
    const int m = t % Lz;
    const int f = t / Lz;
    const C* qf = qb + (size_t)f * a.ny * plane;
    C acc = czero<C>();
    for (int qq = 0; qq < S; ++qq) {
      const int u = m + qq * Lz;
      int kz;
      if (u < nz / 2) kz = u;
      else if (u > mz - nz / 2) kz = u - mz;
      else continue;
      const int row = kz >= 0 ? kz : nz + kz;
      C val = qf[row * nxh + i];
      if (S > 1) val = turn(val, (qq * rank) % S, S, Lz, a.tw_mz);
      acc = acc + val;
    }
    if (rank > 0) acc = cmul(acc, a.tw_mz[m * rank]);
    Z[(f * Lz + m) * nxh + i] = acc;
  }
  __syncthreads();
  fft_dif<+1, R>(Z, 6 * nxh, nxh, a.pz, a.tw_z, false);

  // 2. rows in pairs: x transforms and products
  const int npairs = Lz / 2;
  for (int pb = 0; pb < npairs; pb += NP) {
    for (int w = tid; w < 6 * NP * mx; w += nt) {
      const int k = w % mx;
      const int t = w / mx;
      const int pp = t % NP;
      const int f = t / NP;
      const int r1 = 2 * (pb + pp);
      const C* A = Z + (f * Lz + r1) * nxh;
      const C* Bv = A + nxh;
      C val;
      if (k == 0) {
        val = mk(A[0].x, Bv[0].x);
      } else if (k < nxh) {
        const C av = A[k], bv = Bv[k];
        val = mk(av.x - bv.y, av.y + bv.x);
      } else if (k > mx - nxh) {
        const int kk = mx - k;
        const C av = A[kk], bv = Bv[kk];
        val = mk(av.x + bv.y, bv.x - av.y);
      } else {
        val = czero<C>();
      }
      X[(f * NP + pp) * mx + k] = val;
    }
    __syncthreads();
    fft_dif<+1, R>(X, 6 * NP, 1, a.px, a.tw_x, true);
    for (int w = tid; w < NP * mx; w += nt) {
      const int x = w % mx;
      const int pp = w / mx;
      C* L0 = X + pp * mx;
      const size_t fs = (size_t)NP * mx;
      const C u = L0[x], v = L0[fs + x], ww = L0[2 * fs + x];
      const C ox = L0[3 * fs + x], oy = L0[4 * fs + x], oz = L0[5 * fs + x];
      // real parts: first row of the pair, imaginary parts: second row
      L0[x] = mk(v.x * oz.x - ww.x * oy.x, v.y * oz.y - ww.y * oy.y);
      L0[fs + x] = mk(ww.x * ox.x - u.x * oz.x, ww.y * ox.y - u.y * oz.y);
      L0[2 * fs + x] = mk(u.x * oy.x - v.x * ox.x, u.y * oy.y - v.y * ox.y);
    }
    __syncthreads();
    fft_dit<-1, R>(X, 3 * NP, 1, a.px, a.tw_x, true);
    for (int w = tid; w < 3 * NP * nxh; w += nt) {
      const int i = w % nxh;
      const int t = w / nxh;
      const int pp = t % NP;
      const int f = t / NP;
      const C* line = X + (f * NP + pp) * mx;
      const C zk = line[i];
      const C zm = line[(mx - i) % mx];
      const int r1 = 2 * (pb + pp);
      Z[(f * Lz + r1) * nxh + i] = mk((zk.x + zm.x) * (R)0.5, (zk.y - zm.y) * (R)0.5);
      Z[(f * Lz + r1 + 1) * nxh + i] = mk((zk.y + zm.y) * (R)0.5, (zm.x - zk.x) * (R)0.5);
    }
    __syncthreads();
  }

  // 3. forward z transform of H_x, H_y, H_z and cluster combination
  fft_dit<-1, R>(Z, 3 * nxh, nxh, a.pz, a.tw_z, false);
  if (rank > 0) {
    for (int w = tid; w < 3 * Lz * nxh; w += nt) Z[w] = cmul(Z[w], cconj(a.tw_mz[((w / nxh) % Lz) * rank]));
  }
  if (S > 1) cg::this_cluster().sync();
  for (int w = tid; w < 3 * nz * nxh; w += nt) {
    const int i = w % nxh;
    const int t = w / nxh;
    const int row = t % nz;
    const int f = t / nz;
    if (S > 1 && (row % S) != rank) continue;
    C out = czero<C>();
    if (row != nz / 2) {
      const int kz = row < nz / 2 ? row : row - nz;
      int u = kz % Lz;
      if (u < 0) u += Lz;
      int q = ((kz - u) / Lz) % S;
      if (q < 0) q += S;
      for (int rr = 0; rr < S; ++rr) {
        const C* Zr = Z;
        if (S > 1 && rr != rank) Zr = cg::this_cluster().map_shared_rank(Z, rr);
        C gval = Zr[(f * Lz + u) * nxh + i];
        if (S > 1) gval = turn(gval, (S - (q * rr) % S) % S, S, Lz, a.tw_mz);
        out = out + gval;
      }
      out = a.scale * out;
    }
    hb[(size_t)f * a.ny * plane + row * nxh + i] = out;
  }
  if (S > 1) cg::this_cluster().sync();
}


// The same kernel with the transform lengths, the kept kx count, the row
// pairs per batch and the CTA size fixed at compile time (index arithmetic by
// constants, FFT passes unrolled).  Instantiated for the grids of the
// configurations in use; planes whose shared memory allows one CTA per SM run
// more threads per CTA to hide shared-memory latency.
template <typename R, int MX, int LZ, int NXH, int NP, int NT>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 && NT == 256 && MX == LZ) ? 8 : 0) plane_kernel_ct(PlaneArgs<R> a) {
  using C = typename cpx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Z = reinterpret_cast<C*>(smem_raw);  // [6][LZ][NXH]
  C* X = Z + 6 * LZ * NXH;                // [6][NP][MX]
  // launched only when the cluster size a.S equals MX / LZ (mz = mx)
  constexpr int S = MX / LZ;
  const int nz = a.nz, mz = a.mz;
  const int tid = threadIdx.x;
  int rank = 0;
  if constexpr (S > 1) rank = (int)cg::this_cluster().block_rank();
  const int j = blockIdx.y;
  const int b = blockIdx.z;
  if (a.active && !a.active[b]) return;  // whole cluster (same b) returns together
  pdl_wait_then_release();               // the node values come from stage_pre
  const size_t plane = (size_t)a.P;
  const C* qb = a.q + (size_t)b * 6 * a.ny * plane + (size_t)j * plane;
  C* hb = a.h + (size_t)b * 3 * a.ny * plane + (size_t)j * plane;

  // 1. gather + fold + pre-twiddle
  for (int w = tid; w < 6 * LZ * NXH; w += NT) {
    const int i = w % NXH;
    const int t = w / NXH;
    const int m = t % LZ;
    const int f = t / LZ;
    const C* qf = qb + (size_t)f * a.ny * plane;
    C acc = czero<C>();
    for (int qq = 0; qq < S; ++qq) {
      const int u = m + qq * LZ;
      int kz;
      if (u < nz / 2) kz = u;
      else if (u > mz - nz / 2) kz = u - mz;
      else continue;
      const int row = kz >= 0 ? kz : nz + kz;
      C val = qf[row * NXH + i];
      if (rank > 0) val = turn(val, (qq * rank) % S, S, LZ, a.tw_mz);
      acc = acc + val;
    }
    if (rank > 0) acc = cmul(acc, a.tw_mz[m * rank]);
    Z[(f * LZ + m) * NXH + i] = acc;
  }
  __syncthreads();
  fft_dif_ct<+1, R, LZ, 6 * NXH, NXH, false, NT>(Z, a.tw_z);

  // 2. rows in pairs: x transforms and products
  constexpr int NPAIRS = LZ / 2;
  for (int pb = 0; pb < NPAIRS; pb += NP) {
    for (int w = tid; w < 6 * NP * MX; w += NT) {
      const int k = w % MX;
      const int t = w / MX;
      const int pp = t % NP;
      const int f = t / NP;
      const int r1 = 2 * (pb + pp);
      const C* A = Z + (f * LZ + r1) * NXH;
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
      X[(f * NP + pp) * MX + k] = val;
    }
    __syncthreads();
    fft_dif_ct<+1, R, MX, 6 * NP, 1, true, NT>(X, a.tw_x);
    for (int w = tid; w < NP * MX; w += NT) {
      const int x = w % MX;
      const int pp = w / MX;
      C* L0 = X + pp * MX;
      constexpr int fs = NP * MX;
      const C u = L0[x], v = L0[fs + x], ww = L0[2 * fs + x];
      const C ox = L0[3 * fs + x], oy = L0[4 * fs + x], oz = L0[5 * fs + x];
      L0[x] = mk(v.x * oz.x - ww.x * oy.x, v.y * oz.y - ww.y * oy.y);
      L0[fs + x] = mk(ww.x * ox.x - u.x * oz.x, ww.y * ox.y - u.y * oz.y);
      L0[2 * fs + x] = mk(u.x * oy.x - v.x * ox.x, u.y * oy.y - v.y * ox.y);
    }
    __syncthreads();
    fft_dit_ct<-1, R, MX, 3 * NP, 1, true, NT>(X, a.tw_x);
    for (int w = tid; w < 3 * NP * NXH; w += NT) {
      const int i = w % NXH;
      const int t = w / NXH;
      const int pp = t % NP;
      const int f = t / NP;
      const C* line = X + (f * NP + pp) * MX;
      const C zk = line[i];
      const C zm = line[(MX - i) % MX];
      const int r1 = 2 * (pb + pp);
      Z[(f * LZ + r1) * NXH + i] = mk((zk.x + zm.x) * (R)0.5, (zk.y - zm.y) * (R)0.5);
      Z[(f * LZ + r1 + 1) * NXH + i] = mk((zk.y + zm.y) * (R)0.5, (zm.x - zk.x) * (R)0.5);
    }
    __syncthreads();
  }

  // 3. forward z transform of H_x, H_y, H_z and cluster combination
  fft_dit_ct<-1, R, LZ, 3 * NXH, NXH, false, NT>(Z, a.tw_z);
  if (rank > 0) {
    for (int w = tid; w < 3 * LZ * NXH; w += NT) Z[w] = cmul(Z[w], cconj(a.tw_mz[((w / NXH) % LZ) * rank]));
  }
  if (S > 1) cg::this_cluster().sync();
  for (int w = tid; w < 3 * nz * NXH; w += NT) {
    const int i = w % NXH;
    const int t = w / NXH;
    const int row = t % nz;
    const int f = t / nz;
    if (S > 1 && (row % S) != rank) continue;
    C out = czero<C>();
    if (row != nz / 2) {
      const int kz = row < nz / 2 ? row : row - nz;
      int u = kz % LZ;
      if (u < 0) u += LZ;
      int q = ((kz - u) / LZ) % S;
      if (q < 0) q += S;
      for (int rr = 0; rr < S; ++rr) {
        const C* Zr = Z;
        if (S > 1 && rr != rank) Zr = cg::this_cluster().map_shared_rank(Z, rr);
        C gval = Zr[(f * LZ + u) * NXH + i];
        if (rr > 0) gval = turn(gval, (S - (q * rr) % S) % S, S, LZ, a.tw_mz);
        out = out + gval;
      }
      out = a.scale * out;
    }
    hb[(size_t)f * a.ny * plane + row * NXH + i] = out;
  }
  if (S > 1) cg::this_cluster().sync();
}

template <typename K, typename R>
static cudaError_t launch_with(K kernel, const PlaneArgs<R>& a, int B, size_t smem, cudaStream_t st,
                               SmemLimit* lim, int nt = 256) {
  // clusters above 8 CTAs are a non-portable opt-in
  const cudaError_t e = raise_smem_limit(kernel, lim, smem, a.S > 8);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.S, a.ny, B);
  cfg.blockDim = dim3(nt, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (sizeof(R) == 4) {  // programmatic launch for the FP32 plane only (see launch_pdl_if)
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (a.S > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = a.S;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

// limit of the runtime-size kernel, shared by its launches and the occupancy query
template <typename R>
static SmemLimit& generic_limit() {
  static SmemLimit lim;
  return lim;
}

// compile-time instantiations: (MX, LZ, NXH, NP) of the grids in use
#define CH_PLANE_CT_NT(MX_, LZ_, NXH_, NP_, NT_)                                                      \
  if (a.mx == MX_ && a.Lz == LZ_ && a.nxh == NXH_ && a.NP == NP_ && a.S == MX_ / LZ_) {             \
    static SmemLimit lim_;                                                                            \
    return launch_with(plane_kernel_ct<R, MX_, LZ_, NXH_, NP_, NT_>, a, B, smem, st, &lim_, NT_);     \
  }
#define CH_PLANE_CT(MX_, LZ_, NXH_, NP_) CH_PLANE_CT_NT(MX_, LZ_, NXH_, NP_, 256)

template <typename R>
cudaError_t launch_plane(const PlaneArgs<R>& a, int B, size_t smem, cudaStream_t st) {
  if (a.team16) return launch_plane16<R>(a, B, st);
  if (a.two_pass) return launch_plane_two_pass<R>(a, B, st);
  if constexpr (sizeof(R) == 8) {
    CH_PLANE_CT(24, 6, 8, 3)
    CH_PLANE_CT(24, 24, 8, 12)
    CH_PLANE_CT_NT(96, 24, 32, 3, 512)
    CH_PLANE_CT(48, 12, 16, 6)
    CH_PLANE_CT_NT(192, 24, 64, 4, 1024)
  } else {
    CH_PLANE_CT(24, 6, 8, 3)
    CH_PLANE_CT(24, 24, 8, 12)
    CH_PLANE_CT(96, 24, 32, 12)
    CH_PLANE_CT(48, 12, 16, 6)
    CH_PLANE_CT_NT(192, 48, 64, 8, 1024)
  }
  return launch_with(plane_kernel<R>, a, B, smem, st, &generic_limit<R>());
}

// Clusters of a.S CTAs with `smem` bytes each that the device can hold at
// once for the runtime-size kernel (0: the shape cannot be launched).
template <typename R>
cudaError_t plane_max_clusters(const PlaneArgs<R>& a, size_t smem, int* clusters) {
  *clusters = 0;
  const cudaError_t e = raise_smem_limit(plane_kernel<R>, &generic_limit<R>(), smem, a.S > 8);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.S, a.ny, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, plane_kernel<R>, &cfg);
}

template cudaError_t plane_max_clusters<double>(const PlaneArgs<double>&, size_t, int*);
template cudaError_t plane_max_clusters<float>(const PlaneArgs<float>&, size_t, int*);
template cudaError_t launch_plane<double>(const PlaneArgs<double>&, int, size_t, cudaStream_t);
template cudaError_t launch_plane<float>(const PlaneArgs<float>&, int, size_t, cudaStream_t);

}  // namespace chdns
