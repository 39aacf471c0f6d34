// Shared device helpers of the channel-flow library: complex arithmetic,
// in-place mixed-radix FFT stages in shared memory, and the launch structs
// passed from the host code to the kernels.
#pragma once

#include <cmath>

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <utility>

namespace chdns {

constexpr int kMaxNy = 201;                    // largest Chebyshev node count built
constexpr int kMaxHalf = (kMaxNy + 1) / 2 + 1; // unknowns of one parity, upper bound
constexpr int kMaxRadixStages = 16;

// ---------------------------------------------------------------------------
// complex helpers for double2 / float2
// ---------------------------------------------------------------------------
template <typename R> struct cpx;
template <> struct cpx<double> { using T = double2; };
template <> struct cpx<float> { using T = float2; };

__host__ __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
__host__ __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }

// Round-to-nearest multiply and fused multiply-add that the compiler never
// contracts or splits.  An expression such as a*b - c*d may be fused either
// way, and the choice can differ between kernels that inline the same code;
// the arithmetic that several kernel forms share (so that their results agree
// bit for bit) is written with these.
__host__ __device__ __forceinline__ double fma_rn(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __fma_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
__host__ __device__ __forceinline__ float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
__host__ __device__ __forceinline__ double mul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

#define CH_CPX_OPS(C, R)                                                                   \
  __host__ __device__ __forceinline__ C operator+(C a, C b) { return mk(a.x + b.x, a.y + b.y); } \
  __host__ __device__ __forceinline__ C operator-(C a, C b) { return mk(a.x - b.x, a.y - b.y); } \
  __host__ __device__ __forceinline__ C operator*(R s, C a) { return mk(s * a.x, s * a.y); }     \
  __host__ __device__ __forceinline__ C cmul(C a, C b) {                                  \
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                              \
  }                                                                                       \
  /* the same product with its fused multiply-adds pinned (code shared by several     */ \
  /* kernel forms whose results must agree bit for bit)                                */ \
  __host__ __device__ __forceinline__ C cmul_rn(C a, C b) {                               \
    return mk(fma_rn(a.x, b.x, -mul_rn(a.y, b.y)), fma_rn(a.x, b.y, mul_rn(a.y, b.x)));    \
  }                                                                                       \
  __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }                \
  /* i * s * a */                                                                         \
  __host__ __device__ __forceinline__ C imul(R s, C a) { return mk(-s * a.y, s * a.x); }

CH_CPX_OPS(double2, double)
CH_CPX_OPS(float2, float)
#undef CH_CPX_OPS

template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

// Programmatic dependent launch.  The step's stage and plane kernels may be
// launched with the programmatic-serialisation attribute, so a kernel may start while its
// predecessor in the stream drains.  Each kernel reads its predecessor's
// output only after griddepcontrol.wait (predecessor complete, its writes
// visible), and lets its successor launch only after that wait: a kernel
// that starts early therefore finds every grid before its predecessor
// complete, and may read their outputs (the state, the tables) in its
// prologue.  Both instructions are no-ops in a kernel launched without the
// attribute.
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Asynchronous copy of one 4-, 8- or 16-byte element from global to shared
// memory (cp.async): no register holds the value, so a thread issues all its
// copies of a tile before any completes.  cp_async_wait_all() waits for the
// thread's own copies; a barrier after it publishes the tile to the CTA.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A kernel's dynamic shared-memory limit (and the non-portable cluster-size
// opt-in) as configured so far.  raise_smem_limit only ever raises it, under
// one lock for every kernel, so handles of different sizes driven from
// several host threads never leave a kernel below a size another one needs.
struct SmemLimit {
  size_t bytes = 0;
  bool nonportable = false;
};
inline std::mutex& kernel_attr_mutex() {
  static std::mutex m;
  return m;
}
template <typename K>
inline cudaError_t raise_smem_limit(K kernel, SmemLimit* lim, size_t smem, bool nonportable_cluster = false) {
  std::lock_guard<std::mutex> lock(kernel_attr_mutex());
  if (smem > lim->bytes) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lim->bytes = smem;
  }
  if (nonportable_cluster && !lim->nonportable) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    lim->nonportable = true;
  }
  return cudaSuccess;
}

// launch with the programmatic-serialisation attribute (see above)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The attribute is given to the kernels of FP32-node handles only: measured on
// GB300 it shortens the mixed-precision steps (64x65x64 by 1-4 %, 256 minimal
// channels by 1.2 %) and lengthens the all-FP64 64x65x64 step by 2-3.5 %, also
// when the FP64 plane kernel alone is launched without it.
template <bool PDL, typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_if(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 Args&&... args) {
  if constexpr (PDL) {
    return launch_pdl(kernel, grid, block, smem, st, std::forward<Args>(args)...);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  }
}

// ---------------------------------------------------------------------------
// FFT plans and in-place stages
// ---------------------------------------------------------------------------
struct FftPlan {
  int n;
  int nst;
  int radix[kMaxRadixStages];
};

// e^{SIGN 2 pi i k / n} from a table of e^{+2 pi i k / n}
template <int SIGN, typename C>
__device__ __forceinline__ C twiddle(const C* tw, int k) {
  C w = tw[k];
  if (SIGN < 0) w.y = -w.y;
  return w;
}

// Small DFT y_u = sum_t x_t e^{SIGN 2 pi i t u / r}, r in {2, 3, 4}.
template <int SIGN, typename C, typename R>
__device__ __forceinline__ void small_dft(C* x, int r) {
  if (r == 2) {
    C a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  } else if (r == 3) {
    // sin(2 pi / 3) = sqrt(3) / 2
    const R k = (R)SIGN * (R)0.86602540378443864676372317075293618;
    C s = x[1] + x[2];
    C d = x[1] - x[2];
    C t1 = x[0] - (R)0.5 * s;
    C rot = imul(k, d);
    x[0] = x[0] + s;
    x[1] = t1 + rot;
    x[2] = t1 - rot;
  } else {
    C a0 = x[0] + x[2], a1 = x[0] - x[2];
    C b0 = x[1] + x[3], b1 = x[1] - x[3];
    C wb1 = imul((R)SIGN, b1);
    x[0] = a0 + b0;
    x[1] = a1 + wb1;
    x[2] = a0 - b0;
    x[3] = a1 - wb1;
  }
}

// Line l of a batch starts at (l / g) * (n g) + (l % g) with element stride g
// (g = 1: contiguous lines).  `bf_fastest` picks which index consecutive
// threads walk: butterflies of one line (contiguous lines) or lines
// (strided lines), so that neighbouring threads touch neighbouring words.

// Decimation in frequency: natural-order input, digit-reversed output.
template <int SIGN, typename R>
__device__ void fft_dif(typename cpx<R>::T* buf, int nlines, int g, const FftPlan& pl,
                        const typename cpx<R>::T* tw, bool bf_fastest) {
  using C = typename cpx<R>::T;
  const int n = pl.n;
  int L = n;
  for (int s = 0; s < pl.nst; ++s) {
    const int r = pl.radix[s];
    const int m = L / r;
    const int nb = n / r;
    const int tstep = n / L;
    const int total = nlines * nb;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
      int l, bf;
      if (bf_fastest) { bf = w % nb; l = w / nb; } else { l = w % nlines; bf = w / nlines; }
      C* base = buf + (l / g) * (n * g) + (l % g);
      const int blk = bf / m, q = bf % m;
      const int i0 = blk * L + q;
      C x[4];
      for (int t = 0; t < r; ++t) x[t] = base[(i0 + t * m) * g];
      small_dft<SIGN, C, R>(x, r);
      for (int u = 0; u < r; ++u) {
        C y = x[u];
        if (u > 0 && q > 0) y = cmul(y, twiddle<SIGN>(tw, q * u * tstep));
        base[(i0 + u * m) * g] = y;
      }
    }
    __syncthreads();
    L = m;
  }
}

// Decimation in time with the radices in reverse order: digit-reversed input
// (as produced by fft_dif with the same plan), natural-order output.
template <int SIGN, typename R>
__device__ void fft_dit(typename cpx<R>::T* buf, int nlines, int g, const FftPlan& pl,
                        const typename cpx<R>::T* tw, bool bf_fastest) {
  using C = typename cpx<R>::T;
  const int n = pl.n;
  int L = 1;
  for (int s = pl.nst - 1; s >= 0; --s) {
    const int r = pl.radix[s];
    const int m = L;
    L = L * r;
    const int nb = n / r;
    const int tstep = n / L;
    const int total = nlines * nb;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
      int l, bf;
      if (bf_fastest) { bf = w % nb; l = w / nb; } else { l = w % nlines; bf = w / nlines; }
      C* base = buf + (l / g) * (n * g) + (l % g);
      const int blk = bf / m, q = bf % m;
      const int i0 = blk * L + q;
      C x[4];
      for (int t = 0; t < r; ++t) {
        C v = base[(i0 + t * m) * g];
        if (t > 0 && q > 0) v = cmul(v, twiddle<SIGN>(tw, q * t * tstep));
        x[t] = v;
      }
      small_dft<SIGN, C, R>(x, r);
      for (int u = 0; u < r; ++u) base[(i0 + u * m) * g] = x[u];
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Compile-time FFT plans and stages: the same in-place DIF/DIT passes with
// the length, the radix of every pass and the line layout fixed at compile
// time, so that index arithmetic reduces to constant multiplies and shifts.
// Plan of n = 8^a 4^b 2^c 3^d: radices 8, ..., 8, 4, ..., 4, 2, ..., 2, 3, ..., 3
// (radix 8 first: fewest passes, hence fewest barriers and shared-memory
// round trips per transform).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ct_nst(int n) {
  int s = 0;
  while (n % 8 == 0) { n /= 8; ++s; }
  while (n % 4 == 0) { n /= 4; ++s; }
  while (n % 2 == 0) { n /= 2; ++s; }
  while (n % 3 == 0) { n /= 3; ++s; }
  return s;
}
__host__ __device__ constexpr int ct_radix(int n, int st) {
  int s = 0;
  while (n % 8 == 0) { if (s == st) return 8; n /= 8; ++s; }
  while (n % 4 == 0) { if (s == st) return 4; n /= 4; ++s; }
  while (n % 2 == 0) { if (s == st) return 2; n /= 2; ++s; }
  while (n % 3 == 0) { if (s == st) return 3; n /= 3; ++s; }
  return 1;
}
// true when the radix-8/4/2/3 plan factors n completely
__host__ __device__ constexpr bool ct_plan_ok(int n) {
  if (n < 2) return false;
  while (n % 8 == 0) n /= 8;
  while (n % 4 == 0) n /= 4;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}
// sub-length L before pass st of the DIF order
__host__ __device__ constexpr int ct_len_before(int n, int st) {
  int L = n;
  for (int s = 0; s < st; ++s) L /= ct_radix(n, s);
  return L;
}

template <int SIGN, int RADIX, typename C, typename R>
__device__ __forceinline__ void small_dft_ct(C* x) {
  if constexpr (RADIX == 2) {
    C a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  } else if constexpr (RADIX == 3) {
    const R k = (R)SIGN * (R)0.86602540378443864676372317075293618;
    C s = x[1] + x[2];
    C d = x[1] - x[2];
    C t1 = x[0] - (R)0.5 * s;
    C rot = imul(k, d);
    x[0] = x[0] + s;
    x[1] = t1 + rot;
    x[2] = t1 - rot;
  } else if constexpr (RADIX == 4) {
    C a0 = x[0] + x[2], a1 = x[0] - x[2];
    C b0 = x[1] + x[3], b1 = x[1] - x[3];
    C wb1 = imul((R)SIGN, b1);
    x[0] = a0 + b0;
    x[1] = a1 + wb1;
    x[2] = a0 - b0;
    x[3] = a1 - wb1;
  } else {
    // radix 8: length-4 DFTs of the even and the odd samples, combined with
    // w^u, w = e^{SIGN 2 pi i / 8} = (1 + SIGN i) / sqrt 2
    const C a0 = x[0] + x[4], a1 = x[0] - x[4], a2 = x[2] + x[6], a3 = x[2] - x[6];
    const C e0 = a0 + a2, e2 = a0 - a2;
    const C e1 = a1 + imul((R)SIGN, a3), e3 = a1 - imul((R)SIGN, a3);
    const C b0 = x[1] + x[5], b1 = x[1] - x[5], b2 = x[3] + x[7], b3 = x[3] - x[7];
    const C o0 = b0 + b2;
    const C p2 = b0 - b2;
    const C p1 = b1 + imul((R)SIGN, b3), p3 = b1 - imul((R)SIGN, b3);
    const R h = (R)0.70710678118654752440084436210484904;
    const C o1 = mk(h * (p1.x - (R)SIGN * p1.y), h * (p1.y + (R)SIGN * p1.x));    // p1 w
    const C o2 = imul((R)SIGN, p2);                                               // p2 w^2
    const C o3 = mk(h * (-p3.x - (R)SIGN * p3.y), h * (-p3.y + (R)SIGN * p3.x));  // p3 w^3
    x[0] = e0 + o0;
    x[4] = e0 - o0;
    x[1] = e1 + o1;
    x[5] = e1 - o1;
    x[2] = e2 + o2;
    x[6] = e2 - o2;
    x[3] = e3 + o3;
    x[7] = e3 - o3;
  }
}

// one DIF pass (natural order in, digit-reversed out after all passes)
template <int SIGN, typename R, int N, int ST, int NLINES, int G, bool BF_FASTEST, int NT>
__device__ __forceinline__ void dif_pass(typename cpx<R>::T* buf, const typename cpx<R>::T* tw) {
  using C = typename cpx<R>::T;
  constexpr int r = ct_radix(N, ST);
  constexpr int L = ct_len_before(N, ST);
  constexpr int m = L / r;
  constexpr int nb = N / r;
  constexpr int tstep = N / L;
  constexpr int total = NLINES * nb;
  for (int w = threadIdx.x; w < total; w += NT) {
    int l, bf;
    if (BF_FASTEST) { bf = w % nb; l = w / nb; } else { l = w % NLINES; bf = w / NLINES; }
    C* base = buf + (l / G) * (N * G) + (l % G);
    const int blk = bf / m, q = bf % m;
    const int i0 = blk * L + q;
    C x[r];
#pragma unroll
    for (int t = 0; t < r; ++t) x[t] = base[(i0 + t * m) * G];
    small_dft_ct<SIGN, r, C, R>(x);
#pragma unroll
    for (int u = 0; u < r; ++u) {
      C y = x[u];
      if (u > 0 && q > 0) y = cmul(y, twiddle<SIGN>(tw, q * u * tstep));
      base[(i0 + u * m) * G] = y;
    }
  }
  __syncthreads();
}

// one DIT pass, passes applied in reverse plan order (digit-reversed in, natural out)
template <int SIGN, typename R, int N, int ST, int NLINES, int G, bool BF_FASTEST, int NT>
__device__ __forceinline__ void dit_pass(typename cpx<R>::T* buf, const typename cpx<R>::T* tw) {
  using C = typename cpx<R>::T;
  constexpr int r = ct_radix(N, ST);
  constexpr int m = ct_len_before(N, ST + 1);  // sub-length before this pass in DIT order
  constexpr int L = m * r;
  constexpr int nb = N / r;
  constexpr int tstep = N / L;
  constexpr int total = NLINES * nb;
  for (int w = threadIdx.x; w < total; w += NT) {
    int l, bf;
    if (BF_FASTEST) { bf = w % nb; l = w / nb; } else { l = w % NLINES; bf = w / NLINES; }
    C* base = buf + (l / G) * (N * G) + (l % G);
    const int blk = bf / m, q = bf % m;
    const int i0 = blk * L + q;
    C x[r];
#pragma unroll
    for (int t = 0; t < r; ++t) {
      C v = base[(i0 + t * m) * G];
      if (t > 0 && q > 0) v = cmul(v, twiddle<SIGN>(tw, q * t * tstep));
      x[t] = v;
    }
    small_dft_ct<SIGN, r, C, R>(x);
#pragma unroll
    for (int u = 0; u < r; ++u) base[(i0 + u * m) * G] = x[u];
  }
  __syncthreads();
}

template <int SIGN, typename R, int N, int NLINES, int G, bool BF_FASTEST, int NT, int ST = 0>
__device__ __forceinline__ void fft_dif_ct(typename cpx<R>::T* buf, const typename cpx<R>::T* tw) {
  if constexpr (ST < ct_nst(N)) {
    dif_pass<SIGN, R, N, ST, NLINES, G, BF_FASTEST, NT>(buf, tw);
    fft_dif_ct<SIGN, R, N, NLINES, G, BF_FASTEST, NT, ST + 1>(buf, tw);
  }
}

template <int SIGN, typename R, int N, int NLINES, int G, bool BF_FASTEST, int NT, int ST = ct_nst(N) - 1>
__device__ __forceinline__ void fft_dit_ct(typename cpx<R>::T* buf, const typename cpx<R>::T* tw) {
  if constexpr (ST >= 0) {
    dit_pass<SIGN, R, N, ST, NLINES, G, BF_FASTEST, NT>(buf, tw);
    fft_dit_ct<SIGN, R, N, NLINES, G, BF_FASTEST, NT, ST - 1>(buf, tw);
  }
}

// ---------------------------------------------------------------------------
// launch structs
// ---------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz, nxh, P, N, mx, mz;
};

template <typename R>
struct PlaneArgs {
  using C = typename cpx<R>::T;
  const C* q;          // [B][6][ny][P]
  C* h;                // [B][3][ny][P]
  int nxh, nz, ny, mx, mz, P;
  int S, Lz, NP;
  const C* tw_x;       // [mx]  e^{2 pi i k / mx}
  const C* tw_z;       // [Lz]  e^{2 pi i k / Lz}
  const C* tw_mz;      // [mz]  e^{2 pi i k / mz}
  FftPlan px, pz;
  R scale;             // 1 / (mx mz)
  const int* active;   // [B] slots to process (nullptr: all)
  // planes of 16 x 16 modes in batches that fill the GPU: one plane per team
  // of threads, line transforms in registers (plane_small.cu)
  int team16;
  // planes that fit no cluster's shared memory: three passes through global
  // memory (z inverse, x transforms and products, z forward)
  int two_pass;
  C* y;                // [B][ny][6][mz][nxh] scratch: z-transformed columns, then H in fields 0..2
};

// Per-mode tau tables (device), mode index fastest so that threads owning
// consecutive modes read consecutive words.  Mh = N/2 + 1.
struct TauTables {
  const double* helm;      // [3][2][4][Mh][P]  e, h, b, Q of (D^2 - k^2 - 1/(beta dt nu)) per stage, parity
  const double* helm_isq;  // [3][2][P]         1 / sum Q
  const double* pois;      // [2][4][Mh][P]     same for (D^2 - k^2)
  const double* pois_isq;  // [2][P]
  const double* vh;        // [3][2][Mh][P]     homogeneous v of the influence matrix, parity-indexed
  const double* vh_idv;    // [3][2][P]         1 / sum_{n of parity} n^2 vh_n
  const double* u1;        // [3][Mh]           mean response to unit forcing (even parity)
  const double* u1_iflux;  // [3]               1 / int u1 dy
  const double* rowc;      // [3][ny]           tau row constants cA_n, cB_n, cC_n
  // no-slip top (top_bc = 0): the same factorisations with the row constants
  // folded in, eA = e cA_n, eB = e cB_n, eC = e cC_n, then h, b, the wall
  // weights W (W_{M-1} = 1, W_i = 1 + b_{i+1} W_{i+1}: sum_i P_i = sum_i W_i a_i)
  // and, for the stage's Helmholtz operator, E1 = (1 + alpha/beta) e
  const double* helm_f;    // [3][2][7][Mh][P]  eA, eB, eC, h, b, W, E1 per stage, parity
  const double* pois_f;    // [2][6][Mh][P]     eA, eB, eC, h, b, W
  // free-slip top (top_bc = 1): the wall rows couple the parities
  const double* helm_top;  // [3][2][2][P]      sum Q, sum n^2 Q of the stage's factorisation, per parity
  const double* vh_top;    // [3][2][2][P]      A = sum n^2 (n^2 - 1) / 3 vh_n, B = sum n^2 vh_n, per parity
  int Mh;
  int top_bc;              // 0 no-slip upper wall; 1 free slip (u1 then holds the affine forcing response)
};

// Shared memory of the batched implicit half before its exchange slots: the
// tile of H, [3][ny][ppc] complex in the node precision, then for FP32 nodes
// the staged previous right-hand sides [2][ny][ppc] (FP32 pairs), for FP64
// nodes six more complex values per mode (scratch of the fast analysis);
// 16-byte aligned.
constexpr bool kPostStageHV = true, kPostStageHG = true;
__host__ __device__ inline size_t stage_post_batched_tile_bytes(int ny, int ppc, size_t node_bytes) {
  const size_t staged = (size_t)kPostStageHV + (size_t)kPostStageHG;
  const size_t b = node_bytes == 8 ? (3 + staged) * ny * ppc * 8 : ((size_t)3 * ny + 6) * ppc * 16;
  return (b + 15) & ~(size_t)15;
}

struct StageCoef {
  double alpha, beta, gamma, zeta, dt, nu, theta, flux;
  int k;
};

}  // namespace chdns
