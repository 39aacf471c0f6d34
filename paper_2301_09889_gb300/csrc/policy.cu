// On-device policy: the wall action of every agent from its local observation
// (paper Sec. 3.2: one agent per wall grid point, all sharing one policy that
// maps the observed portion of the sensing plane above the actuator to a
// wall-normal velocity; Sec. 3.2 trains it with DDPG, whose actor is a
// multilayer perceptron).  The paper gives no architecture; this one is a
// perceptron with 0, 1 or 2 ReLU hidden layers of up to 64 units and a
// linear or u_tau tanh output, evaluated in FP32.
//
// Input of agent (b, iz, ix): x[(c wz + dz) wx + dx] = plane c (0: u, 1: v)
// at row (iz + dz - wz/2) mod nz, column (ix + dx - wx/2) mod nx.  Weights, per
// layer: W [out][in] row-major, then the bias [out]; the last layer has one
// output.  One thread per agent; the weights are staged in shared memory and
// every thread reads the same weight at the same time (broadcast).

#include "internal.h"

namespace chdns {

int policy_weight_count(const PolicyDesc& d) {
  const int K = 2 * d.wz * d.wx;
  if (d.n_hidden == 0) return K + 1;
  if (d.n_hidden == 1) return d.h1 * K + d.h1 + d.h1 + 1;
  return d.h1 * K + d.h1 + d.h2 * d.h1 + d.h2 + d.h2 + 1;
}

namespace {

template <int HMAX>
__global__ void __launch_bounds__(256) policy_kernel(int nx, int nz, int B, PolicyDesc d,
                                                     const float* __restrict__ w, const double* __restrict__ plane,
                                                     double* __restrict__ act, double u_tau,
                                                     const int* __restrict__ active) {
  extern __shared__ float sw[];
  for (int i = threadIdx.x; i < d.n_weights; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const long a = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= (long)B * nz * nx) return;
  const int b = (int)(a / ((long)nz * nx));
  const int r = (int)(a % ((long)nz * nx));
  const int iz = r / nx, ix = r % nx;
  if (active && !active[b]) return;
  const double* pl = plane + (size_t)b * 2 * nz * nx;
  const int wz = d.wz, wx = d.wx, K = 2 * wz * wx;
  auto input = [&](int k) -> float {
    const int c = k / (wz * wx), q = k % (wz * wx);
    int zz = iz + q / wx - wz / 2, xx = ix + q % wx - wx / 2;
    zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
    return (float)pl[((size_t)c * nz + zz) * nx + xx];
  };
  float y;
  if (d.n_hidden == 0) {
    y = sw[K];
    for (int k = 0; k < K; ++k) y = fmaf(sw[k], input(k), y);
  } else {
    const int H1 = d.h1;
    const float* W0 = sw;
    const float* b0 = W0 + H1 * K;
    float h[HMAX];
#pragma unroll
    for (int j = 0; j < HMAX; ++j) h[j] = j < H1 ? b0[j] : 0.0f;
    for (int k = 0; k < K; ++k) {
      const float x = input(k);
#pragma unroll
      for (int j = 0; j < HMAX; ++j)
        if (j < H1) h[j] = fmaf(W0[j * K + k], x, h[j]);
    }
#pragma unroll
    for (int j = 0; j < HMAX; ++j) h[j] = fmaxf(h[j], 0.0f);
    const float* L1 = b0 + H1;
    if (d.n_hidden == 1) {
      y = L1[H1];
#pragma unroll
      for (int j = 0; j < HMAX; ++j)
        if (j < H1) y = fmaf(L1[j], h[j], y);
    } else {
      const int H2 = d.h2;
      const float* W1 = L1;
      const float* b1 = W1 + H2 * H1;
      const float* Wo = b1 + H2;
      y = Wo[H2];
      for (int j2 = 0; j2 < H2; ++j2) {
        float s = b1[j2];
#pragma unroll
        for (int j = 0; j < HMAX; ++j)
          if (j < H1) s = fmaf(W1[j2 * H1 + j], h[j], s);
        y = fmaf(Wo[j2], fmaxf(s, 0.0f), y);
      }
    }
  }
  act[a] = d.out_tanh ? u_tau * (double)tanhf(y) : (double)y;
}

// Two hidden layers of 64, the widths in use: the first layer is staged
// transposed (W0t[k][j]) so that both layers read their weights as float4
// broadcasts, and the unit loops have no width predicate.  Same operations in
// the same order as policy_kernel.
__global__ void __launch_bounds__(256) policy_kernel_64x64(int nx, int nz, int B, PolicyDesc d,
                                                           const float* __restrict__ w,
                                                           const double* __restrict__ plane,
                                                           double* __restrict__ act, double u_tau,
                                                           const int* __restrict__ active) {
  constexpr int H = 64;
  extern __shared__ __align__(16) float sw[];
  const int wz = d.wz, wx = d.wx, K = 2 * wz * wx;
  for (int i = threadIdx.x; i < d.n_weights; i += blockDim.x) {
    int o = i;
    if (i < H * K) o = (i % K) * H + i / K;  // W0[j][k] -> W0t[k][j]
    sw[o] = w[i];
  }
  __syncthreads();
  const long a = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= (long)B * nz * nx) return;
  const int b = (int)(a / ((long)nz * nx));
  const int r = (int)(a % ((long)nz * nx));
  const int iz = r / nx, ix = r % nx;
  if (active && !active[b]) return;
  const double* pl = plane + (size_t)b * 2 * nz * nx;
  const float* b0 = sw + H * K;
  const float* W1 = b0 + H;
  const float* b1 = W1 + H * H;
  const float* Wo = b1 + H;
  float h[H];
#pragma unroll
  for (int j = 0; j < H; ++j) h[j] = b0[j];
  for (int k = 0; k < K; ++k) {
    const int c = k / (wz * wx), q = k % (wz * wx);
    int zz = iz + q / wx - wz / 2, xx = ix + q % wx - wx / 2;
    zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
    const float x = (float)pl[((size_t)c * nz + zz) * nx + xx];
    const float4* w4 = reinterpret_cast<const float4*>(sw + k * H);
#pragma unroll
    for (int u = 0; u < H / 4; ++u) {
      const float4 v = w4[u];
      h[4 * u + 0] = fmaf(v.x, x, h[4 * u + 0]);
      h[4 * u + 1] = fmaf(v.y, x, h[4 * u + 1]);
      h[4 * u + 2] = fmaf(v.z, x, h[4 * u + 2]);
      h[4 * u + 3] = fmaf(v.w, x, h[4 * u + 3]);
    }
  }
#pragma unroll
  for (int j = 0; j < H; ++j) h[j] = fmaxf(h[j], 0.0f);
  float y = Wo[H];
  for (int j2 = 0; j2 < H; ++j2) {
    const float4* r4 = reinterpret_cast<const float4*>(W1 + j2 * H);
    float s = b1[j2];
#pragma unroll
    for (int u = 0; u < H / 4; ++u) {
      const float4 v = r4[u];
      s = fmaf(v.x, h[4 * u + 0], s);
      s = fmaf(v.y, h[4 * u + 1], s);
      s = fmaf(v.z, h[4 * u + 2], s);
      s = fmaf(v.w, h[4 * u + 3], s);
    }
    y = fmaf(Wo[j2], fmaxf(s, 0.0f), y);
  }
  act[a] = d.out_tanh ? u_tau * (double)tanhf(y) : (double)y;
}

}  // namespace

cudaError_t launch_policy(int nx, int nz, int B, const PolicyDesc& d, const float* w, const double* plane,
                          double* act, double u_tau, const int* active, cudaStream_t st) {
  const long agents = (long)B * nz * nx;
  constexpr int kThreads = 256;
  const size_t smem = (size_t)d.n_weights * sizeof(float);
  static SmemLimit lim_generic, lim_64x64;
  const size_t bytes = kPolicyMaxWeights * sizeof(float);
  cudaError_t e = raise_smem_limit(policy_kernel<kPolicyMaxWidth>, &lim_generic, bytes);
  if (e == cudaSuccess) e = raise_smem_limit(policy_kernel_64x64, &lim_64x64, bytes);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((agents + kThreads - 1) / kThreads);
  if (d.n_hidden == 2 && d.h1 == 64 && d.h2 == 64) {
    policy_kernel_64x64<<<blocks, kThreads, smem, st>>>(nx, nz, B, d, w, plane, act, u_tau, active);
  } else {
    policy_kernel<kPolicyMaxWidth><<<blocks, kThreads, smem, st>>>(nx, nz, B, d, w, plane, act, u_tau, active);
  }
  return cudaGetLastError();
}

}  // namespace chdns
