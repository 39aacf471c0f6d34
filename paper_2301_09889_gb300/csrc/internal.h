// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace chdns {

template <typename R>
cudaError_t launch_plane(const PlaneArgs<R>& a, int B, size_t smem, cudaStream_t st);
template <typename R>
cudaError_t plane_max_clusters(const PlaneArgs<R>& a, size_t smem, int* clusters);
// nonlinear term of planes of 16 x 16 modes, line transforms in registers (plane_small.cu)
bool plane16_shape(int mx, int mz, int nxh, int nz);
template <typename R>
cudaError_t launch_plane16(const PlaneArgs<R>& a, int B, cudaStream_t st);
// nonlinear term in three passes through global memory (plane2.cu), FP64
bool two_pass_shape_ok(int mx, int mz, int nxh);
bool two_pass_chosen(int mx, int mz, int nxh, bool fp64);
template <typename R>
cudaError_t launch_plane_two_pass(const PlaneArgs<R>& a, int B, cudaStream_t st);

struct PencilBufs {
  double2 *V, *G;               // [B][ny][P]
  double2 *HVP, *HGP;           // [B][ny][P] complex in the node precision (FP32 pairs in mixed mode)
  double *UM, *WM, *HXP, *HZP;  // [B][ny]
  double2* Q;                   // [B][6][ny][P] node values of u, v, w, ox, oy, oz (nonlinear input)
  double2* R;                   // [B][3][ny][P] node values of H
  double2 *vw_old, *vw_new;     // [B][P] wall-velocity spectra
  double2* planes;              // [B][2][P] u, v spectra at the sensing node
  double* tau_acc;              // [B]
  const int* active;            // [B] slots advanced by this step (nullptr: all)
};

struct DevTables {
  const double* kx;    // [nxh]
  const double* kz;    // [nz]
  const double* cheb;  // [ny][ny] cos(pi j n / N)
  const float* cheb_f; // the same table in FP32 (mixed precision)
  const double* dts;   // [ny] T_n'(y_js) at the sensing node
  TauTables tau;
  const double2* tw_nx;  // [nx]
  const double2* tw_nz;  // [nz]
  const double2* tw_cheb;  // [N] e^{2 pi i k / N}: fast Chebyshev synthesis
};

// fused wall-normal halves of a stage (stage.cu); ppc = modes per CTA
size_t stage_pre_smem(const Grid& g, int ppc, size_t node_bytes);  // node_bytes: one complex node value
size_t stage_post_smem(const Grid& g, int Mh, int ppc, int top);
size_t stage_post_batched_smem(const Grid& g, int ppc, int top, size_t node_bytes);
// kernels one launch_stage_post issues (the batched form above 65 nodes: two)
int stage_post_launches(const Grid& g, int top, bool batched);
template <typename RN>
cudaError_t launch_stage_pre(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                             typename cpx<RN>::T* q, int ppc, cudaStream_t st);
// batched: one thread per (mode, class, component) and only H staged in shared
// memory (for batches that supply many modes); otherwise one thread per
// (mode, class, component, equation) on a shared-memory tile
template <typename RN>
cudaError_t launch_stage_post(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                              const typename cpx<RN>::T* h, const StageCoef& sc, int ppc, bool batched,
                              cudaStream_t st);
cudaError_t launch_wall_shear(const Grid& g, int B, const double* UM, double nu, double* acc,
                              const int* active, cudaStream_t st);
cudaError_t launch_sense(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, int js,
                         double alpha, int opposition, cudaStream_t st);
cudaError_t launch_obs(const Grid& g, int B, const double2* planes, const DevTables& t, double* out,
                       size_t out_stride, const int* active, cudaStream_t st);
cudaError_t launch_action(const Grid& g, int B, const double* act, double u_tau, const DevTables& t,
                          const PencilBufs& pb, cudaStream_t st);
cudaError_t launch_finalize(int B, const double* acc, double inv_steps, double tau_ref, double* out,
                            size_t out_stride, size_t out_offset, const int* active, cudaStream_t st);
cudaError_t launch_tau_helmholtz(int ny, int M, const double* lam, const double2* r, const double2* top,
                                 const double2* bot, double2* f, cudaStream_t st);

// on-device policy (policy.cu): a multilayer perceptron shared by every agent
constexpr int kPolicyMaxWidth = 64;
constexpr int kPolicyMaxWindow = 7;
// weights of the largest network: 2 (7 x 7) inputs, two hidden layers of 64
constexpr int kPolicyMaxWeights =
    kPolicyMaxWidth * 2 * kPolicyMaxWindow * kPolicyMaxWindow + kPolicyMaxWidth +
    kPolicyMaxWidth * kPolicyMaxWidth + kPolicyMaxWidth + kPolicyMaxWidth + 1;
struct PolicyDesc {
  int wz, wx;      // observation window (odd)
  int n_hidden;    // 0, 1 or 2 ReLU layers
  int h1, h2;      // hidden widths
  int out_tanh;    // 1: action = u_tau tanh(y)
  int n_weights;   // FP32 values at w
};
int policy_weight_count(const PolicyDesc& d);
// plane [B][2][nz][nx] (u, v on the sensing plane) -> act [B][nz][nx]
cudaError_t launch_policy(int nx, int nz, int B, const PolicyDesc& d, const float* w, const double* plane,
                          double* act, double u_tau, const int* active, cudaStream_t st);

}  // namespace chdns

struct ch_env;
namespace chdns {
// internal entry points of api.cu used by the serving layer
int step_masked(ch_env* env, const double* d_action, const int* d_active, const int* h_active);
double* env_dout(ch_env* env);
double* env_dact(ch_env* env);
size_t env_out_stride(const ch_env* env);
cudaStream_t env_stream(const ch_env* env);
int env_slot_seed(ch_env* env, int e, uint64_t seed, double amplitude, int kmax);
size_t env_footprint(const struct ch_params* p);
}  // namespace chdns
