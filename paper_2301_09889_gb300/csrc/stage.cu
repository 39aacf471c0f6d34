// Dispatch of the fused stage kernels (stage_kernels.cuh) to the register-array
// bucket MH that covers one parity of the Chebyshev unknowns, and their
// shared-memory sizes.
#include "stage_launch.h"

namespace chdns {

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int mh_bucket(int need) {
  const int b[] = {5, 9, 17, 33, 49, 65, 97, 101};
  for (int v : b)
    if (need <= v) return v;
  return 0;
}

// (plus two complex values per line for the fast synthesis)
size_t stage_pre_smem(const Grid& g, int ppc, size_t node_bytes) {
  return (size_t)8 * g.ny * ppc * node_bytes + (size_t)12 * ppc * sizeof(double2);
}
// (both with six complex values per mode for the FP64 fast analysis; the
// coefficient tile is smaller in FP32 node precision, the FP64 size bounds both;
// a free-slip top adds the exchange slots of the parity closures to the
// per-tile form: six values per thread; the batched form exchanges them by
// shuffles)
// Above 65 nodes (no-slip top) the batched form runs in two launches and its
// solve keeps one array of MH doubles per thread in shared memory.
size_t stage_post_batched_smem(const Grid& g, int ppc, int top, size_t node_bytes) {
  const int mh = mh_bucket(g.N / 2 + 1);
  if (!top && mh > 33) return (size_t)4 * ppc * mh * sizeof(double);
  return stage_post_batched_tile_bytes(g.ny, ppc, node_bytes);
}
int stage_post_launches(const Grid& g, int top, bool batched) {
  return (batched && !top && mh_bucket(g.N / 2 + 1) > 33) ? 2 : 1;
}
size_t stage_post_smem(const Grid& g, int Mh, int ppc, int top) {
  return ((size_t)7 * g.ny + 6) * ppc * sizeof(double2) + ((size_t)18 * Mh * ppc + 6 * ppc) * sizeof(double) +
         (top ? (size_t)8 * ppc * 6 * sizeof(double) : 0);
}

template <typename RN>
cudaError_t launch_stage_pre(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                             typename cpx<RN>::T* q, int ppc, cudaStream_t st) {
  const size_t smem = stage_pre_smem(g, ppc, sizeof(typename cpx<RN>::T));
  // 16 (MH - 1) / 16 >= (N + 1) / 2 node pairs per mode
  switch (mh_bucket((g.N + 1) / 2 + 1)) {
    case 5: return pre_mh<RN, 5>(g, B, pb, t, q, ppc, smem, st);
    case 9: return pre_mh<RN, 9>(g, B, pb, t, q, ppc, smem, st);
    case 17: return pre_mh<RN, 17>(g, B, pb, t, q, ppc, smem, st);
    case 33: return pre_mh<RN, 33>(g, B, pb, t, q, ppc, smem, st);
    case 49: return pre_mh<RN, 49>(g, B, pb, t, q, ppc, smem, st);
    case 65: return pre_mh<RN, 65>(g, B, pb, t, q, ppc, smem, st);
    case 97: return pre_mh<RN, 97>(g, B, pb, t, q, ppc, smem, st);
    case 101: return pre_mh<RN, 101>(g, B, pb, t, q, ppc, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename RN>
cudaError_t launch_stage_post(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                              const typename cpx<RN>::T* h, const StageCoef& sc, int ppc, bool batched,
                              cudaStream_t st) {
  const int top = t.tau.top_bc;
  const int mh = mh_bucket(g.N / 2 + 1);
  if (top) {
    // free-slip top: built for MH <= 33 (ny <= 65)
    if (batched) {
      const size_t smem = stage_post_batched_smem(g, ppc, 1, sizeof(typename cpx<RN>::T));
      switch (mh) {
        case 5: return post_batched_mh<RN, 5, 1>(g, B, pb, t, h, sc, ppc, smem, st);
        case 9: return post_batched_mh<RN, 9, 1>(g, B, pb, t, h, sc, ppc, smem, st);
        case 17: return post_batched_mh<RN, 17, 1>(g, B, pb, t, h, sc, ppc, smem, st);
        case 33: return post_batched_mh<RN, 33, 1>(g, B, pb, t, h, sc, ppc, smem, st);
        default: return cudaErrorInvalidValue;
      }
    }
    const size_t smem = stage_post_smem(g, t.tau.Mh, ppc, 1);
    switch (mh) {
      case 5: return post_mh<RN, 5, 1>(g, B, pb, t, h, sc, ppc, smem, st);
      case 9: return post_mh<RN, 9, 1>(g, B, pb, t, h, sc, ppc, smem, st);
      case 17: return post_mh<RN, 17, 1>(g, B, pb, t, h, sc, ppc, smem, st);
      case 33: return post_mh<RN, 33, 1>(g, B, pb, t, h, sc, ppc, smem, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (batched) {
    const size_t smem = stage_post_batched_smem(g, ppc, 0, sizeof(typename cpx<RN>::T));
    switch (mh) {
      case 5: return post_batched_mh<RN, 5, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 9: return post_batched_mh<RN, 9, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 17: return post_batched_mh<RN, 17, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 33: return post_batched_mh<RN, 33, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 49: return post_batched_mh<RN, 49, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 65: return post_batched_mh<RN, 65, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 97: return post_batched_mh<RN, 97, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      case 101: return post_batched_mh<RN, 101, 0>(g, B, pb, t, h, sc, ppc, smem, st);
      default: return cudaErrorInvalidValue;
    }
  }
  const size_t smem = stage_post_smem(g, t.tau.Mh, ppc, 0);
  switch (mh) {
    case 5: return post_mh<RN, 5, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 9: return post_mh<RN, 9, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 17: return post_mh<RN, 17, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 33: return post_mh<RN, 33, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 49: return post_mh<RN, 49, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 65: return post_mh<RN, 65, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 97: return post_mh<RN, 97, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    case 101: return post_mh<RN, 101, 0>(g, B, pb, t, h, sc, ppc, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_stage_pre<double>(const Grid&, int, const PencilBufs&, const DevTables&, double2*, int,
                                              cudaStream_t);
template cudaError_t launch_stage_post<double>(const Grid&, int, const PencilBufs&, const DevTables&, const double2*,
                                               const StageCoef&, int, bool, cudaStream_t);
template cudaError_t launch_stage_pre<float>(const Grid&, int, const PencilBufs&, const DevTables&, float2*, int,
                                             cudaStream_t);
template cudaError_t launch_stage_post<float>(const Grid&, int, const PencilBufs&, const DevTables&, const float2*,
                                              const StageCoef&, int, bool, cudaStream_t);

}  // namespace chdns
