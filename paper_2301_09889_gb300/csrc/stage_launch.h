// Per-MH launchers of the fused stage kernels.  MH bounds the per-thread
// register arrays (unknowns of one parity); each bucket is compiled in its own
// translation unit (stage_mh*.cu) so that the instantiations build in parallel.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace chdns {

template <typename RN, int MH>
cudaError_t pre_mh(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, typename cpx<RN>::T* q, int ppc,
                   size_t smem, cudaStream_t st);
template <typename RN, int MH, int TOP>
cudaError_t post_mh(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, const typename cpx<RN>::T* h,
                    const StageCoef& sc, int ppc, size_t smem, cudaStream_t st);
template <typename RN, int MH, int TOP>
cudaError_t post_batched_mh(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                            const typename cpx<RN>::T* h, const StageCoef& sc, int ppc, size_t smem,
                            cudaStream_t st);

}  // namespace chdns
