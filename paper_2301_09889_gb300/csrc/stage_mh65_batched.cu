// Fused stage kernels instantiated for MH = 65, batched implicit half.
#include "stage_kernels.cuh"

CH_STAGE_POST_BATCHED(65)
