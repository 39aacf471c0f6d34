// Fused stage kernels instantiated for MH = 33.
#include "stage_kernels.cuh"

CH_STAGE_INSTANTIATE(33)
