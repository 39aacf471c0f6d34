// Fused stage kernels instantiated for MH = 49.
#include "stage_kernels.cuh"

CH_STAGE_INSTANTIATE(49)
