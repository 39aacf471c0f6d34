// Fused stage kernels instantiated for MH = 5, 9, 17.
#include "stage_kernels.cuh"

CH_STAGE_INSTANTIATE(5)
CH_STAGE_INSTANTIATE(9)
CH_STAGE_INSTANTIATE(17)
