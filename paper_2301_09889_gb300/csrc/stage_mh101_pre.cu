// Fused stage kernels instantiated for MH = 101, explicit half.
#include "stage_kernels.cuh"

CH_STAGE_PRE(101)
