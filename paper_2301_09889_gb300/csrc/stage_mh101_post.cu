// Fused stage kernels instantiated for MH = 101, per-tile implicit half.
#include "stage_kernels.cuh"

CH_STAGE_POST(101)
