// Fused stage kernels instantiated for MH = 65, per-tile forms.
#include "stage_kernels.cuh"

CH_STAGE_PRE(65)
CH_STAGE_POST(65)
