// Implicit stage halves under a free-slip top (open channel), MH = 33.
#include "stage_kernels.cuh"

CH_STAGE_INSTANTIATE_OPEN(33)
