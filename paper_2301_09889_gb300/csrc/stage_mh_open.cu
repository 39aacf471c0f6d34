// Implicit stage halves under a free-slip top (open channel), MH = 5, 9, 17.
#include "stage_kernels.cuh"

CH_STAGE_INSTANTIATE_OPEN(5)
CH_STAGE_INSTANTIATE_OPEN(9)
CH_STAGE_INSTANTIATE_OPEN(17)
