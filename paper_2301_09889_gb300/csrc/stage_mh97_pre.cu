// Fused stage kernels instantiated for MH = 97 (193 nodes, N = 192: the FFT
// form of the Chebyshev transforms), explicit half.
#include "stage_kernels.cuh"

CH_STAGE_PRE(97)
