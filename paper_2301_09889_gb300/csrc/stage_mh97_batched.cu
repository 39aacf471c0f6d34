// Fused stage kernels instantiated for MH = 97 (193 nodes, N = 192: the FFT
// form of the Chebyshev transforms), batched implicit half.
#include "stage_kernels.cuh"

CH_STAGE_POST_BATCHED(97)
