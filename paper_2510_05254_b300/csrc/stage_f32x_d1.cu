// Fused stage kernels, float, 1D, degrees 1..7, both equations: exact-mass variant.
#define NDG_REAL float
#define NDG_DIM 1
#define NDG_EXACT true
#define NDG_TAG stage_f32x_d1
#include "stage_dispatch.cuh"
