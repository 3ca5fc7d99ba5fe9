// Fused stage kernels, float, 1D, degrees 1..7, both equations.
#define NDG_REAL float
#define NDG_DIM 1
#define NDG_TAG stage_f32_d1
#include "stage_dispatch.cuh"
