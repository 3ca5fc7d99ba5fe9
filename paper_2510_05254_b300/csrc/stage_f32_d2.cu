// Fused stage kernels, float, 2D, degrees 1..7, both equations.
#define NDG_REAL float
#define NDG_DIM 2
#define NDG_TAG stage_f32_d2
#include "stage_dispatch.cuh"
