// Fused stage kernels, float, 3D, degrees 1..7, both equations: exact-mass variant.
#define NDG_REAL float
#define NDG_DIM 3
#define NDG_EXACT true
#define NDG_TAG stage_f32x_d3
#include "stage_dispatch.cuh"
