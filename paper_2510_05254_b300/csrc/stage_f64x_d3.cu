// Fused stage kernels, double, 3D, degrees 1..7, both equations: exact-mass variant.
#define NDG_REAL double
#define NDG_DIM 3
#define NDG_EXACT true
#define NDG_TAG stage_f64x_d3
#include "stage_dispatch.cuh"
