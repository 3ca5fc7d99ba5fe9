// Fused stage kernels, double, 1D, degrees 1..7, both equations: exact-mass variant.
#define NDG_REAL double
#define NDG_DIM 1
#define NDG_EXACT true
#define NDG_TAG stage_f64x_d1
#include "stage_dispatch.cuh"
