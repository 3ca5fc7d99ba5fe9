// Fused stage kernels, double, 2D, degrees 1..7, both equations: exact-mass variant.
#define NDG_REAL double
#define NDG_DIM 2
#define NDG_EXACT true
#define NDG_TAG stage_f64x_d2
#include "stage_dispatch.cuh"
