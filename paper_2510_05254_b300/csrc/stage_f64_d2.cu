// Fused stage kernels, double, 2D, degrees 1..7, both equations.
#define NDG_REAL double
#define NDG_DIM 2
#define NDG_TAG stage_f64_d2
#include "stage_dispatch.cuh"
