// Fused stage kernels, double, 1D, degrees 1..7, both equations.
#define NDG_REAL double
#define NDG_DIM 1
#define NDG_TAG stage_f64_d1
#include "stage_dispatch.cuh"
