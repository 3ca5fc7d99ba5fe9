// Fused stage kernels, FP64 state with the D contraction in float-float, 1D, degrees 1..7.
#define NDG_REAL double
#define NDG_DIM 1
#define NDG_FF true
#define NDG_TAG stage_f64ff_d1
#include "stage_dispatch.cuh"
