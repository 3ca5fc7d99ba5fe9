// Fused stage kernels, FP64 state with the D contraction in float-float, 2D, degrees 1..7.
#define NDG_REAL double
#define NDG_DIM 2
#define NDG_FF true
#define NDG_TAG stage_f64ff_d2
#include "stage_dispatch.cuh"
