// Predictor/corrector kernels of degree N = 3 (one translation unit per degree
// so that the build compiles them in parallel).
#include "dg_step_kernels.cuh"

DG_INSTANTIATE_STEP(3)
