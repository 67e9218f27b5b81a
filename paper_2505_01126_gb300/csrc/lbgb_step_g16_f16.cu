// FP16 shifted populations and FP16 shifted D3Q7 populations: one-site kernels.
#define LBGB_FT __half
#include "lbgb_step_g16_impl.cuh"
