// BF16 shifted populations and BF16 shifted D3Q7 populations: one-site kernels.
#define LBGB_FT __nv_bfloat16
#include "lbgb_step_g16_impl.cuh"
