// BF16 shifted populations and BF16 shifted D3Q7 populations: the paired step kernel.
#define LBGB_FT __nv_bfloat16
#define LBGB_G16_PAIR 1
#include "lbgb_step_g16_impl.cuh"
