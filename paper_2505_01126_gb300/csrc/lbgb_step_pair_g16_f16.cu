// FP16 shifted populations and FP16 shifted D3Q7 populations: the paired step kernel.
#define LBGB_FT __half
#define LBGB_G16_PAIR 1
#include "lbgb_step_g16_impl.cuh"
