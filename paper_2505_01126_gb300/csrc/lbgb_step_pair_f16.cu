// FP16 shifted population storage, paired step kernel.
#define LBGB_FT __half
#include "lbgb_step_pair_impl.cuh"
