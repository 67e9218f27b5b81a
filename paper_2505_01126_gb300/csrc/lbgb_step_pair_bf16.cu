// BF16 shifted population storage, paired step kernel.
#define LBGB_FT __nv_bfloat16
#include "lbgb_step_pair_impl.cuh"
