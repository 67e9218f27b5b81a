// BF16 shifted population storage.
#define LBGB_FT __nv_bfloat16
#include "lbgb_step_impl.cuh"
