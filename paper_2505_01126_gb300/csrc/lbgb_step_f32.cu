// FP32 population storage.
#define LBGB_FT float
#include "lbgb_step_impl.cuh"
