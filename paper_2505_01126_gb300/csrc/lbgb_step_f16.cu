// FP16 shifted population storage.
#define LBGB_FT __half
#include "lbgb_step_impl.cuh"
