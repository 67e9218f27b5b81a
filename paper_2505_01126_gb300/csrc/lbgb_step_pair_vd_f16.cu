// FP16 shifted population storage, paired step kernel with density and viscosity contrasts.
#define LBGB_FT __half
#define LBGB_PAIR_VD 1
#include "lbgb_step_pair_impl.cuh"
