// BF16 shifted population storage, paired step kernel with density and viscosity contrasts.
#define LBGB_FT __nv_bfloat16
#define LBGB_PAIR_VD 1
#include "lbgb_step_pair_impl.cuh"
