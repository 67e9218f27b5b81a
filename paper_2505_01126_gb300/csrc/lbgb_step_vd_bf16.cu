// BF16 shifted population storage, density and viscosity contrasts.
#define LBGB_FT __nv_bfloat16
#define LBGB_MC false
#include "lbgb_step_vd_impl.cuh"
