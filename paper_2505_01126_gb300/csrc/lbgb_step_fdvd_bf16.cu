// BF16 shifted population storage, finite-difference phase field with density and viscosity contrasts.
#define LBGB_FT __nv_bfloat16
#define LBGB_MC false
#define LBGB_VD true
#define LBGB_PF true
#include "lbgb_step_x_impl.cuh"
