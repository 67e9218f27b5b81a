// FP16 shifted population storage, density and viscosity contrasts.
#define LBGB_FT __half
#define LBGB_MC false
#define LBGB_VD true
#define LBGB_PF false
#include "lbgb_step_x_impl.cuh"
