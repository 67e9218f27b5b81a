// FP32 population storage, density and viscosity contrasts.
#define LBGB_FT float
#define LBGB_MC false
#define LBGB_VD true
#define LBGB_PF false
#include "lbgb_step_x_impl.cuh"
