// FP32 population storage, density and viscosity contrasts.
#define LBGB_FT float
#define LBGB_MC false
#include "lbgb_step_vd_impl.cuh"
