// FP16 shifted population storage, density and viscosity contrasts.
#define LBGB_FT __half
#define LBGB_MC false
#include "lbgb_step_vd_impl.cuh"
