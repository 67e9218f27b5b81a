// Moment-only storage, density and viscosity contrasts.
#define LBGB_FT float
#define LBGB_MC true
#include "lbgb_step_vd_impl.cuh"
