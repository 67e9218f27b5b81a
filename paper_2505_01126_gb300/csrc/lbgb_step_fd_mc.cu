// Moment-only storage, finite-difference phase field.
#define LBGB_FT float
#define LBGB_MC true
#define LBGB_VD false
#define LBGB_PF true
#include "lbgb_step_x_impl.cuh"
