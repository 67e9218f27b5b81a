// FP16 shifted population storage, finite-difference phase field.
#define LBGB_FT __half
#define LBGB_MC false
#define LBGB_VD false
#define LBGB_PF true
#include "lbgb_step_x_impl.cuh"
