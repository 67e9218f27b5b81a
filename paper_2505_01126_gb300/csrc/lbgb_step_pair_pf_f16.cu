// FP16 shifted population storage, paired step kernel with the finite-difference phase field.
#define LBGB_FT __half
#define LBGB_PAIR_PF 1
#include "lbgb_step_pair_impl.cuh"
