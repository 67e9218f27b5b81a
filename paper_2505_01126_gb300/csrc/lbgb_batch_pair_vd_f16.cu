// FP16 shifted populations: the batch kernel with the paired tile body and density contrasts.
#define LBGB_FT __half
#include "lbgb_batch_pair_vd_impl.cuh"
