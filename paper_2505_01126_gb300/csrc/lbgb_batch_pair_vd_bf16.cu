// BF16 shifted populations: the batch kernel with the paired tile body and density contrasts.
#define LBGB_FT __nv_bfloat16
#include "lbgb_batch_pair_vd_impl.cuh"
