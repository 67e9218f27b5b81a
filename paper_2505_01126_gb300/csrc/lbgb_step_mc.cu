// Moment-only storage: launcher of the fused kernel with MC = true (the f
// populations are rebuilt from the neighbours' ten post-collision
// coefficients; FP32 throughout).
#include "lbgb_kernels.cuh"

namespace lbgb {

template <int TY, int MODE, bool VEC>
static void launch_mc_kernel(int pull, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (pull) fused_step_kernel<float, TY, MODE, 1, VEC, true><<<grid, 32 * TY, 0, st>>>(a);
    else fused_step_kernel<float, TY, MODE, 0, VEC, true><<<grid, 32 * TY, 0, st>>>(a);
}

cudaError_t launch_fused_mc(int mode, int pull, int ty, bool vec, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (mode == MODE_INIT) {
        if (ty != 8) return cudaErrorInvalidValue;
        fused_step_kernel<float, 8, MODE_INIT, 0, false, true><<<grid, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (mode == MODE_MOMENTS) {
        if (ty != 8) return cudaErrorInvalidValue;
        launch_mc_kernel<8, MODE_MOMENTS, false>(pull, grid, a, st);
        return cudaGetLastError();
    }
    if (mode != MODE_STEP) return cudaErrorInvalidValue;
    if (ty == 4) {
        if (vec) launch_mc_kernel<4, MODE_STEP, true>(pull, grid, a, st);
        else launch_mc_kernel<4, MODE_STEP, false>(pull, grid, a, st);
    } else if (ty == 8) {
        if (vec) launch_mc_kernel<8, MODE_STEP, true>(pull, grid, a, st);
        else launch_mc_kernel<8, MODE_STEP, false>(pull, grid, a, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int TY, bool VEC>
static void launch_batch_mc_ty(int pull, int blocks, const BatchArgs& b, cudaStream_t st) {
    if (pull) batch_step_kernel<float, TY, 1, VEC, true><<<blocks, 32 * TY, 0, st>>>(b);
    else batch_step_kernel<float, TY, 0, VEC, true><<<blocks, 32 * TY, 0, st>>>(b);
}

cudaError_t launch_batch_mc(int pull, int ty, bool vec, int blocks, const BatchArgs& b, cudaStream_t st) {
    if (ty == 4) {
        if (vec) launch_batch_mc_ty<4, true>(pull, blocks, b, st);
        else launch_batch_mc_ty<4, false>(pull, blocks, b, st);
    } else if (ty == 8) {
        if (vec) launch_batch_mc_ty<8, true>(pull, blocks, b, st);
        else launch_batch_mc_ty<8, false>(pull, blocks, b, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int batch_mc_blocks_per_sm(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<float, 4, 1, true, true>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<float, 4, 1, false, true>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<float, 8, 1, true, true>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<float, 8, 1, false, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int fused_mc_blocks_per_sm(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<float, 4, MODE_STEP, 1, true, true>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<float, 4, MODE_STEP, 1, false, true>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<float, 8, MODE_STEP, 1, true, true>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<float, 8, MODE_STEP, 1, false, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace lbgb
