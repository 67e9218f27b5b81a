// lbgb_step_impl.cuh -- host launcher of the fused kernel for one storage type.
// Included once per storage type by lbgb_step_{f32,f16,bf16}.cu so the three
// sets of kernel instances compile in parallel.
#pragma once
#include "lbgb_kernels.cuh"

namespace lbgb {

template <class FT, int TY>
static cudaError_t launch_ty(int mode, int parity, bool vec, dim3 grid, const StepArgs& a, cudaStream_t st) {
    const dim3 block(32 * TY);
    if (mode != MODE_STEP) return cudaErrorInvalidValue;
    if (vec) {
        if (parity == 0) fused_step_kernel<FT, TY, MODE_STEP, 0, true><<<grid, block, 0, st>>>(a);
        else fused_step_kernel<FT, TY, MODE_STEP, 1, true><<<grid, block, 0, st>>>(a);
    } else {
        if (parity == 0) fused_step_kernel<FT, TY, MODE_STEP, 0, false><<<grid, block, 0, st>>>(a);
        else fused_step_kernel<FT, TY, MODE_STEP, 1, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <>
cudaError_t launch_fused<LBGB_FT>(int mode, int parity, int ty, bool vec, dim3 grid, const StepArgs& a,
                                  cudaStream_t st) {
    if (mode == MODE_MOMENTS) {
        if (ty != 8) return cudaErrorInvalidValue;
        if (parity == 0) fused_step_kernel<LBGB_FT, 8, MODE_MOMENTS, 0, false><<<grid, 256, 0, st>>>(a);
        else fused_step_kernel<LBGB_FT, 8, MODE_MOMENTS, 1, false><<<grid, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (mode == MODE_INIT) {
        if (ty != 8) return cudaErrorInvalidValue;
        fused_step_kernel<LBGB_FT, 8, MODE_INIT, 0, false><<<grid, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    switch (ty) {
        case 4: return launch_ty<LBGB_FT, 4>(mode, parity, vec, grid, a, st);
        case 8: return launch_ty<LBGB_FT, 8>(mode, parity, vec, grid, a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <>
int fused_blocks_per_sm<LBGB_FT>(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, false>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, false>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <class FT, int TY, bool VEC>
static cudaError_t launch_batch_ty(int parity, int blocks, const BatchArgs& b, cudaStream_t st) {
    if (parity == 0) batch_step_kernel<FT, TY, 0, VEC><<<blocks, 32 * TY, 0, st>>>(b);
    else batch_step_kernel<FT, TY, 1, VEC><<<blocks, 32 * TY, 0, st>>>(b);
    return cudaGetLastError();
}

template <>
cudaError_t launch_batch<LBGB_FT>(int parity, int ty, bool vec, int blocks, const BatchArgs& b, cudaStream_t st) {
    if (ty == 4) return vec ? launch_batch_ty<LBGB_FT, 4, true>(parity, blocks, b, st)
                            : launch_batch_ty<LBGB_FT, 4, false>(parity, blocks, b, st);
    if (ty == 8) return vec ? launch_batch_ty<LBGB_FT, 8, true>(parity, blocks, b, st)
                            : launch_batch_ty<LBGB_FT, 8, false>(parity, blocks, b, st);
    return cudaErrorInvalidValue;
}

template <>
int batch_blocks_per_sm<LBGB_FT>(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 4, 0, true>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 4, 0, false>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 8, 0, true>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 8, 0, false>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace lbgb
