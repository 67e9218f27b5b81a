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

}  // namespace lbgb
