// lbgb_step_g16_impl.cuh -- host launchers of the kernels of the 16-bit D3Q7
// storage (G16) for one 16-bit storage type LBGB_FT.  Included by
// lbgb_step_g16_{f16,bf16}.cu (one-site kernels: INIT, MOMENTS, STEP) and,
// with LBGB_G16_PAIR defined, by lbgb_step_pair_g16_{f16,bf16}.cu (the paired
// step kernel), so that the four sets compile in parallel.
#pragma once
#include "lbgb_kernels.cuh"

namespace lbgb {

namespace {
int occupancy(const void* kernel, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
}  // namespace

#ifndef LBGB_G16_PAIR
template <class FT, int TY>
static void launch_g16_ty(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity == 0)
        fused_step_kernel<FT, TY, MODE_STEP, 0, true, false, false, false, false, true><<<grid, 32 * TY, 0, st>>>(a);
    else
        fused_step_kernel<FT, TY, MODE_STEP, 1, true, false, false, false, false, true><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_g16<LBGB_FT>(int mode, int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (mode == MODE_INIT) {
        if (ty != 8) return cudaErrorInvalidValue;
        fused_step_kernel<LBGB_FT, 8, MODE_INIT, 0, false, false, false, false, false, true><<<grid, 256, 0, st>>>(a);
    } else if (mode == MODE_MOMENTS) {
        if (ty != 8) return cudaErrorInvalidValue;
        if (parity == 0)
            fused_step_kernel<LBGB_FT, 8, MODE_MOMENTS, 0, true, false, false, false, false, true><<<grid, 256, 0, st>>>(a);
        else
            fused_step_kernel<LBGB_FT, 8, MODE_MOMENTS, 1, true, false, false, false, false, true><<<grid, 256, 0, st>>>(a);
    } else {
        switch (ty) {
            case 4: launch_g16_ty<LBGB_FT, 4>(parity, grid, a, st); break;
            case 8: launch_g16_ty<LBGB_FT, 8>(parity, grid, a, st); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <>
int fused_g16_blocks_per_sm<LBGB_FT>(int ty) {
    if (ty == 4)
        return occupancy((const void*)fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, false, false, false, false, true>,
                         128);
    if (ty == 8)
        return occupancy((const void*)fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, false, false, false, false, true>,
                         256);
    return 0;
}
#else
template <class FT, int TY>
static void launch_pair_g16_ty(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity == 0)
        fused_step_kernel<FT, TY, MODE_STEP, 0, true, false, false, false, true, true><<<grid, 32 * TY, 0, st>>>(a);
    else
        fused_step_kernel<FT, TY, MODE_STEP, 1, true, false, false, false, true, true><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_pair_g16<LBGB_FT>(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st) {
    switch (ty) {
        case 4: launch_pair_g16_ty<LBGB_FT, 4>(parity, grid, a, st); break;
        case 8: launch_pair_g16_ty<LBGB_FT, 8>(parity, grid, a, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
int fused_pair_g16_blocks_per_sm<LBGB_FT>(int ty) {
    if (ty == 4)
        return occupancy((const void*)fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, false, false, false, true, true>,
                         128);
    if (ty == 8)
        return occupancy((const void*)fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, false, false, false, true, true>,
                         256);
    return 0;
}
#endif

}  // namespace lbgb
