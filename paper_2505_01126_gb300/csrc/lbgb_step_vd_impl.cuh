// lbgb_step_vd_impl.cuh -- launchers of the fused kernel with the density and
// viscosity contrasts (VD = true) for one storage: LBGB_FT with LBGB_MC = false
// (AA populations) or float with LBGB_MC = true (moment-only storage).
// Included once per storage by lbgb_step_vd_*.cu so they compile in parallel.
#pragma once
#include "lbgb_kernels.cuh"

namespace lbgb {

template <int TY, int MODE, bool VEC>
static void launch_vd_kernel(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity) fused_step_kernel<LBGB_FT, TY, MODE, 1, VEC, LBGB_MC, true><<<grid, 32 * TY, 0, st>>>(a);
    else fused_step_kernel<LBGB_FT, TY, MODE, 0, VEC, LBGB_MC, true><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_vd<LBGB_FT, LBGB_MC>(int mode, int parity, int ty, bool vec, dim3 grid, const StepArgs& a,
                                              cudaStream_t st) {
    if (mode == MODE_MOMENTS) {
        if (ty != 8) return cudaErrorInvalidValue;
        launch_vd_kernel<8, MODE_MOMENTS, false>(parity, grid, a, st);
        return cudaGetLastError();
    }
    if (mode != MODE_STEP) return cudaErrorInvalidValue;
    if (ty == 4) {
        if (vec) launch_vd_kernel<4, MODE_STEP, true>(parity, grid, a, st);
        else launch_vd_kernel<4, MODE_STEP, false>(parity, grid, a, st);
    } else if (ty == 8) {
        if (vec) launch_vd_kernel<8, MODE_STEP, true>(parity, grid, a, st);
        else launch_vd_kernel<8, MODE_STEP, false>(parity, grid, a, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
int fused_vd_blocks_per_sm<LBGB_FT, LBGB_MC>(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, LBGB_MC, true>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, false, LBGB_MC, true>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, LBGB_MC, true>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, false, LBGB_MC, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace lbgb
