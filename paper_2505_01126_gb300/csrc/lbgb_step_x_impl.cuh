// lbgb_step_x_impl.cuh -- launchers of the fused kernel's optional variants
// for one storage: VD (density and viscosity contrasts) and PF (phase field as
// a stored field, advanced by the finite-difference step).  Included once per
// (storage, VD, PF) by lbgb_step_{vd,fd,fdvd}_*.cu, which compile in parallel:
// LBGB_FT the storage type, LBGB_MC the moment-only storage, LBGB_VD, LBGB_PF.
#pragma once
#include "lbgb_kernels.cuh"

namespace lbgb {

template <int TY, int MODE, bool VEC>
static void launch_x_kernel(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity) fused_step_kernel<LBGB_FT, TY, MODE, 1, VEC, LBGB_MC, LBGB_VD, LBGB_PF><<<grid, 32 * TY, 0, st>>>(a);
    else fused_step_kernel<LBGB_FT, TY, MODE, 0, VEC, LBGB_MC, LBGB_VD, LBGB_PF><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_x<LBGB_FT, LBGB_MC, LBGB_VD, LBGB_PF>(int mode, int parity, int ty, bool vec, dim3 grid,
                                                              const StepArgs& a, cudaStream_t st) {
    if (mode == MODE_INIT) {  // only the PF variant has its own INIT (it stores phi, not g)
        if (!LBGB_PF || LBGB_VD || ty != 8) return cudaErrorInvalidValue;
        launch_x_kernel<8, MODE_INIT, false>(0, grid, a, st);
        return cudaGetLastError();
    }
    if (mode == MODE_MOMENTS) {
        if (ty != 8) return cudaErrorInvalidValue;
        launch_x_kernel<8, MODE_MOMENTS, false>(parity, grid, a, st);
        return cudaGetLastError();
    }
    if (mode != MODE_STEP) return cudaErrorInvalidValue;
    if (ty == 4) {
        if (vec) launch_x_kernel<4, MODE_STEP, true>(parity, grid, a, st);
        else launch_x_kernel<4, MODE_STEP, false>(parity, grid, a, st);
    } else if (ty == 8) {
        if (vec) launch_x_kernel<8, MODE_STEP, true>(parity, grid, a, st);
        else launch_x_kernel<8, MODE_STEP, false>(parity, grid, a, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
int fused_x_blocks_per_sm<LBGB_FT, LBGB_MC, LBGB_VD, LBGB_PF>(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, LBGB_MC, LBGB_VD, LBGB_PF>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, false, LBGB_MC, LBGB_VD, LBGB_PF>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, LBGB_MC, LBGB_VD, LBGB_PF>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, false, LBGB_MC, LBGB_VD, LBGB_PF>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

#if LBGB_VD && !LBGB_PF
template <int TY, bool VEC>
static void launch_batch_vd_ty(int parity, int blocks, const BatchArgs& b, cudaStream_t st) {
    if (parity) batch_step_kernel<LBGB_FT, TY, 1, VEC, LBGB_MC, true><<<blocks, 32 * TY, 0, st>>>(b);
    else batch_step_kernel<LBGB_FT, TY, 0, VEC, LBGB_MC, true><<<blocks, 32 * TY, 0, st>>>(b);
}

template <>
cudaError_t launch_batch_vd<LBGB_FT, LBGB_MC>(int parity, int ty, bool vec, int blocks, const BatchArgs& b,
                                              cudaStream_t st) {
    if (ty == 4) vec ? launch_batch_vd_ty<4, true>(parity, blocks, b, st) : launch_batch_vd_ty<4, false>(parity, blocks, b, st);
    else if (ty == 8) vec ? launch_batch_vd_ty<8, true>(parity, blocks, b, st) : launch_batch_vd_ty<8, false>(parity, blocks, b, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <>
int batch_vd_blocks_per_sm<LBGB_FT, LBGB_MC>(int ty, bool vec) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 4, 1, true, LBGB_MC, true>, 128, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 4, 1, false, LBGB_MC, true>, 128, 0);
    else if (ty == 8)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 8, 1, true, LBGB_MC, true>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<LBGB_FT, 8, 1, false, LBGB_MC, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
#endif

}  // namespace lbgb
