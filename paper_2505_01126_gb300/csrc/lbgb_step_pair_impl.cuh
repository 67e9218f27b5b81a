// lbgb_step_pair_impl.cuh -- host launcher of the paired step kernel (two
// x-adjacent sites per thread, packed two-lane FP32 arithmetic) for one 16-bit
// storage type.  Included by lbgb_step_pair_{f16,bf16}.cu and, with
// LBGB_PAIR_VD defined (the density-contrast instances), by
// lbgb_step_pair_vd_{f16,bf16}.cu, and with LBGB_PAIR_PF (the finite-difference
// phase field) by lbgb_step_pair_pf_{f16,bf16}.cu, which compile in parallel.
#pragma once
#include "lbgb_kernels.cuh"

namespace lbgb {

#if defined(LBGB_PAIR_PF)
// The paired step kernel with the finite-difference phase field (PF: phi read
// from its stored plane, u written for the stage kernels).
template <class FT, int TY>
static void launch_pair_pf_ty(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity == 0) fused_step_kernel<FT, TY, MODE_STEP, 0, true, false, false, true, true><<<grid, 32 * TY, 0, st>>>(a);
    else fused_step_kernel<FT, TY, MODE_STEP, 1, true, false, false, true, true><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_pair_pf<LBGB_FT>(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st) {
    switch (ty) {
        case 4: launch_pair_pf_ty<LBGB_FT, 4>(parity, grid, a, st); break;
        case 8: launch_pair_pf_ty<LBGB_FT, 8>(parity, grid, a, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
int fused_pair_pf_blocks_per_sm<LBGB_FT>(int ty) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, false, false, true, true>, 128, 0);
    else if (ty == 8)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, false, false, true, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
#elif defined(LBGB_PAIR_VD)
// The paired step kernel with density and viscosity contrasts (VD).
template <class FT, int TY>
static void launch_pair_vd_ty(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity == 0) fused_step_kernel<FT, TY, MODE_STEP, 0, true, false, true, false, true><<<grid, 32 * TY, 0, st>>>(a);
    else fused_step_kernel<FT, TY, MODE_STEP, 1, true, false, true, false, true><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_pair_vd<LBGB_FT>(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st) {
    switch (ty) {
        case 4: launch_pair_vd_ty<LBGB_FT, 4>(parity, grid, a, st); break;
        case 8: launch_pair_vd_ty<LBGB_FT, 8>(parity, grid, a, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
int fused_pair_vd_blocks_per_sm<LBGB_FT>(int ty) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, false, true, false, true>, 128, 0);
    else if (ty == 8)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, false, true, false, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
#else
template <class FT, int TY>
static void launch_pair_ty(int parity, dim3 grid, const StepArgs& a, cudaStream_t st) {
    if (parity == 0) fused_step_kernel<FT, TY, MODE_STEP, 0, true, false, false, false, true><<<grid, 32 * TY, 0, st>>>(a);
    else fused_step_kernel<FT, TY, MODE_STEP, 1, true, false, false, false, true><<<grid, 32 * TY, 0, st>>>(a);
}

template <>
cudaError_t launch_fused_pair<LBGB_FT>(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st) {
    switch (ty) {
        case 4: launch_pair_ty<LBGB_FT, 4>(parity, grid, a, st); break;
        case 8: launch_pair_ty<LBGB_FT, 8>(parity, grid, a, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
int fused_pair_blocks_per_sm<LBGB_FT>(int ty) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 4)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, fused_step_kernel<LBGB_FT, 4, MODE_STEP, 1, true, false, false, false, true>, 128, 0);
    else if (ty == 8)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, fused_step_kernel<LBGB_FT, 8, MODE_STEP, 1, true, false, false, false, true>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <class FT, int TY, int PW>
static void launch_batch_pair_ty(int parity, int blocks, const BatchArgs& b, cudaStream_t st) {
    constexpr int threads = PW / 2 * TY;
    if (parity == 0) batch_step_kernel<FT, TY, 0, true, false, false, true, PW><<<blocks, threads, 0, st>>>(b);
    else batch_step_kernel<FT, TY, 1, true, false, false, true, PW><<<blocks, threads, 0, st>>>(b);
}

template <>
cudaError_t launch_batch_pair<LBGB_FT>(int parity, int ty, int pw, int blocks, const BatchArgs& b, cudaStream_t st) {
    if (pw == 64 && ty == 4) launch_batch_pair_ty<LBGB_FT, 4, 64>(parity, blocks, b, st);
    else if (pw == 64 && ty == 8) launch_batch_pair_ty<LBGB_FT, 8, 64>(parity, blocks, b, st);
    else if (pw == 32 && ty == 4) launch_batch_pair_ty<LBGB_FT, 4, 32>(parity, blocks, b, st);
    else if (pw == 32 && ty == 8) launch_batch_pair_ty<LBGB_FT, 8, 32>(parity, blocks, b, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <class FT, int TY, int PW>
static int batch_pair_occupancy() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<FT, TY, 1, true, false, false, true, PW>,
                                                      PW / 2 * TY, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <>
int batch_pair_blocks_per_sm<LBGB_FT>(int ty, int pw) {
    if (pw == 64) return ty == 4 ? batch_pair_occupancy<LBGB_FT, 4, 64>() : ty == 8 ? batch_pair_occupancy<LBGB_FT, 8, 64>() : 0;
    if (pw == 32) return ty == 4 ? batch_pair_occupancy<LBGB_FT, 4, 32>() : ty == 8 ? batch_pair_occupancy<LBGB_FT, 8, 32>() : 0;
    return 0;
}

#endif

}  // namespace lbgb
