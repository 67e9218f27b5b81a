// lbgb_batch_pair_vd_impl.cuh -- host launcher of the batch kernel with the
// paired tile body and density and viscosity contrasts (every box its own),
// for one 16-bit storage type LBGB_FT.  Included by lbgb_batch_pair_vd_{f16,bf16}.cu.
#pragma once
#include "lbgb_kernels.cuh"

namespace lbgb {

// declared beside the batch API (lbgb_batch.cu), which calls them
template <class FT>
cudaError_t launch_batch_pair_vd(int parity, int ty, int pw, int blocks, const BatchArgs& b, cudaStream_t st);
template <class FT>
int batch_pair_vd_blocks_per_sm(int ty, int pw);

template <class FT, int TY, int PW>
static void launch_batch_pair_vd_ty(int parity, int blocks, const BatchArgs& b, cudaStream_t st) {
    constexpr int threads = PW / 2 * TY;
    if (parity == 0) batch_step_kernel<FT, TY, 0, true, false, true, true, PW><<<blocks, threads, 0, st>>>(b);
    else batch_step_kernel<FT, TY, 1, true, false, true, true, PW><<<blocks, threads, 0, st>>>(b);
}

template <>
cudaError_t launch_batch_pair_vd<LBGB_FT>(int parity, int ty, int pw, int blocks, const BatchArgs& b,
                                          cudaStream_t st) {
    if (pw == 64 && ty == 4) launch_batch_pair_vd_ty<LBGB_FT, 4, 64>(parity, blocks, b, st);
    else if (pw == 64 && ty == 8) launch_batch_pair_vd_ty<LBGB_FT, 8, 64>(parity, blocks, b, st);
    else if (pw == 32 && ty == 4) launch_batch_pair_vd_ty<LBGB_FT, 4, 32>(parity, blocks, b, st);
    else if (pw == 32 && ty == 8) launch_batch_pair_vd_ty<LBGB_FT, 8, 32>(parity, blocks, b, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <class FT, int TY, int PW>
static int batch_pair_vd_occupancy() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<FT, TY, 1, true, false, true, true, PW>,
                                                      PW / 2 * TY, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <>
int batch_pair_vd_blocks_per_sm<LBGB_FT>(int ty, int pw) {
    if (pw == 64) return ty == 4 ? batch_pair_vd_occupancy<LBGB_FT, 4, 64>() : ty == 8 ? batch_pair_vd_occupancy<LBGB_FT, 8, 64>() : 0;
    if (pw == 32) return ty == 4 ? batch_pair_vd_occupancy<LBGB_FT, 4, 32>() : ty == 8 ? batch_pair_vd_occupancy<LBGB_FT, 8, 32>() : 0;
    return 0;
}

}  // namespace lbgb
