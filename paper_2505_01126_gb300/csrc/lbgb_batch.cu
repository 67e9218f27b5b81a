// lbgb_batch.cu -- C ABI of the batched ensemble: many independent periodic
// boxes of uneven sizes, advanced together by one persistent kernel launch per
// step (plus one per-box FP64 reduction launch), replayed from a captured CUDA
// graph two steps at a time.  See include/lbgb.h for the contract of each call.
//
// Memory: one population array for all boxes (box b's 27 planes of N_b sites
// start at element f_off_b; with the moment-only storage two buffers of 10
// coefficient planes per box instead, from c_off_b), two D3Q7 arrays likewise,
// per-item FP64 partials, and one DevState per box.  The work list enumerates (box, 32 x ty tile,
// z-chunk) items; the persistent grid strides over it, so every box is
// computed by the same per-tile code as a single box.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lbgb.h"
#include "lbgb_kernels.cuh"

using namespace lbgb;

namespace lbgb {
// The batch kernel with the paired tile body and density contrasts (lbgb_batch_pair_vd_*.cu).
template <class FT>
cudaError_t launch_batch_pair_vd(int parity, int ty, int pw, int blocks, const BatchArgs& b, cudaStream_t st);
template <class FT>
int batch_pair_vd_blocks_per_sm(int ty, int pw);
}  // namespace lbgb

namespace {

int bfail(int code, const char* fmt, ...) {
    char msg[320];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return code;
}

#define BCUDA(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail(e_ == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "%s: %s", \
                         #call, cudaGetErrorString(e_));                                   \
    } while (0)

// Per-box FP64 reduction of a contiguous range of partial records: one block
// per box (the block index plus box_base), fixed summation order.  mode 0 =
// step (Phi, K, eps, max|u|), 1 = init (Phi, K, 0, max|u|).  epsw[box] turns
// the summed a2:a2 partials into eps: 2 nu (3/(2 tau))^2, or 1 with density
// contrasts (the partials then carry each site's own weight).
__global__ void __launch_bounds__(256) batch_reduce_kernel(const double* __restrict__ part,
                                                           const int* __restrict__ start,
                                                           const int* __restrict__ count, int box_base,
                                                           int fixed_count, const double* __restrict__ epsw,
                                                           DevState* st, int mode) {
    const int box = box_base + blockIdx.x;
    const int s0 = start ? start[box] : 0;
    const int n = count ? count[box] : fixed_count;
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0;
    for (int b = threadIdx.x; b < n; b += 256) {
        const double* p = part + (long long)(s0 + b) * NPART;
        v0 += p[0];
        v1 += p[1];
        v2 += p[2];
        v3 += p[3];
        v4 = fmax(v4, p[4]);
    }
    block_reduce5<256>(v0, v1, v2, v3, v4);
    if (threadIdx.x == 0) {
        DevState& S = st[box];
        const bool bad = !isfinite(v0 + v1 + v2 + v3);
        S.diag[0] = v0;
        S.diag[1] = v1;
        S.diag[2] = mode == 0 ? epsw[box] * v2 : 0.0;
        S.diag[3] = sqrt(v4);
        S.diag[4] = 0.0;
        S.mass = mode == 0 ? v3 : 0.0;
        S.A = 0.0;
        if (mode == 1) S.flags = bad ? 1 : 0;
        else if (bad) S.flags |= 1;
    }
}

bool dev_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct lb_batch {
    int count = 0;
    int storage = LB_F32;
    size_t fsize = 4;
    int device = 0;
    std::vector<BoxDesc> boxes;       // host copy (item fields follow the current tile)
    bool mc = false;                  // moment-only storage
    std::vector<double> tau, M, W, sigma;
    bool vd = false;                  // density and viscosity contrasts (lb_batch_set_density)
    int pair = 0;                     // paired tile body preferred, tiles this wide (64 or 32; 0: one
                                      // site per thread; 16-bit storages, see batch_use_pair)
    long long total_sites = 0, max_N = 0;
    bool vec = true;                  // every box has nx % 4 == 0

    void* f = nullptr;
    float* g[2] = {nullptr, nullptr};
    double* partials = nullptr;
    long long part_cap = 0;
    BoxDesc* d_boxes = nullptr;
    int* d_item_box = nullptr;
    int* d_item0 = nullptr;
    int* d_next = nullptr;            // the work queue's next item (zeroed before each step)
    int* d_nitem = nullptr;
    double* d_epsw = nullptr;         // eps per unit of the summed a2:a2 partials, per box
    DevState* d_st = nullptr;
    float* stage = nullptr;           // host I/O staging: 5 * max_N floats
    cudaStream_t stream = nullptr;

    int ty = 4, zc = 32;
    int nitems = 0;
    int grid_blocks = 0;
    long long t = 0;
    std::vector<char> initialized;
    int n_initialized = 0;
    long long launches = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_ty = 0, graph_zc = 0;
};

namespace {

// The paired tile body (two sites per thread, tiles 64 or 32 sites wide) runs
// the step when it is preferred and applies: FP16/BF16 storage, every box with
// nx % 4 == 0 (with or without density contrasts).
bool batch_pair_applies(const lb_batch* B) {
    return (B->storage == LB_F16_SHIFTED || B->storage == LB_BF16_SHIFTED) && B->vec;
}
bool batch_use_pair(const lb_batch* B) { return B->pair != 0 && batch_pair_applies(B); }

long long items_for(const lb_batch* B, int ty, int zc) {
    long long n = 0;
    for (const BoxDesc& d : B->boxes)
        n += (long long)((d.nx + 31) / 32) * ((d.ny + ty - 1) / ty) * ((d.nz + zc - 1) / zc);
    return n;
}

void drop_graph(lb_batch* B) {
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
}

// (Re)build the work list and the persistent grid size for the current tile.
int build_work(lb_batch* B) {
    std::vector<int> item_box, item0(B->count), nitem(B->count);
    int item = 0;
    const int tx = batch_use_pair(B) ? B->pair : 32;
    // Blocks take items from a queue in list order, so the list holds the
    // largest boxes first: their full-height chunks start early and the small
    // boxes' short items fill the end of the step.
    std::vector<int> order(B->count);
    for (int b = 0; b < B->count; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)B->boxes[a].N > (long long)B->boxes[c].N;
    });
    for (int b : order) {
        BoxDesc& d = B->boxes[b];
        d.tiles_x = (d.nx + tx - 1) / tx;
        d.tiles_y = (d.ny + B->ty - 1) / B->ty;
        d.tiles_z = (d.nz + B->zc - 1) / B->zc;
        d.item0 = item;
        const int n = d.tiles_x * d.tiles_y * d.tiles_z;
        item0[b] = item;
        nitem[b] = n;
        for (int k = 0; k < n; ++k) item_box.push_back(b);
        item += n;
    }
    if ((long long)item > B->part_cap) return bfail(LB_EINVAL, "work list of %d items exceeds %lld", item, B->part_cap);
    cudaFree(B->d_item_box);
    B->d_item_box = nullptr;
    BCUDA(cudaMalloc(&B->d_item_box, (size_t)item * sizeof(int)));
    BCUDA(cudaMemcpy(B->d_item_box, item_box.data(), (size_t)item * sizeof(int), cudaMemcpyHostToDevice));
    BCUDA(cudaMemcpy(B->d_boxes, B->boxes.data(), B->boxes.size() * sizeof(BoxDesc), cudaMemcpyHostToDevice));
    BCUDA(cudaMemcpy(B->d_item0, item0.data(), (size_t)B->count * sizeof(int), cudaMemcpyHostToDevice));
    BCUDA(cudaMemcpy(B->d_nitem, nitem.data(), (size_t)B->count * sizeof(int), cudaMemcpyHostToDevice));
    B->nitems = item;
    int per_sm = 0;
    if (batch_use_pair(B) && B->vd)
        per_sm = B->storage == LB_F16_SHIFTED ? batch_pair_vd_blocks_per_sm<__half>(B->ty, B->pair)
                                              : batch_pair_vd_blocks_per_sm<__nv_bfloat16>(B->ty, B->pair);
    else if (batch_use_pair(B)) per_sm = B->storage == LB_F16_SHIFTED ? batch_pair_blocks_per_sm<__half>(B->ty, B->pair)
                                                                  : batch_pair_blocks_per_sm<__nv_bfloat16>(B->ty, B->pair);
    else if (B->vd) switch (B->storage) {
        case LB_F32_MOMENTS: per_sm = batch_vd_blocks_per_sm<float, true>(B->ty, B->vec); break;
        case LB_F32: per_sm = batch_vd_blocks_per_sm<float, false>(B->ty, B->vec); break;
        case LB_F16_SHIFTED: per_sm = batch_vd_blocks_per_sm<__half, false>(B->ty, B->vec); break;
        default: per_sm = batch_vd_blocks_per_sm<__nv_bfloat16, false>(B->ty, B->vec); break;
    } else switch (B->storage) {
        case LB_F32_MOMENTS: per_sm = batch_mc_blocks_per_sm(B->ty, B->vec); break;
        case LB_F32: per_sm = batch_blocks_per_sm<float>(B->ty, B->vec); break;
        case LB_F16_SHIFTED: per_sm = batch_blocks_per_sm<__half>(B->ty, B->vec); break;
        default: per_sm = batch_blocks_per_sm<__nv_bfloat16>(B->ty, B->vec); break;
    }
    cudaDeviceProp prop;
    BCUDA(cudaGetDeviceProperties(&prop, B->device));
    long long blocks = (long long)(per_sm > 0 ? per_sm : 1) * prop.multiProcessorCount;
    B->grid_blocks = (int)(blocks < item ? blocks : item);
    drop_graph(B);
    return LB_OK;
}

StepArgs box_args(const lb_batch* B, int box, int par) {
    const BoxDesc& d = B->boxes[box];
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz;
    a.zc = d.nz < 32 ? d.nz : 32;
    a.N = d.N;
    if (B->mc) {
        float* C = static_cast<float*>(B->f);
        const size_t buf = 10 * (size_t)B->total_sites;
        for (int k = 0; k < 10; ++k) {
            a.cin[k] = C + buf * (size_t)par + (size_t)d.c_off + (size_t)k * d.N;
            a.cout[k] = C + buf * (size_t)(par ^ 1) + (size_t)d.c_off + (size_t)k * d.N;
        }
    } else {
        for (int i = 0; i < 27; ++i) a.fk[i] = (char*)B->f + ((size_t)d.f_off + (size_t)i * d.N) * B->fsize;
    }
    for (int q = 0; q < 7; ++q) {
        a.gin[q] = B->g[par] + d.g_off + (size_t)q * d.N;
        a.gout[q] = B->g[par ^ 1] + d.g_off + (size_t)q * d.N;
    }
    a.force_kind = FK_NONE;
    a.omega = d.omega; a.omega_phi = d.omega_phi; a.sharp = d.sharp; a.beta = d.beta;
    a.rho_g = d.rho_g; a.drho = d.drho; a.tau_g = d.tau_g; a.dtau = d.dtau;
    a.st = B->d_st + box;
    a.partials = B->partials;
    return a;
}

// par: AA parity; for the moment-only storage, 1 to pull (t > 0).
cudaError_t launch_box(const lb_batch* B, int mode, int par, dim3 grid, const StepArgs& a, bool vec) {
    if (B->vd && mode == MODE_MOMENTS) {  // the forced velocity includes the contrast forces
        switch (B->storage) {
            case LB_F32_MOMENTS: return launch_fused_x<float, true, true, false>(mode, par, 8, vec, grid, a, B->stream);
            case LB_F32: return launch_fused_x<float, false, true, false>(mode, par, 8, vec, grid, a, B->stream);
            case LB_F16_SHIFTED: return launch_fused_x<__half, false, true, false>(mode, par, 8, vec, grid, a, B->stream);
            default: return launch_fused_x<__nv_bfloat16, false, true, false>(mode, par, 8, vec, grid, a, B->stream);
        }
    }
    switch (B->storage) {
        case LB_F32_MOMENTS: return launch_fused_mc(mode, par, 8, vec, grid, a, B->stream);
        case LB_F32: return launch_fused<float>(mode, par, 8, vec, grid, a, B->stream);
        case LB_F16_SHIFTED: return launch_fused<__half>(mode, par, 8, vec, grid, a, B->stream);
        default: return launch_fused<__nv_bfloat16>(mode, par, 8, vec, grid, a, B->stream);
    }
}

// One step at parity par; `first` marks the moment-only step from t = 0.
int enqueue_batch_step(lb_batch* B, int par, cudaStream_t s, bool first = false) {
    BatchArgs b;
    b.nitems = B->nitems;
    b.zc = B->zc;
    b.boxes = B->d_boxes;
    b.item_box = B->d_item_box;
    b.f = B->f;
    b.g_in = B->g[par];
    b.g_out = B->g[par ^ 1];
    b.c_in = b.c_out = nullptr;
    if (B->mc) {
        float* C = static_cast<float*>(B->f);
        const size_t buf = 10 * (size_t)B->total_sites;
        b.c_in = C + buf * (size_t)par;
        b.c_out = C + buf * (size_t)(par ^ 1);
    }
    b.partials = B->partials;
    b.next = B->d_next;
    BCUDA(cudaMemsetAsync(B->d_next, 0, sizeof(int), s));
    cudaError_t e;
    if (batch_use_pair(B) && B->vd) {
        e = B->storage == LB_F16_SHIFTED ? launch_batch_pair_vd<__half>(par, B->ty, B->pair, B->grid_blocks, b, s)
                                         : launch_batch_pair_vd<__nv_bfloat16>(par, B->ty, B->pair, B->grid_blocks, b, s);
    } else if (batch_use_pair(B)) {
        e = B->storage == LB_F16_SHIFTED ? launch_batch_pair<__half>(par, B->ty, B->pair, B->grid_blocks, b, s)
                                         : launch_batch_pair<__nv_bfloat16>(par, B->ty, B->pair, B->grid_blocks, b, s);
    } else if (B->vd) {
        switch (B->storage) {
            case LB_F32_MOMENTS: e = launch_batch_vd<float, true>(first ? 0 : 1, B->ty, B->vec, B->grid_blocks, b, s); break;
            case LB_F32: e = launch_batch_vd<float, false>(par, B->ty, B->vec, B->grid_blocks, b, s); break;
            case LB_F16_SHIFTED: e = launch_batch_vd<__half, false>(par, B->ty, B->vec, B->grid_blocks, b, s); break;
            default: e = launch_batch_vd<__nv_bfloat16, false>(par, B->ty, B->vec, B->grid_blocks, b, s); break;
        }
    } else switch (B->storage) {
        case LB_F32_MOMENTS: e = launch_batch_mc(first ? 0 : 1, B->ty, B->vec, B->grid_blocks, b, s); break;
        case LB_F32: e = launch_batch<float>(par, B->ty, B->vec, B->grid_blocks, b, s); break;
        case LB_F16_SHIFTED: e = launch_batch<__half>(par, B->ty, B->vec, B->grid_blocks, b, s); break;
        default: e = launch_batch<__nv_bfloat16>(par, B->ty, B->vec, B->grid_blocks, b, s); break;
    }
    if (e != cudaSuccess) return bfail(LB_ECUDA, "batch step launch: %s", cudaGetErrorString(e));
    batch_reduce_kernel<<<B->count, 256, 0, s>>>(B->partials, B->d_item0, B->d_nitem, 0, 0, B->d_epsw, B->d_st, 0);
    BCUDA(cudaGetLastError());
    B->launches += 2;
    return LB_OK;
}

int capture_batch_graph(lb_batch* B) {
    drop_graph(B);
    cudaStream_t cs;
    BCUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return bfail(LB_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    const long long before = B->launches;
    int rc = enqueue_batch_step(B, 0, cs);
    if (rc == LB_OK) rc = enqueue_batch_step(B, 1, cs);
    B->launches = before;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != LB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bfail(LB_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        B->graph = nullptr;
        return bfail(LB_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    B->graph_ty = B->ty;
    B->graph_zc = B->zc;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_batch_destroy(lb_batch* B) {
    if (!B) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(B->device);
    drop_graph(B);
    cudaFree(B->f);
    cudaFree(B->g[0]);
    cudaFree(B->g[1]);
    cudaFree(B->partials);
    cudaFree(B->d_boxes);
    cudaFree(B->d_item_box);
    cudaFree(B->d_item0);
    cudaFree(B->d_nitem);
    cudaFree(B->d_next);
    cudaFree(B->d_epsw);
    cudaFree(B->d_st);
    cudaFree(B->stage);
    if (prev >= 0) cudaSetDevice(prev);
    delete B;
}

int lb_batch_create(int count, const int* dims, const double* tau, const double* M, const double* W,
                    const double* sigma, int storage, lb_batch** out) {
    if (!out) return bfail(LB_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !dims || !tau || !M || !W || !sigma) return bfail(LB_EINVAL, "lb_batch_create: bad arguments");
    if (storage == LB_F16_SHIFTED_G16 || storage == LB_BF16_SHIFTED_G16)
        return bfail(LB_EINVAL, "the 16-bit D3Q7 storage runs single boxes only (lb_create)");
    if (storage != LB_F32 && storage != LB_F16_SHIFTED && storage != LB_BF16_SHIFTED && storage != LB_F32_MOMENTS)
        return bfail(LB_EINVAL, "unknown storage %d", storage);
    lb_batch* B = new lb_batch();
    B->count = count;
    B->storage = storage;
    B->mc = storage == LB_F32_MOMENTS;
    B->fsize = (storage == LB_F32 || B->mc) ? 4 : 2;
    cudaGetDevice(&B->device);
    long long f_off = 0, g_off = 0, c_off = 0;
    for (int b = 0; b < count; ++b) {
        const int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
        const double t = tau[b], m = M[b], w = W[b], sg = sigma[b];
        if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31) - 1 || !(t > 0.5) || !(m > 0) ||
            !(w > 0) || !(sg >= 0) || (isinf(w) && sg > 0)) {
            delete B;
            return bfail(LB_EINVAL, "box %d: invalid size or parameters", b);
        }
        BoxDesc d;
        memset(&d, 0, sizeof(d));
        d.nx = nx; d.ny = ny; d.nz = nz;
        d.N = nx * ny * nz;
        d.f_off = f_off;
        d.g_off = g_off;
        d.c_off = c_off;
        d.omega = (float)(1.0 / t);
        d.omega_phi = (float)(1.0 / (m / 0.25 + 0.5));
        d.sharp = isinf(w) ? 0.f : (float)((m / 0.25) * (4.0 / w));
        d.beta = sg == 0 ? 0.f : (float)(1.5 * w * sg);
        B->boxes.push_back(d);
        B->tau.push_back(t);
        B->M.push_back(m);
        B->W.push_back(w);
        B->sigma.push_back(sg);
        f_off += 27LL * d.N;
        g_off += 7LL * d.N;
        c_off += 10LL * d.N;
        B->total_sites += d.N;
        if (d.N > B->max_N) B->max_N = d.N;
        if (nx % 4) B->vec = false;
    }
    B->initialized.assign(count, 0);
    B->pair = batch_pair_applies(B) ? 64 : 0;  // the paired body by default where it applies
    // partial records: the work list of the smallest tile, or one box's lb_init grid
    long long cap = items_for(B, 4, 1);
    for (const BoxDesc& d : B->boxes) {
        const long long init_blocks = (long long)((d.nx + 31) / 32) * ((d.ny + 7) / 8) * ((d.nz + 31) / 32);
        if (init_blocks > cap) cap = init_blocks;
    }
    B->part_cap = cap;
    int rc = LB_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc != LB_OK) return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = bfail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "cudaMalloc(%zu bytes): %s", bytes,
                       cudaGetErrorString(e));
        }
    };
    alloc(&B->f, B->mc ? (size_t)(2 * c_off) * sizeof(float) : (size_t)f_off * B->fsize);
    alloc((void**)&B->g[0], (size_t)g_off * sizeof(float));
    alloc((void**)&B->g[1], (size_t)g_off * sizeof(float));
    alloc((void**)&B->partials, (size_t)cap * NPART * sizeof(double));
    alloc((void**)&B->d_boxes, (size_t)count * sizeof(BoxDesc));
    alloc((void**)&B->d_item0, (size_t)count * sizeof(int));
    alloc((void**)&B->d_nitem, (size_t)count * sizeof(int));
    alloc((void**)&B->d_next, sizeof(int));
    alloc((void**)&B->d_epsw, (size_t)count * sizeof(double));
    alloc((void**)&B->d_st, (size_t)count * sizeof(DevState));
    if (rc == LB_OK) {
        std::vector<double> w(count);
        for (int b = 0; b < count; ++b) {
            const double s = 1.5 / B->tau[b];
            w[b] = 2.0 * ((B->tau[b] - 0.5) / 3.0) * s * s;
        }
        cudaError_t e = cudaMemcpy(B->d_epsw, w.data(), (size_t)count * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(B->d_st, 0, (size_t)count * sizeof(DevState));
        if (e != cudaSuccess) rc = bfail(LB_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
    }
    if (rc == LB_OK) rc = build_work(B);
    if (rc != LB_OK) {
        lb_batch_destroy(B);
        return rc;
    }
    *out = B;
    return LB_OK;
}

int lb_batch_set_stream(lb_batch* B, void* stream) {
    if (!B) return bfail(LB_EINVAL, "batch is NULL");
    B->stream = (cudaStream_t)stream;
    return LB_OK;
}

int lb_batch_init(lb_batch* B, int box, const float* phi, const float* u) {
    if (!B || !phi || !u) return bfail(LB_EINVAL, "lb_batch_init: NULL argument");
    if (box < 0 || box >= B->count) return bfail(LB_EINVAL, "box %d out of range", box);
    if (B->t != 0) return bfail(LB_ESTATE, "lb_batch_init after lb_batch_step (every box starts at t = 0)");
    const BoxDesc& d = B->boxes[box];
    const float* dphi = phi;
    const float* du = u;
    if (!dev_ptr(phi) || !dev_ptr(u)) {
        if (!B->stage) BCUDA(cudaMalloc(&B->stage, (size_t)B->max_N * 5 * sizeof(float)));
        if (!dev_ptr(phi)) {
            BCUDA(cudaMemcpyAsync(B->stage, phi, (size_t)d.N * sizeof(float), cudaMemcpyDefault, B->stream));
            dphi = B->stage;
        }
        if (!dev_ptr(u)) {
            BCUDA(cudaMemcpyAsync(B->stage + B->max_N, u, (size_t)d.N * 3 * sizeof(float), cudaMemcpyDefault,
                                  B->stream));
            du = B->stage + B->max_N;
        }
    }
    StepArgs a = box_args(B, box, 1);  // writes g buffer 0
    a.in_phi = dphi;
    a.in_u = du;
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + a.zc - 1) / a.zc);
    BCUDA(launch_box(B, MODE_INIT, 0, grid, a, false));
    batch_reduce_kernel<<<1, 256, 0, B->stream>>>(B->partials, nullptr, nullptr, box, (int)(grid.x * grid.y * grid.z),
                                                  B->d_epsw, B->d_st, 1);
    BCUDA(cudaGetLastError());
    B->launches += 2;
    if (!B->initialized[box]) {
        B->initialized[box] = 1;
        B->n_initialized += 1;
    }
    if (dphi != phi || du != u) BCUDA(cudaStreamSynchronize(B->stream));
    return LB_OK;
}

int lb_batch_step(lb_batch* B, int n) {
    if (!B) return bfail(LB_EINVAL, "batch is NULL");
    if (n < 0) return bfail(LB_EINVAL, "n = %d < 0", n);
    if (B->n_initialized != B->count)
        return bfail(LB_ESTATE, "%d of %d boxes initialised; call lb_batch_init for every box first",
                     B->n_initialized, B->count);
    while (n > 0) {
        const int par = (int)(B->t & 1);
        const bool first = B->mc && B->t == 0;
        if (par == 0 && n >= 2 && !first) {
            if (!B->graph || B->graph_ty != B->ty || B->graph_zc != B->zc) {
                int rc = capture_batch_graph(B);
                if (rc) return rc;
            }
            BCUDA(cudaGraphLaunch(B->graph, B->stream));
            B->launches += 4;
            B->t += 2;
            n -= 2;
        } else {
            int rc = enqueue_batch_step(B, par, B->stream, first);
            if (rc) return rc;
            B->t += 1;
            n -= 1;
        }
    }
    return LB_OK;
}

int lb_batch_moments(lb_batch* B, int box, float* rho, float* u, float* phi) {
    if (!B) return bfail(LB_EINVAL, "batch is NULL");
    if (box < 0 || box >= B->count) return bfail(LB_EINVAL, "box %d out of range", box);
    if (!B->initialized[box]) return bfail(LB_ESTATE, "box %d not initialised", box);
    const BoxDesc& d = B->boxes[box];
    const long long N = d.N;
    const bool hr = rho && !dev_ptr(rho), hu = u && !dev_ptr(u), hp = phi && !dev_ptr(phi);
    if ((hr || hu || hp) && !B->stage) BCUDA(cudaMalloc(&B->stage, (size_t)B->max_N * 5 * sizeof(float)));
    const int par = (int)(B->t & 1);
    StepArgs a = box_args(B, box, par);
    a.out_rho = hr ? B->stage : rho;
    a.out_u = hu ? B->stage + N : u;
    a.out_phi = hp ? B->stage + 4 * N : phi;
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + a.zc - 1) / a.zc);
    BCUDA(launch_box(B, MODE_MOMENTS, B->mc ? (B->t > 0 ? 1 : 0) : par, grid, a, false));
    B->launches += 1;
    if (hr) BCUDA(cudaMemcpyAsync(rho, B->stage, (size_t)N * sizeof(float), cudaMemcpyDefault, B->stream));
    if (hu) BCUDA(cudaMemcpyAsync(u, B->stage + N, (size_t)N * 3 * sizeof(float), cudaMemcpyDefault, B->stream));
    if (hp) BCUDA(cudaMemcpyAsync(phi, B->stage + 4 * N, (size_t)N * sizeof(float), cudaMemcpyDefault, B->stream));
    if (hr || hu || hp) BCUDA(cudaStreamSynchronize(B->stream));
    return LB_OK;
}

int lb_batch_diagnostics(lb_batch* B, int box, double out[5]) {
    if (!B || !out) return bfail(LB_EINVAL, "lb_batch_diagnostics: NULL argument");
    if (box < 0 || box >= B->count) return bfail(LB_EINVAL, "box %d out of range", box);
    DevState h;
    BCUDA(cudaMemcpyAsync(&h, B->d_st + box, sizeof(DevState), cudaMemcpyDeviceToHost, B->stream));
    BCUDA(cudaStreamSynchronize(B->stream));
    for (int k = 0; k < 5; ++k) out[k] = h.diag[k];
    if (h.flags & 1) return bfail(LB_ENONFINITE, "box %d met a NaN or Inf", box);
    return LB_OK;
}

int lb_batch_set_tile(lb_batch* B, int ty, int zc) {
    if (!B) return bfail(LB_EINVAL, "batch is NULL");
    if (ty != 4 && ty != 8) return bfail(LB_EINVAL, "tile height %d not in {4, 8}", ty);
    if (zc < 1) return bfail(LB_EINVAL, "z chunk %d < 1", zc);
    B->ty = ty;
    B->zc = zc;
    return build_work(B);
}

int lb_batch_get_tile(const lb_batch* B, int* ty, int* zc) {
    if (!B || !ty || !zc) return bfail(LB_EINVAL, "lb_batch_get_tile: NULL argument");
    *ty = B->ty;
    *zc = B->zc;
    return LB_OK;
}

int lb_batch_tune(lb_batch* B, int steps) {
    if (!B) return bfail(LB_EINVAL, "batch is NULL");
    if (steps < 1) return bfail(LB_EINVAL, "steps = %d < 1", steps);
    if (B->n_initialized != 0 || B->t != 0)
        return bfail(LB_ESTATE, "lb_batch_tune times steps on the batch's own arrays: call it before lb_batch_init");
    // zero state: the step's cost does not depend on the values
    BCUDA(cudaMemsetAsync(B->f, 0, B->mc ? (size_t)(B->total_sites * 20) * sizeof(float)
                                          : (size_t)(B->total_sites * 27) * B->fsize, B->stream));
    BCUDA(cudaMemsetAsync(B->g[0], 0, (size_t)(B->total_sites * 7) * sizeof(float), B->stream));
    BCUDA(cudaMemsetAsync(B->g[1], 0, (size_t)(B->total_sites * 7) * sizeof(float), B->stream));
    cudaEvent_t e0, e1;
    BCUDA(cudaEventCreate(&e0));
    BCUDA(cudaEventCreate(&e1));
    // As lb_tune: each shape the median of five windows (after one that warms
    // up), the first shape in this order within 1% of the fastest.
    constexpr int WINDOWS = 5;
    constexpr float TIE = 0.01f;
    // with a 16-bit storage the paired body's shapes come first (64 sites wide, then 32)
    const bool try_pair = batch_pair_applies(B);
    const int kinds[6][2] = {{64, 8}, {64, 4}, {32, 8}, {32, 4}, {0, 8}, {0, 4}};  // (paired width, tile height)
    const int zcs[4] = {16, 32, 64, 128};
    float med[24];
    int cty[24], czc[24], cpr[24], ncand = 0;
    int rc = LB_OK;
    for (int a = 0; a < 6 && rc == LB_OK; ++a)
        for (int b = 0; b < 4 && rc == LB_OK; ++b) {
            if (kinds[a][0] && !try_pair) continue;
            B->pair = kinds[a][0];
            if (lb_batch_set_tile(B, kinds[a][1], zcs[b]) != LB_OK) continue;
            float win[WINDOWS + 1];
            int nwin = 0;
            bool ok = true;
            for (int rep = 0; rep <= WINDOWS && ok; ++rep) {
                cudaEventRecord(e0, B->stream);
                int r2 = LB_OK;
                for (int k = 0; k < 2 * steps && r2 == LB_OK; ++k) r2 = enqueue_batch_step(B, k & 1, B->stream);
                cudaEventRecord(e1, B->stream);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r2 != LB_OK) {
                    cudaGetLastError();
                    ok = false;
                } else if (rep > 0) {
                    win[nwin++] = ms;
                }
            }
            if (!ok || nwin == 0) continue;
            for (int i = 1; i < nwin; ++i)
                for (int j = i; j > 0 && win[j] < win[j - 1]; --j) {
                    const float t = win[j];
                    win[j] = win[j - 1];
                    win[j - 1] = t;
                }
            med[ncand] = win[nwin / 2];
            cty[ncand] = kinds[a][1];
            czc[ncand] = zcs[b];
            cpr[ncand] = kinds[a][0];
            ++ncand;
        }
    int bty = B->ty, bzc = B->zc, bpr = B->pair;
    if (ncand > 0) {
        float best = med[0];
        for (int k = 1; k < ncand; ++k) best = med[k] < best ? med[k] : best;
        for (int k = 0; k < ncand; ++k)
            if (med[k] <= best * (1.f + TIE)) {
                bty = cty[k];
                bzc = czc[k];
                bpr = cpr[k];
                break;
            }
    }
    B->pair = bpr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->launches = 0;
    return lb_batch_set_tile(B, bty, bzc);
}

int lb_batch_set_pairing(lb_batch* B, int on) {
    if (!B) return bfail(LB_EINVAL, "batch is NULL");
    if (on != 0 && on != 1 && on != 32 && on != 64)
        return bfail(LB_EINVAL, "lb_batch_set_pairing: %d is none of 0, 1, 32, 64", on);
    if (on && !batch_pair_applies(B))
        return bfail(LB_EINVAL, "the paired tile body needs FP16 or BF16 storage and nx %% 4 == 0 in every box");
    B->pair = on == 1 ? 64 : on;
    return build_work(B);
}

int lb_batch_get_pairing(const lb_batch* B, int* on) {
    if (!B || !on) return bfail(LB_EINVAL, "NULL argument");
    *on = batch_use_pair(B) ? B->pair : 0;
    return LB_OK;
}

int lb_batch_set_density(lb_batch* B, const double* rho_l, const double* rho_g, const double* tau_l,
                         const double* tau_g) {
    if (!B || !rho_l || !rho_g || !tau_l || !tau_g) return bfail(LB_EINVAL, "lb_batch_set_density: NULL argument");
    std::vector<double> w(B->count);
    for (int b = 0; b < B->count; ++b) {
        const double rl = rho_l[b], rg = rho_g[b], tl = tau_l[b], tg = tau_g[b];
        if (!(rl > 0) || !(rg > 0) || !(tl > 0.5) || !(tg > 0.5) || !isfinite(rl) || !isfinite(rg) || !isfinite(tl) ||
            !isfinite(tg))
            return bfail(LB_EINVAL, "lb_batch_set_density: box %d needs rho > 0 and tau > 1/2", b);
    }
    for (int b = 0; b < B->count; ++b) {
        BoxDesc& d = B->boxes[b];
        d.rho_g = (float)rho_g[b];
        d.drho = (float)(rho_l[b] - rho_g[b]);
        d.tau_g = (float)tau_g[b];
        d.dtau = (float)(tau_l[b] - tau_g[b]);
        w[b] = 1.0;  // the contrast kernels weight each site's a2:a2 by its own 2 nu (3/(2 tau))^2
    }
    B->vd = true;
    BCUDA(cudaMemcpy(B->d_epsw, w.data(), (size_t)B->count * sizeof(double), cudaMemcpyHostToDevice));
    return build_work(B);  // uploads the descriptors, sizes the grid for the contrast kernel, drops the graph
}

long long lb_batch_sites(const lb_batch* B) { return B ? B->total_sites : -1; }

long long lb_batch_time(const lb_batch* B) { return B ? B->t : -1; }

}  // extern "C"
