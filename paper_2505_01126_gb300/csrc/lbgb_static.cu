// lbgb_static.cu -- lb_field_stats_static: FP64 field statistics with no
// device allocation.
//
// Why: some callers cannot call cudaMalloc (or anything that allocates
// behind their back).  Examples:
//  - a framework whose caching allocator owns the device memory budget;
//  - code on a latency-critical path, where an allocation may synchronise the
//    device;
//  - a plugin that is handed pre-allocated buffers and must not create its
//    own.
// This entry point gives such callers the FP64 reductions that lb_init and
// lb_diagnostics report (Phi = sum phi, K = 1/2 sum |u|^2, max|u|) for fields
// they own.  It allocates nothing: the per-block partial sums live in a
// file-scope __device__ array of fixed size, which every device that loads
// this library holds until the process exits.
#include <cuda_runtime.h>

#include <math.h>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>

#include "lbgb.h"
#include "lbgb_kernels.cuh"

using namespace lbgb;

namespace {

// Tiles of 32 x 8 sites marching 32 planes, as lb_init's kernel, so a box
// needs ceil(nx/32) * ceil(ny/8) * ceil(nz/32) partial records.
constexpr int ST_TX = 32, ST_TY = 8, ST_ZC = 32, ST_NT = ST_TX * ST_TY;

// Shared by every call on a device; kernel 1 writes every record that kernel
// 2 reads in the same call, so nothing needs clearing between calls.  Calls
// that overlap on the GPU (for example on two streams) race on this array.
static __device__ __align__(256) double g_stat_partials[LB_STATIC_MAX_BLOCKS * NPART];
// Result of the last call, for callers that pass a host output pointer.
static __device__ __align__(256) double g_stat_result[8];

// Failures are reported through lb_last_error().
int fail(int code, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return code;
}

// Per-block FP32 partial sums over each thread's sites (at most ST_ZC), in FP64
// across threads; the same accumulation lb_init's kernel performs.
__global__ void __launch_bounds__(ST_NT) field_stats_kernel(const float* __restrict__ phi,
                                                            const float* __restrict__ u, int nx, int ny,
                                                            int nz, double* __restrict__ partials) {
    const int N = nx * ny * nz;
    const int lx = threadIdx.x % ST_TX, ly = threadIdx.x / ST_TX;
    const int gx = blockIdx.x * ST_TX + lx, gy = blockIdx.y * ST_TY + ly;
    const int z0 = blockIdx.z * ST_ZC, z1 = min(z0 + ST_ZC, nz);
    float s_phi = 0.f, s_K = 0.f, s_umax2 = 0.f;
    if (gx < nx && gy < ny) {
        for (int z = z0; z < z1; ++z) {
            const int s = (z * ny + gy) * nx + gx;
            const float u0 = u[s], u1 = (u + N)[s], u2 = (u + 2 * (long long)N)[s];
            const float uu = u0 * u0 + u1 * u1 + u2 * u2;
            s_phi += phi[s];
            s_K = fmaf(0.5f, uu, s_K);
            s_umax2 = fmaxf(s_umax2, uu);
        }
    }
    double v0 = s_phi, v1 = s_K, v2 = 0.0, v3 = 0.0, v4 = s_umax2;
    block_reduce5<ST_NT>(v0, v1, v2, v3, v4);
    if (threadIdx.x == 0) {
        const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double* out = partials + b * NPART;
        out[0] = v0; out[1] = v1; out[2] = v2; out[3] = v3; out[4] = v4;
    }
}

// One block: fixed-order FP64 sum of the partials into {Phi, K, 0, max|u|, 0}
// and a non-finite flag in out[5] (1.0 if any sum is NaN or Inf).
__global__ void __launch_bounds__(256) field_stats_finalize(const double* __restrict__ partials, int nblk,
                                                            double* __restrict__ out) {
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        const double* p = partials + (long long)b * NPART;
        v0 += p[0];
        v1 += p[1];
        v4 = fmax(v4, p[4]);
    }
    block_reduce5<256>(v0, v1, v2, v3, v4);
    if (threadIdx.x == 0) {
        out[0] = v0;
        out[1] = v1;
        out[2] = 0.0;
        out[3] = sqrt(v4);
        out[4] = 0.0;
        out[5] = isfinite(v0 + v1) ? 0.0 : 1.0;
    }
}

// Device addresses of the two arrays, looked up once per device with that
// device current.  In host code the array names only stand in for the device
// symbols; they are never dereferenced or passed to a kernel.
struct DeviceScratch {
    bool ready = false;
    double* partials = nullptr;
    double* result = nullptr;
};
constexpr int MAX_DEVICES = 64;
DeviceScratch g_scratch[MAX_DEVICES];
std::mutex g_scratch_lock;

int scratch_for_current_device(DeviceScratch** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LB_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(LB_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_lock);
    DeviceScratch& d = g_scratch[dev];
    if (!d.ready) {
        e = cudaGetSymbolAddress((void**)&d.partials, g_stat_partials);
        if (e != cudaSuccess) return fail(LB_ECUDA, "cudaGetSymbolAddress(partials): %s", cudaGetErrorString(e));
        e = cudaGetSymbolAddress((void**)&d.result, g_stat_result);
        if (e != cudaSuccess) return fail(LB_ECUDA, "cudaGetSymbolAddress(result): %s", cudaGetErrorString(e));
        d.ready = true;
    }
    *out = &d;
    return LB_OK;
}

// Device memory of the current device `dev`, or managed memory.  Device
// memory of another GPU is refused: the kernels run on the current device, and
// reading a peer's memory without peer access enabled faults.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

bool is_device_memory(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int lb_field_stats_static(const float* phi, const float* u, int nx, int ny, int nz, void* stream,
                                     double out[5]) {
    if (!phi || !u || !out) return fail(LB_EINVAL, "lb_field_stats_static: NULL argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(LB_EINVAL, "box %d x %d x %d: every edge must be >= 1", nx, ny, nz);
    if ((long long)nx * ny * nz >= (1LL << 31) - 1) return fail(LB_EINVAL, "nx*ny*nz must be < 2^31 - 1");
    const dim3 grid((nx + ST_TX - 1) / ST_TX, (ny + ST_TY - 1) / ST_TY, (nz + ST_ZC - 1) / ST_ZC);
    const long long nblk = (long long)grid.x * grid.y * grid.z;
    if (nblk > LB_STATIC_MAX_BLOCKS)
        return fail(LB_EINVAL,
                    "box %d x %d x %d needs %lld partial records, more than the %d this entry point holds "
                    "(cubic boxes up to 640^3)",
                    nx, ny, nz, nblk, LB_STATIC_MAX_BLOCKS);
    int dev = -1;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return fail(LB_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e0));
    if (!on_device(phi, dev) || !on_device(u, dev))
        return fail(LB_EINVAL, "phi and u must be device memory of the current device (%d)", dev);
    if (is_device_memory(out) && !on_device(out, dev))
        return fail(LB_EINVAL, "a device out must be memory of the current device (%d)", dev);
    DeviceScratch* d = nullptr;
    int rc = scratch_for_current_device(&d);
    if (rc != LB_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    field_stats_kernel<<<grid, ST_NT, 0, s>>>(phi, u, nx, ny, nz, d->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LB_ECUDA, "field_stats_kernel launch: %s", cudaGetErrorString(e));
    const bool dev_out = is_device_memory(out);
    field_stats_finalize<<<1, 256, 0, s>>>(d->partials, (int)nblk, d->result);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LB_ECUDA, "field_stats_finalize launch: %s", cudaGetErrorString(e));
    if (dev_out) {
        e = cudaMemcpyAsync(out, d->result, 5 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(LB_ECUDA, "result copy: %s", cudaGetErrorString(e));
        return LB_OK;
    }
    double h[6];
    e = cudaMemcpyAsync(h, d->result, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LB_ECUDA, "result copy: %s", cudaGetErrorString(e));
    for (int k = 0; k < 5; ++k) out[k] = h[k];
    if (h[5] != 0.0) return fail(LB_ENONFINITE, "a NaN or Inf was met in phi or u");
    return LB_OK;
}
