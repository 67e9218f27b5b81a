// lbgb_stats.cu -- velocity statistics of homogeneous isotropic turbulence
// (Sec. 5.1): moments and histogram of the longitudinal velocity gradient
// (skewness, flatness, PDF), the longitudinal structure functions S_2(r),
// S_3(r), and shell spectra (energy, pressure) of periodic fields on the
// device.  See lb_velocity_statistics and lb_spectrum in include/lbgb.h for
// the definitions.
#include <cuda_runtime.h>
#include <cufft.h>

#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "lbgb.h"
#include "lbgb_kernels.cuh"

using namespace lbgb;

namespace {

constexpr int ST_NT = 256;  // threads per block of every kernel here

struct Field {
    const float* u[3];  // component planes
    int n[3];           // nx, ny, nz
};

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// d_a u_a at (x, y, z) by the lattice gradient in the factorised form
// (1/72) sum k(c1) k(c2) [u_a(+e_a) - u_a(-e_a)], with the additions in the
// fixed order (d(-1) + d(+1)) + 4 d(0) over the first transverse direction,
// then the same over the second, then / 72; every FP32 operation is rounded
// on its own (no contraction), so the value is that of any IEEE FP32
// evaluation in this order.
__device__ float long_grad(const Field& F, int a, const int (&p)[3]) {
    const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;  // transverse directions, in increasing order
    const float* ua = F.u[a];
    float e[3];
#pragma unroll
    for (int c2 = -1; c2 <= 1; ++c2) {
        float d[3];
#pragma unroll
        for (int c1 = -1; c1 <= 1; ++c1) {
            int q[3] = {p[0], p[1], p[2]};
            q[t1] = wrap1(q[t1] + c1, F.n[t1]);
            q[t2] = wrap1(q[t2] + c2, F.n[t2]);
            int qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
            qp[a] = wrap1(q[a] + 1, F.n[a]);
            qm[a] = wrap1(q[a] - 1, F.n[a]);
            const int sp = qp[0] + F.n[0] * (qp[1] + F.n[1] * qp[2]);  // < N < 2^31
            const int sm = qm[0] + F.n[0] * (qm[1] + F.n[1] * qm[2]);
            d[c1 + 1] = __fsub_rn(ua[sp], ua[sm]);
        }
        e[c2 + 1] = __fadd_rn(__fadd_rn(d[0], d[2]), __fmul_rn(4.f, d[1]));
    }
    return __fdiv_rn(__fadd_rn(__fadd_rn(e[0], e[2]), __fmul_rn(4.f, e[1])), 72.f);
}

__device__ __forceinline__ void site_coords(long long s, const Field& F, int (&p)[3]) {
    const int si = (int)s;  // s < N < 2^31
    p[0] = si % F.n[0];
    const int r = si / F.n[0];
    p[1] = r % F.n[1];
    p[2] = r / F.n[1];
}

// Pass 1: per-block sums of g^2, g^3, g^4 over the 3N gradient samples (FP32
// per thread, FP64 across threads).
__global__ void __launch_bounds__(ST_NT) grad_moments_kernel(Field F, long long N, double* partials) {
    float a2 = 0.f, a3 = 0.f, a4 = 0.f;
    for (long long s = blockIdx.x * (long long)ST_NT + threadIdx.x; s < N; s += (long long)gridDim.x * ST_NT) {
        int p[3];
        site_coords(s, F, p);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float g = long_grad(F, a, p);
            const float g2 = g * g;
            a2 += g2;
            a3 = fmaf(g2, g, a3);
            a4 = fmaf(g2, g2, a4);
        }
    }
    double m2 = a2, m3 = a3, m4 = a4, z0 = 0.0, z1 = 0.0;
    block_reduce5<ST_NT>(m2, m3, m4, z0, z1);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = m2;
        partials[3 * blockIdx.x + 1] = m3;
        partials[3 * blockIdx.x + 2] = m4;
    }
}

// Fixed-order sum of `cols` columns of per-block partials (rows = blocks);
// out[c] = sum / denom.  One block.
__global__ void __launch_bounds__(ST_NT) reduce_cols_kernel(const double* part, int rows, int cols, double denom,
                                                           double* out) {
    for (int c = 0; c < cols; ++c) {
        double v = 0.0, z = 0.0, w = 0.0, y = 0.0, x = 0.0;
        for (int r = threadIdx.x; r < rows; r += ST_NT) v += part[(long long)r * cols + c];
        block_reduce5<ST_NT>(v, z, w, y, x);
        if (threadIdx.x == 0) out[c] = v / denom;
        __syncthreads();
    }
}

// Skewness S = M3 / M2^(3/2) and flatness F = M4 / M2^2 from the moments
// mom[0..2], into mom[3], mom[4] (FP64; NaN for a field without gradients).
__global__ void skew_flat_kernel(double* mom) {
    const double m2 = mom[0];
    mom[3] = mom[1] / (m2 * sqrt(m2));
    mom[4] = mom[2] / (m2 * m2);
}

// Pass 2: histogram of g / scale (scale from the host if > 0, else sqrt(M2)
// from pass 1 on the device) in nbins bins on [-range, range), then the
// counts below and above.
__global__ void __launch_bounds__(ST_NT) grad_hist_kernel(Field F, long long N, int nbins, double range,
                                                         double factor, double scale, const double* moments,
                                                         unsigned long long* hist) {
    extern __shared__ unsigned int sh[];
    for (int b = threadIdx.x; b < nbins + 2; b += ST_NT) sh[b] = 0u;
    __syncthreads();
    const double inv = 1.0 / (scale > 0.0 ? scale : sqrt(moments[0]));
    for (long long s = blockIdx.x * (long long)ST_NT + threadIdx.x; s < N; s += (long long)gridDim.x * ST_NT) {
        int p[3];
        site_coords(s, F, p);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double g = (double)long_grad(F, a, p);
            const double b = floor(__dmul_rn(__dadd_rn(__dmul_rn(g, inv), range), factor));
            if (b != b) continue;  // NaN samples are not counted
            const int bin = b < 0.0 ? nbins : (b >= (double)nbins ? nbins + 1 : (int)b);
            // lanes of a warp sample neighbouring sites, mostly in the same bin:
            // one shared-memory atomic per distinct bin
            const unsigned same = __match_any_sync(__activemask(), bin);
            if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&sh[bin], (unsigned)__popc(same));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins + 2; b += ST_NT)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// Pass 3: per-block sums of (u_a(x + r e_a) - u_a(x))^n, n = 2, 3, over the
// sites and the three directions, for the SF_R separations
// r = blockIdx.y * SF_R + 1 .. (up to rmax): u_a(x) is loaded once for all of
// them.  FP32 per thread, FP64 across threads.
constexpr int SF_R = 8;

__global__ void __launch_bounds__(ST_NT) structure_kernel(Field F, long long N, int rmax, double* partials) {
    const int r0 = blockIdx.y * SF_R + 1;
    const int nr = min(SF_R, rmax - r0 + 1);
    float s2[SF_R], s3[SF_R];
#pragma unroll
    for (int j = 0; j < SF_R; ++j) s2[j] = s3[j] = 0.f;
    const int stride[3] = {1, F.n[0], F.n[0] * F.n[1]};
    for (long long s = blockIdx.x * (long long)ST_NT + threadIdx.x; s < N; s += (long long)gridDim.x * ST_NT) {
        int p[3];
        site_coords(s, F, p);
        const int si = (int)s;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float* ua = F.u[a];
            const float u0 = ua[si];
            const int base = si - p[a] * stride[a];
            int q = (int)(((long long)p[a] + r0) % F.n[a]);
#pragma unroll
            for (int j = 0; j < SF_R; ++j) {
                if (j < nr) {
                    const float d = ua[base + q * stride[a]] - u0;
                    const float d2 = d * d;
                    s2[j] += d2;
                    s3[j] = fmaf(d2, d, s3[j]);
                }
                if (++q == F.n[a]) q = 0;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < SF_R; j += 2) {
        double v0 = s2[j], v1 = s3[j], v2 = j + 1 < SF_R ? s2[j + 1] : 0.f, v3 = j + 1 < SF_R ? s3[j + 1] : 0.f;
        double z = 0.0;
        block_reduce5<ST_NT>(v0, v1, v2, v3, z);
        if (threadIdx.x == 0) {
            if (j < nr) {
                double* o = partials + 2 * ((long long)(r0 - 1 + j) * gridDim.x + blockIdx.x);
                o[0] = v0;
                o[1] = v1;
            }
            if (j + 1 < nr) {
                double* o = partials + 2 * ((long long)(r0 + j) * gridDim.x + blockIdx.x);
                o[0] = v2;
                o[1] = v3;
            }
        }
        __syncthreads();
    }
}

// Per-r fixed-order sums of the structure-function partials: out2[r-1], out3[r-1].
__global__ void __launch_bounds__(ST_NT) structure_reduce_kernel(const double* part, int blocks, double denom,
                                                                double* out2, double* out3) {
    const int r = blockIdx.x;
    double v2 = 0.0, v3 = 0.0, z0 = 0.0, z1 = 0.0, z2 = 0.0;
    for (int b = threadIdx.x; b < blocks; b += ST_NT) {
        const double* p = part + 2 * ((long long)r * blocks + b);
        v2 += p[0];
        v3 += p[1];
    }
    block_reduce5<ST_NT>(v2, v3, z0, z1, z2);
    if (threadIdx.x == 0) {
        out2[r] = v2 / denom;
        out3[r] = v3 / denom;
    }
}

// Shell sums of 1/2 |c / N|^2 over one R2C half-spectrum (n x n x (n/2+1)
// complex values), each entry weighted by the number of full-spectrum
// wavevectors it stands for (1 on the planes mx = 0 and mx = n/2, else 2).
// Per-block FP64 shell sums in shared memory, then per-block rows.
__global__ void __launch_bounds__(ST_NT) shell_kernel(const cufftComplex* c, int n, int kmax, double invN,
                                                     double* rows) {
    extern __shared__ double sh_shell[];
    for (int k = threadIdx.x; k <= kmax; k += ST_NT) sh_shell[k] = 0.0;
    __syncthreads();
    const int nh = n / 2 + 1;
    const long long total = (long long)n * n * nh;
    for (long long e = blockIdx.x * (long long)ST_NT + threadIdx.x; e < total; e += (long long)gridDim.x * ST_NT) {
        const int mx = (int)(e % nh);
        const long long r = e / nh;
        const int my0 = (int)(r % n), mz0 = (int)(r / n);
        const int my = my0 <= n / 2 ? my0 : my0 - n, mz = mz0 <= n / 2 ? mz0 : mz0 - n;
        const long long m2 = (long long)mx * mx + (long long)my * my + (long long)mz * mz;
        const int k = (int)floor(sqrt((double)m2) + 0.5);
        if (k > kmax) continue;
        const double re = (double)c[e].x * invN, im = (double)c[e].y * invN;
        const double w = (mx == 0 || (n % 2 == 0 && mx == n / 2)) ? 0.5 : 1.0;  // 1/2 x multiplicity
        atomicAdd(&sh_shell[k], w * (re * re + im * im));
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= kmax; k += ST_NT) rows[(long long)blockIdx.x * (kmax + 1) + k] = sh_shell[k];
}

// out[k] = sum over blocks of rows[b][k] (fixed order), accumulated onto out.
__global__ void __launch_bounds__(ST_NT) shell_reduce_kernel(const double* rows, int blocks, int kmax, double* out) {
    for (int k = blockIdx.x * ST_NT + threadIdx.x; k <= kmax; k += gridDim.x * ST_NT) {
        double v = 0.0;
        for (int b = 0; b < blocks; ++b) v += rows[(long long)b * (kmax + 1) + k];
        out[k] += v;
    }
}

thread_local char s_err[256] = "";

int sfail(int code, const char* msg, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess) cudaGetLastError();
    snprintf(s_err, sizeof(s_err), "lb_velocity_statistics: %s%s%s", msg, e != cudaSuccess ? ": " : "",
             e != cudaSuccess ? cudaGetErrorString(e) : "");
    lbgb::set_last_error(s_err);
    return code;
}

}  // namespace

extern "C" int lb_velocity_statistics(const float* u, int nx, int ny, int nz, int rmax, int nbins, double range,
                                      double scale, void* stream, double* out, unsigned long long* hist) {
    if (!u || !out || (nbins > 0 && !hist)) return sfail(LB_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31) - 1) return sfail(LB_EINVAL, "bad size");
    if (rmax < 0 || rmax > 65535) return sfail(LB_EINVAL, "rmax out of [0, 65535]");
    if (nbins < 0 || nbins > 8192 || (nbins > 0 && !(range > 0.0))) return sfail(LB_EINVAL, "bad histogram arguments");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long N = (long long)nx * ny * nz;
    Field F;
    for (int a = 0; a < 3; ++a) F.u[a] = u + (long long)a * N;
    F.n[0] = nx; F.n[1] = ny; F.n[2] = nz;

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return sfail(LB_ECUDA, "device query", e);
    long long want = (N + ST_NT - 1) / ST_NT;
    const int blocks = (int)(want < 4LL * sms ? want : 4LL * sms);

    // device scratch: moment partials, moments (3), structure partials and results, histogram
    const size_t n_mp = 3 * (size_t)blocks, n_sp = 2 * (size_t)blocks * (size_t)(rmax > 0 ? rmax : 1);
    const size_t n_dbl = n_mp + 5 + n_sp + 2 * (size_t)rmax;
    double* scratch = nullptr;
    unsigned long long* dhist = nullptr;
    e = cudaMalloc(&scratch, n_dbl * sizeof(double));
    if (e != cudaSuccess) return sfail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "cudaMalloc", e);
    if (nbins > 0) {
        e = cudaMalloc(&dhist, (size_t)(nbins + 2) * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(scratch);
            return sfail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "cudaMalloc", e);
        }
    }
    double* mp = scratch;
    double* mom = mp + n_mp;
    double* sp = mom + 5;
    double* sres = sp + n_sp;
    int rc = LB_OK;
    do {
        grad_moments_kernel<<<blocks, ST_NT, 0, st>>>(F, N, mp);
        reduce_cols_kernel<<<1, ST_NT, 0, st>>>(mp, blocks, 3, 3.0 * (double)N, mom);
        skew_flat_kernel<<<1, 1, 0, st>>>(mom);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (nbins > 0) {
            if ((e = cudaMemsetAsync(dhist, 0, (size_t)(nbins + 2) * sizeof(unsigned long long), st)) != cudaSuccess)
                break;
            const double factor = (double)nbins / (2.0 * range);
            grad_hist_kernel<<<blocks, ST_NT, (size_t)(nbins + 2) * sizeof(unsigned int), st>>>(F, N, nbins, range,
                                                                                                  factor, scale, mom,
                                                                                                  dhist);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
        }
        if (rmax > 0) {
            structure_kernel<<<dim3(blocks, (rmax + SF_R - 1) / SF_R), ST_NT, 0, st>>>(F, N, rmax, sp);
            structure_reduce_kernel<<<rmax, ST_NT, 0, st>>>(sp, blocks, 3.0 * (double)N, sres, sres + rmax);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
        }
        if ((e = cudaMemcpyAsync(out, mom, 5 * sizeof(double), cudaMemcpyDefault, st)) != cudaSuccess) break;
        if (rmax > 0 &&
            (e = cudaMemcpyAsync(out + 5, sres, 2 * (size_t)rmax * sizeof(double), cudaMemcpyDefault, st)) !=
                cudaSuccess)
            break;
        if (nbins > 0 && (e = cudaMemcpyAsync(hist, dhist, (size_t)(nbins + 2) * sizeof(unsigned long long),
                                              cudaMemcpyDefault, st)) != cudaSuccess)
            break;
        e = cudaStreamSynchronize(st);
    } while (0);
    if (e != cudaSuccess) rc = sfail(LB_ECUDA, "CUDA error", e);
    cudaFree(scratch);
    if (dhist) cudaFree(dhist);
    return rc;
}

extern "C" int lb_spectrum(const float* f, int ncomp, int n, int kmax, void* stream, double* out) {
    const char* who = "lb_spectrum";
    auto err = [&](int code, const char* msg, cudaError_t e = cudaSuccess) {
        if (e != cudaSuccess) cudaGetLastError();
        snprintf(s_err, sizeof(s_err), "%s: %s%s%s", who, msg, e != cudaSuccess ? ": " : "",
                 e != cudaSuccess ? cudaGetErrorString(e) : "");
        lbgb::set_last_error(s_err);
        return code;
    };
    if (!f || !out) return err(LB_EINVAL, "NULL argument");
    if (ncomp < 1 || ncomp > 3 || n < 2 || (long long)n * n * n >= (1LL << 31) - 1 || kmax < 0 || kmax > 8192)
        return err(LB_EINVAL, "bad size");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long N = (long long)n * n * n;
    const long long nc = (long long)n * n * (n / 2 + 1);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return err(LB_ECUDA, "device query", e);
    const long long want = (nc + ST_NT - 1) / ST_NT;
    const int blocks = (int)(want < 2LL * sms ? want : 2LL * sms);
    if ((size_t)(kmax + 1) * sizeof(double) > 48 * 1024) return err(LB_EINVAL, "kmax too large");

    cufftComplex* c = nullptr;
    double* rows = nullptr;
    double* dout = nullptr;
    float* aligned = nullptr;  // a component plane off an 8-byte boundary is copied here first
    bool need_copy = false;
    for (int q = 0; q < ncomp; ++q)
        if (reinterpret_cast<uintptr_t>(f + (long long)q * N) % sizeof(cufftComplex)) need_copy = true;
    e = cudaMalloc(&c, (size_t)nc * sizeof(cufftComplex));
    if (e == cudaSuccess && need_copy) e = cudaMalloc(&aligned, (size_t)N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&rows, (size_t)blocks * (kmax + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)(kmax + 1) * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(c); cudaFree(rows); cudaFree(dout); cudaFree(aligned);
        return err(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "cudaMalloc", e);
    }
    cufftHandle plan;
    if (cufftPlan3d(&plan, n, n, n, CUFFT_R2C) != CUFFT_SUCCESS) {
        cudaFree(c); cudaFree(rows); cudaFree(dout); cudaFree(aligned);
        return err(LB_ECUDA, "cufftPlan3d failed");
    }
    int rc = LB_OK;
    do {
        if (cufftSetStream(plan, st) != CUFFT_SUCCESS) { rc = err(LB_ECUDA, "cufftSetStream failed"); break; }
        if ((e = cudaMemsetAsync(dout, 0, (size_t)(kmax + 1) * sizeof(double), st)) != cudaSuccess) {
            rc = err(LB_ECUDA, "memset", e);
            break;
        }
        for (int q = 0; q < ncomp && rc == LB_OK; ++q) {
            const float* src = f + (long long)q * N;
            if (reinterpret_cast<uintptr_t>(src) % sizeof(cufftComplex)) {
                if ((e = cudaMemcpyAsync(aligned, src, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, st)) !=
                    cudaSuccess) {
                    rc = err(LB_ECUDA, "copy", e);
                    break;
                }
                src = aligned;
            }
            // out-of-place R2C leaves its input unchanged
            if (cufftExecR2C(plan, const_cast<cufftReal*>(src), c) != CUFFT_SUCCESS) {
                rc = err(LB_ECUDA, "cufftExecR2C failed");
                break;
            }
            shell_kernel<<<blocks, ST_NT, (size_t)(kmax + 1) * sizeof(double), st>>>(c, n, kmax, 1.0 / (double)N, rows);
            shell_reduce_kernel<<<(kmax + ST_NT) / ST_NT, ST_NT, 0, st>>>(rows, blocks, kmax, dout);
            if ((e = cudaGetLastError()) != cudaSuccess) rc = err(LB_ECUDA, "launch", e);
        }
        if (rc != LB_OK) break;
        if ((e = cudaMemcpyAsync(out, dout, (size_t)(kmax + 1) * sizeof(double), cudaMemcpyDefault, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            rc = err(LB_ECUDA, "copy", e);
    } while (0);
    cufftDestroy(plan);
    cudaFree(c);
    cudaFree(rows);
    cudaFree(dout);
    cudaFree(aligned);
    return rc;
}
