// lbgb_kernels.cuh -- sm_103a kernels of the fused two-phase lattice Boltzmann step.
//
// One kernel template does the whole per-site time step of accLB (arXiv
// 2505.01126, Sec. 2); the numbered steps 1-13 are those listed in lbgb.h.
//
// Work decomposition.  A thread block owns a 32 x TY column of sites and
// marches it through a chunk of zc planes.  Per plane z it
//   A. computes phi = sum_q g_q (step 1) on the (32+4) x (TY+4) plane z+2 into
//      a 4-plane shared-memory ring (halo 2: kappa needs phi within radius 2),
//   B. computes grad phi and n (steps 2-3) on the (32+2) x (TY+2) plane z+1
//      into a 4-plane ring,
//   C. for the 32 x TY interior of plane z: kappa from the n ring (step 4),
//      the forces (5-6), the hydrodynamic moments of its own populations (7),
//      velocity, Hermite coefficient and regularized collision (8-10), the
//      D3Q7 BGK (11), streaming stores (12) and FP64 partial sums (13).
// The 27 f and 7 g loads of plane z are issued at the top of the iteration,
// before phase A, so their latency overlaps phases A and B.
//
// Layout in HBM (structure of arrays, site s = x + nx*(y + ny*z)):
//   f: 27 planes of N, in place with the AA access pattern.  Even parity
//      (t even) reads f_i(x) from slot (x, i) and writes f*_i to slot (x, -i);
//      odd parity reads f_i(x) from slot (x - c_i, -i) and writes f*_i to slot
//      (x + c_i, i).  Each slot is read and then written by the same site, so
//      the update is race-free in place.
//   g: two buffers of 7 planes (read g(t), push g(t+1)).  Phase A reads g at
//      sites owned by neighbouring blocks; with a second buffer those values
//      cannot have been overwritten yet.
// D3Q27 direction index i = (cx+1) + 3(cy+1) + 9(cz+1): rest 13, opposite 26-i;
// i = 14..26 are one member of each of the 13 opposite pairs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbgb {

__host__ __device__ constexpr int CX(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int CY(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int NNZ(int i) {
    return (CX(i) != 0) + (CY(i) != 0) + (CZ(i) != 0);
}
// D3Q27 weights by the number of non-zero components: 8/27, 2/27, 1/54, 1/216.
__host__ __device__ constexpr float W27(int i) {
    return NNZ(i) == 0 ? 8.f / 27.f : NNZ(i) == 1 ? 2.f / 27.f : NNZ(i) == 2 ? 1.f / 54.f : 1.f / 216.f;
}
__host__ __device__ constexpr float INVW27(int i) {
    return NNZ(i) == 0 ? 27.f / 8.f : NNZ(i) == 1 ? 13.5f : NNZ(i) == 2 ? 54.f : 216.f;
}

enum Mode { MODE_STEP = 0, MODE_MOMENTS = 1, MODE_INIT = 2 };
enum ForceKind { FK_NONE = 0, FK_CONST = 1, FK_ABC = 2, FK_LINEAR = 3 };

// Device-resident state shared by the step and the reduction kernels.
struct DevState {
    double A;        // linear-forcing amplitude used by the next step
    double K_target; // kinetic-energy target of the controller
    double diag[5];  // Phi, K, eps, max|u|, A_next of the last reduction
    int flags;       // bit 0: a non-finite value was seen
    int pad;
};

constexpr int NPART = 5;  // per-block partials: Phi, K, a2:a2, max|u|, non-finite

struct StepArgs {
    int nx, ny, nz, zc;
    long long N;
    void* f;             // 27 planes of the storage type
    const float* g_in;   // 7 planes, state at t
    float* g_out;        // 7 planes, state at t+1 (INIT: state at 0)
    int force_kind;
    float omega, omega_phi, sharp, beta;  // sharp = (M/cs7^2)(4/W), beta = 3W sigma/2
    float gc0, gc1, gc2; // constant force
    float A_abc;
    const float* abc;    // sin/cos tables: sin(kx) [nx], cos(kx) [nx], sin(ky), cos(ky), sin(kz), cos(kz)
    const DevState* st;
    double* partials;    // NPART per block
    float* out_rho;      // MOMENTS outputs (any may be null)
    float* out_u;
    float* out_phi;
    const float* in_phi; // INIT inputs
    const float* in_u;
};

// ---------------------------------------------------------- storage codecs
template <class T>
struct Codec;

template <>
struct Codec<float> {
    static __device__ __forceinline__ float dec(float v, int) { return v; }
    static __device__ __forceinline__ float enc(float f, int) { return f; }
};

// 16-bit storage holds the shifted, scaled deviation (f_i - w_i)/w_i, so the
// stored number is O(Ma) and never subnormal; arithmetic stays FP32.
template <>
struct Codec<__half> {
    static __device__ __forceinline__ float dec(__half v, int i) {
        return fmaf(W27(i), __half2float(v), W27(i));
    }
    static __device__ __forceinline__ __half enc(float f, int i) {
        return __float2half_rn((f - W27(i)) * INVW27(i));
    }
};

template <>
struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float dec(__nv_bfloat16 v, int i) {
        return fmaf(W27(i), __bfloat162float(v), W27(i));
    }
    static __device__ __forceinline__ __nv_bfloat16 enc(float f, int i) {
        return __float2bfloat16_rn((f - W27(i)) * INVW27(i));
    }
};

__device__ __forceinline__ int wrap_mod(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------- block reduction
// Sums v0..v2 and maxes v3, v4 over the block; thread 0 gets the result.
template <int NT>
__device__ __forceinline__ void block_reduce5(double& v0, double& v1, double& v2, double& v3,
                                              double& v4) {
    __shared__ double red[5][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, off);
        v1 += __shfl_down_sync(0xffffffffu, v1, off);
        v2 += __shfl_down_sync(0xffffffffu, v2, off);
        v3 = fmax(v3, __shfl_down_sync(0xffffffffu, v3, off));
        v4 = fmax(v4, __shfl_down_sync(0xffffffffu, v4, off));
    }
    if (lane == 0) {
        red[0][warp] = v0; red[1][warp] = v1; red[2][warp] = v2;
        red[3][warp] = v3; red[4][warp] = v4;
    }
    __syncthreads();
    if (warp == 0) {
        v0 = lane < NT / 32 ? red[0][lane] : 0.0;
        v1 = lane < NT / 32 ? red[1][lane] : 0.0;
        v2 = lane < NT / 32 ? red[2][lane] : 0.0;
        v3 = lane < NT / 32 ? red[3][lane] : 0.0;
        v4 = lane < NT / 32 ? red[4][lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v0 += __shfl_down_sync(0xffffffffu, v0, off);
            v1 += __shfl_down_sync(0xffffffffu, v1, off);
            v2 += __shfl_down_sync(0xffffffffu, v2, off);
            v3 = fmax(v3, __shfl_down_sync(0xffffffffu, v3, off));
            v4 = fmax(v4, __shfl_down_sync(0xffffffffu, v4, off));
        }
    }
}

// ------------------------------------------------------------ fused kernel
template <class FT, int TY, int MODE, int PAR>
__global__ void __launch_bounds__(32 * TY, (TY >= 16 ? 1 : 512 / (32 * TY)))
fused_step_kernel(const StepArgs a) {
    constexpr int TX = 32;
    constexpr int NT = TX * TY;
    constexpr int HX = TX + 4, HY = TY + 4, NHA = HX * HY;  // halo-2 plane (phi)
    constexpr int BX = TX + 2, BY = TY + 2, NHB = BX * BY;  // halo-1 plane (n)
    constexpr int NA = (NHA + NT - 1) / NT;
    constexpr int NB = (NHB + NT - 1) / NT;

    __shared__ float s_phi[4][HY][HX];
    __shared__ float s_n[4][3][BY][BX];
    __shared__ float s_g[2][4][TY][TX];  // grad phi and |grad phi| of the interior

    using C = Codec<FT>;
    FT* __restrict__ F = static_cast<FT*>(a.f);
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long N = a.N;
    const long long plane = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, nz);

    // phase-A sites (halo-2 plane), fixed for the whole march
    int a_row[NA], a_idx[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        const int idx = tid + k * NT;
        a_idx[k] = idx < NHA ? idx : -1;
        const int ly = idx / HX, lx = idx - (idx / HX) * HX;
        a_row[k] = wrap_mod(y0 + ly - 2, ny) * nx + wrap_mod(x0 + lx - 2, nx);
    }

    // phase-C site
    const int lx = tid % TX, ly = tid / TX;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool active = gx < nx && gy < ny;
    const int cxs = active ? gx : nx - 1, cys = active ? gy : ny - 1;
    const int Xo[3] = {cxs == 0 ? nx - 1 : cxs - 1, cxs, cxs == nx - 1 ? 0 : cxs + 1};
    const int Yo[3] = {(cys == 0 ? ny - 1 : cys - 1) * nx, cys * nx, (cys == ny - 1 ? 0 : cys + 1) * nx};

    float A_lin = 0.f;
    if (MODE != MODE_INIT && a.force_kind == FK_LINEAR) A_lin = (float)a.st->A;

    double d_phi = 0.0, d_K = 0.0, d_aa = 0.0, d_umax = 0.0, d_bad = 0.0;

    auto phaseA = [&](int zp) {
        const long long zb = (long long)wrap_mod(zp, nz) * plane;
        float* ring = &s_phi[zp & 3][0][0];
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            if (a_idx[k] >= 0) {
                const long long s = zb + a_row[k];
                float p;
                if (MODE == MODE_INIT) {
                    p = a.in_phi[s];
                } else {
                    p = 0.f;
#pragma unroll
                    for (int q = 0; q < 7; ++q) p += __ldg(a.g_in + q * N + s);
                }
                ring[a_idx[k]] = p;
            }
        }
    };

    auto phaseB = [&](int zp) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int idx = tid + k * NT;
            if (idx < NHB) {
                const int by = idx / BX, bx = idx - (idx / BX) * BX;
                float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
                for (int i = 14; i < 27; ++i) {
                    const int cx = CX(i), cy = CY(i), cz = CZ(i);
                    const float d = s_phi[(zp + cz) & 3][by + 1 + cy][bx + 1 + cx] -
                                    s_phi[(zp - cz) & 3][by + 1 - cy][bx + 1 - cx];
                    const float wd = W27(i) * d;
                    if (cx > 0) g0 += wd; else if (cx < 0) g0 -= wd;
                    if (cy > 0) g1 += wd; else if (cy < 0) g1 -= wd;
                    if (cz > 0) g2 += wd; else if (cz < 0) g2 -= wd;
                }
                g0 *= 3.f; g1 *= 3.f; g2 *= 3.f;
                const float m = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
                const float den = fmaxf(m, 1e-10f);
                s_n[zp & 3][0][by][bx] = g0 / den;
                s_n[zp & 3][1][by][bx] = g1 / den;
                s_n[zp & 3][2][by][bx] = g2 / den;
                if (bx >= 1 && bx <= TX && by >= 1 && by <= TY) {
                    s_g[zp & 1][0][by - 1][bx - 1] = g0;
                    s_g[zp & 1][1][by - 1][bx - 1] = g1;
                    s_g[zp & 1][2][by - 1][bx - 1] = g2;
                    s_g[zp & 1][3][by - 1][bx - 1] = m;
                }
            }
        }
    };

    // prologue: phi on planes z0-2 .. z0+1, n on z0-1 and z0
    for (int zp = z0 - 2; zp <= z0 + 1; ++zp) phaseA(zp);
    __syncthreads();
    phaseB(z0 - 1);
    phaseB(z0);
    __syncthreads();

    for (int z = z0; z < z1; ++z) {
        const long long Zo[3] = {(long long)(z == 0 ? nz - 1 : z - 1) * plane, (long long)z * plane,
                                 (long long)(z == nz - 1 ? 0 : z + 1) * plane};
        const long long s = Zo[1] + Yo[1] + Xo[1];

        // ---- issue this plane's population loads first
        float fl[27];
        float gl[7];
        float uin0 = 0.f, uin1 = 0.f, uin2 = 0.f;
        if (active) {
            if (MODE == MODE_INIT) {
                uin0 = a.in_u[s];
                uin1 = a.in_u[N + s];
                uin2 = a.in_u[2 * N + s];
            } else {
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    long long src;
                    if (PAR == 0) {
                        src = (long long)i * N + s;
                    } else {  // f_i(x) sits in slot (x - c_i, opposite of i)
                        src = (long long)(26 - i) * N + Zo[1 - CZ(i)] + Yo[1 - CY(i)] + Xo[1 - CX(i)];
                    }
                    fl[i] = C::dec(F[src], i);
                }
                if (MODE == MODE_STEP) {
#pragma unroll
                    for (int q = 0; q < 7; ++q) gl[q] = __ldg(a.g_in + q * N + s);
                }
            }
        }

        phaseA(z + 2);
        __syncthreads();
        phaseB(z + 1);
        __syncthreads();

        if (active) {
            const float phi = s_phi[z & 3][ly + 2][lx + 2];
            const float n0 = s_n[z & 3][0][ly + 1][lx + 1];
            const float n1 = s_n[z & 3][1][ly + 1][lx + 1];
            const float n2 = s_n[z & 3][2][ly + 1][lx + 1];

            if (MODE == MODE_INIT) {
                // f = f^eq(p* = 1, u) in the even-parity layout, g = g^eq(phi, u, n)
                const float u0 = uin0, u1 = uin1, u2 = uin2;
                const float uu = u0 * u0 + u1 * u1 + u2 * u2;
                const float E0 = 1.f - 1.5f * uu;
                F[13 * N + s] = C::enc(W27(13) * E0, 13);
#pragma unroll
                for (int i = 14; i < 27; ++i) {
                    const int cx = CX(i), cy = CY(i), cz = CZ(i);
                    const float cu = cx * u0 + cy * u1 + cz * u2;
                    const float E = E0 + 4.5f * cu * cu;
                    const float O = 3.f * cu;
                    F[(long long)i * N + s] = C::enc(W27(i) * (E + O), i);
                    F[(long long)(26 - i) * N + s] = C::enc(W27(26 - i) * (E - O), 26 - i);
                }
                const float phs = a.sharp * phi * (1.f - phi);
                float* G = a.g_out;
                G[s] = 0.25f * phi;
                G[N + s] = 0.125f * (phi + (4.f * phi * u0 + phs * n0));
                G[2 * N + s] = 0.125f * (phi - (4.f * phi * u0 + phs * n0));
                G[3 * N + s] = 0.125f * (phi + (4.f * phi * u1 + phs * n1));
                G[4 * N + s] = 0.125f * (phi - (4.f * phi * u1 + phs * n1));
                G[5 * N + s] = 0.125f * (phi + (4.f * phi * u2 + phs * n2));
                G[6 * N + s] = 0.125f * (phi - (4.f * phi * u2 + phs * n2));
                d_phi += (double)phi;
                d_K += 0.5 * (double)uu;
                d_umax = fmax(d_umax, (double)sqrtf(uu));
                if (!isfinite(phi + uu)) d_bad = 1.0;
            } else {
                // ---- step 4: kappa = div n (lattice stencil over the n ring)
                float kap = 0.f;
#pragma unroll
                for (int i = 14; i < 27; ++i) {
                    const int cx = CX(i), cy = CY(i), cz = CZ(i);
                    const int zpl = (z + cz) & 3, zmi = (z - cz) & 3;
                    float acc = 0.f;
                    if (cx != 0)
                        acc += cx * (s_n[zpl][0][ly + 1 + cy][lx + 1 + cx] - s_n[zmi][0][ly + 1 - cy][lx + 1 - cx]);
                    if (cy != 0)
                        acc += cy * (s_n[zpl][1][ly + 1 + cy][lx + 1 + cx] - s_n[zmi][1][ly + 1 - cy][lx + 1 - cx]);
                    if (cz != 0)
                        acc += cz * (s_n[zpl][2][ly + 1 + cy][lx + 1 + cx] - s_n[zmi][2][ly + 1 - cy][lx + 1 - cx]);
                    kap += W27(i) * acc;
                }
                kap *= 3.f;

                // ---- steps 5-6: surface tension and external force
                const float gr0 = s_g[z & 1][0][ly][lx], gr1 = s_g[z & 1][1][ly][lx];
                const float gr2 = s_g[z & 1][2][ly][lx], grm = s_g[z & 1][3][ly][lx];
                const float fsc = -a.beta * kap * grm;
                float Fe0 = fsc * gr0, Fe1 = fsc * gr1, Fe2 = fsc * gr2;
                if (a.force_kind == FK_CONST) {
                    Fe0 += a.gc0; Fe1 += a.gc1; Fe2 += a.gc2;
                } else if (a.force_kind == FK_ABC) {
                    const float* T = a.abc;
                    const float sx = T[gx], cxv = T[nx + gx];
                    const float sy = T[2 * nx + gy], cyv = T[2 * nx + ny + gy];
                    const float sz = T[2 * nx + 2 * ny + z], czv = T[2 * nx + 2 * ny + nz + z];
                    Fe0 += a.A_abc * (sz + cyv);
                    Fe1 += a.A_abc * (sx + czv);
                    Fe2 += a.A_abc * (sy + cxv);
                }

                // ---- step 7: moments of f
                float p = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
                float P00 = 0.f, P11 = 0.f, P22 = 0.f, P01 = 0.f, P02 = 0.f, P12 = 0.f;
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    const int cx = CX(i), cy = CY(i), cz = CZ(i);
                    const float v = fl[i];
                    p += v;
                    if (cx > 0) m0 += v; else if (cx < 0) m0 -= v;
                    if (cy > 0) m1 += v; else if (cy < 0) m1 -= v;
                    if (cz > 0) m2 += v; else if (cz < 0) m2 -= v;
                    if (cx != 0) P00 += v;
                    if (cy != 0) P11 += v;
                    if (cz != 0) P22 += v;
                    if (cx * cy > 0) P01 += v; else if (cx * cy < 0) P01 -= v;
                    if (cx * cz > 0) P02 += v; else if (cx * cz < 0) P02 -= v;
                    if (cy * cz > 0) P12 += v; else if (cy * cz < 0) P12 -= v;
                }

                // ---- step 8: forced velocity and total force
                const float inv = 1.f / (1.f - 0.5f * A_lin);
                const float u0 = (m0 + 0.5f * Fe0) * inv;
                const float u1 = (m1 + 0.5f * Fe1) * inv;
                const float u2 = (m2 + 0.5f * Fe2) * inv;

                if (MODE == MODE_MOMENTS) {
                    if (a.out_rho) a.out_rho[s] = p;
                    if (a.out_u) {
                        a.out_u[s] = u0;
                        a.out_u[N + s] = u1;
                        a.out_u[2 * N + s] = u2;
                    }
                    if (a.out_phi) a.out_phi[s] = phi;
                } else {
                    const float F0 = Fe0 + A_lin * u0, F1 = Fe1 + A_lin * u1, F2 = Fe2 + A_lin * u2;

                    // ---- step 9: a2 = Pi - p/3 I - u u + (u F + F u)/2
                    const float p3 = p * (1.f / 3.f);
                    const float a00 = P00 - p3 - u0 * u0 + u0 * F0;
                    const float a11 = P11 - p3 - u1 * u1 + u1 * F1;
                    const float a22 = P22 - p3 - u2 * u2 + u2 * F2;
                    const float a01 = P01 - u0 * u1 + 0.5f * (u0 * F1 + F0 * u1);
                    const float a02 = P02 - u0 * u2 + 0.5f * (u0 * F2 + F0 * u2);
                    const float a12 = P12 - u1 * u2 + 0.5f * (u1 * F2 + F1 * u2);

                    // ---- step 13 (per site): FP64 accumulation
                    const float uu = u0 * u0 + u1 * u1 + u2 * u2;
                    const float aa = a00 * a00 + a11 * a11 + a22 * a22 +
                                     2.f * (a01 * a01 + a02 * a02 + a12 * a12);
                    d_phi += (double)phi;
                    d_K += 0.5 * (double)uu;
                    d_aa += (double)aa;
                    d_umax = fmax(d_umax, (double)sqrtf(uu));
                    if (!isfinite(p + uu + phi + aa)) d_bad = 1.0;

                    // ---- step 10: regularized collision, written per opposite pair
                    const float om1 = 1.f - a.omega;
                    const float B00 = u0 * u0 + om1 * a00, B11 = u1 * u1 + om1 * a11;
                    const float B22 = u2 * u2 + om1 * a22, B01 = u0 * u1 + om1 * a01;
                    const float B02 = u0 * u2 + om1 * a02, B12 = u1 * u2 + om1 * a12;
                    const float trB = B00 + B11 + B22;
                    const float uF = u0 * F0 + u1 * F1 + u2 * F2;
                    const float E0 = p - 1.5f * trB - 1.5f * uF;
                    {
                        const float f13 = W27(13) * E0;
                        const long long dst = (long long)13 * N + s;
                        F[dst] = C::enc(f13, 13);
                    }
#pragma unroll
                    for (int i = 14; i < 27; ++i) {
                        const int cx = CX(i), cy = CY(i), cz = CZ(i);
                        const float cu = cx * u0 + cy * u1 + cz * u2;
                        const float cF = cx * F0 + cy * F1 + cz * F2;
                        const float cBc = cx * cx * B00 + cy * cy * B11 + cz * cz * B22 +
                                          2.f * (cx * cy * B01 + cx * cz * B02 + cy * cz * B12);
                        const float E = E0 + 4.5f * cBc + 4.5f * cu * cF;
                        const float O = 3.f * cu + 1.5f * cF;
                        const float fi = W27(i) * (E + O);        // direction  c
                        const float fj = W27(26 - i) * (E - O);   // direction -c
                        long long di, dj;
                        if (PAR == 0) {  // f*_i to slot (x, opposite of i)
                            di = (long long)(26 - i) * N + s;
                            dj = (long long)i * N + s;
                        } else {         // f*_i to slot (x + c_i, i)
                            di = (long long)i * N + Zo[1 + cz] + Yo[1 + cy] + Xo[1 + cx];
                            dj = (long long)(26 - i) * N + Zo[1 - cz] + Yo[1 - cy] + Xo[1 - cx];
                        }
                        F[di] = C::enc(fi, PAR == 0 ? 26 - i : i);
                        F[dj] = C::enc(fj, PAR == 0 ? i : 26 - i);
                    }

                    // ---- step 11: D3Q7 BGK with the sharpening equilibrium; step 12: push
                    const float om = a.omega_phi;
                    const float phs = a.sharp * phi * (1.f - phi);
                    const float ge0 = 0.25f * phi;
                    const float j0 = 4.f * phi * u0 + phs * n0;
                    const float j1 = 4.f * phi * u1 + phs * n1;
                    const float j2 = 4.f * phi * u2 + phs * n2;
                    float* G = a.g_out;
                    G[s] = gl[0] + om * (ge0 - gl[0]);
                    G[N + Zo[1] + Yo[1] + Xo[2]] = gl[1] + om * (0.125f * (phi + j0) - gl[1]);
                    G[2 * N + Zo[1] + Yo[1] + Xo[0]] = gl[2] + om * (0.125f * (phi - j0) - gl[2]);
                    G[3 * N + Zo[1] + Yo[2] + Xo[1]] = gl[3] + om * (0.125f * (phi + j1) - gl[3]);
                    G[4 * N + Zo[1] + Yo[0] + Xo[1]] = gl[4] + om * (0.125f * (phi - j1) - gl[4]);
                    G[5 * N + Zo[2] + Yo[1] + Xo[1]] = gl[5] + om * (0.125f * (phi + j2) - gl[5]);
                    G[6 * N + Zo[0] + Yo[1] + Xo[1]] = gl[6] + om * (0.125f * (phi - j2) - gl[6]);
                }
            }
        }
    }

    if (MODE != MODE_MOMENTS) {
        block_reduce5<NT>(d_phi, d_K, d_aa, d_umax, d_bad);
        if (tid == 0) {
            const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            double* out = a.partials + b * NPART;
            out[0] = d_phi; out[1] = d_K; out[2] = d_aa; out[3] = d_umax; out[4] = d_bad;
        }
    }
}

// Launch one fused kernel instance.  Defined per storage type in lbgb_step_*.cu.
template <class FT>
cudaError_t launch_fused(int mode, int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st);

}  // namespace lbgb
