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
// Layout in HBM (structure of arrays, site s = x + nx*(y + ny*z), 32-bit):
//   f: 27 planes of N holding delta_i = f_i/w_i - 1, in place with the AA
//      access pattern; each plane has its own base pointer in the kernel
//      arguments, so an access is one 32-bit index add and one wide multiply-add.  Even parity
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
#include <limits.h>
#include <stdint.h>

namespace lbgb {

__host__ __device__ constexpr int CX(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int CY(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int i) { return i / 9 - 1; }
enum Mode { MODE_STEP = 0, MODE_MOMENTS = 1, MODE_INIT = 2 };
enum ForceKind { FK_NONE = 0, FK_CONST = 1, FK_ABC = 2, FK_LINEAR = 3 };

// Device-resident state shared by the step and the reduction kernels.
struct DevState {
    double A;        // linear-forcing amplitude used by the next step
    double K_target; // kinetic-energy target of the controller
    double diag[5];  // Phi, K, eps, max|u|, A_next of the last reduction
    double mass;     // sum of p* - 1 of the last reduction
    int flags;       // bit 0: a non-finite value was seen
    int pad;
};

// per-block partials: Phi, K, a2:a2, sum(p* - 1), max|u|^2
constexpr int NPART = 5;

struct StepArgs {
    int nx, ny, nz, zc;
    int N;                  // sites, < 2^31 (32-bit site indices)
    void* fk[27];           // population plane i (storage type), holding delta_i = f_i/w_i - 1
    const float* gin[7];    // D3Q7 planes at t
    float* gout[7];         // D3Q7 planes at t+1 (INIT: at 0)
    int force_kind;
    float omega, omega_phi, sharp, beta;  // sharp = (M/cs7^2)(4/W), beta = 3W sigma/2
    float gc0, gc1, gc2;    // constant force
    float A_abc;
    const float* abc;       // sin(kx)[nx], cos(kx)[nx], sin(ky)[ny], cos(ky)[ny], sin(kz)[nz], cos(kz)[nz]
    const DevState* st;
    double* partials;       // NPART per block
    float* out_rho;         // MOMENTS outputs (any may be null)
    float* out_u;
    float* out_phi;
    const float* in_phi;    // INIT inputs
    const float* in_u;
};

// ---------------------------------------------------------- storage codecs
// Every storage type holds the shifted, scaled population delta_i = f_i/w_i - 1
// (zero at rest, O(Ma) in a flow, never subnormal in 16 bits); all arithmetic
// is FP32.  The moments and the collision below work on delta directly, so no
// codec multiplies by w_i.
template <class T>
struct Codec;

template <>
struct Codec<float> {
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};

template <>
struct Codec<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};

template <>
struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

__device__ __forceinline__ int wrap_mod(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// 16-byte asynchronous global -> shared copy (L2 only), its group commit and wait.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ constexpr int IDX(int cx, int cy, int cz) { return (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1); }

// ------------------------------------------------------- block reduction
// Sums v0..v3 and maxes v4 over the block; thread 0 gets the result.
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
        v3 += __shfl_down_sync(0xffffffffu, v3, off);
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
            v3 += __shfl_down_sync(0xffffffffu, v3, off);
            v4 = fmax(v4, __shfl_down_sync(0xffffffffu, v4, off));
        }
    }
}

// --------------------------------------------------- per-site arithmetic
// Moments of h_i = w_i delta_i (delta_i = f_i/w_i - 1), using that the D3Q27
// weights factor as w1(cx) w1(cy) w1(cz) with w1 = (1/6, 2/3, 1/6): sums are
// taken along z, then y, then x with integer weights (1, 4, 1) and scaled by
// 1/216 at the end.  Returns p' = p* - 1, m = sum f c, P' = sum f c c - I/3.
__host__ __device__ __forceinline__ void shifted_moments(const float (&d)[27], float& pp, float& m0, float& m1,
                                                float& m2, float& P00, float& P11, float& P22, float& P01,
                                                float& P02, float& P12) {
    float A0[3][3], A1[3][3], A2[3][3];  // [cy+1][cx+1]: z-weighted sums of cz^0, cz^1, cz^2 terms
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
            const int b = cx + 3 * cy;
            const float em = d[b], e0 = d[b + 9], ep = d[b + 18];
            const float s = em + ep;
            A2[cy][cx] = s;
            A0[cy][cx] = fmaf(4.f, e0, s);
            A1[cy][cx] = ep - em;
        }
    float B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];
#pragma unroll
    for (int cx = 0; cx < 3; ++cx) {
        const float s0 = A0[0][cx] + A0[2][cx];
        B00[cx] = fmaf(4.f, A0[1][cx], s0);
        B02[cx] = s0;
        B01[cx] = A0[2][cx] - A0[0][cx];
        B10[cx] = fmaf(4.f, A1[1][cx], A1[0][cx] + A1[2][cx]);
        B11[cx] = A1[2][cx] - A1[0][cx];
        B20[cx] = fmaf(4.f, A2[1][cx], A2[0][cx] + A2[2][cx]);
    }
    constexpr float k = 1.f / 216.f;
    const float t = B00[0] + B00[2];
    pp = fmaf(4.f, B00[1], t) * k;
    m0 = (B00[2] - B00[0]) * k;
    P00 = t * k;
    m1 = fmaf(4.f, B01[1], B01[0] + B01[2]) * k;
    P01 = (B01[2] - B01[0]) * k;
    P11 = fmaf(4.f, B02[1], B02[0] + B02[2]) * k;
    m2 = fmaf(4.f, B10[1], B10[0] + B10[2]) * k;
    P02 = (B10[2] - B10[0]) * k;
    P12 = fmaf(4.f, B11[1], B11[0] + B11[2]) * k;
    P22 = fmaf(4.f, B20[1], B20[0] + B20[2]) * k;
}

// f*_i/w_i - 1 is a quadratic polynomial in c_i:
//   e0 + sum_a P^{sign c_a}_a [c_a != 0] + sum_{a<b} c_a c_b X_ab,
// evaluated for all 27 directions reusing face and xy-edge partial sums.
__host__ __device__ __forceinline__ void quad_poly27(float e0, const float (&Pp)[3], const float (&Pm)[3], float Xxy,
                                            float Xxz, float Xyz, float (&v)[27]) {
    v[IDX(0, 0, 0)] = e0;
    const float fxp = e0 + Pp[0], fxm = e0 + Pm[0];
    const float fyp = e0 + Pp[1], fym = e0 + Pm[1];
    v[IDX(1, 0, 0)] = fxp;
    v[IDX(-1, 0, 0)] = fxm;
    v[IDX(0, 1, 0)] = fyp;
    v[IDX(0, -1, 0)] = fym;
    v[IDX(0, 0, 1)] = e0 + Pp[2];
    v[IDX(0, 0, -1)] = e0 + Pm[2];
    const float epp = fxp + (Pp[1] + Xxy), epm = fxp + (Pm[1] - Xxy);
    const float emp = fxm + (Pp[1] - Xxy), emm = fxm + (Pm[1] + Xxy);
    v[IDX(1, 1, 0)] = epp;
    v[IDX(1, -1, 0)] = epm;
    v[IDX(-1, 1, 0)] = emp;
    v[IDX(-1, -1, 0)] = emm;
    v[IDX(1, 0, 1)] = fxp + (Pp[2] + Xxz);
    v[IDX(1, 0, -1)] = fxp + (Pm[2] - Xxz);
    v[IDX(-1, 0, 1)] = fxm + (Pp[2] - Xxz);
    v[IDX(-1, 0, -1)] = fxm + (Pm[2] + Xxz);
    v[IDX(0, 1, 1)] = fyp + (Pp[2] + Xyz);
    v[IDX(0, 1, -1)] = fyp + (Pm[2] - Xyz);
    v[IDX(0, -1, 1)] = fym + (Pp[2] - Xyz);
    v[IDX(0, -1, -1)] = fym + (Pm[2] + Xyz);
    const float Vpp = Xxz + Xyz, Vpm = Xxz - Xyz;  // (sx Xxz + sy Xyz) for (+,+) and (+,-)
    v[IDX(1, 1, 1)] = epp + (Pp[2] + Vpp);
    v[IDX(1, 1, -1)] = epp + (Pm[2] - Vpp);
    v[IDX(1, -1, 1)] = epm + (Pp[2] + Vpm);
    v[IDX(1, -1, -1)] = epm + (Pm[2] - Vpm);
    v[IDX(-1, 1, 1)] = emp + (Pp[2] - Vpm);
    v[IDX(-1, 1, -1)] = emp + (Pm[2] + Vpm);
    v[IDX(-1, -1, 1)] = emm + (Pp[2] - Vpp);
    v[IDX(-1, -1, -1)] = emm + (Pm[2] + Vpp);
}

// Steps 8-10 for one site from its shifted moments: forced velocity u, total
// force F = Fe + A u, Hermite coefficient a2 (Eq. 8 in closed form), and the
// post-collision shifted populations v_i = f*_i/w_i - 1 of Eq. 7 with the
// regularized non-equilibrium part and the Guo source (Eq. 6):
//   f*_i/w_i = p* + 3 c.u + 4.5 (c.B.c - tr B/3) + 1.5 c.F - 1.5 u.F + 4.5 (c.u)(c.F),
//   B = u u + (1 - omega) a2.
// Also returns a2:a2 for the dissipation estimate.
__host__ __device__ __forceinline__ void collide_site(float pp, float m0, float m1, float m2, float P00, float P11,
                                                      float P22, float P01, float P02, float P12, float Fe0,
                                                      float Fe1, float Fe2, float A_lin, float omega, float& u0,
                                                      float& u1, float& u2, float& aa, float (&v)[27]) {
    const float inv = 1.f / (1.f - 0.5f * A_lin);
    u0 = fmaf(0.5f, Fe0, m0) * inv;
    u1 = fmaf(0.5f, Fe1, m1) * inv;
    u2 = fmaf(0.5f, Fe2, m2) * inv;
    const float F0 = fmaf(A_lin, u0, Fe0), F1 = fmaf(A_lin, u1, Fe1), F2 = fmaf(A_lin, u2, Fe2);
    // a2 = Pi - p*/3 I - u u + (u F + F u)/2, with Pi - p*/3 I = P' - p'/3 I
    const float p3 = pp * (1.f / 3.f);
    const float a00 = P00 - p3 - u0 * u0 + u0 * F0;
    const float a11 = P11 - p3 - u1 * u1 + u1 * F1;
    const float a22 = P22 - p3 - u2 * u2 + u2 * F2;
    const float a01 = P01 - u0 * u1 + 0.5f * (u0 * F1 + F0 * u1);
    const float a02 = P02 - u0 * u2 + 0.5f * (u0 * F2 + F0 * u2);
    const float a12 = P12 - u1 * u2 + 0.5f * (u1 * F2 + F1 * u2);
    aa = a00 * a00 + a11 * a11 + a22 * a22 + 2.f * (a01 * a01 + a02 * a02 + a12 * a12);
    const float om1 = 1.f - omega;
    const float B00 = fmaf(om1, a00, u0 * u0), B11 = fmaf(om1, a11, u1 * u1);
    const float B22 = fmaf(om1, a22, u2 * u2), B01 = fmaf(om1, a01, u0 * u1);
    const float B02 = fmaf(om1, a02, u0 * u2), B12 = fmaf(om1, a12, u1 * u2);
    const float uF = u0 * F0 + u1 * F1 + u2 * F2;
    const float e0 = pp - 1.5f * (B00 + B11 + B22 + uF);
    const float L0 = fmaf(1.5f, F0, 3.f * u0), L1 = fmaf(1.5f, F1, 3.f * u1), L2 = fmaf(1.5f, F2, 3.f * u2);
    const float Q0 = 4.5f * fmaf(u0, F0, B00), Q1 = 4.5f * fmaf(u1, F1, B11), Q2 = 4.5f * fmaf(u2, F2, B22);
    const float Pp[3] = {Q0 + L0, Q1 + L1, Q2 + L2};
    const float Pm[3] = {Q0 - L0, Q1 - L1, Q2 - L2};
    const float Xxy = fmaf(9.f, B01, 4.5f * (u0 * F1 + u1 * F0));
    const float Xxz = fmaf(9.f, B02, 4.5f * (u0 * F2 + u2 * F0));
    const float Xyz = fmaf(9.f, B12, 4.5f * (u1 * F2 + u2 * F1));
    quad_poly27(e0, Pp, Pm, Xxy, Xxz, Xyz, v);
}

// ------------------------------------------------------------ fused kernel
// Shared-memory planes: Z6 = 6 Sz(phi) and D2 = 2 Dz(phi) on the halo-2 plane
// (Sz = (1,4,1)/6 smoothing, Dz = central difference along z), so that the
// lattice gradient of Sec. 2.3 becomes grad phi = G/72 with
//   Gx = sum_y k (Z6(x+1) - Z6(x-1)), Gy = sum_x k (Z6(y+1) - Z6(y-1)),
//   Gz = sum_x sum_y k k D2,  k = (1, 4, 1),
// the same sum as the 26-neighbour stencil, regrouped.  The curvature uses the
// same factorisation on n (planes 6 Sz n_x, 6 Sz n_y, 2 Dz n_z).
//
// Phase A reads the D3Q7 planes either per site (VEC = false) or, when nx is a
// multiple of 4, as float4 quads of 4 consecutive sites covering the halo row
// x0-4 .. x0+TX+3 (VEC = true): 7 vector loads per 4 sites.
template <class FT, int TY, int MODE, int PAR, bool VEC, class Args>
__device__ __forceinline__ void fused_tile(const Args& a, int bx, int by, int bz, long long pblock) {
    constexpr int TX = 32;
    constexpr int NT = TX * TY;
    constexpr int HX = TX + 4, HY = TY + 4, NHA = HX * HY;  // halo-2 plane (phi)
    constexpr int BX = TX + 2, BY = TY + 2, NHB = BX * BY;  // halo-1 plane (n)
    constexpr int NA = (NHA + NT - 1) / NT;
    constexpr int NB = (NHB + NT - 1) / NT;

    __shared__ float s_Z[2][NHA];        // 6 Sz phi, planes by parity
    __shared__ float s_D[2][NHA];        // 2 Dz phi
    __shared__ float s_phi[4][NT];       // phi of the interior, 4-plane ring
    __shared__ float s_n[4][3][NHB];     // unit normal, 4-plane ring
    __shared__ float s_k[3][NHB];        // 6 Sz n_x, 6 Sz n_y, 2 Dz n_z of one plane
    __shared__ float s_grad[2][4][NT];   // grad phi and |grad phi| of the interior
    // VEC: phase-A quads of the D3Q7 planes staged by cp.async one plane ahead (2-plane ring)
    constexpr int NQS = VEC ? (TX / 4 + 2) * HY : 1;  // quad index tid + k*NT < NQS
    __shared__ __align__(16) float4 s_gA[VEC ? 2 : 1][VEC ? 7 : 1][NQS];

    using C = Codec<FT>;
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int N = a.N;
    const int plane = nx * ny;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = bz * a.zc;
    const int z1 = min(z0 + a.zc, nz);

    // phase-A slots (halo-2 plane), fixed for the whole march.  A slot is one
    // site (scalar) or one float4 quad of 4 sites (VEC).
    constexpr int QX = TX / 4 + 2;  // quads per halo row
    constexpr int NQ = QX * HY;
    constexpr int NS = VEC ? (NQ + NT - 1) / NT : NA;
    constexpr int NV = VEC ? 4 : 1;
    int a_row[NS], a_idx[NS], a_int[NS];
    float ph1[NS][NV], ph2[NS][NV];  // phi one and two planes below, per site of a slot
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int idx = tid + k * NT;
        if (VEC) {
            // a_idx: halo-plane index of the quad's row; a_int: halo x of its first
            // site (-2 for the leftmost quad; sites outside [0, HX) are dropped)
            const int ry = idx / QX, qx = idx - (idx / QX) * QX;
            a_idx[k] = idx < NQ ? ry * HX : INT_MIN;
            a_row[k] = wrap_mod(y0 + ry - 2, ny) * nx + wrap_mod(x0 - 4 + 4 * qx, nx);
            a_int[k] = 4 * qx - 2;
        } else {
            a_idx[k] = idx < NHA ? idx : -1;
            const int ly = idx / HX, lx = idx - (idx / HX) * HX;
            a_row[k] = wrap_mod(y0 + ly - 2, ny) * nx + wrap_mod(x0 + lx - 2, nx);
            a_int[k] = 0;
        }
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            ph1[k][j] = 0.f;
            ph2[k][j] = 0.f;
        }
    }

    // phase-C site and its periodic neighbour offsets (32-bit site indices)
    const int lx = tid % TX, ly = tid / TX;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool active = gx < nx && gy < ny;
    const int cxs = active ? gx : nx - 1, cys = active ? gy : ny - 1;
    const int row_s = cys * nx + cxs;
    const int DX0 = cxs == 0 ? nx - 1 : -1, DX2 = cxs == nx - 1 ? 1 - nx : 1;
    const int DY0 = cys == 0 ? (ny - 1) * nx : -nx, DY2 = cys == ny - 1 ? (1 - ny) * nx : nx;
    const int DX[3] = {DX0, 0, DX2};
    const int DY[3] = {DY0, 0, DY2};
    const int c1 = (ly + 1) * BX + (lx + 1);  // own site in the halo-1 plane

    float A_lin = 0.f;
    if (MODE != MODE_INIT && a.force_kind == FK_LINEAR) A_lin = (float)a.st->A;

    // FP32 per-thread partial sums over this thread's <= zc sites; FP64 beyond
    float s_phi_acc = 0.f, s_K = 0.f, s_aa = 0.f, s_mass = 0.f, s_umax2 = 0.f;

    // one site of phase A: z-smoothed planes of zp-1 and the interior phi of zp
    auto a_site = [&](int zp, bool make_zd, int hidx, float p, float& h1, float& h2) {
        if (make_zd) {
            s_Z[(zp - 1) & 1][hidx] = fmaf(4.f, h1, h2 + p);
            s_D[(zp - 1) & 1][hidx] = p - h2;
        }
        const int hy = hidx / HX, hx = hidx - (hidx / HX) * HX;
        if (hx >= 2 && hx < TX + 2 && hy >= 2 && hy < TY + 2) s_phi[zp & 3][(hy - 2) * TX + (hx - 2)] = p;
        h2 = h1;
        h1 = p;
    };

    // VEC: start the asynchronous copies of plane zp's quads into ring slot zp & 1.
    // Every thread commits one group per call (possibly empty) so that the
    // group counts agree across the block.
    auto a_issue = [&](int zp) {
        if (VEC) {
            const int zb = wrap_mod(zp, nz) * plane;
#pragma unroll
            for (int k = 0; k < NS; ++k)
                if (a_idx[k] != INT_MIN) {
#pragma unroll
                    for (int q = 0; q < 7; ++q)
                        cp_async16(&s_gA[zp & 1][q][tid + k * NT], a.gin[q] + zb + a_row[k]);
                }
            cp_async_commit();
        }
    };

    // phi of plane zp (VEC: from the staged quads of slot zp & 1, which this
    // thread copied itself and has waited for)
    auto phaseA = [&](int zp, bool make_zd) {
        const int zb = wrap_mod(zp, nz) * plane;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (VEC) {
                if (a_idx[k] != INT_MIN) {
                    float4 p4 = s_gA[zp & 1][0][tid + k * NT];
#pragma unroll
                    for (int q = 1; q < 7; ++q) {
                        const float4 t = s_gA[zp & 1][q][tid + k * NT];
                        p4.x += t.x; p4.y += t.y; p4.z += t.z; p4.w += t.w;
                    }
                    const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int hx = a_int[k] + j;
                        if (hx >= 0 && hx < HX) a_site(zp, make_zd, a_idx[k] + hx, pv[j], ph1[k][j], ph2[k][j]);
                    }
                }
            } else if (a_idx[k] >= 0) {
                const int s = zb + a_row[k];
                float p;
                if (MODE == MODE_INIT) {
                    p = a.in_phi[s];
                } else {
                    p = __ldg(a.gin[0] + s);
#pragma unroll
                    for (int q = 1; q < 7; ++q) p += __ldg(a.gin[q] + s);
                }
                a_site(zp, make_zd, a_idx[k], p, ph1[k][0], ph2[k][0]);
            }
        }
    };

    // n at plane zp on the halo-1 plane; with make_k also the curvature
    // ingredients of plane zp-1 (needs n at zp-2, zp-1, zp of the same site,
    // which this thread wrote itself).
    auto phaseB = [&](int zp, bool make_k) {
        const float* Z = s_Z[zp & 1];
        const float* D = s_D[zp & 1];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int idx = tid + k * NT;
            if (idx < NHB) {
                const int by = idx / BX, bx = idx - (idx / BX) * BX;
                const int c = (by + 1) * HX + (bx + 1);
                const float zmm = Z[c - HX - 1], zm0 = Z[c - HX], zmp = Z[c - HX + 1];
                const float z0m = Z[c - 1], z0p = Z[c + 1];
                const float zpm = Z[c + HX - 1], zp0 = Z[c + HX], zpp = Z[c + HX + 1];
                // differences before sums keep the small gradients of a nearly uniform phi accurate
                const float Gx = fmaf(4.f, z0p - z0m, (zmp - zmm) + (zpp - zpm));
                const float Gy = fmaf(4.f, zp0 - zm0, (zpm - zmm) + (zpp - zmp));
                const float rm = fmaf(4.f, D[c - 1], D[c - HX - 1] + D[c + HX - 1]);
                const float r0 = fmaf(4.f, D[c], D[c - HX] + D[c + HX]);
                const float rp = fmaf(4.f, D[c + 1], D[c - HX + 1] + D[c + HX + 1]);
                const float Gz = fmaf(4.f, r0, rm + rp);
                constexpr float k72 = 1.f / 72.f;
                const float g0 = Gx * k72, g1 = Gy * k72, g2 = Gz * k72;
                const float gg = g0 * g0 + g1 * g1 + g2 * g2;
                const float r = rsqrtf(fmaxf(gg, 1e-20f));  // 1 / max(|grad phi|, 1e-10)
                const float n0 = g0 * r, n1 = g1 * r, n2 = g2 * r;
                s_n[zp & 3][0][idx] = n0;
                s_n[zp & 3][1][idx] = n1;
                s_n[zp & 3][2][idx] = n2;
                if (bx >= 1 && bx <= TX && by >= 1 && by <= TY) {
                    const int e = (by - 1) * TX + (bx - 1);
                    s_grad[zp & 1][0][e] = g0;
                    s_grad[zp & 1][1][e] = g1;
                    s_grad[zp & 1][2][e] = g2;
                    s_grad[zp & 1][3][e] = gg * r;  // |grad phi|
                }
                if (make_k) {
                    s_k[0][idx] = fmaf(4.f, s_n[(zp - 1) & 3][0][idx], s_n[(zp - 2) & 3][0][idx] + n0);
                    s_k[1][idx] = fmaf(4.f, s_n[(zp - 1) & 3][1][idx], s_n[(zp - 2) & 3][1][idx] + n1);
                    s_k[2][idx] = n2 - s_n[(zp - 2) & 3][2][idx];
                }
            }
        }
    };

    // prologue: phi history from z0-2, gradient planes and n at z0-1, z0
    // (VEC: each plane's copies are waited for at once; plane z0+2 is left in flight)
    a_issue(z0 - 2);
    cp_async_wait<0>();
    phaseA(z0 - 2, false);
    a_issue(z0 - 1);
    cp_async_wait<0>();
    phaseA(z0 - 1, false);
    a_issue(z0);
    cp_async_wait<0>();
    phaseA(z0, true);
    __syncthreads();
    phaseB(z0 - 1, false);
    a_issue(z0 + 1);
    cp_async_wait<0>();
    phaseA(z0 + 1, true);
    __syncthreads();
    phaseB(z0, false);
    a_issue(z0 + 2);

    for (int z = z0; z < z1; ++z) {
        const int DZ0 = z == 0 ? (nz - 1) * plane : -plane;
        const int DZ2 = z == nz - 1 ? (1 - nz) * plane : plane;
        const int DZ[3] = {DZ0, 0, DZ2};
        const int s = z * plane + row_s;

        // ---- issue this plane's population loads first
        float dl[27];
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
                    if (PAR == 0) {
                        dl[i] = C::ld(static_cast<const FT*>(a.fk[i]) + s);
                    } else {  // f_i(x) sits in slot (x - c_i, opposite of i)
                        const int src = s + DZ[1 - CZ(i)] + DY[1 - CY(i)] + DX[1 - CX(i)];
                        dl[i] = C::ld(static_cast<const FT*>(a.fk[26 - i]) + src);
                    }
                }
                if (MODE == MODE_STEP) {
#pragma unroll
                    for (int q = 0; q < 7; ++q) gl[q] = __ldg(a.gin[q] + s);
                }
            }
        }

        a_issue(z + 3);       // next plane's phase-A copies
        cp_async_wait<1>();   // this thread's copies of plane z+2 have landed
        phaseA(z + 2, true);
        __syncthreads();
        phaseB(z + 1, true);
        __syncthreads();

        if (active) {
            const int e = ly * TX + lx;
            const float phi = s_phi[z & 3][e];
            const float n0 = s_n[z & 3][0][c1], n1 = s_n[z & 3][1][c1], n2 = s_n[z & 3][2][c1];

            if (MODE == MODE_INIT) {
                // f = f^eq(p* = 1, u): delta_i = 3 c.u + 4.5 (c.u)^2 - 1.5 u^2 (even layout)
                const float u0 = uin0, u1 = uin1, u2 = uin2;
                const float uu = u0 * u0 + u1 * u1 + u2 * u2;
                const float Pp[3] = {fmaf(4.5f * u0, u0, 3.f * u0), fmaf(4.5f * u1, u1, 3.f * u1),
                                     fmaf(4.5f * u2, u2, 3.f * u2)};
                const float Pm[3] = {fmaf(4.5f * u0, u0, -3.f * u0), fmaf(4.5f * u1, u1, -3.f * u1),
                                     fmaf(4.5f * u2, u2, -3.f * u2)};
                float v[27];
                quad_poly27(-1.5f * uu, Pp, Pm, 9.f * u0 * u1, 9.f * u0 * u2, 9.f * u1 * u2, v);
#pragma unroll
                for (int i = 0; i < 27; ++i) C::st(static_cast<FT*>(a.fk[i]) + s, v[i]);
                const float phs = a.sharp * fmaxf(phi * (1.f - phi), 0.f);  // interface indicator, 0 outside [0, 1]
                const float j0 = fmaf(4.f * phi, u0, phs * n0);
                const float j1 = fmaf(4.f * phi, u1, phs * n1);
                const float j2 = fmaf(4.f * phi, u2, phs * n2);
                a.gout[0][s] = 0.25f * phi;
                a.gout[1][s] = 0.125f * (phi + j0);
                a.gout[2][s] = 0.125f * (phi - j0);
                a.gout[3][s] = 0.125f * (phi + j1);
                a.gout[4][s] = 0.125f * (phi - j1);
                a.gout[5][s] = 0.125f * (phi + j2);
                a.gout[6][s] = 0.125f * (phi - j2);
                s_phi_acc += phi;
                s_K = fmaf(0.5f, uu, s_K);
                s_umax2 = fmaxf(s_umax2, uu);
            } else {
                // ---- step 4: kappa = div n from the factorised planes (sum / 72)
                const float* K0 = s_k[0];
                const float* K1 = s_k[1];
                const float* K2 = s_k[2];
                const float kx = fmaf(4.f, K0[c1 + 1] - K0[c1 - 1],
                                      (K0[c1 - BX + 1] - K0[c1 - BX - 1]) + (K0[c1 + BX + 1] - K0[c1 + BX - 1]));
                const float ky = fmaf(4.f, K1[c1 + BX] - K1[c1 - BX],
                                      (K1[c1 + BX - 1] - K1[c1 - BX - 1]) + (K1[c1 + BX + 1] - K1[c1 - BX + 1]));
                const float qm = fmaf(4.f, K2[c1 - 1], K2[c1 - BX - 1] + K2[c1 + BX - 1]);
                const float q0 = fmaf(4.f, K2[c1], K2[c1 - BX] + K2[c1 + BX]);
                const float qp = fmaf(4.f, K2[c1 + 1], K2[c1 - BX + 1] + K2[c1 + BX + 1]);
                const float kz = fmaf(4.f, q0, qm + qp);
                const float kap = (kx + ky + kz) * (1.f / 72.f);

                // ---- steps 5-6: surface tension and external force
                const float gr0 = s_grad[z & 1][0][e], gr1 = s_grad[z & 1][1][e];
                const float gr2 = s_grad[z & 1][2][e], grm = s_grad[z & 1][3][e];
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

                // ---- step 7: moments of the shifted populations
                float pp, m0, m1, m2, P00, P11, P22, P01, P02, P12;
                shifted_moments(dl, pp, m0, m1, m2, P00, P11, P22, P01, P02, P12);

                if (MODE == MODE_MOMENTS) {
                    // ---- step 8: forced velocity
                    const float inv = 1.f / (1.f - 0.5f * A_lin);
                    const float u0 = fmaf(0.5f, Fe0, m0) * inv;
                    const float u1 = fmaf(0.5f, Fe1, m1) * inv;
                    const float u2 = fmaf(0.5f, Fe2, m2) * inv;
                    if (a.out_rho) a.out_rho[s] = 1.f + pp;
                    if (a.out_u) {
                        a.out_u[s] = u0;
                        a.out_u[N + s] = u1;
                        a.out_u[2 * N + s] = u2;
                    }
                    if (a.out_phi) a.out_phi[s] = phi;
                } else {
                    // ---- steps 8-10: velocity, force, Hermite coefficient, collision
                    float u0, u1, u2, aa, v[27];
                    collide_site(pp, m0, m1, m2, P00, P11, P22, P01, P02, P12, Fe0, Fe1, Fe2, A_lin, a.omega,
                                 u0, u1, u2, aa, v);

                    // ---- step 13 (per site): partial sums
                    const float uu = u0 * u0 + u1 * u1 + u2 * u2;
                    s_phi_acc += phi;
                    s_K = fmaf(0.5f, uu, s_K);
                    s_aa += aa;
                    s_mass += pp;
                    s_umax2 = fmaxf(s_umax2, uu);

                    // ---- step 12: AA streaming stores
#pragma unroll
                    for (int i = 0; i < 27; ++i) {
                        if (PAR == 0) {  // f*_i to slot (x, opposite of i)
                            C::st(static_cast<FT*>(a.fk[26 - i]) + s, v[i]);
                        } else {         // f*_i to slot (x + c_i, i)
                            const int dst = s + DZ[1 + CZ(i)] + DY[1 + CY(i)] + DX[1 + CX(i)];
                            C::st(static_cast<FT*>(a.fk[i]) + dst, v[i]);
                        }
                    }

                    // ---- step 11: D3Q7 BGK with the sharpening equilibrium, push
                    const float om = a.omega_phi;
                    const float phs = a.sharp * fmaxf(phi * (1.f - phi), 0.f);  // interface indicator, 0 outside [0, 1]
                    const float j0 = fmaf(4.f * phi, u0, phs * n0);
                    const float j1 = fmaf(4.f * phi, u1, phs * n1);
                    const float j2 = fmaf(4.f * phi, u2, phs * n2);
                    a.gout[0][s] = fmaf(om, 0.25f * phi - gl[0], gl[0]);
                    a.gout[1][s + DX[2]] = fmaf(om, 0.125f * (phi + j0) - gl[1], gl[1]);
                    a.gout[2][s + DX[0]] = fmaf(om, 0.125f * (phi - j0) - gl[2], gl[2]);
                    a.gout[3][s + DY[2]] = fmaf(om, 0.125f * (phi + j1) - gl[3], gl[3]);
                    a.gout[4][s + DY[0]] = fmaf(om, 0.125f * (phi - j1) - gl[4], gl[4]);
                    a.gout[5][s + DZ[2]] = fmaf(om, 0.125f * (phi + j2) - gl[5], gl[5]);
                    a.gout[6][s + DZ[0]] = fmaf(om, 0.125f * (phi - j2) - gl[6], gl[6]);
                }
            }
        }
    }

    if (MODE != MODE_MOMENTS) {
        double v0 = s_phi_acc, v1 = s_K, v2 = s_aa, v3 = s_mass, v4 = s_umax2;
        block_reduce5<NT>(v0, v1, v2, v3, v4);
        if (tid == 0) {
            double* out = a.partials + pblock * NPART;
            out[0] = v0; out[1] = v1; out[2] = v2; out[3] = v3; out[4] = v4;
        }
    }
}

// One box: a block per (32 x TY tile, z-chunk).
template <class FT, int TY, int MODE, int PAR, bool VEC>
__global__ void __launch_bounds__(32 * TY, (TY >= 16 ? 1 : 512 / (32 * TY)))
fused_step_kernel(const __grid_constant__ StepArgs a) {
    const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    fused_tile<FT, TY, MODE, PAR, VEC>(a, blockIdx.x, blockIdx.y, blockIdx.z, b);
}

// ------------------------------------------------------ batched ensemble
// Many independent periodic boxes in one array set: box b's f planes start at
// element f_off and are N_b apart; its g planes likewise at g_off in each of
// the two g buffers.  The work list enumerates (box, tile, z-chunk) items.
struct BoxDesc {
    int nx, ny, nz, N;
    long long f_off, g_off;                 // element offsets into the batch arrays
    float omega, omega_phi, sharp, beta;
    int item0, tiles_x, tiles_y, tiles_z;   // this box's slice of the work list
};

struct BatchArgs {
    int nitems, zc;
    const BoxDesc* boxes;
    const int* item_box;   // box of each work item
    void* f;               // all boxes' populations (storage type)
    const float* g_in;
    float* g_out;
    double* partials;      // NPART per work item
};

// Plane q of a plane set stored q * stride elements apart.
template <class T>
struct PlaneSet {
    T* base;
    long long stride;
    __device__ __forceinline__ T* operator[](int q) const { return base + q * stride; }
};

// The argument view of one box for fused_tile (steps only, no external force).
template <class FT>
struct BoxTileArgs {
    int nx, ny, nz, zc, N;
    PlaneSet<FT> fk;
    PlaneSet<const float> gin;
    PlaneSet<float> gout;
    int force_kind;
    float omega, omega_phi, sharp, beta, gc0, gc1, gc2, A_abc;
    const float* abc;
    const DevState* st;
    double* partials;
    float *out_rho, *out_u, *out_phi;
    const float *in_phi, *in_u;
};

// Persistent kernel: the grid strides over the work list of all boxes.
template <class FT, int TY, int PAR, bool VEC>
__global__ void __launch_bounds__(32 * TY, (TY >= 16 ? 1 : 512 / (32 * TY)))
batch_step_kernel(const __grid_constant__ BatchArgs b) {
    for (int item = blockIdx.x; item < b.nitems; item += gridDim.x) {
        const BoxDesc d = b.boxes[b.item_box[item]];
        BoxTileArgs<FT> t;
        t.nx = d.nx; t.ny = d.ny; t.nz = d.nz; t.zc = b.zc; t.N = d.N;
        t.fk = PlaneSet<FT>{static_cast<FT*>(b.f) + d.f_off, (long long)d.N};
        t.gin = PlaneSet<const float>{b.g_in + d.g_off, (long long)d.N};
        t.gout = PlaneSet<float>{b.g_out + d.g_off, (long long)d.N};
        t.force_kind = FK_NONE;
        t.omega = d.omega; t.omega_phi = d.omega_phi; t.sharp = d.sharp; t.beta = d.beta;
        t.gc0 = t.gc1 = t.gc2 = t.A_abc = 0.f;
        t.abc = nullptr; t.st = nullptr; t.partials = b.partials;
        t.out_rho = t.out_u = t.out_phi = nullptr;
        t.in_phi = t.in_u = nullptr;
        const int local = item - d.item0;
        const int tx = local % d.tiles_x, rest = local / d.tiles_x;
        fused_tile<FT, TY, MODE_STEP, PAR, VEC>(t, tx, rest % d.tiles_y, rest / d.tiles_y, item);
        __syncthreads();  // the shared rings are reused by the block's next item
    }
}

// Launch one fused kernel instance.  Defined per storage type in lbgb_step_*.cu.
// Records a message for lb_last_error() (defined with the C ABI).
void set_last_error(const char* msg);

// One step of every box of a batch (persistent grid of `blocks` blocks).
template <class FT>
cudaError_t launch_batch(int parity, int ty, bool vec, int blocks, const BatchArgs& b, cudaStream_t st);
// Resident blocks per SM of the batch kernel for this shape (0 on error).
template <class FT>
int batch_blocks_per_sm(int ty, bool vec);

// vec selects the float4 phase-A loads (requires nx % 4 == 0).
template <class FT>
cudaError_t launch_fused(int mode, int parity, int ty, bool vec, dim3 grid, const StepArgs& a, cudaStream_t st);

}  // namespace lbgb
