// lbgb_kernels.cuh -- sm_103a kernels of the fused two-phase lattice Boltzmann step.
//
// One kernel template does the whole per-site time step of accLB (arXiv
// 2505.01126, Sec. 2); the numbered steps 1-13 are those listed in lbgb.h.
//
// Work decomposition.  A thread block owns a 32 x TY column of sites and
// marches it through a chunk of zc planes.  In the interval of plane z it
//   A. computes phi = sum_q g_q (step 1) on the (32+4) x (TY+4) plane z+4
//      (halo 2: kappa needs phi within radius 2) and the z-smoothed planes
//      of z+3,
//   B. computes grad phi and n (steps 2-3) on the (32+2) x (TY+2) plane z+2
//      and the curvature ingredients of plane z+1,
//   C. for the 32 x TY interior of plane z: kappa (step 4), the forces (5-6),
//      the hydrodynamic moments of its populations (7), velocity, Hermite
//      coefficient and regularized collision (8-10), the D3Q7 BGK (11),
//      streaming stores (12) and FP64 partial sums (13),
// with one barrier per plane: each phase reads only what earlier intervals
// wrote, and shared-memory rings keep each plane until its last reader.  The
// 27 f and 7 g loads of plane z+1 are issued by each warp right after its
// phase C of plane z, so they are in flight across the barrier and phases A
// and B.  The moment-only storage (MC) replaces the f loads by coefficient
// planes staged in shared memory and pulled in phase C.
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
    // moment-only storage: the 10 coefficients (e0, P+[3], P-[3], Xxy, Xxz, Xyz)
    // of the post-collision polynomial f*_i/w_i - 1 of each site (see quad_poly27)
    const float* cin[10];   // at t (written by step t-1, or by INIT at t = 0)
    float* cout[10];        // at t+1 (INIT: at 0)
    // density and viscosity contrasts (kernels with VD = true): rho and tau
    // linear in phi, rho = rho_g + phi drho, tau = tau_g + phi dtau; buoyancy
    // (rho - rho_ref) gb (gb = 0 without gravity)
    float rho_g, drho, tau_g, dtau;
    float gb0, gb1, gb2, rho_ref;
    // 16-bit D3Q7 storage (kernels with G16): gin/gout then point at planes of
    // the storage type holding gamma_q = g_q/w_q - phi~, and these at the
    // plane of phi~, each site's phase field of the previous step rounded to
    // the storage type (read at t, written at t+1)
    const void* gphi_in;
    void* gphi_out;
};

// ---------------------------------------------------------- storage codecs
// Every storage type holds the shifted, scaled population delta_i = f_i/w_i - 1
// (zero at rest, O(Ma) in a flow, never subnormal in 16 bits); all arithmetic
// is FP32.  The moments and the collision below work on delta directly, so no
// codec multiplies by w_i.
template <class T>
struct Codec;

// ldr loads the stored value as is and dec widens it to FP32, so that a load
// can be issued well ahead of the conversion that waits for it.
// The pair members serve the paired kernel (two x-adjacent sites per thread):
// raw2 holds both sites' stored values of one direction, ldr2/st2 access an
// aligned pair (even first site), pack joins two single loads.
template <>
struct Codec<float> {
    using raw = float;
    using raw2 = float2;
    static __device__ __forceinline__ raw ldr(const float* p) { return *p; }
    static __device__ __forceinline__ float dec(raw r) { return r; }
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
    static __device__ __forceinline__ raw2 ldr2(const float* p) { return *reinterpret_cast<const float2*>(p); }
    static __device__ __forceinline__ raw2 pack(raw a, raw b) { return make_float2(a, b); }
    static __device__ __forceinline__ float2 dec2(raw2 r) { return r; }
    static __device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
};

// Bit-pattern views of the 16-bit types (the 16-bit D3Q7 storage keeps phi~
// and staged values as raw bits in shared memory): dec2u widens the pair held
// in a 32-bit word (first value in the low half), enc2u rounds a pair into
// one, decu / encu do the same for one value.
template <class T, class R2>
struct Bits16 {
    static __device__ __forceinline__ float2 dec2u(unsigned u) {
        union { unsigned u; R2 r; } c;
        c.u = u;
        return Codec<T>::dec2(c.r);
    }
    static __device__ __forceinline__ unsigned enc2u(float2 v) {
        union { unsigned u; R2 r; } c;
        c.r = Codec<T>::enc2(v);
        return c.u;
    }
    static __device__ __forceinline__ float decu(unsigned short h) {
        union { unsigned short u; T r; } c;
        c.u = h;
        return Codec<T>::dec(c.r);
    }
    static __device__ __forceinline__ unsigned short encu(float v) {
        union { unsigned short u; T r; } c;
        c.r = Codec<T>::enc(v);
        return c.u;
    }
};

template <>
struct Codec<__half> {
    using raw = __half;
    static __device__ __forceinline__ raw ldr(const __half* p) { return *p; }
    static __device__ __forceinline__ float dec(raw r) { return __half2float(r); }
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
    using raw2 = __half2;
    static __device__ __forceinline__ raw2 ldr2(const __half* p) { return *reinterpret_cast<const __half2*>(p); }
    static __device__ __forceinline__ raw2 pack(raw a, raw b) { return __halves2half2(a, b); }
    static __device__ __forceinline__ float2 dec2(raw2 r) { return __half22float2(r); }
    static __device__ __forceinline__ void st2(__half* p, float2 v) {
        *reinterpret_cast<__half2*>(p) = __float22half2_rn(v);
    }
    static __device__ __forceinline__ raw enc(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ raw2 enc2(float2 v) { return __float22half2_rn(v); }
    static __device__ __forceinline__ raw lo(raw2 r) { return __low2half(r); }
    static __device__ __forceinline__ raw hi(raw2 r) { return __high2half(r); }
};

template <>
struct Codec<__nv_bfloat16> {
    using raw = __nv_bfloat16;
    static __device__ __forceinline__ raw ldr(const __nv_bfloat16* p) { return *p; }
    static __device__ __forceinline__ float dec(raw r) { return __bfloat162float(r); }
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    using raw2 = __nv_bfloat162;
    static __device__ __forceinline__ raw2 ldr2(const __nv_bfloat16* p) {
        return *reinterpret_cast<const __nv_bfloat162*>(p);
    }
    static __device__ __forceinline__ raw2 pack(raw a, raw b) { return __halves2bfloat162(a, b); }
    static __device__ __forceinline__ float2 dec2(raw2 r) { return __bfloat1622float2(r); }
    static __device__ __forceinline__ void st2(__nv_bfloat16* p, float2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
    }
    static __device__ __forceinline__ raw enc(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ raw2 enc2(float2 v) { return __float22bfloat162_rn(v); }
    static __device__ __forceinline__ raw lo(raw2 r) { return __low2bfloat16(r); }
    static __device__ __forceinline__ raw hi(raw2 r) { return __high2bfloat16(r); }
};

template <class T>
struct Bits;
template <>
struct Bits<__half> : Bits16<__half, __half2> {};
template <>
struct Bits<__nv_bfloat16> : Bits16<__nv_bfloat16, __nv_bfloat162> {};
template <>
struct Bits<float> {  // never used with FP32 storage; present so that the tile body compiles
    static __device__ __forceinline__ float2 dec2u(unsigned) { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ unsigned enc2u(float2) { return 0u; }
    static __device__ __forceinline__ float decu(unsigned short) { return 0.f; }
    static __device__ __forceinline__ unsigned short encu(float) { return 0; }
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
// 8-byte asynchronous global -> shared copy (both addresses 8-byte aligned).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
// 4-byte asynchronous global -> shared copy (any 4-byte aligned address).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
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
// collide_coefs stops at the ten coefficients of that polynomial (the state
// kept by the moment-only storage); collide_site also evaluates it.
__host__ __device__ __forceinline__ void collide_coefs(float pp, float m0, float m1, float m2, float P00, float P11,
                                                       float P22, float P01, float P02, float P12, float Fe0,
                                                       float Fe1, float Fe2, float A_lin, float omega, float& u0,
                                                       float& u1, float& u2, float& aa, float& e0, float (&Pp)[3],
                                                       float (&Pm)[3], float& Xxy, float& Xxz, float& Xyz) {
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
    e0 = pp - 1.5f * (B00 + B11 + B22 + uF);
    const float L0 = fmaf(1.5f, F0, 3.f * u0), L1 = fmaf(1.5f, F1, 3.f * u1), L2 = fmaf(1.5f, F2, 3.f * u2);
    const float Q0 = 4.5f * fmaf(u0, F0, B00), Q1 = 4.5f * fmaf(u1, F1, B11), Q2 = 4.5f * fmaf(u2, F2, B22);
    Pp[0] = Q0 + L0; Pp[1] = Q1 + L1; Pp[2] = Q2 + L2;
    Pm[0] = Q0 - L0; Pm[1] = Q1 - L1; Pm[2] = Q2 - L2;
    Xxy = fmaf(9.f, B01, 4.5f * (u0 * F1 + u1 * F0));
    Xxz = fmaf(9.f, B02, 4.5f * (u0 * F2 + u2 * F0));
    Xyz = fmaf(9.f, B12, 4.5f * (u1 * F2 + u2 * F1));
}

__host__ __device__ __forceinline__ void collide_site(float pp, float m0, float m1, float m2, float P00, float P11,
                                                      float P22, float P01, float P02, float P12, float Fe0,
                                                      float Fe1, float Fe2, float A_lin, float omega, float& u0,
                                                      float& u1, float& u2, float& aa, float (&v)[27]) {
    float e0, Pp[3], Pm[3], Xxy, Xxz, Xyz;
    collide_coefs(pp, m0, m1, m2, P00, P11, P22, P01, P02, P12, Fe0, Fe1, Fe2, A_lin, omega, u0, u1, u2, aa, e0, Pp,
                  Pm, Xxy, Xxz, Xyz);
    quad_poly27(e0, Pp, Pm, Xxy, Xxz, Xyz, v);
}

// ---------------------------------------------- two sites per thread (PAIR)
// The 16-bit storages are bound by instruction issue, not HBM.  Their paired
// kernel gives each thread two x-adjacent sites and evaluates every per-site
// formula for both at once with sm_100's packed two-lane FP32 instructions
// (FADD2, FMUL2, FFMA2: one instruction, two IEEE-rounded FP32 results), so
// the arithmetic takes half the issue slots.  .x is the even site, .y the odd.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, as b * (-1) + a: the product is exact, so this is the rounded difference
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// shifted_moments for a pair of sites (the same separable sums).
__device__ __forceinline__ void shifted_moments2(const float2 (&d)[27], float2& pp, float2& m0, float2& m1,
                                                 float2& m2, float2& P00, float2& P11, float2& P22, float2& P01,
                                                 float2& P02, float2& P12) {
    const float2 four = f2(4.f);
    float2 A0[3][3], A1[3][3], A2[3][3];
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
            const int b = cx + 3 * cy;
            const float2 s = add2(d[b], d[b + 18]);
            A2[cy][cx] = s;
            A0[cy][cx] = fma2(four, d[b + 9], s);
            A1[cy][cx] = sub2(d[b + 18], d[b]);
        }
    float2 B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];
#pragma unroll
    for (int cx = 0; cx < 3; ++cx) {
        const float2 s0 = add2(A0[0][cx], A0[2][cx]);
        B00[cx] = fma2(four, A0[1][cx], s0);
        B02[cx] = s0;
        B01[cx] = sub2(A0[2][cx], A0[0][cx]);
        B10[cx] = fma2(four, A1[1][cx], add2(A1[0][cx], A1[2][cx]));
        B11[cx] = sub2(A1[2][cx], A1[0][cx]);
        B20[cx] = fma2(four, A2[1][cx], add2(A2[0][cx], A2[2][cx]));
    }
    const float2 k = f2(1.f / 216.f);
    const float2 t = add2(B00[0], B00[2]);
    pp = mul2(fma2(four, B00[1], t), k);
    m0 = mul2(sub2(B00[2], B00[0]), k);
    P00 = mul2(t, k);
    m1 = mul2(fma2(four, B01[1], add2(B01[0], B01[2])), k);
    P01 = mul2(sub2(B01[2], B01[0]), k);
    P11 = mul2(fma2(four, B02[1], add2(B02[0], B02[2])), k);
    m2 = mul2(fma2(four, B10[1], add2(B10[0], B10[2])), k);
    P02 = mul2(sub2(B10[2], B10[0]), k);
    P12 = mul2(fma2(four, B11[1], add2(B11[0], B11[2])), k);
    P22 = mul2(fma2(four, B20[1], add2(B20[0], B20[2])), k);
}

// quad_poly27 for a pair of sites.
__device__ __forceinline__ void quad_poly27_2(float2 e0, const float2 (&Pp)[3], const float2 (&Pm)[3], float2 Xxy,
                                              float2 Xxz, float2 Xyz, float2 (&v)[27]) {
    v[IDX(0, 0, 0)] = e0;
    const float2 fxp = add2(e0, Pp[0]), fxm = add2(e0, Pm[0]);
    const float2 fyp = add2(e0, Pp[1]), fym = add2(e0, Pm[1]);
    v[IDX(1, 0, 0)] = fxp;
    v[IDX(-1, 0, 0)] = fxm;
    v[IDX(0, 1, 0)] = fyp;
    v[IDX(0, -1, 0)] = fym;
    v[IDX(0, 0, 1)] = add2(e0, Pp[2]);
    v[IDX(0, 0, -1)] = add2(e0, Pm[2]);
    const float2 epp = add2(fxp, add2(Pp[1], Xxy)), epm = add2(fxp, sub2(Pm[1], Xxy));
    const float2 emp = add2(fxm, sub2(Pp[1], Xxy)), emm = add2(fxm, add2(Pm[1], Xxy));
    v[IDX(1, 1, 0)] = epp;
    v[IDX(1, -1, 0)] = epm;
    v[IDX(-1, 1, 0)] = emp;
    v[IDX(-1, -1, 0)] = emm;
    v[IDX(1, 0, 1)] = add2(fxp, add2(Pp[2], Xxz));
    v[IDX(1, 0, -1)] = add2(fxp, sub2(Pm[2], Xxz));
    v[IDX(-1, 0, 1)] = add2(fxm, sub2(Pp[2], Xxz));
    v[IDX(-1, 0, -1)] = add2(fxm, add2(Pm[2], Xxz));
    v[IDX(0, 1, 1)] = add2(fyp, add2(Pp[2], Xyz));
    v[IDX(0, 1, -1)] = add2(fyp, sub2(Pm[2], Xyz));
    v[IDX(0, -1, 1)] = add2(fym, sub2(Pp[2], Xyz));
    v[IDX(0, -1, -1)] = add2(fym, add2(Pm[2], Xyz));
    const float2 Vpp = add2(Xxz, Xyz), Vpm = sub2(Xxz, Xyz);
    v[IDX(1, 1, 1)] = add2(epp, add2(Pp[2], Vpp));
    v[IDX(1, 1, -1)] = add2(epp, sub2(Pm[2], Vpp));
    v[IDX(1, -1, 1)] = add2(epm, add2(Pp[2], Vpm));
    v[IDX(1, -1, -1)] = add2(epm, sub2(Pm[2], Vpm));
    v[IDX(-1, 1, 1)] = add2(emp, sub2(Pp[2], Vpm));
    v[IDX(-1, 1, -1)] = add2(emp, add2(Pm[2], Vpm));
    v[IDX(-1, -1, 1)] = add2(emm, sub2(Pp[2], Vpp));
    v[IDX(-1, -1, -1)] = add2(emm, add2(Pm[2], Vpp));
}

// collide_site for a pair of sites: steps 8-10 (inv = 1/(1 - A/2) is the same
// for both; the relaxation rates may differ, with density contrasts).
__device__ __forceinline__ void collide_pair(float2 pp, float2 m0, float2 m1, float2 m2, float2 P00, float2 P11,
                                             float2 P22, float2 P01, float2 P02, float2 P12, float2 Fe0, float2 Fe1,
                                             float2 Fe2, float A_lin, float inv_s, float2 omega, float2& u0,
                                             float2& u1, float2& u2, float2& aa, float2 (&v)[27]) {
    const float2 half = f2(0.5f), inv = f2(inv_s), A = f2(A_lin);
    u0 = mul2(fma2(half, Fe0, m0), inv);
    u1 = mul2(fma2(half, Fe1, m1), inv);
    u2 = mul2(fma2(half, Fe2, m2), inv);
    const float2 F0 = fma2(A, u0, Fe0), F1 = fma2(A, u1, Fe1), F2 = fma2(A, u2, Fe2);
    // a2 = Pi - p*/3 I - u u + (u F + F u)/2, with Pi - p*/3 I = P' - p'/3 I
    const float2 p3 = mul2(pp, f2(1.f / 3.f));
    const float2 a00 = fma2(u0, sub2(F0, u0), sub2(P00, p3));
    const float2 a11 = fma2(u1, sub2(F1, u1), sub2(P11, p3));
    const float2 a22 = fma2(u2, sub2(F2, u2), sub2(P22, p3));
    const float2 a01 = fma2(half, fma2(u0, F1, mul2(F0, u1)), fma2(mul2(u0, f2(-1.f)), u1, P01));
    const float2 a02 = fma2(half, fma2(u0, F2, mul2(F0, u2)), fma2(mul2(u0, f2(-1.f)), u2, P02));
    const float2 a12 = fma2(half, fma2(u1, F2, mul2(F1, u2)), fma2(mul2(u1, f2(-1.f)), u2, P12));
    const float2 offd = fma2(a01, a01, fma2(a02, a02, mul2(a12, a12)));
    aa = fma2(f2(2.f), offd, fma2(a00, a00, fma2(a11, a11, mul2(a22, a22))));
    const float2 om1 = sub2(f2(1.f), omega);
    const float2 B00 = fma2(om1, a00, mul2(u0, u0)), B11 = fma2(om1, a11, mul2(u1, u1));
    const float2 B22 = fma2(om1, a22, mul2(u2, u2)), B01 = fma2(om1, a01, mul2(u0, u1));
    const float2 B02 = fma2(om1, a02, mul2(u0, u2)), B12 = fma2(om1, a12, mul2(u1, u2));
    const float2 uF = fma2(u0, F0, fma2(u1, F1, mul2(u2, F2)));
    const float2 e0 = fma2(f2(-1.5f), add2(add2(B00, B11), add2(B22, uF)), pp);
    const float2 L0 = fma2(f2(1.5f), F0, mul2(f2(3.f), u0)), L1 = fma2(f2(1.5f), F1, mul2(f2(3.f), u1));
    const float2 L2 = fma2(f2(1.5f), F2, mul2(f2(3.f), u2));
    const float2 Q0 = mul2(f2(4.5f), fma2(u0, F0, B00)), Q1 = mul2(f2(4.5f), fma2(u1, F1, B11));
    const float2 Q2 = mul2(f2(4.5f), fma2(u2, F2, B22));
    const float2 Pp[3] = {add2(Q0, L0), add2(Q1, L1), add2(Q2, L2)};
    const float2 Pm[3] = {sub2(Q0, L0), sub2(Q1, L1), sub2(Q2, L2)};
    const float2 Xxy = fma2(f2(9.f), B01, mul2(f2(4.5f), fma2(u0, F1, mul2(u1, F0))));
    const float2 Xxz = fma2(f2(9.f), B02, mul2(f2(4.5f), fma2(u0, F2, mul2(u2, F0))));
    const float2 Xyz = fma2(f2(9.f), B12, mul2(f2(4.5f), fma2(u1, F2, mul2(u2, F1))));
    quad_poly27_2(e0, Pp, Pm, Xxy, Xxz, Xyz, v);
}

// Density and viscosity contrasts (Sec. 2.3), per site, from phi, grad phi,
// the shifted moments (p' = p* - 1, m, P' = Pi - I/3) and the force density
// F = F^s + F^ext:
//   rho = rho_g + phi drho, tau = tau_g + phi dtau, omega = 1/tau;
//   F^b = (rho - rho_ref) gb, buoyancy (Sec. 5.2; zero when gb = 0);
//   F^p = -p' cs^2 grad rho (the pressure measured from its rest value);
//   u0 = (m + F'/(2 rho)) / (1 - A/2), F' = F + F^b + F^p;
//   F^nu = -(nu omega / cs^2) (Pi - Pi^eq(u0)) grad rho, nu omega / cs^2 = 1 - omega/2,
//          Pi - Pi^eq(u0) = P' - (p'/3) I - u0 u0;
// returns the acceleration (F' + F^nu)/rho in F (which collide_coefs then
// treats as the force of a unit-density fluid), omega, and the weight
// 2 nu (3/(2 tau))^2 = 1.5 (1 - omega/2) omega that turns a2:a2 into the
// site's share of eps.
__host__ __device__ __forceinline__ void vd_force(float phi, float gp0, float gp1, float gp2, float pp, float m0,
                                                  float m1, float m2, float P00, float P11, float P22, float P01,
                                                  float P02, float P12, float A_lin, float rho_g, float drho,
                                                  float tau_g, float dtau, float gb0, float gb1, float gb2,
                                                  float rho_ref, float& F0, float& F1, float& F2, float& omega,
                                                  float& aa_w) {
    const float rho = fmaf(phi, drho, rho_g);
    const float irho = 1.f / rho;
    omega = 1.f / fmaf(phi, dtau, tau_g);
    const float q0 = drho * gp0, q1 = drho * gp1, q2 = drho * gp2;  // grad rho
    const float br = rho - rho_ref;
    const float fp = pp * (-1.f / 3.f);
    const float G0 = fmaf(fp, q0, fmaf(br, gb0, F0)), G1 = fmaf(fp, q1, fmaf(br, gb1, F1));
    const float G2 = fmaf(fp, q2, fmaf(br, gb2, F2));
    const float h = 0.5f * irho, inv = 1.f / (1.f - 0.5f * A_lin);
    const float v0 = fmaf(h, G0, m0) * inv, v1 = fmaf(h, G1, m1) * inv, v2 = fmaf(h, G2, m2) * inv;
    const float p3 = pp * (1.f / 3.f);
    const float n00 = P00 - p3 - v0 * v0, n11 = P11 - p3 - v1 * v1, n22 = P22 - p3 - v2 * v2;
    const float n01 = P01 - v0 * v1, n02 = P02 - v0 * v2, n12 = P12 - v1 * v2;
    const float c = 0.5f * omega - 1.f;  // -nu omega / cs^2
    F0 = fmaf(c, fmaf(n00, q0, fmaf(n01, q1, n02 * q2)), G0) * irho;
    F1 = fmaf(c, fmaf(n01, q0, fmaf(n11, q1, n12 * q2)), G1) * irho;
    F2 = fmaf(c, fmaf(n02, q0, fmaf(n12, q1, n22 * q2)), G2) * irho;
    aa_w = 1.5f * (1.f - 0.5f * omega) * omega;
}

// vd_force for a pair of sites (the same formulas, two lanes per instruction;
// grad phi given as |grad phi| n, as the paired kernel keeps it).
__device__ __forceinline__ void vd_force2(float2 phi, float2 gp0, float2 gp1, float2 gp2, float2 pp, float2 m0,
                                          float2 m1, float2 m2, float2 P00, float2 P11, float2 P22, float2 P01,
                                          float2 P02, float2 P12, float A_lin, float rho_g, float drho, float tau_g,
                                          float dtau, float gb0, float gb1, float gb2, float rho_ref, float2& F0,
                                          float2& F1, float2& F2, float2& omega, float2& aa_w) {
    const float2 rho = fma2(phi, f2(drho), f2(rho_g));
    const float2 irho = make_float2(1.f / rho.x, 1.f / rho.y);
    const float2 tau = fma2(phi, f2(dtau), f2(tau_g));
    omega = make_float2(1.f / tau.x, 1.f / tau.y);
    const float2 q0 = mul2(f2(drho), gp0), q1 = mul2(f2(drho), gp1), q2 = mul2(f2(drho), gp2);  // grad rho
    const float2 br = sub2(rho, f2(rho_ref));
    const float2 fp = mul2(pp, f2(-1.f / 3.f));
    const float2 G0 = fma2(fp, q0, fma2(br, f2(gb0), F0)), G1 = fma2(fp, q1, fma2(br, f2(gb1), F1));
    const float2 G2 = fma2(fp, q2, fma2(br, f2(gb2), F2));
    const float2 h = mul2(f2(0.5f), irho), inv = f2(1.f / (1.f - 0.5f * A_lin));
    const float2 v0 = mul2(fma2(h, G0, m0), inv), v1 = mul2(fma2(h, G1, m1), inv), v2 = mul2(fma2(h, G2, m2), inv);
    const float2 p3 = mul2(pp, f2(1.f / 3.f));
    const float2 mv0 = mul2(v0, f2(-1.f)), mv1 = mul2(v1, f2(-1.f));
    const float2 n00 = fma2(mv0, v0, sub2(P00, p3)), n11 = fma2(mv1, v1, sub2(P11, p3));
    const float2 n22 = fma2(mul2(v2, f2(-1.f)), v2, sub2(P22, p3));
    const float2 n01 = fma2(mv0, v1, P01), n02 = fma2(mv0, v2, P02), n12 = fma2(mv1, v2, P12);
    const float2 c = fma2(f2(0.5f), omega, f2(-1.f));  // -nu omega / cs^2
    F0 = mul2(fma2(c, fma2(n00, q0, fma2(n01, q1, mul2(n02, q2))), G0), irho);
    F1 = mul2(fma2(c, fma2(n01, q0, fma2(n11, q1, mul2(n12, q2))), G1), irho);
    F2 = mul2(fma2(c, fma2(n02, q0, fma2(n12, q1, mul2(n22, q2))), G2), irho);
    aa_w = mul2(mul2(f2(1.5f), fma2(f2(-0.5f), omega, f2(1.f))), omega);
}

// One pulled column of the moment-only storage: the three directions
// (cx, cy, -1), (cx, cy, 0), (cx, cy, +1) of the post-collision polynomial of
// a source site whose ten coefficients are read through ld(k), k in the order
// e0, P+x, P+y, P+z, P-x, P-y, P-z, Xxy, Xxz, Xyz.  Each value is formed by
// the same sequence of FP32 additions as in quad_poly27, so it equals, bit for
// bit, the population the AA storage would have stored and reloaded.
template <int CX, int CY, class LD>
__device__ __forceinline__ void pull_column(LD ld, float& vm, float& v0, float& vp) {
    const float e0 = ld(0);
    const float Pp2 = ld(3), Pm2 = ld(6);
    if (CX == 0 && CY == 0) {
        v0 = e0;
        vp = e0 + Pp2;
        vm = e0 + Pm2;
    } else if (CY == 0) {  // x face: fx = e0 + P(cx)_x; z term cx*cz*Xxz
        const float fx = e0 + (CX > 0 ? ld(1) : ld(4));
        const float X = ld(8);
        v0 = fx;
        vp = fx + (CX > 0 ? Pp2 + X : Pp2 - X);
        vm = fx + (CX > 0 ? Pm2 - X : Pm2 + X);
    } else if (CX == 0) {  // y face: fy = e0 + P(cy)_y; z term cy*cz*Xyz
        const float fy = e0 + (CY > 0 ? ld(2) : ld(5));
        const float X = ld(9);
        v0 = fy;
        vp = fy + (CY > 0 ? Pp2 + X : Pp2 - X);
        vm = fy + (CY > 0 ? Pm2 - X : Pm2 + X);
    } else {  // xy edge e = fx + (P(cy)_y +- Xxy); corners add cz (cx Xxz + cy Xyz)
        const float fx = e0 + (CX > 0 ? ld(1) : ld(4));
        const float Xxy = ld(7), Xxz = ld(8), Xyz = ld(9);
        const float Py = CY > 0 ? ld(2) : ld(5);
        const float e = fx + (CX * CY > 0 ? Py + Xxy : Py - Xxy);
        const float V = CX == CY ? Xxz + Xyz : Xxz - Xyz;  // Vpp or Vpm of quad_poly27
        v0 = e;
        vp = e + (CX > 0 ? Pp2 + V : Pp2 - V);
        vm = e + (CX > 0 ? Pm2 - V : Pm2 + V);
    }
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
// One box: a block per (32 x TY tile, z-chunk).
// MC selects the moment-only storage: f is not stored; each site keeps the
// ten coefficients of its post-collision polynomial and the next step pulls
// f_i(x) = w_i (1 + v_i(x - c_i)) from the neighbours' coefficients.  With MC,
// PAR = 0 evaluates the site's own coefficients (t = 0, where lb_init stored
// those of f^eq) and PAR = 1 pulls; FT is float.
// VD adds the density and viscosity contrasts of Sec. 2.3 (see vd_force).
// PF: the phase field is a stored field (one plane, gin[0]) advanced by the
// finite-difference step of lbgb_weno.cu; this kernel then reads phi from it
// and writes u (gout[0..2]) instead of the D3Q7 update (INIT: copies phi).
// PAIR: the paired kernel of the 16-bit AA step (64 x TY tiles, 32 TY threads,
// two sites each; nx a multiple of 4).  Blocks per SM that fit in registers
// and shared memory: three of TY = 4 (168 registers, none spilled), two of
// TY = 8.
// G16: the D3Q7 populations in the 16-bit storage type as well (see the tile
// body), for the AA storages FT = __half or __nv_bfloat16, nx a multiple of 4.
template <class FT, int TY, int MODE, int PAR, bool VEC, bool MC = false, bool VD = false, bool PF = false,
          bool PAIR = false, bool G16 = false>
__global__ void __launch_bounds__(32 * TY, PAIR ? (TY == 4 ? 3 : 2) : (TY >= 16 ? 1 : 512 / (32 * TY)))
fused_step_kernel(const StepArgs a) {
    constexpr int PTX = 64;
#define TILE_BX blockIdx.x
#define TILE_BY blockIdx.y
#define TILE_BZ blockIdx.z
#define TILE_PBLOCK (((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x)
#include "lbgb_tile_body.inc"
#undef TILE_BX
#undef TILE_BY
#undef TILE_BZ
#undef TILE_PBLOCK
}

// ------------------------------------------------------ batched ensemble
// Many independent periodic boxes in one array set: box b's f planes start at
// element f_off and are N_b apart; its g planes likewise at g_off in each of
// the two g buffers.  The work list enumerates (box, tile, z-chunk) items;
// a persistent grid takes them from a queue.
struct BoxDesc {
    int nx, ny, nz, N;
    long long f_off, g_off;                 // element offsets into the batch arrays
    long long c_off;                        // moment-only storage: offset of the box's 10 planes in a buffer
    float omega, omega_phi, sharp, beta;
    int item0, tiles_x, tiles_y, tiles_z;   // this box's slice of the work list
    float rho_g, drho, tau_g, dtau;         // density and viscosity contrasts (kernels with VD)
};

struct BatchArgs {
    int nitems, zc;
    const BoxDesc* boxes;
    const int* item_box;   // box of each work item
    void* f;               // all boxes' populations (storage type)
    const float* g_in;
    float* g_out;
    const float* c_in;     // moment-only storage: coefficient buffers at t and t+1
    float* c_out;
    double* partials;      // NPART per work item
    int* next;             // work queue: the next item to take (zero at the step's start)
};

// Plane q of a plane set stored q * stride elements apart.
template <class T>
struct PlaneSet {
    T* base;
    long long stride;
    __device__ __forceinline__ T* operator[](int q) const { return base + q * stride; }
};

// The argument view of one box for the tile body (steps only, no external force).
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
    PlaneSet<const float> cin;  // moment-only storage
    PlaneSet<float> cout;
    float rho_g, drho, tau_g, dtau;  // density and viscosity contrasts (VD); no buoyancy in a batch
    float gb0, gb1, gb2, rho_ref;
    const void* gphi_in;             // 16-bit D3Q7 storage: not in a batch (null)
    void* gphi_out;
};

// Persistent kernel: the grid strides over the work list of all boxes.  With
// MC_ (moment-only storage, FT float) PAR = 0 evaluates each site's own
// coefficients (the step from t = 0) and PAR = 1 pulls.  VD_: every box with
// its own density and viscosity contrasts (Sec. 2.3).  PAIR_: the paired
// tile body of the 16-bit storages (tiles PW_ = 64 or 32 sites wide, two sites
// per thread, PW_/2 * TY threads).
template <int PW, int TY>
constexpr int pair_threads() { return PW / 2 * TY; }
template <class FT, int TY, int PAR, bool VEC, bool MC_ = false, bool VD_ = false, bool PAIR_ = false, int PW_ = 64>
__global__ void __launch_bounds__(PAIR_ ? pair_threads<PW_, TY>() : 32 * TY,
                                  PAIR_ ? (pair_threads<PW_, TY>() == 64 ? 6 : pair_threads<PW_, TY>() == 128 ? 3 : 2)
                                        : (TY >= 16 ? 1 : 512 / (32 * TY)))
batch_step_kernel(const __grid_constant__ BatchArgs b) {
    __shared__ int s_item;
    for (;;) {
        // each block takes the next item of the queue (items of unequal cost:
        // boxes and z-chunks of different heights)
        if (threadIdx.x == 0) s_item = atomicAdd(b.next, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= b.nitems) break;
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
        t.cin = PlaneSet<const float>{MC_ ? b.c_in + d.c_off : nullptr, (long long)d.N};
        t.cout = PlaneSet<float>{MC_ ? b.c_out + d.c_off : nullptr, (long long)d.N};
        t.rho_g = d.rho_g; t.drho = d.drho; t.tau_g = d.tau_g; t.dtau = d.dtau;
        t.gb0 = t.gb1 = t.gb2 = t.rho_ref = 0.f;
        t.gphi_in = nullptr;
        t.gphi_out = nullptr;
        const int local = item - d.item0;
        const int tbx = local % d.tiles_x, rest = local / d.tiles_x;
        const int tby = rest % d.tiles_y, tbz = rest / d.tiles_y;
        {
            const BoxTileArgs<FT>& a = t;
            constexpr int MODE = MODE_STEP;
            constexpr bool MC = MC_;
            constexpr bool VD = VD_;
            constexpr bool PF = false;
            constexpr bool PAIR = PAIR_;
            constexpr bool G16 = false;
            constexpr int PTX = PW_;
#define TILE_BX tbx
#define TILE_BY tby
#define TILE_BZ tbz
#define TILE_PBLOCK ((long long)item)
#include "lbgb_tile_body.inc"
#undef TILE_BX
#undef TILE_BY
#undef TILE_BZ
#undef TILE_PBLOCK
        }
        __syncthreads();  // the shared rings are reused by the block's next item
    }
}

// Launch one fused kernel instance.  Defined per storage type in lbgb_step_*.cu.
// Records a message for lb_last_error() (defined with the C ABI).
void set_last_error(const char* msg);

// Resident blocks per SM of the single-box STEP kernel (0 if unknown).
template <class FT>
int fused_blocks_per_sm(int ty, bool vec);
int fused_mc_blocks_per_sm(int ty, bool vec);

// One launch of the moment-only storage kernel: mode INIT, MOMENTS or STEP;
// pull = 0 evaluates each site's own coefficients (the state lb_init leaves),
// pull = 1 rebuilds f from the neighbours' coefficients.
cudaError_t launch_fused_mc(int mode, int pull, int ty, bool vec, dim3 grid, const StepArgs& a, cudaStream_t st);
cudaError_t launch_batch_mc(int pull, int ty, bool vec, int blocks, const BatchArgs& b, cudaStream_t st);
int batch_mc_blocks_per_sm(int ty, bool vec);

// One step of every box of a batch (persistent grid of `blocks` blocks).
template <class FT>
cudaError_t launch_batch(int parity, int ty, bool vec, int blocks, const BatchArgs& b, cudaStream_t st);
// Resident blocks per SM of the batch kernel for this shape (0 on error).
template <class FT>
int batch_blocks_per_sm(int ty, bool vec);

// vec selects the float4 phase-A loads (requires nx % 4 == 0).
template <class FT>
cudaError_t launch_fused(int mode, int parity, int ty, bool vec, dim3 grid, const StepArgs& a, cudaStream_t st);

// The paired step kernel of a 16-bit storage (__half or __nv_bfloat16): tiles
// of 64 x ty sites, ty in {4, 8} (32 ty threads per block), nx % 4 == 0,
// MODE_STEP.
// Defined in lbgb_step_pair_*.cu.
template <class FT>
cudaError_t launch_fused_pair(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st);
template <class FT>
int fused_pair_blocks_per_sm(int ty);
// The same with the finite-difference phase field (PF); lbgb_step_pair_pf_*.cu.
template <class FT>
cudaError_t launch_fused_pair_pf(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st);
template <class FT>
int fused_pair_pf_blocks_per_sm(int ty);
// The same with density and viscosity contrasts (VD); lbgb_step_pair_vd_*.cu.
template <class FT>
cudaError_t launch_fused_pair_vd(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st);
template <class FT>
int fused_pair_vd_blocks_per_sm(int ty);
// The kernels of the 16-bit D3Q7 storage (G16; FT __half or __nv_bfloat16,
// nx % 4 == 0): one-site kernels for MODE_INIT (ty 8), MODE_MOMENTS (ty 8) and
// MODE_STEP (ty 4 or 8), defined in lbgb_step_g16_*.cu; the paired step kernel
// (64 x ty tiles, ty 4 or 8), defined in lbgb_step_pair_g16_*.cu.
template <class FT>
cudaError_t launch_fused_g16(int mode, int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st);
template <class FT>
int fused_g16_blocks_per_sm(int ty);
template <class FT>
cudaError_t launch_fused_pair_g16(int parity, int ty, dim3 grid, const StepArgs& a, cudaStream_t st);
template <class FT>
int fused_pair_g16_blocks_per_sm(int ty);
// The batch kernel with the paired tile body (16-bit storages; every box nx % 4 == 0),
// tiles pw = 64 or 32 sites wide and ty = 4 or 8 rows (pw/2 * ty threads).
template <class FT>
cudaError_t launch_batch_pair(int parity, int ty, int pw, int blocks, const BatchArgs& b, cudaStream_t st);
template <class FT>
int batch_pair_blocks_per_sm(int ty, int pw);

// The batch kernel with density and viscosity contrasts (every box its own),
// for the AA storage FT (MC = false) or the moment-only storage (FT float,
// MC = true, parity = pull).  Defined in lbgb_step_vd_*.cu.
template <class FT, bool MC>
cudaError_t launch_batch_vd(int parity, int ty, bool vec, int blocks, const BatchArgs& b, cudaStream_t st);
template <class FT, bool MC>
int batch_vd_blocks_per_sm(int ty, bool vec);

// The same kernels with the density and viscosity contrasts (VD) and/or the
// phase field as a stored field (PF), mode STEP or MOMENTS (and INIT for PF
// without VD), for the AA storage FT (MC = false) or the moment-only storage
// (FT float, MC = true, parity = pull).  Defined in lbgb_step_{vd,fd,fdvd}_*.cu.
template <class FT, bool MC, bool VD, bool PF>
cudaError_t launch_fused_x(int mode, int parity, int ty, bool vec, dim3 grid, const StepArgs& a, cudaStream_t st);
template <class FT, bool MC, bool VD, bool PF>
int fused_x_blocks_per_sm(int ty, bool vec);

// One stage (0, 1, 2) of the finite-difference phase step (lbgb_weno.cu):
// reads pin (with halo), phin (own site), u (3 planes of N) and writes out.
cudaError_t launch_weno_stage(int stage, const float* pin, const float* phin, const float* u, float* out, int nx,
                              int ny, int nz, float D, float kap, cudaStream_t st);

}  // namespace lbgb
