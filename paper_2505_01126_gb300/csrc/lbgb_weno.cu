// lbgb_weno.cu -- the finite-difference phase-field step (Sec. 2.1.1, Eq. 4
// with WENO-5 advection; Sec. 2.3 lattice stencils): one launch per stage of
// the three-stage strong-stability-preserving Runge-Kutta scheme,
//   stage 0: out = p + L(p)                    (p = phi_n)
//   stage 1: out = 3/4 phi_n + 1/4 (p + L(p))  (p = stage-0 result)
//   stage 2: out = 1/3 phi_n + 2/3 (p + L(p))  (p = stage-1 result; out may be phi_n),
//            formed as phi_n + 2/3 (p + L(p) - phi_n)
// with
//   L(p) = -div(p u) + D lap(p) - kappa div(J),  J = max(p (1 - p), 0) n(p),
// D = M, kappa = 4M/W, u the velocity the fused step wrote for this step.
//   - div(p u): face fluxes u_f p_f, u_f the mean of the two sites' normal
//     velocity and p_f the WENO-5 value (Jiang and Shu 1996) from the five
//     values upwind of the face;
//   - lap(p) = (2/cs^2) sum_i w_i (p(x + c_i) - p(x));
//   - grad and div with (1/cs^2) sum_i w_i c_i Psi(x + c_i), in the separable
//     form (1/72) sum over the transverse 3x3 with weights (1, 4, 1)^2 of the
//     difference along the axis;
//   - n = grad p / max(|grad p|, 1e-10).
// A block takes a 32 x 4 x 4 tile: p on the tile with a halo of 3 (the WENO
// reach; 2 would do for the stencils) in shared memory, J on the halo-1 ring,
// then each thread forms L at two sites.  Every read of a stage is of the
// previous stage's array or of phi_n at the thread's own site, so stage 2 may
// write phi_n in place.
#include "lbgb_kernels.cuh"

namespace lbgb {

namespace {

constexpr int WX = 32, WY = 4, WZ = 4, WH = 3;
constexpr int SX = WX + 2 * WH, SY = WY + 2 * WH, SZ = WZ + 2 * WH;  // 38 x 10 x 10
constexpr int JX = WX + 2, JY = WY + 2, JZ = WZ + 2;                 // 34 x 6 x 6
constexpr int WNT = 256;                                             // threads per block

__device__ __forceinline__ float weno5(float vm2, float vm1, float v0, float v1, float v2) {
    const float q0 = (2.f * vm2 - 7.f * vm1 + 11.f * v0) * (1.f / 6.f);
    const float q1 = (-vm1 + 5.f * v0 + 2.f * v1) * (1.f / 6.f);
    const float q2 = (2.f * v0 + 5.f * v1 - v2) * (1.f / 6.f);
    const float d0 = vm2 - 2.f * vm1 + v0, e0 = vm2 - 4.f * vm1 + 3.f * v0;
    const float d1 = vm1 - 2.f * v0 + v1, e1 = vm1 - v1;
    const float d2 = v0 - 2.f * v1 + v2, e2 = 3.f * v0 - 4.f * v1 + v2;
    const float b0 = (13.f / 12.f) * d0 * d0 + 0.25f * e0 * e0;
    const float b1 = (13.f / 12.f) * d1 * d1 + 0.25f * e1 * e1;
    const float b2 = (13.f / 12.f) * d2 * d2 + 0.25f * e2 * e2;
    // weights d_k / (eps + b_k)^2, normalised; multiplied through by the
    // product of the three denominators so that one division remains (each
    // (eps + b)^2 lies in [1e-12, ~1e3], so the products stay normal in FP32)
    constexpr float eps = 1e-6f;
    const float t0 = (eps + b0) * (eps + b0), t1 = (eps + b1) * (eps + b1), t2 = (eps + b2) * (eps + b2);
    const float a0 = 0.1f * (t1 * t2), a1 = 0.6f * (t0 * t2), a2 = 0.3f * (t0 * t1);
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Periodic wrap of v in [-n, 2n).
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Flux u_f p_f through the face between p[2] and p[3] of the six values
// p[0..5] along an axis, u_f = (ul + ur)/2.
__device__ __forceinline__ float face_flux(const float (&p)[6], float ul, float ur) {
    const float uf = 0.5f * (ul + ur);
    const float pf = uf >= 0.f ? weno5(p[0], p[1], p[2], p[3], p[4]) : weno5(p[5], p[4], p[3], p[2], p[1]);
    return uf * pf;
}

__global__ void __launch_bounds__(WNT) weno_stage_kernel(const float* __restrict__ pin, const float* phin,
                                                         const float* __restrict__ ux, const float* __restrict__ uy,
                                                         const float* __restrict__ uz, float* out, int nx, int ny,
                                                         int nz, float D, float kap, int stage) {
    __shared__ float s_p[SZ][SY][SX];
    __shared__ float s_J[3][JZ][JY][JX];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * WX, y0 = blockIdx.y * WY, z0 = blockIdx.z * WZ;
    const long long plane = (long long)nx * ny;

    // the tile and its halo span [x0 - WH, x0 + WX + WH - 1] with x0 < nx, within
    // [-n, 2n) unless the box is shorter than the tile plus its halo
    const bool small = nx < WX + WH || ny < WY + WH || nz < WZ + WH;
    for (int i = tid; i < SX * SY * SZ; i += WNT) {
        const int lx = i % SX, ly = (i / SX) % SY, lz = i / (SX * SY);
        int gx, gy, gz;
        if (small) {
            gx = wrap_mod(x0 - WH + lx, nx); gy = wrap_mod(y0 - WH + ly, ny); gz = wrap_mod(z0 - WH + lz, nz);
        } else {
            gx = wrap1(x0 - WH + lx, nx); gy = wrap1(y0 - WH + ly, ny); gz = wrap1(z0 - WH + lz, nz);
        }
        s_p[lz][ly][lx] = __ldg(pin + gz * plane + (long long)gy * nx + gx);
    }
    __syncthreads();

    // J on the halo-1 ring: site (jx, jy, jz) is s_p[jz + 2][jy + 2][jx + 2]
    for (int i = tid; i < JX * JY * JZ; i += WNT) {
        const int jx = i % JX, jy = (i / JX) % JY, jz = i / (JX * JY);
        const int cx = jx + 2, cy = jy + 2, cz = jz + 2;
        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int b = -1; b <= 1; ++b)
#pragma unroll
            for (int c = -1; c <= 1; ++c) {
                const float wbc = (b == 0 ? 4.f : 1.f) * (c == 0 ? 4.f : 1.f);
                gx = fmaf(wbc, s_p[cz + c][cy + b][cx + 1] - s_p[cz + c][cy + b][cx - 1], gx);
                gy = fmaf(wbc, s_p[cz + c][cy + 1][cx + b] - s_p[cz + c][cy - 1][cx + b], gy);
                gz = fmaf(wbc, s_p[cz + 1][cy + c][cx + b] - s_p[cz - 1][cy + c][cx + b], gz);
            }
        gx *= 1.f / 72.f;
        gy *= 1.f / 72.f;
        gz *= 1.f / 72.f;
        const float m = sqrtf(gx * gx + gy * gy + gz * gz);
        const float p = s_p[cz][cy][cx];
        const float w = fmaxf(p * (1.f - p), 0.f) / fmaxf(m, 1e-10f);
        s_J[0][jz][jy][jx] = w * gx;
        s_J[1][jz][jy][jx] = w * gy;
        s_J[2][jz][jy][jx] = w * gz;
    }
    __syncthreads();

    for (int i = tid; i < WX * WY * WZ; i += WNT) {
        const int tx = i % WX, ty = (i / WX) % WY, tz = i / (WX * WY);
        const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        const int cx = tx + WH, cy = ty + WH, cz = tz + WH;
        const int jx = tx + 1, jy = ty + 1, jz = tz + 1;
        const float p0 = s_p[cz][cy][cx];

        // lap(p) and div(J), the 26 neighbours with weights (1, 4, 1)^3 / 216
        float lap = 0.f, dj = 0.f;
#pragma unroll
        for (int c = -1; c <= 1; ++c)
#pragma unroll
            for (int b = -1; b <= 1; ++b) {
                const float wbc = (b == 0 ? 4.f : 1.f) * (c == 0 ? 4.f : 1.f);
#pragma unroll
                for (int a = -1; a <= 1; ++a) {
                    if (a == 0 && b == 0 && c == 0) continue;
                    const float wabc = wbc * (a == 0 ? 4.f : 1.f);
                    lap = fmaf(wabc, s_p[cz + c][cy + b][cx + a] - p0, lap);
                }
                dj = fmaf(wbc, s_J[0][jz + c][jy + b][jx + 1] - s_J[0][jz + c][jy + b][jx - 1], dj);
                dj = fmaf(wbc, s_J[1][jz + c][jy + 1][jx + b] - s_J[1][jz + c][jy - 1][jx + b], dj);
                dj = fmaf(wbc, s_J[2][jz + 1][jy + c][jx + b] - s_J[2][jz - 1][jy + c][jx + b], dj);
            }
        lap *= 1.f / 36.f;  // (2/cs^2) / 216
        dj *= 1.f / 72.f;

        // advective flux differences
        const long long s = gz * plane + (long long)gy * nx + gx;
        const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
        const int ym = gy == 0 ? ny - 1 : gy - 1, yp = gy == ny - 1 ? 0 : gy + 1;
        const int zm = gz == 0 ? nz - 1 : gz - 1, zp = gz == nz - 1 ? 0 : gz + 1;
        const long long row = gz * plane + (long long)gy * nx;
        const float u0 = __ldg(ux + s), uxm = __ldg(ux + row + xm), uxp = __ldg(ux + row + xp);
        const float v0 = __ldg(uy + s), uym = __ldg(uy + gz * plane + (long long)ym * nx + gx);
        const float uyp = __ldg(uy + gz * plane + (long long)yp * nx + gx);
        const float w0 = __ldg(uz + s), uzm = __ldg(uz + zm * plane + (long long)gy * nx + gx);
        const float uzp = __ldg(uz + zp * plane + (long long)gy * nx + gx);
        float adv = 0.f;
        {
            float pl[6], pr[6];  // the six values around face x-1/2 and around x+1/2
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                pl[j] = s_p[cz][cy][cx - 3 + j];
                pr[j] = s_p[cz][cy][cx - 2 + j];
            }
            adv += face_flux(pr, u0, uxp) - face_flux(pl, uxm, u0);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                pl[j] = s_p[cz][cy - 3 + j][cx];
                pr[j] = s_p[cz][cy - 2 + j][cx];
            }
            adv += face_flux(pr, v0, uyp) - face_flux(pl, uym, v0);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                pl[j] = s_p[cz - 3 + j][cy][cx];
                pr[j] = s_p[cz - 2 + j][cy][cx];
            }
            adv += face_flux(pr, w0, uzp) - face_flux(pl, uzm, w0);
        }
        const float L = fmaf(D, lap, -fmaf(kap, dj, adv));
        const float q = p0 + L;
        float r;
        // weights that sum to exactly 1 in FP32, so that a uniform field stays
        // uniform bit for bit (1/3 + 2/3 rounded separately would not)
        if (stage == 0) r = q;
        else if (stage == 1) r = fmaf(0.75f, phin[s], 0.25f * q);
        else {
            const float pn = phin[s];
            r = fmaf(2.f / 3.f, q - pn, pn);
        }
        out[s] = r;
    }
}

}  // namespace

cudaError_t launch_weno_stage(int stage, const float* pin, const float* phin, const float* u, float* out, int nx,
                              int ny, int nz, float D, float kap, cudaStream_t st) {
    const long long N = (long long)nx * ny * nz;
    const dim3 grid((unsigned)((nx + WX - 1) / WX), (unsigned)((ny + WY - 1) / WY), (unsigned)((nz + WZ - 1) / WZ));
    weno_stage_kernel<<<grid, WNT, 0, st>>>(pin, phin, u, u + N, u + 2 * N, out, nx, ny, nz, D, kap, stage);
    return cudaGetLastError();
}

}  // namespace lbgb
