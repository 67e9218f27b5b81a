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
// A block takes a 32 x 8 x 8 tile: p on the tile with a halo of 3 (the WENO
// reach; 2 would do for the stencils) in shared memory, J on the halo-1 ring,
// D lap - kappa div J in registers, then every face flux of the tile once (in
// the space of J), then L and the stage combination at eight sites per
// thread.  Every read of a stage is of the previous stage's array or of phi_n
// at the thread's own site, so stage 2 may write phi_n in place.
#include "lbgb_kernels.cuh"

namespace lbgb {

namespace {

constexpr int WX = 32, WY = 8, WZ = 8, WH = 3;
constexpr int SX = WX + 2 * WH, SY = WY + 2 * WH, SZ = WZ + 2 * WH;  // 38 x 14 x 14
constexpr int JX = WX + 2, JY = WY + 2, JZ = WZ + 2;                 // 34 x 10 x 10
constexpr int WNT = 256;                                             // threads per block
constexpr int SPT = WX * WY * WZ / WNT;                              // sites per thread
// face fluxes, stored after div(J) is formed, in the space of J
constexpr int NFX = WZ * WY * (WX + 1), NFY = WZ * (WY + 1) * WX, NFZ = (WZ + 1) * WY * WX;
static_assert(NFX + NFY + NFZ <= 3 * JX * JY * JZ, "fluxes fit in the space of J");

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
    // (eps + b)^2 lies in [1e-12, ~1e3], so the products stay normal in FP32,
    // as the fast division needs)
    constexpr float eps = 1e-6f;
    const float t0 = (eps + b0) * (eps + b0), t1 = (eps + b1) * (eps + b1), t2 = (eps + b2) * (eps + b2);
    const float a0 = 0.1f * (t1 * t2), a1 = 0.6f * (t0 * t2), a2 = 0.3f * (t0 * t1);
    return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

// Periodic wrap of v in [-n, 2n).
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__global__ void __launch_bounds__(WNT) weno_stage_kernel(const float* __restrict__ pin, const float* phin,
                                                         const float* __restrict__ ux, const float* __restrict__ uy,
                                                         const float* __restrict__ uz, float* out, int nx, int ny,
                                                         int nz, float D, float kap, int stage) {
    __shared__ float s_p[SZ][SY][SX];
    __shared__ float s_J[3][JZ][JY][JX];
    float* s_F = &s_J[0][0][0][0];  // Fx, Fy, Fz after div(J)
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * WX, y0 = blockIdx.y * WY, z0 = blockIdx.z * WZ;
    const long long plane = (long long)nx * ny;
    // the tile and its halo span [x0 - WH, x0 + WX + WH - 1] with x0 < nx, within
    // [-n, 2n) unless the box is shorter than the tile plus its halo
    const bool small = nx < WX + WH || ny < WY + WH || nz < WZ + WH;
    auto wx = [&](int v) { return small ? wrap_mod(v, nx) : wrap1(v, nx); };
    auto wy = [&](int v) { return small ? wrap_mod(v, ny) : wrap1(v, ny); };
    auto wz = [&](int v) { return small ? wrap_mod(v, nz) : wrap1(v, nz); };

    // a warp per halo row; a lane loads the columns lane and lane + 32 (< SX)
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = WNT / 32;
    const int gxa = wx(x0 - WH + lane), gxb = lane + 32 < SX ? wx(x0 - WH + lane + 32) : 0;
    for (int r = warp; r < SY * SZ; r += NW) {
        const int ly = r % SY, lz = r / SY;
        const float* row = pin + wz(z0 - WH + lz) * plane + (long long)wy(y0 - WH + ly) * nx;
        s_p[lz][ly][lane] = __ldg(row + gxa);
        if (lane + 32 < SX) s_p[lz][ly][lane + 32] = __ldg(row + gxb);
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
        const float w = __fdividef(fmaxf(p * (1.f - p), 0.f), fmaxf(m, 1e-10f));
        s_J[0][jz][jy][jx] = w * gx;
        s_J[1][jz][jy][jx] = w * gy;
        s_J[2][jz][jy][jx] = w * gz;
    }
    __syncthreads();

    // D lap(p) - kappa div(J) at this thread's sites (site i = tid + k WNT)
    float Ld[SPT];
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
        const int i = tid + k * WNT;
        const int tx = i % WX, ty = (i / WX) % WY, tz = i / (WX * WY);
        const int cx = tx + WH, cy = ty + WH, cz = tz + WH;
        const int jx = tx + 1, jy = ty + 1, jz = tz + 1;
        const float p0 = s_p[cz][cy][cx];
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
        // (2/cs^2) / 216 for lap, 1/72 for the divergence
        Ld[k] = fmaf(D * (1.f / 36.f), lap, -kap * (1.f / 72.f) * dj);
    }
    __syncthreads();  // J is read; its space takes the face fluxes

    // advective flux u_f p_f of every face of the tile, once: face f along an
    // axis lies between local sites f - 1 and f.  A warp takes a row of faces
    // (lane = the face's x, or its index along x for the x faces).
    auto flux = [](const float (&v)[6], float ul, float ur) {
        const float uf = 0.5f * (ul + ur);
        // the five values upwind of the face, selected without a branch (a warp
        // holds both signs of u in a flow)
        const bool up = uf >= 0.f;
        return uf * weno5(up ? v[0] : v[5], up ? v[1] : v[4], up ? v[2] : v[3], up ? v[3] : v[2], up ? v[4] : v[1]);
    };
    const int gxl = wx(x0 + lane), gxm = wx(x0 + lane - 1);  // this lane's site and its left neighbour
    {
        float* Fx = s_F;
        for (int r = warp; r < WY * WZ; r += NW) {  // x faces: rows (y, z), faces f = lane and 32
            const int ly = r % WY, lz = r / WY;
            const float* urow = ux + wz(z0 + lz) * plane + (long long)wy(y0 + ly) * nx;
            float v[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) v[j] = s_p[lz + WH][ly + WH][lane + j];
            Fx[(lz * WY + ly) * (WX + 1) + lane] = flux(v, __ldg(urow + gxm), __ldg(urow + gxl));
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) v[j] = s_p[lz + WH][ly + WH][WX + j];
                Fx[(lz * WY + ly) * (WX + 1) + WX] = flux(v, __ldg(urow + wx(x0 + WX - 1)), __ldg(urow + wx(x0 + WX)));
            }
        }
        float* Fy = s_F + NFX;
        for (int r = warp; r < (WY + 1) * WZ; r += NW) {  // y faces: rows (f, z), lane = x
            const int f = r % (WY + 1), lz = r / (WY + 1);
            const long long zb = wz(z0 + lz) * plane;
            float v[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) v[j] = s_p[lz + WH][f + j][lane + WH];
            const float ul = __ldg(uy + zb + (long long)wy(y0 + f - 1) * nx + gxl);
            const float ur = __ldg(uy + zb + (long long)wy(y0 + f) * nx + gxl);
            Fy[(lz * (WY + 1) + f) * WX + lane] = flux(v, ul, ur);
        }
        float* Fz = s_F + NFX + NFY;
        for (int r = warp; r < (WZ + 1) * WY; r += NW) {  // z faces: rows (y, f), lane = x
            const int ly = r % WY, f = r / WY;
            const long long yb = (long long)wy(y0 + ly) * nx + gxl;
            float v[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) v[j] = s_p[f + j][ly + WH][lane + WH];
            const float ul = __ldg(uz + wz(z0 + f - 1) * plane + yb);
            const float ur = __ldg(uz + wz(z0 + f) * plane + yb);
            Fz[(f * WY + ly) * WX + lane] = flux(v, ul, ur);
        }
    }
    __syncthreads();

#pragma unroll
    for (int k = 0; k < SPT; ++k) {
        const int i = tid + k * WNT;
        const int tx = i % WX, ty = (i / WX) % WY, tz = i / (WX * WY);
        const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        const float* Fx = s_F;
        const float* Fy = s_F + NFX;
        const float* Fz = s_F + NFX + NFY;
        const int ix = (tz * WY + ty) * (WX + 1) + tx;
        const int iy = (tz * (WY + 1) + ty) * WX + tx;
        const int iz = (tz * WY + ty) * WX + tx;
        const float adv = (Fx[ix + 1] - Fx[ix]) + (Fy[iy + WX] - Fy[iy]) + (Fz[iz + WX * WY] - Fz[iz]);
        const float q = s_p[tz + WH][ty + WH][tx + WH] + (Ld[k] - adv);
        const long long s = gz * plane + (long long)gy * nx + gx;
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
