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
// Every read of a stage is of the previous stage's array or of phi_n at the
// thread's own site, so stage 2 may write phi_n in place.
#include "lbgb_kernels.cuh"

namespace lbgb {

namespace {

// A block takes a 32 x 8 column tile and marches over a z-chunk: phi planes
// (with a halo of 3 in x and y) in a ring of 8.  The lattice stencils are
// separable, so each plane's in-plane parts are formed once and combined
// across planes:
//   - on the halo-1 ring of the tile, per plane: Gx2 = sum_b w_b dx phi,
//     Gy2 = sum_a w_a dy phi (central differences, weights (1, 4, 1) across)
//     and S2 = sum_ab w_a w_b (phi - phi_c), phi_c the site's own value, in a
//     ring of five planes in shared memory; then
//       grad_x = (1/72) sum_c w_c Gx2(z + c),  likewise y,
//       grad_z = (1/72) (S2(z+1) - S2(z-1) + 36 (phi_c(z+1) - phi_c(z-1))),
//       lap    = sum_c w_c (S2(z + c) + 36 (phi_c(z + c) - phi_c(z))),
//     every term a difference, so that nearly uniform phi keeps its FP32
//     accuracy;
//   - J = max(phi (1 - phi), 0) n on the halo-1 plane (one plane at a time),
//     and for the thread's own site the in-plane parts of div J:
//     A(z) = sum_b w_b dx J_x + sum_a w_a dy J_y and B(z) = sum_ab w_a w_b J_z,
//     carried in registers: div J = sum_c w_c A(z + c) + B(z + 1) - B(z - 1).
// Per plane z: J of plane z + 1; barrier; the x- and y-face fluxes of plane z,
// each once, spread over the block (264 + 288 faces), the partials of plane
// z + 3, A and B of plane z + 1, D lap - kappa div J and the flux through the
// column's upper z face (the lower one carried from the plane below);
// barrier; the stage combination, then the asynchronous copy of plane z + 4.
constexpr int TX = 32, TY = 8, WH = 3;
constexpr int PX = TX + 2 * WH, PY = TY + 2 * WH, NP = PX * PY;  // 38 x 14
constexpr int QX = TX + 2, QY = TY + 2, NQ = QX * QY;            // 34 x 10
constexpr int WNT = TX * TY;                                       // 256 threads
constexpr int NPL = (NP + WNT - 1) / WNT;                          // phi elements per thread
constexpr int NJL = (NQ + WNT - 1) / WNT;                          // halo-1 sites per thread
constexpr int NFX = TY * (TX + 1), NFY = (TY + 1) * TX;            // faces per plane
constexpr int NFL = (NFY + WNT - 1) / WNT;                         // faces per thread (>= x's)
constexpr int PR = 8, GR = 5;                                      // phi ring, partials ring
static_assert(NFX <= NFL * WNT, "x faces fit the per-thread face slots");

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

// Flux u_f p_f through the face between v[2] and v[3] of six values along an
// axis, u_f = (ul + ur)/2; the five values upwind of the face are selected
// without a branch (a warp holds both signs of u in a flow).
__device__ __forceinline__ float face_flux(const float (&v)[6], float ul, float ur) {
    const float uf = 0.5f * (ul + ur);
    const bool up = uf >= 0.f;
    return uf * weno5(up ? v[0] : v[5], up ? v[1] : v[4], up ? v[2] : v[3], up ? v[3] : v[2], up ? v[4] : v[1]);
}

__device__ __forceinline__ int g5(int p) { return (p + 10) % GR; }  // partials ring slot, planes p >= -10

__global__ void __launch_bounds__(WNT, 4) weno_stage_kernel(const float* __restrict__ pin, const float* phin,
                                                         const float* __restrict__ ux, const float* __restrict__ uy,
                                                         const float* __restrict__ uz, float* out, int nx, int ny,
                                                         int nz, int zc, float D, float kap, int stage) {
    __shared__ float s_p[PR][PY][PX];
    __shared__ float s_G[GR][3][NQ];  // Gx2, Gy2, S2 of a plane on the halo-1 ring
    __shared__ float s_J[3][QY][QX];  // J of one plane on the halo-1 ring
    __shared__ float s_Fx[TY][TX + 1];
    __shared__ float s_Fy[TY + 1][TX];
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int z1 = min(z0 + zc, nz);
    const long long plane = (long long)nx * ny;

    // fixed in-plane offsets: this thread's phi-plane elements, faces (left and
    // right site of each) and its own column
    int p_off[NPL], p_dst[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int i = tid + k * WNT;
        p_dst[k] = i < NP ? i : -1;
        const int py = i / PX, px = i - (i / PX) * PX;
        p_off[k] = i < NP ? wrap_mod(y0 - WH + py, ny) * nx + wrap_mod(x0 - WH + px, nx) : 0;
    }
    int fx_i[NFL], fx_l[NFL], fx_r[NFL], fy_i[NFL], fy_l[NFL], fy_r[NFL];
#pragma unroll
    for (int k = 0; k < NFL; ++k) {
        const int i = tid + k * WNT;
        fx_i[k] = i < NFX ? i : -1;  // x face f of row r: between x0 + f - 1 and x0 + f
        const int r = i / (TX + 1), f = i - (i / (TX + 1)) * (TX + 1);
        const int yr = wrap_mod(y0 + r, ny);
        fx_l[k] = i < NFX ? yr * nx + wrap_mod(x0 + f - 1, nx) : 0;
        fx_r[k] = i < NFX ? yr * nx + wrap_mod(x0 + f, nx) : 0;
        fy_i[k] = i < NFY ? i : -1;  // y face f of column c: between y0 + f - 1 and y0 + f
        const int fy = i / TX, c = i - (i / TX) * TX;
        const int xc = wrap_mod(x0 + c, nx);
        fy_l[k] = i < NFY ? wrap_mod(y0 + fy - 1, ny) * nx + xc : 0;
        fy_r[k] = i < NFY ? wrap_mod(y0 + fy, ny) * nx + xc : 0;
    }
    const int own = wrap_mod(y0 + ly, ny) * nx + wrap_mod(x0 + lx, nx);
    const bool active = x0 + lx < nx && y0 + ly < ny;

    // asynchronous copy of phi plane zp into its ring slot (one commit group
    // per call; the caller waits before the barrier that publishes it)
    auto load_plane = [&](int zp) {
        const float* src = pin + (long long)wrap_mod(zp, nz) * plane;
        float* dst = &s_p[zp & (PR - 1)][0][0];
#pragma unroll
        for (int k = 0; k < NPL; ++k)
            if (p_dst[k] >= 0) cp_async4(dst + p_dst[k], src + p_off[k]);
        cp_async_commit();
    };
    // in-plane partials of plane zp on the halo-1 ring (from phi plane zp)
    auto partials = [&](int zp) {
        const float(*P)[PX] = s_p[zp & (PR - 1)];
        float* G = &s_G[g5(zp)][0][0];
#pragma unroll
        for (int k = 0; k < NJL; ++k) {
            const int i = tid + k * WNT;
            if (i >= NQ) continue;
            const int qy = i / QX, qx = i - (i / QX) * QX;
            const int cy = qy + 2, cx = qx + 2;
            const float pc = P[cy][cx];
            const float mm = P[cy - 1][cx - 1], m0 = P[cy - 1][cx], mp = P[cy - 1][cx + 1];
            const float om = P[cy][cx - 1], op = P[cy][cx + 1];
            const float pm = P[cy + 1][cx - 1], p0 = P[cy + 1][cx], pp = P[cy + 1][cx + 1];
            G[i] = fmaf(4.f, op - om, (mp - mm) + (pp - pm));           // Gx2
            G[NQ + i] = fmaf(4.f, p0 - m0, (pm - mm) + (pp - mp));      // Gy2
            G[2 * NQ + i] = fmaf(4.f, (m0 - pc) + (p0 - pc) + (om - pc) + (op - pc),
                                 ((mm - pc) + (mp - pc)) + ((pm - pc) + (pp - pc)));  // S2
        }
    };
    // J of plane zp on the halo-1 ring, from the partials of planes zp - 1 .. zp + 1
    auto make_J = [&](int zp) {
        const float* Gm = &s_G[g5(zp - 1)][0][0];
        const float* G0 = &s_G[g5(zp)][0][0];
        const float* Gp = &s_G[g5(zp + 1)][0][0];
        const float(*Pm)[PX] = s_p[(zp - 1) & (PR - 1)];
        const float(*P0)[PX] = s_p[zp & (PR - 1)];
        const float(*Pp)[PX] = s_p[(zp + 1) & (PR - 1)];
#pragma unroll
        for (int k = 0; k < NJL; ++k) {
            const int i = tid + k * WNT;
            if (i >= NQ) continue;
            const int qy = i / QX, qx = i - (i / QX) * QX;
            const int cy = qy + 2, cx = qx + 2;
            const float gx = fmaf(4.f, G0[i], Gm[i] + Gp[i]) * (1.f / 72.f);
            const float gy = fmaf(4.f, G0[NQ + i], Gm[NQ + i] + Gp[NQ + i]) * (1.f / 72.f);
            const float gz = fmaf(36.f, Pp[cy][cx] - Pm[cy][cx], Gp[2 * NQ + i] - Gm[2 * NQ + i]) * (1.f / 72.f);
            const float m = sqrtf(gx * gx + gy * gy + gz * gz);
            const float p = P0[cy][cx];
            const float w = __fdividef(fmaxf(p * (1.f - p), 0.f), fmaxf(m, 1e-10f));
            s_J[0][qy][qx] = w * gx;
            s_J[1][qy][qx] = w * gy;
            s_J[2][qy][qx] = w * gz;
        }
    };
    // the in-plane parts of div J at this thread's site, from the J plane in place
    const int jy = ly + 1, jx = lx + 1;
    auto divJ_parts = [&](float& A, float& B) {
        const float(*J0)[QX] = s_J[0];
        const float(*J1)[QX] = s_J[1];
        const float(*J2)[QX] = s_J[2];
        A = fmaf(4.f, J0[jy][jx + 1] - J0[jy][jx - 1],
                 (J0[jy - 1][jx + 1] - J0[jy - 1][jx - 1]) + (J0[jy + 1][jx + 1] - J0[jy + 1][jx - 1]));
        A += fmaf(4.f, J1[jy + 1][jx] - J1[jy - 1][jx],
                  (J1[jy + 1][jx - 1] - J1[jy - 1][jx - 1]) + (J1[jy + 1][jx + 1] - J1[jy - 1][jx + 1]));
        B = fmaf(4.f, fmaf(4.f, J2[jy][jx], J2[jy][jx - 1] + J2[jy][jx + 1]),
                 (fmaf(4.f, J2[jy - 1][jx], J2[jy - 1][jx - 1] + J2[jy - 1][jx + 1]) +
                  fmaf(4.f, J2[jy + 1][jx], J2[jy + 1][jx - 1] + J2[jy + 1][jx + 1])));
    };
    // flux through the z face zf + 1/2 of this thread's column
    const int pcy = ly + WH, pcx = lx + WH;
    const int gq = (ly + 1) * QX + (lx + 1);  // own site on the halo-1 ring
    auto z_flux = [&](int zf, float ul, float ur) {
        float v[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = s_p[(zf - 2 + j) & (PR - 1)][pcy][pcx];
        return face_flux(v, ul, ur);
    };

    // prologue: phi planes z0 - 3 .. z0 + 3, partials of z0 - 2 .. z0 + 2, J and
    // the div J parts of z0 - 1 and z0, the z face below z0
    for (int zp = z0 - WH; zp <= z0 + WH; ++zp) load_plane(zp);
    cp_async_wait<0>();
    __syncthreads();
    for (int zp = z0 - 2; zp <= z0 + 2; ++zp) partials(zp);
    __syncthreads();
    float Am, Bm, A0, B0;  // div J parts of the planes below and at the current one
    make_J(z0 - 1);
    __syncthreads();
    divJ_parts(Am, Bm);
    __syncthreads();
    make_J(z0);
    __syncthreads();
    divJ_parts(A0, B0);
    float uzc = __ldg(uz + (long long)wrap_mod(z0, nz) * plane + own);  // uz of the current plane
    float fzm = z_flux(z0 - 1, __ldg(uz + (long long)wrap_mod(z0 - 1, nz) * plane + own), uzc);
    // the face velocities of a plane (left and right site of each x and y face)
    // and uz above the column, loaded one plane ahead of their use so that
    // their latency overlaps the barrier and the J planes
    float vxl[NFL], vxr[NFL], vyl[NFL], vyr[NFL];
    auto load_u = [&](int zq) {  // z0 <= zq < nz
        const long long zb = (long long)zq * plane;
#pragma unroll
        for (int k = 0; k < NFL; ++k) {
            vxl[k] = fx_i[k] >= 0 ? __ldg(ux + zb + fx_l[k]) : 0.f;
            vxr[k] = fx_i[k] >= 0 ? __ldg(ux + zb + fx_r[k]) : 0.f;
            vyl[k] = fy_i[k] >= 0 ? __ldg(uy + zb + fy_l[k]) : 0.f;
            vyr[k] = fy_i[k] >= 0 ? __ldg(uy + zb + fy_r[k]) : 0.f;
        }
    };
    load_u(z0);
    float uzn = __ldg(uz + (long long)wrap_mod(z0 + 1, nz) * plane + own);
    __syncthreads();  // the J plane is rewritten below

    for (int z = z0; z < z1; ++z) {
        make_J(z + 1);
        cp_async_wait<0>();  // this thread's copies of plane z + 3 (issued last iteration) have landed
        __syncthreads();     // J of z + 1 and phi of z + 3 are in place

        const long long zb = (long long)z * plane;  // z < nz
        const float(*P0)[PX] = s_p[z & (PR - 1)];
        // x and y faces of plane z
#pragma unroll
        for (int k = 0; k < NFL; ++k) {
            if (fx_i[k] >= 0) {
                const int r = fx_i[k] / (TX + 1), f = fx_i[k] - r * (TX + 1);
                float v[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) v[j] = P0[r + WH][f + j];
                (&s_Fx[0][0])[fx_i[k]] = face_flux(v, vxl[k], vxr[k]);
            }
            if (fy_i[k] >= 0) {
                const int f = fy_i[k] / TX, c = fy_i[k] - f * TX;
                float v[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) v[j] = P0[f + j][c + WH];
                (&s_Fy[0][0])[fy_i[k]] = face_flux(v, vyl[k], vyr[k]);
            }
        }
        if (z + 3 <= z1 + 1) partials(z + 3);  // make_J(z + 2) of the next plane reads it
        float Ap, Bp;
        divJ_parts(Ap, Bp);
        // D lap(p) - kappa div(J) at (x, y, z) with weights (1, 4, 1)^3
        float lap;
        {
            const float pz = P0[pcy][pcx];
            const float pm = s_p[(z - 1) & (PR - 1)][pcy][pcx], pp = s_p[(z + 1) & (PR - 1)][pcy][pcx];
            const float Sm = s_G[g5(z - 1)][2][gq], S0 = s_G[g5(z)][2][gq], Sp = s_G[g5(z + 1)][2][gq];
            lap = fmaf(4.f, S0, fmaf(36.f, pm - pz, Sm) + fmaf(36.f, pp - pz, Sp));
        }
        const float dj = fmaf(4.f, A0, Am + Ap) + (Bp - Bm);
        Am = A0; Bm = B0; A0 = Ap; B0 = Bp;
        // the upper z face of this column
        const float fzp = z_flux(z, uzc, uzn);
        __syncthreads();  // the plane's x and y face fluxes are in place

        const float adv = (s_Fx[ly][lx + 1] - s_Fx[ly][lx]) + (s_Fy[ly + 1][lx] - s_Fy[ly][lx]) + (fzp - fzm);
        const float L = fmaf(D * (1.f / 36.f), lap, -kap * (1.f / 72.f) * dj) - adv;
        if (active) {
            const long long s = zb + own;
            const float q = P0[pcy][pcx] + L;
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
        fzm = fzp;
        uzc = uzn;
        if (z + 1 < z1) {
            load_plane(z + 4);  // the next plane's; no copy may be in flight when the march ends
            load_u(z + 1);
            uzn = __ldg(uz + (long long)wrap_mod(z + 2, nz) * plane + own);
        }
    }
}

}  // namespace

cudaError_t launch_weno_stage(int stage, const float* pin, const float* phin, const float* u, float* out, int nx,
                              int ny, int nz, float D, float kap, cudaStream_t st) {
    const long long N = (long long)nx * ny * nz;
    const int zc = nz < 32 ? nz : 32;
    const dim3 grid((unsigned)((nx + TX - 1) / TX), (unsigned)((ny + TY - 1) / TY), (unsigned)((nz + zc - 1) / zc));
    weno_stage_kernel<<<grid, WNT, 0, st>>>(pin, phin, u, u + N, u + 2 * N, out, nx, ny, nz, zc, D, kap, stage);
    return cudaGetLastError();
}

}  // namespace lbgb
