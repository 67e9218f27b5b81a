// lbgb_api.cu -- C ABI of the fused two-phase lattice Boltzmann library (see
// include/lbgb.h for the contract of each call).
//
// A context owns, on one device: f (27 planes, in place, AA pattern), g (two
// buffers of 7 planes), the per-block FP64 partial sums, a small DevState
// (forcing amplitude, K_target, last diagnostics, non-finite flag), the ABC
// sin/cos tables and, on demand, staging buffers for host-pointer I/O.
// A step is two launches on the context's stream: the fused step kernel and a
// one-block FP64 reduction that also updates the forcing amplitude on the
// device, so consecutive steps need no host synchronisation and can be
// captured in a CUDA graph (two steps, one of each AA parity).
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "lbgb.h"
#include "lbgb_kernels.cuh"

using namespace lbgb;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define LB_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                   \
    } while (0)

struct FinalizeArgs {
    int mode;        // MODE_STEP or MODE_INIT
    int force_kind;
    double eps_per_aa;  // eps = eps_per_aa * (sum of the per-site a2:a2 partials)
    double T_relax, K_target_param;
};

// One block: deterministic FP64 sum of the per-block partials, then the
// diagnostics (step 13) and the next linear-forcing amplitude.
__global__ void __launch_bounds__(256) finalize_kernel(const double* __restrict__ part, int nblk,
                                                       DevState* st, FinalizeArgs fa) {
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        const double* p = part + (long long)b * NPART;
        v0 += p[0];
        v1 += p[1];
        v2 += p[2];
        v3 += p[3];
        v4 = fmax(v4, p[4]);
    }
    block_reduce5<256>(v0, v1, v2, v3, v4);
    if (threadIdx.x == 0) {
        const double Phi = v0, K = v1, umax = sqrt(v4);
        // a NaN or Inf anywhere reaches the sums (max ignores NaN, the sums do not)
        const bool bad = !isfinite(v0 + v1 + v2 + v3);
        if (fa.mode == MODE_INIT) {
            st->K_target = fa.K_target_param > 0 ? fa.K_target_param : K;
            st->A = 0.0;
            st->diag[0] = Phi; st->diag[1] = K; st->diag[2] = 0.0; st->diag[3] = umax; st->diag[4] = 0.0;
            st->mass = 0.0;
            st->flags = bad ? 1 : 0;
        } else {
            // eps = 2 nu sum S:S, S = -a2/(2 cs^2 tau) = -(3/(2 tau)) a2 (with density
            // contrasts the partials already carry each site's 2 nu (3/(2 tau))^2)
            const double eps = fa.eps_per_aa * v2;
            double An = 0.0;
            if (fa.force_kind == FK_LINEAR && K > 0) An = (eps + (st->K_target - K) / fa.T_relax) / (2.0 * K);
            st->diag[0] = Phi; st->diag[1] = K; st->diag[2] = eps; st->diag[3] = umax; st->diag[4] = An;
            st->mass = v3;
            st->A = An;
            if (bad) st->flags |= 1;
        }
    }
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct lb_ctx {
    int nx, ny, nz;
    long long N;
    double tau, M, W, sigma;
    lb_force force;
    int storage;
    size_t fsize;  // bytes per stored f value
    int device;

    void* f = nullptr;  // AA: 27 planes; LB_F32_MOMENTS: 2 buffers x 10 coefficient planes
    float* g[2] = {nullptr, nullptr};
    double* partials = nullptr;
    long long npart_cap = 0;
    DevState* st = nullptr;
    float* abc = nullptr;
    float* stage = nullptr;  // 5N floats for host I/O, allocated on demand
    cudaStream_t stream = nullptr;

    long long t = 0;
    bool initialized = false;
    int ty = 8, zc = 32;
    long long launches = 0;

    cudaGraphExec_t graph = nullptr;  // two steps starting at even parity
    int graph_ty = 0, graph_zc = 0;
    bool graph_pair = false;

    bool pair = false;  // paired step kernel preferred (16-bit storages; see use_pair)

    bool fd = false;  // phase field by finite differences (lb_set_phase_solver)
    bool vd = false;  // density and viscosity contrasts (lb_set_density)
    double rho_l = 1.0, rho_g = 1.0, tau_l = 1.0, tau_g = 1.0;
    double gb[3] = {0.0, 0.0, 0.0}, rho_ref = 0.0;  // buoyancy (lb_set_gravity)

    bool timing = false;                       // event pairs around fused launches
    std::vector<cudaEvent_t> ev_start, ev_stop;
    size_t ev_used = 0;
};

namespace {

// tx: tile width in sites (32; 64 for the paired kernel)
dim3 grid_for(const lb_ctx* c, int ty, int zc, int tx = 32) {
    return dim3((unsigned)((c->nx + tx - 1) / tx), (unsigned)((c->ny + ty - 1) / ty),
                (unsigned)((c->nz + zc - 1) / zc));
}

bool is_mc(const lb_ctx* c) { return c->storage == LB_F32_MOMENTS; }
// 16-bit D3Q7 populations as well as 16-bit f (the G16 kernels)
bool is_g16(const lb_ctx* c) { return c->storage == LB_F16_SHIFTED_G16 || c->storage == LB_BF16_SHIFTED_G16; }
// f stored as FP16 (LB_F16_SHIFTED, LB_F16_SHIFTED_G16)
bool is_f16(const lb_ctx* c) { return c->storage == LB_F16_SHIFTED || c->storage == LB_F16_SHIFTED_G16; }
// bytes of one D3Q7 buffer: 7 FP32 planes, or (G16) 7 planes of gamma and one of phi~ in 16 bits
size_t g_buf_bytes(const lb_ctx* c) { return (size_t)c->N * (is_g16(c) ? 8 * 2 : 7 * sizeof(float)); }

// The paired step kernel (two x-adjacent sites per thread, packed two-lane FP32
// arithmetic) runs the step when it is preferred and applies: a 16-bit AA
// storage, nx a multiple of 4; the D3Q7 phase field with or without density
// contrasts, or the finite-difference phase field without them.
bool pair_applies(const lb_ctx* c) {
    return (c->fsize == 2 && !is_mc(c)) && c->nx % 4 == 0 && !(c->fd && c->vd);
}
bool use_pair(const lb_ctx* c) { return c->pair && pair_applies(c); }

size_t f_bytes(const lb_ctx* c) { return (size_t)c->N * (is_mc(c) ? 20 * sizeof(float) : 27 * c->fsize); }

StepArgs base_args(const lb_ctx* c) {
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.zc = c->zc;
    a.N = (int)c->N;
    if (!is_mc(c))
        for (int i = 0; i < 27; ++i) a.fk[i] = (char*)c->f + (size_t)i * (size_t)c->N * c->fsize;
    a.force_kind = c->force.kind;
    a.omega = (float)(1.0 / c->tau);
    a.omega_phi = (float)(1.0 / (c->M / 0.25 + 0.5));
    a.sharp = isinf(c->W) ? 0.f : (float)((c->M / 0.25) * (4.0 / c->W));
    a.beta = c->sigma == 0 ? 0.f : (float)(1.5 * c->W * c->sigma);
    a.gc0 = (float)c->force.g[0]; a.gc1 = (float)c->force.g[1]; a.gc2 = (float)c->force.g[2];
    a.A_abc = (float)c->force.A;
    a.abc = c->abc;
    a.st = c->st;
    a.partials = c->partials;
    if (c->vd) {
        a.rho_g = (float)c->rho_g;
        a.drho = (float)(c->rho_l - c->rho_g);
        a.tau_g = (float)c->tau_g;
        a.dtau = (float)(c->tau_l - c->tau_g);
        a.gb0 = (float)c->gb[0]; a.gb1 = (float)c->gb[1]; a.gb2 = (float)c->gb[2];
        a.rho_ref = (float)c->rho_ref;
    }
    return a;
}

// D3Q7 plane pointers: read buffer `par`, write buffer par ^ 1 (and likewise
// the coefficient buffers of the moment-only storage).  With the
// finite-difference phase field, g[0] holds phi (plane 0) and the two RK
// stages (planes 1, 2), g[1] the velocity u (planes 0-2) the step writes; the
// kernel reads phi from gin[0] and writes u to gout[0..2] (INIT: phi to gout[0]).
float* g_plane(const lb_ctx* c, int buf, int q) { return c->g[buf] + (size_t)q * (size_t)c->N; }

void set_g(StepArgs& a, const lb_ctx* c, int par, bool init = false) {
    if (is_g16(c)) {  // planes of 2-byte values: gamma_0..6, then phi~
        const char* gi = reinterpret_cast<const char*>(c->g[par]);
        char* go = reinterpret_cast<char*>(c->g[par ^ 1]);
        for (int q = 0; q < 7; ++q) {
            a.gin[q] = reinterpret_cast<const float*>(gi + (size_t)q * (size_t)c->N * 2);
            a.gout[q] = reinterpret_cast<float*>(go + (size_t)q * (size_t)c->N * 2);
        }
        a.gphi_in = gi + (size_t)7 * (size_t)c->N * 2;
        a.gphi_out = go + (size_t)7 * (size_t)c->N * 2;
        return;
    }
    if (c->fd) {
        for (int q = 0; q < 7; ++q) {
            a.gin[q] = g_plane(c, 0, 0);
            a.gout[q] = init ? g_plane(c, 0, 0) : g_plane(c, 1, q < 3 ? q : 0);
        }
    } else {
        for (int q = 0; q < 7; ++q) {
            a.gin[q] = g_plane(c, par, q);
            a.gout[q] = g_plane(c, par ^ 1, q);
        }
    }
    if (is_mc(c)) {
        float* C = static_cast<float*>(c->f);
        for (int k = 0; k < 10; ++k) {
            a.cin[k] = C + (size_t)(10 * par + k) * (size_t)c->N;
            a.cout[k] = C + (size_t)(10 * (par ^ 1) + k) * (size_t)c->N;
        }
    }
}

// parity: AA parity (t & 1); for the moment-only storage, 1 when the state
// at t is a set of post-collision coefficients to pull from (t > 0).
cudaError_t launch_any(const lb_ctx* c, int mode, int parity, int ty, dim3 grid, const StepArgs& a,
                       cudaStream_t s) {
    // float4 phase-A loads need 16-byte aligned rows: nx % 4 == 0 (planes then start aligned too)
    const bool vec = (c->nx % 4) == 0;
    if (is_g16(c))
        return is_f16(c) ? launch_fused_g16<__half>(mode, parity, ty, grid, a, s)
                         : launch_fused_g16<__nv_bfloat16>(mode, parity, ty, grid, a, s);
    if (c->fd || (c->vd && mode != MODE_INIT)) {
        const bool vd = c->vd && mode != MODE_INIT;
#define LBGB_X(FT, MC)                                                                              \
    (c->fd ? (vd ? launch_fused_x<FT, MC, true, true>(mode, parity, ty, vec, grid, a, s)            \
                 : launch_fused_x<FT, MC, false, true>(mode, parity, ty, vec, grid, a, s))          \
           : launch_fused_x<FT, MC, true, false>(mode, parity, ty, vec, grid, a, s))
        switch (c->storage) {
            case LB_F32_MOMENTS: return LBGB_X(float, true);
            case LB_F32: return LBGB_X(float, false);
            case LB_F16_SHIFTED: return LBGB_X(__half, false);
            case LB_BF16_SHIFTED: return LBGB_X(__nv_bfloat16, false);
        }
#undef LBGB_X
        return cudaErrorInvalidValue;
    }
    switch (c->storage) {
        case LB_F32_MOMENTS: return launch_fused_mc(mode, parity, ty, vec, grid, a, s);
        case LB_F32: return launch_fused<float>(mode, parity, ty, vec, grid, a, s);
        case LB_F16_SHIFTED: return launch_fused<__half>(mode, parity, ty, vec, grid, a, s);
        case LB_BF16_SHIFTED: return launch_fused<__nv_bfloat16>(mode, parity, ty, vec, grid, a, s);
    }
    return cudaErrorInvalidValue;
}

FinalizeArgs fin_args(const lb_ctx* c, int mode) {
    FinalizeArgs fa;
    fa.mode = mode;
    fa.force_kind = c->force.kind;
    if (c->vd) {
        fa.eps_per_aa = 1.0;
    } else {
        const double nu = (c->tau - 0.5) / 3.0, s = 1.5 / c->tau;
        fa.eps_per_aa = 2.0 * nu * s * s;
    }
    fa.T_relax = c->force.T_relax;
    fa.K_target_param = c->force.K_target;
    return fa;
}

// One time step at parity `par` on stream s (2 launches); `first` marks the
// step from t = 0 of the moment-only storage, which evaluates each site's own
// coefficients instead of pulling.
int enqueue_step(lb_ctx* c, int par, cudaStream_t s, bool first = false) {
    StepArgs a = base_args(c);
    a.zc = c->zc;
    set_g(a, c, par);
    const dim3 grid = grid_for(c, c->ty, c->zc, use_pair(c) ? 64 : 32);
    const long long nblk = (long long)grid.x * grid.y * grid.z;
    if (nblk > c->npart_cap) return fail(LB_EINVAL, "tile (%d,%d) needs %lld partials > %lld", c->ty, c->zc, nblk, c->npart_cap);
    const bool timed = c->timing && s == c->stream;
    if (timed) {
        if (c->ev_used == c->ev_start.size()) {
            cudaEvent_t e0, e1;
            LB_CUDA(cudaEventCreate(&e0));
            LB_CUDA(cudaEventCreate(&e1));
            c->ev_start.push_back(e0);
            c->ev_stop.push_back(e1);
        }
        LB_CUDA(cudaEventRecord(c->ev_start[c->ev_used], s));
    }
    if (use_pair(c)) {
        if (is_g16(c))
            LB_CUDA(is_f16(c) ? launch_fused_pair_g16<__half>(par, c->ty, grid, a, s)
                              : launch_fused_pair_g16<__nv_bfloat16>(par, c->ty, grid, a, s));
        else if (c->vd)
            LB_CUDA(is_f16(c) ? launch_fused_pair_vd<__half>(par, c->ty, grid, a, s)
                              : launch_fused_pair_vd<__nv_bfloat16>(par, c->ty, grid, a, s));
        else if (c->fd)
            LB_CUDA(is_f16(c) ? launch_fused_pair_pf<__half>(par, c->ty, grid, a, s)
                              : launch_fused_pair_pf<__nv_bfloat16>(par, c->ty, grid, a, s));
        else
            LB_CUDA(is_f16(c) ? launch_fused_pair<__half>(par, c->ty, grid, a, s)
                              : launch_fused_pair<__nv_bfloat16>(par, c->ty, grid, a, s));
    } else {
        LB_CUDA(launch_any(c, MODE_STEP, is_mc(c) ? (first ? 0 : 1) : par, c->ty, grid, a, s));
    }
    if (timed) {
        LB_CUDA(cudaEventRecord(c->ev_stop[c->ev_used], s));
        c->ev_used += 1;
    }
    if (c->fd) {
        // Eq. 4 by finite differences, three RK stages on the u just written
        const float D = (float)c->M, kap = isinf(c->W) ? 0.f : (float)(4.0 * c->M / c->W);
        float *p0 = g_plane(c, 0, 0), *p1 = g_plane(c, 0, 1), *p2 = g_plane(c, 0, 2);
        const float* u = g_plane(c, 1, 0);
        LB_CUDA(launch_weno_stage(0, p0, p0, u, p1, c->nx, c->ny, c->nz, D, kap, s));
        LB_CUDA(launch_weno_stage(1, p1, p0, u, p2, c->nx, c->ny, c->nz, D, kap, s));
        LB_CUDA(launch_weno_stage(2, p2, p0, u, p0, c->nx, c->ny, c->nz, D, kap, s));
        c->launches += 3;
    }
    finalize_kernel<<<1, 256, 0, s>>>(c->partials, (int)nblk, c->st, fin_args(c, MODE_STEP));
    LB_CUDA(cudaGetLastError());
    c->launches += 2;
    return LB_OK;
}

void drop_graph(lb_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
}

int capture_graph(lb_ctx* c) {
    drop_graph(c);
    cudaStream_t cs;
    LB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(LB_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    long long before = c->launches;
    int rc = enqueue_step(c, 0, cs);
    if (rc == LB_OK) rc = enqueue_step(c, 1, cs);
    c->launches = before;  // captured launches are counted when replayed
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != LB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(LB_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return fail(LB_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    c->graph_ty = c->ty;
    c->graph_zc = c->zc;
    c->graph_pair = use_pair(c);
    return LB_OK;
}

int ensure_stage(lb_ctx* c) {
    if (!c->stage) LB_CUDA(cudaMalloc(&c->stage, (size_t)c->N * 5 * sizeof(float)));
    return LB_OK;
}

// Tile heights: {4, 8} for both the one-site and the paired kernels.
int check_tile(int ty, int zc, bool pair = false) {
    (void)pair;
    if (ty != 4 && ty != 8) return fail(LB_EINVAL, "tile height %d not in {4, 8}", ty);
    if (zc < 1) return fail(LB_EINVAL, "z chunk %d < 1", zc);
    return LB_OK;
}

// Z-chunks the tuner times for tile height ty: 16, 32, 64 and 128 planes
// (those that give distinct launches), plus the two chunkings whose block
// count best fills the last wave of resident blocks (at least 24 planes each,
// so the chunk prologue stays small).  Returns how many were written to zcs.
int tune_chunks(const lb_ctx* c, int ty, int zcs[6]) {
    int n = 0;
    const int fixed[4] = {16, 32, 64, 128};
    for (int b = 0; b < 4; ++b) {
        if (b > 0 && fixed[b - 1] >= c->nz) break;  // larger chunks clamp to the same launch
        zcs[n++] = fixed[b];
    }
    const bool vec = (c->nx % 4) == 0;
    int per_sm = 0;
#define LBGB_XO(FT, MC)                                                                                     \
    (c->fd ? (c->vd ? fused_x_blocks_per_sm<FT, MC, true, true>(ty, vec) : fused_x_blocks_per_sm<FT, MC, false, true>(ty, vec)) \
           : fused_x_blocks_per_sm<FT, MC, true, false>(ty, vec))
    const bool x = c->fd || c->vd;
    switch (c->storage) {
        case LB_F32: per_sm = x ? LBGB_XO(float, false) : fused_blocks_per_sm<float>(ty, vec); break;
        case LB_F16_SHIFTED: per_sm = x ? LBGB_XO(__half, false) : fused_blocks_per_sm<__half>(ty, vec); break;
        case LB_BF16_SHIFTED: per_sm = x ? LBGB_XO(__nv_bfloat16, false) : fused_blocks_per_sm<__nv_bfloat16>(ty, vec); break;
        case LB_F32_MOMENTS: per_sm = x ? LBGB_XO(float, true) : fused_mc_blocks_per_sm(ty, vec); break;
    }
#undef LBGB_XO
    if (is_g16(c))
        per_sm = use_pair(c) ? (is_f16(c) ? fused_pair_g16_blocks_per_sm<__half>(ty)
                                          : fused_pair_g16_blocks_per_sm<__nv_bfloat16>(ty))
                             : (is_f16(c) ? fused_g16_blocks_per_sm<__half>(ty)
                                          : fused_g16_blocks_per_sm<__nv_bfloat16>(ty));
    else if (use_pair(c) && c->fd)
        per_sm = is_f16(c) ? fused_pair_pf_blocks_per_sm<__half>(ty) : fused_pair_pf_blocks_per_sm<__nv_bfloat16>(ty);
    else if (use_pair(c) && c->vd)
        per_sm = is_f16(c) ? fused_pair_vd_blocks_per_sm<__half>(ty) : fused_pair_vd_blocks_per_sm<__nv_bfloat16>(ty);
    else if (use_pair(c))
        per_sm = is_f16(c) ? fused_pair_blocks_per_sm<__half>(ty) : fused_pair_blocks_per_sm<__nv_bfloat16>(ty);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    const long long resident = (long long)sms * per_sm;
    if (resident <= 0) return n;
    const int tx = use_pair(c) ? 64 : 32;
    const long long tiles = (long long)((c->nx + tx - 1) / tx) * ((c->ny + ty - 1) / ty);
    double fill[2] = {0.0, 0.0};
    int pick[2] = {0, 0};
    for (int nc = (c->nz + 127) / 128; nc <= c->nz / 24; ++nc) {
        const int zc = (c->nz + nc - 1) / nc;
        if ((c->nz + zc - 1) / zc != nc) continue;  // this chunking is reached by another zc
        const long long blocks = tiles * nc;
        const long long waves = (blocks + resident - 1) / resident;
        const double f = (double)blocks / (double)(waves * resident);
        if (f > fill[0]) {
            fill[1] = fill[0]; pick[1] = pick[0];
            fill[0] = f; pick[0] = zc;
        } else if (f > fill[1]) {
            fill[1] = f; pick[1] = zc;
        }
    }
    for (int k = 0; k < 2; ++k) {
        bool dup = pick[k] == 0;
        for (int j = 0; j < n && !dup; ++j) dup = zcs[j] == pick[k];
        if (!dup) zcs[n++] = pick[k];
    }
    return n;
}

long long max_blocks(const lb_ctx* c) {
    // the smallest tile (ty = 4) with zc = 1 bounds every configuration
    return (long long)((c->nx + 31) / 32) * ((c->ny + 3) / 4) * c->nz;
}

}  // namespace

namespace lbgb {
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace lbgb

extern "C" {

const char* lb_last_error(void) { return g_err; }

void lb_destroy(lb_ctx* c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    drop_graph(c);
    for (auto e : c->ev_start) cudaEventDestroy(e);
    for (auto e : c->ev_stop) cudaEventDestroy(e);
    cudaFree(c->f);
    cudaFree(c->g[0]);
    cudaFree(c->g[1]);
    cudaFree(c->partials);
    cudaFree(c->st);
    cudaFree(c->abc);
    cudaFree(c->stage);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

int lb_create(int nx, int ny, int nz, double tau, double M, double W, double sigma, const lb_force* force,
              int storage, lb_ctx** out) {
    if (!out) return fail(LB_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(LB_EINVAL, "box %d x %d x %d: every edge must be >= 1", nx, ny, nz);
    if ((long long)nx * ny * nz >= (1LL << 31) - 1)
        return fail(LB_EINVAL, "nx*ny*nz must be < 2^31 - 1 (32-bit site indices)");
    if (!(tau > 0.5) || !isfinite(tau)) return fail(LB_EINVAL, "tau = %g must be > 1/2", tau);
    if (!(M > 0) || !isfinite(M)) return fail(LB_EINVAL, "M = %g must be > 0", M);
    if (!(W > 0)) return fail(LB_EINVAL, "W = %g must be > 0 (or +inf)", W);
    if (!(sigma >= 0) || !isfinite(sigma)) return fail(LB_EINVAL, "sigma = %g must be >= 0", sigma);
    if (isinf(W) && sigma > 0) return fail(LB_EINVAL, "sigma > 0 needs a finite W");
    if (storage != LB_F32 && storage != LB_F16_SHIFTED && storage != LB_BF16_SHIFTED && storage != LB_F32_MOMENTS &&
        storage != LB_F16_SHIFTED_G16 && storage != LB_BF16_SHIFTED_G16)
        return fail(LB_EINVAL, "unknown storage %d", storage);
    if ((storage == LB_F16_SHIFTED_G16 || storage == LB_BF16_SHIFTED_G16) && nx % 4 != 0)
        return fail(LB_EINVAL, "16-bit D3Q7 storage needs nx %% 4 == 0 (got nx = %d)", nx);
    lb_force fz;
    memset(&fz, 0, sizeof(fz));
    if (force) fz = *force;
    if (fz.kind < LB_FORCE_NONE || fz.kind > LB_FORCE_LINEAR) return fail(LB_EINVAL, "unknown force kind %d", fz.kind);
    if (fz.kind == LB_FORCE_LINEAR && !(fz.T_relax > 0)) return fail(LB_EINVAL, "linear forcing needs T_relax > 0");

    lb_ctx* c = new lb_ctx();
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->N = (long long)nx * ny * nz;
    c->tau = tau; c->M = M; c->W = W; c->sigma = sigma;
    c->force = fz;
    c->storage = storage;
    c->fsize = (storage == LB_F32 || storage == LB_F32_MOMENTS) ? 4 : 2;
    cudaGetDevice(&c->device);
    // default launch shape: z chunk of 32 planes, smaller for thin boxes
    c->ty = 8;
    c->zc = nz < 32 ? nz : 32;
    c->pair = pair_applies(c);  // the paired kernel by default where it applies

    int rc = LB_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc != LB_OK) return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "cudaMalloc(%zu bytes): %s", bytes,
                      cudaGetErrorString(e));
        }
    };
    alloc(&c->f, f_bytes(c));
    alloc((void**)&c->g[0], g_buf_bytes(c));
    alloc((void**)&c->g[1], g_buf_bytes(c));
    c->npart_cap = max_blocks(c);
    alloc((void**)&c->partials, (size_t)c->npart_cap * NPART * sizeof(double));
    alloc((void**)&c->st, sizeof(DevState));
    if (rc == LB_OK && fz.kind == LB_FORCE_ABC) {
        const int L = 2 * (nx + ny + nz);
        float* h = (float*)malloc((size_t)L * sizeof(float));
        if (!h) {
            lb_destroy(c);
            return fail(LB_ENOMEM, "host table of %d floats", L);
        }
        int o = 0;
        const int ns[3] = {nx, ny, nz};
        for (int ax = 0; ax < 3; ++ax) {
            for (int k = 0; k < ns[ax]; ++k) h[o + k] = (float)sin(fz.kf * k);
            for (int k = 0; k < ns[ax]; ++k) h[o + ns[ax] + k] = (float)cos(fz.kf * k);
            o += 2 * ns[ax];
        }
        alloc((void**)&c->abc, (size_t)L * sizeof(float));
        if (rc == LB_OK) {
            cudaError_t e = cudaMemcpy(c->abc, h, (size_t)L * sizeof(float), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = fail(LB_ECUDA, "ABC table upload: %s", cudaGetErrorString(e));
        }
        free(h);
    }
    if (rc == LB_OK) {
        cudaError_t e = cudaMemset(c->st, 0, sizeof(DevState));
        if (e != cudaSuccess) rc = fail(LB_ECUDA, "cudaMemset: %s", cudaGetErrorString(e));
    }
    if (rc != LB_OK) {
        lb_destroy(c);
        return rc;
    }
    *out = c;
    return LB_OK;
}

int lb_set_stream(lb_ctx* c, void* stream) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    c->stream = (cudaStream_t)stream;
    return LB_OK;
}

int lb_init(lb_ctx* c, const float* phi, const float* u) {
    if (!c || !phi || !u) return fail(LB_EINVAL, "lb_init: NULL argument");
    const long long N = c->N;
    const float* dphi = phi;
    const float* du = u;
    if (!is_device_pointer(phi) || !is_device_pointer(u)) {
        int rc = ensure_stage(c);
        if (rc) return rc;
        if (!is_device_pointer(phi)) {
            LB_CUDA(cudaMemcpyAsync(c->stage, phi, (size_t)N * sizeof(float), cudaMemcpyDefault, c->stream));
            dphi = c->stage;
        }
        if (!is_device_pointer(u)) {
            LB_CUDA(cudaMemcpyAsync(c->stage + N, u, (size_t)N * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
            du = c->stage + N;
        }
    }
    StepArgs a = base_args(c);
    a.zc = c->nz < 32 ? c->nz : 32;
    set_g(a, c, 1, true);  // writes buffer 0 (finite-difference phase field: phi into g[0] plane 0)
    a.in_phi = dphi;
    a.in_u = du;
    const dim3 grid = grid_for(c, 8, a.zc);
    const long long nblk = (long long)grid.x * grid.y * grid.z;
    LB_CUDA(launch_any(c, MODE_INIT, 0, 8, grid, a, c->stream));
    finalize_kernel<<<1, 256, 0, c->stream>>>(c->partials, (int)nblk, c->st, fin_args(c, MODE_INIT));
    LB_CUDA(cudaGetLastError());
    c->launches += 2;
    c->t = 0;
    c->initialized = true;
    if (dphi != phi || du != u) LB_CUDA(cudaStreamSynchronize(c->stream));  // staging is reused
    return LB_OK;
}

int lb_step(lb_ctx* c, int n) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (n < 0) return fail(LB_EINVAL, "n = %d < 0", n);
    if (!c->initialized) return fail(LB_ESTATE, "lb_step before lb_init");
    int rc = check_tile(c->ty, c->zc, use_pair(c));
    if (rc) return rc;
    while (n > 0) {
        const int par = (int)(c->t & 1);
        const bool first = is_mc(c) && c->t == 0;
        if (par == 0 && n >= 2 && !c->timing && !first) {
            if (!c->graph || c->graph_ty != c->ty || c->graph_zc != c->zc || c->graph_pair != use_pair(c)) {
                rc = capture_graph(c);
                if (rc) return rc;
            }
            LB_CUDA(cudaGraphLaunch(c->graph, c->stream));
            c->launches += 4;
            c->t += 2;
            n -= 2;
        } else {
            rc = enqueue_step(c, par, c->stream, first);
            if (rc) return rc;
            c->t += 1;
            n -= 1;
        }
    }
    return LB_OK;
}

int lb_moments(lb_ctx* c, float* rho, float* u, float* phi) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_moments before lb_init");
    const long long N = c->N;
    const bool hr = rho && !is_device_pointer(rho);
    const bool hu = u && !is_device_pointer(u);
    const bool hp = phi && !is_device_pointer(phi);
    if (hr || hu || hp) {
        int rc = ensure_stage(c);
        if (rc) return rc;
    }
    StepArgs a = base_args(c);
    a.zc = c->nz < 32 ? c->nz : 32;
    const int par = (int)(c->t & 1);
    set_g(a, c, par);
    a.out_rho = hr ? c->stage : rho;
    a.out_u = hu ? c->stage + N : u;
    a.out_phi = hp ? c->stage + 4 * N : phi;
    const int kpar = is_mc(c) ? (c->t > 0 ? 1 : 0) : par;
    LB_CUDA(launch_any(c, MODE_MOMENTS, kpar, 8, grid_for(c, 8, a.zc), a, c->stream));
    c->launches += 1;
    if (hr) LB_CUDA(cudaMemcpyAsync(rho, c->stage, (size_t)N * sizeof(float), cudaMemcpyDefault, c->stream));
    if (hu) LB_CUDA(cudaMemcpyAsync(u, c->stage + N, (size_t)N * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
    if (hp) LB_CUDA(cudaMemcpyAsync(phi, c->stage + 4 * N, (size_t)N * sizeof(float), cudaMemcpyDefault, c->stream));
    if (hr || hu || hp) LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

int lb_diagnostics(lb_ctx* c, double out[5]) {
    if (!c || !out) return fail(LB_EINVAL, "lb_diagnostics: NULL argument");
    if (!c->initialized) return fail(LB_ESTATE, "lb_diagnostics before lb_init");
    DevState h;
    LB_CUDA(cudaMemcpyAsync(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 5; ++k) out[k] = h.diag[k];
    if (h.flags & 1) return fail(LB_ENONFINITE, "a NaN or Inf was met since lb_init");
    return LB_OK;
}

int lb_sync(lb_ctx* c) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

long long lb_time(const lb_ctx* c) { return c ? c->t : -1; }

long long lb_launch_count(const lb_ctx* c) { return c ? c->launches : -1; }

int lb_set_density(lb_ctx* c, double rho_l, double rho_g, double tau_l, double tau_g) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (!(rho_l > 0) || !(rho_g > 0) || !(tau_l > 0.5) || !(tau_g > 0.5) || !isfinite(rho_l) || !isfinite(rho_g) ||
        !isfinite(tau_l) || !isfinite(tau_g))
        return fail(LB_EINVAL, "lb_set_density: need rho > 0 and tau > 1/2, got rho %g, %g, tau %g, %g", rho_l, rho_g,
                    tau_l, tau_g);
    if (is_g16(c)) return fail(LB_EINVAL, "lb_set_density: density contrasts need FP32 D3Q7 populations");
    c->vd = true;
    c->rho_l = rho_l; c->rho_g = rho_g; c->tau_l = tau_l; c->tau_g = tau_g;
    drop_graph(c);  // the captured launches carry the old kernel and arguments
    return LB_OK;
}

int lb_set_phase_solver(lb_ctx* c, int solver) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (solver != LB_PHASE_LB && solver != LB_PHASE_WENO5) return fail(LB_EINVAL, "unknown phase solver %d", solver);
    if (solver == LB_PHASE_WENO5 && is_g16(c))
        return fail(LB_EINVAL, "the WENO-5 phase field holds no D3Q7 populations: use LB_F16_SHIFTED or LB_BF16_SHIFTED");
    if (c->initialized && (solver == LB_PHASE_WENO5) != c->fd)
        return fail(LB_ESTATE, "lb_set_phase_solver after lb_init (the state is held differently)");
    c->fd = solver == LB_PHASE_WENO5;
    drop_graph(c);
    return LB_OK;
}

int lb_set_gravity(lb_ctx* c, double gx, double gy, double gz, double rho_ref) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (!c->vd) return fail(LB_ESTATE, "lb_set_gravity needs lb_set_density first");
    if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz) || !isfinite(rho_ref))
        return fail(LB_EINVAL, "lb_set_gravity: non-finite argument");
    c->gb[0] = gx; c->gb[1] = gy; c->gb[2] = gz;
    c->rho_ref = rho_ref;
    drop_graph(c);  // the captured launches carry the old arguments
    return LB_OK;
}

int lb_set_timing(lb_ctx* c, int on) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    c->timing = on != 0;
    c->ev_used = 0;
    return LB_OK;
}

int lb_kernel_time(lb_ctx* c, double* ms, long long* launches) {
    if (!c || !ms || !launches) return fail(LB_EINVAL, "lb_kernel_time: NULL argument");
    LB_CUDA(cudaStreamSynchronize(c->stream));
    double total = 0.0;
    for (size_t k = 0; k < c->ev_used; ++k) {
        float m = 0.f;
        LB_CUDA(cudaEventElapsedTime(&m, c->ev_start[k], c->ev_stop[k]));
        total += m;
    }
    *ms = total;
    *launches = (long long)c->ev_used;
    return LB_OK;
}

int lb_set_tile(lb_ctx* c, int ty, int zc) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    int rc = check_tile(ty, zc, use_pair(c));
    if (rc) return rc;
    c->ty = ty;
    c->zc = zc > c->nz ? c->nz : zc;
    return LB_OK;
}

int lb_set_pairing(lb_ctx* c, int on) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (on && !pair_applies(c))
        return fail(LB_EINVAL, "the paired step kernel needs FP16 or BF16 storage and nx %% 4 == 0 (and not density "
                               "contrasts together with the finite-difference phase field)");
    c->pair = on != 0;
    return LB_OK;
}

int lb_get_pairing(const lb_ctx* c, int* on) {
    if (!c || !on) return fail(LB_EINVAL, "lb_get_pairing: NULL argument");
    *on = use_pair(c) ? 1 : 0;
    return LB_OK;
}

int lb_get_tile(const lb_ctx* c, int* ty, int* zc) {
    if (!c || !ty || !zc) return fail(LB_EINVAL, "lb_get_tile: NULL argument");
    *ty = c->ty;
    *zc = c->zc;
    return LB_OK;
}

// Checkpoint layout: header, DevState, the populations of time t (the AA
// array, or the coefficient buffer the next step reads), the D3Q7 buffer of
// time t.
struct CkptHeader {
    char magic[8];  // "LBGBCKP3"
    int nx, ny, nz, storage;
    int phase;      // LB_PHASE_LB or LB_PHASE_WENO5: how the phase buffer is laid out
    int vd;         // density contrasts on (1) or off (0)
    long long t;
    long long f_bytes, g_bytes;
    // the settings the saved run stepped with: density contrasts (rho_l, rho_g,
    // tau_l, tau_g) and buoyancy (g, rho_ref); zero when contrasts are off
    double rho_l, rho_g, tau_l, tau_g, gb[3], rho_ref;
};

static size_t ckpt_f_bytes(const lb_ctx* c) {
    return is_mc(c) ? (size_t)c->N * 10 * sizeof(float) : (size_t)c->N * 27 * c->fsize;
}

// The D3Q7 buffer of time t, or (finite-difference phase field) the buffer
// whose plane 0 holds phi.
static float* g_state(const lb_ctx* c) { return c->fd ? c->g[0] : c->g[c->t & 1]; }
static size_t ckpt_g_bytes(const lb_ctx* c) { return g_buf_bytes(c); }

static char* ckpt_f_ptr(const lb_ctx* c) {
    if (!is_mc(c)) return static_cast<char*>(c->f);
    return static_cast<char*>(c->f) + (size_t)(c->t & 1) * (size_t)c->N * 10 * sizeof(float);
}

size_t lb_state_bytes(const lb_ctx* c) {
    if (!c) return 0;
    return sizeof(CkptHeader) + sizeof(DevState) + ckpt_f_bytes(c) + ckpt_g_bytes(c);
}

int lb_save(lb_ctx* c, void* buf, size_t bytes) {
    if (!c || !buf) return fail(LB_EINVAL, "lb_save: NULL argument");
    if (!c->initialized) return fail(LB_ESTATE, "lb_save before lb_init");
    if (bytes < lb_state_bytes(c)) return fail(LB_EINVAL, "lb_save: buffer of %zu bytes < %zu", bytes, lb_state_bytes(c));
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "LBGBCKP3", 8);
    h.nx = c->nx; h.ny = c->ny; h.nz = c->nz; h.storage = c->storage;
    h.phase = c->fd ? LB_PHASE_WENO5 : LB_PHASE_LB;
    h.vd = c->vd ? 1 : 0;
    if (c->vd) {
        h.rho_l = c->rho_l; h.rho_g = c->rho_g; h.tau_l = c->tau_l; h.tau_g = c->tau_g;
        for (int k = 0; k < 3; ++k) h.gb[k] = c->gb[k];
        h.rho_ref = c->rho_ref;
    }
    h.t = c->t;
    h.f_bytes = (long long)ckpt_f_bytes(c);
    h.g_bytes = (long long)ckpt_g_bytes(c);
    char* p = static_cast<char*>(buf);
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    LB_CUDA(cudaMemcpyAsync(p, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(DevState);
    LB_CUDA(cudaMemcpyAsync(p, ckpt_f_ptr(c), (size_t)h.f_bytes, cudaMemcpyDeviceToHost, c->stream));
    p += h.f_bytes;
    LB_CUDA(cudaMemcpyAsync(p, g_state(c), (size_t)h.g_bytes, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

int lb_load(lb_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf) return fail(LB_EINVAL, "lb_load: NULL argument");
    if (bytes < sizeof(CkptHeader)) return fail(LB_EINVAL, "lb_load: %zu bytes hold no checkpoint", bytes);
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, "LBGBCKP3", 8) != 0) return fail(LB_EINVAL, "lb_load: not a checkpoint of this library");
    // the saved run's physics must be the context's: a state stepped with density
    // contrasts continued without them (or with other ones) would change the flow
    if (h.vd != (c->vd ? 1 : 0))
        return fail(LB_EINVAL, "lb_load: checkpoint %s density contrasts, the context %s", h.vd ? "with" : "without",
                    c->vd ? "has them" : "has none (call lb_set_density first)");
    if (c->vd && (h.rho_l != c->rho_l || h.rho_g != c->rho_g || h.tau_l != c->tau_l || h.tau_g != c->tau_g ||
                  h.gb[0] != c->gb[0] || h.gb[1] != c->gb[1] || h.gb[2] != c->gb[2] || h.rho_ref != c->rho_ref))
        return fail(LB_EINVAL,
                    "lb_load: checkpoint stepped with rho %g/%g, tau %g/%g, g (%g, %g, %g), rho_ref %g; the context "
                    "has other density, viscosity or gravity settings",
                    h.rho_l, h.rho_g, h.tau_l, h.tau_g, h.gb[0], h.gb[1], h.gb[2], h.rho_ref);
    if (h.phase != (c->fd ? LB_PHASE_WENO5 : LB_PHASE_LB))
        return fail(LB_EINVAL, "lb_load: checkpoint of phase solver %d, context uses %d", h.phase,
                    c->fd ? LB_PHASE_WENO5 : LB_PHASE_LB);
    if (h.nx != c->nx || h.ny != c->ny || h.nz != c->nz || h.storage != c->storage)
        return fail(LB_EINVAL, "lb_load: checkpoint of a %dx%dx%d box in storage %d, context is %dx%dx%d in %d", h.nx,
                    h.ny, h.nz, h.storage, c->nx, c->ny, c->nz, c->storage);
    if (h.t < 0 || bytes < lb_state_bytes(c) || h.f_bytes != (long long)ckpt_f_bytes(c) ||
        h.g_bytes != (long long)ckpt_g_bytes(c))
        return fail(LB_EINVAL, "lb_load: truncated or inconsistent checkpoint");
    c->t = h.t;  // selects the buffers the state goes to
    const char* p = static_cast<const char*>(buf) + sizeof(h);
    LB_CUDA(cudaMemcpyAsync(c->st, p, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    p += sizeof(DevState);
    LB_CUDA(cudaMemcpyAsync(ckpt_f_ptr(c), p, (size_t)h.f_bytes, cudaMemcpyHostToDevice, c->stream));
    p += h.f_bytes;
    LB_CUDA(cudaMemcpyAsync(g_state(c), p, (size_t)h.g_bytes, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    c->initialized = true;
    return LB_OK;
}

double lb_bytes_per_site(const lb_ctx* c) {
    if (!c) return 0.0;
    // phase part: D3Q7 read + write, or (finite-difference phase field) phi read + u written
    // (G16: gamma_0..6 and phi~, 2 bytes each, read + write)
    const double ph = c->fd ? 4.0 + 3.0 * 4.0 : is_g16(c) ? 8.0 * 2.0 * 2.0 : 7.0 * 2.0 * 4.0;
    if (is_mc(c)) return 10.0 * 2.0 * 4.0 + ph;
    return 27.0 * 2.0 * (double)c->fsize + ph;
}

int lb_tune(lb_ctx* c, int steps) {
    if (!c) return fail(LB_EINVAL, "ctx is NULL");
    if (steps < 1) return fail(LB_EINVAL, "steps = %d < 1", steps);
    char dev_name[256] = "";
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) snprintf(dev_name, sizeof(dev_name), "%s", prop.name);
    }
    for (char* p = dev_name; *p; ++p)
        if (*p == ' ') *p = '_';
    const char* cache = getenv("LBGB_TUNE_CACHE");
    char key[512];
    snprintf(key, sizeof(key), "%s %d %d %d %d%s%s", dev_name, c->nx, c->ny, c->nz, c->storage, c->vd ? "vd" : "",
             c->fd ? "fd" : "");
    if (cache) {
        FILE* fp = fopen(cache, "r");
        if (fp) {
            char line[640];
            while (fgets(line, sizeof(line), fp)) {
                int ty, zc, pr = 0;
                size_t kl = strlen(key);
                if (strncmp(line, key, kl) == 0 && sscanf(line + kl, " %d %d %d", &ty, &zc, &pr) >= 2 &&
                    (!pr || pair_applies(c)) && check_tile(ty, zc, pr != 0) == LB_OK) {
                    fclose(fp);
                    c->pair = pr != 0;
                    return lb_set_tile(c, ty, zc);
                }
            }
            fclose(fp);
        }
    }
    // Before lb_init the context's own arrays are free: time the shapes on them
    // (zeroed; the step's cost does not depend on the values) so the block
    // counts are those of the real box.  After lb_init, time on a scratch box
    // with this box's nx, ny and min(nz, 128) planes.
    const bool in_place = !c->initialized;
    lb_ctx* s = nullptr;
    float* z = nullptr;
    int rc = LB_OK;
    if (in_place) {
        s = c;
        LB_CUDA(cudaMemsetAsync(c->f, 0, f_bytes(c), c->stream));
        LB_CUDA(cudaMemsetAsync(c->g[0], 0, g_buf_bytes(c), c->stream));
        LB_CUDA(cudaMemsetAsync(c->g[1], 0, g_buf_bytes(c), c->stream));
        LB_CUDA(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
        c->initialized = true;
        c->t = 0;
    } else {
        const int nzt = c->nz < 128 ? c->nz : 128;
        rc = lb_create(c->nx, c->ny, nzt, c->tau, c->M, c->W, c->sigma, &c->force, c->storage, &s);
        if (rc) return rc;
        lb_set_stream(s, c->stream);
        if (c->fd) lb_set_phase_solver(s, LB_PHASE_WENO5);
        if (c->vd) {
            lb_set_density(s, c->rho_l, c->rho_g, c->tau_l, c->tau_g);
            lb_set_gravity(s, c->gb[0], c->gb[1], c->gb[2], c->rho_ref);
        }
        cudaError_t e = cudaMalloc(&z, (size_t)s->N * 4 * sizeof(float));
        if (e != cudaSuccess) {
            lb_destroy(s);
            return fail(LB_ENOMEM, "tune scratch: %s", cudaGetErrorString(e));
        }
        cudaMemsetAsync(z, 0, (size_t)s->N * 4 * sizeof(float), c->stream);
        rc = lb_init(s, z, z + s->N);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // Candidates in a fixed order (tile height 8 first); each is timed as the
    // median of TUNE_WINDOWS windows.  The pick is the first candidate whose
    // median is within TUNE_TIE of the fastest, so shapes that time alike do
    // not trade places from run to run on noise.
    // With a 16-bit storage the paired kernel's shapes (tile heights 8, 4) come
    // first, then the one-site kernel's.
    constexpr int TUNE_WINDOWS = 5;
    constexpr float TUNE_TIE = 0.01f;
    const bool try_pair = pair_applies(s);
    const int kinds[4][2] = {{1, 8}, {1, 4}, {0, 8}, {0, 4}};  // (paired, tile height)
    int cand_ty[30], cand_zc[30], cand_pr[30];
    float cand_ms[30];
    int ncand = 0;
    for (int a = 0; a < 4 && rc == LB_OK; ++a) {
        if (kinds[a][0] && !try_pair) continue;
        s->pair = kinds[a][0] != 0;
        int zcs[6];
        const int nzc = tune_chunks(s, kinds[a][1], zcs);
        for (int b = 0; b < nzc && rc == LB_OK; ++b) {
            if (lb_set_tile(s, kinds[a][1], zcs[b]) != LB_OK) continue;
            if (lb_step(s, 2) != LB_OK) {  // warm-up and graph capture; skip shapes that fail
                cudaGetLastError();
                continue;
            }
            float win[TUNE_WINDOWS];
            int nwin = 0;
            for (int rep = 0; rep < TUNE_WINDOWS; ++rep) {
                cudaEventRecord(e0, c->stream);
                int r2 = lb_step(s, 2 * steps);
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r2 == LB_OK) win[nwin++] = ms;
            }
            if (nwin == 0) continue;
            for (int i = 1; i < nwin; ++i)  // insertion sort of the windows
                for (int j = i; j > 0 && win[j] < win[j - 1]; --j) {
                    const float t = win[j];
                    win[j] = win[j - 1];
                    win[j - 1] = t;
                }
            cand_ty[ncand] = kinds[a][1];
            cand_zc[ncand] = zcs[b];
            cand_pr[ncand] = kinds[a][0];
            cand_ms[ncand] = win[nwin / 2];
            ++ncand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int bty = c->ty, bzc = c->zc, bpr = c->pair ? 1 : 0;
    if (ncand > 0) {
        float best = cand_ms[0];
        for (int k = 1; k < ncand; ++k) best = cand_ms[k] < best ? cand_ms[k] : best;
        for (int k = 0; k < ncand; ++k)
            if (cand_ms[k] <= best * (1.f + TUNE_TIE)) {
                bty = cand_ty[k];
                bzc = cand_zc[k];
                bpr = cand_pr[k];
                break;
            }
    }
    if (in_place) {
        LB_CUDA(cudaStreamSynchronize(c->stream));
        c->initialized = false;  // the timed steps left no usable state
        c->t = 0;
        c->launches = 0;
    } else {
        cudaFree(z);
        lb_destroy(s);
    }
    if (rc) return rc;
    if (cache) {
        FILE* fp = fopen(cache, "a");
        if (fp) {
            fprintf(fp, "%s %d %d %d\n", key, bty, bzc, bpr);
            fclose(fp);
        }
    }
    c->pair = bpr != 0 && pair_applies(c);
    return lb_set_tile(c, bty, bzc);
}

}  // extern "C"
