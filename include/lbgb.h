/*
 * lbgb.h -- C ABI of the GB300 (sm_103a) two-phase lattice Boltzmann library.
 *
 * The library advances one periodic box (or a batch of independent boxes) by
 * the fused per-site time step of accLB (arXiv 2505.01126, Sec. 2):
 *   1. phi = sum_q g_q                  (D3Q7 phase populations)
 *   2. grad phi with the lattice stencil of Sec. 2.3
 *   3. n = grad phi / max(|grad phi|, 1e-10)
 *   4. kappa = div n (same stencil, so phi is read within radius 2)
 *   5. surface tension F^s = -(3W/2) sigma kappa |grad phi| grad phi (Sec. 2.3)
 *   6. external force: none, constant, ABC (Sec. 5.1) or linear A_t u
 *   7. hydrodynamic moments p* = sum f, m = sum f c, Pi = sum f c c (Sec. 2.2)
 *   8. u = (m + (F^s + F^ext)/2) / (1 - A_t/2), F = F^s + F^ext + A_t u
 *   9. a2 = Pi - cs^2 p* I - u u + (u F + F u)/2   (Eq. 8 in closed form)
 *  10. f*_i = w_i [p* + c_i.u/cs^2 + H_i:(u u + (1-omega) a2)/(2 cs^4)] + S_i/2
 *      (Eq. 7 with the Hermite-regularized non-equilibrium; S_i is Eq. 6)
 *  11. g*_q = g_q + omega_phi (g^eq_q - g_q),
 *      g^eq_q = w_q phi (1 + c_q.u/cs7^2) + w_q (M/cs7^2)(4/W) max(phi (1-phi), 0) c_q.n
 *      (D3Q7 BGK whose Chapman-Enskog limit is the Allen-Cahn Eq. 4, D = M;
 *      the interface indicator phi (1-phi) is taken as 0 where phi overshoots [0, 1])
 *  12. streaming f_i(x + c_i) <- f*_i, g_q(x + c_q) <- g*_q, periodic
 *  13. FP64 reductions Phi = sum phi, K = 1/2 sum |u|^2,
 *      eps = 2 nu sum S:S with S = -a2/(2 cs^2 tau), max|u|, and the next
 *      linear-forcing amplitude A_{t+1} = [eps + (K_target - K)/T_relax]/(2K).
 * D3Q27: cs^2 = 1/3, weights 8/27, 2/27, 1/54, 1/216.  D3Q7: cs7^2 = 1/4,
 * weights 1/4 (rest), 1/8.  nu = cs^2 (tau - 1/2) (Sec. 2.2).
 *
 * Conventions for every call:
 *  - Fields are FP32 structure-of-arrays over the site index
 *    s = x + nx*(y + ny*z) (x fastest); a vector field is three consecutive
 *    planes (ux | uy | uz), 3*N floats.  N = nx*ny*nz < 2^31 - 1.
 *  - Field pointers may be host or device memory (the library asks the CUDA
 *    runtime which); they are borrowed for the duration of the call only and
 *    never freed by the library.  Device pointers must belong to the current
 *    device.  Host pointers make the call synchronous.
 *  - Every call that can fail returns LB_OK (0) or a negative LB_E* code and
 *    records a message for lb_last_error().  No exception, trap or device
 *    assert crosses the ABI.
 *  - Work is queued on the context's stream (default: the legacy default
 *    stream; see lb_set_stream).  lb_step is asynchronous.
 */
#ifndef LBGB_H
#define LBGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ return codes */
#define LB_OK 0
#define LB_EINVAL (-1)     /* invalid argument (sizes, parameters, NULL, state) */
#define LB_ENOMEM (-2)     /* device allocation failed */
#define LB_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define LB_ENONFINITE (-4) /* a NaN/Inf was seen by the step's reductions */
#define LB_ESTATE (-5)     /* call out of order (e.g. lb_step before lb_init) */

/* ---------------------------------------------------- population storage */
/* The first three hold the shifted population delta_i = (f_i - w_i)/w_i, 27
 * planes updated in place with the AA access pattern.  LB_F32_MOMENTS holds no
 * populations: each site keeps the ten FP32 coefficients of its post-collision
 * population, a quadratic polynomial in c_i fixed by p*, u, a2 and F (Eq. 7,
 * the reconstruction from macroscopic fields of the thread-safe scheme,
 * Sec. 3), in two buffers; a step rebuilds f_i(x) from the coefficients of the
 * neighbour x - c_i.  It computes the same FP32 numbers as LB_F32 and moves
 * 136 instead of 272 bytes per site and step.  In these four the D3Q7
 * populations g are FP32.  The last two store g in 16 bits as well, shifted so
 * that both bulk phases are near zero: gamma_q = g_q/w_q - phi~, phi~ the
 * phase field of the step before at the site that reads g_q (the D3Q7
 * population of Eq. 4 streamed into it), rounded to the same 16-bit type and
 * kept as an eighth plane; 140 bytes per site and step.  They need nx % 4 == 0
 * and exclude density contrasts and the WENO-5 phase field.  In all six the
 * arithmetic is FP32. */
#define LB_F32 0          /* delta_i stored as FP32 */
#define LB_F16_SHIFTED 1  /* delta_i stored as FP16 */
#define LB_BF16_SHIFTED 2 /* delta_i stored as BF16 */
#define LB_F32_MOMENTS 3  /* post-collision coefficients, FP32 */
#define LB_F16_SHIFTED_G16 4  /* delta_i and gamma_q (and phi~) stored as FP16 */
#define LB_BF16_SHIFTED_G16 5 /* delta_i and gamma_q (and phi~) stored as BF16 */

/* ------------------------------------------------------------ forcing */
#define LB_FORCE_NONE 0
#define LB_FORCE_CONST 1  /* F^ext = g (uniform body force) */
#define LB_FORCE_ABC 2    /* F^ext = A (sin kz + cos ky, sin kx + cos kz, sin ky + cos kx), Sec. 5.1 */
#define LB_FORCE_LINEAR 3 /* F^ext = A_t u with the kinetic-energy controller of step 13 */

typedef struct lb_force {
    int kind;        /* LB_FORCE_* */
    double g[3];     /* LB_FORCE_CONST: force per site, lattice units */
    double A;        /* LB_FORCE_ABC: amplitude */
    double kf;       /* LB_FORCE_ABC: wavenumber in radians per lattice spacing */
    double K_target; /* LB_FORCE_LINEAR: target K = 1/2 sum |u|^2; <= 0 takes the K of lb_init's u */
    double T_relax;  /* LB_FORCE_LINEAR: relaxation time of the controller in steps (> 0) */
} lb_force;

typedef struct lb_ctx lb_ctx;

/*
 * lb_create -- allocate a periodic nx*ny*nz box on the current CUDA device.
 *   tau    hydrodynamic relaxation time, > 1/2 (Sec. 2.2: nu = (tau - 1/2)/3)
 *   M      phase-field mobility D = M of Eq. 4, > 0 (omega_phi = 1/(4M + 1/2))
 *   W      interface width delta of Eq. 4, > 0; +INFINITY switches the
 *          sharpening flux off (then sigma must be 0)
 *   sigma  surface tension, >= 0
 *   force  NULL for no external force
 *   storage  LB_F32, LB_F16_SHIFTED, LB_BF16_SHIFTED, LB_F32_MOMENTS,
 *            LB_F16_SHIFTED_G16 or LB_BF16_SHIFTED_G16
 * The context owns the populations (f: 27 planes, in place with the AA access
 * pattern, or two buffers of 10 coefficient planes; g: two buffers of 7
 * planes), the reduction scratch and the device state.  Sizes: 1 <= nx, ny, nz and nx*ny*nz < 2^31 - 1 (1024^3 fits).
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA; *out is set to NULL on error.
 */
int lb_create(int nx, int ny, int nz, double tau, double M, double W, double sigma,
              const lb_force* force, int storage, lb_ctx** out);

/* Use `stream` (a cudaStream_t, e.g. torch.cuda.Stream.cuda_stream) for all
 * later work of this context; NULL selects the legacy default stream. */
int lb_set_stream(lb_ctx* ctx, void* stream);

/*
 * lb_init -- set the state at t = 0 from phi (N floats) and u (3N floats):
 * n from phi (steps 2-3), f_i = f^eq_i(p* = 1, u), g_q = g^eq_q(phi, u, n).
 * u is the physical velocity.  Resets t, the forcing amplitude (A_0 = 0) and,
 * for LB_FORCE_LINEAR with K_target <= 0, sets K_target = 1/2 sum |u|^2 (FP64).
 */
int lb_init(lb_ctx* ctx, const float* phi, const float* u);

/*
 * lb_set_density -- density and viscosity contrasts (Sec. 2.3, after Fakhari
 * et al. 2017).  From the next step on, the mixture density and the relaxation
 * time follow phi linearly,
 *   rho = rho_g + phi (rho_l - rho_g),  tau = tau_g + phi (tau_l - tau_g),
 * (phi = 1 is the liquid, phi = 0 the gas; tau of lb_create is no longer used)
 * and the total force F = F^s + F^ext + F^p + F^nu enters the velocity, the
 * Guo source and a2 as the acceleration F/rho, with
 *   F^p  = -(p* - 1) cs^2 grad rho   (the pressure measured from its rest value),
 *   F^nu = -(1 - omega/2) [Pi - Pi^eq] grad rho,  omega = 1/tau of the site,
 * Pi the second moment of the pre-collision populations and Pi^eq that of the
 * equilibrium at the velocity without F^nu's own half-force.  The external
 * force of lb_force is a force density.  eps in lb_diagnostics sums each
 * site's own nu.  lb_moments still returns p* as rho; the pressure is
 * p = p* rho(phi) cs^2.  Put the denser phase at phi = 1: the phase-field step
 * overshoots phi slightly above 1 but not below 0, and an overshoot into a light
 * phase at phi = 1 drives rho(phi) towards 0 (such runs blow up within tens of
 * steps at ratio 10).  Every storage supports it; it stays on for the life
 * of the context (a checkpoint records these parameters, and lb_load accepts
 * it only into a context with the same ones: set them before loading).
 * Errors: LB_EINVAL unless rho_l, rho_g > 0 and tau_l, tau_g > 1/2 (finite).
 */
int lb_set_density(lb_ctx* ctx, double rho_l, double rho_g, double tau_l, double tau_g);

/*
 * lb_set_phase_solver -- how the phase field advances (Sec. 2.1.1, Eq. 4):
 *   LB_PHASE_LB     the D3Q7 lattice Boltzmann model (default);
 *   LB_PHASE_WENO5  Eq. 4 by finite differences: the advection in flux form
 *                   div(phi u) with WENO-5 face values (Jiang and Shu), the
 *                   diffusion D lap(phi) and the sharpening
 *                   -kappa div(max(phi (1 - phi), 0) n) with the lattice
 *                   stencils of Sec. 2.3 (D = M, kappa = 4M/W), and the
 *                   three-stage SSP Runge-Kutta scheme in time with u held at
 *                   the step's forced velocity.
 * With LB_PHASE_WENO5 phi is stored as one field (the D3Q7 buffers hold phi,
 * the two Runge-Kutta stages and the velocity), each step launches the fused
 * kernel (which reads phi and writes u), three stage kernels and the
 * reduction.  Call before lb_init (LB_ESTATE after it, unless the solver does
 * not change).  Every storage, density contrasts and checkpoints support it.
 * Errors: LB_EINVAL for an unknown solver.
 */
#define LB_PHASE_LB 0
#define LB_PHASE_WENO5 1
int lb_set_phase_solver(lb_ctx* ctx, int solver);

/*
 * lb_set_gravity -- buoyancy (the rising bubbles of Sec. 5.2) with density
 * contrasts on: from the next step the force density gains
 *   F^b = (rho(phi) - rho_ref) g,  g = (gx, gy, gz).
 * In a periodic box gravity must be balanced by a mean pressure gradient; the
 * paper does not say how, so the caller passes rho_ref.  The mean density of
 * the initial field makes the total buoyancy force zero (it stays zero: sum
 * phi is conserved).  The step does not conserve momentum exactly across a
 * density gradient (O(dx^2) in the lattice product rule), so buoyant layers
 * drift slowly (2% of g at a W = 4 interface, ratio 10).  g = 0 switches it off.
 * Errors: LB_ESTATE before lb_set_density; LB_EINVAL for non-finite arguments.
 */
int lb_set_gravity(lb_ctx* ctx, double gx, double gy, double gz, double rho_ref);

/* lb_step -- advance n >= 0 full time steps (steps 1-13), asynchronously.
 * Runs of two or more steps replay a captured CUDA graph. */
int lb_step(lb_ctx* ctx, int n);

/*
 * lb_moments -- fields at the current time t: rho = p* = sum f (N floats),
 * u = the forced velocity of step 8 (3N floats), phi = sum g (N floats).
 * Any output may be NULL.  Waits for completion when an output is host memory.
 */
int lb_moments(lb_ctx* ctx, float* rho, float* u, float* phi);

/*
 * lb_diagnostics -- FP64 reductions of the most recent step (of lb_init's
 * fields before the first step): out = {Phi, K, eps, max|u|, A_next}.
 * Synchronises the context's stream.  Returns LB_ENONFINITE (out still
 * filled) if any step since lb_init met a NaN or Inf.
 */
int lb_diagnostics(lb_ctx* ctx, double out[5]);

/* Wait for the context's queued work; LB_ECUDA if a kernel failed. */
int lb_sync(lb_ctx* ctx);

/* Steps taken since lb_init. */
long long lb_time(const lb_ctx* ctx);

/* Launch shape of the fused step kernel: tile height ty (x tile is 32 sites)
 * in {4, 8} and z-chunk zc >= 1 planes per block.  Takes effect at the
 * next lb_step; lb_tune picks it by measurement. */
int lb_set_tile(lb_ctx* ctx, int ty, int zc);
int lb_get_tile(const lb_ctx* ctx, int* ty, int* zc);

/*
 * lb_set_pairing -- which kernel runs the step of the FP16 and BF16 storages.
 * on = 1 (the default where it applies): the paired kernel, in which each
 * thread owns two x-adjacent sites, evaluates steps 4-13 for both with packed
 * two-lane FP32 instructions (sm_100's FADD2 / FMUL2 / FFMA2: one instruction,
 * two IEEE-rounded FP32 results) and loads and stores the two sites' stored
 * populations as one 32-bit pair wherever their AA slots are adjacent (every
 * direction at even t, those with c_x = 0 at odd t).  These storages are
 * bound by instruction issue, which this halves for the arithmetic.  on = 0:
 * one site per thread, as for every other storage.  The two compute the same
 * formulas in FP32; their results agree to FP32 rounding, not bit for bit.
 * The paired kernel applies to FP16/BF16 storage with nx % 4 == 0: with the
 * D3Q7 phase field, with or without density contrasts (lb_set_density), and
 * with the WENO-5 phase field (lb_set_phase_solver) without them; the two
 * together run the one-site kernel.
 * lb_get_pairing reports whether the paired kernel runs the step.
 * Errors: LB_EINVAL for on = 1 where the paired kernel does not apply.
 */
int lb_set_pairing(lb_ctx* ctx, int on);
int lb_get_pairing(const lb_ctx* ctx, int* on);

/*
 * lb_tune -- time tile heights ty in {8, 4} with z-chunks zc in {16, 32, 64,
 * 128} and the two chunkings whose block count best fills the last wave of
 * resident blocks (with FP16/BF16 storage first the paired kernel's heights
 * 8, 4, then the one-site kernel's), each as the median of five windows of
 * 2*steps steps, and keep the first shape in that order whose median is within
 * 1% of the fastest (so shapes that time alike do not trade places on noise).  Before lb_init it times on the context's own
 * arrays, so the timed launches have the real box's block counts, and leaves
 * the context uninitialised; after lb_init it times on a scratch box with this
 * box's nx, ny, storage and min(nz, 128) planes, allocated and freed here,
 * and leaves the state untouched.  Results are cached per (device name, nx,
 * ny, nz, storage, density contrasts on or off, phase solver), with the
 * pairing choice, in the file named by LBGB_TUNE_CACHE, if set.
 */
int lb_tune(lb_ctx* ctx, int steps);

/*
 * Checkpoint / restart.  lb_save copies the complete state of time t to host
 * memory: a header (sizes, storage, phase solver, t, and the density,
 * viscosity and gravity settings of lb_set_density / lb_set_gravity), the device state
 * (forcing amplitude and target, last diagnostics, non-finite flag), the
 * populations of time t (the AA array, or the moment-only coefficients the
 * next step reads) and the D3Q7 populations of time t (with LB_PHASE_WENO5:
 * the buffer holding phi).  lb_load restores it into a context of the same
 * sizes, storage, phase solver and density, viscosity and gravity settings
 * (initialised or not; call lb_set_density and lb_set_gravity as on the saving
 * context before lb_load), after which lb_step continues
 * exactly as the saved run would have: the results are bitwise those of an
 * uninterrupted run.  Both calls are synchronous on the context's stream.
 *   buf    host memory of at least lb_state_bytes(ctx) bytes (pinned memory
 *          makes the copies faster); caller-owned
 * Errors: LB_EINVAL (NULL, short buffer, foreign checkpoint, or one whose sizes,
 * storage, phase solver or density/gravity settings differ from the context's),
 * LB_ESTATE (lb_save before lb_init), LB_ECUDA.
 */
size_t lb_state_bytes(const lb_ctx* ctx);
int lb_save(lb_ctx* ctx, void* buf, size_t bytes);
int lb_load(lb_ctx* ctx, const void* buf, size_t bytes);

/* Algorithmic bytes moved per site per step by the fused kernel (population
 * reads and writes): 27*2*sizeof(f) + 7*2*sizeof(g), or 10*2*4 + 7*2*4 for
 * LB_F32_MOMENTS, or 27*2*2 + 8*2*2 = 140 for the 16-bit D3Q7 storages (gamma
 * and phi~); with LB_PHASE_WENO5 the 7*2*4 of g become 4 + 3*4 (phi read,
 * u written; the three stage kernels move 3*(4 + 3*4 + 4) + 2*4 = 68 more). */
double lb_bytes_per_site(const lb_ctx* ctx);

/* Free everything the context owns.  NULL is ignored. */
void lb_destroy(lb_ctx* ctx);

/*
 * lb_velocity_statistics -- statistics of homogeneous isotropic turbulence
 * (Sec. 5.1) of a periodic velocity field, computed on the device.
 *   u        device array of 3N floats, planes u_x | u_y | u_z (the layout
 *            lb_moments writes), N = nx*ny*nz < 2^31 - 1; caller-owned, read only
 *   rmax     structure functions for r = 1 .. rmax (0: none; at most 65535)
 *   nbins    histogram bins (0: no histogram; at most 8192)
 *   range    histogram range [-range, range) in units of `scale` (> 0 if nbins > 0)
 *   scale    bin unit: > 0 as given, <= 0 the RMS gradient sqrt(M2)
 *   stream   cudaStream_t (NULL: legacy default stream); the call returns
 *            when its results are on the host
 *   out      host, 5 + 2*rmax doubles: M2, M3, M4, the skewness S and the
 *            flatness F, then S_2(1..rmax), then S_3(1..rmax)
 *   hist     host, nbins + 2 counts (NULL allowed when nbins == 0): the bins,
 *            then the samples below and above the range
 * The samples are the longitudinal gradients g = d_a u_a, a = x, y, z, at
 * every site (3N samples), with the lattice gradient of Sec. 2.3 evaluated in
 * FP32 with each operation rounded on its own; M_n is the mean of g^n (FP32
 * per-thread sums, FP64 across threads); S = M3 / M2^(3/2) and F = M4 / M2^2
 * are formed in FP64 on the device (NaN when M2 = 0).  Sample g falls in bin
 * floor((g * (1/scale) + range) * (nbins / (2 range))), evaluated in FP64.
 * S_n(r) is the mean over a and sites of (u_a(x + r e_a) - u_a(x))^n (FP32
 * differences and per-thread sums, FP64 across threads).  Scratch memory is
 * allocated and freed here.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA.
 */
int lb_velocity_statistics(const float* u, int nx, int ny, int nz, int rmax, int nbins, double range, double scale,
                           void* stream, double* out, unsigned long long* hist);

/*
 * lb_spectrum -- shell spectrum of a periodic cubic field (the energy and
 * pressure spectra of Sec. 5.1), computed on the device.
 *   f       device array of ncomp * n^3 floats (ncomp = 1 .. 3 component
 *           planes, x fastest); caller-owned, read only
 *   n       edge of the cubic box, n^3 < 2^31 - 1
 *   kmax    last shell (shells 0 .. kmax; at most 6143)
 *   stream  cudaStream_t (NULL: legacy default stream); the call returns when
 *           the result is on the host
 *   out     host, kmax + 1 doubles: E(k) = 1/2 sum over the components and the
 *           integer wavevectors m with round(|m|) = k of |f_hat(m)|^2, with
 *           f_hat = FFT(f) / n^3.  For a velocity field the shells sum to the
 *           mean kinetic energy per site (Parseval) once kmax >= sqrt(3) n/2;
 *           for the pressure pass p = p^* c_s^2 from lb_moments (one component).
 * The FFT is cuFFT's single-precision R2C; shell sums are FP64 (per-block
 * shared-memory sums, then a fixed-order sum over blocks).  Scratch is
 * allocated and freed here.  Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA.
 */
int lb_spectrum(const float* f, int ncomp, int n, int kmax, void* stream, double* out);

/*
 * lb_measure_fp32_peak -- the FP32 throughput this device sustains, measured:
 * a grid filling every SM (64 resident warps each) runs independent FP32
 * fused multiply-add chains for about 10 ms (best of three timed launches
 * after one warm-up, CUDA events on `stream`, NULL: the legacy default
 * stream), once as scalar FMAs and once as packed two-lane FMAs (__ffma2_rn,
 * two FP32 FMAs per instruction).  The roofline of the kernels that are bound
 * by instruction issue rather than HBM (the 16-bit and moment-only storages,
 * the finite-difference stages) is taken against it.  Not part of the method
 * (the paper has no counterpart).
 *   out  host, 6 doubles: FP32 FLOP/s with scalar FMAs (2 per FMA), scalar FMA
 *        warp-instructions issued per second (one per scheduler and cycle at
 *        most), that kernel's time in ms, the SM clock in MHz seen by the first
 *        block (clock64 cycles over the global timer), FP32 FLOP/s with packed
 *        FMAs, packed FMA warp-instructions per second
 * Allocates and frees a few bytes of device memory.  Errors: LB_EINVAL,
 * LB_ENOMEM, LB_ECUDA.
 */
int lb_measure_fp32_peak(void* stream, double out[6]);

/* Message of the last failed call on this thread ("" if none). */
const char* lb_last_error(void);

/* Kernel launches queued by the library since the context was created. */
long long lb_launch_count(const lb_ctx* ctx);

/*
 * Kernel timing.  While on (on != 0), lb_step launches step by step (no
 * graph) and records a CUDA event pair on the context's stream around every
 * fused step kernel.  lb_kernel_time waits for the stream, returns the summed
 * kernel time in milliseconds and the number of timed launches since timing
 * was switched on, and keeps timing on.  Turning timing on again resets both.
 */
int lb_set_timing(lb_ctx* ctx, int on);
int lb_kernel_time(lb_ctx* ctx, double* ms, long long* launches);

/* --------------------------------------------------------- batched ensemble
 * Many independent periodic boxes of uneven sizes advanced together: each step
 * is ONE persistent kernel launch over a work list of (box, tile, z-chunk)
 * items of all boxes, plus one per-box FP64 reduction launch; runs of two or
 * more steps replay a captured CUDA graph.  Every box is computed by the same
 * per-tile code as a single box (lb_step), so its fields are bitwise those of
 * lb_step with the same tile shape and the same kernel (one-site, or paired
 * for FP16/BF16; lb_batch_set_pairing, lb_set_pairing).  No external force
 * (LB_FORCE_NONE).
 */
typedef struct lb_batch lb_batch;

/* count boxes; dims = count triples (nx, ny, nz); tau, M, W, sigma = count
 * values each, with the meaning and limits of lb_create.  The batch owns one
 * population array for all boxes (same storage), two D3Q7 arrays and the
 * reduction scratch.  storage is LB_F32, LB_F16_SHIFTED, LB_BF16_SHIFTED or
 * LB_F32_MOMENTS (the 16-bit D3Q7 storages run single boxes only).
 * Errors: LB_EINVAL (also for LB_F16_SHIFTED_G16 / LB_BF16_SHIFTED_G16),
 * LB_ENOMEM, LB_ECUDA. */
int lb_batch_create(int count, const int* dims, const double* tau, const double* M, const double* W,
                    const double* sigma, int storage, lb_batch** out);
int lb_batch_set_stream(lb_batch* batch, void* stream);
/* State of box `box` at t = 0 from phi (N_box floats) and u (3 N_box floats),
 * host or device; as lb_init.  LB_ESTATE once the batch has stepped. */
int lb_batch_init(lb_batch* batch, int box, const float* phi, const float* u);
/* Advance every box n >= 0 steps; LB_ESTATE until every box is initialised. */
int lb_batch_step(lb_batch* batch, int n);
/* Fields of one box at the current time, as lb_moments. */
int lb_batch_moments(lb_batch* batch, int box, float* rho, float* u, float* phi);
/* FP64 reductions of one box's last step: {Phi, K, eps, max|u|, 0}; syncs. */
int lb_batch_diagnostics(lb_batch* batch, int box, double out[5]);
/* Tile height ty in {4, 8} and z-chunk zc >= 1 of the work items. */
int lb_batch_set_tile(lb_batch* batch, int ty, int zc);
int lb_batch_get_tile(const lb_batch* batch, int* ty, int* zc);
/* Time every tile shape (heights 8 and 4, z-chunks 16 to 128) on the batch's
 * own arrays (zeroed), each as the median of five windows of 2*steps steps, and
 * keep the first shape in that order within 1% of the fastest; call before
 * lb_batch_init (LB_ESTATE otherwise). */
int lb_batch_tune(lb_batch* batch, int steps);
/* Density and viscosity contrasts (Sec. 2.3, as lb_set_density) for every box,
 * each with its own rho_l, rho_g, tau_l, tau_g (count values each; tau of
 * lb_batch_create is then no longer used).  From the next step every box runs
 * the contrast step, in the same persistent launch; the denser phase belongs
 * at phi = 1.  No buoyancy in a batch.
 * Errors: LB_EINVAL unless every rho > 0 and tau > 1/2 (finite). */
int lb_batch_set_density(lb_batch* batch, const double* rho_l, const double* rho_g, const double* tau_l,
                         const double* tau_g);
/* Which tile body runs the batch step of the FP16/BF16 storages: the paired
 * one of lb_set_pairing on tiles 64 (on = 64 or 1, the default where it
 * applies) or 32 sites wide (on = 32, which idles fewer columns on boxes of 24
 * or 48 sites), or one site per thread (on = 0).  The paired body applies when
 * every box has nx % 4 == 0, with or without density contrasts.  lb_batch_tune
 * times all three.  Errors: LB_EINVAL for another value, or a paired body
 * where it does not apply. */
int lb_batch_set_pairing(lb_batch* batch, int on);
/* *on = the paired tile's width (64 or 32) when the paired body runs, else 0 */
int lb_batch_get_pairing(const lb_batch* batch, int* on);
long long lb_batch_sites(const lb_batch* batch);  /* sum of the boxes' sites */
long long lb_batch_time(const lb_batch* batch);   /* steps taken */
void lb_batch_destroy(lb_batch* batch);            /* NULL is ignored */

/*
 * lb_field_stats_static -- FP64 statistics of caller fields without any device
 * allocation.  The paper has no counterpart; this call exists for callers that
 * must not call cudaMalloc: a framework whose caching allocator owns the device
 * memory budget, a latency-critical path where an allocation may synchronise
 * the device, or a plugin that is handed its buffers.
 *   phi    N floats, device memory of the current device (or managed), read only
 *   u      3N floats (ux | uy | uz planes), as phi
 *   stream cudaStream_t for the work, or NULL for the legacy default stream
 *   out    5 doubles: {Phi = sum phi, K = 1/2 sum |u|^2, 0, max|u|, 0}, the
 *          numbers lb_diagnostics reports right after lb_init with these
 *          fields.  Host memory: the call waits for the result.  Device
 *          memory (of the current device): the result is written in stream
 *          order and the call returns at once, with no non-finite report (a
 *          NaN or Inf in the fields shows as a non-finite Phi or K).
 * Scratch is a file-scope __device__ array of LB_STATIC_MAX_BLOCKS * 5 doubles
 * (1.25 MiB), which every device that loads the library holds until the process
 * exits.  A box needs ceil(nx/32)*ceil(ny/8)*ceil(nz/32) records; larger boxes
 * (beyond 640^3 for a cube) are rejected with LB_EINVAL.  The first call on a
 * device looks up the array's device address, so make that first call before
 * any stream capture.  All calls on a device share the array: calls that
 * overlap on the GPU (e.g. on two streams) race.
 * Errors: LB_EINVAL (NULL, sizes, phi/u/out in host memory or in another
 * device's memory), LB_ECUDA, LB_ENONFINITE (a NaN or Inf in phi or u; host out
 * only, out still filled).
 */
#define LB_STATIC_MAX_BLOCKS 32768
int lb_field_stats_static(const float* phi, const float* u, int nx, int ny, int nz, void* stream,
                          double out[5]);

#ifdef __cplusplus
}
#endif
#endif /* LBGB_H */
