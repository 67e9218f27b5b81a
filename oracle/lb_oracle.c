/*
 * lb_oracle.c -- plain FP64 CPU oracle of the two-phase lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE.  This is the slow, literal statement of what one time
 * step computes, used to check the CUDA library.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Method: accLB (arXiv 2505.01126), Sec. 2.
 *   - phase field phi: conservative Allen-Cahn equation (Sec. 2.1.1, Eq. 4),
 *     solved here with a D3Q7 BGK lattice Boltzmann model whose equilibrium
 *     carries the sharpening flux (4M/W) phi(1-phi) n as its first moment;
 *   - lattice gradient of Sec. 2.3 (d_a Psi = (1/cs^2) sum_i w_i c_ia Psi(x+c_i))
 *     for grad(phi); the normal n = grad(phi)/|grad(phi)|; the curvature
 *     kappa = div(n) with the same stencil;
 *   - surface tension (Sec. 2.3, after Kim 2005): F^s = -(3W/2) sigma kappa
 *     |grad phi| grad phi;
 *   - hydrodynamics: D3Q27, pressure-based equilibrium (Sec. 2.2), Guo force
 *     (Eq. 6), push form of the collision (Eq. 7) with the non-equilibrium part
 *     rebuilt from the second-order Hermite coefficient (Eq. 8);
 *   - FP64 diagnostics and the linear-forcing amplitude controller;
 *   - optional (orc_set_density): density and viscosity contrasts (Sec. 2.3),
 *     mixture density rho(phi) and relaxation time tau(phi) linear in phi, the
 *     pressure force F^p and the viscous correction F^nu added to the total
 *     force, which enters the velocity, the source and a2 as F/rho; optional
 *     (orc_set_gravity) buoyancy (rho(phi) - rho_ref) g (Sec. 5.2);
 *   - optional (orc_set_phase_solver): Eq. 4 by finite differences, WENO-5
 *     advection (Sec. 2.1.1) and the lattice stencils of Sec. 2.3, in place of
 *     the D3Q7 model.
 *
 * Every stage is a separate loop over all sites writing a full field, in the
 * order of the method.  Two copies of each population set are kept; streaming
 * pushes f*_i(x) into f_new(x + c_i).  Per-site loops may run under OpenMP:
 * every site writes only its own outputs (or its own streamed slots), so the
 * result does not depend on the thread count.  Sums are serial, in site order.
 *
 * Readings of the paper taken here (the CUDA library takes the same ones):
 *   - the equilibrium tanh profile is phi = 1/2 - 1/2 tanh(2(d-R)/W) in the
 *     Euclidean distance d; it is the 1D steady state of Eq. 4 with kappa=4D/W;
 *   - the surface-tension prefactor 3W/2 makes the Laplace jump 2 sigma/R;
 *   - n uses the guard max(|grad phi|, 1e-10);
 *   - the sharpening flux uses max(phi (1-phi), 0) (no flux where phi
 *     overshoots [0, 1]);
 *   - the regularized non-equilibrium is w_i H_i:a2/(2 cs^4) (the printed form
 *     omits w_i and the trace part of H_i);
 *   - u = sum_i f_i c_i + F/2 (the printed sum of S_i vanishes identically);
 *   - linear forcing F = A u, A_{t+1} = [eps_t + (K_target-K_t)/T_relax]/(2K_t);
 *   - density contrasts: F^p = -(p* - 1) cs^2 grad rho (p* measured from its
 *     rest value 1, which the equilibrium here carries); F^nu with the
 *     coefficient nu omega / cs^2 = 1 - omega/2 and f - f^eq taken from the
 *     pre-collision populations, f^eq at the velocity without F^nu's own
 *     half-force; tau (so nu) linear in phi; the body force is a force density
 *     (acceleration F/rho); eps sums each site's own nu;
 *   - buoyancy: the paper does not say how the net force of gravity on a
 *     periodic box is closed; here the caller gives a reference density, and
 *     rho_ref = the mean density makes the total buoyancy force zero.
 */
#include "lb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- lattices */

/* D3Q27 in textbook order: rest, 6 faces, 12 edges, 8 corners; every direction
 * is followed by its opposite, so (1,2), (3,4), ... (25,26) are opposite pairs. */
static const int C27[27][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1},
    {1, 0, -1},  {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
    {-1, 1, 1},  {1, -1, -1}};

/* Weights by the number of non-zero components of c_i: 8/27, 2/27, 1/54, 1/216. */
#define WR (8.0 / 27)
#define WF (2.0 / 27)
#define WE (1.0 / 54)
#define WC (1.0 / 216)
static const double W27[27] = {WR, WF, WF, WF, WF, WF, WF, WE, WE, WE, WE, WE, WE, WE,
                               WE, WE, WE, WE, WE, WC, WC, WC, WC, WC, WC, WC, WC};
static const double CS2 = 1.0 / 3.0; /* D3Q27 speed of sound squared */

/* D3Q7: rest and the 6 faces, opposite pairs (1,2), (3,4), (5,6). */
static const int C7[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                             {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double W7[7] = {1.0 / 4, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8};
static const double CS2_7 = 1.0 / 4.0; /* D3Q7 speed of sound squared */

static const double NORMAL_GUARD = 1e-10;

void orc_lattice27(int c[27][3], double w[27]) {
    for (int i = 0; i < 27; ++i) {
        for (int a = 0; a < 3; ++a) c[i][a] = C27[i][a];
        w[i] = W27[i];
    }
}

void orc_lattice7(int c[7][3], double w[7]) {
    for (int i = 0; i < 7; ++i) {
        for (int a = 0; a < 3; ++a) c[i][a] = C7[i][a];
        w[i] = W7[i];
    }
}

/* ------------------------------------------------------------------- state */

struct orc_state {
    int nx, ny, nz;
    long long N;
    double tau, omega, nu, M, W, sigma, omega_phi, sharp, beta;
    int force_kind;
    double g_const[3], A_abc, kf, K_target, T_relax;
    int regularize;
    double A;       /* linear forcing amplitude used by the next step */
    long long t;    /* steps taken */
    double diag[5]; /* Phi, K, eps, max|u|, A_next of the last step */

    double *f, *fn, *g, *gn;           /* populations, two copies each */
    double *phi, *grad, *nrm, *kappa;  /* phase field and its derivatives */
    double *Fs, *rho, *mom, *Pi;       /* surface force, hydrodynamic moments */
    double *u, *F, *a2;                /* velocity, total force, Hermite coeff. */

    /* variable density and viscosity (Sec. 2.3), off unless orc_set_density */
    int vd;
    double rho_l, rho_g, tau_l, tau_g; /* of the phi = 1 and phi = 0 phases */
    double* om;                        /* per-site relaxation rate 1/tau(phi) */
    double gb[3], rho_ref;             /* buoyancy (rho(phi) - rho_ref) g, off while g = 0 */

    /* phase field by finite differences (Sec. 2.1.1: WENO-5 advection), off
     * unless orc_set_phase_solver; phs is then the state and g is unused */
    int fd;
    double *phs, *ph1, *ph2, *rhs, *wv; /* state, RK3 stages, right-hand side, 3N work */
};

static int g_threads = 0;

void orc_set_threads(int n) { g_threads = n; }

int orc_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static inline int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

static inline long long site(const orc_state* s, int x, int y, int z) {
    return (long long)x + (long long)s->nx * ((long long)y + (long long)s->ny * z);
}

orc_state* orc_create(int nx, int ny, int nz, double tau, double M, double W, double sigma,
                      int force_kind, const double g_const[3], double A_abc, double kf,
                      double K_target, double T_relax, int regularize) {
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || !(M > 0) || !(W > 0) || !(sigma >= 0))
        return NULL;
    if (isinf(W) && sigma > 0) return NULL;
    if (force_kind < ORC_FORCE_NONE || force_kind > ORC_FORCE_LINEAR) return NULL;
    if (force_kind == ORC_FORCE_LINEAR && !(T_relax > 0)) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->N = (long long)nx * ny * nz;
    s->tau = tau;
    s->omega = 1.0 / tau;
    s->nu = CS2 * (tau - 0.5);                /* Sec. 2.2: nu = cs^2 (tau - 1/2) */
    s->M = M; s->W = W; s->sigma = sigma;
    s->omega_phi = 1.0 / (M / CS2_7 + 0.5);  /* M = cs7^2 (tau_phi - 1/2) */
    s->sharp = isinf(W) ? 0.0 : (M / CS2_7) * (4.0 / W);
    s->beta = sigma == 0 ? 0.0 : 1.5 * W * sigma;
    s->force_kind = force_kind;
    for (int a = 0; a < 3; ++a) s->g_const[a] = g_const ? g_const[a] : 0.0;
    s->A_abc = A_abc; s->kf = kf; s->K_target = K_target; s->T_relax = T_relax;
    s->regularize = regularize;
    long long N = s->N;
    s->f = (double*)calloc((size_t)(27 * N), sizeof(double));
    s->fn = (double*)calloc((size_t)(27 * N), sizeof(double));
    s->g = (double*)calloc((size_t)(7 * N), sizeof(double));
    s->gn = (double*)calloc((size_t)(7 * N), sizeof(double));
    s->phi = (double*)calloc((size_t)N, sizeof(double));
    s->grad = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->nrm = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->kappa = (double*)calloc((size_t)N, sizeof(double));
    s->Fs = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->rho = (double*)calloc((size_t)N, sizeof(double));
    s->mom = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->Pi = (double*)calloc((size_t)(6 * N), sizeof(double));
    s->u = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->F = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->a2 = (double*)calloc((size_t)(6 * N), sizeof(double));
    if (!s->f || !s->fn || !s->g || !s->gn || !s->phi || !s->grad || !s->nrm || !s->kappa ||
        !s->Fs || !s->rho || !s->mom || !s->Pi || !s->u || !s->F || !s->a2) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_state* s) {
    if (!s) return;
    free(s->f); free(s->fn); free(s->g); free(s->gn);
    free(s->phi); free(s->grad); free(s->nrm); free(s->kappa);
    free(s->Fs); free(s->rho); free(s->mom); free(s->Pi);
    free(s->u); free(s->F); free(s->a2);
    free(s->om);
    free(s->phs); free(s->ph1); free(s->ph2); free(s->rhs); free(s->wv);
    free(s);
}

long long orc_time(const orc_state* s) { return s->t; }

/* ------------------------------------------------- per-site building blocks */

/* Pressure-based equilibrium (Sec. 2.2):
 * f^eq_i = w_i (p* + c_i.u/cs^2 + (c_ia c_ib - cs^2 d_ab) u_a u_b / (2 cs^4)). */
void orc_equilibrium(double p, const double u[3], double feq[27]) {
    for (int i = 0; i < 27; ++i) {
        double cu = 0, Huu = 0;
        for (int a = 0; a < 3; ++a) cu += C27[i][a] * u[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Huu += (C27[i][a] * C27[i][b] - (a == b ? CS2 : 0.0)) * u[a] * u[b];
        feq[i] = W27[i] * (p + cu / CS2 + Huu / (2 * CS2 * CS2));
    }
}

/* Guo forcing term, Eq. 6: S_i = w_i ((c_ia - u_a)/cs^2 + (c_ib u_b) c_ia / cs^4) F_a. */
void orc_guo_source(const double u[3], const double F[3], double S[27]) {
    for (int i = 0; i < 27; ++i) {
        double cu = 0;
        for (int b = 0; b < 3; ++b) cu += C27[i][b] * u[b];
        double acc = 0;
        for (int a = 0; a < 3; ++a)
            acc += ((C27[i][a] - u[a]) / CS2 + cu * C27[i][a] / (CS2 * CS2)) * F[a];
        S[i] = W27[i] * acc;
    }
}

/* Symmetric tensor component (a,b) from storage order xx, yy, zz, xy, xz, yz. */
static inline double sym(const double t[6], int a, int b) {
    if (a == b) return t[a];
    int k = a + b; /* xy -> 1, xz -> 2, yz -> 3 */
    return t[2 + k];
}

/* Regularized non-equilibrium (Sec. 2.2, Hermite reconstruction):
 * f^neq_i = w_i H_i : a2 / (2 cs^4), H_i = c_i c_i - cs^2 I. */
void orc_regularized_neq(const double a2[6], double fneq[27]) {
    for (int i = 0; i < 27; ++i) {
        double Ha = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Ha += (C27[i][a] * C27[i][b] - (a == b ? CS2 : 0.0)) * sym(a2, a, b);
        fneq[i] = W27[i] * Ha / (2 * CS2 * CS2);
    }
}

/* D3Q7 phase-field equilibrium: the zeroth moment is phi, the first moment is
 * phi u + (4M/W) max(phi (1-phi), 0) n, so the Chapman-Enskog limit is Eq. 4
 * with D = M = cs7^2 (tau_phi - 1/2).  sharp = (M/cs7^2)(4/W).
 * phi (1-phi) is Eq. 4's interface indicator, zero in both bulk phases; where
 * numerical overshoot puts phi outside [0, 1] it is taken as 0 (bulk), since
 * the unclamped flux there reverses into -c grad phi/|grad phi|, a normalised
 * diffusion that is ill-conditioned where |grad phi| is small. */
void orc_phase_equilibrium(double phi, const double u[3], const double n[3], double sharp,
                           double geq[7]) {
    double ind = phi * (1 - phi);
    if (ind < 0) ind = 0;
    for (int i = 0; i < 7; ++i) {
        double cu = 0, cn = 0;
        for (int a = 0; a < 3; ++a) {
            cu += C7[i][a] * u[a];
            cn += C7[i][a] * n[a];
        }
        geq[i] = W7[i] * phi * (1 + cu / CS2_7) + W7[i] * sharp * ind * cn;
    }
}

/* Periodic neighbour coordinate tables: nb[c+1][x] = (x + c) mod n, c in {-1,0,1}. */
static int* neighbour_table(int n) {
    int* t = (int*)malloc((size_t)(3 * n) * sizeof(int));
    for (int c = -1; c <= 1; ++c)
        for (int x = 0; x < n; ++x) t[(c + 1) * n + x] = wrap(x + c, n);
    return t;
}

/* Lattice gradient (Sec. 2.3): d_a Psi(x) = (1/cs^2) sum_i w_i c_ia Psi(x + c_i),
 * summed over the 13 opposite pairs (the rest direction has c = 0), periodic. */
void orc_gradient(int nx, int ny, int nz, const double* psi, double* grad) {
    long long N = (long long)nx * ny * nz;
    int* tx = neighbour_table(nx);
    int* ty = neighbour_table(ny);
    int* tz = neighbour_table(nz);
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long long s = (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
                double d[3] = {0, 0, 0};
                for (int i = 1; i < 27; i += 2) {
                    const int* c = C27[i];
                    long long sp = tx[(1 + c[0]) * nx + x] +
                                   (long long)nx * (ty[(1 + c[1]) * ny + y] + (long long)ny * tz[(1 + c[2]) * nz + z]);
                    long long sm = tx[(1 - c[0]) * nx + x] +
                                   (long long)nx * (ty[(1 - c[1]) * ny + y] + (long long)ny * tz[(1 - c[2]) * nz + z]);
                    double diff = psi[sp] - psi[sm];
                    for (int a = 0; a < 3; ++a) d[a] += W27[i] * c[a] * diff;
                }
                for (int a = 0; a < 3; ++a) grad[a * N + s] = d[a] / CS2;
            }
    free(tx); free(ty); free(tz);
}

/* ------------------------------------------------------------ step stages */

/* phi = sum_i g_i (zeroth moment of the phase populations); with the
 * finite-difference phase solver phi is the stored field itself. */
static void stage_phase_field(orc_state* s) {
    long long N = s->N;
    if (s->fd) {
        memcpy(s->phi, s->phs, (size_t)N * sizeof(double));
        return;
    }
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (long long x = 0; x < N; ++x) {
        double p = 0;
        for (int i = 0; i < 7; ++i) p += s->g[i * N + x];
        s->phi[x] = p;
    }
}

/* n = grad phi / max(|grad phi|, 1e-10). */
static void stage_normal(orc_state* s) {
    long long N = s->N;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (long long x = 0; x < N; ++x) {
        double gx = s->grad[x], gy = s->grad[N + x], gz = s->grad[2 * N + x];
        double m = sqrt(gx * gx + gy * gy + gz * gz);
        double d = m > NORMAL_GUARD ? m : NORMAL_GUARD;
        s->nrm[x] = gx / d;
        s->nrm[N + x] = gy / d;
        s->nrm[2 * N + x] = gz / d;
    }
}

/* kappa = div n = d_x n_x + d_y n_y + d_z n_z, each with the lattice gradient. */
static void stage_curvature(orc_state* s) {
    long long N = s->N;
    double* tmp = (double*)malloc((size_t)(3 * N) * sizeof(double));
    for (long long x = 0; x < N; ++x) s->kappa[x] = 0;
    for (int a = 0; a < 3; ++a) {
        orc_gradient(s->nx, s->ny, s->nz, s->nrm + a * N, tmp);
        for (long long x = 0; x < N; ++x) s->kappa[x] += tmp[a * N + x];
    }
    free(tmp);
}

/* Surface tension (Sec. 2.3): F^s = -(3W/2) sigma kappa |grad phi| grad phi. */
static void stage_surface_force(orc_state* s) {
    long long N = s->N;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (long long x = 0; x < N; ++x) {
        double gx = s->grad[x], gy = s->grad[N + x], gz = s->grad[2 * N + x];
        double m = sqrt(gx * gx + gy * gy + gz * gz);
        double c = -s->beta * s->kappa[x] * m;
        s->Fs[x] = c * gx;
        s->Fs[N + x] = c * gy;
        s->Fs[2 * N + x] = c * gz;
    }
}

/* p* = sum_i f_i, m = sum_i f_i c_i, Pi = sum_i f_i c_i c_i (Sec. 2.2). */
static void stage_hydro_moments(orc_state* s) {
    long long N = s->N;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (long long x = 0; x < N; ++x) {
        double p = 0, m[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 27; ++i) {
            double fi = s->f[i * N + x];
            const int* c = C27[i];
            p += fi;
            for (int a = 0; a < 3; ++a) m[a] += fi * c[a];
            P[0] += fi * c[0] * c[0];
            P[1] += fi * c[1] * c[1];
            P[2] += fi * c[2] * c[2];
            P[3] += fi * c[0] * c[1];
            P[4] += fi * c[0] * c[2];
            P[5] += fi * c[1] * c[2];
        }
        s->rho[x] = p;
        for (int a = 0; a < 3; ++a) s->mom[a * N + x] = m[a];
        for (int k = 0; k < 6; ++k) s->Pi[k * N + x] = P[k];
    }
}

/* Velocity-independent part of the external force at site (x,y,z). */
static void external_force(const orc_state* s, int x, int y, int z, double Fe[3]) {
    Fe[0] = Fe[1] = Fe[2] = 0;
    if (s->force_kind == ORC_FORCE_CONST) {
        for (int a = 0; a < 3; ++a) Fe[a] = s->g_const[a];
    } else if (s->force_kind == ORC_FORCE_ABC) {
        /* ABC forcing (Sec. 5.1) */
        double k = s->kf;
        Fe[0] = s->A_abc * (sin(k * z) + cos(k * y));
        Fe[1] = s->A_abc * (sin(k * x) + cos(k * z));
        Fe[2] = s->A_abc * (sin(k * y) + cos(k * x));
    }
}

/* Variable density and viscosity (Sec. 2.3), per site:
 *   rho = rho_g + phi (rho_l - rho_g), grad rho = (rho_l - rho_g) grad phi,
 *   tau = tau_g + phi (tau_l - tau_g) (linear in tau, so in nu), omega = 1/tau;
 *   F^p = -(p* - 1) cs^2 grad rho, the pressure p* measured from its rest value 1
 *         (the equilibrium carries p* = 1 at rest);
 *   F^b = (rho - rho_ref) g, buoyancy (zero unless orc_set_gravity);
 *   u0  = (m + (F^s + F^ext + F^b + F^p)/(2 rho)) / (1 - A/2);
 *   F^nu_a = -(nu omega / cs^2) sum_b [Pi_ab - (p* cs^2 d_ab + u0_a u0_b)] d_b rho,
 *          nu omega / cs^2 = (tau - 1/2) / tau = 1 - omega/2; Pi the second
 *          moment of the pre-collision f, the equilibrium taken at u0 (before
 *          F^nu's own half-force);
 *   u = (m + F/(2 rho)) / (1 - A/2), F = F^s + F^ext + F^b + F^p + F^nu,
 * and the source, the Hermite coefficient and the collision see the
 * acceleration F/rho + A u.  With rho_l = rho_g = 1 and tau_l = tau_g every
 * added term is an exact zero and these are the density-ratio-1 values. */
static void velocity_force_vd(orc_state* s, double A) {
    long long N = s->N;
    const double dr = s->rho_l - s->rho_g, dt = s->tau_l - s->tau_g;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long long i = site(s, x, y, z);
                const double ph = s->phi[i];
                const double rho = s->rho_g + ph * dr;
                const double om = 1.0 / (s->tau_g + ph * dt);
                const double pp = s->rho[i] - 1.0;
                double Fe[3], grho[3], Fo[3], u0[3];
                external_force(s, x, y, z, Fe);
                for (int a = 0; a < 3; ++a) {
                    grho[a] = dr * s->grad[a * N + i];
                    Fo[a] = s->Fs[a * N + i] + Fe[a] + (rho - s->rho_ref) * s->gb[a] - pp * CS2 * grho[a];
                    u0[a] = (s->mom[a * N + i] + 0.5 * Fo[a] / rho) / (1 - 0.5 * A);
                }
                /* Pi - Pi^eq at u0; Pi is stored xx, yy, zz, xy, xz, yz */
                const double p = s->rho[i];
                double Pn[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const int k = a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
                        Pn[a][b] = s->Pi[k * N + i] - ((a == b ? p * CS2 : 0.0) + u0[a] * u0[b]);
                    }
                for (int a = 0; a < 3; ++a) {
                    double Fnu = 0;
                    for (int b = 0; b < 3; ++b) Fnu += Pn[a][b] * grho[b];
                    const double Fa = Fo[a] - (1 - 0.5 * om) * Fnu;
                    const double ua = (s->mom[a * N + i] + 0.5 * Fa / rho) / (1 - 0.5 * A);
                    s->u[a * N + i] = ua;
                    s->F[a * N + i] = Fa / rho + A * ua;
                }
                s->om[i] = om;
            }
}

/* u = sum f c + F/2 with F = F^s + F^ext + A u (linear forcing solved in closed
 * form: u = (m + (F^s + F^ext)/2) / (1 - A/2)). */
static void stage_velocity_force(orc_state* s) {
    long long N = s->N;
    double A = s->force_kind == ORC_FORCE_LINEAR ? s->A : 0.0;
    if (s->vd) {
        velocity_force_vd(s, A);
        return;
    }
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long long i = site(s, x, y, z);
                double Fe[3];
                external_force(s, x, y, z, Fe);
                for (int a = 0; a < 3; ++a) {
                    double Fa = s->Fs[a * N + i] + Fe[a];
                    double ua = (s->mom[a * N + i] + 0.5 * Fa) / (1 - 0.5 * A);
                    s->u[a * N + i] = ua;
                    s->F[a * N + i] = Fa + A * ua;
                }
            }
}

/* Eq. 8: a2_ab = sum_i f^neq_i (c_ia c_ib - cs^2 d_ab), f^neq_i = f_i - f^eq_i + S_i/2. */
static void stage_hermite(orc_state* s) {
    long long N = s->N;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (long long x = 0; x < N; ++x) {
        double u[3] = {s->u[x], s->u[N + x], s->u[2 * N + x]};
        double F[3] = {s->F[x], s->F[N + x], s->F[2 * N + x]};
        double feq[27], S[27];
        orc_equilibrium(s->rho[x], u, feq);
        orc_guo_source(u, F, S);
        double A[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 27; ++i) {
            const int* c = C27[i];
            double fneq = s->f[i * N + x] - feq[i] + 0.5 * S[i];
            A[0] += fneq * (c[0] * c[0] - CS2);
            A[1] += fneq * (c[1] * c[1] - CS2);
            A[2] += fneq * (c[2] * c[2] - CS2);
            A[3] += fneq * c[0] * c[1];
            A[4] += fneq * c[0] * c[2];
            A[5] += fneq * c[1] * c[2];
        }
        for (int k = 0; k < 6; ++k) s->a2[k * N + x] = A[k];
    }
}

/* Eq. 7 (push form): f_i(x + c_i, t+1) = f^eq_i + (1 - omega) f^neq_i + S_i/2. */
static void stage_collide_stream_hydro(orc_state* s) {
    long long N = s->N;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long long k = site(s, x, y, z);
                double u[3] = {s->u[k], s->u[N + k], s->u[2 * N + k]};
                double F[3] = {s->F[k], s->F[N + k], s->F[2 * N + k]};
                double a2[6];
                for (int q = 0; q < 6; ++q) a2[q] = s->a2[q * N + k];
                double feq[27], S[27], fneq[27];
                orc_equilibrium(s->rho[k], u, feq);
                orc_guo_source(u, F, S);
                if (s->regularize) {
                    orc_regularized_neq(a2, fneq);
                } else {
                    for (int i = 0; i < 27; ++i) fneq[i] = s->f[i * N + k] - feq[i] + 0.5 * S[i];
                }
                const double om = s->vd ? s->om[k] : s->omega;
                for (int i = 0; i < 27; ++i) {
                    const int* c = C27[i];
                    long long dst = site(s, wrap(x + c[0], s->nx), wrap(y + c[1], s->ny),
                                         wrap(z + c[2], s->nz));
                    s->fn[i * N + dst] = feq[i] + (1 - om) * fneq[i] + 0.5 * S[i];
                }
            }
    double* t = s->f; s->f = s->fn; s->fn = t;
}

/* D3Q7 BGK: g_i(x + c_i, t+1) = g_i + omega_phi (g^eq_i - g_i). */
static void stage_collide_stream_phase(orc_state* s) {
    long long N = s->N;
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long long k = site(s, x, y, z);
                double u[3] = {s->u[k], s->u[N + k], s->u[2 * N + k]};
                double n[3] = {s->nrm[k], s->nrm[N + k], s->nrm[2 * N + k]};
                double geq[7];
                orc_phase_equilibrium(s->phi[k], u, n, s->sharp, geq);
                for (int i = 0; i < 7; ++i) {
                    const int* c = C7[i];
                    long long dst = site(s, wrap(x + c[0], s->nx), wrap(y + c[1], s->ny),
                                         wrap(z + c[2], s->nz));
                    double gi = s->g[i * N + k];
                    s->gn[i * N + dst] = gi + s->omega_phi * (geq[i] - gi);
                }
            }
    double* t = s->g; s->g = s->gn; s->gn = t;
}

/* ----------------------------------- phase field by finite differences
 * Eq. 4 with the advection in flux form (reading: the printed u.grad phi
 * equals div(phi u) for a solenoidal u; the flux form keeps sum phi exact):
 *   d phi/dt = L(phi) = -div(phi u) + D lap(phi) - kappa_ace div(J),
 *   J = max(phi (1 - phi), 0) n,  n = grad phi / max(|grad phi|, 1e-10),
 * D = M and kappa_ace = 4M/W (the same constants as the D3Q7 model).  The
 * derivatives of the diffusion and sharpening terms use the lattice stencils
 * of Sec. 2.3: grad with (1/cs^2) sum_i w_i c_i Psi(x + c_i), and
 * lap(Psi) = (2/cs^2) sum_i w_i (Psi(x + c_i) - Psi(x)).  The advective flux
 * through the face between x and x + e_a is u_f phi_f with u_f the mean of
 * the two sites' u_a and phi_f the WENO-5 reconstruction of Jiang and Shu
 * (1996) from the five values upwind of the face (smoothness indicators,
 * linear weights 1/10, 6/10, 3/10, epsilon 1e-6, squared).  Time: the
 * three-stage strong-stability-preserving Runge-Kutta scheme of Shu and Osher
 * with u held at its value of step 8 over the step (dt = 1). */

/* WENO-5 value at the face between v0 and v1 for flow from v0 towards v1,
 * from the values vm2, vm1, v0, v1, v2 along the flow. */
static double weno5_face(double vm2, double vm1, double v0, double v1, double v2) {
    const double q0 = (2 * vm2 - 7 * vm1 + 11 * v0) / 6;
    const double q1 = (-vm1 + 5 * v0 + 2 * v1) / 6;
    const double q2 = (2 * v0 + 5 * v1 - v2) / 6;
    const double b0 = 13.0 / 12 * (vm2 - 2 * vm1 + v0) * (vm2 - 2 * vm1 + v0) +
                      0.25 * (vm2 - 4 * vm1 + 3 * v0) * (vm2 - 4 * vm1 + 3 * v0);
    const double b1 = 13.0 / 12 * (vm1 - 2 * v0 + v1) * (vm1 - 2 * v0 + v1) + 0.25 * (vm1 - v1) * (vm1 - v1);
    const double b2 = 13.0 / 12 * (v0 - 2 * v1 + v2) * (v0 - 2 * v1 + v2) +
                      0.25 * (3 * v0 - 4 * v1 + v2) * (3 * v0 - 4 * v1 + v2);
    const double eps = 1e-6;
    const double a0 = 0.1 / ((eps + b0) * (eps + b0));
    const double a1 = 0.6 / ((eps + b1) * (eps + b1));
    const double a2 = 0.3 / ((eps + b2) * (eps + b2));
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

double orc_weno5_face(const double v[5]) { return weno5_face(v[0], v[1], v[2], v[3], v[4]); }

/* L(ph) into out, u = s->u. */
static void phase_rhs(orc_state* s, const double* ph, double* out) {
    long long N = s->N;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const double D = s->M, kap = isinf(s->W) ? 0.0 : 4.0 * s->M / s->W;
    double* J = s->wv;
    /* J = max(ph (1 - ph), 0) n */
    orc_gradient(nx, ny, nz, ph, J);
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (long long x = 0; x < N; ++x) {
        double gx = J[x], gy = J[N + x], gz = J[2 * N + x];
        double m = sqrt(gx * gx + gy * gy + gz * gz);
        double d = m > NORMAL_GUARD ? m : NORMAL_GUARD;
        double w = ph[x] * (1 - ph[x]);
        if (w < 0) w = 0;
        J[x] = w * gx / d;
        J[N + x] = w * gy / d;
        J[2 * N + x] = w * gz / d;
    }
#pragma omp parallel for schedule(static) num_threads(orc_threads())
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long long k = site(s, x, y, z);
                /* div J and lap(ph) with the lattice stencils */
                double divJ = 0, lap = 0;
                for (int i = 1; i < 27; ++i) {
                    const int* c = C27[i];
                    long long q = site(s, wrap(x + c[0], nx), wrap(y + c[1], ny), wrap(z + c[2], nz));
                    for (int a = 0; a < 3; ++a) divJ += W27[i] * c[a] * J[a * N + q];
                    lap += W27[i] * (ph[q] - ph[k]);
                }
                divJ /= CS2;
                lap *= 2 / CS2;
                /* advective flux differences, face by face */
                double adv = 0;
                for (int a = 0; a < 3; ++a) {
                    const int n = a == 0 ? nx : (a == 1 ? ny : nz);
                    const int p = a == 0 ? x : (a == 1 ? y : z);
                    for (int side = 0; side < 2; ++side) {   /* faces p - 1/2 (side 0) and p + 1/2 */
                        const int lo = p - 1 + side;         /* the face lies between lo and lo + 1 */
                        double v[6];                         /* ph at lo - 2 .. lo + 3 along axis a */
                        double ul = 0, ur = 0;
                        for (int j = 0; j < 6; ++j) {
                            int e[3] = {x, y, z};
                            e[a] = wrap(lo - 2 + j, n);
                            v[j] = ph[site(s, e[0], e[1], e[2])];
                        }
                        {
                            int e[3] = {x, y, z};
                            e[a] = wrap(lo, n);
                            ul = s->u[a * N + site(s, e[0], e[1], e[2])];
                            e[a] = wrap(lo + 1, n);
                            ur = s->u[a * N + site(s, e[0], e[1], e[2])];
                        }
                        const double uf = 0.5 * (ul + ur);
                        const double pf = uf >= 0 ? weno5_face(v[0], v[1], v[2], v[3], v[4])
                                                  : weno5_face(v[5], v[4], v[3], v[2], v[1]);
                        adv += (side ? 1.0 : -1.0) * uf * pf;
                    }
                }
                out[k] = -adv + D * lap - kap * divJ;
            }
}

static void stage_phase_fd(orc_state* s) {
    long long N = s->N;
    double *p0 = s->phs, *p1 = s->ph1, *p2 = s->ph2, *L = s->rhs;
    phase_rhs(s, p0, L);
    for (long long x = 0; x < N; ++x) p1[x] = p0[x] + L[x];
    phase_rhs(s, p1, L);
    for (long long x = 0; x < N; ++x) p2[x] = 0.75 * p0[x] + 0.25 * (p1[x] + L[x]);
    phase_rhs(s, p2, L);
    for (long long x = 0; x < N; ++x) p0[x] = p0[x] / 3 + 2.0 / 3 * (p2[x] + L[x]);
}

/* FP64 reductions: Phi = sum phi, K = 1/2 sum |u|^2, eps = 2 nu sum S:S with
 * S = -a2/(2 cs^2 tau) (the Chapman-Enskog estimate of Sec. 2.2), max|u|;
 * then the linear-forcing amplitude for the next step. */
static void stage_diagnostics(orc_state* s) {
    long long N = s->N;
    double Phi = 0, K = 0, SS = 0, umax = 0;
    double scale = 1.0 / (2 * CS2 * s->tau);
    const double nu_g = s->vd ? CS2 * (s->tau_g - 0.5) : s->nu;
    for (long long x = 0; x < N; ++x) {
        Phi += s->phi[x];
        double u2 = s->u[x] * s->u[x] + s->u[N + x] * s->u[N + x] + s->u[2 * N + x] * s->u[2 * N + x];
        K += 0.5 * u2;
        double um = sqrt(u2);
        if (um > umax || um != um) umax = um;
        double ss = 0;
        double A[6];
        for (int q = 0; q < 6; ++q) A[q] = s->a2[q * N + x];
        /* variable viscosity: each site's own tau in S and nu_s in the sum,
         * eps = 2 nu_g sum (nu_s / nu_g) S:S (exactly the single-viscosity sum
         * when tau_l = tau_g = tau) */
        const double tx = s->vd ? s->tau_g + s->phi[x] * (s->tau_l - s->tau_g) : s->tau;
        const double sc = s->vd ? 1.0 / (2 * CS2 * tx) : scale;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double Sab = -sc * sym(A, a, b);
                ss += Sab * Sab;
            }
        SS += s->vd ? (CS2 * (tx - 0.5)) / nu_g * ss : ss;
    }
    double eps = 2 * nu_g * SS;
    double Anext = 0;
    if (s->force_kind == ORC_FORCE_LINEAR && K > 0)
        Anext = (eps + (s->K_target - K) / s->T_relax) / (2 * K);
    s->diag[0] = Phi;
    s->diag[1] = K;
    s->diag[2] = eps;
    s->diag[3] = umax;
    s->diag[4] = Anext;
    s->A = Anext;
}

/* Stages that need only the state at time t: phi, its derivatives, the forces,
 * the moments and the velocity. */
static void prepare(orc_state* s) {
    stage_phase_field(s);
    orc_gradient(s->nx, s->ny, s->nz, s->phi, s->grad);
    stage_normal(s);
    stage_curvature(s);
    stage_surface_force(s);
    stage_hydro_moments(s);
    stage_velocity_force(s);
}

int orc_step(orc_state* s, int n) {
    if (!s || n < 0) return -1;
    for (int k = 0; k < n; ++k) {
        prepare(s);
        stage_hermite(s);
        stage_diagnostics(s);
        stage_collide_stream_hydro(s);
        if (s->fd) stage_phase_fd(s);
        else stage_collide_stream_phase(s);
        s->t += 1;
    }
    return 0;
}

int orc_init(orc_state* s, const double* phi, const double* u) {
    if (!s || !phi || !u) return -1;
    long long N = s->N;
    memcpy(s->phi, phi, (size_t)N * sizeof(double));
    if (s->fd) memcpy(s->phs, phi, (size_t)N * sizeof(double));
    orc_gradient(s->nx, s->ny, s->nz, s->phi, s->grad);
    stage_normal(s);
    for (long long x = 0; x < N; ++x) {
        double ux[3] = {u[x], u[N + x], u[2 * N + x]};
        double n[3] = {s->nrm[x], s->nrm[N + x], s->nrm[2 * N + x]};
        double feq[27], geq[7];
        orc_equilibrium(1.0, ux, feq);
        orc_phase_equilibrium(phi[x], ux, n, s->sharp, geq);
        for (int i = 0; i < 27; ++i) s->f[i * N + x] = feq[i];
        for (int i = 0; i < 7; ++i) s->g[i * N + x] = geq[i];
    }
    if (s->force_kind == ORC_FORCE_LINEAR && !(s->K_target > 0)) {
        double K = 0;
        for (long long x = 0; x < N; ++x)
            K += 0.5 * (u[x] * u[x] + u[N + x] * u[N + x] + u[2 * N + x] * u[2 * N + x]);
        s->K_target = K;
    }
    s->A = 0;
    s->t = 0;
    for (int q = 0; q < 5; ++q) s->diag[q] = 0;
    return 0;
}

void orc_moments(orc_state* s, double* rho, double* u, double* phi) {
    prepare(s);
    long long N = s->N;
    if (rho) memcpy(rho, s->rho, (size_t)N * sizeof(double));
    if (u) memcpy(u, s->u, (size_t)(3 * N) * sizeof(double));
    if (phi) memcpy(phi, s->phi, (size_t)N * sizeof(double));
}

/* phi -> grad phi, n, kappa and F^s (sigma, W as given), through the same stages as
 * the step. */
int orc_interface(int nx, int ny, int nz, double W, double sigma, const double* phi,
                  double* grad, double* nrm, double* kappa, double* Fs) {
    orc_state* s = orc_create(nx, ny, nz, 1.0, 0.1, W, sigma, ORC_FORCE_NONE, NULL, 0, 0, 0, 1, 1);
    if (!s) return -1;
    long long N = s->N;
    memcpy(s->phi, phi, (size_t)N * sizeof(double));
    orc_gradient(nx, ny, nz, s->phi, s->grad);
    stage_normal(s);
    stage_curvature(s);
    stage_surface_force(s);
    if (grad) memcpy(grad, s->grad, (size_t)(3 * N) * sizeof(double));
    if (nrm) memcpy(nrm, s->nrm, (size_t)(3 * N) * sizeof(double));
    if (kappa) memcpy(kappa, s->kappa, (size_t)N * sizeof(double));
    if (Fs) memcpy(Fs, s->Fs, (size_t)(3 * N) * sizeof(double));
    orc_destroy(s);
    return 0;
}

void orc_diagnostics(const orc_state* s, double out[5]) {
    for (int q = 0; q < 5; ++q) out[q] = s->diag[q];
}

int orc_set_density(orc_state* s, double rho_l, double rho_g, double tau_l, double tau_g) {
    if (!s || !(rho_l > 0) || !(rho_g > 0) || !(tau_l > 0.5) || !(tau_g > 0.5)) return -1;
    if (!s->om) {
        s->om = (double*)calloc((size_t)s->N, sizeof(double));
        if (!s->om) return -1;
    }
    s->vd = 1;
    s->rho_l = rho_l; s->rho_g = rho_g; s->tau_l = tau_l; s->tau_g = tau_g;
    return 0;
}

int orc_set_phase_solver(orc_state* s, int solver) {
    if (!s || (solver != ORC_PHASE_LB && solver != ORC_PHASE_WENO5)) return -1;
    if (solver == ORC_PHASE_WENO5 && !s->phs) {
        long long N = s->N;
        s->phs = (double*)calloc((size_t)N, sizeof(double));
        s->ph1 = (double*)calloc((size_t)N, sizeof(double));
        s->ph2 = (double*)calloc((size_t)N, sizeof(double));
        s->rhs = (double*)calloc((size_t)N, sizeof(double));
        s->wv = (double*)calloc((size_t)(3 * N), sizeof(double));
        if (!s->phs || !s->ph1 || !s->ph2 || !s->rhs || !s->wv) return -1;
    }
    s->fd = solver == ORC_PHASE_WENO5;
    return 0;
}

int orc_set_gravity(orc_state* s, const double g[3], double rho_ref) {
    if (!s || !s->vd || !g || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2]) || !isfinite(rho_ref)) return -1;
    for (int a = 0; a < 3; ++a) s->gb[a] = g[a];
    s->rho_ref = rho_ref;
    return 0;
}

void orc_get_populations(const orc_state* s, double* f, double* g) {
    if (f) memcpy(f, s->f, (size_t)(27 * s->N) * sizeof(double));
    if (g) memcpy(g, s->g, (size_t)(7 * s->N) * sizeof(double));
}

void orc_set_populations(orc_state* s, const double* f, const double* g) {
    if (f) memcpy(s->f, f, (size_t)(27 * s->N) * sizeof(double));
    if (g) memcpy(s->g, g, (size_t)(7 * s->N) * sizeof(double));
}

/* The stored phase field of the finite-difference solver (the state when
 * orc_set_phase_solver selected WENO-5); -1 when that solver is not selected.
 * Test access only: the tests round the state to FP32 storage between steps. */
int orc_get_phase(const orc_state* s, double* phi) {
    if (!s->fd) return -1;
    memcpy(phi, s->phs, (size_t)s->N * sizeof(double));
    return 0;
}

int orc_set_phase(orc_state* s, const double* phi) {
    if (!s->fd) return -1;
    memcpy(s->phs, phi, (size_t)s->N * sizeof(double));
    return 0;
}

void orc_last_force(const orc_state* s, double* F) {
    memcpy(F, s->F, (size_t)(3 * s->N) * sizeof(double));
}
