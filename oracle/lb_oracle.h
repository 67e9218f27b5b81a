/*
 * lb_oracle.h -- plain FP64 CPU oracle of the two-phase lattice Boltzmann step
 * (conservative Allen-Cahn phase field + regularized D3Q27 hydrodynamics with
 * Guo forcing, accLB, arXiv 2505.01126, Sec. 2).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant with the CUDA library under paper_2505_01126_gb300/.
 *
 * All arrays are host FP64, structure-of-arrays, site index
 * s = x + nx*(y + ny*z), periodic in every axis.  Vector fields are stored as
 * consecutive planes (component c at offset c*N).
 */
#ifndef LB_ORACLE_H
#define LB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_state orc_state;

enum { ORC_FORCE_NONE = 0, ORC_FORCE_CONST = 1, ORC_FORCE_ABC = 2, ORC_FORCE_LINEAR = 3 };

/* Creates a state.  W may be +inf (no interface sharpening); sigma 0 disables
 * surface tension.  regularize=1 is the method (Sec. 2.2, Hermite-regularized
 * non-equilibrium); regularize=0 keeps the full non-equilibrium part in Eq. 7
 * (used only by tests that check Eq. 5 <=> Eq. 7).  Returns NULL on bad input. */
orc_state* orc_create(int nx, int ny, int nz, double tau, double M, double W, double sigma,
                      int force_kind, const double g_const[3], double A_abc, double kf,
                      double K_target, double T_relax, int regularize);
void orc_destroy(orc_state* s);
void orc_set_threads(int n);            /* OpenMP threads for per-site loops */
int  orc_threads(void);

/* phi: N values, u: 3N (ux | uy | uz planes).  Sets f = f^eq(p*=1,u), g = g^eq(phi,u,n). */
int  orc_init(orc_state* s, const double* phi, const double* u);
int  orc_step(orc_state* s, int n);
/* Moments of the current state: rho (= p*), u (forced velocity, 3N), phi. */
void orc_moments(orc_state* s, double* rho, double* u, double* phi);
/* Reductions of the last step: Phi, K, eps, max|u|, A for the next step. */
void orc_diagnostics(const orc_state* s, double out[5]);
long long orc_time(const orc_state* s);

/* Variable density and viscosity (Sec. 2.3): rho and tau of the phi = 1 and
 * phi = 0 phases, interpolated linearly in phi; adds the pressure and viscous
 * forces F^p, F^nu and divides the force by rho in the source.  rho_l = rho_g
 * = 1 with tau_l = tau_g = tau reproduces the density-ratio-1 step exactly.
 * Returns -1 on bad input. */
int  orc_set_density(orc_state* s, double rho_l, double rho_g, double tau_l, double tau_g);

/* Buoyancy (Sec. 5.2) with density contrasts on: adds (rho(phi) - rho_ref) g
 * to the force density.  Returns -1 unless orc_set_density was called and the
 * arguments are finite. */
int  orc_set_gravity(orc_state* s, const double g[3], double rho_ref);

/* Phase-field solver: ORC_PHASE_LB (the D3Q7 model, default) or
 * ORC_PHASE_WENO5 (Eq. 4 by finite differences with WENO-5 advection and
 * SSP-RK3 in time).  Call before orc_init.  Returns -1 on bad input. */
#define ORC_PHASE_LB 0
#define ORC_PHASE_WENO5 1
int  orc_set_phase_solver(orc_state* s, int solver);

/* The WENO-5 face value of Jiang and Shu from the five values v[0..4] along
 * the flow (the face lies between v[2] and v[3]). */
double orc_weno5_face(const double v[5]);

/* Raw populations: f is 27N in the oracle's own direction order (see
 * orc_lattice27), g is 7N in the order of orc_lattice7. */
void orc_get_populations(const orc_state* s, double* f, double* g);
int orc_get_phase(const orc_state* s, double* phi);
int orc_set_phase(orc_state* s, const double* phi);
void orc_set_populations(orc_state* s, const double* f, const double* g);
/* Body force F of the last step (3N). */
void orc_last_force(const orc_state* s, double* F);

/* Building blocks, exposed so tests can pin them individually. */
void orc_lattice27(int c[27][3], double w[27]);
void orc_lattice7(int c[7][3], double w[7]);
void orc_gradient(int nx, int ny, int nz, const double* psi, double* grad);
void orc_equilibrium(double p, const double u[3], double feq[27]);
void orc_guo_source(const double u[3], const double F[3], double S[27]);
void orc_regularized_neq(const double a2[6], double fneq[27]);
/* grad phi (3N), n (3N), kappa (N), F^s (3N) of a given phase field; any output may be NULL. */
int  orc_interface(int nx, int ny, int nz, double W, double sigma, const double* phi,
                   double* grad, double* nrm, double* kappa, double* Fs);
void orc_phase_equilibrium(double phi, const double u[3], const double n[3],
                           double sharp, double geq[7]);

#ifdef __cplusplus
}
#endif
#endif
