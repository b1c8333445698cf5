/*
 * lbm_oracle.h -- FP64 CPU oracle of the difference-free conservative
 * phase-field lattice Boltzmann method (Zhao, Patel & Lee, arXiv:2407.12263).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path (the
 * CUDA library and its Python binding) never calls it and shares no source
 * with it.
 *
 * Conventions (lattice units): dx = 1, dt = 1 in every collision, moment and
 * forcing formula; the Courant number c enters only the Lax-Wendroff
 * propagation (Sec. 2.2). Fluid 2 (phi = 0) has density 1 and dynamic
 * viscosity eta2 = cs^2 * tau_f; fluid 1 (phi = 1) has density rho_ratio and
 * viscosity mu_ratio * eta2.
 *
 * Storage: populations are planes [Q][nz][ny][nx], x fastest, FP64, in the
 * velocity order of oracle_lattice(). The stored state is the post-collision
 * set f*, g* (Sec. 2.2, Sec. 2.3).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle oracle;

/* Lattice tables: d, e[Q][3], t[Q]. Returns 0, or -1 for an unknown Q. */
int oracle_lattice(int Q, int *d, int *e, double *t);

/* Lax-Wendroff propagation of one population along its link (Sec. 2.2). */
double oracle_lax_wendroff(double c, double at_minus, double at_x, double at_plus);

/* Continuous surface stress Pi_s = sigma |grad phi| (I - n n) (Eq. surface), 3x3 row-major. */
void oracle_css_tensor(int d, double sigma, double grad_norm, const double *n, double *pis);

/* f_i^eq of Eq. geq_s; pis_sign = -1 is the reading this oracle uses, +1 the printed sign. */
void oracle_feq(int Q, double p, double rho, const double *u, const double *pis, int pis_sign,
                double *feq);

/* g_i^eq of Eq. geq; src_scale multiplies t_i e_i.S (tau_phi in the reading used here). */
void oracle_geq(int Q, double phi, const double *u, const double *S, double src_scale,
                double *geq);

/* Compensation forcing S_i (App. A) and body force R_i (Eq. body). */
void oracle_forcing(int Q, double rho, const double *u, const double *grad_rho, const double *G,
                    double *Si, double *Ri);

/* Isotropic central-difference gradient of a periodic field (the finite-difference variant). */
void oracle_isotropic_gradient(int Q, int nx, int ny, int nz, const double *field,
                               double *grad /* 3 planes */);

/* Create / destroy. scheme: 0 = difference-free, 1 = isotropic finite difference.
 * pis_sign, half_force_sign, geq_source_tau select readings of ambiguous
 * passages (defaults -1, +1, 1). Returns NULL on invalid arguments. */
oracle *oracle_create(int Q, int nx, int ny, int nz, double tau_f, double tau_g, double M,
                      double xi, double sigma, double rho_ratio, double mu_ratio,
                      const double *G, double courant, int scheme, int pis_sign,
                      int half_force_sign, int geq_source_tau);
void oracle_destroy(oracle *o);
double oracle_tau_phi(const oracle *o);

/* Walls (bit 0: x, bit 1: y, bit 2: z), half-way between the last cell and the next:
 * bounce-back in the Lax-Wendroff stencil, mirror image for gradients of phi. Returns -1 for
 * an invalid mask. Default 0 (fully periodic). */
int oracle_set_walls(oracle *o, int walls);

/* Macroscopic stage of one cell from its propagated populations fbar, g.
 * fd_grad = NULL selects the moment-based gradient. out receives, packed:
 * phi, rho, u[3], K1[3], n[3], S[3], grad_phi[3], grad_rho[3], p  (21 doubles). */
void oracle_macroscopic_cell(const oracle *o, const double *fbar, const double *g,
                             const double *fd_grad, double *out);

/* Collision of one cell: fbar, g and the packed macroscopic record -> f*, g*. */
void oracle_collide_cell(const oracle *o, const double *fbar, const double *g,
                         const double *macro, double *fstar, double *gstar);

/* Initial post-collision populations from phi0 (N), u0 (3 planes or NULL), p0. */
int oracle_init_phi(oracle *o, const double *phi0, const double *u0, double p0);
/* As oracle_init_phi, with the pressure of f^eq taken per cell from p (N values) when p is not
 * NULL (p0 is then unused): the initial state of the Taylor-Green case of Sec. 3.4, whose
 * pressure field is part of the initial condition. */
int oracle_init_fields(oracle *o, const double *phi0, const double *u0, const double *p, double p0);
int oracle_step(oracle *o, int nsteps);

/* Fields of the propagated current state (what the next collision uses).
 * Any output may be NULL. u, grad_phi and n are 3 planes each. */
int oracle_moments(oracle *o, double *phi, double *p, double *u, double *grad_phi, double *n);
int oracle_mass(oracle *o, double *sum_phi, double *sum_rho_phi);
int oracle_get_pops(const oracle *o, double *f, double *g);
int oracle_set_pops(oracle *o, const double *f, const double *g);
int oracle_num_threads(void);
/* Threads the following oracle calls use (n >= 1; a no-op without OpenMP). Results do not depend
 * on it: every cell writes only its own outputs. */
void oracle_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
