/*
 * lbm_oracle.c -- FP64 CPU oracle of the difference-free conservative
 * phase-field lattice Boltzmann method (Zhao, Patel & Lee, arXiv:2407.12263).
 *
 * TEST INFRASTRUCTURE: plain, slow and written to be checked against the
 * paper by eye. It is loaded only by the test suite, the smoke check and the
 * CPU baseline leg of the benchmark; the CUDA path neither links nor calls it.
 *
 * One time step, for every cell, in the order the paper lists (end of Sec. 2.3):
 *   Lax-Wendroff propagation of f* and g*          (Sec. 2.2, also used for g in Sec. 2.3)
 *   phi = sum g_i, rho = rho1 phi + rho2 (1 - phi) (Sec. 2.3)
 *   rho u = sum fbar_i e_i + rho G / 2             (Eq. momentum, sign reading below)
 *   K1 = sum g_i (e_i - u)                         (Sec. 2.3)
 *   n = -K1 / |K1|                                 (Eq. norm)
 *   S = 4 phi (1 - phi) / delta n                  (Sec. 2.3)
 *   grad phi = (tau_phi cs^2 S - K1) / ((tau_phi + 1/2) cs^2), grad rho = (rho1 - rho2) grad phi
 *   p = cs^2 sum fbar_i + cs^2/2 u . grad rho      (Eq. pressure)
 *   Pi_s = sigma |grad phi| (I - n n)              (Eq. surface)
 *   f^eq (Eq. geq_s), S_i (App. A), R_i (Eq. body), Crank-Nicolson collision (Eq. c-n_m)
 *   g^eq (Eq. geq), Crank-Nicolson collision (Eq. c-n_c)
 * The finite-difference variant replaces K1 -> n -> grad phi by the isotropic
 * central difference of the propagated phi field and n = grad phi / |grad phi| (Sec. 3.4).
 *
 * Readings of passages the paper leaves silent, garbled or inconsistent:
 *   - D2Q9 weights follow the speed of each velocity: 4/9, 1/9 (|e| = 1), 1/36 (|e|^2 = 2).
 *   - 3D runs use D3Q19 (the paper names no 3D lattice).
 *   - Eq. geq_s enters Pi_s with a minus sign (pis_sign = -1), so that the second
 *     moment of f^eq is p I + rho u u - Pi_s as App. A requires.
 *   - Eq. momentum adds rho G / 2 (half_force_sign = +1), consistent with
 *     fbar = f - F/2 and sum_i F_i e_i = rho G.
 *   - The sharpening source in g^eq is tau_phi t_i e_i.S (geq_source_tau = 1), the
 *     scale the gradient formula of Sec. 2.3 and the flux M (grad phi - S) require.
 *   - n = 0 where |K1|^2 <= 1e-24 (or |grad phi|^2 <= 1e-24 in the FD variant).
 *   - dt = 1; the Courant number enters only the propagation.
 *   - M > 0 fixes tau_phi = M / cs^2; otherwise tau_phi = tau_g.
 *   - Local viscosity eta(phi) = eta2 + (eta1 - eta2) phi, tau_rho = eta / (rho cs^2).
 *   - Initial state: f* = f^eq(p0, u0, rho0, Pi_s0) and
 *     g* = g^eq(phi0, u0, S0) - t_i (tau_phi - 1/2) e_i . grad phi0, with grad phi0 the
 *     isotropic central difference of phi0.
 *   - No clamping of phi anywhere.
 *   - Walls (the paper gives no wall treatment; its Rayleigh-Taylor and rising-bubble runs have
 *     walls): a wall lies half-way between the last cell and the next. Where the Lax-Wendroff
 *     stencil of population i reaches across a wall, the value there is the opposite population
 *     of the same cell, f_ibar(x) (half-way bounce-back written for the three-point stencil; at
 *     c = 1 it is the usual bounce-back). The wall-face fluxes of i and ibar then cancel, so
 *     sum phi is conserved. Gradients of phi (initialisation, finite-difference variant) read
 *     the mirror image of the cell across the wall (zero normal gradient).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)
#define NORMAL_GUARD 1e-24

/* ----------------------------------------------------------------------------
 * Lattices. D2Q9 velocities in the paper's order (Sec. 2.2): i = 1..4 along
 * theta = (i-1) pi/2, i = 5..8 along theta = (i-5) pi/2 + pi/4 with length sqrt 2.
 * D3Q19: rest, the six axis directions, the twelve face diagonals.
 * ------------------------------------------------------------------------- */
static const int E_D2Q9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};

static const int E_D3Q19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
    int Q, d;
    int e[19][3];
    double t[19];
} lattice;

static int lattice_setup(int Q, lattice *L)
{
    int i, a;
    if (Q != 9 && Q != 19) return -1;
    L->Q = Q;
    L->d = (Q == 9) ? 2 : 3;
    for (i = 0; i < Q; ++i) {
        int e2 = 0;
        for (a = 0; a < 3; ++a) {
            L->e[i][a] = (Q == 9) ? E_D2Q9[i][a] : E_D3Q19[i][a];
            e2 += L->e[i][a] * L->e[i][a];
        }
        /* weights by speed */
        if (Q == 9) L->t[i] = (e2 == 0) ? 4.0 / 9.0 : (e2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
        else L->t[i] = (e2 == 0) ? 1.0 / 3.0 : (e2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
    }
    return 0;
}

int oracle_lattice(int Q, int *d, int *e, double *t)
{
    lattice L;
    int i, a;
    if (lattice_setup(Q, &L)) return -1;
    *d = L.d;
    for (i = 0; i < Q; ++i) {
        for (a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
        t[i] = L.t[i];
    }
    return 0;
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double edot(const lattice *L, int i, const double *v)
{
    return L->e[i][0] * v[0] + L->e[i][1] * v[1] + L->e[i][2] * v[2];
}

/* ----------------------------------------------------------------------------
 * Lax-Wendroff propagation along link e_i with Courant number c (Sec. 2.2):
 *   fbar(x) = f*(x) - c [f*(x) - f*(x - e)] - c (1 - c)/2 [f*(x + e) - 2 f*(x) + f*(x - e)]
 * ------------------------------------------------------------------------- */
double oracle_lax_wendroff(double c, double at_minus, double at_x, double at_plus)
{
    return at_x - c * (at_x - at_minus) - 0.5 * c * (1.0 - c) * (at_plus - 2.0 * at_x + at_minus);
}

/* Pi_s = sigma |grad phi| (I - n (x) n) in d dimensions (Eq. surface). */
void oracle_css_tensor(int d, double sigma, double grad_norm, const double *n, double *pis)
{
    int a, b;
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            double I_ab = (a == b && a < d) ? 1.0 : 0.0;
            pis[3 * a + b] = (a < d && b < d) ? sigma * grad_norm * (I_ab - n[a] * n[b]) : 0.0;
        }
}

/* f_i^eq = t_i ( p/cs^2 + rho (e.u/cs^2 + (e.u)^2/(2 cs^4) - |u|^2/(2 cs^2))
 *               + sign/(2 cs^4) Pi_s : (e e - cs^2 I) )              (Eq. geq_s) */
void oracle_feq(int Q, double p, double rho, const double *u, const double *pis, int pis_sign,
                double *feq)
{
    lattice L;
    int i, a, b;
    lattice_setup(Q, &L);
    for (i = 0; i < Q; ++i) {
        double eu = edot(&L, i, u), uu = dot3(u, u), contraction = 0.0;
        for (a = 0; a < L.d; ++a)
            for (b = 0; b < L.d; ++b) {
                double eeab = (double)L.e[i][a] * L.e[i][b] - ((a == b) ? CS2 : 0.0);
                contraction += pis[3 * a + b] * eeab;
            }
        feq[i] = L.t[i] * (p / CS2 + rho * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)) +
                           (double)pis_sign / (2.0 * CS2 * CS2) * contraction);
    }
}

/* g_i^eq = t_i phi [1 + e.u/cs^2 + (e.u)^2/(2 cs^4) - |u|^2/(2 cs^2)] + scale t_i e_i . S  (Eq. geq) */
void oracle_geq(int Q, double phi, const double *u, const double *S, double src_scale, double *geq)
{
    lattice L;
    int i;
    lattice_setup(Q, &L);
    for (i = 0; i < Q; ++i) {
        double eu = edot(&L, i, u), uu = dot3(u, u);
        geq[i] = L.t[i] * phi * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)) +
                 src_scale * L.t[i] * edot(&L, i, S);
    }
}

/* S_i = (Gamma_i - t_i)(e_i - u) . grad rho (App. A), with
 * Gamma_i = t_i [1 + e.u/cs^2 + (e.u)^2/(2 cs^4) - |u|^2/(2 cs^2)];
 * R_i = t_i [ (e_i - u)/cs^2 + (e_i . u)/cs^4 e_i ] . (rho G)  (Eq. body). */
void oracle_forcing(int Q, double rho, const double *u, const double *grad_rho, const double *G,
                    double *Si, double *Ri)
{
    lattice L;
    int i, a;
    lattice_setup(Q, &L);
    for (i = 0; i < Q; ++i) {
        double eu = edot(&L, i, u), uu = dot3(u, u);
        double Gamma = L.t[i] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        double emu_grad = 0.0, body = 0.0;
        for (a = 0; a < 3; ++a) {
            double emu = L.e[i][a] - u[a];
            emu_grad += emu * grad_rho[a];
            body += (emu / CS2 + eu / (CS2 * CS2) * L.e[i][a]) * (rho * G[a]);
        }
        Si[i] = (Gamma - L.t[i]) * emu_grad;
        Ri[i] = L.t[i] * body;
    }
}

static long wrap(long a, long n) { return ((a % n) + n) % n; }

static int opposite(const lattice *L, int i)
{
    int j;
    for (j = 0; j < L->Q; ++j)
        if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == -L->e[i][2]) return j;
    return -1;
}

/* 1 if coordinate a (before wrapping) lies beyond a wall of its axis */
static int beyond(int walls, int axis, long a, long n) { return ((walls >> axis) & 1) && (a < 0 || a >= n); }

/* coordinate of the cell a step `a` lands on: periodic wrap, or the mirror image across a wall */
static long land(int walls, int axis, long a, long n)
{
    if ((walls >> axis) & 1) {
        if (a < 0) return -1 - a;
        if (a >= n) return 2 * n - 1 - a;
        return a;
    }
    return wrap(a, n);
}

/* grad phi(x) = sum_{i != 0} t_i e_i [phi(x + e_i) - phi(x - e_i)] / (2 cs^2): the isotropic
 * central difference of the finite-difference method the paper compares against (Sec. 3.4). */
static void isotropic_gradient_walls(int Q, int nx, int ny, int nz, int walls, const double *field, double *grad);

void oracle_isotropic_gradient(int Q, int nx, int ny, int nz, const double *field, double *grad)
{
    isotropic_gradient_walls(Q, nx, ny, nz, 0, field, grad);
}

static void isotropic_gradient_walls(int Q, int nx, int ny, int nz, int walls, const double *field, double *grad)
{
    lattice L;
    long N = (long)nx * ny * nz;
    long row;
    lattice_setup(Q, &L);
#pragma omp parallel for schedule(static)
    for (row = 0; row < (long)nz * ny; ++row) {
        long z = row / ny, y = row % ny, x;
        int i, a;
            for (x = 0; x < nx; ++x) {
                long c = (z * ny + y) * nx + x;
                for (a = 0; a < 3; ++a) grad[a * N + c] = 0.0;
                for (i = 1; i < L.Q; ++i) {
                    long xp = land(walls, 0, x + L.e[i][0], nx), yp = land(walls, 1, y + L.e[i][1], ny);
                    long zp = land(walls, 2, z + L.e[i][2], nz);
                    long xm = land(walls, 0, x - L.e[i][0], nx), ym = land(walls, 1, y - L.e[i][1], ny);
                    long zm = land(walls, 2, z - L.e[i][2], nz);
                    double diff = field[(zp * ny + yp) * nx + xp] - field[(zm * ny + ym) * nx + xm];
                    for (a = 0; a < 3; ++a) grad[a * N + c] += L.t[i] * L.e[i][a] * diff / (2.0 * CS2);
                }
            }
    }
}

/* ----------------------------------------------------------------------------
 * The scheme.
 * ------------------------------------------------------------------------- */
struct oracle {
    lattice L;
    int nx, ny, nz;
    long N;
    double tau_f, tau_phi, delta, sigma;
    double rho1, rho2, eta1, eta2;
    double G[3];
    double c;
    int scheme;
    int pis_sign, half_force_sign, geq_source_tau;
    int walls; /* bit 0: walls at x = -1/2 and nx - 1/2; bit 1: the same in y; bit 2: in z */
    int initialised;
    double *f, *g;   /* post-collision state f*, g*: [Q][N] */
    double *fn, *gn; /* next state */
    double *phi;     /* propagated phi (finite-difference variant) */
    double *grad;    /* isotropic gradient of phi, 3 planes (finite-difference variant) */
};

/* packed macroscopic record */
enum { M_PHI = 0, M_RHO = 1, M_U = 2, M_K1 = 5, M_N = 8, M_S = 11, M_GPHI = 14, M_GRHO = 17, M_P = 20, M_LEN = 21 };

oracle *oracle_create(int Q, int nx, int ny, int nz, double tau_f, double tau_g, double M,
                      double xi, double sigma, double rho_ratio, double mu_ratio,
                      const double *G, double courant, int scheme, int pis_sign,
                      int half_force_sign, int geq_source_tau)
{
    oracle *o;
    size_t bytes;
    if (nx < 3 || ny < 3 || nz < 1) return NULL;
    if (Q == 9 && nz != 1) return NULL;
    if (Q == 19 && nz < 3) return NULL;
    if (tau_f <= 0 || xi <= 0 || rho_ratio <= 0 || mu_ratio <= 0) return NULL;
    if (M <= 0 && tau_g <= 0) return NULL;
    o = (oracle *)calloc(1, sizeof(oracle));
    if (!o) return NULL;
    if (lattice_setup(Q, &o->L)) { free(o); return NULL; }
    o->nx = nx; o->ny = ny; o->nz = nz;
    o->N = (long)nx * ny * nz;
    o->tau_f = tau_f;
    /* mobility M = tau_phi cs^2 dt (Sec. 2.3) */
    o->tau_phi = (M > 0) ? M / CS2 : tau_g;
    o->delta = xi;
    o->sigma = sigma;
    o->rho2 = 1.0;
    o->rho1 = rho_ratio;
    o->eta2 = o->rho2 * CS2 * tau_f;
    o->eta1 = mu_ratio * o->eta2;
    o->G[0] = G ? G[0] : 0.0; o->G[1] = G ? G[1] : 0.0; o->G[2] = G ? G[2] : 0.0;
    o->c = courant;
    o->scheme = scheme;
    o->pis_sign = pis_sign;
    o->half_force_sign = half_force_sign;
    o->geq_source_tau = geq_source_tau;
    bytes = (size_t)Q * o->N * sizeof(double);
    o->f = (double *)malloc(bytes);
    o->g = (double *)malloc(bytes);
    o->fn = (double *)malloc(bytes);
    o->gn = (double *)malloc(bytes);
    o->phi = (double *)malloc((size_t)o->N * sizeof(double));
    o->grad = (double *)malloc((size_t)3 * o->N * sizeof(double));
    if (!o->f || !o->g || !o->fn || !o->gn || !o->phi || !o->grad) { oracle_destroy(o); return NULL; }
    return o;
}

void oracle_destroy(oracle *o)
{
    if (!o) return;
    free(o->f); free(o->g); free(o->fn); free(o->gn); free(o->phi); free(o->grad);
    free(o);
}

double oracle_tau_phi(const oracle *o) { return o->tau_phi; }

int oracle_set_walls(oracle *o, int walls)
{
    if (walls < 0 || walls > 7 || (o->L.Q == 9 && (walls & 4))) return -1;
    o->walls = walls;
    return 0;
}

void oracle_macroscopic_cell(const oracle *o, const double *fbar, const double *g,
                             const double *fd_grad, double *m)
{
    const lattice *L = &o->L;
    double *u = m + M_U, *K1 = m + M_K1, *n = m + M_N, *S = m + M_S;
    double *gphi = m + M_GPHI, *grho = m + M_GRHO;
    double phi = 0.0, rho, rhou[3] = {0, 0, 0}, sum_f = 0.0, norm2, smag;
    int i, a;

    /* phi = sum_i g_i ; rho = rho1 phi + rho2 (1 - phi) (Sec. 2.3) */
    for (i = 0; i < L->Q; ++i) phi += g[i];
    rho = o->rho1 * phi + o->rho2 * (1.0 - phi);

    /* rho u = sum_i fbar_i e_i + (dt/2) rho G (Eq. momentum) */
    for (i = 0; i < L->Q; ++i)
        for (a = 0; a < 3; ++a) rhou[a] += fbar[i] * L->e[i][a];
    for (a = 0; a < 3; ++a) {
        rhou[a] += o->half_force_sign * 0.5 * rho * o->G[a];
        u[a] = rhou[a] / rho;
    }

    if (fd_grad == NULL) {
        /* K1 = sum_i g_i (e_i - u) (Sec. 2.3) */
        for (a = 0; a < 3; ++a) {
            K1[a] = 0.0;
            for (i = 0; i < L->Q; ++i) K1[a] += g[i] * (L->e[i][a] - u[a]);
        }
        /* n = -K1 / |K1| (Eq. norm) */
        norm2 = dot3(K1, K1);
        for (a = 0; a < 3; ++a) n[a] = (norm2 > NORMAL_GUARD) ? -K1[a] / sqrt(norm2) : 0.0;
        /* S = 4 phi (1 - phi) / delta n */
        smag = 4.0 * phi * (1.0 - phi) / o->delta;
        for (a = 0; a < 3; ++a) S[a] = smag * n[a];
        /* grad phi = (tau_phi cs^2 S - K1) / ((tau_phi + 0.5) cs^2) */
        for (a = 0; a < 3; ++a) gphi[a] = (o->tau_phi * CS2 * S[a] - K1[a]) / ((o->tau_phi + 0.5) * CS2);
    } else {
        /* finite-difference variant: n = grad phi / |grad phi| (Sec. 3.4) */
        for (a = 0; a < 3; ++a) { gphi[a] = fd_grad[a]; K1[a] = 0.0; }
        norm2 = dot3(gphi, gphi);
        for (a = 0; a < 3; ++a) n[a] = (norm2 > NORMAL_GUARD) ? gphi[a] / sqrt(norm2) : 0.0;
        smag = 4.0 * phi * (1.0 - phi) / o->delta;
        for (a = 0; a < 3; ++a) S[a] = smag * n[a];
    }
    /* grad rho = (rho1 - rho2) grad phi (Sec. 2.3) */
    for (a = 0; a < 3; ++a) grho[a] = (o->rho1 - o->rho2) * gphi[a];

    /* p = cs^2 sum fbar + (cs^2 dt / 2) u . grad rho (Eq. pressure) */
    for (i = 0; i < L->Q; ++i) sum_f += fbar[i];
    m[M_P] = CS2 * sum_f + 0.5 * CS2 * dot3(u, grho);
    m[M_PHI] = phi;
    m[M_RHO] = rho;
}

void oracle_collide_cell(const oracle *o, const double *fbar, const double *g,
                         const double *m, double *fstar, double *gstar)
{
    const lattice *L = &o->L;
    const int Q = L->Q;
    const double phi = m[M_PHI], rho = m[M_RHO], p = m[M_P];
    const double *u = m + M_U, *n = m + M_N, *S = m + M_S, *gphi = m + M_GPHI, *grho = m + M_GRHO;
    double pis[9], feq[19], geq[19], Si[19], Ri[19];
    double eta, tau_rho, src;
    int i;

    /* Pi_s = sigma |grad phi| (I - n n) */
    oracle_css_tensor(L->d, o->sigma, sqrt(dot3(gphi, gphi)), n, pis);
    oracle_feq(Q, p, rho, u, pis, o->pis_sign, feq);
    oracle_forcing(Q, rho, u, grho, o->G, Si, Ri);

    /* local relaxation time: eta(phi) = eta2 + (eta1 - eta2) phi, nu = eta/rho = tau_rho cs^2 */
    eta = o->eta2 + (o->eta1 - o->eta2) * phi;
    tau_rho = eta / (rho * CS2);

    for (i = 0; i < Q; ++i) {
        double F = Si[i] + Ri[i];
        double fbar_eq = feq[i] - 0.5 * F; /* modified equilibrium (Sec. 2.2) */
        /* f* = fbar - (fbar - fbar^eq)/(tau_rho + 0.5) + dt F (Eq. c-n_m) */
        fstar[i] = fbar[i] - (fbar[i] - fbar_eq) / (tau_rho + 0.5) + F;
    }

    src = o->geq_source_tau ? o->tau_phi : 1.0;
    oracle_geq(Q, phi, u, S, src, geq);
    for (i = 0; i < Q; ++i) {
        /* g* = g - (g - g^eq)/(tau_phi + 0.5) (Eq. c-n_c) */
        gstar[i] = g[i] - (g[i] - geq[i]) / (o->tau_phi + 0.5);
    }
}

/* Propagated populations of cell (x, y, z) from the stored post-collision planes. */
static void propagate_cell(const oracle *o, const double *fs, const double *gs, long x, long y, long z,
                           double *fbar, double *g)
{
    const lattice *L = &o->L;
    long c = (z * o->ny + y) * o->nx + x;
    int i;
    for (i = 0; i < L->Q; ++i) {
        long xm = x - L->e[i][0], ym = y - L->e[i][1], zm = z - L->e[i][2];
        long xp = x + L->e[i][0], yp = y + L->e[i][1], zp = z + L->e[i][2];
        int wall_m = beyond(o->walls, 0, xm, o->nx) || beyond(o->walls, 1, ym, o->ny) || beyond(o->walls, 2, zm, o->nz);
        int wall_p = beyond(o->walls, 0, xp, o->nx) || beyond(o->walls, 1, yp, o->ny) || beyond(o->walls, 2, zp, o->nz);
        long cm = (wrap(zm, o->nz) * o->ny + wrap(ym, o->ny)) * o->nx + wrap(xm, o->nx);
        long cp = (wrap(zp, o->nz) * o->ny + wrap(yp, o->ny)) * o->nx + wrap(xp, o->nx);
        const double *F = fs + (long)i * o->N, *G = gs + (long)i * o->N;
        int ib = opposite(L, i);
        const double *Fb = fs + (long)ib * o->N, *Gb = gs + (long)ib * o->N;
        /* across a wall the stencil reads the opposite population of this cell */
        double fm = wall_m ? Fb[c] : F[cm], fp = wall_p ? Fb[c] : F[cp];
        double gm = wall_m ? Gb[c] : G[cm], gp = wall_p ? Gb[c] : G[cp];
        fbar[i] = oracle_lax_wendroff(o->c, fm, F[c], fp);
        g[i] = oracle_lax_wendroff(o->c, gm, G[c], gp);
    }
}

/* Finite-difference variant, first pass: propagated phi everywhere, then its gradient. */
static void fd_phi_pass(oracle *o)
{
    long row;
#pragma omp parallel for schedule(static)
    for (row = 0; row < (long)o->nz * o->ny; ++row) {
        long z = row / o->ny, y = row % o->ny, x;
        int i;
        double fbar[19], g[19];
            for (x = 0; x < o->nx; ++x) {
                double phi = 0.0;
                propagate_cell(o, o->f, o->g, x, y, z, fbar, g);
                for (i = 0; i < o->L.Q; ++i) phi += g[i];
                o->phi[(z * o->ny + y) * o->nx + x] = phi;
            }
    }
    isotropic_gradient_walls(o->L.Q, o->nx, o->ny, o->nz, o->walls, o->phi, o->grad);
}

int oracle_init_phi(oracle *o, const double *phi0, const double *u0, double p0)
{
    return oracle_init_fields(o, phi0, u0, NULL, p0);
}

int oracle_init_fields(oracle *o, const double *phi0, const double *u0, const double *p, double p0)
{
    const lattice *L = &o->L;
    long c;
    double *grad = o->grad;
    isotropic_gradient_walls(L->Q, o->nx, o->ny, o->nz, o->walls, phi0, grad);
#pragma omp parallel for schedule(static)
    for (c = 0; c < o->N; ++c) {
        double gphi[3], n[3], S[3], u[3], pis[9], feq[19], geq[19];
        double norm2, gn, smag, rho;
        int a, i;
        for (a = 0; a < 3; ++a) {
            gphi[a] = grad[a * o->N + c];
            u[a] = u0 ? u0[a * o->N + c] : 0.0;
        }
        norm2 = dot3(gphi, gphi);
        gn = sqrt(norm2);
        for (a = 0; a < 3; ++a) n[a] = (norm2 > NORMAL_GUARD) ? gphi[a] / gn : 0.0;
        smag = 4.0 * phi0[c] * (1.0 - phi0[c]) / o->delta;
        for (a = 0; a < 3; ++a) S[a] = smag * n[a];
        rho = o->rho1 * phi0[c] + o->rho2 * (1.0 - phi0[c]);
        oracle_css_tensor(L->d, o->sigma, gn, n, pis);
        oracle_feq(L->Q, p ? p[c] : p0, rho, u, pis, o->pis_sign, feq);
        oracle_geq(L->Q, phi0[c], u, S, o->geq_source_tau ? o->tau_phi : 1.0, geq);
        for (i = 0; i < L->Q; ++i) {
            o->f[(long)i * o->N + c] = feq[i];
            o->g[(long)i * o->N + c] = geq[i] - L->t[i] * (o->tau_phi - 0.5) * edot(L, i, gphi);
        }
    }
    o->initialised = 1;
    return 0;
}

int oracle_step(oracle *o, int nsteps)
{
    int s;
    if (!o->initialised) return -6;
    for (s = 0; s < nsteps; ++s) {
        long row;
        double *tmp;
        if (o->scheme == 1) fd_phi_pass(o);
#pragma omp parallel for schedule(static)
        for (row = 0; row < (long)o->nz * o->ny; ++row) {
            long z = row / o->ny, y = row % o->ny, x;
            double fbar[19], g[19], fstar[19], gstar[19], m[M_LEN], fd[3];
            int i, a;
                for (x = 0; x < o->nx; ++x) {
                    long c = (z * o->ny + y) * o->nx + x;
                    propagate_cell(o, o->f, o->g, x, y, z, fbar, g);
                    if (o->scheme == 1)
                        for (a = 0; a < 3; ++a) fd[a] = o->grad[a * o->N + c];
                    oracle_macroscopic_cell(o, fbar, g, o->scheme == 1 ? fd : NULL, m);
                    oracle_collide_cell(o, fbar, g, m, fstar, gstar);
                    for (i = 0; i < o->L.Q; ++i) {
                        o->fn[(long)i * o->N + c] = fstar[i];
                        o->gn[(long)i * o->N + c] = gstar[i];
                    }
                }
        }
        tmp = o->f; o->f = o->fn; o->fn = tmp;
        tmp = o->g; o->g = o->gn; o->gn = tmp;
    }
    return 0;
}

int oracle_moments(oracle *o, double *phi, double *p, double *u, double *grad_phi, double *n)
{
    long row;
    if (!o->initialised) return -6;
    if (o->scheme == 1) fd_phi_pass(o);
#pragma omp parallel for schedule(static)
    for (row = 0; row < (long)o->nz * o->ny; ++row) {
        long z = row / o->ny, y = row % o->ny, x;
        double fbar[19], g[19], m[M_LEN], fd[3];
        int a;
            for (x = 0; x < o->nx; ++x) {
                long c = (z * o->ny + y) * o->nx + x;
                propagate_cell(o, o->f, o->g, x, y, z, fbar, g);
                if (o->scheme == 1)
                    for (a = 0; a < 3; ++a) fd[a] = o->grad[a * o->N + c];
                oracle_macroscopic_cell(o, fbar, g, o->scheme == 1 ? fd : NULL, m);
                if (phi) phi[c] = m[M_PHI];
                if (p) p[c] = m[M_P];
                for (a = 0; a < 3; ++a) {
                    if (u) u[a * o->N + c] = m[M_U + a];
                    if (grad_phi) grad_phi[a * o->N + c] = m[M_GPHI + a];
                    if (n) n[a * o->N + c] = m[M_N + a];
                }
            }
    }
    return 0;
}

/* Sum of phi and of rho phi over the propagated current state (m = sum rho phi dx^3, Sec. 3.3). */
int oracle_mass(oracle *o, double *sum_phi, double *sum_rho_phi)
{
    double *phi;
    long c;
    double s1 = 0.0, s2 = 0.0;
    if (!o->initialised) return -6;
    phi = (double *)malloc((size_t)o->N * sizeof(double));
    if (!phi) return -2;
    oracle_moments(o, phi, NULL, NULL, NULL, NULL);
    for (c = 0; c < o->N; ++c) {
        double rho = o->rho1 * phi[c] + o->rho2 * (1.0 - phi[c]);
        s1 += phi[c];
        s2 += rho * phi[c];
    }
    free(phi);
    *sum_phi = s1;
    *sum_rho_phi = s2;
    return 0;
}

int oracle_get_pops(const oracle *o, double *f, double *g)
{
    size_t bytes = (size_t)o->L.Q * o->N * sizeof(double);
    if (f) memcpy(f, o->f, bytes);
    if (g) memcpy(g, o->g, bytes);
    return 0;
}

int oracle_set_pops(oracle *o, const double *f, const double *g)
{
    size_t bytes = (size_t)o->L.Q * o->N * sizeof(double);
    memcpy(o->f, f, bytes);
    memcpy(o->g, g, bytes);
    o->initialised = 1;
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
