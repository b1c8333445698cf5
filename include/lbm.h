/*
 * lbm.h -- C ABI of the GB300 (sm_103a) difference-free conservative phase-field
 * lattice Boltzmann solver (Zhao, Patel & Lee, arXiv:2407.12263).
 *
 * One handle owns one periodic lattice (D2Q9 or D3Q19) and its device state: the
 * post-collision populations f* (one-fluid pressure PDF, Sec. 2.2) and g* (conservative
 * phase-field PDF, Sec. 2.3), held as (f_i, g_i) pairs with x fastest, in two ping-pong
 * copies; the moving pairs are FP32, FP16 or BF16 (lbm_storage), all arithmetic is FP32. A
 * state buffer holds the zeroth-moment plane (8 B per cell, padded to a multiple of 16 B for
 * FP32 storage), then one plane of words [nz][ny][nx] per opposite pair of populations (i, and
 * j with e_j = -e_i): per cell the pair of i then that of j, 16 B for FP32, 8 B for 16-bit.
 * Every step is one fused stream-collide kernel launch (difference-free scheme), or two
 * launches for the finite-difference variant.
 *
 * Units are lattice units: dx = 1 and dt = 1 in every collision, moment and forcing
 * formula; the Courant number only enters the Lax-Wendroff propagation (Sec. 2.2).
 * Fluid 2 (phi = 0) has density 1 and dynamic viscosity eta2 = tau_f / 3; fluid 1
 * (phi = 1) has density rho_ratio and viscosity mu_ratio * eta2.
 *
 * Host arrays passed to or from the library are FP64, owned by the caller, never
 * retained, and laid out like the device planes: scalar fields have nx*ny*nz entries with
 * x fastest; vector fields are 3 such planes (x, y, z components). Population arrays are
 * Q planes in the velocity order given below.
 *
 * Velocity order. D2Q9 follows Sec. 2.2: 0 rest; 1..4 = (1,0), (0,1), (-1,0), (0,-1);
 * 5..8 = (1,1), (-1,1), (-1,-1), (1,-1). D3Q19: 0 rest; 1..6 = +x, -x, +y, -y, +z, -z;
 * 7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
 * (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1). Weights follow the speed: 4/9, 1/9, 1/36 (D2Q9)
 * and 1/3, 1/18, 1/36 (D3Q19).
 *
 * Errors: every call returns an lbm_status; nothing throws across the ABI. The message
 * of the last failure on a handle is available from lbm_last_error(handle) until the next
 * call on that handle; failures of lbm_create are reported by lbm_last_error(NULL) on the
 * calling thread. A handle must not be used from two host threads at once. Calls that
 * return data to the host synchronise the handle's stream; lbm_step does not, so a fault
 * in an asynchronous launch surfaces at the next synchronising call.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

enum lbm_lattice { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };

enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* an argument is out of range or inconsistent */
    LBM_ENOMEM = -2,     /* a device allocation failed */
    LBM_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    LBM_ENONFINITE = -4, /* the state holds a NaN or an infinity */
    LBM_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    LBM_ESTATE = -6      /* the call needs lbm_init_phi (or lbm_set_pops) first */
};

enum lbm_storage {
    LBM_STORAGE_FP32 = 0, /* (f_i, g_i) pairs as 2 x FP32: 304 B per D3Q19 cell and step */
    LBM_STORAGE_FP16 = 1, /* moving pairs as 2 x FP16 (deviations scaled by 2^12 and 2^10), the
                             zeroth-moment plane in FP32: 160 B per D3Q19 cell and step */
    LBM_STORAGE_BF16 = 2, /* moving pairs as 2 x BF16, zeroth-moment plane in FP32: 160 B */
    LBM_STORAGE_AUTO = 3  /* batch cases only: lbm_batch_tune picks the fastest of the three */
};

enum lbm_scheme {
    LBM_SCHEME_DIFFERENCE_FREE = 0, /* grad phi and n from the central moment K1 (Sec. 2.3) */
    LBM_SCHEME_FINITE_DIFFERENCE = 1 /* isotropic central difference of phi (Sec. 3.4) */
};

typedef struct {
    int scheme;     /* enum lbm_scheme; default difference-free */
    int storage;    /* enum lbm_storage; default FP32. Arithmetic is FP32 in every case */
    double courant; /* Lax-Wendroff Courant number c, 0 < c <= 1; default 0.997 (Sec. 2.2) */
    int walls;      /* mask of walled axes: 1 = x, 2 = y, 4 = z (D3Q19 only); 0 = fully periodic.
                       A wall lies half-way beyond the first and last cell of its axis:
                       half-way bounce-back in the Lax-Wendroff stencil (sum phi conserved),
                       zero normal gradient of phi for the initial and finite-difference
                       gradients */
    void *stream;   /* cudaStream_t the handle launches on; NULL = a stream the handle owns */
    int graph_steps; /* lbm_step replays CUDA graphs of this many steps (even, >= 2; default 32);
                        0 launches every step directly. Steps run inside a caller's own stream
                        capture are always launched directly, so they land in that graph */
} lbm_opts;

/* Fill *opts with the defaults above. */
void lbm_default_opts(lbm_opts *opts);

/*
 * Create a handle and allocate its device state (no kernel runs).
 *   grid[3]    nx, ny, nz; nx, ny >= 3; D2Q9 needs nz = 1, D3Q19 nz >= 3; nz <= 65535;
 *              nx*ny*nz < 2^31.
 *   lattice    LBM_D2Q9 or LBM_D3Q19.
 *   tau_f      relaxation time tau_rho of fluid 2 (Eq. c-n_m), > 0; nu2 = tau_f / 3.
 *   tau_g, M   phase-field relaxation time and mobility, related by M = tau_phi cs^2 dt
 *              (Sec. 2.3). If M > 0 it fixes tau_phi = 3 M; otherwise tau_phi = tau_g > 0.
 *   xi         interface thickness delta of Eq. cac, >= 2.
 *   sigma      surface tension of Eq. surface, >= 0.
 *   rho_ratio  rho1 / rho2 (> 0); mu_ratio eta1 / eta2 (> 0). Local viscosity
 *              eta(phi) = eta2 + (eta1 - eta2) phi and tau_rho = eta / (rho / 3).
 *   body_force G of Eq. body (3 components; NULL = 0; the z component must be 0 for D2Q9).
 *   opts       NULL = defaults.
 * Returns LBM_OK and *out, or LBM_EINVAL / LBM_ENOMEM / LBM_ECUDA with *out = NULL.
 */
int lbm_create(lbm_ctx **out, const int grid[3], int lattice, double tau_f, double tau_g,
               double M, double xi, double sigma, double rho_ratio, double mu_ratio,
               const double body_force[3], const lbm_opts *opts);

/* Bytes of one state buffer (a handle holds two) for this lattice, grid and storage: 8 B per
 * cell for the zeroth moments (padded to a multiple of 16 B for FP32 storage), plus Q - 1
 * moving (f, g) pairs of 8 B (FP32) or 4 B (FP16, BF16) per cell. Host-only; 0 for invalid
 * arguments. */
long long lbm_state_bytes(int lattice, const int grid[3], int storage);

/*
 * lbm_create with the two state buffers owned by the caller (a framework's tensors, a pool or
 * an arena the caller manages). fg0 and fg1: device memory of the current device, starting on
 * 16-byte boundaries, not overlapping, bytes_each >= lbm_state_bytes(lattice, grid,
 * opts->storage) each. The handle keeps its state in them for its lifetime, in the layout of
 * lbm.h's storage description, and never frees them: lbm_destroy leaves them to the caller,
 * who must not free or reuse them before it. The library still allocates its small buffers
 * (reduction scratch, the finite-difference phi plane, host staging on first use, the surrogate
 * workspace). LBM_EINVAL for NULL, misaligned, overlapping, too small or non-device buffers;
 * otherwise as lbm_create. (The paper does not discuss memory ownership; Sec. 3.4 runs
 * IMEXLBM, which owns its arrays.)
 */
int lbm_create_ext(lbm_ctx **out, const int grid[3], int lattice, double tau_f, double tau_g,
                   double M, double xi, double sigma, double rho_ratio, double mu_ratio,
                   const double body_force[3], const lbm_opts *opts, void *fg0, void *fg1,
                   size_t bytes_each);

/*
 * Initial state from the order parameter (host FP64, nx*ny*nz), an optional velocity
 * (3 host planes, NULL = rest) and a uniform pressure p0 > 0. Builds the post-collision
 * populations f* = f^eq(p0, u0, rho(phi0), Pi_s) (Eq. geq_s) and
 * g* = g^eq(phi0, u0, S0) - t_i (tau_phi - 1/2) e_i . grad phi0 (Eq. geq), with grad phi0
 * the isotropic central difference of phi0 and n0 = grad phi0 / |grad phi0|. Every phi0 value
 * must lie in [-1, 1.5] (LBM_EINVAL otherwise): the handle holds phi as a fixed-point number
 * with range [-2, 2) and resolution 2^-30. Synchronous.
 */
int lbm_init_phi(lbm_ctx *ctx, const double *phi0, const double *u0, double p0);

/*
 * lbm_init_phi with the pressure of f^eq given per cell: p (host FP64, nx*ny*nz, every value
 * > 0 and finite) replaces the uniform p0, which remains the reference level the f storage is
 * shifted by (take the mean pressure). The initial condition of the Taylor-Green case of
 * Sec. 3.4 includes such a field; without it the vortex starts out of balance and launches an
 * acoustic transient. p = NULL is lbm_init_phi. Synchronous.
 */
int lbm_init_fields(lbm_ctx *ctx, const double *phi0, const double *u0, const double *p, double p0);

/* Advance n >= 0 time steps (asynchronous on the handle's stream). Whole multiples of
 * opts.graph_steps are replayed from CUDA graphs the handle captures on first use; the rest
 * are launched directly. Both give bit-identical results. */
int lbm_step(lbm_ctx *ctx, int n);

/* Capture the step graph that lbm_step replays from the current state's buffer, if it is not
 * captured yet, and upload it to the device, without running it: the state does not change and
 * no launch is counted. A later lbm_step(n) with n a multiple of graph_steps from this buffer
 * then replays it with no capture and no first-launch upload. Synchronous. LBM_EINVAL if the
 * handle replays no graphs (graph_steps 0), LBM_ESTATE before lbm_init_phi. */
int lbm_graph_prepare(lbm_ctx *ctx);

/*
 * Macroscopic fields of the current state: phi, p and u computed from the propagated
 * populations exactly as the next step computes them before colliding (phi = sum g_i,
 * Eq. momentum, Eq. pressure). Any output may be NULL. Synchronous.
 */
int lbm_moments(lbm_ctx *ctx, double *phi, double *p, double *u);

/*
 * grad phi and the unit normal n of the current state as the scheme computes them:
 * from K1 (Sec. 2.3, Eq. norm) or from the isotropic central difference (Sec. 3.4).
 * 3 host planes each; either may be NULL. Synchronous.
 */
int lbm_gradients(lbm_ctx *ctx, double *grad_phi, double *normal);

/*
 * Global sums over the propagated current state: sum phi and sum rho phi (the mass
 * m = sum rho phi dx^3 of Sec. 3.3). sum phi is the exact sum of the fixed-point phi values
 * (a 64-bit integer sum; the time step conserves it bit for bit, walls included); sum rho phi
 * is rho2 sum phi + (rho1 - rho2) sum phi^2, the squares of the fixed-point values summed in
 * FP64. Also scans every stored population and returns LBM_ENONFINITE if one
 * is not finite. Synchronous.
 */
int lbm_mass(lbm_ctx *ctx, double *sum_phi, double *sum_rho_phi);

/*
 * State diagnostics for the static-droplet checks of Sec. 3.1: the spurious currents (the
 * largest |u|, Table 1) and the pressure inside and outside the droplet for Laplace's law,
 * reduced on the device from the fields lbm_moments returns (u and p of the propagated current
 * state), without moving the fields to the host. The largest speed, its cell and the masks are
 * exact as defined here in FP64, every product and sum rounded once (the device decides in
 * FP32 where that cannot change the outcome and takes FP64 where it can):
 *   max_speed  sqrt of the largest (u_x^2 + u_y^2) + u_z^2 over the cells;
 *   argmax     the cell index (x fastest) of that value, the smallest index on ties;
 *   kinetic    sum over cells of rho |u|^2 / 2, rho = 1 + (rho_ratio - 1) phi, each cell's term
 *              and runs of 8 cells summed in FP32 (rho and u are FP32 fields), the runs in FP64:
 *              within about 1e-6 relative of the same sum in FP64;
 *   p_in/n_in  mean p over, and count of, the cells whose centre (integer coordinates) lies
 *              closer than r_in to centre; p_out/n_out the same farther than r_out. The
 *              distance takes the minimum image along periodic axes, the plain difference
 *              along walled axes, and leaves out an axis of extent 1. A mean over no cell is NaN.
 * The reduction order is fixed (per thread, per block, then the blocks in order): the same bits
 * on every run. The per-cell fields are computed by the code lbm_moments uses; compiled into
 * another kernel, a fused multiply-add may round differently, so a field value can differ from
 * lbm_moments' in its last FP32 bit. centre: 3 host doubles (x, y, z). Synchronous. LBM_EINVAL for NULL pointers or
 * a non-finite centre or radius; LBM_ESTATE before lbm_init_phi.
 */
typedef struct {
    double max_speed;
    long long argmax;
    double kinetic;
    double p_in, p_out;
    long long n_in, n_out;
} lbm_diag;
int lbm_diagnostics(lbm_ctx *ctx, const double centre[3], double r_in, double r_out, lbm_diag *out);

/* Copy the post-collision populations f*, g* to / from host FP64 arrays (Q planes each;
 * either pointer of lbm_get_pops may be NULL). lbm_set_pops also marks the state
 * initialised; sum_i g_i must lie in [-1, 1.5] in every cell (LBM_EINVAL otherwise), and is
 * rounded to the fixed-point grid of phi (2^-30). Synchronous. */
int lbm_get_pops(lbm_ctx *ctx, double *f, double *g);
int lbm_set_pops(lbm_ctx *ctx, const double *f, const double *g);

/* Kernel launches issued by this handle since creation (one per step for the
 * difference-free scheme, two for the finite-difference variant, plus auxiliaries). */
long long lbm_launch_count(const lbm_ctx *ctx);

/* tau_phi the handle resolved from (tau_g, M). */
double lbm_tau_phi(const lbm_ctx *ctx);

/* The velocity set the CUDA path uses: d, e[Q][3] (row-major) and weights w[Q]; any output
 * may be NULL. Host-only (needs no GPU). LBM_EINVAL for an unknown lattice. */
int lbm_lattice_tables(int lattice, int *d, int *e, double *w);

/*
 * Mass diagnostic for callers that cannot allocate device memory. Such callers include a
 * solver whose populations already fill the GPU, code whose device memory is all owned by a
 * framework's pool or a fixed arena, and a loop that must not stall on the driver's
 * allocator. This entry point has no counterpart in the paper; it is a variant of the
 * reduction behind lbm_mass that needs no handle and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   g         device pointer to FP32 plain populations g_i (not the handle's storage):
 *             Q planes [Q][nz][ny][nx], x fastest, plane 0 the rest population, in the
 *             velocity order above. Read only.
 *   lattice   LBM_D2Q9 or LBM_D3Q19; grid[3] as for lbm_create.
 *   walls     the mask of walled axes, as lbm_opts.walls (0 = fully periodic). Where the
 *             propagation stencil of a cell crosses a wall it reads the opposite population of
 *             the same cell (half-way bounce-back), as the time step does.
 *   courant   Lax-Wendroff Courant number, 0 < c <= 1. rho_ratio > 0 as for lbm_create.
 *   result    device pointer to 3 doubles, written with: sum phi and sum rho phi (the mass
 *             m = sum rho phi of Sec. 3.3) over the propagated state, then the count of
 *             non-finite values among the stored populations. phi of each cell is the FP32
 *             sum of its propagated g_i, accumulated in FP64. It is therefore not the exact
 *             fixed-point sum lbm_mass reports for a handle, which the time step conserves bit
 *             for bit: for the same state the two agree to about 1e-7 relative (FP32 rounding
 *             of each cell's phi).
 *   stream    cudaStream_t to launch on (NULL = the default stream). Asynchronous: result is
 *             ready when the stream reaches this point.
 * Scratch. The per-block partial sums live in a static device array that every GPU loading
 * the library holds until exit. It has room for 2048 blocks (48 KB), and each z-layer takes
 * at least one block, so nz must be <= 2048; larger grids, like every other invalid argument,
 * return LBM_EINVAL without launching. Every call shares that array: the blocks of a call
 * write their slots before the call's final sum reads them, so nothing needs clearing between
 * calls, but calls that overlap on the GPU (two streams, two threads) race on it and must be
 * serialised by the caller.
 * Each call looks up the array's device address in the current context, so the entry point
 * stays valid after a device reset. Returns LBM_ECUDA if the lookup or a launch fails; an
 * error left on the thread by earlier work is neither reported nor cleared by this call.
 */
int lbm_mass_noalloc(const float *g, int lattice, const int grid[3], int walls, double courant,
                     double rho_ratio, double *result, void *stream);

/* Message of the last failure (see the error notes above); never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Free the handle and its device memory; NULL is a no-op. Synchronises the stream. A case
 * handle of a batch (lbm_batch_case) is left alone: lbm_batch_destroy frees it. */
void lbm_destroy(lbm_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Batches: many independent cases advanced together.
 *
 * The paper advances one problem at a time; this interface has no counterpart there. It
 * exists because a small grid cannot fill the GPU: a 32^3 case is 256 blocks of 128 cells,
 * fewer than the 608 that 152 SMs keep resident. A step of the batch is a set of launches on
 * eight branch streams that run concurrently:
 *   - group launches: all cases of one grid size (and tile shape, storage) in one grid of
 *     128-cell tiles, the case picked by blockIdx.y, its parameters read from the launch's
 *     parameter block;
 *   - dedicated launches: the single-case step kernel of lbm_step for one case.
 * Every cell runs the same code as lbm_step, so a case gives the same bits whether the batch
 * or its own handle advances it. lbm_batch_tune picks, per size class, the faster of the two
 * forms on this GPU. Each case's steps stay on one branch, so a graph of many steps has one
 * fork and one join and no barrier between steps; nothing spins.
 * ------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* One case: the arguments of lbm_create and its options. Every case of a batch uses the
 * difference-free scheme and the same lattice. */
typedef struct {
    int grid[3];
    int lattice;
    double tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio;
    double body_force[3];
    int walls;      /* as lbm_opts.walls */
    int storage;    /* LBM_STORAGE_FP32 / FP16 / BF16, or LBM_STORAGE_AUTO: lbm_batch_tune
                       times the three on this GPU and keeps the fastest (the state buffers are
                       sized for FP32); FP32 until then */
    double courant; /* 0 = the default 0.997 */
} lbm_case;

typedef struct {
    void *stream;    /* cudaStream_t shared by the batch and its cases; NULL = one it owns */
    int graph_steps; /* lbm_batch_step replays CUDA graphs of this many steps (even, >= 2;
                        default 32); 0 launches every step directly */
} lbm_batch_opts;

void lbm_batch_default_opts(lbm_batch_opts *opts);

/* Create the cases (each as lbm_create would, with the same argument checks) and the batch.
 * n_cases >= 1; cases[] is read only during the call. Returns LBM_OK and *out, or an error
 * with *out = NULL and the message in lbm_batch_last_error(NULL). */
int lbm_batch_create(lbm_batch **out, int n_cases, const lbm_case *cases, const lbm_batch_opts *opts);

/* The handle of case k (0 <= k < n_cases), owned by the batch, or NULL. Every single-case
 * entry point works on it: lbm_init_phi (required before lbm_batch_step), lbm_moments,
 * lbm_gradients, lbm_mass, lbm_get_pops / lbm_set_pops, and lbm_step, which advances that
 * case alone. */
lbm_ctx *lbm_batch_case(lbm_batch *b, int k);

/* Tuner. For every size class (cases of one grid size) it times trial_steps steps of the
 * class alone in each form: a group launch per tile shape 2^a x 2^b x 2^c = 128 (a >= 3, no
 * extent beyond the grid's next power of two) and dedicated launches; where a case asks for
 * LBM_STORAGE_AUTO and holds no state yet, each storage as well. The fastest form (and storage)
 * is kept for the class. Trial launches read each case's current state and write only its
 * other buffer, so the state is unchanged; cases without state are timed on the uniform rest
 * state. Synchronous. Without it a case with nx a multiple of 32 and at least 2^15 cells runs in
 * dedicated launches and the others in group launches of tiles 2^a x 8 x 128/(2^a 8) (2^a the
 * largest power of two up to 32 that divides nx, at least 8; 2D: 2^a x 128/2^a x 1). */
int lbm_batch_tune(lbm_batch *b, int trial_steps);

/* Tile shape (cells in x, y, z) of case k's group launch, its storage, and 1 if the case runs
 * in dedicated launches instead; any output may be NULL. */
int lbm_batch_case_config(const lbm_batch *b, int k, int tile[3], int *storage, int *dedicated);

/* Fix case k's form by hand (to restore choices the tuner made in an earlier run, say): tile
 * (cells in x, y, z; powers of two with product 128, z = 1 in 2D; NULL keeps the current one)
 * and dedicated (nonzero: dedicated launches). LBM_EINVAL for an invalid tile or case. */
int lbm_batch_set_config(lbm_batch *b, int k, const int tile[3], int dedicated);

/* Advance every case by n >= 0 steps (asynchronous on the batch's stream, which the branches
 * fork from and join back to; whole multiples of graph_steps are replayed from CUDA graphs).
 * LBM_ESTATE if a case has no state. */
int lbm_batch_step(lbm_batch *b, int n);

/* Kernel launches of the batch so far (steps plus tuner trials), and total cells. */
long long lbm_batch_launch_count(const lbm_batch *b);
long long lbm_batch_cells(const lbm_batch *b);

/* Message of the last failure of a batch call (b = NULL: of the last lbm_batch_create). */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Free the batch and all its cases; NULL is a no-op. */
void lbm_batch_destroy(lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif
