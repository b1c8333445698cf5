/*
 * lbm_surrogate.h -- a small 3D convolutional surrogate that fast-forwards the coarsened state
 * of the difference-free conservative phase-field LBM (include/lbm.h), with the solver as its
 * judge and fallback.
 *
 * The paper has no counterpart: it advances every step with the LBM. This part stands on its
 * own. It is trained only on trajectories this solver generates. It has its own forward and
 * backward kernels, and is checked against an FP64 restatement of the same network.
 *
 * The network. C = 5 field channels (phi, u, v, w, p), each normalised as (value - mean) / std.
 * Four periodic 3x3x3 convolutions, 5 -> 32 -> 32 -> 32 -> 5 channels, ReLU after the first
 * three; the prediction is input + output (a residual step). Convolutions accumulate in FP32;
 * activations between layers are stored in FP16 (or FP32, for gradient checks). With FP16
 * activations every layer (channels zero-padded to 32), its adjoint and its weight gradients
 * run on the tensor cores (tcgen05, FP16 operands, FP32 accumulation in tensor memory); in
 * FP32 mode everything runs on the CUDA cores. A tensor-core wait that times out makes the
 * next synchronising call return LBM_ETIMEOUT. Weights are
 * FP32 ([Cout][Cin][27] then bias [Cout] per layer, tap = 9 dz + 3 dy + dx for the input offset
 * (dz-1, dy-1, dx-1)). Training minimises the (channel-weighted) mean squared error with Adam
 * (0.9, 0.999, 1e-8).
 *
 * Arrays of fields are device FP32 [B][5][D][H][W], W fastest, owned by the caller.
 * Every call returns an lbm_status; nothing throws. Calls on one network are asynchronous on
 * its stream unless marked synchronous.
 */
#ifndef LBM_SURROGATE_H
#define LBM_SURROGATE_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_net lbm_net;

/* Create a network with seeded weights: He-normal (std sqrt(2 / (27 Cin))) drawn from a
 * SplitMix64 stream started at `seed`, the last layer scaled by 0.1, biases 0.
 * activations_fp16: 1 stores activations in FP16, 0 in FP32. stream: cudaStream_t or NULL (one
 * the network owns). */
int lbm_net_create(lbm_net **out, int activations_fp16, unsigned long long seed, void *stream);

/* Number of FP32 parameters, and host copies of the parameters, of the gradients of the last
 * lbm_net_gradients call, and into the parameters (synchronous). */
long long lbm_net_param_count(const lbm_net *net);
int lbm_net_get_params(lbm_net *net, float *host);
int lbm_net_set_params(lbm_net *net, const float *host);
int lbm_net_get_grads(lbm_net *net, float *host);

/* y = x + net(x) for a batch on a grid (each extent >= 1). x and y may not alias. */
int lbm_net_forward(lbm_net *net, const float *x, float *y, int batch, const int grid[3]);

/* Per-channel weights w_c >= 0 of the loss (default 1): fields whose changes are small next to
 * their spread (the velocity over a short jump) can be weighted up. */
int lbm_net_set_loss_weights(lbm_net *net, const float w[5]);

/* The loss mean(w_c (x + net(x) - target)^2) over every element of the batch into *loss
 * (synchronous) and its gradients with respect to all parameters (kept on the device). */
int lbm_net_gradients(lbm_net *net, const float *x, const float *target, int batch, const int grid[3], double *loss);

/* One Adam step with learning rate lr from the gradients of the last lbm_net_gradients. */
int lbm_net_adam(lbm_net *net, float lr);

/* Every wait of the tensor-core kernels polls its mbarrier a bounded number of times (2^26)
 * and gives up after that. on = 1 makes every wait for a step's MMAs give up at once instead:
 * the kernel then stops issuing, waits (with the full bound) for the MMAs it issued, frees its
 * tensor memory and returns, and the next synchronising call on the network returns
 * LBM_ETIMEOUT once; the network stays usable. on = 0 restores the normal waits. This exists to
 * test the timeout path without a hung GPU; the paper has no counterpart. */
int lbm_net_fail_waits(lbm_net *net, int on);

const char *lbm_net_last_error(const lbm_net *net);
void lbm_net_destroy(lbm_net *net);

/* The lattice side. factor f divides nx, ny, nz; the handle uses the difference-free scheme.
 * lbm_coarse_fields: device out [5][nz/f][ny/f][nx/f] = block means over f^3 cells of phi, u,
 * v, w and p as lbm_moments computes them. */
int lbm_coarse_fields(lbm_ctx *ctx, int factor, float *out);

/* Block means over f^3 cells of the state's own phi (the fixed-point zeroth moment of g, before
 * propagation), device out [nz/f][ny/f][nx/f]: what the judge of lbm_surrogate_jump measures
 * right after a restart and judge_steps later. f must divide 32 as well as nx, ny and nz. */
int lbm_coarse_phi(lbm_ctx *ctx, int factor, float *out);

/* Replace the state by the one lbm_init_fields builds from coarse fields (device [5][...] as
 * above) upsampled trilinearly between coarse cell centres (periodic; clamped across walls),
 * with p0 the reference pressure of the storage; the construction runs in FP32 in one pass, and
 * the upsampled phi is clamped to [-1, 1.5]. sum phi is then set back exactly to its value
 * before the call (the difference, in units of 2^-30, spread over the cells). */
int lbm_restart_from_coarse(lbm_ctx *ctx, int factor, const float *coarse, double p0);

/* The divergence-free part of a periodic velocity field: the field closest to u in the sum of
 * squares over all cells and components whose central-difference divergence
 *   div u = sum_a (u_a(x + e_a) - u_a(x - e_a)) / 2
 * vanishes (the orthogonal projection onto the kernel of div; u minus it is a central-difference
 * gradient). At low Mach number the flow is divergence-free (Sec. 2.1, with the pressure
 * evolution equation), and a lattice restarted from a compressive velocity relaxes it away
 * through pressure waves; lbm_surrogate_jump applies this to the predicted velocity.
 * Evaluated per Fourier mode, U <- U - s (s . U) / |s|^2 with s_a = sin(2 pi k_a / n_a) (modes with
 * s = 0 are kept), between a forward and an inverse discrete Fourier transform along each axis,
 * as direct sums in FP32 in a fixed order: the same bits on every run.
 * u: device FP32 [3][nz][ny][nx] (components x, y, z, x fastest), replaced in place; grid
 * (nx, ny, nz), each extent 1 .. 512; work: device scratch of at least
 * lbm_project_workspace_bytes(grid) bytes (caller-owned; nothing is allocated), 16-byte
 * aligned; stream: cudaStream_t or NULL (the legacy default stream). Asynchronous: 9
 * kernel launches on the stream. Returns LBM_EINVAL for a NULL pointer, an extent outside
 * 1 .. 512, a misaligned pointer or too small a workspace (nothing is launched), LBM_ECUDA if a
 * launch fails. */
long long lbm_project_workspace_bytes(const int grid[3]); /* -1 for an invalid grid */
int lbm_project_solenoidal(float *u, const int grid[3], void *work, long long work_bytes, void *stream);

typedef struct {
    int accepted;       /* 1: the state holds the prediction advanced by judge_steps steps;
                           0: it holds the LBM's own k steps from the starting state */
    double mass_error;  /* |sum phi of the prediction - sum phi before| / sum phi before */
    double relax_ratio; /* how fast the LBM moves phi after the restart from the prediction,
                           relative to after the same restart from the starting state's own
                           coarse fields (1 = as consistent as the starting state); 0 if the
                           prediction was rejected before any restart */
    double interface_shift; /* mean displacement of the interface from the starting state to the
                               prediction, in cells: f sum |phi_pred - phi_start| / sum |grad phi_start|
                               over the coarse cells (central differences in coarse cells) */
    double interface_limit; /* the largest shift accepted: interface_tol * k * the largest speed
                               |u| of the starting and the predicted coarse fields */
    double seconds_surrogate; /* host wall time of the jump, judge included */
    int projected;      /* 1 if the predicted velocity was replaced by its divergence-free part
                           (grids periodic in every axis), 0 if it was used as predicted */
} lbm_jump_report;

/*
 * Fast-forward k steps with the surrogate, judged by the LBM:
 *   1. coarsen the state by `factor`, normalise with mean_std (5 means, then 5 stds), predict,
 *      denormalise; on a grid without walls (coarse extents at most 512), replace the predicted
 *      velocity by its divergence-free part (lbm_project_solenoidal);
 *   2. reject if the prediction's sum phi is off by more than mass_tol (relative), or if its
 *      interface moved farther than the flow can carry it: interface_shift > interface_limit
 *      (see lbm_jump_report). The phi = 1/2 surface of the conservative phase field moves with
 *      the fluid, because the sharpening flux vanishes on the equilibrium profile (Sec. 2.3), so
 *      in k steps no part of it moves farther than max |u| k; interface_tol = 1 is that bound;
 *   3. restart the lattice from the starting state's own coarse fields, run judge_steps LBM
 *      steps and measure how fast phi moves (|phi_after - phi_restart| / judge_steps, coarse,
 *      L1; phi_restart the coarse phi right after the restart, both block means of the state's
 *      own phi when factor divides 32): the relaxation a restart alone causes;
 *   4. restart from the prediction (sum phi held exactly), measure the same, and reject if it
 *      exceeds relax_tol times the rate of step 3: a prediction whose phi, u and p do not fit
 *      together relaxes faster than the starting state does after the same restart;
 *   5. on rejection restore the starting state and advance it k steps with the LBM.
 * Synchronous. Needs a workspace of one more state buffer, four coarse field arrays and the
 * projection's scratch (lbm_project_workspace_bytes of the coarse grid): the
 * first jump on a handle allocates it (or lbm_surrogate_reserve, beforehand) and the handle keeps
 * it until lbm_destroy, so later jumps allocate nothing.
 */
int lbm_surrogate_jump(lbm_ctx *ctx, lbm_net *net, int factor, const float mean_std[10], int k, int judge_steps,
                       double mass_tol, double relax_tol, double interface_tol, lbm_jump_report *report);

/* Allocate the workspace of lbm_surrogate_jump for this factor now (LBM_ENOMEM if it does not
 * fit), so that the jumps themselves allocate nothing. Synchronous. */
int lbm_surrogate_reserve(lbm_ctx *ctx, int factor);

#ifdef __cplusplus
}
#endif
#endif
