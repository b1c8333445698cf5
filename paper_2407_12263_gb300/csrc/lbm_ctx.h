// lbm_ctx.h -- the handle behind the C ABI (include/lbm.h), shared by the single-case entry
// points (lbm_api.cu) and the batch entry points (lbm_batch.cu). Internal: not installed.
#pragma once

#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

struct lbm_ctx {
    lbm::Params P;
    int scheme;
    double courant;
    int device;
    cudaStream_t stream;
    bool own_stream;
    void* fg[2];           // ping-pong state: Q planes of N (f, g) pairs each (storage.cuh)
    bool own_fg;           // false: the caller's buffers (lbm_create_ext), never freed here
    size_t fg_bytes;       // bytes allocated per state buffer (the largest storage the case may take)
    int cur;               // index of the buffer holding the current state
    float* phi_fd;         // propagated phi plane of the finite-difference variant
    double* partials;      // per-block FP64 partial sums of the mass reduction
    int n_partials;
    double* result;        // 3 doubles: sum phi, sum rho phi, non-finite count
    double* staging;       // FP64 staging for host transfers, allocated on first use
    size_t staging_elems;
    bool initialised;
    long long launches;
    int graph_steps;                  // steps per replayed CUDA graph (0 = none)
    cudaGraphExec_t graph_exec[2];    // graph of graph_steps steps starting from buffer 0 / 1
    bool batch_owned;      // a case of an lbm_batch: lbm_destroy leaves it to lbm_batch_destroy
    void* jump_ws;         // surrogate jumps: a backup state, then four coarse field arrays
    size_t jump_ws_bytes;  // (allocated by the first jump or lbm_surrogate_reserve, kept until destroy)
    long long version;     // bumped whenever the parameters or the whole state are replaced
    char err[512];
};

namespace lbm {

// lbm_create with the state buffers sized for alloc_storage (>= the bytes of opts->storage), so
// that set_ctx_storage may later switch to any storage that fits. Messages of a failed create
// are in lbm_last_error(NULL).
// ext_fg, ext_bytes: two caller-owned state buffers of ext_bytes each (lbm_create_ext), or
// nullptr to allocate them.
int create_ctx(lbm_ctx** out, const int grid[3], int lattice, double tau_f, double tau_g, double M, double xi,
               double sigma, double rho_ratio, double mu_ratio, const double body_force[3], const lbm_opts* opts,
               int alloc_storage, void* const* ext_fg = nullptr, size_t ext_bytes = 0);

// Switches the storage of a handle that holds no state yet (LBM_ESTATE after lbm_init_phi or
// lbm_set_pops, LBM_EINVAL if the buffers are too small for it).
int set_ctx_storage(lbm_ctx* c, int storage);

// Helpers of the surrogate entry points (lbm_surrogate.cu).
int ctx_error(lbm_ctx* c, int code, const char* msg);
int ctx_check(lbm_ctx* c);
// The exact 64-bit sum of the fixed-point phi values of the propagated state. Synchronous.
int ctx_mass_fixed(lbm_ctx* c, long long* sum);
// Replace the state by the one lbm_init_fields builds from the coarse fields [5][nz/f][ny/f][nx/f]
// (device FP32: phi, u, v, w, p) upsampled trilinearly; p0 = the storage reference pressure.
int ctx_restart_from_coarse(lbm_ctx* c, int f, const float* coarse, double p0);
// Add delta fixed-point units of phi, spread so that the sum changes by exactly delta.
int ctx_adjust_phi(lbm_ctx* c, long long delta);

}  // namespace lbm
