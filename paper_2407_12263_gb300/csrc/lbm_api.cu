// lbm_api.cu -- the C ABI (include/lbm.h): handle management, argument checks, slab-wise
// host <-> device transfers and kernel launches on the handle's stream.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lattice.cuh"
#include "diagnostics.h"
#include "lbm_ctx.h"
#include "lbm_internal.h"
#include "storage.cuh"
#include "surrogate.h"

using lbm::Params;

namespace {

constexpr size_t kStagingCap = size_t(32) << 20;  // doubles (256 MB) per staging slab at most
// phi is held as the fixed-point integer phi * 2^30 (range [-2, 2)); initial and restored
// states must leave room for the overshoot of a running interface.
constexpr double kPhiMin = -1.0, kPhiMax = 1.5;

thread_local char g_create_error[512] = "no error";

int set_error(lbm_ctx* ctx, int code, const char* fmt, ...) {
    char* buf = ctx ? ctx->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    // a failed allocation is reported here, synchronously, and is not sticky: clear it, or the
    // next launch's error check would report it again
    if (code == LBM_ENOMEM) (void)cudaGetLastError();
    return code;
}

#define LBM_CUDA(ctx, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_error((ctx), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, \
                             "%s failed: %s", #call, cudaGetErrorString(e_));                 \
    } while (0)

bool is_fin(double v) { return std::isfinite(v); }

void free_ctx(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->own_fg)
        for (int k = 0; k < 2; ++k) cudaFree(c->fg[k]);
    cudaFree(c->phi_fd);
    cudaFree(c->partials);
    cudaFree(c->result);
    cudaFree(c->staging);
    cudaFree(c->jump_ws);
    for (int k = 0; k < 2; ++k)
        if (c->graph_exec[k]) cudaGraphExecDestroy(c->graph_exec[k]);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int ensure_staging(lbm_ctx* c, size_t elems) {
    if (c->staging_elems >= elems) return LBM_OK;
    cudaFree(c->staging);
    c->staging = nullptr;
    c->staging_elems = 0;
    LBM_CUDA(c, cudaMalloc(&c->staging, elems * sizeof(double)));
    c->staging_elems = elems;
    return LBM_OK;
}

// z-planes per slab so that slab_planes(nzs) * nxy doubles fit the staging cap.
int slab_depth(const lbm_ctx* c, int planes_per_z, int extra_planes) {
    const size_t nxy = (size_t)c->P.nxy;
    long long nzs = (long long)(kStagingCap / nxy) - extra_planes;
    nzs = planes_per_z > 0 ? nzs / planes_per_z : nzs;
    if (nzs < 1) nzs = 1;
    if (nzs > c->P.nz) nzs = c->P.nz;
    return (int)nzs;
}

void drop_graphs(lbm_ctx* c) {
    for (int k = 0; k < 2; ++k)
        if (c->graph_exec[k]) {
            cudaGraphExecDestroy(c->graph_exec[k]);
            c->graph_exec[k] = nullptr;
        }
}

// Captures graph_steps steps starting from buffer `start` (an even count returns to it).
int capture_graph(lbm_ctx* c, int start) {
    cudaGraph_t graph = nullptr;
    LBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int launches = 0, cur = start;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < c->graph_steps && e == cudaSuccess; ++k) {
        e = lbm::launch_step(c->P, c->scheme, c->fg[cur], c->fg[1 - cur], c->phi_fd, c->stream, &launches);
        cur = 1 - cur;
    }
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec[start], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->graph_exec[start] = nullptr;
        return set_error(c, LBM_ECUDA, "capturing the step graph failed: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

// The storage of the moving pairs (the FP16 scaling is a compile-time constant of Store<S>),
// and the face-flux weights for g held in that storage's units.
void apply_storage(Params& P, int storage) {
    P.storage = storage;
    P.flux_as = P.flux_a * lbm::storage_inv_g(storage);
    P.flux_bs = P.flux_b * lbm::storage_inv_g(storage);
}

int check_ctx(lbm_ctx* c) {
    if (!c) return set_error(nullptr, LBM_EINVAL, "null handle");
    LBM_CUDA(c, cudaSetDevice(c->device));
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_opts(lbm_opts* o) {
    if (!o) return;
    o->scheme = LBM_SCHEME_DIFFERENCE_FREE;
    o->storage = 0;
    o->courant = 0.997;
    o->walls = 0;
    o->stream = nullptr;
    o->graph_steps = 32;
}

int lbm_create(lbm_ctx** out, const int grid[3], int lattice, double tau_f, double tau_g, double M, double xi,
               double sigma, double rho_ratio, double mu_ratio, const double body_force[3], const lbm_opts* opts) {
    lbm_opts o;
    lbm_default_opts(&o);
    if (opts) o = *opts;
    return lbm::create_ctx(out, grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio, body_force, &o,
                           o.storage);
}

long long lbm_state_bytes(int lattice, const int grid[3], int storage) {
    if (!grid || (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) || storage < 0 || storage > 2) return 0;
    if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1) return 0;
    const long long N = (long long)grid[0] * grid[1] * grid[2];
    if (N >= (long long)INT_MAX) return 0;
    return (long long)lbm::state_bytes(lattice, N, storage);
}

int lbm_create_ext(lbm_ctx** out, const int grid[3], int lattice, double tau_f, double tau_g, double M, double xi,
                   double sigma, double rho_ratio, double mu_ratio, const double body_force[3], const lbm_opts* opts,
                   void* fg0, void* fg1, size_t bytes_each) {
    lbm_opts o;
    lbm_default_opts(&o);
    if (opts) o = *opts;
    if (out) *out = nullptr;
    if (!fg0 || !fg1) return set_error(nullptr, LBM_EINVAL, "the two state buffers may not be NULL");
    if ((reinterpret_cast<uintptr_t>(fg0) | reinterpret_cast<uintptr_t>(fg1)) % 16)
        return set_error(nullptr, LBM_EINVAL, "the state buffers must start on 16-byte boundaries");
    const uintptr_t a = reinterpret_cast<uintptr_t>(fg0), b = reinterpret_cast<uintptr_t>(fg1);
    if ((a < b ? b - a : a - b) < bytes_each)
        return set_error(nullptr, LBM_EINVAL, "the state buffers overlap");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(nullptr, LBM_ECUDA, "no CUDA device available");
    for (void* ptr : {fg0, fg1}) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
            (void)cudaGetLastError();
            return set_error(nullptr, LBM_EINVAL, "a state buffer is not memory the CUDA runtime knows");
        }
        if (attr.type != cudaMemoryTypeDevice || attr.device != dev)
            return set_error(nullptr, LBM_EINVAL, "the state buffers must be device memory of the current device");
    }
    void* fg[2] = {fg0, fg1};
    return lbm::create_ctx(out, grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio, body_force, &o,
                           o.storage, fg, bytes_each);
}

}  // extern "C"

int lbm::create_ctx(lbm_ctx** out, const int grid[3], int lattice, double tau_f, double tau_g, double M, double xi,
                    double sigma, double rho_ratio, double mu_ratio, const double body_force[3], const lbm_opts* opts,
                    int alloc_storage, void* const* ext_fg, size_t ext_bytes) {
    if (!out) return set_error(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid) return set_error(nullptr, LBM_EINVAL, "grid is NULL");
    lbm_opts o;
    lbm_default_opts(&o);
    if (opts) o = *opts;
    const int nx = grid[0], ny = grid[1], nz = grid[2];
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19)
        return set_error(nullptr, LBM_EINVAL, "lattice must be 9 (D2Q9) or 19 (D3Q19), got %d", lattice);
    if (nx < 3 || ny < 3) return set_error(nullptr, LBM_EINVAL, "nx and ny must be >= 3 (got %d, %d)", nx, ny);
    if (lattice == LBM_D2Q9 && nz != 1) return set_error(nullptr, LBM_EINVAL, "D2Q9 needs nz = 1 (got %d)", nz);
    if (lattice == LBM_D3Q19 && (nz < 3 || nz > 65535))
        return set_error(nullptr, LBM_EINVAL, "D3Q19 needs 3 <= nz <= 65535 (got %d)", nz);
    const long long N = (long long)nx * ny * nz;
    if (N >= (long long)INT_MAX) return set_error(nullptr, LBM_EINVAL, "nx*ny*nz must be < 2^31 (got %lld)", N);
    if (!(tau_f > 0) || !is_fin(tau_f)) return set_error(nullptr, LBM_EINVAL, "tau_f must be > 0");
    if (!is_fin(M) || !is_fin(tau_g) || (!(M > 0) && !(tau_g > 0)))
        return set_error(nullptr, LBM_EINVAL, "need M > 0 or tau_g > 0");
    if (!(xi >= 2) || !is_fin(xi)) return set_error(nullptr, LBM_EINVAL, "xi must be >= 2 (got %g)", xi);
    if (!(sigma >= 0) || !is_fin(sigma)) return set_error(nullptr, LBM_EINVAL, "sigma must be >= 0");
    if (!(rho_ratio > 0) || !is_fin(rho_ratio) || !(mu_ratio > 0) || !is_fin(mu_ratio))
        return set_error(nullptr, LBM_EINVAL, "rho_ratio and mu_ratio must be > 0");
    double G[3] = {0, 0, 0};
    if (body_force)
        for (int a = 0; a < 3; ++a) G[a] = body_force[a];
    for (int a = 0; a < 3; ++a)
        if (!is_fin(G[a])) return set_error(nullptr, LBM_EINVAL, "body_force must be finite");
    if (lattice == LBM_D2Q9 && G[2] != 0) return set_error(nullptr, LBM_EINVAL, "D2Q9 needs body_force[2] = 0");
    if (o.scheme != LBM_SCHEME_DIFFERENCE_FREE && o.scheme != LBM_SCHEME_FINITE_DIFFERENCE)
        return set_error(nullptr, LBM_EINVAL, "unknown scheme %d", o.scheme);
    if (o.storage < 0 || o.storage > 2)
        return set_error(nullptr, LBM_EINVAL, "storage must be 0 (FP32), 1 (FP16) or 2 (BF16), got %d", o.storage);
    if (o.walls < 0 || o.walls > 7 || (lattice == LBM_D2Q9 && (o.walls & 4)))
        return set_error(nullptr, LBM_EINVAL, "walls must be a mask of 1 (x), 2 (y), 4 (z, D3Q19 only); got %d",
                         o.walls);
    if (!(o.courant > 0 && o.courant <= 1)) return set_error(nullptr, LBM_EINVAL, "courant must be in (0, 1]");
    if (o.graph_steps < 0 || o.graph_steps == 1 || (o.graph_steps & 1))
        return set_error(nullptr, LBM_EINVAL, "graph_steps must be 0 or an even count >= 2 (got %d)", o.graph_steps);

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return set_error(nullptr, LBM_ENOMEM, "host allocation failed");
    std::memset(c, 0, sizeof(*c));
    std::snprintf(c->err, sizeof c->err, "no error");
    c->scheme = o.scheme;
    c->courant = o.courant;
    c->graph_steps = o.graph_steps;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return set_error(nullptr, LBM_ECUDA, "no CUDA device available");
    }

    // Parameters (Sec. 2.2, Sec. 2.3). tau_phi from M = tau_phi cs^2 dt when M > 0.
    Params& P = c->P;
    const double cs2 = 1.0 / 3.0;
    const double cc = o.courant;
    const double tau_phi = (M > 0) ? M / cs2 : tau_g;
    P.Q = lattice;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.nxy = nx * ny;
    P.N = N;
    P.lw_m = (float)(0.5 * cc * (1.0 + cc));   // c - c(1-c)/2: weight of f*(x - e) - f*(x)
    P.lw_p = (float)(-0.5 * cc * (1.0 - cc));  // -c(1-c)/2:    weight of f*(x + e) - f*(x)
    P.flux_a = (float)(0.5 * cc * (1.0 + cc) * 1073741824.0);  // face-flux weights times 2^30
    P.flux_b = (float)(0.5 * cc * (1.0 - cc) * 1073741824.0);
    P.tau_phi = (float)tau_phi;
    P.omega_g = (float)(1.0 / (tau_phi + 0.5));
    P.grad_s = (float)(tau_phi / (tau_phi + 0.5));
    P.grad_k = (float)(1.0 / ((tau_phi + 0.5) * cs2));
    P.tau_f = (float)tau_f;
    P.omega_f = (float)(1.0 / (tau_f + 0.5));
    P.rho2 = 1.0f;
    P.drho = (float)(rho_ratio - 1.0);
    P.mu_m1 = (float)(mu_ratio - 1.0);
    P.sigma = (float)sigma;
    P.four_over_delta = (float)(4.0 / xi);
    for (int a = 0; a < 3; ++a) P.G[a] = (float)G[a];
    P.w0 = 1.0f;       // p0 = cs^2 until lbm_init_phi sets it
    P.phi_ref = 1.0f;  // until lbm_init_phi picks the bulk phase of phi0
    P.phi_ref_fx = 1 << 30;
    P.walls = o.walls;
    P.general = (rho_ratio != 1.0 || mu_ratio != 1.0 || G[0] != 0 || G[1] != 0 || G[2] != 0 || o.walls) ? 1 : 0;
    apply_storage(P, o.storage);
    P.w0d = 1.0;
    P.phi_ref_d = 1.0;
    P.tau_phi_d = tau_phi;
    P.sigma_d = sigma;
    P.four_over_delta_d = 4.0 / xi;
    P.drho_d = rho_ratio - 1.0;
    P.rho2_d = 1.0;

    int rc = LBM_OK;
    auto fail = [&](int code) {
        std::snprintf(g_create_error, sizeof g_create_error, "%s", c->err);
        free_ctx(c);
        return code;
    };
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            set_error(c, LBM_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
            return fail(LBM_ECUDA);
        }
        c->own_stream = true;
    }
    if (alloc_storage < 0 || alloc_storage > 2 ||
        lbm::state_bytes(lattice, N, alloc_storage) < lbm::state_bytes(lattice, N, o.storage))
        alloc_storage = o.storage;
    const size_t pop_bytes = lbm::state_bytes(lattice, N, alloc_storage);
    if (ext_fg) {
        // the caller's buffers: used for the handle's lifetime, never freed here
        if (ext_bytes < pop_bytes) {
            set_error(c, LBM_EINVAL, "the state buffers hold %zu bytes each; this grid and storage need %zu", ext_bytes,
                      pop_bytes);
            return fail(LBM_EINVAL);
        }
        c->fg[0] = ext_fg[0];
        c->fg[1] = ext_fg[1];
        c->fg_bytes = ext_bytes;
        c->own_fg = false;
    } else {
        c->fg_bytes = pop_bytes;
        c->own_fg = true;
        for (int k = 0; k < 2 && rc == LBM_OK; ++k) {
            cudaError_t e = cudaMalloc(&c->fg[k], pop_bytes);
            if (e != cudaSuccess)
                rc = set_error(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                               "allocating %zu bytes of populations failed: %s", 2 * pop_bytes, cudaGetErrorString(e));
        }
    }
    if (rc == LBM_OK && c->scheme == LBM_SCHEME_FINITE_DIFFERENCE) {
        cudaError_t e = cudaMalloc(&c->phi_fd, (size_t)N * sizeof(float));
        if (e != cudaSuccess) rc = set_error(c, LBM_ENOMEM, "allocating the phi plane failed: %s", cudaGetErrorString(e));
    }
    if (rc == LBM_OK) {
        c->n_partials = lbm::mass_partials_needed(P);
        cudaError_t e = cudaMalloc(&c->partials, (size_t)3 * c->n_partials * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->result, 4 * sizeof(double));
        if (e != cudaSuccess) rc = set_error(c, LBM_ENOMEM, "allocating reduction scratch failed: %s", cudaGetErrorString(e));
    }
    if (rc != LBM_OK) return fail(rc);
    *out = c;
    return LBM_OK;
}

int lbm::ctx_error(lbm_ctx* c, int code, const char* msg) { return set_error(c, code, "%s", msg); }

int lbm::ctx_check(lbm_ctx* c) { return check_ctx(c); }

int lbm::ctx_mass_fixed(lbm_ctx* c, long long* sum) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->initialised) return set_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    LBM_CUDA(c, lbm::launch_phi_fixed_sum(c->P, c->fg[c->cur], c->partials, c->n_partials, c->result, c->stream));
    c->launches += 2;
    double r3;
    LBM_CUDA(c, cudaMemcpyAsync(&r3, c->result + 3, sizeof r3, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    std::memcpy(sum, &r3, sizeof *sum);
    return LBM_OK;
}

int lbm::ctx_restart_from_coarse(lbm_ctx* c, int f, const float* coarse, double p0) {
    int rc = check_ctx(c);
    if (rc) return rc;
    Params& P = c->P;
    P.w0d = p0 * 3.0;
    P.w0 = (float)P.w0d;
    drop_graphs(c);
    rc = ensure_staging(c, ((size_t)P.N + 1) / 2);  // N floats of upsampled phi
    if (rc) return rc;
    LBM_CUDA(c, lbm::launch_restart(P, coarse, f, p0, reinterpret_cast<float*>(c->staging), c->fg[c->cur], c->stream));
    c->launches += 2;
    c->initialised = true;
    c->version += 1;
    return LBM_OK;
}

int lbm::ctx_adjust_phi(lbm_ctx* c, long long delta) {
    LBM_CUDA(c, lbm::launch_adjust_phi(c->P, c->fg[c->cur], delta, c->stream));
    c->launches += 1;
    return LBM_OK;
}

int lbm::set_ctx_storage(lbm_ctx* c, int storage) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->initialised) return set_error(c, LBM_ESTATE, "the storage of a handle with state cannot change");
    if (storage < 0 || storage > 2 || lbm::state_bytes(c->P.Q, c->P.N, storage) > c->fg_bytes)
        return set_error(c, LBM_EINVAL, "storage %d does not fit this handle", storage);
    apply_storage(c->P, storage);
    drop_graphs(c);
    c->version += 1;
    return LBM_OK;
}

extern "C" {

int lbm_init_phi(lbm_ctx* c, const double* phi0, const double* u0, double p0) {
    return lbm_init_fields(c, phi0, u0, nullptr, p0);
}

int lbm_init_fields(lbm_ctx* c, const double* phi0, const double* u0, const double* p, double p0) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!phi0) return set_error(c, LBM_EINVAL, "phi0 is NULL");
    if (!(p0 > 0) || !is_fin(p0)) return set_error(c, LBM_EINVAL, "p0 must be > 0 and finite");
    Params& P = c->P;
    const long long Ncells = P.N;
    const size_t nxy = (size_t)P.nxy;
    const int per_z = 1 + (u0 ? 3 : 0) + (p ? 1 : 0);
    const int nzs = slab_depth(c, per_z, 2);
    rc = ensure_staging(c, (size_t)(nzs + 2 + (u0 ? 3 * nzs : 0) + (p ? nzs : 0)) * nxy);
    if (rc) return rc;
    double* phis = c->staging;
    double* us = c->staging + (size_t)(nzs + 2) * nxy;
    double* ps = us + (u0 ? (size_t)3 * nzs * nxy : 0);
    // one slab holds the whole grid: pass 1 copies phi0 and p to where pass 2 reads them, and
    // pass 2 copies them no more
    const bool one_slab = nzs >= P.nz;
    // Pass 1, before anything is written: every phi0 in [kPhiMin, kPhiMax] and every p > 0 and
    // finite, and the sum of phi0, checked on the device slab by slab (block partials added on
    // the host in a fixed order). Only when a value fails is the host array searched for it.
    double mean = 0.0;
    {
        const int nb = std::max(1, std::min(3 * c->n_partials / 2, 1024));
        std::vector<double> part(2 * (size_t)nb);
        double sum = 0.0, bad_phi = 0.0, bad_p = 0.0;
        auto check = [&](const double* dev, long long n, double lo, double hi, int open_low, double* bad,
                         double* total) -> int {
            LBM_CUDA(c, lbm::launch_check_values(dev, n, lo, hi, open_low, c->partials, nb, c->stream));
            LBM_CUDA(c, cudaMemcpyAsync(part.data(), c->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                        c->stream));
            LBM_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int b = 0; b < nb; ++b) {
                *bad += part[2 * b];
                if (total) *total += part[2 * b + 1];
            }
            return LBM_OK;
        };
        for (int z0 = 0; z0 < P.nz; z0 += nzs) {
            const int n = (z0 + nzs <= P.nz) ? nzs : P.nz - z0;
            const size_t cells = (size_t)n * nxy;
            double* dphi = one_slab ? phis + nxy : c->staging;
            LBM_CUDA(c, cudaMemcpyAsync(dphi, phi0 + (size_t)z0 * nxy, cells * sizeof(double), cudaMemcpyHostToDevice,
                                        c->stream));
            if ((rc = check(dphi, (long long)cells, kPhiMin, kPhiMax, 0, &bad_phi, &sum))) return rc;
            if (p) {
                double* dp = one_slab ? ps : c->staging;
                LBM_CUDA(c, cudaMemcpyAsync(dp, p + (size_t)z0 * nxy, cells * sizeof(double), cudaMemcpyHostToDevice,
                                            c->stream));
                if ((rc = check(dp, (long long)cells, 0.0, INFINITY, 1, &bad_p, nullptr))) return rc;
            }
        }
        if (bad_p > 0)
            for (long long k = 0; k < Ncells; ++k)
                if (!(p[k] > 0) || !is_fin(p[k])) return set_error(c, LBM_EINVAL, "p[%lld] = %g must be > 0 and finite", k, p[k]);
        if (bad_phi > 0)
            for (long long k = 0; k < Ncells; ++k)
                if (!(phi0[k] >= kPhiMin && phi0[k] <= kPhiMax))
                    return set_error(c, LBM_EINVAL, "phi0[%lld] = %g outside [%g, %g]", k, phi0[k], kPhiMin, kPhiMax);
        if (bad_p > 0 || bad_phi > 0) return set_error(c, LBM_EINVAL, "non-finite phi0 or p");
        mean = sum / (double)Ncells;
    }
    P.w0d = p0 * 3.0;  // w0 = p0 / cs^2: the level the f storage is shifted by
    P.w0 = (float)P.w0d;
    // g is stored as the deviation from the bulk phase (phi = 0 or 1) that covers most cells
    P.phi_ref_d = (mean >= 0.5) ? 1.0 : 0.0;
    P.phi_ref = (float)P.phi_ref_d;
    P.phi_ref_fx = (mean >= 0.5) ? (1 << 30) : 0;
    drop_graphs(c);  // captured steps carry the old parameters
    for (int z0 = 0; z0 < P.nz; z0 += nzs) {
        const int n = (z0 + nzs <= P.nz) ? nzs : P.nz - z0;
        // phi0 planes z0-1 .. z0+n: the slab's own planes in one copy, and the two halo planes,
        // periodic images or across a z wall the mirror image (zero normal gradient); D2Q9 has
        // only its one plane. With one slab the halos are copies of staged planes.
        if (!one_slab)
            LBM_CUDA(c, cudaMemcpyAsync(phis + nxy, phi0 + (size_t)z0 * nxy, (size_t)n * nxy * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream));
        if (P.Q != 9)
            for (int l : {-1, n}) {
                const int z = (P.walls & 4) ? std::min(std::max(z0 + l, 0), P.nz - 1) : ((z0 + l) % P.nz + P.nz) % P.nz;
                if (one_slab)
                    LBM_CUDA(c, cudaMemcpyAsync(phis + (size_t)(l + 1) * nxy, phis + (size_t)(z + 1) * nxy,
                                                nxy * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
                else
                    LBM_CUDA(c, cudaMemcpyAsync(phis + (size_t)(l + 1) * nxy, phi0 + (size_t)z * nxy,
                                                nxy * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            }
        if (u0)
            for (int a = 0; a < 3; ++a)
                LBM_CUDA(c, cudaMemcpyAsync(us + (size_t)a * n * nxy, u0 + (size_t)a * P.N + (size_t)z0 * nxy,
                                            (size_t)n * nxy * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (p && !one_slab)
            LBM_CUDA(c, cudaMemcpyAsync(ps, p + (size_t)z0 * nxy, (size_t)n * nxy * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream));
        LBM_CUDA(c, lbm::launch_init(P, z0, n, phis, u0 ? us : nullptr, p ? ps : nullptr, p0, c->fg[c->cur],
                                     c->stream));
        c->launches += 1;
    }
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->initialised = true;
    c->version += 1;
    return LBM_OK;
}

int lbm_graph_prepare(lbm_ctx* c) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->graph_steps <= 0) return set_error(c, LBM_EINVAL, "the handle replays no graphs (graph_steps 0)");
    if (!c->initialised) return set_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    if (!c->graph_exec[c->cur]) {
        rc = capture_graph(c, c->cur);
        if (rc) return rc;
    }
    LBM_CUDA(c, cudaGraphUpload(c->graph_exec[c->cur], c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n < 0) return set_error(c, LBM_EINVAL, "n must be >= 0 (got %d)", n);
    if (!c->initialised) return set_error(c, LBM_ESTATE, "lbm_step before lbm_init_phi");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LBM_CUDA(c, cudaStreamIsCapturing(c->stream, &cap));
    if (c->graph_steps > 0 && cap == cudaStreamCaptureStatusNone) {
        const int per_step = (c->scheme == LBM_SCHEME_FINITE_DIFFERENCE) ? 2 : 1;
        while (n >= c->graph_steps) {
            if (!c->graph_exec[c->cur]) {
                rc = capture_graph(c, c->cur);
                if (rc) return rc;
            }
            LBM_CUDA(c, cudaGraphLaunch(c->graph_exec[c->cur], c->stream));
            c->launches += (long long)per_step * c->graph_steps;
            n -= c->graph_steps;  // an even number of steps leaves the current buffer unchanged
        }
    }
    for (int k = 0; k < n; ++k) {
        const int a = c->cur, b = 1 - c->cur;
        int launches = 0;
        LBM_CUDA(c, lbm::launch_step(c->P, c->scheme, c->fg[a], c->fg[b], c->phi_fd, c->stream, &launches));
        c->launches += launches;
        c->cur = b;
    }
    return LBM_OK;
}

static int fields_out(lbm_ctx* c, int mask, double* const* dst /* 11 planes, NULL = skip */) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->initialised) return set_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    Params& P = c->P;
    const size_t nxy = (size_t)P.nxy;
    const void* fg = c->fg[c->cur];
    if (c->scheme == LBM_SCHEME_FINITE_DIFFERENCE) {
        LBM_CUDA(c, lbm::launch_fd_phi(P, fg, c->phi_fd, c->stream));
        c->launches += 1;
    }
    // Destinations in page-locked host memory are written by the kernel itself across the host
    // link, in one launch over the grid, with no staging copy; any other host memory goes slab
    // by slab through device staging and cudaMemcpyAsync.
    lbm::FieldOut direct{};
    bool all_direct = P.nz <= 65535;
    for (int j = 0; j < 11 && all_direct; ++j) {
        if (!dst[j]) continue;
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, dst[j]) != cudaSuccess) {
            (void)cudaGetLastError();
            all_direct = false;
        } else if (a.type != cudaMemoryTypeHost || !a.devicePointer) {
            all_direct = false;
        } else {
            direct.p[j] = static_cast<double*>(a.devicePointer);
        }
    }
    if (all_direct) {
        LBM_CUDA(c, lbm::launch_moments(P, c->scheme, 0, P.nz, fg, c->phi_fd, mask, direct, c->stream));
        c->launches += 1;
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    const int nzs = slab_depth(c, 11, 0);
    rc = ensure_staging(c, (size_t)11 * nzs * nxy);
    if (rc) return rc;
    for (int z0 = 0; z0 < P.nz; z0 += nzs) {
        const int n = (z0 + nzs <= P.nz) ? nzs : P.nz - z0;
        const size_t slab = (size_t)n * nxy;
        lbm::FieldOut staged{};
        for (int j = 0; j < 11; ++j) staged.p[j] = c->staging + (size_t)j * slab;
        LBM_CUDA(c, lbm::launch_moments(P, c->scheme, z0, n, fg, c->phi_fd, mask, staged, c->stream));
        c->launches += 1;
        for (int j = 0; j < 11; ++j) {
            if (!dst[j]) continue;
            LBM_CUDA(c, cudaMemcpyAsync(dst[j] + (size_t)z0 * nxy, c->staging + (size_t)j * slab, slab * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream));
        }
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* phi, double* p, double* u) {
    if (!c) return set_error(nullptr, LBM_EINVAL, "null handle");
    const size_t N = c ? (size_t)c->P.N : 0;
    double* dst[11] = {phi, p, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr,
                       nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const int mask = (phi ? 1 : 0) | (p ? 2 : 0) | (u ? 4 : 0);
    if (!mask) return LBM_OK;
    return fields_out(c, mask, dst);
}

int lbm_gradients(lbm_ctx* c, double* grad_phi, double* normal) {
    if (!c) return set_error(nullptr, LBM_EINVAL, "null handle");
    const size_t N = (size_t)c->P.N;
    double* dst[11] = {nullptr, nullptr, nullptr, nullptr, nullptr,
                       grad_phi, grad_phi ? grad_phi + N : nullptr, grad_phi ? grad_phi + 2 * N : nullptr,
                       normal, normal ? normal + N : nullptr, normal ? normal + 2 * N : nullptr};
    const int mask = (grad_phi ? 8 : 0) | (normal ? 16 : 0);
    if (!mask) return LBM_OK;
    return fields_out(c, mask, dst);
}

int lbm_mass(lbm_ctx* c, double* sum_phi, double* sum_rho_phi) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->initialised) return set_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    LBM_CUDA(c, lbm::launch_mass(c->P, c->fg[c->cur], c->partials, c->n_partials, c->result, c->stream));
    c->launches += 2;
    double r[3];
    LBM_CUDA(c, cudaMemcpyAsync(r, c->result, sizeof r, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sum_phi) *sum_phi = r[0];
    if (sum_rho_phi) *sum_rho_phi = r[1];
    if (r[2] != 0.0) return set_error(c, LBM_ENONFINITE, "%.0f stored populations are not finite", r[2]);
    return LBM_OK;
}

int lbm_diagnostics(lbm_ctx* c, const double centre[3], double r_in, double r_out, lbm_diag* out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!centre || !out) return set_error(c, LBM_EINVAL, "centre and out may not be NULL");
    if (!is_fin(centre[0]) || !is_fin(centre[1]) || !is_fin(centre[2]) || !is_fin(r_in) || !is_fin(r_out))
        return set_error(c, LBM_EINVAL, "centre, r_in and r_out must be finite");
    if (!c->initialised) return set_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    const Params& P = c->P;
    // a few cells per thread: after its first, a thread rarely needs FP64 for the largest u^2
    const int nb = std::max(1, std::min(c->n_partials, 1024));
    // scratch: the per-block partials, then the 7 result doubles
    const size_t part_doubles = (lbm::diag_partial_bytes(nb) + sizeof(double) - 1) / sizeof(double);
    const size_t n_axes = (size_t)P.nx + P.ny + P.nz;
    rc = ensure_staging(c, part_doubles + 8 + n_axes + (n_axes + 1) / 2);
    if (rc) return rc;
    // the squared distance along each axis per coordinate, evaluated here with the operations the
    // definition names (minimum image on periodic axes), then the same rounded to FP32
    std::vector<double> d2(n_axes + (n_axes + 1) / 2);
    for (int i = 0; i < P.nx; ++i) d2[i] = lbm::axis_d2_host(i, centre[0], P.nx, P.walls & 1);
    for (int i = 0; i < P.ny; ++i) d2[P.nx + i] = lbm::axis_d2_host(i, centre[1], P.ny, P.walls & 2);
    for (int i = 0; i < P.nz; ++i) d2[P.nx + P.ny + i] = lbm::axis_d2_host(i, centre[2], P.nz, P.walls & 4);
    float* f2 = reinterpret_cast<float*>(d2.data() + n_axes);
    for (size_t i = 0; i < n_axes; ++i) f2[i] = (float)d2[i];
    double* d2_dev = c->staging + part_doubles + 8;
    LBM_CUDA(c, cudaMemcpyAsync(d2_dev, d2.data(), d2.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const void* fg = c->fg[c->cur];
    if (c->scheme == LBM_SCHEME_FINITE_DIFFERENCE) {
        LBM_CUDA(c, lbm::launch_fd_phi(P, fg, c->phi_fd, c->stream));
        c->launches += 1;
    }
    double* result = c->staging + part_doubles;
    LBM_CUDA(c, lbm::launch_diagnostics(P, c->scheme, fg, c->phi_fd, d2_dev, r_in, r_out, c->staging, nb, result,
                                        c->stream));
    c->launches += 2;
    double r[7];
    LBM_CUDA(c, cudaMemcpyAsync(r, result, sizeof r, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    out->max_speed = r[0];
    long long arg;
    std::memcpy(&arg, &r[1], sizeof arg);
    out->argmax = arg;
    out->kinetic = r[2];
    out->p_in = r[3];
    out->p_out = r[4];
    out->n_in = (long long)r[5];
    out->n_out = (long long)r[6];
    return LBM_OK;
}

static int pops_io(lbm_ctx* c, double* f_out, double* g_out, const double* f_in, const double* g_in) {
    int rc = check_ctx(c);
    if (rc) return rc;
    Params& P = c->P;
    const size_t nxy = (size_t)P.nxy;
    const int nzs = slab_depth(c, P.Q, 0);
    rc = ensure_staging(c, (size_t)P.Q * nzs * nxy);
    if (rc) return rc;
    for (int is_f = 1; is_f >= 0; --is_f) {
        double* host_out = is_f ? f_out : g_out;
        const double* host_in = is_f ? f_in : g_in;
        void* dev = c->fg[c->cur];
        if (!host_out && !host_in) continue;
        for (int z0 = 0; z0 < P.nz; z0 += nzs) {
            const int n = (z0 + nzs <= P.nz) ? nzs : P.nz - z0;
            const size_t slab = (size_t)n * nxy, bytes = slab * sizeof(double);
            if (host_in) {
                for (int q = 0; q < P.Q; ++q)
                    LBM_CUDA(c, cudaMemcpyAsync(c->staging + q * slab, host_in + (size_t)q * P.N + (size_t)z0 * nxy,
                                                bytes, cudaMemcpyHostToDevice, c->stream));
                LBM_CUDA(c, lbm::launch_pops_from_f64(P, c->staging, is_f, z0, n, dev, c->stream));
            } else {
                LBM_CUDA(c, lbm::launch_pops_to_f64(P, dev, is_f, z0, n, c->staging, c->stream));
                for (int q = 0; q < P.Q; ++q)
                    LBM_CUDA(c, cudaMemcpyAsync(host_out + (size_t)q * P.N + (size_t)z0 * nxy, c->staging + q * slab,
                                                bytes, cudaMemcpyDeviceToHost, c->stream));
            }
            c->launches += 1;
            LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        }
    }
    return LBM_OK;
}

int lbm_get_pops(lbm_ctx* c, double* f, double* g) {
    if (!c) return set_error(nullptr, LBM_EINVAL, "null handle");
    if (!c->initialised) return set_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    return pops_io(c, f, g, nullptr, nullptr);
}

int lbm_set_pops(lbm_ctx* c, const double* f, const double* g) {
    if (!c) return set_error(nullptr, LBM_EINVAL, "null handle");
    if (!f || !g) return set_error(c, LBM_EINVAL, "f and g are required");
    for (long long k = 0; k < c->P.N; ++k) {
        double phi = 0.0;
        for (int q = 0; q < c->P.Q; ++q) phi += g[(size_t)q * c->P.N + k];
        if (!(phi >= kPhiMin && phi <= kPhiMax))
            return set_error(c, LBM_EINVAL, "sum of g at cell %lld = %g outside [%g, %g]", k, phi, kPhiMin, kPhiMax);
    }
    int rc = pops_io(c, nullptr, nullptr, f, g);
    c->version += 1;
    if (rc == LBM_OK) c->initialised = true;
    return rc;
}

long long lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : 0; }

double lbm_tau_phi(const lbm_ctx* c) { return c ? c->P.tau_phi_d : 0.0; }

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : g_create_error; }

void lbm_destroy(lbm_ctx* c) {
    if (c && c->batch_owned) return;  // a case of a batch: freed by lbm_batch_destroy
    free_ctx(c);
}

int lbm_lattice_tables(int lattice, int* d, int* e, double* w) {
    if (lattice == LBM_D2Q9) {
        if (d) *d = lbm::Lat<9>::D;
        for (int i = 0; i < 9; ++i) {
            if (e) {
                e[3 * i] = lbm::Lat<9>::cx(i);
                e[3 * i + 1] = lbm::Lat<9>::cy(i);
                e[3 * i + 2] = lbm::Lat<9>::cz(i);
            }
            if (w) w[i] = lbm::Lat<9>::wd(i);
        }
        return LBM_OK;
    }
    if (lattice == LBM_D3Q19) {
        if (d) *d = lbm::Lat<19>::D;
        for (int i = 0; i < 19; ++i) {
            if (e) {
                e[3 * i] = lbm::Lat<19>::cx(i);
                e[3 * i + 1] = lbm::Lat<19>::cy(i);
                e[3 * i + 2] = lbm::Lat<19>::cz(i);
            }
            if (w) w[i] = lbm::Lat<19>::wd(i);
        }
        return LBM_OK;
    }
    return LBM_EINVAL;
}

}  // extern "C"
