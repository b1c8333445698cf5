// lbm_surrogate.cu -- the surrogate entry points (include/lbm_surrogate.h): the network's
// parameters and workspaces, its forward pass, gradients and Adam step (surrogate_kernels.cu),
// and the judged jump of a lattice (surrogate_glue.cu for the field transfers).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "../../include/lbm_surrogate.h"
#include "lbm_ctx.h"
#include "surrogate.h"

using lbm::net::kFieldChannels;
using lbm::net::kHidden;
using lbm::net::kLayers;

struct lbm_net {
    int fp16;
    cudaStream_t stream;
    bool own_stream;
    int cin[kLayers], cout[kLayers];
    long long w_off[kLayers], b_off[kLayers], n_params;
    float *params, *grads, *m, *v;   // device, n_params each
    float* wt;                        // adjoint weights of one layer
    __half* wimg;                     // FP16 tensor-core weight image of one 32 -> 32 layer
    int* tc_err;                      // set by the tensor-core kernel if a wait timed out
    long long tc_spin;                // polls of an mbarrier before a tensor-core wait for a step gives up
    float* wscratch;                  // partial sums of the tensor-core weight gradients
    int adam_step;
    float loss_w[kFieldChannels];     // per-channel weights of the loss
    // workspace for (batch, voxels)
    long long ws_elems;               // batch * voxels the workspace holds
    void* x_t;                        // input in the activation type
    void* h[kLayers - 1];             // hidden activations
    float* d;                         // last layer's output [B][5]
    float *ga, *gb;                   // gradient ping-pong [B][32]
    double* partials;
    int n_partials;
    char err[512];
};

namespace {

thread_local char g_net_error[512] = "no error";

int nerr(lbm_net* n, int code, const char* fmt, ...) {
    char* dst = n ? n->err : g_net_error;
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    // a failed allocation is reported here, synchronously, and is not sticky: clear it, or the
    // next launch's error check would report it again
    if (code == LBM_ENOMEM) (void)cudaGetLastError();
    return code;
}

#define LBM_NCUDA(n, call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return nerr((n), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,          \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

void free_ws(lbm_net* n) {
    cudaFree(n->x_t);
    for (int l = 0; l < kLayers - 1; ++l) cudaFree(n->h[l]);
    cudaFree(n->d);
    cudaFree(n->ga);
    cudaFree(n->gb);
    cudaFree(n->partials);
    n->x_t = nullptr;
    for (int l = 0; l < kLayers - 1; ++l) n->h[l] = nullptr;
    n->d = n->ga = n->gb = nullptr;
    n->partials = nullptr;
    n->ws_elems = 0;
}

void free_net(lbm_net* n) {
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    free_ws(n);
    cudaFree(n->params);
    cudaFree(n->grads);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->wt);
    cudaFree(n->wimg);
    cudaFree(n->tc_err);
    cudaFree(n->wscratch);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

int ensure_ws(lbm_net* n, int batch, long long vox) {
    const long long e = (long long)batch * vox;
    const size_t act = n->fp16 ? 2 : 4;
    if (e <= n->ws_elems) return LBM_OK;
    free_ws(n);
    LBM_NCUDA(n, cudaMalloc(&n->x_t, (size_t)e * kFieldChannels * act));
    for (int l = 0; l < kLayers - 1; ++l) LBM_NCUDA(n, cudaMalloc(&n->h[l], (size_t)e * kHidden * act));
    LBM_NCUDA(n, cudaMalloc(&n->d, (size_t)e * kFieldChannels * sizeof(float)));
    LBM_NCUDA(n, cudaMalloc(&n->ga, (size_t)e * kHidden * sizeof(float)));
    LBM_NCUDA(n, cudaMalloc(&n->gb, (size_t)e * kHidden * sizeof(float)));
    n->n_partials = lbm::net::loss_blocks(e * kFieldChannels);
    LBM_NCUDA(n, cudaMalloc(&n->partials, (size_t)n->n_partials * sizeof(double)));
    n->ws_elems = e;
    return LBM_OK;
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014)
// and a Box-Muller normal from two of its outputs.
struct SplitMix64 {
    unsigned long long s;
    unsigned long long next() {
        unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

int check_grid(lbm_net* n, int batch, const int grid[3]) {
    if (!grid || batch < 1 || grid[0] < 1 || grid[1] < 1 || grid[2] < 1)
        return nerr(n, LBM_EINVAL, "need batch >= 1 and a grid of positive extents");
    return LBM_OK;
}

// The layers run on the tensor cores with FP16 activations (channels zero-padded to 32); the FP32
// mode stays on the CUDA-core kernels, whose results the gradient checks compare with FP64 at 1e-5.
bool on_tensor_cores(const lbm_net* n) { return n->fp16 != 0; }

// A timeout of the tensor-core kernel, read at a point where the stream has been synchronised.
// The flag is cleared once reported, so the network stays usable: the kernel that timed out has
// waited for its MMAs in flight and freed its tensor memory before it returned.
int check_tc(lbm_net* n) {
    int flag = 0;
    LBM_NCUDA(n, cudaMemcpy(&flag, n->tc_err, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        LBM_NCUDA(n, cudaMemset(n->tc_err, 0, sizeof(int)));
        return nerr(n, LBM_ETIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
    }
    return LBM_OK;
}

// Forward pass keeping the activations; the last layer's output in n->d.
int forward_keep(lbm_net* n, const float* x, int batch, const int grid[3]) {
    const int D = grid[2], H = grid[1], W = grid[0];
    const long long vox = (long long)D * H * W;
    int rc = ensure_ws(n, batch, vox);
    if (rc) return rc;
    LBM_NCUDA(n, lbm::net::cast_to(x, n->x_t, n->fp16, (long long)batch * kFieldChannels * vox, n->stream));
    const void* in = n->x_t;
    for (int l = 0; l < kLayers; ++l) {
        const bool last = l == kLayers - 1;
        void* out = last ? (void*)n->d : n->h[l];
        if (on_tensor_cores(n)) {
            LBM_NCUDA(n, lbm::net::weight_image(n->params + n->w_off[l], n->cout[l], n->cin[l], n->wimg, n->stream));
            LBM_NCUDA(n, lbm::net::conv32_tc(in, 1, n->cin[l], 1.0f, n->wimg, n->params + n->b_off[l], out, last ? 0 : 1,
                                             n->cout[l], last ? 0 : 1, batch, D, H, W, n->tc_spin, n->tc_err,
                                             n->stream));
        } else {
            LBM_NCUDA(n, lbm::net::conv_forward(in, n->fp16, n->cin[l], n->params + n->w_off[l], n->params + n->b_off[l],
                                                out, last ? 0 : n->fp16, n->cout[l], last ? 0 : 1, batch, D, H, W, n->stream));
        }
        in = out;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_net_create(lbm_net** out, int activations_fp16, unsigned long long seed, void* stream) {
    if (!out) return nerr(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_net* n = new (std::nothrow) lbm_net();
    if (!n) return nerr(nullptr, LBM_ENOMEM, "host allocation failed");
    std::snprintf(n->err, sizeof n->err, "no error");
    n->fp16 = activations_fp16 ? 1 : 0;
    n->tc_spin = lbm::net::kTcWaitPolls;
    for (int c = 0; c < kFieldChannels; ++c) n->loss_w[c] = 1.f;
    auto fail = [&](int code) {
        std::snprintf(g_net_error, sizeof g_net_error, "%s", n->err);
        free_net(n);
        return code;
    };
    if (stream) {
        n->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(nerr(n, LBM_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e)));
        n->own_stream = true;
    }
    const int chans[kLayers + 1] = {kFieldChannels, kHidden, kHidden, kHidden, kFieldChannels};
    long long off = 0;
    for (int l = 0; l < kLayers; ++l) {
        n->cin[l] = chans[l];
        n->cout[l] = chans[l + 1];
        n->w_off[l] = off;
        off += (long long)n->cout[l] * n->cin[l] * 27;
        n->b_off[l] = off;
        off += n->cout[l];
    }
    n->n_params = off;
    std::vector<float> h((size_t)off, 0.f);
    SplitMix64 rng{seed};
    for (int l = 0; l < kLayers; ++l) {
        const double sd = std::sqrt(2.0 / (27.0 * n->cin[l])) * (l == kLayers - 1 ? 0.1 : 1.0);
        for (long long i = 0; i < (long long)n->cout[l] * n->cin[l] * 27; ++i) h[n->w_off[l] + i] = (float)(sd * rng.normal());
    }
    const size_t bytes = (size_t)off * sizeof(float);
    cudaError_t e = cudaMalloc(&n->params, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&n->grads, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&n->wt, (size_t)kHidden * kHidden * 27 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->wimg, lbm::net::weight_image_bytes());
    if (e == cudaSuccess) e = cudaMalloc(&n->tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&n->wscratch, lbm::net::wgrad_scratch_floats() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(n->params, h.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->grads, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, bytes);
    if (e != cudaSuccess) return fail(nerr(n, LBM_ENOMEM, "allocating the network failed: %s", cudaGetErrorString(e)));
    *out = n;
    return LBM_OK;
}

long long lbm_net_param_count(const lbm_net* n) { return n ? n->n_params : 0; }

int lbm_net_get_params(lbm_net* n, float* host) {
    if (!n || !host) return nerr(n, LBM_EINVAL, "null argument");
    LBM_NCUDA(n, cudaMemcpyAsync(host, n->params, (size_t)n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    LBM_NCUDA(n, cudaStreamSynchronize(n->stream));
    return check_tc(n);
}

int lbm_net_set_params(lbm_net* n, const float* host) {
    if (!n || !host) return nerr(n, LBM_EINVAL, "null argument");
    LBM_NCUDA(n, cudaMemcpyAsync(n->params, host, (size_t)n->n_params * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    LBM_NCUDA(n, cudaStreamSynchronize(n->stream));
    return LBM_OK;
}

int lbm_net_get_grads(lbm_net* n, float* host) {
    if (!n || !host) return nerr(n, LBM_EINVAL, "null argument");
    LBM_NCUDA(n, cudaMemcpyAsync(host, n->grads, (size_t)n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    LBM_NCUDA(n, cudaStreamSynchronize(n->stream));
    return LBM_OK;
}

int lbm_net_forward(lbm_net* n, const float* x, float* y, int batch, const int grid[3]) {
    if (!n || !x || !y) return nerr(n, LBM_EINVAL, "null argument");
    int rc = check_grid(n, batch, grid);
    if (rc) return rc;
    rc = forward_keep(n, x, batch, grid);
    if (rc) return rc;
    const long long e = (long long)batch * kFieldChannels * grid[0] * grid[1] * grid[2];
    LBM_NCUDA(n, lbm::net::residual(x, n->d, y, e, n->stream));
    return LBM_OK;
}

int lbm_net_gradients(lbm_net* n, const float* x, const float* target, int batch, const int grid[3], double* loss) {
    if (!n || !x || !target) return nerr(n, LBM_EINVAL, "null argument");
    int rc = check_grid(n, batch, grid);
    if (rc) return rc;
    rc = forward_keep(n, x, batch, grid);
    if (rc) return rc;
    const int D = grid[2], H = grid[1], W = grid[0];
    const long long vox = (long long)D * H * W, e = (long long)batch * kFieldChannels * vox;
    LBM_NCUDA(n, lbm::net::loss_and_grad(x, n->d, target, n->ga, e, vox, n->loss_w, n->partials, n->stream));
    LBM_NCUDA(n, cudaMemsetAsync(n->grads, 0, (size_t)n->n_params * sizeof(float), n->stream));
    float* g = n->ga;      // gradient of the current layer's output
    float* other = n->gb;
    const float grad_scale = std::ldexp(1.0f, std::ilogb((double)e));  // the power of two nearest below e
    for (int l = kLayers - 1; l >= 0; --l) {
        const void* h_in = (l == 0) ? n->x_t : n->h[l - 1];
        if (on_tensor_cores(n))
            LBM_NCUDA(n, lbm::net::wgrad32_tc(g, n->cout[l], grad_scale, h_in, n->fp16, n->cin[l], n->grads + n->w_off[l],
                                              n->grads + n->b_off[l], batch, D, H, W, n->tc_spin, n->wscratch,
                                              n->tc_err, n->stream));
        else
            LBM_NCUDA(n, lbm::net::conv_wgrad(g, n->cout[l], h_in, n->fp16, n->cin[l], n->grads + n->w_off[l],
                                              n->grads + n->b_off[l], batch, D, H, W, n->stream));
        if (l == 0) break;
        LBM_NCUDA(n, lbm::net::flip_transpose(n->params + n->w_off[l], n->cout[l], n->cin[l], n->wt, n->stream));
        if (on_tensor_cores(n)) {
            LBM_NCUDA(n, lbm::net::weight_image(n->wt, n->cin[l], n->cout[l], n->wimg, n->stream));
            // the loss gradient is 2 diff / (elements): scale it back to order one before FP16
            LBM_NCUDA(n, lbm::net::conv32_tc(g, 0, n->cout[l], grad_scale, n->wimg, nullptr, other, 0, n->cin[l], 0, batch,
                                             D, H, W, n->tc_spin, n->tc_err, n->stream));
        } else {
            LBM_NCUDA(n, lbm::net::conv_forward(g, 0, n->cout[l], n->wt, nullptr, other, 0, n->cin[l], 0, batch, D, H, W,
                                                n->stream));
        }
        LBM_NCUDA(n, lbm::net::relu_mask(other, n->h[l - 1], n->fp16, (long long)batch * n->cin[l] * vox, n->stream));
        float* t = g;
        g = other;
        other = t;
    }
    if (loss) {
        std::vector<double> part((size_t)n->n_partials);
        LBM_NCUDA(n, cudaMemcpyAsync(part.data(), n->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                     n->stream));
        LBM_NCUDA(n, cudaStreamSynchronize(n->stream));
        double s = 0.0;
        for (double v : part) s += v;
        *loss = s / (double)e;
    } else {
        LBM_NCUDA(n, cudaStreamSynchronize(n->stream));
    }
    return check_tc(n);
}

int lbm_net_set_loss_weights(lbm_net* n, const float w[5]) {
    if (!n || !w) return nerr(n, LBM_EINVAL, "null argument");
    for (int c = 0; c < kFieldChannels; ++c)
        if (!(w[c] >= 0.f) || !std::isfinite(w[c])) return nerr(n, LBM_EINVAL, "loss weights must be finite and >= 0");
    for (int c = 0; c < kFieldChannels; ++c) n->loss_w[c] = w[c];
    return LBM_OK;
}

int lbm_net_adam(lbm_net* n, float lr) {
    if (!n) return nerr(nullptr, LBM_EINVAL, "null network");
    if (!(lr > 0.f)) return nerr(n, LBM_EINVAL, "lr must be > 0");
    n->adam_step += 1;
    LBM_NCUDA(n, lbm::net::adam(n->params, n->grads, n->m, n->v, n->n_params, lr, n->adam_step, n->stream));
    return LBM_OK;
}

int lbm_net_fail_waits(lbm_net* n, int on) {
    if (!n) return nerr(nullptr, LBM_EINVAL, "null network");
    n->tc_spin = on ? 0 : lbm::net::kTcWaitPolls;
    return LBM_OK;
}

const char* lbm_net_last_error(const lbm_net* n) { return n ? n->err : g_net_error; }

void lbm_net_destroy(lbm_net* n) { free_net(n); }

int lbm_coarse_fields(lbm_ctx* c, int f, float* out) {
    int rc = lbm::ctx_check(c);
    if (rc) return rc;
    if (!out || f < 1 || c->P.nx % f || c->P.ny % f || c->P.nz % f)
        return lbm::ctx_error(c, LBM_EINVAL, "factor must divide nx, ny and nz, and out may not be NULL");
    if (!c->initialised) return lbm::ctx_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    if (c->scheme != LBM_SCHEME_DIFFERENCE_FREE) return lbm::ctx_error(c, LBM_EINVAL, "coarse fields need the difference-free scheme");
    cudaError_t e = lbm::launch_coarsen(c->P, c->fg[c->cur], f, out, c->stream);
    if (e != cudaSuccess) return lbm::ctx_error(c, LBM_ECUDA, cudaGetErrorString(e));
    c->launches += 1;
    return LBM_OK;
}

int lbm_coarse_phi(lbm_ctx* c, int f, float* out) {
    int rc = lbm::ctx_check(c);
    if (rc) return rc;
    if (!out || f < 1 || f > 32 || 32 % f || c->P.nx % f || c->P.ny % f || c->P.nz % f)
        return lbm::ctx_error(c, LBM_EINVAL, "factor must divide 32, nx, ny and nz, and out may not be NULL");
    if (!c->initialised) return lbm::ctx_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    cudaError_t e = lbm::launch_coarse_phi(c->P, c->fg[c->cur], f, out, c->stream);
    if (e != cudaSuccess) return lbm::ctx_error(c, LBM_ECUDA, cudaGetErrorString(e));
    c->launches += 1;
    return LBM_OK;
}

int lbm_restart_from_coarse(lbm_ctx* c, int f, const float* coarse, double p0) {
    int rc = lbm::ctx_check(c);
    if (rc) return rc;
    if (!coarse || f < 1 || c->P.nx % f || c->P.ny % f || c->P.nz % f)
        return lbm::ctx_error(c, LBM_EINVAL, "factor must divide nx, ny and nz, and coarse may not be NULL");
    if (!(p0 > 0) || !std::isfinite(p0)) return lbm::ctx_error(c, LBM_EINVAL, "p0 must be > 0 and finite");
    if (!c->initialised) return lbm::ctx_error(c, LBM_ESTATE, "no state to hold the mass of: call lbm_init_phi first");
    long long before = 0, after = 0;
    rc = lbm::ctx_mass_fixed(c, &before);
    if (rc) return rc;
    rc = lbm::ctx_restart_from_coarse(c, f, coarse, p0);
    if (rc) return rc;
    rc = lbm::ctx_mass_fixed(c, &after);
    if (rc) return rc;
    if (after != before) {
        rc = lbm::ctx_adjust_phi(c, before - after);
        if (rc) return rc;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return lbm::ctx_error(c, LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}

namespace {

// Whether the jump projects the predicted velocity: a grid without walls whose coarse extents
// the projection takes.
bool jump_projects(const lbm_ctx* c, int f) {
    const int grid_c[3] = {c->P.nx / f, c->P.ny / f, c->P.nz / f};
    return c->P.walls == 0 && lbm::project_extents_ok(grid_c);
}

// Carves the jump's buffers out of the handle's workspace, growing it if it is too small: a
// backup state, four coarse field arrays, the judge's four FP64 measures and the projection's
// scratch (*proj, NULL when the jump does not project).
int jump_workspace(lbm_ctx* c, int f, void** backup, float* fields[4], double** measures, void** proj) {
    const long long nc = (long long)(c->P.nx / f) * (c->P.ny / f) * (c->P.nz / f);
    const size_t align = 256;
    const size_t sb = (c->fg_bytes + align - 1) / align * align;
    const size_t fb = ((size_t)5 * nc * sizeof(float) + align - 1) / align * align;
    const size_t pb = jump_projects(c, f) ? lbm::project_workspace_bytes(c->P.nx / f, c->P.ny / f, c->P.nz / f) : 0;
    const size_t need = sb + 4 * fb + align + pb;
    if (c->jump_ws_bytes < need) {
        cudaFree(c->jump_ws);
        c->jump_ws = nullptr;
        c->jump_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&c->jump_ws, need);
        if (e != cudaSuccess) return lbm::ctx_error(c, LBM_ENOMEM, cudaGetErrorString(e));
        c->jump_ws_bytes = need;
    }
    char* base = static_cast<char*>(c->jump_ws);
    *backup = base;
    for (int i = 0; i < 4; ++i) fields[i] = reinterpret_cast<float*>(base + sb + i * fb);
    *measures = reinterpret_cast<double*>(base + sb + 4 * fb);
    *proj = pb ? base + sb + 4 * fb + align : nullptr;
    return LBM_OK;
}

}  // namespace

int lbm_surrogate_reserve(lbm_ctx* c, int f) {
    int rc = lbm::ctx_check(c);
    if (rc) return rc;
    if (f < 1 || c->P.nx % f || c->P.ny % f || c->P.nz % f)
        return lbm::ctx_error(c, LBM_EINVAL, "factor must divide nx, ny and nz");
    void* backup;
    float* fields[4];
    double* measures;
    void* proj;
    return jump_workspace(c, f, &backup, fields, &measures, &proj);
}

int lbm_surrogate_jump(lbm_ctx* c, lbm_net* n, int f, const float mean_std[10], int k, int judge_steps, double mass_tol,
                       double relax_tol, double interface_tol, lbm_jump_report* rep) {
    int rc = lbm::ctx_check(c);
    if (rc) return rc;
    if (!n || !mean_std || !rep || k < 1 || judge_steps < 1 || !(mass_tol >= 0) || !(relax_tol > 0) ||
        !(interface_tol >= 0) || std::isnan(relax_tol))
        return lbm::ctx_error(c, LBM_EINVAL, "need a network, mean_std, a report, k >= 1, judge_steps >= 1 and tolerances");
    if (f < 1 || c->P.nx % f || c->P.ny % f || c->P.nz % f)
        return lbm::ctx_error(c, LBM_EINVAL, "factor must divide nx, ny and nz");
    if (!c->initialised) return lbm::ctx_error(c, LBM_ESTATE, "no state: call lbm_init_phi first");
    const auto t0 = std::chrono::steady_clock::now();
    std::memset(rep, 0, sizeof *rep);
    const int grid_c[3] = {c->P.nx / f, c->P.ny / f, c->P.nz / f};
    const long long nc = (long long)grid_c[0] * grid_c[1] * grid_c[2];
    void* backup;
    float* fields[4];
    double* measures;
    void* proj;
    if ((rc = jump_workspace(c, f, &backup, fields, &measures, &proj))) return rc;
    float *in = fields[0], *xin = fields[1], *yout = fields[2], *pred = fields[3];
    auto cu = [&](cudaError_t e) { return e == cudaSuccess ? LBM_OK : lbm::ctx_error(c, LBM_ECUDA, cudaGetErrorString(e)); };
    const int saved_cur = c->cur;
    const lbm::Params saved_P = c->P;
    if ((rc = cu(cudaMemcpyAsync(backup, c->fg[c->cur], c->fg_bytes, cudaMemcpyDeviceToDevice, c->stream)))) return rc;
    long long m_before = 0;
    if ((rc = lbm::ctx_mass_fixed(c, &m_before))) return rc;
    // 1. predict
    if ((rc = lbm_coarse_fields(c, f, in))) return rc;
    if ((rc = cu(cudaStreamSynchronize(c->stream)))) return rc;
    if ((rc = cu(lbm::launch_normalize(in, xin, nc, mean_std, +1, n->stream)))) return rc;
    if ((rc = lbm_net_forward(n, xin, yout, 1, grid_c))) return lbm::ctx_error(c, rc, lbm_net_last_error(n));
    if ((rc = cu(lbm::launch_normalize(yout, pred, nc, mean_std, -1, n->stream)))) return rc;
    if ((rc = cu(cudaStreamSynchronize(n->stream)))) return rc;
    if ((rc = check_tc(n))) return lbm::ctx_error(c, rc, lbm_net_last_error(n));
    // the predicted velocity (channels 1-3) replaced by its divergence-free part
    if (proj) {
        if ((rc = cu(lbm::launch_project_solenoidal(pred + nc, grid_c[0], grid_c[1], grid_c[2], proj, c->stream))))
            return rc;
        c->launches += 9;
        rep->projected = 1;
    }
    // 2. mass and interface position of the prediction, measured on the coarse grid
    if ((rc = cu(cudaMemsetAsync(measures, 0, 4 * sizeof(double), c->stream)))) return rc;
    if ((rc = cu(lbm::launch_jump_measures(in, pred, grid_c[0], grid_c[1], grid_c[2], c->P.walls, measures, c->stream))))
        return rc;
    double m[4];
    if ((rc = cu(cudaMemcpyAsync(m, measures, sizeof m, cudaMemcpyDeviceToHost, c->stream)))) return rc;
    if ((rc = cu(cudaStreamSynchronize(c->stream)))) return rc;
    c->launches += 1;
    const double mass_before = (double)m_before / 1073741824.0;
    const double mass_pred = m[0] * f * f * f, jump = m[1];
    rep->mass_error = std::fabs(mass_pred - mass_before) / std::fabs(mass_before);
    // Mean displacement of the interface, in fine cells: a profile moved by d along its normal
    // changes phi by |grad phi| d, so int |phi_pred - phi_start| dV = d int |grad phi| dV. On the
    // coarse grid both integrals are sums over coarse cells (f^3 fine cells each; the coarse
    // gradient is f times the fine one), so d = f sum |dphi| / sum |grad_c phi|.
    rep->interface_shift = m[2] > 0 ? f * jump / m[2] : (jump > 0 ? INFINITY : 0.0);
    // Kinematic bound: the phi = 1/2 surface is carried by the flow (the sharpening flux of the
    // conservative phase-field equation vanishes on the equilibrium profile), so in k steps no
    // part of it moves farther than the largest speed times k.
    rep->interface_limit = interface_tol * std::sqrt(m[3]) * k;
    bool accept = rep->mass_error <= mass_tol && rep->interface_shift <= rep->interface_limit;
    // 3-4. restart and judge. How fast phi moves in the LBM's first judge_steps steps after a
    // restart, as the L1 rate of its coarse block means: after the restart from the prediction,
    // against the same after the restart from the starting state's own coarse fields. Both carry
    // the relaxation a restart causes (upsampled fields are smoother than the lattice's); a
    // prediction whose phi, u and p do not fit together relaxes faster than that.
    if (accept) {
        auto coarse_phi_into = [&](float* dst) -> int {
            if (f <= 32 && 32 % f == 0) return cu(lbm::launch_coarse_phi(c->P, c->fg[c->cur], f, dst, c->stream));
            return lbm_coarse_fields(c, f, dst);  // phi is channel 0 of the five it writes
        };
        std::vector<float> h_r((size_t)nc), h_after((size_t)nc);
        auto restart_and_relax = [&](const float* src, double* rate) -> int {
            int r = lbm_restart_from_coarse(c, f, src, saved_P.w0d / 3.0);
            if (r) return r;
            if ((r = coarse_phi_into(xin))) return r;
            if ((r = lbm_step(c, judge_steps))) return r;
            if ((r = coarse_phi_into(yout))) return r;
            if ((r = cu(cudaStreamSynchronize(c->stream)))) return r;
            if ((r = cu(cudaMemcpy(h_r.data(), xin, (size_t)nc * sizeof(float), cudaMemcpyDeviceToHost)))) return r;
            if ((r = cu(cudaMemcpy(h_after.data(), yout, (size_t)nc * sizeof(float), cudaMemcpyDeviceToHost)))) return r;
            double sum = 0.0;
            for (long long i = 0; i < nc; ++i) sum += std::fabs((double)h_after[i] - (double)h_r[i]);
            *rate = sum / judge_steps;
            return LBM_OK;
        };
        double rate_ref = 0.0, rate_pred = 0.0;
        if ((rc = restart_and_relax(in, &rate_ref))) return rc;
        if ((rc = restart_and_relax(pred, &rate_pred))) return rc;
        rep->relax_ratio = rate_ref > 0 ? rate_pred / rate_ref : (rate_pred > 0 ? INFINITY : 0.0);
        accept = rep->relax_ratio <= relax_tol;
    }
    // 5. fallback
    if (!accept) {
        c->P = saved_P;
        c->cur = saved_cur;
        if ((rc = cu(cudaMemcpyAsync(c->fg[c->cur], backup, c->fg_bytes, cudaMemcpyDeviceToDevice, c->stream)))) return rc;
        c->initialised = true;
        c->version += 1;
        if ((rc = lbm_step(c, k))) return rc;
        if ((rc = cu(cudaStreamSynchronize(c->stream)))) return rc;
    }
    rep->accepted = accept ? 1 : 0;
    rep->seconds_surrogate = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return LBM_OK;
}

}  // extern "C"
