// surrogate_kernels.cu -- the kernels of the 3D convolutional surrogate (lbm_net_*): periodic
// 3x3x3 convolutions (FP32 accumulation over FP16 or FP32 activations), their weight
// gradients, the loss of the residual prediction, ReLU masks and the Adam update. The network
// and the use the solver makes of it have no counterpart in the paper.
//
// Layout: a batch of fields is [B][C][D][H][W], W fastest. Weights of a layer are [Cout][Cin][27]
// (tap = 9 dz + 3 dy + dx, the input offset of a tap is (dz-1, dy-1, dx-1)), then bias [Cout].
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "surrogate.h"

namespace lbm {
namespace net {

constexpr int TX = 8, TY = 8, TZ = 4;             // output tile per block: 256 voxels
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;  // the tile with its halo
constexpr int HALO = HX * HY * HZ;                  // 600
constexpr int CCH = 8;                             // input channels staged at a time
constexpr int kThreads = TX * TY * TZ;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// periodic index for any i (tiles may reach more than one period past a grid smaller than them)
__device__ __forceinline__ int wrap(int i, int n) { return ((i % n) + n) % n; }

struct Tiles {
    int tx, ty, tz;  // tiles per axis
};

__device__ __forceinline__ void tile_origin(const Tiles& T, int t, int& x0, int& y0, int& z0) {
    const int ix = t % T.tx, iy = (t / T.tx) % T.ty, iz = t / (T.tx * T.ty);
    x0 = ix * TX;
    y0 = iy * TY;
    z0 = iz * TZ;
}

// out[b][o][v] = bias[o] + sum_{c, tap} W[o][c][tap] in[b][c][v + off(tap)] (periodic), then
// MODE 0: stored as FP32; MODE 1: relu, stored in TOUT.
template <typename TIN, int COUT, int MODE, typename TOUT>
__global__ void __launch_bounds__(kThreads)
conv3_kernel(const TIN* __restrict__ in, int cin, const float* __restrict__ W, const float* __restrict__ bias,
             TOUT* __restrict__ out, int D, int H, int Wd, Tiles T) {
    __shared__ float s_in[CCH][HZ][HY][HX];
    __shared__ float s_w[CCH][27][COUT];
    const int b = blockIdx.y;
    int x0, y0, z0;
    tile_origin(T, blockIdx.x, x0, y0, z0);
    const int t = threadIdx.x;
    const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
    const long long vox = (long long)D * H * Wd;
    const TIN* inb = in + (long long)b * cin * vox;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias ? bias[o] : 0.f;
    for (int c0 = 0; c0 < cin; c0 += CCH) {
        const int nc = min(CCH, cin - c0);
        __syncthreads();
        for (int i = t; i < nc * HALO; i += kThreads) {
            const int c = i / HALO, r = i - c * HALO;
            const int hx = r % HX, hy = (r / HX) % HY, hz = r / (HX * HY);
            const int gx = wrap(x0 + hx - 1, Wd), gy = wrap(y0 + hy - 1, H), gz = wrap(z0 + hz - 1, D);
            s_in[c][hz][hy][hx] = to_f(inb[(long long)(c0 + c) * vox + ((long long)gz * H + gy) * Wd + gx]);
        }
        for (int i = t; i < nc * 27 * COUT; i += kThreads) {
            const int c = i / (27 * COUT), r = i - c * 27 * COUT;
            const int tap = r / COUT, o = r - tap * COUT;
            s_w[c][tap][o] = W[((long long)o * cin + c0 + c) * 27 + tap];
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                const float v = s_in[c][lz + dz][ly + dy][lx + dx];
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[o] = fmaf(s_w[c][tap][o], v, acc[o]);
            }
        }
    }
    const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
    if (x >= Wd || y >= H || z >= D) return;
    const long long v = ((long long)z * H + y) * Wd + x;
    TOUT* outb = out + (long long)b * COUT * vox;
#pragma unroll
    for (int o = 0; o < COUT; ++o) outb[(long long)o * vox + v] = from_f<TOUT>(MODE == 1 ? fmaxf(acc[o], 0.f) : acc[o]);
}

// gW[o][c][tap] += sum_{b, v} g[b][o][v] h[b][c][v + off(tap)] and gb[o] += sum g[b][o][v]. Block
// (k, o) strides over the tiles of all samples; thread t < CCH * 27 owns the pair
// (c = c0 + t / 27, tap = t % 27) of every chunk c0 of input channels, thread CCH * 27 the bias.
template <typename TH>
__global__ void __launch_bounds__(kThreads)
conv3_wgrad_kernel(const float* __restrict__ g, int cout, const TH* __restrict__ h, int cin, float* __restrict__ gW,
                   float* __restrict__ gb, int D, int H, int Wd, Tiles T, int batch) {
    constexpr int kMaxChunks = 4;  // cin <= 32
    __shared__ float s_h[CCH][HZ][HY][HX];
    __shared__ float s_g[kThreads];
    const int o = blockIdx.y;
    const int t = threadIdx.x;
    const long long vox = (long long)D * H * Wd;
    const int tiles = T.tx * T.ty * T.tz;
    const int nchunks = (cin + CCH - 1) / CCH;
    float acc[kMaxChunks] = {0.f, 0.f, 0.f, 0.f};
    float accb = 0.f;
    const int pc = t / 27, ptap = t - (t / 27) * 27;
    const int dz = ptap / 9, dy = (ptap / 3) % 3, dx = ptap % 3;
    for (int w = blockIdx.x; w < tiles * batch; w += gridDim.x) {
        const int b = w / tiles;
        int x0, y0, z0;
        tile_origin(T, w - b * tiles, x0, y0, z0);
        __syncthreads();
        {
            const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
            const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
            s_g[t] = (x < Wd && y < H && z < D) ? g[((long long)b * cout + o) * vox + ((long long)z * H + y) * Wd + x] : 0.f;
        }
        __syncthreads();
        if (t == CCH * 27)
            for (int v = 0; v < kThreads; ++v) accb += s_g[v];
#pragma unroll
        for (int k = 0; k < kMaxChunks; ++k) {
            if (k >= nchunks) break;
            const int c0 = k * CCH, nc = min(CCH, cin - c0);
            __syncthreads();
            for (int i = t; i < nc * HALO; i += kThreads) {
                const int c = i / HALO, r = i - c * HALO;
                const int hx = r % HX, hy = (r / HX) % HY, hz = r / (HX * HY);
                const int gx = wrap(x0 + hx - 1, Wd), gy = wrap(y0 + hy - 1, H), gz = wrap(z0 + hz - 1, D);
                s_h[c][hz][hy][hx] = to_f(h[((long long)b * cin + c0 + c) * vox + ((long long)gz * H + gy) * Wd + gx]);
            }
            __syncthreads();
            if (pc < nc) {
                float a = 0.f;
                for (int v = 0; v < kThreads; ++v) {
                    const int lx = v % TX, ly = (v / TX) % TY, lz = v / (TX * TY);
                    a = fmaf(s_g[v], s_h[pc][lz + dz][ly + dy][lx + dx], a);
                }
                acc[k] += a;
            }
        }
    }
    for (int k = 0; k < nchunks && k < kMaxChunks; ++k) {
        const int c = k * CCH + pc;
        if (pc < CCH && c < cin && t < CCH * 27) atomicAdd(&gW[((long long)o * cin + c) * 27 + ptap], acc[k]);
    }
    if (t == CCH * 27) atomicAdd(&gb[o], accb);
}

// Wt[c][o][tap] = W[o][c][26 - tap]: the weights of the adjoint convolution.
__global__ void flip_transpose_kernel(const float* __restrict__ W, int cout, int cin, float* __restrict__ Wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cout * cin * 27) return;
    const int tap = i % 27, c = (i / 27) % cin, o = i / (27 * cin);
    Wt[((long long)c * cout + o) * 27 + (26 - tap)] = W[i];
}

template <typename T>
__global__ void relu_mask_kernel(float* __restrict__ g, const T* __restrict__ h, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(to_f(h[i]) > 0.f)) g[i] = 0.f;
}

template <typename T>
__global__ void cast_kernel(const float* __restrict__ x, T* __restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = from_f<T>(x[i]);
}

// y = x + d (the residual prediction)
__global__ void residual_kernel(const float* __restrict__ x, const float* __restrict__ d, float* __restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] + d[i];
}

// diff = x + d - target; loss term w_c diff^2 and its gradient g = 2 w_c diff / n, with w_c the
// weight of the element's channel (elements [B][5][vox]); per-block partial sums (FP64).
__global__ void loss_kernel(const float* __restrict__ x, const float* __restrict__ d, const float* __restrict__ target,
                            float* __restrict__ g, long long n, long long vox, float w0, float w1, float w2, float w3,
                            float w4, double* __restrict__ partials) {
    __shared__ double red[256 / 32];
    const float w[kFieldChannels] = {w0, w1, w2, w3, w4};
    double acc = 0.0;
    const float scale = (float)(2.0 / (double)n);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float wc = w[(i / vox) % kFieldChannels];
        const float diff = x[i] + d[i] - target[i];
        g[i] = scale * wc * diff;
        acc += (double)wc * (double)diff * (double)diff;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

static Tiles tiles_of(int D, int H, int Wd) { return Tiles{(Wd + TX - 1) / TX, (H + TY - 1) / TY, (D + TZ - 1) / TZ}; }

static unsigned ew_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? b : 4096);
}

template <typename TIN, typename TOUT>
static cudaError_t conv_dispatch(const TIN* in, int cin, const float* W, const float* bias, TOUT* out, int cout, int relu,
                                 int batch, int D, int H, int Wd, cudaStream_t s) {
    const Tiles T = tiles_of(D, H, Wd);
    const dim3 grid((unsigned)(T.tx * T.ty * T.tz), (unsigned)batch);
    if (cout == 32) {
        if (relu) conv3_kernel<TIN, 32, 1, TOUT><<<grid, kThreads, 0, s>>>(in, cin, W, bias, out, D, H, Wd, T);
        else conv3_kernel<TIN, 32, 0, TOUT><<<grid, kThreads, 0, s>>>(in, cin, W, bias, out, D, H, Wd, T);
    } else if (cout == kFieldChannels) {
        if (relu) conv3_kernel<TIN, kFieldChannels, 1, TOUT><<<grid, kThreads, 0, s>>>(in, cin, W, bias, out, D, H, Wd, T);
        else conv3_kernel<TIN, kFieldChannels, 0, TOUT><<<grid, kThreads, 0, s>>>(in, cin, W, bias, out, D, H, Wd, T);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t conv_forward(const void* in, int in_fp16, int cin, const float* W, const float* bias, void* out, int out_fp16,
                         int cout, int relu, int batch, int D, int H, int Wd, cudaStream_t s) {
    if (in_fp16 && out_fp16)
        return conv_dispatch((const __half*)in, cin, W, bias, (__half*)out, cout, relu, batch, D, H, Wd, s);
    if (in_fp16)
        return conv_dispatch((const __half*)in, cin, W, bias, (float*)out, cout, relu, batch, D, H, Wd, s);
    if (out_fp16)
        return conv_dispatch((const float*)in, cin, W, bias, (__half*)out, cout, relu, batch, D, H, Wd, s);
    return conv_dispatch((const float*)in, cin, W, bias, (float*)out, cout, relu, batch, D, H, Wd, s);
}

cudaError_t conv_wgrad(const float* g, int cout, const void* h, int h_fp16, int cin, float* gW, float* gb, int batch,
                       int D, int H, int Wd, cudaStream_t s) {
    if (cin > 32) return cudaErrorInvalidValue;
    const Tiles T = tiles_of(D, H, Wd);
    const int tiles = T.tx * T.ty * T.tz * batch;
    const dim3 grid((unsigned)(tiles < 64 ? tiles : 64), (unsigned)cout);
    if (h_fp16) conv3_wgrad_kernel<__half><<<grid, kThreads, 0, s>>>(g, cout, (const __half*)h, cin, gW, gb, D, H, Wd, T, batch);
    else conv3_wgrad_kernel<float><<<grid, kThreads, 0, s>>>(g, cout, (const float*)h, cin, gW, gb, D, H, Wd, T, batch);
    return cudaGetLastError();
}

cudaError_t flip_transpose(const float* W, int cout, int cin, float* Wt, cudaStream_t s) {
    const int n = cout * cin * 27;
    flip_transpose_kernel<<<(n + 255) / 256, 256, 0, s>>>(W, cout, cin, Wt);
    return cudaGetLastError();
}

cudaError_t relu_mask(float* g, const void* h, int h_fp16, long long n, cudaStream_t s) {
    if (h_fp16) relu_mask_kernel<__half><<<ew_blocks(n), 256, 0, s>>>(g, (const __half*)h, n);
    else relu_mask_kernel<float><<<ew_blocks(n), 256, 0, s>>>(g, (const float*)h, n);
    return cudaGetLastError();
}

cudaError_t cast_to(const float* x, void* y, int fp16, long long n, cudaStream_t s) {
    if (fp16) cast_kernel<__half><<<ew_blocks(n), 256, 0, s>>>(x, (__half*)y, n);
    else cast_kernel<float><<<ew_blocks(n), 256, 0, s>>>(x, (float*)y, n);
    return cudaGetLastError();
}

cudaError_t residual(const float* x, const float* d, float* y, long long n, cudaStream_t s) {
    residual_kernel<<<ew_blocks(n), 256, 0, s>>>(x, d, y, n);
    return cudaGetLastError();
}

int loss_blocks(long long n) { return (int)ew_blocks(n); }

cudaError_t loss_and_grad(const float* x, const float* d, const float* target, float* g, long long n, long long vox,
                          const float* w, double* partials, cudaStream_t s) {
    loss_kernel<<<ew_blocks(n), 256, 0, s>>>(x, d, target, g, n, vox, w[0], w[1], w[2], w[3], w[4], partials);
    return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 / (1.0 - pow((double)b1, step))), c2 = (float)(1.0 / (1.0 - pow((double)b2, step)));
    adam_kernel<<<ew_blocks(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace net
}  // namespace lbm
