// surrogate_kernels.cu -- the kernels of the 3D convolutional surrogate (lbm_net_*): periodic
// 3x3x3 convolutions (FP32 accumulation over FP16 or FP32 activations), their weight
// gradients, the loss of the residual prediction, ReLU masks and the Adam update. The network
// and the use the solver makes of it have no counterpart in the paper.
//
// Layout: a batch of fields is [B][C][D][H][W], W fastest. Weights of a layer are [Cout][Cin][27]
// (tap = 9 dz + 3 dy + dx, the input offset of a tap is (dz-1, dy-1, dx-1)), then bias [Cout].
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

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

// periodic index for any i: in range, one period off, or (a grid smaller than a tile) further
__device__ __forceinline__ int wrap(int i, int n) {
    if (i >= 0 && i < n) return i;
    if (i < 0 && i + n >= 0) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    return ((i % n) + n) % n;
}

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

// ---------------------------------------------------------------------------------------
// The 32 -> 32 channel convolution on the fifth-generation tensor cores (tcgen05), FP16
// operands, FP32 accumulation in tensor memory.
//
// Implicit GEMM: a step of 128 output voxels (8 in x, 16 in y, one z plane) is the M = 128 side,
// the 32 output channels the N = 32 side, and the reduction runs over 27 taps x 32 input
// channels. A haloed input plane (10 x 18 voxels, 32 channels) sits in shared memory in "chunk
// planes": element (haloed voxel v, channel k) at (k / 8) * PLP + 16 v + 2 (k % 8). In the
// canonical no-swizzle K-major operand layout (core matrices of 8 rows x 16 bytes), the rows of
// an 8-voxel x-run are then 16 bytes apart and successive y-runs one haloed row (160 bytes)
// apart, so the A operand of every tap is the same descriptor at a different start address.
// The weights of all taps are a preformatted FP16 image (2 KB per tap) loaded once per CTA.
//
// A CTA walks a column of steps along z (a chunk of z planes of one (x, y) tile) with the
// haloed planes in a ring of four and two accumulators in tensor memory: one thread issues the
// 54 MMAs of step z (27 taps x 2 of K = 16) and commits them to an mbarrier; meanwhile four
// warps read the accumulator of step z - 1 (tcgen05.ld) and write its output, and seven warps
// write plane z + 2 (loaded during step z - 1) into the slot step z - 1 read and issue the
// loads of plane z + 3. Waits are bounded: on a timeout the kernel raises *err, waits once more
// for its MMAs, frees its tensor memory and returns.
// ---------------------------------------------------------------------------------------
namespace tc {

constexpr int TX = 8, TY = 16, HX = TX + 2, HY = TY + 2;
constexpr int HPLANE = HX * HY;               // 180 haloed voxels per z plane
constexpr uint32_t PLP = HPLANE * 16;         // bytes of one chunk plane (8 channels) of a z plane
constexpr uint32_t SLOT_BYTES = 4 * PLP;      // 32 channels: 11,520
constexpr int CONV_THREADS = 256;
constexpr int CONV_STAGERS = CONV_THREADS - 32;  // warps 0..6 stage; warp 7 issues the MMAs
constexpr int kIssuer = CONV_THREADS - 32;
constexpr uint32_t W_TAP = 2048;             // bytes of one tap's 32 x 32 FP16 weights
constexpr uint32_t W_BYTES = 27 * W_TAP;
constexpr uint32_t SMEM = 4 * SLOT_BYTES + W_BYTES;  // 101,376: two CTAs per SM
constexpr long long kSpin = kTcWaitPolls;     // polls of an mbarrier before giving up, at most

// offset of weight (out n, in k) of a tap inside its 2 KB block: core matrix (k/8, n/8)
__host__ __device__ inline uint32_t w_off(int n, int k) { return (k / 8) * 512 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2; }

__device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);  // no swizzle, version 1
}

// kind::f16 instruction descriptor: FP32 D, FP16 A and B, both K-major, M = 128, N = 32
constexpr uint32_t kIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// One MMA from descriptors given as 32-bit halves. A descriptor's start address sits in the
// low 14 bits as address / 16 and every shared-memory address stays below 2^18 bytes, so an
// operand at byte offset d from a described base is the same descriptor with d / 16 added to
// its low half.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 ad, bd;\n\t"
        "mov.b64 ad, {%1, %2};\n\tmov.b64 bd, {%3, %4};\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(kIdesc), "r"(accumulate));
}

// The FP16 weight image of a layer with cout, cin <= 32: zero where n >= cout or k >= cin.
__global__ void weight_image_kernel(const float* __restrict__ W, int cout, int cin, __half* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over [32 out][32 in][27]
    if (i >= 32 * 32 * 27) return;
    const int tap = i % 27, k = (i / 27) % 32, n = i / (27 * 32);
    const float w = (n < cout && k < cin) ? W[((long long)n * cin + k) * 27 + tap] : 0.f;
    *reinterpret_cast<__half*>(reinterpret_cast<unsigned char*>(img) + tap * W_TAP + w_off(n, k)) = __float2half_rn(w);
}

// Polls mbarrier `mbar` until phase `parity` completes, at most `limit` times (limit 0 gives up
// at once without polling).
__device__ inline bool wait_parity(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\tselp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity));
        if (ok) return true;
    }
    return false;
}

// A haloed row of one channel as loaded: the 8 values x0 .. x0 + 7 and the halo values x0 - 1
// and x0 + 8 (periodic), kept in the storage type until they are written to shared memory.
// vec: the row start is 16-byte aligned and x0 .. x0 + 7 lie inside the row.
constexpr int kRunX = 8;
template <typename TH>
struct HRow;
template <>
struct HRow<__half> {
    uint4 m;
    __half l, r;
    __device__ __forceinline__ void load(const __half* __restrict__ row, bool vec, int x0, int Wd) {
        if (vec) {
            m = __ldg(reinterpret_cast<const uint4*>(row + x0));
        } else {
            __half2 q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = __halves2half2(row[wrap(x0 + 2 * j, Wd)], row[wrap(x0 + 2 * j + 1, Wd)]);
            m = *reinterpret_cast<const uint4*>(q);
        }
        l = row[wrap(x0 - 1, Wd)];
        r = row[wrap(x0 + kRunX, Wd)];
    }
    __device__ __forceinline__ void zero() {
        m = make_uint4(0, 0, 0, 0);
        l = r = __float2half_rn(0.f);
    }
    __device__ __forceinline__ void get(float (&v)[kRunX + 2]) const {
        const __half2* h2 = reinterpret_cast<const __half2*>(&m);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 f = __half22float2(h2[j]);
            v[1 + 2 * j] = f.x;
            v[2 + 2 * j] = f.y;
        }
        v[0] = __half2float(l);
        v[kRunX + 1] = __half2float(r);
    }
};
template <>
struct HRow<float> {
    float4 a, b;
    float l, r;
    __device__ __forceinline__ void load(const float* __restrict__ row, bool vec, int x0, int Wd) {
        if (vec) {
            a = __ldg(reinterpret_cast<const float4*>(row + x0));
            b = __ldg(reinterpret_cast<const float4*>(row + x0 + 4));
        } else {
            a = make_float4(row[wrap(x0, Wd)], row[wrap(x0 + 1, Wd)], row[wrap(x0 + 2, Wd)], row[wrap(x0 + 3, Wd)]);
            b = make_float4(row[wrap(x0 + 4, Wd)], row[wrap(x0 + 5, Wd)], row[wrap(x0 + 6, Wd)], row[wrap(x0 + 7, Wd)]);
        }
        l = row[wrap(x0 - 1, Wd)];
        r = row[wrap(x0 + kRunX, Wd)];
    }
    __device__ __forceinline__ void zero() {
        a = b = make_float4(0.f, 0.f, 0.f, 0.f);
        l = r = 0.f;
    }
    __device__ __forceinline__ void get(float (&v)[kRunX + 2]) const {
        v[0] = l;
        v[1] = a.x; v[2] = a.y; v[3] = a.z; v[4] = a.w;
        v[5] = b.x; v[6] = b.y; v[7] = b.z; v[8] = b.w;
        v[kRunX + 1] = r;
    }
};

// One haloed z plane of the input, a thread's share as loaded: tasks are (row, channel), ten
// x-values each. Warps 0..6 stage; the MMA warp takes no tasks.
constexpr int CV_TASKS = HY * 32, CV_PER = (CV_TASKS + CONV_STAGERS - 1) / CONV_STAGERS;

template <typename TIN>
struct ConvStage {
    HRow<TIN> h[CV_PER];
};

template <typename TIN>
__device__ __forceinline__ void conv_load_plane(ConvStage<TIN>& st, const TIN* __restrict__ inb, int cin, long long vox,
                                                int zz, int y0, int x0, int H, int Wd, bool vec) {
    if (threadIdx.x >= CONV_STAGERS) return;
#pragma unroll
    for (int i = 0; i < CV_PER; ++i) {
        const int task = threadIdx.x + i * CONV_STAGERS;
        const int r = task / 32, c = task % 32;
        if (task < CV_TASKS && c < cin)
            st.h[i].load(inb + (long long)c * vox + ((long long)zz * H + wrap(y0 + r - 1, H)) * Wd, vec, x0, Wd);
        else
            st.h[i].zero();
    }
}

// The loaded rows into a ring slot in chunk planes, converted to FP16 and scaled: element
// (haloed voxel v = HX r + hx, channel c) at (c / 8) PLP + 16 v + 2 (c % 8). Channels >= cin
// are zero.
template <typename TIN>
__device__ __forceinline__ void conv_store_plane(unsigned char* __restrict__ slot, const ConvStage<TIN>& st, float in_scale) {
    if (threadIdx.x >= CONV_STAGERS) return;
#pragma unroll
    for (int i = 0; i < CV_PER; ++i) {
        const int task = threadIdx.x + i * CONV_STAGERS;
        if (task >= CV_TASKS) break;
        const int r = task / 32, c = task % 32;
        float v[kRunX + 2];
        st.h[i].get(v);
        unsigned char* base = slot + (c >> 3) * PLP + (c & 7) * 2 + r * HX * 16;
#pragma unroll
        for (int hx = 0; hx < HX; ++hx) *reinterpret_cast<__half*>(base + hx * 16) = __float2half_rn(v[hx] * in_scale);
    }
}

template <typename TIN, int MODE, typename TOUT>
__global__ void __launch_bounds__(CONV_THREADS, 2)
conv32_tc_kernel(const TIN* __restrict__ in, int cin, float in_scale, const __half* __restrict__ wimg,
                 const float* __restrict__ bias, TOUT* __restrict__ out, int cout, int D, int H, int Wd, int tiles_x,
                 int tiles_y, int zchunk, int n_chunks, int n_columns, int vec_in, long long spin, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                   // ring of four haloed planes
    unsigned char* sW = smem + 4 * SLOT_BYTES;  // weights of the 27 taps
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    __shared__ __align__(16) float s_bias[32];
    const int t = threadIdx.x;
    const uint32_t mbar0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);  // barrier k at mbar0 + 8 k
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8));
        s_fail = 0;
    }
    if (t < 32) s_bias[t] = (bias && t < cout) ? bias[t] : 0.f;
    if (t < 32) {  // two 32-column accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
            (uint32_t)__cvta_generic_to_shared(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // weights: the preformatted image, 16 bytes at a time
    for (int i = t; i < (int)(W_BYTES / 16); i += CONV_THREADS)
        reinterpret_cast<uint4*>(sW)[i] = __ldg(reinterpret_cast<const uint4*>(wimg) + i);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t a_addr = (uint32_t)__cvta_generic_to_shared(sA), w_addr = (uint32_t)__cvta_generic_to_shared(sW);
    const uint64_t a_desc = smem_desc(a_addr, PLP, HX * 16), b_desc = smem_desc(w_addr, 512, 128);
    const uint32_t a_lo0 = (uint32_t)a_desc, a_hi = (uint32_t)(a_desc >> 32);
    const uint32_t b_lo0 = (uint32_t)b_desc, b_hi = (uint32_t)(b_desc >> 32);
    const long long vox = (long long)D * H * Wd;
    const float out_scale = 1.0f / in_scale;  // in_scale is a power of two: exact
    const bool vin = vec_in != 0;
    uint32_t phase = 0u, pending = 0u;        // per barrier k (bit k): the parity it waits for; a commit not waited for
    // waits for the MMAs committed on barrier k, if any, polling at most `limit` times; false on a
    // timeout (they stay pending)
    auto drain = [&](int k, long long limit) {
        if (!((pending >> k) & 1u)) return true;
        if (!wait_parity(mbar0 + 8u * (uint32_t)k, (phase >> k) & 1u, limit)) return false;
        phase ^= 1u << k;
        pending &= ~(1u << k);
        return true;
    };
    // the output of a finished step from accumulator k: warp w < 4 holds rows 32 w .. 32 w + 31
    // (row m = 8 ly + lx)
    auto epilogue = [&](int k, int b, int z, int x0, int y0) {
        if (t >= 128) return;
        const int warp = t / 32;
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
              "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
              "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(k * 32)));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int lx = t % TX, ly = t / TX;
        const int x = x0 + lx, y = y0 + ly;
        if (x < Wd && y < H) {
            // channel o of this voxel at p + o vox; the biases come four at a time
            TOUT* p = out + (long long)b * cout * vox + ((long long)z * H + y) * Wd + x;
            const float4* b4 = reinterpret_cast<const float4*>(s_bias);
#pragma unroll
            for (int o4 = 0; o4 < 8; ++o4) {
                const float4 bq = b4[o4];
                const float bias4[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int o = 4 * o4 + q;
                    if (o < cout) {
                        float a = fmaf(__uint_as_float(v[o]), out_scale, bias4[q]);
                        if (MODE == 1) a = fmaxf(a, 0.f);
                        *p = from_f<TOUT>(a);
                        p += vox;
                    }
                }
            }
        }
    };
    for (int col = blockIdx.x; col < n_columns && !s_fail; col += gridDim.x) {
        int r = col;
        const int zc = r % n_chunks;
        r /= n_chunks;
        const int tx = r % tiles_x;
        r /= tiles_x;
        const int ty = r % tiles_y;
        const int b = r / tiles_y;
        const int x0 = tx * TX, y0 = ty * TY;
        const int z_begin = zc * zchunk, z_end = min(z_begin + zchunk, D);
        const TIN* inb = in + (long long)b * cin * vox;
        // prologue: planes z_begin - 1 .. z_begin + 1 in ring slots 0..2, and the loads of the
        // plane the first step stages in flight
        ConvStage<TIN> st;
        for (int j = 0; j < 3; ++j) {
            conv_load_plane(st, inb, cin, vox, wrap(z_begin - 1 + j, D), y0, x0, H, Wd, vin);
            conv_store_plane(sA + j * SLOT_BYTES, st, in_scale);
        }
        if (z_begin + 1 < z_end) conv_load_plane(st, inb, cin, vox, wrap(z_begin + 2, D), y0, x0, H, Wd, vin);
        for (int z = z_begin; z < z_end; ++z) {
            const int zi = z - z_begin, k = zi & 1;  // accumulator and barrier of this step
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (s_fail) break;
            if (t == kIssuer) {
                uint32_t alo[3];  // plane z + dz - 1 in its ring slot
#pragma unroll
                for (int dz = 0; dz < 3; ++dz) alo[dz] = a_lo0 + ((uint32_t)((zi + dz) & 3) * SLOT_BYTES >> 4);
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)  // haloed voxel of output (0, 0) shifted by (dx - 1, dy - 1)
                        mma_f16(tmem + (uint32_t)(k * 32), alo[dz] + (((uint32_t)(dy * HX + dx) * 16 + (uint32_t)(2 * kk) * PLP) >> 4),
                                a_hi, b_lo0 + (((uint32_t)tap * W_TAP + (uint32_t)(2 * kk) * 512) >> 4), b_hi, (tap | kk) ? 1u : 0u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar0 + 8u * (uint32_t)k));
            }
            pending |= 1u << k;
            if (zi > 0) {
                // step z - 1 is done: its output, then its ring slot takes plane z + 2
                if (!drain(k ^ 1, spin)) {
                    s_fail = 1;
                    atomicExch(err, 1);
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    epilogue(k ^ 1, b, z - 1, x0, y0);
                }
            }
            if (z + 1 < z_end) {  // plane z + 2, loaded during the previous step, and the next loads
                conv_store_plane(sA + (uint32_t)((zi + 3) & 3) * SLOT_BYTES, st, in_scale);
                if (z + 2 < z_end) conv_load_plane(st, inb, cin, vox, wrap(z + 3, D), y0, x0, H, Wd, vin);
            }
            // the epilogue's reads of accumulator k ^ 1 come before the next step's MMAs into it
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
        // the column's last step
        const int kl = (z_end - 1 - z_begin) & 1;
        if (!s_fail) {
            if (!drain(kl, spin)) {
                s_fail = 1;
                atomicExch(err, 1);
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;");
                epilogue(kl, b, z_end - 1, x0, y0);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    // on a timeout, one more wait, bounded by the full limit whatever `spin` was, for MMAs still
    // in flight before the memory is freed
    for (int kb = 0; kb < 2; ++kb) drain(kb, kSpin);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------------------------------
// Weight gradients on the tensor cores:
//   gW[o][c][tap] = sum over voxels v of h[c][v + off(tap)] g[o][v],
// a GEMM over the voxels for each of the 9 (dz, dy) pairs: D_(dz,dy)[m][o] with the M = 128 rows
// m = 32 dx + c (dx = 0, 1, 2 and a fourth, zero, slot) and N = 32 columns o. A step is 8 voxels
// in x by 16 in y in one z plane (K = 128). A haloed row of h (18 y-rows per z plane) is staged
// as three x-shifted copies of its 8-voxel run side by side: element (row r, dx, c, lx) at
// 2048 r + 512 dx + 16 c + 2 lx holds h[c][z][y0 + r - 1][x0 + lx + dx - 1]. In the K-major
// no-swizzle layout that is an operand with 128 bytes between groups of 8 rows (SBO) and 2 KB
// between successive 8-voxel K chunks (LBO), the pair (dz, dy) selecting the plane and the start
// row. g is staged the same way as the N x K operand (16 o + 2 lx within a 512-byte row).
//
// A CTA walks a column of steps along z (a chunk of z planes of one (x, y) tile), keeping the
// haloed planes in a ring of four: step z reads planes z - 1, z, z + 1 while seven warps write
// plane z + 2 and g of step z + 1 into the plane and g buffers that step z - 1 read (waited for
// on its mbarrier), from registers loaded during step z - 1, and issue the loads for step z + 1. Nine 128 x 32 FP32 accumulators live in tensor memory (288 of 512
// columns; one CTA per SM) for all the columns a CTA takes, and are added to gW at the end.
// ---------------------------------------------------------------------------------------
constexpr int WG_TX = 8, WG_TY = 16, WG_HY = WG_TY + 2;        // 18 haloed rows per plane
constexpr int WG_THREADS = 256;
constexpr int WG_STAGERS = WG_THREADS - 32;  // warps 0..6 stage; warp 7 issues the MMAs
constexpr int WG_ZCHUNK = 16;                                   // z planes per column
constexpr uint32_t WG_ROW_BYTES = 4 * 512;                      // 4 dx slots x 32 channels x 8 voxels
constexpr uint32_t WG_PLANE_BYTES = WG_HY * WG_ROW_BYTES;        // 36,864
constexpr uint32_t WG_G_BYTES = WG_TY * 512;                     // 8,192
constexpr uint32_t WG_SMEM = 4 * WG_PLANE_BYTES + 2 * WG_G_BYTES; // 163,840

// A thread's share of one haloed plane of h (tasks are (row, channel)) and of one step of g
// (tasks are (row, output channel), 8 voxels each), as loaded. Loading and writing to shared
// memory are separate so that the loads of the plane a step will need can be issued a whole
// step ahead.
constexpr int WG_H_TASKS = WG_HY * 32, WG_H_PER = (WG_H_TASKS + WG_STAGERS - 1) / WG_STAGERS;
constexpr int WG_G_TASKS = WG_TY * 32, WG_G_PER = (WG_G_TASKS + WG_STAGERS - 1) / WG_STAGERS;

template <typename TH>
struct WgStage {
    HRow<TH> h[WG_H_PER];
    float4 ga[WG_G_PER], gb[WG_G_PER];
};

template <typename TH>
__device__ __forceinline__ void wg_load_plane(WgStage<TH>& st, const TH* __restrict__ hb, int cin, long long vox, int zz,
                                              int y0, int x0, int H, int Wd, bool vec) {
    if (threadIdx.x >= WG_STAGERS) return;  // the MMA warp takes no tasks
#pragma unroll
    for (int i = 0; i < WG_H_PER; ++i) {
        const int task = threadIdx.x + i * WG_STAGERS;
        const int r = task / 32, c = task % 32;
        if (task < WG_H_TASKS && c < cin)
            st.h[i].load(hb + (long long)c * vox + ((long long)zz * H + wrap(y0 + r - 1, H)) * Wd, vec, x0, Wd);
        else
            st.h[i].zero();
    }
}

// The three x-shifted 8-voxel windows of every loaded row, 16 bytes each.
template <typename TH>
__device__ __forceinline__ void wg_store_plane(unsigned char* __restrict__ slot, const WgStage<TH>& st) {
    if (threadIdx.x >= WG_STAGERS) return;
#pragma unroll
    for (int i = 0; i < WG_H_PER; ++i) {
        const int task = threadIdx.x + i * WG_STAGERS;
        if (task >= WG_H_TASKS) break;
        const int r = task / 32, c = task % 32;
        float v[WG_TX + 2];
        st.h[i].get(v);
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            __half2 w2[4];
#pragma unroll
            for (int j2 = 0; j2 < 4; ++j2) w2[j2] = __floats2half2_rn(v[dx + 2 * j2], v[dx + 2 * j2 + 1]);
            *reinterpret_cast<uint4*>(slot + r * WG_ROW_BYTES + dx * 512 + c * 16) = *reinterpret_cast<const uint4*>(w2);
        }
    }
}

// g of one step's own voxels: zero outside the grid and for o >= cout.
template <typename TH>
__device__ __forceinline__ void wg_load_g(WgStage<TH>& st, const float* __restrict__ gb, int cout, long long vox, int z,
                                          int y0, int x0, int H, int Wd, bool vec) {
    if (threadIdx.x >= WG_STAGERS) return;
#pragma unroll
    for (int i = 0; i < WG_G_PER; ++i) {
        const int task = threadIdx.x + i * WG_STAGERS;
        const int ly = task / 32, o = task % 32;
        const int y = y0 + ly;
        st.ga[i] = st.gb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (task < WG_G_TASKS && o < cout && y < H) {
            const float* row = gb + (long long)o * vox + ((long long)z * H + y) * Wd + x0;
            if (vec) {
                st.ga[i] = __ldg(reinterpret_cast<const float4*>(row));
                st.gb[i] = __ldg(reinterpret_cast<const float4*>(row + 4));
            } else {
                float v[8];
#pragma unroll
                for (int lx = 0; lx < WG_TX; ++lx) v[lx] = (x0 + lx < Wd) ? row[lx] : 0.f;
                st.ga[i] = make_float4(v[0], v[1], v[2], v[3]);
                st.gb[i] = make_float4(v[4], v[5], v[6], v[7]);
            }
        }
    }
}

// g scaled and rounded to FP16, one (row, output channel) per 16-byte store.
template <typename TH>
__device__ __forceinline__ void wg_store_g(unsigned char* __restrict__ buf, const WgStage<TH>& st, float g_scale) {
    if (threadIdx.x >= WG_STAGERS) return;
#pragma unroll
    for (int i = 0; i < WG_G_PER; ++i) {
        const int task = threadIdx.x + i * WG_STAGERS;
        if (task >= WG_G_TASKS) break;
        const int ly = task / 32, o = task % 32;
        const float4 a = st.ga[i], b = st.gb[i];
        const __half2 w2[4] = {__floats2half2_rn(a.x * g_scale, a.y * g_scale), __floats2half2_rn(a.z * g_scale, a.w * g_scale),
                               __floats2half2_rn(b.x * g_scale, b.y * g_scale), __floats2half2_rn(b.z * g_scale, b.w * g_scale)};
        *reinterpret_cast<uint4*>(buf + ly * 512 + o * 16) = *reinterpret_cast<const uint4*>(w2);
    }
}

template <typename TH>
__global__ void __launch_bounds__(WG_THREADS, 1)
wgrad32_tc_kernel(const float* __restrict__ g, int cout, float g_scale, const TH* __restrict__ h, int cin,
                  float* __restrict__ part, int D, int H, int Wd, int tiles_x, int tiles_y, int n_chunks, int n_columns,
                  int vec_h, int vec_g, long long spin, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sH = smem;                       // ring of four haloed planes
    unsigned char* sG = smem + 4 * WG_PLANE_BYTES;  // two g buffers
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int t = threadIdx.x;
    const uint32_t mbar0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);  // barrier k at mbar0 + 8 k
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8));
        s_fail = 0;
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            (uint32_t)__cvta_generic_to_shared(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the fourth dx slot of every row stays zero
    for (int i = t; i < (int)(4 * WG_PLANE_BYTES / 16); i += WG_THREADS) reinterpret_cast<uint4*>(sH)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t h_addr = (uint32_t)__cvta_generic_to_shared(sH), g_addr = (uint32_t)__cvta_generic_to_shared(sG);
    const uint64_t h_desc = smem_desc(h_addr, WG_ROW_BYTES, 128), g_desc = smem_desc(g_addr, 512, 128);
    const uint32_t h_lo0 = (uint32_t)h_desc, h_hi = (uint32_t)(h_desc >> 32);
    const uint32_t g_lo0 = (uint32_t)g_desc, g_hi = (uint32_t)(g_desc >> 32);
    const long long vox = (long long)D * H * Wd;
    uint32_t phase = 0u, pending = 0u;  // bit k: the parity barrier k waits for; a commit on it not yet waited for
    bool first = true;
    // waits for the MMAs committed on barrier k, if any, polling at most `limit` times; false on a
    // timeout (they stay pending)
    auto drain = [&](int k, long long limit) {
        if (!((pending >> k) & 1u)) return true;
        if (!wait_parity(mbar0 + 8u * (uint32_t)k, (phase >> k) & 1u, limit)) return false;
        phase ^= 1u << k;
        pending &= ~(1u << k);
        return true;
    };
    const bool vh = vec_h != 0, vg = vec_g != 0;
    for (int col = blockIdx.x; col < n_columns && !s_fail; col += gridDim.x) {
        int r = col;
        const int zc = r % n_chunks;
        r /= n_chunks;
        const int tx = r % tiles_x;
        r /= tiles_x;
        const int ty = r % tiles_y;
        const int b = r / tiles_y;
        const int x0 = tx * WG_TX, y0 = ty * WG_TY;
        const int z_begin = zc * WG_ZCHUNK, z_end = min(z_begin + WG_ZCHUNK, D);
        const TH* hb = h + (long long)b * cin * vox;
        const float* gbat = g + (long long)b * cout * vox;
        // prologue: planes z_begin - 1 .. z_begin + 1 (ring slots 0..2) and g of the first step
        // in shared memory, and the loads of what the first step stages already in flight
        WgStage<TH> st;
        for (int j = 0; j < 3; ++j) {
            wg_load_plane(st, hb, cin, vox, wrap(z_begin - 1 + j, D), y0, x0, H, Wd, vh);
            wg_store_plane(sH + j * WG_PLANE_BYTES, st);
        }
        wg_load_g(st, gbat, cout, vox, z_begin, y0, x0, H, Wd, vg);
        wg_store_g(sG, st, g_scale);
        if (z_begin + 1 < z_end) {
            wg_load_plane(st, hb, cin, vox, wrap(z_begin + 2, D), y0, x0, H, Wd, vh);
            wg_load_g(st, gbat, cout, vox, z_begin + 1, y0, x0, H, Wd, vg);
        }
        for (int z = z_begin; z < z_end; ++z) {
            const int zi = z - z_begin;
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (s_fail) break;
            const int k = zi & 1;  // barrier and g buffer of this step
            if (t == WG_STAGERS) {
                uint32_t alo[3];  // plane z + dz - 1 in its ring slot
#pragma unroll
                for (int dz = 0; dz < 3; ++dz) alo[dz] = h_lo0 + ((uint32_t)((zi + dz) & 3) * WG_PLANE_BYTES >> 4);
                const uint32_t glo = g_lo0 + ((uint32_t)k * WG_G_BYTES >> 4);
#pragma unroll
                for (int pr = 0; pr < 9; ++pr) {
                    const int dz = pr / 3, dy = pr % 3;
#pragma unroll
                    for (int kk = 0; kk < WG_TY / 2; ++kk)  // two 8-voxel rows per MMA (K = 16)
                        mma_f16(tmem + (uint32_t)(pr * 32), alo[dz] + ((uint32_t)(dy + 2 * kk) * WG_ROW_BYTES >> 4), h_hi,
                                glo + ((uint32_t)(2 * kk) * 512 >> 4), g_hi, (first && kk == 0) ? 0u : 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar0 + 8u * (uint32_t)k));
            }
            pending |= 1u << k;
            first = false;
            if (z + 1 < z_end) {
                // the buffers of step z - 1 are free once its MMAs are done; stage into them
                if (!drain(k ^ 1, spin)) {
                    s_fail = 1;
                    atomicExch(err, 1);
                }
                // plane z + 2 and g of step z + 1, loaded during the previous step
                wg_store_plane(sH + (uint32_t)((zi + 3) & 3) * WG_PLANE_BYTES, st);
                wg_store_g(sG + (uint32_t)(k ^ 1) * WG_G_BYTES, st, g_scale);
                if (z + 2 < z_end) {  // and the loads of what step z + 1 stages
                    wg_load_plane(st, hb, cin, vox, wrap(z + 3, D), y0, x0, H, Wd, vh);
                    wg_load_g(st, gbat, cout, vox, z + 2, y0, x0, H, Wd, vg);
                }
            }
        }
        // the column's last MMAs read the ring: wait for them before the next prologue
        for (int kb = 0; kb < 2; ++kb)
            if (!drain(kb, spin)) {
                s_fail = 1;
                atomicExch(err, 1);
            }
        __syncthreads();
    }
    // on a timeout, one more wait, bounded by the full limit whatever `spin` was, for MMAs still
    // in flight before the memory is freed
    for (int kb = 0; kb < 2; ++kb) drain(kb, kSpin);
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    // read the nine accumulators out: warp w < 4 holds rows 32 w .. 32 w + 31, i.e. dx = w, c = lane
    if (!s_fail && !first && t < 128) {
        const int warp = t / 32, c = t % 32;
        const float inv = 1.0f / g_scale;
        for (int pr = 0; pr < 9; ++pr) {
            uint32_t v[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
                  "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                  "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                  "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(pr * 32)));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (warp < 3 && c < cin) {
                const int tap = 9 * (pr / 3) + 3 * (pr % 3) + warp;
                float* pb = part + (long long)blockIdx.x * cout * cin * 27;
#pragma unroll
                for (int o = 0; o < 32; ++o)
                    if (o < cout) pb[((long long)o * cin + c) * 27 + tap] = __uint_as_float(v[o]) * inv;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// y[i] += sum over k < parts of x[k n + i], k in increasing order (the same bits on every run)
__global__ void sum_parts_kernel(const float* __restrict__ x, int parts, long long n, float* __restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int k = 0; k < parts; ++k) acc += x[(long long)k * n + i];
        y[i] += acc;
    }
}

// partial[blockIdx.x][o] = this block's sum over the batch and the voxels of g[b][o][v]
__global__ void bias_grad_kernel(const float* __restrict__ g, int cout, long long vox, int batch, float* __restrict__ part) {
    __shared__ float red[256 / 32];
    const int o = blockIdx.y;
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < vox * batch; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / vox, v = i - b * vox;
        acc += g[(b * cout + o) * vox + v];
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[(long long)blockIdx.x * cout + o] = s;
    }
}

}  // namespace tc

cudaError_t weight_image(const float* W, int cout, int cin, __half* img, cudaStream_t s) {
    if (cout > 32 || cin > 32) return cudaErrorInvalidValue;
    const int n = 32 * 32 * 27;
    tc::weight_image_kernel<<<(n + 255) / 256, 256, 0, s>>>(W, cout, cin, img);
    return cudaGetLastError();
}

size_t weight_image_bytes() { return tc::W_BYTES; }

// Two persistent CTAs per SM of the current device.
static int tc_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 2 * (sms > 0 ? sms : 1);
}

int wgrad_parts() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

size_t wgrad_scratch_floats() { return (size_t)wgrad_parts() * 32 * 32 * 27 + (size_t)kBiasParts * 32; }

cudaError_t wgrad32_tc(const float* g, int cout, float g_scale, const void* h, int h_fp16, int cin, float* gW, float* gb,
                       int batch, int D, int H, int Wd, long long spin, float* scratch, int* err, cudaStream_t s) {
    if (cin > 32 || cout > 32) return cudaErrorInvalidValue;
    const int tx = (Wd + tc::WG_TX - 1) / tc::WG_TX, ty = (H + tc::WG_TY - 1) / tc::WG_TY;
    const int n_chunks = (D + tc::WG_ZCHUNK - 1) / tc::WG_ZCHUNK;
    const int n_columns = tx * ty * n_chunks * batch;
    const int sms = wgrad_parts();
    const int blocks = n_columns < sms ? n_columns : sms;  // 512 tensor-memory columns each: one per SM
    // each CTA writes its sums over its columns to its own slice of the scratch; the slices are
    // then added in CTA order, so the gradients are the same bits on every run
    float* wpart = scratch;
    float* bpart = scratch + (size_t)sms * 32 * 32 * 27;
    // 16-byte row loads where every 8-voxel run is aligned and inside its row
    const int vec_h = (Wd % 8 == 0) && ((uintptr_t)h % 16 == 0);
    const int vec_g = (Wd % 8 == 0) && ((uintptr_t)g % 16 == 0);
    cudaError_t e;
    if (h_fp16) {
        e = cudaFuncSetAttribute(tc::wgrad32_tc_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::WG_SMEM);
        if (e != cudaSuccess) return e;
        tc::wgrad32_tc_kernel<__half><<<blocks, tc::WG_THREADS, tc::WG_SMEM, s>>>(
            g, cout, g_scale, (const __half*)h, cin, wpart, D, H, Wd, tx, ty, n_chunks, n_columns, vec_h, vec_g, spin, err);
    } else {
        e = cudaFuncSetAttribute(tc::wgrad32_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::WG_SMEM);
        if (e != cudaSuccess) return e;
        tc::wgrad32_tc_kernel<float><<<blocks, tc::WG_THREADS, tc::WG_SMEM, s>>>(
            g, cout, g_scale, (const float*)h, cin, wpart, D, H, Wd, tx, ty, n_chunks, n_columns, vec_h, vec_g, spin, err);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long nw = (long long)cout * cin * 27;
    tc::sum_parts_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(wpart, blocks, nw, gW);
    const long long vox = (long long)D * H * Wd;
    const long long blk = (vox * batch + 255) / 256;
    const int bblocks = (int)(blk < kBiasParts ? blk : kBiasParts);
    tc::bias_grad_kernel<<<dim3((unsigned)bblocks, (unsigned)cout), 256, 0, s>>>(g, cout, vox, batch, bpart);
    tc::sum_parts_kernel<<<1, 256, 0, s>>>(bpart, bblocks, cout, gb);
    return cudaGetLastError();
}

cudaError_t conv32_tc(const void* in, int in_fp16, int cin, float in_scale, const __half* wimg, const float* bias, void* out,
                      int out_fp16, int cout, int relu, int batch, int D, int H, int Wd, long long spin, int* err,
                      cudaStream_t s) {
    if (cin > 32 || cout > 32) return cudaErrorInvalidValue;
    const int tx = (Wd + tc::TX - 1) / tc::TX, ty = (H + tc::TY - 1) / tc::TY;
    // z chunks of 8 planes: 10 staged planes per 8 steps, and enough columns to fill the GPU
    const int zchunk = D < 8 ? D : 8;
    const int n_chunks = (D + zchunk - 1) / zchunk;
    const int n_columns = tx * ty * n_chunks * batch;
    const int blocks = n_columns < tc_blocks() ? n_columns : tc_blocks();
    // 16-byte row loads where every 8-voxel run is aligned and inside its row
    const int vec_in = (Wd % 8 == 0) && ((uintptr_t)in % 16 == 0);
#define LBM_TC(TIN, MODE, TOUT)                                                                                    \
    do {                                                                                                           \
        cudaError_t e_ = cudaFuncSetAttribute(tc::conv32_tc_kernel<TIN, MODE, TOUT>,                              \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);         \
        if (e_ != cudaSuccess) return e_;                                                                          \
        tc::conv32_tc_kernel<TIN, MODE, TOUT><<<blocks, tc::CONV_THREADS, tc::SMEM, s>>>(                          \
            (const TIN*)in, cin, in_scale, wimg, bias, (TOUT*)out, cout, D, H, Wd, tx, ty, zchunk, n_chunks,       \
            n_columns, vec_in, spin, err);                                                                         \
    } while (0)
    if (in_fp16 && out_fp16 && relu) LBM_TC(__half, 1, __half);
    else if (!in_fp16 && !out_fp16 && !relu) LBM_TC(float, 0, float);
    else if (in_fp16 && !out_fp16 && !relu) LBM_TC(__half, 0, float);
    else return cudaErrorInvalidValue;
#undef LBM_TC
    return cudaGetLastError();
}

}  // namespace net
}  // namespace lbm
