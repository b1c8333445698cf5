// project.cu -- the divergence-free projection of a periodic velocity field
// (lbm_project_solenoidal, include/lbm_surrogate.h): the surrogate's predicted velocity is
// replaced by the closest field whose central-difference divergence vanishes before the lattice
// restarts from it. At low Mach number the flow is divergence-free (Sec. 2.1 of arXiv:2407.12263,
// with the pressure evolution equation); a compressive prediction would be relaxed away by the
// lattice through pressure waves.
//
// The discrete Fourier transform diagonalises the central difference D_a: a mode of wavenumber
// k_a along axis a is multiplied by i s_a, s_a = sin(2 pi k_a / n_a). The projection is
// U <- U - s (s . U) / |s|^2 per mode (modes with s = 0 carry no divergence and stay), between a
// forward and an inverse transform along x, y and z.
//
// Each transform pass is one kernel: a block stages 8 lines along its axis (with the twiddles
// of that axis) in shared memory and evaluates every output of those lines as a direct sum in
// FP32, in a fixed order (the same bits on every run). Lines along x are rows; along y and z a
// block takes 8 neighbouring x positions, so every global access covers 8 consecutive values.
// The coarse grids this serves are small (64^3 for a 256^3 lattice at factor 4): the direct sums
// cost n complex multiply-adds per output, 6 passes of 3 components.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "../../include/lbm.h"
#include "../../include/lbm_surrogate.h"
#include "surrogate.h"

namespace lbm {
namespace proj {

constexpr int kLines = 8;       // lines per block
constexpr int kThreads = 256;
constexpr int kMaxExtent = 512;  // (kLines + 1) (n + 1) float2 of shared memory stay below 48 KB

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace: the twiddles of the three axes (nx + ny + nz float2), then the spectrum
// [3][nz][ny][nx] float2.
inline size_t twiddle_bytes(int nx, int ny, int nz) { return align256((size_t)(nx + ny + nz) * sizeof(float2)); }
inline size_t workspace_bytes(int nx, int ny, int nz) {
    return twiddle_bytes(nx, ny, nz) + (size_t)3 * nx * ny * nz * sizeof(float2);
}

// w[m] = exp(-2 pi i m / n) for each axis, from the FP64 cospi / sinpi, which are exactly 0 and
// +-1 where 2 m / n is an integer or a half-integer.
__global__ void twiddle_kernel(float2* tw, int nx, int ny, int nz) {
    const int total = nx + ny + nz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int n = t < nx ? nx : t < nx + ny ? ny : nz;
        const int m = t < nx ? t : t < nx + ny ? t - nx : t - nx - ny;
        double s, c;
        sincospi(2.0 * m / n, &s, &c);
        tw[t] = make_float2((float)c, (float)-s);
    }
}

// One transform pass along AXIS (0 x, 1 y, 2 z) over the spectrum W (in place). inverse: the
// conjugate twiddles. in_real (pass along x only): read the real field [3][N] instead of W.
// out_real (pass along x only): write scale times the real part to [3][N] instead of W.
template <int AXIS>
__global__ void __launch_bounds__(kThreads) dft_kernel(float2* __restrict__ W, const float2* __restrict__ tw_axis,
                                                       const float* __restrict__ in_real, float* __restrict__ out_real,
                                                       int nx, int ny, int nz, int inverse, float scale) {
    extern __shared__ float2 sm[];
    const int n = AXIS == 0 ? nx : AXIS == 1 ? ny : nz;
    const int ld = n + 1;  // padded line: the 8 lines of a warp's reads sit in different banks
    float2* tw = sm;
    float2* tile = sm + ld;
    long long base, lstride, estride;
    int nl;
    if (AXIS == 0) {
        const long long l0 = (long long)blockIdx.x * kLines, lines = 3ll * nz * ny;
        nl = (int)min((long long)kLines, lines - l0);
        base = l0 * nx;
        lstride = nx;
        estride = 1;
    } else {
        const int xt = (nx + kLines - 1) / kLines;
        const int x0 = (int)(blockIdx.x % xt) * kLines;
        const long long outer = blockIdx.x / xt;  // (component, z) for y lines, (component, y) for z lines
        nl = min(kLines, nx - x0);
        if (AXIS == 1) {
            base = outer * ny * (long long)nx + x0;
            estride = nx;
        } else {
            const long long c = outer / ny, y = outer % ny;
            base = c * (long long)nz * ny * nx + y * nx + x0;
            estride = (long long)nx * ny;
        }
        lstride = 1;
    }
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const float2 w = tw_axis[m];
        tw[m] = inverse ? make_float2(w.x, -w.y) : w;
    }
    // element (l, j): line l, position j; l fastest, so a warp touches 4 positions of 8 lines
    for (int t = threadIdx.x; t < kLines * n; t += blockDim.x) {
        const int l = t % kLines, j = t / kLines;
        float2 v = make_float2(0.f, 0.f);
        if (l < nl) {
            const long long o = base + l * lstride + j * estride;
            v = in_real ? make_float2(in_real[o], 0.f) : W[o];
        }
        tile[l * ld + j] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kLines * n; t += blockDim.x) {
        const int l = t % kLines, k = t / kLines;
        if (l >= nl) continue;
        const float2* x = tile + l * ld;
        float re = 0.f, im = 0.f;
        int m = 0;  // j k mod n
        for (int j = 0; j < n; ++j) {
            const float2 a = x[j], w = tw[m];
            re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
            im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
            m += k;
            if (m >= n) m -= n;
        }
        const long long o = base + l * lstride + k * estride;
        if (out_real) out_real[o] = re * scale;
        else W[o] = make_float2(re, im);
    }
}

// U <- U - s (s . U) / |s|^2 for every mode (kx, ky, kz); s_a = sin(2 pi k_a / n_a) = -Im w_a[k_a].
__global__ void project_modes_kernel(float2* __restrict__ W, const float2* __restrict__ tw, int nx, int ny, int nz) {
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nx), ky = (int)((i / nx) % ny), kz = (int)(i / ((long long)nx * ny));
        const float sx = -tw[kx].y, sy = -tw[nx + ky].y, sz = -tw[nx + ny + kz].y;
        const float s2 = sx * sx + sy * sy + sz * sz;
        if (!(s2 > 0.f)) continue;
        const float2 ux = W[i], uy = W[N + i], uz = W[2 * N + i];
        const float dre = (sx * ux.x + sy * uy.x + sz * uz.x) / s2;
        const float dim = (sx * ux.y + sy * uy.y + sz * uz.y) / s2;
        W[i] = make_float2(ux.x - sx * dre, ux.y - sx * dim);
        W[N + i] = make_float2(uy.x - sy * dre, uy.y - sy * dim);
        W[2 * N + i] = make_float2(uz.x - sz * dre, uz.y - sz * dim);
    }
}

inline size_t dft_smem(int n) { return (size_t)(kLines + 1) * (n + 1) * sizeof(float2); }

template <int AXIS>
cudaError_t dft(float2* W, const float2* tw, const float* in_real, float* out_real, int nx, int ny, int nz, int inverse,
                float scale, cudaStream_t s) {
    const int n = AXIS == 0 ? nx : AXIS == 1 ? ny : nz;
    const long long blocks = AXIS == 0 ? (3ll * nz * ny + kLines - 1) / kLines
                                       : 3ll * (AXIS == 1 ? nz : ny) * ((nx + kLines - 1) / kLines);
    const float2* tw_axis = tw + (AXIS == 0 ? 0 : AXIS == 1 ? nx : nx + ny);
    dft_kernel<AXIS><<<(unsigned)blocks, kThreads, dft_smem(n), s>>>(W, tw_axis, in_real, out_real, nx, ny, nz, inverse,
                                                                     scale);
    return cudaGetLastError();
}

}  // namespace proj

// The whole projection of u [3][nz][ny][nx] in place: 9 launches on stream s.
cudaError_t launch_project_solenoidal(float* u, int nx, int ny, int nz, void* work, cudaStream_t s) {
    using namespace proj;
    float2* tw = static_cast<float2*>(work);
    float2* W = reinterpret_cast<float2*>(static_cast<char*>(work) + twiddle_bytes(nx, ny, nz));
    const long long N = (long long)nx * ny * nz;
    cudaError_t e;
    twiddle_kernel<<<1, kThreads, 0, s>>>(tw, nx, ny, nz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = dft<0>(W, tw, u, nullptr, nx, ny, nz, 0, 1.f, s)) != cudaSuccess) return e;
    if ((e = dft<1>(W, tw, nullptr, nullptr, nx, ny, nz, 0, 1.f, s)) != cudaSuccess) return e;
    if ((e = dft<2>(W, tw, nullptr, nullptr, nx, ny, nz, 0, 1.f, s)) != cudaSuccess) return e;
    const long long pb = (N + kThreads - 1) / kThreads;
    project_modes_kernel<<<(unsigned)(pb < 4096 ? pb : 4096), kThreads, 0, s>>>(W, tw, nx, ny, nz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = dft<2>(W, tw, nullptr, nullptr, nx, ny, nz, 1, 1.f, s)) != cudaSuccess) return e;
    if ((e = dft<1>(W, tw, nullptr, nullptr, nx, ny, nz, 1, 1.f, s)) != cudaSuccess) return e;
    return dft<0>(W, tw, nullptr, u, nx, ny, nz, 1, (float)(1.0 / (double)N), s);
}

size_t project_workspace_bytes(int nx, int ny, int nz) { return proj::workspace_bytes(nx, ny, nz); }

bool project_extents_ok(const int grid[3]) {
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1 || grid[a] > proj::kMaxExtent) return false;
    return true;
}

}  // namespace lbm

extern "C" {

long long lbm_project_workspace_bytes(const int grid[3]) {
    if (!grid || !lbm::project_extents_ok(grid)) return -1;
    return (long long)lbm::project_workspace_bytes(grid[0], grid[1], grid[2]);
}

int lbm_project_solenoidal(float* u, const int grid[3], void* work, long long work_bytes, void* stream) {
    if (!u || !grid || !work || !lbm::project_extents_ok(grid)) return LBM_EINVAL;
    if (reinterpret_cast<uintptr_t>(u) % sizeof(float) || reinterpret_cast<uintptr_t>(work) % 16) return LBM_EINVAL;
    if (work_bytes < (long long)lbm::project_workspace_bytes(grid[0], grid[1], grid[2])) return LBM_EINVAL;
    const cudaError_t e = lbm::launch_project_solenoidal(u, grid[0], grid[1], grid[2], work, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // this call's own launch failure, reported by the return code
        return LBM_ECUDA;
    }
    return LBM_OK;
}

}  // extern "C"
