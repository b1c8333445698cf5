// mass_noalloc.cu -- lbm_mass_noalloc: the FP64 mass reduction for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc. Examples:
//  * a solver whose populations already fill the GPU, so there is nothing left to allocate;
//  * code that runs under a memory manager which owns every device allocation (a framework's
//    caching pool, a fixed arena sized at start-up);
//  * a loop that must not stall on the driver's allocator between steps.
// The handle-based lbm_mass needs scratch for its per-block partial sums and gets it from
// cudaMalloc in lbm_create. This entry point instead keeps that scratch in a file-scope
// __device__ array with a fixed maximum size. Every GPU that loads the library holds the array
// until the process exits. The caller owns the input populations and the output.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "../../include/lbm.h"
#include "cell.cuh"

namespace lbm {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 2048;  // partial triples the static scratch holds

// One FP64 triple (sum phi, sum rho phi, non-finite count) per block of the last call.
static __device__ __align__(256) double g_noalloc_partials[3 * kNoallocMaxBlocks];

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_sum3_d(double (&v)[3], double* out) {
    __shared__ double red[3][kNoallocThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = warp_sum_d(v[k]);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double w = (lane < kNoallocThreads / 32) ? red[k][lane] : 0.0;
            w = warp_sum_d(w);
            if (lane == 0) out[k] = w;
        }
    }
}

// Block b covers z-layer b / bpl, rows [r0, r1) of it; it writes its triple to partials[b].
// phi = sum_i of the Lax-Wendroff-propagated g_i (plane 0, the rest population, does not move).
// Where a stencil point x -+ e_i lies beyond a wall, it reads the opposite population of this
// cell (half-way bounce-back), as the time step does.
template <int Q>
__global__ void __launch_bounds__(kNoallocThreads)
mass_noalloc_kernel(const Params P, const float* __restrict__ g, int blocks_per_layer, double* __restrict__ partials) {
    const int z = blockIdx.x / blocks_per_layer, part = blockIdx.x % blocks_per_layer;
    const int rows_per = (P.ny + blocks_per_layer - 1) / blocks_per_layer;
    const int r0 = part * rows_per, r1 = min(P.ny, r0 + rows_per);
    const size_t N = (size_t)P.N;
    double acc[3] = {0.0, 0.0, 0.0};
    const int n = (r1 > r0) ? (r1 - r0) * P.nx : 0;
    for (int k = threadIdx.x; k < n; k += kNoallocThreads) {
        const int y = r0 + k / P.nx, x = k % P.nx;
        const int c = (z * P.ny + y) * P.nx + x;
        const Nbr nb = make_nbr(P, x, y, z);
        const WallSide ws = make_wall_side(P, x, y, z);
        float phi = __ldg(g + c);
        int bad = !isfinite(phi);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float* gq = g + i * N;
            const float* back = g + Lat<Q>::opp(i) * N + c;
            const float g0 = __ldg(gq + c);
            const float gm = __ldg(crosses_wall<Q>(ws, i, -1) ? back : gq + c + link_offset<Q>(nb, i, -1));
            const float gp = __ldg(crosses_wall<Q>(ws, i, +1) ? back : gq + c + link_offset<Q>(nb, i, +1));
            phi += g0 + (P.lw_m * (gm - g0) + P.lw_p * (gp - g0));
            bad += !isfinite(g0);
        }
        const double pd = (double)phi;
        acc[0] += pd;
        acc[1] += (P.rho2_d + P.drho_d * pd) * pd;
        acc[2] += (double)bad;
    }
    block_sum3_d(acc, partials + 3 * blockIdx.x);
}

__global__ void __launch_bounds__(kNoallocThreads)
mass_noalloc_finish(const double* __restrict__ partials, int n, double* __restrict__ result) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < n; b += kNoallocThreads)
        for (int k = 0; k < 3; ++k) acc[k] += partials[3 * b + k];
    block_sum3_d(acc, result);
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_mass_noalloc(const float* g, int lattice, const int grid[3], int walls, double courant,
                                double rho_ratio, double* result, void* stream) {
    if (!g || !grid || !result) return LBM_EINVAL;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) return LBM_EINVAL;
    const int nx = grid[0], ny = grid[1], nz = grid[2];
    if (nx < 3 || ny < 3 || (lattice == LBM_D2Q9 && nz != 1) || (lattice == LBM_D3Q19 && nz < 3)) return LBM_EINVAL;
    if ((long long)nx * ny * nz >= (long long)INT_MAX) return LBM_EINVAL;
    // The static scratch holds kNoallocMaxBlocks partial triples and each z-layer takes at least
    // one block, so grids deeper than that are rejected.
    if (nz > lbm::kNoallocMaxBlocks) return LBM_EINVAL;
    if (walls < 0 || walls > 7 || (lattice == LBM_D2Q9 && (walls & 4))) return LBM_EINVAL;
    if (!(courant > 0 && courant <= 1) || !(rho_ratio > 0) || !std::isfinite(rho_ratio)) return LBM_EINVAL;

    // The array's device address in the current context, looked up on every call: host code
    // only knows a host-side stand-in for the symbol, and the address changes if the caller
    // resets the device and a new context loads the module.
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, lbm::g_noalloc_partials) != cudaSuccess) {
        (void)cudaGetLastError();  // this call's own failure, reported by the return code
        return LBM_ECUDA;
    }
    double* partials = static_cast<double*>(scratch);

    lbm::Params P = {};
    P.Q = lattice;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.nxy = nx * ny;
    P.N = (long long)nx * ny * nz;
    P.walls = walls;
    P.lw_m = (float)(0.5 * courant * (1.0 + courant));
    P.lw_p = (float)(-0.5 * courant * (1.0 - courant));
    P.rho2_d = 1.0;
    P.drho_d = rho_ratio - 1.0;
    int bpl = lbm::kNoallocMaxBlocks / nz;
    if (bpl > ny) bpl = ny;
    if (bpl < 1) bpl = 1;
    int blocks = nz * bpl;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Launched through cudaLaunchKernel so that each launch's own status is checked: an error
    // that earlier, unrelated work left on this thread is neither blamed on this call nor
    // cleared by it.
    const void* kernel = (lattice == LBM_D2Q9) ? (const void*)lbm::mass_noalloc_kernel<9>
                                               : (const void*)lbm::mass_noalloc_kernel<19>;
    void* args1[] = {&P, (void*)&g, &bpl, &partials};
    cudaError_t e = cudaLaunchKernel(kernel, dim3(blocks), dim3(lbm::kNoallocThreads), args1, 0, s);
    if (e == cudaSuccess) {
        void* args2[] = {&partials, &blocks, &result};
        e = cudaLaunchKernel((const void*)lbm::mass_noalloc_finish, dim3(1), dim3(lbm::kNoallocThreads), args2, 0, s);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return LBM_ECUDA;
    }
    return LBM_OK;
}
