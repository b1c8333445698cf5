// batch_kernels.cu -- many independent cases of the difference-free conservative phase-field
// LBM (arXiv:2407.12263) of one grid size advanced by ONE launch ("group launch").
//
// The group's cases (up to 128, each with its own fluid properties and buffers) travel in the
// kernel's parameter block. Block (t, k, tz) runs one tile of 128 cells, a 2^a x 2^b x 2^c box
// chosen by the tuner, of case k = blockIdx.y: the case index is uniform over the block, so its
// parameter reads are uniform loads from the constant bank. Each thread runs step_cell,
// the same per-cell code as the single-case kernel, so a case gives the same bits either way.
// A group of 35 cases of 32^3 cells is 8960 blocks, where each case alone is 256: the group
// fills the 152 SMs that a single small case cannot.
#include "cell.cuh"

namespace lbm {

// Register budget: 5 blocks (96 registers) per SM for the general kernels (walls, forces,
// density ratio), 4 (128) for the periodic ones. The wall-bounded boxes batches hold keep a
// group launch waiting on DRAM latency at 16 warps per SM; at 20 the FP32 group launches of
// 256 rising-bubble cases ran 4.7% faster (15.94 -> 16.69 G cell/s) although the FP32 kernel
// spills 16 bytes there, and the 16-bit ones fit without spilling. The periodic 16-bit kernels
// would spill 8 to 16 bytes at 96.
template <bool GEN, int S>
constexpr int batch_min_blocks() {
    return GEN ? 5 : 4;
}

template <int Q, bool GEN, int S>
__global__ void __launch_bounds__(kBatchThreads, (batch_min_blocks<GEN, S>()))
batch_step_kernel(const __grid_constant__ BatchLaunch L) {
    const LaunchCase& C = L.cases[blockIdx.y];
    // The host groups cases that share every parameter except their fluid properties (see
    // group_key in lbm_batch.cu), so those shared fields are read from case 0, at fixed offsets
    // of the parameter block: operands of the instructions that use them, not loads. Only the
    // fluid properties of case blockIdx.y are loads through a run-time index.
    Params P = L.cases[0].P;
    P.tau_f = C.P.tau_f;
    P.omega_f = C.P.omega_f;
    P.drho = C.P.drho;
    P.mu_m1 = C.P.mu_m1;
    P.sigma = C.P.sigma;
    P.G[0] = C.P.G[0];
    P.G[1] = C.P.G[1];
    P.G[2] = C.P.G[2];
    const int txs = L.tx_shift, tys = L.ty_shift, tzs = 7 - txs - tys;
    const int ty_i = blockIdx.x / L.ntx;
    const int tx_i = blockIdx.x - ty_i * L.ntx;
    const int tid = threadIdx.x;
    const int x = (tx_i << txs) + (tid & ((1 << txs) - 1));
    const int y = (ty_i << tys) + ((tid >> txs) & ((1 << tys) - 1));
    const int z = ((int)blockIdx.z << tzs) + (tid >> (txs + tys));
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const int par = C.cur ^ L.flip;
    step_cell<Q, SCHEME_DF, GEN, S>(P, C.fg[par], C.fg[1 - par], nullptr, x, y, z);
}

template <int Q>
static void launch_q(const BatchLaunch& L, dim3 grid, cudaStream_t s) {
    if (L.general) {
        if (L.storage == STORE_F16) batch_step_kernel<Q, true, STORE_F16><<<grid, kBatchThreads, 0, s>>>(L);
        else if (L.storage == STORE_BF16) batch_step_kernel<Q, true, STORE_BF16><<<grid, kBatchThreads, 0, s>>>(L);
        else batch_step_kernel<Q, true, STORE_F32><<<grid, kBatchThreads, 0, s>>>(L);
    } else {
        if (L.storage == STORE_F16) batch_step_kernel<Q, false, STORE_F16><<<grid, kBatchThreads, 0, s>>>(L);
        else if (L.storage == STORE_BF16) batch_step_kernel<Q, false, STORE_BF16><<<grid, kBatchThreads, 0, s>>>(L);
        else batch_step_kernel<Q, false, STORE_F32><<<grid, kBatchThreads, 0, s>>>(L);
    }
}

cudaError_t launch_batch_group(int Q, const BatchLaunch& L, cudaStream_t s) {
    if (L.n_cases <= 0) return cudaSuccess;
    const dim3 grid((unsigned)(L.ntx * L.nty), (unsigned)L.n_cases, (unsigned)L.ntz);
    if (Q == 9) launch_q<9>(L, grid, s);
    else launch_q<19>(L, grid, s);
    return cudaGetLastError();
}

__global__ void fill_plane0_kernel(float2* plane0, long long N) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        plane0[c] = make_float2(0.0f, __int_as_float(1 << 30));
}

cudaError_t launch_fill_rest(const Params& P, void* fg, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(fg, 0, state_bytes(P.Q, P.N, P.storage), s);
    if (e != cudaSuccess) return e;
    const long long blocks = (P.N + 255) / 256;
    fill_plane0_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(moment_plane(fg), P.N);
    return cudaGetLastError();
}

}  // namespace lbm
