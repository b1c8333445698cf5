// step_kernels.cu -- the fused time step of the difference-free conservative phase-field LBM
// (Zhao, Patel & Lee, arXiv:2407.12263) and its finite-difference twin.
//
// Difference-free step: ONE kernel per time step. Each thread owns one cell; it pulls the
// Lax-Wendroff-propagated f and g (Sec. 2.2: for each opposite pair of populations, three loads
// of the word that holds both (f, g) pairs, at x - e_i, x and x + e_i), computes phi, rho, u,
// the central moment K1, n, S, grad phi and p in registers (Sec. 2.3), collides both sets
// (Eqs. c-n_m and c-n_c) and streams the Q post-collision pairs out, one word per opposite
// pair. The neighbour loads of adjacent threads overlap, so DRAM sees each stored value about
// once per step; everything else is L1/L2 reuse. Interleaving f with g, and a population with
// its opposite, divides the memory instructions per cell by four, and that count (not bytes) is
// what limits a 3-point stencil over 38 planes: with separate planes the same step ran at 74%
// of the HBM copy bandwidth, with (f, g) pairs at 0.98, with opposite pairs interleaved too at
// the copy bandwidth.
//
// Finite-difference variant (the "previous method" of Sec. 3.4): a first kernel propagates g
// and writes the phi plane; the second is the fused step with grad phi taken from the
// isotropic central difference of that plane instead of K1.
#include "cell.cuh"

namespace lbm {

// Thread block: 128 threads, one cell per thread, x fastest. The host picks the shape: one
// 128-cell row per block where rows are at least that long, else 32 x 4 (a warp spans 32
// consecutive cells of a row either way). With FP32 storage the register budget allows 4
// blocks (16 warps) per SM: the difference-free step needs ~122 registers and runs at that
// occupancy with every (f, g) load of a cell in flight. A 16-bit cell moves half the bytes, so
// the same bandwidth needs more cells in flight: the 16-bit steps are held to 96 registers for
// 5 blocks (20 warps), which they fit without spilling.
constexpr int kStepThreads = 128;
constexpr int LBM_STEP_MINB = 4;

template <int S>
constexpr int step_min_blocks() {
    return S == STORE_F32 ? LBM_STEP_MINB : 5;
}

template <int Q, int SCHEME, bool GEN, int S>
__global__ void __launch_bounds__(kStepThreads, (step_min_blocks<S>()))
step_kernel(const Params P, const void* __restrict__ fg_in, void* __restrict__ fg_out,
            const float* __restrict__ phi_fd) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    step_cell<Q, SCHEME, GEN, S>(P, fg_in, fg_out, phi_fd, x, y, z);
}

// Finite-difference variant, pass 1: the propagated phi (held as phi - phi_ref), one FP32 plane.
template <int Q, int S, bool WALLS>
__global__ void __launch_bounds__(kStepThreads, LBM_STEP_MINB)
fd_phi_kernel(const Params P, const void* __restrict__ fg_in, float* __restrict__ phi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const Nbr nb = make_nbr(P, x, y, z);
    const int c = (z * P.ny + y) * P.nx + x;
    float fb[Q], gb[Q];
    int phi_fx;
    pull<Q, false, S, WALLS>(P, fg_in, c, nb, fb, gb, phi_fx, WALLS ? make_wall_side(P, x, y, z) : WallSide{});
    phi[c] = gb[0];
}

static dim3 step_block(const Params& P) { return P.nx >= 128 ? dim3(128, 1, 1) : dim3(32, 4, 1); }

static dim3 step_grid(const Params& P) {
    const dim3 b = step_block(P);
    return dim3((P.nx + b.x - 1) / b.x, (P.ny + b.y - 1) / b.y, P.nz);
}

template <int Q, int S>
static cudaError_t step_qs(const Params& P, int scheme, const void* in, void* out, float* phi, cudaStream_t s,
                           int* launches) {
    const dim3 grid = step_grid(P), block = step_block(P);
    if (scheme == SCHEME_DF) {
        if (P.general) step_kernel<Q, SCHEME_DF, true, S><<<grid, block, 0, s>>>(P, in, out, nullptr);
        else step_kernel<Q, SCHEME_DF, false, S><<<grid, block, 0, s>>>(P, in, out, nullptr);
        *launches += 1;
    } else {
        if (P.walls) fd_phi_kernel<Q, S, true><<<grid, block, 0, s>>>(P, in, phi);
        else fd_phi_kernel<Q, S, false><<<grid, block, 0, s>>>(P, in, phi);
        if (P.general) step_kernel<Q, SCHEME_FD, true, S><<<grid, block, 0, s>>>(P, in, out, phi);
        else step_kernel<Q, SCHEME_FD, false, S><<<grid, block, 0, s>>>(P, in, out, phi);
        *launches += 2;
    }
    return cudaGetLastError();
}

template <int Q>
static cudaError_t step_q(const Params& P, int scheme, const void* in, void* out, float* phi, cudaStream_t s,
                          int* launches) {
    if (P.storage == STORE_F16) return step_qs<Q, STORE_F16>(P, scheme, in, out, phi, s, launches);
    if (P.storage == STORE_BF16) return step_qs<Q, STORE_BF16>(P, scheme, in, out, phi, s, launches);
    return step_qs<Q, STORE_F32>(P, scheme, in, out, phi, s, launches);
}

cudaError_t launch_step(const Params& P, int scheme, const void* fg_in, void* fg_out, float* phi_fd, cudaStream_t s,
                        int* launches) {
    if (P.Q == 9) return step_q<9>(P, scheme, fg_in, fg_out, phi_fd, s, launches);
    return step_q<19>(P, scheme, fg_in, fg_out, phi_fd, s, launches);
}

template <int Q, int S>
static void fd_phi_qs(const Params& P, const void* in, float* phi, cudaStream_t s) {
    if (P.walls) fd_phi_kernel<Q, S, true><<<step_grid(P), step_block(P), 0, s>>>(P, in, phi);
    else fd_phi_kernel<Q, S, false><<<step_grid(P), step_block(P), 0, s>>>(P, in, phi);
}

cudaError_t launch_fd_phi(const Params& P, const void* fg_in, float* phi_fd, cudaStream_t s) {
    if (P.Q == 9) {
        if (P.storage == STORE_F16) fd_phi_qs<9, STORE_F16>(P, fg_in, phi_fd, s);
        else if (P.storage == STORE_BF16) fd_phi_qs<9, STORE_BF16>(P, fg_in, phi_fd, s);
        else fd_phi_qs<9, STORE_F32>(P, fg_in, phi_fd, s);
    } else {
        if (P.storage == STORE_F16) fd_phi_qs<19, STORE_F16>(P, fg_in, phi_fd, s);
        else if (P.storage == STORE_BF16) fd_phi_qs<19, STORE_BF16>(P, fg_in, phi_fd, s);
        else fd_phi_qs<19, STORE_F32>(P, fg_in, phi_fd, s);
    }
    return cudaGetLastError();
}

}  // namespace lbm
