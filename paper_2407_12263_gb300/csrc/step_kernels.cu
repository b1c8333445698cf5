// step_kernels.cu -- the fused time step of the difference-free conservative phase-field LBM
// (Zhao, Patel & Lee, arXiv:2407.12263) and its finite-difference twin.
//
// Difference-free step: ONE kernel per time step. Each thread owns one cell; it pulls the
// Lax-Wendroff-propagated f and g (three loads per moving population, Sec. 2.2), computes
// phi, rho, u, the central moment K1, n, S, grad phi and p in registers (Sec. 2.3), collides
// both sets (Eqs. c-n_m and c-n_c) and streams the 2Q post-collision values out. The
// neighbour loads of adjacent threads overlap, so DRAM sees each stored value about once per
// step; everything else is L1/L2 reuse.
//
// Finite-difference variant (the "previous method" of Sec. 3.4): a first kernel propagates g
// and writes the phi plane; the second is the fused step with grad phi taken from the
// isotropic central difference of that plane instead of K1.
#include "cell.cuh"

namespace lbm {

// Thread block: one cell per thread, x fastest (a warp spans 32 consecutive cells of a row).
// 32 x 4 threads with a 72-register budget (7 blocks per SM) measured best among the shapes
// and budgets tried on the 128^3 workload (all within 69-75% of the HBM roofline).
#ifndef LBM_STEP_BX
#define LBM_STEP_BX 32
#endif
#ifndef LBM_STEP_BY
#define LBM_STEP_BY 4
#endif
#ifndef LBM_STEP_BZ
#define LBM_STEP_BZ 1
#endif
#ifndef LBM_STEP_MINB
#define LBM_STEP_MINB 7
#endif
constexpr int kStepBX = LBM_STEP_BX, kStepBY = LBM_STEP_BY, kStepBZ = LBM_STEP_BZ;
constexpr int kStepThreads = kStepBX * kStepBY * kStepBZ;

template <int Q, int SCHEME, bool GEN>
__global__ void __launch_bounds__(kStepThreads, LBM_STEP_MINB)
step_kernel(const Params P, const float* __restrict__ f_in, const float* __restrict__ g_in,
            float* __restrict__ f_out, float* __restrict__ g_out, const float* __restrict__ phi_fd) {
    const int x = blockIdx.x * kStepBX + threadIdx.x;
    const int y = blockIdx.y * kStepBY + threadIdx.y;
    const int z = blockIdx.z * kStepBZ + threadIdx.z;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const Nbr nb = make_nbr(P, x, y, z);
    const int c = (z * P.ny + y) * P.nx + x;

    float fb[Q], gb[Q];
    pull<Q, true>(P, f_in, g_in, c, nb, fb, gb);

    Macro m;
    macro_flow<Q, GEN>(P, fb, gb, m);
    if (SCHEME == SCHEME_DF) {
        macro_interface_df<Q>(P, gb, m);
    } else {
        float gx, gy, gz;
        fd_gradient<Q>(phi_fd, c, nb, gx, gy, gz);
        macro_interface_fd(P, gx, gy, gz, m);
    }
    macro_pressure<GEN>(P, m);
    collide<Q, GEN>(P, m, fb, gb);

    const size_t N = (size_t)P.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        __stcs(f_out + i * N + c, fb[i]);   // streaming stores: the output is not re-read this step
        __stcs(g_out + i * N + c, gb[i]);
    }
}

// Finite-difference variant, pass 1: the propagated phi (held as phi - phi_ref), one FP32 plane.
template <int Q>
__global__ void __launch_bounds__(kStepThreads)
fd_phi_kernel(const Params P, const float* __restrict__ g_in, float* __restrict__ phi) {
    const int x = blockIdx.x * kStepBX + threadIdx.x;
    const int y = blockIdx.y * kStepBY + threadIdx.y;
    const int z = blockIdx.z * kStepBZ + threadIdx.z;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const Nbr nb = make_nbr(P, x, y, z);
    const int c = (z * P.ny + y) * P.nx + x;
    float fb[Q], gb[Q];
    pull<Q, false>(P, nullptr, g_in, c, nb, fb, gb);
    phi[c] = gb[0];
}

static dim3 step_grid(const Params& P) {
    return dim3((P.nx + kStepBX - 1) / kStepBX, (P.ny + kStepBY - 1) / kStepBY, (P.nz + kStepBZ - 1) / kStepBZ);
}

template <int Q>
static cudaError_t step_q(const Params& P, int scheme, const float* fi, const float* gi, float* fo,
                          float* go, float* phi, cudaStream_t s, int* launches) {
    const dim3 grid = step_grid(P), block(kStepBX, kStepBY, kStepBZ);
    if (scheme == SCHEME_DF) {
        if (P.general) step_kernel<Q, SCHEME_DF, true><<<grid, block, 0, s>>>(P, fi, gi, fo, go, nullptr);
        else step_kernel<Q, SCHEME_DF, false><<<grid, block, 0, s>>>(P, fi, gi, fo, go, nullptr);
        *launches += 1;
    } else {
        fd_phi_kernel<Q><<<grid, block, 0, s>>>(P, gi, phi);
        if (P.general) step_kernel<Q, SCHEME_FD, true><<<grid, block, 0, s>>>(P, fi, gi, fo, go, phi);
        else step_kernel<Q, SCHEME_FD, false><<<grid, block, 0, s>>>(P, fi, gi, fo, go, phi);
        *launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_step(const Params& P, int scheme, const float* f_in, const float* g_in,
                        float* f_out, float* g_out, float* phi_fd, cudaStream_t s, int* launches) {
    if (P.Q == 9) return step_q<9>(P, scheme, f_in, g_in, f_out, g_out, phi_fd, s, launches);
    return step_q<19>(P, scheme, f_in, g_in, f_out, g_out, phi_fd, s, launches);
}

cudaError_t launch_fd_phi(const Params& P, const float* g_in, float* phi_fd, cudaStream_t s) {
    const dim3 grid = step_grid(P), block(kStepBX, kStepBY, kStepBZ);
    if (P.Q == 9) fd_phi_kernel<9><<<grid, block, 0, s>>>(P, g_in, phi_fd);
    else fd_phi_kernel<19><<<grid, block, 0, s>>>(P, g_in, phi_fd);
    return cudaGetLastError();
}

}  // namespace lbm
