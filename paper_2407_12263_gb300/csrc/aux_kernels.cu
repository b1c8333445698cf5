// aux_kernels.cu -- initialisation, field output, FP64 mass reduction and population
// conversion for the difference-free conservative phase-field LBM (arXiv:2407.12263).
// None of these runs inside the time-step loop.
#include <cmath>

#include "cell.cuh"
#include "diagnostics.h"

namespace lbm {

constexpr int kAuxBX = 32, kAuxBY = 4;

// ---------------------------------------------------------------------------------------
// Initial post-collision populations:
//   grad phi0 = 3 sum_{i != 0} t_i e_i phi0(x + e_i)   (isotropic central difference)
//   n0 = grad phi0 / |grad phi0|, S0 = 4 phi0 (1 - phi0) / delta n0, rho0 = rho2 + drho phi0
//   f*_i = f^eq_i(p0, u0, rho0, Pi_s0)                                   (Eq. geq_s)
//   g*_i = g^eq_i(phi0, u0, S0) - t_i (tau_phi - 1/2) e_i . grad phi0     (Eq. geq)
// The g term is the first-order non-equilibrium part a relaxed state carries after collision,
// so the first K1 already points along -grad phi for any tau_phi.
// The moving populations are computed in FP32, directly as deviations from the storage's
// reference levels (the values are stored in FP32 or 16 bits anyway; GB300's FP64 rate made the
// FP64 version of this kernel a millisecond at 128^3). Plane 0 takes the zeroth moments from
// their closed forms in FP64: sum_i f*_i = p / cs^2 (sum_i t_i gam_i = 0 and the Pi_s term has no
// trace over the velocity set) and sum_i g*_i = phi0 (the first moments of t_i e_i vanish).
// ---------------------------------------------------------------------------------------
template <int Q, int S>
__global__ void init_kernel(const Params P, int z0, const double* __restrict__ phi0s,
                            const double* __restrict__ u0s, const double* __restrict__ ps, double p0,
                            void* __restrict__ fg) {
    const int x = blockIdx.x * kAuxBX + threadIdx.x;
    const int y = blockIdx.y * kAuxBY + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int nzs = gridDim.z;
    const int ls = (zl + 1) * P.nxy + y * P.nx + x;  // this cell in the staged phi0 slab
    const double phid = phi0s[ls];
    const float phi = (float)phid;

    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        int xx = x + Lat<Q>::cx(i), yy = y + Lat<Q>::cy(i);
        // across a wall: the mirror image of this cell (zero normal gradient); else periodic
        xx = (P.walls & 1) ? min(max(xx, 0), P.nx - 1) : (xx + P.nx) % P.nx;
        yy = (P.walls & 2) ? min(max(yy, 0), P.ny - 1) : (yy + P.ny) % P.ny;
        const int ll = (zl + 1 + Lat<Q>::cz(i)) * P.nxy + yy * P.nx + xx;
        const float v = Lat<Q>::w(i) * (float)phi0s[ll];
        gx += Lat<Q>::cx(i) * v;
        gy += Lat<Q>::cy(i) * v;
        gz += Lat<Q>::cz(i) * v;
    }
    gx *= 3.f;
    gy *= 3.f;
    gz *= 3.f;
    const float g2 = gx * gx + gy * gy + gz * gz;
    const float gn = sqrtf(g2);
    const float inv = (g2 > kNormalGuard) ? 1.0f / gn : 0.f;
    const float n[3] = {gx * inv, gy * inv, gz * inv};
    const float smag = P.four_over_delta * phi * (1.f - phi);
    const float Sv[3] = {smag * n[0], smag * n[1], smag * n[2]};
    const float rho = P.rho2 + P.drho * phi;
    const size_t slab = (size_t)nzs * P.nxy;
    const int lu = zl * P.nxy + y * P.nx + x;
    const float u[3] = {u0s ? (float)u0s[lu] : 0.f, u0s ? (float)u0s[slab + lu] : 0.f, u0s ? (float)u0s[2 * slab + lu] : 0.f};
    const double pc = ps ? ps[lu] : p0;
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float sg = P.sigma * gn;
    const float trc3 = ((float)Lat<Q>::D - (n[0] * n[0] + n[1] * n[1] + n[2] * n[2])) * (1.0f / 3.0f);
    const float dP = (float)(3.0 * pc - P.w0d);     // p / cs^2 - w0
    const float Phi = (float)(phid - P.phi_ref_d);  // phi - phi_ref
    const float tnq = P.tau_phi - 0.5f;

    const size_t c = (size_t)(z0 + zl) * P.nxy + (size_t)y * P.nx + x;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float t = Lat<Q>::w(i);
        const float eu = Lat<Q>::cx(i) * u[0] + Lat<Q>::cy(i) * u[1] + Lat<Q>::cz(i) * u[2];
        const float en = Lat<Q>::cx(i) * n[0] + Lat<Q>::cy(i) * n[1] + Lat<Q>::cz(i) * n[2];
        const float es = Lat<Q>::cx(i) * Sv[0] + Lat<Q>::cy(i) * Sv[1] + Lat<Q>::cz(i) * Sv[2];
        const float eg = Lat<Q>::cx(i) * gx + Lat<Q>::cy(i) * gy + Lat<Q>::cz(i) * gz;
        const float gam = 3.f * eu + 4.5f * eu * eu - 1.5f * u2;
        const float pis = sg * ((float)Lat<Q>::e2(i) - en * en - trc3);
        const float fdev = t * (dP + rho * gam - 4.5f * pis);                       // f*_i - t_i w0
        const float gdev = t * (Phi + phi * gam + P.tau_phi * es) - t * tnq * eg;  // g*_i - t_i phi_ref
        Store<S>::store(pop_ptr<Q, S>(fg, P.N, i, c), fdev, gdev, P);
    }
    // plane 0: the zeroth moments sum f - w0 = p / cs^2 - w0 (FP32) and phi as the integer phi * 2^30
    moment_plane(fg)[c] = make_float2((float)(3.0 * pc - P.w0d), __int_as_float((int)llrint(phid * kPhiFx)));
}

cudaError_t launch_init(const Params& P, int z0, int nzs, const double* phi0s, const double* u0s,
                        const double* ps, double p0, void* fg, cudaStream_t s) {
    const dim3 grid((P.nx + kAuxBX - 1) / kAuxBX, (P.ny + kAuxBY - 1) / kAuxBY, nzs), block(kAuxBX, kAuxBY);
#define LBM_INIT(Q, S) init_kernel<Q, S><<<grid, block, 0, s>>>(P, z0, phi0s, u0s, ps, p0, fg)
    if (P.Q == 9) {
        if (P.storage == STORE_F16) LBM_INIT(9, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_INIT(9, STORE_BF16);
        else LBM_INIT(9, STORE_F32);
    } else {
        if (P.storage == STORE_F16) LBM_INIT(19, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_INIT(19, STORE_BF16);
        else LBM_INIT(19, STORE_F32);
    }
#undef LBM_INIT
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Fields of the propagated current state (the values the next step collides with), each as FP64
// planes of the slab at its own destination (FieldOut): phi, p, u(3), grad phi(3), n(3).
// ---------------------------------------------------------------------------------------
// The macroscopic fields of cell (x, y, z) of the propagated state, as the next step's
// collision sees them; the fixed-point phi in phi_fx.
template <int Q, int SCHEME, bool GEN, int S>
__device__ __forceinline__ void cell_fields(const Params& P, const void* __restrict__ fg, const float* __restrict__ phi_fd,
                                            int x, int y, int z, Macro& m, int& phi_fx) {
    const Nbr nb = make_nbr(P, x, y, z);
    const int c = (z * P.ny + y) * P.nx + x;
    const WallSide ws = GEN ? make_wall_side(P, x, y, z) : WallSide{};
    float fb[Q], gb[Q];
    pull<Q, true, S, GEN>(P, fg, c, nb, fb, gb, phi_fx, ws);
    macro_flow<Q, GEN>(P, fb, gb, m);
    if (SCHEME == SCHEME_DF) {
        macro_interface_df<Q>(P, m);
    } else {
        float gx, gy, gz;
        fd_gradient<Q>(phi_fd, c, GEN ? mirror_at_walls(nb, ws) : nb, gx, gy, gz);
        macro_interface_fd(P, gx, gy, gz, m);
    }
    macro_pressure<GEN>(P, m);
}

template <int Q, int SCHEME, bool GEN, int S>
__global__ void moments_kernel(const Params P, int z0, const void* __restrict__ fg,
                               const float* __restrict__ phi_fd, int mask, const FieldOut out) {
    const int x = blockIdx.x * kAuxBX + threadIdx.x;
    const int y = blockIdx.y * kAuxBY + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int z = z0 + zl;
    Macro m;
    int phi_fx;
    cell_fields<Q, SCHEME, GEN, S>(P, fg, phi_fd, x, y, z, m, phi_fx);
    const size_t l = (size_t)zl * P.nxy + (size_t)y * P.nx + x;
    if (mask & 1) out.p[0][l] = (double)phi_fx / kPhiFx;
    if (mask & 2) out.p[1][l] = (P.w0d + (double)m.P) / 3.0;  // p = cs^2 (w0 + P)
    for (int a = 0; a < 3; ++a) {
        if (mask & 4) out.p[2 + a][l] = (double)m.u[a];
        if (mask & 8) out.p[5 + a][l] = (double)m.gphi[a];
        if (mask & 16) out.p[8 + a][l] = (double)m.n[a];
    }
}

template <int Q, int SCHEME, int S>
static void moments_qs(const Params& P, int z0, int nzs, const void* fg, const float* phi, int mask,
                       const FieldOut& out, cudaStream_t s) {
    const dim3 grid((P.nx + kAuxBX - 1) / kAuxBX, (P.ny + kAuxBY - 1) / kAuxBY, nzs), block(kAuxBX, kAuxBY);
    if (P.general) moments_kernel<Q, SCHEME, true, S><<<grid, block, 0, s>>>(P, z0, fg, phi, mask, out);
    else moments_kernel<Q, SCHEME, false, S><<<grid, block, 0, s>>>(P, z0, fg, phi, mask, out);
}

template <int Q, int SCHEME>
static void moments_q(const Params& P, int z0, int nzs, const void* fg, const float* phi, int mask,
                      const FieldOut& out, cudaStream_t s) {
    if (P.storage == STORE_F16) moments_qs<Q, SCHEME, STORE_F16>(P, z0, nzs, fg, phi, mask, out, s);
    else if (P.storage == STORE_BF16) moments_qs<Q, SCHEME, STORE_BF16>(P, z0, nzs, fg, phi, mask, out, s);
    else moments_qs<Q, SCHEME, STORE_F32>(P, z0, nzs, fg, phi, mask, out, s);
}

cudaError_t launch_moments(const Params& P, int scheme, int z0, int nzs, const void* fg, const float* phi_fd,
                           int mask, const FieldOut& out, cudaStream_t s) {
    if (P.Q == 9) {
        if (scheme == SCHEME_DF) moments_q<9, SCHEME_DF>(P, z0, nzs, fg, phi_fd, mask, out, s);
        else moments_q<9, SCHEME_FD>(P, z0, nzs, fg, phi_fd, mask, out, s);
    } else {
        if (scheme == SCHEME_DF) moments_q<19, SCHEME_DF>(P, z0, nzs, fg, phi_fd, mask, out, s);
        else moments_q<19, SCHEME_FD>(P, z0, nzs, fg, phi_fd, mask, out, s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Mass: sum phi and sum rho phi over the propagated state, plus a count of non-finite stored
// populations. sum phi is the exact integer sum of the fixed-point phi values (64-bit), so it
// reports conservation bit for bit; the other two accumulate in FP64. Grid-stride per thread,
// warp shuffle, shared memory per block, one partial triple per block (the integer held in the
// bits of the first double); a single block then sums the partials in a fixed order.
// ---------------------------------------------------------------------------------------
constexpr int kRedThreads = 256;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block totals of s and v[0..1]; valid in thread 0.
__device__ __forceinline__ void block_sum(long long& s, double (&v)[2]) {
    __shared__ long long rs[kRedThreads / 32];
    __shared__ double rv[2][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s = warp_sum(s);
    v[0] = warp_sum(v[0]);
    v[1] = warp_sum(v[1]);
    if (lane == 0) {
        rs[warp] = s;
        rv[0][warp] = v[0];
        rv[1][warp] = v[1];
    }
    __syncthreads();
    if (warp == 0) {
        const bool in = lane < kRedThreads / 32;
        s = warp_sum(in ? rs[lane] : 0ll);
        v[0] = warp_sum(in ? rv[0][lane] : 0.0);
        v[1] = warp_sum(in ? rv[1][lane] : 0.0);
    }
}

template <int Q, int S>
__global__ void __launch_bounds__(kRedThreads)
mass_kernel(const Params P, const void* __restrict__ fg, double* __restrict__ partials) {
    long long phi_sum = 0, bad_sum = 0;
    double acc[2] = {0.0, 0.0};
    // sum rho phi = rho2 sum phi + drho sum phi^2: sum phi is the exact integer sum, and only the
    // squares of the fixed-point values are summed in FP64 (GB300 issues FP64 at a small fraction
    // of its FP32 rate); mass_finish scales them by 2^-60
    for (long long c = (long long)blockIdx.x * kRedThreads + threadIdx.x; c < P.N;
         c += (long long)gridDim.x * kRedThreads) {
        const int z = (int)(c / P.nxy);
        const int r = (int)(c - (long long)z * P.nxy);
        const int y = r / P.nx, x = r - y * P.nx;
        const Nbr nb = make_nbr(P, x, y, z);
        float fb[Q], gb[Q];
        int phi_fx;
        pull<Q, false, S, true>(P, fg, (int)c, nb, fb, gb, phi_fx, make_wall_side(P, x, y, z));
        const double q = (double)phi_fx;
        phi_sum += phi_fx;
        acc[0] += q * q;
        int bad = 0;
        const float2 m0 = __ldg(moment_plane(fg) + c);
        bad += !isfinite(m0.x);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float2 v = Store<S>::load(pop_ptr<Q, S>(fg, P.N, i, c), P);
            bad += !isfinite(v.x) + !isfinite(v.y);
        }
        bad_sum += bad;
    }
    acc[1] = (double)bad_sum;
    block_sum(phi_sum, acc);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = __longlong_as_double(phi_sum);
        partials[3 * blockIdx.x + 1] = acc[0];
        partials[3 * blockIdx.x + 2] = acc[1];
    }
}

__global__ void __launch_bounds__(kRedThreads)
mass_finish(const double* __restrict__ partials, int n, double rho2, double drho, double* __restrict__ result) {
    long long phi_sum = 0;
    double acc[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < n; b += kRedThreads) {
        phi_sum += __double_as_longlong(partials[3 * b]);
        acc[0] += partials[3 * b + 1];
        acc[1] += partials[3 * b + 2];
    }
    block_sum(phi_sum, acc);
    if (threadIdx.x == 0) {
        result[0] = (double)phi_sum / kPhiFx;
        result[1] = rho2 * result[0] + drho * (acc[0] / (kPhiFx * kPhiFx));
        result[2] = acc[1];
        result[3] = __longlong_as_double(phi_sum);  // the exact integer sum, bit for bit
    }
}

// The exact sum of the fixed-point phi values of plane 0. The propagation only moves phi across
// faces in integer amounts that cancel in pairs, so this equals the sum over the propagated
// state that launch_mass reports in result[3], without reading the moving populations.
__global__ void __launch_bounds__(kRedThreads)
phi_fixed_sum_kernel(const float2* __restrict__ plane0, long long N, double* __restrict__ partials) {
    long long s = 0;
    for (long long c = (long long)blockIdx.x * kRedThreads + threadIdx.x; c < N; c += (long long)gridDim.x * kRedThreads)
        s += __float_as_int(__ldg(plane0 + c).y);
    double unused[2] = {0.0, 0.0};
    block_sum(s, unused);
    if (threadIdx.x == 0) partials[3 * blockIdx.x] = __longlong_as_double(s);
}

__global__ void __launch_bounds__(kRedThreads)
phi_fixed_finish(const double* __restrict__ partials, int n, double* __restrict__ result) {
    long long s = 0;
    for (int b = threadIdx.x; b < n; b += kRedThreads) s += __double_as_longlong(partials[3 * b]);
    double unused[2] = {0.0, 0.0};
    block_sum(s, unused);
    if (threadIdx.x == 0) result[3] = __longlong_as_double(s);
}

cudaError_t launch_phi_fixed_sum(const Params& P, const void* fg, double* partials, int n_partials, double* result,
                                 cudaStream_t s) {
    phi_fixed_sum_kernel<<<n_partials, kRedThreads, 0, s>>>(moment_plane(fg), P.N, partials);
    phi_fixed_finish<<<1, kRedThreads, 0, s>>>(partials, n_partials, result);
    return cudaGetLastError();
}

// Validation of host input staged on the device: per block, the number of values outside
// [lo, hi] ((lo, hi] with open_low; NaN and infinities count as outside) and the sum of the
// values, in partials[2 b], partials[2 b + 1]. Each block sums its grid-stride elements in a
// fixed order and the tree of block_sum is fixed, so the partials are the same bits on every run.
__global__ void __launch_bounds__(kRedThreads)
check_values_kernel(const double* __restrict__ v, long long n, double lo, double hi, int open_low,
                    double* __restrict__ partials) {
    long long unused = 0;
    double acc[2] = {0.0, 0.0};
    for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kRedThreads) {
        const double x = v[i];
        const bool ok = (open_low ? (x > lo) : (x >= lo)) && x <= hi && isfinite(x);
        acc[0] += ok ? 0.0 : 1.0;
        acc[1] += x;
    }
    block_sum(unused, acc);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = acc[0];
        partials[2 * blockIdx.x + 1] = acc[1];
    }
}

cudaError_t launch_check_values(const double* v, long long n, double lo, double hi, int open_low, double* partials,
                                int n_blocks, cudaStream_t s) {
    check_values_kernel<<<n_blocks, kRedThreads, 0, s>>>(v, n, lo, hi, open_low, partials);
    return cudaGetLastError();
}

int mass_partials_needed(const Params& P) {
    const long long blocks = (P.N + kRedThreads - 1) / kRedThreads;
    return (int)(blocks < 1024 ? blocks : 1024);
}

cudaError_t launch_mass(const Params& P, const void* fg, double* partials, int n_partials, double* result,
                        cudaStream_t s) {
#define LBM_MASS(Q, S) mass_kernel<Q, S><<<n_partials, kRedThreads, 0, s>>>(P, fg, partials)
    if (P.Q == 9) {
        if (P.storage == STORE_F16) LBM_MASS(9, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_MASS(9, STORE_BF16);
        else LBM_MASS(9, STORE_F32);
    } else {
        if (P.storage == STORE_F16) LBM_MASS(19, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_MASS(19, STORE_BF16);
        else LBM_MASS(19, STORE_F32);
    }
#undef LBM_MASS
    mass_finish<<<1, kRedThreads, 0, s>>>(partials, n_partials, P.rho2_d, P.drho_d, result);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Diagnostics (lbm_diagnostics): the largest u^2 and its cell, the kinetic energy and the mean
// pressure inside and outside a sphere, from the same per-cell fields lbm_moments returns, in
// FP64 with every product and sum rounded once (no contraction), so that a host evaluation of
// the same definitions on lbm_moments' output gives the same maximum and cell. Each thread takes
// a grid-stride set of cells in a fixed order, a block combines its threads with warp shuffles
// and shared memory in a fixed tree, and one block combines the per-block partials in order:
// the same bits on every run.
// ---------------------------------------------------------------------------------------
struct DiagAcc {
    double s2;      // the largest u^2 so far
    long long arg;  // its cell (the smallest index among equal values)
    double kin, pin, pout;
    long long nin, nout;
};

__device__ __forceinline__ void diag_merge(DiagAcc& a, const DiagAcc& b) {
    if (b.s2 > a.s2 || (b.s2 == a.s2 && b.arg < a.arg)) {
        a.s2 = b.s2;
        a.arg = b.arg;
    }
    a.kin += b.kin;
    a.pin += b.pin;
    a.pout += b.pout;
    a.nin += b.nin;
    a.nout += b.nout;
}

__device__ __forceinline__ DiagAcc diag_shfl_down(const DiagAcc& a, int o) {
    DiagAcc b;
    b.s2 = __shfl_down_sync(0xffffffffu, a.s2, o);
    b.arg = __shfl_down_sync(0xffffffffu, a.arg, o);
    b.kin = __shfl_down_sync(0xffffffffu, a.kin, o);
    b.pin = __shfl_down_sync(0xffffffffu, a.pin, o);
    b.pout = __shfl_down_sync(0xffffffffu, a.pout, o);
    b.nin = __shfl_down_sync(0xffffffffu, a.nin, o);
    b.nout = __shfl_down_sync(0xffffffffu, a.nout, o);
    return b;
}

// Block total of a, valid in thread 0.
__device__ __forceinline__ void diag_block(DiagAcc& a) {
    __shared__ DiagAcc rs[kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DiagAcc b = diag_shfl_down(a, o);
        diag_merge(a, b);
    }
    if (lane == 0) rs[warp] = a;
    __syncthreads();
    if (warp == 0) {
        a = lane < kRedThreads / 32 ? rs[lane] : DiagAcc{-1.0, -1, 0.0, 0.0, 0.0, 0, 0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DiagAcc b = diag_shfl_down(a, o);
            diag_merge(a, b);
        }
    }
}

// r_in, r_out, and the squared distance along each axis per coordinate (d2x, d2y, d2z; the
// host evaluates them in FP64 with the operations of the definition), FP64 and FP32 copies.
struct DiagArgs {
    double r_in, r_out;
    float in2_lo, in2_hi, out2_lo, out2_hi;  // FP32 bands around r^2 outside which FP32 decides
    const double* d2x;
    const double* d2y;
    const double* d2z;
    const float* f2x;
    const float* f2y;
    const float* f2z;
};

// GB300 issues FP64 instructions at a small fraction of its FP32 rate, so the per-cell work is
// FP32 and FP64 is taken only where the result needs it:
//  * the largest u^2: each cell's FP32 estimate (within 4e-7 relative of the FP64 value) is
//    compared with the thread's best so far; the warp takes the FP64 path only if one of its
//    lanes may reach it, which after a thread's first cell is rare;
//  * the sphere masks: FP32 decides outside a band of 1e-5 relative around r^2; a cell inside
//    the band takes the FP64 distance and the correctly rounded square root;
//  * the energy and pressure sums: FP32 per cell and over runs of 8 of a thread's cells, each run
//    then added to FP64 sums (one FP64 add per 8 cells whatever the grid size).
template <int Q, int SCHEME, bool GEN, int S>
__global__ void __launch_bounds__(kRedThreads, 2)
diag_kernel(const Params P, const void* __restrict__ fg, const float* __restrict__ phi_fd, const DiagArgs A,
            DiagAcc* __restrict__ partials) {
    double best = -1.0;  // FP64 u^2 of the thread's best cell
    long long arg = -1;
    float best_lo = -1.0f;  // FP32 threshold a cell's estimate must reach to be a candidate
    float kin = 0.f, pin = 0.f, pout = 0.f;        // the current run of 8 cells
    double kin_d = 0.0, pin_d = 0.0, pout_d = 0.0;  // the finished runs
    long long nin = 0, nout = 0;
    const unsigned lane_mask = 0xffffffffu;
    int run = 0;  // the same in every thread of the block: the loop bounds are block-uniform
    for (long long base = (long long)blockIdx.x * kRedThreads; base < P.N; base += (long long)gridDim.x * kRedThreads) {
        const long long c = base + threadIdx.x;
        const bool valid = c < P.N;
        float s2f = -1.0f;
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (valid) {
            const int z = (int)(c / P.nxy);
            const int r = (int)(c - (long long)z * P.nxy);
            const int y = r / P.nx, x = r - y * P.nx;
            Macro m;
            int phi_fx;
            cell_fields<Q, SCHEME, GEN, S>(P, fg, phi_fd, x, y, z, m, phi_fx);
            ux = m.u[0];
            uy = m.u[1];
            uz = m.u[2];
            s2f = __fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(uz, uz));
            kin = __fadd_rn(kin, __fmul_rn(__fmul_rn(0.5f, m.rho), s2f));
            const float d2f = __fadd_rn(__fadd_rn(__ldg(A.f2x + x), __ldg(A.f2y + y)), __ldg(A.f2z + z));
            const bool near_in = d2f >= A.in2_lo && d2f <= A.in2_hi;
            const bool near_out = d2f >= A.out2_lo && d2f <= A.out2_hi;
            bool inside = d2f < A.in2_lo, outside = d2f > A.out2_hi;
            if (near_in || near_out) {  // FP64, as the definition evaluates it
                const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__ldg(A.d2x + x), __ldg(A.d2y + y)), __ldg(A.d2z + z)));
                if (near_in) inside = d < A.r_in;
                if (near_out) outside = d > A.r_out;
            }
            if (inside) {
                pin = __fadd_rn(pin, m.P);
                nin += 1;
            }
            if (outside) {
                pout = __fadd_rn(pout, m.P);
                nout += 1;
            }
        }
        const bool cand = valid && s2f >= best_lo;
        if (__any_sync(lane_mask, cand)) {
            if (cand) {
                const double dx = ux, dy = uy, dz = uz;
                const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (s2 > best) {  // a thread's cells come in increasing order: the first of equal values stays
                    best = s2;
                    arg = c;
                    // below 1e-30 the FP32 squares lose precision to underflow: every cell stays a candidate
                    best_lo = best < 1e-30 ? 0.0f : __double2float_rd(best * (1.0 - 1e-6));
                }
            }
        }
        if (++run == 8) {
            kin_d += (double)kin;
            pin_d += (double)pin;
            pout_d += (double)pout;
            kin = pin = pout = 0.f;
            run = 0;
        }
    }
    DiagAcc a{best, arg, kin_d + (double)kin, pin_d + (double)pin, pout_d + (double)pout, nin, nout};
    diag_block(a);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

// result: max |u|, its cell (as double bits of the integer), kinetic, p_in, p_out, n_in, n_out
// (doubles of the counts)
__global__ void __launch_bounds__(kRedThreads)
diag_finish(const DiagAcc* __restrict__ partials, int n, double w0, double* __restrict__ result) {
    DiagAcc a{-1.0, -1, 0.0, 0.0, 0.0, 0, 0};
    for (int b = threadIdx.x; b < n; b += kRedThreads) diag_merge(a, partials[b]);
    diag_block(a);
    if (threadIdx.x == 0) {
        result[0] = __dsqrt_rn(a.s2);
        result[1] = __longlong_as_double(a.arg);
        result[2] = a.kin;
        result[3] = a.nin ? (w0 + a.pin / (double)a.nin) / 3.0 : __longlong_as_double(0x7ff8000000000000ll);
        result[4] = a.nout ? (w0 + a.pout / (double)a.nout) / 3.0 : __longlong_as_double(0x7ff8000000000000ll);
        result[5] = (double)a.nin;
        result[6] = (double)a.nout;
    }
}

size_t diag_partial_bytes(int n_blocks) { return (size_t)n_blocks * sizeof(DiagAcc); }

template <int Q, int SCHEME, int S>
static void diag_qs(const Params& P, const void* fg, const float* phi_fd, const DiagArgs& A, DiagAcc* part, int nb,
                    cudaStream_t s) {
    if (P.general) diag_kernel<Q, SCHEME, true, S><<<nb, kRedThreads, 0, s>>>(P, fg, phi_fd, A, part);
    else diag_kernel<Q, SCHEME, false, S><<<nb, kRedThreads, 0, s>>>(P, fg, phi_fd, A, part);
}

template <int Q, int SCHEME>
static void diag_q(const Params& P, const void* fg, const float* phi_fd, const DiagArgs& A, DiagAcc* part, int nb,
                   cudaStream_t s) {
    if (P.storage == STORE_F16) diag_qs<Q, SCHEME, STORE_F16>(P, fg, phi_fd, A, part, nb, s);
    else if (P.storage == STORE_BF16) diag_qs<Q, SCHEME, STORE_BF16>(P, fg, phi_fd, A, part, nb, s);
    else diag_qs<Q, SCHEME, STORE_F32>(P, fg, phi_fd, A, part, nb, s);
}

double axis_d2_host(int i, double c, int n, bool wall) {
    if (n == 1) return 0.0;
    double d = std::fabs((double)i - c);
    if (!wall) {
        if (d >= (double)n) d = std::fmod(d, (double)n);
        d = std::fmin(d, (double)n - d);
    }
    return d * d;
}

cudaError_t launch_diagnostics(const Params& P, int scheme, const void* fg, const float* phi_fd, const double* d2_axes,
                               double r_in, double r_out, void* partials, int n_blocks, double* result, cudaStream_t s) {
    // bands of 1e-5 relative around r^2: far wider than the FP32 rounding of the axis terms and
    // their sum (outside, FP32 decides the comparison of the correctly rounded FP64 distance)
    auto band = [](double r, double& lo, double& hi) {
        const double r2 = r * r;
        lo = r > 0 ? r2 * (1.0 - 1e-5) : -1.0;
        hi = r > 0 ? r2 * (1.0 + 1e-5) : 0.0;
    };
    const int n_axes = P.nx + P.ny + P.nz;
    const float* f2 = reinterpret_cast<const float*>(d2_axes + n_axes);
    DiagArgs A{r_in, r_out, 0, 0, 0, 0, d2_axes, d2_axes + P.nx, d2_axes + P.nx + P.ny, f2, f2 + P.nx, f2 + P.nx + P.ny};
    double lo, hi;
    band(r_in, lo, hi);
    A.in2_lo = (float)lo;
    A.in2_hi = (float)hi;
    band(r_out, lo, hi);
    A.out2_lo = (float)lo;
    A.out2_hi = (float)hi;
    DiagAcc* part = static_cast<DiagAcc*>(partials);
    if (P.Q == 9) {
        if (scheme == SCHEME_DF) diag_q<9, SCHEME_DF>(P, fg, phi_fd, A, part, n_blocks, s);
        else diag_q<9, SCHEME_FD>(P, fg, phi_fd, A, part, n_blocks, s);
    } else {
        if (scheme == SCHEME_DF) diag_q<19, SCHEME_DF>(P, fg, phi_fd, A, part, n_blocks, s);
        else diag_q<19, SCHEME_FD>(P, fg, phi_fd, A, part, n_blocks, s);
    }
    diag_finish<<<1, kRedThreads, 0, s>>>(part, n_blocks, P.w0d, result);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Device storage <-> plain FP64 populations, all Q planes of a slab (staging [Q][nzs * nxy]).
// Plane i >= 1: v_i + t_i ref; plane 0: the rest population, the zeroth moment held in plane 0
// (w0 + v_0 for f, phi_fx / 2^30 for g) minus sum_{i>=1} of the set.
// Writing one set (f or g) re-encodes the other member of each stored pair unchanged: decoding
// and re-encoding a stored FP32, scaled FP16 or BF16 value returns the same bits.
// ---------------------------------------------------------------------------------------
template <int Q, int S>
__global__ void pops_to_f64(const Params P, const void* __restrict__ src, int is_f, int z0, int nzs,
                            double* __restrict__ dst) {
    const size_t n = (size_t)nzs * P.nxy, base = (size_t)z0 * P.nxy;
    const double ref = is_f ? P.w0d : P.phi_ref_d;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        const float2 m0 = moment_plane(src)[base + l];
        double rest = is_f ? ref + (double)m0.x : (double)__float_as_int(m0.y) / kPhiFx;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float2 p = Store<S>::load(pop_ptr<Q, S>(src, P.N, i, (long long)(base + l)), P);
            const double v = (double)(is_f ? p.x : p.y) + Lat<Q>::wd(i) * ref;
            dst[i * n + l] = v;
            rest -= v;
        }
        dst[l] = rest;
    }
}

template <int Q, int S>
__global__ void pops_from_f64(const Params P, const double* __restrict__ src, int is_f, int z0, int nzs,
                              void* __restrict__ dst) {
    const size_t n = (size_t)nzs * P.nxy, base = (size_t)z0 * P.nxy;
    const double ref = is_f ? P.w0d : P.phi_ref_d;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        double sum = src[l];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const double v = src[i * n + l];
            sum += v;
            typename Store<S>::T* slot = pop_ptr<Q, S>(dst, P.N, i, (long long)(base + l));
            float2 p = Store<S>::load(slot, P);
            const float w = (float)(v - Lat<Q>::wd(i) * ref);
            if (is_f) p.x = w;
            else p.y = w;
            Store<S>::store(slot, p.x, p.y, P);
        }
        float2* m0 = moment_plane(dst) + base + l;
        if (is_f) m0->x = (float)(sum - ref);
        else m0->y = __int_as_float((int)llrint(sum * kPhiFx));  // |sum| < 2 checked by the host
    }
}

static unsigned conv_blocks(const Params& P, int nzs) {
    const size_t n = (size_t)nzs * P.nxy;
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? b : 4096);
}

#define LBM_DISPATCH_QS(KERNEL, ...)                                                       \
    do {                                                                                   \
        const unsigned nb_ = conv_blocks(P, nzs);                                          \
        if (P.Q == 9) {                                                                    \
            if (P.storage == STORE_F16) KERNEL<9, STORE_F16><<<nb_, 256, 0, s>>>(__VA_ARGS__);   \
            else if (P.storage == STORE_BF16) KERNEL<9, STORE_BF16><<<nb_, 256, 0, s>>>(__VA_ARGS__); \
            else KERNEL<9, STORE_F32><<<nb_, 256, 0, s>>>(__VA_ARGS__);                    \
        } else {                                                                           \
            if (P.storage == STORE_F16) KERNEL<19, STORE_F16><<<nb_, 256, 0, s>>>(__VA_ARGS__);  \
            else if (P.storage == STORE_BF16) KERNEL<19, STORE_BF16><<<nb_, 256, 0, s>>>(__VA_ARGS__); \
            else KERNEL<19, STORE_F32><<<nb_, 256, 0, s>>>(__VA_ARGS__);                   \
        }                                                                                  \
    } while (0)

cudaError_t launch_pops_to_f64(const Params& P, const void* src, int is_f, int z0, int nzs, double* dst,
                               cudaStream_t s) {
    LBM_DISPATCH_QS(pops_to_f64, P, src, is_f, z0, nzs, dst);
    return cudaGetLastError();
}

cudaError_t launch_pops_from_f64(const Params& P, const double* src, int is_f, int z0, int nzs, void* dst,
                                 cudaStream_t s) {
    LBM_DISPATCH_QS(pops_from_f64, P, src, is_f, z0, nzs, dst);
    return cudaGetLastError();
}
#undef LBM_DISPATCH_QS

}  // namespace lbm
