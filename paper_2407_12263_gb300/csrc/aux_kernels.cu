// aux_kernels.cu -- initialisation, field output, FP64 mass reduction and population
// conversion for the difference-free conservative phase-field LBM (arXiv:2407.12263).
// None of these runs inside the time-step loop.
#include "cell.cuh"

namespace lbm {

constexpr int kAuxBX = 32, kAuxBY = 4;

// ---------------------------------------------------------------------------------------
// Initial post-collision populations (FP64 arithmetic, stored FP32):
//   grad phi0 = 3 sum_{i != 0} t_i e_i phi0(x + e_i)   (isotropic central difference)
//   n0 = grad phi0 / |grad phi0|, S0 = 4 phi0 (1 - phi0) / delta n0, rho0 = rho2 + drho phi0
//   f*_i = f^eq_i(p0, u0, rho0, Pi_s0)                                   (Eq. geq_s)
//   g*_i = g^eq_i(phi0, u0, S0) - t_i (tau_phi - 1/2) e_i . grad phi0     (Eq. geq)
// The g term is the first-order non-equilibrium part a relaxed state carries after collision,
// so the first K1 already points along -grad phi for any tau_phi.
// ---------------------------------------------------------------------------------------
template <int Q, int S>
__global__ void init_kernel(const Params P, int z0, const double* __restrict__ phi0s,
                            const double* __restrict__ u0s, double p0, void* __restrict__ fg) {
    const int x = blockIdx.x * kAuxBX + threadIdx.x;
    const int y = blockIdx.y * kAuxBY + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int nzs = gridDim.z;
    const int ls = (zl + 1) * P.nxy + y * P.nx + x;  // this cell in the staged phi0 slab
    const double phi = phi0s[ls];

    double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int xx = (x + Lat<Q>::cx(i) + P.nx) % P.nx;
        const int yy = (y + Lat<Q>::cy(i) + P.ny) % P.ny;
        const int ll = (zl + 1 + Lat<Q>::cz(i)) * P.nxy + yy * P.nx + xx;
        const double v = Lat<Q>::wd(i) * phi0s[ll];
        gx += Lat<Q>::cx(i) * v;
        gy += Lat<Q>::cy(i) * v;
        gz += Lat<Q>::cz(i) * v;
    }
    gx *= 3.0;
    gy *= 3.0;
    gz *= 3.0;
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double gn = sqrt(g2);
    const double inv = (g2 > 1e-24) ? 1.0 / gn : 0.0;
    const double n[3] = {gx * inv, gy * inv, gz * inv};
    const double smag = P.four_over_delta_d * phi * (1.0 - phi);
    const double Sv[3] = {smag * n[0], smag * n[1], smag * n[2]};
    const double rho = P.rho2_d + P.drho_d * phi;
    const size_t slab = (size_t)nzs * P.nxy;
    const int lu = zl * P.nxy + y * P.nx + x;
    const double u[3] = {u0s ? u0s[lu] : 0.0, u0s ? u0s[slab + lu] : 0.0, u0s ? u0s[2 * slab + lu] : 0.0};
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double sg = P.sigma_d * gn;
    const double trc = (double)Lat<Q>::D - (n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);

    const size_t c = (size_t)(z0 + zl) * P.nxy + (size_t)y * P.nx + x;
    double fsum = 0.0, gsum = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double t = Lat<Q>::wd(i);
        const double eu = Lat<Q>::cx(i) * u[0] + Lat<Q>::cy(i) * u[1] + Lat<Q>::cz(i) * u[2];
        const double en = Lat<Q>::cx(i) * n[0] + Lat<Q>::cy(i) * n[1] + Lat<Q>::cz(i) * n[2];
        const double es = Lat<Q>::cx(i) * Sv[0] + Lat<Q>::cy(i) * Sv[1] + Lat<Q>::cz(i) * Sv[2];
        const double eg = Lat<Q>::cx(i) * gx + Lat<Q>::cy(i) * gy + Lat<Q>::cz(i) * gz;
        const double gam = 3.0 * eu + 4.5 * eu * eu - 1.5 * u2;
        const double pis = sg * ((double)Lat<Q>::e2(i) - en * en - trc / 3.0);
        const double fstar = t * (3.0 * p0 + rho * gam - 4.5 * pis);
        const double gstar = t * (phi * (1.0 + gam) + P.tau_phi_d * es) - t * (P.tau_phi_d - 0.5) * eg;
        fsum += fstar;
        gsum += gstar;
        if (i > 0)
            Store<S>::store(moving_plane<S>(fg, P.N, i) + c, (float)(fstar - t * P.w0d), (float)(gstar - t * P.phi_ref_d), P);
    }
    moment_plane(fg)[c] = make_float2((float)(fsum - P.w0d), (float)(gsum - P.phi_ref_d));  // plane 0: zeroth moments
}

cudaError_t launch_init(const Params& P, int z0, int nzs, const double* phi0s, const double* u0s,
                        double p0, void* fg, cudaStream_t s) {
    const dim3 grid((P.nx + kAuxBX - 1) / kAuxBX, (P.ny + kAuxBY - 1) / kAuxBY, nzs), block(kAuxBX, kAuxBY);
#define LBM_INIT(Q, S) init_kernel<Q, S><<<grid, block, 0, s>>>(P, z0, phi0s, u0s, p0, fg)
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
// Fields of the propagated current state (the values the next step collides with).
// Output slab layout: 11 FP64 planes of nzs * nxy values: phi, p, u(3), grad phi(3), n(3).
// ---------------------------------------------------------------------------------------
template <int Q, int SCHEME, bool GEN, int S>
__global__ void moments_kernel(const Params P, int z0, const void* __restrict__ fg,
                               const float* __restrict__ phi_fd, int mask, double* __restrict__ out) {
    const int x = blockIdx.x * kAuxBX + threadIdx.x;
    const int y = blockIdx.y * kAuxBY + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int z = z0 + zl;
    const Nbr nb = make_nbr(P, x, y, z);
    const int c = (z * P.ny + y) * P.nx + x;
    float fb[Q], gb[Q];
    pull<Q, true, S>(P, fg, c, nb, fb, gb);
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
    const size_t slab = (size_t)gridDim.z * P.nxy;
    const size_t l = (size_t)zl * P.nxy + (size_t)y * P.nx + x;
    if (mask & 1) out[l] = P.phi_ref_d + (double)m.Phi;
    if (mask & 2) out[slab + l] = (P.w0d + (double)m.P) / 3.0;  // p = cs^2 (w0 + P)
    for (int a = 0; a < 3; ++a) {
        if (mask & 4) out[(2 + a) * slab + l] = (double)m.u[a];
        if (mask & 8) out[(5 + a) * slab + l] = (double)m.gphi[a];
        if (mask & 16) out[(8 + a) * slab + l] = (double)m.n[a];
    }
}

template <int Q, int SCHEME, int S>
static void moments_qs(const Params& P, int z0, int nzs, const void* fg, const float* phi, int mask, double* out,
                       cudaStream_t s) {
    const dim3 grid((P.nx + kAuxBX - 1) / kAuxBX, (P.ny + kAuxBY - 1) / kAuxBY, nzs), block(kAuxBX, kAuxBY);
    if (P.general) moments_kernel<Q, SCHEME, true, S><<<grid, block, 0, s>>>(P, z0, fg, phi, mask, out);
    else moments_kernel<Q, SCHEME, false, S><<<grid, block, 0, s>>>(P, z0, fg, phi, mask, out);
}

template <int Q, int SCHEME>
static void moments_q(const Params& P, int z0, int nzs, const void* fg, const float* phi, int mask, double* out,
                      cudaStream_t s) {
    if (P.storage == STORE_F16) moments_qs<Q, SCHEME, STORE_F16>(P, z0, nzs, fg, phi, mask, out, s);
    else if (P.storage == STORE_BF16) moments_qs<Q, SCHEME, STORE_BF16>(P, z0, nzs, fg, phi, mask, out, s);
    else moments_qs<Q, SCHEME, STORE_F32>(P, z0, nzs, fg, phi, mask, out, s);
}

cudaError_t launch_moments(const Params& P, int scheme, int z0, int nzs, const void* fg, const float* phi_fd,
                           int mask, double* out, cudaStream_t s) {
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
// Mass: sum phi and sum rho phi over the propagated state, FP64 accumulation, plus a count of
// non-finite stored populations. Grid-stride per thread, warp shuffle, shared memory per block,
// one partial triple per block; a single block then sums the partials in a fixed order, so the
// result does not depend on scheduling.
// ---------------------------------------------------------------------------------------
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_sum3(double (&v)[3], double* out) {
    __shared__ double red[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = warp_sum(v[k]);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double w = (lane < kRedThreads / 32) ? red[k][lane] : 0.0;
            w = warp_sum(w);
            if (lane == 0) out[k] = w;
        }
    }
}

template <int Q, int S>
__global__ void __launch_bounds__(kRedThreads)
mass_kernel(const Params P, const void* __restrict__ fg, double* __restrict__ partials) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * kRedThreads + threadIdx.x; c < P.N;
         c += (long long)gridDim.x * kRedThreads) {
        const int z = (int)(c / P.nxy);
        const int r = (int)(c - (long long)z * P.nxy);
        const int y = r / P.nx, x = r - y * P.nx;
        const Nbr nb = make_nbr(P, x, y, z);
        float fb[Q], gb[Q];
        pull<Q, false, S>(P, fg, (int)c, nb, fb, gb);
        const double phi = P.phi_ref_d + (double)gb[0];
        acc[0] += phi;
        acc[1] += (P.rho2_d + P.drho_d * phi) * phi;
        int bad = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float2 v = (i == 0) ? __ldg(moment_plane(fg) + c) : Store<S>::load(moving_plane<S>(fg, P.N, i) + c, P);
            bad += !isfinite(v.x) + !isfinite(v.y);
        }
        acc[2] += (double)bad;
    }
    block_sum3(acc, partials + 3 * blockIdx.x);
}

__global__ void __launch_bounds__(kRedThreads)
mass_finish(const double* __restrict__ partials, int n, double* __restrict__ result) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < n; b += kRedThreads)
        for (int k = 0; k < 3; ++k) acc[k] += partials[3 * b + k];
    block_sum3(acc, result);
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
    mass_finish<<<1, kRedThreads, 0, s>>>(partials, n_partials, result);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Device storage <-> plain FP64 populations, all Q planes of a slab (staging [Q][nzs * nxy]).
// Plane i >= 1: v_i + t_i ref; plane 0: the rest population (ref + v_0) - sum_{i>=1} f_i.
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
        double rest = ref + (double)(is_f ? m0.x : m0.y);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float2 p = Store<S>::load(moving_plane<S>(src, P.N, i) + base + l, P);
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
            typename Store<S>::T* slot = moving_plane<S>(dst, P.N, i) + base + l;
            float2 p = Store<S>::load(slot, P);
            const float w = (float)(v - Lat<Q>::wd(i) * ref);
            if (is_f) p.x = w;
            else p.y = w;
            Store<S>::store(slot, p.x, p.y, P);
        }
        float2* m0 = moment_plane(dst) + base + l;
        if (is_f) m0->x = (float)(sum - ref);
        else m0->y = (float)(sum - ref);
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
