// surrogate_glue.cu -- field transfers between the lattice and the surrogate's coarse grid:
// block means of the macroscopic fields, the restart from trilinearly upsampled coarse fields
// (the same equilibrium-plus-non-equilibrium construction as the initial state, in FP32), and
// the exact correction of sum phi after a restart.
#include "cell.cuh"
#include "surrogate.h"

namespace lbm {

template <int Q, int S, bool GEN>
__global__ void coarsen_kernel(const Params P, const void* __restrict__ fg, int f, float* __restrict__ out) {
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    const int cz = blockIdx.z;
    const int ncx = P.nx / f, ncy = P.ny / f, ncz = P.nz / f;
    if (cx >= ncx || cy >= ncy) return;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int dz = 0; dz < f; ++dz)
        for (int dy = 0; dy < f; ++dy)
            for (int dx = 0; dx < f; ++dx) {
                const int x = cx * f + dx, y = cy * f + dy, z = cz * f + dz;
                const Nbr nb = make_nbr(P, x, y, z);
                const int c = (z * P.ny + y) * P.nx + x;
                const WallSide ws = GEN ? make_wall_side(P, x, y, z) : WallSide{};
                float fb[Q], gb[Q];
                int phi_fx;
                pull<Q, true, S, GEN>(P, fg, c, nb, fb, gb, phi_fx, ws);
                Macro m;
                macro_flow<Q, GEN>(P, fb, gb, m);
                macro_interface_df<Q>(P, m);
                macro_pressure<GEN>(P, m);
                acc[0] += (double)phi_fx / kPhiFx;
                acc[1] += m.u[0];
                acc[2] += m.u[1];
                acc[3] += m.u[2];
                acc[4] += (P.w0d + (double)m.P) / 3.0;
            }
    const double inv = 1.0 / ((double)f * f * f);
    const long long nc = (long long)ncx * ncy * ncz, l = ((long long)cz * ncy + cy) * ncx + cx;
    for (int k = 0; k < 5; ++k) out[k * nc + l] = (float)(acc[k] * inv);
}

// The same block means for factors f that divide 32: lane l of a warp takes fine x = 32 b + l,
// so a warp reads 32 consecutive cells of each plane, loops over the f x f rows of its coarse
// cells and sums across each aligned group of f lanes (one coarse cell) with shuffles.
template <int Q, int S, bool GEN>
__global__ void coarsen_lanes_kernel(const Params P, const void* __restrict__ fg, int f, float* __restrict__ out) {
    const int lane = threadIdx.x;
    const int x = blockIdx.x * 32 + lane;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    const int cz = blockIdx.z;
    const int ncx = P.nx / f, ncy = P.ny / f, ncz = P.nz / f;
    if (cy >= ncy) return;  // whole warps leave together
    const bool valid = x < P.nx;  // whole groups of f lanes are valid or not: f divides nx and 32
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (valid)
        for (int dz = 0; dz < f; ++dz)
            for (int dy = 0; dy < f; ++dy) {
                const int y = cy * f + dy, z = cz * f + dz;
                const Nbr nb = make_nbr(P, x, y, z);
                const int c = (z * P.ny + y) * P.nx + x;
                const WallSide ws = GEN ? make_wall_side(P, x, y, z) : WallSide{};
                float fb[Q], gb[Q];
                int phi_fx;
                pull<Q, true, S, GEN>(P, fg, c, nb, fb, gb, phi_fx, ws);
                Macro m;
                macro_flow<Q, GEN>(P, fb, gb, m);
                macro_interface_df<Q>(P, m);
                macro_pressure<GEN>(P, m);
                acc[0] += (double)phi_fx / kPhiFx;
                acc[1] += m.u[0];
                acc[2] += m.u[1];
                acc[3] += m.u[2];
                acc[4] += (P.w0d + (double)m.P) / 3.0;
            }
    for (int o = f >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (!valid || lane % f) return;
    const double inv = 1.0 / ((double)f * f * f);
    const long long nc = (long long)ncx * ncy * ncz, l = ((long long)cz * ncy + cy) * ncx + x / f;
    for (int k = 0; k < 5; ++k) out[k * nc + l] = (float)(acc[k] * inv);
}

cudaError_t launch_coarsen(const Params& P, const void* fg, int factor, float* out, cudaStream_t s) {
    const int ncx = P.nx / factor, ncy = P.ny / factor, ncz = P.nz / factor;
    if (factor <= 32 && 32 % factor == 0) {
        const dim3 block(32, 4), grid((P.nx + 31) / 32, (ncy + 3) / 4, ncz);
#define LBM_COARSEN_LANES(Q, S)                                                                   \
    (P.general ? (coarsen_lanes_kernel<Q, S, true><<<grid, block, 0, s>>>(P, fg, factor, out), 0) \
               : (coarsen_lanes_kernel<Q, S, false><<<grid, block, 0, s>>>(P, fg, factor, out), 0))
        if (P.Q == 9) {
            if (P.storage == STORE_F16) LBM_COARSEN_LANES(9, STORE_F16);
            else if (P.storage == STORE_BF16) LBM_COARSEN_LANES(9, STORE_BF16);
            else LBM_COARSEN_LANES(9, STORE_F32);
        } else {
            if (P.storage == STORE_F16) LBM_COARSEN_LANES(19, STORE_F16);
            else if (P.storage == STORE_BF16) LBM_COARSEN_LANES(19, STORE_BF16);
            else LBM_COARSEN_LANES(19, STORE_F32);
        }
#undef LBM_COARSEN_LANES
        return cudaGetLastError();
    }
    const dim3 block(32, 4), grid((ncx + 31) / 32, (ncy + 3) / 4, ncz);
#define LBM_COARSEN(Q, S)                                                                   \
    (P.general ? (coarsen_kernel<Q, S, true><<<grid, block, 0, s>>>(P, fg, factor, out), 0) \
               : (coarsen_kernel<Q, S, false><<<grid, block, 0, s>>>(P, fg, factor, out), 0))
    if (P.Q == 9) {
        if (P.storage == STORE_F16) LBM_COARSEN(9, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_COARSEN(9, STORE_BF16);
        else LBM_COARSEN(9, STORE_F32);
    } else {
        if (P.storage == STORE_F16) LBM_COARSEN(19, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_COARSEN(19, STORE_BF16);
        else LBM_COARSEN(19, STORE_F32);
    }
#undef LBM_COARSEN
    return cudaGetLastError();
}

// Block means over f^3 cells of the state's own phi, the fixed-point value of plane 0 (no
// propagation: 8 bytes read per cell). Lane l of a warp takes fine x = 32 b + l; f divides 32,
// and each aligned group of f lanes is summed with shuffles.
__global__ void coarse_phi_kernel(const float2* __restrict__ plane0, int nx, int ny, int nz, int f, float* __restrict__ out) {
    const int lane = threadIdx.x;
    const int x = blockIdx.x * 32 + lane;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    const int cz = blockIdx.z;
    const int ncx = nx / f, ncy = ny / f;
    if (cy >= ncy) return;  // whole warps leave together
    const bool valid = x < nx;
    long long acc = 0;
    if (valid)
        for (int dz = 0; dz < f; ++dz)
            for (int dy = 0; dy < f; ++dy)
                acc += __float_as_int(__ldg(plane0 + ((long long)(cz * f + dz) * ny + (cy * f + dy)) * nx + x).y);
    for (int o = f >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!valid || lane % f) return;
    out[((long long)cz * ncy + cy) * ncx + x / f] = (float)((double)acc / (kPhiFx * (double)f * f * f));
}

cudaError_t launch_coarse_phi(const Params& P, const void* fg, int factor, float* out, cudaStream_t s) {
    if (factor > 32 || 32 % factor) return cudaErrorInvalidValue;
    const dim3 block(32, 4), grid((P.nx + 31) / 32, (P.ny / factor + 3) / 4, P.nz / factor);
    coarse_phi_kernel<<<grid, block, 0, s>>>(moment_plane(fg), P.nx, P.ny, P.nz, factor, out);
    return cudaGetLastError();
}

// Where fine coordinate i (of n = nc f cells) falls between coarse cell centres: the two coarse
// indices and the weight of the second. Periodic, or clamped to the end centres across a wall.
struct Axis {
    int a, b;
    float t;
};

__device__ __forceinline__ Axis interp_axis(int i, int f, int nc, bool wall) {
    const float xc = ((float)i + 0.5f) / (float)f - 0.5f;
    Axis r;
    r.a = (int)floorf(xc);
    r.t = xc - (float)r.a;
    r.b = r.a + 1;
    if (wall) {
        if (r.a < 0) {
            r.a = 0;
            r.t = 0.f;
        }
        if (r.b > nc - 1) {
            r.b = nc - 1;
            if (r.a == r.b) r.t = 0.f;
        }
    } else {  // r.a is in [-1, nc - 1] and r.b = r.a + 1: one period at most on either side
        if (r.a < 0) r.a += nc;
        if (r.b >= nc) r.b -= nc;
    }
    return r;
}

// The offsets of the eight coarse corners around a fine cell (the coarse grid holds fewer than
// 2^31 cells), computed once for all the fields interpolated there.
struct Corners {
    int o[8];  // (z, y, x) in {a, b}^3, x fastest
    float tx, ty, tz;
};

__device__ __forceinline__ Corners corners(int ncx, int ncy, const Axis& X, const Axis& Y, const Axis& Z) {
    Corners c;
    const int za = Z.a * ncy, zb = Z.b * ncy;
    const int r00 = (za + Y.a) * ncx, r01 = (za + Y.b) * ncx, r10 = (zb + Y.a) * ncx, r11 = (zb + Y.b) * ncx;
    c.o[0] = r00 + X.a;
    c.o[1] = r00 + X.b;
    c.o[2] = r01 + X.a;
    c.o[3] = r01 + X.b;
    c.o[4] = r10 + X.a;
    c.o[5] = r10 + X.b;
    c.o[6] = r11 + X.a;
    c.o[7] = r11 + X.b;
    c.tx = X.t;
    c.ty = Y.t;
    c.tz = Z.t;
    return c;
}

// Trilinear interpolation of q at the corners: along x, then y, then z
__device__ __forceinline__ float trilinear(const float* __restrict__ q, const Corners& c) {
    auto lerp = [](float u, float v, float t) { return fmaf(t, v - u, u); };
    const float c00 = lerp(__ldg(q + c.o[0]), __ldg(q + c.o[1]), c.tx);
    const float c01 = lerp(__ldg(q + c.o[2]), __ldg(q + c.o[3]), c.tx);
    const float c10 = lerp(__ldg(q + c.o[4]), __ldg(q + c.o[5]), c.tx);
    const float c11 = lerp(__ldg(q + c.o[6]), __ldg(q + c.o[7]), c.tx);
    return lerp(lerp(c00, c01, c.ty), lerp(c10, c11, c.ty), c.tz);
}

// The initial-state construction of init_kernel (equilibria of the upsampled phi, u, p plus the
// first-order non-equilibrium part of g, grad phi from the isotropic central difference of the
// upsampled phi, which phi_fine_kernel writes first) in FP32, written directly as deviations
// from the storage's reference levels. phi is clamped to [-1, 1.5], the range lbm_init_fields
// accepts, so that its fixed-point value stays in range whatever the prediction holds.
// The upsampled phi of every cell (clamped as below), the first pass of the restart.
__global__ void phi_fine_kernel(const Params P, const float* __restrict__ coarse, int f, float* __restrict__ phi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int ncx = P.nx / f, ncy = P.ny / f, ncz = P.nz / f;
    const float v = trilinear(coarse, corners(ncx, ncy, interp_axis(x, f, ncx, P.walls & 1),
                                              interp_axis(y, f, ncy, P.walls & 2), interp_axis(z, f, ncz, P.walls & 4)));
    phi[((long long)z * P.ny + y) * P.nx + x] = fminf(fmaxf(v, -1.0f), 1.5f);
}

template <int Q, int S>
__global__ void restart_kernel(const Params P, const float* __restrict__ coarse, const float* __restrict__ phi_fine, int f,
                               float p0, void* __restrict__ fg) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int ncx = P.nx / f, ncy = P.ny / f, ncz = P.nz / f;
    const long long nc = (long long)ncx * ncy * ncz;
    // neighbour rows and columns: periodic images, or across a wall the cell itself (so that
    // the normal gradient vanishes there)
    int xs[3], ys[3], zs[3];
    // x + d lies in [-1, nx]: a periodic image is one period away at most
    auto wrap1 = [](int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); };
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        xs[d + 1] = (P.walls & 1) ? min(max(x + d, 0), P.nx - 1) : wrap1(x + d, P.nx);
        ys[d + 1] = (P.walls & 2) ? min(max(y + d, 0), P.ny - 1) : wrap1(y + d, P.ny);
        zs[d + 1] = (P.walls & 4) ? min(max(z + d, 0), P.nz - 1) : wrap1(z + d, P.nz);
    }
    auto phi_at = [&](int dx, int dy, int dz) {  // the grid holds fewer than 2^31 cells
        return __ldg(phi_fine + (zs[dz + 1] * P.ny + ys[dy + 1]) * P.nx + xs[dx + 1]);
    };
    const float phi = phi_at(0, 0, 0);
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float v = Lat<Q>::w(i) * phi_at(Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i));
        gx += Lat<Q>::cx(i) * v;
        gy += Lat<Q>::cy(i) * v;
        gz += Lat<Q>::cz(i) * v;
    }
    gx *= 3.f;
    gy *= 3.f;
    gz *= 3.f;
    const Corners cc = corners(ncx, ncy, interp_axis(x, f, ncx, P.walls & 1), interp_axis(y, f, ncy, P.walls & 2),
                               interp_axis(z, f, ncz, P.walls & 4));
    const float u[3] = {trilinear(coarse + nc, cc), trilinear(coarse + 2 * nc, cc), trilinear(coarse + 3 * nc, cc)};
    const float pc = trilinear(coarse + 4 * nc, cc);
    const float g2 = gx * gx + gy * gy + gz * gz;
    const float gn = sqrtf(g2);
    const float inv = (g2 > kNormalGuard) ? 1.0f / gn : 0.f;
    const float n[3] = {gx * inv, gy * inv, gz * inv};
    const float smag = P.four_over_delta * phi * (1.f - phi);
    const float Sv[3] = {smag * n[0], smag * n[1], smag * n[2]};
    const float rho = P.rho2 + P.drho * phi;
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float sg = P.sigma * gn;
    const float trc3 = ((float)Lat<Q>::D - (n[0] * n[0] + n[1] * n[1] + n[2] * n[2])) * (1.0f / 3.0f);
    const float dP = 3.f * (pc - p0);  // p / cs^2 - w0
    const float Phi = phi - P.phi_ref;
    const float tnq = P.tau_phi - 0.5f;
    const long long c = ((long long)z * P.ny + y) * P.nx + x;
    float fsum = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float t = Lat<Q>::w(i);
        const float eu = Lat<Q>::cx(i) * u[0] + Lat<Q>::cy(i) * u[1] + Lat<Q>::cz(i) * u[2];
        const float en = Lat<Q>::cx(i) * n[0] + Lat<Q>::cy(i) * n[1] + Lat<Q>::cz(i) * n[2];
        const float es = Lat<Q>::cx(i) * Sv[0] + Lat<Q>::cy(i) * Sv[1] + Lat<Q>::cz(i) * Sv[2];
        const float eg = Lat<Q>::cx(i) * gx + Lat<Q>::cy(i) * gy + Lat<Q>::cz(i) * gz;
        const float gam = 3.f * eu + 4.5f * eu * eu - 1.5f * u2;
        const float pis = sg * ((float)Lat<Q>::e2(i) - en * en - trc3);
        const float fdev = t * (dP + rho * gam - 4.5f * pis);                        // f*_i - t_i w0
        const float gdev = t * (Phi + phi * gam + P.tau_phi * es) - t * tnq * eg;  // g*_i - t_i phi_ref
        fsum += fdev;
        if (i > 0) Store<S>::store(pop_ptr<Q, S>(fg, P.N, i, c), fdev, gdev, P);
    }
    // plane 0: sum_i f*_i - w0, and phi (= sum_i g*_i) as the integer phi * 2^30
    moment_plane(fg)[c] = make_float2(fsum, __int_as_float(__float2int_rn(phi * 1073741824.0f)));
}

cudaError_t launch_restart(const Params& P, const float* coarse, int factor, double p0, float* phi_fine, void* fg,
                           cudaStream_t s) {
    const dim3 block(32, 4), grid((P.nx + 31) / 32, (P.ny + 3) / 4, P.nz);
    phi_fine_kernel<<<grid, block, 0, s>>>(P, coarse, factor, phi_fine);
#define LBM_RESTART(Q, S) restart_kernel<Q, S><<<grid, block, 0, s>>>(P, coarse, phi_fine, factor, (float)p0, fg)
    if (P.Q == 9) {
        if (P.storage == STORE_F16) LBM_RESTART(9, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_RESTART(9, STORE_BF16);
        else LBM_RESTART(9, STORE_F32);
    } else {
        if (P.storage == STORE_F16) LBM_RESTART(19, STORE_F16);
        else if (P.storage == STORE_BF16) LBM_RESTART(19, STORE_BF16);
        else LBM_RESTART(19, STORE_F32);
    }
#undef LBM_RESTART
    return cudaGetLastError();
}

__global__ void adjust_phi_kernel(float2* __restrict__ plane0, long long N, long long q, long long r) {
    const long long sign = r < 0 ? -1 : 1, ar = r < 0 ? -r : r;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const long long add = q + (c < ar ? sign : 0);
        const int v = __float_as_int(plane0[c].y);
        plane0[c].y = __int_as_float((int)((unsigned int)v + (unsigned int)add));
    }
}

cudaError_t launch_adjust_phi(const Params& P, void* fg, long long delta, cudaStream_t s) {
    const long long q = delta / P.N, r = delta - q * P.N;
    const long long blocks = (P.N + 255) / 256;
    adjust_phi_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(moment_plane(fg), P.N, q, r);
    return cudaGetLastError();
}

__device__ __forceinline__ double warp_sum_jm(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_jm(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kJumpThreads = 256;

__global__ void __launch_bounds__(kJumpThreads)
jump_measures_kernel(const float* __restrict__ start, const float* __restrict__ pred, int ncx, int ncy, int ncz,
                     int walls, double* __restrict__ out) {
    const long long nc = (long long)ncx * ncy * ncz;
    double acc[3] = {0.0, 0.0, 0.0}, umax = 0.0;
    for (long long l = (long long)blockIdx.x * kJumpThreads + threadIdx.x; l < nc; l += (long long)gridDim.x * kJumpThreads) {
        const int x = (int)(l % ncx), y = (int)((l / ncx) % ncy), z = (int)(l / ((long long)ncx * ncy));
        auto idx = [&](int xx, int yy, int zz) { return ((long long)zz * ncy + yy) * ncx + xx; };
        auto nb = [](int i, int d, int n, bool wall) { return wall ? min(max(i + d, 0), n - 1) : (i + d + n) % n; };
        const float ps = __ldg(start + l), pp = __ldg(pred + l);
        acc[0] += (double)pp;
        acc[1] += fabs((double)pp - (double)ps);
        const double gx = 0.5 * ((double)__ldg(start + idx(nb(x, 1, ncx, walls & 1), y, z)) -
                                 (double)__ldg(start + idx(nb(x, -1, ncx, walls & 1), y, z)));
        const double gy = 0.5 * ((double)__ldg(start + idx(x, nb(y, 1, ncy, walls & 2), z)) -
                                 (double)__ldg(start + idx(x, nb(y, -1, ncy, walls & 2), z)));
        const double gz = 0.5 * ((double)__ldg(start + idx(x, y, nb(z, 1, ncz, walls & 4))) -
                                 (double)__ldg(start + idx(x, y, nb(z, -1, ncz, walls & 4))));
        acc[2] += sqrt(gx * gx + gy * gy + gz * gz);
        double u2s = 0.0, u2p = 0.0;
#pragma unroll
        for (int a = 1; a <= 3; ++a) {
            const double us = __ldg(start + a * nc + l), up = __ldg(pred + a * nc + l);
            u2s += us * us;
            u2p += up * up;
        }
        umax = fmax(umax, fmax(u2s, u2p));
    }
    __shared__ double red[4][kJumpThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] = warp_sum_jm(acc[k]);
    umax = warp_max_jm(umax);
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) red[k][warp] = acc[k];
        red[3][warp] = umax;
    }
    __syncthreads();
    if (warp == 0) {
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (lane < kJumpThreads / 32) ? red[k][lane] : 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = warp_sum_jm(v[k]);
        v[3] = warp_max_jm(v[3]);
        if (lane == 0) {
            for (int k = 0; k < 3; ++k) atomicAdd(out + k, v[k]);
            // non-negative doubles order like their bit patterns
            atomicMax(reinterpret_cast<unsigned long long*>(out + 3), (unsigned long long)__double_as_longlong(v[3]));
        }
    }
}

cudaError_t launch_jump_measures(const float* start, const float* pred, int ncx, int ncy, int ncz, int walls, double* out,
                                 cudaStream_t s) {
    const long long nc = (long long)ncx * ncy * ncz;
    const long long blocks = (nc + kJumpThreads - 1) / kJumpThreads;
    jump_measures_kernel<<<(unsigned)(blocks < 1216 ? blocks : 1216), kJumpThreads, 0, s>>>(start, pred, ncx, ncy, ncz,
                                                                                           walls, out);
    return cudaGetLastError();
}

__global__ void normalize_kernel(const float* __restrict__ x, float* __restrict__ y, long long n, float m0, float m1,
                                 float m2, float m3, float m4, float s0, float s1, float s2, float s3, float s4, int dir) {
    const float mean[5] = {m0, m1, m2, m3, m4}, sd[5] = {s0, s1, s2, s3, s4};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 5 * n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / n);
        y[i] = dir > 0 ? (x[i] - mean[c]) / sd[c] : x[i] * sd[c] + mean[c];
    }
}

cudaError_t launch_normalize(const float* x, float* y, long long n, const float* ms, int dir, cudaStream_t s) {
    const long long blocks = (5 * n + 255) / 256;
    normalize_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(x, y, n, ms[0], ms[1], ms[2], ms[3], ms[4],
                                                                              ms[5], ms[6], ms[7], ms[8], ms[9], dir);
    return cudaGetLastError();
}

}  // namespace lbm
