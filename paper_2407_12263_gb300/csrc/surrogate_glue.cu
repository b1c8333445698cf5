// surrogate_glue.cu -- field transfers between the lattice and the surrogate's coarse grid:
// block means of the macroscopic fields, trilinear upsampling into the initialisation's
// staging (the restart is then the same equilibrium-plus-non-equilibrium construction as the
// initial state), and the exact correction of sum phi after a restart.
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
                macro_interface_df<Q>(P, gb, m);
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

cudaError_t launch_coarsen(const Params& P, const void* fg, int factor, float* out, cudaStream_t s) {
    const int ncx = P.nx / factor, ncy = P.ny / factor, ncz = P.nz / factor;
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

// coarse index and weight of fine cell i along an axis of n fine cells (nc coarse ones)
__device__ __forceinline__ void interp_axis(int i, int f, int nc, bool wall, int& i0, int& i1, double& t) {
    const double xc = (i + 0.5) / f - 0.5;
    int a = (int)floor(xc);
    t = xc - a;
    int b = a + 1;
    if (wall) {
        if (a < 0) { a = 0; t = 0.0; }
        if (b > nc - 1) { b = nc - 1; t = (a == b) ? 0.0 : t; }
    } else {
        a = (a % nc + nc) % nc;
        b = (b % nc + nc) % nc;
    }
    i0 = a;
    i1 = b;
}

__device__ __forceinline__ double trilinear(const float* __restrict__ q, int ncx, int ncy, int x0, int x1, double tx,
                                            int y0, int y1, double ty, int z0, int z1, double tz) {
    auto at = [&](int z, int y, int x) { return (double)q[((long long)z * ncy + y) * ncx + x]; };
    const double c00 = at(z0, y0, x0) * (1 - tx) + at(z0, y0, x1) * tx;
    const double c01 = at(z0, y1, x0) * (1 - tx) + at(z0, y1, x1) * tx;
    const double c10 = at(z1, y0, x0) * (1 - tx) + at(z1, y0, x1) * tx;
    const double c11 = at(z1, y1, x0) * (1 - tx) + at(z1, y1, x1) * tx;
    return (c00 * (1 - ty) + c01 * ty) * (1 - tz) + (c10 * (1 - ty) + c11 * ty) * tz;
}

__global__ void upsample_kernel(const Params P, const float* __restrict__ coarse, int f, int z0, int nzs,
                                double* __restrict__ phis, double* __restrict__ us, double* __restrict__ ps) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int l = (int)blockIdx.z - 1;  // plane z0 + l, l = -1 .. nzs
    if (x >= P.nx || y >= P.ny) return;
    const int ncx = P.nx / f, ncy = P.ny / f, ncz = P.nz / f;
    const long long nc = (long long)ncx * ncy * ncz;
    int z = z0 + l;
    if (P.walls & 4) z = min(max(z, 0), P.nz - 1);
    else z = ((z % P.nz) + P.nz) % P.nz;
    int x0, x1, y0, y1, zz0, zz1;
    double tx, ty, tz;
    interp_axis(x, f, ncx, P.walls & 1, x0, x1, tx);
    interp_axis(y, f, ncy, P.walls & 2, y0, y1, ty);
    interp_axis(z, f, ncz, P.walls & 4, zz0, zz1, tz);
    const size_t nxy = (size_t)P.nxy;
    const size_t cell = (size_t)y * P.nx + x;
    phis[(size_t)(l + 1) * nxy + cell] = trilinear(coarse, ncx, ncy, x0, x1, tx, y0, y1, ty, zz0, zz1, tz);
    if (l < 0 || l >= nzs) return;
    const size_t slab = (size_t)nzs * nxy, lu = (size_t)l * nxy + cell;
    for (int a = 0; a < 3; ++a)
        us[a * slab + lu] = trilinear(coarse + (1 + a) * nc, ncx, ncy, x0, x1, tx, y0, y1, ty, zz0, zz1, tz);
    ps[lu] = trilinear(coarse + 4 * nc, ncx, ncy, x0, x1, tx, y0, y1, ty, zz0, zz1, tz);
}

cudaError_t launch_upsample_slab(const Params& P, const float* coarse, int factor, int z0, int nzs, double* phis,
                                 double* us, double* ps, cudaStream_t s) {
    const dim3 block(32, 4), grid((P.nx + 31) / 32, (P.ny + 3) / 4, nzs + 2);
    upsample_kernel<<<grid, block, 0, s>>>(P, coarse, factor, z0, nzs, phis, us, ps);
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
