// lbm_internal.h -- parameters and kernel launchers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Scalar parameters of one lattice, derived on the host once (lbm_create / lbm_init_phi).
struct Params {
    int Q;                 // 9 or 19
    int nx, ny, nz;
    int nxy;               // nx * ny
    long long N;           // nx * ny * nz
    float lw_m, lw_p;      // Lax-Wendroff, difference form (Sec. 2.2):
                           // fbar(x) = f*(x) + lw_m [f*(x - e) - f*(x)] + lw_p [f*(x + e) - f*(x)]
    float flux_a, flux_b;  // the same update in flux form, weights times 2^30: the flux of a
                           // population across the face between an upwind cell u and its
                           // downwind neighbour d is 2^-30 (flux_a g*(u) + flux_b g*(d)),
                           // flux_a = 2^30 lw_m, flux_b = -2^30 lw_p
    float flux_as, flux_bs;  // flux_a, flux_b for g in the storage's units (set with the storage)
    float tau_phi;         // phase-field relaxation time
    float omega_g;         // 1 / (tau_phi + 1/2)           (Eq. c-n_c)
    float grad_s;          // tau_phi / (tau_phi + 1/2)      grad phi = grad_s S - grad_k K1
    float grad_k;          // 1 / ((tau_phi + 1/2) cs^2)
    float tau_f;           // tau_rho of fluid 2
    float omega_f;         // 1 / (tau_f + 1/2), used where the kinematic viscosity is uniform
    float rho2, drho;      // rho2 = 1, drho = rho1 - rho2
    float mu_m1;           // eta1 / eta2 - 1
    float sigma;           // surface tension
    float four_over_delta; // 4 / delta
    float G[3];            // body force
    float w0;              // storage shift of f: f_i is held as f_i - t_i w0 (w0 = p0 / cs^2)
    float phi_ref;         // storage shift of g: g_i is held as g_i - t_i phi_ref (phi_ref = 0 or 1)
    int phi_ref_fx;        // phi_ref * 2^30, the same level in the fixed-point units of plane 0
    int general;           // 1 if any of drho, G, mu_m1, walls is non-zero (selects the full kernels)
    int storage;           // enum StorageKind of the moving planes
    int walls;             // bit 0: walls at x = -1/2 and nx - 1/2; bit 1: the same in y; bit 2: in z
    // FP64 copies for the initialisation and the conversions to and from FP64 host arrays
    double w0d, phi_ref_d, tau_phi_d, sigma_d, four_over_delta_d, drho_d, rho2_d;
};

enum Scheme { SCHEME_DF = 0, SCHEME_FD = 1 };
enum StorageKind { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2 };

// Launchers (return the launch's cudaError_t). The state is one buffer (storage.cuh): plane 0
// holds the zeroth moments, sum_i f_i - w0 as FP32 and phi = sum_i g_i as a 32-bit fixed-point
// integer phi * 2^30, in place of the rest populations, which they determine exactly; then one
// plane of words per opposite pair of moving populations (i, j), each word the pairs
// (f_i - t_i w0, g_i - t_i phi_ref) and (f_j - t_j w0, g_j - t_j phi_ref) of one cell in the
// storage type (FP32, FP16 or BF16). f_i and g_i share their propagation stencil, and so do a
// population and its opposite, so one load serves all four values.
cudaError_t launch_step(const Params& P, int scheme, const void* fg_in, void* fg_out, float* phi_fd,
                        cudaStream_t s, int* launches);
cudaError_t launch_fd_phi(const Params& P, const void* fg_in, float* phi_fd, cudaStream_t s);

// Initial populations for z in [z0, z0 + nzs). phi0s holds planes z0-1 .. z0+nzs of phi0
// (periodic images for the two halo planes; D2Q9 holds the single plane at index 1);
// u0s (or nullptr) holds 3 x nzs planes of the velocity for the slab; ps (or nullptr) holds nzs
// planes of the pressure, else the pressure is p0 everywhere.
cudaError_t launch_init(const Params& P, int z0, int nzs, const double* phi0s, const double* u0s,
                        const double* ps, double p0, void* fg, cudaStream_t s);

// Where the macroscopic fields go: field j (0 phi, 1 p, 2-4 u, 5-7 grad phi, 8-10 n) of cell
// (x, y, z0 + zl) is written to p[j][zl * nxy + y * nx + x]; device memory or page-locked host
// memory the device can address.
struct FieldOut {
    double* p[11];
};
// Macroscopic fields for z in [z0, z0 + nzs) as FP64. mask selects the fields: bit 0 phi, 1 p,
// 2 u (3 planes), 3 grad phi (3), 4 n (3); the pointers of the selected fields must be set.
cudaError_t launch_moments(const Params& P, int scheme, int z0, int nzs, const void* fg,
                           const float* phi_fd, int mask, const FieldOut& out, cudaStream_t s);

// sum phi, sum rho phi (FP64), the count of non-finite stored populations, and in result[3]
// the bits of the exact 64-bit sum of the fixed-point phi values.
cudaError_t launch_mass(const Params& P, const void* fg, double* partials, int n_partials,
                        double* result /* 4 doubles */, cudaStream_t s);
int mass_partials_needed(const Params& P);
// Per block b < n_blocks: the count of
// values of v[0, n) outside [lo, hi] ((lo, hi] with open_low; non-finite values count) and their
// sum, in partials[2 b] and partials[2 b + 1]; fixed order, the same bits on every run.
cudaError_t launch_check_values(const double* v, long long n, double lo, double hi, int open_low, double* partials,
                                int n_blocks, cudaStream_t s);
// Only result[3] of launch_mass (the exact fixed-point sum of phi), from plane 0 alone.
cudaError_t launch_phi_fixed_sum(const Params& P, const void* fg, double* partials, int n_partials,
                                 double* result /* 4 doubles */, cudaStream_t s);

// All Q populations of the slab [z0, z0 + nzs) between the device storage and FP64 staging
// holding plain populations (Q planes of nzs * nxy values).
cudaError_t launch_pops_to_f64(const Params& P, const void* src, int is_f, int z0, int nzs, double* dst,
                               cudaStream_t s);
cudaError_t launch_pops_from_f64(const Params& P, const double* src, int is_f, int z0, int nzs, void* dst,
                                 cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Batches of independent cases (lbm_batch_*).
// ---------------------------------------------------------------------------------------
constexpr int kBatchThreads = 128;    // cells per tile and threads per block
constexpr int kMaxLaunchCases = 128;  // cases per group launch: their table fits the 32 KB parameter space

// One case of a group launch, as the kernel reads it from its parameter block.
struct LaunchCase {
    Params P;
    void* fg[2];    // the case's ping-pong state buffers
    int cur;        // buffer holding the state when the group was built
    int pad_;
};

// The whole parameter block of a group launch: up to kMaxLaunchCases cases of one grid size,
// tile shape, kernel variant and storage.
struct BatchLaunch {
    int n_cases;
    int flip;       // step parity: reads fg[cur ^ flip]
    int tx_shift;   // tile of 2^tx_shift x 2^ty_shift x 2^(7 - tx_shift - ty_shift) cells
    int ty_shift;
    int ntx;        // tiles along x, y and z
    int nty;
    int ntz;
    int general;
    int storage;
    int pad_;
    LaunchCase cases[kMaxLaunchCases];
};
static_assert(sizeof(BatchLaunch) <= 32764, "a group launch's parameters must fit the kernel parameter space");

// One step of every case of the group: grid (ntx * nty, n_cases, ntz), one tile per block.
cudaError_t launch_batch_group(int Q, const BatchLaunch& L, cudaStream_t s);
// The uniform rest state phi = 1, p = 1/3, u = 0 in the storage of P (plane 0 = (0, 2^30),
// moving planes 0), used by the tuner on cases that hold no state yet.
cudaError_t launch_fill_rest(const Params& P, void* fg, cudaStream_t s);

}  // namespace lbm
