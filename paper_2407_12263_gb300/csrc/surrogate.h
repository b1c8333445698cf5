// surrogate.h -- launchers of the convolutional surrogate's kernels (surrogate_kernels.cu) and
// of the field transfers between the lattice and the coarse grid (surrogate_glue.cu).
// Internal to the library.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {
namespace net {

constexpr int kFieldChannels = 5;  // phi, u, v, w, p
constexpr int kHidden = 32;        // channels of the hidden layers
constexpr int kLayers = 4;

// Periodic 3x3x3 convolution of a batch [B][cin][D][H][W] into [B][cout][D][H][W]
// (cout = 32 or 5), FP32 accumulation; inputs and outputs FP16 or FP32; relu on the output if
// asked. bias may be NULL.
cudaError_t conv_forward(const void* in, int in_fp16, int cin, const float* W, const float* bias, void* out, int out_fp16,
                         int cout, int relu, int batch, int D, int H, int Wd, cudaStream_t s);
// gW [cout][cin][27] += correlation of g [B][cout] with h [B][cin]; gb [cout] += sum of g.
cudaError_t conv_wgrad(const float* g, int cout, const void* h, int h_fp16, int cin, float* gW, float* gb, int batch,
                       int D, int H, int Wd, cudaStream_t s);
// Wt [cin][cout][27] with the taps reversed: the adjoint convolution's weights.
cudaError_t flip_transpose(const float* W, int cout, int cin, float* Wt, cudaStream_t s);
cudaError_t relu_mask(float* g, const void* h, int h_fp16, long long n, cudaStream_t s);
cudaError_t cast_to(const float* x, void* y, int fp16, long long n, cudaStream_t s);
cudaError_t residual(const float* x, const float* d, float* y, long long n, cudaStream_t s);
int loss_blocks(long long n);
// loss sum_i w_c(i) (x + d - target)_i^2 / n and its gradient; w: 5 host weights, vox: cells per channel.
cudaError_t loss_and_grad(const float* x, const float* d, const float* target, float* g, long long n, long long vox,
                          const float* w, double* partials, cudaStream_t s);
cudaError_t adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s);

// The 32 -> 32 convolution on the tensor cores (tcgen05): FP16 operands, FP32 accumulation.
// wimg is the layer's weight image (weight_image, weight_image_bytes() bytes); inputs FP16 or
// FP32, multiplied by in_scale (a power of two) before they are rounded to FP16 and the sums
// divided by it again (so small gradients keep their bits); outputs FP16 with relu or FP32
// without. *err is set to 1 if a wait for the tensor cores timed out: each wait for a step's
// MMAs polls its mbarrier at most `spin` times, kTcWaitPolls normally or 0 (give up at once,
// the same in every thread: a test of the timeout path); the last wait for MMAs still in
// flight, before the tensor memory is freed, always allows kTcWaitPolls.
// Layers with cin, cout <= 32 (the unused channels are zero-padded).
constexpr long long kTcWaitPolls = 1ll << 26;
size_t weight_image_bytes();
cudaError_t weight_image(const float* W, int cout, int cin, __half* img, cudaStream_t s);
cudaError_t conv32_tc(const void* in, int in_fp16, int cin, float in_scale, const __half* wimg, const float* bias, void* out,
                      int out_fp16, int cout, int relu, int batch, int D, int H, int Wd, long long spin, int* err,
                      cudaStream_t s);
// gW [cout][cin][27] += correlation of g [B][cout] with h [B][cin] on the tensor cores (g scaled by
// g_scale, a power of two, before FP16 rounding and unscaled after); gb [cout] += sum of g.
// scratch: wgrad_scratch_floats() floats of device memory for the per-CTA and per-block partial
// sums, which are added in a fixed order: the gradients are the same bits on every run.
constexpr int kBiasParts = 256;
size_t wgrad_scratch_floats();
cudaError_t wgrad32_tc(const float* g, int cout, float g_scale, const void* h, int h_fp16, int cin, float* gW, float* gb,
                       int batch, int D, int H, int Wd, long long spin, float* scratch, int* err, cudaStream_t s);

}  // namespace net

// Coarse fields [5][nz/f][ny/f][nx/f] (phi, u, v, w, p; means over f^3 cells of the macroscopic
// fields of the difference-free scheme) of the propagated state fg.
cudaError_t launch_coarsen(const Params& P, const void* fg, int factor, float* out, cudaStream_t s);
// Block means of the state's own phi (plane 0, before propagation) into out [nz/f][ny/f][nx/f];
// factor must divide 32 (cudaErrorInvalidValue otherwise).
cudaError_t launch_coarse_phi(const Params& P, const void* fg, int factor, float* out, cudaStream_t s);
// The state launch_init builds (equilibrium plus the first-order non-equilibrium part of g) from
// coarse fields upsampled trilinearly between coarse cell centres (periodic, clamped across
// walls), in FP32 arithmetic: the upsampled phi of every cell into phi_fine (N floats), then the
// populations.
cudaError_t launch_restart(const Params& P, const float* coarse, int factor, double p0, float* phi_fine, void* fg,
                           cudaStream_t s);
// Adds delta units (2^-30) of phi to the state, spread over the cells so that it sums exactly.
cudaError_t launch_adjust_phi(const Params& P, void* fg, long long delta, cudaStream_t s);
// What the judge of a jump measures on the coarse grid [5][ncz][ncy][ncx] of the starting fields
// `start` and of the prediction `pred`, accumulated into out[4] (zeroed by the caller):
//   out[0] += sum of the predicted phi;
//   out[1] += sum |phi_pred - phi_start|;
//   out[2] += sum |grad phi_start|, central differences in coarse cells (periodic, or the cell
//             itself beyond a wall, bit 0 x, bit 1 y, bit 2 z of walls);
//   out[3]  = max(out[3], largest |u|^2 of start and prediction) (as non-negative double bits).
cudaError_t launch_jump_measures(const float* start, const float* pred, int ncx, int ncy, int ncz, int walls, double* out,
                                 cudaStream_t s);
// The divergence-free part of the periodic velocity u [3][nz][ny][nx] in place
// (lbm_project_solenoidal); work holds project_workspace_bytes() bytes, 16-byte aligned.
cudaError_t launch_project_solenoidal(float* u, int nx, int ny, int nz, void* work, cudaStream_t s);
size_t project_workspace_bytes(int nx, int ny, int nz);
bool project_extents_ok(const int grid[3]);  // every extent in 1 .. 512
// (x - mean[c]) / std[c] per channel of [5][n] (dir = +1) or x std[c] + mean[c] (dir = -1).
cudaError_t launch_normalize(const float* x, float* y, long long n, const float* mean_std, int dir, cudaStream_t s);

}  // namespace lbm
