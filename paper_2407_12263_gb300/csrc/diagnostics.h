// diagnostics.h -- launcher of the state diagnostics (lbm_diagnostics), internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// Per-block partials of n_blocks blocks (diag_partial_bytes(n_blocks) bytes of device scratch,
// 8-byte aligned) and the result, 7 doubles on the device: the largest |u|, its cell index (the
// bits of a 64-bit integer), the kinetic energy, the mean p inside r_in and outside r_out (NaN
// where no cell qualifies) and the two cell counts. FD needs phi_fd from launch_fd_phi first.
// d2_axes: device, nx + ny + nz doubles, the squared distance along x, y and z of each cell
// coordinate from the centre (axis_d2_host).
size_t diag_partial_bytes(int n_blocks);
double axis_d2_host(int i, double c, int n, bool wall);
cudaError_t launch_diagnostics(const Params& P, int scheme, const void* fg, const float* phi_fd, const double* d2_axes,
                               double r_in, double r_out, void* partials, int n_blocks, double* result, cudaStream_t s);

}  // namespace lbm
