// Internal entry of the learned-coefficient network used by the runtime.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fd.h"

namespace fd {

// Per-cell weights c_1..c_4 of every padded cell of a grid from its model
// term A (x0 = sqrt(A) = v dt / h); field j is written at coef + j * ncell.
fd_status mlp_grid_coefficients(fd_mlp net, const float* A, size_t ncell, int pitch, int Nx,
                                double h, double dt, double f_hz, float* coef,
                                cudaStream_t s);

}  // namespace fd
