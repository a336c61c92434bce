// Helper kernels of libfd.so (model set-up, reductions, gradient fold).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace fd {

// Library-wide kernel launch counter (defined in fd_runtime.cu).
void count_launch(long long n = 1);

// min/max velocity of a physical model (v in km/s, or m -> 1/sqrt(m)) and the
// number of non-positive or non-finite values.  Synchronises `s`.
cudaError_t model_stats(const float* data, size_t n, int kind, float* vmin,
                        float* vmax, int* nbad, unsigned int* scratch,
                        cudaStream_t s);
// A = dt^2/(m h^2) on the padded, pitched grid (edge-replicated model).
cudaError_t model_to_A(const float* data, int kind, int nx, int ny, int nz, int nbl,
                       int Nx, int Ny, int Nz, int pitch, double dt2_h2, float* A,
                       cudaStream_t s);
// Number of NaN/Inf values in x (synchronises `s`).
cudaError_t count_nonfinite(const float* x, size_t n, int* dcnt, int* hcnt,
                            cudaStream_t s);
// r = rec - obs and *dloss = sum r^2 / 2 (double, on the device).
cudaError_t residual(const float* rec, const float* obs, float* r, size_t n,
                     double* dloss, cudaStream_t s);
// Physical gradient from the padded one (sum over replicated layer cells).
cudaError_t fold_grad(const float* gpad, int nx, int ny, int nz, int nbl, int Nx,
                      int Ny, int Nz, int pitch, float* gphys, cudaStream_t s);

// Per-cell weights [nz][ny][nx][R] (physical) -> R padded, pitched fields
// (edge replication into the layer).
cudaError_t pad_coefficients(const float* phys, int R, int nx, int ny, int nz, int nbl, int Nx,
                             int Ny, int Nz, int pitch, size_t ncell, float* coef,
                             cudaStream_t s);

}  // namespace fd
