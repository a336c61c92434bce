// Small helper kernels of libfd.so: model set-up, reductions, gradient fold.
#include <math.h>
#include <string.h>

#include "fd_aux.h"

namespace fd {

namespace {

__global__ void k_model_stats(const float* __restrict__ data, size_t n, int kind,
                              unsigned int* vmin_bits, unsigned int* vmax_bits,
                              int* bad) {
  float lo = INFINITY, hi = 0.0f;
  int nbad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float x = data[i];
    if (!(x > 0.0f) || !isfinite(x)) {
      ++nbad;
      continue;
    }
    const float v = kind == 0 ? x : 1.0f / sqrtf(x);
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  // positive floats order like their bit patterns
  if (nbad) atomicAdd(bad, nbad);
  if (hi > 0.0f) {
    atomicMin(vmin_bits, __float_as_uint(lo));
    atomicMax(vmax_bits, __float_as_uint(hi));
  }
}

// A = dt^2 / (m h^2) on every padded cell, the model edge-replicated into the
// layer.  Computed in double, rounded once to float.
__global__ void k_model_to_A(const float* __restrict__ data, int kind, int nx,
                             int ny, int nz, int nbl, int Nx, int Ny, int Nz,
                             int pitch, double dt2_h2, float* __restrict__ A) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= pitch) return;
  float* row = A + ((size_t)z * Ny + y) * pitch;
  if (x >= Nx) {
    row[x] = 0.0f;
    return;
  }
  const int px = min(max(x - nbl, 0), nx - 1);
  const int py = min(max(y - nbl, 0), ny - 1);
  const int pz = min(max(z - nbl, 0), nz - 1);
  const double val = data[((size_t)pz * ny + py) * nx + px];
  const double a = kind == 0 ? dt2_h2 * val * val : dt2_h2 / val;
  row[x] = (float)a;
}

__global__ void k_count_nonfinite(const float* __restrict__ x, size_t n, int* cnt) {
  int c = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    c += isfinite(x[i]) ? 0 : 1;
  if (c) atomicAdd(cnt, c);
}

__global__ void k_residual(const float* __restrict__ rec, const float* __restrict__ obs,
                           float* __restrict__ r, size_t n, double* loss) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float d = rec[i] - obs[i];
    r[i] = d;
    acc += 0.5 * (double)d * (double)d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(loss, acc);
}

// Physical gradient: each physical cell sums the padded cells that replicate
// it (only cells on the faces of the physical box have more than one).
__global__ void k_fold_grad(const float* __restrict__ gpad, int nx, int ny, int nz,
                            int nbl, int Nx, int Ny, int Nz, int pitch,
                            float* __restrict__ gphys) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= nx) return;
  const int xa = x == 0 ? 0 : x + nbl, xb = x == nx - 1 ? Nx - 1 : x + nbl;
  const int ya = y == 0 ? 0 : y + nbl, yb = y == ny - 1 ? Ny - 1 : y + nbl;
  const int za = z == 0 ? 0 : z + nbl, zb = z == nz - 1 ? Nz - 1 : z + nbl;
  double acc = 0.0;
  for (int k = za; k <= zb; ++k)
    for (int j = ya; j <= yb; ++j)
      for (int i = xa; i <= xb; ++i) acc += gpad[((size_t)k * Ny + j) * pitch + i];
  gphys[((size_t)z * ny + y) * nx + x] = (float)acc;
}

__global__ void k_pad_coef(const float* __restrict__ phys, int R, int nx, int ny, int nz,
                           int nbl, int Nx, int Ny, int Nz, int pitch, size_t ncell,
                           float* __restrict__ coef) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= Nx) return;
  const int px = min(max(x - nbl, 0), nx - 1);
  const int py = min(max(y - nbl, 0), ny - 1);
  const int pz = min(max(z - nbl, 0), nz - 1);
  const size_t src = (((size_t)pz * ny + py) * nx + px) * R;
  const size_t dst = ((size_t)z * Ny + y) * pitch + x;
  for (int j = 0; j < R; ++j) coef[j * ncell + dst] = phys[src + j];
}

}  // namespace

cudaError_t pad_coefficients(const float* phys, int R, int nx, int ny, int nz, int nbl, int Nx,
                             int Ny, int Nz, int pitch, size_t ncell, float* coef,
                             cudaStream_t s) {
  dim3 grid((Nx + 127) / 128, Ny, Nz);
  k_pad_coef<<<grid, 128, 0, s>>>(phys, R, nx, ny, nz, nbl, Nx, Ny, Nz, pitch, ncell, coef);
  count_launch();
  return cudaGetLastError();
}

cudaError_t model_stats(const float* data, size_t n, int kind, float* vmin,
                        float* vmax, int* nbad, unsigned int* scratch,
                        cudaStream_t s) {
  // scratch: [vmin_bits, vmax_bits, bad]
  unsigned int init[3] = {0x7f800000u, 0u, 0u};
  cudaError_t e = cudaMemcpyAsync(scratch, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_model_stats<<<1024, 256, 0, s>>>(data, n, kind, scratch, scratch + 1,
                                     reinterpret_cast<int*>(scratch + 2));
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  unsigned int out[3];
  e = cudaMemcpyAsync(out, scratch, sizeof(out), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  memcpy(vmin, &out[0], sizeof(float));
  memcpy(vmax, &out[1], sizeof(float));
  *nbad = static_cast<int>(out[2]);
  return cudaSuccess;
}

cudaError_t model_to_A(const float* data, int kind, int nx, int ny, int nz, int nbl,
                       int Nx, int Ny, int Nz, int pitch, double dt2_h2, float* A,
                       cudaStream_t s) {
  dim3 grid((pitch + 127) / 128, Ny, Nz);
  k_model_to_A<<<grid, 128, 0, s>>>(data, kind, nx, ny, nz, nbl, Nx, Ny, Nz, pitch,
                                    dt2_h2, A);
  count_launch();
  return cudaGetLastError();
}

cudaError_t count_nonfinite(const float* x, size_t n, int* dcnt, int* hcnt,
                            cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dcnt, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (n) {
    k_count_nonfinite<<<256, 256, 0, s>>>(x, n, dcnt);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(hcnt, dcnt, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t residual(const float* rec, const float* obs, float* r, size_t n,
                     double* dloss, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dloss, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (n) {
    k_residual<<<256, 256, 0, s>>>(rec, obs, r, n, dloss);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t fold_grad(const float* gpad, int nx, int ny, int nz, int nbl, int Nx,
                      int Ny, int Nz, int pitch, float* gphys, cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny, nz);
  k_fold_grad<<<grid, 128, 0, s>>>(gpad, nx, ny, nz, nbl, Nx, Ny, Nz, pitch, gphys);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fd
