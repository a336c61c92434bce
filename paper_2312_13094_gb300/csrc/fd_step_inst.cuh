// Instantiation of the step kernel for one stencil radius.  Each
// fd_step_rN.cu includes this with FD_R defined, so the radii compile in
// parallel translation units.
#pragma once

#include "fd_step.cuh"

namespace fd {
namespace {

template <int R, int TX, int TY, int PF, int MODE>
cudaError_t launch_one(const CUtensorMap& h, const CUtensorMap& p,
                       const CUtensorMap& A, const CUtensorMap& Cm, const StepArgs& a,
                       cudaStream_t s) {
  using C = Cfg<R, TX, TY, PF, MODE == kModePerCell ? R : 0>;
  static unsigned long long attr_done = 0;  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  auto k = step_kernel<R, TX, TY, PF, MODE>;
  if (!(attr_done & (1ull << (dev & 63)))) {
    cudaError_t e = cudaFuncSetAttribute(
        k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_done |= 1ull << (dev & 63);
  }
  dim3 grid(a.tiles_x, a.tiles_y, a.zsplit);
  k<<<grid, C::NT, C::SMEM, s>>>(h, p, A, Cm, a);
  return cudaGetLastError();
}

template <int R, int TX, int TY, int PF>
cudaError_t launch_batch_one(const BatchShot* shots, const int4* work, int nwork,
                             int* counter, int step, int grid, cudaStream_t s) {
  using C = Cfg<R, TX, TY, PF>;
  static unsigned long long attr_done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  auto k = batch_kernel<R, TX, TY, PF>;
  if (!(attr_done & (1ull << (dev & 63)))) {
    cudaError_t e = cudaFuncSetAttribute(
        k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_done |= 1ull << (dev & 63);
  }
  k<<<grid, C::NT, C::SMEM, s>>>(shots, work, nwork, counter, step);
  return cudaGetLastError();
}

template <int R, int TX, int TY, int PF>
int batch_occupancy() {
  using C = Cfg<R, TX, TY, PF>;
  auto k = batch_kernel<R, TX, TY, PF>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, C::NT, C::SMEM) != cudaSuccess)
    return 0;
  return nb;
}

template <int R, int TX, int TY, int PF>
int regs_of() {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, step_kernel<R, TX, TY, PF, 0>) != cudaSuccess)
    return -1;
  return fa.numRegs;
}

}  // namespace

// Tile shapes compiled for every radius: (threads in x, rows, prefetch).
#define FD_FOR_EACH_SHAPE(X) X(16, 16, 2) X(32, 8, 2) X(8, 32, 2) X(16, 8, 3)

#if FD_R == 4
#define FD_PERCELL(TX, TY, PF) \
  case kModePerCell: return launch_one<FD_R, TX, TY, PF, 3>(h, p, A, Cm, a, s);
#else
#define FD_PERCELL(TX, TY, PF)
#endif

template <>
cudaError_t launch_step_r<FD_R>(const TileShape& t, int mode,
                                const CUtensorMap& h, const CUtensorMap& p,
                                const CUtensorMap& A, const CUtensorMap& Cm,
                                const StepArgs& a, cudaStream_t s) {
#define FD_SHAPE(TX, TY, PF)                                                        \
  if (t.tx == TX && t.ty == TY && t.pf == PF) {                                     \
    switch (mode) {                                                                 \
      case kModeForward: return launch_one<FD_R, TX, TY, PF, 0>(h, p, A, Cm, a, s); \
      case kModeStoreE: return launch_one<FD_R, TX, TY, PF, 1>(h, p, A, Cm, a, s);  \
      case kModeAdjoint: return launch_one<FD_R, TX, TY, PF, 2>(h, p, A, Cm, a, s); \
      FD_PERCELL(TX, TY, PF)                                                        \
      default: return cudaErrorInvalidValue;                                        \
    }                                                                               \
  }
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_batch_r<FD_R>(const TileShape& t, const BatchShot* shots, const int4* work,
                                 int nwork, int* counter, int step, int grid,
                                 cudaStream_t s) {
#define FD_SHAPE(TX, TY, PF)                  \
  if (t.tx == TX && t.ty == TY && t.pf == PF) \
    return launch_batch_one<FD_R, TX, TY, PF>(shots, work, nwork, counter, step, grid, s);
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return cudaErrorInvalidValue;
}

template <>
int batch_blocks_per_sm_r<FD_R>(const TileShape& t) {
#define FD_SHAPE(TX, TY, PF) \
  if (t.tx == TX && t.ty == TY && t.pf == PF) return batch_occupancy<FD_R, TX, TY, PF>();
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return 0;
}

template <>
size_t smem_r<FD_R>(const TileShape& t) {
#define FD_SHAPE(TX, TY, PF) \
  if (t.tx == TX && t.ty == TY && t.pf == PF) return Cfg<FD_R, TX, TY, PF>::SMEM;
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return 0;
}

template <>
int regs_r<FD_R>(const TileShape& t) {
#define FD_SHAPE(TX, TY, PF) \
  if (t.tx == TX && t.ty == TY && t.pf == PF) return regs_of<FD_R, TX, TY, PF>();
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return -1;
}

}  // namespace fd
