// Instantiation of the sweep kernel for one stencil radius.  Each
// fd_step_rN.cu includes this with FD_R defined, so the radii compile in
// parallel translation units.
#pragma once

#include "fd_step.cuh"
#if FD_R == 2 || FD_R == 4
#include "fd_tblock.cuh"
#endif

namespace fd {
namespace {

template <int R, int TX, int TY, int MODE>
constexpr int pf_of() {
  return auto_pf<R, TX, TY, MODE == kModePerCell ? R : 0, MODE>();
}

template <int R, int TX, int TY, int PF, int MODE>
constexpr uint32_t sweep_smem() {
  return Cfg<R, TX, TY, PF, MODE == kModePerCell ? R : 0>::SMEM;
}

template <int R, int TX, int TY, int PF, int MODE>
cudaError_t set_smem_attr() {
  static unsigned long long done = 0;  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (done & (1ull << (dev & 63))) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel<R, TX, TY, PF, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       sweep_smem<R, TX, TY, PF, MODE>());
  if (e == cudaSuccess) done |= 1ull << (dev & 63);
  return e;
}

// The scheduled sweep (every mode but per-cell weights): the same shared
// memory and launch bounds as the equal-share kernel, so the same CTAs fit on
// an SM.
template <int R, int TX, int TY, int PF, int MODE>
cudaError_t set_sched_smem_attr() {
  static unsigned long long done = 0;  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (done & (1ull << (dev & 63))) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(sched_kernel<R, TX, TY, PF, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       sweep_smem<R, TX, TY, PF, MODE>());
  if (e == cudaSuccess) done |= 1ull << (dev & 63);
  return e;
}

template <int R, int TX, int TY, int PF, int MODE>
cudaError_t launch_one(const ShotDesc* shots, const long long* prefix, int nshots,
                       const StepOverride& ov, int grid, cudaStream_t s) {
  if (ov.items) {
    if constexpr (MODE != kModePerCell) {
      cudaError_t e = set_sched_smem_attr<R, TX, TY, PF, MODE>();
      if (e != cudaSuccess) return e;
      sched_kernel<R, TX, TY, PF, MODE><<<grid, TX * TY, sweep_smem<R, TX, TY, PF, MODE>(), s>>>(
          shots, ov);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  cudaError_t e = set_smem_attr<R, TX, TY, PF, MODE>();
  if (e != cudaSuccess) return e;
  sweep_kernel<R, TX, TY, PF, MODE><<<grid, TX * TY, sweep_smem<R, TX, TY, PF, MODE>(), s>>>(
      shots, prefix, nshots, ov);
  return cudaGetLastError();
}

template <int R, int TX, int TY, int PF, int MODE>
int occupancy_one() {
  if (set_smem_attr<R, TX, TY, PF, MODE>() != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<R, TX, TY, PF, MODE>,
                                                    TX * TY,
                                                    sweep_smem<R, TX, TY, PF, MODE>()) !=
      cudaSuccess)
    return 0;
  return nb;
}

}  // namespace

// Tile shapes compiled for every radius: (threads in x, rows); the prefetch
// depth of each follows from its shared-memory budget (auto_pf).
#define FD_FOR_EACH_SHAPE(X) X(16, 16) X(32, 8) X(8, 16) X(16, 8) X(8, 8)

// Per-cell and table weights exist for space order 8 only; other radii map
// those modes to the plain forward kernel (the runtime never asks for them).
#if FD_R == 4
#define FD_MODE_PERCELL 3
#define FD_MODE_TABLE 4
#else
#define FD_MODE_PERCELL 0
#define FD_MODE_TABLE 0
#endif
#define FD_PERCELL_LAUNCH(TX, TY)                                                          \
  case kModePerCell:                                                                       \
    return launch_one<FD_R, TX, TY, pf_of<FD_R, TX, TY, FD_MODE_PERCELL>(), FD_MODE_PERCELL>( \
        shots, prefix, nshots, ov, grid, s);                                               \
  case kModeTable:                                                                         \
    return launch_one<FD_R, TX, TY, pf_of<FD_R, TX, TY, FD_MODE_TABLE>(), FD_MODE_TABLE>(     \
        shots, prefix, nshots, ov, grid, s);
#define FD_PERCELL_OCC(TX, TY)                                                                \
  case kModePerCell:                                                                          \
    return occupancy_one<FD_R, TX, TY, pf_of<FD_R, TX, TY, FD_MODE_PERCELL>(), FD_MODE_PERCELL>(); \
  case kModeTable:                                                                            \
    return occupancy_one<FD_R, TX, TY, pf_of<FD_R, TX, TY, FD_MODE_TABLE>(), FD_MODE_TABLE>();
#define FD_PF(TX, TY) pf_of<FD_R, TX, TY, 0>()

template <>
cudaError_t launch_sweep_r<FD_R>(const TileShape& t, int mode, const ShotDesc* shots,
                                 const long long* prefix, int nshots, const StepOverride& ov,
                                 int grid, cudaStream_t s) {
#define FD_SHAPE(TX, TY)                                                                  \
  if (t.tx == TX && t.ty == TY) {                                                         \
    switch (mode) {                                                                       \
      case kModeForward:                                                                  \
        return launch_one<FD_R, TX, TY, FD_PF(TX, TY), 0>(shots, prefix, nshots, ov, grid, s); \
      case kModeStoreE:                                                                   \
        return launch_one<FD_R, TX, TY, FD_PF(TX, TY), 1>(shots, prefix, nshots, ov, grid, s); \
      case kModeAdjoint:                                                                  \
        return launch_one<FD_R, TX, TY, FD_PF(TX, TY), 2>(shots, prefix, nshots, ov, grid, s); \
      FD_PERCELL_LAUNCH(TX, TY)                                                           \
      default: return cudaErrorInvalidValue;                                              \
    }                                                                                     \
  }
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return cudaErrorInvalidValue;
}

template <>
int sweep_blocks_per_sm_r<FD_R>(const TileShape& t, int mode) {
#define FD_SHAPE(TX, TY)                                                        \
  if (t.tx == TX && t.ty == TY) {                                               \
    switch (mode) {                                                             \
      case kModeForward: return occupancy_one<FD_R, TX, TY, FD_PF(TX, TY), 0>(); \
      case kModeStoreE: return occupancy_one<FD_R, TX, TY, FD_PF(TX, TY), 1>();  \
      case kModeAdjoint: return occupancy_one<FD_R, TX, TY, FD_PF(TX, TY), 2>(); \
      FD_PERCELL_OCC(TX, TY)                                                    \
      default: return 0;                                                        \
    }                                                                           \
  }
  FD_FOR_EACH_SHAPE(FD_SHAPE)
#undef FD_SHAPE
  return 0;
}

#if FD_R == 2 || FD_R == 4
template <>
void tblock_tile_r<FD_R>(int* bx, int* by) {
  *bx = TbGeom<FD_R>::BX;
  *by = TbGeom<FD_R>::BY;
}

template <>
cudaError_t launch_tblock_r<FD_R>(const TbDesc* d, const TbLaunch& l, int grid, cudaStream_t s) {
  static unsigned long long done = 0;  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(done & (1ull << (dev & 63)))) {
    cudaError_t e = cudaFuncSetAttribute(tblock_kernel<FD_R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TbGeom<FD_R>::SMEM);
    if (e != cudaSuccess) return e;
    done |= 1ull << (dev & 63);
  }
  tblock_kernel<FD_R><<<grid, TbGeom<FD_R>::NT, TbGeom<FD_R>::SMEM, s>>>(d, l);
  return cudaGetLastError();
}
#endif

}  // namespace fd
