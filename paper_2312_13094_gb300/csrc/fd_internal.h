// Internal types shared by the CUDA translation units of libfd.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fd {

constexpr int kMaxR = 8;  // space order up to 16
constexpr int kTableNodes = 256;  // largest weight table of kModeTable

// One source node: padded z, tile-local x/y of the node, scaled weight and the
// column of the value table (wavelet or residual) that feeds it.
struct InjEntry {
  int32_t z;
  int16_t lx, ly;
  float w;
  int32_t col;
};

// One receiver: padded z of its floor node, tile-local floor x/y, the three
// fractional offsets and its output column.
struct RecEntry {
  int32_t z;
  int16_t lx, ly;
  float fx, fy, fz;
  int32_t col;
};

enum StepMode : int {
  kModeForward = 0,    // u^{n+1} only
  kModeStoreE = 1,     // also e = (dt^2/m)(L u + s) for the imaging condition
  kModeAdjoint = 2,    // also grad -= u_cur * e_in / dt^2 (u_cur = z^{n+1})
  kModePerCell = 3,    // forward with per-cell weights c_1..c_R (space order 8)
  kModeTable = 4       // forward with weights c_1..c_4 interpolated per point from a
                       // table over A = (v dt / h)^2 (space order 8)
};

// Everything one launch of the step kernel needs besides the tensor maps.
struct StepArgs {
  int32_t Nx, Ny, Nz;      // padded extents (Nz: updated planes per tile column)
  int32_t pitch;           // floats per row of every device array
  int32_t nbl, nx, ny, nz; // layer width and physical extents
  int32_t tiles_x, tiles_y;
  float bscale;            // gamma_max * dt / 2 / nbl^2
  float c[kMaxR + 1];      // second-derivative weights c_0..c_R
  float* out;              // u^{n+1}: the u^{n-1} buffer, updated in place
  const int32_t* inj_start;  // [tiles_x*tiles_y + 1] or nullptr
  const InjEntry* inj;
  const float* inj_val;      // [step][inj_ncol]
  int32_t inj_ncol;
  const int32_t* rec_start;  // [tiles_x*tiles_y + 1] or nullptr
  const RecEntry* recs;
  float* rec_out;            // [step][rec_ncol]
  int32_t rec_ncol;
  int32_t inj_row;           // row of inj_val read by this launch
  int32_t rec_row;           // row of rec_out written by this launch
  float* e_out;              // kModeStoreE
  const float* e_in;         // kModeAdjoint
  float* grad;               // kModeAdjoint (padded, pitched)
  const float4* table;       // kModeTable: per node i, c_1..c_4 at node i and the
                             // step to node i + 1 (2 float4 per node)
  float tab_lo, tab_inv;     // node i sits at A = tab_lo + i / tab_inv (tab_inv 0: one)
  int32_t tab_nodes;
  float inv_dt2;
  int32_t* err;              // device error word (bit 0: wait timed out)
  long long spin_limit;      // clock cycles before a wait gives up
  int32_t debug_skip_plane;  // test hook: never issue this plane's load (-1)
  // Subdomain of a Cartesian decomposition (whole grids: 0, 0, Nx, Ny, 0, 0,
  // 0): tiles start at array column xfirst and row yfirst, updated points lie
  // below xend and yend, and the padded-grid coordinate of a point is its
  // array coordinate plus (offx, offy, offz), which places the damping layer.
  int32_t xfirst, yfirst, xend, yend;
  int32_t offx, offy, offz;
};

// One grid of a sweep launch (device memory): its tensor maps, constants and
// buffers.  Step-dependent values come from StepOverride.
struct ShotDesc {
  CUtensorMap halo[2];  // u^n with halo, per buffer
  CUtensorMap tile[2];  // tiles without halo, per buffer (u^{n-1}; u^n for R >= 5)
  CUtensorMap A;        // model term tiles
  CUtensorMap C;        // per-cell weight tiles (fields stacked along z) or A
  StepArgs args;
  float* u[2];
};

// One work item of a scheduled sweep: planes [zb, ze) of tile column `tile`
// of grid `shot` of the launch.
struct WorkItem {
  int32_t shot, tile, zb, ze;
};

// Per-launch values of a sweep: buffer parity, table rows, imaging fields.
struct StepOverride {
  int cur;            // u[cur] holds u^n
  int zfirst;         // array plane of the first updated plane of every grid of the
                      // launch (0 for whole grids; a slab part: its first plane)
  int nblz;           // layer width in the launch's array planes along z: nbl minus the
                      // padded z of array plane 0 (nbl for whole grids)
  int inj_row;
  int rec_row;
  int debug_skip_plane;      // test hook: never issue this plane's load (-1)
  float* e_out;
  const float* e_in;
  long long spin_limit;      // clock cycles before a wait gives up
  float c[kMaxR + 2];        // stencil weights shared by every shot of the launch:
                             // c[0] the centre weight -6 sum c_j (hi part, see
                             // launch_weights), c[1..R] the weights c_j, c[kMaxR+1] the
                             // centre weight's lo part
  const int32_t* item_start; // scheduled sweep: CTA c runs items [item_start[c],
  const WorkItem* items;     // item_start[c+1]); nullptr: equal contiguous shares
};

// Two-step (temporally blocked) pass, fd_tblock.cuh: what does not change
// from one pass to the next.  Source entries carry extended-tile coordinates
// (lx, ly relative to the extended tile's corner); receiver entries are
// relative to the output tile.
struct TbArgs {
  int32_t Nx, Ny, Nz, pitch, nbl, nx, ny, nz, tiles_x, tiles_y;
  float bscale;
  const int32_t* inj1_start;  // [tiles + 1]: step-1 sources, nodes of the extended tile
  const InjEntry* inj1;
  const int32_t* inj2_start;  // [tiles + 1]: step-2 sources, nodes of the output tile
  const InjEntry* inj2;
  const float* inj_val;       // [step][inj_ncol]
  int32_t inj_ncol;
  const int32_t* rec_start;   // [tiles + 1]
  const RecEntry* recs;
  float* rec_out;             // [step][rec_ncol]
  int32_t rec_ncol;
  const float* A;             // model term (step 2 reads its own points)
  int32_t* err;
};

// Device descriptor of a two-step pass: tensor maps of the four wavefield
// buffers (u^n with the two-step halo, extended tiles of u^{n-1}), of A, and
// the buffers themselves.
struct TbDesc {
  CUtensorMap halo2[4];
  CUtensorMap ext[4];
  CUtensorMap extA;
  float* u[4];
  TbArgs args;
};

// Per-pass values: which buffers hold u^{n-1}, u^n and receive u^{n+1},
// u^{n+2}; the value-table rows of the pass's first step; the work items.
struct TbLaunch {
  int in_prev, in_cur, out1, out2;
  int inj_row, rec_row;
  long long spin_limit;
  float c[kMaxR + 2];  // as StepOverride::c
  const int32_t* item_start;
  const WorkItem* items;
};

// The weights of a uniform-stencil launch from the FP64 weights c[0..R]
// (host side): out[j] = c_j rounded to FP32 for j = 1..R, and the centre
// weight T = -6 sum_j out[j] (exact in FP64) as out[0] + out[kMaxR+1], the
// FP32 hi and lo parts; zero beyond R.
inline void launch_weights(const double* c, int R, float* out) {
  double t = 0.0;
  for (int j = 0; j < kMaxR + 2; ++j) out[j] = 0.0f;
  for (int j = 1; j <= R; ++j) {
    out[j] = static_cast<float>(c[j]);
    t += static_cast<double>(out[j]);
  }
  t *= -6.0;
  out[0] = static_cast<float>(t);
  out[kMaxR + 1] = static_cast<float>(t - static_cast<double>(out[0]));
}

struct TileShape {
  int tx, ty, pf;   // threads in x (4 points each), rows, prefetch depth
  int ctas;         // persistent CTAs per sweep (0: resident CTAs per SM x SMs)
};

// Per-radius launchers, specialised in fd_step_r<R>.cu.
template <int R>
cudaError_t launch_sweep_r(const TileShape& t, int mode, const ShotDesc* shots,
                           const long long* prefix, int nshots, const StepOverride& ov,
                           int grid, cudaStream_t s);
template <int R>
int sweep_blocks_per_sm_r(const TileShape& t, int mode);

// Two-step passes (space orders 4 and 8), specialised in fd_step_r2.cu and
// fd_step_r4.cu: the output tile and the launch.
template <int R>
void tblock_tile_r(int* bx, int* by);
template <int R>
cudaError_t launch_tblock_r(const TbDesc* d, const TbLaunch& l, int grid, cudaStream_t s);

}  // namespace fd
