// Host-side state of a grid and the runtime helpers shared by the host
// translation units (forward, adjoint, batch).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/fd.h"
#include "fd_internal.h"

namespace fd {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes);
  void release();
};

struct Tables {
  DevBuf inj_start, inj, rec_start, recs;
  int n_inj = 0, n_rec = 0;
};

// A pair of wavefield buffers with their tensor maps; u[cur] holds the
// current field, u[cur^1] the previous one (overwritten by the next).
struct Fields {
  float* u[2] = {nullptr, nullptr};
  CUtensorMap halo[2];
  CUtensorMap tile[2];
  int cur = 0;
};

// One run of consecutive steps.
struct RunSpec {
  Fields* f;
  int allow_graph;
  int mode;
  int nsteps;
  const int32_t* inj_start;
  const InjEntry* inj;
  const float* inj_val;
  int inj_ncol, inj_row0, inj_row_step;
  const int32_t* rec_start;
  const RecEntry* recs;
  float* rec_out;
  int rec_ncol, rec_row0, rec_row_step;
  float* e_base;      // kModeStoreE: e of step t at e_base + t*ncell
  int e_idx0, e_idx_step;  // kModeAdjoint: e_in index of step t
  float* grad;
};

// Everything that fixes the launches of a captured run (the descriptor
// contents are refreshed before each replay and are not part of it).
struct GraphKey {
  int mode, nsteps, cur, slot;
  int inj_row0, inj_row_step, rec_row0, rec_row_step;
  float* e_base;
  int e_idx0, e_idx_step;
  TileShape shape;
  int ctas;
  void* desc;
  const void* sched;  // work items of a wave-scheduled sweep (nullptr: equal shares)
  int skip;
  long long spin;
  float c[kMaxR + 2];
};

struct Decomp;  // domain decomposition state of a grid (fd_decomp.cu)
struct TbState;  // buffers of the two-step passes (fd_tblock.cu)
struct Cart;     // boxes of a Cartesian decomposition (fd_cart.cu)

constexpr int kNumShapes = 5;
constexpr int kTuneMinSteps = 400;  // shorter forward runs are not worth tuning
extern const TileShape kShapes[kNumShapes];

}  // namespace fd

struct fd_grid_s {
  fd_grid_desc d;
  int R = 1;
  int Nx = 0, Ny = 0, Nz = 0;
  int pitch = 0;
  size_t ncell = 0;  // pitch * Ny * Nz
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  fd::Fields F;  // forward wavefields u^{n-1}, u^n
  fd::Fields Z;  // adjoint wavefields (allocated on first use)
  float* A = nullptr;
  CUtensorMap mapA;
  float* coef = nullptr;   // per-cell weights c_1..c_R, field j at coef + j*ncell
  CUtensorMap mapC;
  bool percell = false;
  // kModeTable: c_1..c_4 at tab_nodes Courant numbers tab_lo + i / tab_inv
  float4* table = nullptr;
  int tab_nodes = 0;
  float tab_lo = 0.0f, tab_inv = 0.0f;
  bool table_mode = false;
  bool model_set = false;
  double vmin = 0.0, vmax = 0.0;
  float bscale = 0.0f;
  double c[fd::kMaxR + 1] = {};
  double cfl = 0.0;
  fd::TileShape shape = {};
  int tiles_x = 0, tiles_y = 0;
  fd::Tables tab, tab_adj;
  fd::DevBuf stage_val, stage_rec, stage_aux, recbuf;
  fd::DevBuf ckpt, ebuf, gpad, resid;
  fd::DevBuf desc;  // sweep descriptors (forward and adjoint slots)
  int32_t* d_err = nullptr;  // [0] wait-timeout word, [1] finite count, [4..6] scratch
  long long spin_limit = 0;
  int debug_skip_plane = -1;
  bool no_graph = false;
  bool profiling = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double step_ms = 0.0;
  long long steps_timed = 0;
  bool graph_valid = false;
  cudaGraphExec_t gexec = nullptr;
  fd::GraphKey gkey = {};
  fd::Decomp* dmp = nullptr;  // z slabs of fd_set_decomposition (nullptr: whole grid)
  fd::TbState* tb = nullptr;  // second wavefield pair etc. of FD_SCHED_TEMPORAL runs
  fd::Cart* cart = nullptr;   // boxes of fd_set_topology (nullptr: not decomposed)
  int sched_mode = FD_SCHED_AUTO;  // fd_set_schedule
  fd::DevBuf sched;                // wave schedule: CTA starts, then the work items
  long long sched_key[5] = {};     // tile, grid and CTA count it was built for
  int sched_ctas = 0;              // CTAs of the wave-scheduled launch
  size_t sched_off = 0;            // byte offset of the items in g->sched
  int last_sched = 0;              // schedule of the last forward run (fd_grid_info)
  fd::TileShape base_shape = {};   // tile of every run but tuned forward runs
  bool auto_tile = false;          // no fd_set_tile: plain forward runs may be tuned
  bool tuned = false;              // tuned_shape / tuned_waves hold the tuner's pick
  fd::TileShape tuned_shape = {};
  bool tuned_waves = false;
};

namespace fd {

fd_status fail(fd_status st, const char* fmt, ...);
fd_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
cudaError_t dev_alloc(void** p, size_t bytes);
long long alloc_count();         // device allocations made through dev_alloc so far
long long default_spin_limit();  // FD_SPIN_LIMIT, else ~0.1 s of clock cycles
bool is_device_ptr(const void* p);
fd_status make_map(CUtensorMap* m, const float* base, int Nx, int Ny, int Nz, int pitch, int bx,
                   int by);
int radius_halo_x(int R);
fd_status build_maps(fd_grid g);
fd_status build_field_maps(fd_grid g, Fields& f);
void set_shape(fd_grid g, TileShape t);
// Puts the grid on the tile its next run uses: the tuned one for plain forward
// runs of a tuned grid, else the base tile (rebuilding the tensor maps).
fd_status use_shape(fd_grid g, bool plain_forward);
// Times every compiled tile under both schedules on the grid's zeroed
// wavefields (a few source-free steps each) and records the fastest for plain
// forward runs; picks are cached per device and padded size.
fd_status autotune_grid(fd_grid g);
TileShape default_shape(int R, int Nx, int Ny, int Nz);
cudaError_t launch_sweep(int R, const TileShape& t, int mode, const ShotDesc* shots,
                         const long long* prefix, int nshots, const StepOverride& ov, int grid,
                         cudaStream_t s);
int sweep_ctas(int R, const TileShape& t, int mode);
// CTAs of one step launch: k z chunks per column when the columns fit in the
// resident slots (lockstep), else every resident slot; k = slots / columns,
// capped so that a chunk holds at least 8R of the Nz planes
int lockstep_chunks(int R, long long slots, long long columns, int Nz);
int lockstep_ctas(int R, const TileShape& t, int mode, long long columns, int Nz);
void fill_desc(fd_grid g, const RunSpec& rs, ShotDesc* d);
StepArgs base_args(fd_grid g);
int forward_mode(fd_grid g);  // kModeForward, kModePerCell or kModeTable
fd_status upload_tables(fd_grid g, const fd_points* src, double src_scale,
                        const fd_points* rec, Tables& t);
fd_status build_injection(fd_grid g, const fd_points* pts, double scale,
                          std::vector<int32_t>& start, std::vector<InjEntry>& out);
fd_status build_receivers(fd_grid g, const fd_points* pts, std::vector<int32_t>& start,
                          std::vector<RecEntry>& out);
// Padded floor node and fractions of a point in metres (FD_ERR_ARG outside
// the physical box).
fd_status locate_point(fd_grid g, const float* xyz, int i0[3], double f[3]);
// The same over bx x by tiles whose regions are widened by hx columns and hy
// rows per side (entries relative to the widened region's corner).
fd_status build_injection_tiles(fd_grid g, const fd_points* pts, double scale, int bx, int by,
                                int hx, int hy, std::vector<int32_t>& start,
                                std::vector<InjEntry>& out);
fd_status build_receivers_tiles(fd_grid g, const fd_points* pts, int bx, int by,
                                std::vector<int32_t>& start, std::vector<RecEntry>& out);
// Host vector to a device buffer (grown as needed) on the grid's stream.
template <class T>
fd_status upload(fd_grid g, DevBuf& buf, const std::vector<T>& v);
// Two-step passes (fd_tblock.cu): whether the grid's next forward run takes
// them, the run itself (nsteps steps, the last one single-step when nsteps is
// odd), and the release of their buffers with the grid.
bool tblock_eligible(fd_grid g);
fd_status tblock_propagate(fd_grid g, int n0, int nsteps, const fd_points* src,
                           const float* dval, const fd_points* rec, float* drec);
void tblock_destroy(fd_grid g);
fd_status stage_in(fd_grid g, DevBuf& buf, const float* p, size_t n, const float** out);
fd_status stage_out(fd_grid g, DevBuf& buf, float* p, size_t n, float** out);
fd_status finish_out(fd_grid g, float* host, const float* dev, size_t n);
fd_status run_steps(fd_grid g, const RunSpec& rs);
// Wave schedule of the grid's forward sweeps (built once per tile shape and
// CTA count, uploaded to g->sched); fills the item pointers of a launch and
// returns its CTA count, or 0 when the grid runs equal shares.
int grid_schedule(fd_grid g, int mode, StepOverride* ov, fd_status* st);
fd_status check_device_error(fd_grid g);
fd_status check_finite(fd_grid g, const float* dev, size_t n);
fd_status copy_field(fd_grid g, float* dev_field, void* user, int region, bool to_user);
// decomposed runs (fd_decomp.cu): steps of fd_forward / fd_propagate when the
// grid has slabs, and the release of the slabs with the grid
fd_status decomp_propagate(fd_grid g, int n0, int nsteps, const fd_points* src,
                           const float* wavelet, const fd_points* rec, float* rec_out);
void decomp_destroy(fd_grid g);
// Cartesian boxes (fd_cart.cu): the steps of fd_forward / fd_propagate when
// the grid has a px x py x pz topology, and the release of the boxes
fd_status cart_propagate(fd_grid g, int n0, int nsteps, const fd_points* src,
                         const float* wavelet, const fd_points* rec, float* rec_out);
void cart_destroy(fd_grid g);

}  // namespace fd
