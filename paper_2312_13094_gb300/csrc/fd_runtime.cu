// Host runtime of libfd.so: the C ABI declared in include/fd.h.
//
// Owns the device state of a grid (two wavefields, the model term A, the
// per-tile source/receiver tables, checkpoints), builds the TMA tensor maps,
// captures the time loop in a CUDA graph and maps every failure to a status
// code with a thread-local message.
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fd.h"
#include "fd_aux.h"
#include "fd_internal.h"
#include "fd_mlp.h"
#include "fd_runtime.h"
#include "fd_sched.h"

namespace fd {

static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local std::string t_err;

fd_status fail(fd_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return st;
}

fd_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(FD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(FD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { t_err.clear(); }

// --------------------------------------------------------------------------
// allocation with a host-side failure-injection hook: FD_FAULT_ALLOC_AT=k makes
// the k-th device allocation of the process (1-based) fail with OOM.
// --------------------------------------------------------------------------
static std::atomic<long long> g_alloc_count{0};

cudaError_t dev_alloc(void** p, size_t bytes) {
  const long long k = g_alloc_count.fetch_add(1) + 1;
  const char* env = getenv("FD_FAULT_ALLOC_AT");
  if (env && atoll(env) == k) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

long long alloc_count() { return g_alloc_count.load(); }

// Clock cycles a device-side wait spins before it gives up: ~0.1 s at 2 GHz
// (a tile load takes microseconds), or FD_SPIN_LIMIT when set.
long long default_spin_limit() {
  long long v = 200000000LL;
  if (const char* s = getenv("FD_SPIN_LIMIT")) {
    const long long e = atoll(s);
    if (e > 0) v = e;
  }
  return v;
}

cudaError_t DevBuf::ensure(size_t bytes) {
  if (bytes <= cap) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = dev_alloc(&p, bytes);
  if (e == cudaSuccess) cap = bytes;
  return e;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// --------------------------------------------------------------------------
// tensor maps
// --------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

fd_status make_map(CUtensorMap* m, const float* base, int Nx, int Ny, int Nz,
                   int pitch, int bx, int by) {
  auto fn = encode_fn();
  if (!fn) return fail(FD_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)Nx, (cuuint64_t)Ny, (cuuint64_t)Nz};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * Ny};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                  strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for box %dx%d", (int)r,
                bx, by);
  return FD_OK;
}

int radius_halo_x(int R) { return ((R + 3) / 4) * 4; }

fd_status build_field_maps(fd_grid g, Fields& f) {
  const int bx = 4 * g->shape.tx, by = g->shape.ty;
  const int W = bx + 2 * radius_halo_x(g->R), H = by + 2 * g->R;
  for (int b = 0; b < 2; ++b) {
    if (!f.u[b]) continue;
    fd_status st = make_map(&f.halo[b], f.u[b], g->Nx, g->Ny, g->Nz, g->pitch, W, H);
    if (st) return st;
    st = make_map(&f.tile[b], f.u[b], g->Nx, g->Ny, g->Nz, g->pitch, bx, by);
    if (st) return st;
  }
  return FD_OK;
}

fd_status build_maps(fd_grid g) {
  fd_status st = build_field_maps(g, g->F);
  if (!st) st = build_field_maps(g, g->Z);
  if (st) return st;
  const int bx = 4 * g->shape.tx, by = g->shape.ty;
  st = make_map(&g->mapA, g->A, g->Nx, g->Ny, g->Nz, g->pitch, bx, by);
  if (st) return st;
  if (g->coef)  // the R coefficient fields stacked along z
    return make_map(&g->mapC, g->coef, g->Nx, g->Ny, g->R * g->Nz, g->pitch, bx, by);
  return FD_OK;
}

// --------------------------------------------------------------------------
// dispatch over radius
// --------------------------------------------------------------------------
cudaError_t launch_sweep(int R, const TileShape& t, int mode, const ShotDesc* shots,
                         const long long* prefix, int nshots, const StepOverride& ov, int grid,
                         cudaStream_t s) {
  count_launch();
  switch (R) {
    case 1: return launch_sweep_r<1>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 2: return launch_sweep_r<2>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 3: return launch_sweep_r<3>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 4: return launch_sweep_r<4>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 5: return launch_sweep_r<5>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 6: return launch_sweep_r<6>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 7: return launch_sweep_r<7>(t, mode, shots, prefix, nshots, ov, grid, s);
    case 8: return launch_sweep_r<8>(t, mode, shots, prefix, nshots, ov, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Persistent CTAs of a sweep: the explicit count of the tile shape, else the
// CTAs that fit on all SMs at once.
int sweep_ctas(int R, const TileShape& t, int mode) {
  if (t.ctas > 0) return t.ctas;
  int per = 0;
  switch (R) {
    case 1: per = sweep_blocks_per_sm_r<1>(t, mode); break;
    case 2: per = sweep_blocks_per_sm_r<2>(t, mode); break;
    case 3: per = sweep_blocks_per_sm_r<3>(t, mode); break;
    case 4: per = sweep_blocks_per_sm_r<4>(t, mode); break;
    case 5: per = sweep_blocks_per_sm_r<5>(t, mode); break;
    case 6: per = sweep_blocks_per_sm_r<6>(t, mode); break;
    case 7: per = sweep_blocks_per_sm_r<7>(t, mode); break;
    case 8: per = sweep_blocks_per_sm_r<8>(t, mode); break;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, per) * std::max(1, sms);
}

int lockstep_chunks(int R, long long slots, long long columns, int Nz) {
  // at least 8R planes per chunk: each chunk re-reads 2R halo planes
  const long long kmax = std::max<long long>(1, Nz / (8 * R));
  return int(std::min<long long>(slots / columns, kmax));
}

int lockstep_ctas(int R, const TileShape& t, int mode, long long columns, int Nz) {
  const int slots = sweep_ctas(R, t, mode);
  if (t.ctas > 0 || columns <= 0 || columns > slots) return slots;
  return int(columns * lockstep_chunks(R, slots, columns, Nz));
}

const TileShape kShapes[kNumShapes] = {
    {16, 16, 2, 0}, {32, 8, 2, 0}, {8, 16, 1, 0}, {16, 8, 2, 0}, {8, 8, 1, 0}};

// Default tile.  A shape whose T columns can all be resident at once runs in
// lockstep (k = slots / T z chunks per column, all in step), sharing halos in
// L2.  The k T chunks land on the SMs as evenly as the block scheduler can
// place them, so the slowest SM holds ceil(k T / SMs) chunks: among the
// lockstep shapes the one with the fewest points on that SM wins, then the
// wider tile, then the taller one.  Without a lockstep shape the widest tile
// (then the tallest) among those with the most resident warps, counting 16
// or more warps per SM as enough, runs the equal-share sweep, whose shares
// are balanced by construction.  Measured on GB300 (Gpts/s): SO 8 592^3
// lockstep 64x8 293, 32x16 285, 32x8 260, 128x8 246 and 64x16 221 (sweeps);
// SO 8 768^3 sweep 128x8 (16 warps per SM) 260, 64x16 (16) 235, 64x8 (20)
// 206, 32x16 (20) 178, 32x8 (20) 155; SO 16 592^3 sweep 32x16 (12) 160,
// 128x8 (8) 145.
TileShape default_shape(int R, int Nx, int Ny, int Nz) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = std::max(1, sms);
  auto wider = [](const TileShape& p, const TileShape& q) {  // p before q
    return p.tx != q.tx ? p.tx > q.tx : p.ty > q.ty;
  };
  int best = -1, best_sweep = -1;
  long long best_load = 0, best_warps = 0;
  for (int i = 0; i < kNumShapes; ++i) {
    const TileShape& t = kShapes[i];
    const int bx = 4 * t.tx, by = t.ty;
    const long long T = (long long)((Nx + bx - 1) / bx) * ((Ny + by - 1) / by);
    const long long slots = sweep_ctas(R, t, kModeForward);
    const long long warps = std::min<long long>(16, slots / sms * (t.tx * t.ty / 32));
    if (best_sweep < 0 || warps > best_warps ||
        (warps == best_warps && wider(t, kShapes[best_sweep]))) {
      best_sweep = i;
      best_warps = warps;
    }
    if (T <= slots) {
      // k chunks of Nz / k planes per column; the busiest SM holds
      // ceil(k T / SMs) chunks
      const long long k = lockstep_chunks(R, slots, T, Nz);
      const long long load = (k * T + sms - 1) / sms * (long long)(bx * by) * Nz / k;
      if (best < 0 || load < best_load || (load == best_load && wider(t, kShapes[best]))) {
        best = i;
        best_load = load;
      }
    }
  }
  return kShapes[best >= 0 ? best : best_sweep];
}

void set_shape(fd_grid g, TileShape t) {
  const int bx = 4 * t.tx, by = t.ty;
  g->shape = t;
  g->tiles_x = (g->Nx + bx - 1) / bx;
  g->tiles_y = (g->Ny + by - 1) / by;
  g->graph_valid = false;
}

// FD weights: c_j = 2(-1)^{j+1}(R!)^2/(j^2 (R-j)!(R+j)!), c_0 = -2 sum c_j.
void fd_weights(int R, double* c) {
  double sum = 0.0;
  for (int j = 1; j <= R; ++j) {
    double ratio = 1.0;
    for (int k = 1; k <= j; ++k) ratio *= double(R - k + 1) / double(R + k);
    c[j] = ((j & 1) ? 2.0 : -2.0) * ratio / (double(j) * j);
    sum += c[j];
  }
  c[0] = -2.0 * sum;
}

// Largest stable v dt / h of the 3D leapfrog: sqrt(4 / (3 S)) with S the
// magnitude of the 1D stencil symbol at the Nyquist wavenumber.
double cfl_limit(const double* c, int R) {
  double S = -c[0];
  for (int j = 1; j <= R; ++j) S -= 2.0 * ((j & 1) ? -c[j] : c[j]);
  return sqrt(4.0 / (3.0 * S));
}

// --------------------------------------------------------------------------
// source / receiver tables
// --------------------------------------------------------------------------
struct PointCell {
  int i0[3];
  double f[3];
};

fd_status locate_point(fd_grid g, const float* xyz, int i0[3], double f[3]);

static fd_status locate(fd_grid g, const float* xyz, PointCell* pc) {
  return locate_point(g, xyz, pc->i0, pc->f);
}

// Padded floor node i0 and fractions f of a point given in metres from the
// physical origin; FD_ERR_ARG outside the physical box.
fd_status locate_point(fd_grid g, const float* xyz, int i0[3], double f[3]) {
  PointCell c;
  PointCell* pc = &c;
  const int n[3] = {g->d.nx, g->d.ny, g->d.nz};
  for (int a = 0; a < 3; ++a) {
    const double s = double(xyz[a]) / g->d.h;
    if (!(s >= 0.0) || s > double(n[a] - 1))
      return fail(FD_ERR_ARG, "point (%g, %g, %g) outside the physical box", xyz[0], xyz[1],
                  xyz[2]);
    const double fl = floor(s);
    pc->i0[a] = int(fl) + g->d.nbl;
    pc->f[a] = s - fl;
  }
  for (int a = 0; a < 3; ++a) {
    i0[a] = c.i0[a];
    f[a] = c.f[a];
  }
  return FD_OK;
}

// Trilinear injection entries of every point, scaled by `scale`, grouped per
// tile and sorted by z within a tile (stable: a node's entries keep the order
// of the points).  Tiles are bx x by; a tile's region is extended by hx
// columns and hy rows on each side, so a node near a tile edge can belong to
// several tiles, and lx, ly are relative to the extended region's corner.
fd_status build_injection_tiles(fd_grid g, const fd_points* pts, double scale, int bx, int by,
                                int hx, int hy, std::vector<int32_t>& start,
                                std::vector<InjEntry>& out) {
  const int tiles_x = (g->Nx + bx - 1) / bx, tiles_y = (g->Ny + by - 1) / by;
  const int ntiles = tiles_x * tiles_y;
  std::vector<std::pair<int, InjEntry>> ent;
  for (int p = 0; p < (pts ? pts->n : 0); ++p) {
    PointCell pc;
    fd_status st = locate(g, pts->xyz + 3 * p, &pc);
    if (st) return st;
    for (int c = 0; c < 8; ++c) {
      int node[3];
      double w = 1.0;
      for (int a = 0; a < 3; ++a) {
        const int hi = (c >> a) & 1;
        node[a] = pc.i0[a] + hi;
        w *= hi ? pc.f[a] : 1.0 - pc.f[a];
      }
      if (w == 0.0) continue;
      if (node[0] >= g->Nx || node[1] >= g->Ny || node[2] >= g->Nz) continue;
      const int tx0 = std::max(0, (node[0] - hx) / bx);
      const int tx1 = std::min(tiles_x - 1, (node[0] + hx) / bx);
      const int ty0 = std::max(0, (node[1] - hy) / by);
      const int ty1 = std::min(tiles_y - 1, (node[1] + hy) / by);
      for (int ty = ty0; ty <= ty1; ++ty) {
        for (int tx = tx0; tx <= tx1; ++tx) {
          const int lx = node[0] - (tx * bx - hx), ly = node[1] - (ty * by - hy);
          if (lx < 0 || lx >= bx + 2 * hx || ly < 0 || ly >= by + 2 * hy) continue;
          InjEntry e;
          e.z = node[2];
          e.lx = int16_t(lx);
          e.ly = int16_t(ly);
          e.w = float(w * scale);
          e.col = p;
          ent.push_back({ty * tiles_x + tx, e});
        }
      }
    }
  }
  std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) {
    return a.first != b.first ? a.first < b.first : a.second.z < b.second.z;
  });
  start.assign(ntiles + 1, 0);
  out.clear();
  for (auto& e : ent) {
    start[e.first + 1]++;
    out.push_back(e.second);
  }
  for (int t = 0; t < ntiles; ++t) start[t + 1] += start[t];
  return FD_OK;
}

fd_status build_injection(fd_grid g, const fd_points* pts, double scale,
                          std::vector<int32_t>& start, std::vector<InjEntry>& out) {
  return build_injection_tiles(g, pts, scale, 4 * g->shape.tx, g->shape.ty, 0, 0, start, out);
}

// Receivers grouped per bx x by tile (floor node's tile), sorted by z.
fd_status build_receivers_tiles(fd_grid g, const fd_points* pts, int bx, int by,
                                std::vector<int32_t>& start, std::vector<RecEntry>& out) {
  const int tiles_x = (g->Nx + bx - 1) / bx, tiles_y = (g->Ny + by - 1) / by;
  const int ntiles = tiles_x * tiles_y;
  std::vector<std::pair<int, RecEntry>> ent;
  for (int p = 0; p < (pts ? pts->n : 0); ++p) {
    PointCell pc;
    fd_status st = locate(g, pts->xyz + 3 * p, &pc);
    if (st) return st;
    RecEntry e;
    e.z = pc.i0[2];
    e.lx = int16_t(pc.i0[0] % bx);
    e.ly = int16_t(pc.i0[1] % by);
    e.fx = float(pc.f[0]);
    e.fy = float(pc.f[1]);
    e.fz = float(pc.f[2]);
    e.col = p;
    ent.push_back({(pc.i0[1] / by) * tiles_x + pc.i0[0] / bx, e});
  }
  std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) {
    return a.first != b.first ? a.first < b.first : a.second.z < b.second.z;
  });
  start.assign(ntiles + 1, 0);
  out.clear();
  for (auto& e : ent) {
    start[e.first + 1]++;
    out.push_back(e.second);
  }
  for (int t = 0; t < ntiles; ++t) start[t + 1] += start[t];
  return FD_OK;
}

fd_status build_receivers(fd_grid g, const fd_points* pts, std::vector<int32_t>& start,
                          std::vector<RecEntry>& out) {
  return build_receivers_tiles(g, pts, 4 * g->shape.tx, g->shape.ty, start, out);
}

template <class T>
fd_status upload(fd_grid g, DevBuf& buf, const std::vector<T>& v) {
  cudaError_t e = buf.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
  if (e) return cuda_fail(e, "table allocation");
  if (!v.empty()) {
    e = cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                        g->stream);
    if (e) return cuda_fail(e, "table upload");
  }
  return FD_OK;
}
template fd_status upload<int32_t>(fd_grid, DevBuf&, const std::vector<int32_t>&);
template fd_status upload<InjEntry>(fd_grid, DevBuf&, const std::vector<InjEntry>&);
template fd_status upload<RecEntry>(fd_grid, DevBuf&, const std::vector<RecEntry>&);

fd_status upload_tables(fd_grid g, const fd_points* src, double src_scale,
                        const fd_points* rec, Tables& t) {
  std::vector<int32_t> is, rs;
  std::vector<InjEntry> ie;
  std::vector<RecEntry> re;
  fd_status st = build_injection(g, src, src_scale, is, ie);
  if (st) return st;
  st = build_receivers(g, rec, rs, re);
  if (st) return st;
  if ((st = upload(g, t.inj_start, is))) return st;
  if ((st = upload(g, t.inj, ie))) return st;
  if ((st = upload(g, t.rec_start, rs))) return st;
  if ((st = upload(g, t.recs, re))) return st;
  t.n_inj = int(ie.size());
  t.n_rec = int(re.size());
  // keep the uploads ordered before the host vectors go away
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "table upload");
  return FD_OK;
}

// Device view of a caller array: the pointer itself if it is device memory,
// else a staging buffer (filled from the host when `in`).
fd_status stage_in(fd_grid g, DevBuf& buf, const float* p, size_t n, const float** out) {
  if (!p || n == 0) {
    *out = nullptr;
    return FD_OK;
  }
  if (is_device_ptr(p)) {
    *out = p;
    return FD_OK;
  }
  cudaError_t e = buf.ensure(n * sizeof(float));
  if (e) return cuda_fail(e, "staging allocation");
  e = cudaMemcpyAsync(buf.p, p, n * sizeof(float), cudaMemcpyHostToDevice, g->stream);
  if (e) return cuda_fail(e, "host to device copy");
  *out = static_cast<const float*>(buf.p);
  return FD_OK;
}

fd_status stage_out(fd_grid g, DevBuf& buf, float* p, size_t n, float** out) {
  if (!p || n == 0) {
    *out = nullptr;
    return FD_OK;
  }
  if (is_device_ptr(p)) {
    *out = p;
    return FD_OK;
  }
  cudaError_t e = buf.ensure(n * sizeof(float));
  if (e) return cuda_fail(e, "staging allocation");
  *out = static_cast<float*>(buf.p);
  return FD_OK;
}

fd_status finish_out(fd_grid g, float* host, const float* dev, size_t n) {
  if (!host || host == dev || n == 0) return FD_OK;
  cudaError_t e =
      cudaMemcpyAsync(host, dev, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream);
  if (e) return cuda_fail(e, "device to host copy");
  return FD_OK;
}

// --------------------------------------------------------------------------
// time loop
// --------------------------------------------------------------------------
StepArgs base_args(fd_grid g) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.Nx = g->Nx;
  a.Ny = g->Ny;
  a.Nz = g->Nz;
  a.pitch = g->pitch;
  a.nbl = g->d.nbl;
  a.nx = g->d.nx;
  a.ny = g->d.ny;
  a.nz = g->d.nz;
  a.tiles_x = g->tiles_x;
  a.tiles_y = g->tiles_y;
  a.bscale = g->bscale;
  for (int j = 0; j <= kMaxR; ++j) a.c[j] = j <= g->R ? float(g->c[j]) : 0.0f;
  a.err = g->d_err;
  a.spin_limit = g->spin_limit;
  a.debug_skip_plane = -1;
  a.table = g->table;
  a.tab_lo = g->tab_lo;
  a.tab_inv = g->tab_inv;
  a.tab_nodes = g->tab_nodes;
  a.xend = g->Nx;
  a.yend = g->Ny;
  return a;
}

int forward_mode(fd_grid g) {
  if (g->percell) return kModePerCell;
  if (g->table_mode) return kModeTable;
  return kModeForward;
}

// Host image of the sweep descriptor of one run (grid, field pair, tables).
void fill_desc(fd_grid g, const RunSpec& rs, ShotDesc* d) {
  memset(d, 0, sizeof(*d));
  Fields& F = *rs.f;
  for (int b = 0; b < 2; ++b) {
    d->halo[b] = F.halo[b];
    d->tile[b] = F.tile[b];
    d->u[b] = F.u[b];
  }
  d->A = g->mapA;
  d->C = g->coef ? g->mapC : g->mapA;
  d->args = base_args(g);
  if (rs.inj_val) {
    d->args.inj_start = rs.inj_start;
    d->args.inj = rs.inj;
    d->args.inj_val = rs.inj_val;
    d->args.inj_ncol = rs.inj_ncol;
  }
  if (rs.rec_out) {
    d->args.rec_start = rs.rec_start;
    d->args.recs = rs.recs;
    d->args.rec_out = rs.rec_out;
    d->args.rec_ncol = rs.rec_ncol;
  }
  d->args.grad = rs.grad;
  d->args.inv_dt2 = float(1.0 / (g->d.dt * g->d.dt));
  d->args.out = nullptr;
}

// FD_SCHED_WAVES runs every forward sweep of the grid on the wave schedule of
// fd_sched.cu; FD_SCHED_AUTO does so for plain forward runs when the tuner
// picked it, else the equal-share sweep (lockstep when the columns fit).
int grid_schedule(fd_grid g, int mode, StepOverride* ov, fd_status* st) {
  *st = FD_OK;
  const bool tuned_waves = g->sched_mode == FD_SCHED_AUTO && g->tuned && g->tuned_waves &&
                           g->shape.tx == g->tuned_shape.tx && g->shape.ty == g->tuned_shape.ty;
  if (mode == kModePerCell || g->shape.ctas > 0 ||
      !(g->sched_mode == FD_SCHED_WAVES || tuned_waves))
    return 0;
  const int slots = sweep_ctas(g->R, g->shape, mode);
  const long long key[5] = {g->shape.tx, g->shape.ty, g->Nz,
                            (long long)g->tiles_x * g->tiles_y, slots};
  if (memcmp(key, g->sched_key, sizeof(key)) != 0 || !g->sched.p) {
    std::vector<int32_t> start;
    std::vector<WorkItem> items;
    const std::vector<SchedGrid> grids = {{0, g->tiles_x * g->tiles_y, g->Nz}};
    const int used = wave_schedule(grids, slots, g->R, start, items);
    const size_t off = (start.size() * 4 + 15) / 16 * 16;
    cudaError_t e = g->sched.ensure(off + items.size() * sizeof(WorkItem));
    if (!e) e = cudaMemcpyAsync(g->sched.p, start.data(), start.size() * 4,
                                cudaMemcpyHostToDevice, g->stream);
    if (!e)
      e = cudaMemcpyAsync(static_cast<char*>(g->sched.p) + off, items.data(),
                          items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, g->stream);
    if (!e) e = cudaStreamSynchronize(g->stream);
    if (e) {
      *st = cuda_fail(e, "schedule upload");
      return 0;
    }
    memcpy(g->sched_key, key, sizeof(key));
    g->sched_ctas = used;
    g->sched_off = off;
  }
  ov->item_start = static_cast<const int32_t*>(g->sched.p);
  ov->items = reinterpret_cast<const WorkItem*>(static_cast<const char*>(g->sched.p) +
                                                g->sched_off);
  return g->sched_ctas;
}

fd_status use_shape(fd_grid g, bool plain_forward) {
  const TileShape want = (plain_forward && g->tuned && g->sched_mode == FD_SCHED_AUTO)
                             ? g->tuned_shape
                             : g->base_shape;
  if (want.tx == 0) return FD_OK;  // a grid without a base tile keeps its own
  if (want.tx == g->shape.tx && want.ty == g->shape.ty && want.ctas == g->shape.ctas)
    return FD_OK;
  set_shape(g, want);
  return build_maps(g);
}

// Tuner picks per (device, radius, padded size, kernel mode).
static std::mutex g_tune_mu;
static std::map<std::string, std::pair<TileShape, bool>> g_tune_cache;

fd_status autotune_grid(fd_grid g) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, g->d.device);
  const std::string key = std::string(prop.name) + "|R" + std::to_string(g->R) + "|" +
                          std::to_string(g->Nx) + "x" + std::to_string(g->Ny) + "x" +
                          std::to_string(g->Nz) + "|M" + std::to_string(forward_mode(g));
  std::pair<TileShape, bool> pick = {g->base_shape, false};
  bool found = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      pick = it->second;
      found = true;
    }
  }
  fd_status st = FD_OK;
  if (!found) {
    const bool prof = g->profiling;
    g->profiling = false;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    if (e) st = cuda_fail(e, "tuner events");
    RunSpec rs;
    memset(&rs, 0, sizeof(rs));
    rs.f = &g->F;
    rs.allow_graph = 0;
    rs.mode = kModeForward;
    // every (tile, schedule) pair is timed twice, in one order and then in
    // the reverse one, and keeps its faster time: one pass of short trials
    // misranked pairs within a few percent of each other
    const int trial = 6;
    constexpr int kPairs = 2 * kNumShapes;
    float best_of[kPairs];
    for (int c = 0; c < kPairs; ++c) best_of[c] = 1e30f;
    float best = 1e30f;
    for (int r = 0; r < 2 * kPairs && !st; ++r) {
      const int c = r < kPairs ? r : 2 * kPairs - 1 - r;
      const TileShape t = kShapes[c / 2];
      g->tuned = true;
      g->tuned_shape = t;
      g->tuned_waves = (c & 1) != 0;
      if ((st = use_shape(g, true))) break;
      rs.nsteps = 1;  // warm-up (builds the schedule)
      if ((st = run_steps(g, rs))) break;
      cudaEventRecord(a, g->stream);
      rs.nsteps = trial;
      if ((st = run_steps(g, rs))) break;
      cudaEventRecord(b, g->stream);
      if ((e = cudaEventSynchronize(b))) {
        st = cuda_fail(e, "tuner timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      best_of[c] = std::min(best_of[c], ms);
      if (r >= kPairs && best_of[c] < best) {
        best = best_of[c];
        pick = {t, g->tuned_waves};
      }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    g->profiling = prof;
    if (!st) st = check_device_error(g);
    if (st) {
      g->tuned = false;
      use_shape(g, false);
      return st;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = pick;
  }
  g->tuned = true;
  g->tuned_shape = pick.first;
  g->tuned_waves = pick.second;
  return use_shape(g, true);
}

fd_status run_steps(fd_grid g, const RunSpec& rs) {
  if (rs.nsteps <= 0) return FD_OK;
  cudaError_t e;
  Fields& F = *rs.f;
  const int mode = rs.mode == kModeForward ? forward_mode(g) : rs.mode;
  // lockstep when all columns fit in the resident slots: k = slots / T CTAs
  // per column, each taking one of k equal z chunks (the shares below then
  // fall on chunk boundaries), so every CTA walks z in step with its
  // neighbours, which share halos in L2; otherwise equal contiguous shares
  // of all the (tile, plane) units over every resident slot
  int G = lockstep_ctas(g->R, g->shape, mode, (long long)g->tiles_x * g->tiles_y, g->Nz);
  StepOverride sched_ov;
  memset(&sched_ov, 0, sizeof(sched_ov));
  {
    fd_status st = FD_OK;
    const int Gs = grid_schedule(g, mode, &sched_ov, &st);
    if (st) return st;
    if (Gs > 0) G = Gs;
    if (mode == kModeForward || mode == kModeTable)
      g->last_sched = Gs > 0 ? FD_SCHED_WAVES : FD_SCHED_SHARES;
  }
  // descriptor + unit prefix, refreshed before every run (stream ordered),
  // so a captured graph stays valid when tables or caller arrays move
  struct {
    ShotDesc d;
    long long prefix[2];
  } host;
  fill_desc(g, rs, &host.d);
  host.prefix[0] = 0;
  host.prefix[1] = (long long)g->tiles_x * g->tiles_y * g->Nz;
  const int slot = (&F == &g->Z) ? 1 : 0;
  e = g->desc.ensure(2 * sizeof(host));
  if (e) return cuda_fail(e, "descriptor allocation");
  char* dslot = static_cast<char*>(g->desc.p) + slot * sizeof(host);
  e = cudaMemcpyAsync(dslot, &host, sizeof(host), cudaMemcpyHostToDevice, g->stream);
  if (e) return cuda_fail(e, "descriptor upload");
  const ShotDesc* dshot = reinterpret_cast<const ShotDesc*>(dslot);
  const long long* dprefix = reinterpret_cast<const long long*>(dslot + sizeof(ShotDesc));

  const bool use_graph = rs.allow_graph && rs.nsteps >= 2 && !g->no_graph;
  GraphKey key;
  memset(&key, 0, sizeof(key));
  key.mode = mode;
  key.nsteps = rs.nsteps;
  key.cur = F.cur;
  key.slot = slot;
  key.inj_row0 = rs.inj_row0;
  key.inj_row_step = rs.inj_row_step;
  key.rec_row0 = rs.rec_row0;
  key.rec_row_step = rs.rec_row_step;
  key.e_base = rs.e_base;
  key.e_idx0 = rs.e_idx0;
  key.e_idx_step = rs.e_idx_step;
  key.shape = g->shape;
  key.ctas = G;
  key.desc = dslot;
  key.sched = sched_ov.items;
  key.skip = g->debug_skip_plane;
  key.spin = g->spin_limit;
  launch_weights(g->c, g->R, key.c);
  const bool reuse = use_graph && g->graph_valid && memcmp(&key, &g->gkey, sizeof(key)) == 0;
  if (g->profiling) cudaEventRecord(g->ev0, g->stream);
  const int cur0 = F.cur;
  if (!reuse) {
    if (use_graph) {
      if (g->graph_valid) {
        cudaGraphExecDestroy(g->gexec);
        g->graph_valid = false;
      }
      e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed);
      if (e) return cuda_fail(e, "stream capture");
    }
    const long long before = g_launches.load();
    for (int t = 0; t < rs.nsteps; ++t) {
      StepOverride ov;
      memset(&ov, 0, sizeof(ov));
      ov.cur = (cur0 + t) & 1;
      ov.zfirst = 0;
      ov.nblz = g->d.nbl;
      ov.item_start = sched_ov.item_start;
      ov.items = sched_ov.items;
      ov.spin_limit = g->spin_limit;
      ov.debug_skip_plane = (t == 0) ? g->debug_skip_plane : -1;
      launch_weights(g->c, g->R, ov.c);
      ov.inj_row = rs.inj_row0 + rs.inj_row_step * t;
      ov.rec_row = rs.rec_row0 + rs.rec_row_step * t;
      if (mode == kModeStoreE) ov.e_out = rs.e_base + size_t(t) * g->ncell;
      if (mode == kModeAdjoint)
        ov.e_in = rs.e_base + size_t(rs.e_idx0 + rs.e_idx_step * t) * g->ncell;
      e = launch_sweep(g->R, g->shape, mode, dshot, dprefix, 1, ov, G, g->stream);
      if (e) {
        if (use_graph) {
          cudaGraph_t dummy = nullptr;
          cudaStreamEndCapture(g->stream, &dummy);
          if (dummy) cudaGraphDestroy(dummy);
        }
        return cuda_fail(e, "step launch");
      }
    }
    if (use_graph) {
      g_launches.store(before);  // counted when the graph runs
      cudaGraph_t graph;
      e = cudaStreamEndCapture(g->stream, &graph);
      if (e) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&g->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e) return cuda_fail(e, "graph instantiate");
      g->graph_valid = true;
      g->gkey = key;
    }
  }
  if (use_graph) {
    e = cudaGraphLaunch(g->gexec, g->stream);
    if (e) return cuda_fail(e, "graph launch");
    count_launch(rs.nsteps);
  }
  F.cur = (cur0 + rs.nsteps) & 1;
  if (g->profiling) {
    cudaEventRecord(g->ev1, g->stream);
    e = cudaEventSynchronize(g->ev1);
    if (e) return cuda_fail(e, "profiling event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    g->step_ms += ms;
    g->steps_timed += rs.nsteps;
  }
  return FD_OK;
}

fd_status check_device_error(fd_grid g) {
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "stream synchronize");
  int h = 0;
  e = cudaMemcpy(&h, g->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(e, "error word read");
  if (h) {
    cudaMemset(g->d_err, 0, sizeof(int));
    return fail(FD_ERR_TIMEOUT, "a device-side wait ran out (error word %d)", h);
  }
  return FD_OK;
}

fd_status check_finite(fd_grid g, const float* dev, size_t n) {
  int h = 0;
  cudaError_t e = count_nonfinite(dev, n, g->d_err + 1, &h, g->stream);
  if (e) return cuda_fail(e, "finite check");
  if (h) return fail(FD_ERR_NONFINITE, "%d receiver samples are NaN or Inf", h);
  return FD_OK;
}

// Copy between the padded pitched wavefield and a dense caller array.
fd_status copy_field(fd_grid g, float* dev_field, void* user, int region, bool to_user) {
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof(p));
  const bool phys = region == FD_REGION_PHYSICAL;
  const int ex = phys ? g->d.nx : g->Nx, ey = phys ? g->d.ny : g->Ny,
            ez = phys ? g->d.nz : g->Nz;
  const int off = phys ? g->d.nbl : 0;
  cudaPitchedPtr dev = make_cudaPitchedPtr(dev_field, size_t(g->pitch) * 4, g->Nx * 4, g->Ny);
  cudaPitchedPtr usr = make_cudaPitchedPtr(user, size_t(ex) * 4, ex * 4, ey);
  if (to_user) {
    p.srcPtr = dev;
    p.srcPos = make_cudaPos(size_t(off) * 4, off, off);
    p.dstPtr = usr;
  } else {
    p.srcPtr = usr;
    p.dstPtr = dev;
    p.dstPos = make_cudaPos(size_t(off) * 4, off, off);
  }
  p.extent = make_cudaExtent(size_t(ex) * 4, ey, ez);
  p.kind = cudaMemcpyDefault;
  cudaError_t e = cudaMemcpy3DAsync(&p, g->stream);
  if (e) return cuda_fail(e, "wavefield copy");
  return FD_OK;
}

}  // namespace fd

using namespace fd;

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

const char* fd_status_string(fd_status s) {
  switch (s) {
    case FD_OK: return "ok";
    case FD_ERR_ARG: return "invalid argument";
    case FD_ERR_CUDA: return "CUDA error";
    case FD_ERR_OOM: return "out of device memory";
    case FD_ERR_UNSTABLE: return "time step above the stability limit";
    case FD_ERR_STATE: return "call out of order";
    case FD_ERR_TIMEOUT: return "device-side wait timed out";
    case FD_ERR_NONFINITE: return "non-finite receiver data";
  }
  return "unknown status";
}

const char* fd_last_error(void) { return t_err.c_str(); }

int64_t fd_launch_count(void) { return g_launches.load(); }

int64_t fd_alloc_count(void) { return alloc_count(); }

fd_status fd_create_grid(const fd_grid_desc* d, fd_grid* out) {
  clear_error();
  if (!d || !out) return fail(FD_ERR_ARG, "null argument");
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1)
    return fail(FD_ERR_ARG, "grid sizes must be positive");
  if (!(d->h > 0.0) || !(d->dt > 0.0)) return fail(FD_ERR_ARG, "h and dt must be positive");
  if (d->space_order < 2 || d->space_order > 16 || (d->space_order & 1))
    return fail(FD_ERR_ARG, "space_order must be even, 2..16");
  if (d->nbl < 0 || d->nt < 0) return fail(FD_ERR_ARG, "nbl and nt must be >= 0");
  const long long Nx = d->nx + 2LL * d->nbl, Ny = d->ny + 2LL * d->nbl,
                  Nz = d->nz + 2LL * d->nbl;
  if (Nx > (1 << 24) || Ny > 65535 || Nz > 65535)
    return fail(FD_ERR_ARG, "padded grid too large for the launch shape");
  cudaError_t e = cudaSetDevice(d->device);
  if (e) return cuda_fail(e, "cudaSetDevice");

  fd_grid g = new fd_grid_s();
  g->d = *d;
  g->R = d->space_order / 2;
  g->Nx = int(Nx);
  g->Ny = int(Ny);
  g->Nz = int(Nz);
  g->pitch = int((Nx + 31) / 32 * 32);
  g->ncell = size_t(g->pitch) * g->Ny * g->Nz;
  fd_weights(g->R, g->c);
  g->cfl = cfl_limit(g->c, g->R);
  g->spin_limit = default_spin_limit();
  set_shape(g, default_shape(g->R, g->Nx, g->Ny, g->Nz));
  g->base_shape = g->shape;
  g->auto_tile = true;

  fd_status st = FD_OK;
  if (d->stream) {
    g->stream = static_cast<cudaStream_t>(d->stream);
  } else {
    // blocking: ordered after work the caller queued on the legacy default stream
    e = cudaStreamCreateWithFlags(&g->stream, cudaStreamDefault);
    if (e) st = cuda_fail(e, "stream create");
    g->own_stream = true;
  }
  for (int b = 0; b < 2 && !st; ++b) {
    e = dev_alloc(reinterpret_cast<void**>(&g->F.u[b]), g->ncell * 4);
    if (e) st = cuda_fail(e, "wavefield allocation");
  }
  if (!st) {
    e = dev_alloc(reinterpret_cast<void**>(&g->A), g->ncell * 4);
    if (e) st = cuda_fail(e, "model allocation");
  }
  if (!st) {
    e = dev_alloc(reinterpret_cast<void**>(&g->d_err), 64);
    if (e) st = cuda_fail(e, "status allocation");
  }
  if (!st) {
    e = cudaMemsetAsync(g->d_err, 0, 64, g->stream);
    for (int b = 0; b < 2 && !e; ++b) e = cudaMemsetAsync(g->F.u[b], 0, g->ncell * 4, g->stream);
    if (!e) e = cudaMemsetAsync(g->A, 0, g->ncell * 4, g->stream);
    if (!e) e = cudaEventCreate(&g->ev0);
    if (!e) e = cudaEventCreate(&g->ev1);
    if (!e) e = cudaStreamSynchronize(g->stream);
    if (e) st = cuda_fail(e, "grid initialisation");
  }
  if (!st) st = build_maps(g);
  if (st) {
    std::string keep = t_err;
    fd_destroy_grid(g);
    t_err = keep;
    return st;
  }
  *out = g;
  return FD_OK;
}

fd_status fd_destroy_grid(fd_grid g) {
  if (!g) return FD_OK;
  cudaSetDevice(g->d.device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  decomp_destroy(g);
  cart_destroy(g);
  tblock_destroy(g);
  if (g->graph_valid) cudaGraphExecDestroy(g->gexec);
  for (int b = 0; b < 2; ++b) {
    if (g->F.u[b]) cudaFree(g->F.u[b]);
    if (g->Z.u[b]) cudaFree(g->Z.u[b]);
  }
  if (g->A) cudaFree(g->A);
  if (g->coef) cudaFree(g->coef);
  if (g->table) cudaFree(g->table);
  if (g->d_err) cudaFree(g->d_err);
  for (DevBuf* b : {&g->tab.inj_start, &g->tab.inj, &g->tab.rec_start, &g->tab.recs,
                    &g->tab_adj.inj_start, &g->tab_adj.inj, &g->tab_adj.rec_start,
                    &g->tab_adj.recs,
                    &g->stage_val, &g->stage_rec, &g->stage_aux, &g->ckpt, &g->ebuf,
                    &g->gpad, &g->resid, &g->recbuf, &g->desc, &g->sched})
    b->release();
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return FD_OK;
}

fd_status fd_set_model(fd_grid g, const float* data, int32_t kind) {
  clear_error();
  if (!g || !data) return fail(FD_ERR_ARG, "null argument");
  if (kind != FD_MODEL_VP_KMS && kind != FD_MODEL_M) return fail(FD_ERR_ARG, "bad model kind");
  cudaSetDevice(g->d.device);
  const size_t np = size_t(g->d.nx) * g->d.ny * g->d.nz;
  const float* dev = data;
  cudaError_t e;
  if (!is_device_ptr(data)) {
    // stage through the second wavefield (it is reset below)
    e = cudaMemcpyAsync(g->F.u[1], data, np * 4, cudaMemcpyHostToDevice, g->stream);
    if (e) return cuda_fail(e, "model upload");
    dev = g->F.u[1];
  }
  float vmin = 0, vmax = 0;
  int nbad = 0;
  e = model_stats(dev, np, kind, &vmin, &vmax, &nbad,
                  reinterpret_cast<unsigned int*>(g->d_err + 4), g->stream);
  if (e) return cuda_fail(e, "model statistics");
  if (nbad) return fail(FD_ERR_ARG, "%d model values are not positive and finite", nbad);
  const double courant = double(vmax) * g->d.dt / g->d.h;
  if (courant > g->cfl)
    return fail(FD_ERR_UNSTABLE, "v_max dt / h = %.4f exceeds the limit %.4f for SO %d",
                courant, g->cfl, g->d.space_order);
  e = model_to_A(dev, kind, g->d.nx, g->d.ny, g->d.nz, g->d.nbl, g->Nx, g->Ny, g->Nz,
                 g->pitch, g->d.dt * g->d.dt / (g->d.h * g->d.h), g->A, g->stream);
  if (e) return cuda_fail(e, "model set-up");
  g->vmin = vmin;
  g->vmax = vmax;
  if (g->d.nbl > 0) {
    const double gmax = 3.0 * double(vmax) * log(1000.0) / (2.0 * g->d.nbl * g->d.h);
    g->bscale = float(gmax * g->d.dt / 2.0 / (double(g->d.nbl) * g->d.nbl));
  } else {
    g->bscale = 0.0f;
  }
  for (int b = 0; b < 2; ++b) {
    e = cudaMemsetAsync(g->F.u[b], 0, g->ncell * 4, g->stream);
    if (e) return cuda_fail(e, "wavefield reset");
  }
  g->F.cur = 0;
  g->model_set = true;
  e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "model set-up");
  return FD_OK;
}

static fd_status propagate_impl(fd_grid g, int32_t n0, int32_t nsteps, const fd_points* src,
                                const float* wavelet, const fd_points* rec, float* rec_out) {
  if (!g->model_set) return fail(FD_ERR_STATE, "fd_set_model has not been called");
  if (n0 < 0 || nsteps < 0) return fail(FD_ERR_ARG, "negative step range");
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;
  if ((nsrc && (!src->xyz || !wavelet)) || (nrec && (!rec->xyz || !rec_out)))
    return fail(FD_ERR_ARG, "points given without their data array");
  // plain and table-weight forward runs take the tuner's pick (tile and
  // schedule) for the grid's size; per-cell weight fields keep the base tile
  fd_status st = use_shape(g, !g->dmp && !g->cart && forward_mode(g) != kModePerCell);
  if (st) return st;
  if (g->dmp) return decomp_propagate(g, n0, nsteps, src, wavelet, rec, rec_out);
  if (g->cart) return cart_propagate(g, n0, nsteps, src, wavelet, rec, rec_out);
  st = upload_tables(g, src, 1.0 / g->d.h, rec, g->tab);
  if (st) return st;
  const float* dval = nullptr;
  float* drec = nullptr;
  if ((st = stage_in(g, g->stage_val, nsrc ? wavelet : nullptr, size_t(n0 + nsteps) * nsrc,
                     &dval)))
    return st;
  if ((st = stage_out(g, g->stage_rec, nrec ? rec_out : nullptr, size_t(nsteps) * nrec,
                      &drec)))
    return st;
  if (tblock_eligible(g) && nsteps >= 2) {
    // two steps per pass (temporal blocking), fd_tblock.cu
    if ((st = tblock_propagate(g, n0, nsteps, src, dval, rec, drec))) return st;
  } else {
  RunSpec rs;
  memset(&rs, 0, sizeof(rs));
  rs.f = &g->F;
  rs.allow_graph = 1;
  rs.mode = kModeForward;
  rs.nsteps = nsteps;
  if (nsrc) {
    rs.inj_start = static_cast<const int32_t*>(g->tab.inj_start.p);
    rs.inj = static_cast<const InjEntry*>(g->tab.inj.p);
    rs.inj_val = dval;
    rs.inj_ncol = nsrc;
    rs.inj_row0 = n0;
    rs.inj_row_step = 1;
  }
  if (nrec) {
    rs.rec_start = static_cast<const int32_t*>(g->tab.rec_start.p);
    rs.recs = static_cast<const RecEntry*>(g->tab.recs.p);
    rs.rec_out = drec;
    rs.rec_ncol = nrec;
    rs.rec_row0 = 0;
    rs.rec_row_step = 1;
  }
  if ((st = run_steps(g, rs))) return st;
  }
  if ((st = check_device_error(g))) return st;
  if (nrec) {
    if ((st = check_finite(g, drec, size_t(nsteps) * nrec))) return st;
    if ((st = finish_out(g, rec_out, drec, size_t(nsteps) * nrec))) return st;
  }
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "stream synchronize");
  return FD_OK;
}

fd_status fd_propagate(fd_grid g, int32_t n0, int32_t nsteps, const fd_points* src,
                       const float* wavelet, const fd_points* rec, float* rec_out) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(g->d.device);
  return propagate_impl(g, n0, nsteps, src, wavelet, rec, rec_out);
}

fd_status fd_forward(fd_grid g, const fd_points* src, const float* wavelet,
                     const fd_points* rec, float* rec_out, float* u_out) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(g->d.device);
  if (!g->model_set) return fail(FD_ERR_STATE, "fd_set_model has not been called");
  cudaError_t e;
  for (int b = 0; b < 2; ++b) {
    e = cudaMemsetAsync(g->F.u[b], 0, g->ncell * 4, g->stream);
    if (e) return cuda_fail(e, "wavefield reset");
  }
  g->F.cur = 0;
  // plain and table-weight forward runs of grids left on the default tile
  // are tuned once (on the grid's own kernel), on the zeroed wavefields,
  // which are cleared again afterwards
  if (g->auto_tile && !g->tuned && g->sched_mode == FD_SCHED_AUTO && !g->dmp && !g->cart &&
      forward_mode(g) != kModePerCell && g->d.nt >= kTuneMinSteps && g->debug_skip_plane < 0) {
    fd_status st = autotune_grid(g);
    if (st) return st;
    for (int b = 0; b < 2; ++b) {
      e = cudaMemsetAsync(g->F.u[b], 0, g->ncell * 4, g->stream);
      if (e) return cuda_fail(e, "wavefield reset");
    }
    g->F.cur = 0;
  }
  fd_status st = propagate_impl(g, 0, g->d.nt, src, wavelet, rec, rec_out);
  if (st) return st;
  if (u_out) {
    if ((st = copy_field(g, g->F.u[g->F.cur], u_out, FD_REGION_PHYSICAL, true))) return st;
    e = cudaStreamSynchronize(g->stream);
    if (e) return cuda_fail(e, "wavefield copy");
  }
  return FD_OK;
}

fd_status fd_set_wavefield(fd_grid g, const float* u_prev, const float* u_cur, int32_t region) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (region != FD_REGION_PHYSICAL && region != FD_REGION_PADDED)
    return fail(FD_ERR_ARG, "bad region");
  cudaSetDevice(g->d.device);
  fd_status st;
  if (u_prev &&
      (st = copy_field(g, g->F.u[g->F.cur ^ 1], const_cast<float*>(u_prev), region, false)))
    return st;
  if (u_cur && (st = copy_field(g, g->F.u[g->F.cur], const_cast<float*>(u_cur), region, false)))
    return st;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "wavefield copy");
  return FD_OK;
}

fd_status fd_get_wavefield(fd_grid g, float* u_prev, float* u_cur, int32_t region) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (region != FD_REGION_PHYSICAL && region != FD_REGION_PADDED)
    return fail(FD_ERR_ARG, "bad region");
  cudaSetDevice(g->d.device);
  fd_status st;
  if (u_prev && (st = copy_field(g, g->F.u[g->F.cur ^ 1], u_prev, region, true))) return st;
  if (u_cur && (st = copy_field(g, g->F.u[g->F.cur], u_cur, region, true))) return st;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "wavefield copy");
  return FD_OK;
}

fd_status fd_get_info(fd_grid g, fd_grid_info* info) {
  clear_error();
  if (!g || !info) return fail(FD_ERR_ARG, "null argument");
  info->nx_pad = g->Nx;
  info->ny_pad = g->Ny;
  info->nz_pad = g->Nz;
  info->pitch = g->pitch;
  info->tile_x = 4 * g->shape.tx;
  info->tile_y = g->shape.ty;
  info->ctas = sweep_ctas(g->R, g->shape, forward_mode(g));
  info->v_max = g->vmax;
  info->cfl_limit = g->cfl;
  info->launches = g_launches.load();
  info->step_ms = g->step_ms;
  info->steps_timed = g->steps_timed;
  info->schedule = g->last_sched;
  return FD_OK;
}

static fd_status ensure_coef(fd_grid g) {
  if (g->coef) return FD_OK;
  cudaError_t e = dev_alloc(reinterpret_cast<void**>(&g->coef), size_t(g->R) * g->ncell * 4);
  if (e) return cuda_fail(e, "coefficient allocation");
  return build_maps(g);
}

fd_status fd_set_coefficients(fd_grid g, const float* c, int32_t mode) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(g->d.device);
  g->graph_valid = false;
  g->table_mode = false;
  g->tuned = false;  // the tuner's pick is per kernel mode: picked again
  if (mode == FD_COEF_TAYLOR) {
    fd_weights(g->R, g->c);
    g->percell = false;
    return FD_OK;
  }
  if (!c) return fail(FD_ERR_ARG, "coefficients required");
  if (mode == FD_COEF_UNIFORM) {
    float h[kMaxR + 1];
    cudaError_t e = cudaMemcpy(h, c, sizeof(float) * (g->R + 1), cudaMemcpyDefault);
    if (e) return cuda_fail(e, "coefficient read");
    for (int j = 0; j <= g->R; ++j) g->c[j] = h[j];
    g->percell = false;
    return FD_OK;
  }
  if (mode != FD_COEF_PER_CELL) return fail(FD_ERR_ARG, "bad coefficient mode");
  if (g->R != 4) return fail(FD_ERR_ARG, "per-cell weights are compiled for space order 8");
  fd_status st = ensure_coef(g);
  if (st) return st;
  const size_t np = size_t(g->d.nx) * g->d.ny * g->d.nz;
  const float* dev = nullptr;
  if ((st = stage_in(g, g->stage_aux, c, np * g->R, &dev))) return st;
  cudaError_t e = pad_coefficients(dev, g->R, g->d.nx, g->d.ny, g->d.nz, g->d.nbl, g->Nx, g->Ny,
                                   g->Nz, g->pitch, g->ncell, g->coef, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "coefficient set-up");
  g->percell = true;
  return FD_OK;
}

fd_status fd_set_learned_coefficients(fd_grid g, fd_mlp net, double f_hz) {
  clear_error();
  if (!g || !net) return fail(FD_ERR_ARG, "null argument");
  if (g->R != 4) return fail(FD_ERR_ARG, "the network predicts space-order-8 weights");
  if (!g->model_set) return fail(FD_ERR_STATE, "fd_set_model has not been called");
  cudaSetDevice(g->d.device);
  fd_status st = ensure_coef(g);
  if (st) return st;
  st = mlp_grid_coefficients(net, g->A, g->ncell, g->pitch, g->Nx, g->d.h, g->d.dt, f_hz,
                             g->coef, g->stream);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "learned coefficients");
  g->percell = true;
  g->table_mode = false;
  g->graph_valid = false;
  g->tuned = false;
  return FD_OK;
}

fd_status fd_set_learned_table(fd_grid g, fd_mlp net, double f_hz, int32_t nodes) {
  clear_error();
  if (!g || !net) return fail(FD_ERR_ARG, "null argument");
  if (g->R != 4) return fail(FD_ERR_ARG, "the network predicts space-order-8 weights");
  if (nodes < 2 || nodes > kTableNodes)
    return fail(FD_ERR_ARG, "table nodes must be in [2, %d]", kTableNodes);
  if (!g->model_set) return fail(FD_ERR_STATE, "fd_set_model has not been called");
  cudaSetDevice(g->d.device);
  if (!g->table) {
    cudaError_t e =
        dev_alloc(reinterpret_cast<void**>(&g->table), 2 * kTableNodes * sizeof(float4));
    if (e) return cuda_fail(e, "table allocation");
  }
  // nodes evenly spaced in A = C^2 over the model's Courant numbers
  // C = v dt / h; the network sees C_i = sqrt(A_i)
  const double clo = g->vmin * g->d.dt / g->d.h, chi = g->vmax * g->d.dt / g->d.h;
  const double alo = clo * clo, ahi = chi * chi;
  std::vector<float> feat(size_t(nodes) * 4), coef(size_t(nodes) * 4);
  for (int i = 0; i < nodes; ++i) {
    feat[4 * i + 0] = float(std::sqrt(alo + (ahi - alo) * i / (nodes - 1)));
    feat[4 * i + 1] = float(g->d.h / 10.0);
    feat[4 * i + 2] = float(g->d.dt / 1.0);
    feat[4 * i + 3] = float(f_hz / 10.0);
  }
  fd_status st = fd_mlp_coefficients(net, nodes, feat.data(), coef.data());
  if (st) return st;
  // per node: the weights and the step to the next node (zero at the last)
  std::vector<float> tab(size_t(nodes) * 8);
  for (int i = 0; i < nodes; ++i) {
    for (int j = 0; j < 4; ++j) {
      tab[8 * i + j] = coef[4 * i + j];
      tab[8 * i + 4 + j] = i + 1 < nodes ? coef[4 * (i + 1) + j] - coef[4 * i + j] : 0.0f;
    }
  }
  cudaError_t e = cudaMemcpyAsync(g->table, tab.data(), tab.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "table upload");
  g->tab_nodes = nodes;
  g->tab_lo = float(alo);
  g->tab_inv = ahi > alo ? float((nodes - 1) / (ahi - alo)) : 0.0f;
  g->table_mode = true;
  g->percell = false;
  g->graph_valid = false;
  g->tuned = false;
  return FD_OK;
}

fd_status fd_set_tile(fd_grid g, int32_t tile_x, int32_t tile_y, int32_t ctas) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (ctas < 0) return fail(FD_ERR_ARG, "ctas must be >= 0");
  for (int i = 0; i < kNumShapes; ++i) {
    if (4 * kShapes[i].tx == tile_x && kShapes[i].ty == tile_y) {
      cudaSetDevice(g->d.device);
      TileShape t = kShapes[i];
      t.ctas = ctas;
      set_shape(g, t);
      g->base_shape = t;
      g->auto_tile = false;
      g->tuned = false;
      return build_maps(g);
    }
  }
  return fail(FD_ERR_ARG, "tile %dx%d is not compiled", tile_x, tile_y);
}

fd_status fd_set_schedule(fd_grid g, int32_t mode) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (mode != FD_SCHED_AUTO && mode != FD_SCHED_SHARES && mode != FD_SCHED_WAVES &&
      mode != FD_SCHED_TEMPORAL)
    return fail(FD_ERR_ARG, "bad schedule %d", mode);
  g->sched_mode = mode;
  g->graph_valid = false;
  return FD_OK;
}

fd_status fd_set_debug(fd_grid g, int32_t key, int64_t value) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  switch (key) {
    case FD_DEBUG_SKIP_PLANE:
      g->debug_skip_plane = value < 0 ? -1 : int(value);
      return FD_OK;
    case FD_DEBUG_SPIN_LIMIT:
      if (value <= 0) return fail(FD_ERR_ARG, "spin limit must be positive");
      g->spin_limit = value;
      return FD_OK;
    case FD_DEBUG_NO_GRAPH:
      g->no_graph = value != 0;
      return FD_OK;
  }
  return fail(FD_ERR_ARG, "unknown debug key %d", key);
}

fd_status fd_set_profiling(fd_grid g, int32_t enabled) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  g->profiling = enabled != 0;
  g->step_ms = 0.0;
  g->steps_timed = 0;
  return FD_OK;
}

}  // extern "C"
