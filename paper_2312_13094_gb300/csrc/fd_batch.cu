// Batched multi-shot forward modelling: every time step of all shots is one
// persistent sweep launch over the concatenated (shot, tile, plane) units of
// the batch, each resident CTA taking an equal contiguous share or running
// the items of a column-wave schedule (fd_sched.cu), and the nt launches are
// captured in one CUDA graph.  An autotuner times the compiled tile shapes
// under both schedules on the actual batch once per (GPU, space order, window
// sizes) and caches the pick in memory and, if FD_AUTOTUNE_CACHE names a
// file, on disk (the paper tunes loop blocking the same way, Sec. IV-C).
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fd_aux.h"
#include "fd_runtime.h"
#include "fd_sched.h"

using namespace fd;

namespace {

struct BatchWorkspace {
  DevBuf desc;  // ShotDesc[nshots] followed by the unit prefix [nshots + 1]
  bool graph_valid = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<char> key;
};

std::mutex g_mu;
std::map<int, BatchWorkspace> g_ws;        // per device
struct Pick {
  TileShape t;
  bool waves;  // wave schedule instead of equal shares
};
std::map<std::string, Pick> g_tuned;  // autotuner picks

std::string tune_key(int device, int R, int nshots, const fd_shot* shots) {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, device);
  std::vector<std::string> dims;
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    dims.push_back(std::to_string(g->Nx) + "x" + std::to_string(g->Ny) + "x" +
                   std::to_string(g->Nz));
  }
  std::sort(dims.begin(), dims.end());
  std::string k = std::string(p.name) + "|v2|R" + std::to_string(R);
  for (auto& d : dims) k += "|" + d;
  for (auto& c : k)
    if (c == ' ') c = '_';
  return k;
}

void load_cache_file() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = getenv("FD_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[8192], key[4096];
  TileShape t;
  int waves = 0;
  while (fgets(line, sizeof(line), f)) {
    if (sscanf(line, "%4095s %d %d %d %d %d", key, &t.tx, &t.ty, &t.pf, &t.ctas, &waves) == 6)
      g_tuned[key] = {t, waves != 0};
  }
  fclose(f);
}

void save_cache_entry(const std::string& key, const Pick& p) {
  const char* path = getenv("FD_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), p.t.tx, p.t.ty, p.t.pf, p.t.ctas,
          p.waves ? 1 : 0);
  fclose(f);
}

struct Prepared {
  std::vector<char> host;  // descriptors + prefix (+ wave schedule), as uploaded
  std::vector<float*> drec;
  int nshots = 0;
  int ctas = 0;
  bool waves = false;
  size_t off_start = 0, off_items = 0;  // wave schedule within `host`
  float c[kMaxR + 2] = {};  // stencil weights (the same for every shot; launch_weights)
  int nbl = 0;              // layer width (the same for every shot)
  long long spin_limit = 0;
};

// Puts every shot on tile shape t and builds the descriptors and the unit
// prefix of the batch.
fd_status prepare(int nshots, const fd_shot* shots, const TileShape& t, bool waves,
                  Prepared& P) {
  const int R = shots[0].grid->R;
  P.nshots = nshots;
  P.drec.assign(nshots, nullptr);
  P.host.assign(nshots * sizeof(ShotDesc) + (nshots + 1) * sizeof(long long), 0);
  ShotDesc* desc = reinterpret_cast<ShotDesc*>(P.host.data());
  long long* prefix = reinterpret_cast<long long*>(P.host.data() + nshots * sizeof(ShotDesc));
  prefix[0] = 0;
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    const TileShape old = g->shape;
    if (old.tx != t.tx || old.ty != t.ty || old.ctas != t.ctas) {
      set_shape(g, t);
      fd_status st = build_maps(g);
      if (st) return st;
    }
    const int nsrc = shots[i].src ? shots[i].src->n : 0;
    const int nrec = shots[i].rec ? shots[i].rec->n : 0;
    fd_status st = upload_tables(g, shots[i].src, 1.0 / g->d.h, shots[i].rec, g->tab);
    if (st) return st;
    const float* dval = nullptr;
    float* drec = nullptr;
    if ((st = stage_in(g, g->stage_val, nsrc ? shots[i].wavelet : nullptr,
                       size_t(g->d.nt) * nsrc, &dval)))
      return st;
    if ((st = stage_out(g, g->stage_rec, nrec ? shots[i].rec_out : nullptr,
                        size_t(g->d.nt) * nrec, &drec)))
      return st;
    P.drec[i] = drec;
    RunSpec rs;
    memset(&rs, 0, sizeof(rs));
    rs.f = &g->F;
    if (nsrc) {
      rs.inj_start = static_cast<const int32_t*>(g->tab.inj_start.p);
      rs.inj = static_cast<const InjEntry*>(g->tab.inj.p);
      rs.inj_val = dval;
      rs.inj_ncol = nsrc;
    }
    if (nrec) {
      rs.rec_start = static_cast<const int32_t*>(g->tab.rec_start.p);
      rs.recs = static_cast<const RecEntry*>(g->tab.recs.p);
      rs.rec_out = drec;
      rs.rec_ncol = nrec;
    }
    fill_desc(g, rs, &desc[i]);
    prefix[i + 1] = prefix[i] + (long long)g->tiles_x * g->tiles_y * g->Nz;
  }
  P.ctas = sweep_ctas(R, t, kModeForward);
  P.waves = waves;
  if (waves) {
    // taller windows first, so that a wave holds chunks of similar height
    std::vector<SchedGrid> grids;
    for (int i = 0; i < nshots; ++i) {
      fd_grid g = shots[i].grid;
      grids.push_back({i, g->tiles_x * g->tiles_y, g->Nz});
    }
    std::stable_sort(grids.begin(), grids.end(),
                     [](const SchedGrid& a, const SchedGrid& b) { return a.nz > b.nz; });
    std::vector<int32_t> start;
    std::vector<WorkItem> items;
    P.ctas = wave_schedule(grids, P.ctas, R, start, items);
    P.off_start = (P.host.size() + 15) / 16 * 16;
    P.off_items = (P.off_start + start.size() * 4 + 15) / 16 * 16;
    P.host.resize(P.off_items + items.size() * sizeof(WorkItem), 0);
    memcpy(P.host.data() + P.off_start, start.data(), start.size() * 4);
    memcpy(P.host.data() + P.off_items, items.data(), items.size() * sizeof(WorkItem));
  }
  fd_grid g0 = shots[0].grid;
  launch_weights(g0->c, R, P.c);
  P.spin_limit = g0->spin_limit;
  P.nbl = g0->d.nbl;
  return FD_OK;
}

fd_status upload_prepared(BatchWorkspace& ws, const Prepared& P, cudaStream_t s) {
  cudaError_t e = ws.desc.ensure(P.host.size());
  if (e) return cuda_fail(e, "batch descriptor allocation");
  e = cudaMemcpyAsync(ws.desc.p, P.host.data(), P.host.size(), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "batch descriptor upload");
  return FD_OK;
}

fd_status zero_state(int nshots, const fd_shot* shots, cudaStream_t s) {
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    for (int b = 0; b < 2; ++b) {
      cudaError_t e = cudaMemsetAsync(g->F.u[b], 0, g->ncell * 4, s);
      if (e) return cuda_fail(e, "wavefield reset");
    }
    g->F.cur = 0;
  }
  return FD_OK;
}

// Issues steps [0, nsteps) of the prepared batch on stream s.
fd_status issue_steps(BatchWorkspace& ws, const Prepared& P, int R, const TileShape& t,
                      int nsteps, cudaStream_t s) {
  const ShotDesc* d = static_cast<const ShotDesc*>(ws.desc.p);
  const long long* prefix = reinterpret_cast<const long long*>(
      static_cast<const char*>(ws.desc.p) + P.nshots * sizeof(ShotDesc));
  for (int step = 0; step < nsteps; ++step) {
    StepOverride ov;
    memset(&ov, 0, sizeof(ov));
    ov.cur = step & 1;
    ov.zfirst = 0;
    ov.nblz = P.nbl;
    ov.inj_row = step;
    ov.rec_row = step;
    ov.spin_limit = P.spin_limit;
    ov.debug_skip_plane = -1;
    for (int j = 0; j < kMaxR + 2; ++j) ov.c[j] = P.c[j];
    if (P.waves) {
      const char* base = static_cast<const char*>(ws.desc.p);
      ov.item_start = reinterpret_cast<const int32_t*>(base + P.off_start);
      ov.items = reinterpret_cast<const WorkItem*>(base + P.off_items);
    }
    cudaError_t e = launch_sweep(R, t, kModeForward, d, prefix, P.nshots, ov, P.ctas, s);
    if (e) return cuda_fail(e, "batch launch");
  }
  return FD_OK;
}

fd_status autotune(BatchWorkspace& ws, int nshots, const fd_shot* shots, int R, int nt,
                   cudaStream_t s, Pick* best) {
  const int trial = std::max(1, std::min(nt, 6));
  float best_ms = 1e30f;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fd_status st = FD_OK;
  for (int c = 0; c < 2 * kNumShapes && !st; ++c) {
    TileShape t = kShapes[c / 2];
    const bool waves = (c & 1) != 0;
    Prepared P;
    st = prepare(nshots, shots, t, waves, P);
    if (!st) st = upload_prepared(ws, P, s);
    if (!st) st = zero_state(nshots, shots, s);
    if (!st) st = issue_steps(ws, P, R, t, 1, s);  // warm-up
    if (st) break;
    cudaEventRecord(a, s);
    st = issue_steps(ws, P, R, t, trial, s);
    cudaEventRecord(b, s);
    if (st) break;
    if (cudaEventSynchronize(b) != cudaSuccess) {
      st = fail(FD_ERR_CUDA, "autotune timing failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best_ms) {
      best_ms = ms;
      *best = {t, waves};
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

}  // namespace

extern "C" fd_status fd_batch_forward(int32_t nshots, const fd_shot* shots, int32_t flags) {
  clear_error();
  if (nshots < 1 || !shots) return fail(FD_ERR_ARG, "no shots");
  fd_grid g0 = shots[0].grid;
  if (!g0) return fail(FD_ERR_ARG, "shot 0 has no grid");
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    if (!g) return fail(FD_ERR_ARG, "shot %d has no grid", i);
    if (!g->model_set) return fail(FD_ERR_STATE, "shot %d has no model", i);
    if (g->percell || g->table_mode)
      return fail(FD_ERR_STATE, "shot %d uses per-cell weights", i);
    for (int j = 0; j <= g->R && j <= g0->R; ++j)
      if (g->c[j] != g0->c[j]) return fail(FD_ERR_ARG, "shots must share stencil weights");
    if (g->d.device != g0->d.device || g->R != g0->R || g->d.nt != g0->d.nt ||
        g->d.nbl != g0->d.nbl)
      return fail(FD_ERR_ARG, "shots must share device, space order, nt and layer width");
    for (int j = 0; j < i; ++j)
      if (shots[j].grid == g) return fail(FD_ERR_ARG, "grid used by two shots");
    const int nsrc = shots[i].src ? shots[i].src->n : 0;
    const int nrec = shots[i].rec ? shots[i].rec->n : 0;
    if ((nsrc && (!shots[i].wavelet || !shots[i].src->xyz)) ||
        (nrec && (!shots[i].rec_out || !shots[i].rec->xyz)))
      return fail(FD_ERR_ARG, "shot %d: points given without their data array", i);
  }
  cudaSetDevice(g0->d.device);
  const int R = g0->R, nt = g0->d.nt;
  cudaStream_t s = g0->stream;
  std::lock_guard<std::mutex> lock(g_mu);
  BatchWorkspace& ws = g_ws[g0->d.device];

  // tile shape: autotuned (cached), else the single-grid default
  Pick pick = {default_shape(R, g0->Nx, g0->Ny, g0->Nz), g0->sched_mode == FD_SCHED_WAVES};
  load_cache_file();
  const std::string key = tune_key(g0->d.device, R, nshots, shots);
  auto it = g_tuned.find(key);
  fd_status st;
  if (it != g_tuned.end()) {
    pick = it->second;
  } else if (flags & FD_BATCH_AUTOTUNE) {
    if ((st = autotune(ws, nshots, shots, R, nt, s, &pick))) return st;
    g_tuned[key] = pick;
    save_cache_entry(key, pick);
  }
  const TileShape t = pick.t;

  Prepared P;
  if ((st = prepare(nshots, shots, t, pick.waves, P))) return st;
  if ((st = upload_prepared(ws, P, s))) return st;
  if ((st = zero_state(nshots, shots, s))) return st;

  const bool use_graph = (flags & FD_BATCH_GRAPH) && nt >= 2;
  // the captured launches depend on the shape, sizes and workspace address;
  // the descriptors are re-uploaded before each replay
  std::vector<char> key_bytes(sizeof(TileShape) + 4 * sizeof(int) + sizeof(void*));
  {
    char* q = key_bytes.data();
    memcpy(q, &t, sizeof(t));
    q += sizeof(t);
    int ints[4] = {R, nt, P.nshots, P.ctas * 2 + (P.waves ? 1 : 0)};
    memcpy(q, ints, sizeof(ints));
    q += sizeof(ints);
    memcpy(q, &ws.desc.p, sizeof(void*));
  }
  if (g0->profiling) cudaEventRecord(g0->ev0, s);
  cudaError_t e;
  if (use_graph) {
    if (!(ws.graph_valid && ws.key == key_bytes)) {
      if (ws.graph_valid) cudaGraphExecDestroy(ws.gexec);
      ws.graph_valid = false;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
      if (e) return cuda_fail(e, "stream capture");
      const long long before = fd_launch_count();
      st = issue_steps(ws, P, R, t, nt, s);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(s, &graph);
      count_launch(before - fd_launch_count());  // counted when the graph runs
      if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&ws.gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e) return cuda_fail(e, "graph instantiate");
      ws.graph_valid = true;
      ws.key = key_bytes;
    }
    e = cudaGraphLaunch(ws.gexec, s);
    if (e) return cuda_fail(e, "graph launch");
    count_launch(nt);
  } else {
    if ((st = issue_steps(ws, P, R, t, nt, s))) return st;
  }
  if (g0->profiling) {
    cudaEventRecord(g0->ev1, s);
    if ((e = cudaEventSynchronize(g0->ev1))) return cuda_fail(e, "profiling event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g0->ev0, g0->ev1);
    g0->step_ms += ms;
    g0->steps_timed += nt;
  }
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    g->F.cur = nt & 1;
    g->last_sched = pick.waves ? FD_SCHED_WAVES : FD_SCHED_SHARES;
    // every grid's error word and receivers were written on stream s
    cudaStream_t own = g->stream;
    g->stream = s;
    st = check_device_error(g);
    const int nrec = shots[i].rec ? shots[i].rec->n : 0;
    if (!st && nrec) st = check_finite(g, P.drec[i], size_t(nt) * nrec);
    if (!st && nrec) st = finish_out(g, shots[i].rec_out, P.drec[i], size_t(nt) * nrec);
    g->stream = own;
    if (st) return st;
  }
  e = cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "stream synchronize");
  return FD_OK;
}
