// Batched multi-shot forward modelling: every time step of all shots is one
// persistent launch over a shared work list, and the nt launches are captured
// in one CUDA graph.  A tile autotuner times the compiled tile shapes on the
// actual batch once per (GPU, space order, window sizes) and caches the pick
// in memory and, if FD_AUTOTUNE_CACHE names a file, on disk.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fd_aux.h"
#include "fd_runtime.h"

using namespace fd;

namespace {

struct BatchWorkspace {
  DevBuf shots, work, counters;
  bool graph_valid = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<char> key;
};

std::mutex g_mu;
std::map<int, BatchWorkspace> g_ws;           // per device
std::map<std::string, TileShape> g_tuned;     // autotuner picks

cudaError_t launch_batch(int R, const TileShape& t, const BatchShot* shots, const int4* work,
                         int nwork, int* counter, int step, int grid, cudaStream_t s) {
  count_launch();
  switch (R) {
    case 1: return launch_batch_r<1>(t, shots, work, nwork, counter, step, grid, s);
    case 2: return launch_batch_r<2>(t, shots, work, nwork, counter, step, grid, s);
    case 3: return launch_batch_r<3>(t, shots, work, nwork, counter, step, grid, s);
    case 4: return launch_batch_r<4>(t, shots, work, nwork, counter, step, grid, s);
    case 5: return launch_batch_r<5>(t, shots, work, nwork, counter, step, grid, s);
    case 6: return launch_batch_r<6>(t, shots, work, nwork, counter, step, grid, s);
    case 7: return launch_batch_r<7>(t, shots, work, nwork, counter, step, grid, s);
    case 8: return launch_batch_r<8>(t, shots, work, nwork, counter, step, grid, s);
  }
  return cudaErrorInvalidValue;
}

int blocks_per_sm(int R, const TileShape& t) {
  switch (R) {
    case 1: return batch_blocks_per_sm_r<1>(t);
    case 2: return batch_blocks_per_sm_r<2>(t);
    case 3: return batch_blocks_per_sm_r<3>(t);
    case 4: return batch_blocks_per_sm_r<4>(t);
    case 5: return batch_blocks_per_sm_r<5>(t);
    case 6: return batch_blocks_per_sm_r<6>(t);
    case 7: return batch_blocks_per_sm_r<7>(t);
    case 8: return batch_blocks_per_sm_r<8>(t);
  }
  return 0;
}

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
  std::string k = std::string(p.name) + "|R" + std::to_string(R);
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
  char key[4096];
  TileShape t;
  while (fscanf(f, "%4095s %d %d %d %d", key, &t.tx, &t.ty, &t.pf, &t.zsplit) == 5)
    g_tuned[key] = t;
  fclose(f);
}

void save_cache_entry(const std::string& key, const TileShape& t) {
  const char* path = getenv("FD_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d\n", key.c_str(), t.tx, t.ty, t.pf, t.zsplit);
  fclose(f);
}

struct Prepared {
  std::vector<BatchShot> hs;
  std::vector<int4> work;
  std::vector<float*> drec;
  int nwork = 0;
  int grid = 0;
};

// Puts every shot on tile shape t and builds the device descriptors and the
// longest-first work list.
fd_status prepare(int nshots, const fd_shot* shots, const TileShape& t, Prepared& P) {
  const int R = shots[0].grid->R;
  P.hs.assign(nshots, BatchShot());
  P.drec.assign(nshots, nullptr);
  std::vector<std::pair<int, int4>> items;
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    const TileShape old = g->shape;
    if (old.tx != t.tx || old.ty != t.ty || old.pf != t.pf || old.zsplit != t.zsplit) {
      TileShape tt = t;
      tt.zsplit = std::min(t.zsplit, g->Nz);
      set_shape(g, tt);
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
    BatchShot& b = P.hs[i];
    memset(&b, 0, sizeof(b));
    for (int k = 0; k < 2; ++k) {
      b.halo[k] = g->F.halo[k];
      b.tile[k] = g->F.tile[k];
      b.u[k] = g->F.u[k];
    }
    b.A = g->mapA;
    b.args = base_args(g);
    if (nsrc) {
      b.args.inj_start = static_cast<const int32_t*>(g->tab.inj_start.p);
      b.args.inj = static_cast<const InjEntry*>(g->tab.inj.p);
      b.args.inj_val = dval;
      b.args.inj_ncol = nsrc;
    }
    if (nrec) {
      b.args.rec_start = static_cast<const int32_t*>(g->tab.rec_start.p);
      b.args.recs = static_cast<const RecEntry*>(g->tab.recs.p);
      b.args.rec_out = drec;
      b.args.rec_ncol = nrec;
    }
    for (int zc = 0; zc < g->shape.zsplit; ++zc) {
      const int zl = std::min(g->Nz, (zc + 1) * g->zlen) - zc * g->zlen;
      if (zl <= 0) continue;
      for (int ty = 0; ty < g->tiles_y; ++ty)
        for (int tx = 0; tx < g->tiles_x; ++tx)
          items.push_back({zl + 2 * R, make_int4(i, tx, ty, zc)});
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const auto& a, const auto& b) { return a.first > b.first; });
  P.work.clear();
  for (auto& it : items) P.work.push_back(it.second);
  P.nwork = int(P.work.size());
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = std::max(1, blocks_per_sm(R, t));
  P.grid = std::max(1, std::min(P.nwork, per * sms));
  return FD_OK;
}

fd_status upload_prepared(BatchWorkspace& ws, const Prepared& P, int nt, cudaStream_t s) {
  cudaError_t e = ws.shots.ensure(P.hs.size() * sizeof(BatchShot));
  if (!e) e = ws.work.ensure(std::max<size_t>(P.work.size() * sizeof(int4), 16));
  if (!e) e = ws.counters.ensure(size_t(std::max(nt, 1)) * sizeof(int));
  if (e) return cuda_fail(e, "batch workspace allocation");
  e = cudaMemcpyAsync(ws.shots.p, P.hs.data(), P.hs.size() * sizeof(BatchShot),
                      cudaMemcpyHostToDevice, s);
  if (!e && !P.work.empty())
    e = cudaMemcpyAsync(ws.work.p, P.work.data(), P.work.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "batch workspace upload");
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
  cudaError_t e = cudaMemsetAsync(ws.counters.p, 0, size_t(nsteps) * sizeof(int), s);
  if (e) return cuda_fail(e, "counter reset");
  for (int step = 0; step < nsteps; ++step) {
    e = launch_batch(R, t, static_cast<const BatchShot*>(ws.shots.p),
                     static_cast<const int4*>(ws.work.p), P.nwork,
                     static_cast<int*>(ws.counters.p) + step, step, P.grid, s);
    if (e) return cuda_fail(e, "batch launch");
  }
  return FD_OK;
}

fd_status autotune(BatchWorkspace& ws, int nshots, const fd_shot* shots, int R, int nt,
                   cudaStream_t s, TileShape* best) {
  const int trial = std::max(1, std::min(nt, 6));
  float best_ms = 1e30f;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int i = 0; i < kNumShapes; ++i) {
    for (int zs : {1, 2}) {
      TileShape t = kShapes[i];
      t.zsplit = zs;
      Prepared P;
      fd_status st = prepare(nshots, shots, t, P);
      if (!st) st = upload_prepared(ws, P, nt, s);
      if (!st) st = zero_state(nshots, shots, s);
      if (!st) st = issue_steps(ws, P, R, t, 1, s);  // warm-up
      if (st) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return st;
      }
      cudaEventRecord(a, s);
      st = issue_steps(ws, P, R, t, trial, s);
      cudaEventRecord(b, s);
      if (st || cudaEventSynchronize(b)) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return st ? st : fail(FD_ERR_CUDA, "autotune timing failed");
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best_ms) {
        best_ms = ms;
        *best = t;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return FD_OK;
}

}  // namespace

extern "C" fd_status fd_batch_forward(int32_t nshots, const fd_shot* shots, int32_t flags) {
  clear_error();
  if (nshots < 1 || !shots) return fail(FD_ERR_ARG, "no shots");
  fd_grid g0 = shots[0].grid;
  for (int i = 0; i < nshots; ++i) {
    fd_grid g = shots[i].grid;
    if (!g) return fail(FD_ERR_ARG, "shot %d has no grid", i);
    if (!g->model_set) return fail(FD_ERR_STATE, "shot %d has no model", i);
    if (g->percell) return fail(FD_ERR_STATE, "shot %d uses per-cell weights", i);
    if (g->d.device != g0->d.device || g->R != g0->R || g->d.nt != g0->d.nt)
      return fail(FD_ERR_ARG, "shots must share device, space order and nt");
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
  TileShape t = default_shape(R, g0->Nx, g0->Ny, g0->Nz);
  load_cache_file();
  const std::string key = tune_key(g0->d.device, R, nshots, shots);
  auto it = g_tuned.find(key);
  fd_status st;
  if (it != g_tuned.end()) {
    t = it->second;
  } else if (flags & FD_BATCH_AUTOTUNE) {
    if ((st = autotune(ws, nshots, shots, R, nt, s, &t))) return st;
    g_tuned[key] = t;
    save_cache_entry(key, t);
    ws.graph_valid = false;
  }

  Prepared P;
  if ((st = prepare(nshots, shots, t, P))) return st;
  if ((st = upload_prepared(ws, P, nt, s))) return st;
  if ((st = zero_state(nshots, shots, s))) return st;

  const bool use_graph = (flags & FD_BATCH_GRAPH) && nt >= 2;
  // the graph depends on the launch shape and the workspace pointers only;
  // descriptors live in device memory and were just refreshed
  std::vector<char> key_bytes(sizeof(TileShape) + 4 * sizeof(int) + 3 * sizeof(void*));
  {
    char* q = key_bytes.data();
    memcpy(q, &t, sizeof(t));
    q += sizeof(t);
    int ints[4] = {R, nt, P.nwork, P.grid};
    memcpy(q, ints, sizeof(ints));
    q += sizeof(ints);
    void* ptrs[3] = {ws.shots.p, ws.work.p, ws.counters.p};
    memcpy(q, ptrs, sizeof(ptrs));
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
    // every grid's error word is written on stream s
    std::swap(g->stream, s);
    st = check_device_error(g);
    const int nrec = shots[i].rec ? shots[i].rec->n : 0;
    if (!st && nrec) st = check_finite(g, P.drec[i], size_t(nt) * nrec);
    if (!st && nrec) st = finish_out(g, shots[i].rec_out, P.drec[i], size_t(nt) * nrec);
    std::swap(g->stream, s);
    if (st) return st;
  }
  e = cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "stream synchronize");
  return FD_OK;
}
