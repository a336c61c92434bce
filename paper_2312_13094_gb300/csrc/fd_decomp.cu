// Domain decomposition of one grid along z, on the device.
//
// Sec. III of the paper splits the grid into subdomains, one per rank, each
// exchanging an R-deep halo with its neighbours before the stencil reads it.
// Its "basic" mode exchanges synchronously before every step; its "full" mode
// computes the CORE points, whose stencils stay inside the subdomain, while
// the exchange is in flight, and the REMAINDER (the OWNED points next to a
// face) once the halo has arrived.  Both are built here for slabs along z.
//
// Layout.  Slab s owns the padded planes [z0, z0 + nloc) and keeps its two
// wavefields and its model term A in arrays of nloc + 2R planes (pitch and y
// extent of the whole grid): R ghost planes, the owned planes, R ghost planes.
// Ghost planes beyond the ends of the grid are zero and never written: the
// zero halo that the whole-grid kernel gets from the TMA unit's out-of-bounds
// fill.  Ghost planes between slabs receive the neighbour's edge planes.
// With x fastest an R-plane z face is one contiguous block, so the exchange
// is one device copy per face and direction, with no pack or unpack kernel.
//
// Step.  Each slab runs the whole-grid sweep kernel over a range of its array
// planes (launch parameters zfirst, the first updated array plane, and nblz,
// the layer width shifted into the slab's planes, so that the damping profile
// stays that of the whole grid):
//  * basic:   one launch per slab over its owned planes, then the copies that
//             refill every inner ghost plane with the new u^{n+1};
//  * overlap: per slab first the REMAINDER planes (the R owned planes beside
//             an inner face, whose stencils reach into the ghosts); the copies
//             of those planes then run on a second stream while the CORE
//             planes are computed on the first; the next step's remainder
//             waits for the copies.
// Every point goes through the same arithmetic as in the undecomposed run, so
// both give the same wavefields and receivers bit for bit.  All slabs live on
// the grid's device; across GPUs the copies would become peer copies.
#include <string.h>

#include <algorithm>
#include <vector>

#include "fd_aux.h"
#include "fd_runtime.h"

namespace fd {

struct Slab {
  int z0 = 0, nloc = 0;  // owned padded planes [z0, z0 + nloc)
  size_t ncell = 0;      // pitch * Ny * (nloc + 2R)
  Fields F;              // u^{n-1}, u^n with R ghost planes on either side
  float* A = nullptr;    // model term on the same planes (ghost planes unused)
  CUtensorMap mapA;
  Tables tab;            // source/receiver entries of the owned planes
};

// One launch: the owned planes [p0, p0 + cnt) of slab s (p0 counted from the
// slab's first owned plane).
struct Part {
  int s, p0, cnt;
};

struct Decomp {
  int nsub = 1, mode = FD_DMP_BASIC;
  std::vector<Slab> slab;
  TileShape shape = {};      // tile the maps were built for
  std::vector<Part> before;  // launches of a step before the exchange is issued
  std::vector<Part> after;   // launches after it (overlap: the CORE planes)
  DevBuf desc;               // per part: ShotDesc + unit prefix, kBlock bytes
  cudaStream_t side = nullptr;  // overlap: the exchange stream
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool graph_valid = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<char> gkey;
  long long graph_launches = 0;  // kernel launches of one replay
};

namespace {

constexpr size_t kBlock = (sizeof(ShotDesc) + 2 * sizeof(long long) + 127) / 128 * 128;

size_t plane_floats(fd_grid g) { return size_t(g->pitch) * g->Ny; }

fd_status build_slab_maps(fd_grid g, Slab& sl) {
  const int bx = 4 * g->shape.tx, by = g->shape.ty;
  const int W = bx + 2 * radius_halo_x(g->R), H = by + 2 * g->R;
  const int Nza = sl.nloc + 2 * g->R;
  for (int b = 0; b < 2; ++b) {
    fd_status st = make_map(&sl.F.halo[b], sl.F.u[b], g->Nx, g->Ny, Nza, g->pitch, W, H);
    if (!st) st = make_map(&sl.F.tile[b], sl.F.u[b], g->Nx, g->Ny, Nza, g->pitch, bx, by);
    if (st) return st;
  }
  return make_map(&sl.mapA, sl.A, g->Nx, g->Ny, Nza, g->pitch, bx, by);
}

void release(fd_grid g, Decomp* d) {
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (d->side) cudaStreamSynchronize(d->side);
  for (Slab& sl : d->slab) {
    for (int b = 0; b < 2; ++b)
      if (sl.F.u[b]) cudaFree(sl.F.u[b]);
    if (sl.A) cudaFree(sl.A);
    for (DevBuf* b : {&sl.tab.inj_start, &sl.tab.inj, &sl.tab.rec_start, &sl.tab.recs})
      b->release();
  }
  d->desc.release();
  if (d->graph_valid) cudaGraphExecDestroy(d->gexec);
  if (d->ev_fork) cudaEventDestroy(d->ev_fork);
  if (d->ev_join) cudaEventDestroy(d->ev_join);
  if (d->side) cudaStreamDestroy(d->side);
  delete d;
}

// Per-slab entry lists: the whole-grid lists of each tile restricted to the
// slab's owned planes, with z moved to the slab's array planes.
template <class E>
void split_entries(const std::vector<int32_t>& start, const std::vector<E>& ent, int ntiles,
                   int zlo, int zhi, int zshift, std::vector<int32_t>& st_out,
                   std::vector<E>& out) {
  st_out.assign(ntiles + 1, 0);
  out.clear();
  for (int t = 0; t < ntiles; ++t) {
    for (int i = start[t]; i < start[t + 1]; ++i) {
      if (ent[i].z < zlo || ent[i].z >= zhi) continue;
      E e = ent[i];
      e.z -= zshift;
      out.push_back(e);
      st_out[t + 1]++;
    }
  }
  for (int t = 0; t < ntiles; ++t) st_out[t + 1] += st_out[t];
}

template <class T>
fd_status upload_vec(fd_grid g, DevBuf& buf, const std::vector<T>& v) {
  cudaError_t e = buf.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
  if (e) return cuda_fail(e, "slab table allocation");
  if (!v.empty()) {
    e = cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                        g->stream);
    if (e) return cuda_fail(e, "slab table upload");
  }
  return FD_OK;
}

fd_status upload_slab_tables(fd_grid g, Decomp* d, const fd_points* src, const fd_points* rec) {
  std::vector<int32_t> is, rs;
  std::vector<InjEntry> ie;
  std::vector<RecEntry> re;
  fd_status st = build_injection(g, src, 1.0 / g->d.h, is, ie);
  if (!st) st = build_receivers(g, rec, rs, re);
  if (st) return st;
  const int ntiles = g->tiles_x * g->tiles_y;
  const int nsub = int(d->slab.size());
  std::vector<std::vector<int32_t>> s_is(nsub), s_rs(nsub);
  std::vector<std::vector<InjEntry>> s_ie(nsub);
  std::vector<std::vector<RecEntry>> s_re(nsub);
  for (int s = 0; s < nsub && !st; ++s) {
    Slab& sl = d->slab[s];
    const int shift = sl.z0 - g->R;  // padded z of array plane 0
    split_entries(is, ie, ntiles, sl.z0, sl.z0 + sl.nloc, shift, s_is[s], s_ie[s]);
    split_entries(rs, re, ntiles, sl.z0, sl.z0 + sl.nloc, shift, s_rs[s], s_re[s]);
    if (!st) st = upload_vec(g, sl.tab.inj_start, s_is[s]);
    if (!st) st = upload_vec(g, sl.tab.inj, s_ie[s]);
    if (!st) st = upload_vec(g, sl.tab.rec_start, s_rs[s]);
    if (!st) st = upload_vec(g, sl.tab.recs, s_re[s]);
  }
  // keep the uploads ordered before the host vectors go away
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (!st && e) st = cuda_fail(e, "slab table upload");
  return st;
}

cudaError_t copy_planes(float* dst, const float* src, size_t planes, size_t plane,
                        cudaStream_t s) {
  if (planes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, planes * plane * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

// Whole-grid state and model term -> slabs: owned planes plus the in-grid
// ghost planes of both wavefields, owned planes of A.
fd_status scatter(fd_grid g, Decomp* d) {
  const size_t pl = plane_floats(g);
  const int R = g->R;
  for (Slab& sl : d->slab) {
    const int zlo = std::max(0, sl.z0 - R), zhi = std::min(g->Nz, sl.z0 + sl.nloc + R);
    const size_t dst0 = size_t(zlo - (sl.z0 - R)) * pl;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && !e; ++b)
      e = copy_planes(sl.F.u[b] + dst0, g->F.u[b] + size_t(zlo) * pl, zhi - zlo, pl, g->stream);
    if (!e) e = copy_planes(sl.A + size_t(R) * pl, g->A + size_t(sl.z0) * pl, sl.nloc, pl,
                            g->stream);
    if (e) return cuda_fail(e, "slab scatter");
  }
  return FD_OK;
}

// Slabs -> whole-grid state (owned planes of both wavefields).
fd_status gather(fd_grid g, Decomp* d) {
  const size_t pl = plane_floats(g);
  for (Slab& sl : d->slab) {
    for (int b = 0; b < 2; ++b) {
      cudaError_t e = copy_planes(g->F.u[b] + size_t(sl.z0) * pl, sl.F.u[b] + size_t(g->R) * pl,
                                  sl.nloc, pl, g->stream);
      if (e) return cuda_fail(e, "slab gather");
    }
  }
  return FD_OK;
}

// The exchange after a step wrote buffer nb: across every inner face the
// lower slab's top R owned planes become the upper slab's lower ghosts and
// the upper slab's first R owned planes the lower slab's upper ghosts.
cudaError_t exchange(fd_grid g, Decomp* d, int nb, cudaStream_t s) {
  const size_t pl = plane_floats(g);
  const int R = g->R;
  for (size_t i = 0; i + 1 < d->slab.size(); ++i) {
    Slab& lo = d->slab[i];
    Slab& hi = d->slab[i + 1];
    cudaError_t e = copy_planes(hi.F.u[nb], lo.F.u[nb] + size_t(lo.nloc) * pl, R, pl, s);
    if (!e) e = copy_planes(lo.F.u[nb] + size_t(R + lo.nloc) * pl, hi.F.u[nb] + size_t(R) * pl,
                            R, pl, s);
    if (e) return e;
  }
  return cudaSuccess;
}

void make_parts(Decomp* d, int R) {
  d->before.clear();
  d->after.clear();
  const int P = int(d->slab.size());
  for (int s = 0; s < P; ++s) {
    const int n = d->slab[s].nloc;
    if (d->mode == FD_DMP_BASIC) {
      d->before.push_back({s, 0, n});
      continue;
    }
    const int lo = s > 0 ? R : 0, hi = s + 1 < P ? R : 0;
    if (lo) d->before.push_back({s, 0, R});
    if (hi) d->before.push_back({s, n - R, R});
    if (n - lo - hi > 0) d->after.push_back({s, lo, n - lo - hi});
  }
}

}  // namespace

void decomp_destroy(fd_grid g) {
  if (!g->dmp) return;
  release(g, g->dmp);
  g->dmp = nullptr;
}

fd_status decomp_propagate(fd_grid g, int n0, int nsteps, const fd_points* src,
                           const float* wavelet, const fd_points* rec, float* rec_out) {
  Decomp* d = g->dmp;
  if (g->percell)
    return fail(FD_ERR_STATE, "per-cell weight fields are not split into slabs");
  const int R = g->R;
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;
  fd_status st;
  if (d->shape.tx != g->shape.tx || d->shape.ty != g->shape.ty) {
    for (Slab& sl : d->slab)
      if ((st = build_slab_maps(g, sl))) return st;
    d->shape = g->shape;
    if (d->graph_valid) cudaGraphExecDestroy(d->gexec);
    d->graph_valid = false;
  }
  d->shape.ctas = g->shape.ctas;
  if ((st = upload_slab_tables(g, d, src, rec))) return st;
  const float* dval = nullptr;
  float* drec = nullptr;
  if ((st = stage_in(g, g->stage_val, nsrc ? wavelet : nullptr, size_t(n0 + nsteps) * nsrc,
                     &dval)))
    return st;
  if ((st = stage_out(g, g->stage_rec, nrec ? rec_out : nullptr, size_t(nsteps) * nrec,
                      &drec)))
    return st;

  // descriptors of every part, refreshed before each run (stream ordered)
  const int mode = forward_mode(g);
  std::vector<Part> parts = d->before;
  parts.insert(parts.end(), d->after.begin(), d->after.end());
  std::vector<char> host(parts.size() * kBlock, 0);
  const long long columns = (long long)g->tiles_x * g->tiles_y;
  std::vector<int> ctas(parts.size());
  for (size_t i = 0; i < parts.size(); ++i) {
    const Part& p = parts[i];
    Slab& sl = d->slab[p.s];
    RunSpec rs;
    memset(&rs, 0, sizeof(rs));
    rs.f = &sl.F;
    if (nsrc) {
      rs.inj_start = static_cast<const int32_t*>(sl.tab.inj_start.p);
      rs.inj = static_cast<const InjEntry*>(sl.tab.inj.p);
      rs.inj_val = dval;
      rs.inj_ncol = nsrc;
    }
    if (nrec) {
      rs.rec_start = static_cast<const int32_t*>(sl.tab.rec_start.p);
      rs.recs = static_cast<const RecEntry*>(sl.tab.recs.p);
      rs.rec_out = drec;
      rs.rec_ncol = nrec;
    }
    ShotDesc* sd = reinterpret_cast<ShotDesc*>(host.data() + i * kBlock);
    fill_desc(g, rs, sd);
    sd->A = sl.mapA;
    sd->C = sl.mapA;
    sd->args.Nz = p.cnt;  // updated planes per tile column
    long long* prefix = reinterpret_cast<long long*>(host.data() + i * kBlock + sizeof(ShotDesc));
    prefix[0] = 0;
    prefix[1] = columns * p.cnt;
    ctas[i] = lockstep_ctas(R, g->shape, mode, columns, p.cnt);
  }
  cudaError_t e = d->desc.ensure(host.size());
  if (e) return cuda_fail(e, "slab descriptor allocation");
  e = cudaMemcpyAsync(d->desc.p, host.data(), host.size(), cudaMemcpyHostToDevice, g->stream);
  if (e) return cuda_fail(e, "slab descriptor upload");
  if ((st = scatter(g, d))) return st;

  const int cur0 = g->F.cur;
  const bool use_graph = nsteps >= 2 && !g->no_graph;
  std::vector<char> key;
  {
    long long v[10] = {mode, nsteps, cur0, n0, nsrc > 0, nrec > 0, g->shape.tx, g->shape.ty,
                       g->shape.ctas, g->spin_limit};
    key.assign(reinterpret_cast<char*>(v), reinterpret_cast<char*>(v) + sizeof(v));
    const char* dp = reinterpret_cast<const char*>(&d->desc.p);
    key.insert(key.end(), dp, dp + sizeof(void*));
    for (int j = 0; j <= R; ++j) {
      const float c = float(g->c[j]);
      const char* cp = reinterpret_cast<const char*>(&c);
      key.insert(key.end(), cp, cp + sizeof(c));
    }
  }
  const bool reuse = use_graph && d->graph_valid && d->gkey == key;

  auto issue = [&](cudaStream_t s) -> fd_status {
    const char* base = static_cast<const char*>(d->desc.p);
    auto launch = [&](size_t i, int t) -> cudaError_t {
      const Part& p = parts[i];
      const Slab& sl = d->slab[p.s];
      StepOverride ov;
      memset(&ov, 0, sizeof(ov));
      ov.cur = (cur0 + t) & 1;
      ov.zfirst = R + p.p0;
      ov.nblz = g->d.nbl - (sl.z0 - R);
      ov.inj_row = n0 + t;
      ov.rec_row = t;
      ov.spin_limit = g->spin_limit;
      ov.debug_skip_plane = -1;
      launch_weights(g->c, R, ov.c);
      const ShotDesc* sd = reinterpret_cast<const ShotDesc*>(base + i * kBlock);
      const long long* pf = reinterpret_cast<const long long*>(base + i * kBlock + sizeof(ShotDesc));
      return launch_sweep(R, g->shape, mode, sd, pf, 1, ov, ctas[i], s);
    };
    const size_t nb4 = d->before.size();
    for (int t = 0; t < nsteps; ++t) {
      const int nb = ((cur0 + t) & 1) ^ 1;  // buffer receiving u^{n+1}
      cudaError_t e2 = cudaSuccess;
      if (d->mode == FD_DMP_OVERLAP && t > 0) e2 = cudaStreamWaitEvent(s, d->ev_join, 0);
      for (size_t i = 0; i < nb4 && !e2; ++i) e2 = launch(i, t);
      if (!e2) {
        if (d->mode == FD_DMP_BASIC) {
          e2 = exchange(g, d, nb, s);
        } else {
          e2 = cudaEventRecord(d->ev_fork, s);
          if (!e2) e2 = cudaStreamWaitEvent(d->side, d->ev_fork, 0);
          if (!e2) e2 = exchange(g, d, nb, d->side);
          if (!e2) e2 = cudaEventRecord(d->ev_join, d->side);
        }
      }
      for (size_t i = nb4; i < parts.size() && !e2; ++i) e2 = launch(i, t);
      if (e2) return cuda_fail(e2, "decomposed step");
    }
    if (d->mode == FD_DMP_OVERLAP) {
      cudaError_t e2 = cudaStreamWaitEvent(s, d->ev_join, 0);
      if (e2) return cuda_fail(e2, "exchange join");
    }
    return FD_OK;
  };

  if (g->profiling) cudaEventRecord(g->ev0, g->stream);
  if (use_graph) {
    if (!reuse) {
      if (d->graph_valid) cudaGraphExecDestroy(d->gexec);
      d->graph_valid = false;
      e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed);
      if (e) return cuda_fail(e, "stream capture");
      const long long before = fd_launch_count();
      st = issue(g->stream);
      const long long captured = fd_launch_count() - before;
      count_launch(-captured);  // counted when the graph runs
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(g->stream, &graph);
      if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&d->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e) return cuda_fail(e, "graph instantiate");
      d->graph_valid = true;
      d->gkey = key;
      d->graph_launches = captured;
    }
    e = cudaGraphLaunch(d->gexec, g->stream);
    if (e) return cuda_fail(e, "graph launch");
    count_launch(d->graph_launches);
  } else if ((st = issue(g->stream))) {
    return st;
  }
  if (g->profiling) {
    cudaEventRecord(g->ev1, g->stream);
    e = cudaEventSynchronize(g->ev1);
    if (e) return cuda_fail(e, "profiling event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    g->step_ms += ms;
    g->steps_timed += nsteps;
  }
  g->F.cur = (cur0 + nsteps) & 1;
  if ((st = gather(g, d))) return st;
  if ((st = check_device_error(g))) return st;
  if (nrec) {
    if ((st = check_finite(g, drec, size_t(nsteps) * nrec))) return st;
    if ((st = finish_out(g, rec_out, drec, size_t(nsteps) * nrec))) return st;
  }
  e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "stream synchronize");
  return FD_OK;
}

}  // namespace fd

using namespace fd;

extern "C" fd_status fd_set_decomposition(fd_grid g, int32_t nsub, int32_t mode) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (mode != FD_DMP_BASIC && mode != FD_DMP_OVERLAP)
    return fail(FD_ERR_ARG, "bad exchange mode %d", mode);
  if (nsub < 1) return fail(FD_ERR_ARG, "nsub must be >= 1");
  cudaSetDevice(g->d.device);
  const int R = g->R;
  const int need = mode == FD_DMP_OVERLAP ? 2 * R : R;
  if (nsub > 1 && g->Nz / nsub < need)
    return fail(FD_ERR_ARG,
                "cannot split %d planes into %d slabs of at least %d planes (SO %d, %s mode)",
                g->Nz, nsub, need, g->d.space_order,
                mode == FD_DMP_OVERLAP ? "overlap" : "basic");
  decomp_destroy(g);
  if (nsub == 1) return FD_OK;
  cart_destroy(g);  // slabs and boxes exclude each other

  Decomp* d = new Decomp();
  d->nsub = nsub;
  d->mode = mode;
  d->slab.resize(nsub);
  fd_status st = FD_OK;
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < nsub && !st; ++s) {
    Slab& sl = d->slab[s];
    sl.z0 = int((long long)g->Nz * s / nsub);
    sl.nloc = int((long long)g->Nz * (s + 1) / nsub) - sl.z0;
    sl.ncell = plane_floats(g) * size_t(sl.nloc + 2 * R);
    for (int b = 0; b < 2 && !st; ++b) {
      e = dev_alloc(reinterpret_cast<void**>(&sl.F.u[b]), sl.ncell * 4);
      if (!e) e = cudaMemsetAsync(sl.F.u[b], 0, sl.ncell * 4, g->stream);
      if (e) st = cuda_fail(e, "slab wavefield allocation");
    }
    if (!st) {
      e = dev_alloc(reinterpret_cast<void**>(&sl.A), sl.ncell * 4);
      if (!e) e = cudaMemsetAsync(sl.A, 0, sl.ncell * 4, g->stream);
      if (e) st = cuda_fail(e, "slab model allocation");
    }
    if (!st) st = build_slab_maps(g, sl);
  }
  d->shape = g->shape;
  if (!st && mode == FD_DMP_OVERLAP) {
    e = cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming);
    if (e) st = cuda_fail(e, "exchange stream");
  }
  if (!st) {
    e = cudaStreamSynchronize(g->stream);
    if (e) st = cuda_fail(e, "slab initialisation");
  }
  if (st) {
    release(g, d);
    return st;
  }
  make_parts(d, R);
  g->dmp = d;
  return FD_OK;
}
