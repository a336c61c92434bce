// Host side of the two-step (temporally blocked) passes of fd_tblock.cuh.
//
// A run of nsteps forward steps becomes nsteps / 2 passes, each reading the
// wavefield pair (u^{n-1}, u^n) of one pair of buffers and writing
// (u^{n+1}, u^{n+2}) into the other pair, plus one single step of the regular
// kernel when nsteps is odd.  The four buffers are the grid's own pair F and a
// second pair allocated on first use; when a run ends in the second pair the
// two pairs are swapped, so that F holds the state afterwards as after any
// other run.  The work is cut into column waves over the output tiles
// (fd_sched.cu), one CTA per SM.
#include <string.h>

#include <algorithm>
#include <vector>

#include "fd_aux.h"
#include "fd_runtime.h"
#include "fd_sched.h"

namespace fd {

struct TbState {
  Fields T;                      // second wavefield pair
  DevBuf desc;                   // TbDesc
  DevBuf sched;                  // CTA starts, then the work items
  DevBuf inj1s, inj1, inj2s, inj2, recs_s, recs;
  int bx = 0, by = 0;            // output tile
  int sched_ctas = 0;
  size_t sched_off = 0;
  long long sched_key[3] = {};
};

bool tblock_eligible(fd_grid g) {
  return g->sched_mode == FD_SCHED_TEMPORAL && (g->R == 2 || g->R == 4) && !g->dmp && !g->cart &&
         forward_mode(g) == kModeForward;
}

void tblock_destroy(fd_grid g) {
  if (!g->tb) return;
  TbState* t = g->tb;
  for (int b = 0; b < 2; ++b)
    if (t->T.u[b]) cudaFree(t->T.u[b]);
  for (DevBuf* b : {&t->desc, &t->sched, &t->inj1s, &t->inj1, &t->inj2s, &t->inj2, &t->recs_s,
                    &t->recs})
    b->release();
  delete t;
  g->tb = nullptr;
}

static fd_status tb_setup(fd_grid g) {
  if (!g->tb) g->tb = new TbState();
  TbState* t = g->tb;
  if (g->R == 2) tblock_tile_r<2>(&t->bx, &t->by);
  else tblock_tile_r<4>(&t->bx, &t->by);
  for (int b = 0; b < 2; ++b) {
    if (t->T.u[b]) continue;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&t->T.u[b]), g->ncell * 4);
    if (!e) e = cudaMemsetAsync(t->T.u[b], 0, g->ncell * 4, g->stream);
    if (e) return cuda_fail(e, "second wavefield pair");
  }
  return FD_OK;
}

// Column-wave schedule of the output tiles, one CTA per SM.
static fd_status tb_schedule(fd_grid g, int tiles) {
  TbState* t = g->tb;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long key[3] = {tiles, g->Nz, sms};
  if (t->sched.p && memcmp(key, t->sched_key, sizeof(key)) == 0) return FD_OK;
  std::vector<int32_t> start;
  std::vector<WorkItem> items;
  // each item streams 4R halo planes of u^n and 2R of step 1 besides its own
  t->sched_ctas = wave_schedule({{0, tiles, g->Nz}}, std::max(1, sms), 2 * g->R, start, items);
  t->sched_off = (start.size() * 4 + 15) / 16 * 16;
  cudaError_t e = t->sched.ensure(t->sched_off + items.size() * sizeof(WorkItem));
  if (!e) e = cudaMemcpyAsync(t->sched.p, start.data(), start.size() * 4,
                              cudaMemcpyHostToDevice, g->stream);
  if (!e)
    e = cudaMemcpyAsync(static_cast<char*>(t->sched.p) + t->sched_off, items.data(),
                        items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "two-step schedule upload");
  memcpy(t->sched_key, key, sizeof(key));
  return FD_OK;
}

fd_status tblock_propagate(fd_grid g, int n0, int nsteps, const fd_points* src,
                           const float* dval, const fd_points* rec, float* drec) {
  fd_status st = tb_setup(g);
  if (st) return st;
  TbState* t = g->tb;
  const int bx = t->bx, by = t->by, R = g->R;
  const int tiles_x = (g->Nx + bx - 1) / bx, tiles_y = (g->Ny + by - 1) / by;
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;

  // tables: step-1 sources over the extended tiles, step-2 sources over the
  // output tiles (both in extended-tile coordinates), receivers per output tile
  std::vector<int32_t> s1, s2, rs;
  std::vector<InjEntry> e1, e2;
  std::vector<RecEntry> re;
  const double scale = 1.0 / g->d.h;
  if ((st = build_injection_tiles(g, src, scale, bx, by, 4, R, s1, e1))) return st;
  if ((st = build_injection_tiles(g, src, scale, bx, by, 0, 0, s2, e2))) return st;
  for (InjEntry& e : e2) {
    e.lx = int16_t(e.lx + 4);
    e.ly = int16_t(e.ly + R);
  }
  if ((st = build_receivers_tiles(g, rec, bx, by, rs, re))) return st;
  if ((st = upload(g, t->inj1s, s1)) || (st = upload(g, t->inj1, e1)) ||
      (st = upload(g, t->inj2s, s2)) || (st = upload(g, t->inj2, e2)) ||
      (st = upload(g, t->recs_s, rs)) || (st = upload(g, t->recs, re)))
    return st;
  if ((st = tb_schedule(g, tiles_x * tiles_y))) return st;

  // descriptor: tensor maps of the four buffers and of A
  float* buf[4] = {g->F.u[0], g->F.u[1], t->T.u[0], t->T.u[1]};
  const int W2 = bx + 16, H2 = by + 4 * R, EX = bx + 8, EY = by + 2 * R;
  TbDesc host;
  memset(&host, 0, sizeof(host));
  for (int b = 0; b < 4; ++b) {
    if ((st = make_map(&host.halo2[b], buf[b], g->Nx, g->Ny, g->Nz, g->pitch, W2, H2))) return st;
    if ((st = make_map(&host.ext[b], buf[b], g->Nx, g->Ny, g->Nz, g->pitch, EX, EY))) return st;
    host.u[b] = buf[b];
  }
  if ((st = make_map(&host.extA, g->A, g->Nx, g->Ny, g->Nz, g->pitch, EX, EY))) return st;
  TbArgs& a = host.args;
  a.Nx = g->Nx;
  a.Ny = g->Ny;
  a.Nz = g->Nz;
  a.pitch = g->pitch;
  a.nbl = g->d.nbl;
  a.nx = g->d.nx;
  a.ny = g->d.ny;
  a.nz = g->d.nz;
  a.tiles_x = tiles_x;
  a.tiles_y = tiles_y;
  a.bscale = g->bscale;
  a.inj1_start = static_cast<const int32_t*>(t->inj1s.p);
  a.inj1 = static_cast<const InjEntry*>(t->inj1.p);
  a.inj2_start = static_cast<const int32_t*>(t->inj2s.p);
  a.inj2 = static_cast<const InjEntry*>(t->inj2.p);
  a.inj_val = dval;
  a.inj_ncol = nsrc;
  a.rec_start = static_cast<const int32_t*>(t->recs_s.p);
  a.recs = static_cast<const RecEntry*>(t->recs.p);
  a.rec_out = drec;
  a.rec_ncol = nrec;
  a.A = g->A;
  a.err = g->d_err;
  cudaError_t e = t->desc.ensure(sizeof(TbDesc));
  if (!e) e = cudaMemcpyAsync(t->desc.p, &host, sizeof(host), cudaMemcpyHostToDevice, g->stream);
  if (e) return cuda_fail(e, "two-step descriptor");

  TbLaunch L;
  memset(&L, 0, sizeof(L));
  L.spin_limit = g->spin_limit;
  launch_weights(g->c, R, L.c);
  L.item_start = static_cast<const int32_t*>(t->sched.p);
  L.items = reinterpret_cast<const WorkItem*>(static_cast<const char*>(t->sched.p) +
                                              t->sched_off);
  int prev = g->F.cur ^ 1, cur = g->F.cur;  // buffer indices 0..3
  const TbDesc* dd = static_cast<const TbDesc*>(t->desc.p);
  if (g->profiling) cudaEventRecord(g->ev0, g->stream);
  const int npass = nsteps / 2;
  for (int p = 0; p < npass; ++p) {
    const int other = cur < 2 ? 2 : 0;  // the pair that does not hold the state
    L.in_prev = prev;
    L.in_cur = cur;
    L.out1 = other;
    L.out2 = other + 1;
    L.inj_row = n0 + 2 * p;
    L.rec_row = 2 * p;
    count_launch();
    e = R == 2 ? launch_tblock_r<2>(dd, L, t->sched_ctas, g->stream)
               : launch_tblock_r<4>(dd, L, t->sched_ctas, g->stream);
    if (e) return cuda_fail(e, "two-step launch");
    prev = other;
    cur = other + 1;
  }
  if (g->profiling) {
    cudaEventRecord(g->ev1, g->stream);
    e = cudaEventSynchronize(g->ev1);
    if (e) return cuda_fail(e, "profiling event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    g->step_ms += ms;
    g->steps_timed += 2LL * npass;
  }
  // the state back in the grid's own pair F
  if (cur >= 2) {
    std::swap(g->F.u[0], t->T.u[0]);
    std::swap(g->F.u[1], t->T.u[1]);
    g->graph_valid = false;
    if ((st = build_field_maps(g, g->F))) return st;
  }
  g->F.cur = cur & 1;
  g->last_sched = FD_SCHED_TEMPORAL;
  if (nsteps & 1) {
    // the last step on the regular kernel
    Tables& tab = g->tab;
    if ((st = upload_tables(g, src, scale, rec, tab))) return st;
    RunSpec rs;
    memset(&rs, 0, sizeof(rs));
    rs.f = &g->F;
    rs.allow_graph = 0;
    rs.mode = kModeForward;
    rs.nsteps = 1;
    if (nsrc) {
      rs.inj_start = static_cast<const int32_t*>(tab.inj_start.p);
      rs.inj = static_cast<const InjEntry*>(tab.inj.p);
      rs.inj_val = dval;
      rs.inj_ncol = nsrc;
      rs.inj_row0 = n0 + nsteps - 1;
    }
    if (nrec) {
      rs.rec_start = static_cast<const int32_t*>(tab.rec_start.p);
      rs.recs = static_cast<const RecEntry*>(tab.recs.p);
      rs.rec_out = drec;
      rs.rec_ncol = nrec;
      rs.rec_row0 = nsteps - 1;
    }
    const int keep = g->last_sched;
    if ((st = run_steps(g, rs))) return st;
    g->last_sched = keep;
  }
  return FD_OK;
}

}  // namespace fd
