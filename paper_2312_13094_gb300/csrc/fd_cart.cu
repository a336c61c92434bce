// Cartesian domain decomposition of one grid on the device: px x py x pz
// boxes exchanging their halo before every step.
//
// Sec. III of the paper splits the grid over a Cartesian topology of ranks
// (MPI_Dims_create or a user-given topology); before every step each rank
// packs the R owned layers next to its neighbours into messages, sends them
// and unpacks what it receives into its halo.  Its "basic" mode fills edges
// and corners of the halo by exchanging axis after axis; its "diagonal" mode
// sends one message per neighbour, faces, edges and corners (26 in 3-D), in
// a single exchange.  Here six face messages of owned values are packed and
// every ghost block, faces, edges and corners, is filled from them in one
// exchange (an edge or corner block is part of a diagonal neighbour's face
// message).  The star stencil itself reads only the six faces; the edge and
// corner ghosts serve the trilinear receivers whose eight nodes straddle two
// or three cuts.
//
// Layout.  Box b owns the padded ranges [gx0, gx0 + onx) x [gy0, gy0 + ony)
// x [gz0, gz0 + onz) (per axis the balanced split of the padded extent) and
// keeps its two wavefields and its model term in arrays of
// (onx + 2 GX) x (ony + 2R) x (onz + 2R) points, GX = R rounded up to four
// floats so that every tile's TMA x coordinate stays 16-byte aligned.  Ghost
// layers beyond the grid are zero and never written.
//
// Step.  One launch of the plain step kernel steps every box (the boxes are
// the "shots" of the launch, with their own tensor maps, tables and array
// offsets that keep the damping layer in global coordinates), on column
// waves over the boxes one after another unless the grid asks for equal
// shares or a CTA count.  A pack kernel
// then copies the R updated layers next to each face with a neighbour into
// that face's contiguous message, and an unpack kernel copies every message
// block into the receiving box's ghost layers: the whole message for a face
// neighbour, a sub-block of it (the first or last R rows or planes) for an
// edge or corner neighbour, whose points the face messages hold too.  On one
// GPU the unpack reads the sender's message directly; across GPUs a peer
// copy (or NCCL send/recv) of each contiguous message into the receiver's
// memory would come in between.  (Writing the messages from the step's own
// epilogue was measured 1.7x slower than the plain step: the extra code made
// the kernel's hot loop execute 1.25x the instructions even for points that
// store nothing; the two copy kernels cost a fraction of that.)  Every point
// goes through the same arithmetic as in the undecomposed run, so both give
// the same wavefields and receivers bit for bit.
#include <string.h>

#include <algorithm>
#include <vector>

#include "fd_aux.h"
#include "fd_runtime.h"
#include "fd_sched.h"

namespace fd {

struct Box {
  int g0[3] = {0, 0, 0};  // padded coordinates of the first owned point
  int on[3] = {0, 0, 0};  // owned extents
  int ax = 0, ay = 0, az = 0, pitch = 0;  // array extents and row pitch (floats)
  size_t ncell = 0;
  Fields F;
  float* A = nullptr;
  CUtensorMap mapA;
  Tables tab;
  float* msg[6] = {};  // face messages x-, x+, y-, y+, z-, z+ (faces with a neighbour)
  int nb[27];           // neighbour box per direction (dx+1) + 3(dy+1) + 9(dz+1), -1: none
};

// One block copy of n0 x n1 x n2 points between strided regions (row and
// plane strides in floats); the side that is a box wavefield has one address
// per buffer of the pair, the step's parity chooses.  Pack: box -> message;
// unpack: message (or a sub-block of it) -> box ghost layers.
struct Msg {
  const float* src[2];
  float* dst[2];
  int n0, n1, n2;
  long long s1, s2;  // source strides
  long long d1, d2;  // destination strides
};

struct Cart {
  int p[3] = {1, 1, 1};
  int gx = 4;  // x ghost width
  std::vector<Box> box;
  TileShape shape = {};
  DevBuf desc;   // ShotDesc per box, then the unit prefix
  DevBuf msgs;   // pack blocks, then unpack blocks
  int npack = 0, nunpack = 0, maxlen = 0;  // block counts; most points in one block
  DevBuf sched;  // column-wave work items over all boxes: CTA starts, then items
  long long sched_key[3] = {0, 0, 0};  // tile x, tile y, slots of the schedule
  int sched_ctas = 0;
  size_t sched_off = 0;
  bool graph_valid = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<char> gkey;
  long long graph_launches = 0;
};

namespace {

// Block copies, one block per blockIdx.y: every point of a block is one
// thread's (32-bit indices: a block holds at most (N + 2R)^2 R points).
__global__ void k_copy_blocks(const Msg* __restrict__ list, int nb) {
  const Msg m = list[blockIdx.y];
  const int n = m.n0 * m.n1 * m.n2;
  const float* src = m.src[nb];
  float* dst = m.dst[nb];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int i0 = i % m.n0, r = i / m.n0;
    const int i1 = r % m.n1, i2 = r / m.n1;
    dst[i2 * m.d2 + i1 * m.d1 + i0] = src[i2 * m.s2 + i1 * m.s1 + i0];
  }
}

fd_status build_box_maps(fd_grid g, Cart* c, Box& b) {
  const int bx = 4 * g->shape.tx, by = g->shape.ty;
  const int W = bx + 2 * radius_halo_x(g->R), H = by + 2 * g->R;
  for (int k = 0; k < 2; ++k) {
    fd_status st = make_map(&b.F.halo[k], b.F.u[k], b.ax, b.ay, b.az, b.pitch, W, H);
    if (!st) st = make_map(&b.F.tile[k], b.F.u[k], b.ax, b.ay, b.az, b.pitch, bx, by);
    if (st) return st;
  }
  (void)c;
  return make_map(&b.mapA, b.A, b.ax, b.ay, b.az, b.pitch, bx, by);
}

void release(fd_grid g, Cart* c) {
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (Box& b : c->box) {
    for (int k = 0; k < 2; ++k)
      if (b.F.u[k]) cudaFree(b.F.u[k]);
    if (b.A) cudaFree(b.A);
    for (int f = 0; f < 6; ++f)
      if (b.msg[f]) cudaFree(b.msg[f]);
    for (DevBuf* d : {&b.tab.inj_start, &b.tab.inj, &b.tab.rec_start, &b.tab.recs}) d->release();
  }
  c->desc.release();
  c->msgs.release();
  c->sched.release();
  if (c->graph_valid) cudaGraphExecDestroy(c->gexec);
  delete c;
}

// array coordinate = padded coordinate - off
int off_x(const Cart* c, const Box& b) { return b.g0[0] - c->gx; }
int off_y(fd_grid g, const Box& b) { return b.g0[1] - g->R; }
int off_z(fd_grid g, const Box& b) { return b.g0[2] - g->R; }

int owner(const Cart* c, const fd_grid g, const int node[3], int* idx) {
  const int N[3] = {g->Nx, g->Ny, g->Nz};
  int q[3];
  for (int a = 0; a < 3; ++a) {
    q[a] = int((long long)(node[a] + 1) * c->p[a] / N[a]);  // first guess, then correct
    q[a] = std::min(std::max(q[a], 0), c->p[a] - 1);
    while (q[a] > 0 && node[a] < int((long long)N[a] * q[a] / c->p[a])) --q[a];
    while (q[a] + 1 < c->p[a] && node[a] >= int((long long)N[a] * (q[a] + 1) / c->p[a])) ++q[a];
  }
  *idx = (q[2] * c->p[1] + q[1]) * c->p[0] + q[0];
  return 0;
}

// Per-box source and receiver tables in the box's tiling and array planes,
// entries of a node in the order of the points (as the whole-grid tables).
fd_status upload_box_tables(fd_grid g, Cart* c, const fd_points* src, const fd_points* rec) {
  const int bx = 4 * g->shape.tx, by = g->shape.ty;
  const int nbox = int(c->box.size());
  struct KI { int box, tile; InjEntry e; };
  struct KR { int box, tile; RecEntry e; };
  std::vector<KI> inj;
  std::vector<KR> re;
  const double scale = 1.0 / g->d.h;
  for (int p = 0; p < (src ? src->n : 0); ++p) {
    int i0[3];
    double f[3];
    fd_status st = locate_point(g, src->xyz + 3 * p, i0, f);
    if (st) return st;
    for (int cc = 0; cc < 8; ++cc) {
      int node[3];
      double w = 1.0;
      for (int a = 0; a < 3; ++a) {
        const int hi = (cc >> a) & 1;
        node[a] = i0[a] + hi;
        w *= hi ? f[a] : 1.0 - f[a];
      }
      if (w == 0.0) continue;
      if (node[0] >= g->Nx || node[1] >= g->Ny || node[2] >= g->Nz) continue;
      int b = 0;
      owner(c, g, node, &b);
      const Box& B = c->box[b];
      const int lx = node[0] - B.g0[0], ly = node[1] - B.g0[1];
      const int tiles_x = (B.on[0] + bx - 1) / bx;
      InjEntry e;
      e.z = node[2] - off_z(g, B);
      e.lx = int16_t(lx % bx);
      e.ly = int16_t(ly % by);
      e.w = float(w * scale);
      e.col = p;
      inj.push_back({b, (ly / by) * tiles_x + lx / bx, e});
    }
  }
  for (int p = 0; p < (rec ? rec->n : 0); ++p) {
    int i0[3];
    double f[3];
    fd_status st = locate_point(g, rec->xyz + 3 * p, i0, f);
    if (st) return st;
    int b = 0;
    owner(c, g, i0, &b);
    const Box& B = c->box[b];
    const int lx = i0[0] - B.g0[0], ly = i0[1] - B.g0[1];
    const int tiles_x = (B.on[0] + bx - 1) / bx;
    RecEntry e;
    e.z = i0[2] - off_z(g, B);
    e.lx = int16_t(lx % bx);
    e.ly = int16_t(ly % by);
    e.fx = float(f[0]);
    e.fy = float(f[1]);
    e.fz = float(f[2]);
    e.col = p;
    re.push_back({b, (ly / by) * tiles_x + lx / bx, e});
  }
  std::stable_sort(inj.begin(), inj.end(), [](const KI& a, const KI& b) {
    return a.box != b.box ? a.box < b.box : a.tile != b.tile ? a.tile < b.tile : a.e.z < b.e.z;
  });
  std::stable_sort(re.begin(), re.end(), [](const KR& a, const KR& b) {
    return a.box != b.box ? a.box < b.box : a.tile != b.tile ? a.tile < b.tile : a.e.z < b.e.z;
  });
  size_t ii = 0, rr = 0;
  for (int b = 0; b < nbox; ++b) {
    Box& B = c->box[b];
    const int ntiles = ((B.on[0] + bx - 1) / bx) * ((B.on[1] + by - 1) / by);
    std::vector<int32_t> is(ntiles + 1, 0), rs(ntiles + 1, 0);
    std::vector<InjEntry> ie;
    std::vector<RecEntry> rv;
    for (; ii < inj.size() && inj[ii].box == b; ++ii) {
      is[inj[ii].tile + 1]++;
      ie.push_back(inj[ii].e);
    }
    for (; rr < re.size() && re[rr].box == b; ++rr) {
      rs[re[rr].tile + 1]++;
      rv.push_back(re[rr].e);
    }
    for (int t = 0; t < ntiles; ++t) {
      is[t + 1] += is[t];
      rs[t + 1] += rs[t];
    }
    fd_status st;
    if ((st = upload(g, B.tab.inj_start, is)) || (st = upload(g, B.tab.inj, ie)) ||
        (st = upload(g, B.tab.rec_start, rs)) || (st = upload(g, B.tab.recs, rv)))
      return st;
  }
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "box table upload");
  return FD_OK;
}

// Copy the padded-grid region [lo, hi) (per axis) between the whole grid's
// field and a box array.
cudaError_t copy_region(fd_grid g, const Cart* c, const Box& b, float* whole, float* arr,
                        const int lo[3], const int hi[3], bool to_box) {
  if (hi[0] <= lo[0] || hi[1] <= lo[1] || hi[2] <= lo[2]) return cudaSuccess;
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof(p));
  cudaPitchedPtr W = make_cudaPitchedPtr(whole, size_t(g->pitch) * 4, g->Nx * 4, g->Ny);
  cudaPitchedPtr B = make_cudaPitchedPtr(arr, size_t(b.pitch) * 4, b.ax * 4, b.ay);
  const cudaPos pw = make_cudaPos(size_t(lo[0]) * 4, lo[1], lo[2]);
  const cudaPos pb = make_cudaPos(size_t(lo[0] - off_x(c, b)) * 4, lo[1] - off_y(g, b),
                                  lo[2] - off_z(g, b));
  if (to_box) {
    p.srcPtr = W;
    p.srcPos = pw;
    p.dstPtr = B;
    p.dstPos = pb;
  } else {
    p.srcPtr = B;
    p.srcPos = pb;
    p.dstPtr = W;
    p.dstPos = pw;
  }
  p.extent = make_cudaExtent(size_t(hi[0] - lo[0]) * 4, hi[1] - lo[1], hi[2] - lo[2]);
  p.kind = cudaMemcpyDeviceToDevice;
  return cudaMemcpy3DAsync(&p, g->stream);
}

fd_status scatter(fd_grid g, Cart* c) {
  const int R = g->R;
  const int N[3] = {g->Nx, g->Ny, g->Nz};
  for (Box& b : c->box) {
    int lo[3], hi[3], olo[3], ohi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::max(0, b.g0[a] - R);
      hi[a] = std::min(N[a], b.g0[a] + b.on[a] + R);
      olo[a] = b.g0[a];
      ohi[a] = b.g0[a] + b.on[a];
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && !e; ++k) e = copy_region(g, c, b, g->F.u[k], b.F.u[k], lo, hi, true);
    if (!e) e = copy_region(g, c, b, g->A, b.A, olo, ohi, true);
    if (e) return cuda_fail(e, "box scatter");
  }
  return FD_OK;
}

fd_status gather(fd_grid g, Cart* c) {
  for (Box& b : c->box) {
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = b.g0[a];
      hi[a] = b.g0[a] + b.on[a];
    }
    for (int k = 0; k < 2; ++k) {
      cudaError_t e = copy_region(g, c, b, g->F.u[k], b.F.u[k], lo, hi, false);
      if (e) return cuda_fail(e, "box gather");
    }
  }
  return FD_OK;
}

// Pack list: face f of box b (axis f / 2, low side for even f), where it has
// a neighbour, copies b's R owned layers next to it into its message, stored
// [z][y][x] over that block.  Unpack list: box b's ghost block towards
// direction d is the neighbour n = b + d's owned block next to b: along an
// axis with d = 0 the owned range, with d = -1 the R layers below b's first
// owned one (n's last R), with d = +1 the R above b's last (n's first R).
// That block lies in one of n's face messages, the one of the first axis a
// with d_a != 0 (n's face towards b on that axis): the whole message for a
// face neighbour, a sub-block of it (the first or last R rows or planes of
// the other axes) for an edge or corner neighbour.
fd_status build_messages(fd_grid g, Cart* c) {
  const int R = g->R;
  const int first[3] = {c->gx, R, R};
  std::vector<Msg> pack, unpack;
  c->maxlen = 0;
  for (Box& b : c->box) {
    const long long row = b.pitch, plane = (long long)b.pitch * b.ay;
    for (int f = 0; f < 6; ++f) {
      if (!b.msg[f]) continue;
      const int ax = f / 2;
      int e[3], o[3];
      for (int a = 0; a < 3; ++a) {
        e[a] = a == ax ? R : b.on[a];
        o[a] = first[a] + (a == ax && (f & 1) ? b.on[a] - R : 0);
      }
      Msg m;
      const long long off = o[2] * plane + o[1] * row + o[0];
      for (int q = 0; q < 2; ++q) {
        m.src[q] = b.F.u[q] + off;
        m.dst[q] = b.msg[f];
      }
      m.n0 = e[0];
      m.n1 = e[1];
      m.n2 = e[2];
      m.s1 = row;
      m.s2 = plane;
      m.d1 = e[0];
      m.d2 = (long long)e[0] * e[1];
      pack.push_back(m);
      c->maxlen = std::max(c->maxlen, e[0] * e[1] * e[2]);
    }
  }
  for (Box& b : c->box) {
    for (int k = 0; k < 27; ++k) {
      if (k == 13 || b.nb[k] < 0) continue;
      const int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
      const Box& n = c->box[b.nb[k]];
      int ax = 0;
      while (d[ax] == 0) ++ax;
      const int f = 2 * ax + (d[ax] < 0 ? 1 : 0);  // n's face towards b
      // extents of n's face message, the first point of the block within
      // it, the block's extents and its first point in b's arrays
      int me[3], mo[3], e[3], o[3];
      for (int a = 0; a < 3; ++a) {
        me[a] = a == ax ? R : n.on[a];
        e[a] = d[a] ? R : b.on[a];
        mo[a] = (a == ax || d[a] >= 0) ? 0 : n.on[a] - R;  // d = -1: n's last R
        o[a] = d[a] == 0 ? first[a] : (d[a] > 0 ? first[a] + b.on[a] : first[a] - R);
      }
      Msg m;
      const float* src = n.msg[f] + ((long long)mo[2] * me[1] + mo[1]) * me[0] + mo[0];
      m.s1 = me[0];
      m.s2 = (long long)me[0] * me[1];
      m.n0 = e[0];
      m.n1 = e[1];
      m.n2 = e[2];
      m.d1 = b.pitch;
      m.d2 = (long long)b.pitch * b.ay;
      const long long off = (long long)o[2] * m.d2 + (long long)o[1] * b.pitch + o[0];
      for (int q = 0; q < 2; ++q) {
        m.src[q] = src;
        m.dst[q] = b.F.u[q] + off;
      }
      unpack.push_back(m);
      c->maxlen = std::max(c->maxlen, e[0] * e[1] * e[2]);
    }
  }
  c->npack = int(pack.size());
  c->nunpack = int(unpack.size());
  pack.insert(pack.end(), unpack.begin(), unpack.end());
  cudaError_t e = c->msgs.ensure(std::max<size_t>(16, pack.size() * sizeof(Msg)));
  if (!e && !pack.empty())
    e = cudaMemcpyAsync(c->msgs.p, pack.data(), pack.size() * sizeof(Msg),
                        cudaMemcpyHostToDevice, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "message list upload");
  return FD_OK;
}

}  // namespace

void cart_destroy(fd_grid g) {
  if (!g->cart) return;
  release(g, g->cart);
  g->cart = nullptr;
}

fd_status cart_propagate(fd_grid g, int n0, int nsteps, const fd_points* src,
                         const float* wavelet, const fd_points* rec, float* rec_out) {
  Cart* c = g->cart;
  if (g->percell || g->table_mode)
    return fail(FD_ERR_STATE, "per-cell and table weights are not split into boxes");
  const int R = g->R;
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;
  fd_status st;
  if (c->shape.tx != g->shape.tx || c->shape.ty != g->shape.ty) {
    for (Box& b : c->box)
      if ((st = build_box_maps(g, c, b))) return st;
    c->shape = g->shape;
    if (c->graph_valid) cudaGraphExecDestroy(c->gexec);
    c->graph_valid = false;
  }
  c->shape.ctas = g->shape.ctas;
  if ((st = upload_box_tables(g, c, src, rec))) return st;
  const float* dval = nullptr;
  float* drec = nullptr;
  if ((st = stage_in(g, g->stage_val, nsrc ? wavelet : nullptr, size_t(n0 + nsteps) * nsrc,
                     &dval)))
    return st;
  if ((st = stage_out(g, g->stage_rec, nrec ? rec_out : nullptr, size_t(nsteps) * nrec,
                      &drec)))
    return st;

  // one descriptor per box (a "shot" of the launch), then the unit prefix
  const int nbox = int(c->box.size());
  const int bx = 4 * g->shape.tx, by = g->shape.ty;
  const size_t dbytes = nbox * sizeof(ShotDesc);
  std::vector<char> host(dbytes + (nbox + 1) * sizeof(long long), 0);
  long long* prefix = reinterpret_cast<long long*>(host.data() + dbytes);
  prefix[0] = 0;
  for (int i = 0; i < nbox; ++i) {
    Box& b = c->box[i];
    RunSpec rs;
    memset(&rs, 0, sizeof(rs));
    rs.f = &b.F;
    if (nsrc) {
      rs.inj_start = static_cast<const int32_t*>(b.tab.inj_start.p);
      rs.inj = static_cast<const InjEntry*>(b.tab.inj.p);
      rs.inj_val = dval;
      rs.inj_ncol = nsrc;
    }
    if (nrec) {
      rs.rec_start = static_cast<const int32_t*>(b.tab.rec_start.p);
      rs.recs = static_cast<const RecEntry*>(b.tab.recs.p);
      rs.rec_out = drec;
      rs.rec_ncol = nrec;
    }
    ShotDesc* sd = reinterpret_cast<ShotDesc*>(host.data()) + i;
    fill_desc(g, rs, sd);
    sd->A = b.mapA;
    sd->C = b.mapA;
    StepArgs& a = sd->args;
    a.Nx = b.ax;
    a.Ny = b.ay;
    a.Nz = b.on[2];  // updated planes per tile column
    a.pitch = b.pitch;
    a.tiles_x = (b.on[0] + bx - 1) / bx;
    a.tiles_y = (b.on[1] + by - 1) / by;
    a.xfirst = c->gx;
    a.yfirst = R;
    a.xend = c->gx + b.on[0];
    a.yend = R + b.on[1];
    a.offx = off_x(c, b);
    a.offy = off_y(g, b);
    a.offz = off_z(g, b);
    prefix[i + 1] = prefix[i] + (long long)a.tiles_x * a.tiles_y * b.on[2];
  }
  cudaError_t e = c->desc.ensure(host.size());
  if (e) return cuda_fail(e, "box descriptor allocation");
  e = cudaMemcpyAsync(c->desc.p, host.data(), host.size(), cudaMemcpyHostToDevice, g->stream);
  if (e) return cuda_fail(e, "box descriptor upload");
  if ((st = scatter(g, c))) return st;

  // lockstep as for whole grids: when every box's columns fit in the
  // resident CTAs, k equal z chunks per column, all advancing together so
  // that neighbouring columns find each other's halo rows in L2
  long long columns = 0;
  int onz_min = g->Nz;
  for (const Box& b : c->box) {
    columns += (long long)((b.on[0] + bx - 1) / bx) * ((b.on[1] + by - 1) / by);
    onz_min = std::min(onz_min, b.on[2]);
  }
  int ctas = lockstep_ctas(R, g->shape, kModeForward, columns, onz_min);
  // column waves over all boxes (the boxes one after another, as the shots of
  // a batch), unless the grid asks for equal shares or a CTA count: the
  // columns of a wave advance together, so the y and x halo rows that
  // neighbouring columns share are read from L2
  const WorkItem* items = nullptr;
  const int32_t* item_start = nullptr;
  if (g->sched_mode != FD_SCHED_SHARES && g->shape.ctas == 0) {
    const int slots = sweep_ctas(R, g->shape, kModeForward);
    const long long key[3] = {g->shape.tx, g->shape.ty, slots};
    if (memcmp(key, c->sched_key, sizeof(key)) != 0 || !c->sched.p) {
      std::vector<SchedGrid> grids;
      for (int i = 0; i < nbox; ++i) {
        const Box& b = c->box[i];
        grids.push_back({i, ((b.on[0] + bx - 1) / bx) * ((b.on[1] + by - 1) / by), b.on[2]});
      }
      std::vector<int32_t> start;
      std::vector<WorkItem> witems;
      const int used = wave_schedule(grids, slots, R, start, witems);
      const size_t off = (start.size() * 4 + 15) / 16 * 16;
      e = c->sched.ensure(off + witems.size() * sizeof(WorkItem));
      if (!e) e = cudaMemcpyAsync(c->sched.p, start.data(), start.size() * 4,
                                  cudaMemcpyHostToDevice, g->stream);
      if (!e)
        e = cudaMemcpyAsync(static_cast<char*>(c->sched.p) + off, witems.data(),
                            witems.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, g->stream);
      if (!e) e = cudaStreamSynchronize(g->stream);
      if (e) return cuda_fail(e, "box schedule upload");
      memcpy(c->sched_key, key, sizeof(key));
      c->sched_ctas = used;
      c->sched_off = off;
    }
    item_start = static_cast<const int32_t*>(c->sched.p);
    items = reinterpret_cast<const WorkItem*>(static_cast<const char*>(c->sched.p) +
                                              c->sched_off);
    ctas = c->sched_ctas;
  }
  const int cur0 = g->F.cur;
  const bool use_graph = nsteps >= 2 && !g->no_graph;
  std::vector<char> key;
  {
    long long v[11] = {nsteps, cur0, n0, nsrc > 0, nrec > 0, g->shape.tx, g->shape.ty, ctas,
                       g->spin_limit, (long long)c->msgs.p, (long long)items};
    key.assign(reinterpret_cast<char*>(v), reinterpret_cast<char*>(v) + sizeof(v));
    const char* dp = reinterpret_cast<const char*>(&c->desc.p);
    key.insert(key.end(), dp, dp + sizeof(void*));
    for (int j = 0; j <= R; ++j) {
      const float cf = float(g->c[j]);
      const char* cp = reinterpret_cast<const char*>(&cf);
      key.insert(key.end(), cp, cp + sizeof(cf));
    }
  }
  const bool reuse = use_graph && c->graph_valid && c->gkey == key;
  // copy kernels: 256 threads, enough blocks to cover the largest block copy
  const int cblocks = std::max(1, std::min(1024, (c->maxlen + 255) / 256));

  auto issue = [&](cudaStream_t s) -> fd_status {
    const ShotDesc* sd = static_cast<const ShotDesc*>(c->desc.p);
    const long long* pf =
        reinterpret_cast<const long long*>(static_cast<const char*>(c->desc.p) + dbytes);
    for (int t = 0; t < nsteps; ++t) {
      StepOverride ov;
      memset(&ov, 0, sizeof(ov));
      ov.cur = (cur0 + t) & 1;
      ov.zfirst = R;
      ov.nblz = g->d.nbl;
      ov.inj_row = n0 + t;
      ov.rec_row = t;
      ov.spin_limit = g->spin_limit;
      ov.debug_skip_plane = -1;
      ov.item_start = item_start;
      ov.items = items;
      launch_weights(g->c, R, ov.c);
      cudaError_t e2 = launch_sweep(R, g->shape, kModeForward, sd, pf, nbox, ov, ctas, s);
      // pack the faces of the buffer the step wrote, then unpack into it
      const Msg* list = static_cast<const Msg*>(c->msgs.p);
      if (!e2 && c->npack > 0) {
        count_launch();
        k_copy_blocks<<<dim3(cblocks, c->npack), 256, 0, s>>>(list, ov.cur ^ 1);
        e2 = cudaGetLastError();
      }
      if (!e2 && c->nunpack > 0) {
        count_launch();
        k_copy_blocks<<<dim3(cblocks, c->nunpack), 256, 0, s>>>(list + c->npack, ov.cur ^ 1);
        e2 = cudaGetLastError();
      }
      if (e2) return cuda_fail(e2, "decomposed step");
    }
    return FD_OK;
  };

  if (g->profiling) cudaEventRecord(g->ev0, g->stream);
  if (use_graph) {
    if (!reuse) {
      if (c->graph_valid) cudaGraphExecDestroy(c->gexec);
      c->graph_valid = false;
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
      e = cudaGraphInstantiate(&c->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e) return cuda_fail(e, "graph instantiate");
      c->graph_valid = true;
      c->gkey = key;
      c->graph_launches = captured;
    }
    e = cudaGraphLaunch(c->gexec, g->stream);
    if (e) return cuda_fail(e, "graph launch");
    count_launch(c->graph_launches);
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
  g->last_sched = FD_SCHED_SHARES;
  if ((st = gather(g, c))) return st;
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

extern "C" fd_status fd_set_topology(fd_grid g, int32_t px, int32_t py, int32_t pz) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (px < 1 || py < 1 || pz < 1) return fail(FD_ERR_ARG, "topology sizes must be >= 1");
  cudaSetDevice(g->d.device);
  const int R = g->R;
  const int N[3] = {g->Nx, g->Ny, g->Nz};
  const int P[3] = {px, py, pz};
  for (int a = 0; a < 3; ++a)
    if (P[a] > 1 && N[a] / P[a] < R)
      return fail(FD_ERR_ARG, "cannot split %d points along axis %d into %d boxes of at least %d",
                  N[a], a, P[a], R);
  cart_destroy(g);
  if (px * py * pz == 1) return FD_OK;
  decomp_destroy(g);  // slabs and boxes exclude each other

  Cart* c = new Cart();
  for (int a = 0; a < 3; ++a) c->p[a] = P[a];
  c->gx = radius_halo_x(R);
  c->box.resize(size_t(px) * py * pz);
  fd_status st = FD_OK;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < pz && !st; ++k)
    for (int j = 0; j < py && !st; ++j)
      for (int i = 0; i < px && !st; ++i) {
        const int q[3] = {i, j, k};
        Box& b = c->box[(size_t(k) * py + j) * px + i];
        for (int a = 0; a < 3; ++a) {
          b.g0[a] = int((long long)N[a] * q[a] / P[a]);
          b.on[a] = int((long long)N[a] * (q[a] + 1) / P[a]) - b.g0[a];
        }
        for (int f = 0; f < 27; ++f) {
          const int n[3] = {i + f % 3 - 1, j + (f / 3) % 3 - 1, k + f / 9 - 1};
          b.nb[f] = -1;
          if (f != 13 && n[0] >= 0 && n[0] < px && n[1] >= 0 && n[1] < py && n[2] >= 0 &&
              n[2] < pz)
            b.nb[f] = (n[2] * py + n[1]) * px + n[0];
        }
        b.ax = b.on[0] + 2 * c->gx;
        b.ay = b.on[1] + 2 * R;
        b.az = b.on[2] + 2 * R;
        b.pitch = (b.ax + 31) / 32 * 32;
        b.ncell = size_t(b.pitch) * b.ay * b.az;
        for (int m = 0; m < 2 && !st; ++m) {
          e = dev_alloc(reinterpret_cast<void**>(&b.F.u[m]), b.ncell * 4);
          if (!e) e = cudaMemsetAsync(b.F.u[m], 0, b.ncell * 4, g->stream);
          if (e) st = cuda_fail(e, "box wavefield allocation");
        }
        if (!st) {
          e = dev_alloc(reinterpret_cast<void**>(&b.A), b.ncell * 4);
          if (!e) e = cudaMemsetAsync(b.A, 0, b.ncell * 4, g->stream);
          if (e) st = cuda_fail(e, "box model allocation");
        }
        // face messages: face f (axis f / 2, low side for even f) towards the
        // neighbour in direction index 13 -/+ 1, 3, 9
        for (int f = 0; f < 6 && !st; ++f) {
          const int step = f < 2 ? 1 : f < 4 ? 3 : 9;
          if (b.nb[13 + (f & 1 ? step : -step)] < 0) continue;
          size_t n = R;
          for (int a = 0; a < 3; ++a)
            if (a != f / 2) n *= size_t(b.on[a]);
          e = dev_alloc(reinterpret_cast<void**>(&b.msg[f]), n * 4);
          if (e) st = cuda_fail(e, "message buffer allocation");
        }
        if (!st) st = build_box_maps(g, c, b);
      }
  c->shape = g->shape;
  if (!st) st = build_messages(g, c);
  if (!st) {
    e = cudaStreamSynchronize(g->stream);
    if (e) st = cuda_fail(e, "box initialisation");
  }
  if (st) {
    release(g, c);
    return st;
  }
  g->cart = c;
  return FD_OK;
}
