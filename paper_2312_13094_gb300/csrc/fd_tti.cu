// Anisotropic acoustic (TTI) propagation for sm_103a.
//
// Sec. IV-B ("Anisotropic acoustic") and App. A (Eq. rot): two scalar fields
// p, q coupled through a rotated anisotropic Laplacian,
//     m p_tt + eta p_t = (1+2 eps) H_0 p + sqrt(1+2 delta) H_z q + s,
//     m q_tt + eta q_t = sqrt(1+2 delta) H_0 p + H_z q + s,
// H_z u = sum_ab n_a n_b D_ab u along the symmetry axis
// n = (sin t cos p, sin t sin p, cos t) (t the tilt, p the azimuth, per cell)
// and H_0 = Laplacian - H_z (the xbar and ybar directions of Eq. rot), D_aa
// the centred order-2R second-derivative weights and D_ab (a != b) the product
// of centred order-2R first-derivative weights along a and b: at space order
// 16 the 769-point stencil of the paper's TTI figure (the 49-point star and
// the 16 x 16 squares of the xy, xz and yz planes through the point).  Time
// stepping, damping layer (strength from the fastest speed v sqrt(1+2 eps)),
// zero ghost, source scaling and trilinear points as in the isotropic path;
// the source enters both fields, receivers interpolate p.
//
// Step kernel (2.5D, one point per thread, a CTA owning a 32 x 8 xy tile and
// a run of z planes; k_tti_q, fd_tti_q.cuh): each plane of p and q enters
// once, by TMA, with an R-wide halo; its in-plane second derivatives and its
// first x and y differences are formed then, and every z sum (D_zz, D_xz,
// D_yz) runs over per-thread register queues, so shared memory holds only
// the entering plane, one plane of first x differences and the update's
// per-point tiles.  The model enters through six per-cell fields
// (dt^2 v^2 / h^2, 1 + 2 eps, sqrt(1 + 2 delta) and the axis n), computed
// once per model in double precision.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/fd.h"
#include "fd_aux.h"
#include "fd_internal.h"
#include "fd_runtime.h"
#include "fd_tti_q.cuh"

namespace fd {
void fd_weights(int R, double* c);
double cfl_limit(const double* c, int R);
}  // namespace fd

using namespace fd;

struct fd_tti_s {
  fd_grid_desc d;
  int R = 1;
  int Nx = 0, Ny = 0, Nz = 0, pitch = 0;
  size_t ncell = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* p[2] = {nullptr, nullptr};  // p[cur] = p^n, p[cur^1] = p^{n-1}
  float* q[2] = {nullptr, nullptr};
  float* coef = nullptr;  // six padded fields: A, e2, dl, nx, ny, nz
  int cur = 0;
  bool model_set = false;
  double vmax = 0.0, cfl = 0.0;
  float bscale = 0.0f;
  double c[kMaxR + 1] = {}, d1[kMaxR + 1] = {};
  DevBuf inj, rec, stage_val, stage_rec, stage_in, scratch;
  DevBuf err;  // error word of the TMA kernel's bounded waits
  // tensor maps of the step kernel, per buffer
  CUtensorMap halo_p[2], halo_q[2], tile_p[2], tile_q[2], coef_map;
  long long spin_limit = 0;
  int n_inj = 0, n_rec = 0;
  bool profiling = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double step_ms = 0.0;
  long long steps_timed = 0;
};

namespace {

struct TtiInj {
  long long off;
  int x, y, z;
  float w;  // trilinear weight / h
  int col;
};

struct TtiRec {
  long long off[8];
  float w[8];
};

__device__ __forceinline__ int depth(int g, int nbl, int n) {
  int d = nbl - g;
  const int e = g - (n + nbl - 1);
  d = d > e ? d : e;
  return d > 0 ? d : 0;
}

// Model fields on the padded, pitched grid (edge replication into the layer),
// in double, rounded once: A = dt^2 v^2 / h^2, 1 + 2 eps, sqrt(1 + 2 delta),
// n = (sin t cos p, sin t sin p, cos t).
__global__ void k_tti_coef(const float* __restrict__ vp, const float* __restrict__ eps,
                           const float* __restrict__ del, const float* __restrict__ th,
                           const float* __restrict__ ph, int nx, int ny, int nz, int nbl,
                           int Nx, int Ny, int pitch, size_t ncell, double dt2_h2,
                           float* __restrict__ coef) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= pitch) return;
  const size_t o = (static_cast<size_t>(z) * Ny + y) * pitch + x;
  if (x >= Nx) {
    for (int f = 0; f < 6; ++f) coef[f * ncell + o] = 0.f;
    return;
  }
  const int px = min(max(x - nbl, 0), nx - 1);
  const int py = min(max(y - nbl, 0), ny - 1);
  const int pz = min(max(z - nbl, 0), nz - 1);
  const size_t i = (static_cast<size_t>(pz) * ny + py) * nx + px;
  const double v = vp[i], t = th[i], p = ph[i];
  coef[o] = static_cast<float>(dt2_h2 * v * v);
  coef[ncell + o] = static_cast<float>(1.0 + 2.0 * static_cast<double>(eps[i]));
  coef[2 * ncell + o] = static_cast<float>(sqrt(1.0 + 2.0 * static_cast<double>(del[i])));
  coef[3 * ncell + o] = static_cast<float>(sin(t) * cos(p));
  coef[4 * ncell + o] = static_cast<float>(sin(t) * sin(p));
  coef[5 * ncell + o] = static_cast<float>(cos(t));
}

// max of v sqrt(1+2 eps) (bits of a non-negative float) and the count of
// invalid cells (v not positive, 1+2eps or 1+2delta not positive, anything
// not finite).
__global__ void k_tti_stats(const float* __restrict__ vp, const float* __restrict__ eps,
                            const float* __restrict__ del, const float* __restrict__ th,
                            const float* __restrict__ ph, size_t n, unsigned int* out) {
  float hi = 0.f;
  int bad = 0;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float v = vp[i], e = eps[i], d = del[i];
    if (!(v > 0.f) || !isfinite(v) || !(1.f + 2.f * e > 0.f) || !isfinite(e) ||
        !(1.f + 2.f * d > 0.f) || !isfinite(d) || !isfinite(th[i]) || !isfinite(ph[i])) {
      ++bad;
      continue;
    }
    hi = fmaxf(hi, v * sqrtf(1.f + 2.f * e));
  }
  for (int o = 16; o > 0; o >>= 1) {
    hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(hi));
    if (bad) atomicAdd(out + 1, static_cast<unsigned int>(bad));
  }
}

// rec[row][r] = sum_k w_k p[off_k]
__global__ void k_tti_gather(const float* __restrict__ p, const TtiRec* __restrict__ recs, int n,
                             float* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const TtiRec e = recs[r];
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc = fmaf(e.w[k], p[e.off[k]], acc);
  out[r] = acc;
}

// p, q at each source node += A w q(t_n) / (h (1 + b)) (s^n = w q / h^3 scaled
// by dt^2 v^2 and the damping division of the update)
__global__ void k_tti_inject(const TtiInj* __restrict__ inj, int n, const float* __restrict__ val,
                             const float* __restrict__ A, float bscale, int nbl, int nx, int ny,
                             int nz, float* p, float* q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const TtiInj e = inj[i];
  const int dx = depth(e.x, nbl, nx), dy = depth(e.y, nbl, ny), dz = depth(e.z, nbl, nz);
  const float b = bscale * static_cast<float>(dx * dx + dy * dy + dz * dz);
  const float s = A[e.off] * e.w * val[e.col] / (1.f + b);
  atomicAdd(p + e.off, s);
  atomicAdd(q + e.off, s);
}

template <int R>
cudaError_t launch_q(const tti::QMaps& M, const tti::QArgs& qa, dim3 grid, cudaStream_t s) {
  static unsigned long long done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(done & (1ull << (dev & 63)))) {
    cudaError_t e = cudaFuncSetAttribute(tti::k_tti_q<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(tti::QGeom<R>::SMEM));
    if (e) return e;
    done |= 1ull << (dev & 63);
  }
  tti::k_tti_q<R><<<grid, tti::kQT, tti::QGeom<R>::SMEM, s>>>(M, qa);
  return cudaGetLastError();
}

cudaError_t launch_q_r(int R, const tti::QMaps& M, const tti::QArgs& qa, dim3 grid,
                       cudaStream_t s) {
  count_launch();
  switch (R) {
    case 1: return launch_q<1>(M, qa, grid, s);
    case 2: return launch_q<2>(M, qa, grid, s);
    case 3: return launch_q<3>(M, qa, grid, s);
    case 4: return launch_q<4>(M, qa, grid, s);
    case 5: return launch_q<5>(M, qa, grid, s);
    case 6: return launch_q<6>(M, qa, grid, s);
    case 7: return launch_q<7>(M, qa, grid, s);
    case 8: return launch_q<8>(M, qa, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Centred first-derivative weights of order 2R:
// d_j = (-1)^(j+1) (R!)^2 / (j (R-j)! (R+j)!), d_0 = 0.
void first_weights(int R, double* d) {
  d[0] = 0.0;
  for (int j = 1; j <= R; ++j) {
    double ratio = 1.0;  // (R!)^2 / ((R-j)! (R+j)!)
    for (int k = 1; k <= j; ++k) ratio *= double(R - k + 1) / double(R + k);
    d[j] = ((j & 1) ? 1.0 : -1.0) * ratio / double(j);
  }
}

fd_status stage(fd_tti t, DevBuf& buf, const float* p, size_t n, size_t off_floats,
                const float** out) {
  if (is_device_ptr(p)) {
    *out = p;
    return FD_OK;
  }
  cudaError_t e = cudaMemcpyAsync(static_cast<float*>(buf.p) + off_floats, p, n * sizeof(float),
                                  cudaMemcpyHostToDevice, t->stream);
  if (e) return cuda_fail(e, "host to device copy");
  *out = static_cast<const float*>(buf.p) + off_floats;
  return FD_OK;
}

fd_status locate(fd_tti t, const float* xyz, int i0[3], double f[3]) {
  const int n[3] = {t->d.nx, t->d.ny, t->d.nz};
  for (int a = 0; a < 3; ++a) {
    const double s = double(xyz[a]) / t->d.h;
    if (!(s >= 0.0) || s > double(n[a] - 1))
      return fail(FD_ERR_ARG, "point (%g, %g, %g) outside the physical box", xyz[0], xyz[1],
                  xyz[2]);
    const double fl = floor(s);
    i0[a] = int(fl) + t->d.nbl;
    f[a] = s - fl;
  }
  return FD_OK;
}

size_t offset(fd_tti t, int x, int y, int z) {
  return (size_t(z) * t->Ny + y) * t->pitch + x;
}

fd_status tables(fd_tti t, const fd_points* src, const fd_points* rec) {
  std::vector<TtiInj> inj;
  std::vector<TtiRec> recs;
  const int N[3] = {t->Nx, t->Ny, t->Nz};
  for (int p = 0; p < (src ? src->n : 0); ++p) {
    int i0[3];
    double f[3];
    fd_status st = locate(t, src->xyz + 3 * p, i0, f);
    if (st) return st;
    for (int c = 0; c < 8; ++c) {
      int node[3];
      double w = 1.0;
      for (int a = 0; a < 3; ++a) {
        const int hi = (c >> a) & 1;
        node[a] = i0[a] + hi;
        w *= hi ? f[a] : 1.0 - f[a];
      }
      if (w == 0.0 || node[0] >= N[0] || node[1] >= N[1] || node[2] >= N[2]) continue;
      inj.push_back({(long long)offset(t, node[0], node[1], node[2]), node[0], node[1], node[2],
                     float(w / t->d.h), p});
    }
  }
  for (int p = 0; p < (rec ? rec->n : 0); ++p) {
    int i0[3];
    double f[3];
    fd_status st = locate(t, rec->xyz + 3 * p, i0, f);
    if (st) return st;
    TtiRec e;
    for (int c = 0; c < 8; ++c) {
      int node[3];
      double w = 1.0;
      for (int a = 0; a < 3; ++a) {
        const int hi = (c >> a) & 1;
        node[a] = i0[a] + hi;
        w *= hi ? f[a] : 1.0 - f[a];
      }
      const bool ok = node[0] < N[0] && node[1] < N[1] && node[2] < N[2];
      e.off[c] = ok ? (long long)offset(t, node[0], node[1], node[2]) : 0;
      e.w[c] = ok ? float(w) : 0.f;
    }
    recs.push_back(e);
  }
  cudaError_t e = t->inj.ensure(std::max<size_t>(inj.size() * sizeof(TtiInj), 16));
  if (!e) e = t->rec.ensure(std::max<size_t>(recs.size() * sizeof(TtiRec), 16));
  if (!e && !inj.empty())
    e = cudaMemcpyAsync(t->inj.p, inj.data(), inj.size() * sizeof(TtiInj),
                        cudaMemcpyHostToDevice, t->stream);
  if (!e && !recs.empty())
    e = cudaMemcpyAsync(t->rec.p, recs.data(), recs.size() * sizeof(TtiRec),
                        cudaMemcpyHostToDevice, t->stream);
  if (!e) e = cudaStreamSynchronize(t->stream);
  if (e) return cuda_fail(e, "point tables");
  t->n_inj = int(inj.size());
  t->n_rec = int(recs.size());
  return FD_OK;
}

fd_status copy_state(fd_tti t, float* dev, void* user, bool to_user) {
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof(p));
  cudaPitchedPtr dv = make_cudaPitchedPtr(dev, size_t(t->pitch) * 4, t->Nx * 4, t->Ny);
  cudaPitchedPtr us = make_cudaPitchedPtr(user, size_t(t->Nx) * 4, t->Nx * 4, t->Ny);
  p.srcPtr = to_user ? dv : us;
  p.dstPtr = to_user ? us : dv;
  p.extent = make_cudaExtent(size_t(t->Nx) * 4, t->Ny, t->Nz);
  p.kind = cudaMemcpyDefault;
  cudaError_t e = cudaMemcpy3DAsync(&p, t->stream);
  if (e) return cuda_fail(e, "wavefield copy");
  return FD_OK;
}

fd_status propagate(fd_tti t, int n0, int nsteps, const fd_points* src, const float* wavelet,
                    const fd_points* rec, float* rec_out) {
  if (!t->model_set) return fail(FD_ERR_STATE, "fd_tti_set_model has not been called");
  if (n0 < 0 || nsteps < 0) return fail(FD_ERR_ARG, "negative step range");
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;
  if ((nsrc && (!src->xyz || !wavelet)) || (nrec && (!rec->xyz || !rec_out)))
    return fail(FD_ERR_ARG, "points given without their data array");
  fd_status st = tables(t, src, rec);
  if (st) return st;
  cudaError_t e;
  const float* dval = nullptr;
  if (nsrc) {
    const size_t n = size_t(n0 + nsteps) * nsrc;
    if (!is_device_ptr(wavelet) && (e = t->stage_val.ensure(n * 4))) return cuda_fail(e, "staging");
    if ((st = stage(t, t->stage_val, wavelet, n, 0, &dval))) return st;
  }
  float* drec = nullptr;
  if (nrec) {
    if (is_device_ptr(rec_out)) {
      drec = rec_out;
    } else {
      if ((e = t->stage_rec.ensure(size_t(nsteps) * nrec * 4))) return cuda_fail(e, "staging");
      drec = static_cast<float*>(t->stage_rec.p);
    }
  }
  // the step kernel's arguments; its z chunks are cut so that the launch
  // fills at least four waves of the resident CTAs
  tti::QArgs qa;
  memset(&qa, 0, sizeof(qa));
  qa.err = static_cast<int*>(t->err.p);
  qa.Nx = t->Nx;
  qa.Ny = t->Ny;
  qa.Nz = t->Nz;
  qa.pitch = t->pitch;
  qa.nbl = t->d.nbl;
  qa.nx = t->d.nx;
  qa.ny = t->d.ny;
  qa.nz = t->d.nz;
  qa.spin_limit = t->spin_limit;
  qa.bscale = t->bscale;
  for (int j = 0; j <= kMaxR; ++j) {
    qa.c[j] = j <= t->R ? float(t->c[j]) : 0.f;
    qa.d[j] = j <= t->R ? float(t->d1[j]) : 0.f;
  }
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long cols = (long long)((t->Nx + tti::kQX - 1) / tti::kQX) *
                           ((t->Ny + tti::kQY - 1) / tti::kQY);
    const long long want = 4LL * (t->R <= 4 ? 2 : 1) * std::max(sms, 1);
    int chunks = int(std::max<long long>(1, (want + cols - 1) / cols));
    chunks = std::min(chunks, std::max(1, t->Nz / (8 * t->R)));
    qa.zchunk = (t->Nz + chunks - 1) / chunks;
  }
  const dim3 qgrid((t->Nx + tti::kQX - 1) / tti::kQX, (t->Ny + tti::kQY - 1) / tti::kQY,
                   (t->Nz + qa.zchunk - 1) / qa.zchunk);
  if (t->profiling) cudaEventRecord(t->ev0, t->stream);
  for (int s = 0; s < nsteps; ++s) {
    const int cur = t->cur;
    if (nrec) {
      k_tti_gather<<<(nrec + 127) / 128, 128, 0, t->stream>>>(
          t->p[cur], static_cast<const TtiRec*>(t->rec.p), nrec, drec + size_t(s) * nrec);
      count_launch();
    }
    tti::QMaps M;
    M.halo_p = t->halo_p[cur];
    M.halo_q = t->halo_q[cur];
    M.prev_p = t->tile_p[cur ^ 1];
    M.prev_q = t->tile_q[cur ^ 1];
    M.coef = t->coef_map;
    qa.pn = t->p[cur ^ 1];
    qa.qn = t->q[cur ^ 1];
    if ((e = launch_q_r(t->R, M, qa, qgrid, t->stream))) return cuda_fail(e, "TTI step launch");
    if (t->n_inj) {
      k_tti_inject<<<(t->n_inj + 127) / 128, 128, 0, t->stream>>>(
          static_cast<const TtiInj*>(t->inj.p), t->n_inj, dval + size_t(n0 + s) * nsrc, t->coef,
          t->bscale, t->d.nbl, t->d.nx, t->d.ny, t->d.nz, t->p[cur ^ 1], t->q[cur ^ 1]);
      count_launch();
    }
    t->cur = cur ^ 1;
  }
  if (t->profiling) {
    cudaEventRecord(t->ev1, t->stream);
    if ((e = cudaEventSynchronize(t->ev1))) return cuda_fail(e, "profiling event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t->ev0, t->ev1);
    t->step_ms += ms;
    t->steps_timed += nsteps;
  }
  if ((e = cudaGetLastError())) return cuda_fail(e, "TTI launch");
  if (nrec) {
    int bad = 0;
    e = count_nonfinite(drec, size_t(nsteps) * nrec, reinterpret_cast<int*>(t->scratch.p), &bad,
                        t->stream);
    if (e) return cuda_fail(e, "finite check");
    if (bad) return fail(FD_ERR_NONFINITE, "%d receiver samples are NaN or Inf", bad);
    if (drec != rec_out && nsteps > 0) {
      e = cudaMemcpyAsync(rec_out, drec, size_t(nsteps) * nrec * 4, cudaMemcpyDeviceToHost,
                          t->stream);
      if (e) return cuda_fail(e, "device to host copy");
    }
  }
  e = cudaStreamSynchronize(t->stream);
  if (e) return cuda_fail(e, "stream synchronize");
  if (nsteps > 0) {
    int flag = 0;
    e = cudaMemcpyAsync(&flag, t->err.p, sizeof(flag), cudaMemcpyDeviceToHost, t->stream);
    if (!e) e = cudaStreamSynchronize(t->stream);
    if (e) return cuda_fail(e, "error word");
    if (flag) {
      cudaMemsetAsync(t->err.p, 0, sizeof(int), t->stream);
      cudaStreamSynchronize(t->stream);
      return fail(FD_ERR_TIMEOUT, "a bounded wait of the TTI step ran out");
    }
  }
  return FD_OK;
}

}  // namespace

extern "C" {

fd_status fd_tti_create(const fd_grid_desc* d, fd_tti* out) {
  clear_error();
  if (!d || !out) return fail(FD_ERR_ARG, "null argument");
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(FD_ERR_ARG, "grid sizes must be positive");
  if (!(d->h > 0.0) || !(d->dt > 0.0)) return fail(FD_ERR_ARG, "h and dt must be positive");
  if (d->space_order < 2 || d->space_order > 16 || (d->space_order & 1))
    return fail(FD_ERR_ARG, "space_order must be even, 2..16");
  if (d->nbl < 0 || d->nt < 0) return fail(FD_ERR_ARG, "nbl and nt must be >= 0");
  const long long Nx = d->nx + 2LL * d->nbl, Ny = d->ny + 2LL * d->nbl, Nz = d->nz + 2LL * d->nbl;
  if (Nx > (1 << 24) || Ny > 65535 || Nz > 65535) return fail(FD_ERR_ARG, "padded grid too large");
  cudaError_t e = cudaSetDevice(d->device);
  if (e) return cuda_fail(e, "cudaSetDevice");
  fd_tti t = new fd_tti_s();
  t->d = *d;
  t->R = d->space_order / 2;
  t->Nx = int(Nx);
  t->Ny = int(Ny);
  t->Nz = int(Nz);
  t->pitch = int((Nx + 31) / 32 * 32);
  t->ncell = size_t(t->pitch) * t->Ny * t->Nz;
  fd_weights(t->R, t->c);
  first_weights(t->R, t->d1);
  t->cfl = cfl_limit(t->c, t->R);
  fd_status st = FD_OK;
  if (d->stream) {
    t->stream = static_cast<cudaStream_t>(d->stream);
  } else {
    e = cudaStreamCreateWithFlags(&t->stream, cudaStreamDefault);
    if (e) st = cuda_fail(e, "stream create");
    t->own_stream = true;
  }
  for (int b = 0; b < 2 && !st; ++b) {
    e = dev_alloc(reinterpret_cast<void**>(&t->p[b]), t->ncell * 4);
    if (!e) e = dev_alloc(reinterpret_cast<void**>(&t->q[b]), t->ncell * 4);
    if (e) st = cuda_fail(e, "wavefield allocation");
  }
  if (!st) {
    e = dev_alloc(reinterpret_cast<void**>(&t->coef), 6 * t->ncell * 4);
    if (!e) e = t->scratch.ensure(64);
    if (!e) e = t->err.ensure(16);
    if (!e) e = cudaMemsetAsync(t->err.p, 0, 16, t->stream);
    if (e) st = cuda_fail(e, "model allocation");
  }
  t->spin_limit = default_spin_limit();
  if (!st) {
    // tensor maps of the TMA kernel: staged planes with the x halo rounded
    // up to four floats and R rows, per-point tiles, the six model fields
    // stacked along z
    const int W = tti::kQX + 2 * ((t->R + 3) / 4 * 4), H = tti::kQY + 2 * t->R;
    for (int b = 0; b < 2 && !st; ++b) {
      st = make_map(&t->halo_p[b], t->p[b], t->Nx, t->Ny, t->Nz, t->pitch, W, H);
      if (!st) st = make_map(&t->halo_q[b], t->q[b], t->Nx, t->Ny, t->Nz, t->pitch, W, H);
      if (!st)
        st = make_map(&t->tile_p[b], t->p[b], t->Nx, t->Ny, t->Nz, t->pitch, tti::kQX, tti::kQY);
      if (!st)
        st = make_map(&t->tile_q[b], t->q[b], t->Nx, t->Ny, t->Nz, t->pitch, tti::kQX, tti::kQY);
    }
    if (!st)
      st = make_map(&t->coef_map, t->coef, t->Nx, t->Ny, 6 * t->Nz, t->pitch, tti::kQX,
                    tti::kQY);
  }
  if (!st) {
    for (int b = 0; b < 2 && !e; ++b) {
      e = cudaMemsetAsync(t->p[b], 0, t->ncell * 4, t->stream);
      if (!e) e = cudaMemsetAsync(t->q[b], 0, t->ncell * 4, t->stream);
    }
    if (!e) e = cudaMemsetAsync(t->coef, 0, 6 * t->ncell * 4, t->stream);
    if (!e) e = cudaEventCreate(&t->ev0);
    if (!e) e = cudaEventCreate(&t->ev1);
    if (!e) e = cudaStreamSynchronize(t->stream);
    if (e) st = cuda_fail(e, "grid initialisation");
  }
  if (st) {
    fd_tti_destroy(t);
    return st;
  }
  *out = t;
  return FD_OK;
}

fd_status fd_tti_destroy(fd_tti t) {
  if (!t) return FD_OK;
  cudaSetDevice(t->d.device);
  if (t->stream) cudaStreamSynchronize(t->stream);
  for (int b = 0; b < 2; ++b) {
    if (t->p[b]) cudaFree(t->p[b]);
    if (t->q[b]) cudaFree(t->q[b]);
  }
  if (t->coef) cudaFree(t->coef);
  for (DevBuf* b : {&t->inj, &t->rec, &t->stage_val, &t->stage_rec, &t->stage_in, &t->scratch,
                    &t->err})
    b->release();
  if (t->ev0) cudaEventDestroy(t->ev0);
  if (t->ev1) cudaEventDestroy(t->ev1);
  if (t->own_stream && t->stream) cudaStreamDestroy(t->stream);
  delete t;
  return FD_OK;
}

fd_status fd_tti_set_model(fd_tti t, const float* vp, const float* epsilon, const float* delta,
                           const float* theta, const float* phi) {
  clear_error();
  if (!t || !vp || !epsilon || !delta || !theta || !phi) return fail(FD_ERR_ARG, "null argument");
  cudaSetDevice(t->d.device);
  const size_t np = size_t(t->d.nx) * t->d.ny * t->d.nz;
  const float* in[5] = {vp, epsilon, delta, theta, phi};
  const float* dev[5];
  bool host = false;
  for (int f = 0; f < 5; ++f) host |= !is_device_ptr(in[f]);
  cudaError_t e;
  if (host && (e = t->stage_in.ensure(5 * np * 4))) return cuda_fail(e, "model staging");
  for (int f = 0; f < 5; ++f) {
    fd_status st = stage(t, t->stage_in, in[f], np, size_t(f) * np, &dev[f]);
    if (st) return st;
  }
  // the staging copy of host arrays is only needed inside this call: freed
  // on every return, after the work that reads it has finished
  struct Release {
    DevBuf& b;
    cudaStream_t s;
    ~Release() {
      if (b.p) cudaStreamSynchronize(s);
      b.release();
    }
  } release_staging{t->stage_in, t->stream};
  unsigned int h[2] = {0, 0};
  unsigned int* s = static_cast<unsigned int*>(t->scratch.p);
  e = cudaMemsetAsync(s, 0, 8, t->stream);
  if (!e) {
    k_tti_stats<<<1024, 256, 0, t->stream>>>(dev[0], dev[1], dev[2], dev[3], dev[4], np, s);
    count_launch();
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(h, s, 8, cudaMemcpyDeviceToHost, t->stream);
  if (!e) e = cudaStreamSynchronize(t->stream);
  if (e) return cuda_fail(e, "model statistics");
  if (h[1]) return fail(FD_ERR_ARG, "%u model cells are invalid", h[1]);
  float vmax;
  memcpy(&vmax, &h[0], 4);
  const double courant = double(vmax) * t->d.dt / t->d.h;
  if (courant > t->cfl)
    return fail(FD_ERR_UNSTABLE, "v_max sqrt(1+2 eps) dt / h = %.4f exceeds the limit %.4f",
                courant, t->cfl);
  dim3 grid((t->pitch + 127) / 128, t->Ny, t->Nz);
  k_tti_coef<<<grid, 128, 0, t->stream>>>(dev[0], dev[1], dev[2], dev[3], dev[4], t->d.nx,
                                          t->d.ny, t->d.nz, t->d.nbl, t->Nx, t->Ny, t->pitch,
                                          t->ncell, t->d.dt * t->d.dt / (t->d.h * t->d.h), t->coef);
  count_launch();
  if ((e = cudaGetLastError())) return cuda_fail(e, "model set-up");
  t->vmax = vmax;
  if (t->d.nbl > 0) {
    const double gmax = 3.0 * double(vmax) * log(1000.0) / (2.0 * t->d.nbl * t->d.h);
    t->bscale = float(gmax * t->d.dt / 2.0 / (double(t->d.nbl) * t->d.nbl));
  } else {
    t->bscale = 0.f;
  }
  for (int b = 0; b < 2 && !e; ++b) {
    e = cudaMemsetAsync(t->p[b], 0, t->ncell * 4, t->stream);
    if (!e) e = cudaMemsetAsync(t->q[b], 0, t->ncell * 4, t->stream);
  }
  if (!e) e = cudaStreamSynchronize(t->stream);
  if (e) return cuda_fail(e, "model set-up");
  t->cur = 0;
  t->model_set = true;
  return FD_OK;
}

fd_status fd_tti_forward(fd_tti t, const fd_points* src, const float* wavelet,
                         const fd_points* rec, float* rec_out) {
  clear_error();
  if (!t) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(t->d.device);
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaMemsetAsync(t->p[b], 0, t->ncell * 4, t->stream);
    if (!e) e = cudaMemsetAsync(t->q[b], 0, t->ncell * 4, t->stream);
    if (e) return cuda_fail(e, "wavefield reset");
  }
  t->cur = 0;
  return propagate(t, 0, t->d.nt, src, wavelet, rec, rec_out);
}

fd_status fd_tti_propagate(fd_tti t, int32_t n0, int32_t nsteps, const fd_points* src,
                           const float* wavelet, const fd_points* rec, float* rec_out) {
  clear_error();
  if (!t) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(t->d.device);
  return propagate(t, n0, nsteps, src, wavelet, rec, rec_out);
}

fd_status fd_tti_set_state(fd_tti t, const float* p_prev, const float* p, const float* q_prev,
                           const float* q) {
  clear_error();
  if (!t) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(t->d.device);
  const float* in[4] = {p_prev, p, q_prev, q};
  float* dst[4] = {t->p[t->cur ^ 1], t->p[t->cur], t->q[t->cur ^ 1], t->q[t->cur]};
  for (int f = 0; f < 4; ++f) {
    if (!in[f]) continue;
    fd_status st = copy_state(t, dst[f], const_cast<float*>(in[f]), false);
    if (st) return st;
  }
  cudaError_t e = cudaStreamSynchronize(t->stream);
  if (e) return cuda_fail(e, "wavefield copy");
  return FD_OK;
}

fd_status fd_tti_get_state(fd_tti t, float* p_prev, float* p, float* q_prev, float* q) {
  clear_error();
  if (!t) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(t->d.device);
  float* out[4] = {p_prev, p, q_prev, q};
  float* src[4] = {t->p[t->cur ^ 1], t->p[t->cur], t->q[t->cur ^ 1], t->q[t->cur]};
  for (int f = 0; f < 4; ++f) {
    if (!out[f]) continue;
    fd_status st = copy_state(t, src[f], out[f], true);
    if (st) return st;
  }
  cudaError_t e = cudaStreamSynchronize(t->stream);
  if (e) return cuda_fail(e, "wavefield copy");
  return FD_OK;
}

fd_status fd_tti_set_profiling(fd_tti t, int32_t enabled) {
  clear_error();
  if (!t) return fail(FD_ERR_ARG, "null grid");
  t->profiling = enabled != 0;
  if (t->profiling) {
    t->step_ms = 0.0;
    t->steps_timed = 0;
  }
  return FD_OK;
}

fd_status fd_tti_get_info(fd_tti t, fd_grid_info* info) {
  clear_error();
  if (!t || !info) return fail(FD_ERR_ARG, "null argument");
  memset(info, 0, sizeof(*info));
  info->nx_pad = t->Nx;
  info->ny_pad = t->Ny;
  info->nz_pad = t->Nz;
  info->pitch = t->pitch;
  info->tile_x = tti::kQX;
  info->tile_y = tti::kQY;
  info->v_max = t->vmax;
  info->cfl_limit = t->cfl;
  info->launches = fd_launch_count();
  info->step_ms = t->step_ms;
  info->steps_timed = t->steps_timed;
  return FD_OK;
}

}  // extern "C"
