// Adjoint-state gradient of the receiver misfit with respect to m.
//
// The forward recurrence (damped leapfrog of Eq. 1)
//     D u^{n+1} = 2u^n - E u^{n-1} + M (L u^n + s^n),  D = 1+b, E = 1-b, M = dt^2/m
// has, for J = 1/2 sum_n ||I(u^n) - d^n||^2, the exact discrete adjoint
//     D z^n = 2z^{n+1} - E z^{n+2} + M (L z^{n+1} + I^T r^n),  z^{nt} = z^{nt+1} = 0,
// i.e. the same step run backwards in time with the residual injected through
// the transpose of the receiver interpolation (L is symmetric), and
//     dJ/dm = - sum_n z^{n+1} e^{n+1} / dt^2,   e^{n+1} = M (L u^n + s^n),
// folded from the padded grid onto the physical cells that the layer
// replicates.  (The paper names FWI/RTM as users of these propagators,
// Sec. I and IV-B; the adjoint itself is derived here from the recurrence.)
//
// Memory plan: the forward sweep keeps (u^{k-1}, u^k) at the start of each of
// `nc` segments in device memory; the backward sweep restores a segment,
// recomputes it storing e per step (one field per step of the segment), then
// runs the adjoint steps of that segment, which fuse the imaging condition.
#include <string.h>

#include <algorithm>
#include <vector>

#include "fd_aux.h"
#include "fd_runtime.h"

using namespace fd;

namespace {

fd_status ensure_adjoint_fields(fd_grid g) {
  if (g->Z.u[0] && g->Z.u[1]) return FD_OK;
  for (int b = 0; b < 2; ++b) {
    if (g->Z.u[b]) continue;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&g->Z.u[b]), g->ncell * 4);
    if (e) return cuda_fail(e, "adjoint wavefield allocation");
  }
  return build_field_maps(g, g->Z);
}

fd_status copy_async(fd_grid g, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, g->stream);
  if (e) return cuda_fail(e, "device copy");
  return FD_OK;
}

// Shared body of fd_adjoint_gradient (d_obs given) and fd_backward
// (residual given).
fd_status adjoint_impl(fd_grid g, const fd_points* src, const float* wavelet,
                       const fd_points* rec, const float* d_obs, const float* resid_in,
                       int32_t n_checkpoints, float* grad_m, double* loss_out) {
  {
    // the adjoint's launches (recompute and adjoint modes) take the tuner's
    // pick of tile and schedule for the grid's size, as plain forward runs do
    // (every tile and schedule gives the same bits)
    fd_status st0 = use_shape(g, true);
    if (st0) return st0;
  }
  if (!g->model_set) return fail(FD_ERR_STATE, "fd_set_model has not been called");
  if (g->percell || g->table_mode)
    return fail(FD_ERR_STATE, "the adjoint is built for the symmetric uniform-weight stencil");
  const int nt = g->d.nt;
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;
  if (!grad_m) return fail(FD_ERR_ARG, "grad_m is required");
  if ((nsrc && (!src->xyz || !wavelet)) || (nrec && !rec->xyz))
    return fail(FD_ERR_ARG, "points given without their data array");
  if (nrec && !d_obs && !resid_in) return fail(FD_ERR_ARG, "d_obs or residual is required");
  const int nc = std::max(1, std::min(n_checkpoints, std::max(nt, 1)));
  const int L = nt > 0 ? (nt + nc - 1) / nc : 0;
  const int nseg = L > 0 ? (nt + L - 1) / L : 0;
  const size_t cell_bytes = g->ncell * 4;
  cudaError_t e;
  fd_status st;

  // a grid left on the default tile is tuned by its first long run, whether
  // that is a forward run or this one (source-free steps on zeroed
  // wavefields), before the point tables are built for the tile in use
  if (g->auto_tile && !g->tuned && g->sched_mode == FD_SCHED_AUTO && !g->dmp && !g->cart &&
      nt >= kTuneMinSteps && g->debug_skip_plane < 0) {
    for (int b = 0; b < 2; ++b)
      if ((e = cudaMemsetAsync(g->F.u[b], 0, cell_bytes, g->stream)))
        return cuda_fail(e, "wavefield reset");
    g->F.cur = 0;
    if ((st = autotune_grid(g))) return st;
  }
  if ((st = ensure_adjoint_fields(g))) return st;
  if ((e = g->ckpt.ensure(std::max<size_t>(size_t(std::max(nseg - 1, 0)) * 2 * cell_bytes, 16))))
    return cuda_fail(e, "checkpoint allocation");
  if ((e = g->ebuf.ensure(std::max<size_t>(size_t(L) * cell_bytes, 16))))
    return cuda_fail(e, "imaging buffer allocation");
  if ((e = g->gpad.ensure(cell_bytes))) return cuda_fail(e, "gradient allocation");
  if ((e = g->recbuf.ensure(std::max<size_t>(size_t(nt) * nrec * 4, 16))))
    return cuda_fail(e, "receiver buffer allocation");
  if ((e = g->resid.ensure(std::max<size_t>(size_t(nt) * nrec * 4 + 64, 80))))
    return cuda_fail(e, "residual allocation");

  // tables: forward injection (1/h) and gather, adjoint injection at the
  // receivers (transpose of the gather, scaled by h^2 as A holds 1/h^2)
  if ((st = upload_tables(g, src, 1.0 / g->d.h, rec, g->tab))) return st;
  if ((st = upload_tables(g, rec, g->d.h * g->d.h, nullptr, g->tab_adj))) return st;
  const float* dval = nullptr;
  if ((st = stage_in(g, g->stage_val, nsrc ? wavelet : nullptr, size_t(nt) * nsrc, &dval)))
    return st;

  // ---- forward sweep with checkpoints --------------------------------------
  for (int b = 0; b < 2; ++b)
    if ((e = cudaMemsetAsync(g->F.u[b], 0, cell_bytes, g->stream)))
      return cuda_fail(e, "wavefield reset");
  g->F.cur = 0;
  float* drec = static_cast<float*>(g->recbuf.p);
  char* ck = static_cast<char*>(g->ckpt.p);
  for (int s = 0; s < nseg; ++s) {
    const int n0 = s * L, n1 = std::min(nt, n0 + L);
    if (s > 0) {
      char* slot = ck + size_t(s - 1) * 2 * cell_bytes;
      if ((st = copy_async(g, slot, g->F.u[g->F.cur ^ 1], cell_bytes))) return st;
      if ((st = copy_async(g, slot + cell_bytes, g->F.u[g->F.cur], cell_bytes))) return st;
    }
    RunSpec rs;
    memset(&rs, 0, sizeof(rs));
    rs.f = &g->F;
    rs.mode = kModeForward;
    rs.nsteps = n1 - n0;
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
      rs.rec_row0 = n0;
      rs.rec_row_step = 1;
    }
    if ((st = run_steps(g, rs))) return st;
  }
  if ((st = check_device_error(g))) return st;

  // ---- residual -------------------------------------------------------------
  float* dres = static_cast<float*>(g->resid.p);
  double* dloss = reinterpret_cast<double*>(static_cast<char*>(g->resid.p) +
                                            ((size_t(nt) * nrec * 4 + 15) / 16) * 16);
  if (nrec) {
    if ((st = check_finite(g, drec, size_t(nt) * nrec))) return st;
    if (d_obs) {
      const float* dobs = nullptr;
      if ((st = stage_in(g, g->stage_aux, d_obs, size_t(nt) * nrec, &dobs))) return st;
      if ((e = residual(drec, dobs, dres, size_t(nt) * nrec, dloss, g->stream)))
        return cuda_fail(e, "residual");
    } else {
      const float* dr = nullptr;
      if ((st = stage_in(g, g->stage_aux, resid_in, size_t(nt) * nrec, &dr))) return st;
      if ((st = copy_async(g, dres, dr, size_t(nt) * nrec * 4))) return st;
      if ((e = cudaMemsetAsync(dloss, 0, sizeof(double), g->stream)))
        return cuda_fail(e, "loss reset");
    }
  }

  // ---- backward sweep ---------------------------------------------------------
  if ((e = cudaMemsetAsync(g->gpad.p, 0, cell_bytes, g->stream)))
    return cuda_fail(e, "gradient reset");
  for (int b = 0; b < 2; ++b)
    if ((e = cudaMemsetAsync(g->Z.u[b], 0, cell_bytes, g->stream)))
      return cuda_fail(e, "adjoint reset");
  g->Z.cur = 0;
  float* ebase = static_cast<float*>(g->ebuf.p);
  for (int s = nseg - 1; s >= 0; --s) {
    const int n0 = s * L, n1 = std::min(nt, n0 + L);
    // restore (u^{n0-1}, u^{n0}) and recompute the segment storing e^{n+1}
    g->F.cur = 0;
    if (s == 0) {
      for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(g->F.u[b], 0, cell_bytes, g->stream)))
          return cuda_fail(e, "wavefield reset");
    } else {
      const char* slot = ck + size_t(s - 1) * 2 * cell_bytes;
      if ((st = copy_async(g, g->F.u[1], slot, cell_bytes))) return st;
      if ((st = copy_async(g, g->F.u[0], slot + cell_bytes, cell_bytes))) return st;
    }
    RunSpec rf;
    memset(&rf, 0, sizeof(rf));
    rf.f = &g->F;
    rf.mode = kModeStoreE;
    rf.nsteps = n1 - n0;
    rf.e_base = ebase;
    if (nsrc) {
      rf.inj_start = static_cast<const int32_t*>(g->tab.inj_start.p);
      rf.inj = static_cast<const InjEntry*>(g->tab.inj.p);
      rf.inj_val = dval;
      rf.inj_ncol = nsrc;
      rf.inj_row0 = n0;
      rf.inj_row_step = 1;
    }
    if ((st = run_steps(g, rf))) return st;
    // adjoint steps n = n1-1 .. n0: z^n from z^{n+1}, z^{n+2}; imaging with
    // z^{n+1} and e^{n+1} (stored at index n - n0)
    RunSpec ra;
    memset(&ra, 0, sizeof(ra));
    ra.f = &g->Z;
    ra.mode = kModeAdjoint;
    ra.nsteps = n1 - n0;
    ra.e_base = ebase;
    ra.e_idx0 = n1 - 1 - n0;
    ra.e_idx_step = -1;
    ra.grad = static_cast<float*>(g->gpad.p);
    if (nrec) {
      ra.inj_start = static_cast<const int32_t*>(g->tab_adj.inj_start.p);
      ra.inj = static_cast<const InjEntry*>(g->tab_adj.inj.p);
      ra.inj_val = dres;
      ra.inj_ncol = nrec;
      ra.inj_row0 = n1 - 1;
      ra.inj_row_step = -1;
    }
    if ((st = run_steps(g, ra))) return st;
  }
  if ((st = check_device_error(g))) return st;

  // ---- fold onto the physical grid -------------------------------------------
  const size_t np = size_t(g->d.nx) * g->d.ny * g->d.nz;
  float* dgrad = nullptr;
  if ((st = stage_out(g, g->stage_aux, grad_m, np, &dgrad))) return st;
  if ((e = fold_grad(static_cast<const float*>(g->gpad.p), g->d.nx, g->d.ny, g->d.nz,
                     g->d.nbl, g->Nx, g->Ny, g->Nz, g->pitch, dgrad, g->stream)))
    return cuda_fail(e, "gradient fold");
  if ((st = finish_out(g, grad_m, dgrad, np))) return st;
  if (loss_out) {
    double h = 0.0;
    if (nrec) {
      e = cudaMemcpyAsync(&h, dloss, sizeof(double), cudaMemcpyDeviceToHost, g->stream);
      if (e) return cuda_fail(e, "loss read");
    }
    e = cudaStreamSynchronize(g->stream);
    if (e) return cuda_fail(e, "stream synchronize");
    *loss_out = h;
  }
  e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "stream synchronize");
  return FD_OK;
}

}  // namespace

extern "C" {

fd_status fd_adjoint_gradient(fd_grid g, const fd_points* src, const float* wavelet,
                              const fd_points* rec, const float* d_obs,
                              int32_t n_checkpoints, float* grad_m, double* loss_out) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  cudaSetDevice(g->d.device);
  return adjoint_impl(g, src, wavelet, rec, d_obs, nullptr, n_checkpoints, grad_m, loss_out);
}

fd_status fd_backward(fd_grid g, const fd_points* src, const float* wavelet,
                      const fd_points* rec, const float* grad_rec, int32_t n_checkpoints,
                      float* grad_m) {
  clear_error();
  if (!g) return fail(FD_ERR_ARG, "null grid");
  if (rec && rec->n && !grad_rec) return fail(FD_ERR_ARG, "grad_rec is required");
  cudaSetDevice(g->d.device);
  return adjoint_impl(g, src, wavelet, rec, nullptr, grad_rec, n_checkpoints, grad_m,
                      nullptr);
}

}  // extern "C"
