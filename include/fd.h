/*
 * fd.h -- C ABI of libfd.so: explicit high-order finite-difference time
 * stepping of the isotropic acoustic wave equation on one GB300 (sm_103a).
 *
 * The operation (paper: "Automated MPI-X code generation for scalable
 * finite-difference solvers", Eq. 1 in App. A and Sec. IV-B/IV-C):
 *
 *     m(x) u_tt - Laplace(u) + eta(x) u_t = delta(x - x_s) q(t),
 *     u = u_t = 0 at t = 0,   d(t) = u(t, x_r),   m = 1/c^2,
 *
 * discretised with the centred order-2R second-derivative stencil in each
 * axis (space order SO = 2R, 2..16) and second-order leapfrog in time, with a
 * sponge layer of `nbl` cells added outside each face of the physical grid in
 * which eta = m * gamma(x) damps outgoing waves (Sec. IV-C: "40-point deep
 * ABC").  One step is
 *
 *     (1+b) u^{n+1} = 2 u^n - (1-b) u^{n-1} + (dt^2/m) (L u^n + s^n),
 *
 * b = gamma dt / 2, gamma = gamma_max * sum_a (depth_a / nbl)^2,
 * gamma_max = 3 v_max ln(1000) / (2 nbl h); the ghost cells beyond the layer
 * are zero (Sec. III "Access alignment": the halo is read-only).  Sources
 * are injected and receivers interpolated with trilinear weights (Sec. III
 * "Sparse data"); s^n = sum_src w q(t_n) / h^3 and rec[n] = I(u^n).
 *
 * Beyond that step the library has: the adjoint gradient (fd_adjoint_gradient,
 * fd_backward), many shots per launch (fd_batch_forward), learned stencil
 * weights (fd_mlp_*, fd_set_learned_*), work schedules and their tuning
 * (fd_set_tile, fd_set_schedule), a z decomposition into slabs with halo
 * exchange on the device (fd_set_decomposition, Sec. III), the model update
 * of an inversion loop (fd_descent_step), the anisotropic TTI system of
 * Sec. IV-B (fd_tti_*) and a forward run that allocates nothing
 * (fd_forward_noalloc).
 *
 * Units: h in metres, dt in milliseconds, velocity in km/s, m in (ms/m)^2.
 *
 * Memory: every float array argument may be HOST or DEVICE memory on the
 * grid's device; the library tells them apart with cudaPointerGetAttributes
 * and stages host data through its own device buffers.  Point coordinate
 * tables (fd_points.xyz) are host memory.  The caller owns every pointer it
 * passes; the library never frees or retains them past the call.  The
 * library owns all grid buffers (wavefields, model, checkpoints, tables).
 *
 * Ordering: calls run on the grid's stream and return after the work has
 * completed, so the returned status reflects completion.  A grid must not be
 * used from two threads at once.  Errors are returned as fd_status codes and
 * never thrown across the ABI; fd_last_error() gives a thread-local message.
 */
#ifndef FD_H
#define FD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fd_grid_s* fd_grid; /* opaque, library-owned */

typedef enum {
  FD_OK = 0,
  FD_ERR_ARG = 1,       /* invalid argument (sizes, points outside the box) */
  FD_ERR_CUDA = 2,      /* a CUDA call failed (message in fd_last_error) */
  FD_ERR_OOM = 3,       /* device allocation failed */
  FD_ERR_UNSTABLE = 4,  /* v_max dt / h above the stability limit */
  FD_ERR_STATE = 5,     /* call out of order (e.g. no model set) */
  FD_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out */
  FD_ERR_NONFINITE = 7  /* NaN or Inf in the receiver data */
} fd_status;

/* kinds for fd_set_model */
enum { FD_MODEL_VP_KMS = 0, /* P velocity in km/s */
       FD_MODEL_M = 1 };    /* squared slowness m = 1/v^2 in (ms/m)^2 */

/* regions for fd_set_wavefield / fd_get_wavefield */
enum { FD_REGION_PHYSICAL = 0, /* nz*ny*nx physical cells */
       FD_REGION_PADDED = 1 };  /* (nz+2nbl)*(ny+2nbl)*(nx+2nbl) cells */

typedef struct {
  int32_t nx, ny, nz;    /* physical cells, x fastest in every array */
  double h;              /* grid spacing [m], the same on all axes */
  int32_t space_order;   /* even, 2..16 */
  int32_t nbl;           /* sponge cells added outside each face (>= 0) */
  double dt;             /* time step [ms] */
  int32_t nt;            /* number of steps run by fd_forward */
  int32_t device;        /* CUDA device ordinal */
  void* stream;          /* cudaStream_t to run on, or NULL for an own one */
} fd_grid_desc;

typedef struct {
  int32_t n;             /* number of points */
  const float* xyz;      /* host [n][3], metres from physical cell (0,0,0);
                            each point must satisfy 0 <= x <= (nx-1) h etc. */
} fd_points;

typedef struct {
  int32_t nx_pad, ny_pad, nz_pad; /* padded (physical + 2 nbl) extents */
  int32_t pitch;                  /* floats between rows of device arrays */
  int32_t tile_x, tile_y, ctas;   /* stencil tile and persistent CTAs per sweep */
  double v_max;                   /* from the model, km/s */
  double cfl_limit;               /* largest stable v_max dt / h */
  int64_t launches;               /* library kernels launched so far */
  double step_ms;                 /* summed device time of profiled steps */
  int64_t steps_timed;            /* steps inside that time */
  int32_t schedule;               /* of the last forward run: FD_SCHED_SHARES,
                                     FD_SCHED_WAVES or FD_SCHED_TEMPORAL (0 before
                                     the first run) */
} fd_grid_info;

/* Creates a grid; allocates the two wavefields and the model on `device`.
 * Errors: FD_ERR_ARG (sizes), FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_create_grid(const fd_grid_desc* desc, fd_grid* out);

/* Frees every buffer of the grid.  NULL is accepted. */
fd_status fd_destroy_grid(fd_grid grid);

/* Sets the medium from nz*ny*nx physical values (`kind` FD_MODEL_*), padded
 * into the sponge by edge replication, and resets the wavefields to zero.
 * Errors: FD_ERR_ARG (non-positive or non-finite values), FD_ERR_UNSTABLE
 * (v_max dt / h above the limit sqrt(4 / (3 S)), S = -c0 - 2 sum (-1)^j c_j). */
fd_status fd_set_model(fd_grid grid, const float* data, int32_t kind);

/* Forward modelling from rest (Eq. 1): runs desc.nt steps.
 *   wavelet  [nt][src->n] source signatures q(t_n), t_n = n dt
 *   rec_out  [nt][rec->n] receives I(u^n), n = 0..nt-1 (rec_out[0] = 0)
 *   u_out    optional nz*ny*nx physical u^{nt} (NULL to skip)
 * Errors: FD_ERR_STATE (no model), FD_ERR_ARG (points), FD_ERR_TIMEOUT,
 * FD_ERR_NONFINITE (receiver data not finite). */
fd_status fd_forward(fd_grid grid, const fd_points* src, const float* wavelet,
                     const fd_points* rec, float* rec_out, float* u_out);

/* Continues from the current wavefield state (u^{n0-1}, u^{n0}) for
 * `nsteps` steps, using wavelet rows n0..n0+nsteps-1 (wavelet has
 * n0+nsteps rows) and writing rec_out rows 0..nsteps-1 = I(u^{n0+t}).
 * src, rec, wavelet and rec_out may be NULL for a source-free run. */
fd_status fd_propagate(fd_grid grid, int32_t n0, int32_t nsteps,
                       const fd_points* src, const float* wavelet,
                       const fd_points* rec, float* rec_out);

/* Replaces / reads the state (u^{n-1}, u^n); either pointer may be NULL. */
fd_status fd_set_wavefield(fd_grid grid, const float* u_prev,
                           const float* u_cur, int32_t region);
fd_status fd_get_wavefield(fd_grid grid, float* u_prev, float* u_cur,
                           int32_t region);

/* Gradient of J = 1/2 sum_n ||I(u^n) - d_obs[n]||^2 with respect to the
 * physical squared slowness m (nz*ny*nx floats), by the adjoint-state method
 * with `n_checkpoints` stored states and recomputation between them.  The
 * layer strength gamma_max is held fixed.  d_obs is [nt][rec->n]; the loss
 * is written to *loss_out if not NULL.  Errors as fd_forward. */
fd_status fd_adjoint_gradient(fd_grid grid, const fd_points* src,
                              const float* wavelet, const fd_points* rec,
                              const float* d_obs, int32_t n_checkpoints,
                              float* grad_m, double* loss_out);

/* Vector-Jacobian product: grad_m = (d rec / d m)^T grad_rec, with grad_rec
 * [nt][rec->n] (the residual slot of the adjoint).  Used by autograd. */
fd_status fd_backward(fd_grid grid, const fd_points* src, const float* wavelet,
                      const fd_points* rec, const float* grad_rec,
                      int32_t n_checkpoints, float* grad_m);

/* Many independent shots (each its own grid, all with the same space order,
 * nt and layer width nbl) advanced together: each time step is one
 * persistent launch over a shared {shot, tile} work list; the nt launches
 * are captured in a CUDA
 * graph when flags has FD_BATCH_GRAPH.  FD_BATCH_AUTOTUNE times the tile
 * candidates once per (space order, window sizes) and caches the choice.
 * All grids must be on the same device; the first grid's stream is used. */
enum { FD_BATCH_GRAPH = 1, FD_BATCH_AUTOTUNE = 2 };
typedef struct {
  fd_grid grid;
  const fd_points* src;
  const float* wavelet;   /* [nt][src->n] */
  const fd_points* rec;
  float* rec_out;         /* [nt][rec->n] */
} fd_shot;
fd_status fd_batch_forward(int32_t nshots, const fd_shot* shots,
                           int32_t flags);

/* Domain decomposition along z (Sec. III: the grid is split into
 * subdomains that each exchange an R-deep halo with their neighbours, in a
 * "basic" mode that exchanges before every step and a "full" mode that
 * overlaps the exchange with the CORE points, whose stencils need no halo,
 * and computes the REMAINDER afterwards).  With nsub > 1 the padded grid's
 * nz + 2 nbl planes are cut into nsub contiguous slabs of balanced size
 * (sizes differ by at most one plane); each slab keeps its own two
 * wavefields and model term with R ghost planes on either side, and every
 * later fd_forward / fd_propagate on this grid steps the slabs:
 *   FD_DMP_BASIC    per step, one launch per slab, then device copies that
 *                   refill every inner ghost plane with the neighbour's
 *                   edge planes (one copy per face and direction: a z face
 *                   is contiguous, so nothing is packed);
 *   FD_DMP_OVERLAP  per step, first the R planes beside each inner face of
 *                   every slab, then their copies to the neighbours on a
 *                   second stream while the remaining (core) planes are
 *                   computed; the next step waits for the copies.
 * Every point is computed exactly as in the undecomposed run, so receivers
 * and wavefields are the same bit for bit; the whole-grid state is scattered
 * into the slabs before a run and gathered back after it, so fd_get_wavefield
 * and u_out see the usual layout.  All slabs live on the grid's device.
 * The slabs add 3 (nz + 2 nbl + 2 R nsub) planes of device memory, allocated
 * here.  nsub = 1 removes the decomposition.  fd_adjoint_gradient,
 * fd_backward and fd_batch_forward ignore it and step the whole grid; the
 * FD_DEBUG_SKIP_PLANE hook does not reach slab runs.
 * Errors: FD_ERR_ARG (bad mode; a slab would hold fewer than R planes, 2R in
 * overlap mode), FD_ERR_OOM, FD_ERR_CUDA; a run with per-cell weight fields
 * returns FD_ERR_STATE. */
enum { FD_DMP_BASIC = 0, FD_DMP_OVERLAP = 1 };
fd_status fd_set_decomposition(fd_grid grid, int32_t nsub, int32_t mode);

/* Cartesian domain decomposition (Sec. III: a topology of px x py x pz ranks,
 * each owning a box of the grid and exchanging an R-deep halo with its
 * neighbours before every step).  The padded extents are split per axis into
 * balanced ranges (sizes differ by at most one point); box (i, j, k), x
 * fastest, keeps its two wavefields and model term with ghost layers (R
 * rounded up to four floats in x, R in y and z), and every later
 * fd_forward / fd_propagate on this grid steps all boxes in one launch per
 * step (column waves over the boxes one after another; equal shares under
 * FD_SCHED_SHARES or an explicit CTA count).  After the step a pack kernel copies the R updated layers next to
 * each face with a neighbour into that face's contiguous message, and an
 * unpack kernel fills every ghost block from them: faces from the face
 * neighbour's message, edges and corners (read by receivers next to two or
 * three cuts; the stencil reads faces only) from sub-blocks of the diagonal
 * neighbour's face messages.  Every point is computed exactly as in the
 * undecomposed run (receivers and wavefields equal bit for bit); the
 * whole-grid state is scattered before a run and gathered after it.  All
 * boxes live on the grid's device; across GPUs each message would be one
 * peer copy (or NCCL send/recv) into the receiver's memory before the unpack.
 * px = py = pz = 1 removes the topology; setting one removes any slabs of
 * fd_set_decomposition and the reverse.  fd_adjoint_gradient, fd_backward and
 * fd_batch_forward step the whole grid; temporal blocking is not applied to
 * boxes.
 * Errors: FD_ERR_ARG (a size < 1; a box thinner than R points along a split
 * axis), FD_ERR_OOM, FD_ERR_CUDA; a run with per-cell or table weights
 * returns FD_ERR_STATE. */
fd_status fd_set_topology(fd_grid grid, int32_t px, int32_t py, int32_t pz);

/* One model update of a full-waveform-inversion loop (the paper names FWI
 * as a user of the propagator, Sec. I and IV-B, without an update rule):
 * normalised steepest descent on n values,
 *     alpha = step * max|m| / max|grad|,
 *     m[i] <- min(max(m[i] - alpha grad[i], m_min), m_max),
 * so the largest change is `step` times the model's scale.  m (updated in
 * place) and grad are DEVICE arrays on the current device; the work runs on
 * `stream` (NULL: the legacy default stream) and has completed on return.
 * *alpha_out (optional) receives alpha; a zero gradient (or step 0) leaves m
 * unchanged with alpha 0.  Errors: FD_ERR_ARG (n < 0, null or host arrays,
 * step < 0, m_min > m_max), FD_ERR_NONFINITE (NaN or Inf in grad; m is then
 * unchanged), FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_descent_step(int64_t n, float* m, const float* grad, double step,
                          double m_min, double m_max, void* stream,
                          double* alpha_out);

/* Chooses the stencil tile (tile_x x tile_y points per CTA column) and the
 * number of persistent CTAs of each step launch (and turns off the tuning
 * of FD_SCHED_AUTO for this grid).  Each CTA sweeps an equal
 * contiguous share of the grid's (tile, z plane) units.  ctas = 0 picks the
 * count: when all tile columns fit in the CTAs resident at once, k equal z
 * chunks per column (all columns advance together and share halos in L2),
 * else as many CTAs as are resident on all SMs.  Compiled tiles: 64x16,
 * 128x8, 32x16, 64x8, 32x8.  fd_create_grid starts from a default chosen by
 * the load of the busiest SM.
 * Errors: FD_ERR_ARG for a tile that is not compiled or ctas < 0. */
fd_status fd_set_tile(fd_grid grid, int32_t tile_x, int32_t tile_y, int32_t ctas);

/* How the persistent CTAs of a forward step share the grid's work units
 * (one xy tile column over a range of z planes each):
 *   FD_SCHED_SHARES  every resident CTA takes an equal contiguous share of
 *                    the (tile, plane) units; when all tile columns fit in
 *                    the resident CTAs, k equal z chunks per column instead
 *                    (lockstep: all columns advance together and neighbours
 *                    find each other's halo rows in L2);
 *   FD_SCHED_WAVES   columns cut into z chunks of a common height, handed to
 *                    the CTAs in waves of neighbouring chunks at the same
 *                    depth, so neighbours share halos in L2 however many
 *                    columns there are; the chunk height minimises the load
 *                    of the busiest CTA (a host-side simulation);
 *   FD_SCHED_AUTO    the default: equal shares, except that a grid left on
 *                    its default tile (no fd_set_tile call) is tuned by its
 *                    first fd_forward, fd_adjoint_gradient or fd_backward of
 *                    at least 400 steps: every compiled tile is timed under
 *                    both schedules for a few source-free steps on the
 *                    zeroed wavefields (cleared again before the run), twice,
 *                    and the fastest pair serves all later runs of grids of
 *                    that padded size and kernel mode on that device
 *                    (fd_forward, fd_propagate and the adjoint; the pick is
 *                    cached per process; fd_grid_info shows the tile and
 *                    schedule in use).
 *   FD_SCHED_TEMPORAL  temporal blocking (the paper's Discussion, Sec. IV,
 *                    names it as future work): space orders 4 and 8 with
 *                    uniform weights advance two steps per pass over the
 *                    grid, reading u^{n-1}, u^n and the model once and
 *                    writing u^{n+1} and u^{n+2} to a second pair of
 *                    wavefield buffers (allocated on first use: two more
 *                    grid fields); the first step is recomputed on an R-wide
 *                    halo of each 56 x 24 (SO 8) or 56 x 28 (SO 4) tile.  An
 *                    odd step count ends with one single step.  Other space
 *                    orders, per-cell or table weights and decomposed grids
 *                    run single steps with equal shares instead.
 * The adjoint's steps (fd_adjoint, fd_gradient) and table-weight forward
 * steps follow the same choice as plain forward runs (the tuner's tile and
 * schedule once the grid has been tuned); per-cell weight fields always use
 * equal shares on the default tile, and so does an explicit CTA count
 * (fd_set_tile ctas > 0).  Every schedule and tile gives the same results
 * bit for bit.
 * Errors: FD_ERR_ARG (unknown mode). */
enum { FD_SCHED_AUTO = 0, FD_SCHED_SHARES = 1, FD_SCHED_WAVES = 2, FD_SCHED_TEMPORAL = 3 };
fd_status fd_set_schedule(fd_grid grid, int32_t mode);

/* Test hooks, host-side fault injection only:
 *   FD_DEBUG_SKIP_PLANE  value z >= 0: the first step of the next run never
 *                        issues the load of padded plane z, so the bounded
 *                        waits for it run out and the call returns
 *                        FD_ERR_TIMEOUT; -1 turns it off
 *   FD_DEBUG_SPIN_LIMIT  clock cycles a device-side wait may take (> 0)
 *   FD_DEBUG_NO_GRAPH    1: launch steps one by one instead of a CUDA graph
 * Device allocations can be made to fail with FD_ERR_OOM by setting the
 * environment variable FD_FAULT_ALLOC_AT=k (k-th allocation, 1-based). */
enum { FD_DEBUG_SKIP_PLANE = 1, FD_DEBUG_SPIN_LIMIT = 2, FD_DEBUG_NO_GRAPH = 3 };
fd_status fd_set_debug(fd_grid grid, int32_t key, int64_t value);

/* Stencil weights.  FD_COEF_TAYLOR restores the order-2R Taylor weights;
 * FD_COEF_UNIFORM takes c[0..R] (c[0] the centre weight per axis);
 * FD_COEF_PER_CELL takes physical [nz][ny][nx][R] weights c_1..c_R per cell
 * (c_0 = -2 sum c_j per cell), padded into the layer by edge replication;
 * per-cell weights are compiled for space order 8 and forward runs only
 * (fd_adjoint_gradient / fd_batch_forward then return FD_ERR_STATE).
 * Errors: FD_ERR_ARG. */
enum { FD_COEF_TAYLOR = 0, FD_COEF_UNIFORM = 1, FD_COEF_PER_CELL = 2 };
fd_status fd_set_coefficients(fd_grid grid, const float* c, int32_t mode);

/* ---- learned per-cell weights (no counterpart in the paper; follows the
 * learned-discretisation idea of Bar-Sinai et al., PNAS 2019) -------------
 * A 4 -> 64 -> 64 -> 8 ReLU network (FP32) maps x = [v dt/h, h/10 m,
 * dt/1 ms, f/10 Hz] to outputs o_1..o_8; s_j = (o_j + o_{j+4})/2 and
 * c_j = cT_j (1 + tanh(s_j)/2), j = 1..4, cT the SO 8 Taylor weights, so a
 * zero output layer reproduces the plain stencil.  Parameters (5000 floats):
 * W1[64][4] b1[64] W2[64][64] b2[64] W3[8][64] b3[8].  A training sample is
 * 10 floats: x[4], T[4] (T_j = sum of the 6 neighbours at distance j minus
 * 6 u), target y and weight w; loss (1/n) sum w (sum_j c_j T_j - y)^2. */
#define FD_MLP_NPARAM 5000
#define FD_MLP_SAMPLE 10
typedef struct fd_mlp_s* fd_mlp;
/* params: FD_MLP_NPARAM floats (host or device) or NULL for zeros. */
fd_status fd_mlp_create(int32_t device, const float* params, fd_mlp* out);
fd_status fd_mlp_destroy(fd_mlp net);
fd_status fd_mlp_get_params(fd_mlp net, float* out);
/* also resets the Adam state */
fd_status fd_mlp_set_params(fd_mlp net, const float* in);
/* loss and gradient over n samples ([n][FD_MLP_SAMPLE]); grad_out optional */
fd_status fd_mlp_loss_grad(fd_mlp net, int64_t n, const float* samples, double* loss,
                           float* grad_out);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient */
fd_status fd_mlp_adam_step(fd_mlp net, float lr);
/* `epochs` passes over the samples in mini-batches of `batch`, one Adam step
 * per mini-batch; *loss_out = loss of the whole set at the end */
fd_status fd_mlp_train(fd_mlp net, int64_t n, const float* samples, int32_t epochs,
                       int32_t batch, float lr, double* loss_out);
/* inference: coef_out[n][4] = c_1..c_4 of features[n][4] */
fd_status fd_mlp_coefficients(fd_mlp net, int64_t n, const float* features, float* coef_out);
/* per-cell weights of every cell of a space-order-8 grid from its model,
 * computed by the network on the device (call after fd_set_model) */
fd_status fd_set_learned_coefficients(fd_grid grid, fd_mlp net, double f_hz);
/* The same weights without per-cell fields: for fixed h, dt and f the
 * network's input varies only with the Courant number C = v dt / h, so the
 * network is evaluated (on the device) at `nodes` values A_i evenly spaced
 * from (v_min dt/h)^2 to (v_max dt/h)^2 of the current model (input
 * C_i = sqrt(A_i)), and each point of every step takes c_1..c_4 interpolated
 * linearly in A between the two nodes around its own A = dt^2 v^2 / h^2
 * (clamped to the end nodes).  The step then moves the 16 bytes per point of
 * the plain stencil instead of 32.  The
 * table is rebuilt by the next call, and dropped by fd_set_coefficients or
 * fd_set_learned_coefficients; call again after fd_set_model.
 * Errors: FD_ERR_ARG (null, space order not 8, nodes outside [2, 256]),
 * FD_ERR_STATE (no model), FD_ERR_CUDA. */
fd_status fd_set_learned_table(fd_grid grid, fd_mlp net, double f_hz, int32_t nodes);
/* Training-data helpers.  fd_sample_stencil writes, for each padded cell
 * (x, y, z) of cells[n][3], the current wavefield at the cell and at
 * distances j*stride (j = 1..radius) along -x, +x, -y, +y, -z, +z:
 * out[n][1 + 6 radius]; outside the grid reads 0.  fd_mlp_make_samples
 * turns three such arrays (radius 4; coarse times t-dt, t, t+dt) and the
 * velocity at each cell into samples: x as above, T_j from `cur`,
 * y = (next - 2 cur + prev) / C^2 with C = v dt / h at the centre, and
 * w = 1 / (scale + mean square of the cur stencil).  Device arrays only. */
fd_status fd_sample_stencil(fd_grid grid, int32_t n, const int32_t* cells, int32_t stride,
                            int32_t radius, float* out);
fd_status fd_mlp_make_samples(int32_t n, const float* prev, const float* cur, const float* next,
                              const float* vel, double h, double dt, double f_hz, double scale,
                              float* out);

/* Forward modelling for callers that cannot allocate device memory (for
 * example while another framework owns the memory pool and forbids new
 * cudaMalloc calls, or when the device footprint must stay fixed).  It does
 * what fd_create_grid + fd_set_model + fd_forward + fd_destroy_grid do, but
 * every buffer it needs (wavefields, model term, tables, descriptors) lives in
 * one static device array of FD_NOALLOC_MAX_BYTES that the library keeps on
 * each GPU that loads it, and it calls no allocating routine.  The paper has
 * no counterpart of this entry point.
 *   desc     as for fd_create_grid (desc->stream may be NULL: legacy stream);
 *            no graph, events or stream are created
 *   model    DEVICE array, nz*ny*nx values of `kind` (FD_MODEL_*)
 *   wavelet  DEVICE [nt][src->n];  rec_out DEVICE [nt][rec->n]
 * Errors: FD_ERR_ARG when the padded grid and tables do not fit in the array
 * (the message gives the bytes needed) or an array is host memory; otherwise
 * as fd_set_model and fd_forward.  Each call whose stream is not being
 * captured looks up the array's device address (cudaGetSymbolAddress), so a
 * cudaDeviceReset by the caller between calls is harmless; a call on a
 * capturing stream reuses the address found by the device's last call, so
 * make the first call on a device before any stream capture.  Device waits
 * give up after FD_SPIN_LIMIT clock cycles when that variable is set, as for
 * fd_create_grid.  All calls share the array and leave the last call's
 * contents in it; calls that overlap on the GPU race and must be serialised
 * by the caller. */
#define FD_NOALLOC_MAX_BYTES (32 * 1024 * 1024)
fd_status fd_forward_noalloc(const fd_grid_desc* desc, const float* model, int32_t kind,
                             const fd_points* src, const float* wavelet,
                             const fd_points* rec, float* rec_out);

/* ---- Anisotropic acoustic (TTI) propagation -------------------------------
 * Sec. IV-B ("Anisotropic acoustic") and App. A (Eq. rot): two fields p, q
 * coupled through a rotated anisotropic Laplacian (the pseudo-acoustic system
 * of Zhang et al. 2011, the formulation the paper cites):
 *     m p_tt + eta p_t = (1+2 eps) H_0 p + sqrt(1+2 delta) H_z q + s,
 *     m q_tt + eta q_t = sqrt(1+2 delta) H_0 p + H_z q + s,
 * H_z u = sum_ab n_a n_b D_ab u with the symmetry axis
 * n = (sin(theta) cos(phi), sin(theta) sin(phi), cos(theta)) (theta the tilt,
 * phi the azimuth, per cell; Eq. rot's xbar = (cos t cos p, cos t sin p,
 * -sin t) and ybar = n x xbar complete the rotated frame), H_0 = Laplacian
 * - H_z, D_aa the centred order-2R second-derivative weights and D_ab (a != b)
 * the product of the centred order-2R first-derivative weights along a and
 * b (at space order 16 the paper's 769-point TTI stencil).  Leapfrog in time
 * with the damping layer, zero ghost, source scaling and trilinear points of
 * the isotropic path; the layer strength uses v_max sqrt(1+2 eps_max); the
 * source enters p and q, receivers record I(p^n).  The grid descriptor,
 * units, memory rules and error codes are those of fd_grid; the library owns
 * six model fields and two wavefields of each of p and q. */
typedef struct fd_tti_s* fd_tti;
fd_status fd_tti_create(const fd_grid_desc* desc, fd_tti* out);
fd_status fd_tti_destroy(fd_tti grid);
/* Physical nz*ny*nx arrays (host or device): vp [km/s], Thomsen epsilon and
 * delta, tilt theta and azimuth phi [rad]; padded into the layer by edge
 * replication; resets the wavefields.  Errors: FD_ERR_ARG (vp not positive,
 * 1+2 eps or 1+2 delta not positive, a value not finite), FD_ERR_UNSTABLE
 * (v_max sqrt(1+2 eps_max) dt / h above the isotropic limit of the space
 * order; strongly tilted media may need a larger margin). */
fd_status fd_tti_set_model(fd_tti grid, const float* vp, const float* epsilon,
                           const float* delta, const float* theta, const float* phi);
/* desc.nt steps from rest; wavelet [nt][src->n], rec_out [nt][rec->n] = I(p^n).
 * Errors (here and in fd_tti_propagate): those of fd_forward; FD_ERR_TIMEOUT
 * when a bounded wait of the step kernel for its staged planes ran out (the
 * state is then undefined). */
fd_status fd_tti_forward(fd_tti grid, const fd_points* src, const float* wavelet,
                         const fd_points* rec, float* rec_out);
/* Continues from the current state for nsteps steps (wavelet rows
 * n0..n0+nsteps-1; rec_out rows 0..nsteps-1); pointers may be NULL. */
fd_status fd_tti_propagate(fd_tti grid, int32_t n0, int32_t nsteps, const fd_points* src,
                           const float* wavelet, const fd_points* rec, float* rec_out);
/* Replace / read the state (p^{n-1}, p^n, q^{n-1}, q^n) as padded
 * (nz+2nbl)(ny+2nbl)(nx+2nbl) arrays; any pointer may be NULL. */
fd_status fd_tti_set_state(fd_tti grid, const float* p_prev, const float* p,
                           const float* q_prev, const float* q);
fd_status fd_tti_get_state(fd_tti grid, float* p_prev, float* p, float* q_prev, float* q);
/* Device time of the steps of later runs (reset when enabled), reported by
 * fd_tti_get_info in step_ms / steps_timed with the grid's extents. */
fd_status fd_tti_set_profiling(fd_tti grid, int32_t enabled);
fd_status fd_tti_get_info(fd_tti grid, fd_grid_info* info);

/* Diagnostics. */
fd_status fd_get_info(fd_grid grid, fd_grid_info* info);
/* When enabled, fd_forward / fd_propagate / fd_batch_forward record CUDA
 * events around the step launches on the grid's stream and add the time to
 * fd_grid_info.step_ms. */
fd_status fd_set_profiling(fd_grid grid, int32_t enabled);
/* Library-wide count of kernel launches issued so far. */
int64_t fd_launch_count(void);
/* Library-wide count of the device allocations (cudaMalloc) the library has
 * made so far for grids, tables, staging and checkpoints. */
int64_t fd_alloc_count(void);

const char* fd_status_string(fd_status status);
const char* fd_last_error(void); /* thread-local; "" when none */

#ifdef __cplusplus
}
#endif

#endif /* FD_H */
