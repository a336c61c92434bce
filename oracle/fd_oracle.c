/*
 * FP64 CPU oracle for the explicit finite-difference acoustic time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the GPU path computes.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and it never imports it.
 *
 * What it follows (paper: "Automated MPI-X code generation for scalable
 * finite-difference solvers"):
 *   - Eq. 1 (App. A, isotropic acoustic): m u_tt - Laplace(u) = delta(x_s) q(t),
 *     u = u_t = 0 at t = 0, d(t) = u(t, x_r), m = 1/c^2.
 *   - Sec. IV-B ("Isotropic acoustic"): the update is obtained by solving the
 *     discretised equation for u.forward (explicit leapfrog, star stencil).
 *   - Sec. IV-C ("Problem setup"): a 40-cell absorbing layer is added outside
 *     the stated grid; the halo beyond it is read-only.
 *   - Sec. III ("Access alignment"): data / halo regions; with no neighbour the
 *     halo is a read-only ghost region, here zero.
 *   - Sec. III ("Sparse data"): off-grid sources are injected into, and
 *     receivers interpolated from, the grid points around them.
 *   - Sec. II, Listing 1 and Sec. III Listings 2-3: heat-diffusion worked
 *     example (forward Euler of u_t = Laplace(u)), used as an indexing pin.
 *
 * Readings where the paper is silent (each repeated in the design notes):
 *   - Laplacian weights: the unique centred second-derivative weights of
 *     order 2R, c_j = 2(-1)^{j+1}(R!)^2 / (j^2 (R-j)!(R+j)!), c_0 = -2 sum c_j.
 *   - Damping: eta = m*gamma(x), discretised centred in time, so the update is
 *       (1+b) u^{n+1} = 2u^n - (1-b) u^{n-1} + (dt^2/m)(L u^n + s^n),
 *     b = gamma dt/2, gamma = gamma_max * sum_a d_a^2, d_a the normalised
 *     depth into the layer along axis a, gamma_max = 3 v_max ln(1/Rc)/(2 nbl h).
 *   - The model inside the layer is the edge-replicated physical model.
 *   - Source: multilinear weights / h^dims (discrete delta); q sampled at t_n
 *     is injected into the update that produces u^{n+1}; rec[n] = I(u^n).
 *   - Multilinear weights: floor index i0 and fraction f along each axis,
 *     weights (1-f, f); a point exactly on a node puts weight 1 on it.
 *
 * Units: h in m, dt in ms, velocity in km/s (= m/ms), m in (ms/m)^2.
 *
 * Layout: padded arrays of N[0]*N[1]*N[2] doubles, x fastest, where
 * N[a] = n[a] + 2*nbl on active axes and 1 on inactive ones.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t dims;     /* number of active axes: 1 (x), 2 (x,y) or 3 (x,y,z) */
  int32_t n[3];     /* physical cells per axis (1 on inactive axes) */
  int32_t nbl;      /* absorbing-layer cells added outside each active face */
  int32_t R;        /* stencil half width; space order is 2R */
  int32_t periodic; /* 1: wrap-around neighbours instead of the zero ghost */
  int32_t pad_;
  double h;         /* grid spacing [m] */
  double dt;        /* time step [ms] */
  double rc;        /* target reflection coefficient of the layer */
} or_grid;

static void padded_dims(const or_grid* g, int64_t N[3]) {
  for (int a = 0; a < 3; ++a)
    N[a] = (a < g->dims) ? (int64_t)g->n[a] + 2 * (int64_t)g->nbl : 1;
}

int64_t or_ncell(const or_grid* g) {
  int64_t N[3];
  padded_dims(g, N);
  return N[0] * N[1] * N[2];
}

/* Centred second-derivative weights of order 2R (reading above). */
void or_fd_coefficients(int32_t R, double* c) {
  double sum = 0.0;
  for (int j = 1; j <= R; ++j) {
    /* (R!)^2 / ((R-j)! (R+j)!) = prod_{k=1..j} (R-k+1)/(R+k) */
    double ratio = 1.0;
    for (int k = 1; k <= j; ++k) ratio *= (double)(R - k + 1) / (double)(R + k);
    double sign = (j % 2 == 1) ? 1.0 : -1.0;
    c[j] = 2.0 * sign * ratio / ((double)j * (double)j);
    sum += c[j];
  }
  c[0] = -2.0 * sum;
}

/* Edge replication of the physical model into the absorbing layer. */
void or_pad_model(const or_grid* g, const double* m_phys, double* m_pad) {
  int64_t N[3];
  padded_dims(g, N);
  int nbl = g->nbl;
  for (int64_t k = 0; k < N[2]; ++k)
    for (int64_t j = 0; j < N[1]; ++j)
      for (int64_t i = 0; i < N[0]; ++i) {
        int64_t p[3] = {i, j, k};
        int64_t q[3];
        for (int a = 0; a < 3; ++a) {
          if (a < g->dims) {
            int64_t v = p[a] - nbl;
            if (v < 0) v = 0;
            if (v > g->n[a] - 1) v = g->n[a] - 1;
            q[a] = v;
          } else {
            q[a] = 0;
          }
        }
        m_pad[i + N[0] * (j + N[1] * k)] =
            m_phys[q[0] + (int64_t)g->n[0] * (q[1] + (int64_t)g->n[1] * q[2])];
      }
}

/* b = gamma*dt/2 per padded cell; gamma = gamma_max * sum_a d_a^2. */
void or_damping(const or_grid* g, double vmax, double* b) {
  int64_t N[3];
  padded_dims(g, N);
  double gmax = 0.0;
  if (g->nbl > 0)
    gmax = 3.0 * vmax * log(1.0 / g->rc) / (2.0 * g->nbl * g->h);
  for (int64_t k = 0; k < N[2]; ++k)
    for (int64_t j = 0; j < N[1]; ++j)
      for (int64_t i = 0; i < N[0]; ++i) {
        int64_t p[3] = {i, j, k};
        double s = 0.0;
        for (int a = 0; a < g->dims; ++a) {
          double lo = (double)(g->nbl - p[a]);
          double hi = (double)(p[a] - (g->n[a] + g->nbl - 1));
          double d = 0.0;
          if (lo > d) d = lo;
          if (hi > d) d = hi;
          if (g->nbl > 0) d /= g->nbl;
          s += d * d;
        }
        b[i + N[0] * (j + N[1] * k)] = gmax * s * g->dt / 2.0;
      }
}

/* Value of u at padded index p along axis a displaced by `off`, honouring the
 * zero ghost (or wrap-around). */
static double neighbour(const or_grid* g, const int64_t N[3], const double* u,
                        int64_t i, int64_t j, int64_t k, int a, int off) {
  int64_t p[3] = {i, j, k};
  p[a] += off;
  if (p[a] < 0 || p[a] >= N[a]) {
    if (!g->periodic) return 0.0;
    p[a] = ((p[a] % N[a]) + N[a]) % N[a];
  }
  return u[p[0] + N[0] * (p[1] + N[1] * p[2])];
}

/*
 * L u = h^-2 * sum over active axes of sum_{j=-R..R} c_|j| u(i + j e_a).
 * coef: [R+1] uniform weights, or NULL to use `percell` = [ncell][R+1]
 * weights that vary per cell (the centre weight is percell[.][0]).
 */
void or_laplacian(const or_grid* g, const double* coef, const double* percell,
                  const double* u, double* out) {
  int64_t N[3];
  padded_dims(g, N);
  int R = g->R;
  double ih2 = 1.0 / (g->h * g->h);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t k = 0; k < N[2]; ++k)
    for (int64_t j = 0; j < N[1]; ++j)
      for (int64_t i = 0; i < N[0]; ++i) {
        int64_t idx = i + N[0] * (j + N[1] * k);
        const double* c = coef ? coef : percell + idx * (R + 1);
        double acc = 0.0;
        for (int a = 0; a < g->dims; ++a) {
          acc += c[0] * u[idx];
          for (int r = 1; r <= R; ++r)
            acc += c[r] * (neighbour(g, N, u, i, j, k, a, r) +
                           neighbour(g, N, u, i, j, k, a, -r));
        }
        out[idx] = acc * ih2;
      }
}

/*
 * Multilinear weights of a point given in metres from the physical origin.
 * Writes up to 2^dims (padded index, weight) pairs; returns how many, or -1
 * if the point lies outside the physical box [0, (n-1) h] on an active axis.
 */
int32_t or_point_weights(const or_grid* g, const double* xyz, int64_t* idx,
                         double* w) {
  int64_t N[3];
  padded_dims(g, N);
  int64_t i0[3] = {0, 0, 0};
  double f[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < g->dims; ++a) {
    double s = xyz[a] / g->h;
    if (!(s >= 0.0) || s > (double)(g->n[a] - 1)) return -1;
    double fl = floor(s);
    i0[a] = (int64_t)fl + g->nbl;
    f[a] = s - fl;
  }
  int cnt = 0;
  int corners = 1 << g->dims;
  for (int c = 0; c < corners; ++c) {
    int64_t p[3] = {i0[0], i0[1], i0[2]};
    double wt = 1.0;
    for (int a = 0; a < g->dims; ++a) {
      int hi = (c >> a) & 1;
      p[a] += hi;
      wt *= hi ? f[a] : (1.0 - f[a]);
    }
    if (wt == 0.0) continue; /* far node of a point sitting on a node */
    if (p[0] >= N[0] || p[1] >= N[1] || p[2] >= N[2]) continue;
    idx[cnt] = p[0] + N[0] * (p[1] + N[1] * p[2]);
    w[cnt] = wt;
    ++cnt;
  }
  return cnt;
}

/*
 * One damped leapfrog step over every padded cell:
 *   u_next = (2 u_cur - (1-b) u_prev + (dt^2/m) (L u_cur + s)) / (1+b)
 * where s is zero except at the nsrc_nodes listed cells, which receive
 * src_val (already multiplied by q(t_n) and divided by h^dims).
 * If e_out is not NULL it receives (dt^2/m)(L u_cur + s).
 */
void or_step(const or_grid* g, const double* m_pad, const double* b,
             const double* coef, const double* percell, const double* u_prev,
             const double* u_cur, int32_t nsrc_nodes, const int64_t* src_idx,
             const double* src_val, double* scratch_L, double* u_next,
             double* e_out) {
  int64_t n = or_ncell(g);
  or_laplacian(g, coef, percell, u_cur, scratch_L);
  for (int32_t s = 0; s < nsrc_nodes; ++s) scratch_L[src_idx[s]] += src_val[s];
  double dt2 = g->dt * g->dt;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double e = dt2 / m_pad[i] * scratch_L[i];
    u_next[i] = (2.0 * u_cur[i] - (1.0 - b[i]) * u_prev[i] + e) / (1.0 + b[i]);
    if (e_out) e_out[i] = e;
  }
}

/*
 * The same damped leapfrog step on a z slab of the padded grid, as one rank of
 * a domain decomposition along z computes it (the paper's basic mode, Sec. III
 * "halo exchange": each subdomain reads R ghost planes of u^n from its
 * neighbours before the step).  Owned planes are nzs consecutive padded z
 * planes; u_cur_x holds them with R ghost planes before and after
 * ([nzs + 2R][N1][N0], zero where the ghost lies beyond the global grid);
 * m_pad_s, b_s, u_prev_s and u_next_s cover the owned planes only.  Sources
 * are not handled here.  Every point is summed in the order of or_laplacian
 * and updated as in or_step, so a decomposed run reproduces the undecomposed
 * one bit for bit.  Returns 0, or -1 for a grid that is not 3-D and
 * non-periodic.
 */
int32_t or_step_slab(const or_grid* g, const double* m_pad_s, const double* b_s,
                     const double* coef, const double* u_prev_s, const double* u_cur_x,
                     int64_t nzs, double* u_next_s) {
  if (g->dims != 3 || g->periodic) return -1;
  int64_t N[3];
  padded_dims(g, N);
  const int R = g->R;
  const double ih2 = 1.0 / (g->h * g->h);
  const double dt2 = g->dt * g->dt;
  const int64_t plane = N[0] * N[1];
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t kk = 0; kk < nzs; ++kk)
    for (int64_t j = 0; j < N[1]; ++j)
      for (int64_t i = 0; i < N[0]; ++i) {
        const int64_t o = i + N[0] * j;
        const double* uc = u_cur_x + (kk + R) * plane;  /* centre plane */
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) {
          acc += coef[0] * uc[o];
          for (int r = 1; r <= R; ++r) {
            double up_v, dn_v;
            if (a == 0) {
              up_v = i + r < N[0] ? uc[o + r] : 0.0;
              dn_v = i - r >= 0 ? uc[o - r] : 0.0;
            } else if (a == 1) {
              up_v = j + r < N[1] ? uc[o + r * N[0]] : 0.0;
              dn_v = j - r >= 0 ? uc[o - r * N[0]] : 0.0;
            } else {
              up_v = uc[o + r * plane];
              dn_v = uc[o - r * plane];
            }
            acc += coef[r] * (up_v + dn_v);
          }
        }
        const double L = acc * ih2;
        const int64_t idx = o + kk * plane;
        const double e = dt2 / m_pad_s[idx] * L;
        u_next_s[idx] = (2.0 * uc[o] - (1.0 - b_s[idx]) * u_prev_s[idx] + e) / (1.0 + b_s[idx]);
      }
  return 0;
}

/*
 * The same step on a block of a Cartesian domain decomposition (Sec. III: a
 * topology of px x py x pz ranks, each owning a box of the padded grid and
 * reading an R-wide halo of u^n from its neighbours).  The owned box has
 * nb[0] x nb[1] x nb[2] points (x fastest); u_cur_x holds it with R ghost
 * layers on every side ([nb2+2R][nb1+2R][nb0+2R], zero where the ghost lies
 * beyond the global grid); m_pad_b, b_b, u_prev_b and u_next_b cover the
 * owned box.  Sources are not handled here.  Each point is summed in the
 * order of or_laplacian and updated as in or_step, so a decomposed run
 * reproduces the undecomposed one bit for bit.  Returns 0, or -1 for a grid
 * that is not 3-D and non-periodic.
 */
int32_t or_step_block(const or_grid* g, const double* m_pad_b, const double* b_b,
                      const double* coef, const double* u_prev_b, const double* u_cur_x,
                      const int64_t* nb, double* u_next_b) {
  if (g->dims != 3 || g->periodic) return -1;
  const int R = g->R;
  const double ih2 = 1.0 / (g->h * g->h);
  const double dt2 = g->dt * g->dt;
  const int64_t X0 = nb[0] + 2 * R, X1 = nb[1] + 2 * R;
  const int64_t stride[3] = {1, X0, X0 * X1};
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t k = 0; k < nb[2]; ++k)
    for (int64_t j = 0; j < nb[1]; ++j)
      for (int64_t i = 0; i < nb[0]; ++i) {
        const int64_t ox = (i + R) + X0 * ((j + R) + X1 * (k + R));
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) {
          acc += coef[0] * u_cur_x[ox];
          for (int r = 1; r <= R; ++r)
            acc += coef[r] * (u_cur_x[ox + r * stride[a]] + u_cur_x[ox - r * stride[a]]);
        }
        const double L = acc * ih2;
        const int64_t idx = i + nb[0] * (j + nb[1] * k);
        const double e = dt2 / m_pad_b[idx] * L;
        u_next_b[idx] =
            (2.0 * u_cur_x[ox] - (1.0 - b_b[idx]) * u_prev_b[idx] + e) / (1.0 + b_b[idx]);
      }
  return 0;
}

/* Forward-Euler heat step u_next = u + dt * L u (Sec. II, Listing 1). */
void or_heat_step(const or_grid* g, const double* u, double* scratch_L,
                  double* u_next) {
  double c[17];
  or_fd_coefficients(g->R, c);
  or_laplacian(g, c, NULL, u, scratch_L);
  int64_t n = or_ncell(g);
  for (int64_t i = 0; i < n; ++i) u_next[i] = u[i] + g->dt * scratch_L[i];
}

static double vmax_of(const or_grid* g, const double* m_phys) {
  int64_t np = (int64_t)g->n[0] * g->n[1] * g->n[2];
  double mmin = m_phys[0];
  for (int64_t i = 1; i < np; ++i)
    if (m_phys[i] < mmin) mmin = m_phys[i];
  return 1.0 / sqrt(mmin);
}

typedef struct {
  int32_t cnt;
  int64_t idx[8];
  double w[8];
} pt_w;

static int build_points(const or_grid* g, int32_t npts, const double* xyz,
                        pt_w* out) {
  for (int32_t p = 0; p < npts; ++p) {
    out[p].cnt = or_point_weights(g, xyz + 3 * p, out[p].idx, out[p].w);
    if (out[p].cnt < 0) return -1;
  }
  return 0;
}

/*
 * Full forward modelling (Eq. 1 discretised), nt steps from the state
 * (u_prev, u_cur) given in `state` (2 * ncell doubles, overwritten with the
 * final state u^{n0+nt-1}, u^{n0+nt}); pass zeros for the quiescent start.
 *   m_phys  [n2][n1][n0] squared slowness of the physical cells
 *   coef    [R+1] uniform weights, or NULL with `percell` ([ncell][R+1])
 *   wavelet [nt_total][nsrc], row n0+t used at step t
 *   rec_out [nt][nrec] receives I(u^{n0+t}) for t = 0..nt-1 (may be NULL)
 *   e_hist  optional [nt][ncell]: (dt^2/m)(L u + s) of every step
 *   u_hist  optional [nt+1][ncell]: u^{n0}, ..., u^{n0+nt}
 * Returns 0, or -1 when a point lies outside the physical box.
 */
int32_t or_forward(const or_grid* g, const double* m_phys, const double* coef,
                   const double* percell, int32_t n0, int32_t nt,
                   int32_t nsrc, const double* src_xyz, const double* wavelet,
                   int32_t nrec, const double* rec_xyz, double* rec_out,
                   double* state, double* e_hist, double* u_hist) {
  int64_t n = or_ncell(g);
  double* m_pad = malloc(sizeof(double) * n);
  double* b = malloc(sizeof(double) * n);
  double* L = malloc(sizeof(double) * n);
  double* u_next = malloc(sizeof(double) * n);
  pt_w* sp = malloc(sizeof(pt_w) * (nsrc > 0 ? nsrc : 1));
  pt_w* rp = malloc(sizeof(pt_w) * (nrec > 0 ? nrec : 1));
  int64_t* sidx = malloc(sizeof(int64_t) * 8 * (nsrc > 0 ? nsrc : 1));
  double* sval = malloc(sizeof(double) * 8 * (nsrc > 0 ? nsrc : 1));
  int32_t rc = 0;
  if (build_points(g, nsrc, src_xyz, sp) || build_points(g, nrec, rec_xyz, rp)) {
    rc = -1;
    goto done;
  }
  or_pad_model(g, m_phys, m_pad);
  or_damping(g, vmax_of(g, m_phys), b);
  double hd = pow(g->h, g->dims);
  double* u_prev = state;
  double* u_cur = state + n;
  if (u_hist) memcpy(u_hist, u_cur, sizeof(double) * n);
  for (int32_t t = 0; t < nt; ++t) {
    int32_t step = n0 + t;
    if (rec_out)
      for (int32_t r = 0; r < nrec; ++r) {
        double v = 0.0;
        for (int k = 0; k < rp[r].cnt; ++k) v += rp[r].w[k] * u_cur[rp[r].idx[k]];
        rec_out[(int64_t)t * nrec + r] = v;
      }
    int32_t ns = 0;
    for (int32_t s = 0; s < nsrc; ++s)
      for (int k = 0; k < sp[s].cnt; ++k) {
        sidx[ns] = sp[s].idx[k];
        sval[ns] = sp[s].w[k] * wavelet[(int64_t)step * nsrc + s] / hd;
        ++ns;
      }
    or_step(g, m_pad, b, coef, percell, u_prev, u_cur, ns, sidx, sval, L,
            u_next, e_hist ? e_hist + (int64_t)t * n : NULL);
    memcpy(u_prev, u_cur, sizeof(double) * n);
    memcpy(u_cur, u_next, sizeof(double) * n);
    if (u_hist) memcpy(u_hist + (int64_t)(t + 1) * n, u_cur, sizeof(double) * n);
  }
done:
  free(m_pad); free(b); free(L); free(u_next); free(sp); free(rp);
  free(sidx); free(sval);
  return rc;
}

/*
 * Gradient of J = 1/2 sum_n || I(u^n) - d_obs[n] ||^2 (n = 0..nt-1, forward
 * from rest) with respect to the physical squared slowness, by the exact
 * transpose of the damped leapfrog recurrence (derived by hand from it):
 *
 *   forward   D u^{n+1} = 2u^n - E u^{n-1} + M (L u^n + s^n),
 *             D = diag(1+b), E = diag(1-b), M = diag(dt^2/m)
 *   adjoint   z^{nt} = z^{nt+1} = 0 and, for n = nt-1 .. 0,
 *             D z^n = 2z^{n+1} - E z^{n+2} + M (L z^{n+1} + I^T r^n),
 *             with r^n = I(u^n) - d_obs[n]  (z = M * dJ/dDu, L symmetric)
 *   gradient  g_pad = - sum_{n=0}^{nt-1} z^{n+1} (L u^n + s^n) / m
 *             = - sum_n z^{n+1} e^{n+1} / dt^2,  e^{n+1} = M (L u^n + s^n)
 *   g_phys[i] = sum of g_pad over the padded cells that replicate cell i.
 * The layer strength gamma_max is held fixed (its dependence on max(v) is
 * not differentiated).  The whole forward history is kept in memory, so this
 * is for small grids only.  `residual` (if not NULL) receives r.
 * Returns 0, or -1 on bad points.
 */
int32_t or_adjoint_gradient(const or_grid* g, const double* m_phys,
                            int32_t nt, int32_t nsrc, const double* src_xyz,
                            const double* wavelet, int32_t nrec,
                            const double* rec_xyz, const double* d_obs,
                            const double* residual_in, double* grad_phys,
                            double* loss_out, double* residual) {
  int64_t n = or_ncell(g);
  int R = g->R;
  double c[17];
  or_fd_coefficients(R, c);
  double* state = calloc(2 * n, sizeof(double));
  double* e_hist = malloc(sizeof(double) * n * nt);
  double* rec = malloc(sizeof(double) * (int64_t)nt * (nrec > 0 ? nrec : 1));
  double* r = malloc(sizeof(double) * (int64_t)nt * (nrec > 0 ? nrec : 1));
  double* m_pad = malloc(sizeof(double) * n);
  double* b = malloc(sizeof(double) * n);
  double* z0 = calloc(n, sizeof(double)); /* z^{n+2} */
  double* z1 = calloc(n, sizeof(double)); /* z^{n+1} */
  double* z2 = malloc(sizeof(double) * n); /* z^{n} */
  double* L = malloc(sizeof(double) * n);
  double* gpad = calloc(n, sizeof(double));
  pt_w* rp = malloc(sizeof(pt_w) * (nrec > 0 ? nrec : 1));
  int32_t rcode = or_forward(g, m_phys, c, NULL, 0, nt, nsrc, src_xyz, wavelet,
                             nrec, rec_xyz, rec, state, e_hist, NULL);
  if (rcode || build_points(g, nrec, rec_xyz, rp)) { rcode = -1; goto done; }
  or_pad_model(g, m_phys, m_pad);
  or_damping(g, vmax_of(g, m_phys), b);
  double loss = 0.0;
  for (int64_t i = 0; i < (int64_t)nt * nrec; ++i) {
    r[i] = residual_in ? residual_in[i] : rec[i] - d_obs[i];
    loss += 0.5 * r[i] * r[i];
  }
  if (residual) memcpy(residual, r, sizeof(double) * (int64_t)nt * nrec);
  if (loss_out) *loss_out = loss;
  double dt2 = g->dt * g->dt;
  for (int32_t t = nt - 1; t >= 0; --t) {
    /* imaging with z^{t+1} and e^{t+1} (stored at e_hist[t]) */
    const double* e = e_hist + (int64_t)t * n;
    for (int64_t i = 0; i < n; ++i) gpad[i] -= z1[i] * e[i] / dt2;
    /* z^t from z^{t+1}, z^{t+2} with the residual r^t injected by I^T */
    or_laplacian(g, c, NULL, z1, L);
    for (int32_t q = 0; q < nrec; ++q)
      for (int k = 0; k < rp[q].cnt; ++k)
        L[rp[q].idx[k]] += rp[q].w[k] * r[(int64_t)t * nrec + q];
    for (int64_t i = 0; i < n; ++i)
      z2[i] = (2.0 * z1[i] - (1.0 - b[i]) * z0[i] + dt2 / m_pad[i] * L[i]) /
              (1.0 + b[i]);
    double* tmp = z0; z0 = z1; z1 = z2; z2 = tmp;
  }
  /* fold the padded gradient back onto the physical cells */
  {
    int64_t N[3];
    padded_dims(g, N);
    int64_t np = (int64_t)g->n[0] * g->n[1] * g->n[2];
    memset(grad_phys, 0, sizeof(double) * np);
    for (int64_t k = 0; k < N[2]; ++k)
      for (int64_t j = 0; j < N[1]; ++j)
        for (int64_t i = 0; i < N[0]; ++i) {
          int64_t p[3] = {i, j, k}, q[3] = {0, 0, 0};
          for (int a = 0; a < g->dims; ++a) {
            int64_t v = p[a] - g->nbl;
            if (v < 0) v = 0;
            if (v > g->n[a] - 1) v = g->n[a] - 1;
            q[a] = v;
          }
          grad_phys[q[0] + g->n[0] * (q[1] + (int64_t)g->n[1] * q[2])] +=
              gpad[i + N[0] * (j + N[1] * k)];
        }
  }
done:
  free(state); free(e_hist); free(rec); free(r); free(m_pad); free(b);
  free(z0); free(z1); free(z2); free(L); free(gpad); free(rp);
  return rcode;
}

/*
 * The damped leapfrog update (same definition as or_step) evaluated only at
 * the listed padded cells, for checking sampled outputs of grids too large
 * to step on the CPU.  m_phys is the physical model; v_max sets the layer.
 * No source term.
 */
void or_step_points(const or_grid* g, const double* m_phys, double vmax,
                    const double* coef, const double* u_prev, const double* u_cur,
                    int64_t npts, const int64_t* idx, double* out) {
  int64_t N[3];
  padded_dims(g, N);
  int R = g->R;
  double ih2 = 1.0 / (g->h * g->h);
  double dt2 = g->dt * g->dt;
  double gmax = 0.0;
  if (g->nbl > 0)
    gmax = 3.0 * vmax * log(1.0 / g->rc) / (2.0 * g->nbl * g->h);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < npts; ++s) {
    int64_t id = idx[s];
    int64_t p[3] = {id % N[0], (id / N[0]) % N[1], id / (N[0] * N[1])};
    double acc = 0.0, damp = 0.0;
    int64_t q[3] = {0, 0, 0};
    for (int a = 0; a < g->dims; ++a) {
      acc += coef[0] * u_cur[id];
      for (int r = 1; r <= R; ++r)
        acc += coef[r] * (neighbour(g, N, u_cur, p[0], p[1], p[2], a, r) +
                          neighbour(g, N, u_cur, p[0], p[1], p[2], a, -r));
      double lo = (double)(g->nbl - p[a]);
      double hi = (double)(p[a] - (g->n[a] + g->nbl - 1));
      double d = 0.0;
      if (lo > d) d = lo;
      if (hi > d) d = hi;
      if (g->nbl > 0) d /= g->nbl;
      damp += d * d;
      int64_t v = p[a] - g->nbl;
      if (v < 0) v = 0;
      if (v > g->n[a] - 1) v = g->n[a] - 1;
      q[a] = v;
    }
    double m = m_phys[q[0] + (int64_t)g->n[0] * (q[1] + (int64_t)g->n[1] * q[2])];
    double b = gmax * damp * g->dt / 2.0;
    double e = dt2 / m * acc * ih2;
    out[s] = (2.0 * u_cur[id] - (1.0 - b) * u_prev[id] + e) / (1.0 + b);
  }
}
