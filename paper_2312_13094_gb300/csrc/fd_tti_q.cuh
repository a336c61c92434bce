// TTI step with register queues and TMA staging (included by fd_tti.cu;
// Sec. IV-B and App. A, Eq. rot).  Space orders up to 8 run two 256-thread
// CTAs per SM; the wider stencils, whose queues take about 200 registers,
// one.
//
// One point per thread on a 32 x 8 tile, a CTA streaming a run of z planes.
// Every derivative is split by what it needs:
//  * the in-plane terms D_xx, D_yy and D_xy of a plane need only that plane,
//    so they are formed once, when the plane enters (p = k + R for output
//    plane k), and wait R planes in per-thread register queues;
//  * the z terms D_zz, D_xz and D_yz are sums over planes k-R .. k+R of the
//    thread's own u and of its first x and y differences dx, dy, which also
//    enter with their plane and live in register queues of 2R+1 entries.
// So shared memory holds only the entering plane of p and q with its halo
// (one 3D TMA tile load per field into a ring of PF+1 slots), the first x
// differences of that plane on the tile and its R halo rows (for D_xy, two
// buffers), and the update's eight per-point values of the output plane
// (six model fields, p^{n-1}, q^{n-1}; TMA tiles, L2 evict-first, PF+1
// slots).  Loads outside the grid are zero-filled by the TMA unit (the zero
// ghost).  Every mbarrier wait is bounded; on expiry the CTA records an
// error, waits (bounded) for its own copies in flight and returns.
#pragma once

#include "fd_step.cuh"

namespace fd {
namespace tti {

constexpr int kQX = 32, kQY = 8, kQT = kQX * kQY;  // tile and threads
constexpr int kQPF = 2;                             // planes in flight ahead

template <int R>
struct QGeom {
  // x halo of the staged tile: R rounded up to 4 floats (16-byte aligned TMA x coordinate)
  static constexpr int RX = ((R + 3) / 4) * 4;
  static constexpr int W = kQX + 2 * RX, H = kQY + 2 * R;
  static constexpr uint32_t UBYTES = W * H * 4;
  static constexpr uint32_t UP = (UBYTES + 127) / 128 * 128;  // one field's staged plane
  static constexpr int SU = kQPF + 1, SA = kQPF + 1;
  static constexpr int EH = kQY + 2 * R;  // rows of the dx scratch
  static constexpr int NE = (EH + kQY - 1) / kQY;  // scratch rows per thread
  static constexpr int CTAS = R <= 4 ? 2 : 1;       // resident CTAs per SM
  static constexpr uint32_t XP = (kQX * EH * 4 + 127) / 128 * 128;
  static constexpr uint32_t TBYTES = kQX * kQY * 4;  // one per-point tile
  static constexpr uint32_t OFF_X = 2 * SU * UP;      // dx scratch: [field][buffer]
  static constexpr uint32_t OFF_A = OFF_X + 4 * XP;   // per-point tiles: [slot][8]
  static constexpr uint32_t OFF_BAR = OFF_A + SA * 8 * TBYTES;
  static constexpr uint32_t SMEM = OFF_BAR + 8 * (SU + SA) + 128;  // + alignment slack
};

struct QMaps {
  CUtensorMap halo_p, halo_q;  // p^n, q^n: 40 x (8 + 2R) boxes
  CUtensorMap prev_p, prev_q;  // p^{n-1}, q^{n-1}: 32 x 8 boxes
  CUtensorMap coef;            // the six model fields stacked along z: 32 x 8 boxes
};

struct QArgs {
  float* pn;  // p^{n-1} in, p^{n+1} out (in place)
  float* qn;
  int* err;   // set on an expired wait
  int Nx, Ny, Nz, pitch;
  int nbl, nx, ny, nz;
  int zchunk;
  long long spin_limit;
  float bscale;
  float c[kMaxR + 1];
  float d[kMaxR + 1];
};

__device__ __forceinline__ int qdepth(int g, int nbl, int n) {
  int d = nbl - g;
  const int e = g - (n + nbl - 1);
  d = d > e ? d : e;
  return d > 0 ? d : 0;
}

template <int N>
__device__ __forceinline__ void qpush(float (&q)[N], float v) {
#pragma unroll
  for (int i = 0; i < N - 1; ++i) q[i] = q[i + 1];
  q[N - 1] = v;
}

template <int R>
__global__ void __launch_bounds__(kQT, QGeom<R>::CTAS)
    k_tti_q(const __grid_constant__ QMaps M, const __grid_constant__ QArgs a) {
  using G = QGeom<R>;
  extern __shared__ unsigned char qsm_raw[];
  // aligned by an offset from the shared array, so the address space is kept
  unsigned char* qsm =
      qsm_raw + ((128u - (static_cast<uint32_t>(__cvta_generic_to_shared(qsm_raw)) & 127u)) &
                 127u);
  const uint32_t sbase = smem_u32(qsm);
  const uint32_t bar_u0 = sbase + G::OFF_BAR, bar_a0 = bar_u0 + 8 * G::SU;
  const int tid = threadIdx.x, tx = tid % kQX, ty = tid / kQX;
  const int x0 = blockIdx.x * kQX, y0 = blockIdx.y * kQY;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.Nz);
  if (z0 >= z1) return;
  const int nin = z1 - z0 + 2 * R;  // entering planes z0-R .. z1+R-1
  const int nout = z1 - z0;
  constexpr int kAux = 32;

  if (tid == 0) {
    for (int s = 0; s < G::SU; ++s) mbar_init(bar_u0 + 8 * s, 1);
    for (int s = 0; s < G::SA; ++s) mbar_init(bar_a0 + 8 * s, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // producers: thread 0 the staged planes (entering plane i: z = z0-R+i),
  // thread 32 the per-point tiles (output plane i: z = z0+i)
  int iu_next = 0, ia_next = 0;
  auto issue_u = [&](int i) {
    if (i >= nin) return;
    iu_next = i + 1;
    const int s = i % G::SU;
    const uint32_t bar = bar_u0 + 8 * s;
    mbar_expect_tx(bar, 2 * G::UBYTES);
    const int z = z0 - R + i;
    tma_load_3d(sbase + (2 * s) * G::UP, &M.halo_p, x0 - G::RX, y0 - R, z, bar);
    tma_load_3d(sbase + (2 * s + 1) * G::UP, &M.halo_q, x0 - G::RX, y0 - R, z, bar);
  };
  auto issue_a = [&](int i) {
    if (i >= nout) return;
    ia_next = i + 1;
    const int s = i % G::SA;
    const uint32_t bar = bar_a0 + 8 * s;
    mbar_expect_tx(bar, 8 * G::TBYTES);
    const int z = z0 + i;
    const uint32_t dst = sbase + G::OFF_A + s * 8 * G::TBYTES;
#pragma unroll
    for (int f = 0; f < 6; ++f)
      tma_load_3d_stream(dst + f * G::TBYTES, &M.coef, x0, y0, z + f * a.Nz, bar);
    tma_load_3d_stream(dst + 6 * G::TBYTES, &M.prev_p, x0, y0, z, bar);
    tma_load_3d_stream(dst + 7 * G::TBYTES, &M.prev_q, x0, y0, z, bar);
  };
  if (tid == 0)
    for (int i = 0; i < G::SU; ++i) issue_u(i);
  if (tid == kAux)
    for (int i = 0; i < G::SA; ++i) issue_a(i);

  // register queues per field: own u, dx, dy of planes k-R .. k+R (centre at
  // R) and D_xx, D_yy, D_xy of planes k .. k+R (centre at 0)
  float qu[2][2 * R + 1], qdx[2][2 * R + 1], qdy[2][2 * R + 1];
  float qxx[2][R + 1], qyy[2][R + 1], qxy[2][R + 1];
#pragma unroll
  for (int f = 0; f < 2; ++f) {
#pragma unroll
    for (int i = 0; i < 2 * R + 1; ++i) qu[f][i] = qdx[f][i] = qdy[f][i] = 0.f;
#pragma unroll
    for (int i = 0; i < R + 1; ++i) qxx[f][i] = qyy[f][i] = qxy[f][i] = 0.f;
  }

  const int gx = x0 + tx, gy = y0 + ty;
  const bool inside = gx < a.Nx && gy < a.Ny;
  const int dxy = qdepth(gx, a.nbl, a.nx) * qdepth(gx, a.nbl, a.nx) +
                  qdepth(gy, a.nbl, a.ny) * qdepth(gy, a.nbl, a.ny);
  // byte offsets: own point in a staged plane; the scratch rows this thread
  // fills are e = ty + 8m (scratch row e = staged row e, tile row e - R)
  const uint32_t cown = 4u * ((ty + R) * G::W + tx + G::RX);
  const uint32_t cx = 4u * ((ty + R) * kQX + tx);
  const size_t plane = static_cast<size_t>(a.Ny) * a.pitch;
  size_t off = static_cast<size_t>(z0) * plane + static_cast<size_t>(gy) * a.pitch + gx;

  bool bad = false;
  int su = 0;
  uint32_t pu = 0;
  int sa = 0;
  uint32_t pa = 0;

  // one entering plane: its in-plane terms and first differences into the
  // queues (one barrier: the dx scratch of both fields); returns false when
  // the CTA must stop
  auto enter = [&](int i) -> bool {
    bad |= !mbar_wait(bar_u0 + 8 * su, pu, a.spin_limit);
    const int buf = i & 1;
    float dyo[2], xxo[2], yyo[2], uo[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const uint32_t P = sbase + (2 * su + f) * G::UP;
      const float u0 = lds1(P + cown);
      float xx = a.c[0] * u0, yy = a.c[0] * u0, dy = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const float xp = lds1(P + cown + 4 * j), xm = lds1(P + cown - 4 * j);
        const float yp = lds1(P + cown + 4 * j * G::W), ym = lds1(P + cown - 4 * j * G::W);
        xx = fmaf(a.c[j], xp + xm, xx);
        yy = fmaf(a.c[j], yp + ym, yy);
        dy = fmaf(a.d[j], yp - ym, dy);
      }
      // first x differences of the scratch rows ty + 8m (staged rows)
      const uint32_t X = sbase + G::OFF_X + (2 * f + buf) * G::XP;
#pragma unroll
      for (int m = 0; m < G::NE; ++m) {
        const int e = ty + m * kQY;
        if (m == 0 || e < G::EH) {
          const uint32_t re = 4u * (e * G::W + tx + G::RX);
          float ex = 0.f;
#pragma unroll
          for (int j = 1; j <= R; ++j)
            ex = fmaf(a.d[j], lds1(P + re + 4 * j) - lds1(P + re - 4 * j), ex);
          asm volatile("st.shared.f32 [%0], %1;" ::"r"(X + 4u * (e * kQX + tx)), "f"(ex)
                       : "memory");
        }
      }
      uo[f] = u0;
      xxo[f] = xx;
      yyo[f] = yy;
      dyo[f] = dy;
    }
    if (__syncthreads_or(bad)) return false;
    // every thread is past this plane's staged tiles and the previous
    // plane's compute: refill this slot and the last output plane's tiles
    if (tid == 0) issue_u(i + G::SU);
    if (tid == kAux && i > 2 * R) issue_a(i - 2 * R - 1 + G::SA);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const uint32_t X = sbase + G::OFF_X + (2 * f + buf) * G::XP;
      float xy = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j)
        xy = fmaf(a.d[j], lds1(X + cx + 4 * j * kQX) - lds1(X + cx - 4 * j * kQX), xy);
      // the own row's first x difference is scratch row ty + R, written before
      // the barrier (the same sum in the same order)
      qpush(qu[f], uo[f]);
      qpush(qdx[f], lds1(X + cx));
      qpush(qdy[f], dyo[f]);
      qpush(qxx[f], xxo[f]);
      qpush(qyy[f], yyo[f]);
      qpush(qxy[f], xy);
    }
    su = (su + 1 == G::SU) ? 0 : su + 1;
    pu ^= (su == 0) ? 1u : 0u;
    return true;
  };

  for (int i = 0; i < 2 * R; ++i)
    if (!enter(i)) goto fail;

  // four planes per loop trip: the compiler renames the queues for three of
  // them instead of shifting
#pragma unroll 4
  for (int k = 0; k < nout; ++k) {
    if (!enter(k + 2 * R)) goto fail;
    bad |= !mbar_wait(bar_a0 + 8 * sa, pa, a.spin_limit);
    {
      const uint32_t T = sbase + G::OFF_A + sa * 8 * G::TBYTES + 4u * (ty * kQX + tx);
      const float A = lds1(T), e2 = lds1(T + G::TBYTES), dl = lds1(T + 2 * G::TBYTES);
      const float nx = lds1(T + 3 * G::TBYTES), ny = lds1(T + 4 * G::TBYTES),
                  nz = lds1(T + 5 * G::TBYTES);
      const float pm = lds1(T + 6 * G::TBYTES), qm = lds1(T + 7 * G::TBYTES);
      float D[2][6];
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        float zz = a.c[0] * qu[f][R], xz = 0.f, yz = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          zz = fmaf(a.c[j], qu[f][R + j] + qu[f][R - j], zz);
          xz = fmaf(a.d[j], qdx[f][R + j] - qdx[f][R - j], xz);
          yz = fmaf(a.d[j], qdy[f][R + j] - qdy[f][R - j], yz);
        }
        D[f][0] = qxx[f][0];
        D[f][1] = qyy[f][0];
        D[f][2] = zz;
        D[f][3] = qxy[f][0];
        D[f][4] = xz;
        D[f][5] = yz;
      }
      const float wxx = nx * nx, wyy = ny * ny, wzz = nz * nz;
      const float wxy = 2.f * nx * ny, wxz = 2.f * nx * nz, wyz = 2.f * ny * nz;
      const float* dp = D[0];
      const float* dq = D[1];
      const float lap_p = dp[0] + dp[1] + dp[2];
      const float hz_p = wxx * dp[0] + wyy * dp[1] + wzz * dp[2] + wxy * dp[3] + wxz * dp[4] +
                         wyz * dp[5];
      const float hz_q = wxx * dq[0] + wyy * dq[1] + wzz * dq[2] + wxy * dq[3] + wxz * dq[4] +
                         wyz * dq[5];
      const float h0_p = lap_p - hz_p;
      const float rp = e2 * h0_p + dl * hz_q;
      const float rq = dl * h0_p + hz_q;
      const int dz = qdepth(z0 + k, a.nbl, a.nz);
      const float b = a.bscale * static_cast<float>(dxy + dz * dz);
      const float pc = qu[0][R], qc = qu[1][R];
      // outside the layer b = 0 and the division by 1 + b is exact: skipped
      float np_ = 2.f * pc - (1.f - b) * pm + A * rp;
      float nq_ = 2.f * qc - (1.f - b) * qm + A * rq;
      if (b != 0.f) {
        np_ = np_ / (1.f + b);
        nq_ = nq_ / (1.f + b);
      }
      if (inside) {
        a.pn[off] = np_;
        a.qn[off] = nq_;
      }
    }
    off += plane;
    sa = (sa + 1 == G::SA) ? 0 : sa + 1;
    pa ^= (sa == 0) ? 1u : 0u;
  }
  // every issued copy has been waited for (the entering planes up to nin-1,
  // the per-point tiles up to nout-1); release the barriers
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < G::SU; ++s) mbar_inval(bar_u0 + 8 * s);
    for (int s = 0; s < G::SA; ++s) mbar_inval(bar_a0 + 8 * s);
  }
  return;

fail:
  if (tid == 0) {
    atomicOr(a.err, 1);
    for (int i = max(0, iu_next - G::SU); i < iu_next; ++i)
      mbar_wait(bar_u0 + 8 * (i % G::SU), (i / G::SU) & 1, a.spin_limit);
  }
  if (tid == kAux) {
    for (int i = max(0, ia_next - G::SA); i < ia_next; ++i)
      mbar_wait(bar_a0 + 8 * (i % G::SA), (i / G::SA) & 1, a.spin_limit);
  }
}

}  // namespace tti
}  // namespace fd
