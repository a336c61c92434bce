// Temporal blocking: two damped leapfrog steps of Eq. 1 (App. A) per pass
// over the grid, for space orders 4 and 8.
//
// The paper names temporal blocking (several time steps per pass) as future
// work in the Discussion of Sec. IV.  One pass here reads u^{n-1}, u^n and A
// and writes u^{n+1} and u^{n+2}: 20 bytes per point for two steps instead of
// the 32 of two single-step passes.  The price is recomputation: the second
// step needs u^{n+1} on an R-wide halo around its tile, so the first step runs
// on the extended tile.
//
// Design (2.5D streaming as in fd_step.cuh, one CTA per SM):
//  * A CTA owns an output tile of BX x BY points and the extended tile of
//    EX x EY = (BX + 2 RX) x (BY + 2R) points around it, one thread per four
//    consecutive x points of the extended tile (16 x 32 = 512 threads).
//  * u^n planes arrive by 3D TMA with a halo of 2 RX columns and 2R rows
//    (zero-filled outside the grid: the read-only zero halo); u^{n-1} and A
//    on the extended tile through a second TMA ring.
//  * Step 1 computes u^{n+1} of plane k on the extended tile (z neighbours
//    from a register queue of u^n) into a shared-memory ring of 2R + 2
//    planes, and stores its output-tile part.  Step 2 then computes u^{n+2}
//    of plane k - R on the output tile from that ring (x, y and z
//    neighbours), with u^n of that plane from the bottom of the queue.
//  * Both steps use the shared Laplacian and update helpers of the
//    single-step kernel, point by point in the same order of operations, so
//    two steps of one pass equal two single-step passes bit for bit.
//  * Sources inject q(t_n) into step 1 (entries of the extended tile) and
//    q(t_{n+1}) into step 2 (entries of the output tile); receivers read
//    I(u^n) from the staged u^n planes and I(u^{n+1}) from the ring.
//  * One barrier per plane: the 2R + 2 ring slots mean the slot step 1
//    overwrites was last read by step 2 two planes earlier.
//  * Every mbarrier wait is bounded; on expiry the CTA records an error,
//    drains its own copies (bounded) and returns.
#pragma once

#include "fd_step.cuh"

namespace fd {

template <int R>
struct TbCfg;
template <>
struct TbCfg<2> {
  static constexpr int BX = 56, BY = 28, PF = 3;
};
template <>
struct TbCfg<4> {
  static constexpr int BX = 56, BY = 24, PF = 2;
};

template <int R>
struct TbGeom {
  static constexpr int BX = TbCfg<R>::BX;
  static constexpr int BY = TbCfg<R>::BY;
  static constexpr int PF = TbCfg<R>::PF;
  static constexpr int RX = 4;                 // x halo rounded to 16 bytes (R <= 4)
  static constexpr int EX = BX + 2 * RX;       // extended tile of step 1
  static constexpr int EY = BY + 2 * R;
  static constexpr int TXE = EX / 4;
  static constexpr int NT = TXE * EY;          // threads
  static constexpr int W2 = EX + 2 * RX;       // staged u^n box
  static constexpr int H2 = EY + 2 * R;
  static constexpr int SU = R + 1 + PF;        // u^n ring slots
  static constexpr int SA = PF + 1;            // u^{n-1} / A ring slots
  static constexpr int S1 = 2 * R + 2;         // u^{n+1} ring slots
  static constexpr uint32_t UBYTES = W2 * H2 * 4;
  static constexpr uint32_t UPITCH = (UBYTES + 127) / 128 * 128;
  static constexpr uint32_t EBYTES = EX * EY * 4;
  static constexpr uint32_t EPITCH = (EBYTES + 127) / 128 * 128;
  static constexpr uint32_t OFF_P = SU * UPITCH;
  static constexpr uint32_t OFF_A = OFF_P + SA * EPITCH;
  static constexpr uint32_t OFF_1 = OFF_A + SA * EPITCH;
  static constexpr uint32_t OFF_BAR = OFF_1 + S1 * EPITCH;
  static constexpr uint32_t SMEM = OFF_BAR + (SU + SA) * 8 + 128;
  static constexpr int NROW4 = 3;
  static_assert(R <= 4, "one 16-byte x halo");
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
  static_assert(W2 <= 256 && H2 <= 256, "TMA box too large");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// One column (output tile (tile_x, tile_y), output planes [zb, ze)) of a
// two-step pass.  Step-1 planes run from zb - R to ze + R - 1 (index i,
// k1 = zb - R + i), u^n planes from zb - 2R to ze + 2R - 1 (index j,
// z = zb - 2R + j; staged plane jk = i + R holds k1's x/y neighbours), and
// step 2 produces plane k2 = k1 - R once i >= 2R.
template <int R>
__device__ __forceinline__ void tb_column(const TbDesc* __restrict__ D, const TbLaunch& L,
                                          const TbArgs& a, int tile_x, int tile_y, int zb,
                                          int ze, unsigned char* smem) {
  using G = TbGeom<R>;
  constexpr int NQ = 2 * R + 1;
  const int tid = threadIdx.x;
  const int tx = tid % G::TXE;
  const int ty = tid / G::TXE;
  const int x0 = tile_x * G::BX;
  const int y0 = tile_y * G::BY;
  if (zb >= ze) return;
  const int ZL = ze - zb;
  const int J = ZL + 4 * R;   // u^n planes
  const int Z1 = ZL + 2 * R;  // step-1 planes
  __shared__ int s_abort;
  if (tid == 0) s_abort = *reinterpret_cast<volatile const int*>(a.err);
  __syncthreads();
  if (s_abort) return;

  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_u0 = sbase + G::OFF_BAR;
  const uint32_t bar_a0 = bar_u0 + 8 * G::SU;
  const unsigned char* ubuf = smem;
  const unsigned char* pbuf = smem + G::OFF_P;
  const unsigned char* abuf = smem + G::OFF_A;
  unsigned char* ring1 = smem + G::OFF_1;
  if (tid == 0) {
    for (int s = 0; s < G::SU; ++s) mbar_init(bar_u0 + 8 * s, 1);
    for (int s = 0; s < G::SA; ++s) mbar_init(bar_a0 + 8 * s, 1);
    fence_mbar_init();
  }
  __syncthreads();

  int ju_next = 0, ia_next = 0;
  auto issue_u = [&](int j, uint32_t uoff) {
    if (j >= J) return;
    ju_next = j + 1;
    const uint32_t bar = bar_u0 + 8 * (uoff / G::UPITCH);
    mbar_expect_tx(bar, G::UBYTES);
    tma_load_3d(sbase + uoff, &D->halo2[L.in_cur], x0 - 2 * G::RX, y0 - 2 * R,
                zb - 2 * R + j, bar);
  };
  auto issue_a = [&](int i, uint32_t aoff) {
    if (i >= Z1) return;
    ia_next = i + 1;
    const uint32_t bar = bar_a0 + 8 * (aoff / G::EPITCH);
    mbar_expect_tx(bar, 2 * G::EBYTES);
    // plain L2 policy: neighbouring columns read these extended tiles too
    tma_load_3d(sbase + G::OFF_P + aoff, &D->ext[L.in_prev], x0 - G::RX, y0 - R, zb - R + i,
                bar);
    tma_load_3d(sbase + G::OFF_A + aoff, &D->extA, x0 - G::RX, y0 - R, zb - R + i, bar);
  };
  constexpr int kAuxTid = 32;
  if (tid == 0)
    for (int j = 0; j < G::SU; ++j) issue_u(j, j * G::UPITCH);
  if (tid == kAuxTid)
    for (int i = 0; i < G::SA; ++i) issue_a(i, i * G::EPITCH);

  // the thread's point: extended-tile column 4 tx, row ty
  const int gx = x0 - G::RX + 4 * tx;
  const int gy = y0 - R + ty;
  const uint32_t crow = 4u * ((ty + R) * G::W2 + 4 * tx + G::RX);  // in a staged u^n plane
  const uint32_t cext = 4u * (ty * G::EX + 4 * tx);                // in an extended tile
  const bool interior = tx >= G::RX / 4 && tx < G::RX / 4 + G::BX / 4 && ty >= R && ty < R + G::BY;
  const bool in_y = gy >= 0 && gy < a.Ny;
  bool okx[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) okx[l] = in_y && gx + l >= 0 && gx + l < a.Nx;
  const bool store_ok = interior && in_y && gx < a.Nx;

  float4 q[NQ];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) {
    const int slot = j % G::SU;
    bad |= !mbar_wait(bar_u0 + 8 * slot, (j / G::SU) & 1, L.spin_limit);
    q[j] = *reinterpret_cast<const float4*>(ubuf + slot * G::UPITCH + crow);
    if (j < R) {
      if (__syncthreads_or(bad)) goto fail;
      if (tid == 0) issue_u(j + G::SU, slot * G::UPITCH);
    }
  }

  {
    const int tile = tile_y * a.tiles_x + tile_x;
    // step-1 sources (extended tile), step-2 sources (output tile), receivers
    int ip1 = a.inj1_start[tile], iend1 = a.inj1_start[tile + 1];
    int ip2 = a.inj2_start[tile], iend2 = a.inj2_start[tile + 1];
    int rp = a.rec_start[tile], rend = a.rec_start[tile + 1];
    while (ip1 < iend1 && a.inj1[ip1].z < zb - R) ++ip1;
    while (ip2 < iend2 && a.inj2[ip2].z < zb) ++ip2;
    while (rp < rend && a.recs[rp].z < zb) ++rp;
    int iz1 = ip1 < iend1 ? a.inj1[ip1].z : INT_MAX;
    int iz2 = ip2 < iend2 ? a.inj2[ip2].z : INT_MAX;
    int rz1 = rp < rend ? a.recs[rp].z : INT_MAX;  // I(u^n) of the plane at step 1
    int rp2 = rp;                                   // I(u^{n+1}) of the plane at step 2
    int rz2 = rz1;

    const int dyv = sponge_depth(gy, a.nbl, a.ny);
    float dxx[4];
    bool xy_inner = true;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int d = sponge_depth(gx + l, a.nbl, a.nx);
      dxx[l] = static_cast<float>(d * d + dyv * dyv);
      xy_inner = xy_inner && d == 0 && okx[l];
    }
    xy_inner = xy_inner && dyv == 0;  // inside the physical box in x and y: b = 0
    const size_t plane_stride = static_cast<size_t>(a.Ny) * a.pitch;
    const size_t col = static_cast<size_t>(gy) * a.pitch + gx;
    const float c0hi = L.c[0], c0lo = L.c[kMaxR + 1];  // centre weight (launch_weights)
    float* out1 = D->u[L.out1];
    float* out2 = D->u[L.out2];

    int sk = R % G::SU;  // slot of staged plane jk
    int sn = (2 * R) % G::SU;
    uint32_t pn = ((2 * R) / G::SU) & 1;
    int sa = 0;
    uint32_t pa = 0;

    for (int i = 0; i < Z1; ++i) {
      const int k1 = zb - R + i;
      const int k2 = k1 - R;
      const bool step2 = i >= 2 * R;
      // u^n, A of step 2's point, fetched early (L2: loaded R planes ago)
      float4 A2 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (step2 && store_ok) A2 = __ldg(reinterpret_cast<const float4*>(a.A + k2 * plane_stride + col));
#define FD_Q(o) q[R + (o)]
      bad |= !mbar_wait(bar_u0 + 8 * sn, pn, L.spin_limit);
      FD_Q(R) = *reinterpret_cast<const float4*>(ubuf + sn * G::UPITCH + crow);
      bad |= !mbar_wait(bar_a0 + 8 * sa, pa, L.spin_limit);

      // ---- step 1: u^{n+1} of plane k1 on the extended tile ----
      {
        const unsigned char* P = ubuf + sk * G::UPITCH + crow;
        float xr[4 * G::NROW4];
#pragma unroll
        for (int m = 0; m < G::NROW4; ++m) {
          const float4 v = (m == 1) ? FD_Q(0) : *reinterpret_cast<const float4*>(P + 16 * (m - 1));
          xr[4 * m + 0] = v.x;
          xr[4 * m + 1] = v.y;
          xr[4 * m + 2] = v.z;
          xr[4 * m + 3] = v.w;
        }
        float lap[4];
        lap4_packed<R, G::RX>(
            xr,
            [&](int jj, float4& ym, float4& yp) {
              ym = *reinterpret_cast<const float4*>(P - 4 * jj * G::W2);
              yp = *reinterpret_cast<const float4*>(P + 4 * jj * G::W2);
            },
            [&](int o) { return FD_Q(o); }, L.c, c0hi, c0lo, lap);
        float src[4] = {0.f, 0.f, 0.f, 0.f};
        if (k1 == iz1) {
          while (ip1 < iend1) {
            const InjEntry e = a.inj1[ip1];
            if (e.z != k1) break;
            if (e.ly == ty && (e.lx >> 2) == tx) {
              const float val =
                  e.w * a.inj_val[static_cast<size_t>(L.inj_row) * a.inj_ncol + e.col];
#pragma unroll
              for (int l = 0; l < 4; ++l) src[l] += ((e.lx & 3) == l) ? val : 0.f;
            }
            ++ip1;
          }
          iz1 = ip1 < iend1 ? a.inj1[ip1].z : INT_MAX;
        }
        const float4 up = *reinterpret_cast<const float4*>(pbuf + sa * G::EPITCH + cext);
        const float4 Av = *reinterpret_cast<const float4*>(abuf + sa * G::EPITCH + cext);
        float res[4], ev[4];
        const bool in_z = k1 >= 0 && k1 < a.Nz;
        if (xy_inner && k1 >= a.nbl && k1 < a.nbl + a.nz) {
          update4_inner(lap, src, FD_Q(0), up, Av, res, ev);
        } else {
          const int dz = sponge_depth(k1, a.nbl, a.nz);
          const bool ok[4] = {okx[0] && in_z, okx[1] && in_z, okx[2] && in_z, okx[3] && in_z};
          update4_layer(lap, src, FD_Q(0), up, Av, dxx, static_cast<float>(dz * dz), a.bscale,
                        ok, res, ev);
        }
        *reinterpret_cast<float4*>(ring1 + (i % G::S1) * G::EPITCH + cext) =
            make_float4(res[0], res[1], res[2], res[3]);
        if (store_ok && k1 >= zb && k1 < ze)
          st_stream(out1 + k1 * plane_stride + col, res[0], res[1], res[2], res[3]);

        // receivers I(u^n) with their floor node in plane k1 (output tile,
        // planes of this column only)
        if (k1 == rz1 && k1 < ze) {
          int rq = rp;
          while (rq < rend && a.recs[rq].z == k1) ++rq;
          const float* P0 = reinterpret_cast<const float*>(ubuf + sk * G::UPITCH);
          const float* P1 =
              reinterpret_cast<const float*>(ubuf + (sk + 1 == G::SU ? 0 : sk + 1) * G::UPITCH);
          for (int e = rp + tid; e < rq; e += G::NT) {
            const RecEntry r = a.recs[e];
            const int o = (r.ly + 2 * R) * G::W2 + r.lx + 2 * G::RX;
            const float gx0 = 1.0f - r.fx, gy0 = 1.0f - r.fy;
            const float p0 = gy0 * (gx0 * P0[o] + r.fx * P0[o + 1]) +
                             r.fy * (gx0 * P0[o + G::W2] + r.fx * P0[o + G::W2 + 1]);
            const float p1 = gy0 * (gx0 * P1[o] + r.fx * P1[o + 1]) +
                             r.fy * (gx0 * P1[o + G::W2] + r.fx * P1[o + G::W2 + 1]);
            a.rec_out[static_cast<size_t>(L.rec_row) * a.rec_ncol + r.col] =
                (1.0f - r.fz) * p0 + r.fz * p1;
          }
          rp = rq;
          rz1 = rp < rend ? a.recs[rp].z : INT_MAX;
        }
      }

      if (__syncthreads_or(bad)) goto fail;
      if (tid == 0) issue_u(i + R + G::SU, sk * G::UPITCH);
      if (tid == kAuxTid) issue_a(i + G::SA, sa * G::EPITCH);

      // ---- step 2: u^{n+2} of plane k2 = k1 - R on the output tile ----
      if (step2) {
        const int s2 = (i - R) % G::S1;
        const unsigned char* Q = ring1 + s2 * G::EPITCH + cext;
        if (interior) {
          float xr[4 * G::NROW4];
#pragma unroll
          for (int m = 0; m < G::NROW4; ++m) {
            const float4 v = *reinterpret_cast<const float4*>(Q + 16 * (m - 1));
            xr[4 * m + 0] = v.x;
            xr[4 * m + 1] = v.y;
            xr[4 * m + 2] = v.z;
            xr[4 * m + 3] = v.w;
          }
          float lap[4];
          lap4_packed<R, G::RX>(
              xr,
              [&](int jj, float4& ym, float4& yp) {
                ym = *reinterpret_cast<const float4*>(Q - 4 * jj * G::EX);
                yp = *reinterpret_cast<const float4*>(Q + 4 * jj * G::EX);
              },
              [&](int o) {
                if (o == 0) return make_float4(xr[4], xr[5], xr[6], xr[7]);
                const int s = (i - R + o + G::S1) % G::S1;
                return *reinterpret_cast<const float4*>(ring1 + s * G::EPITCH + cext);
              },
              L.c, c0hi, c0lo, lap);
          float src[4] = {0.f, 0.f, 0.f, 0.f};
          if (k2 == iz2) {
            while (ip2 < iend2) {
              const InjEntry e = a.inj2[ip2];
              if (e.z != k2) break;
              if (e.ly == ty && (e.lx >> 2) == tx) {
                const float val =
                    e.w * a.inj_val[static_cast<size_t>(L.inj_row + 1) * a.inj_ncol + e.col];
#pragma unroll
                for (int l = 0; l < 4; ++l) src[l] += ((e.lx & 3) == l) ? val : 0.f;
              }
              ++ip2;
            }
            iz2 = ip2 < iend2 ? a.inj2[ip2].z : INT_MAX;
          }
          const float4 uc = make_float4(xr[4], xr[5], xr[6], xr[7]);
          float res[4], ev[4];
          if (xy_inner && k2 >= a.nbl && k2 < a.nbl + a.nz) {
            update4_inner(lap, src, uc, FD_Q(-R), A2, res, ev);
          } else {
            const int dz = sponge_depth(k2, a.nbl, a.nz);
            update4_layer(lap, src, uc, FD_Q(-R), A2, dxx, static_cast<float>(dz * dz),
                          a.bscale, okx, res, ev);
          }
          if (store_ok) st_stream(out2 + k2 * plane_stride + col, res[0], res[1], res[2], res[3]);
        }
        // receivers I(u^{n+1}) with their floor node in plane k2
        if (k2 == rz2) {
          int rq = rp2;
          while (rq < rend && a.recs[rq].z == k2) ++rq;
          const float* P0 = reinterpret_cast<const float*>(ring1 + s2 * G::EPITCH);
          const float* P1 = reinterpret_cast<const float*>(
              ring1 + ((i - R + 1) % G::S1) * G::EPITCH);
          for (int e = rp2 + tid; e < rq; e += G::NT) {
            const RecEntry r = a.recs[e];
            const int o = (r.ly + R) * G::EX + r.lx + G::RX;
            const float gx0 = 1.0f - r.fx, gy0 = 1.0f - r.fy;
            const float p0 = gy0 * (gx0 * P0[o] + r.fx * P0[o + 1]) +
                             r.fy * (gx0 * P0[o + G::EX] + r.fx * P0[o + G::EX + 1]);
            const float p1 = gy0 * (gx0 * P1[o] + r.fx * P1[o + 1]) +
                             r.fy * (gx0 * P1[o + G::EX] + r.fx * P1[o + G::EX + 1]);
            a.rec_out[static_cast<size_t>(L.rec_row + 1) * a.rec_ncol + r.col] =
                (1.0f - r.fz) * p0 + r.fz * p1;
          }
          rp2 = rq;
          rz2 = rp2 < rend ? a.recs[rp2].z : INT_MAX;
        }
      }

      sk = (sk + 1 == G::SU) ? 0 : sk + 1;
      sn = (sn + 1 == G::SU) ? 0 : sn + 1;
      pn ^= (sn == 0) ? 1u : 0u;
      sa = (sa + 1 == G::SA) ? 0 : sa + 1;
      pa ^= (sa == 0) ? 1u : 0u;
#pragma unroll
      for (int j = 0; j < 2 * R; ++j) q[j] = q[j + 1];
#undef FD_Q
    }
  }
  if (tid == 0) {
    for (int s = 0; s < G::SU; ++s) mbar_inval(bar_u0 + 8 * s);
    for (int s = 0; s < G::SA; ++s) mbar_inval(bar_a0 + 8 * s);
  }
  __syncthreads();
  return;

fail:
  if (tid == 0) {
    atomicOr(a.err, 1);
    for (int j = max(0, ju_next - G::SU); j < ju_next; ++j)
      mbar_wait(bar_u0 + 8 * (j % G::SU), (j / G::SU) & 1, L.spin_limit);
  }
  if (tid == kAuxTid) {
    for (int i = max(0, ia_next - G::SA); i < ia_next; ++i)
      mbar_wait(bar_a0 + 8 * (i % G::SA), (i / G::SA) & 1, L.spin_limit);
  }
}

// CTA c runs the work items [item_start[c], item_start[c+1]) (column waves
// of fd_sched.cu over the output tiles).
template <int R>
__global__ void __launch_bounds__(TbGeom<R>::NT, 1)
    tblock_kernel(const TbDesc* __restrict__ D, const __grid_constant__ TbLaunch L) {
  extern __shared__ unsigned char smem_raw[];
  // aligned to 128 bytes by an offset from the shared array itself, so that
  // the compiler keeps the address space and issues shared-memory loads and
  // stores (through a pointer rebuilt from an integer it issued generic ones)
  unsigned char* smem =
      smem_raw + ((128u - (static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw)) & 127u)) &
                  127u);
  __shared__ TbArgs a;
  if (threadIdx.x == 0) a = D->args;
  __syncthreads();
  const int i1 = L.item_start[blockIdx.x + 1];
  for (int i = L.item_start[blockIdx.x]; i < i1; ++i) {
    const WorkItem w = L.items[i];
    tb_column<R>(D, L, a, w.tile % a.tiles_x, w.tile / a.tiles_x, w.zb, w.ze, smem);
    __syncthreads();
  }
}

}  // namespace fd
