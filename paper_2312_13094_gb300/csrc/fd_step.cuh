// Damped leapfrog step of the acoustic wave equation for sm_103a.
//
// Eq. 1 (App. A) discretised as in Sec. IV-B: one launch advances
//   (1+b) u^{n+1} = 2u^n - (1-b) u^{n-1} + A (lap(u^n) + s^n),
// A = dt^2 / (m h^2) (stored per cell), lap = sum_axes sum_j c_|j| u(i+j e_a)
// with the zero ghost of Sec. III beyond the padded grid, b from the sponge
// depth, s^n the trilinear source term, and rec[n] = I(u^n) (Sec. III
// "Sparse data") read from the same staged planes.
//
// Design (2.5D streaming, Blackwell-native):
//  * A CTA owns an xy tile of BX x BY points (4 consecutive x per thread,
//    one row per thread) and sweeps a range of z planes.
//  * Each plane of u^n, with an R-row and RX-column halo (RX = R rounded up
//    to 4 floats so that the TMA x coordinate stays 16-byte aligned), is
//    brought into shared memory by one 3D TMA tile load into a ring of
//    SU = R + 1 + PF slots, each completed on its own mbarrier.  Loads that
//    fall outside the grid are zero-filled by the TMA unit, which is exactly
//    the read-only zero halo, so no ghost cells are stored in HBM.
//  * u^{n-1} and A tiles come through a second TMA ring of PF + 1 slots.
//  * z neighbours live in a per-thread register queue of 2R+1 float4s; x and
//    y neighbours are read from the staged plane with 128-bit loads.
//  * The wide stencils (R >= 5) split the u^n staging: the ring of halo
//    tiles holds only the centre plane and PF planes ahead (SU = PF + 1),
//    and the queue is fed R planes ahead of the centre from a third ring of
//    PF + 1 interior tiles.  Each plane is then copied twice from L2 (once as
//    an interior tile, R planes later with its halo), but a CTA holds
//    2 (PF + 1) tiles instead of R + 1 + PF halo tiles, so that the
//    512 threads per SM that the registers allow are not cut by shared
//    memory (a 32 x 16 tile at R = 8: 70 KB per CTA, three CTAs per SM,
//    with the single ring).
//  * Shared memory is read with explicit ld.shared at 32-bit addresses.
//  * Source injection and receiver interpolation use per-tile entry lists
//    sorted by z, so a tile without points pays one compare per plane.
//  * Every mbarrier wait is bounded (clock64); on expiry the CTA records an
//    error, waits (bounded) for its own copies still in flight, and returns.
#pragma once

#include <climits>

#include "fd_internal.h"

namespace fd {

template <int R, int TX, int TY, int PF, int NC = 0>
struct Cfg {
  static constexpr int RX = ((R + 3) / 4) * 4;
  static constexpr int BX = 4 * TX;
  static constexpr int BY = TY;
  static constexpr int NT = TX * TY;
  static constexpr int W = BX + 2 * RX;
  static constexpr int H = BY + 2 * R;
  static constexpr bool SPLIT = R >= 5;  // split u^n staging (see above)
  static constexpr int SU = SPLIT ? PF + 1 : R + 1 + PF;  // halo-tile slots
  static constexpr int SA = PF + 1;
  static constexpr int SI = SPLIT ? PF + 1 : 0;  // interior-tile slots of u^n
  static constexpr uint32_t UBYTES = W * H * 4;
  static constexpr uint32_t UPITCH = (UBYTES + 127) / 128 * 128;
  static constexpr uint32_t TBYTES = BX * BY * 4;
  static constexpr uint32_t TPITCH = (TBYTES + 127) / 128 * 128;
  static constexpr uint32_t OFF_P = SU * UPITCH;
  static constexpr uint32_t OFF_A = OFF_P + SA * TPITCH;
  static constexpr uint32_t OFF_C = OFF_A + SA * TPITCH;      // NC coefficient tiles
  static constexpr uint32_t OFF_I = OFF_C + SA * NC * TPITCH;  // u^n interior tiles
  static constexpr uint32_t OFF_BAR = OFF_I + SI * TPITCH;
  // one barrier per ring slot (twice the room: kept as before)
  static constexpr uint32_t SMEM = OFF_BAR + 2 * (SU + SA + SI) * 8 + 128;
  static constexpr int NROW4 = 2 * RX / 4 + 1;
  static_assert(W <= 256 && H <= 256, "TMA box too large");
};

// Threads per SM that the launch bounds aim for.  SO <= 8: 640, five
// 128-thread CTAs with 96 registers each (no spills) and room for a 2-plane
// prefetch on the 64x8 tile; six CTAs at 80 registers with a 1-plane prefetch
// measured 282 against 293 Gpts/s on 592^3.  The wider stencils need more
// registers for their register queue (2R+1 float4 per thread): 512.
constexpr int threads_per_sm(int R, int /*MODE*/ = kModeForward) { return R <= 4 ? 640 : 512; }

// Static shared memory of a mode beyond the rings (the weight table).
constexpr uint32_t static_smem(int MODE) {
  return MODE == kModeTable ? 2u * kTableNodes * 16u : 0u;
}


// Prefetch depth of a tile shape: the deepest ring (1..6 planes beyond the
// R+1 in use) whose shared memory still lets the CTAs that the launch bounds
// admit be resident together (640 threads per SM for R <= 4: two CTAs of
// 256 threads, five of 128 or ten of 64; 512 for the wider stencils).
template <int R, int TX, int TY, int NC, int MODE = kModeForward>
constexpr int auto_pf() {
  const uint32_t budget =
      219u * 1024u / (threads_per_sm(R, MODE) / (TX * TY)) - static_smem(MODE);
  const int rx = ((R + 3) / 4) * 4;
  const uint32_t up = ((4 * TX + 2 * rx) * (TY + 2 * R) * 4 + 127) / 128 * 128;
  const uint32_t tp = (4 * TX * TY * 4 + 127) / 128 * 128;
  const bool split = R >= 5;
  for (int pf = 6; pf > 1; --pf) {
    const int su = split ? pf + 1 : R + 1 + pf, si = split ? pf + 1 : 0;
    const uint32_t smem =
        su * up + (pf + 1) * (2 + NC) * tp + si * tp + 2 * (su + pf + 1 + si) * 8 + 128;
    if (smem <= budget) return pf;
  }
  return 1;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Loads from shared memory at a 32-bit shared address.  Volatile, so that no
// load of a ring slot is merged with an earlier load of the same slot or
// moved across the mbarrier wait that makes the slot's new plane visible.
__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}

__device__ __forceinline__ float lds1(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map,
                                            int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// 3D tile load whose lines are marked first for eviction from L2: for
// tiles that are read exactly once (u^{n-1}, A), so that they do not push out
// the u^n planes that neighbouring columns are about to read as halos.
__device__ __forceinline__ void tma_load_3d_stream(uint32_t dst, const CUtensorMap* map,
                                                   int x, int y, int z, uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::"
      "bytes.L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], pol;\n\t}" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Streaming 128-bit store (evict-first): u^{n+1} is not read again in this
// launch.
__device__ __forceinline__ void st_stream(float* p, float a, float b, float c, float d) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ int sponge_depth(int g, int nbl, int n) {
  int d = nbl - g;
  int e = g - (n + nbl - 1);
  d = d > e ? d : e;
  return d > 0 ? d : 0;
}

__device__ __forceinline__ float lane(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Lanes (0,1) (p = 0) or (2,3) (p = 1) of a float4 as a packed pair.
__device__ __forceinline__ float2 half2of(const float4& v, int p) {
  return p == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
}

// h^2 times the Laplacian of four consecutive x points with uniform weights:
// lap = (hi + lo) u + sum_{j=1..R} c_j S_j, S_j the sum of the six neighbours
// at distance j, hi + lo = -6 sum c_j the centre weight of the FP32 weights c_j
// (launch_weights: exact in FP64, split into FP32 hi and lo parts).  With hi
// alone the rounded centre weight leaves the stencil a row sum of ~1e-7: the
// Laplacian of a constant field is then not zero but that constant times a
// fixed bias, a spurious mass term whose phase error grows with every step
// (about 1e-5 of the wavefield after 200 steps at space order 8).  With the
// pair the residual is rounding noise without a bias.  Lanes (0,1) and (2,3) run as
// packed pairs: each packed operation rounds every lane exactly as its scalar
// form.  xr holds the row through the points (the points at xr[XO .. XO+3]),
// yn(j, lo, hi) gives the float4s j rows below and above, zn(o) the float4 of
// the plane at z offset o.
template <int R, int XO, class YN, class ZN>
__device__ __forceinline__ void lap4_packed(const float* xr, YN yn, ZN zn, const float* c,
                                            float c0hi, float c0lo, float lap[4]) {
  const float4 uc = zn(0);
  const float2 hi2 = make_float2(c0hi, c0hi), lo2 = make_float2(c0lo, c0lo);
  float2 lp[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 u2 = half2of(uc, p);
    lp[p] = __ffma2_rn(hi2, u2, __fmul2_rn(lo2, u2));
  }
#pragma unroll
  for (int jj = 1; jj <= R; ++jj) {
    float4 ym, yp;
    yn(jj, ym, yp);
    const float4 zm = zn(-jj), zp = zn(jj);
    const float2 cj = make_float2(c[jj], c[jj]);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int xa = XO + 2 * p - jj, xb = XO + 2 * p + jj;
      // even distances pair aligned register halves; odd ones would
      // straddle two and are summed lane by lane
      const float2 sx =
          (jj & 1) ? make_float2(__fadd_rn(xr[xa], xr[xb]), __fadd_rn(xr[xa + 1], xr[xb + 1]))
                   : __fadd2_rn(make_float2(xr[xa], xr[xa + 1]), make_float2(xr[xb], xr[xb + 1]));
      const float2 sy = __fadd2_rn(half2of(ym, p), half2of(yp, p));
      const float2 sz = __fadd2_rn(half2of(zm, p), half2of(zp, p));
      lp[p] = __ffma2_rn(cj, __fadd2_rn(__fadd2_rn(sx, sy), sz), lp[p]);
    }
  }
  lap[0] = lp[0].x;
  lap[1] = lp[0].y;
  lap[2] = lp[1].x;
  lap[3] = lp[1].y;
}

// Leapfrog update of four points where b = 0: u^{n+1} = A(lap + s) + (2u - u^{n-1})
// with e = A(lap + s), as packed pairs (the roundings of the scalar form).
__device__ __forceinline__ void update4_inner(const float lap[4], const float src[4],
                                              const float4& uc, const float4& up,
                                              const float4& Av, float res[4], float ev[4]) {
  const float2 two = make_float2(2.0f, 2.0f);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 ls = __fadd2_rn(make_float2(lap[2 * p], lap[2 * p + 1]),
                                 make_float2(src[2 * p], src[2 * p + 1]));
    const float2 a2 = half2of(Av, p);
    const float2 u2 = half2of(up, p);
    const float2 e2 = __fmul2_rn(a2, ls);
    const float2 r2 =
        __ffma2_rn(a2, ls, __ffma2_rn(two, half2of(uc, p), make_float2(-u2.x, -u2.y)));
    ev[2 * p] = e2.x;
    ev[2 * p + 1] = e2.y;
    res[2 * p] = r2.x;
    res[2 * p + 1] = r2.y;
  }
}

// The general damped update, (1+b) u^{n+1} = A(lap + s) + 2u - (1-b) u^{n-1},
// b = bscale (dxx + dzz) per lane; lanes with ok[l] false give 0 (points
// outside the grid).  For b = 0 it rounds exactly as update4_inner.
__device__ __forceinline__ void update4_layer(const float lap[4], const float src[4],
                                              const float4& uc4, const float4& up,
                                              const float4& Av, const float dxx[4], float dzz,
                                              float bscale, const bool ok[4], float res[4],
                                              float ev[4]) {
  // lanes (0,1) and (2,3) as packed pairs, each operation rounding every lane
  // exactly as its scalar form; the division stays per lane
  const float2 one = make_float2(1.0f, 1.0f), two = make_float2(2.0f, 2.0f);
  const float2 bs2 = make_float2(bscale, bscale), dz2 = make_float2(dzz, dzz);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 b = __fmul2_rn(bs2, __fadd2_rn(make_float2(dxx[2 * p], dxx[2 * p + 1]), dz2));
    const float2 ls = __fadd2_rn(make_float2(lap[2 * p], lap[2 * p + 1]),
                                 make_float2(src[2 * p], src[2 * p + 1]));
    const float2 a2 = half2of(Av, p);
    const float2 e = __fmul2_rn(a2, ls);
    const float2 omb = __fadd2_rn(one, make_float2(-b.x, -b.y));  // 1 - b
    const float2 t2 = __ffma2_rn(a2, ls,
                                 __ffma2_rn(make_float2(-omb.x, -omb.y), half2of(up, p),
                                            __fmul2_rn(two, half2of(uc4, p))));
    const float2 d = __fadd2_rn(one, b);
    // inside the layer divide by 1+b (fast reciprocal; select, no branch)
    const float tx = (b.x != 0.0f) ? __fdividef(t2.x, d.x) : t2.x;
    const float ty = (b.y != 0.0f) ? __fdividef(t2.y, d.y) : t2.y;
    res[2 * p] = ok[2 * p] ? tx : 0.0f;
    res[2 * p + 1] = ok[2 * p + 1] ? ty : 0.0f;
    ev[2 * p] = ok[2 * p] ? e.x : 0.0f;
    ev[2 * p + 1] = ok[2 * p + 1] ? e.y : 0.0f;
  }
}

// One CTA: the xy tile (tile_x, tile_y), output planes [zbeg, zend).  All
// threads of the CTA must call this with the same arguments.
//
// Ring bookkeeping.  u planes are numbered j = 0 .. J-1 (z = zbeg - R + j) and
// live in slot j mod SU; u^{n-1}/A tiles i = 0 .. zl-1 (z = zbeg + i) in slot
// i mod SA.  Output plane k (i = k - zbeg) reads the staged plane jk = i + R
// for its x and y neighbours and takes plane jn = i + 2R into the register
// queue; once every thread has passed the plane, thread 0 refills slot
// jk mod SU with plane jk + SU and slot i mod SA with tile i + SA.  The slots
// are tracked as byte offsets that advance by one pitch per plane.
//
// Split staging (R >= 5).  The halo ring holds the centre planes h = 0 .. zl
// (z = zbeg + h; plane zl only for receivers of the last plane) in slot
// h mod SU; the interior ring holds planes j = 0 .. J-1 (numbered as above)
// in slot j mod SI.  The prologue takes planes 0 .. 2R-1 into the queue in
// batches of SI, refilling the batch's slots after a barrier; output plane k
// then takes plane jn = i + 2R from the interior ring and its x and y
// neighbours from halo plane i.
//
// Register queue: q[R + o] holds the thread's own float4 of plane jk + o,
// o = -R .. R; it shifts by one entry per plane.  (Unrolling the z loop by
// 2R+1 so that the queue rotates by register naming instead was measured
// slower on GB300: the SO 8 body then overflows the instruction cache, 234
// against 280 Gpts/s on 592^3; two planes per block ran 1.5 % slower.)
template <int R, int TX, int TY, int PF, int MODE>
__device__ __forceinline__ void run_column(const CUtensorMap* tm_halo,
                                           const CUtensorMap* tm_cur,
                                           const CUtensorMap* tm_prev,
                                           const CUtensorMap* tm_A,
                                           const CUtensorMap* tm_C,
                                           const StepArgs& a, const StepOverride& ov,
                                           float* __restrict__ out,
                                           int tile_x, int tile_y, int zbeg, int zend,
                                           unsigned char* smem) {
  constexpr int NC = (MODE == kModePerCell) ? R : 0;
  using C = Cfg<R, TX, TY, PF, NC>;
  constexpr bool SPLIT = C::SPLIT;
  constexpr int NQ = 2 * R + 1;
  const int tid = threadIdx.x;
  const int tx = tid % TX;
  const int ty = tid / TX;
  const int x0 = a.xfirst + tile_x * C::BX;
  const int y0 = a.yfirst + tile_y * C::BY;
  if (zbeg >= zend) return;
  const int zl = zend - zbeg;
  const int J = zl + 2 * R;  // u planes zbeg-R .. zend-1+R
  // once any CTA has recorded a failed wait, later columns and launches of
  // the same run return at once instead of waiting again (read by one
  // thread and shared, so the whole CTA takes the same branch)
  __shared__ int s_abort;
  if (tid == 0) s_abort = *reinterpret_cast<volatile const int*>(a.err);
  __syncthreads();
  if (s_abort) return;

  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_u0 = sbase + C::OFF_BAR;
  const uint32_t bar_a0 = bar_u0 + 8 * C::SU;
  const uint32_t bar_i0 = bar_a0 + 8 * C::SA;
  // shared addresses of the rings
  const uint32_t ubuf = sbase;
  const uint32_t pbuf = sbase + C::OFF_P;
  const uint32_t abuf = sbase + C::OFF_A;
  const uint32_t cbuf = sbase + C::OFF_C;
  const uint32_t ibuf = sbase + C::OFF_I;

  // kModeTable: the weight table of this grid, read from every point's
  // Courant number (made visible by the barrier below)
  __shared__ float4 s_tab[MODE == kModeTable ? 2 * kTableNodes : 1];
  if (MODE == kModeTable) {
    for (int i = tid; i < 2 * a.tab_nodes; i += C::NT) s_tab[i] = a.table[i];
  }
  if (tid == 0) {
    for (int s = 0; s < C::SU; ++s) mbar_init(bar_u0 + 8 * s, 1);
    for (int s = 0; s < C::SA; ++s) mbar_init(bar_a0 + 8 * s, 1);
    for (int s = 0; s < C::SI; ++s) mbar_init(bar_i0 + 8 * s, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // producer (thread 0): next plane / tile to issue.  Halo tiles: planes
  // j of the single ring, or centre planes h (z = zbeg + h) when split.
  int ju_next = 0, ia_next = 0, ji_next = 0;
  const int UN = SPLIT ? zl + 1 : J;
  const int z_u0 = SPLIT ? zbeg : zbeg - R;
  auto issue_u = [&](int j, uint32_t uoff) {
    if (j >= UN) return;
    ju_next = j + 1;
    const int z = z_u0 + j;
    if (ov.debug_skip_plane >= 0 && z == ov.debug_skip_plane) return;
    const uint32_t bar = bar_u0 + 8 * (uoff / C::UPITCH);
    mbar_expect_tx(bar, C::UBYTES);
    tma_load_3d(sbase + uoff, tm_halo, x0 - C::RX, y0 - R, z, bar);
  };
  // interior tiles of u^n (split staging): plane j, z = zbeg - R + j
  auto issue_i = [&](int j, uint32_t ioff) {
    if (j >= J) return;
    ji_next = j + 1;
    const int z = zbeg - R + j;
    if (ov.debug_skip_plane >= 0 && z == ov.debug_skip_plane) return;
    const uint32_t bar = bar_i0 + 8 * (ioff / C::TPITCH);
    mbar_expect_tx(bar, C::TBYTES);
    tma_load_3d(ibuf + ioff, tm_cur, x0, y0, z, bar);
  };
  auto issue_a = [&](int i, uint32_t aoff) {
    if (i >= zl) return;
    ia_next = i + 1;
    const int z = zbeg + i;
    const uint32_t bar = bar_a0 + 8 * (aoff / C::TPITCH);
    mbar_expect_tx(bar, (2 + NC) * C::TBYTES);
    tma_load_3d_stream(sbase + C::OFF_P + aoff, tm_prev, x0, y0, z, bar);
    tma_load_3d_stream(sbase + C::OFF_A + aoff, tm_A, x0, y0, z, bar);
#pragma unroll
    for (int j = 0; j < NC; ++j)  // coefficient field j sits j*Nz planes further
      tma_load_3d(sbase + C::OFF_C + ((aoff / C::TPITCH) * NC + j) * C::TPITCH, tm_C, x0, y0,
                  z + j * a.Nz, bar);
  };

  // the u^n ring is refilled by thread 0, the u^{n-1}/A ring by the first
  // thread of warp 1, so that no single warp carries both after the barrier
  constexpr int kAuxTid = 32;
  static_assert(C::NT > kAuxTid, "CTAs have at least two warps");
  if (tid == 0) {
    for (int j = 0; j < C::SU; ++j) issue_u(j, j * C::UPITCH);
    for (int j = 0; j < C::SI; ++j) issue_i(j, j * C::TPITCH);
  }
  if (tid == kAuxTid) {
    for (int i = 0; i < C::SA; ++i) issue_a(i, i * C::TPITCH);
  }

  // byte offsets of the thread's own float4 in a staged plane / tile
  const uint32_t crow = 4u * ((ty + R) * C::W + 4 * tx + C::RX);
  const uint32_t ctile = 4u * (ty * C::BX + 4 * tx);
  float4 q[NQ];
  bool bad = false;

  if constexpr (SPLIT) {
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      const int slot = j % C::SI;
      bad |= !mbar_wait(bar_i0 + 8 * slot, (j / C::SI) & 1, ov.spin_limit);
      q[j] = lds4(ibuf + slot * C::TPITCH + ctile);
      if (slot == C::SI - 1 || j == 2 * R - 1) {
        if (__syncthreads_or(bad)) goto fail;
        if (tid == 0)
          for (int jj = j - slot; jj <= j; ++jj) issue_i(jj + C::SI, (jj % C::SI) * C::TPITCH);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      const int slot = j % C::SU;
      bad |= !mbar_wait(bar_u0 + 8 * slot, (j / C::SU) & 1, ov.spin_limit);
      q[j] = lds4(ubuf + slot * C::UPITCH + crow);
      if (j < R) {
        if (__syncthreads_or(bad)) goto fail;
        if (tid == 0) issue_u(j + C::SU, slot * C::UPITCH);
      }
    }
  }

  {
    // entry ranges of this tile, skipping entries below this z chunk
    const int tile = tile_y * a.tiles_x + tile_x;
    int ip = 0, iend = 0, rp = 0, rend = 0;
    if (a.inj_start) {
      ip = a.inj_start[tile];
      iend = a.inj_start[tile + 1];
      while (ip < iend && a.inj[ip].z < zbeg) ++ip;
    }
    if (a.rec_start) {
      rp = a.rec_start[tile];
      rend = a.rec_start[tile + 1];
      while (rp < rend && a.recs[rp].z < zbeg) ++rp;
    }
    // plane of the next entry of each list (INT_MAX: none), kept in a
    // register so that planes without entries touch neither list
    int iz = ip < iend ? a.inj[ip].z : INT_MAX;
    int rz = rp < rend ? a.recs[rp].z : INT_MAX;

    const int gy = y0 + ty;
    const int gx = x0 + 4 * tx;
    const bool in_grid = gy < a.yend && gx < a.xend;
    const float c0hi = ov.c[0], c0lo = ov.c[kMaxR + 1];  // centre weight (launch_weights)
    // the layer in array coordinates (shifted for subdomains)
    const int nblx = a.nbl - a.offx, nbly = a.nbl - a.offy, nblz = ov.nblz - a.offz;
    const int dyv = sponge_depth(gy, nbly, a.ny);
    float dxx[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int d = sponge_depth(gx + l, nblx, a.nx);
      dxx[l] = static_cast<float>(d * d + dyv * dyv);
    }
    // planes [zf_lo, zf_hi) of this column have b = 0 at every point and no
    // point outside the grid: there the update needs no sponge terms or masks
    int zf_lo = nblz, zf_hi = nblz + a.nz;
    {
      const bool no_sponge = a.bscale == 0.0f;
      const bool full = x0 + C::BX <= a.xend && y0 + C::BY <= a.yend;
      const bool inner_xy = x0 >= nblx && x0 + C::BX <= nblx + a.nx && y0 >= nbly &&
                            y0 + C::BY <= nbly + a.ny;
      if (no_sponge) {
        zf_lo = zbeg;
        zf_hi = zend;
      }
      if (!full || !(no_sponge || inner_xy)) {
        zf_lo = 0;
        zf_hi = 0;
      }
    }
    size_t off = (static_cast<size_t>(zbeg) * a.Ny + gy) * a.pitch + gx;
    const size_t plane_stride = static_cast<size_t>(a.Ny) * a.pitch;
    // adjoint mode: the imaging condition's e and gradient of the next plane
    // are read one plane ahead, so their global-load latency overlaps the
    // current plane (each point of the chunk is touched by this thread only);
    // up to SO 8 (the wider stencils have no registers to spare and load them
    // in the update)
    constexpr bool kAdjAhead = MODE == kModeAdjoint && R <= 4;
    float4 ein_nx = make_float4(0.f, 0.f, 0.f, 0.f), g_nx = ein_nx;
    if (kAdjAhead && in_grid) {
      ein_nx = __ldg(reinterpret_cast<const float4*>(a.e_in + off));
      g_nx = *reinterpret_cast<const float4*>(a.grad + off);
    }

    // ring slots: sk holds plane jk (split: halo plane ik, parity pk), sn
    // plane jn (parity pn; split: in the interior ring), sa tile ik
    constexpr int SN = SPLIT ? C::SI : C::SU;
    int sk = SPLIT ? 0 : R % C::SU;
    uint32_t pk = 0;
    int sn = (2 * R) % SN;
    uint32_t pn = ((2 * R) / SN) & 1;
    int sa = 0;
    uint32_t pa = 0;

    // several planes per loop trip: the compiler renames the queue for all
    // but the last of them instead of shifting it.  Measured on 592^3
    // (Gpts/s, trips of 1 / 2 / 3 / 4 planes): SO 8 -, 350, 360, 345;
    // SO 16 196, 210, 217, 220 (6: 204, 8: 212); SO 12 248, 261, 266, 277.
    // Per-cell weights keep one plane per trip (more would spill).
    constexpr int kUnroll = MODE == kModePerCell ? 1 : (R >= 5 ? 4 : 3);
#pragma unroll kUnroll
    for (int k = zbeg; k < zend; ++k) {
      {
#define FD_Q(o) q[R + (o)]
        const int ik = k - zbeg;
        const int jk = ik + R;
        float4 ein_c = ein_nx, g_c = g_nx;
        if (kAdjAhead) {
          if (in_grid && k + 1 < zend) {
            ein_nx = __ldg(reinterpret_cast<const float4*>(a.e_in + off + plane_stride));
            g_nx = *reinterpret_cast<const float4*>(a.grad + off + plane_stride);
          }
        }
        if constexpr (SPLIT) {
          bad |= !mbar_wait(bar_u0 + 8 * sk, pk, ov.spin_limit);
          bad |= !mbar_wait(bar_i0 + 8 * sn, pn, ov.spin_limit);
          q[2 * R] = lds4(ibuf + sn * C::TPITCH + ctile);
        } else {
          bad |= !mbar_wait(bar_u0 + 8 * sn, pn, ov.spin_limit);
          q[2 * R] = lds4(ubuf + sn * C::UPITCH + crow);
        }
        bad |= !mbar_wait(bar_a0 + 8 * sa, pa, ov.spin_limit);
        // the float4 of the plane at z offset o (-R .. R)
        auto zq = [&](int o) -> float4 { return q[R + o]; };

        const uint32_t P = ubuf + sk * C::UPITCH + crow;
        float xr[4 * C::NROW4];
#pragma unroll
        for (int m = 0; m < C::NROW4; ++m) {
          const float4 v = (m == C::NROW4 / 2) ? FD_Q(0) : lds4(P + 16 * (m - C::NROW4 / 2));
          xr[4 * m + 0] = v.x;
          xr[4 * m + 1] = v.y;
          xr[4 * m + 2] = v.z;
          xr[4 * m + 3] = v.w;
        }
        float lap[4];
        // per-point weights: lap = sum_j c_j (S_j - 6u), so no FP32 centre weight
        // carries a rounding bias into the row sum
        if (MODE == kModePerCell || MODE == kModeTable) {
          // per-point weights c_1..c_R: from the staged coefficient tiles, or
          // interpolated linearly in the table at the point's own
          // A = (v dt / h)^2
          float ct[4][R];
          if (MODE == kModeTable) {
            const float4 At = lds4(abuf + sa * C::TPITCH + ctile);
            const float top = static_cast<float>(a.tab_nodes - 1);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              const float x = fminf(fmaxf((lane(At, l) - a.tab_lo) * a.tab_inv, 0.0f), top);
              const int i = min(static_cast<int>(x), a.tab_nodes - 2);
              const float f = x - static_cast<float>(i);
              const float4 t0 = s_tab[2 * i];
              const float4 dt = s_tab[2 * i + 1];
#pragma unroll
              for (int jj = 1; jj <= R; ++jj)
                ct[l][jj - 1] = fmaf(f, lane(dt, jj - 1), lane(t0, jj - 1));
            }
          }
          if (MODE == kModeTable) {
            // lane by lane (the sixteen interpolated weights stay live: as
            // packed pairs they would spill)
#pragma unroll
            for (int jj = 1; jj <= R; ++jj) {
              const float4 ym = lds4(P - 4 * jj * C::W);
              const float4 yp = lds4(P + 4 * jj * C::W);
#pragma unroll
              for (int l = 0; l < 4; ++l) {
                const float sx = xr[C::RX + l - jj] + xr[C::RX + l + jj];
                const float sy = lane(ym, l) + lane(yp, l);
                const float sz = lane(zq(-jj), l) + lane(zq(jj), l);
                const float d = fmaf(-6.0f, xr[C::RX + l], (sx + sy) + sz);
                lap[l] = (jj == 1) ? ct[l][jj - 1] * d : fmaf(ct[l][jj - 1], d, lap[l]);
              }
            }
          } else {
          // per-cell weights: lanes (0,1) and (2,3) as packed pairs, each with
          // its own weights (the roundings of the scalar form, lane by lane)
          const float2 m6 = make_float2(-6.0f, -6.0f);
          float2 lp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
          for (int jj = 1; jj <= R; ++jj) {
            float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (MODE == kModePerCell)
              cv = lds4(cbuf + (sa * NC + (jj - 1)) * C::TPITCH + ctile);
            const float4 ym = lds4(P - 4 * jj * C::W);
            const float4 yp = lds4(P + 4 * jj * C::W);
            const float4 zm = zq(-jj), zp = zq(jj);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              const int xa = C::RX + 2 * p - jj, xb = C::RX + 2 * p + jj;
              const float2 sx =
                  (jj & 1) ? make_float2(__fadd_rn(xr[xa], xr[xb]), __fadd_rn(xr[xa + 1], xr[xb + 1]))
                           : __fadd2_rn(make_float2(xr[xa], xr[xa + 1]),
                                        make_float2(xr[xb], xr[xb + 1]));
              const float2 sy = __fadd2_rn(half2of(ym, p), half2of(yp, p));
              const float2 sz = __fadd2_rn(half2of(zm, p), half2of(zp, p));
              const float2 u2 = make_float2(xr[C::RX + 2 * p], xr[C::RX + 2 * p + 1]);
              const float2 d = __ffma2_rn(m6, u2, __fadd2_rn(__fadd2_rn(sx, sy), sz));
              const float2 cj = half2of(cv, p);
              lp[p] = (jj == 1) ? __fmul2_rn(cj, d) : __ffma2_rn(cj, d, lp[p]);
            }
          }
          lap[0] = lp[0].x;
          lap[1] = lp[0].y;
          lap[2] = lp[1].x;
          lap[3] = lp[1].y;
          }
        } else {
          lap4_packed<R, C::RX>(
              xr,
              [&](int jj, float4& ym, float4& yp) {
                ym = lds4(P - 4 * jj * C::W);
                yp = lds4(P + 4 * jj * C::W);
              },
              zq, ov.c, c0hi, c0lo, lap);
        }

        // point sources of this plane (owner thread adds its share)
        float src[4] = {0.f, 0.f, 0.f, 0.f};
        if (k == iz) {
          while (ip < iend) {
            const InjEntry e = a.inj[ip];
            if (e.z != k) break;
            if (e.ly == ty && (e.lx >> 2) == tx) {
              const float val =
                  e.w * a.inj_val[static_cast<size_t>(a.inj_row) * a.inj_ncol + e.col];
#pragma unroll
              for (int l = 0; l < 4; ++l) src[l] += ((e.lx & 3) == l) ? val : 0.f;
            }
            ++ip;
          }
          iz = ip < iend ? a.inj[ip].z : INT_MAX;
        }

        const float4 up = lds4(pbuf + sa * C::TPITCH + ctile);
        const float4 Av = lds4(abuf + sa * C::TPITCH + ctile);
        float res[4], ev[4];
        // the same explicit roundings in every mode and on both branches, so
        // that a recomputed segment reproduces the stored states bit for bit
        if (k >= zf_lo && k < zf_hi) {
          // b = 0: (1-b) = 1 and no division; every column is inside the grid
          update4_inner(lap, src, FD_Q(0), up, Av, res, ev);
        } else {
          const int dz = sponge_depth(k, nblz, a.nz);
          const bool ok[4] = {gx < a.xend, gx + 1 < a.xend, gx + 2 < a.xend, gx + 3 < a.xend};
          update4_layer(lap, src, FD_Q(0), up, Av, dxx, static_cast<float>(dz * dz), a.bscale, ok,
                        res, ev);
        }
        if (in_grid) {
          st_stream(out + off, res[0], res[1], res[2], res[3]);
          if (MODE == kModeStoreE)  // read back after the whole segment: not kept in L2
            st_stream(a.e_out + off, ev[0], ev[1], ev[2], ev[3]);
          if (MODE == kModeAdjoint) {
            const float4 ein =
                kAdjAhead ? ein_c : __ldg(reinterpret_cast<const float4*>(a.e_in + off));
            const float4 uc = FD_Q(0);
            float4 g = kAdjAhead ? g_c : *reinterpret_cast<const float4*>(a.grad + off);
            g.x -= uc.x * ein.x * a.inv_dt2;
            g.y -= uc.y * ein.y * a.inv_dt2;
            g.z -= uc.z * ein.z * a.inv_dt2;
            g.w -= uc.w * ein.w * a.inv_dt2;
            *reinterpret_cast<float4*>(a.grad + off) = g;
          }
        }
        off += plane_stride;

        // receivers whose floor node lies in this plane: one thread each,
        // trilinear over planes k and k+1 (both staged)
        if (k == rz) {
          int rq = rp;
          while (rq < rend && a.recs[rq].z == k) ++rq;
          const int s1 = sk + 1 == C::SU ? 0 : sk + 1;
          // split staging: halo plane ik + 1 is in flight, not yet waited for
          if (SPLIT) bad |= !mbar_wait(bar_u0 + 8 * s1, s1 == 0 ? pk ^ 1u : pk, ov.spin_limit);
          const uint32_t P0 = ubuf + sk * C::UPITCH;
          const uint32_t P1 = ubuf + s1 * C::UPITCH;
          for (int e = rp + tid; e < rq; e += C::NT) {
            const RecEntry r = a.recs[e];
            const uint32_t o = 4u * ((r.ly + R) * C::W + r.lx + C::RX);
            constexpr uint32_t W4 = 4u * C::W;
            const float gx0 = 1.0f - r.fx, gy0 = 1.0f - r.fy;
            const float p0 = gy0 * (gx0 * lds1(P0 + o) + r.fx * lds1(P0 + o + 4)) +
                             r.fy * (gx0 * lds1(P0 + o + W4) + r.fx * lds1(P0 + o + W4 + 4));
            const float p1 = gy0 * (gx0 * lds1(P1 + o) + r.fx * lds1(P1 + o + 4)) +
                             r.fy * (gx0 * lds1(P1 + o + W4) + r.fx * lds1(P1 + o + W4 + 4));
            a.rec_out[static_cast<size_t>(a.rec_row) * a.rec_ncol + r.col] =
                (1.0f - r.fz) * p0 + r.fz * p1;
          }
          rp = rq;
          rz = rp < rend ? a.recs[rp].z : INT_MAX;
        }

        if (__syncthreads_or(bad)) goto fail;
        if (tid == 0) {
          if constexpr (SPLIT) {
            issue_u(ik + C::SU, sk * C::UPITCH);
            issue_i(jk + R + C::SI, sn * C::TPITCH);
          } else {
            issue_u(jk + C::SU, sk * C::UPITCH);
          }
        }
        if (tid == kAuxTid) issue_a(ik + C::SA, sa * C::TPITCH);
        sk = (sk + 1 == C::SU) ? 0 : sk + 1;
        pk ^= (sk == 0) ? 1u : 0u;
        sn = (sn + 1 == SN) ? 0 : sn + 1;
        pn ^= (sn == 0) ? 1u : 0u;
        sa = (sa + 1 == C::SA) ? 0 : sa + 1;
        pa ^= (sa == 0) ? 1u : 0u;
#pragma unroll
        for (int j = 0; j < NQ - 1; ++j) q[j] = q[j + 1];
#undef FD_Q
      }
    }
  }
  // every issued copy has been waited for (split staging: but for halo
  // plane zl, which only receivers on the last plane wait for, so thread 0
  // waits for it here); release the barriers so the shared memory can host
  // the next column
  if (tid == 0) {
    if (SPLIT && ju_next > zl && !(ov.debug_skip_plane >= 0 && zend == ov.debug_skip_plane)) {
      if (!mbar_wait(bar_u0 + 8 * (zl % C::SU), (zl / C::SU) & 1, ov.spin_limit))
        atomicOr(a.err, 1);
    }
    for (int s = 0; s < C::SU; ++s) mbar_inval(bar_u0 + 8 * s);
    for (int s = 0; s < C::SA; ++s) mbar_inval(bar_a0 + 8 * s);
    for (int s = 0; s < C::SI; ++s) mbar_inval(bar_i0 + 8 * s);
  }
  __syncthreads();
  return;

fail:
  // each issuing thread waits (bounded) for the copies it still has in flight
  if (tid == 0) {
    atomicOr(a.err, 1);
    for (int j = max(0, ju_next - C::SU); j < ju_next; ++j) {
      if (ov.debug_skip_plane >= 0 && z_u0 + j == ov.debug_skip_plane) continue;
      mbar_wait(bar_u0 + 8 * (j % C::SU), (j / C::SU) & 1, ov.spin_limit);
    }
    if constexpr (SPLIT) {
      for (int j = max(0, ji_next - C::SI); j < ji_next; ++j) {
        if (ov.debug_skip_plane >= 0 && zbeg - R + j == ov.debug_skip_plane) continue;
        mbar_wait(bar_i0 + 8 * (j % C::SI), (j / C::SI) & 1, ov.spin_limit);
      }
    }
  }
  if (tid == kAuxTid) {
    for (int i = max(0, ia_next - C::SA); i < ia_next; ++i)
      mbar_wait(bar_a0 + 8 * (i % C::SA), (i / C::SA) & 1, ov.spin_limit);
  }
}

// Persistent sweep over every (tile, plane) work unit of one or more grids.
// The units of shot s are numbered tile-major (unit = tile * Nz + z) after the
// units of shots 0..s-1; CTA c of G takes the contiguous share
// [c*total/G, (c+1)*total/G), cut into per-tile z segments.  With G equal to
// the number of resident CTAs every SM streams the same number of planes and
// no CTA waits for a second wave.  A scheduled sweep (ov.items set) instead
// runs the host-built work items [item_start[c], item_start[c+1]) of CTA c:
// z ranges of tile columns in any order (column waves, see fd_sched.cu).
template <int R, int TX, int TY, int PF, int MODE>
__global__ void __launch_bounds__(TX* TY, threads_per_sm(R, MODE) / (TX * TY))
    sweep_kernel(const ShotDesc* __restrict__ shots, const long long* __restrict__ prefix,
                 int nshots, const __grid_constant__ StepOverride ov) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  __shared__ StepArgs sa;
  const long long total = prefix[nshots];
  const long long lo = total * blockIdx.x / gridDim.x;
  const long long hi = total * (blockIdx.x + 1) / gridDim.x;
  const int cur = ov.cur;
  int s = 0;
  for (long long pos = lo; pos < hi;) {
    while (pos >= prefix[s + 1]) ++s;
    const ShotDesc* S = shots + s;
    const long long local = pos - prefix[s];
    const int Nz = S->args.Nz;
    const int tile = static_cast<int>(local / Nz);
    const int zb = static_cast<int>(local % Nz);
    const long long left = hi - pos;
    const int ze = left < Nz - zb ? zb + static_cast<int>(left) : Nz;
    if (threadIdx.x == 0) {
      sa = S->args;
      sa.inj_row = ov.inj_row;
      sa.rec_row = ov.rec_row;
      sa.e_out = ov.e_out;
      sa.e_in = ov.e_in;
    }
    __syncthreads();
    run_column<R, TX, TY, PF, MODE>(&S->halo[cur], &S->tile[cur], &S->tile[cur ^ 1], &S->A,
                                    &S->C, sa, ov,
                                    S->u[cur ^ 1], tile % sa.tiles_x, tile / sa.tiles_x,
                                    zb + ov.zfirst, ze + ov.zfirst, smem);
    __syncthreads();
    pos += ze - zb;
  }
}

// Scheduled sweep: CTA c runs the host-built work items
// [ov.item_start[c], ov.item_start[c+1]) in order, each the planes [zb, ze)
// of one tile column of one grid (column waves, fd_sched.cu).  A kernel of
// its own, so that the equal-share sweep above keeps its register allocation.
template <int R, int TX, int TY, int PF, int MODE>
__global__ void __launch_bounds__(TX* TY, threads_per_sm(R, MODE) / (TX * TY))
    sched_kernel(const ShotDesc* __restrict__ shots, const __grid_constant__ StepOverride ov) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  __shared__ StepArgs sa;
  const int cur = ov.cur;
  const int i1 = ov.item_start[blockIdx.x + 1];
  for (int i = ov.item_start[blockIdx.x]; i < i1; ++i) {
    const WorkItem w = ov.items[i];
    const ShotDesc* S = shots + w.shot;
    if (threadIdx.x == 0) {
      sa = S->args;
      sa.inj_row = ov.inj_row;
      sa.rec_row = ov.rec_row;
      sa.e_out = ov.e_out;
      sa.e_in = ov.e_in;
    }
    __syncthreads();
    run_column<R, TX, TY, PF, MODE>(&S->halo[cur], &S->tile[cur], &S->tile[cur ^ 1], &S->A,
                                    &S->C, sa, ov,
                                    S->u[cur ^ 1], w.tile % sa.tiles_x, w.tile / sa.tiles_x,
                                    w.zb + ov.zfirst, w.ze + ov.zfirst, smem);
    __syncthreads();
  }
}

}  // namespace fd
