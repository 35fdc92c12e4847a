// Feature description (§II-B: 6x6 grid of No-bin MIM histograms; §III: dominant index
// s = argmax of the patch histogram, Eq. 1, recoding MIM_n = (MIM - s) mod No, Eq. 2,
// and a second descriptor when the second-highest bin is within the dominant ratio of
// the peak).
//
//   desc_hist  : each warp takes several keypoints.  The 96x96 MIM patch (rows
//                y-48..y+47, columns x-48..x+47) is staged into shared memory in two
//                halves by TMA tensor copies whose x start is rounded down to 16 bytes
//                (112 x 48 boxes), the next half in flight while the current one is
//                counted; each lane counts a 16-pixel cell row through three bit planes
//                and popc, and the cell totals are reduced over the 16 lanes of a
//                half-warp.  Writes the unrecoded cell counts, s, s2 and the
//                second-descriptor flag.
//   desc_scan  : one CTA per image: exclusive scan of descriptors per keypoint (1 or 2;
//                for RIFT's baseline modes 1 from the unshifted MIM, or the No members of
//                the convolution-sequence ring, §II-C).
//   desc_write : one warp per keypoint: the recoded count vectors (a cyclic shift of the
//                bins of every cell) and their L2 norms.
#include <type_traits>

#include "kernels.h"

namespace rift2 {

constexpr int BOX_W = PATCH + 16;                 // 112 bytes: x start rounded down to 16
constexpr int HALF_ROWS = PATCH / 2;              // one job stages half a patch (3 cell rows)
constexpr int HBUF = (BOX_W * HALF_ROWS + 128 + 127) / 128 * 128;   // + slack for the
                                                                    // 4-byte realignment reads
constexpr int DH_WARPS = 8;
constexpr int DH_KPW = 4;                         // keypoints per warp

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

constexpr long long kWaitIters = 1ll << 24;   // try_wait polls before a wait gives up

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase, long long max_iter) {
  for (long long it = 0; it < max_iter; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Each warp takes the keypoints gw, gw + stride, ... of its image (gw its global warp
// index).  Every keypoint is two jobs, the upper and lower half of its patch; a job's
// 112 x 48 box is staged while the previous job is counted (two buffers per warp).
__global__ void __launch_bounds__(DH_WARPS * 32) desc_hist(const __grid_constant__ CUtensorMap tmap,
                                                           const __grid_constant__ Group gr,
                                                           KParams kp, DescribeWs ws,
                                                           FeatPtrs fp) {
  // [DH_WARPS][2 half-patch buffers][DH_WARPS][2 mbarriers]; no static shared memory, so
  // the dynamic block starts at the (16-byte aligned) base the TMA destination needs.
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(dsm + DH_WARPS * 2 * HBUF);
  const int img = blockIdx.y;
  const int row0 = gr.mrow[img];   // the image's first row in the stacked MIM
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkp = fp.counts[img][0];
  const int gw = blockIdx.x * DH_WARPS + warp, gstride = gridDim.x * DH_WARPS;
  if (gw >= nkp) return;   // warp-uniform
  const int njobs = 2 * ((nkp - gw + gstride - 1) / gstride);
  unsigned char* buf0 = dsm + warp * 2 * HBUF;
  const unsigned bar0 = smem_u32(&bars[2 * warp]);
  const int* kxy = fp.kp_xy[img];
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // lane 0: stage job q into buffer q & 1 (its previous contents were read before the
  // warp's last __syncwarp; the proxy fence orders those reads before the async write)
  auto issue = [&](int q) {
    const int k = gw + (q >> 1) * gstride;
    const int x = kxy[2 * k], y = kxy[2 * k + 1];
    const unsigned b = bar0 + 8 * (q & 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                 "r"(BOX_W * HALF_ROWS)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(buf0 + (q & 1) * HBUF)),
        "l"(&tmap), "r"((x - HALF_PATCH) & ~15),
        "r"(row0 + y - HALF_PATCH + (q & 1) * HALF_ROWS), "r"(b)
        : "memory");
  };
  if (lane == 0) issue(0);
  const int rho = lane & 15, half = lane >> 4;
  unsigned wsum[3] = {0, 0, 0};   // whole-patch bins as u16 pairs (each total <= 9216)
  for (int q = 0; q < njobs; ++q) {
    if (lane == 0 && q + 1 < njobs) issue(q + 1);
    const int k = gw + (q >> 1) * gstride, hh = q & 1;
    const int px = kxy[2 * k] - HALF_PATCH;
    const int sh = px - (px & ~15);
    if (!mbar_wait(bar0 + 8 * (q & 1), (q >> 1) & 1, ws.wait_iters)) {
      if (lane == 0) atomicExch(ws.status, ST_TIMEOUT);
      // the copies in flight may still land: wait for them with the full limit before
      // exiting, so that no copy into this CTA's shared memory outlives the kernel.  The
      // keypoints this warp leaves keep stale info words; desc_shifts reduces every shift
      // modulo No, so the descriptor kernels stay in bounds on them.
      mbar_wait(bar0 + 8 * (q & 1), (q >> 1) & 1, kWaitIters);
      if (q + 1 < njobs) mbar_wait(bar0 + 8 * ((q + 1) & 1), ((q + 1) >> 1) & 1, kWaitIters);
      return;
    }
    const unsigned char* buf = buf0 + (q & 1) * HBUF;
    unsigned short* raw = ws.raw + ((size_t)img * kp.kp_cap + k) * DESC_DIM;
    // A lane's 16 pixels start sh bytes into a 16-byte aligned 32-byte window, read with
    // two 16-byte loads (the 112-byte row pitch puts a quarter-warp's loads on distinct
    // banks); the window's words d .. d+4, d = sh / 4 (uniform over the warp), feed the
    // byte realignment through a uniform switch so that every index is static.
    const int a8 = (sh & 3) * 8;
    auto count_cells = [&](auto dc) {
      constexpr int d = decltype(dc)::value;
#pragma unroll 3
      for (int m = 0; m < CELLS * CELLS / 4; ++m) {
        const int cl = 2 * m + half;                 // cell within this half: 3 rows of 6
        const int ci = cl / CELLS, cj = cl % CELLS;
        const int c = hh * (CELLS * CELLS / 2) + cl;
        const uint4* wp = reinterpret_cast<const uint4*>(buf + (ci * CELL + rho) * BOX_W + cj * CELL);
        const uint4 lo = wp[0], hi = wp[1];
        const unsigned qw[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        // bit planes of the 16 pixels (MIM values 0..5 need three bits): bit i of byte j of
        // plane k is bit k of pixel 4i + j; a bin count is one 3-input logic op and a popc
        // (values 6 and 7 never occur, so 5 = b2 b0 and 4 = b2 !b0)
        static_assert(NO == 6, "bit-plane counting covers the values 0..5");
        unsigned p0b = 0, p1b = 0, p2b = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const unsigned v = __funnelshift_r(qw[d + i], qw[d + i + 1], a8);
          p0b |= (v & 0x01010101u) << i;
          p1b |= ((v >> 1) & 0x01010101u) << i;
          p2b |= ((v >> 2) & 0x01010101u) << i;
        }
        unsigned cnt[NO];
        cnt[5] = __popc(p2b & p0b);
        cnt[4] = __popc(p2b & ~p0b);
        cnt[3] = __popc(~p2b & p1b & p0b);
        cnt[2] = __popc(~p2b & p1b & ~p0b);
        cnt[1] = __popc(~p2b & ~p1b & p0b);
        cnt[0] = 16u - cnt[1] - cnt[2] - cnt[3] - cnt[4] - cnt[5];
        // pack two bins per word (cell totals <= 256)
        unsigned p0 = cnt[0] | (cnt[1] << 16);
        unsigned p1 = cnt[2] | (cnt[3] << 16);
        unsigned p2 = cnt[4] | (cnt[5] << 16);
#pragma unroll
        for (int dd = 1; dd < 16; dd <<= 1) {
          p0 += __shfl_xor_sync(0xffffffffu, p0, dd);
          p1 += __shfl_xor_sync(0xffffffffu, p1, dd);
          p2 += __shfl_xor_sync(0xffffffffu, p2, dd);
        }
        // p0, p1, p2 are the cell's bins (0,1), (2,3), (4,5) as u16 pairs: the raw layout
        wsum[0] += p0;
        wsum[1] += p1;
        wsum[2] += p2;
        if (rho < 3)
          reinterpret_cast<unsigned*>(raw + c * NO)[rho] = (rho == 0) ? p0 : (rho == 1) ? p1 : p2;
      }
    };
    switch (sh >> 2) {
      case 0: count_cells(std::integral_constant<int, 0>{}); break;
      case 1: count_cells(std::integral_constant<int, 1>{}); break;
      case 2: count_cells(std::integral_constant<int, 2>{}); break;
      default: count_cells(std::integral_constant<int, 3>{}); break;
    }
    if (hh == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) wsum[i] += __shfl_xor_sync(0xffffffffu, wsum[i], 16);
      const unsigned whole[NO] = {wsum[0] & 0xFFFFu, wsum[0] >> 16, wsum[1] & 0xFFFFu,
                                  wsum[1] >> 16, wsum[2] & 0xFFFFu, wsum[2] >> 16};
      if (lane == 0) {
        int s = 0;
        for (int b = 1; b < NO; ++b)
          if (whole[b] > whole[s]) s = b;
        int s2 = (s == 0) ? 1 : 0;
        for (int b = 0; b < NO; ++b)
          if (b != s && whole[b] > whole[s2]) s2 = b;
        unsigned has2 = (1000u * whole[s2] >= (unsigned)kp.ratio_pm * whole[s]) ? 1u : 0u;
        ws.info[(size_t)img * kp.kp_cap + k] = (unsigned)s | ((unsigned)s2 << 4) | (has2 << 8);
      }
      wsum[0] = wsum[1] = wsum[2] = 0;
    }
    __syncwarp();   // every lane's reads of this buffer precede its next staging
  }
}

// ------------------------------------------- spatial orientation normalisation (variant)
// desc_spatial: one warp per keypoint (several in turn).  The window of MIM rows y-66..y+66
// and 160 columns from (x-66) rounded down to 16 bytes is staged by one TMA box: it holds
// the disc |d| <= 48 and every sample of the rotated grid (|rnd(R d)| <= 48 (cos 30 +
// sin 30) < 66).  Out-of-image pixels are excluded by explicit bounds tests, never by the
// copy's fill value.
//  1. Disc histogram and centroid sums: each lane takes 16-pixel row segments, forms the
//     three bit planes of their MIM values (as desc_hist does), masks them to the disc
//     row and the image, and adds per bin the popcount, the sum of the pixels' dx (from
//     popcounts against the four bit-weight masks of the pixel index) and dy x count.
//  2. Dominant index s, secondary s2 and the ratio test (Eq. 1, §III) on the disc counts.
//  3. Per descriptor index w: frame (cos, sin) of w pi / No in Q14, negated when the
//     centroid of the w-pixels projects negatively on the axis (cos, -sin); the grid
//     d = (dx, dy) in [-48, 47]^2 is sampled at p + (rnd(c dx + s dy), rnd(-s dx + c dy)),
//     rnd rounding x / 2^14 half away from zero; a lane counts 8 samples of a cell in
//     4-bit fields, the warp adds them with one redux per three bins.
//  The raw (unrecoded) counts of grid w go to raw[k][d], d = 0 for s and 1 for s2.
constexpr int SP_R = 66;
constexpr int SP_BOX_W = 160;
constexpr int SP_BOX_H = 2 * SP_R + 1;
constexpr int SP_BUF = (SP_BOX_W * SP_BOX_H + 127) / 128 * 128;
constexpr int SP_WARPS = 4;
static_assert(SP_BOX_W >= 2 * SP_R + 1 + 15, "window holds the rounded-down x start");

__device__ __forceinline__ int rnd_q14(int v) { return (v + 8192 - (v < 0 ? 1 : 0)) >> 14; }

__global__ void __launch_bounds__(SP_WARPS * 32) desc_spatial(const __grid_constant__ CUtensorMap tmap,
                                                              const __grid_constant__ Group gr,
                                                              KParams kp, DescribeWs ws,
                                                              FeatPtrs fp) {
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(dsm + SP_WARPS * SP_BUF);
  const int img = blockIdx.y;
  const int H = gr.H[img], W = gr.W[img];
  const int row0 = gr.mrow[img];   // the image's first row in the stacked MIM
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkp = fp.counts[img][0];
  const int gw = blockIdx.x * SP_WARPS + warp, gstride = gridDim.x * SP_WARPS;
  if (gw >= nkp) return;   // warp-uniform
  unsigned char* buf = dsm + warp * SP_BUF;
  const unsigned bar = smem_u32(&bars[warp]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int* kxy = fp.kp_xy[img];
  const unsigned FULL = 0xffffffffu;
  unsigned phase = 0;
  for (int k = gw; k < nkp; k += gstride, phase ^= 1u) {
    const int x = kxy[2 * k], y = kxy[2 * k + 1];
    const int wx0 = (x - SP_R) & ~15, wy0 = y - SP_R;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(SP_BOX_W * SP_BOX_H)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(buf)),
          "l"(&tmap), "r"(wx0), "r"(row0 + wy0), "r"(bar)
          : "memory");
    }
    if (!mbar_wait(bar, phase, ws.wait_iters)) {
      if (lane == 0) atomicExch(ws.status, ST_TIMEOUT);
      mbar_wait(bar, phase, kWaitIters);   // the copy lands before the kernel exits
      return;
    }
    // ---- 1. disc histogram and centroid sums (rows dy = -48..48, segments of 16 columns)
    int cnt[NO], sx[NO], sy[NO];
#pragma unroll
    for (int b = 0; b < NO; ++b) cnt[b] = sx[b] = sy[b] = 0;
    const int xoff = x - wx0;   // window column of the keypoint
    for (int u = lane; u < 97 * (SP_BOX_W / 16); u += 32) {
      const int ri = u / (SP_BOX_W / 16), sk = u - ri * (SP_BOX_W / 16);
      const int dy = ri - HALF_PATCH;
      if ((unsigned)(y + dy) >= (unsigned)H) continue;
      const int r2 = HALF_PATCH * HALF_PATCH - dy * dy;
      int rr = (int)sqrtf((float)r2);
      while ((rr + 1) * (rr + 1) <= r2) ++rr;
      while (rr * rr > r2) --rr;
      const int lo = max(-rr, -x), hi = min(rr, W - 1 - x);
      const int off = xoff - 16 * sk;          // pixel j of the segment is dx = j - off
      const int jl = max(lo + off, 0), jh = min(hi + off, 15);
      if (jl > jh) continue;
      const uint4 v4 = *reinterpret_cast<const uint4*>(buf + (dy + SP_R) * SP_BOX_W + 16 * sk);
      const unsigned wv[4] = {v4.x, v4.y, v4.z, v4.w};
      unsigned p0 = 0, p1 = 0, p2 = 0, pv = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned idx = 0x03020100u + 0x04040404u * (unsigned)i;
        const unsigned val = __vcmpgeu4(idx, 0x01010101u * (unsigned)jl) &
                             __vcmpleu4(idx, 0x01010101u * (unsigned)jh) & 0x01010101u;
        p0 |= (wv[i] & 0x01010101u) << i;
        p1 |= ((wv[i] >> 1) & 0x01010101u) << i;
        p2 |= ((wv[i] >> 2) & 0x01010101u) << i;
        pv |= val << i;
      }
      // bit 8 j + i holds pixel 4 i + j: pixel-index bit b is set on these masks
      const unsigned m[NO] = {~p2 & ~p1 & ~p0 & pv, ~p2 & ~p1 & p0 & pv, ~p2 & p1 & ~p0 & pv,
                              ~p2 & p1 & p0 & pv,   p2 & ~p0 & pv,        p2 & p0 & pv};
#pragma unroll
      for (int b = 0; b < NO; ++b) {
        const int n = __popc(m[b]);
        const int sj = __popc(m[b] & 0x0F000F00u) + 2 * __popc(m[b] & 0x0F0F0000u) +
                       4 * __popc(m[b] & 0x0A0A0A0Au) + 8 * __popc(m[b] & 0x0C0C0C0Cu);
        cnt[b] += n;
        sx[b] += sj - off * n;
        sy[b] += dy * n;
      }
    }
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      cnt[b] = __reduce_add_sync(FULL, cnt[b]);
      sx[b] = __reduce_add_sync(FULL, sx[b]);
      sy[b] = __reduce_add_sync(FULL, sy[b]);
    }
    // ---- 2. dominant and secondary index (lowest bin on ties), ratio test in integers
    int s = 0;
#pragma unroll
    for (int b = 1; b < NO; ++b)
      if (cnt[b] > cnt[s]) s = b;
    int s2 = (s == 0) ? 1 : 0;
#pragma unroll
    for (int b = 0; b < NO; ++b)
      if (b != s && cnt[b] > cnt[s2]) s2 = b;
    const bool has2 = 1000ll * cnt[s2] >= (long long)kp.ratio_pm * cnt[s];
    if (lane == 0)
      ws.info[(size_t)img * kp.kp_cap + k] = (unsigned)s | ((unsigned)s2 << 4) | ((has2 ? 1u : 0u) << 8);
    // ---- 3. the rotated grids
    const bool interior = x >= SP_R && y >= SP_R && x + SP_R < W && y + SP_R < H;
    unsigned short* raw = ws.raw + ((size_t)img * kp.kp_cap + k) * (2 * DESC_DIM);
    for (int d = 0; d < (has2 ? 2 : 1); ++d) {
      const int wi = d ? s2 : s;
      int sxw = 0, syw = 0, c = 0, sn = 0;   // static indices only (no local copies)
#pragma unroll
      for (int b = 0; b < NO; ++b)
        if (b == wi) { sxw = sx[b]; syw = sy[b]; c = kp.rot_c[b]; sn = kp.rot_s[b]; }
      if ((long long)sxw * c - (long long)syw * sn < 0) { c = -c; sn = -sn; }
      const int dx = -HALF_PATCH + (lane & 15);
      const int dyl = -HALF_PATCH + (lane >> 4);
      for (int cl = 0; cl < CELLS * CELLS; ++cl) {
        const int ci = cl / CELLS, cj = cl - ci * CELLS;
        const int ddx = dx + CELL * cj, ddy = dyl + CELL * ci;
        int X = c * ddx + sn * ddy, Y = -sn * ddx + c * ddy;
        unsigned acc = 0;
#pragma unroll
        for (int r = 0; r < CELL / 2; ++r) {
          const int rx = rnd_q14(X), ry = rnd_q14(Y);
          const bool ok = interior || ((unsigned)(x + rx) < (unsigned)W &&
                                       (unsigned)(y + ry) < (unsigned)H);
          if (ok) {
            const unsigned mv = buf[(ry + SP_R) * SP_BOX_W + xoff + rx];
            acc += 1u << (4 * mv);
          }
          X += 2 * sn;
          Y += 2 * c;
        }
        // nibbles of bins 0..2 and 3..5 into 10-bit fields, summed over the warp
        const unsigned e0 = (acc & 0xFu) | (((acc >> 4) & 0xFu) << 10) | (((acc >> 8) & 0xFu) << 20);
        const unsigned e1 = ((acc >> 12) & 0xFu) | (((acc >> 16) & 0xFu) << 10) |
                            (((acc >> 20) & 0xFu) << 20);
        const unsigned t0 = __reduce_add_sync(FULL, e0), t1 = __reduce_add_sync(FULL, e1);
        if (lane < NO) {
          const unsigned t = lane < 3 ? t0 : t1;
          raw[d * DESC_DIM + cl * NO + lane] = (unsigned short)((t >> (10 * (lane % 3))) & 1023u);
        }
      }
    }
    __syncwarp();   // every lane's reads of the window precede the next copy into it
  }
}

// Descriptors of keypoint info `inf` under the mode: count, and the recoding shift of each.
__device__ __forceinline__ int desc_shifts(unsigned inf, int mode, int (&sh)[NO]) {
  if (mode == DESC_RIFT_RING) {
#pragma unroll
    for (int w = 0; w < NO; ++w) sh[w] = w;
    return NO;
  }
  if (mode == DESC_RIFT_TEMPLATE) {
    sh[0] = 0;
    return 1;
  }
  sh[0] = (int)((inf & 15u) % NO);
  sh[1] = (int)(((inf >> 4) & 15u) % NO);
  return 1 + (int)((inf >> 8) & 1u);
}

__global__ void __launch_bounds__(1024) desc_scan(KParams kp, DescribeWs ws, FeatPtrs fp) {
  __shared__ int wsum[32];
  const int img = blockIdx.x;
  const int nkp = fp.counts[img][0];
  const int per = (nkp + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  const unsigned* info = ws.info + (size_t)img * kp.kp_cap;
  int local = 0;
  for (int i = 0; i < per; ++i) {
    int kk = beg + i;
    if (kk < nkp) {
      int sh[NO];
      local += desc_shifts(info[kk], kp.desc_mode, sh);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    int yv = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += yv;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
    int inc = v;
    for (int d = 1; d < 32; d <<= 1) {
      int yv = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += yv;
    }
    wsum[lane] = inc - v;
  }
  __syncthreads();
  int run = wsum[warp] + incl - local;
  int* off = ws.off + (size_t)img * kp.kp_cap;
  for (int i = 0; i < per; ++i) {
    int kk = beg + i;
    if (kk >= nkp) break;
    int sh[NO];
    const int nd = desc_shifts(info[kk], kp.desc_mode, sh);
    off[kk] = run;
    for (int d = 0; d < nd; ++d) {
      fp.desc_kp[img][run] = kk;
      fp.desc_dom[img][run] = (unsigned char)sh[d];
      ++run;
    }
  }
  if (threadIdx.x == blockDim.x - 1) fp.counts[img][1] = run;
  if (nkp == 0 && threadIdx.x == 0) fp.counts[img][1] = 0;
}

__global__ void __launch_bounds__(256) desc_write(KParams kp, DescribeWs ws, FeatPtrs fp) {
  const int img = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + warp;
  if (k >= fp.counts[img][0]) return;
  int sh[NO];
  const int nd = desc_shifts(ws.info[(size_t)img * kp.kp_cap + k], kp.desc_mode, sh);
  const int off = ws.off[(size_t)img * kp.kp_cap + k];
  unsigned short* d0 = fp.desc[img] + (size_t)off * DESC_DIM;
  if (kp.desc_mode == DESC_SPATIAL) {
    // one raw count vector per descriptor (each from its own rotated grid), recoded by its
    // index; its own norm
    const unsigned short* rk = ws.raw + ((size_t)img * kp.kp_cap + k) * (2 * DESC_DIM);
    for (int d = 0; d < nd; ++d) {
      unsigned n2 = 0;
      for (int e = lane; e < DESC_DIM; e += 32) {
        const unsigned v = rk[d * DESC_DIM + e];
        n2 += v * v;
        const int c = e / NO, b = e - c * NO;
        d0[(size_t)d * DESC_DIM + c * NO + (b - sh[d] + NO) % NO] = (unsigned short)v;
      }
      for (int dd = 16; dd > 0; dd >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, dd);
      if (lane == 0) fp.desc_norm[img][off + d] = sqrtf((float)n2);
    }
    return;
  }
  const unsigned short* raw = ws.raw + ((size_t)img * kp.kp_cap + k) * DESC_DIM;
  unsigned n2 = 0;
  for (int e = lane; e < DESC_DIM; e += 32) {
    const unsigned v = raw[e];
    n2 += v * v;
    const int c = e / NO, b = e - c * NO;
    for (int d = 0; d < nd; ++d) d0[(size_t)d * DESC_DIM + c * NO + (b - sh[d] + NO) % NO] = (unsigned short)v;
  }
  for (int d = 16; d > 0; d >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, d);
  if (lane < nd) fp.desc_norm[img][off + lane] = sqrtf((float)n2);   // exact: n2 < 2^24
}

void describe_box(int desc_mode, int* cols, int* rows) {
  if (desc_mode == DESC_SPATIAL) {
    *cols = SP_BOX_W;
    *rows = SP_BOX_H;
  } else {
    *cols = BOX_W;
    *rows = HALF_ROWS;
  }
}

cudaError_t launch_describe(const CUtensorMap* mim_map, const Group& gr, const KParams& kp,
                            DescribeWs ws, const FeatPtrs& fp, cudaStream_t st) {
  const int nimg = gr.n;
  if (kp.desc_mode == DESC_SPATIAL) {
    const size_t sm = (size_t)SP_WARPS * SP_BUF + SP_WARPS * sizeof(unsigned long long);
    cudaFuncSetAttribute(desc_spatial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int blocks = (kp.kp_cap + SP_WARPS * DH_KPW - 1) / (SP_WARPS * DH_KPW);
    desc_spatial<<<dim3(blocks, nimg), SP_WARPS * 32, sm, st>>>(*mim_map, gr, kp, ws, fp);
  } else {
    const size_t sm = (size_t)DH_WARPS * 2 * HBUF + DH_WARPS * 2 * sizeof(unsigned long long);
    cudaFuncSetAttribute(desc_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int blocks = (kp.kp_cap + DH_WARPS * DH_KPW - 1) / (DH_WARPS * DH_KPW);
    desc_hist<<<dim3(blocks, nimg), DH_WARPS * 32, sm, st>>>(*mim_map, gr, kp, ws, fp);
  }
  desc_scan<<<nimg, 1024, 0, st>>>(kp, ws, fp);
  desc_write<<<dim3((kp.kp_cap + 7) / 8, nimg), 256, 0, st>>>(kp, ws, fp);
  return cudaGetLastError();
}

}  // namespace rift2
