// Feature description (§II-B: 6x6 grid of No-bin MIM histograms; §III: dominant index
// s = argmax of the patch histogram, Eq. 1, recoding MIM_n = (MIM - s) mod No, Eq. 2,
// and a second descriptor when the second-highest bin is within the dominant ratio of
// the peak).
//
//   desc_hist  : one warp per keypoint.  The 96x96 MIM patch (rows y-48..y+47, columns
//                x-48..x+47) is staged into shared memory by a TMA tensor copy whose x
//                start is rounded down to 16 bytes (a 112-byte wide box); each lane
//                counts 16-byte cell rows with byte-wise compares (__vcmpeq4 + popc) and
//                the cell totals are reduced over the 16 lanes of a half-warp.  Writes the
//                unrecoded cell counts, s, s2 and the second-descriptor flag.
//   desc_scan  : one CTA per image: exclusive scan of descriptors per keypoint (1 or 2;
//                for RIFT's baseline modes 1 from the unshifted MIM, or the No members of
//                the convolution-sequence ring, §II-C).
//   desc_write : one warp per keypoint: the recoded count vectors (a cyclic shift of the
//                bins of every cell) and their L2 norms.
#include "kernels.h"

namespace rift2 {

constexpr int BOX_W = PATCH + 16;                 // 112 bytes: x start rounded down to 16
constexpr int WARP_BUF = BOX_W * PATCH + 128;     // + slack for the 4-byte realignment reads
constexpr int DH_WARPS = 8;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

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

__global__ void __launch_bounds__(DH_WARPS * 32) desc_hist(const __grid_constant__ CUtensorMap tmap,
                                                           int H, int W, KParams kp,
                                                           DescribeWs ws, FeatPtrs fp) {
  // [DH_WARPS patch buffers][DH_WARPS mbarriers]; no static shared memory, so the dynamic
  // block starts at the (16-byte aligned) base the TMA destination needs.
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(dsm + DH_WARPS * WARP_BUF);
  const int img = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * DH_WARPS + warp;
  const int nkp = fp.counts[img][0];
  if (k >= nkp) return;   // warp-uniform
  const int x = fp.kp_xy[img][2 * k], y = fp.kp_xy[img][2 * k + 1];
  const int px = x - HALF_PATCH;          // first patch column
  const int x0 = px & ~15;                // TMA x start: 16-byte aligned (u8 elements)
  const int sh = px - x0;
  unsigned char* buf = dsm + warp * WARP_BUF;
  const unsigned bar = smem_u32(&bars[warp]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  if (lane == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(BOX_W * PATCH)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(buf)),
        "l"(&tmap), "r"(x0), "r"(y - HALF_PATCH), "r"(img), "r"(bar)
        : "memory");
  }
  if (!mbar_wait(bar, 0, 1ll << 24)) {
    if (lane == 0) atomicExch(ws.status, ST_TIMEOUT);
    mbar_wait(bar, 0, 1ll << 24);   // the copy may still land: give it a bounded chance
    return;
  }
  const int rho = lane & 15, half = lane >> 4;
  unsigned whole[NO] = {0, 0, 0, 0, 0, 0};
  unsigned short* raw = ws.raw + ((size_t)img * kp.max_kp + k) * DESC_DIM;
#pragma unroll 2
  for (int m = 0; m < CELLS * CELLS / 2; ++m) {
    const int c = 2 * m + half;
    const int ci = c / CELLS, cj = c % CELLS;
    const int s0 = (ci * CELL + rho) * BOX_W + sh + cj * CELL;
    const unsigned* wp = reinterpret_cast<const unsigned*>(buf + (s0 & ~3));
    const int a8 = (s0 & 3) * 8;
    unsigned w[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) w[i] = wp[i];
    // bins 0..No-2 by byte-wise compares; the last bin is what remains of the 16 pixels
    // (MIM values are 0..No-1)
    unsigned cnt[NO] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      unsigned v = __funnelshift_r(w[i], w[i + 1], a8);
#pragma unroll
      for (int b = 0; b < NO - 1; ++b) cnt[b] += __popc(__vcmpeq4(v, 0x01010101u * b));
    }
    unsigned rest = 16;
#pragma unroll
    for (int b = 0; b < NO - 1; ++b) {
      cnt[b] >>= 3;   // 8 bits per matching byte
      rest -= cnt[b];
    }
    cnt[NO - 1] = rest;
    // pack two bins per word (cell totals <= 256)
    unsigned p0 = cnt[0] | (cnt[1] << 16);
    unsigned p1 = cnt[2] | (cnt[3] << 16);
    unsigned p2 = cnt[4] | (cnt[5] << 16);
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      p0 += __shfl_xor_sync(0xffffffffu, p0, d);
      p1 += __shfl_xor_sync(0xffffffffu, p1, d);
      p2 += __shfl_xor_sync(0xffffffffu, p2, d);
    }
    unsigned tot[NO] = {p0 & 0xFFFFu, p0 >> 16, p1 & 0xFFFFu, p1 >> 16, p2 & 0xFFFFu, p2 >> 16};
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      whole[b] += tot[b];
      if (rho == b) raw[c * NO + b] = (unsigned short)tot[b];
    }
  }
#pragma unroll
  for (int b = 0; b < NO; ++b) whole[b] += __shfl_xor_sync(0xffffffffu, whole[b], 16);
  if (lane == 0) {
    int s = 0;
    for (int b = 1; b < NO; ++b)
      if (whole[b] > whole[s]) s = b;
    int s2 = (s == 0) ? 1 : 0;
    for (int b = 0; b < NO; ++b)
      if (b != s && whole[b] > whole[s2]) s2 = b;
    unsigned has2 = (1000u * whole[s2] >= (unsigned)kp.ratio_pm * whole[s]) ? 1u : 0u;
    ws.info[(size_t)img * kp.max_kp + k] = (unsigned)s | ((unsigned)s2 << 4) | (has2 << 8);
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
  sh[0] = inf & 15u;
  sh[1] = (inf >> 4) & 15u;
  return 1 + (int)((inf >> 8) & 1u);
}

__global__ void __launch_bounds__(1024) desc_scan(KParams kp, DescribeWs ws, FeatPtrs fp) {
  __shared__ int wsum[32];
  const int img = blockIdx.x;
  const int nkp = fp.counts[img][0];
  const int per = (nkp + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  const unsigned* info = ws.info + (size_t)img * kp.max_kp;
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
  int* off = ws.off + (size_t)img * kp.max_kp;
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
  const int nd = desc_shifts(ws.info[(size_t)img * kp.max_kp + k], kp.desc_mode, sh);
  const int off = ws.off[(size_t)img * kp.max_kp + k];
  const unsigned short* raw = ws.raw + ((size_t)img * kp.max_kp + k) * DESC_DIM;
  unsigned short* d0 = fp.desc[img] + (size_t)off * DESC_DIM;
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

cudaError_t launch_describe(const CUtensorMap* mim_map, int nimg, int H, int W,
                            const KParams& kp, DescribeWs ws, const FeatPtrs& fp,
                            cudaStream_t st) {
  size_t sm = (size_t)DH_WARPS * WARP_BUF + DH_WARPS * sizeof(unsigned long long);
  cudaFuncSetAttribute(desc_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int blocks = (kp.max_kp + DH_WARPS - 1) / DH_WARPS;
  desc_hist<<<dim3(blocks, nimg), DH_WARPS * 32, sm, st>>>(*mim_map, H, W, kp, ws, fp);
  desc_scan<<<nimg, 1024, 0, st>>>(kp, ws, fp);
  desc_write<<<dim3((kp.max_kp + 7) / 8, nimg), 256, 0, st>>>(kp, ws, fp);
  return cudaGetLastError();
}

}  // namespace rift2
