// Brute-force nearest-neighbour matching on the tcgen05 tensor cores (§IV: nearest
// feature distance over all descriptor pairs).  The only dense contraction of the path.
//
//   nn_prep   : descriptor counts -> BF16 rows padded to K = 256 (counts <= 256 are exact
//               in BF16), exact squared norms, 1/|b| for the screening scores.
//   nn_tc     : per CTA 128 queries x a range of 256-wide tiles of B.  One thread issues
//               TMA loads (128-byte swizzle, three 32 KB K-atom slots in flight), one issues
//               tcgen05.mma (BF16 x BF16 -> FP32 in TMEM, M = 128, N = 256, 14 K-steps of 16
//               cover K = 216) into two accumulators of 256 TMEM columns (all 512), so the
//               next tile's MMAs overlap the epilogue of this one; eight epilogue warps (two
//               per TMEM lane quadrant, one 128-column half each) read the accumulators with
//               tcgen05.ld and keep each query's 4 best candidates per half by the FP32
//               score dot / |b|, screening 32 columns at a time against the larger of the two
//               halves' 4th-best scores.  No score matrix ever reaches HBM.
//   nn_rerank : one thread per query: the exact comparison of match_common.cuh over its
//               candidates, distances and near-tie flags, and the certification that no
//               screened-out column can enter the top two (else the query is listed).
//   nn_exact  : the listed queries against all of B with exact integer dots.
// The products and partial sums of integer counts stay below 2^24, so every FP32 addition
// in the tensor-core accumulation is exact: the accumulators hold the exact integer dot
// products, which the epilogue stores with each candidate for the re-rank.
#include <cuda_bf16.h>

#include "kernels.h"
#include "match_common.cuh"

namespace rift2 {

constexpr int TC_BM = 128, TC_BN = 256, TC_KP = 256, TC_KATOM = 64, TC_NATOM = 4;
constexpr int TC_KSTEPS = 14;                             // 14 x 16 = 224 >= 216
constexpr int TC_A_ATOM = TC_BM * 128;                    // 128 rows x 128 bytes = 16 KB
constexpr int TC_B_ATOM = TC_BN * 128;                    // 32 KB: one K-atom of a B tile
constexpr int TC_A_BYTES = TC_NATOM * TC_A_ATOM;          // 64 KB
constexpr int TC_SLOTS = 3;                               // B K-atoms in flight
constexpr int TC_ACC = 2;                                 // accumulators in TMEM
constexpr int TC_TOPK = 4;
constexpr int TC_EPI_WARPS = 8;                           // two per TMEM lane quadrant
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;        // warp 0 TMA, warp 1 MMA, epilogue
constexpr int TC_HALVES = TC_EPI_WARPS / 4;               // column slices per quadrant
constexpr int TC_SLICE = TC_BN / TC_HALVES;               // 128 columns per epilogue warp
constexpr int TC_TMEM_COLS = TC_ACC * TC_BN;              // 512: all of TMEM
constexpr long long TC_WAIT = 1ll << 26;                  // bounded mbarrier polls
constexpr int TC_NBARS = 1 + 2 * TC_SLOTS + 3 * TC_ACC;
// per epilogue warp: 32 lanes x 32 accumulator values, the chunk a lane is screening
constexpr int TC_STAGE_FLOATS = TC_EPI_WARPS * 32 * 32;
constexpr size_t TC_SMEM = 1024 + TC_A_BYTES + TC_SLOTS * TC_B_ATOM + 256 +
                           (TC_ACC * TC_BN + TC_HALVES * TC_BM + TC_STAGE_FLOATS) * sizeof(float);
static_assert(TC_HALVES == 2, "threshold sharing pairs the two column halves of a row");
static_assert(TC_NBARS * 8 + 8 <= 256, "barrier block");
static_assert(TC_SMEM <= 232448, "shared memory");

// --------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < TC_WAIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand stored with the 128-byte swizzle:
// start address >> 4, leading offset unused (1), stride between 8-row groups 1024 B,
// descriptor version 1, layout SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N and M.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane, without the wait
// (several loads share one tcgen05.wait::ld).
__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// Largest of 32 values with three-input maxima (17 instructions).
__device__ __forceinline__ float max32(const float (&v)[32]) {
  float a[11];
#pragma unroll
  for (int k = 0; k < 10; ++k) a[k] = max3f(v[3 * k], v[3 * k + 1], v[3 * k + 2]);
  a[10] = fmaxf(v[30], v[31]);
  const float b0 = max3f(a[0], a[1], a[2]), b1 = max3f(a[3], a[4], a[5]);
  const float b2 = max3f(a[6], a[7], a[8]), b3 = fmaxf(a[9], a[10]);
  return fmaxf(max3f(b0, b1, b2), b3);
}
// Two IEEE round-to-nearest products in one packed instruction.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  const unsigned long long x = ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
  const unsigned long long y = ((unsigned long long)__float_as_uint(b.y) << 32) | __float_as_uint(b.x);
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  return make_float2(__uint_as_float((unsigned)d), __uint_as_float((unsigned)(d >> 32)));
}

// --------------------------------------------------------------------------- prep
// grid (rows / 8, 2 sides, pairs); warp per descriptor row.
__global__ void __launch_bounds__(256) nn_prep(MatchPtrs mp, __nv_bfloat16* __restrict__ abf,
                                               __nv_bfloat16* __restrict__ bbf,
                                               float* __restrict__ rinv_b,
                                               int* __restrict__ n2_a, int* __restrict__ n2_b,
                                               int cap, int* __restrict__ n_unsure) {
  const int pr = blockIdx.z, side = blockIdx.y;
  if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *n_unsure = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  const int n = side ? mp.counts_b[pr][1] : mp.counts_a[pr][1];
  if (row >= n) return;
  const unsigned short* src = (side ? mp.desc_b[pr] : mp.desc_a[pr]) + (size_t)row * DESC_DIM;
  __nv_bfloat16* dst = (side ? bbf : abf) + ((size_t)pr * cap + row) * TC_KP;
  unsigned n2 = 0;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = lane * 8 + i;
    const unsigned c = (k < DESC_DIM) ? src[k] : 0u;
    n2 += c * c;
    v[i] = __float2bfloat16_rn((float)c);   // counts <= 256: exact
  }
  *reinterpret_cast<uint4*>(dst + lane * 8) = *reinterpret_cast<const uint4*>(v);
  for (int d = 16; d > 0; d >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, d);
  if (lane == 0) {
    if (side) {
      n2_b[(size_t)pr * cap + row] = (int)n2;
      rinv_b[(size_t)pr * cap + row] = 1.f / sqrtf((float)n2);
    } else {
      n2_a[(size_t)pr * cap + row] = (int)n2;
    }
  }
}

// ------------------------------------------------------------------------- GEMM
struct TcArgs {
  const int* counts_a[MAXB];
  const int* counts_b[MAXB];
  const float* rinv_b;   // [pairs][cap]
  int2* cand;            // [pairs][nsplit * TC_HALVES][cap][TOPK] (index, dot bits)
  int cap, nsplit;
  int* status;
};

__global__ void __launch_bounds__(TC_THREADS, 1) nn_tc(const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB,
                                                       TcArgs args) {
  extern __shared__ unsigned char tsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pr = blockIdx.z, split = blockIdx.y;
  const int m0 = blockIdx.x * TC_BM;
  const int nA = *args.counts_a[pr], nB = *args.counts_b[pr];
  if (m0 >= nA) return;   // uniform: before any barrier, TMEM or TMA work
  const int ntiles = (nB + TC_BN - 1) / TC_BN;
  const int t0 = (int)((long long)split * ntiles / args.nsplit);
  const int t1 = (int)((long long)(split + 1) * ntiles / args.nsplit);
  const int nt = t1 - t0;

  // 1024-byte aligned: A | B K-atom slots | barriers, TMEM slot, flag (256 B) | 1/|b| slots
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tsm) + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  unsigned char* sB = base + TC_A_BYTES;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(sB + TC_SLOTS * TC_B_ATOM);
  const uint32_t full_a = su32(&bars[0]);
  const uint32_t full0 = su32(&bars[1]);             // B slot filled
  const uint32_t empty0 = full0 + 8 * TC_SLOTS;      // B slot read by its MMAs
  const uint32_t tfull0 = empty0 + 8 * TC_SLOTS;     // accumulator ready
  const uint32_t tempty0 = tfull0 + 8 * TC_ACC;      // accumulator drained
  const uint32_t rfull0 = tempty0 + 8 * TC_ACC;      // 1/|b| slice staged
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(&bars[TC_NBARS]);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* rinv_s = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(bars) + 256);
  float* thr_s = rinv_s + TC_ACC * TC_BN;          // [half][row]: TC_TOPK-th best score of a list
  float* stage_s = thr_s + TC_HALVES * TC_BM;      // [epilogue warp][lane][32], swizzled
  for (int i = threadIdx.x; i < TC_HALVES * TC_BM; i += TC_THREADS) thr_s[i] = -1.f;

  if (threadIdx.x == 0) {
    mbar_init(full_a, 1);
    for (int i = 0; i < TC_SLOTS; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int i = 0; i < TC_ACC; ++i) {
      mbar_init(tfull0 + 8 * i, 1);
      mbar_init(tempty0 + 8 * i, 32 * TC_EPI_WARPS);
      mbar_init(rfull0 + 8 * i, TC_BN);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(args.status, ST_TIMEOUT);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ TMA producer
      mbar_expect_tx(full_a, TC_A_BYTES);
      for (int a = 0; a < TC_NATOM; ++a)
        tma_load_3d(su32(sA + a * TC_A_ATOM), &tmA, a * TC_KATOM, m0, pr, full_a);
      for (int u = 0; u < nt * TC_NATOM && !*abort_flag; ++u) {
        const int slot = u % TC_SLOTS, a = u % TC_NATOM;
        if (u >= TC_SLOTS && !mbar_wait_bounded(empty0 + 8 * slot, ((u / TC_SLOTS) - 1) & 1)) {
          fail();
          break;
        }
        mbar_expect_tx(full0 + 8 * slot, TC_B_ATOM);
        tma_load_3d(su32(sB + slot * TC_B_ATOM), &tmB, a * TC_KATOM, (t0 + u / TC_NATOM) * TC_BN,
                    pr, full0 + 8 * slot);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = umma_idesc_bf16(TC_BM, TC_BN);
      bool ok = mbar_wait_bounded(full_a, 0);
      if (!ok) fail();
      const uint32_t a0 = su32(sA), b0 = su32(sB);
      for (int i = 0; ok && i < nt && !*abort_flag; ++i) {
        const int acc = i % TC_ACC;
        if (i >= TC_ACC && !mbar_wait_bounded(tempty0 + 8 * acc, ((i / TC_ACC) - 1) & 1)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * TC_BN);
        for (int a = 0; a < TC_NATOM; ++a) {
          const int u = i * TC_NATOM + a, slot = u % TC_SLOTS;
          if (!mbar_wait_bounded(full0 + 8 * slot, (u / TC_SLOTS) & 1)) { ok = false; break; }
          tc_fence_after();
          const int ks_end = (a == TC_NATOM - 1) ? TC_KSTEPS - 4 * a : 4;
          for (int kk = 0; kk < ks_end; ++kk) {
            umma_bf16(d, umma_desc_sw128(a0 + a * TC_A_ATOM + kk * 32),
                      umma_desc_sw128(b0 + slot * TC_B_ATOM + kk * 32), idesc, (a | kk) != 0);
          }
          umma_commit(empty0 + 8 * slot);   // slot free once these MMAs have read it
        }
        if (!ok) { fail(); break; }
        umma_commit(tfull0 + 8 * acc);      // accumulator ready for the epilogue
      }
    }
  } else {
    // ----------------------------------------------------------------- epilogue
    // Warp w reads TMEM lanes 32 (w % 4) .. +31 (the quadrant the hardware lets it access)
    // and one half (TC_SLICE columns) of every accumulator tile.  Each lane keeps the
    // TC_TOPK best candidates of its row within its half.  The two halves of a row publish
    // their TC_TOPK-th best score in shared memory and each screens against the larger of
    // the two: a candidate below the partner's TC_TOPK-th best has TC_TOPK better ones in
    // the partner's half and cannot be among the row's TC_TOPK best, so the union of the
    // two lists still holds them.
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int etid = threadIdx.x - 64;
    const int rl = q * 32 + lane;
    const int row = m0 + rl;
    float sc[TC_TOPK], dt[TC_TOPK];
    int id[TC_TOPK];
#pragma unroll
    for (int k = 0; k < TC_TOPK; ++k) { sc[k] = -1.f; dt[k] = 0.f; id[k] = -1; }
    volatile float* my_thr = thr_s + half * TC_BM + rl;
    const volatile float* pa_thr = thr_s + (half ^ 1) * TC_BM + rl;
    // this lane's row of the staging area: 8 float4 slots, slot k stored at k ^ (lane & 7)
    float4* stg = reinterpret_cast<float4*>(stage_s + ((warp - 2) * 32 + lane) * 32);
    const int swz = lane & 7;
    const float* rinv = args.rinv_b + (size_t)pr * args.cap;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    // 1/|b| of the next tile, prefetched one tile ahead into registers, staged in smem
    float rnext = (nt > 0 && etid < TC_BN) ? __ldg(rinv + t0 * TC_BN + etid) : 0.f;
    for (int i = 0; i < nt; ++i) {
      const int acc = i % TC_ACC;
      bool ok = true;
      if (etid < TC_BN) {
        // slot `acc` was last read for tile i - TC_ACC; every epilogue thread arrived on
        // tempty[acc] for that tile once its reads were done
        if (i >= TC_ACC) ok = mbar_wait_bounded(tempty0 + 8 * acc, ((i / TC_ACC) - 1) & 1);
        rinv_s[acc * TC_BN + etid] = rnext;
        mbar_arrive(rfull0 + 8 * acc);
        if (i + 1 < nt) rnext = __ldg(rinv + (t0 + i + 1) * TC_BN + etid);
      }
      ok = ok && mbar_wait_bounded(rfull0 + 8 * acc, (i / TC_ACC) & 1);
      // warp-uniform decision: tcgen05.ld below is a warp-collective instruction
      const bool ready =
          __all_sync(0xffffffffu, ok && mbar_wait_bounded(tfull0 + 8 * acc, (i / TC_ACC) & 1));
      if (!ready) {
        if (lane == 0) fail();
        break;
      }
      tc_fence_after();
      // two rounds of two 32-column chunks: one tcgen05.wait::ld per round
#pragma unroll 1
      for (int rd = 0; rd < TC_SLICE / 64; ++rd) {
        uint32_t r[2][32];
        const uint32_t cb = (uint32_t)(acc * TC_BN + half * TC_SLICE + rd * 64);
        tmem_ld32_nw(lane_base + cb, r[0]);
        tmem_ld32_nw(lane_base + cb + 32, r[1]);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int j0 = (t0 + i) * TC_BN + half * TC_SLICE + rd * 64 + c * 32;
          const float* rs = rinv_s + acc * TC_BN + half * TC_SLICE + rd * 64 + c * 32;
          float sv[32];
#pragma unroll
          for (int e4 = 0; e4 < 8; ++e4) {
            const float4 rb = *reinterpret_cast<const float4*>(rs + e4 * 4);
            const float2 lo = mul2(make_float2(__uint_as_float(r[c][4 * e4]), __uint_as_float(r[c][4 * e4 + 1])),
                                   make_float2(rb.x, rb.y));
            const float2 hi = mul2(make_float2(__uint_as_float(r[c][4 * e4 + 2]), __uint_as_float(r[c][4 * e4 + 3])),
                                   make_float2(rb.z, rb.w));
            sv[4 * e4] = lo.x; sv[4 * e4 + 1] = lo.y; sv[4 * e4 + 2] = hi.x; sv[4 * e4 + 3] = hi.y;
          }
          float thr = fmaxf(sc[TC_TOPK - 1], *pa_thr);
          if (max32(sv) > thr) {
            // stage this lane's 32 exact dots, then visit only the groups of four whose
            // maximum passes; scores are recomputed with the same rounded product
#pragma unroll
            for (int k = 0; k < 8; ++k)
              stg[k ^ swz] = make_float4(__uint_as_float(r[c][4 * k]), __uint_as_float(r[c][4 * k + 1]),
                                         __uint_as_float(r[c][4 * k + 2]), __uint_as_float(r[c][4 * k + 3]));
            unsigned gm = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
              gm |= (fmaxf(fmaxf(sv[4 * k], sv[4 * k + 1]), fmaxf(sv[4 * k + 2], sv[4 * k + 3])) > thr ? 1u : 0u) << k;
            while (gm) {
              const int k = __ffs(gm) - 1;
              gm &= gm - 1;
              const float4 d4 = stg[k ^ swz];
              const float4 r4 = *reinterpret_cast<const float4*>(rs + 4 * k);
              const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
              const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float s = __fmul_rn(dv[e], rv[e]);
                const int j = j0 + 4 * k + e;
                if (s > thr && j < nB) {
                  sc[TC_TOPK - 1] = s;
                  dt[TC_TOPK - 1] = dv[e];
                  id[TC_TOPK - 1] = j;
#pragma unroll
                  for (int k2 = TC_TOPK - 1; k2 > 0; --k2) {
                    if (sc[k2] > sc[k2 - 1]) {
                      const float ts = sc[k2]; sc[k2] = sc[k2 - 1]; sc[k2 - 1] = ts;
                      const float td = dt[k2]; dt[k2] = dt[k2 - 1]; dt[k2 - 1] = td;
                      const int ti = id[k2]; id[k2] = id[k2 - 1]; id[k2 - 1] = ti;
                    }
                  }
                  thr = fmaxf(sc[TC_TOPK - 1], thr);
                }
              }
            }
            *my_thr = sc[TC_TOPK - 1];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(tempty0 + 8 * acc);
    }
    if (row < nA) {
      int2* out = args.cand +
                  (((size_t)pr * args.nsplit * TC_HALVES + split * TC_HALVES + half) * args.cap + row) *
                      TC_TOPK;
#pragma unroll
      for (int k = 0; k < TC_TOPK; ++k) out[k] = make_int2(id[k], __float_as_int(dt[k]));
    }
  }
  __syncthreads();
  if (warp == 1) {
    if (*abort_flag && nt > 0) {
      // let the last committed MMAs land before the accumulator memory is released
      mbar_wait_bounded(tfull0 + 8 * ((nt - 1) % TC_ACC), ((nt - 1) / TC_ACC) & 1);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------------ re-rank
// One thread per query.  The exact comparison of match_common.cuh over the candidates of
// all its lists gives c1, c2.  The screen is certified afterwards: every column left out
// of a list scored at most that list's last (4th) FP32 score s, and the exact similarity
// dot / |b| of any column is at most its FP32 score times (1 + 3 * 2^-24) (one rounding
// each in sqrt, reciprocal and product; dots and squared norms are exact).  If the
// second-best similarity beats the largest such s by more than a factor 1 + 2^-21, no
// column outside the lists can displace c1 or c2; otherwise the query goes to the
// exhaustive pass below (it needs several columns within FP32 rounding of c2).
__device__ __forceinline__ void write_match(const MatchPtrs& mp, int pr, int q, float na2,
                                            const Cand& c1, const Cand& c2) {
  const bool ok1 = c1.j != 0x7fffffff, ok2 = c2.j != 0x7fffffff;
  const float d1 = ok1 ? exact_dist(na2, c1) : __int_as_float(0x7f800000);
  const float d2 = ok2 ? exact_dist(na2, c2) : __int_as_float(0x7f800000);
  mp.q_desc[pr][q] = q;
  mp.nn_desc[pr][q] = ok1 ? c1.j : -1;
  mp.kp_a[pr][q] = mp.desc_kp_a[pr][q];
  mp.kp_b[pr][q] = ok1 ? mp.desc_kp_b[pr][c1.j] : -1;
  mp.d1[pr][q] = d1;
  mp.d2[pr][q] = d2;
  mp.near_tie[pr][q] = (ok2 && (d2 - d1) < 1e-5f * fmaxf(d1, 1e-12f)) ? 1 : 0;
}

__global__ void __launch_bounds__(256) nn_rerank(MatchPtrs mp, const int2* __restrict__ cand,
                                                 const int* __restrict__ n2_a,
                                                 const int* __restrict__ n2_b,
                                                 const float* __restrict__ rinv_b, int cap,
                                                 int nsplit, int* __restrict__ unsure,
                                                 int* __restrict__ n_unsure) {
  const int pr = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nA = mp.counts_a[pr][1], nB = mp.counts_b[pr][1];
  if (blockIdx.x == 0 && threadIdx.x == 0) *mp.count[pr] = nA;
  if (q >= nA) return;
  const int nl = nsplit * TC_HALVES;
  Cand c1{0.f, 1.f, 0x7fffffff}, c2 = c1;
  float s_cut = -1.f;   // largest last score of a full list
  for (int l = 0; l < nl; ++l) {
    const int4* cl = reinterpret_cast<const int4*>(cand + (((size_t)pr * nl + l) * cap + q) * TC_TOPK);
    int2 e[TC_TOPK];
#pragma unroll
    for (int k = 0; k < TC_TOPK / 2; ++k) {
      const int4 v = __ldg(cl + k);
      e[2 * k] = make_int2(v.x, v.y);
      e[2 * k + 1] = make_int2(v.z, v.w);
    }
    float n2[TC_TOPK];
#pragma unroll
    for (int k = 0; k < TC_TOPK; ++k)
      n2[k] = (e[k].x >= 0 && e[k].x < nB) ? (float)__ldg(n2_b + (size_t)pr * cap + e[k].x) : 0.f;
#pragma unroll
    for (int k = 0; k < TC_TOPK; ++k)
      if (e[k].x >= 0 && e[k].x < nB) push2(c1, c2, Cand{__int_as_float(e[k].y), n2[k], e[k].x});
    const int2 last = e[TC_TOPK - 1];
    if (last.x >= 0 && last.x < nB)
      s_cut = fmaxf(s_cut, __fmul_rn(__int_as_float(last.y), __ldg(rinv_b + (size_t)pr * cap + last.x)));
  }
  if (s_cut >= 0.f) {
    const Cand& w = (c2.j != 0x7fffffff) ? c2 : c1;
    const double bound = (double)s_cut * (1.0 + 1.0 / (double)(1 << 21));
    if (!(w.j != 0x7fffffff && (double)w.dot / sqrt((double)w.n2) > bound)) {
      const int slot = atomicAdd(n_unsure, 1);
      unsure[slot] = pr * cap + q;
      return;
    }
  }
  write_match(mp, pr, q, (float)n2_a[(size_t)pr * cap + q], c1, c2);
}

// Exhaustive exact search for the queries the screen could not certify: one CTA per
// query, integer dots against every descriptor of B, the exact order of match_common.cuh.
constexpr int NN_EXACT_THREADS = 256;
__global__ void __launch_bounds__(NN_EXACT_THREADS) nn_exact(MatchPtrs mp,
                                                             const int* __restrict__ n2_a,
                                                             const int* __restrict__ n2_b,
                                                             int cap,
                                                             const int* __restrict__ unsure,
                                                             const int* __restrict__ n_unsure) {
  __shared__ int qa[DESC_DIM];
  __shared__ Cand best[2 * NN_EXACT_THREADS];
  const int nu = *n_unsure;
  for (int f = blockIdx.x; f < nu; f += gridDim.x) {
    const int pr = unsure[f] / cap, q = unsure[f] % cap;
    const int nB = mp.counts_b[pr][1];
    __syncthreads();   // qa / best of the previous query are no longer read
    for (int k = threadIdx.x; k < DESC_DIM; k += blockDim.x)
      qa[k] = mp.desc_a[pr][(size_t)q * DESC_DIM + k];
    __syncthreads();
    Cand c1{0.f, 1.f, 0x7fffffff}, c2 = c1;
    for (int j = threadIdx.x; j < nB; j += blockDim.x) {
      const unsigned short* bj = mp.desc_b[pr] + (size_t)j * DESC_DIM;
      int dot = 0;
      for (int k = 0; k < DESC_DIM; ++k) dot += qa[k] * (int)bj[k];
      push2(c1, c2, Cand{(float)dot, (float)n2_b[(size_t)pr * cap + j], j});
    }
    best[2 * threadIdx.x] = c1;
    best[2 * threadIdx.x + 1] = c2;
    __syncthreads();
    if (threadIdx.x == 0) {
      Cand b1{0.f, 1.f, 0x7fffffff}, b2 = b1;
      for (int i = 0; i < 2 * NN_EXACT_THREADS; ++i)
        if (best[i].j != 0x7fffffff) push2(b1, b2, best[i]);
      write_match(mp, pr, q, (float)n2_a[(size_t)pr * cap + q], b1, b2);
    }
  }
}

// ---------------------------------------------------------------------- launcher
size_t match_tc_ws_bytes(int npairs, int cap, int nsplit) {
  size_t bf = (size_t)npairs * cap * TC_KP * 2;
  size_t per = (size_t)npairs * cap * 4;
  return 2 * bf + 4 * per + (size_t)npairs * nsplit * TC_HALVES * cap * TC_TOPK * 8 + 4096;
}

int match_tc_nsplit(int npairs, int cap) {
  const int mtiles = (cap + TC_BM - 1) / TC_BM;
  int ns = (2 * 152 + npairs * mtiles - 1) / (npairs * mtiles);
  return ns < 1 ? 1 : (ns > 4 ? 4 : ns);
}

cudaError_t launch_match_tc(const MatchPtrs& mp, int npairs, int cap, void* ws,
                            const CUtensorMap* tmA, const CUtensorMap* tmB, int nsplit,
                            int* status, cudaStream_t st) {
  char* p = static_cast<char*>(ws);
  __nv_bfloat16* abf = reinterpret_cast<__nv_bfloat16*>(p);
  p += (size_t)npairs * cap * TC_KP * 2;
  __nv_bfloat16* bbf = reinterpret_cast<__nv_bfloat16*>(p);
  p += (size_t)npairs * cap * TC_KP * 2;
  float* rinv = reinterpret_cast<float*>(p);
  p += (size_t)npairs * cap * 4;
  int* n2a = reinterpret_cast<int*>(p);
  p += (size_t)npairs * cap * 4;
  int* n2b = reinterpret_cast<int*>(p);
  p += (size_t)npairs * cap * 4;
  int* unsure = reinterpret_cast<int*>(p);
  p += (size_t)npairs * cap * 4;
  int2* cand = reinterpret_cast<int2*>(p);
  p += (size_t)npairs * nsplit * TC_HALVES * cap * TC_TOPK * 8;
  int* n_unsure = reinterpret_cast<int*>(p);
  nn_prep<<<dim3((cap + 7) / 8, 2, npairs), 256, 0, st>>>(mp, abf, bbf, rinv, n2a, n2b, cap, n_unsure);
  TcArgs ta{};
  for (int i = 0; i < npairs; ++i) {
    ta.counts_a[i] = mp.counts_a[i] + 1;
    ta.counts_b[i] = mp.counts_b[i] + 1;
  }
  ta.rinv_b = rinv;
  ta.cand = cand;
  ta.cap = cap;
  ta.nsplit = nsplit;
  ta.status = status;
  const size_t sm = TC_SMEM;
  cudaFuncSetAttribute(nn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  nn_tc<<<dim3((cap + TC_BM - 1) / TC_BM, nsplit, npairs), TC_THREADS, sm, st>>>(*tmA, *tmB, ta);
  nn_rerank<<<dim3((cap + 255) / 256, npairs), 256, 0, st>>>(mp, cand, n2a, n2b, rinv, cap, nsplit,
                                                             unsure, n_unsure);
  nn_exact<<<152, NN_EXACT_THREADS, 0, st>>>(mp, n2a, n2b, cap, unsure, n_unsure);
  return cudaGetLastError();
}

// The BF16 operand arrays [pairs][cap][256] inside the workspace; the A map uses boxes of
// 64 x TC_BM x 1 and the B map boxes of 64 x TC_BN x 1 (128-byte swizzle).
int match_tc_box_rows(int operand) { return operand == 0 ? TC_BM : TC_BN; }
void match_tc_operands(void* ws, int npairs, int cap, void** abf, void** bbf) {
  char* p = static_cast<char*>(ws);
  *abf = p;
  *bbf = p + (size_t)npairs * cap * TC_KP * 2;
}

}  // namespace rift2
