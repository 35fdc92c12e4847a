// Keypoint detection on the maximum-moment map (§II-A: FAST "detects edge features on
// the maximum moment map"; Table 1: FAST threshold 0.001, at most 5000 keypoints).
//
//   fast_nms  : min-max normalisation of M (times one reciprocal of the range per tile;
//               1.5 ulp, far inside the 1e-5 near-tie margin), FAST segment test (a
//               compass-pixel precheck, then >= arc contiguous pixels of
//               the radius-3 Bresenham circle all brighter than p + t or all darker than
//               p - t), sum-of-differences score V, 3x3 non-maximum suppression on
//               (V, -raster index); survivors are appended as 64-bit keys
//               (~bits(V) << 32 | raster index), whose ascending order is (V desc, index asc),
//               and counted in a histogram of their leading 16 bits.
//   topk_select / topk_gather : from that histogram, the digit holding rank K - 1; the keys
//               up to it (the K smallest and the rest of that digit's bucket) compacted by
//               many CTAs when they fit the shared-memory sort.
//   topk_sort : one CTA per image sorts the compacted keys; without a fast selection it
//               keeps the max_keypoints smallest keys itself: radix refinement
//               on 8-bit digits until the boundary bucket fits in shared memory, then a
//               bitonic sort (a power-of-two size up to 16384 keys; any size up to 26624
//               keys with the missing tail treated as +inf; global memory beyond that).
//               The result order is deterministic.
#include "kernels.h"

namespace rift2 {

constexpr int FTX = 64, FTY = 32;   // output tile
constexpr int FH = 4;                // halo: 3 for the circle + 1 for the NMS
constexpr int FSX = FTX + 2 * FH, FSY = FTY + 2 * FH;
constexpr int VSX = FTX + 2, VSY = FTY + 2;   // score map (1-pixel halo)

// The 16-pixel Bresenham circle of radius 3 in cyclic order; compile-time offsets, so the
// unrolled segment test reads the tile at immediate displacements.
__device__ constexpr int kCircleDx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
__device__ constexpr int kCircleDy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

// A run of >= arc cyclically contiguous set bits in the 16-bit circle mask (1 <= arc <= 16).
// acc holds the AND of r >> 0 .. h-1 (bit i set: bits i .. i+h-1 of r all set); doubling h
// and one final shift by arc - h (<= h) extend it to arc.
// ARC > 0: the arc length as a compile-time constant (the loop unrolls into a fixed
// sequence of shifts); ARC = 0 reads it from `arc`.
template <int ARC = 0>
__device__ __forceinline__ bool has_arc(unsigned m16, int arc) {
  if constexpr (ARC > 0) arc = ARC;
  if (__popc(m16) < arc) return false;
  const unsigned r = m16 | (m16 << 16);   // cyclic: any run of length <= 16 appears linearly
  unsigned acc = r;
  int h = 1;
  while (2 * h <= arc) {
    acc &= acc >> h;
    h *= 2;
  }
  if (h < arc) acc &= acc >> (arc - h);
  return acc != 0;
}

template <int ARC>
__global__ void __launch_bounds__(256) fast_nms(const float* __restrict__ moment,
                                                const __grid_constant__ Group gr, KParams kp,
                                                DetectWs ws) {
  __shared__ float mn[FSY][FSX];
  __shared__ float vs[VSY][VSX];
  const int img = blockIdx.z;
  const int H = gr.H[img], W = gr.W[img];
  const int tx0 = blockIdx.x * FTX, ty0 = blockIdx.y * FTY;
  const int ylo = HALF_PATCH, yhi = H - HALF_PATCH, xlo = HALF_PATCH, xhi = W - HALF_PATCH;
  // tiles with no candidate pixel in or next to them do nothing
  if (tx0 - 1 >= xhi || tx0 + FTX + 1 <= xlo || ty0 - 1 >= yhi || ty0 + FTY + 1 <= ylo) return;
  const float lo = __uint_as_float(ws.minmax[2 * img]);
  const float hi = __uint_as_float(ws.minmax[2 * img + 1]);
  if (!(hi > lo)) return;   // constant map: no keypoints
  const float rinv = 1.f / (hi - lo);
  const float* M = moment + gr.poff[img];
  for (int i = threadIdx.x; i < FSX * FSY; i += blockDim.x) {
    int y = ty0 - FH + i / FSX, x = tx0 - FH + i % FSX;
    float v = 0.f;
    if (y >= 0 && y < H && x >= 0 && x < W) v = (__ldg(M + (size_t)y * W + x) - lo) * rinv;
    mn[i / FSX][i % FSX] = v;
  }
  __syncthreads();
  const float t = kp.fast_t;
  for (int i = threadIdx.x; i < VSX * VSY; i += blockDim.x) {
    int ly = i / VSX, lx = i % VSX;
    int y = ty0 - 1 + ly, x = tx0 - 1 + lx;
    float score = 0.f;
    if (y >= ylo && y < yhi && x >= xlo && x < xhi) {
      int sy = ly + FH - 1, sx = lx + FH - 1;
      float p = mn[sy][sx];
      // any run of >= arc contiguous circle pixels holds >= arc / 4 of the compass pixels
      // 0, 4, 8, 12 (every 4 consecutive positions hold one): a pixel without that many
      // brighter or that many darker compass pixels fails the segment test
      int nb = 0, nd = 0;
#pragma unroll
      for (int k = 0; k < 16; k += 4) {
        const float q = mn[sy + kCircleDy[k]][sx + kCircleDx[k]];
        nb += (q > p + t) ? 1 : 0;
        nd += (q < p - t) ? 1 : 0;
      }
      if (max(nb, nd) >= ((ARC > 0 ? ARC : kp.fast_arc) >> 2)) {
        unsigned bright = 0, dark = 0;
        float vb = 0.f, vd = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          float q = mn[sy + kCircleDy[k]][sx + kCircleDx[k]];
          if (q > p + t) { bright |= 1u << k; vb += q - p - t; }
          if (q < p - t) { dark |= 1u << k; vd += p - q - t; }
        }
        if (has_arc<ARC>(bright, kp.fast_arc) || has_arc<ARC>(dark, kp.fast_arc))
          score = fmaxf(vb, vd);
      }
    }
    vs[ly][lx] = score;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < FTX * FTY; i += blockDim.x) {
    int ly = i / FTX + 1, lx = i % FTX + 1;
    float v = vs[ly][lx];
    bool keep = v > 0.f;
    if (keep) {
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          if (dy == 0 && dx == 0) continue;
          float qv = vs[ly + dy][lx + dx];
          if (qv > 0.f) {
            bool q_before = dy < 0 || (dy == 0 && dx < 0);
            bool wins = q_before ? (v > qv) : (v >= qv);
            keep = keep && wins;
          }
        }
    }
    unsigned ballot = __ballot_sync(0xffffffffu, keep);
    if (ballot) {
      int lane = threadIdx.x & 31;
      int leader = __ffs(ballot) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(ws.cand_count + img, (unsigned)__popc(ballot));
      base = __shfl_sync(0xffffffffu, base, leader);
      unsigned dig = 0xFFFFFFFFu;   // top 16 key bits of a stored key, else none
      if (keep) {
        unsigned pos = base + __popc(ballot & ((1u << lane) - 1));
        int y = ty0 + ly - 1, x = tx0 + lx - 1;
        unsigned long long key = ((unsigned long long)(~__float_as_uint(v)) << 32) |
                                 (unsigned)(y * W + x);
        if (pos < (unsigned)ws.cap_cand) {
          ws.cand[(size_t)img * ws.cap_cand + pos] = key;
          dig = (unsigned)(key >> (64 - TOPK_DIGIT_BITS));
        }
      }
      if (ws.cand_hist) {   // histogram of the stored keys' leading digits (warp-aggregated)
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        if (dig != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
          atomicAdd(ws.cand_hist + ((size_t)img << TOPK_DIGIT_BITS) + dig, (unsigned)__popc(peers));
      }
    }
  }
}

constexpr int SORT_CAP = TOPK_SMEM_CAP;

// Ascending bitonic sort of n (a power of two) keys in shared memory; every thread
// iteration performs one compare-exchange (n / 2 per stage).
__device__ void bitonic_sort(unsigned long long* s, int n) {
  const int half = n >> 1;
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int p = threadIdx.x; p < half; p += blockDim.x) {
        const int i = 2 * j * (p / j) + (p % j);
        const int l = i + j;
        const unsigned long long a = s[i], b = s[l];
        const bool up = (i & k) == 0;
        if ((a > b) == up) { s[i] = b; s[l] = a; }
      }
      __syncthreads();
    }
  }
}

// Ascending sort of n keys (any n) in shared memory as a bitonic network over the next
// power of two N >= n, positions >= n standing for +inf keys that are never stored.  Each
// stage k merges with the mirrored comparison (i against i ^ (k - 1)) followed by
// half-cleaners (i against i + j), every comparator ascending; a comparator whose upper
// position is >= n would only confirm that +inf stays on top, so it is skipped.
__device__ void bitonic_sort_any(unsigned long long* s, int n) {
  int N = 1;
  while (N < n) N <<= 1;
  const int half = N >> 1;
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int p = threadIdx.x; p < half; p += blockDim.x) {
        const int i = 2 * j * (p / j) + (p % j);
        const int l = (j == (k >> 1)) ? (i ^ (k - 1)) : (i + j);
        if (l < n) {
          const unsigned long long a = s[i], b = s[l];
          if (a > b) { s[i] = b; s[l] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// The same sort for n = 1024 E keys in shared memory with 1024 threads: warp w owns
// positions w 32E .. +32E-1, lane l the positions w 32E + l + 32 e (e < E).  Compare-exchange
// distances j < 32 run as lane shuffles, 32 <= j < 32E inside a thread's registers, and only
// j >= 32E through shared memory (15 block-wide barriers instead of 91 for n = 8192).
template <int E>
__device__ void bitonic_sort_reg(unsigned long long* s, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int base = warp * 32 * E + lane;
  unsigned long long v[E];
  for (int k = 2; k <= n; k <<= 1) {
    int j = k >> 1;
    for (; j >= 32 * E; j >>= 1) {   // partners in another warp
      for (int p = threadIdx.x; p < (n >> 1); p += blockDim.x) {
        const int i = 2 * j * (p / j) + (p % j);
        const int l = i + j;
        const unsigned long long a = s[i], b = s[l];
        const bool up = (i & k) == 0;
        if ((a > b) == up) { s[i] = b; s[l] = a; }
      }
      __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = s[base + 32 * e];
    for (; j > 0; j >>= 1) {
      if (j >= 32) {   // partner e ^ (j / 32) in this thread (static register indices)
#pragma unroll
        for (int sb = 1; sb < E; sb <<= 1) {
          if ((j >> 5) == sb) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              if ((e & sb) == 0) {
                const bool up = ((base + 32 * e) & k) == 0;
                const unsigned long long a = v[e], b = v[e | sb];
                if ((a > b) == up) { v[e] = b; v[e | sb] = a; }
              }
            }
          }
        }
      } else {         // partner lane ^ j
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pos = base + 32 * e;
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[e], j);
          const bool keep_min = ((pos & j) == 0) == ((pos & k) == 0);
          v[e] = keep_min ? (v[e] < o ? v[e] : o) : (v[e] > o ? v[e] : o);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) s[base + 32 * e] = v[e];
    __syncthreads();
  }
}

// Top-K selection from the leading-digit histogram fast_nms built: one CTA per image finds
// the digit d holding rank K - 1 of the stored keys (or takes every digit when at most
// topk_fast_cap keys are stored).  The keys with digit <= d are exactly the K smallest
// plus the rest of d's bucket; when they fit the sort (below + bucket <= topk_fast_cap) the
// gather kernel compacts them and the sort reads only those, else the sort refines on the
// full candidate list.  sel[img] = {d, below + bucket, fast, gathered count}.
__global__ void __launch_bounds__(1024) topk_select(KParams kp, DetectWs ws) {
  __shared__ unsigned part[1024];
  __shared__ unsigned s_d, s_below, s_found;
  const int img = blockIdx.x;
  const unsigned* h = ws.cand_hist + ((size_t)img << TOPK_DIGIT_BITS);
  unsigned n = ws.cand_count[img];
  if (n > (unsigned)ws.cap_cand) n = ws.cap_cand;
  const unsigned capf = (unsigned)topk_fast_cap(kp.max_kp);
  unsigned* sel = ws.sel + 4 * img;
  if (n <= capf) {   // every stored key fits: no selection
    if (threadIdx.x == 0) {
      sel[0] = (1u << TOPK_DIGIT_BITS) - 1;
      sel[1] = n;
      sel[2] = 1;
      sel[3] = 0;
    }
    return;
  }
  constexpr int PER = (1 << TOPK_DIGIT_BITS) / 1024;
  if (threadIdx.x == 0) s_found = 0;
  unsigned loc = 0;
  for (int i = 0; i < PER; ++i) loc += h[threadIdx.x * PER + i];
  part[threadIdx.x] = loc;
  __syncthreads();
  // inclusive block scan (Hillis-Steele in shared memory)
  for (int d = 1; d < 1024; d <<= 1) {
    const unsigned add = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  const unsigned rank = (unsigned)kp.max_kp - 1;
  const unsigned incl = part[threadIdx.x], excl = incl - loc;
  if (excl <= rank && rank < incl) {   // exactly one thread holds the rank
    unsigned acc = excl;
    int i = 0;
    for (; i < PER - 1; ++i) {
      const unsigned c = h[threadIdx.x * PER + i];
      if (rank < acc + c) break;
      acc += c;
    }
    s_d = threadIdx.x * PER + i;
    s_below = acc;
    s_found = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned d = s_found ? s_d : 0u, tot = s_found ? s_below + h[d] : 0u;
    sel[0] = d;
    sel[1] = tot;
    sel[2] = (s_found && tot <= capf) ? 1u : 0u;
    sel[3] = 0;
  }
}

// Compacts the keys whose leading digit is <= sel.d into ws.comp (fast selections only).
__global__ void __launch_bounds__(256) topk_gather(KParams kp, DetectWs ws) {
  const int img = blockIdx.y;
  unsigned* sel = ws.sel + 4 * img;
  if (!sel[2]) return;
  const unsigned d = sel[0];
  unsigned n = ws.cand_count[img];
  if (n > (unsigned)ws.cap_cand) n = ws.cap_cand;
  const unsigned capf = (unsigned)topk_fast_cap(kp.max_kp);
  const unsigned long long* cand = ws.cand + (size_t)img * ws.cap_cand;
  unsigned long long* comp = ws.comp + (size_t)img * capf;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b0 < n; b0 += stride) {
    const unsigned i = b0 + lane;
    unsigned long long k = 0;
    bool take = false;
    if (i < n) {
      k = cand[i];
      take = (unsigned)(k >> (64 - TOPK_DIGIT_BITS)) <= d;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    unsigned base = 0;
    if (lane == 0 && bal) base = atomicAdd(sel + 3, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) {
      const unsigned pos = base + __popc(bal & ((1u << lane) - 1u));
      if (pos < capf) comp[pos] = k;
    }
  }
}

__global__ void __launch_bounds__(1024) topk_sort(const __grid_constant__ Group gr, KParams kp,
                                                  DetectWs ws, FeatPtrs fp) {
  extern __shared__ unsigned long long skeys[];
  __shared__ unsigned hist[256];
  __shared__ unsigned s_sel[4];
  const int img = blockIdx.x;
  const unsigned W = (unsigned)gr.W[img];
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long* cand = ws.cand + (size_t)img * ws.cap_cand;
  unsigned n = ws.cand_count[img];
  if (n > (unsigned)ws.cap_cand) n = ws.cap_cand;
  const unsigned K = kp.max_kp;
  unsigned kcap = 256;                 // sort size: the smallest power of two >= K
  while (kcap < K) kcap <<= 1;
  // keys live in shared memory (a power-of-two sort of kcap keys, or K above that but
  // within TOPK_SMEM_ANY_CAP: an any-size sort of at most that many keys), or in this
  // image's global sort buffer; the block-wide barriers order the global accesses the
  // same way
  const bool any = kcap > (unsigned)SORT_CAP && K <= (unsigned)TOPK_SMEM_ANY_CAP;
  if (any) kcap = TOPK_SMEM_ANY_CAP;
  unsigned long long* keys =
      (kcap <= (unsigned)SORT_CAP || any) ? skeys : ws.sortbuf + (size_t)img * kcap;
  int pbits = 0;
  unsigned long long prefix = 0;
  unsigned nsel = n;   // keys to gather: those whose top pbits bits are <= prefix
  // a fast selection already compacted the keys to sort (topk_select / topk_gather)
  const bool fast = ws.sel && ws.sel[4 * img + 2];
  if (fast) nsel = ws.sel[4 * img + 1];
  if (!fast && n > kcap) {
    unsigned below = 0, rank = K - 1;
    while (true) {
      for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
      __syncthreads();
      // warp-aggregated: most keys share the leading digits, so lanes with equal digits
      // add their count with one atomic
      // while the prefix lies in the keys' upper words (the score bits), the digits and
      // the prefix test use 32-bit shifts of that word
      const bool hi32 = pbits < 32;
      const unsigned prefix32 = (unsigned)prefix;
      for (unsigned b0 = threadIdx.x & ~31u; b0 < n; b0 += blockDim.x) {
        const unsigned i = b0 + lane;
        unsigned dig = 256u;   // not counted
        if (i < n) {
          const unsigned long long k = cand[i];
          if (hi32) {
            const unsigned h = (unsigned)(k >> 32);
            if (pbits == 0 || (h >> (32 - pbits)) == prefix32) dig = (h >> (24 - pbits)) & 0xFFu;
          } else if ((k >> (64 - pbits)) == prefix) {
            dig = (unsigned)(k >> (56 - pbits)) & 0xFFu;
          }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        if (dig < 256u && lane == __ffs(peers) - 1) atomicAdd(&hist[dig], (unsigned)__popc(peers));
      }
      __syncthreads();
      // the digit holding rank: the first bin whose inclusive count exceeds it (bin 255 if
      // none), found by warp 0 with eight bins per lane and a shuffle scan
      if (threadIdx.x < 32) {
        unsigned c[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) { c[j] = hist[lane * 8 + j]; sum += c[j]; }
        unsigned incl = sum;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const unsigned a = __shfl_up_sync(0xffffffffu, incl, dd);
          if (lane >= (unsigned)dd) incl += a;
        }
        const unsigned over = __ballot_sync(0xffffffffu, rank < incl);
        const unsigned owner = over ? (unsigned)(__ffs(over) - 1) : 31u;
        if (lane == owner) {
          unsigned cum = incl - sum;
          int j = 0;
#pragma unroll
          for (int u = 0; u < 7; ++u) {
            if (j == u && rank >= cum + c[u]) { cum += c[u]; j = u + 1; }
          }
          unsigned hd = c[0];
#pragma unroll
          for (int u = 1; u < 8; ++u) hd = (j == u) ? c[u] : hd;
          s_sel[0] = lane * 8 + j;
          s_sel[1] = cum;
          s_sel[2] = hd;
        }
      }
      __syncthreads();
      unsigned d = s_sel[0], cum = s_sel[1], hd = s_sel[2];
      below += cum;
      rank -= cum;
      prefix = (prefix << 8) | d;
      pbits += 8;
      __syncthreads();
      if (below + hd <= kcap || pbits >= 64) { nsel = below + hd; break; }
    }
  }
  int nsort = 1;
  while (nsort < (int)nsel) nsort <<= 1;
  if (nsort < 2) nsort = 2;
  if (any) nsort = (int)nsel;   // exactly the gathered keys, no padding
  if (threadIdx.x == 0) s_sel[3] = 0;
  for (int i = threadIdx.x; i < nsort; i += blockDim.x) keys[i] = ~0ull;
  __syncthreads();
  if (fast) {
    const unsigned long long* comp = ws.comp + (size_t)img * topk_fast_cap(kp.max_kp);
    for (unsigned i = threadIdx.x; i < nsel; i += blockDim.x) keys[i] = comp[i];
  }
  for (unsigned b0 = threadIdx.x & ~31u; !fast && b0 < n; b0 += blockDim.x) {
    const unsigned i = b0 + lane;
    unsigned long long k = 0;
    bool take = false;
    if (i < n) {
      k = cand[i];
      take = pbits == 0 || (k >> (64 - pbits)) <= prefix;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    unsigned base = 0;
    if (lane == 0 && bal) base = atomicAdd(&s_sel[3], (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) {
      const unsigned pos = base + __popc(bal & ((1u << lane) - 1u));
      if (pos < (unsigned)nsort) keys[pos] = k;
    }
  }
  __syncthreads();
  // keys in shared memory with 2048 .. 8192 of them: the register / shuffle form
  if (keys == skeys && nsort == 2048) bitonic_sort_reg<2>(keys, nsort);
  else if (keys == skeys && nsort == 4096) bitonic_sort_reg<4>(keys, nsort);
  else if (keys == skeys && nsort == 8192) bitonic_sort_reg<8>(keys, nsort);
  else if (any) bitonic_sort_any(keys, nsort);
  else bitonic_sort(keys, nsort);
  unsigned nout = n < K ? n : K;
  int* xy = fp.kp_xy[img];
  float* sc = fp.kp_score[img];
  for (unsigned r = threadIdx.x; r < nout; r += blockDim.x) {
    unsigned long long k = keys[r];
    unsigned idx = (unsigned)k;
    xy[2 * r] = (int)(idx % W);
    xy[2 * r + 1] = (int)(idx / W);
    sc[r] = __uint_as_float(~(unsigned)(k >> 32));
  }
  if (threadIdx.x == 0) {
    fp.counts[img][0] = (int)nout;
    fp.counts[img][1] = 0;
  }
}

__global__ void init_detect(unsigned* minmax, unsigned* ccount, int g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < g) {
    minmax[2 * i] = 0xFFFFFFFFu;
    minmax[2 * i + 1] = 0u;
    ccount[i] = 0u;
  }
}

__global__ void minmax_kernel(const float* __restrict__ m, long long P, unsigned* minmax) {
  const int img = blockIdx.y;
  float lo = 3.0e38f, hi = -3.0e38f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    float v = m[(size_t)img * P + i];
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  for (int d = 16; d > 0; d >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, d));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, d));
  }
  if ((threadIdx.x & 31) == 0) {
    // callers of the stage entry pass non-negative moment maps (M >= eps / 2 > 0)
    atomicMin(minmax + 2 * img, __float_as_uint(fmaxf(lo, 0.f)));
    atomicMax(minmax + 2 * img + 1, __float_as_uint(fmaxf(hi, 0.f)));
  }
}

// Corner keypoints after the edge keypoints (RIFT's corner and edge features, §II-A): one
// CTA per image marks the edge keypoints' pixels in a bitmap, then compacts the corner
// list (already in (score desc, index asc) order) without the marked pixels, block-wide
// scans keeping the order.
__global__ void __launch_bounds__(1024) merge_corners(const __grid_constant__ Group gr, KParams kp,
                                                      FeatPtrs fp,
                                                      const int* __restrict__ cxy,
                                                      const float* __restrict__ csc,
                                                      const int* __restrict__ ccnt,
                                                      unsigned* __restrict__ bits,
                                                      long long bits_stride) {
  __shared__ unsigned wsum[32];
  __shared__ int s_base;
  const int img = blockIdx.x;
  const int H = gr.H[img], W = gr.W[img];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const size_t nw = ((size_t)H * W + 31) / 32;
  unsigned* bm = bits + (size_t)img * bits_stride;
  for (size_t i = threadIdx.x; i < nw; i += blockDim.x) bm[i] = 0u;
  __syncthreads();
  int* xy = fp.kp_xy[img];
  float* sc = fp.kp_score[img];
  const int ne = fp.counts[img][0];
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    const unsigned idx = (unsigned)xy[2 * i + 1] * (unsigned)W + (unsigned)xy[2 * i];
    atomicOr(bm + idx / 32, 1u << (idx % 32));
  }
  if (threadIdx.x == 0) s_base = ne;
  __syncthreads();
  const int nc = ccnt[2 * img];
  const int* cx = cxy + (size_t)img * kp.max_kp * 2;
  const float* cs = csc + (size_t)img * kp.max_kp;
  for (int c0 = 0; c0 < nc; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    int x = 0, y = 0;
    float v = 0.f;
    bool keep = false;
    if (i < nc) {
      x = cx[2 * i];
      y = cx[2 * i + 1];
      v = cs[i];
      const unsigned idx = (unsigned)y * (unsigned)W + (unsigned)x;
      keep = ((bm[idx / 32] >> (idx % 32)) & 1u) == 0u;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = (unsigned)__popc(bal);
    __syncthreads();
    if (warp == 0) {
      const unsigned own = lane < nwarp ? wsum[lane] : 0u;
      unsigned inc = own;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
      }
      wsum[lane] = inc - own;   // exclusive prefix over warps
    }
    __syncthreads();
    const int base = s_base;
    const int pos = base + (int)wsum[warp] + __popc(bal & ((1u << lane) - 1u));
    if (keep) {
      xy[2 * pos] = x;
      xy[2 * pos + 1] = y;
      sc[pos] = v;
    }
    __syncthreads();   // every thread has read s_base
    if (threadIdx.x == blockDim.x - 1) s_base = pos + (keep ? 1 : 0);
    __syncthreads();
  }
  if (threadIdx.x == 0) fp.counts[img][0] = s_base;
}

cudaError_t launch_merge_corners(const Group& gr, const KParams& kp, const FeatPtrs& fp,
                                 const int* cxy, const float* csc, const int* ccnt,
                                 unsigned* bits, long long bits_stride, cudaStream_t st) {
  merge_corners<<<gr.n, 1024, 0, st>>>(gr, kp, fp, cxy, csc, ccnt, bits, bits_stride);
  return cudaGetLastError();
}

void launch_init_detect(unsigned* minmax, unsigned* ccount, int g, cudaStream_t st) {
  init_detect<<<(g + 127) / 128, 128, 0, st>>>(minmax, ccount, g);
}

void launch_minmax(const float* m, int g, long long P, unsigned* minmax, cudaStream_t st) {
  minmax_kernel<<<dim3(256, g), 256, 0, st>>>(m, P, minmax);
}

cudaError_t launch_detect(const float* moment, const Group& gr, const KParams& kp, DetectWs ws,
                          const FeatPtrs& fp, cudaStream_t st) {
  int hmax = 1, wmax = 1;
  for (int i = 0; i < gr.n; ++i) {
    hmax = gr.H[i] > hmax ? gr.H[i] : hmax;
    wmax = gr.W[i] > wmax ? gr.W[i] : wmax;
  }
  dim3 grid((wmax + FTX - 1) / FTX, (hmax + FTY - 1) / FTY, gr.n);
  if (!ws.cand_hist || !ws.sel || !ws.comp || !topk_multi_group(kp.max_kp, gr)) {
    ws.cand_hist = nullptr;   // single-CTA refinement only
    ws.sel = nullptr;
    ws.comp = nullptr;
  } else {
    cudaError_t e = cudaMemsetAsync(ws.cand_hist, 0, ((size_t)gr.n << TOPK_DIGIT_BITS) * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  if (kp.fast_arc == 9) fast_nms<9><<<grid, 256, 0, st>>>(moment, gr, kp, ws);
  else fast_nms<0><<<grid, 256, 0, st>>>(moment, gr, kp, ws);
  if (ws.cand_hist) {
    topk_select<<<gr.n, 1024, 0, st>>>(kp, ws);
    topk_gather<<<dim3(16, gr.n), 256, 0, st>>>(kp, ws);
  }
  const int kc = topk_sort_cap(kp.max_kp);
  const int skeys = kc <= SORT_CAP ? kc : (kp.max_kp <= TOPK_SMEM_ANY_CAP ? TOPK_SMEM_ANY_CAP : 0);
  size_t sm = (size_t)skeys * sizeof(unsigned long long);
  cudaFuncSetAttribute(topk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  topk_sort<<<gr.n, 1024, sm, st>>>(gr, kp, ws, fp);
  return cudaGetLastError();
}

}  // namespace rift2
