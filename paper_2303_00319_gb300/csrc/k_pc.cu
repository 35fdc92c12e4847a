// Noise threshold and phase congruency (§II-A: "one-dimensional phase congruency for
// each orientation of the log-Gabor convolutions", "analyzes the change of moment with
// orientations").  The noise model follows the phase-congruency model RIFT builds on:
// T_o is a fixed multiple of the median smallest-scale amplitude.
//
//   median_hist0/1, median_select0/1 : exact median of |EO_0,o| over the whole image by a
//     two-round radix select on the float bit patterns (16 + 16 bits).  The amplitudes
//     are non-negative, so their bit patterns order like the values.  For an even pixel
//     count the two middle values are selected and averaged.
//   pc_moment : PC_o = q_o max(Er_o - T_o, 0), covariance moments over the orientations,
//     maximum moment M, and the image-wide min / max of M for the FAST normalisation.
#include "kernels.h"

namespace rift2 {

// Digits of the two rounds.  Round 0 counts the upper 16 bits of every pattern (bit 31 is
// 0 for non-negative values, so 32768 buckets) in shared memory with 16-bit counters, two
// buckets per word; a CTA counts at most MED_SLICE values, so no counter can overflow into
// its neighbour.  Round 1 counts the lower 16 bits of only the values whose upper half is
// a middle rank's bucket (a small fraction of the slice: the bucket spans 1/128 of an
// octave) directly in the global histogram of that rank.
constexpr int MED_B0 = 32768;        // round-0 buckets
constexpr int MED_B1 = 65536;        // round-1 buckets per middle rank
constexpr int MED_SLICE = 65532;     // values per round-0 CTA (a multiple of 4, < 2^16)
// After the buckets: the counts of 512 equal chunks of the round-0 buckets, then of each
// round-1 histogram, kept beside the buckets so that a selection reads the chunk counts
// and one chunk instead of every bucket.
constexpr int MED_CH0 = MED_B0 + 2 * MED_B1;   // 512 chunk counts of round 0
constexpr int MED_CH1 = MED_CH0 + 512;          // 2 x 512 chunk counts of round 1
static_assert(MED_CH1 + 1024 == MEDIAN_HIST_WORDS, "median histogram layout");

// Streams this CTA's slice of (image, orientation) plane `src` of P values and calls
// one(bits) per value: 16-byte loads when the slice is 16-byte aligned (P % 4 == 0),
// scalar otherwise; four loads per thread in flight before their values are counted.
template <class F>
__device__ __forceinline__ void med_stream(const float* __restrict__ src, long long beg,
                                           long long end, long long P, F&& one) {
  if ((P & 3) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const long long e4 = end / 4;
    long long i = beg / 4 + threadIdx.x;
    for (; i + 3 * (long long)blockDim.x < e4; i += 4 * (long long)blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(s4 + i + u * (long long)blockDim.x);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        one(__float_as_uint(v[u].x));
        one(__float_as_uint(v[u].y));
        one(__float_as_uint(v[u].z));
        one(__float_as_uint(v[u].w));
      }
    }
    for (; i < e4; i += blockDim.x) {
      const float4 v = __ldg(s4 + i);
      one(__float_as_uint(v.x));
      one(__float_as_uint(v.y));
      one(__float_as_uint(v.z));
      one(__float_as_uint(v.w));
    }
  } else {
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) one(__float_as_uint(__ldg(src + i)));
  }
}

__device__ __forceinline__ void med_slice(const Group& gr, int img, long long& beg, long long& end) {
  const long long P = gr.P(img);
  const long long chunk = ((P + gridDim.x - 1) / gridDim.x + 3) & ~3ll;
  beg = blockIdx.x * chunk;
  end = min(P, beg + chunk);
}

// The bin of `hist` holding rank r (0-based, counting from bin 0) and r minus the count of
// the bins before it, into res[0], res[1].  A block of 512 threads, thread t holding the
// count cs of chunk t (NB / 512 bins): a block-wide scan over the chunks, then one warp
// scans the chunk.
template <int NB>
__device__ void med_find(const unsigned* hist, unsigned cs, unsigned r, unsigned* wsum,
                         unsigned* res) {
  constexpr int C = NB / 512, PER = C / 32;   // 2 or 4 bins per lane in the last step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned incl = cs;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned a = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += a;
  }
  if (lane == 31) wsum[warp] = incl;
  if (tid == 0) { res[0] = NB - 1; res[1] = 0; res[2] = 0; res[3] = 0; }
  __syncthreads();
  unsigned wb = 0;
  for (int w = 0; w < warp; ++w) wb += wsum[w];
  const unsigned excl = wb + incl - cs;
  if (excl <= r && r < excl + cs) { res[2] = tid; res[3] = excl; }
  __syncthreads();
  if (tid < 32) {
    const unsigned k = res[2], rr = r - res[3];
    const unsigned* hc = hist + (size_t)k * C + lane * PER;
    unsigned v[PER], s = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) { v[j] = __ldcg(hc + j); s += v[j]; }
    unsigned inc2 = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned a = __shfl_up_sync(0xffffffffu, inc2, d);
      if (lane >= d) inc2 += a;
    }
    unsigned acc = inc2 - s;
    if (acc <= rr && rr < inc2) {
      int j = 0;
#pragma unroll
      for (int u = 0; u < PER - 1; ++u) {
        if (j == u && rr >= acc + v[u]) { acc += v[u]; j = u + 1; }
      }
      res[0] = (unsigned)(k * C + lane * PER + j);
      res[1] = rr - acc;
    }
  }
  __syncthreads();
}

// Round 0: the 32768-bucket histogram of the upper halves (64 KB of shared memory).
// 512 threads (every warp takes part in every step of the flush).
__global__ void __launch_bounds__(512, 3) median_hist0(const float* __restrict__ an0,
                                                       const __grid_constant__ Group gr,
                                                       MedianWs ws) {
  extern __shared__ uint4 med_smem[];
  unsigned* h = reinterpret_cast<unsigned*>(med_smem);   // bucket b: half (b & 1) of word b >> 1
  const int o = blockIdx.y, img = blockIdx.z;
  long long beg, end;
  med_slice(gr, img, beg, end);
  if (beg >= end) return;   // the whole CTA: a smaller image's slices are used up
  for (int i = threadIdx.x; i < MED_B0 / 8; i += blockDim.x) med_smem[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  const long long P = gr.P(img);
  const float* src = an0 + (size_t)NO * gr.poff[img] + (size_t)o * P;
  med_stream(src, beg, end, P, [&](unsigned bits) {
    const unsigned b = (bits >> 16) & 0x7FFFu;
    atomicAdd(&h[b >> 1], 1u << ((b & 1u) << 4));
  });
  __syncthreads();
  // a warp's 32 consecutive words are one chunk (64 buckets): the nonzero buckets are
  // added by their lanes, the chunk's count (when not zero) by lane 0
  unsigned* gh = ws.hist + ((size_t)img * NO + o) * MEDIAN_HIST_WORDS;
  for (int i = threadIdx.x; i < MED_B0 / 2; i += blockDim.x) {
    const unsigned w = h[i], lo = w & 0xFFFFu, hi = w >> 16;
    if (lo) atomicAdd(gh + 2 * i, lo);
    if (hi) atomicAdd(gh + 2 * i + 1, hi);
    if (__any_sync(0xffffffffu, w != 0)) {
      unsigned c = lo + hi;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
      if ((threadIdx.x & 31) == 0) atomicAdd(gh + MED_CH0 + (i >> 5), c);
    }
  }
}

// After round 0: state = (bucket, rank within it) of the lower and upper middle ranks
// (P - 1) / 2 and P / 2.  One 512-thread CTA per (image, orientation).
__global__ void __launch_bounds__(512) median_select0(const __grid_constant__ Group gr, MedianWs ws) {
  __shared__ unsigned wsum[16], res[4];
  const int o = blockIdx.x, img = blockIdx.y;
  const long long P = gr.P(img);
  const unsigned* gh = ws.hist + ((size_t)img * NO + o) * MEDIAN_HIST_WORDS;
  const unsigned cs = __ldcg(gh + MED_CH0 + threadIdx.x);
  med_find<MED_B0>(gh, cs, (unsigned)((P - 1) / 2), wsum, res);
  const unsigned b0 = res[0], k0 = res[1];
  __syncthreads();   // res is rewritten by the next search
  med_find<MED_B0>(gh, cs, (unsigned)(P / 2), wsum, res);
  if (threadIdx.x == 0) {
    unsigned* st = ws.state + ((size_t)img * NO + o) * 4;
    st[0] = b0;
    st[1] = k0;
    st[2] = res[0];
    st[3] = res[1];
  }
}

// Round 1: the lower halves of the values in the middle ranks' buckets (state words 0 and
// 2), into 65536 global buckets per rank (the upper rank's only when its bucket differs).
// Each hit also counts in its 128-bucket chunk.  Where eight or more lanes of a warp hit
// at once (a plane with many equal values), the lanes with equal buckets add their count
// once.
__global__ void __launch_bounds__(512) median_hist1(const float* __restrict__ an0,
                                                    const __grid_constant__ Group gr,
                                                    MedianWs ws) {
  const int o = blockIdx.y, img = blockIdx.z;
  long long beg, end;
  med_slice(gr, img, beg, end);
  if (beg >= end) return;
  const unsigned* st = ws.state + ((size_t)img * NO + o) * 4;
  const unsigned pre0 = st[0], pre1 = st[2];
  const bool two = pre1 != pre0;
  unsigned* gh = ws.hist + ((size_t)img * NO + o) * MEDIAN_HIST_WORDS + MED_B0;
  const long long P = gr.P(img);
  const float* src = an0 + (size_t)NO * gr.poff[img] + (size_t)o * P;
  unsigned* gc = ws.hist + ((size_t)img * NO + o) * MEDIAN_HIST_WORDS + MED_CH1;
  med_stream(src, beg, end, P, [&](unsigned bits) {
    const unsigned pre = bits >> 16;
    const int slot = (pre == pre0) ? 0 : (two && pre == pre1) ? 1 : -1;
    if (slot < 0) return;   // nearly every value
    // the lanes that hit together: the bucket and its chunk count once per equal key
    const unsigned key = ((unsigned)slot << 16) | (bits & 0xFFFFu);
    const unsigned act = __activemask();
    unsigned n = 1;
    bool lead = true;
    if (__popc(act) >= 8) {
      const unsigned same = __match_any_sync(act, key);
      n = (unsigned)__popc(same);
      lead = (int)(threadIdx.x & 31) == __ffs(same) - 1;
    }
    if (lead) {
      atomicAdd(gh + key, n);
      atomicAdd(gc + (key >> 7), n);
    }
  });
}

// After round 1: each middle value = (bucket << 16) | lower half, and T_o = noise_c times
// their mean.  One 512-thread CTA per (image, orientation).
__global__ void __launch_bounds__(512) median_select1(const __grid_constant__ Group gr,
                                                      float noise_c, MedianWs ws) {
  __shared__ unsigned wsum[16], res[4];
  const int o = blockIdx.x, img = blockIdx.y;
  const unsigned* st = ws.state + ((size_t)img * NO + o) * 4;
  const unsigned pre0 = st[0], r0 = st[1], pre1 = st[2], r1 = st[3];
  const bool two = pre1 != pre0;
  const unsigned* gh = ws.hist + ((size_t)img * NO + o) * MEDIAN_HIST_WORDS + MED_B0;
  const unsigned* gc = gh - MED_B0 + MED_CH1;
  const unsigned cs0 = __ldcg(gc + threadIdx.x);
  const unsigned cs1 = two ? __ldcg(gc + 512 + threadIdx.x) : cs0;
  med_find<MED_B1>(gh, cs0, r0, wsum, res);
  const unsigned v0 = (pre0 << 16) | res[0];
  __syncthreads();
  med_find<MED_B1>(gh + (two ? MED_B1 : 0), cs1, r1, wsum, res);
  const unsigned v1 = (pre1 << 16) | res[0];
  if (threadIdx.x == 0) ws.noise_t[img * NO + o] = 0.5f * (__uint_as_float(v0) + __uint_as_float(v1)) * noise_c;
}

cudaError_t launch_noise_threshold(const float* an0, const Group& gr, const KParams& kp,
                                   MedianWs ws, cudaStream_t st) {
  // at most MED_SLICE values per CTA of the largest image (a smaller image's CTAs take
  // smaller slices); the histograms (MEDIAN_HIST_WORDS per image and orientation) are zero
  long long pmax = 1;
  for (int i = 0; i < gr.n; ++i) pmax = gr.P(i) > pmax ? gr.P(i) : pmax;
  const int chunks = (int)((pmax + MED_SLICE - 1) / MED_SLICE);
  const int sm0 = MED_B0 / 2 * (int)sizeof(unsigned);
  cudaFuncSetAttribute(median_hist0, cudaFuncAttributeMaxDynamicSharedMemorySize, sm0);
  median_hist0<<<dim3(chunks, NO, gr.n), 512, sm0, st>>>(an0, gr, ws);
  median_select0<<<dim3(NO, gr.n), 512, 0, st>>>(gr, ws);
  median_hist1<<<dim3(chunks, NO, gr.n), 512, 0, st>>>(an0, gr, ws);
  median_select1<<<dim3(NO, gr.n), 512, 0, st>>>(gr, kp.noise_c, ws);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ PC and moments
// Maximum moment of one pixel from its six (q_o, Er_o); mc = the minimum moment plus eps/2,
// clamped at 0 (the covariance's smaller eigenvalue).
__device__ __forceinline__ float moment_px(const float (&qv)[NO], const float (&ev)[NO],
                                           const float (&tn)[NO], const KParams& kp,
                                           float (&pc)[NO], float& mc) {
  float sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    pc[o] = qv[o] * fmaxf(ev[o] - tn[o], 0.f);
    const float a = pc[o] * kp.cos_o[o], b = pc[o] * kp.sin_o[o];
    sxx += a * a;
    syy += b * b;
    sxy += a * b;
  }
  sxx *= 2.f / NO;
  syy *= 2.f / NO;
  sxy *= 4.f / NO;
  const float d = sxx - syy;
  const float sq = sqrtf(sxy * sxy + d * d);
  const float den = sq + kp.eps;
  mc = fmaxf(0.5f * (sxx + syy - sq), 0.f);
  return 0.5f * (sxx + syy + den);
}

__global__ void __launch_bounds__(256) pc_moment(const float* __restrict__ er,
                                                 const float* __restrict__ q,
                                                 const float* __restrict__ noise_t,
                                                 const __grid_constant__ Group gr,
                                                 KParams kp, float* __restrict__ moment,
                                                 unsigned* __restrict__ minmax,
                                                 float* __restrict__ pc_out,
                                                 float* __restrict__ mcorner,
                                                 unsigned* __restrict__ minmax_c) {
  const int img = blockIdx.y;
  const long long P = gr.P(img);
  const size_t pb = (size_t)gr.poff[img];
  float tn[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) tn[o] = __ldg(noise_t + img * NO + o);
  float lo = 3.0e38f, hi = 0.f, loc = 3.0e38f, hic = 0.f;
  const size_t ib = NO * pb;
  if ((P & 3) == 0) {
    // four pixels per thread and step: twelve 16-byte loads in flight
    const long long P4 = P >> 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P4;
         i += (long long)gridDim.x * blockDim.x) {
      float4 q4[NO], e4[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        q4[o] = __ldg(reinterpret_cast<const float4*>(q + ib + (size_t)o * P) + i);
        e4[o] = __ldg(reinterpret_cast<const float4*>(er + ib + (size_t)o * P) + i);
      }
      float mv[4], mcv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float qv[NO], ev[NO], pc[NO];
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          qv[o] = c == 0 ? q4[o].x : c == 1 ? q4[o].y : c == 2 ? q4[o].z : q4[o].w;
          ev[o] = c == 0 ? e4[o].x : c == 1 ? e4[o].y : c == 2 ? e4[o].z : e4[o].w;
        }
        mv[c] = moment_px(qv, ev, tn, kp, pc, mcv[c]);
        loc = fminf(loc, mcv[c]);
        hic = fmaxf(hic, mcv[c]);
        if (pc_out) {
#pragma unroll
          for (int o = 0; o < NO; ++o) pc_out[ib + (size_t)o * P + 4 * i + c] = pc[o];
        }
        lo = fminf(lo, mv[c]);
        hi = fmaxf(hi, mv[c]);
      }
      reinterpret_cast<float4*>(moment + pb)[i] = make_float4(mv[0], mv[1], mv[2], mv[3]);
      if (mcorner)
        reinterpret_cast<float4*>(mcorner + pb)[i] = make_float4(mcv[0], mcv[1], mcv[2], mcv[3]);
    }
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
      float qv[NO], ev[NO], pc[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        qv[o] = __ldg(q + ib + (size_t)o * P + i);
        ev[o] = __ldg(er + ib + (size_t)o * P + i);
      }
      float mc;
      const float m = moment_px(qv, ev, tn, kp, pc, mc);
      if (mcorner) mcorner[pb + i] = mc;
      loc = fminf(loc, mc);
      hic = fmaxf(hic, mc);
      if (pc_out) {
#pragma unroll
        for (int o = 0; o < NO; ++o) pc_out[ib + (size_t)o * P + i] = pc[o];
      }
      moment[pb + i] = m;
      lo = fminf(lo, m);
      hi = fmaxf(hi, m);
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, d));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    loc = fminf(loc, __shfl_xor_sync(0xffffffffu, loc, d));
    hic = fmaxf(hic, __shfl_xor_sync(0xffffffffu, hic, d));
  }
  __shared__ float slo[8], shi[8], sloc[8], shic[8];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { slo[w] = lo; shi[w] = hi; sloc[w] = loc; shic[w] = hic; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      lo = fminf(lo, slo[k]);
      hi = fmaxf(hi, shi[k]);
      loc = fminf(loc, sloc[k]);
      hic = fmaxf(hic, shic[k]);
    }
    // M > 0 and the corner map >= 0, so the bit patterns order like the values
    atomicMin(minmax + 2 * img, __float_as_uint(lo));
    atomicMax(minmax + 2 * img + 1, __float_as_uint(hi));
    if (minmax_c) {
      atomicMin(minmax_c + 2 * img, __float_as_uint(loc));
      atomicMax(minmax_c + 2 * img + 1, __float_as_uint(hic));
    }
  }
}

cudaError_t launch_pc_moment(const float* er, const float* q, const float* noise_t,
                             const Group& gr, const KParams& kp, float* moment, unsigned* minmax,
                             float* pc_out, float* mcorner, unsigned* minmax_c, cudaStream_t st) {
  long long pmax = 1;
  for (int i = 0; i < gr.n; ++i) pmax = gr.P(i) > pmax ? gr.P(i) : pmax;
  long long blocks = (pmax / 4 + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1216) blocks = 1216;   // 8 per SM on 152 SMs; grid-stride beyond
  pc_moment<<<dim3((unsigned)blocks, gr.n), 256, 0, st>>>(er, q, noise_t, gr, kp, moment, minmax,
                                                          pc_out, mcorner, minmax_c);
  return cudaGetLastError();
}

}  // namespace rift2
