// Noise threshold and phase congruency (§II-A: "one-dimensional phase congruency for
// each orientation of the log-Gabor convolutions", "analyzes the change of moment with
// orientations").  The noise model follows the phase-congruency model RIFT builds on:
// T_o is a fixed multiple of the median smallest-scale amplitude.
//
//   median_hist / median_select : exact median of |EO_0,o| over the whole image by a
//     three-round radix select on the float bit patterns (12 + 12 + 8 bits).  The
//     amplitudes are non-negative, so their bit patterns order like the values.  For an
//     even pixel count the two middle values are selected and averaged.
//   pc_moment : PC_o = q_o max(Er_o - T_o, 0), covariance moments over the orientations,
//     maximum moment M, and the image-wide min / max of M for the FAST normalisation.
#include "kernels.h"

namespace rift2 {

constexpr int MED_BINS = 4096;

__device__ __forceinline__ void med_digit(unsigned bits, int round, unsigned& pre, unsigned& dig) {
  if (round == 0) { pre = 0; dig = bits >> 20; }
  else if (round == 1) { pre = bits >> 20; dig = (bits >> 8) & 0xFFFu; }
  else { pre = bits >> 8; dig = bits & 0xFFu; }
}

__global__ void __launch_bounds__(512) median_hist(const float* __restrict__ an0,
                                                   const __grid_constant__ Group gr, int round,
                                                   MedianWs ws) {
  __shared__ unsigned h[2][MED_BINS];
  const int nslot = (round == 0) ? 1 : 2;   // round 0: both ranks share one histogram
  const int o = blockIdx.y, img = blockIdx.z;
  const long long P = gr.P(img);
  for (int i = threadIdx.x; i < nslot * MED_BINS; i += blockDim.x) (&h[0][0])[i] = 0;
  const unsigned* st = ws.state + ((size_t)img * NO + o) * 4;
  const unsigned pre0 = st[0], pre1 = st[2];
  __syncthreads();
  const float* src = an0 + (size_t)NO * gr.poff[img] + (size_t)o * P;
  const long long chunk = ((P + gridDim.x - 1) / gridDim.x + 3) & ~3ll;
  const long long beg = blockIdx.x * chunk;
  const long long end = min(P, beg + chunk);
  auto one = [&](unsigned bits) {
    unsigned pre, dig;
    med_digit(bits, round, pre, dig);
    if (round == 0) {
      atomicAdd(&h[0][dig], 1u);
    } else {
      if (pre == pre0) atomicAdd(&h[0][dig], 1u);
      if (pre == pre1) atomicAdd(&h[1][dig], 1u);
    }
  };
  // 16-byte loads when the slice is 16-byte aligned (P % 4 == 0), scalar otherwise; four
  // loads per thread in flight before their values are counted
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
  __syncthreads();
  unsigned* gh = ws.hist + ((size_t)img * NO + o) * 2 * MED_BINS;
  for (int i = threadIdx.x; i < nslot * MED_BINS; i += blockDim.x) {
    unsigned c = (&h[0][0])[i];
    if (c) atomicAdd(gh + i, c);
  }
}

// One CTA per (image, orientation) and round, for both middle ranks (lower = (P-1)/2,
// upper = P/2): each of 256 threads sums its slice of the bins of both ranks' histograms,
// a block-wide scan locates the bin holding each rank, and the state becomes (prefix with
// that digit appended, rank within the bin).  The histograms are cleared for the next
// round; after the last round T_o follows from the two middle values.
__global__ void __launch_bounds__(256) median_select(const __grid_constant__ Group gr, int round,
                                                     float noise_c, MedianWs ws) {
  __shared__ unsigned part[2][256];
  __shared__ unsigned s_dig[2], s_rank[2];
  const int o = blockIdx.x, img = blockIdx.y;
  const long long P = gr.P(img);
  const int tid = threadIdx.x;
  unsigned* gh = ws.hist + ((size_t)img * NO + o) * 2 * MED_BINS;
  unsigned* st = ws.state + ((size_t)img * NO + o) * 4;
  const int nbins = (round == 2) ? 256 : MED_BINS;
  const int shift = (round == 2) ? 8 : 12;
  const int per = nbins / 256;
  unsigned prefix[2], rank[2], loc[2];
  for (int t = 0; t < 2; ++t) {
    if (round == 0) {
      prefix[t] = 0;
      rank[t] = (unsigned)(t == 0 ? (P - 1) / 2 : P / 2);
    } else {
      prefix[t] = st[2 * t];
      rank[t] = st[2 * t + 1];
    }
    const unsigned* hist = gh + ((round == 0) ? 0 : t) * MED_BINS;
    unsigned sum = 0;
    for (int i = 0; i < per; ++i) sum += hist[tid * per + i];
    loc[t] = sum;
    part[t][tid] = sum;
  }
  if (tid < 2) {
    s_dig[tid] = nbins - 1;
    s_rank[tid] = 0;
  }
  __syncthreads();
  for (int d = 1; d < 256; d <<= 1) {
    const unsigned a0 = tid >= d ? part[0][tid - d] : 0u, a1 = tid >= d ? part[1][tid - d] : 0u;
    __syncthreads();
    part[0][tid] += a0;
    part[1][tid] += a1;
    __syncthreads();
  }
  for (int t = 0; t < 2; ++t) {
    const unsigned incl = part[t][tid], excl = incl - loc[t];
    if (excl <= rank[t] && rank[t] < incl) {
      const unsigned* hist = gh + ((round == 0) ? 0 : t) * MED_BINS;
      unsigned acc = excl;
      int i = 0;
      for (; i < per - 1; ++i) {
        const unsigned c = hist[tid * per + i];
        if (rank[t] < acc + c) break;
        acc += c;
      }
      s_dig[t] = tid * per + i;
      s_rank[t] = rank[t] - acc;
    }
  }
  __syncthreads();   // every thread has read the histogram
  if (tid < 2) {
    st[2 * tid] = (prefix[tid] << shift) | s_dig[tid];
    st[2 * tid + 1] = s_rank[tid];
  }
  for (int i = tid; i < 2 * MED_BINS; i += blockDim.x) gh[i] = 0;   // ready for next round
  if (round == 2) {
    __syncthreads();
    if (tid == 0) {
      const float v0 = __uint_as_float(st[0]), v1 = __uint_as_float(st[2]);
      ws.noise_t[img * NO + o] = 0.5f * (v0 + v1) * noise_c;
    }
  }
}

cudaError_t launch_noise_threshold(const float* an0, const Group& gr, const KParams& kp,
                                   MedianWs ws, cudaStream_t st) {
  // ~64K values per CTA of the largest image (a smaller image's CTAs take smaller
  // slices): the histogram set-up and flush stay small next to the scan
  long long pmax = 1;
  for (int i = 0; i < gr.n; ++i) pmax = gr.P(i) > pmax ? gr.P(i) : pmax;
  int chunks = (int)((pmax + 65535) / 65536);
  if (chunks > 64) chunks = 64;
  if (chunks < 1) chunks = 1;
  for (int r = 0; r < 3; ++r) {
    median_hist<<<dim3(chunks, NO, gr.n), 512, 0, st>>>(an0, gr, r, ws);
    median_select<<<dim3(NO, gr.n), 256, 0, st>>>(gr, r, kp.noise_c, ws);
  }
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
