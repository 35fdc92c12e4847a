// Brute-force nearest-feature matching (§IV: "brute force matching with the nearest
// feature distance"; no ratio test and no RANSAC in the evaluation).
//
// The distance between descriptors a, b is ||a/|a| - b/|b|||^2 = 2 - 2 a.b / (|a||b|).
// Descriptor entries are integer counts (each cell sums to 256), so a.b and |a|^2 are
// integers below 2^24: float accumulation is exact, and the comparison
//     a.b_j / |b_j|  >  a.b_k / |b_k|   <=>   (a.b_j)^2 |b_k|^2  >  (a.b_k)^2 |b_j|^2
// is decided exactly in 64-bit integers (the products stay below 2^64), lowest index on
// ties.  The reported distance uses the exact integer numerator |a|^2|b|^2 - (a.b)^2.
//
//   match_simt : CUDA-core form.  A CTA holds 64 queries and streams B in tiles of 64,
//                each thread owning a 4x4 block of dot products and a running top-2.
#include "kernels.h"
#include "match_common.cuh"

namespace rift2 {

constexpr int MT = 64;   // queries per CTA and candidates per tile

__device__ __forceinline__ void load_tile(float* dst, const unsigned short* src, int r0, int n,
                                          float* n2) {
  for (int i = threadIdx.x; i < MT * DESC_DIM; i += blockDim.x) {
    int r = i / DESC_DIM, k = i - r * DESC_DIM;
    float v = (r0 + r < n) ? (float)src[(size_t)(r0 + r) * DESC_DIM + k] : 0.f;
    dst[k * MT + r] = v;
  }
  __syncthreads();
  if (threadIdx.x < MT) {
    float acc = 0.f;
    for (int k = 0; k < DESC_DIM; ++k) {
      float v = dst[k * MT + threadIdx.x];
      acc += v * v;
    }
    n2[threadIdx.x] = acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) match_simt(MatchPtrs mp) {
  extern __shared__ float msm[];
  float* As = msm;                       // [216][64]
  float* Bs = msm + DESC_DIM * MT;       // [216][64]
  __shared__ float n2a[MT], n2b[MT];
  const int pr = blockIdx.y;
  const int nA = mp.counts_a[pr][1], nB = mp.counts_b[pr][1];
  const int q0 = blockIdx.x * MT;
  if (blockIdx.x == 0 && threadIdx.x == 0) *mp.count[pr] = nA;
  if (q0 >= nA) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  load_tile(As, mp.desc_a[pr], q0, nA, n2a);
  Cand c1[4], c2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    c1[i] = Cand{0.f, 1.f, 0x7fffffff};
    c2[i] = c1[i];
  }
  for (int j0 = 0; j0 < nB; j0 += MT) {
    load_tile(Bs, mp.desc_b[pr], j0, nB, n2b);
    float acc[4][4] = {};
    for (int k = 0; k < DESC_DIM; ++k) {
      float4 a = *reinterpret_cast<const float4*>(As + k * MT + 4 * ty);
      float4 b = *reinterpret_cast<const float4*>(Bs + k * MT + 4 * tx);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(av[i], bv[c], acc[i][c]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int j = j0 + 4 * tx + c;
      if (j < nB) {
#pragma unroll
        for (int i = 0; i < 4; ++i) push2(c1[i], c2[i], Cand{acc[i][c], n2b[4 * tx + c], j});
      }
    }
    __syncthreads();   // Bs is overwritten by the next tile
  }
  // merge the 16 partial top-2 lists of each query (lanes with equal ty share a warp half)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      Cand o1{__shfl_xor_sync(0xffffffffu, c1[i].dot, d), __shfl_xor_sync(0xffffffffu, c1[i].n2, d),
              __shfl_xor_sync(0xffffffffu, c1[i].j, d)};
      Cand o2{__shfl_xor_sync(0xffffffffu, c2[i].dot, d), __shfl_xor_sync(0xffffffffu, c2[i].n2, d),
              __shfl_xor_sync(0xffffffffu, c2[i].j, d)};
      push2(c1[i], c2[i], o1);
      push2(c1[i], c2[i], o2);
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int q = q0 + 4 * ty + i;
      if (q >= nA) continue;
      float na2 = n2a[4 * ty + i];
      bool ok1 = c1[i].j != 0x7fffffff, ok2 = c2[i].j != 0x7fffffff;
      float d1 = ok1 ? exact_dist(na2, c1[i]) : __int_as_float(0x7f800000);
      float d2 = ok2 ? exact_dist(na2, c2[i]) : __int_as_float(0x7f800000);
      mp.q_desc[pr][q] = q;
      mp.nn_desc[pr][q] = ok1 ? c1[i].j : -1;
      mp.kp_a[pr][q] = mp.desc_kp_a[pr][q];
      mp.kp_b[pr][q] = ok1 ? mp.desc_kp_b[pr][c1[i].j] : -1;
      mp.d1[pr][q] = d1;
      mp.d2[pr][q] = d2;
      mp.near_tie[pr][q] = (ok2 && (d2 - d1) < 1e-5f * fmaxf(d1, 1e-12f)) ? 1 : 0;
    }
  }
}

cudaError_t launch_match_simt(const MatchPtrs& mp, int npairs, int max_desc, cudaStream_t st) {
  size_t sm = 2 * (size_t)DESC_DIM * MT * sizeof(float);
  cudaFuncSetAttribute(match_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  match_simt<<<dim3((max_desc + MT - 1) / MT, npairs), 256, sm, st>>>(mp);
  return cudaGetLastError();
}

}  // namespace rift2
