// Batched mixed-radix Stockham FFT over shared memory (radices 2, 3, 4, 5, 7, 8, 11, 13).
//
// A Stockham (auto-sorting) pass of radix R over an n-point transform, with ns the
// product of the radices already applied, maps butterfly j (0 <= j < n/R, k = j mod ns)
//     v_r = in[j + r n/R] * W_{ns R}^{k r},   v = DFT_R(v),
//     out[(j / ns) ns R + k + r ns] = v_r,
// and leaves the result in natural order after the last pass.  Twiddles come from one
// table per length, tw[e] = exp(-2 pi i e / n), generated in double precision.
#pragma once

#include "common.cuh"

namespace rift2 {

constexpr int FFT_MAX_STAGES = 16;

struct FftPlan {
  int n;
  int nst;
  int radix[FFT_MAX_STAGES];
  const float2* tw;   // device, n entries
};

template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e) {
  float2 w = __ldg(tw + e);
  return INV ? make_float2(w.x, -w.y) : w;
}

// Multiply by -i (forward) or +i (inverse).
template <bool INV>
__device__ __forceinline__ float2 rot_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
  float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  float2 a2 = cadd(v[1], v[3]), a3 = rot_mi<INV>(csub(v[1], v[3]));
  v[0] = cadd(a0, a2);
  v[2] = csub(a0, a2);
  v[1] = cadd(a1, a3);
  v[3] = csub(a1, a3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float c = 0.70710678118654752440f;
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // o_k *= W8^k (conjugated for the inverse)
  float2 o1 = INV ? make_float2(c * (o[1].x - o[1].y), c * (o[1].x + o[1].y))
                  : make_float2(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x));
  float2 o2 = rot_mi<INV>(o[2]);
  float2 o3 = INV ? make_float2(-c * (o[3].x + o[3].y), c * (o[3].x - o[3].y))
                  : make_float2(c * (o[3].y - o[3].x), -c * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

// Odd radix: direct R-point DFT with roots of unity read from the length-n table.
template <int R, bool INV>
__device__ __forceinline__ void dft_odd(float2* v, const float2* __restrict__ tw, int n) {
  float2 out[R];
  const int step = n / R;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    float2 acc = v[0];
#pragma unroll
    for (int m = 1; m < R; ++m) {
      float2 w = twiddle<INV>(tw, ((m * k) % R) * step);
      acc = cadd(acc, cmul(v[m], w));
    }
    out[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v, const float2* __restrict__ tw, int n) {
  if constexpr (R == 2) dft2<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else dft_odd<R, INV>(v, tw, n);
}

// One Stockham pass over nb transforms; element k of transform b at buf[b*bs + k*ks].
// BFAST: consecutive threads take consecutive transforms (column tiles, ks > 1);
// otherwise consecutive butterflies of one transform (rows, ks == 1).
template <int R, bool INV, bool BFAST>
__device__ __forceinline__ void fft_pass(const float2* __restrict__ in, float2* __restrict__ out,
                                         int n, int ns, int nb, int bs, int ks,
                                         const float2* __restrict__ tw, int tid, int nthr) {
  const int m = n / R;
  const int tstep = n / (ns * R);
  const int total = nb * m;
  for (int idx = tid; idx < total; idx += nthr) {
    int b, j;
    if (BFAST) { j = idx / nb; b = idx - j * nb; }
    else       { b = idx / m;  j = idx - b * m; }
    const int k = j % ns;
    const float2* src = in + b * bs;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * m) * ks];
    if (ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle<INV>(tw, k * r * tstep));
    }
    dft_r<R, INV>(v, tw, n);
    float2* dst = out + b * bs;
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * ns) * ks] = v[r];
  }
}

// Full transform; data starts in `a`, `b` is scratch of the same size.  Returns the
// buffer holding the result.  Ends with a __syncthreads().
template <bool INV, bool BFAST>
__device__ float2* fft_smem(float2* a, float2* b, const FftPlan& pl, int nb, int bs, int ks) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  int ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.radix[st];
    switch (R) {
      case 8: fft_pass<8, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 4: fft_pass<4, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 2: fft_pass<2, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 3: fft_pass<3, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 5: fft_pass<5, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 7: fft_pass<7, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 11: fft_pass<11, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      case 13: fft_pass<13, INV, BFAST>(a, b, pl.n, ns, nb, bs, ks, pl.tw, tid, nthr); break;
      default: break;
    }
    __syncthreads();
    ns *= R;
    float2* t = a; a = b; b = t;
  }
  return a;
}

}  // namespace rift2
