// Register-tiled Stockham FFT for power-of-two lengths: a group of T threads owns one
// N-point transform, each thread holding E = N / T elements in registers.  Each pass of
// radix R runs E / R radix-R butterflies per thread entirely in registers; passes talk
// through one padded shared-memory buffer per transform, so an N = 1024 transform is two
// radix-32 passes with a single exchange and only warp-level synchronisation.
//
// Pass with radix R after NS = product of the earlier radices, butterfly j (k = j mod NS):
//     v_r = x[j + r N/R] * W_{NS R}^{k r},  v = DFT_R(v),  y[(j - k) R + k + r NS] = v_r.
#pragma once

#include "fft.cuh"

namespace rift2 {

// cos / sin (2 pi m / 32), m = 0..31: the roots of unity the in-register DFTs use.
__device__ constexpr float kCos32[32] = {
    1.000000000e+00f,  9.807852804e-01f,  9.238795325e-01f,  8.314696123e-01f,
    7.071067812e-01f,  5.555702330e-01f,  3.826834324e-01f,  1.950903220e-01f,
    0.0f,              -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
    -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
    -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
    -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f,
    0.0f,              1.950903220e-01f,  3.826834324e-01f,  5.555702330e-01f,
    7.071067812e-01f,  8.314696123e-01f,  9.238795325e-01f,  9.807852804e-01f};
__device__ constexpr float kSin32[32] = {
    0.0f,              1.950903220e-01f,  3.826834324e-01f,  5.555702330e-01f,
    7.071067812e-01f,  8.314696123e-01f,  9.238795325e-01f,  9.807852804e-01f,
    1.000000000e+00f,  9.807852804e-01f,  9.238795325e-01f,  8.314696123e-01f,
    7.071067812e-01f,  5.555702330e-01f,  3.826834324e-01f,  1.950903220e-01f,
    0.0f,              -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
    -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
    -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
    -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f};

// exp(-+ 2 pi i m / R) for R | 32 (forward sign; INV conjugates).  m is a compile-time
// constant after unrolling, so the table reads fold into immediates.
template <int R, bool INV>
__device__ __forceinline__ float2 wr(int m) {
  const int e = (m * (32 / R)) & 31;
  return make_float2(kCos32[e], INV ? kSin32[e] : -kSin32[e]);
}

// In-register DFT of length R in natural order (R = 1, 2, 4, 8, 16, 32).  R = 16, 32 are
// split as R1 x 4: R1-point DFTs over n1 of x[4 n1 + n2], internal twiddles W_R^{n2 k1},
// then 4-point DFTs over n2, with output k1 + R1 k2.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v);
  } else if constexpr (R == 8) {
    dft8<INV>(v);
  } else {
    constexpr int R2 = 4, R1 = R / 4;
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      float2 t[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
      dft_reg<R1, INV>(t);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1)
        v[R2 * k1 + n2] = (n2 * k1 == 0) ? t[k1] : cmul(t[k1], wr<R, INV>(n2 * k1));
    }
    float2 out[R];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 t[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) t[n2] = v[R2 * k1 + n2];
      dft4<INV>(t);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) out[k1 + R1 * k2] = t[k2];
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = out[i];
  }
}

// Padded index into a transform's exchange buffer: one spare slot per 32 elements keeps
// the strided butterfly stores free of bank conflicts.
__device__ __forceinline__ int xpad(int i) { return i + (i >> 5); }
template <int N>
struct XBuf {
  static constexpr int SIZE = N + N / 32 + 2;   // +2: staggers consecutive buffers' banks
};

// Stride between the exchange buffers of the COLS columns a CTA transposes through shared
// memory (row segments of COLS columns in global memory <-> one buffer per column): a
// stride of 16 / COLS (mod 16) float2 puts the COLS columns of the (16 / COLS) rows a
// half-warp touches on 32 distinct banks.
template <int N, int COLS>
struct ColStride {
  static_assert(COLS >= 1 && COLS <= 16 && 16 % COLS == 0, "columns per CTA");
  static constexpr int BASE = XBuf<N>::SIZE;
  static constexpr int SIZE = BASE + ((16 / COLS - BASE % 16) % 16 + 16) % 16;
};

// log2 of a power-of-two radix.
template <int R>
constexpr int log2_radix() { return R >= 32 ? 5 : R >= 16 ? 4 : R >= 8 ? 3 : R >= 4 ? 2 : 1; }

// The twiddle powers one thread's butterflies of a pass need: for butterfly i (k = the
// butterfly's index modulo NS) the table values W^(k 2^b TSTEP), b < log2(R).  They depend
// only on the thread, so a transform loads them before its first pass runs and the loads'
// latency hides behind that pass.
template <int N, int T, int R, int NS>
struct PassTw {
  static constexpr int B = (N / T) / R, LOGR = log2_radix<R>();
  float2 w[B][LOGR];
  template <bool INV>
  __device__ __forceinline__ void load(int t, const float2* __restrict__ tw) {
    if constexpr (NS > 1) {
      constexpr int TSTEP = N / (NS * R);
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const int k = (t + T * i) % NS;
#pragma unroll
        for (int b = 0; b < LOGR; ++b) w[i][b] = twiddle<INV>(tw, k * (1 << b) * TSTEP);
      }
    }
  }
};

// One pass.  Inputs come from `ld(i, r, index)` (FIRST; i = butterfly of this thread,
// r = butterfly input, both compile-time) or the exchange buffer; outputs go to
// `st(index, value)` (LAST) or the exchange buffer.  `sync()` synchronises the group.
// Twiddles W^(k r TSTEP), r = 1..R-1: the powers r = 2^b come from `tp` (table values
// generated in FP64); every other r is the product of the powers of its set bits, taken
// from the lowest bit up, so each shares its prefix product with a smaller r: log2(R)
// table reads instead of R - 1, at most log2(R) - 1 extra roundings per twiddle (relative
// error below 1e-6).
template <int N, int T, int R, int NS, bool INV, bool FIRST, bool LAST, class Ld, class St,
          class Sync>
__device__ __forceinline__ void reg_pass(float2* xb, int t, const PassTw<N, T, R, NS>& tp,
                                         Ld& ld, St& st, Sync& sync) {
  constexpr int E = N / T, B = E / R, M = N / R;
  static_assert(E % R == 0, "radix must divide the elements per thread");
  float2 v[B][R];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int j = t + T * i;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = FIRST ? ld(i, r, j + r * M) : xb[xpad(j + r * M)];
  }
  if (!FIRST) sync();   // every read of xb is done before this pass overwrites it
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int j = t + T * i;
    const int k = j % NS;
    if constexpr (NS > 1) {
      constexpr int LOGR = PassTw<N, T, R, NS>::LOGR;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = make_float2(1.f, 0.f);
        bool first = true;
#pragma unroll
        for (int b = 0; b < LOGR; ++b)
          if (r & (1 << b)) {
            w = first ? tp.w[i][b] : cmul(w, tp.w[i][b]);
            first = false;
          }
        v[i][r] = cmul(v[i][r], w);
      }
    }
    dft_reg<R, INV>(v[i]);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (LAST) st(base + r * NS, v[i][r]);
      else xb[xpad(base + r * NS)] = v[i][r];
    }
  }
  if (!LAST) sync();
}

// Full transform as up to three passes of radices R0, R1, R2 (1 = unused).  The later
// passes' twiddle powers are loaded before the first pass.
template <int N, int T, int R0, int R1, int R2, bool INV, class Ld, class St, class Sync>
__device__ __forceinline__ void group_fft(float2* xb, int t, const float2* __restrict__ tw, Ld& ld,
                                          St& st, Sync& sync) {
  static_assert(R0 * R1 * R2 == N, "radices must multiply to N");
  PassTw<N, T, R0, 1> p0;
  if constexpr (R1 == 1) {
    reg_pass<N, T, R0, 1, INV, true, true>(xb, t, p0, ld, st, sync);
  } else if constexpr (R2 == 1) {
    PassTw<N, T, R1, R0> p1;
    p1.template load<INV>(t, tw);
    reg_pass<N, T, R0, 1, INV, true, false>(xb, t, p0, ld, st, sync);
    reg_pass<N, T, R1, R0, INV, false, true>(xb, t, p1, ld, st, sync);
  } else {
    PassTw<N, T, R1, R0> p1;
    PassTw<N, T, R2, R0 * R1> p2;
    p1.template load<INV>(t, tw);
    p2.template load<INV>(t, tw);
    reg_pass<N, T, R0, 1, INV, true, false>(xb, t, p0, ld, st, sync);
    reg_pass<N, T, R1, R0, INV, false, false>(xb, t, p1, ld, st, sync);
    reg_pass<N, T, R2, R0 * R1, INV, false, true>(xb, t, p2, ld, st, sync);
  }
}

// The same transform when the input already sits in the exchange buffer: every pass
// (the first included) reads xb and synchronises before overwriting it.
template <int N, int T, int R0, int R1, int R2, bool INV, class St, class Sync>
__device__ __forceinline__ void group_fft_xb(float2* xb, int t, const float2* __restrict__ tw,
                                             St& st, Sync& sync) {
  static_assert(R0 * R1 * R2 == N, "radices must multiply to N");
  auto none = [](int, int, int) { return make_float2(0.f, 0.f); };
  PassTw<N, T, R0, 1> p0;
  if constexpr (R1 == 1) {
    reg_pass<N, T, R0, 1, INV, false, true>(xb, t, p0, none, st, sync);
  } else if constexpr (R2 == 1) {
    PassTw<N, T, R1, R0> p1;
    p1.template load<INV>(t, tw);
    reg_pass<N, T, R0, 1, INV, false, false>(xb, t, p0, none, st, sync);
    reg_pass<N, T, R1, R0, INV, false, true>(xb, t, p1, none, st, sync);
  } else {
    PassTw<N, T, R1, R0> p1;
    PassTw<N, T, R2, R0 * R1> p2;
    p1.template load<INV>(t, tw);
    p2.template load<INV>(t, tw);
    reg_pass<N, T, R0, 1, INV, false, false>(xb, t, p0, none, st, sync);
    reg_pass<N, T, R1, R0, INV, false, false>(xb, t, p1, none, st, sync);
    reg_pass<N, T, R2, R0 * R1, INV, false, true>(xb, t, p2, none, st, sync);
  }
}

// Column-pass shapes (more threads per transform, fewer registers per thread).
template <int N>
struct ColShape;
template <>
struct ColShape<256> {
  static constexpr int T = 16, R0 = 16, R1 = 16, R2 = 1, NT = 256;
};
template <>
struct ColShape<512> {
  static constexpr int T = 32, R0 = 16, R1 = 16, R2 = 2, NT = 256;
};
template <>
struct ColShape<1024> {
  static constexpr int T = 32, R0 = 32, R1 = 32, R2 = 1, NT = 128;
};
template <>
struct ColShape<2048> {
  static constexpr int T = 128, R0 = 16, R1 = 16, R2 = 8, NT = 512;
};
template <>
struct ColShape<4096> {
  static constexpr int T = 128, R0 = 32, R1 = 8, R2 = 16, NT = 256;
};

// Register-path shapes: transform length -> threads per transform and pass radices.
template <int N>
struct RegShape;
template <>
struct RegShape<256> {
  static constexpr int T = 16, R0 = 16, R1 = 16, R2 = 1, NT = 256;
};
template <>
struct RegShape<512> {
  static constexpr int T = 16, R0 = 32, R1 = 16, R2 = 1, NT = 256;
};
template <>
struct RegShape<1024> {   // one row (its four scale transforms) per 128-thread CTA
  static constexpr int T = 32, R0 = 32, R1 = 32, R2 = 1, NT = 128;
};
template <>
struct RegShape<2048> {
  static constexpr int T = 64, R0 = 32, R1 = 8, R2 = 8, NT = 256;
};
template <>
struct RegShape<4096> {
  static constexpr int T = 128, R0 = 32, R1 = 8, R2 = 16, NT = 512;
};

}  // namespace rift2
