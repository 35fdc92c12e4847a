// Batched mixed-radix Stockham FFT over shared memory (radices 2, 3, 4, 5, 7, 8, 9, 11, 13, 16).
//
// A Stockham (auto-sorting) pass of radix R over an n-point transform, with ns the
// product of the radices already applied, maps butterfly j (0 <= j < n/R, k = j mod ns)
//     v_r = in[j + r n/R] * W_{ns R}^{k r},   v = DFT_R(v),
//     out[(j / ns) ns R + k + r ns] = v_r,
// and leaves the result in natural order after the last pass.  Twiddles come from one
// table per length, tw[e] = exp(-2 pi i e / n), generated in double precision, gathered
// once per plan into a per-pass table (FftPasses::ptw); the odd radices' own roots are
// compile-time constants.
#pragma once

#include "common.cuh"

namespace rift2 {

constexpr int FFT_MAX_STAGES = 12;   // 13-smooth lengths up to 10240 need at most 9 passes

// Unsigned division by a run-time divisor d >= 1 for dividends below 2^31: the
// multiply-shift method (Granlund and Montgomery), q = (umulhi(n, m) + n) >> s with
// s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  unsigned m = 1, s = 0, d = 1;
  FastDiv() = default;
  __host__ __device__ explicit FastDiv(unsigned dv) : d(dv) {
    s = 0;
    while ((1u << s) < dv) ++s;
    m = (unsigned)(((1ull << 32) * ((1ull << s) - dv)) / dv + 1);
  }
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(n, m) + n) >> s; }
};

// One Stockham pass of a length-L transform as the shared-memory kernels run it.
struct FftPass {
  int R;        // radix
  int ns;       // product of the radices of the passes before this one
  FastDiv q;    // L / R: butterflies per transform
  FastDiv k;    // ns
  int tw;       // offset of the pass's twiddles in FftPasses::ptw, laid out [ns][R - 1]
};

// The device copy of a plan the shared-memory kernels read (made once per length): the
// passes at the transform length L (n, or the Bluestein convolution length) with their
// divisors precomputed on the host, and every pass's twiddles W_(ns R)^(k r), k < ns,
// 1 <= r < R, gathered from the FP64-generated length-L table.
struct FftPasses {
  int n, L, nst;
  FftPass p[FFT_MAX_STAGES];
  FastDiv dL, dn;
  const float2* ptw;
  const float2* chirp;      // Bluestein only: [n] c_j (NULL for a direct transform)
  const float2* kern_fwd;   // Bluestein only: [L]
  const float2* kern_inv;   // Bluestein only: [L]
};

// A transform of length n: directly (n 13-smooth: radices of n, twiddles of length n), or
// by Bluestein's chirp-z identity when n has a larger prime factor.  With c_j =
// exp(-i pi j^2 / n), jk = (j^2 + k^2 - (k - j)^2) / 2 turns the DFT into a convolution:
//     X_k = c_k sum_j (x_j c_j) conj(c_(k-j))          (forward; the inverse conjugates c)
// evaluated as a cyclic convolution of length m >= 2n - 1 (m 13-smooth, chosen by the
// planner's cost estimate, at most 2.5 n) with FFTs of
// length m: the radices and twiddles below are then those of m, and kern_* hold
// FFT_m(conj(c)) / m (forward) and FFT_m(c) / m (inverse), c extended cyclically
// (c_(m-j) = c_j for 0 < j < n, 0 between).  All tables are generated in FP64.
struct FftPlan {
  int n;
  int nst;
  int radix[FFT_MAX_STAGES];
  const float2* tw;   // device, m entries (twiddles of the length the passes run at)
  int m;              // length of one transform's shared-memory slot: n, or the convolution length
  const float2* chirp;      // Bluestein only: [n] c_j
  const float2* kern_fwd;   // Bluestein only: [m]
  const float2* kern_inv;   // Bluestein only: [m]
  const FftPasses* dev;     // device: the shared-memory kernels' copy
  const FftPasses* dev_r;   // device: the same transform without radix 16 (row kernels)
};

// Per-image transform data of one shared-memory-path launch over a Group: the device plan
// of the transformed side, the tile (rows or columns per CTA) with its divisor, and the
// zero-window column table of the image's size ([NO][W]: 1 where orientation o's angular
// window is zero on the whole column).
struct FftGroup {
  const FftPasses* pass[MAXB];
  int tile[MAXB];
  FastDiv dtile[MAXB];
  const unsigned char* zc[MAXB];
};

template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e) {
  float2 w = __ldg(tw + e);
  return INV ? make_float2(w.x, -w.y) : w;
}

template <bool INV>
__device__ __forceinline__ float2 twiddle_s(const float2* tw, int e) {
  float2 w = tw[e];
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

// cos / sin (2 pi j / R) of the odd radices (written out to 10 significant digits).
__device__ constexpr float kCos3[3] = {1.000000000e+00f, -5.000000000e-01f, -5.000000000e-01f};
__device__ constexpr float kSin3[3] = {0.000000000e+00f, 8.660254038e-01f, -8.660254038e-01f};
__device__ constexpr float kCos5[5] = {1.000000000e+00f, 3.090169944e-01f, -8.090169944e-01f, -8.090169944e-01f, 3.090169944e-01f};
__device__ constexpr float kSin5[5] = {0.000000000e+00f, 9.510565163e-01f, 5.877852523e-01f, -5.877852523e-01f, -9.510565163e-01f};
__device__ constexpr float kCos7[7] = {1.000000000e+00f, 6.234898019e-01f, -2.225209340e-01f, -9.009688679e-01f, -9.009688679e-01f, -2.225209340e-01f, 6.234898019e-01f};
__device__ constexpr float kSin7[7] = {0.000000000e+00f, 7.818314825e-01f, 9.749279122e-01f, 4.338837391e-01f, -4.338837391e-01f, -9.749279122e-01f, -7.818314825e-01f};
__device__ constexpr float kCos11[11] = {1.000000000e+00f, 8.412535328e-01f, 4.154150130e-01f, -1.423148383e-01f, -6.548607339e-01f, -9.594929736e-01f, -9.594929736e-01f, -6.548607339e-01f, -1.423148383e-01f, 4.154150130e-01f, 8.412535328e-01f};
__device__ constexpr float kSin11[11] = {0.000000000e+00f, 5.406408175e-01f, 9.096319954e-01f, 9.898214419e-01f, 7.557495744e-01f, 2.817325568e-01f, -2.817325568e-01f, -7.557495744e-01f, -9.898214419e-01f, -9.096319954e-01f, -5.406408175e-01f};
__device__ constexpr float kCos13[13] = {1.000000000e+00f, 8.854560257e-01f, 5.680647467e-01f, 1.205366803e-01f, -3.546048870e-01f, -7.485107482e-01f, -9.709418174e-01f, -9.709418174e-01f, -7.485107482e-01f, -3.546048870e-01f, 1.205366803e-01f, 5.680647467e-01f, 8.854560257e-01f};
__device__ constexpr float kSin13[13] = {0.000000000e+00f, 4.647231720e-01f, 8.229838659e-01f, 9.927088741e-01f, 9.350162427e-01f, 6.631226582e-01f, 2.393156643e-01f, -2.393156643e-01f, -6.631226582e-01f, -9.350162427e-01f, -9.927088741e-01f, -8.229838659e-01f, -4.647231720e-01f};
// radix 9 (3 x 3 as one pass): the same symmetric-pair DFT as the odd primes
__device__ constexpr float kCos9[9] = {1.000000000e+00f, 7.660444431e-01f, 1.736481777e-01f, -5.000000000e-01f, -9.396926208e-01f, -9.396926208e-01f, -5.000000000e-01f, 1.736481777e-01f, 7.660444431e-01f};
__device__ constexpr float kSin9[9] = {0.000000000e+00f, 6.427876097e-01f, 9.848077530e-01f, 8.660254038e-01f, 3.420201433e-01f, -3.420201433e-01f, -8.660254038e-01f, -9.848077530e-01f, -6.427876097e-01f};
template <int R>
__device__ __forceinline__ float odd_cos(int j) {
  if constexpr (R == 3) return kCos3[j];
  else if constexpr (R == 5) return kCos5[j];
  else if constexpr (R == 7) return kCos7[j];
  else if constexpr (R == 9) return kCos9[j];
  else if constexpr (R == 11) return kCos11[j];
  else return kCos13[j];
}
template <int R>
__device__ __forceinline__ float odd_sin(int j) {
  if constexpr (R == 3) return kSin3[j];
  else if constexpr (R == 5) return kSin5[j];
  else if constexpr (R == 7) return kSin7[j];
  else if constexpr (R == 9) return kSin9[j];
  else if constexpr (R == 11) return kSin11[j];
  else return kSin13[j];
}

// 16-point DFT as 4 x 4: four 4-point DFTs over the residues p of the index mod 4, the
// products by W16^(p k1) (conjugated for the inverse), four 4-point DFTs across p; output
// k1 + 4 k2.
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  float2 y[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float2 t[4] = {v[p], v[p + 4], v[p + 8], v[p + 12]};
    dft4<INV>(t);
#pragma unroll
    for (int k = 0; k < 4; ++k) y[p][k] = t[k];
  }
  // W16^e = (cos(pi e / 8), -sin(pi e / 8)) for e = p k1 in 0..9
  auto tw = [&](float2 a, int e) -> float2 {
    float cr, ci;
    switch (e) {
      case 1: cr = c1; ci = s1; break;
      case 2: cr = h; ci = h; break;
      case 3: cr = s1; ci = c1; break;
      case 4: cr = 0.f; ci = 1.f; break;
      case 6: cr = -h; ci = h; break;
      case 9: cr = -c1; ci = -s1; break;
      default: return a;
    }
    if (!INV) ci = -ci;
    return make_float2(a.x * cr - a.y * ci, a.x * ci + a.y * cr);
  };
#pragma unroll
  for (int p = 1; p < 4; ++p)
#pragma unroll
    for (int k = 1; k < 4; ++k) y[p][k] = tw(y[p][k], p * k);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 t[4] = {y[0][k], y[1][k], y[2][k], y[3][k]};
    dft4<INV>(t);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[k + 4 * q] = t[q];
  }
}

// Odd radix R: with a_m = x_m + x_{R-m}, b_m = x_m - x_{R-m} (m = 1 .. (R-1)/2),
//     X_0 = x_0 + sum a_m,   C_k = x_0 + sum a_m cos(2 pi m k / R),   S_k = sum b_m sin(..),
//     X_k = C_k -+ i S_k,  X_{R-k} = C_k +- i S_k   (upper signs forward, lower inverse),
// about a third of the direct form's multiplications; the roots fold into constants.
template <int R, bool INV>
__device__ __forceinline__ void dft_odd(float2* v) {
  constexpr int h = (R - 1) / 2;
  const float2 x0 = v[0];
  float2 a[h + 1], b[h + 1];
  float2 sum = x0;
#pragma unroll
  for (int m = 1; m <= h; ++m) {
    a[m] = cadd(v[m], v[R - m]);
    b[m] = csub(v[m], v[R - m]);
    sum = cadd(sum, a[m]);
  }
#pragma unroll
  for (int k = 1; k <= h; ++k) {
    float2 c = x0, sn = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 1; m <= h; ++m) {
      const int e = (m * k) % R;
      c.x = fmaf(a[m].x, odd_cos<R>(e), c.x);
      c.y = fmaf(a[m].y, odd_cos<R>(e), c.y);
      sn.x = fmaf(b[m].x, odd_sin<R>(e), sn.x);
      sn.y = fmaf(b[m].y, odd_sin<R>(e), sn.y);
    }
    const float2 minus_is = make_float2(c.x + sn.y, c.y - sn.x);   // C - i S
    const float2 plus_is = make_float2(c.x - sn.y, c.y + sn.x);    // C + i S
    v[k] = INV ? plus_is : minus_is;
    v[R - k] = INV ? minus_is : plus_is;
  }
  v[0] = sum;
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v) {
  if constexpr (R == 2) dft2<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else dft_odd<R, INV>(v);
}

// One Stockham pass over nb transforms with its input and output as functors: src(t, e)
// returns element e of transform t, dst(t, e, v) stores it.  BFAST: consecutive threads
// take consecutive transforms (column tiles; dnb is the divisor nb); otherwise consecutive
// butterflies of one transform (rows).  The first pass of a transform can read its input
// from wherever it lives (a window applied on the fly, global memory) and the last pass
// can write its output there, without a staging round trip through shared memory.
// TWS: ptw points to shared memory (a copy of the plan's twiddles the kernel made).
// The pass parameters are copied to registers first: the loop's shared-memory stores could
// alias the generic references as far as the compiler knows, and would force reloads.
template <int R, bool INV, bool BFAST, bool TWS = false, class Src, class Dst>
__device__ __forceinline__ void fft_pass_io(Src&& src, Dst&& dst, const FftPass& ps_,
                                            const float2* __restrict__ ptw, const FastDiv& dnb_,
                                            int nb, int tid, int nthr) {
  const FftPass ps = ps_;
  const FastDiv dnb = dnb_;
  const int m = (int)ps.q.d;
  const int ns = ps.ns;
  const int total = nb * m;
  const float2* __restrict__ pw = ptw + ps.tw;
  for (int idx = tid; idx < total; idx += nthr) {
    int b, j;
    if (BFAST) { j = (int)dnb.div((unsigned)idx); b = idx - j * nb; }
    else       { b = (int)ps.q.div((unsigned)idx); j = idx - b * m; }
    const int k = j - (int)ps.k.div((unsigned)j) * ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src(b, j + r * m);
    if (ns > 1) {
      const float2* w = pw + k * (R - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], TWS ? twiddle_s<INV>(w, r - 1) : twiddle<INV>(w, r - 1));
    }
    dft_r<R, INV>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst(b, base + r * ns, v[r]);
  }
}

// R16: the plan may hold radix-16 passes (kernels with the registers for them).
template <bool INV, bool BFAST, bool R16, bool TWS = false, class Src, class Dst>
__device__ __forceinline__ void fft_pass_io_r(int R, Src&& src, Dst&& dst, const FftPass& ps,
                                              const float2* __restrict__ ptw,
                                              const FastDiv& dnb, int nb, int tid, int nthr) {
  switch (R) {
    case 16:
      if constexpr (R16) fft_pass_io<16, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr);
      break;
    case 8: fft_pass_io<8, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 9: fft_pass_io<9, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 4: fft_pass_io<4, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 2: fft_pass_io<2, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 3: fft_pass_io<3, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 5: fft_pass_io<5, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 7: fft_pass_io<7, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 11: fft_pass_io<11, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    case 13: fft_pass_io<13, INV, BFAST, TWS>(src, dst, ps, ptw, dnb, nb, tid, nthr); break;
    default: break;
  }
}

// A direct (non-Bluestein) transform of nb transforms whose first pass reads src and whose
// last pass writes dst (functors as fft_pass_io); the passes between use the shared-memory
// buffers a and b (element e of transform t at t * bs + e * ks).  With last_smem the last
// pass writes to shared memory instead, and the buffer holding the result is returned
// (dst unused).  Ends with a __syncthreads().
// PAD > 0 (rows, ks == 1): element e of a slot sits at e + (e >> PAD), which spreads the
// first pass's radix-strided stores over the shared-memory banks (slots then need
// L + (L >> PAD) + 1 entries; pad_at() gives the position).  PAD < 0 (column tiles): the
// flattened index q = t * bs + e * ks sits at q + (q >> -PAD) (a buffer of q entries then
// needs q + (q >> -PAD) + 1).
template <int PAD>
__host__ __device__ __forceinline__ int pad_at(int e) { return PAD > 0 ? e + (e >> PAD) : e; }
template <int PAD>
__host__ __device__ __forceinline__ int slot_at(int t, int e, int bs, int ks) {
  if constexpr (PAD > 0) return t * bs + e + (e >> PAD);
  else if constexpr (PAD < 0) {
    const int q = t * bs + e * ks;
    return q + (q >> (-PAD));
  } else return t * bs + e * ks;
}

// TWS: the passes read their twiddles from tws, the kernel's shared-memory copy of
// pl.ptw (L - 1 entries), instead of global memory.
template <bool INV, bool BFAST, int PAD = 0, bool R16 = true, bool TWS = false, class Src,
          class Dst>
__device__ float2* fft_direct_io(Src&& src, Dst&& dst, bool last_smem, float2* a, float2* b,
                                 const FftPasses& pl, const FastDiv& dnb, int nb, int bs,
                                 int ks, const float2* tws = nullptr) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float2* ptw = TWS ? tws : pl.ptw;
  auto lds = [&](float2* buf) {
    return [buf, bs, ks](int t, int e) { return buf[slot_at<PAD>(t, e, bs, ks)]; };
  };
  auto sts = [&](float2* buf) {
    return [buf, bs, ks](int t, int e, float2 v) { buf[slot_at<PAD>(t, e, bs, ks)] = v; };
  };
  const int last = pl.nst - 1;
  for (int st = 0; st <= last; ++st) {
    const FftPass& ps = pl.p[st];
    if (st == last && !last_smem) {
      if (st == 0) fft_pass_io_r<INV, BFAST, R16, TWS>(ps.R, src, dst, ps, ptw, dnb, nb, tid, nthr);
      else fft_pass_io_r<INV, BFAST, R16, TWS>(ps.R, lds(a), dst, ps, ptw, dnb, nb, tid, nthr);
    } else if (st == 0) {
      fft_pass_io_r<INV, BFAST, R16, TWS>(ps.R, src, sts(b), ps, ptw, dnb, nb, tid, nthr);
    } else {
      fft_pass_io_r<INV, BFAST, R16, TWS>(ps.R, lds(a), sts(b), ps, ptw, dnb, nb, tid, nthr);
    }
    __syncthreads();
    if (st < last || last_smem) { float2* t = a; a = b; b = t; }
  }
  return a;
}

// A Bluestein transform (pl.chirp != NULL) of nb transforms of length pl.n as two
// length-L pass sequences: the forward sequence's first pass reads src(t, j) times c_j
// (conj(c_j) for the inverse) for j < n and zeros beyond; the kernel product rides on the
// first pass of the inverse sequence, whose last pass hands dst(t, k, X_k) the outputs
// k < n times c_k (conj(c_k) for the inverse).  With last_smem the outputs stay in shared
// memory WITHOUT that last chirp product (the caller applies it as it reads them) and the
// buffer holding them is returned.  Ends with a __syncthreads().
template <bool INV, bool BFAST, int PAD = 0, bool R16 = true, bool TWS = false, class Src,
          class Dst>
__device__ float2* fft_bluestein_io(Src&& src, Dst&& dst, bool last_smem, float2* a, float2* b,
                                    const FftPasses& pl, const FastDiv& dnb, int nb, int bs,
                                    int ks, const float2* tws = nullptr) {
  const int n = pl.n;
  const float2* __restrict__ chirp = pl.chirp;
  auto s1 = [&](int t, int j) -> float2 {
    if (j >= n) return make_float2(0.f, 0.f);
    const float2 c = __ldg(chirp + j);
    const float2 x = src(t, j);
    return INV ? cmulc(x, c) : cmul(x, c);
  };
  float2* r1 = fft_direct_io<false, BFAST, PAD, R16, TWS>(s1, [](int, int, float2) {}, true, a, b,
                                                     pl, dnb, nb, bs, ks, tws);
  float2* o = (r1 == a) ? b : a;
  const float2* __restrict__ kern = INV ? pl.kern_inv : pl.kern_fwd;
  auto s2 = [r1, kern, bs, ks](int t, int j) -> float2 {
    const float2 x = r1[slot_at<PAD>(t, j, bs, ks)];
    return cmul(x, __ldg(kern + j));
  };
  auto d2 = [&](int t, int k, float2 v) {
    if (k < n) {
      const float2 c = __ldg(chirp + k);
      dst(t, k, INV ? cmulc(v, c) : cmul(v, c));
    }
  };
  return fft_direct_io<true, BFAST, PAD, R16, TWS>(s2, d2, last_smem, r1, o, pl, dnb, nb, bs, ks,
                                                  tws);
}

}  // namespace rift2
