// Log-Gabor filter bank in the frequency domain (§II-B: "response components of the
// Log-Gabor filter"; the bank itself is the RIFT / phase-congruency one, §II-A).
//
//   fwd_rows / fwd_cols : F = FFT2(I), full complex spectrum [H][W]
//   lg_cols_inverse     : for each (s, o): column inverse DFT of F * G_so, G evaluated in
//                         registers from its closed form -> scratch [s][o][H][W]
//   lg_rows_reduce      : row inverse DFT of the four scales of each orientation, fused
//                         with the per-pixel reductions (amplitude sum A_o, MIM argmax,
//                         phase-congruency energy Er_o, spread weight / A_o, |EO_0,o|).
#include "fft.cuh"
#include "fft_reg.cuh"
#include "kernels.h"
#include "tmem.cuh"

namespace rift2 {

// Column tiles' Stockham buffers: in tiles of at most CC_NARROW columns the flattened index
// q (element e of column t at e tc + t) sits at q + (q >> CC_PAD), so that the
// radix-strided stores spread over the shared-memory banks (wider tiles spread them
// already and run faster unpadded); a buffer for q entries holds col_buf(q) either way.
constexpr int CC_PAD = 4, CC_NARROW = 3;
__host__ __device__ __forceinline__ int col_buf(int q) { return q + (q >> CC_PAD) + 1; }

// ------------------------------------------------------------------ twiddle tables
// tw[e] = exp(-2 pi i e / n), computed in double precision (the only FP64 step).
__global__ void twiddle_gen(float2* tw, int n) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s, c;
  sincospi(-2.0 * (double)e / (double)n, &s, &c);
  tw[e] = make_float2((float)c, (float)s);
}

// Per-pass twiddles of a Stockham plan: pass st (radix R, ns) holds W_(ns R)^(k r) =
// tw[k r L / (ns R)] for k < ns, 1 <= r < R at ptw[off_st + k (R - 1) + r - 1] (a gather
// from the FP64-generated length-L table, so the values are the table's own).
__global__ void pass_twiddle_gather(float2* __restrict__ ptw, const float2* __restrict__ tw,
                                    int L, PassDims pd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pd.total) return;
  int st = 0;
  while (st + 1 < pd.nst && i >= pd.off[st + 1]) ++st;
  const int e = i - pd.off[st], R = pd.R[st], ns = pd.ns[st];
  const int k = e / (R - 1), r = e - k * (R - 1) + 1;
  ptw[i] = tw[(long long)k * r * (L / (ns * R))];
}

// Bluestein tables (FP64 arithmetic, rounded once to FP32).  c_j = exp(-i pi j^2 / n) with
// j^2 reduced modulo 2n first (exact in 64-bit integers), so the argument stays small.
__global__ void chirp_gen(float2* c32, double2* c64, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long r = ((long long)j * j) % (2ll * n);
  double sn, cs;
  sincospi(-(double)r / (double)n, &sn, &cs);
  c64[j] = make_double2(cs, sn);
  c32[j] = make_float2((float)cs, (float)sn);
}
__global__ void twiddle64_gen(double2* tw, int m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  double sn, cs;
  sincospi(-2.0 * (double)e / (double)m, &sn, &cs);
  tw[e] = make_double2(cs, sn);
}
// kern_fwd[k] = (1/m) sum_j conj(c~_j) W_m^(jk), kern_inv[k] = (1/m) sum_j c~_j W_m^(jk),
// c~ the cyclic extension of c to length m (c~_j = c_j, c~_(m-j) = c_j for 0 < j < n, zero
// between): a direct DFT in FP64, one output per thread.
__global__ void bluestein_kern_gen(float2* kf, float2* ki, const double2* __restrict__ c64,
                                   const double2* __restrict__ tw64, int n, int m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  double fr = 0.0, fi = 0.0, ir = 0.0, ii = 0.0;
  for (int j = 0; j < m; ++j) {
    const int jj = (j < n) ? j : ((j > m - n) ? m - j : -1);
    if (jj < 0) continue;
    const double2 c = c64[jj];
    const double2 w = tw64[(int)(((long long)j * k) % m)];
    // conj(c) w and c w
    fr += c.x * w.x + c.y * w.y;
    fi += c.x * w.y - c.y * w.x;
    ir += c.x * w.x - c.y * w.y;
    ii += c.x * w.y + c.y * w.x;
  }
  const double s = 1.0 / (double)m;
  kf[k] = make_float2((float)(fr * s), (float)(fi * s));
  ki[k] = make_float2((float)(ir * s), (float)(ii * s));
}

void launch_bluestein_tables(float2* chirp, float2* kf, float2* ki, double2* c64, double2* tw64,
                             int n, int m, cudaStream_t st) {
  chirp_gen<<<(n + 255) / 256, 256, 0, st>>>(chirp, c64, n);
  twiddle64_gen<<<(m + 255) / 256, 256, 0, st>>>(tw64, m);
  bluestein_kern_gen<<<(m + 127) / 128, 128, 0, st>>>(kf, ki, c64, tw64, n, m);
}

// ------------------------------------------------------------------ forward 2-D DFT
// The large DC term dominates the rounding error of an FP32 FFT.  Each 1-D transform
// therefore runs on its input minus the input's mean and gets its bin 0 back as the
// input sum afterwards: DFT(x) = DFT(x - m) + m N delta_0 exactly, so the result is the
// same transform with an error set by the non-DC content only.
__device__ __forceinline__ void seg_means(const float2* a, int nseg, int len, int es, int ss,
                                          float2* mean) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int g = warp; g < nseg; g += nw) {
    float sx = 0.f, sy = 0.f;
    for (int i = lane; i < len; i += 32) {
      float2 v = a[g * ss + i * es];
      sx += v.x;
      sy += v.y;
    }
    for (int d = 16; d > 0; d >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, d);
      sy += __shfl_xor_sync(0xffffffffu, sy, d);
    }
    if (lane == 0) mean[g] = make_float2(sx / len, sy / len);
  }
}

// Rows of real images: tile of `tr` rows (fg.tile of the image), complex FFT with zero
// imaginary part.  Image blockIdx.y of the group; dense (if not NULL) holds the images
// packed like the spectrum.
__global__ void __launch_bounds__(512, 1) fwd_rows(ImgPtrs ip, const float* __restrict__ dense,
                                                float2* __restrict__ spec,
                                                const __grid_constant__ Group gr,
                                                const __grid_constant__ FftGroup fg) {
  extern __shared__ float2 sm[];
  __shared__ float2 mean[256];
  const int img = blockIdx.y;
  const int H = gr.H[img], W = gr.W[img], tr = fg.tile[img];
  const FftPasses& pw = *fg.pass[img];
  const int r0 = blockIdx.x * tr;
  if (r0 >= H) return;
  const int nel = tr * W;
  const int L = pw.L;   // shared-memory slot of one row transform (> W for Bluestein plans)
  float2* a = sm;
  float2* b = sm + tr * L;
  const float* src = dense ? dense + gr.poff[img] : ip.img[img];
  const long long pitch = dense ? W : ip.pitch[img];
  const FastDiv dW((unsigned)W);
  for (int i = threadIdx.x; i < nel; i += blockDim.x) {
    const int rr = (int)dW.div((unsigned)i), x = i - rr * W, r = r0 + rr;
    float v = (r < H) ? __ldg(src + (size_t)r * pitch + x) : 0.f;
    a[rr * L + x] = make_float2(v, 0.f);
  }
  __syncthreads();
  seg_means(a, tr, W, 1, L, mean);
  __syncthreads();
  // the first pass reads the rows minus their means, the last pass restores bin 0 and
  // stores the spectrum rows
  float2* dst = spec + gr.poff[img];
  auto src_m = [&](int t, int e) -> float2 {
    const float2 x = a[t * L + e];
    return make_float2(x.x - mean[t].x, x.y);
  };
  auto out = [&](int t, int e, float2 v) {
    if (e == 0) v.x += mean[t].x * W;
    if (r0 + t < H) dst[(size_t)(r0 + t) * W + e] = v;
  };
  if (!pw.chirp) fft_direct_io<false, false>(src_m, out, false, a, b, pw, fg.dtile[img], tr, L, 1);
  else fft_bluestein_io<false, false>(src_m, out, false, a, b, pw, fg.dtile[img], tr, L, 1);
}

// Columns, in place on spec [H][W]: tile of `tc` columns (fg.tile of the image).
__global__ void __launch_bounds__(512, 1) fwd_cols(float2* __restrict__ spec,
                                                const __grid_constant__ Group gr,
                                                const __grid_constant__ FftGroup fg) {
  extern __shared__ float2 sm[];
  __shared__ float2 mean[64];
  const int img = blockIdx.y;
  const int H = gr.H[img], W = gr.W[img], tc = fg.tile[img];
  const FftPasses& ph = *fg.pass[img];
  const int c0 = blockIdx.x * tc;
  if (c0 >= W) return;
  const int nel = H * tc;
  float2* a = sm;
  float2* b = sm + col_buf(ph.L * tc);   // [ph.L][tc] each (padded): a column's slot is ph.L long
  float2* base = spec + gr.poff[img];
  const FastDiv& dtc = fg.dtile[img];
  for (int i = threadIdx.x; i < nel; i += blockDim.x) {
    const int v = (int)dtc.div((unsigned)i), c = i - v * tc;
    a[i] = (c0 + c < W) ? base[(size_t)v * W + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  seg_means(a, tc, H, tc, 1, mean);
  __syncthreads();
  // the first pass reads the columns minus their means, the last pass restores bin 0 and
  // writes the columns back
  auto src_m = [&](int t, int e) -> float2 {
    const float2 x = a[e * tc + t];
    return make_float2(x.x - mean[t].x, x.y - mean[t].y);
  };
  auto out = [&](int t, int e, float2 v) {
    if (e == 0) {
      v.x += mean[t].x * H;
      v.y += mean[t].y * H;
    }
    if (c0 + t < W) base[(size_t)e * W + c0 + t] = v;
  };
  if (tc <= CC_NARROW) {
    if (!ph.chirp) fft_direct_io<false, true, -CC_PAD>(src_m, out, false, a, b, ph, dtc, tc, 1, tc);
    else fft_bluestein_io<false, true, -CC_PAD>(src_m, out, false, a, b, ph, dtc, tc, 1, tc);
  } else {
    if (!ph.chirp) fft_direct_io<false, true>(src_m, out, false, a, b, ph, dtc, tc, 1, tc);
    else fft_bluestein_io<false, true>(src_m, out, false, a, b, ph, dtc, tc, 1, tc);
  }
}

constexpr int REG_NT = 256;   // threads per CTA of the register-tiled row kernels

// ------------------------------------------------------- register-tiled forward DFT
// Sum over the T threads of one transform group (T <= 32: shuffles inside the group's
// lanes; T > 32: through shared memory, one slot per thread).
template <int T>
__device__ __forceinline__ float2 group_sum(float2 v, float2* red) {
  if constexpr (T <= 32) {
#pragma unroll
    for (int d = 1; d < T; d <<= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, d);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, d);
    }
    return v;
  } else {
    const int t = threadIdx.x % T, g0 = threadIdx.x - t;
    red[threadIdx.x] = v;
    __syncthreads();
    float2 a = make_float2(0.f, 0.f);
    for (int k = 0; k < T; ++k) {
      const float2 b = red[g0 + k];
      a.x += b.x;
      a.y += b.y;
    }
    __syncthreads();
    return a;
  }
}

// Rows of real images, one group of T threads per row, mean removed and restored.
template <int WN>
__global__ void __launch_bounds__(RegShape<WN>::NT) fwd_rows_reg(ImgPtrs ip, const float* __restrict__ dense,
                                                       float2* __restrict__ spec, int H,
                                                       const float2* __restrict__ tww) {
  using S = RegShape<WN>;
  constexpr int T = S::T, ROWS = S::NT / T, E = WN / T, XS = XBuf<WN>::SIZE;
  extern __shared__ float2 sm[];   // [ROWS][XS] exchange + [NT] reduction slots
  float2* red = sm + ROWS * XS;
  const int img = blockIdx.y;
  const int grp = threadIdx.x / T, t = threadIdx.x % T;
  const int row = blockIdx.x * ROWS + grp;
  const bool live = row < H;
  const float* src = dense ? dense + (size_t)img * H * WN : ip.img[img];
  const long long pitch = dense ? WN : ip.pitch[img];
  float xr[E];
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < E; ++k) {   // the first pass's inputs: x = t + T k
    xr[k] = live ? __ldg(src + (size_t)row * pitch + t + T * k) : 0.f;
    sum += xr[k];
  }
  const float mean = group_sum<T>(make_float2(sum, 0.f), red).x / WN;
  float2* xb = sm + grp * XS;
  auto ld = [&](int, int r, int) -> float2 { return make_float2(xr[r] - mean, 0.f); };
  float2* dst = spec + ((size_t)img * H + row) * WN;
  auto st = [&](int x, float2 val) {
    if (x == 0) val.x += mean * WN;
    if (live) dst[x] = val;
  };
  auto sync = [] {
    if constexpr (T <= 32) __syncwarp();
    else __syncthreads();
  };
  group_fft<WN, T, S::R0, S::R1, S::R2, false>(xb, t, tww, ld, st, sync);
}

// Columns of the spectrum in place, COLS columns per CTA, mean removed and restored.
template <int HN>
__global__ void __launch_bounds__(ColShape<HN>::NT) fwd_cols_reg(float2* __restrict__ spec, int W,
                                                                const float2* __restrict__ twh) {
  using S = ColShape<HN>;
  constexpr int T = S::T, NT = S::NT, COLS = NT / T, E = HN / T, XS = ColStride<HN, COLS>::SIZE;
  extern __shared__ float2 sm[];   // [COLS][XS] + [NT] reduction slots
  float2* red = sm + COLS * XS;
  const int img = blockIdx.y;
  const int c0 = blockIdx.x * COLS;
  float2* base = spec + (size_t)img * HN * W;
  {
    // the tile's loads all in flight together, then into the exchange buffers
    constexpr int NF = HN * COLS / NT;
    float2 fx[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const int i = threadIdx.x + k * NT;
      const int v = i / COLS, c = i % COLS;
      fx[k] = (c0 + c < W) ? base[(size_t)v * W + c0 + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const int i = threadIdx.x + k * NT;
      sm[(i % COLS) * XS + xpad(i / COLS)] = fx[k];
    }
  }
  __syncthreads();
  const int col = threadIdx.x / T, t = threadIdx.x % T;
  float2* xb = sm + col * XS;
  float2 s = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const float2 v = xb[xpad(t + T * k)];
    s.x += v.x;
    s.y += v.y;
  }
  const float2 tot = group_sum<T>(s, red);
  const float2 mean = make_float2(tot.x / HN, tot.y / HN);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    float2& v = xb[xpad(t + T * k)];
    v.x -= mean.x;
    v.y -= mean.y;
  }
  auto sync = [] {
    if constexpr (T <= 32) __syncwarp();
    else __syncthreads();
  };
  sync();
  auto st = [&](int v, float2 val) {
    if (v == 0) {
      val.x += tot.x;
      val.y += tot.y;
    }
    xb[xpad(v)] = val;
  };
  group_fft_xb<HN, T, S::R0, S::R1, S::R2, false>(xb, t, twh, st, sync);
  __syncthreads();
  {
    // thread (row v0, column c) writes rows v0 + RSTEP k: a warp stores row segments
    constexpr int RSTEP = NT / COLS;
    const int c = threadIdx.x % COLS, v0 = threadIdx.x / COLS;
    if (c0 + c < W) {
#pragma unroll 8
      for (int k = 0; k < HN / RSTEP; ++k) {
        const int v = v0 + RSTEP * k;
        base[(size_t)v * W + c0 + c] = sm[c * XS + xpad(v)];
      }
    }
  }
}

// ------------------------------------------------------------- log-Gabor transfer
// Radial part of scale s at squared radius r2 (cycles/px)^2:
//   exp(-(ln r - ln f_s)^2 / (2 ln^2 sigma_onf)) / (1 + (r^2 / c^2)^n), zero at DC.
// The logarithm, exponential and quotient use the SFU approximations (relative error of
// the filter value a few 1e-7; (r/c)^(2n) stays below 1e6 on the grid).  (r/c)^(2n) is
// taken by square-and-multiply over the bits of n: with LP > 0 the order n = LP is a
// compile-time constant (the loop unrolls into the same products), LP = 0 reads it from
// the parameters.
template <int LP = 0>
__device__ __forceinline__ float lg_radial(float r2, float log_fs, const KParams& kp) {
  if (r2 <= 0.f) return 0.f;
  float lr = 0.5f * __logf(r2);
  float d = lr - log_fs;
  float x = r2 * kp.inv_lp_c2;   // (r/c)^2
  float p = 1.f, base = x;
  if constexpr (LP > 0) {
#pragma unroll
    for (int e = LP; e > 0; e >>= 1) {
      if (e & 1) p *= base;
      base *= base;
    }
  } else {
    for (int e = kp.lp_order; e > 0; e >>= 1) {
      if (e & 1) p *= base;
      base *= base;
    }
  }
  return __fdividef(__expf(-d * d * kp.inv_2ls2), 1.f + p);
}

// Angular raised-cosine window.  With c = cos(theta - theta_o) (theta = atan2(-v, u)),
// the window (1 + cos(3 dtheta)) / 2 for |dtheta| < pi/3 equals (1 + c)(2c - 1)^2 / 2 =
// 2c^3 - 1.5c + 0.5 (triple-angle identity, cos 3x = 4c^3 - 3c), evaluated as
// c (2c^2 - 1.5) + 0.5 with two fused multiply-adds, and 0 beyond.  c = (fu cos_o -
// fv sin_o) / r is formed from fuco = fu cos_o, fv, sin_o and ri = 1/r (0 at DC).  Every kernel that evaluates the
// window, and the zero-column table, goes through lg_rinv and lg_window with explicitly
// rounded products, so they agree bit for bit on which bins are zero.
__device__ __forceinline__ float lg_rinv(float fu, float fv) {
  const float r2 = fmaf(fv, fv, __fmul_rn(fu, fu));
  return (r2 > 0.f) ? rsqrtf(r2) : 0.f;
}
// The cubic is exactly 0 at c = 0.5 (fmaf(0.5, fmaf(1, 0.5, -1.5), 0.5) = 0 with exact
// intermediate values), so clamping c below at 0.5 gives the window's zero without a branch.
__device__ __forceinline__ float lg_window(float fuco, float fv, float so, float ri) {
  const float c = fmaxf(__fmul_rn(fmaf(-fv, so, fuco), ri), 0.5f);
  return fmaf(c, fmaf(2.f * c, c, -1.5f), 0.5f);
}

// Columns u whose angular window is zero on every row: S_o(u, v) = 0 for all v, so the
// filtered spectrum column and its inverse transform are exactly zero.  The one-sided
// wedge of each orientation misses about a third of all (o, u) columns.  Evaluated with
// the very expression the column pass uses, so the table is exact for that pass.
__global__ void angular_zero_cols(int H, int W, KParams kp, unsigned char* __restrict__ zc) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y;
  if (u >= W) return;
  const float fu = fftfreq(u, W);
  const float fuco = __fmul_rn(fu, kp.cos_o[o]), so = kp.sin_o[o];
  bool zero = true;
  for (int v = 0; v < H && zero; ++v) {
    const float fv = fftfreq(v, H);
    zero = (lg_window(fuco, fv, so, lg_rinv(fu, fv)) == 0.f);
  }
  zc[o * W + u] = zero ? 1 : 0;
}

void launch_zero_cols(int H, int W, const KParams& kp, unsigned char* zc, cudaStream_t st) {
  angular_zero_cols<<<dim3((W + 127) / 128, NO), 128, 0, st>>>(H, W, kp, zc);
}

// Column pass of the inverse for the six orientations of scale blockIdx.y.
// smem: base (F * R_s) [H][tc], a, b [L][tc] each (padded, col_buf), with tw_smem the
// plan's pass twiddles [L - 1] (read by every butterfly of every pass: from shared memory
// instead of global memory, where the launch's tiles leave room for them), fftfreq(v, H)
// [H].  A tile whose columns all have a zero angular window for an orientation (fg.zc)
// writes nothing for it.
__global__ void __launch_bounds__(512, 1) lg_cols_inverse(const float2* __restrict__ spec,
                                                       float2* __restrict__ scratch,
                                                       const __grid_constant__ Group gr,
                                                       const __grid_constant__ FftGroup fg,
                                                       KParams kp, int tw_smem) {
  extern __shared__ float2 sm[];
  const int s = blockIdx.y;
  const int img = blockIdx.z;
  const int H = gr.H[img], W = gr.W[img], tc = fg.tile[img];
  const FftPasses& ph = *fg.pass[img];
  const int c0 = blockIdx.x * tc;
  if (c0 >= W) return;
  const size_t P = (size_t)H * W;
  const int nel = H * tc;
  const int nl = col_buf(ph.L * tc);   // transform slots ph.L long (> H for Bluestein plans), padded
  float2* base = sm;
  float2* a = sm + nel;
  float2* b = sm + nel + nl;
  float2* tws = sm + nel + 2 * nl;
  float* fvt = reinterpret_cast<float*>(tws + (tw_smem ? ph.L : 0));   // fftfreq(v, H) per row
  __shared__ float fut[16];                               // fftfreq(u, W) per column
  if (tw_smem)
    for (int i = threadIdx.x; i < ph.L - 1; i += blockDim.x) tws[i] = __ldg(ph.ptw + i);
  const float2* twp = tw_smem ? tws : ph.ptw;
  const float2* F = spec + gr.poff[img];
  const float log_fs = kp.log_fs[s];
  const float inv_hw = 1.f / ((float)H * (float)W);   // the inverse DFT's normalisation
  const FastDiv& dtc = fg.dtile[img];
  for (int v = threadIdx.x; v < H; v += blockDim.x) fvt[v] = fftfreq(v, H);
  if (threadIdx.x < tc) fut[threadIdx.x] = fftfreq(c0 + threadIdx.x, W);
  __syncthreads();
  for (int i = threadIdx.x; i < nel; i += blockDim.x) {
    const int v = (int)dtc.div((unsigned)i), c = i - v * tc, u = c0 + c;
    float2 f = make_float2(0.f, 0.f);
    if (u < W) {
      const float fu = fut[c], fv = fvt[v];
      const float rs = lg_radial(fu * fu + fv * fv, log_fs, kp) * inv_hw;
      const float2 x = __ldg(F + (size_t)v * W + u);
      f = make_float2(x.x * rs, x.y * rs);
    }
    base[i] = f;
  }
  const unsigned char* __restrict__ zc = fg.zc[img];
  for (int o = 0; o < NO; ++o) {
    // a tile whose columns all have a zero window for o has nothing to transform or
    // store: the row pass reads those columns as zeros from the same table
    const int t = threadIdx.x;
    const bool zt = t >= tc || c0 + t >= W || (zc && zc[o * W + c0 + t]);
    if (__syncthreads_and(zt)) continue;
    const float co = kp.cos_o[o], so = kp.sin_o[o];
    float2* dst = scratch + (size_t)NS * NO * gr.poff[img] + ((size_t)s * NO + o) * P;
    // the first pass reads F R_s and applies the window, the last pass writes the
    // responses to HBM (through the chirp products and the convolution for Bluestein
    // heights)
    auto src = [&](int t, int e) -> float2 {
      if (c0 + t >= W) return make_float2(0.f, 0.f);
      const float fu = fut[t], fv = fvt[e];
      const float g = lg_window(__fmul_rn(fu, co), fv, so, lg_rinv(fu, fv));
      const float2 x = base[e * tc + t];
      return make_float2(x.x * g, x.y * g);
    };
    auto out = [&](int t, int e, float2 v) {
      if (c0 + t < W) dst[(size_t)e * W + c0 + t] = v;
    };
    if (tc <= CC_NARROW) {
      if (!ph.chirp)
        fft_direct_io<true, true, -CC_PAD, true, true>(src, out, false, a, b, ph, dtc, tc, 1, tc, twp);
      else
        fft_bluestein_io<true, true, -CC_PAD, true, true>(src, out, false, a, b, ph, dtc, tc, 1, tc, twp);
    } else {
      if (!ph.chirp)
        fft_direct_io<true, true, 0, true, true>(src, out, false, a, b, ph, dtc, tc, 1, tc, twp);
      else
        fft_bluestein_io<true, true, 0, true, true>(src, out, false, a, b, ph, dtc, tc, 1, tc, twp);
    }
    // the next orientation overwrites a/b only after everyone has stored (loop-top sync)
  }
}

// Per-pixel reductions over the Ns scales of one orientation (phase-congruency model of
// §II-A; MIM amplitude sum of §II-B).  z[s] = EO_{s,o}(x): the column pass applies the
// inverse DFT's 1/(HW) to the filtered spectrum, so the row pass output is EO itself.
//   A = sum_s |EO_s|, Er = sum_s (E mE + O mO - |E mO - O mE|) with (mE, mO) the unit mean
//   phase vector, q = w / A with the frequency-spread weight w, an0 = |EO_0|.
// Square roots, reciprocals and the exponential use the SFU approximations (relative
// error a few 1e-7), well inside the 1e-4 value tolerance and the 1e-5 near-tie margin.
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

__device__ __forceinline__ void reduce_pixel(const float2 (&z)[NS], const KParams& kp,
                                             float& er, float& q, float& an0, float& sum_an) {
  float e[NS], od[NS];
  float2 sum_eo = z[0];
  float max_an = 0.f;
  sum_an = 0.f;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    e[s] = z[s].x;
    od[s] = z[s].y;
    const float an = fast_sqrt(e[s] * e[s] + od[s] * od[s]);
    if (s == 0) an0 = an;
    if (s > 0) sum_eo = cadd(sum_eo, z[s]);
    sum_an += an;
    max_an = fmaxf(max_an, an);
  }
  const float sum_e = sum_eo.x, sum_o = sum_eo.y;
  const float ixe = __fdividef(1.f, fast_sqrt(sum_e * sum_e + sum_o * sum_o) + kp.eps);
  const float me = sum_e * ixe, mo = sum_o * ixe;
  // sum_s (E_s mE + O_s mO) = mE sum E + mO sum O: the projections once, on the sums
  float energy = fmaf(sum_e, me, sum_o * mo);
#pragma unroll
  for (int s = 0; s < NS; ++s) energy -= fabsf(e[s] * mo - od[s] * me);
  const float width = (sum_an * __fdividef(1.f, max_an + kp.eps) - 1.f) * kp.inv_ns1;
  const float wgt = __fdividef(1.f, 1.f + __expf((kp.cutoff - width) * kp.g));
  er = energy;
  q = (sum_an > 0.f) ? wgt * __fdividef(1.f, sum_an) : 0.f;
}

// Row pass of the inverse with the fused per-pixel reductions.  One row per CTA;
// for each orientation the four scales are transformed together.
constexpr int RR_MAXPIX = 8;   // pixels per thread: W <= 8 * blockDim.x
// Row transforms' shared-memory slots: element e at e + (e >> RR_PAD) (conflict-free radix
// strides in the first pass), so a slot of a length-L transform holds row_slot(L) entries.
constexpr int RR_PAD = 4;
__host__ __device__ __forceinline__ int row_slot(int L) { return L + (L >> RR_PAD) + 1; }

// HALVES: the four scales are transformed two at a time and the first two parked in
// shared memory ([2][W], chirp applied), which halves the transform buffers (two CTAs per
// SM for wider rows, and rows too wide for four scales at once without the split pass).
template <bool HALVES>
__global__ void __launch_bounds__(512, 2) lg_rows_reduce(const float2* __restrict__ scratch,
                                                      const __grid_constant__ Group gr,
                                                      const __grid_constant__ FftGroup fg,
                                                      KParams kp,
                                                      float* __restrict__ er_out,
                                                      float* __restrict__ q_out,
                                                      float* __restrict__ an0_out,
                                                      float* __restrict__ amp_out,
                                                      unsigned char* __restrict__ mim_out,
                                                      int mim_pitch) {
  extern __shared__ float2 sm[];
  constexpr int NT = HALVES ? NS / 2 : NS;   // transforms per pass sequence
  const int row = blockIdx.x;
  const int img = blockIdx.y;
  const int H = gr.H[img], W = gr.W[img];
  if (row >= H) return;
  const FftPasses& pw = *fg.pass[img];
  const unsigned char* __restrict__ zc = fg.zc[img];
  const float2* __restrict__ chirp = pw.chirp;
  const int L = row_slot(pw.L);   // a row transform's padded slot (pw.L > W for Bluestein)
  float2* a = sm;
  float2* b = sm + NT * L;
  float2* stash = sm + 2 * NT * L;   // HALVES: scales 0 and 1 of the row
  const size_t P = (size_t)H * W;
  const size_t pb = (size_t)gr.poff[img];
  float best[RR_MAXPIX];
  unsigned besto = 0;   // the argmax orientation of pixel k in bits 3k..3k+2
#pragma unroll
  for (int k = 0; k < RR_MAXPIX; ++k) best[k] = -1.f;

  const float2* rows = scratch + NS * NO * pb + (size_t)row * W;
  auto nop = [](int, int, float2) {};
  // the transforms of scales s0 .. s0 + NT - 1: the first pass loads their rows from HBM
  // (zero-window columns are not read: the column pass may not have written them); for a
  // Bluestein width the result still lacks its chirp product, applied as it is read
  auto transform = [&](int o, int s0) -> float2* {
    auto src = [&](int t, int e) -> float2 {
      if (zc[o * W + e]) return make_float2(0.f, 0.f);
      return __ldg(rows + ((size_t)(s0 + t) * NO + o) * P + e);
    };
    return !chirp ? fft_direct_io<true, false, RR_PAD, false>(src, nop, true, a, b, pw, fg.dtile[img], NT, L, 1)
                  : fft_bluestein_io<true, false, RR_PAD, false>(src, nop, true, a, b, pw, fg.dtile[img], NT, L, 1);
  };
  for (int o = 0; o < NO; ++o) {
    float2* res = transform(o, 0);
    if constexpr (HALVES) {
      for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const float2 c = chirp ? __ldg(chirp + x) : make_float2(1.f, 0.f);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const float2 v = res[t * L + pad_at<RR_PAD>(x)];
          stash[t * W + x] = chirp ? cmulc(v, c) : v;
        }
      }
      __syncthreads();
      res = transform(o, NT);
    }
#pragma unroll
    for (int k = 0; k < RR_MAXPIX; ++k) {
      int x = threadIdx.x + k * blockDim.x;
      if (x >= W) break;
      float2 z[NS];
      const float2 c = chirp ? __ldg(chirp + x) : make_float2(1.f, 0.f);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (HALVES && s < NT) {
          z[s] = stash[s * W + x];
        } else {
          const float2 v = res[(s - (HALVES ? NT : 0)) * L + pad_at<RR_PAD>(x)];
          z[s] = chirp ? cmulc(v, c) : v;
        }
      }
      float energy, q, an0, sum_an;
      reduce_pixel(z, kp, energy, q, an0, sum_an);
      size_t off = NO * pb + o * P + (size_t)row * W + x;
      er_out[off] = energy;
      q_out[off] = q;
      an0_out[off] = an0;
      if (amp_out) amp_out[off] = sum_an;
      if (sum_an > best[k]) {   // lowest o on ties
        best[k] = sum_an;
        besto = (besto & ~(7u << (3 * k))) | ((unsigned)o << (3 * k));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < RR_MAXPIX; ++k) {
    int x = threadIdx.x + k * blockDim.x;
    if (x >= W) break;
    mim_out[((size_t)gr.mrow[img] + row) * mim_pitch + x] = (unsigned char)((besto >> (3 * k)) & 7u);
  }
}

// Row pass for rows too wide for lg_rows_reduce: each CTA transforms one (row, scale) for
// the six orientations and writes the responses back in place (zero-window columns are
// read as zeros and every column is written), then lg_rows_pixels reduces each pixel from
// its 24 responses exactly as lg_rows_reduce does.
__global__ void __launch_bounds__(512) lg_rows_split(float2* __restrict__ scratch,
                                                     const __grid_constant__ Group gr,
                                                     const __grid_constant__ FftGroup fg) {
  extern __shared__ float2 sm[];
  const int row = blockIdx.x, s = blockIdx.y, img = blockIdx.z;
  const int H = gr.H[img], W = gr.W[img];
  if (row >= H) return;
  const FftPasses& pw = *fg.pass[img];
  const unsigned char* __restrict__ zc = fg.zc[img];
  float2* a = sm;
  const int Ls = row_slot(pw.L);
  float2* b = sm + Ls;
  const size_t P = (size_t)H * W;
  for (int o = 0; o < NO; ++o) {
    float2* rowp = scratch + (size_t)NS * NO * gr.poff[img] + ((size_t)s * NO + o) * P +
                   (size_t)row * W;
    // in place: the first pass reads the row (barriers separate it from the last pass,
    // which writes the row back)
    auto src = [&](int, int e) -> float2 {
      return zc[o * W + e] ? make_float2(0.f, 0.f) : rowp[e];
    };
    auto out = [&](int, int e, float2 v) { rowp[e] = v; };
    if (!pw.chirp) fft_direct_io<true, false, RR_PAD>(src, out, false, a, b, pw, fg.dtile[img], 1, Ls, 1);
    else fft_bluestein_io<true, false, RR_PAD>(src, out, false, a, b, pw, fg.dtile[img], 1, Ls, 1);
  }
}

__global__ void __launch_bounds__(256) lg_rows_pixels(const float2* __restrict__ scratch,
                                                      const __grid_constant__ Group gr,
                                                      KParams kp,
                                                      float* __restrict__ er_out,
                                                      float* __restrict__ q_out,
                                                      float* __restrict__ an0_out,
                                                      float* __restrict__ amp_out,
                                                      unsigned char* __restrict__ mim_out,
                                                      int mim_pitch) {
  const int img = blockIdx.y;
  const int W = gr.W[img];
  const long long P = gr.P(img);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const size_t pb = (size_t)gr.poff[img];
  float best = -1.f;
  int besto = 0;
  for (int o = 0; o < NO; ++o) {
    float2 z[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) z[s] = __ldg(scratch + NS * NO * pb + ((size_t)s * NO + o) * P + i);
    float energy, q, an0, sum_an;
    reduce_pixel(z, kp, energy, q, an0, sum_an);
    const size_t off = NO * pb + o * P + i;
    er_out[off] = energy;
    q_out[off] = q;
    an0_out[off] = an0;
    if (amp_out) amp_out[off] = sum_an;
    if (sum_an > best) { best = sum_an; besto = o; }   // lowest o on ties
  }
  const long long y = i / W, x = i - y * W;
  mim_out[((size_t)gr.mrow[img] + y) * mim_pitch + x] = (unsigned char)besto;
}

// ------------------------------------------------------- register-tiled fast path
// Column pass for power-of-two H: one group of T threads per column, COLS columns per
// CTA.  F * R_s is staged once per CTA (coalesced rows of COLS columns); each orientation
// multiplies the angular window in the first FFT pass, and the results are written back
// through the exchange buffers as coalesced row segments.

template <int H>
__global__ void __launch_bounds__(ColShape<H>::NT) lg_cols_reg(const float2* __restrict__ spec,
                                                              float2* __restrict__ scratch, int W,
                                                              const float2* __restrict__ twh,
                                                              KParams kp,
                                                              const unsigned char* __restrict__ zc) {
  using S = ColShape<H>;
  constexpr int T = S::T, NT = S::NT;
  constexpr int COLS = NT / T;
  constexpr int E = H / T;
  constexpr int XS = ColStride<H, COLS>::SIZE;
  extern __shared__ float2 sm[];
  float2* base = sm;               // [COLS][XS]  F * R_s
  float2* xbuf = sm + COLS * XS;   // [COLS][XS]  exchange buffers
  __shared__ unsigned char zcs[NO][COLS];   // zero-window flags of this CTA's columns
  const int s = blockIdx.y, img = blockIdx.z;
  const int c0 = blockIdx.x * COLS;
  const int tid = threadIdx.x;
  // The CTA's spectrum tile (H rows x COLS columns) is loaded into registers first, all
  // loads in flight together; their latency hides behind the set-up below.
  const float2* F = spec + (size_t)img * H * W;
  static_assert((H * COLS) % NT == 0, "fill tile");
  constexpr int NF = H * COLS / NT;
  float2 fx[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int i = tid + k * NT;
    const int v = i / COLS, c = i % COLS, u = c0 + c;
    fx[k] = (u < W) ? __ldg(F + (size_t)v * W + u) : make_float2(0.f, 0.f);
  }
  for (int i = tid; i < NO * COLS; i += NT) {
    const int o = i / COLS, c = i % COLS;
    zcs[o][c] = (c0 + c < W) ? zc[o * W + c0 + c] : 1;
  }
  const int col = tid / T, t = tid % T;
  const int u = c0 + col;
  float2* xb = xbuf + col * XS;
  const float2* bc = base + col * XS;
  const float fu = (u < W) ? fftfreq(u, W) : 0.f;
  // The first FFT pass reads this thread's elements v = t + T r (r < E, one butterfly of
  // radix E): 1/r of those bins stays in registers across the six windows, and each
  // window is applied as the pass loads its input.
  static_assert(E == S::R0, "first pass: one butterfly of radix E per thread");
  float ri[E];
#pragma unroll
  for (int r = 0; r < E; ++r) ri[r] = (u < W) ? lg_rinv(fu, fftfreq(t + T * r, H)) : 0.f;
  // fftfreq(t + T r, H) as t / H plus a constant per r (exact: H is a power of two and
  // t + T r < H / 2 exactly when r < E / 2)
  const float fv0 = (float)t * (1.f / H);
  // F * R_s * 1/(HW) into shared memory
  const float log_fs = kp.log_fs[s];
  const float inv_hw = 1.f / ((float)H * (float)W);   // the inverse DFT's normalisation
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int i = tid + k * NT;
    const int v = i / COLS, c = i % COLS, uu = c0 + c;
    float2 f = make_float2(0.f, 0.f);
    if (uu < W) {
      const float fuu = fftfreq(uu, W), fv = fftfreq(v, H);
      const float rs = lg_radial(fuu * fuu + fv * fv, log_fs, kp) * inv_hw;
      f = make_float2(fx[k].x * rs, fx[k].y * rs);
    }
    base[c * XS + xpad(v)] = f;
  }
  __syncthreads();
  auto sync = [] {
    if constexpr (T <= 32) __syncwarp();
    else __syncthreads();
  };
  for (int o = 0; o < NO; ++o) {
    const float fuco = __fmul_rn(fu, kp.cos_o[o]), so = kp.sin_o[o];
    // a column whose window is zero everywhere transforms to zero: skip it, and leave it
    // unwritten (the row pass reads the same table and substitutes zeros).  The skip is
    // taken per synchronisation domain of the FFT: a warp, or the CTA when T > 32.
    const bool zcol = zcs[o][col] != 0;
    bool skip;
    if constexpr (T <= 32) skip = __all_sync(0xffffffffu, zcol);
    else skip = __syncthreads_and(zcol);
    if (!skip) {
      auto ld = [&](int, int r, int v) -> float2 {
        const float fv = fv0 + (float)(T * r - (2 * r >= E ? H : 0)) * (1.f / H);
        const float g = lg_window(fuco, fv, so, ri[r]);
        const float2 x = bc[xpad(v)];
        return make_float2(x.x * g, x.y * g);
      };
      auto st = [&](int v, float2 val) { xb[xpad(v)] = val; };
      group_fft<H, T, S::R0, S::R1, S::R2, true>(xb, t, twh, ld, st, sync);
    }
    __syncthreads();
    {
      // thread (row v0 = tid / COLS, column c = tid % COLS) copies rows v0 + RSTEP k: a
      // warp stores row segments of COLS columns
      constexpr int RSTEP = NT / COLS;
      const int c = tid % COLS, v0 = tid / COLS;
      if (!zcs[o][c]) {
        const float2* srcb = xbuf + c * XS;
        float2* dstc = scratch + (((size_t)img * NS + s) * NO + o) * (size_t)H * W + c0 + c;
#pragma unroll 2
        for (int k = 0; k < H / RSTEP; ++k) {
          const int v = v0 + RSTEP * k;
          dstc[(size_t)v * W] = srcb[xpad(v)];
        }
      }
    }
    __syncthreads();
  }
}

// Column pass for H = 1024 with the filtered spectrum in tensor memory.  CTA = 8 columns,
// one warp each (two warps per TMEM lane quadrant), two CTAs per SM.  Thread t of a column
// reads the same 32 elements v = t + 32 r of F * R_s in the first FFT pass of every
// orientation, so those 64 floats live in its own TMEM lane (64 columns) instead of shared
// memory; shared memory holds only the exchange buffers, which also stage the coalesced
// copy-out (row segments of 8 columns = 64 bytes).  The window is applied as the first pass
// loads its inputs (1/r recomputed there: fewer registers), the transform is two radix-32
// passes with the addresses of t < 32 folded: pass 1 writes xb[33 t + r], pass 2 reads and
// writes xb[t + 33 r].
constexpr int CT_COLS = 8;
constexpr int CT_NT = 32 * CT_COLS;
constexpr int CT_TMEM_COLS = 64 * (CT_COLS / 4);

template <class Ld>
__device__ __forceinline__ void fft1024_inverse_col(float2* xb, int t, const float2* __restrict__ tw,
                                                    Ld& ld) {
  PassTw<1024, 32, 32, 32> p1;
  p1.template load<true>(t, tw);
  float2 v[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = ld(r);
  dft_reg<32, true>(v);
  float2* w1 = xb + 33 * t;   // xpad(32 t + r)
#pragma unroll
  for (int r = 0; r < 32; ++r) w1[r] = v[r];
  __syncwarp();
  const float2* r2p = xb + t;   // xpad(t + 32 r)
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = r2p[33 * r];
  __syncwarp();
#pragma unroll
  for (int r = 1; r < 32; ++r) {
    // W^(t r) from the powers r = 2^b (FP64-generated table values), as reg_pass does
    float2 w = make_float2(1.f, 0.f);
    bool first = true;
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (r & (1 << b)) {
        w = first ? p1.w[0][b] : cmul(w, p1.w[0][b]);
        first = false;
      }
    v[r] = cmul(v[r], w);
  }
  dft_reg<32, true>(v);
  float2* w2 = xb + t;
#pragma unroll
  for (int r = 0; r < 32; ++r) w2[33 * r] = v[r];
}

template <int LP>
__global__ void __launch_bounds__(CT_NT, 2) lg_cols_tm1024(const float2* __restrict__ spec,
                                                          float2* __restrict__ scratch, int W,
                                                          const float2* __restrict__ twh,
                                                          KParams kp,
                                                          const unsigned char* __restrict__ zc) {
  constexpr int H = 1024, T = 32, E = H / T, COLS = CT_COLS, NT = CT_NT;
  constexpr int XS = ColStride<H, COLS>::SIZE;
  static_assert(COLS % 4 == 0, "whole TMEM lane quadrants");
  extern __shared__ float2 sm[];
  float2* xbuf = sm;   // [COLS][XS]
  __shared__ unsigned char zcs[NO][COLS];
  __shared__ uint32_t tm_slot;
  const int s = blockIdx.y, img = blockIdx.z;
  const int c0 = blockIdx.x * COLS;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, t = tid & 31, col = warp;
  if (warp == 0) tmem_alloc(&tm_slot, CT_TMEM_COLS);
  for (int i = tid; i < NO * COLS; i += NT) {
    const int o = i / COLS, c = i % COLS;
    zcs[o][c] = (c0 + c < W) ? zc[o * W + c0 + c] : 1;
  }
  {
    // F * R_s * 1/(HW) into the exchange buffers: thread (row v0 = tid / COLS, column c)
    // loads rows v0 + 32 k of its column, all loads in flight together
    const float2* F = spec + (size_t)img * H * W;
    const float log_fs = kp.log_fs[s];
    const float inv_hw = 1.f / ((float)H * (float)W);
    const int c = tid % COLS, v0 = tid / COLS, uu = c0 + c;
    const float fuu = (uu < W) ? fftfreq(uu, W) : 0.f;
    float2 fx[E];
#pragma unroll
    for (int k = 0; k < E; ++k)
      fx[k] = (uu < W) ? __ldg(F + (size_t)(v0 + 32 * k) * W + uu) : make_float2(0.f, 0.f);
    float2* xc = xbuf + c * XS + v0;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      float2 f = make_float2(0.f, 0.f);
      if (uu < W) {
        const float fv = fftfreq(v0 + 32 * k, H);
        const float rs = lg_radial<LP>(fuu * fuu + fv * fv, log_fs, kp) * inv_hw;
        f = make_float2(fx[k].x * rs, fx[k].y * rs);
      }
      xc[33 * k] = f;   // xpad(v0 + 32 k)
    }
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this warp's TMEM: lanes of quadrant warp % 4, 64 columns from 64 (warp / 4)
  const uint32_t tm = tm_slot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  float2* xb = xbuf + col * XS;
  {
    float bv[64];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const float2 x = xb[t + 33 * r];
      bv[2 * r] = x.x;
      bv[2 * r + 1] = x.y;
    }
    tmem_st64(tm, bv);
    tmem_wait_st();
  }
  __syncthreads();   // the staging reads precede the first pass's writes
  const int u = c0 + col;
  const float fu = (u < W) ? fftfreq(u, W) : 0.f;
  const float fu2 = __fmul_rn(fu, fu);
  // fftfreq(t + 32 r, H) as t / H plus a constant per r (exact: H is a power of two)
  const float fv0 = (float)t * (1.f / H);
  for (int o = 0; o < NO; ++o) {
    const float fuco = __fmul_rn(fu, kp.cos_o[o]), so = kp.sin_o[o];
    // a column whose window is zero everywhere transforms to zero: skipped and left
    // unwritten (the row pass substitutes zeros from the same table)
    if (!__all_sync(0xffffffffu, zcs[o][col] != 0)) {
      float bv[64];
      tmem_ld64(tm, bv);
      tmem_wait_ld_all();
      auto ld = [&](int r) -> float2 {
        const float fv = fv0 + (float)(T * r - (2 * r >= E ? H : 0)) * (1.f / H);
        // 1/r of max(r^2, tiny): at DC both frequencies are 0, so c and the window are 0
        const float ri = rsqrtf(fmaxf(fmaf(fv, fv, fu2), 1e-30f));
        const float g = lg_window(fuco, fv, so, ri);
        return make_float2(bv[2 * r] * g, bv[2 * r + 1] * g);
      };
      fft1024_inverse_col(xb, t, twh, ld);
    }
    __syncthreads();
    {
      // thread (row v0 = tid / COLS, column c) copies rows v0 + 32 k
      const int c = tid % COLS, v0 = tid / COLS;
      if (!zcs[o][c]) {
        const float2* srcb = xbuf + c * XS + v0;
        float2* dstc = scratch + (((size_t)img * NS + s) * NO + o) * (size_t)H * W + c0 + c +
                       (size_t)v0 * W;
#pragma unroll 4
        for (int k = 0; k < E; ++k) dstc[(size_t)(32 * k) * W] = srcb[33 * k];
      }
    }
    __syncthreads();
  }
  tmem_fence_before();
  __syncthreads();
  if (warp == 0) {
    tmem_fence_after();
    tmem_dealloc(tm_slot, CT_TMEM_COLS);
  }
}

template <int LP>
static cudaError_t cols_tm1024(const float2* spec, float2* scratch, int nimg, int W,
                               const FftPlan& ph, const KParams& kp, const unsigned char* zc,
                               cudaStream_t st) {
  const size_t sm = (size_t)CT_COLS * ColStride<1024, CT_COLS>::SIZE * sizeof(float2);
  cudaFuncSetAttribute(lg_cols_tm1024<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  lg_cols_tm1024<LP><<<dim3((W + CT_COLS - 1) / CT_COLS, NS, nimg), CT_NT, sm, st>>>(
      spec, scratch, W, ph.tw, kp, zc);
  return cudaGetLastError();
}

// Row pass for power-of-two W: one group per (row, scale) transform, ROWS rows per CTA;
// after each orientation's four scales are in shared memory every thread reduces its
// pixels (same formulas as lg_rows_reduce).
template <int WN>
__global__ void __launch_bounds__(RegShape<WN>::NT) lg_rows_reg(const float2* __restrict__ scratch, int H,
                                                           const float2* __restrict__ tww,
                                                           KParams kp, float* __restrict__ er_out,
                                                           float* __restrict__ q_out,
                                                           float* __restrict__ an0_out,
                                                           float* __restrict__ amp_out,
                                                           unsigned char* __restrict__ mim_out,
                                                           int mim_pitch,
                                                           const unsigned char* __restrict__ zc) {
  using S = RegShape<WN>;
  constexpr int T = S::T, NT = S::NT;
  constexpr int GROUPS = NT / T;
  constexpr int ROWS = GROUPS / NS;
  constexpr int XS = XBuf<WN>::SIZE;
  constexpr int PIX = ROWS * WN / NT;
  static_assert(ROWS >= 1 && PIX >= 1, "row tile");
  extern __shared__ float2 sm[];   // [GROUPS][XS], group g = (row g / NS, scale g % NS)
  // bit r of zmask[o][t]: column t + T r has a zero window for orientation o (the first
  // FFT pass reads exactly those columns, one radix-E butterfly per thread)
  constexpr int E = WN / T;
  static_assert(E == S::R0 && E <= 32, "first pass: one butterfly of radix E per thread");
  __shared__ unsigned zmask[NO][T];
  for (int i = threadIdx.x; i < NO * T; i += NT) {
    const int o = i / T, tt = i % T;
    unsigned m = 0;
    for (int r = 0; r < E; ++r) m |= (zc[o * WN + tt + T * r] ? 1u : 0u) << r;
    zmask[o][tt] = m;
  }
  __syncthreads();
  const int img = blockIdx.y;
  const int row0 = blockIdx.x * ROWS;
  const int tid = threadIdx.x;
  const int grp = tid / T, t = tid % T;
  const int rr = grp / NS, sc = grp % NS;
  const int row = row0 + rr;
  float2* xb = sm + grp * XS;
  const size_t P = (size_t)H * WN;
  float best[PIX];
  int besto[PIX];
#pragma unroll
  for (int k = 0; k < PIX; ++k) { best[k] = -1.f; besto[k] = 0; }
  auto sync = [] {
    if constexpr (T <= 32) __syncwarp();
    else __syncthreads();
  };
  for (int o = 0; o < NO; ++o) {
    const float2* src = scratch + (((size_t)img * NS + sc) * NO + o) * P + (size_t)row * WN;
    const unsigned zm = (row < H) ? ~zmask[o][t] : 0u;   // bit r set: load element r
    auto ld = [&](int, int r, int x) -> float2 {
      return ((zm >> r) & 1u) ? __ldg(src + x) : make_float2(0.f, 0.f);
    };
    auto st = [&](int x, float2 val) { xb[xpad(x)] = val; };
    group_fft<WN, T, S::R0, S::R1, S::R2, true>(xb, t, tww, ld, st, sync);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
      const int pix = tid + NT * k;
      const int r2 = pix / WN, x = pix % WN;
      if (row0 + r2 >= H) continue;
      float2 z[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) z[s] = sm[(r2 * NS + s) * XS + xpad(x)];
      float energy, q, an0, sum_an;
      reduce_pixel(z, kp, energy, q, an0, sum_an);
      const size_t off = ((size_t)img * NO + o) * P + (size_t)(row0 + r2) * WN + x;
      er_out[off] = energy;
      q_out[off] = q;
      an0_out[off] = an0;
      if (amp_out) amp_out[off] = sum_an;
      if (sum_an > best[k]) { best[k] = sum_an; besto[k] = o; }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PIX; ++k) {
    const int pix = tid + NT * k;
    const int r2 = pix / WN, x = pix % WN;
    if (row0 + r2 < H)
      mim_out[(size_t)img * H * mim_pitch + (size_t)(row0 + r2) * mim_pitch + x] =
          (unsigned char)besto[k];
  }
}

// Row pass for W = 1024: one row per 128-thread CTA, warp s transforms scale s with the
// folded-address two-pass transform (the same arithmetic and order as the generic row
// pass), then every thread reduces 8 pixels as lg_rows_reg does.
__global__ void __launch_bounds__(128) lg_rows_1024(const float2* __restrict__ scratch, int H,
                                                   const float2* __restrict__ tww, KParams kp,
                                                   float* __restrict__ er_out,
                                                   float* __restrict__ q_out,
                                                   float* __restrict__ an0_out,
                                                   float* __restrict__ amp_out,
                                                   unsigned char* __restrict__ mim_out,
                                                   int mim_pitch,
                                                   const unsigned char* __restrict__ zc) {
  constexpr int WN = 1024, T = 32, NT = 128, E = WN / T, PIX = WN / NT;
  constexpr int XS = XBuf<WN>::SIZE;
  extern __shared__ float2 sm[];   // [NS][XS]
  // bit r of zmask[o][t]: column t + 32 r has a zero window for orientation o
  __shared__ unsigned zmask[NO][T];
  for (int i = threadIdx.x; i < NO * T; i += NT) {
    const int o = i / T, tt = i % T;
    unsigned m = 0;
    for (int r = 0; r < E; ++r) m |= (zc[o * WN + tt + T * r] ? 1u : 0u) << r;
    zmask[o][tt] = m;
  }
  __syncthreads();
  const int img = blockIdx.y, row = blockIdx.x;
  const int tid = threadIdx.x, sc = tid >> 5, t = tid & 31;
  float2* xb = sm + sc * XS;
  const size_t P = (size_t)H * WN;
  float best[PIX];
  int besto[PIX];
#pragma unroll
  for (int k = 0; k < PIX; ++k) { best[k] = -1.f; besto[k] = 0; }
  const float2* pix0 = sm + tid + (tid >> 5);   // xpad(tid + 128 k) = tid + tid / 32 + 132 k
  for (int o = 0; o < NO; ++o) {
    const float2* src = scratch + (((size_t)img * NS + sc) * NO + o) * P + (size_t)row * WN + t;
    const unsigned zm = ~zmask[o][t];   // bit r set: load element r
    auto ld = [&](int r) -> float2 {
      return ((zm >> r) & 1u) ? __ldg(src + T * r) : make_float2(0.f, 0.f);
    };
    fft1024_inverse_col(xb, t, tww, ld);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
      const int x = tid + NT * k;
      float2 z[NS];
#pragma unroll
      for (int s2 = 0; s2 < NS; ++s2) z[s2] = pix0[s2 * XS + 132 * k];
      float energy, q, an0, sum_an;
      reduce_pixel(z, kp, energy, q, an0, sum_an);
      const size_t off = ((size_t)img * NO + o) * P + (size_t)row * WN + x;
      er_out[off] = energy;
      q_out[off] = q;
      an0_out[off] = an0;
      if (amp_out) amp_out[off] = sum_an;
      if (sum_an > best[k]) { best[k] = sum_an; besto[k] = o; }   // lowest o on ties
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PIX; ++k)
    mim_out[(size_t)img * H * mim_pitch + (size_t)row * mim_pitch + tid + NT * k] =
        (unsigned char)besto[k];
}

template <int H>
static cudaError_t cols_reg(const float2* spec, float2* scratch, int nimg, int W,
                            const FftPlan& ph, const KParams& kp, const unsigned char* zc,
                            cudaStream_t st) {
  constexpr int NT = ColShape<H>::NT;
  constexpr int COLS = NT / ColShape<H>::T;
  const size_t sm = 2 * (size_t)COLS * ColStride<H, COLS>::SIZE * sizeof(float2);
  cudaFuncSetAttribute(lg_cols_reg<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  lg_cols_reg<H><<<dim3((W + COLS - 1) / COLS, NS, nimg), NT, sm, st>>>(spec, scratch, W, ph.tw,
                                                                       kp, zc);
  return cudaGetLastError();
}

template <int WN>
static cudaError_t rows_reg(const float2* scratch, int nimg, int H, const FftPlan& pw,
                            const KParams& kp, float* er, float* q, float* an0, float* amp,
                            unsigned char* mim, int mim_pitch, const unsigned char* zc,
                            cudaStream_t st) {
  constexpr int NT = RegShape<WN>::NT, GROUPS = NT / RegShape<WN>::T;
  constexpr int ROWS = GROUPS / NS;
  const size_t sm = (size_t)GROUPS * XBuf<WN>::SIZE * sizeof(float2);
  cudaFuncSetAttribute(lg_rows_reg<WN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  lg_rows_reg<WN><<<dim3((H + ROWS - 1) / ROWS, nimg), NT, sm, st>>>(
      scratch, H, pw.tw, kp, er, q, an0, amp, mim, mim_pitch, zc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
void launch_twiddles(float2* tw, int n, cudaStream_t st) {
  twiddle_gen<<<(n + 255) / 256, 256, 0, st>>>(tw, n);
}

void launch_pass_twiddles(float2* ptw, const float2* tw, int L, const PassDims& pd,
                          cudaStream_t st) {
  if (pd.total > 0)
    pass_twiddle_gather<<<(pd.total + 255) / 256, 256, 0, st>>>(ptw, tw, L, pd);
}

static int rows_tile(int W) { return W >= 4096 ? 1 : (4096 / W > 256 ? 256 : 4096 / W); }
static int cols_tile(int H) {
  int tc = 8192 / H;
  if (tc > 16) tc = 16;
  if (tc < 1) tc = 1;
  return tc;
}

template <int WN>
static void rows_fwd_reg(const ImgPtrs& ip, const float* dense, float2* spec, int nimg, int H,
                         const FftPlan& pw, cudaStream_t st) {
  constexpr int NT = RegShape<WN>::NT, ROWS = NT / RegShape<WN>::T;
  const size_t sm = ((size_t)ROWS * XBuf<WN>::SIZE + NT) * sizeof(float2);
  cudaFuncSetAttribute(fwd_rows_reg<WN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  fwd_rows_reg<WN><<<dim3((H + ROWS - 1) / ROWS, nimg), NT, sm, st>>>(ip, dense, spec, H, pw.tw);
}

template <int HN>
static void cols_fwd_reg(float2* spec, int nimg, int W, const FftPlan& ph, cudaStream_t st) {
  constexpr int NT = ColShape<HN>::NT, COLS = NT / ColShape<HN>::T;
  const size_t sm = ((size_t)COLS * ColStride<HN, COLS>::SIZE + NT) * sizeof(float2);
  cudaFuncSetAttribute(fwd_cols_reg<HN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  fwd_cols_reg<HN><<<dim3((W + COLS - 1) / COLS, nimg), NT, sm, st>>>(spec, W, ph.tw);
}

// ------------------------------------------------------------------ group launchers
// A launch group is walked in runs of consecutive images of one size.  A run whose
// transformed side has a register-tiled kernel (a power-of-two side, direct transform)
// gets that kernel on the run's slice of the packed buffers (the run's images lie H W
// pixels apart there, as those kernels expect); every other image joins one shared-memory
// launch over the images of all sizes, in which each CTA reads its image's size, plan and
// tile from the group tables.
namespace {

bool reg_side(int n, const FftPlan& p) {
  if (p.m != n) return false;
  switch (n) {
    case 256: case 512: case 1024: case 2048: case 4096: return true;
    default: return false;
  }
}

template <class F>
void for_runs(const Group& gr, F&& f) {
  int i = 0;
  while (i < gr.n) {
    int j = i + 1;
    while (j < gr.n && gr.H[j] == gr.H[i] && gr.W[j] == gr.W[i]) ++j;
    f(i, j - i);
    i = j;
  }
}

// Appends image i of gr to the shared-memory launch's tables.
void sub_add(Group& sub, FftGroup& sf, const Group& gr, int i, const FftPlan& pl, int tile,
             const unsigned char* zc, bool rows = false) {
  const int k = sub.n++;
  sub.H[k] = gr.H[i];
  sub.W[k] = gr.W[i];
  sub.poff[k] = gr.poff[i];
  sub.mrow[k] = gr.mrow[i];
  sf.pass[k] = rows ? pl.dev_r : pl.dev;
  sf.tile[k] = tile;
  sf.dtile[k] = FastDiv((unsigned)(tile > 0 ? tile : 1));
  sf.zc[k] = zc;
}

template <class T>
inline T max_of(T a, T b) { return a > b ? a : b; }

}  // namespace

cudaError_t launch_fft2_forward(const ImgPtrs* ip, const float* dense, float2* spec,
                                const Group& gr, const FbImage* fi, cudaStream_t st,
                                int* launches) {
  ImgPtrs none{};
  const ImgPtrs& ipr = ip ? *ip : none;
  int nl = 0;
  // rows of the real images
  {
    Group sub{};
    FftGroup sf{};
    ImgPtrs sip{};
    int grid_x = 0;
    size_t smr = 0;
    for_runs(gr, [&](int i0, int cnt) {
      const int H = gr.H[i0], W = gr.W[i0];
      const FftPlan& pw = fi[i0].pw;
      if (reg_side(W, pw)) {
        ImgPtrs rp{};
        for (int k = 0; k < cnt; ++k) {
          rp.img[k] = ipr.img[i0 + k];
          rp.pitch[k] = ipr.pitch[i0 + k];
        }
        const float* d = dense ? dense + gr.poff[i0] : nullptr;
        float2* sp = spec + gr.poff[i0];
        switch (W) {
          case 256: rows_fwd_reg<256>(rp, d, sp, cnt, H, pw, st); break;
          case 512: rows_fwd_reg<512>(rp, d, sp, cnt, H, pw, st); break;
          case 1024: rows_fwd_reg<1024>(rp, d, sp, cnt, H, pw, st); break;
          case 2048: rows_fwd_reg<2048>(rp, d, sp, cnt, H, pw, st); break;
          default: rows_fwd_reg<4096>(rp, d, sp, cnt, H, pw, st); break;
        }
        ++nl;
        return;
      }
      const int tr = rows_tile(pw.m);
      for (int k = 0; k < cnt; ++k) {
        sip.img[sub.n] = ipr.img[i0 + k];
        sip.pitch[sub.n] = ipr.pitch[i0 + k];
        sub_add(sub, sf, gr, i0 + k, pw, tr, nullptr);
      }
      grid_x = max_of(grid_x, (H + tr - 1) / tr);
      smr = max_of(smr, 2 * (size_t)tr * pw.m * sizeof(float2));
    });
    if (sub.n) {
      cudaFuncSetAttribute(fwd_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
      fwd_rows<<<dim3(grid_x, sub.n), 512, smr, st>>>(sip, dense, spec, sub, sf);
      ++nl;
    }
  }
  // columns, in place
  {
    Group sub{};
    FftGroup sf{};
    int grid_x = 0;
    size_t smc = 0;
    for_runs(gr, [&](int i0, int cnt) {
      const int H = gr.H[i0], W = gr.W[i0];
      const FftPlan& ph = fi[i0].ph;
      if (reg_side(H, ph)) {
        float2* sp = spec + gr.poff[i0];
        switch (H) {
          case 256: cols_fwd_reg<256>(sp, cnt, W, ph, st); break;
          case 512: cols_fwd_reg<512>(sp, cnt, W, ph, st); break;
          case 1024: cols_fwd_reg<1024>(sp, cnt, W, ph, st); break;
          case 2048: cols_fwd_reg<2048>(sp, cnt, W, ph, st); break;
          default: cols_fwd_reg<4096>(sp, cnt, W, ph, st); break;
        }
        ++nl;
        return;
      }
      const int tc = cols_tile(ph.m);
      for (int k = 0; k < cnt; ++k) sub_add(sub, sf, gr, i0 + k, ph, tc, nullptr);
      grid_x = max_of(grid_x, (W + tc - 1) / tc);
      smc = max_of(smc, 2 * (size_t)col_buf(tc * ph.m) * sizeof(float2));
    });
    if (sub.n) {
      cudaFuncSetAttribute(fwd_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
      fwd_cols<<<dim3(grid_x, sub.n), 512, smc, st>>>(spec, sub, sf);
      ++nl;
    }
  }
  if (launches) *launches = nl;
  return cudaGetLastError();
}

// Shared memory of the generic column pass for a tile of tc columns: F R_s (H rows), the
// two transform buffers (slot length L each) and the per-row frequencies.
// Shared memory of a column tile, with (tw) or without the twiddle copy.
static constexpr size_t kColSmemMax = 227 * 1024;
static size_t cols_inverse_smem(int H, int L, int tc, bool tw) {
  return ((size_t)H * tc + 2 * (size_t)col_buf(L * tc) + (tw ? L : 0)) * sizeof(float2) +
         (size_t)H * sizeof(float);
}
// The twiddle copy is made where a one-column tile leaves room for it (all but the
// tallest Bluestein heights, whose convolution slots fill the shared memory).
static bool cols_inverse_tw(int H, int L) { return cols_inverse_smem(H, L, 1, true) <= kColSmemMax; }
static int cols_inverse_tile(int H, int L) {
  const bool tw = cols_inverse_tw(H, L);
  int tc = cols_tile(L);
  while (tc > 1 && cols_inverse_smem(H, L, tc, tw) > kColSmemMax) tc /= 2;
  return tc;
}

int lg_cols_tile_candidates(int H, int L, int* out, int max_n) {
  if (L == H) {
    switch (H) {
      case 256: case 512: case 1024: case 2048: case 4096: return 0;   // register path
      default: break;
    }
  }
  int n = 0;
  for (int tc = cols_inverse_tile(H, L); tc >= 1 && n < max_n; tc /= 2) out[n++] = tc;
  return n;
}

cudaError_t launch_lg_cols(const float2* spec, float2* scratch, const Group& gr,
                           const FbImage* fi, const KParams& kp, cudaStream_t st, int* launches) {
  int nl = 0;
  Group sub{};
  FftGroup sf{};
  int grid_x = 0;
  size_t smx = 0;
  bool tw_all = true;
  struct TileDims { int H, L, tc; };
  TileDims tiles[MAXB];
  int ntiles = 0;
  cudaError_t err = cudaSuccess;
  for_runs(gr, [&](int i0, int cnt) {
    const int H = gr.H[i0], W = gr.W[i0];
    const FftPlan& ph = fi[i0].ph;
    if (reg_side(H, ph)) {
      const float2* sp = spec + gr.poff[i0];
      float2* sc = scratch + (size_t)NS * NO * gr.poff[i0];
      const unsigned char* zc = fi[i0].zc;
      cudaError_t e;
      switch (H) {
        case 256: e = cols_reg<256>(sp, sc, cnt, W, ph, kp, zc, st); break;
        case 512: e = cols_reg<512>(sp, sc, cnt, W, ph, kp, zc, st); break;
        case 1024:
          e = kp.lp_order == 15 ? cols_tm1024<15>(sp, sc, cnt, W, ph, kp, zc, st)
                                : cols_tm1024<0>(sp, sc, cnt, W, ph, kp, zc, st);
          break;
        case 2048: e = cols_reg<2048>(sp, sc, cnt, W, ph, kp, zc, st); break;
        default: e = cols_reg<4096>(sp, sc, cnt, W, ph, kp, zc, st); break;
      }
      if (e != cudaSuccess) err = e;
      ++nl;
      return;
    }
    int tc = cols_inverse_tile(H, ph.m);
    const int tuned = fi[i0].col_tile;
    if (tuned >= 1 && tuned <= tc) tc = tuned;   // a tuned (smaller) tile; same result
    for (int k = 0; k < cnt; ++k) sub_add(sub, sf, gr, i0 + k, ph, tc, fi[i0].zc);
    grid_x = max_of(grid_x, (W + tc - 1) / tc);
    tw_all = tw_all && cols_inverse_tw(H, ph.m);
    tiles[ntiles++] = {H, ph.m, tc};
  });
  if (err != cudaSuccess) return err;
  if (sub.n) {
    // one launch: the twiddle copy only when every image's tile has room for it (each
    // tile was sized with the copy where its height allows; without it every tile fits)
    for (int i = 0; i < ntiles; ++i)
      smx = max_of(smx, cols_inverse_smem(tiles[i].H, tiles[i].L, tiles[i].tc, tw_all));
    cudaFuncSetAttribute(lg_cols_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx);
    lg_cols_inverse<<<dim3(grid_x, NS, sub.n), 512, smx, st>>>(spec, scratch, sub, sf, kp,
                                                                tw_all ? 1 : 0);
    ++nl;
  }
  if (launches) *launches = nl;
  return cudaGetLastError();
}

cudaError_t launch_lg_rows(float2* scratch, const Group& gr, const FbImage* fi,
                           const KParams& kp, float* er, float* q, float* an0, float* amp,
                           unsigned char* mim, int mim_pitch, cudaStream_t st, int* launches) {
  int nl = 0;
  // red[0]: rows whose four scales fit two CTAs per SM; red[1]: wider rows, transformed
  // two scales at a time (one launch each, so that a wide image does not set the
  // occupancy of the narrow ones); spl: rows too wide even for that
  Group red[2] = {}, spl{};
  FftGroup rf[2] = {}, sf{};
  int red_rows[2] = {0, 0}, spl_rows = 0;
  long long spl_px = 0;
  size_t red_sm[2] = {0, 0}, spl_sm = 0;
  cudaError_t err = cudaSuccess;
  for_runs(gr, [&](int i0, int cnt) {
    const int H = gr.H[i0], W = gr.W[i0];
    const FftPlan& pw = fi[i0].pw;
    const unsigned char* zc = fi[i0].zc;
    if (reg_side(W, pw)) {
      const size_t pb = (size_t)gr.poff[i0];
      const float2* sc = scratch + NS * NO * pb;
      float* e_ = er + NO * pb;
      float* q_ = q + NO * pb;
      float* a0 = an0 + NO * pb;
      float* am = amp ? amp + NO * pb : nullptr;
      unsigned char* mm = mim + (size_t)gr.mrow[i0] * mim_pitch;
      cudaError_t e;
      switch (W) {
        case 256: e = rows_reg<256>(sc, cnt, H, pw, kp, e_, q_, a0, am, mm, mim_pitch, zc, st); break;
        case 512: e = rows_reg<512>(sc, cnt, H, pw, kp, e_, q_, a0, am, mm, mim_pitch, zc, st); break;
        case 1024: {
          const size_t sm = (size_t)NS * XBuf<1024>::SIZE * sizeof(float2);
          cudaFuncSetAttribute(lg_rows_1024, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          lg_rows_1024<<<dim3(H, cnt), 128, sm, st>>>(sc, H, pw.tw, kp, e_, q_, a0, am, mm,
                                                      mim_pitch, zc);
          e = cudaGetLastError();
          break;
        }
        case 2048: e = rows_reg<2048>(sc, cnt, H, pw, kp, e_, q_, a0, am, mm, mim_pitch, zc, st); break;
        default: e = rows_reg<4096>(sc, cnt, H, pw, kp, e_, q_, a0, am, mm, mim_pitch, zc, st); break;
      }
      if (e != cudaSuccess) err = e;
      ++nl;
      return;
    }
    const size_t sm_full = 2 * (size_t)NS * row_slot(pw.m) * sizeof(float2);
    const size_t sm_half = (2 * (size_t)(NS / 2) * row_slot(pw.m) + 2 * (size_t)W) * sizeof(float2);
    const int cl = sm_full <= 113 * 1024 ? 0 : (sm_half <= 227 * 1024 ? 1 : 2);
    if (cl < 2 && W <= RR_MAXPIX * 512) {
      for (int k = 0; k < cnt; ++k) sub_add(red[cl], rf[cl], gr, i0 + k, pw, 0, zc, true);
      red_rows[cl] = max_of(red_rows[cl], H);
      red_sm[cl] = max_of(red_sm[cl], cl == 0 ? sm_full : sm_half);
    } else {
      // rows too wide for four scales in shared memory: transform each (row, scale) in
      // place, then reduce the pixels from the transformed responses
      for (int k = 0; k < cnt; ++k) sub_add(spl, sf, gr, i0 + k, pw, 0, zc);
      spl_rows = max_of(spl_rows, H);
      spl_px = max_of(spl_px, (long long)H * W);
      spl_sm = max_of(spl_sm, 2 * (size_t)row_slot(pw.m) * sizeof(float2));
    }
  });
  if (err != cudaSuccess) return err;
  if (red[0].n) {
    cudaFuncSetAttribute(lg_rows_reduce<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)red_sm[0]);
    lg_rows_reduce<false><<<dim3(red_rows[0], red[0].n), 512, red_sm[0], st>>>(
        scratch, red[0], rf[0], kp, er, q, an0, amp, mim, mim_pitch);
    ++nl;
  }
  if (red[1].n) {
    cudaFuncSetAttribute(lg_rows_reduce<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)red_sm[1]);
    lg_rows_reduce<true><<<dim3(red_rows[1], red[1].n), 512, red_sm[1], st>>>(
        scratch, red[1], rf[1], kp, er, q, an0, amp, mim, mim_pitch);
    ++nl;
  }
  if (spl.n) {
    cudaFuncSetAttribute(lg_rows_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spl_sm);
    lg_rows_split<<<dim3(spl_rows, NS, spl.n), 512, spl_sm, st>>>(scratch, spl, sf);
    const int blocks = (int)((spl_px + 255) / 256);
    lg_rows_pixels<<<dim3(blocks, spl.n), 256, 0, st>>>(scratch, spl, kp, er, q, an0, amp, mim,
                                                        mim_pitch);
    nl += 2;
  }
  if (launches) *launches = nl;
  return cudaGetLastError();
}

}  // namespace rift2
