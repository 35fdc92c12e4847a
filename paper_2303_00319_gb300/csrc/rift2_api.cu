// C ABI of the RIFT2 pipeline (include/rift2.h): context, FFT plans, workspace arena and
// the launch sequences of rift2_extract / rift2_match and the stage entry points.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"

using namespace rift2;

namespace rift2 {
void derive_kparams(const rift2_params& p, KParams& k) {
  for (int s = 0; s < NS; ++s)
    k.log_fs[s] = (float)(-std::log((double)p.min_wavelength) - s * std::log((double)p.mult));
  double ls = std::log((double)p.sigma_onf);
  k.inv_2ls2 = (float)(1.0 / (2.0 * ls * ls));
  k.inv_lp_c2 = (float)(1.0 / ((double)p.lp_cutoff * p.lp_cutoff));
  k.lp_order = p.lp_order;
  for (int o = 0; o < NO; ++o) {
    double a = o * M_PI / NO;
    k.cos_o[o] = (float)std::cos(a);
    k.sin_o[o] = (float)std::sin(a);
  }
  k.eps = p.eps;
  k.g = p.g;
  k.cutoff = p.cutoff;
  k.inv_ns1 = (float)(1.0 / (p.n_scales - 1));
  double inv_mult = 1.0 / p.mult;
  double scale_sum = (1.0 - std::pow(inv_mult, p.n_scales)) / (1.0 - inv_mult);
  k.noise_c = (float)(scale_sum / std::sqrt(std::log(4.0)) *
                      (std::sqrt(M_PI / 2.0) + p.k * std::sqrt((4.0 - M_PI) / 2.0)));
  k.fast_t = p.fast_threshold;
  k.fast_arc = p.fast_arc;
  k.max_kp = p.max_keypoints;
  k.kp_cap = p.max_keypoints * ((p.flags & RIFT2_FLAG_CORNERS) ? 2 : 1);
  k.ratio_pm = (int)std::lround(p.second_ratio * 1000.0);
  k.desc_mode = (p.flags & RIFT2_FLAG_RIFT_RING)       ? DESC_RIFT_RING
                : (p.flags & RIFT2_FLAG_RIFT_TEMPLATE) ? DESC_RIFT_TEMPLATE
                : (p.flags & RIFT2_FLAG_SPATIAL_NORM)  ? DESC_SPATIAL
                                                       : DESC_RIFT2;
  for (int o = 0; o < NO; ++o) {   // Q14, half away from zero (std::round)
    const double a = o * M_PI / NO;
    k.rot_c[o] = (int)std::round(std::cos(a) * 16384.0);
    k.rot_s[o] = (int)std::round(std::sin(a) * 16384.0);
  }
}

}  // namespace rift2

struct rift2_ctx {
  int device = 0;
  rift2_params p{};
  KParams kp{};
  size_t budget = 0;
  void* ws = nullptr;
  size_t ws_size = 0;
  int* status = nullptr;
  long long wait_iters = 1ll << 24;   // first-wait limit of the descriptor kernel's staging
  std::map<int, FftPlan> plans;
  std::vector<float2*> pass_tw;   // per-pass twiddle tables of the plans (freed at destroy)
  std::vector<FftPasses*> pass_dev;   // the plans' device pass tables (freed at destroy)
  std::map<std::pair<int, int>, unsigned char*> zero_cols;   // (H, W) -> [NO][W]
  std::map<std::pair<int, int>, int> col_tiles;              // (H, W) -> tuned column tile
  std::map<std::pair<int, int>, int> match_splits;           // (pairs, cap) -> tuned split
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  // tracing
  long long launches = 0;
  bool prof = false;
  struct Mark { int stage; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> free_events;
  double acc_ms[RIFT2_N_STAGES] = {};
  long long acc_n[RIFT2_N_STAGES] = {};
  // RIFT2_FLAG_TWO_LANES: the second lane's context and stream, and the events that fork
  // it from and join it back to the caller's stream (made on first use)
  rift2_ctx* lane = nullptr;
  cudaStream_t lane_st = nullptr;
  cudaEvent_t lane_fork = nullptr, lane_join = nullptr;
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

#define RIFT2_CU(call)                                                     \
  do {                                                                     \
    cudaError_t e__ = (call);                                              \
    if (e__ != cudaSuccess) {                                              \
      fprintf(stderr, "rift2: %s failed: %s\n", #call, cudaGetErrorString(e__)); \
      return RIFT2_E_CUDA;                                                 \
    }                                                                      \
  } while (0)

// The planner.  A pass of the shared-memory transforms costs about the same per element
// whatever its radix (index arithmetic, a shared-memory load and store, the twiddle
// product) plus a butterfly whose cost per element grows with the radix; pass_cost() is
// that sum in units of instructions per element (counted from the butterflies and the
// pass loop).  A length's radices minimise the summed cost: the power-of-two part by a
// small dynamic program over radices 16, 8, 4, 2, powers of 3 as 9s (and one 3), then
// 5, 7, 11, 13; power-of-two radices run first.  The choice is a pure function of n.
double pass_cost(int R) {
  switch (R) {
    case 2: return 18.5;
    case 4: return 16.0;
    case 8: return 15.9;
    case 16: return 17.2;
    case 3: return 17.0;
    case 9: return 20.7;
    case 5: return 18.0;
    case 7: return 19.1;
    case 11: return 22.4;
    default: return 24.2;   // 13
  }
}

// Radices of n (false when n has a prime factor above 13 or needs too many passes);
// *cost: the plan's summed pass cost per element.  allow16: radix 16 among the
// power-of-two radices (the row kernels, which run in 64 registers, take plans without).
bool factor_plan(int n, FftPlan& pl, double* cost = nullptr, bool allow16 = true) {
  pl.n = n;
  pl.nst = 0;
  int m = n, a = 0;
  while (m % 2 == 0) { m /= 2; ++a; }
  // power-of-two part: best[k] = cheapest passes for 2^k, from[k] = the last radix
  double best[32];
  int from[32];
  best[0] = 0.0;
  from[0] = 0;
  for (int k = 1; k <= a; ++k) {
    best[k] = 1e30;
    from[k] = 0;
    for (int lr = 1; lr <= (allow16 ? 4 : 3) && lr <= k; ++lr) {
      const double c = best[k - lr] + pass_cost(1 << lr);
      if (c < best[k]) { best[k] = c; from[k] = lr; }
    }
  }
  std::vector<int> rs;
  for (int k = a; k > 0; k -= from[k]) rs.push_back(1 << from[k]);
  std::sort(rs.begin(), rs.end(), [](int x, int y) { return x > y; });
  int b3 = 0;
  while (m % 3 == 0) { m /= 3; ++b3; }
  for (int i = 0; i < b3 / 2; ++i) rs.push_back(9);
  if (b3 % 2) rs.push_back(3);
  for (int f : {5, 7, 11, 13})
    while (m % f == 0) { m /= f; rs.push_back(f); }
  if (m != 1 || (int)rs.size() > FFT_MAX_STAGES) return false;
  pl.nst = (int)rs.size();
  double c = 0.0;
  for (int i = 0; i < pl.nst; ++i) {
    pl.radix[i] = rs[i];
    c += pass_cost(rs[i]);
  }
  if (cost) *cost = c;
  return true;
}

// Occupancy factor of the row kernels for a row of width n transformed at length m: their
// shared memory holds two padded slots (m + m/16 + 1 entries, as the row kernels lay them
// out) for each of the four scales, or for two scales plus a parked copy of the other two
// (2 n entries); two CTAs share an SM below 113 KB, one below 227 KB, else the row pass
// splits into a transform pass and a pixel pass.  The factors weigh the estimated work.
double row_occupancy_factor(int n, int m) {
  const double slot = (double)(m + (m >> 4) + 1) * sizeof(float2);
  const double full = 8.0 * slot, halves = 4.0 * slot + 2.0 * n * sizeof(float2);
  if (full <= 113.0 * 1024 || halves <= 113.0 * 1024) return 1.0;
  if (halves <= 227.0 * 1024) return 1.35;
  return 2.0;
}

// Length of the Bluestein convolution for a length-n transform: among the lengths
// m >= 2n - 1 up to 2.5 n that the passes take, the one with the least estimated work
// (m times its summed pass cost, times the row kernels' occupancy factor); 0 if none.
int bluestein_length(int n) {
  FftPlan t{};
  int best = 0;
  double best_work = 1e300;
  for (int m = 2 * n - 1; m <= 5 * n / 2 + 1; ++m) {
    double c = 0.0;
    if (!factor_plan(m, t, &c)) continue;
    const double work = (double)m * c * row_occupancy_factor(n, m);
    if (work < best_work) { best_work = work; best = m; }
  }
  return best;
}

// The device copy of plan pl's passes (FftPasses) with its per-pass twiddle table.
int make_passes(rift2_ctx* c, const FftPlan& pl, cudaStream_t st, const FftPasses** out) {
  const int n = pl.n, m = pl.m;
  FftPasses pp{};
  PassDims pd{};
  pp.n = n;
  pp.L = m;
  pp.nst = pl.nst;
  pd.nst = pl.nst;
  int ns = 1, off = 0;
  for (int st2 = 0; st2 < pl.nst; ++st2) {
    const int R = pl.radix[st2];
    FftPass& ps = pp.p[st2];
    ps.R = R;
    ps.ns = ns;
    ps.q = FastDiv((unsigned)(m / R));
    ps.k = FastDiv((unsigned)ns);
    ps.tw = off;
    pd.R[st2] = R;
    pd.ns[st2] = ns;
    pd.off[st2] = off;
    off += ns * (R - 1);
    ns *= R;
  }
  pd.total = off;
  pp.dL = FastDiv((unsigned)m);
  pp.dn = FastDiv((unsigned)n);
  pp.chirp = pl.chirp;
  pp.kern_fwd = pl.kern_fwd;
  pp.kern_inv = pl.kern_inv;
  float2* ptw = nullptr;
  RIFT2_CU(cudaMalloc(&ptw, sizeof(float2) * (off > 0 ? off : 1)));
  launch_pass_twiddles(ptw, pl.tw, m, pd, st);
  c->launches += 1;
  RIFT2_CU(cudaGetLastError());
  pp.ptw = ptw;
  FftPasses* dev = nullptr;
  RIFT2_CU(cudaMalloc(&dev, sizeof(FftPasses)));
  RIFT2_CU(cudaMemcpyAsync(dev, &pp, sizeof(FftPasses), cudaMemcpyHostToDevice, st));
  RIFT2_CU(cudaStreamSynchronize(st));   // pp is on this stack frame
  c->pass_tw.push_back(ptw);
  c->pass_dev.push_back(dev);
  *out = dev;
  return RIFT2_OK;
}

int get_plan(rift2_ctx* c, int n, cudaStream_t st, FftPlan* out) {
  auto it = c->plans.find(n);
  if (it != c->plans.end()) { *out = it->second; return RIFT2_OK; }
  FftPlan pl{};
  int m = n;
  if (!factor_plan(n, pl)) {
    m = bluestein_length(n);
    if (!m || !factor_plan(m, pl)) return RIFT2_E_UNIMPL;
    pl.n = n;
  }
  pl.m = m;
  float2* tw = nullptr;
  RIFT2_CU(cudaMalloc(&tw, sizeof(float2) * m));
  launch_twiddles(tw, m, st);
  c->launches += 1;
  RIFT2_CU(cudaGetLastError());
  pl.tw = tw;
  if (m != n) {
    float2 *ch = nullptr, *kf = nullptr, *ki = nullptr;
    double2 *c64 = nullptr, *tw64 = nullptr;
    RIFT2_CU(cudaMalloc(&ch, sizeof(float2) * n));
    RIFT2_CU(cudaMalloc(&kf, sizeof(float2) * m));
    RIFT2_CU(cudaMalloc(&ki, sizeof(float2) * m));
    RIFT2_CU(cudaMalloc(&c64, sizeof(double2) * n));
    RIFT2_CU(cudaMalloc(&tw64, sizeof(double2) * m));
    launch_bluestein_tables(ch, kf, ki, c64, tw64, n, m, st);
    c->launches += 3;
    RIFT2_CU(cudaGetLastError());
    RIFT2_CU(cudaStreamSynchronize(st));
    cudaFree(c64);
    cudaFree(tw64);
    pl.chirp = ch;
    pl.kern_fwd = kf;
    pl.kern_inv = ki;
  }
  // the shared-memory kernels' device copies (passes with precomputed divisors, per-pass
  // twiddles gathered from tw): one with radix 16 for the column and forward kernels, one
  // without for the row kernels (the same when the radices agree)
  FftPlan pr = pl;
  if (!factor_plan(m, pr, nullptr, false)) return RIFT2_E_UNIMPL;
  pr.n = n;
  int rc = make_passes(c, pl, st, &pl.dev);
  if (rc) return rc;
  bool same = pr.nst == pl.nst;
  for (int i = 0; same && i < pl.nst; ++i) same = pr.radix[i] == pl.radix[i];
  if (same) {
    pl.dev_r = pl.dev;
  } else {
    rc = make_passes(c, pr, st, &pl.dev_r);
    if (rc) return rc;
  }
  RIFT2_CU(cudaStreamSynchronize(st));
  c->plans[n] = pl;
  *out = pl;
  return RIFT2_OK;
}

int get_zero_cols(rift2_ctx* c, int H, int W, cudaStream_t st, unsigned char** out) {
  auto key = std::make_pair(H, W);
  auto it = c->zero_cols.find(key);
  if (it != c->zero_cols.end()) { *out = it->second; return RIFT2_OK; }
  unsigned char* zc = nullptr;
  RIFT2_CU(cudaMalloc(&zc, (size_t)NO * W));
  launch_zero_cols(H, W, c->kp, zc, st);
  c->launches += 1;
  RIFT2_CU(cudaGetLastError());
  RIFT2_CU(cudaStreamSynchronize(st));
  c->zero_cols[key] = zc;
  *out = zc;
  return RIFT2_OK;
}

int ensure_ws(rift2_ctx* c, size_t need) {
  if (need <= c->ws_size) return RIFT2_OK;
  if (need > c->budget) return RIFT2_E_NOMEM;
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_size = 0;
  }
  size_t sz = align_up(need, 1 << 20);
  if (sz > c->budget) sz = need;
  if (cudaMalloc(&c->ws, sz) != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    return RIFT2_E_NOMEM;
  }
  c->ws_size = sz;
  return RIFT2_OK;
}

// Sides the transforms take: 13-smooth up to 8192 (direct), any other length up to 4096
// (Bluestein: a convolution of 13-smooth length between 2n - 1 and 2.5 n).
int check_size(int H, int W) {
  if (H < 16 || W < 16) return RIFT2_E_INVAL;
  if (H > 8192 || W > 8192) return RIFT2_E_UNIMPL;
  FftPlan t{};
  for (int n : {H, W})
    if (!factor_plan(n, t) && (n > 4096 || !bluestein_length(n))) return RIFT2_E_UNIMPL;
  return RIFT2_OK;
}

// ------------------------------------------------------------------ tracing
// Kernels enqueued by each launcher (kept next to the launch sequences they count).
constexpr int K_FFT_FWD = 2, K_LG_COLS = 1, K_NOISE = 4, K_MOMENT = 1,
              K_DESCRIBE = 3, K_MATCH = 1, K_MATCH_TC = 4, K_INIT = 1,
              K_MERGE = 1;

cudaEvent_t take_event(rift2_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct StageScope {
  rift2_ctx* c;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageScope(rift2_ctx* c_, int stage_, cudaStream_t st_, int kernels) : c(c_), stage(stage_), st(st_) {
    c->launches += kernels;
    if (c->prof) {
      a = take_event(c);
      cudaEventRecord(a, st);
    }
  }
  ~StageScope() {
    if (c->prof && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, st);
      c->marks.push_back({stage, a, b});
    }
  }
};

// ------------------------------------------------------------------ autotuning
// First extraction of a size with a shared-memory column pass: run that pass once per
// candidate tile on image i of the group (its own spectrum; two timed repetitions each,
// events on the stream, one synchronisation), keep the fastest.  The outputs of every
// candidate are identical, so the scratch the last run leaves is as good as any.
int tune_col_tile(rift2_ctx* c, const float2* spec, float2* scratch, const Group& gr, int i,
                  const FbImage& fim, cudaStream_t st, int* tile) {
  const int H = gr.H[i], W = gr.W[i];
  const auto key = std::make_pair(H, W);
  auto it = c->col_tiles.find(key);
  if (it != c->col_tiles.end()) { *tile = it->second; return RIFT2_OK; }
  int cand[8];
  const int n = lg_cols_tile_candidates(H, fim.ph.m, cand, 8);
  if (n <= 1) { *tile = n ? cand[0] : 0; c->col_tiles[key] = *tile; return RIFT2_OK; }
  Group one{};
  one.n = 1;
  one.H[0] = H;
  one.W[0] = W;
  one.poff[0] = gr.poff[i];
  one.mrow[0] = gr.mrow[i];
  FbImage f = fim;
  cudaEvent_t ev[9];
  for (int k = 0; k <= n; ++k) RIFT2_CU(cudaEventCreate(&ev[k]));
  f.col_tile = cand[0];
  RIFT2_CU(launch_lg_cols(spec, scratch, one, &f, c->kp, st, nullptr));   // warm-up
  c->launches += 1 + 2 * n;
  RIFT2_CU(cudaEventRecord(ev[0], st));
  for (int k = 0; k < n; ++k) {
    f.col_tile = cand[k];
    for (int r = 0; r < 2; ++r) RIFT2_CU(launch_lg_cols(spec, scratch, one, &f, c->kp, st, nullptr));
    RIFT2_CU(cudaEventRecord(ev[k + 1], st));
  }
  RIFT2_CU(cudaEventSynchronize(ev[n]));
  int best = cand[0];
  float best_ms = 1e30f;
  for (int k = 0; k < n; ++k) {
    float ms = 0.f;
    RIFT2_CU(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
    if (ms < best_ms) { best_ms = ms; best = cand[k]; }
  }
  for (int k = 0; k <= n; ++k) cudaEventDestroy(ev[k]);
  c->col_tiles[key] = best;
  *tile = best;
  return RIFT2_OK;
}

// ------------------------------------------------------------------ workspace layout
// Kernels one launch_detect issues: FAST + sort, plus the multi-CTA selection's two
// kernels when it runs for this keypoint budget and map size.
static int detect_launches(int max_kp, const Group& gr) {
  return topk_multi_group(max_kp, gr) ? 4 : 2;
}

struct Layout {
  size_t spec, scratch, er, q, an0, amp, pc, moment, mim, mhist, mstate, noise, minmax, ccount,
      cand, sortbuf, chist, sel, comp, raw, info, off, total;
  // corner keypoints (RIFT2_FLAG_CORNERS): minimum-moment map, its min / max, candidate
  // count, the corner list before the merge, and the bitmap of edge-keypoint pixels
  size_t mcorner, minmax_c, ccount_c, cxy, csc, ccnt, bits;
  int mim_pitch, mim_rows, cap_cand;
  long long bits_words;   // words of the edge-keypoint bitmap per image
};

// Pixels of an image in the packed per-pixel planes: a multiple of 64, so that every
// plane of every image starts 256-byte aligned.
inline long long padded_px(int H, int W) { return ((long long)H * W + 63) / 64 * 64; }

// The packed layout of n images (Group): pixel offsets from padded counts, MIM rows
// stacked.  *ptot / *rows: pixels of one plane and MIM rows of the whole group.
Group make_group(int n, const int* H, const int* W, long long* ptot, int* rows) {
  Group gr{};
  gr.n = n;
  long long p = 0;
  int r = 0;
  for (int i = 0; i < n; ++i) {
    gr.H[i] = H[i];
    gr.W[i] = W[i];
    gr.poff[i] = p;
    gr.mrow[i] = r;
    p += padded_px(H[i], W[i]);
    r += H[i];
  }
  if (ptot) *ptot = p;
  if (rows) *rows = r;
  return gr;
}

// g images of one size whose pixels lie `stride` apart (a caller's dense [g][H][W] array:
// stride H W; the packed workspace: padded_px).
Group uniform_group(int g, int H, int W, long long stride) {
  Group gr{};
  gr.n = g;
  for (int i = 0; i < g; ++i) {
    gr.H[i] = H;
    gr.W[i] = W;
    gr.poff[i] = i * stride;
    gr.mrow[i] = i * H;
  }
  return gr;
}

// max_kp: keypoints one detector pass keeps; kp_cap: keypoint list capacity per image.
Layout extract_layout(const Group& gr, int max_kp, int kp_cap, bool corners, int debug,
                      bool spatial) {
  Layout L{};
  const int g = gr.n;
  size_t P = 0;      // pixels of one packed plane
  int rows = 0, wmax = 0;
  long long cc = 1, bw = 1;
  for (int i = 0; i < g; ++i) {
    P += (size_t)padded_px(gr.H[i], gr.W[i]);
    rows += gr.H[i];
    wmax = gr.W[i] > wmax ? gr.W[i] : wmax;
    const long long c = detect_cap_candidates(gr.H[i], gr.W[i]);
    cc = c > cc ? c : cc;
    const long long w = (gr.P(i) + 31) / 32;
    bw = w > bw ? w : bw;
  }
  // at least one TMA box wide (112 bytes; 160 for the spatial variant's window)
  const size_t box_w = spatial ? 160 : 112;
  L.mim_pitch = (int)align_up((size_t)wmax > box_w ? (size_t)wmax : box_w, 16);
  L.cap_cand = (int)cc;
  L.bits_words = bw;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
  L.spec = take(P * sizeof(float2));
  L.scratch = take((size_t)NS * NO * P * sizeof(float2));
  L.er = take((size_t)NO * P * 4);
  L.q = take((size_t)NO * P * 4);
  L.an0 = take((size_t)NO * P * 4);
  L.amp = (debug & 1) ? take((size_t)NO * P * 4) : (size_t)-1;
  L.pc = (debug & 2) ? take((size_t)NO * P * 4) : (size_t)-1;
  L.moment = take(P * 4);
  // rows of the stacked MIMs, at least one TMA box high (the tensor map covers them all)
  L.mim_rows = rows > 160 ? rows : 160;
  L.mim = take((size_t)L.mim_rows * L.mim_pitch);
  L.mhist = take((size_t)g * NO * MEDIAN_HIST_WORDS * 4);
  L.mstate = take((size_t)g * NO * 4 * 4);
  L.noise = take((size_t)g * NO * 4);
  L.minmax = take((size_t)g * 2 * 4);
  L.ccount = take((size_t)g * 4);
  L.cand = take((size_t)g * L.cap_cand * 8);
  const int kc = topk_sort_cap(max_kp);
  L.sortbuf = take(topk_needs_sortbuf(max_kp) ? (size_t)g * kc * 8 : 0);
  const bool multi = topk_multi_group(max_kp, gr);
  L.chist = take(multi ? (size_t)g * ((size_t)1 << TOPK_DIGIT_BITS) * 4 : 0);
  L.sel = take(multi ? (size_t)g * 4 * 4 : 0);
  L.comp = take(multi ? (size_t)g * topk_fast_cap(max_kp) * 8 : 0);
  L.raw = take((size_t)g * kp_cap * DESC_DIM * 2 * (spatial ? 2 : 1));
  L.info = take((size_t)g * kp_cap * 4);
  L.off = take((size_t)g * kp_cap * 4);
  const size_t none = (size_t)-1;
  L.mcorner = corners ? take(P * 4) : none;
  L.minmax_c = corners ? take((size_t)g * 2 * 4) : none;
  L.ccount_c = corners ? take((size_t)g * 4) : none;
  L.cxy = corners ? take((size_t)g * max_kp * 2 * 4) : none;
  L.csc = corners ? take((size_t)g * max_kp * 4) : none;
  L.ccnt = corners ? take((size_t)g * 2 * 4) : none;
  L.bits = corners ? take((size_t)g * L.bits_words * 4) : none;
  L.total = o;
  return L;
}

Layout ctx_layout(const rift2_ctx* c, const Group& gr, int debug) {
  return extract_layout(gr, c->kp.max_kp, c->kp.kp_cap, (c->p.flags & RIFT2_FLAG_CORNERS) != 0,
                        debug, c->kp.desc_mode == DESC_SPATIAL);
}

template <typename T>
T* at(void* base, size_t off) {
  return off == (size_t)-1 ? nullptr : reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// The MIM as a [g][H][pitch] uint8 tensor for the descriptor kernel's TMA staging (box
// shape: describe_box(), which depends on the descriptor mode).
// The MIMs of a group stacked row after row ([rows][pitch] uint8) as one 2-D tensor map
// for the descriptor kernel's TMA staging (box shape: describe_box(), which depends on
// the descriptor mode).  A box reaching past an image's rows reads a neighbour's rows or
// the fill value; the descriptor kernels only count pixels inside their own image.
int make_mim_map(rift2_ctx* c, CUtensorMap* tm, unsigned char* mim, int rows, int pitch) {
  cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch};
  int bw = 0, bh = 0;
  describe_box(c->kp.desc_mode, &bw, &bh);
  cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  cuuint32_t es[2] = {1, 1};
  CUresult r = c->encode(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, mim, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fprintf(stderr, "rift2: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
    return RIFT2_E_CUDA;
  }
  return RIFT2_OK;
}

int make_operand_map(rift2_ctx* c, CUtensorMap* tm, void* base, int npairs, int cap,
                     int box_rows) {
  cuuint64_t dims[3] = {256, (cuuint64_t)cap, (cuuint64_t)npairs};
  cuuint64_t strides[2] = {256 * 2, (cuuint64_t)cap * 256 * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = c->encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fprintf(stderr, "rift2: cuTensorMapEncodeTiled (operands) failed (%d)\n", (int)r);
    return RIFT2_E_CUDA;
  }
  return RIFT2_OK;
}

// Most descriptors one image can produce per keypoint under the context's mode.
int desc_per_kp(const rift2_ctx* c) { return (c->p.flags & RIFT2_FLAG_RIFT_RING) ? NO : 2; }

int check_features(const rift2_ctx* c, const rift2_features& f, bool need_desc) {
  if (!f.kp_xy || !f.kp_score || !f.counts) return RIFT2_E_INVAL;
  if (f.cap_kp < c->kp.kp_cap) return RIFT2_E_CAPACITY;
  if (need_desc) {
    if (!f.desc || !f.desc_norm || !f.desc_kp || !f.desc_dom) return RIFT2_E_INVAL;
    if (f.cap_desc < desc_per_kp(c) * c->kp.kp_cap) return RIFT2_E_CAPACITY;
  }
  return RIFT2_OK;
}

FeatPtrs feat_ptrs(const rift2_features* f, int n) {
  FeatPtrs fp{};
  for (int i = 0; i < n; ++i) {
    fp.kp_xy[i] = f[i].kp_xy;
    fp.kp_score[i] = f[i].kp_score;
    fp.desc[i] = f[i].desc;
    fp.desc_norm[i] = f[i].desc_norm;
    fp.desc_kp[i] = f[i].desc_kp;
    fp.desc_dom[i] = f[i].desc_dom;
    fp.counts[i] = f[i].counts;
  }
  return fp;
}

int copy_debug(const rift2_features* f, const Group& gr, void* ws, const Layout& L,
               cudaStream_t st) {
  for (int i = 0; i < gr.n; ++i) {
    const rift2_debug_maps* d = f[i].debug;
    if (!d) continue;
    const size_t P = (size_t)gr.P(i), pb = (size_t)gr.poff[i];
    auto cp = [&](void* dst, size_t off, size_t planes, size_t esize) -> cudaError_t {
      if (!dst || off == (size_t)-1) return cudaSuccess;
      return cudaMemcpyAsync(dst, static_cast<char*>(ws) + off + planes * pb * esize,
                             planes * P * esize, cudaMemcpyDeviceToDevice, st);
    };
    RIFT2_CU(cp(d->amp, L.amp, NO, 4));
    RIFT2_CU(cp(d->er, L.er, NO, 4));
    RIFT2_CU(cp(d->q, L.q, NO, 4));
    RIFT2_CU(cp(d->an0, L.an0, NO, 4));
    RIFT2_CU(cp(d->pc, L.pc, NO, 4));
    RIFT2_CU(cp(d->moment, L.moment, 1, 4));
    RIFT2_CU(cp(d->spectrum, L.spec, 1, sizeof(float2)));
    if (d->noise_t)
      RIFT2_CU(cudaMemcpyAsync(d->noise_t, static_cast<char*>(ws) + L.noise + (size_t)i * NO * 4,
                               NO * 4, cudaMemcpyDeviceToDevice, st));
    if (d->mim)
      RIFT2_CU(cudaMemcpy2DAsync(d->mim, gr.W[i],
                                 static_cast<char*>(ws) + L.mim + (size_t)gr.mrow[i] * L.mim_pitch,
                                 L.mim_pitch, gr.W[i], gr.H[i], cudaMemcpyDeviceToDevice, st));
  }
  return RIFT2_OK;
}

// Which optional outputs a launch group needs: bit 0 the amplitude sums, bit 1 PC (both
// need workspace of their own), bit 2 any other debug copy (no extra workspace).
int wants_debug(const rift2_features* f, int n) {
  int w = 0;
  for (int i = 0; i < n; ++i) {
    const rift2_debug_maps* d = f[i].debug;
    if (!d) continue;
    if (d->amp) w |= 1;
    if (d->pc) w |= 2;
    w |= 4;
  }
  return w;
}

// The group of images imgs[0..g) (any sizes) in the packed layout.
Group image_group(int g, const rift2_image* imgs) {
  int H[MAXB], W[MAXB];
  for (int i = 0; i < g; ++i) {
    H[i] = imgs[i].height;
    W[i] = imgs[i].width;
  }
  return make_group(g, H, W, nullptr, nullptr);
}

// One launch group: g <= MAXB images of any sizes, one launch per stage (plus one per run of
// a register-tiled size in the transform stages).
int extract_group(rift2_ctx* c, int g, const rift2_image* imgs, rift2_features* out,
                  cudaStream_t st) {
  const Group gr = image_group(g, imgs);
  FbImage fi[MAXB];
  for (int i = 0; i < g; ++i) {
    const int H = gr.H[i], W = gr.W[i];
    fi[i] = FbImage{};
    int rc = get_plan(c, H, st, &fi[i].ph);
    if (rc) return rc;
    rc = get_plan(c, W, st, &fi[i].pw);
    if (rc) return rc;
    unsigned char* zc = nullptr;
    rc = get_zero_cols(c, H, W, st, &zc);
    if (rc) return rc;
    fi[i].zc = zc;
    auto it = c->col_tiles.find(std::make_pair(H, W));
    fi[i].col_tile = it == c->col_tiles.end() ? 0 : it->second;
  }
  const int dbg = wants_debug(out, g);
  Layout L = ctx_layout(c, gr, dbg);
  int rc = ensure_ws(c, L.total);
  if (rc) return rc;
  void* ws = c->ws;
  ImgPtrs ip{};
  for (int i = 0; i < g; ++i) {
    ip.img[i] = imgs[i].data;
    ip.pitch[i] = imgs[i].pitch;
  }
  FeatPtrs fp = feat_ptrs(out, g);
  unsigned* minmax = at<unsigned>(ws, L.minmax);
  unsigned* ccount = at<unsigned>(ws, L.ccount);
  c->launches += K_INIT;
  launch_init_detect(minmax, ccount, g, st);
  const bool corners = (c->p.flags & RIFT2_FLAG_CORNERS) != 0;
  unsigned* minmax_c = corners ? at<unsigned>(ws, L.minmax_c) : nullptr;
  unsigned* ccount_c = corners ? at<unsigned>(ws, L.ccount_c) : nullptr;
  if (corners) {
    c->launches += K_INIT;
    launch_init_detect(minmax_c, ccount_c, g, st);
  }
  RIFT2_CU(cudaMemsetAsync(at<char>(ws, L.mhist), 0, (size_t)g * NO * MEDIAN_HIST_WORDS * 4, st));
  float2* spec = at<float2>(ws, L.spec);
  int nl = 0;
  {
    StageScope sc(c, RIFT2_STAGE_FFT_FWD, st, 0);
    RIFT2_CU(launch_fft2_forward(&ip, nullptr, spec, gr, fi, st, &nl));
    c->launches += nl;
  }
  float* er = at<float>(ws, L.er);
  float* q = at<float>(ws, L.q);
  float* an0 = at<float>(ws, L.an0);
  unsigned char* mim = at<unsigned char>(ws, L.mim);
  float2* scratch = at<float2>(ws, L.scratch);
  if (c->p.flags & RIFT2_FLAG_AUTOTUNE) {
    for (int i = 0; i < g; ++i) {   // each size once, on its first image
      if (i > 0 && gr.H[i] == gr.H[i - 1] && gr.W[i] == gr.W[i - 1]) {
        fi[i].col_tile = fi[i - 1].col_tile;
        continue;
      }
      rc = tune_col_tile(c, spec, scratch, gr, i, fi[i], st, &fi[i].col_tile);
      if (rc) return rc;
    }
  }
  {
    StageScope sc(c, RIFT2_STAGE_LG_COLS, st, 0);
    RIFT2_CU(launch_lg_cols(spec, scratch, gr, fi, c->kp, st, &nl));
    c->launches += nl;
  }
  {
    StageScope sc(c, RIFT2_STAGE_LG_ROWS, st, 0);
    RIFT2_CU(launch_lg_rows(scratch, gr, fi, c->kp, er, q, an0, at<float>(ws, L.amp), mim,
                            L.mim_pitch, st, &nl));
    c->launches += nl;
  }
  MedianWs mw{at<unsigned>(ws, L.mhist), at<unsigned>(ws, L.mstate), at<float>(ws, L.noise)};
  {
    StageScope sc(c, RIFT2_STAGE_NOISE, st, K_NOISE);
    RIFT2_CU(launch_noise_threshold(an0, gr, c->kp, mw, st));
  }
  float* moment = at<float>(ws, L.moment);
  {
    StageScope sc(c, RIFT2_STAGE_MOMENT, st, K_MOMENT);
    RIFT2_CU(launch_pc_moment(er, q, mw.noise_t, gr, c->kp, moment, minmax, at<float>(ws, L.pc),
                              corners ? at<float>(ws, L.mcorner) : nullptr, minmax_c, st));
  }
  DetectWs dw{minmax, at<unsigned long long>(ws, L.cand), ccount, L.cap_cand,
              at<unsigned long long>(ws, L.sortbuf), at<unsigned>(ws, L.chist),
              at<unsigned>(ws, L.sel), at<unsigned long long>(ws, L.comp)};
  {
    const int kd = detect_launches(c->kp.max_kp, gr);
    StageScope sc(c, RIFT2_STAGE_DETECT, st, corners ? 2 * kd + K_MERGE : kd);
    RIFT2_CU(launch_detect(moment, gr, c->kp, dw, fp, st));
    if (corners) {
      // corner keypoints on the minimum moment into the side list, then appended
      FeatPtrs fc{};
      int* cxy = at<int>(ws, L.cxy);
      float* csc = at<float>(ws, L.csc);
      int* ccnt = at<int>(ws, L.ccnt);
      for (int i = 0; i < g; ++i) {
        fc.kp_xy[i] = cxy + (size_t)i * c->kp.max_kp * 2;
        fc.kp_score[i] = csc + (size_t)i * c->kp.max_kp;
        fc.counts[i] = ccnt + 2 * i;
      }
      DetectWs dwc{minmax_c, at<unsigned long long>(ws, L.cand), ccount_c, L.cap_cand,
                   at<unsigned long long>(ws, L.sortbuf), at<unsigned>(ws, L.chist),
                   at<unsigned>(ws, L.sel), at<unsigned long long>(ws, L.comp)};
      RIFT2_CU(launch_detect(at<float>(ws, L.mcorner), gr, c->kp, dwc, fc, st));
      RIFT2_CU(launch_merge_corners(gr, c->kp, fp, cxy, csc, ccnt, at<unsigned>(ws, L.bits),
                                    L.bits_words, st));
    }
  }
  // images smaller than the patch keep no keypoint (fast_nms has no candidate pixel there;
  // topk_sort wrote their descriptor count 0)
  bool any_patch = false;
  for (int i = 0; i < g; ++i) any_patch |= gr.H[i] >= RIFT2_PATCH && gr.W[i] >= RIFT2_PATCH;
  if (any_patch) {
    CUtensorMap tm;
    rc = make_mim_map(c, &tm, mim, L.mim_rows, L.mim_pitch);
    if (rc) return rc;
    DescribeWs dsw{at<unsigned short>(ws, L.raw), at<unsigned>(ws, L.info), at<int>(ws, L.off),
                   c->status, c->wait_iters};
    StageScope sc(c, RIFT2_STAGE_DESCRIBE, st, K_DESCRIBE);
    RIFT2_CU(launch_describe(&tm, gr, c->kp, dsw, fp, st));
  }
  return copy_debug(out, gr, ws, L, st);
}

// The launch groups rift2_extract forms (rift2_workspace_bytes applies the same): with
// RIFT2_FLAG_NO_GROUPING one image each; with RIFT2_FLAG_SIZE_GROUPS runs of consecutive
// images of one size; otherwise all images in order of size (height, then width; equal
// sizes keep their order) cut into groups of up to MAXB images.  A group whose workspace
// exceeds the budget is halved until it fits or holds one image.  dbg[i]: the optional
// outputs image i wants (wants_debug bits; NULL: none).
void plan_groups(const rift2_ctx* c, int n, const int* H, const int* W, const int* dbg,
                 std::vector<int>& order, std::vector<int>& sizes) {
  order.resize(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  const int fl = c->p.flags;
  const bool none = (fl & RIFT2_FLAG_NO_GROUPING) != 0, same = (fl & RIFT2_FLAG_SIZE_GROUPS) != 0;
  if (!none && !same)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return H[x] != H[y] ? H[x] < H[y] : W[x] < W[y];
    });
  sizes.clear();
  int i = 0;
  while (i < n) {
    int j = i + 1;
    if (!none)
      while (j < n && j - i < MAXB &&
             (!same || (H[order[j]] == H[order[i]] && W[order[j]] == W[order[i]])))
        ++j;
    auto total = [&](int g) {
      int hh[MAXB], ww[MAXB], d = 0;
      for (int k = 0; k < g; ++k) {
        hh[k] = H[order[i + k]];
        ww[k] = W[order[i + k]];
        if (dbg) d |= dbg[order[i + k]];
      }
      return ctx_layout(c, make_group(g, hh, ww, nullptr, nullptr), d).total;
    };
    int g = j - i;
    while (g > 1 && total(g) > c->budget) g = (g + 1) / 2;
    sizes.push_back(g);
    i += g;
  }
}

// One lane's share of rift2_extract / rift2_match (defined after the C ABI entry points).
int extract_impl(rift2_ctx* c, int n, const rift2_image* imgs, rift2_features* out,
                 cudaStream_t st);
int match_impl(rift2_ctx* c, int n, const rift2_features* a, const rift2_features* b,
               rift2_matches* out, cudaStream_t st);

// RIFT2_FLAG_TWO_LANES applies to a call of n images or pairs (not while profiling, whose
// stage events are recorded on one stream).
bool two_lanes(const rift2_ctx* c, int n) {
  return (c->p.flags & RIFT2_FLAG_TWO_LANES) && !c->prof && n >= 2;
}

// The second lane: a context with the same parameters (without the flag) and budget, its
// own non-blocking stream and the fork / join events; made on first use.
int lane_of(rift2_ctx* c, rift2_ctx** out) {
  if (!c->lane) {
    rift2_params p2 = c->p;
    p2.flags &= ~RIFT2_FLAG_TWO_LANES;
    rift2_ctx* ln = nullptr;
    int rc = rift2_create(&p2, c->device, c->budget, &ln);
    if (rc) return rc;
    ln->wait_iters = c->wait_iters;
    if (cudaStreamCreateWithFlags(&c->lane_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->lane_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->lane_join, cudaEventDisableTiming) != cudaSuccess) {
      rift2_destroy(ln);
      return RIFT2_E_CUDA;
    }
    c->lane = ln;
  }
  *out = c->lane;
  return RIFT2_OK;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

void rift2_default_params(rift2_params* p) {
  if (!p) return;
  p->n_scales = 4;
  p->n_orient = 6;
  p->min_wavelength = 3.0f;
  p->mult = 1.6f;
  p->sigma_onf = 0.75f;
  p->k = 1.0f;
  p->g = 3.0f;
  p->cutoff = 0.5f;
  p->eps = 1e-4f;
  p->lp_cutoff = 0.45f;
  p->lp_order = 15;
  p->fast_threshold = 0.001f;
  p->fast_arc = 9;
  p->max_keypoints = 5000;
  p->patch = 96;
  p->cells = 6;
  p->second_ratio = 0.8f;
  p->flags = 0;
}

const char* rift2_status_str(int s) {
  switch (s) {
    case RIFT2_OK: return "ok";
    case RIFT2_E_INVAL: return "invalid argument";
    case RIFT2_E_NOMEM: return "workspace exceeds the HBM budget or allocation failed";
    case RIFT2_E_CAPACITY: return "output buffer capacity too small";
    case RIFT2_E_CUDA: return "CUDA error";
    case RIFT2_E_TIMEOUT: return "bounded device wait timed out";
    case RIFT2_E_UNIMPL: return "not implemented for this size or geometry";
    default: return "unknown status";
  }
}

}  // extern "C"

namespace {
// The parameters rift2_create accepts (defaults where params is NULL) into *p.
int validate_params(const rift2_params* params, rift2_params* out) {
  rift2_params p;
  rift2_default_params(&p);
  if (params) p = *params;
  if (p.n_scales != NS || p.n_orient != NO || p.patch != PATCH || p.cells != CELLS)
    return RIFT2_E_UNIMPL;
  if (!(p.min_wavelength > 0) || !(p.mult > 1) || !(p.sigma_onf > 0 && p.sigma_onf < 1) ||
      !(p.lp_cutoff > 0) || p.lp_order < 1 || p.fast_arc < 1 || p.fast_arc > 16 ||
      p.max_keypoints < 1 || p.max_keypoints > 32768 || !(p.fast_threshold >= 0) ||
      ((p.flags & RIFT2_FLAG_RIFT_RING) && (p.flags & RIFT2_FLAG_RIFT_TEMPLATE)) ||
      ((p.flags & RIFT2_FLAG_SPATIAL_NORM) &&
       (p.flags & (RIFT2_FLAG_RIFT_RING | RIFT2_FLAG_RIFT_TEMPLATE))) ||
      !(p.second_ratio >= 0) || !(p.eps > 0))
    return RIFT2_E_INVAL;
  *out = p;
  return RIFT2_OK;
}
constexpr size_t kDefaultBudget = (size_t)16 << 30;
}  // namespace

extern "C" {

int rift2_fft_plan(int n, int rows, int* length, int* radices, int max_radices) {
  if (n < 2 || !length || !radices || max_radices < 1) return RIFT2_E_INVAL;
  FftPlan pl{};
  int m = n;
  if (!factor_plan(n, pl, nullptr, rows == 0)) {
    if (n > 4096) return RIFT2_E_UNIMPL;
    m = bluestein_length(n);
    if (!m || !factor_plan(m, pl, nullptr, rows == 0)) return RIFT2_E_UNIMPL;
  } else if (n > 8192) {
    return RIFT2_E_UNIMPL;
  }
  if (pl.nst > max_radices) return RIFT2_E_INVAL;
  *length = m;
  for (int i = 0; i < pl.nst; ++i) radices[i] = pl.radix[i];
  return pl.nst;
}

int rift2_plan_groups(const rift2_params* params, size_t hbm_budget_bytes, int n,
                      const int* heights, const int* widths, int* order, int* sizes,
                      int* n_groups) {
  if (n < 0 || !n_groups || (n > 0 && (!heights || !widths || !order || !sizes)))
    return RIFT2_E_INVAL;
  rift2_ctx c;   // host state only: parameters, derived constants, budget
  const int rc = validate_params(params, &c.p);
  if (rc) return rc;
  derive_kparams(c.p, c.kp);
  c.budget = hbm_budget_bytes ? hbm_budget_bytes : kDefaultBudget;
  std::vector<int> ord, sz;
  plan_groups(&c, n, heights, widths, nullptr, ord, sz);
  for (int i = 0; i < n; ++i) order[i] = ord[i];
  for (size_t g = 0; g < sz.size(); ++g) sizes[g] = sz[g];
  *n_groups = (int)sz.size();
  return RIFT2_OK;
}

int rift2_create(const rift2_params* params, int device, size_t hbm_budget_bytes, rift2_ctx** out) {
  if (!out) return RIFT2_E_INVAL;
  *out = nullptr;
  rift2_params p;
  const int vrc = validate_params(params, &p);
  if (vrc) return vrc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return RIFT2_E_CUDA;
  }
  DeviceGuard dg(device);
  rift2_ctx* c = new rift2_ctx();
  c->device = device;
  c->p = p;
  derive_kparams(p, c->kp);
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : kDefaultBudget;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn) {
    delete c;
    return RIFT2_E_CUDA;
  }
  c->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) {
    delete c;
    return RIFT2_E_CUDA;
  }
  *out = c;
  return RIFT2_OK;
}

int rift2_destroy(rift2_ctx* c) {
  if (!c) return RIFT2_E_INVAL;
  DeviceGuard dg(c->device);
  cudaDeviceSynchronize();
  if (c->lane) {
    rift2_destroy(c->lane);
    cudaStreamDestroy(c->lane_st);
    cudaEventDestroy(c->lane_fork);
    cudaEventDestroy(c->lane_join);
  }
  for (auto& kv : c->plans) {
    cudaFree(const_cast<float2*>(kv.second.tw));
    if (kv.second.chirp) {
      cudaFree(const_cast<float2*>(kv.second.chirp));
      cudaFree(const_cast<float2*>(kv.second.kern_fwd));
      cudaFree(const_cast<float2*>(kv.second.kern_inv));
    }
  }
  for (float2* p : c->pass_tw) cudaFree(p);
  for (FftPasses* p : c->pass_dev) cudaFree(p);
  for (auto& kv : c->zero_cols) cudaFree(kv.second);
  for (auto& m : c->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : c->free_events) cudaEventDestroy(e);
  if (c->ws) cudaFree(c->ws);
  if (c->status) cudaFree(c->status);
  delete c;
  return RIFT2_OK;
}

int rift2_set_profiling(rift2_ctx* c, int enable) {
  if (!c) return RIFT2_E_INVAL;
  c->prof = enable != 0;
  return RIFT2_OK;
}

int rift2_profile_read(rift2_ctx* c, int n, double* ms, long long* count) {
  if (!c || n < 0) return RIFT2_E_INVAL;
  DeviceGuard dg(c->device);
  for (auto& m : c->marks) {
    if (cudaEventSynchronize(m.b) != cudaSuccess) return RIFT2_E_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) != cudaSuccess) return RIFT2_E_CUDA;
    c->acc_ms[m.stage] += t;
    c->acc_n[m.stage] += 1;
    c->free_events.push_back(m.a);
    c->free_events.push_back(m.b);
  }
  c->marks.clear();
  for (int s = 0; s < n && s < RIFT2_N_STAGES; ++s) {
    if (ms) ms[s] = c->acc_ms[s];
    if (count) count[s] = c->acc_n[s];
  }
  for (int s = 0; s < RIFT2_N_STAGES; ++s) { c->acc_ms[s] = 0; c->acc_n[s] = 0; }
  return RIFT2_OK;
}

long long rift2_launch_count(const rift2_ctx* c) {
  return c ? c->launches + (c->lane ? c->lane->launches : 0) : -1;
}

}  // extern "C"

namespace {
// Workspace of one lane for n images and n_pairs pairs (the larger of its largest launch
// group's layout and the matcher's).
size_t lane_need(const rift2_ctx* c, int n, const int* heights, const int* widths, int n_pairs) {
  size_t need = 0;
  std::vector<int> order, sizes;
  plan_groups(c, n, heights, widths, nullptr, order, sizes);   // the groups rift2_extract forms
  int i = 0;
  for (int g : sizes) {
    int hh[MAXB], ww[MAXB];
    for (int k = 0; k < g; ++k) {
      hh[k] = heights[order[i + k]];
      ww[k] = widths[order[i + k]];
    }
    const size_t t = ctx_layout(c, make_group(g, hh, ww, nullptr, nullptr), 0).total;
    if (t > need) need = t;
    i += g;
  }
  if (n_pairs > 0 && !(c->p.flags & RIFT2_FLAG_PLAIN_MATCH)) {
    const int gp = (c->p.flags & RIFT2_FLAG_NO_GROUPING) ? 1 : (n_pairs < MAXB ? n_pairs : MAXB);
    const int cap = (desc_per_kp(c) * c->kp.kp_cap + 127) / 128 * 128;
    // the autotuner's first match of a batch shape runs every split up to 4
    const int ns = (c->p.flags & RIFT2_FLAG_AUTOTUNE) ? 4 : match_tc_nsplit(gp, cap);
    const size_t t = match_tc_ws_bytes(gp, cap, ns);
    if (t > need) need = t;
  }
  return need;
}
}  // namespace

extern "C" {

int rift2_workspace_bytes(const rift2_ctx* c, int n, const int* heights, const int* widths,
                          int n_pairs, size_t* bytes) {
  if (!c || n < 0 || n_pairs < 0 || !bytes || (n > 0 && (!heights || !widths))) return RIFT2_E_INVAL;
  if (c->p.flags & RIFT2_FLAG_TWO_LANES) {
    // both lanes' workspaces: the first half of the images and pairs on this context, the
    // rest on the second lane (a call of one image or pair stays on the first)
    const int h = n >= 2 ? n / 2 : n, hp = n_pairs >= 2 ? n_pairs / 2 : n_pairs;
    *bytes = lane_need(c, h, heights, widths, hp) +
             lane_need(c, n - h, heights + h, widths + h, n_pairs - hp);
    return RIFT2_OK;
  }
  *bytes = lane_need(c, n, heights, widths, n_pairs);
  return RIFT2_OK;
}

int rift2_set_wait_limit(rift2_ctx* c, long long iters) {
  if (!c || iters < 0) return RIFT2_E_INVAL;
  c->wait_iters = iters;
  if (c->lane) c->lane->wait_iters = iters;
  return RIFT2_OK;
}

int rift2_required_capacity(const rift2_ctx* c, int* cap_kp, int* cap_desc, int* cap_match) {
  if (!c) return RIFT2_E_INVAL;
  if (cap_kp) *cap_kp = c->kp.kp_cap;
  if (cap_desc) *cap_desc = desc_per_kp(c) * c->kp.kp_cap;
  if (cap_match) *cap_match = desc_per_kp(c) * c->kp.kp_cap;
  return RIFT2_OK;
}

int rift2_tuned_tile(const rift2_ctx* c, int height, int width) {
  if (!c) return RIFT2_E_INVAL;
  auto it = c->col_tiles.find(std::make_pair(height, width));
  return it == c->col_tiles.end() ? 0 : it->second;
}

int rift2_tuned_match_split(const rift2_ctx* c, int n_pairs) {
  if (!c || n_pairs < 1) return RIFT2_E_INVAL;
  const int g = n_pairs < MAXB ? n_pairs : MAXB;
  const int cap = (desc_per_kp(c) * c->kp.kp_cap + 127) / 128 * 128;
  auto it = c->match_splits.find(std::make_pair(g, cap));
  return it == c->match_splits.end() ? 0 : it->second;
}

int rift2_sync(rift2_ctx* c, void* stream) {
  if (!c) return RIFT2_E_INVAL;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the second lane's work was joined back to the caller's stream, so its status word is
  // read in order too
  int h = 0, h2 = 0;
  if (cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (c->lane && cudaMemcpyAsync(&h2, c->lane->status, sizeof(int), cudaMemcpyDeviceToHost,
                                  st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RIFT2_E_CUDA;
  if (h || h2) {
    cudaMemsetAsync(c->status, 0, sizeof(int), st);
    if (c->lane) cudaMemsetAsync(c->lane->status, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return RIFT2_E_TIMEOUT;
  }
  return RIFT2_OK;
}

int rift2_extract(rift2_ctx* c, int n, const rift2_image* imgs, rift2_features* out, void* stream) {
  if (!c || n < 0 || (n > 0 && (!imgs || !out))) return RIFT2_E_INVAL;
  for (int i = 0; i < n; ++i) {
    if (!imgs[i].data || imgs[i].pitch < imgs[i].width) return RIFT2_E_INVAL;
    int rc = check_size(imgs[i].height, imgs[i].width);
    if (rc) return rc;
    rc = check_features(c, out[i], true);
    if (rc) return rc;
  }
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (two_lanes(c, n)) {
    rift2_ctx* ln = nullptr;
    int rc = lane_of(c, &ln);
    if (rc) return rc;
    const int h = n / 2;
    RIFT2_CU(cudaEventRecord(c->lane_fork, st));
    RIFT2_CU(cudaStreamWaitEvent(c->lane_st, c->lane_fork, 0));
    rc = extract_impl(c, h, imgs, out, st);
    if (rc) return rc;
    rc = extract_impl(ln, n - h, imgs + h, out + h, c->lane_st);
    if (rc) return rc;
    RIFT2_CU(cudaEventRecord(c->lane_join, c->lane_st));
    RIFT2_CU(cudaStreamWaitEvent(st, c->lane_join, 0));
    return RIFT2_OK;
  }
  return extract_impl(c, n, imgs, out, st);
}

}  // extern "C"

namespace {
// The extraction of n images on one lane (context c, stream st): launch groups as
// plan_groups forms them.
int extract_impl(rift2_ctx* c, int n, const rift2_image* imgs, rift2_features* out,
                 cudaStream_t st) {
  std::vector<int> hh(n), ww(n), dbg(n), order, sizes;
  for (int i = 0; i < n; ++i) {
    hh[i] = imgs[i].height;
    ww[i] = imgs[i].width;
    dbg[i] = wants_debug(out + i, 1);
  }
  plan_groups(c, n, hh.data(), ww.data(), dbg.data(), order, sizes);
  int i = 0;
  for (int g : sizes) {
    rift2_image gi[MAXB];
    rift2_features go[MAXB];
    for (int k = 0; k < g; ++k) {
      gi[k] = imgs[order[i + k]];
      go[k] = out[order[i + k]];
    }
    int rc = extract_group(c, g, gi, go, st);
    if (rc) return rc;
    i += g;
  }
  return RIFT2_OK;
}
}  // namespace

extern "C" {

int rift2_match(rift2_ctx* c, int n, const rift2_features* a, const rift2_features* b,
                rift2_matches* out, void* stream) {
  if (!c || n < 0 || (n > 0 && (!a || !b || !out))) return RIFT2_E_INVAL;
  for (int i = 0; i < n; ++i) {
    if (!a[i].desc || !b[i].desc || !a[i].counts || !b[i].counts || !a[i].desc_kp ||
        !b[i].desc_kp)
      return RIFT2_E_INVAL;
    const rift2_matches& m = out[i];
    if (!m.q_desc || !m.nn_desc || !m.kp_a || !m.kp_b || !m.d1 || !m.d2 || !m.near_tie ||
        !m.count)
      return RIFT2_E_INVAL;
    if (m.cap < desc_per_kp(c) * c->kp.kp_cap) return RIFT2_E_CAPACITY;
  }
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (two_lanes(c, n)) {
    rift2_ctx* ln = nullptr;
    int rc = lane_of(c, &ln);
    if (rc) return rc;
    const int h = n / 2;
    RIFT2_CU(cudaEventRecord(c->lane_fork, st));
    RIFT2_CU(cudaStreamWaitEvent(c->lane_st, c->lane_fork, 0));
    rc = match_impl(c, h, a, b, out, st);
    if (rc) return rc;
    rc = match_impl(ln, n - h, a + h, b + h, out + h, c->lane_st);
    if (rc) return rc;
    RIFT2_CU(cudaEventRecord(c->lane_join, c->lane_st));
    RIFT2_CU(cudaStreamWaitEvent(st, c->lane_join, 0));
    return RIFT2_OK;
  }
  return match_impl(c, n, a, b, out, st);
}

}  // extern "C"

namespace {
// The matching of n pairs on one lane (context c, stream st).
int match_impl(rift2_ctx* c, int n, const rift2_features* a, const rift2_features* b,
               rift2_matches* out, cudaStream_t st) {
  const int step = (c->p.flags & RIFT2_FLAG_NO_GROUPING) ? 1 : MAXB;
  for (int i0 = 0; i0 < n; i0 += step) {
    int g = n - i0 < step ? n - i0 : step;
    MatchPtrs mp{};
    for (int k = 0; k < g; ++k) {
      const rift2_features& fa = a[i0 + k];
      const rift2_features& fb = b[i0 + k];
      const rift2_matches& m = out[i0 + k];
      mp.desc_a[k] = fa.desc;
      mp.desc_b[k] = fb.desc;
      mp.counts_a[k] = fa.counts;
      mp.counts_b[k] = fb.counts;
      mp.desc_kp_a[k] = fa.desc_kp;
      mp.desc_kp_b[k] = fb.desc_kp;
      mp.q_desc[k] = m.q_desc;
      mp.nn_desc[k] = m.nn_desc;
      mp.kp_a[k] = m.kp_a;
      mp.kp_b[k] = m.kp_b;
      mp.d1[k] = m.d1;
      mp.d2[k] = m.d2;
      mp.near_tie[k] = m.near_tie;
      mp.count[k] = m.count;
    }
    if (c->p.flags & RIFT2_FLAG_PLAIN_MATCH) {
      StageScope sc(c, RIFT2_STAGE_MATCH, st, K_MATCH);
      RIFT2_CU(launch_match_simt(mp, g, desc_per_kp(c) * c->kp.kp_cap, st));
    } else {
      const int cap = (desc_per_kp(c) * c->kp.kp_cap + 127) / 128 * 128;
      const auto key = std::make_pair(g, cap);
      auto it = c->match_splits.find(key);
      const bool tune = (c->p.flags & RIFT2_FLAG_AUTOTUNE) && it == c->match_splits.end();
      const int nsplit = it != c->match_splits.end() ? it->second : match_tc_nsplit(g, cap);
      int rc = ensure_ws(c, match_tc_ws_bytes(g, cap, tune ? 4 : nsplit));
      if (rc) return rc;
      void *abf, *bbf;
      match_tc_operands(c->ws, g, cap, &abf, &bbf);
      CUtensorMap ta, tb;
      rc = make_operand_map(c, &ta, abf, g, cap, match_tc_box_rows(0));
      if (rc) return rc;
      rc = make_operand_map(c, &tb, bbf, g, cap, match_tc_box_rows(1));
      if (rc) return rc;
      if (tune) {
        // every split computes the same matches: time each on this call's descriptors
        // (a warm-up, then two timed launches each) and keep the fastest; the last run
        // leaves the call's results in place
        cudaEvent_t ev[5];
        for (int k = 0; k < 5; ++k) RIFT2_CU(cudaEventCreate(&ev[k]));
        RIFT2_CU(launch_match_tc(mp, g, cap, c->ws, &ta, &tb, 1, c->status, st));
        c->launches += K_MATCH_TC * 9;
        RIFT2_CU(cudaEventRecord(ev[0], st));
        for (int k = 1; k <= 4; ++k) {
          for (int r = 0; r < 2; ++r)
            RIFT2_CU(launch_match_tc(mp, g, cap, c->ws, &ta, &tb, k, c->status, st));
          RIFT2_CU(cudaEventRecord(ev[k], st));
        }
        RIFT2_CU(cudaEventSynchronize(ev[4]));
        int best = 1;
        float best_ms = 1e30f;
        for (int k = 1; k <= 4; ++k) {
          float ms = 0.f;
          RIFT2_CU(cudaEventElapsedTime(&ms, ev[k - 1], ev[k]));
          if (ms < best_ms) { best_ms = ms; best = k; }
        }
        for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
        c->match_splits[key] = best;
        continue;
      }
      StageScope sc(c, RIFT2_STAGE_MATCH, st, K_MATCH_TC);
      RIFT2_CU(launch_match_tc(mp, g, cap, c->ws, &ta, &tb, nsplit, c->status, st));
    }
  }
  return RIFT2_OK;
  return RIFT2_OK;
}
}  // namespace

extern "C" {

int rift2_evaluate(rift2_ctx* c, int n, const rift2_features* a, const rift2_features* b,
                   const rift2_matches* m, const double* affine, double tol, double rmse_cap,
                   int min_correct, rift2_evaluation* out, void* stream) {
  if (!c || n < 1 || n > MAXB || !a || !b || !m || !affine || !out || !(tol > 0) ||
      !(rmse_cap >= 0))
    return RIFT2_E_INVAL;
  EvalPtrs ep{};
  for (int i = 0; i < n; ++i) {
    if (!a[i].kp_xy || !b[i].kp_xy || !m[i].kp_a || !m[i].kp_b || !m[i].count)
      return RIFT2_E_INVAL;
    ep.xy_a[i] = a[i].kp_xy;
    ep.xy_b[i] = b[i].kp_xy;
    ep.kp_a[i] = m[i].kp_a;
    ep.kp_b[i] = m[i].kp_b;
    ep.count[i] = m[i].count;
  }
  for (int i = 0; i < 6 * n; ++i) ep.affine[i] = affine[i];   // passed by value
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ep.out = out;
  c->launches += 1;
  RIFT2_CU(launch_evaluate(ep, n, tol, rmse_cap, min_correct, st));
  return RIFT2_OK;
}

int rift2_fft2(rift2_ctx* c, int n, const float* img, int H, int W, float* out, void* stream) {
  if (!c || n < 1 || !img || !out) return RIFT2_E_INVAL;
  int rc = check_size(H, W);
  if (rc) return rc;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FbImage f{};
  rc = get_plan(c, H, st, &f.ph);
  if (rc) return rc;
  rc = get_plan(c, W, st, &f.pw);
  if (rc) return rc;
  FbImage fi[MAXB];
  for (int k = 0; k < MAXB; ++k) fi[k] = f;
  const long long P = (long long)H * W;
  for (int i0 = 0; i0 < n; i0 += MAXB) {
    const int g = n - i0 < MAXB ? n - i0 : MAXB;
    Group gr = uniform_group(g, H, W, P);   // the caller's dense [n][H][W] layout
    int nl = 0;
    RIFT2_CU(launch_fft2_forward(nullptr, img + (size_t)i0 * P,
                                 reinterpret_cast<float2*>(out) + (size_t)i0 * P, gr, fi, st, &nl));
    c->launches += nl;
  }
  return RIFT2_OK;
}

int rift2_detect(rift2_ctx* c, int n, const float* moment, int H, int W, rift2_features* out,
                 void* stream) {
  if (!c || n < 1 || !moment || !out || H < 16 || W < 16) return RIFT2_E_INVAL;
  for (int i = 0; i < n; ++i) {
    int rc = check_features(c, out[i], false);
    if (rc) return rc;
  }
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long P = (long long)H * W;
  for (int i0 = 0; i0 < n; i0 += MAXB) {
    int g = n - i0 < MAXB ? n - i0 : MAXB;
    const Group gr = uniform_group(g, H, W, P);   // the caller's dense [n][H][W] maps
    Layout L = ctx_layout(c, gr, 0);
    int rc = ensure_ws(c, L.total);
    if (rc) return rc;
    unsigned* minmax = at<unsigned>(c->ws, L.minmax);
    unsigned* ccount = at<unsigned>(c->ws, L.ccount);
    c->launches += K_INIT + 1 + detect_launches(c->kp.max_kp, gr);
    launch_init_detect(minmax, ccount, g, st);
    const float* m = moment + (size_t)i0 * P;
    launch_minmax(m, g, P, minmax, st);
    FeatPtrs fp = feat_ptrs(out + i0, g);
    DetectWs dw{minmax, at<unsigned long long>(c->ws, L.cand), ccount, L.cap_cand,
                at<unsigned long long>(c->ws, L.sortbuf), at<unsigned>(c->ws, L.chist),
                at<unsigned>(c->ws, L.sel), at<unsigned long long>(c->ws, L.comp)};
    RIFT2_CU(launch_detect(m, gr, c->kp, dw, fp, st));
  }
  return RIFT2_OK;
}

int rift2_describe(rift2_ctx* c, int n, const unsigned char* mim, int H, int W,
                   rift2_features* feats, void* stream) {
  if (!c || n < 1 || !mim || !feats || H < RIFT2_PATCH || W < RIFT2_PATCH) return RIFT2_E_INVAL;
  for (int i = 0; i < n; ++i) {
    int rc = check_features(c, feats[i], true);
    if (rc) return rc;
  }
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i0 = 0; i0 < n; i0 += MAXB) {
    int g = n - i0 < MAXB ? n - i0 : MAXB;
    const Group gr = uniform_group(g, H, W, padded_px(H, W));
    Layout L = ctx_layout(c, gr, 0);
    int rc = ensure_ws(c, L.total);
    if (rc) return rc;
    unsigned char* wm = at<unsigned char>(c->ws, L.mim);
    RIFT2_CU(cudaMemcpy2DAsync(wm, L.mim_pitch, mim + (size_t)i0 * H * W, W, W, (size_t)g * H,
                               cudaMemcpyDeviceToDevice, st));
    CUtensorMap tm;
    rc = make_mim_map(c, &tm, wm, L.mim_rows, L.mim_pitch);
    if (rc) return rc;
    FeatPtrs fp = feat_ptrs(feats + i0, g);
    c->launches += K_DESCRIBE;
    DescribeWs dsw{at<unsigned short>(c->ws, L.raw), at<unsigned>(c->ws, L.info),
                   at<int>(c->ws, L.off), c->status, c->wait_iters};
    RIFT2_CU(launch_describe(&tm, gr, c->kp, dsw, fp, st));
  }
  return RIFT2_OK;
}

}  // extern "C"
