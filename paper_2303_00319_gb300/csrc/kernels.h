// Host-side launchers of the RIFT2 kernels (one translation unit per stage group).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"

namespace rift2 {

// k_filterbank.cu
void launch_twiddles(float2* tw, int n, cudaStream_t st);
// The passes of a plan as pass_twiddle_gather reads them: pass st has radix R[st], ns[st]
// and its twiddles from off[st] on; total = sum of ns (R - 1) = L - 1.
struct PassDims {
  int nst, total;
  int R[FFT_MAX_STAGES], ns[FFT_MAX_STAGES], off[FFT_MAX_STAGES];
};
void launch_pass_twiddles(float2* ptw, const float2* tw, int L, const PassDims& pd,
                          cudaStream_t st);
// Bluestein tables of a length-n transform run as a length-m convolution (FftPlan);
// c64 [n] and tw64 [m] are FP64 scratch the caller frees after the stream has passed.
void launch_bluestein_tables(float2* chirp, float2* kf, float2* ki, double2* c64, double2* tw64,
                             int n, int m, cudaStream_t st);
// Per-image inputs of the filter-bank launchers: the plans of the image's height and
// width, its zero-window column table (zc [NO][W]: 1 where orientation o's angular window
// is zero on the whole column u) and its column tile (0: the default).
struct FbImage {
  FftPlan ph, pw;
  const unsigned char* zc;
  int col_tile;
};
// Each launcher walks the group in runs of one size (register-tiled kernels per run where
// the side allows, one shared-memory launch for the rest) and reports the kernels it
// enqueued in *launches.  Buffers are packed as the Group describes.
cudaError_t launch_fft2_forward(const ImgPtrs* ip, const float* dense, float2* spec,
                                const Group& gr, const FbImage* fi, cudaStream_t st,
                                int* launches);
void launch_zero_cols(int H, int W, const KParams& kp, unsigned char* zc, cudaStream_t st);
// Column tiles (columns per CTA) the shared-memory column pass can use for height H, the
// default first; none for the register-tiled heights.  FbImage::col_tile picks one; every
// tile computes the same result.
int lg_cols_tile_candidates(int H, int L, int* out, int max_n);
cudaError_t launch_lg_cols(const float2* spec, float2* scratch, const Group& gr,
                           const FbImage* fi, const KParams& kp, cudaStream_t st, int* launches);
cudaError_t launch_lg_rows(float2* scratch, const Group& gr, const FbImage* fi,
                           const KParams& kp, float* er, float* q, float* an0, float* amp,
                           unsigned char* mim, int mim_pitch, cudaStream_t st, int* launches);

// k_pc.cu — exact median of |EO_0,o| (radix select), noise thresholds, PC, moments.
// Global histogram words per (image, orientation): 32768 round-0 buckets, 65536 round-1
// buckets for each middle rank, then the counts of 512 chunks of each of the three
// histograms.  Zero before launch_noise_threshold.
constexpr int MEDIAN_HIST_WORDS = 32768 + 2 * 65536 + 3 * 512;
struct MedianWs {
  unsigned* hist;    // [nimg][NO][MEDIAN_HIST_WORDS]
  unsigned* state;   // [nimg][NO][2][2]  (prefix, rank)
  float* noise_t;    // [nimg][NO]
};
cudaError_t launch_noise_threshold(const float* an0, const Group& gr, const KParams& kp,
                                   MedianWs ws, cudaStream_t st);
// mcorner / minmax_c (both NULL unless corners are wanted): the minimum moment without its
// -eps/2 offset (>= 0, the same FAST input up to the min-max normalisation) and its min / max.
cudaError_t launch_pc_moment(const float* er, const float* q, const float* noise_t,
                             const Group& gr, const KParams& kp, float* moment, unsigned* minmax,
                             float* pc_out, float* mcorner, unsigned* minmax_c, cudaStream_t st);

// k_detect.cu — FAST + NMS on the normalised moment map, then top-K.
struct DetectWs {
  const unsigned* minmax;       // [nimg][2] float bits of min / max of M
  unsigned long long* cand;     // [nimg][cap_cand]
  unsigned* cand_count;         // [nimg]
  int cap_cand;
  unsigned long long* sortbuf;  // [nimg][topk_sort_cap(max_kp)] when max_kp exceeds both
                                // shared-memory sorts (max_kp > TOPK_SMEM_ANY_CAP), else unused
  // Multi-CTA selection (all NULL: topk_sort refines on the full list by itself):
  unsigned* cand_hist;          // [nimg][2^TOPK_DIGIT_BITS] counts of the stored keys' leading digits
  unsigned* sel;                // [nimg][4] digit, keys selected, fast flag, gathered count
  unsigned long long* comp;     // [nimg][topk_fast_cap(max_kp)] the compacted selection
};
// Keys the top-K sort holds: the smallest power of two >= max_kp (at least 256).
__host__ __device__ inline int topk_sort_cap(int max_kp) {
  int c = 256;
  while (c < max_kp) c <<= 1;
  return c;
}
constexpr int TOPK_SMEM_CAP = 16384;       // power-of-two sort in shared memory
constexpr int TOPK_SMEM_ANY_CAP = 26624;   // any-size sort in shared memory (208 KB)
constexpr int TOPK_DIGIT_BITS = 16;       // leading key bits of the selection histogram
// Keys a fast selection may hand to the shared-memory sort (0: the global-memory sort
// always refines on the full list).
__host__ __device__ inline int topk_fast_cap(int max_kp) {
  const int kc = topk_sort_cap(max_kp);
  return kc <= TOPK_SMEM_CAP ? kc : (max_kp <= TOPK_SMEM_ANY_CAP ? TOPK_SMEM_ANY_CAP : 0);
}
// The multi-CTA selection pays for its histogram and two extra launches only when an image
// can hold many more candidates than one CTA scans quickly: maps above 4 MPix.
inline bool topk_multi(int max_kp, int H, int W) {
  return topk_fast_cap(max_kp) > 0 && (long long)H * W > (1ll << 22);
}
// A group takes the multi-CTA selection for all its images when one of them needs it (the
// selected keypoints are the same either way).
inline bool topk_multi_group(int max_kp, const Group& gr) {
  for (int i = 0; i < gr.n; ++i)
    if (topk_multi(max_kp, gr.H[i], gr.W[i])) return true;
  return false;
}
inline bool topk_needs_sortbuf(int max_kp) {
  return topk_sort_cap(max_kp) > TOPK_SMEM_CAP && max_kp > TOPK_SMEM_ANY_CAP;
}
cudaError_t launch_detect(const float* moment, const Group& gr, const KParams& kp, DetectWs ws,
                          const FeatPtrs& fp, cudaStream_t st);
// min = +inf bits, max = 0, candidate counts = 0 for g images
void launch_init_detect(unsigned* minmax, unsigned* ccount, int g, cudaStream_t st);
// Appends each image's corner keypoints (cxy / csc / ccnt[2 i], max_kp per image) after its
// edge keypoints in fp, leaving out pixels already among the edge keypoints (order kept);
// bits: scratch of bits_stride >= ceil(H W / 32) words per image.
cudaError_t launch_merge_corners(const Group& gr, const KParams& kp, const FeatPtrs& fp,
                                 const int* cxy, const float* csc, const int* ccnt,
                                 unsigned* bits, long long bits_stride, cudaStream_t st);
// image-wide min / max of g non-negative maps [g][P] (ordered-int atomics)
void launch_minmax(const float* m, int g, long long P, unsigned* minmax, cudaStream_t st);
// worst-case number of NMS survivors of an H x W map (one per 2 x 2 block)
inline int detect_cap_candidates(int H, int W) { return ((H + 1) / 2) * ((W + 1) / 2); }

// rift2_api.cu — scalar kernel parameters derived from the public parameter struct
void derive_kparams(const rift2_params& p, KParams& k);

// k_describe.cu — MIM patch histograms, dominant index, recoded descriptors.
struct DescribeWs {
  unsigned short* raw;   // [nimg][max_kp][216]
  unsigned* info;        // [nimg][max_kp]
  int* off;              // [nimg][max_kp]
  int* status;           // device status word
  long long wait_iters;  // limit of the first wait on each staged patch half
};
// Box (columns, rows) of the MIM tensor map the descriptor kernel of `desc_mode` stages.
void describe_box(int desc_mode, int* cols, int* rows);
// mim_map: 2-D tensor map over the group's MIMs stacked row after row (Group::mrow).
cudaError_t launch_describe(const CUtensorMap* mim_map, const Group& gr, const KParams& kp,
                            DescribeWs ws, const FeatPtrs& fp, cudaStream_t st);

// k_match.cu — brute-force nearest neighbour.
struct MatchPtrs {
  const unsigned short* desc_a[MAXB];
  const unsigned short* desc_b[MAXB];
  const int* counts_a[MAXB];
  const int* counts_b[MAXB];
  const int* desc_kp_a[MAXB];
  const int* desc_kp_b[MAXB];
  int* q_desc[MAXB];
  int* nn_desc[MAXB];
  int* kp_a[MAXB];
  int* kp_b[MAXB];
  float* d1[MAXB];
  float* d2[MAXB];
  unsigned char* near_tie[MAXB];
  int* count[MAXB];
};
cudaError_t launch_match_simt(const MatchPtrs& mp, int npairs, int max_desc, cudaStream_t st);

// k_evaluate.cu — ground-truth evaluation of correspondences under known transforms.
struct EvalPtrs {
  const int* xy_a[MAXB];
  const int* xy_b[MAXB];
  const int* kp_a[MAXB];
  const int* kp_b[MAXB];
  const int* count[MAXB];
  double affine[MAXB * 6];     // per pair (x', y') = (t0 x + t1 y + t2, t3 x + t4 y + t5)
  rift2_evaluation* out;       // device [npairs]
};
cudaError_t launch_evaluate(const EvalPtrs& ep, int npairs, double tol, double rmse_cap,
                            int min_correct, cudaStream_t st);

// k_match_tc.cu — tcgen05 BF16 distance GEMM fused with a top-4 screen per column half,
// certified exact re-rank, exhaustive pass for the uncertified queries.
// `cap` (descriptor rows per pair) must be a multiple of 128.
size_t match_tc_ws_bytes(int npairs, int cap, int nsplit);
int match_tc_nsplit(int npairs, int cap);
void match_tc_operands(void* ws, int npairs, int cap, void** abf, void** bbf);
int match_tc_box_rows(int operand);   // 0: A (queries), 1: B
cudaError_t launch_match_tc(const MatchPtrs& mp, int npairs, int cap, void* ws,
                            const CUtensorMap* tmA, const CUtensorMap* tmB, int nsplit,
                            int* status, cudaStream_t st);

}  // namespace rift2
