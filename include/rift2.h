/*
 * rift2.h — C ABI of the GB300 (sm_103a) RIFT2 feature pipeline.
 *
 * RIFT2 (Li, Shi, Hu, Zhang, "RIFT2: Speeding-up RIFT with A New Rotation-Invariance
 * Technique") matches multimodal images in three stages (§II, Fig. 1): keypoint
 * detection on the phase-congruency maximum-moment map (§II-A), description by
 * 6x6-cell histograms of the maximum index map (MIM, §II-B) normalised by the dominant
 * index (§III, Eq. 1 and Eq. 2), and brute-force nearest-feature matching (§IV).
 * This library runs those stages as hand-written CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 *  - All data pointers are DEVICE pointers on the context's device unless stated.
 *    The caller owns every image, feature and match buffer; the context owns its plans,
 *    twiddle tables and workspace.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Every call only enqueues work on that stream and returns; results are ready once
 *    the stream has reached that point.  Calls on one context must not run concurrently
 *    from several host threads, and work on one context is serialised on the streams it
 *    is given (the workspace is shared).
 *  - Return codes: RIFT2_OK (0) or a negative RIFT2_E_*.  Argument errors are detected
 *    on the host before anything is enqueued.  Errors found on the device (a bounded
 *    wait that ran out) are latched in a device status word that rift2_sync() returns.
 *  - Indices are 0-based.  The paper's 1-based orientation / bin index is value + 1.
 */
#ifndef RIFT2_H_
#define RIFT2_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RIFT2_VERSION_MAJOR 0
#define RIFT2_VERSION_MINOR 1

/* The kernels are compiled for the paper's bank and descriptor geometry:
 * Ns = 4 scales, No = 6 orientations (§II), patch 96 (Table 1), 6x6 cells (§II-B). */
#define RIFT2_NS 4
#define RIFT2_NO 6
#define RIFT2_PATCH 96
#define RIFT2_CELLS 6
#define RIFT2_DESC_DIM (RIFT2_CELLS * RIFT2_CELLS * RIFT2_NO) /* 216 */
#define RIFT2_MAX_BATCH 32      /* images (or pairs) per internal launch group */

enum {
  RIFT2_OK = 0,
  RIFT2_E_INVAL = -1,     /* bad argument (NULL pointer, size, parameter out of range) */
  RIFT2_E_NOMEM = -2,     /* workspace would exceed the HBM budget or cudaMalloc failed */
  RIFT2_E_CAPACITY = -3,  /* a caller buffer is smaller than the worst case it may hold */
  RIFT2_E_CUDA = -4,      /* a CUDA runtime call failed (launch, copy, sync) */
  RIFT2_E_TIMEOUT = -5,   /* a bounded device wait gave up (reported by rift2_sync) */
  RIFT2_E_UNIMPL = -6     /* valid request outside what the kernels are built for */
};

/* Flags (rift2_params.flags). */
#define RIFT2_FLAG_PLAIN_MATCH 0x1   /* CUDA-core matcher instead of the tcgen05 one */
#define RIFT2_FLAG_NO_GROUPING 0x2   /* one image / pair per launch (plain form) */
/* RIFT's own rotation handling (§II-C), the baseline RIFT2 replaces: a "template" image gets
 * one descriptor per keypoint from the unshifted MIM, a "reference" image gets the No
 * descriptors of the convolution-sequence ring, one per initial layer w = 0..No-1, i.e. the
 * MIM recoded by (MIM - w) mod No.  Without either flag: RIFT2's dominant-index descriptors
 * (§III).  The ring needs cap_desc >= No * max_keypoints. */
#define RIFT2_FLAG_RIFT_TEMPLATE 0x4
#define RIFT2_FLAG_RIFT_RING 0x8
/* RIFT's corner keypoints (§II-A: FAST on the minimum moment, which measures cornerness,
 * beside the edge keypoints on the maximum moment): FAST with the same threshold, NMS and
 * ordering on the min-max normalised minimum moment, at most max_keypoints of them,
 * appended after the edge keypoints with pixels already among the edge keypoints left out.
 * The keypoint capacity doubles: cap_kp >= 2 * max_keypoints, and cap_desc / the match
 * capacity double with it.  rift2_detect (the stage entry) ignores the flag. */
#define RIFT2_FLAG_CORNERS 0x10
/* Tune per image size and per match batch (no counterpart in the paper): the first
 * extraction of a size whose column transforms run in shared memory times each candidate
 * column tile (columns per CTA) on that call's own data, and the first tensor-core match
 * of a batch shape (pairs per launch group, descriptor capacity) times each split of B's
 * columns over 1 to 4 CTAs per query block; each synchronises the stream once and keeps
 * the fastest for the context.  Every tile and every split computes bit-identical results
 * (the matcher's candidates are re-ranked exactly and certified).  Without the flag the
 * defaults are used.  rift2_tuned_tile and rift2_tuned_match_split report the choices. */
#define RIFT2_FLAG_AUTOTUNE 0x20
/* Spatial orientation normalisation of the patch (a variant the paper does not have: §III
 * normalises rotation through the dominant index alone, which leaves the 6x6 cell layout
 * axis-aligned).  The dominant / secondary index comes from the MIM histogram over the
 * disc of radius 48 around the keypoint; each descriptor's 96 x 96 grid is rotated by
 * w pi / No (w its index), or that + 180 degrees when the centroid of the disc pixels with
 * MIM == w lies behind the axis, in Q14 fixed point with rounding half away from zero;
 * samples outside the image are not counted; counts are recoded by w (Eq. 2).  Not with
 * RIFT2_FLAG_RIFT_TEMPLATE / RIFT2_FLAG_RIFT_RING (RIFT2_E_INVAL). */
#define RIFT2_FLAG_SPATIAL_NORM 0x40
/* Launch groups of one image size only (consecutive images of equal size share launches,
 * in call order).  Without it rift2_extract orders the call's images by size and lets up
 * to RIFT2_MAX_BATCH images of any sizes share one launch per stage; each image's results
 * are bit-identical either way. */
#define RIFT2_FLAG_SIZE_GROUPS 0x80
/* Two lanes (no counterpart in the paper): rift2_extract and rift2_match run the second
 * half of a call's images / pairs on a second internal stream and context (forked from
 * and joined back to the caller's stream with events), so that one half's under-filled
 * stages (top-K sort, median selection, re-rank) overlap the other half's kernels.  Each
 * lane keeps its own workspace within the HBM budget, so the context may hold up to twice
 * the budget; results are bit-identical to one lane.  Calls with one image or one pair,
 * and calls with profiling on, run on one lane. */
#define RIFT2_FLAG_TWO_LANES 0x100

/*
 * Pipeline parameters.  Defaults (rift2_default_params) follow Table 1 (5000 keypoints,
 * patch 96, FAST threshold 0.001, dominant ratio 0.8), §II-B (6x6 grid, No bins) and
 * the log-Gabor bank of §II (Ns = 4, No = 6, minimum wavelength 3, multiplier 1.6);
 * the paper is silent on the remaining values, which follow the Kovesi phase-congruency
 * model RIFT builds on: sigma_onf 0.75, k 1, g 3, cutoff 0.5, eps 1e-4, low-pass cutoff
 * 0.45 of order 15.  n_scales, n_orient, patch and cells must equal the RIFT2_* values
 * above; anything else returns RIFT2_E_UNIMPL.
 */
typedef struct rift2_params {
  int   n_scales;        /* Ns */
  int   n_orient;        /* No */
  float min_wavelength;  /* wavelength of the finest scale, px */
  float mult;            /* wavelength ratio between scales */
  float sigma_onf;       /* radial bandwidth: sigma of the log-Gaussian / centre freq */
  float k;               /* noise threshold = mean + k sigma of the noise energy */
  float g;               /* sharpness of the frequency-spread weight */
  float cutoff;          /* frequency-spread cutoff of the weight */
  float eps;             /* small constant guarding divisions */
  float lp_cutoff;       /* low-pass cutoff, cycles/px */
  int   lp_order;        /* low-pass order n: 1 / (1 + (r/c)^(2n)) */
  float fast_threshold;  /* FAST threshold on the min-max normalised moment map */
  int   fast_arc;        /* contiguous circle pixels required (9 of 16) */
  int   max_keypoints;   /* strongest keypoints kept per image (1..32768) */
  int   patch;           /* descriptor patch side, px */
  int   cells;           /* cells per patch side */
  float second_ratio;    /* second dominant bin kept if >= ratio * peak (integer test) */
  int   flags;           /* RIFT2_FLAG_* */
} rift2_params;

typedef struct rift2_ctx rift2_ctx;

/* One grey image: float32 in [0, 1], row-major, `pitch` elements between rows. */
typedef struct rift2_image {
  const float* data;
  int height, width;
  long long pitch;
} rift2_image;

/*
 * Optional per-image intermediate maps (any member may be NULL; all float32 unless
 * stated).  Used to check each stage against the oracle.
 *   amp    [No][H][W]  A_o = sum_s |EO_s,o|                                (§II-B)
 *   er     [No][H][W]  phase-congruency energy before the noise threshold
 *   q      [No][H][W]  frequency-spread weight / A_o
 *   an0    [No][H][W]  |EO_0,o|, the smallest-scale amplitude (noise estimate)
 *   pc     [No][H][W]  PC_o                                                 (§II-A)
 *   moment [H][W]      maximum moment M (edge map FAST runs on)             (§II-A)
 *   mim    [H][W]      uint8 maximum index map, values 0..No-1              (§II-B)
 *   noise_t [No]       noise thresholds T_o
 *   spectrum [H][W]    complex (re, im float32) forward DFT F of the image (§II-B)
 * amp and pc need workspace of their own (NO * H * W * 4 bytes each per image of the launch
 * group); the others are copies of what the pipeline keeps anyway.
 */
typedef struct rift2_debug_maps {
  float* amp;
  float* er;
  float* q;
  float* an0;
  float* pc;
  float* moment;
  unsigned char* mim;
  float* noise_t;
  float* spectrum;
} rift2_debug_maps;

/*
 * Features of one image (outputs of rift2_extract; inputs of rift2_match).
 *   kp_xy     int32 [cap_kp][2]      keypoint (x, y), strongest first
 *   kp_score  float [cap_kp]         FAST score
 *   desc      uint16 [cap_desc][216] descriptor counts, cell-major (6x6 row-major), bin
 *                                    minor, bins recoded by the dominant index (Eq. 2)
 *   desc_norm float [cap_desc]       L2 norm of the count vector (descriptor = desc/norm)
 *   desc_kp   int32 [cap_desc]       keypoint each descriptor belongs to
 *   desc_dom  uint8 [cap_desc]       index the MIM was recoded by (dominant index, or the
 *                                    ring's initial layer; 0..No-1)
 *   counts    int32 [2]              written on the device: n_kp, n_desc
 * cap_kp >= max_keypoints and cap_desc >= 2 * max_keypoints are required (each keypoint
 * yields one or two descriptors, §III; No * max_keypoints with RIFT2_FLAG_RIFT_RING; both
 * doubled with RIFT2_FLAG_CORNERS), otherwise RIFT2_E_CAPACITY.
 */
typedef struct rift2_features {
  int cap_kp, cap_desc;
  int* kp_xy;
  float* kp_score;
  unsigned short* desc;
  float* desc_norm;
  int* desc_kp;
  unsigned char* desc_dom;
  int* counts;
  rift2_debug_maps* debug;   /* HOST pointer to a struct of device pointers, or NULL */
} rift2_features;

/*
 * Putative correspondences of one pair (§IV: nearest feature distance, no ratio test,
 * no RANSAC).  Row i is descriptor i of image A:
 *   q_desc = i, nn_desc = nearest descriptor of B, kp_a / kp_b their keypoints,
 *   d1 / d2 = smallest and second-smallest ||a/|a| - b/|b|||^2 (d2 = +inf if B has one
 *   descriptor), near_tie = 1 if (d2 - d1) < 1e-5 * max(d1, 1e-12).
 *   count = number of rows (= n_desc of A), written on the device.
 * cap >= 2 * max_keypoints is required (No * max_keypoints with RIFT2_FLAG_RIFT_RING;
 * doubled with RIFT2_FLAG_CORNERS).
 */
typedef struct rift2_matches {
  int cap;
  int* q_desc;
  int* nn_desc;
  int* kp_a;
  int* kp_b;
  float* d1;
  float* d2;
  unsigned char* near_tie;
  int* count;
} rift2_matches;

/* Fills *p with the defaults listed above. */
void rift2_default_params(rift2_params* p);

/* Human-readable name of a status code (static storage). */
const char* rift2_status_str(int status);

/*
 * Creates a context on CUDA device `device`.  `params` may be NULL (defaults); it is
 * copied.  `hbm_budget_bytes` caps the workspace the context may allocate (0 = 16 GiB);
 * the workspace grows on demand up to it and is freed by rift2_destroy.
 * Errors: RIFT2_E_INVAL (bad params / out == NULL), RIFT2_E_UNIMPL (geometry other
 * than Ns=4, No=6, patch 96, 6x6 cells), RIFT2_E_CUDA (device cannot be used).
 */
int rift2_create(const rift2_params* params, int device, size_t hbm_budget_bytes,
                 rift2_ctx** out);

/*
 * Extracts keypoints and descriptors of `n_images` images (§II-A, §II-B, §III):
 * log-Gabor bank in the frequency domain -> MIM and phase congruency -> maximum
 * moment -> FAST + NMS + top-K -> dominant-index-recoded 6x6xNo descriptors.
 * imgs[i] (host array of n_images structs; data on the device) -> out[i] (host array).
 * Each side must be >= 16, and either 13-smooth (prime factors in {2, 3, 5, 7, 11, 13})
 * up to 8192 or any length up to 4096 (Bluestein transforms); images smaller than patch
 * + 6 on a side produce zero keypoints.  Launch groups: up to RIFT2_MAX_BATCH images of
 * any sizes share one launch per stage (the images taken in order of size; one launch per
 * run of equal size for the register-tiled transforms of power-of-two sides), split
 * further while a group's workspace exceeds the HBM budget; RIFT2_FLAG_SIZE_GROUPS keeps
 * one size per group, RIFT2_FLAG_NO_GROUPING one image.
 * Errors: RIFT2_E_INVAL, RIFT2_E_UNIMPL (size), RIFT2_E_CAPACITY, RIFT2_E_NOMEM,
 * RIFT2_E_CUDA.
 */
int rift2_extract(rift2_ctx* ctx, int n_images, const rift2_image* imgs,
                  rift2_features* out, void* stream);

/*
 * Brute-force nearest-neighbour matching of `n_pairs` feature pairs, A -> B (§IV).
 * a[i], b[i], out[i] are host arrays of structs whose buffers are on the device; the
 * descriptor counts are read on the device (counts[1]).  Lowest B index wins exact ties.
 * Errors: RIFT2_E_INVAL, RIFT2_E_CAPACITY, RIFT2_E_NOMEM, RIFT2_E_CUDA.
 */
int rift2_match(rift2_ctx* ctx, int n_pairs, const rift2_features* a,
                const rift2_features* b, rift2_matches* out, void* stream);

/*
 * Ground-truth evaluation of putative correspondences (§IV: a correspondence is correct
 * when the matched keypoint of image B lies within `tol` px (3 in the paper) of where the
 * keypoint of image A lands under the known transform; the RMSE is taken over the correct
 * ones and capped at `rmse_cap` (20); a pair succeeds with at least `min_correct` (10)
 * correct ones).  Pair i: a[i], b[i] the features (kp_xy read on the device), m[i] its
 * matches A -> B (m.count rows; rows whose kp_a or kp_b is -1 are not correspondences),
 * affine: HOST array [n_pairs][6] of the transform of image A's pixel coordinates into
 * image B's, (x', y') = (t0 x + t1 y + t2, t3 x + t4 y + t5).  out: DEVICE array of
 * n_pairs structs, written asynchronously.  Residuals in FP64.  The transforms travel in
 * the kernel's parameters: the host array may be reused once the call returns.
 * Errors: RIFT2_E_INVAL (NULL pointers, n_pairs outside 1..32, tol <= 0), RIFT2_E_CUDA.
 */
typedef struct rift2_evaluation {
  int n_matches;   /* rows that are correspondences */
  int n_correct;   /* residual < tol */
  int success;     /* n_correct >= min_correct */
  int reserved;
  double rmse;     /* over the correct rows, capped at rmse_cap (rmse_cap if none) */
} rift2_evaluation;
int rift2_evaluate(rift2_ctx* ctx, int n_pairs, const rift2_features* a,
                   const rift2_features* b, const rift2_matches* m, const double* affine,
                   double tol, double rmse_cap, int min_correct, rift2_evaluation* out,
                   void* stream);

/* Waits for `stream`, then returns and clears the device status word (RIFT2_OK or
 * RIFT2_E_TIMEOUT), or RIFT2_E_CUDA if the stream reported an error. */
int rift2_sync(rift2_ctx* ctx, void* stream);

/* Frees the context and its workspace (waits for the device first). */
int rift2_destroy(rift2_ctx* ctx);

/* The column tile the autotuner chose for images of H x W in this context: the tile (>= 1),
 * 0 if none was tuned (flag off, the size not seen yet, or a register-tiled height), or
 * RIFT2_E_INVAL for a NULL context.  No counterpart in the paper. */
int rift2_tuned_tile(const rift2_ctx* ctx, int height, int width);

/* The split of B's columns the autotuner chose for tensor-core match launches of n_pairs
 * pairs in this context (1 to 4 CTAs per block of 128 queries), 0 if none was tuned, or
 * RIFT2_E_INVAL for a NULL context.  No counterpart in the paper. */
int rift2_tuned_match_split(const rift2_ctx* ctx, int n_pairs);

/* ------------------------------------------------------------------------------
 * Tracing.  With profiling on, the context brackets every stage of every launch group
 * with CUDA events on the call's stream (a few microseconds of overhead per stage);
 * rift2_profile_read waits for those events and reports the accumulated device time.
 * The launch counter counts every kernel the library enqueues, profiling on or off.
 * ---------------------------------------------------------------------------- */
enum {
  RIFT2_STAGE_FFT_FWD = 0,   /* forward 2-D DFT of the images                       */
  RIFT2_STAGE_LG_COLS = 1,   /* column pass of the 24 filtered inverse DFTs          */
  RIFT2_STAGE_LG_ROWS = 2,   /* row pass + amplitude / MIM / PC-energy reductions    */
  RIFT2_STAGE_NOISE = 3,     /* exact median of |EO_0,o| and noise thresholds        */
  RIFT2_STAGE_MOMENT = 4,    /* phase congruency and maximum moment                  */
  RIFT2_STAGE_DETECT = 5,    /* FAST + NMS + top-K                                   */
  RIFT2_STAGE_DESCRIBE = 6,  /* patch histograms, dominant index, descriptors        */
  RIFT2_STAGE_MATCH = 7,     /* nearest-neighbour matching                           */
  RIFT2_N_STAGES = 8
};

/* Turns per-stage event timing on (1) or off (0). */
int rift2_set_profiling(rift2_ctx* ctx, int enable);

/* Waits for the recorded events and writes, for each stage s < n, the device time
 * accumulated since the last reset (ms[s]) and the number of timed launches of that
 * stage (count[s]); either array may be NULL.  Then clears the accumulators. */
int rift2_profile_read(rift2_ctx* ctx, int n, double* ms, long long* count);

/* Kernels enqueued by this context since it was created. */
long long rift2_launch_count(const rift2_ctx* ctx);

/* Host-only planning queries (no device, no context): what the library decides before it
 * launches anything, so that a caller (or a test) can inspect it.  No counterpart in the
 * paper.
 *
 * rift2_fft_plan: the transform the shared-memory kernels run for a side of length n: the
 * pass length (*length = n for 13-smooth n, else the Bluestein convolution length chosen
 * by the planner, 2n - 1 <= *length <= 2.5 n + 1) and its radices in pass order (radices
 * [max_radices] host array; rows != 0: the row kernels' plan, which has no radix 16).
 * Returns the number of passes, RIFT2_E_UNIMPL when n cannot be planned (n > 4096 with a
 * prime factor above 13, n > 8192), RIFT2_E_INVAL for n < 2, NULL pointers or too small
 * a radices array. */
int rift2_fft_plan(int n, int rows, int* length, int* radices, int max_radices);

/* rift2_plan_groups: the launch groups rift2_extract forms for n_images images of the
 * given sizes under params (flags NO_GROUPING / SIZE_GROUPS, the descriptor mode and the
 * keypoint budget set the workspace) and an HBM budget (0: rift2_create's default,
 * 16 GiB): order[n_images]
 * receives the images in launch order, sizes[n_images] the size of each group in turn;
 * *n_groups their number.  Host arrays.  Errors: RIFT2_E_INVAL (params as rift2_create
 * validates them, NULL arrays, n_images < 0). */
int rift2_plan_groups(const rift2_params* params, size_t hbm_budget_bytes, int n_images,
                      const int* heights, const int* widths, int* order, int* sizes,
                      int* n_groups);

/* Device workspace the context needs for rift2_extract of n_images images of the given
 * sizes (host arrays; grouped as rift2_extract groups them, no debug maps) followed by
 * rift2_match of n_pairs pairs: the largest launch group's layout or the matcher's (the
 * workspace is one buffer reused by every group and by the matcher; with
 * RIFT2_FLAG_TWO_LANES the sum of both lanes' workspaces for their halves).  For admission
 * control by a serving loop; no counterpart in the paper.  *bytes is written.
 * Errors: RIFT2_E_INVAL. */
int rift2_workspace_bytes(const rift2_ctx* ctx, int n_images, const int* heights,
                          const int* widths, int n_pairs, size_t* bytes);

/* ------------------------------------------------------------------------------
 * Capacities and failure paths (no counterpart in the paper).
 * ---------------------------------------------------------------------------- */

/* The buffer capacities this context's calls require (the worst case of its parameters):
 * rift2_features.cap_kp, .cap_desc and rift2_matches.cap.  A call given less returns
 * RIFT2_E_CAPACITY before enqueuing anything; this reports the counts it needed.  Any
 * pointer may be NULL.  Errors: RIFT2_E_INVAL (NULL context). */
int rift2_required_capacity(const rift2_ctx* ctx, int* cap_kp, int* cap_desc, int* cap_match);

/* Iteration limit of the FIRST bounded wait on each staged patch half in the descriptor
 * kernel (default 2^24 polls of mbarrier.try_wait, far beyond a copy's latency).  When it
 * runs out the kernel latches RIFT2_E_TIMEOUT in the status word, waits for its copies in
 * flight with the full default limit (so none outlives the kernel) and returns; the
 * descriptors of that call are then invalid and rift2_sync reports RIFT2_E_TIMEOUT.  0
 * makes every such wait give up at once: a way to exercise the timeout path without a
 * fault.  Errors: RIFT2_E_INVAL (NULL context, iters < 0). */
int rift2_set_wait_limit(rift2_ctx* ctx, long long iters);

/* ------------------------------------------------------------------------------
 * Stage entry points.  Each runs one stage of the pipeline on caller-supplied inputs
 * so that the stage can be checked against the oracle in isolation (an oracle near-tie
 * upstream then cannot cascade).  Same conventions as above.
 * ---------------------------------------------------------------------------- */

/* Forward 2-D DFT (no scaling) of n real images img [n][H][W] -> out [n][H][W] complex
 * (interleaved re, im float32): the first step of the frequency-domain log-Gabor
 * filtering of §II-B. */
int rift2_fft2(rift2_ctx* ctx, int n, const float* img, int height, int width,
               float* out, void* stream);

/* Keypoints from given maximum-moment maps moment [n][H][W] (§II-A, Table 1): min-max
 * normalisation, FAST, 3x3 NMS, top max_keypoints.  Writes kp_xy, kp_score and
 * counts[0] of out[i]; counts[1] is set to 0. */
int rift2_detect(rift2_ctx* ctx, int n, const float* moment, int height, int width,
                 rift2_features* out, void* stream);

/* Descriptors (§II-B, §III, Eq. 1-2) of given keypoints on given MIMs mim [n][H][W]
 * (uint8, 0..No-1).  feats[i].kp_xy and feats[i].counts[0] are inputs (every keypoint
 * must satisfy 48 <= x < W-48, 48 <= y < H-48); desc, desc_norm, desc_kp, desc_dom and
 * counts[1] are written. */
int rift2_describe(rift2_ctx* ctx, int n, const unsigned char* mim, int height, int width,
                   rift2_features* feats, void* stream);

/* ------------------------------------------------------------------------------
 * Allocation-free keypoint detection.  The paper has no counterpart: this is a service
 * for callers that must not allocate device memory — code whose device memory belongs
 * to a framework's caching allocator, real-time loops that cannot absorb the implicit
 * device synchronisation of cudaMalloc / cudaFree, and hosts that budget every byte of
 * device memory in advance.
 *
 * rift2_detect_static does what rift2_detect does for ONE map (min-max normalisation,
 * FAST, 3x3 NMS, top max_keypoints of moment [H][W], device pointer) without a context:
 * it calls no cudaMalloc, cudaFree or allocating library routine.  Its only scratch
 * memory is a fixed file-scope device array of RIFT2_STATIC_MAX_CANDIDATES candidate
 * slots (about 2 MiB), which every GPU that loads the library holds until the process
 * exits.  A map needs ceil(H/2) * ceil(W/2) slots (any 1024 x 1024 map fits); larger
 * maps are refused with RIFT2_E_CAPACITY before anything is enqueued.
 *  - params: NULL for the defaults; out: kp_xy, kp_score, counts (cap_kp >= max_keypoints).
 *  - Runs on the calling thread's current device and the given stream; `moment` and the
 *    three output buffers must be device memory of that device (RIFT2_E_INVAL otherwise,
 *    checked with cudaPointerGetAttributes before anything is enqueued).
 *  - The first call on a device looks up the array's device address; make that first call
 *    before any CUDA stream capture.  The address belongs to the device's primary context:
 *    the library keeps the context's handle beside it and looks the address up again when
 *    a later call finds another context current (e.g. after cudaDeviceReset); such a call
 *    is again a first call and must not happen during a capture.
 *  - Every call shares the one array (it keeps the last call's contents; each call resets
 *    what must start at zero).  Calls whose work overlaps on the GPU (other streams, other
 *    host threads, concurrent graph launches) race on it: serialise them.
 * ---------------------------------------------------------------------------- */
#define RIFT2_STATIC_MAX_CANDIDATES 262144
int rift2_detect_static(const rift2_params* params, const float* moment, int height, int width,
                        rift2_features* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RIFT2_H_ */
