// Shared device-side definitions of the RIFT2 kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rift2.h"

namespace rift2 {

constexpr int NS = RIFT2_NS;
constexpr int NO = RIFT2_NO;
constexpr int PATCH = RIFT2_PATCH;
constexpr int HALF_PATCH = RIFT2_PATCH / 2;
constexpr int CELLS = RIFT2_CELLS;
constexpr int CELL = RIFT2_PATCH / RIFT2_CELLS;  // 16
constexpr int DESC_DIM = RIFT2_DESC_DIM;         // 216
constexpr int MAXB = RIFT2_MAX_BATCH;

// Device status word values (latched by bounded waits).
constexpr int ST_TIMEOUT = 1;

// Scalar parameters the kernels read, derived on the host in double precision and
// rounded once to float.
struct KParams {
  float log_fs[NS];      // ln(centre frequency of scale s)
  float inv_2ls2;        // 1 / (2 ln^2 sigma_onf)
  float inv_lp_c2;       // 1 / lp_cutoff^2
  int lp_order;
  float cos_o[NO], sin_o[NO];   // orientation angle o*pi/No
  float eps, g, cutoff, inv_ns1;
  float noise_c;         // T_o = median * noise_c (tau, scale sum and Rayleigh stats)
  float fast_t;
  int fast_arc;
  int max_kp;            // keypoints one detector pass keeps
  int kp_cap;            // keypoint list capacity per image (2 max_kp with corners)
  int ratio_pm;          // dominant ratio in per mille (integer comparison)
  int desc_mode;         // DESC_RIFT2, DESC_RIFT_TEMPLATE, DESC_RIFT_RING or DESC_SPATIAL
  int rot_c[NO], rot_s[NO];   // cos / sin of o pi / No in Q14, rounded half away from zero
};

// Descriptor modes: RIFT2's dominant index (one or two per keypoint), RIFT's template
// (unshifted MIM, one per keypoint) and RIFT's reference ring (No per keypoint).
// DESC_SPATIAL: RIFT2's descriptors on a patch grid rotated into the dominant index's frame
// (a variant the paper does not have; see desc_spatial).
constexpr int DESC_RIFT2 = 0, DESC_RIFT_TEMPLATE = 1, DESC_RIFT_RING = 2, DESC_SPATIAL = 3;

// Per-launch-group pointers to the caller's buffers (passed by value).
struct FeatPtrs {
  int* kp_xy[MAXB];
  float* kp_score[MAXB];
  unsigned short* desc[MAXB];
  float* desc_norm[MAXB];
  int* desc_kp[MAXB];
  unsigned char* desc_dom[MAXB];
  int* counts[MAXB];
};

struct ImgPtrs {
  const float* img[MAXB];
  long long pitch[MAXB];
};

// The images of one launch group, which may differ in size (passed by value to the
// kernels of every stage; image i of the group is blockIdx.y or .z == i, and CTAs past
// the extent of a smaller image return at once).  Per-pixel workspace planes are packed
// image after image: image i's pixels start at pixel poff[i] of a plane, so a buffer of k
// planes per pixel holds image i from k * poff[i] on; its MIM rows start at row mrow[i]
// of the MIM buffer.  The extraction pads each image's pixel count to a multiple of 64,
// so every plane of every image starts 256-byte aligned.
struct Group {
  int n;
  int H[MAXB], W[MAXB];
  int mrow[MAXB];
  long long poff[MAXB];
  __host__ __device__ long long P(int i) const { return (long long)H[i] * W[i]; }
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// Complex add / subtract as one packed two-lane f32 instruction each (sm_100 and later):
// the same round-to-nearest sums as two scalar adds, in half the issue slots.  The FFT
// butterflies are mostly these.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
      "add.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
      "sub.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// DFT bin k of an n-point transform in cycles per sample (numpy fftfreq order).
__device__ __forceinline__ float fftfreq(int k, int n) {
  int kk = (k < (n + 1) / 2) ? k : k - n;
  return (float)kk / (float)n;
}

}  // namespace rift2
