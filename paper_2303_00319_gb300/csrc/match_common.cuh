// Exact nearest-neighbour comparisons shared by the matching kernels.
//
// Descriptor entries are integer counts (each cell sums to 256), so a.b and |b|^2 are
// integers below 2^24 and the comparison of normalised similarities
//     a.b_j / |b_j|  >  a.b_k / |b_k|   <=>   (a.b_j)^2 |b_k|^2  >  (a.b_k)^2 |b_j|^2
// is decided exactly in 64-bit integers (the products stay below 2^64); ties go to the
// lower index.  The distance ||a/|a| - b/|b|||^2 = 2 (|a|^2|b|^2 - (a.b)^2) /
// ((|a||b| + a.b) |a||b|) uses the exact integer numerator, so it keeps full relative
// precision even for nearly identical descriptors.
#pragma once

#include "common.cuh"

namespace rift2 {

struct Cand {
  float dot;
  float n2;
  int j;
};

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  unsigned long long da = (unsigned long long)a.dot, db = (unsigned long long)b.dot;
  unsigned long long lhs = da * da * (unsigned long long)b.n2;
  unsigned long long rhs = db * db * (unsigned long long)a.n2;
  return lhs > rhs || (lhs == rhs && a.j < b.j);
}

__device__ __forceinline__ void push2(Cand& c1, Cand& c2, const Cand& x) {
  if (better(x, c1)) { c2 = c1; c1 = x; }
  else if (better(x, c2)) { c2 = x; }
}

__device__ __forceinline__ float exact_dist(float n2a, const Cand& c) {
  unsigned long long na = (unsigned long long)n2a, nb = (unsigned long long)c.n2;
  unsigned long long dt = (unsigned long long)c.dot;
  unsigned long long num = na * nb - dt * dt;        // >= 0 (Cauchy-Schwarz), exact
  float nn = sqrtf((float)(na * nb));
  return 2.f * (float)num / ((nn + c.dot) * nn);
}


}  // namespace rift2
