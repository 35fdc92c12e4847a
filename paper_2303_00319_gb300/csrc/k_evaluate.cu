// Ground-truth evaluation of putative correspondences (§IV's protocol: a correspondence is
// correct when the matched keypoint of image B lies within tol pixels of where the keypoint
// of image A lands under the known transform; RMSE over the correct ones, capped; a pair
// succeeds with at least min_correct correct correspondences).
//
//   eval_pairs : one CTA per pair.  Thread t takes the rows t, t + 256, ...; residuals in
//                FP64 (the same formula and order for every row), then a fixed-shape tree
//                reduction of the count and the squared residuals, so the result does not
//                depend on scheduling.
#include "kernels.h"

namespace rift2 {

constexpr int EV_NT = 256;

__global__ void __launch_bounds__(EV_NT) eval_pairs(const __grid_constant__ EvalPtrs ep, double tol, double rmse_cap,
                                                   int min_correct) {
  __shared__ double ssq[EV_NT];
  __shared__ int scnt[EV_NT], sval[EV_NT];
  const int pr = blockIdx.x;
  const int n = *ep.count[pr];
  const double* t = ep.affine + 6 * pr;   // kernel parameter space
  const double t0 = t[0], t1 = t[1], t2 = t[2], t3 = t[3], t4 = t[4], t5 = t[5];
  double sq = 0.0;
  int cnt = 0, valid = 0;
  for (int i = threadIdx.x; i < n; i += EV_NT) {
    const int ka = ep.kp_a[pr][i], kb = ep.kp_b[pr][i];
    if (ka < 0 || kb < 0) continue;   // no correspondence (image B had no descriptor)
    ++valid;
    const double ax = ep.xy_a[pr][2 * ka], ay = ep.xy_a[pr][2 * ka + 1];
    const double bx = ep.xy_b[pr][2 * kb], by = ep.xy_b[pr][2 * kb + 1];
    const double ex = fma(t0, ax, fma(t1, ay, t2)) - bx;
    const double ey = fma(t3, ax, fma(t4, ay, t5)) - by;
    const double r2 = fma(ex, ex, ey * ey);
    if (r2 < tol * tol) {
      ++cnt;
      sq += r2;
    }
  }
  ssq[threadIdx.x] = sq;
  scnt[threadIdx.x] = cnt;
  sval[threadIdx.x] = valid;
  __syncthreads();
  for (int h = EV_NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      ssq[threadIdx.x] += ssq[threadIdx.x + h];
      scnt[threadIdx.x] += scnt[threadIdx.x + h];
      sval[threadIdx.x] += sval[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rift2_evaluation r{};
    r.n_matches = sval[0];
    r.n_correct = scnt[0];
    r.success = scnt[0] >= min_correct ? 1 : 0;
    const double rmse = scnt[0] ? sqrt(ssq[0] / scnt[0]) : rmse_cap;
    r.rmse = rmse < rmse_cap ? rmse : rmse_cap;
    ep.out[pr] = r;
  }
}

cudaError_t launch_evaluate(const EvalPtrs& ep, int npairs, double tol, double rmse_cap,
                            int min_correct, cudaStream_t st) {
  eval_pairs<<<npairs, EV_NT, 0, st>>>(ep, tol, rmse_cap, min_correct);
  return cudaGetLastError();
}

}  // namespace rift2
