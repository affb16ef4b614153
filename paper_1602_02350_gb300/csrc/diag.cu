// Speed-up diagnostic of Sec. 2 (the ratio after Thm 1, plotted against k in Fig. 1):
//   ratio(k) = sum_i lambda_i / (k lambda_k + sum_{i>k} lambda_i),
// evaluated from a sketch: the numerator is tr(C) (exact, one pass), lambda_i (i <= k) are the
// sketched eigenvalues sigma~_i^2 and the tail sum is tr(C) - sum_{i<=k} sigma~_i^2.  With
// acceleration the paper's speed-up is the square root of the same ratio.
#include <cmath>

#include "common.cuh"

namespace {

// One thread walks k = 1..kmax in order (the prefix sum is a fixed left-to-right sum, so the
// result does not depend on the launch shape); kmax is at most a few thousand.
__global__ void speedup_ratio_kernel(const double* __restrict__ sigma2, int64_t kmax, double trace_c,
                                     double* __restrict__ ratio, double* __restrict__ ratio_accel) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double head = 0.0;
  for (int64_t k = 1; k <= kmax; ++k) {
    const double s = sigma2[k - 1];
    head += s;
    const double den = (double)k * s + (trace_c - head);
    const double r = den > 0.0 ? trace_c / den : NAN;
    ratio[k - 1] = r;
    if (ratio_accel) ratio_accel[k - 1] = r >= 0.0 ? sqrt(r) : NAN;
  }
}

}  // namespace

extern "C" int rs_speedup_ratio(rs_ctx* ctx, const double* sigma2, int64_t kmax, double trace_c, double* ratio,
                                double* ratio_accel) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(sigma2 && ratio, "rs_speedup_ratio: null argument");
  RS_CHECK_ARG(kmax >= 1 && kmax <= 65536, "rs_speedup_ratio: need 1 <= kmax <= 65536 (got %lld)", (long long)kmax);
  RS_CHECK_ARG(std::isfinite(trace_c) && trace_c > 0.0, "rs_speedup_ratio: tr(C) must be finite and positive");
  speedup_ratio_kernel<<<1, 32, 0, ctx->stream>>>(sigma2, kmax, trace_c, ratio, ratio_accel);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}
