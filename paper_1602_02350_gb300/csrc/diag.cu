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

// ------------------------------------------------------------------ bounded-wait check
// Every device-side wait of this library is bounded: it gives up after a budget of clock cycles,
// sets the timeout bit of the context's status word and lets the kernel finish, so that the host
// reports RS_ETIMEOUT and the context stays usable.  rs_wait_probe runs that path on purpose:
// one thread initialises an mbarrier expecting one arrival, arrives on it only if `complete`, and
// waits for its phase with the same bounded wait the pipelined kernels use.
namespace {
__global__ void wait_probe_kernel(long long budget, int complete, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init_cta(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  if (complete) mbar_arrive_cta(&bar);
  if (!mbar_wait_bounded(&bar, 0u, budget)) atomicOr(status, STATUS_TIMEOUT);
}
}  // namespace

extern "C" int rs_wait_probe(rs_ctx* ctx, int64_t budget_cycles, int32_t complete) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(budget_cycles >= 1 && budget_cycles <= 4000000000LL,
               "rs_wait_probe: budget must be in [1, 4e9] cycles (about two seconds)");
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  wait_probe_kernel<<<1, 32, 0, ctx->stream>>>((long long)budget_cycles, complete ? 1 : 0, ctx->d_status);
  RS_LAUNCH_CHECK(ctx);
  int st = 0;
  RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (st & STATUS_TIMEOUT) return rs_fail(RS_ETIMEOUT, "rs_wait_probe: the bounded wait gave up after %lld cycles",
                                          (long long)budget_cycles);
  return RS_OK;
}
