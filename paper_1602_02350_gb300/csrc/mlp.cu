// Parameter-proposal network on the GPU: batched inference, training steps (a fused forward and
// backward pass per block of 32 samples that writes per-block gradient partials, then one kernel
// that sums the partials in block order and applies Adam), and rs_propose with the theory-set
// fallback of Sec. 3 / Thm 1.
#include <cmath>

#include "common.cuh"

namespace {

constexpr int IN = RS_MLP_IN, HID = RS_MLP_HIDDEN, OUT = RS_MLP_OUT, NP = RS_MLP_NPARAM;
constexpr float kInputClip = 3.0f;   // normalised inputs are clipped to this many training spreads
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + OUT * HID;
static_assert(OB3 + OUT == NP, "parameter layout");
static_assert(HID == 128 && OUT <= 4, "one thread per hidden unit, one warp per output");
constexpr int TS = 32;       // samples per thread block
constexpr int NT = HID;      // threads per block: thread i owns hidden unit i
constexpr int W1S = IN + 2;  // row strides in shared memory, chosen so that the accesses of a
constexpr int XS = IN + 1;   // warp fall on distinct banks (odd word strides for per-thread rows)
constexpr int HS = HID + 1;
constexpr int W2S = HID + 1;

constexpr size_t mlp_smem_bytes(bool train) {
  return sizeof(float) * ((size_t)HID * W1S + (size_t)HID * W2S + TS * XS + 2 * TS * HS +
                          (train ? 2 * TS * HS + TS * OUT + NT / 32 : 0));
}

template <bool TRAIN>
__global__ void __launch_bounds__(NT) mlp_kernel(const float* __restrict__ theta, const float* __restrict__ X,
                                                 int64_t B, const float* __restrict__ T, float* __restrict__ out,
                                                 float* __restrict__ part, float* __restrict__ loss_part) {
  extern __shared__ __align__(16) float mlp_sh[];
  float* w1 = mlp_sh;              // [HID][W1S]  W1 row-major
  float* w2 = w1 + HID * W1S;      // [HID][W2S]  W2 row-major
  float* xs = w2 + HID * W2S;      // [TS][XS]    inputs (zero rows beyond the batch)
  float* h1 = xs + TS * XS;        // [TS][HS]    ReLU(a1)
  float* h2 = h1 + TS * HS;        // [TS][HS]    ReLU(a2)
  float* g2 = h2 + TS * HS;        // [TS][HS]    d loss / d a2       (training only)
  float* g1 = g2 + TS * HS;        // [TS][HS]    d loss / d a1
  float* go = g1 + TS * HS;        // [TS][OUT]   d loss / d output
  float* red = go + TS * OUT;      // [NT / 32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const int nb = (int)min64(TS, B - s0);
  for (int e = tid; e < HID * IN; e += NT) w1[(e / IN) * W1S + e % IN] = theta[OW1 + e];
  for (int e = tid; e < HID * HID; e += NT) w2[(e / HID) * W2S + e % HID] = theta[OW2 + e];
  for (int e = tid; e < TS * IN; e += NT) {
    const int s = e / IN, j = e % IN;
    xs[s * XS + j] = s < nb ? X[(s0 + s) * IN + j] : 0.f;
  }
  __syncthreads();
  const int i = tid;
  {
    float acc[TS];
    const float bi = theta[OB1 + i];
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = bi;
    for (int j = 0; j < IN; ++j) {
      const float w = w1[i * W1S + j];
#pragma unroll
      for (int s = 0; s < TS; ++s) acc[s] = fmaf(w, xs[s * XS + j], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TS; ++s) h1[s * HS + i] = fmaxf(acc[s], 0.f);
  }
  __syncthreads();
  {
    float acc[TS];
    const float bi = theta[OB2 + i];
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = bi;
    for (int j = 0; j < HID; ++j) {
      const float w = w2[i * W2S + j];
#pragma unroll
      for (int s = 0; s < TS; ++s) acc[s] = fmaf(w, h1[s * HS + j], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TS; ++s) h2[s * HS + i] = fmaxf(acc[s], 0.f);
  }
  __syncthreads();
  // output layer: warp o computes output o, lane s sample s
  float sq = 0.f;
  if (warp < OUT) {
    const int o = warp, s = lane;
    float a = theta[OB3 + o];
    for (int j = 0; j < HID; ++j) a = fmaf(theta[OW3 + o * HID + j], h2[s * HS + j], a);
    if constexpr (!TRAIN) {
      if (s < nb) out[(s0 + s) * OUT + o] = a;
    } else {
      const float dlt = s < nb ? a - T[(s0 + s) * OUT + o] : 0.f;
      go[s * OUT + o] = 2.f * dlt / (float)B;
      sq = dlt * dlt;
    }
  }
  if constexpr (TRAIN) {
    sq = warp_sum(sq);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      loss_part[blockIdx.x] = t;
    }
    {   // g2 = relu'(a2) (W3^T go)
      float w3[OUT];
#pragma unroll
      for (int o = 0; o < OUT; ++o) w3[o] = theta[OW3 + o * HID + i];
#pragma unroll 4
      for (int s = 0; s < TS; ++s) {
        float g = 0.f;
#pragma unroll
        for (int o = 0; o < OUT; ++o) g = fmaf(w3[o], go[s * OUT + o], g);
        g2[s * HS + i] = h2[s * HS + i] > 0.f ? g : 0.f;
      }
    }
    __syncthreads();
    {   // g1 = relu'(a1) (W2^T g2)
      float acc[TS];
#pragma unroll
      for (int s = 0; s < TS; ++s) acc[s] = 0.f;
      for (int j = 0; j < HID; ++j) {
        const float w = w2[j * W2S + i];
#pragma unroll
        for (int s = 0; s < TS; ++s) acc[s] = fmaf(w, g2[s * HS + j], acc[s]);
      }
#pragma unroll
      for (int s = 0; s < TS; ++s) g1[s * HS + i] = h1[s * HS + i] > 0.f ? acc[s] : 0.f;
    }
    __syncthreads();
    // this block's share of the gradient (samples beyond the batch have zero go, g2, g1)
    float* P = part + (int64_t)blockIdx.x * NP;
#pragma unroll
    for (int o = 0; o < OUT; ++o) {
      float a = 0.f;
#pragma unroll 8
      for (int s = 0; s < TS; ++s) a = fmaf(go[s * OUT + o], h2[s * HS + tid], a);
      P[OW3 + o * HID + tid] = a;
    }
    if (tid < OUT) {
      float a = 0.f;
      for (int s = 0; s < TS; ++s) a += go[s * OUT + tid];
      P[OB3 + tid] = a;
    }
    for (int r = 0; r < HID; ++r) {
      float a = 0.f;
#pragma unroll 8
      for (int s = 0; s < TS; ++s) a = fmaf(g2[s * HS + r], h1[s * HS + tid], a);
      P[OW2 + r * HID + tid] = a;
    }
    {
      float a = 0.f;
      for (int s = 0; s < TS; ++s) a += g2[s * HS + tid];
      P[OB2 + tid] = a;
    }
    for (int e = tid; e < HID * IN; e += NT) {
      const int r = e / IN, j = e % IN;
      float a = 0.f;
#pragma unroll 8
      for (int s = 0; s < TS; ++s) a = fmaf(g1[s * HS + r], xs[s * XS + j], a);
      P[OW1 + e] = a;
    }
    {
      float a = 0.f;
      for (int s = 0; s < TS; ++s) a += g1[s * HS + tid];
      P[OB1 + tid] = a;
    }
  }
}

// g = sum of the block partials in block order; Adam with bias corrections bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t.  Thread 0 also reduces the loss partials.
__global__ void mlp_adam_kernel(float* __restrict__ theta, float* __restrict__ am, float* __restrict__ av,
                                const float* __restrict__ part, int nblk, float lr, float b1, float b2, float eps,
                                float bc1, float bc2, float inv_b, float* __restrict__ grad_out,
                                const float* __restrict__ loss_part, float* __restrict__ loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    float t = 0.f;
    for (int b = 0; b < nblk; ++b) t += loss_part[b];
    *loss_out = t * inv_b;
  }
  if (p >= NP) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += part[(int64_t)b * NP + p];
  if (grad_out) grad_out[p] = g;
  const float m = b1 * am[p] + (1.f - b1) * g;
  const float v = b2 * av[p] + (1.f - b2) * g * g;
  am[p] = m;
  av[p] = v;
  theta[p] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

int launch_forward(rs_ctx* ctx, const float* theta, const float* X, int64_t B, float* out) {
  constexpr size_t shm = mlp_smem_bytes(false);
  RS_CUDA_TRY(cudaFuncSetAttribute(mlp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  mlp_kernel<false><<<(unsigned)((B + TS - 1) / TS), NT, shm, ctx->stream>>>(theta, X, B, nullptr, out, nullptr,
                                                                              nullptr);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

// Thm 1 runtime model: kappa~(k) = (k sigma_k^2 + tr(C) - sum_{i<=k} sigma_i^2) / lambda
double kappa_tilde(const double* sigma2, double trace_c, double lambda, int k) {
  double head = 0.0;
  for (int i = 0; i < k; ++i) head += sigma2[i];
  return ((double)k * sigma2[k - 1] + (trace_c - head)) / lambda;
}

}  // namespace

extern "C" {

int rs_mlp_forward(rs_ctx* ctx, const float* theta, const float* X, int64_t B, float* out) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(theta && X && out && B >= 1, "rs_mlp_forward: null argument or empty batch");
  return launch_forward(ctx, theta, X, B, out);
}

int rs_mlp_train_step(rs_ctx* ctx, float* theta, float* adam_m, float* adam_v, const float* X, const float* T,
                      int64_t B, const rs_adam_params* p, float* grad_out, float* loss_out) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(theta && adam_m && adam_v && X && T && p && B >= 1, "rs_mlp_train_step: null argument or empty batch");
  RS_CHECK_ARG(p->step >= 1 && p->lr > 0.f && p->beta1 >= 0.f && p->beta1 < 1.f && p->beta2 >= 0.f && p->beta2 < 1.f &&
                   p->eps > 0.f,
               "rs_mlp_train_step: bad Adam parameters");
  const int64_t nblk = (B + TS - 1) / TS;
  RS_CHECK_ARG(nblk <= (1 << 20), "rs_mlp_train_step: batch too large");
  float* part = static_cast<float*>(rs_scratch(ctx, SCR_MLP_PART, ((size_t)nblk * NP + nblk) * sizeof(float)));
  if (!part) return RS_ENOMEM;
  float* loss_part = part + (size_t)nblk * NP;
  constexpr size_t shm = mlp_smem_bytes(true);
  RS_CUDA_TRY(cudaFuncSetAttribute(mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  mlp_kernel<true><<<(unsigned)nblk, NT, shm, ctx->stream>>>(theta, X, B, T, nullptr, part, loss_part);
  RS_LAUNCH_CHECK(ctx);
  const double bc1 = 1.0 - std::pow((double)p->beta1, (double)p->step);
  const double bc2 = 1.0 - std::pow((double)p->beta2, (double)p->step);
  mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, ctx->stream>>>(theta, adam_m, adam_v, part, (int)nblk, p->lr, p->beta1,
                                                             p->beta2, p->eps, (float)bc1, (float)bc2,
                                                             (float)(1.0 / (double)B), grad_out, loss_part, loss_out);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int rs_propose(rs_ctx* ctx, const float* theta, const rs_mlp_norm* norm, const double* sigma2, double lambda,
               int64_t n, int64_t d, double trace_c, int32_t* k, double* eta_mult, int64_t* m,
               int32_t* used_fallback) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(sigma2 && k && eta_mult && m && used_fallback, "rs_propose: null argument");
  RS_CHECK_ARG(lambda > 0.0 && n >= 1 && d >= 1 && std::isfinite(trace_c) && trace_c >= 0.0,
               "rs_propose: need lambda > 0, n, d >= 1 and a finite tr(C) >= 0");
  for (int i = 0; i < 64; ++i)
    RS_CHECK_ARG(std::isfinite(sigma2[i]) && sigma2[i] >= 0.0 && (i == 0 || sigma2[i] <= sigma2[i - 1]),
                 "rs_propose: sigma2 must hold 64 finite, non-negative, descending values");
  const int K = (int)min64(64, d);
  // theory setting: k minimises the Thm 1 runtime model, eta = 0.1 / beta^, m = ceil(beta^ / lambda)
  int kb = 1;
  double cb = INFINITY;
  for (int kk = 1; kk <= K; ++kk) {
    const double c = (double)n * (double)d * kk + (kappa_tilde(sigma2, trace_c, lambda, kk) + (double)n + (double)d) * d;
    if (c < cb) {
      cb = c;
      kb = kk;
    }
  }
  *k = kb;
  *eta_mult = 0.1;
  *m = (int64_t)std::ceil(kappa_tilde(sigma2, trace_c, lambda, kb) + (double)d);
  *used_fallback = 1;
  if (!theta || !norm) return RS_OK;
  float x[IN];
  // log-spectrum and log lambda relative to the leading sketched value (invariant to the scale of
  // X), log n, log d; normalised, then clipped to kInputClip training spreads
  const double ls0 = 0.5 * std::log(std::fmax(sigma2[0], 1e-60));
  for (int j = 0; j < 64; ++j) x[j] = (float)(0.5 * std::log(std::fmax(sigma2[j], 1e-60)) - ls0);
  x[64] = (float)(std::log(lambda) - 2.0 * ls0);
  x[65] = (float)std::log((double)n);
  x[66] = (float)std::log((double)d);
  for (int j = 0; j < IN; ++j)
    x[j] = std::fmin(std::fmax((x[j] - norm->in_mean[j]) / norm->in_std[j], -kInputClip), kInputClip);
  float* io = static_cast<float*>(rs_scratch(ctx, SCR_MLP_IO, (IN + OUT) * sizeof(float)));
  if (!io) return RS_ENOMEM;
  RS_CUDA_TRY(cudaMemcpyAsync(io, x, IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  RS_TRY(launch_forward(ctx, theta, io, 1, io + IN));
  float o[OUT];
  RS_CUDA_TRY(cudaMemcpyAsync(o, io + IN, OUT * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  double v[OUT];
  for (int j = 0; j < OUT; ++j) v[j] = (double)o[j] * norm->out_std[j] + norm->out_mean[j];
  const double kr = std::exp2(v[0]), em = std::exp(v[1]), mr = std::exp2(v[2]);
  if (!std::isfinite(kr) || !std::isfinite(em) || !std::isfinite(mr)) return RS_OK;
  if (em < 0.01 || em > 8.0 || mr < 1.0 / 256.0 || mr > 64.0) return RS_OK;
  *k = (int32_t)std::lround(std::fmin(std::fmax(kr, 1.0), (double)K));
  *eta_mult = em;
  *m = std::max<int64_t>(1, (int64_t)std::llround((double)n * mr));
  *used_fallback = 0;
  return RS_OK;
}

}  // extern "C"
