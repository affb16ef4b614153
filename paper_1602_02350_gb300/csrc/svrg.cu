// SVRG on the preconditioned components (Alg. 1 with the n+d decomposition of Sec. 5.1):
// the full-gradient streaming pass, the blocked inner loop (a parallel per-block
// preparation plus a sequential thread-block-cluster chain), the epoch driver and
// Alg. 3 end to end.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace cg = cooperative_groups;

int scan_u32_to_u64(rs_ctx* ctx, const uint32_t* in, uint64_t* out, int64_t N);
int sampling_weights_dispatch(rs_ctx* ctx, const void* beta, int32_t dtype, int64_t N, uint32_t* W);
int index_stream_dispatch(rs_ctx* ctx, const uint32_t* W, const uint64_t* cum, int64_t N, uint64_t seed,
                          int64_t epoch, int64_t t0, int64_t m, int32_t sampling, int32_t dtype, uint32_t* idx,
                          void* inv_nq);
int map_output_dispatch(rs_ctx* ctx, const void* V, const double* sigma2, int64_t d, int64_t k, double lam,
                        int32_t dtype, const void* wt, void* w);
int sketch_dispatch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* V, double* sigma2);
template <typename S, typename T>
int tune_chain_t(rs_ctx* ctx, const rs_matrix* Z, const uint32_t* idx, int64_t m, TuneEntry* best, int* tried);   // epoch.cu
int precondition_dispatch(rs_ctx* ctx, const rs_matrix* X, const void* V, const double* sigma2, int64_t k, double lam,
                          rs_matrix* Xt, void* beta, double* beta_hat);

namespace {


int blocks_for(rs_ctx* ctx, int64_t work, int threads = 256) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// ------------------------------------------------------------------ full gradient
// mu = (1/N) sum_i gamma_i (z_i^T w - y_i) z_i: a warp streams one row at a time (VPL 16-byte
// vectors per lane), reduces the dot product with shuffles and accumulates r_i z_i in registers;
// per-block partial vectors are summed in a fixed order by fullgrad_reduce_kernel.
template <typename T, int VPL>
__global__ void __launch_bounds__(256) fullgrad_kernel(const T* __restrict__ Z, int64_t N, int64_t n, int64_t d,
                                                       int64_t ld, const T* __restrict__ y, T lam,
                                                       const T* __restrict__ w, T* __restrict__ part) {
  using V = typename Vec<T>::type;
  constexpr int E = Vec<T>::N;
  extern __shared__ unsigned char fg_sh[];
  T* sh = reinterpret_cast<T*>(fg_sh);   // [warps][d]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T wr[VPL][E], acc[VPL][E];
#pragma unroll
  for (int q = 0; q < VPL; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t c = (int64_t)(lane + 32 * q) * E + e;
      wr[q][e] = c < d ? w[c] : T(0);
      acc[q][e] = T(0);
    }
  const T inv_n = T(1) / (T)n;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < N; i += (int64_t)gridDim.x * nw) {
    const T* row = Z + i * ld;
    T z[VPL][E];
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
      const int64_t c0 = (int64_t)(lane + 32 * q) * E;
      if (c0 < d) {
        V v = *reinterpret_cast<const V*>(row + c0);
        vec_to_arr(v, z[q]);
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (c0 + e >= d) z[q][e] = T(0);
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) z[q][e] = T(0);
      }
    }
    T dot = T(0);
#pragma unroll
    for (int q = 0; q < VPL; ++q)
#pragma unroll
      for (int e = 0; e < E; ++e) dot = fma(z[q][e], wr[q][e], dot);
    dot = warp_sum(dot);
    const T r = i < n ? (dot - y[i]) * inv_n : lam * dot;
#pragma unroll
    for (int q = 0; q < VPL; ++q)
#pragma unroll
      for (int e = 0; e < E; ++e) acc[q][e] = fma(r, z[q][e], acc[q][e]);
  }
#pragma unroll
  for (int q = 0; q < VPL; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t c = (int64_t)(lane + 32 * q) * E + e;
      if (c < d) sh[warp * d + c] = acc[q][e];
    }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
    T s = T(0);
    for (int w2 = 0; w2 < nw; ++w2) s += sh[w2 * d + c];
    part[(int64_t)blockIdx.x * d + c] = s;
  }
}

// Bulk-copy staged variant of fullgrad_kernel (one CTA per SM): a producer warp streams tiles of
// eight rows into a ring of shared-memory stages with cp.async.bulk, the copied bytes counted on
// the stage's mbarrier; eight consumer warps take one row of each tile (vectorised shared-memory
// reads, shuffle dot product, register accumulation) and release the stage.  Up to
// kFgStages x 8 rows are in flight per SM whatever the register pressure.  Waits are bounded.
constexpr int kFgStages = 6, kFgRows = 8;
constexpr long long kFgWait = 2000000000LL;   // about a second

template <typename T, int VPL>
__global__ void __launch_bounds__(32 * (kFgRows + 1)) fullgrad_bulk_kernel(const T* __restrict__ Z, int64_t N,
                                                                          int64_t n, int64_t d, int64_t ld,
                                                                          const T* __restrict__ y, T lam,
                                                                          const T* __restrict__ w,
                                                                          T* __restrict__ part, int* status) {
  using V = typename Vec<T>::type;
  constexpr int E = Vec<T>::N;
  extern __shared__ __align__(128) unsigned char fb_sh[];
  __shared__ uint64_t full[kFgStages], empty[kFgStages];
  const int64_t rs = ((d * (int64_t)sizeof(T) + 127) / 128) * 128 / (int64_t)sizeof(T);   // staged row stride
  T* stage = reinterpret_cast<T*>(fb_sh);   // [kFgStages][kFgRows][rs]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (N + kFgRows - 1) / kFgRows;
  // bulk copies move whole 16-byte units: the row is read up to the next 16-byte boundary, which
  // lies inside its row stride (ld * sizeof(T) is a multiple of 16); staged elements >= d are ignored
  const uint32_t row_bytes = (uint32_t)((d * (int64_t)sizeof(T) + 15) / 16 * 16);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kFgStages; ++s) {
      mbar_init_cta(&full[s], 1);
      mbar_init_cta(&empty[s], kFgRows);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  T acc[VPL][E];
#pragma unroll
  for (int q = 0; q < VPL; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[q][e] = T(0);
  if (warp == kFgRows) {
    if (lane == 0) {   // producer
      int64_t it = 0;
      int64_t last_use[kFgStages];
      for (int s = 0; s < kFgStages; ++s) last_use[s] = -1;
      for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = (int)(it % kFgStages);
        const int64_t u = it / kFgStages;
        if (u >= 1 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kFgWait)) {
          atomicOr(status, STATUS_TIMEOUT);
          break;
        }
        const int64_t r0 = t * kFgRows;
        const int rows = (int)min64(kFgRows, N - r0);
        mbar_expect_tx_cta(&full[s], (uint32_t)rows * row_bytes);
        for (int r = 0; r < rows; ++r)
          bulk_copy_g2s(stage + ((int64_t)s * kFgRows + r) * rs, Z + (r0 + r) * ld, row_bytes, &full[s]);
        last_use[s] = u;
      }
      // every issued copy has landed before the stages are reused for the reduction below
      for (int s = 0; s < kFgStages; ++s)
        if (last_use[s] >= 0 && !mbar_wait_bounded(&full[s], (uint32_t)(last_use[s] & 1), kFgWait))
          atomicOr(status, STATUS_TIMEOUT);
    }
  } else {   // consumers
    T wr[VPL][E];
#pragma unroll
    for (int q = 0; q < VPL; ++q)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = (int64_t)(lane + 32 * q) * E + e;
        wr[q][e] = c < d ? w[c] : T(0);
      }
    const T inv_n = T(1) / (T)n;
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int s = (int)(it % kFgStages);
      const int64_t u = it / kFgStages;
      const int64_t i = t * kFgRows + warp;
      const T yi = (i < n) ? y[i] : T(0);
      if (!mbar_wait_bounded(&full[s], (uint32_t)(u & 1), kFgWait)) {
        if (lane == 0) atomicOr(status, STATUS_TIMEOUT);
        break;
      }
      if (i < N) {
        const T* row = stage + ((int64_t)s * kFgRows + warp) * rs;
        T z[VPL][E];
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
          const int64_t c0 = (int64_t)(lane + 32 * q) * E;
          if (c0 < d) {
            vec_to_arr(*reinterpret_cast<const V*>(row + c0), z[q]);
#pragma unroll
            for (int e = 0; e < E; ++e)
              if (c0 + e >= d) z[q][e] = T(0);
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) z[q][e] = T(0);
          }
        }
        T dot = T(0);
#pragma unroll
        for (int q = 0; q < VPL; ++q)
#pragma unroll
          for (int e = 0; e < E; ++e) dot = fma(z[q][e], wr[q][e], dot);
        dot = warp_sum(dot);
        const T r = i < n ? (dot - yi) * inv_n : lam * dot;
#pragma unroll
        for (int q = 0; q < VPL; ++q)
#pragma unroll
          for (int e = 0; e < E; ++e) acc[q][e] = fma(r, z[q][e], acc[q][e]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&empty[s]);
    }
  }
  __syncthreads();
  // per-warp sums in the (now idle) stage memory, then a fixed-order sum over the warps
  T* sh = stage;   // [kFgRows][d]
  if (warp < kFgRows) {
#pragma unroll
    for (int q = 0; q < VPL; ++q)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = (int64_t)(lane + 32 * q) * E + e;
        if (c < d) sh[warp * d + c] = acc[q][e];
      }
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
    T s2 = T(0);
    for (int w2 = 0; w2 < kFgRows; ++w2) s2 += sh[w2 * d + c];
    part[(int64_t)blockIdx.x * d + c] = s2;
  }
}

// Wide rows (float or bfloat16 storage, float arithmetic): column ownership.  A producer warp
// streams tiles of R rows into a ring of shared-memory stages with cp.async.bulk (bytes counted on
// the stage's mbarrier, bounded waits).  Each of the 256 consumer threads owns the 16-byte column
// chunks q = tid + 256 u (u < U), keeps w and the gradient accumulators of those columns in
// registers, and loads each staged element exactly once: it forms its partial dot products for
// the R rows of the tile, the partials are summed across the block (shuffles, then the eight warp
// sums in a fixed order after one named barrier), and the same registers then take
// acc += r_i z_i.  Every column of the block's partial gradient has one owner, so no shared-memory
// accumulation is needed.  A wait that gives up sets the status bit and every consumer leaves the
// loop together (the decision is taken after the barrier).
constexpr int kFcThreads = 256, kFcMaxStages = 8;
constexpr size_t kFcSmemBudget = 200 * 1024;

template <typename S, int U, int R>
__global__ void __launch_bounds__(kFcThreads + 32, 1)
    fullgrad_cols_kernel(const S* __restrict__ Z, int64_t N, int64_t n, int64_t d, int64_t ld,
                         const float* __restrict__ y, float lam, const float* __restrict__ w,
                         float* __restrict__ part, int stages, int* status) {
  constexpr int E = 16 / (int)sizeof(S);
  extern __shared__ __align__(128) unsigned char fc_sh[];
  __shared__ uint64_t full[kFcMaxStages], empty[kFcMaxStages];
  __shared__ __align__(16) float dpart[kFcMaxStages][kFcThreads / 32][R];
  __shared__ int abort_flag;
  const int64_t nch = (d + E - 1) / E;                          // 16-byte chunks per row
  const uint32_t row_bytes = (uint32_t)(nch * 16);
  const int64_t rstride = ((int64_t)row_bytes + 127) / 128 * 128;   // staged row stride (bytes)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (N + R - 1) / R;
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init_cta(&full[s], 1);
      mbar_init_cta(&empty[s], kFcThreads / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  float acc[U][E];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[u][e] = 0.0f;
  if (warp == kFcThreads / 32) {
    if (lane == 0) {   // producer
      int64_t it = 0, last_use[kFcMaxStages];
      for (int s = 0; s < stages; ++s) last_use[s] = -1;
      for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = (int)(it % stages);
        const int64_t u = it / stages;
        if (u >= 1 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kFgWait)) {
          atomicOr(status, STATUS_TIMEOUT);
          break;
        }
        const int64_t r0 = t * R;
        const int rows = (int)min64(R, N - r0);
        mbar_expect_tx_cta(&full[s], (uint32_t)rows * row_bytes);
        for (int r = 0; r < rows; ++r)
          bulk_copy_g2s(fc_sh + ((int64_t)s * R + r) * rstride, Z + (r0 + r) * ld, row_bytes, &full[s]);
        last_use[s] = u;
      }
      for (int s = 0; s < stages; ++s)   // every issued copy has landed before the block exits
        if (last_use[s] >= 0 && !mbar_wait_bounded(&full[s], (uint32_t)(last_use[s] & 1), kFgWait))
          atomicOr(status, STATUS_TIMEOUT);
    }
  } else {   // consumers
    float wr[U][E];
    // the last chunk may run past d: its extra elements get weight 0 and are masked to zero on load
    // (the row padding need not hold finite values); chunks beyond the row are not loaded at all
    uint4 msk[U];
    int lim[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = tid + (int64_t)kFcThreads * u;
      lim[u] = q < nch ? (int)min64(E, d - q * E) : 0;
      uint32_t mw[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (E == 8) {
          mw[k] = (2 * k < lim[u] ? 0x0000FFFFu : 0u) | (2 * k + 1 < lim[u] ? 0xFFFF0000u : 0u);
        } else {
          mw[k] = k < lim[u] ? 0xFFFFFFFFu : 0u;
        }
      }
      msk[u] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
#pragma unroll
      for (int e = 0; e < E; ++e) wr[u][e] = e < lim[u] ? w[q * E + e] : 0.0f;
    }
    const float inv_n = 1.0f / (float)n;
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int s = (int)(it % stages);
      const int64_t uu = it / stages;
      const int64_t r0 = t * R;
      const int rows = (int)min64(R, N - r0);
      // the tile's labels are read before waiting for its rows, so their latency overlaps the copy
      float yv[R];
#pragma unroll
      for (int j = 0; j < R; ++j) yv[j] = (r0 + j < n) ? y[r0 + j] : 0.0f;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(uu & 1), kFgWait)) abort_flag = 1;
      const unsigned char* st = fc_sh + (int64_t)s * R * rstride;
      uint4 zr[R][U];
      float pd[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        pd[j] = 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t q = tid + (int64_t)kFcThreads * u;
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (j < rows && lim[u] > 0) v = *reinterpret_cast<const uint4*>(st + j * rstride + q * 16);
          v.x &= msk[u].x;
          v.y &= msk[u].y;
          v.z &= msk[u].z;
          v.w &= msk[u].w;
          zr[j][u] = v;
          const S* sv = reinterpret_cast<const S*>(&zr[j][u]);
#pragma unroll
          for (int e = 0; e < E; ++e) pd[j] = fmaf(cvt<float>(sv[e]), wr[u][e], pd[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float v = warp_sum(pd[j]);
        if (lane == 0) dpart[s][warp][j] = v;
      }
      asm volatile("bar.sync 1, %0;\n" ::"r"(kFcThreads) : "memory");
      if (abort_flag) {
        if (lane == 0) atomicOr(status, STATUS_TIMEOUT);
        break;
      }
      float dots[R];
#pragma unroll
      for (int j = 0; j < R; ++j) dots[j] = 0.0f;
#pragma unroll
      for (int w2 = 0; w2 < kFcThreads / 32; ++w2) {   // fixed order
        if constexpr (R % 4 == 0) {
#pragma unroll
          for (int j = 0; j < R; j += 4) {
            const float4 q = *reinterpret_cast<const float4*>(&dpart[s][w2][j]);
            dots[j] += q.x;
            dots[j + 1] += q.y;
            dots[j + 2] += q.z;
            dots[j + 3] += q.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < R; ++j) dots[j] += dpart[s][w2][j];
        }
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (j < rows) {
          const float dot = dots[j];
          const int64_t i = r0 + j;
          const float r = i < n ? (dot - yv[j]) * inv_n : lam * dot;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const S* sv = reinterpret_cast<const S*>(&zr[j][u]);
#pragma unroll
            for (int e = 0; e < E; ++e) acc[u][e] = fmaf(r, cvt<float>(sv[e]), acc[u][e]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&empty[s]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = tid + (int64_t)kFcThreads * u;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < lim[u]) part[(int64_t)blockIdx.x * d + q * E + e] = acc[u][e];
    }
  }
}

// mu[c] = sum over the per-block partials, 32 columns per thread block: eight interleaved
// partial sums per column, then a fixed-order sum of the eight (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) fullgrad_reduce_kernel(const T* __restrict__ part, int np, int64_t d,
                                                              T* __restrict__ mu) {
  __shared__ T sh[8][33];
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  T s = T(0);
  if (c < d)
    for (int p = g; p < np; p += 8) s += part[(int64_t)p * d + c];
  sh[g][lane] = s;
  __syncthreads();
  if (g == 0 && c < d) {
    T t = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) t += sh[q][lane];
    mu[c] = t;
  }
}

template <typename T>
__global__ void norm2_kernel(const T* v, int64_t d, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) s += (double)v[c] * (double)v[c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sh[w2];
    *out = t;
  }
}

// Rows of any width and storage type S (double, float or bfloat16), compute type T: a warp
// streams one row at a time (16-byte vector loads, eight in flight per lane), reduces the dot
// product, re-reads the row (an L1 hit) and accumulates r_i z_i into its own shared-memory copy
// of the gradient; the eight warp copies are summed in a fixed order.
template <typename S, typename T>
__global__ void __launch_bounds__(256) fullgrad_wide_kernel(const S* __restrict__ Z, int64_t N, int64_t n, int64_t d,
                                                            int64_t ld, const T* __restrict__ y, T lam,
                                                            const T* __restrict__ w, T* __restrict__ part) {
  constexpr int E = 16 / sizeof(S);
  extern __shared__ __align__(16) unsigned char fw_sh[];
  T* ws = reinterpret_cast<T*>(fw_sh);        // [d]
  T* acc = ws + ((d + 3) & ~int64_t(3));      // [warps][d]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) ws[c] = w[c];
  for (int64_t c = threadIdx.x; c < (int64_t)nw * d; c += blockDim.x) acc[c] = T(0);
  __syncthreads();
  T* my = acc + (int64_t)warp * d;
  const int64_t nvec = (d + E - 1) / E;
  const T inv_n = T(1) / (T)n;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < N; i += (int64_t)gridDim.x * nw) {
    const S* row = Z + i * ld;
    T dot = T(0);
#pragma unroll 8
    for (int64_t q = lane; q < nvec; q += 32) {
      S v[E];
      *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(row + q * E);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = q * E + e;
        if (c < d) dot = fma(cvt<T>(v[e]), ws[c], dot);
      }
    }
    dot = warp_sum(dot);
    const T r = i < n ? (dot - y[i]) * inv_n : lam * dot;
#pragma unroll 8
    for (int64_t q = lane; q < nvec; q += 32) {
      S v[E];
      *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(row + q * E);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = q * E + e;
        if (c < d) my[c] = fma(r, cvt<T>(v[e]), my[c]);
      }
    }
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
    T t = T(0);
    for (int w2 = 0; w2 < nw; ++w2) t += acc[(int64_t)w2 * d + c];
    part[(int64_t)blockIdx.x * d + c] = t;
  }
}

template <typename T>
__global__ void convert_kernel(const double* in, int64_t count, T* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)in[e];
}

template <typename T>
__global__ void finite_check_kernel(const T* w, int64_t d, double limit, int* status) {
  bool bad = false, big = false;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d; c += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)w[c];
    if (!isfinite(v)) bad = true;
    else if (fabs(v) > limit) big = true;
  }
  if (bad) atomicOr(status, 1);
  if (big) atomicOr(status, 8);
}

template <typename S, typename T>
__global__ void row_beta_only_kernel(const S* Z, int64_t N, int64_t n, int64_t d, int64_t ld, double lam, T* beta) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double gd = (double)N / (double)n, gr = lam * (double)N;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < N; i += (int64_t)gridDim.x * nw) {
    T s = T(0);
    for (int64_t c = lane; c < d; c += 32) {
      const T v = cvt<T>(Z[i * ld + c]);
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) beta[i] = (T)((i < n ? gd : gr) * (double)s);
  }
}

template <typename T>
__global__ void mean_kernel(const T* v, int64_t N, double* out) {
  __shared__ double sh[32];
  // per-thread sums in T (a few dozen terms each; double adds are slow on this GPU), then double
  T st = T(0);
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) st += v[i];
  double s = warp_sum((double)st);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sh[w2];
    *out = t / (double)N;
  }
}

}  // namespace

// ====================================================================== launchers

// mu over the rows of Z (storage S, compute T); the rows i >= n are regulariser rows.  Called
// with Z = X and n = X->n it gives the data part of the gradient on the stored data.
template <typename S, typename T>
static int full_gradient_t(rs_ctx* ctx, const rs_matrix* Z, const T* y, int64_t n, double lam, const T* w, T* mu,
                           double* norm2_dev) {
  const int64_t N = Z->n, d = Z->d;
  constexpr int E = 16 / sizeof(S);
  const int64_t vecs = (d + E - 1) / E;
  const int vpl = (int)((vecs + 31) / 32);
  const int threads = 256;
  if constexpr (std::is_same<S, T>::value) if (vpl <= 8) {
    const T* Zd = static_cast<const T*>(Z->data);
    const int blocks = ctx->num_sms;
    T* part = static_cast<T*>(rs_scratch(ctx, SCR_PART2, (size_t)blocks * d * sizeof(T)));
    if (!part) return RS_ENOMEM;
    const int64_t rs_bytes = (d * (int64_t)sizeof(T) + 127) / 128 * 128;
    const size_t shm = std::max((size_t)kFgStages * kFgRows * rs_bytes, (size_t)kFgRows * d * sizeof(T));
    (void)threads;
#define RS_FG(VV)                                                                                              \
  do {                                                                                                         \
    RS_CUDA_TRY(cudaFuncSetAttribute(fullgrad_bulk_kernel<T, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)shm));                                                               \
    fullgrad_bulk_kernel<T, VV><<<blocks, 32 * (kFgRows + 1), shm, ctx->stream>>>(Zd, N, n, d, Z->ld, y,       \
                                                                                   (T)lam, w, part,            \
                                                                                   ctx->d_status);             \
  } while (0)
    if (vpl <= 1) RS_FG(1);
    else if (vpl <= 2) RS_FG(2);
    else if (vpl <= 4) RS_FG(4);
    else RS_FG(8);
#undef RS_FG
    RS_LAUNCH_CHECK(ctx);
    fullgrad_reduce_kernel<T><<<(unsigned)((d + 31) / 32), 256, 0, ctx->stream>>>(part, blocks, d, mu);
    RS_LAUNCH_CHECK(ctx);
    if (norm2_dev) {
      norm2_kernel<T><<<1, 256, 0, ctx->stream>>>(mu, d, norm2_dev);
      RS_LAUNCH_CHECK(ctx);
    }
    return RS_OK;
  }
  // wide float rows or bfloat16 storage: column-owner kernel with a bulk-copy ring
  if constexpr (std::is_same<T, float>::value && (std::is_same<S, float>::value ||
                                                  std::is_same<S, __nv_bfloat16>::value)) {
    constexpr int E = 16 / (int)sizeof(S);
    const int64_t nch = (d + E - 1) / E;
    // rows per tile R and chunks per thread U keep R U 16-byte chunks in registers: 16 for float
    // rows, 8 for bfloat16 rows (whose widened values take twice the registers)
    constexpr int RU = E == 8 ? 8 : 16;
    constexpr int UMAX = E == 8 ? 4 : 8;
    if (nch <= (int64_t)kFcThreads * UMAX) {
      const int U = nch <= kFcThreads ? 1 : nch <= 2 * kFcThreads ? 2 : nch <= 4 * kFcThreads ? 4 : 8;
      const int R = RU / U;
      const int64_t rstride = (nch * 16 + 127) / 128 * 128;
      int stages = (int)std::min<int64_t>(kFcMaxStages, (int64_t)kFcSmemBudget / (R * rstride));
      if (const TuneEntry* te = tune_find(ctx, TUNE_FULLGRAD, dtype_code<S>(), d))   // rs_autotune's choice
        stages = std::min(stages, te->a);
      if (stages >= 2) {
        const size_t shm = (size_t)stages * R * rstride;
        const int blocks = ctx->num_sms;
        T* part = static_cast<T*>(rs_scratch(ctx, SCR_PART2, (size_t)blocks * d * sizeof(T)));
        if (!part) return RS_ENOMEM;
        const S* Zd = static_cast<const S*>(Z->data);
#define RS_FC(UU)                                                                                             \
  do {                                                                                                        \
    constexpr int UC = UU <= UMAX ? UU : UMAX;                                                                \
    RS_CUDA_TRY(cudaFuncSetAttribute(fullgrad_cols_kernel<S, UC, RU / UC>,                                     \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));                  \
    fullgrad_cols_kernel<S, UC, RU / UC><<<blocks, kFcThreads + 32, shm, ctx->stream>>>(                      \
        Zd, N, n, d, Z->ld, y, (float)lam, w, part, stages, ctx->d_status);                                   \
  } while (0)
        if (U == 1) RS_FC(1);
        else if (U == 2) RS_FC(2);
        else if (U == 4) RS_FC(4);
        else RS_FC(8);
#undef RS_FC
        RS_LAUNCH_CHECK(ctx);
        fullgrad_reduce_kernel<T><<<(unsigned)((d + 31) / 32), 256, 0, ctx->stream>>>(part, blocks, d, mu);
        RS_LAUNCH_CHECK(ctx);
        if (norm2_dev) {
          norm2_kernel<T><<<1, 256, 0, ctx->stream>>>(mu, d, norm2_dev);
          RS_LAUNCH_CHECK(ctx);
        }
        return RS_OK;
      }
    }
  }
  // wider rows: shared-memory accumulators
  const size_t shm = ((size_t)((d + 3) & ~int64_t(3)) + (size_t)(threads / 32) * d) * sizeof(T);
  if (shm > 220 * 1024) return rs_fail(RS_EUNSUPPORTED, "full gradient: d = %lld too wide for on-chip accumulators", (long long)d);
  const int blocks = ctx->num_sms * (shm <= 100 * 1024 ? 2 : 1);
  T* part = static_cast<T*>(rs_scratch(ctx, SCR_PART2, (size_t)blocks * d * sizeof(T)));
  if (!part) return RS_ENOMEM;
  RS_CUDA_TRY(cudaFuncSetAttribute(fullgrad_wide_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  fullgrad_wide_kernel<S, T><<<blocks, threads, shm, ctx->stream>>>(static_cast<const S*>(Z->data), N, n, d, Z->ld, y,
                                                                    (T)lam, w, part);
  RS_LAUNCH_CHECK(ctx);
  fullgrad_reduce_kernel<T><<<(unsigned)((d + 31) / 32), 256, 0, ctx->stream>>>(part, blocks, d, mu);
  RS_LAUNCH_CHECK(ctx);
  if (norm2_dev) {
    norm2_kernel<T><<<1, 256, 0, ctx->stream>>>(mu, d, norm2_dev);
    RS_LAUNCH_CHECK(ctx);
  }
  return RS_OK;
}

template <typename S, typename T>
int svrg_epoch_t(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lam, const uint32_t* idx, const T* inv_nq,
                 int64_t m, double eta, const T* wbar, const T* mu, int average, T* wnext);   // epoch.cu
template <typename S, typename T>
int epoch_prep_r_t(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lam, const uint32_t* idx, const T* inv_nq,
                   int64_t m, double eta, T* Rt, T* cv);                                      // epoch.cu
template <typename S, typename T>
int epoch_finish_t(rs_ctx* ctx, const rs_matrix* Z, const uint32_t* idx, int64_t m, double eta, const T* Rt, T* cv,
                   const T* wbar, const T* mu, int average, T* wnext);                        // epoch.cu

// A second stream and its events for the look-ahead preparation of the next epoch; the context's
// stream is restored on every exit.
struct SideStream {
  rs_ctx* ctx = nullptr;
  cudaStream_t main = nullptr, side = nullptr;
  cudaEvent_t ready[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr}, start = nullptr;
  ~SideStream() {
    if (ctx) ctx->stream = main;
    for (int q = 0; q < 2; ++q) {
      if (ready[q]) cudaEventDestroy(ready[q]);
      if (used[q]) cudaEventDestroy(used[q]);
    }
    if (start) cudaEventDestroy(start);
    if (side) cudaStreamDestroy(side);
  }
};

// v = g + lam u (the gradient of Eq. (1) at u from its data part g)
template <typename T>
__global__ void add_ridge_kernel(const T* g, const T* u, int64_t d, double lam, T* v) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d; c += (int64_t)gridDim.x * blockDim.x)
    v[c] = g[c] + (T)lam * u[c];
}

static int check_components(const rs_matrix* Z, int64_t n, bool allow_fp8 = false) {
  RS_TRY(check_matrix(Z, "Z"));
  RS_CHECK_ARG(Z->dtype == RS_F64 || Z->dtype == RS_F32 || Z->dtype == RS_BF16 || (allow_fp8 && Z->dtype == RS_FP8E4M3),
               "components: dtype must be RS_F64, RS_F32 or RS_BF16 (RS_FP8E4M3 where stated)");
  RS_CHECK_ARG(n >= 1 && n < Z->n && Z->n - n == Z->d, "components: Z must have n + d rows");
  return RS_OK;
}

// Options of the proximal subproblems of accelerated SVRG (rs_catalyst_solve): the output map uses
// the preconditioner's lambda (lam_pre) while p->lambda is the subproblem's regularisation; mc
// (nullable) is subtracted from every snapshot gradient (kappa M c for the proximal centre c); the
// final preconditioned iterate is copied to wt_out (nullable).
template <typename T>
struct CenterOpt {
  double lam_pre;
  const T* mc;
  T* wt_out;
};

template <typename T>
__global__ void sub_vec_kernel(T* v, const T* u, int64_t d) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d; c += (int64_t)gridDim.x * blockDim.x)
    v[c] -= u[c];
}

// Alg. 1 epochs on the components Z (storage S, compute T).  With p->refine the full gradient
// is formed on the stored data X instead (mu = M (X^T (X M w - y)/n + lam M w), storage SX), so
// that the fixed point is exact for the data as stored even when Z is a rounded copy.
template <typename S, typename T, typename SX>
static int svrg_solve_t(rs_ctx* ctx, const rs_matrix* Z, const rs_matrix* X, const T* y, const T* beta_in,
                        const T* V, const double* sigma2, int64_t k, const rs_svrg_params* p, const T* w0, T* w_out,
                        rs_history* hist, double* eta_used, int64_t* m_used, const CenterOpt<T>* opt = nullptr) {
  const int64_t N = Z->n, d = Z->d, n = N - d;
  const int32_t dt = sizeof(T) == 8 ? RS_F64 : RS_F32;
  const double lam = p->lambda;
  const double lam_m = opt ? opt->lam_pre : lam;   // lambda of the preconditioner M (output maps)
  T* beta = const_cast<T*>(beta_in);
  if constexpr (IsFp8<S>::value) {
    if (!beta || !(p->refine && X))
      return rs_fail(RS_EINVAL, "rs_svrg_solve: FP8 components need beta (from rs_precondition) and refine with X");
  }
  if (!beta) {
    beta = static_cast<T*>(rs_scratch(ctx, SCR_BETA, N * sizeof(T)));
    if (!beta) return RS_ENOMEM;
    if constexpr (!IsFp8<S>::value) {
      row_beta_only_kernel<S, T><<<blocks_for(ctx, N * 32), 256, 0, ctx->stream>>>(static_cast<const S*>(Z->data), N,
                                                                                    n, d, Z->ld, lam, beta);
      RS_LAUNCH_CHECK(ctx);
    }
  }
  uint32_t* W = static_cast<uint32_t*>(rs_scratch(ctx, SCR_W, N * sizeof(uint32_t)));
  uint64_t* cum = static_cast<uint64_t*>(rs_scratch(ctx, SCR_CUM, N * sizeof(uint64_t)));
  double* scal = static_cast<double*>(rs_scratch(ctx, SCR_S2, (size_t)(4 + std::max(1, p->epochs)) * sizeof(double)));
  if (!W || !cum || !scal) return RS_ENOMEM;
  RS_TRY(sampling_weights_dispatch(ctx, beta, dt, N, W));   // synchronises, checks finiteness
  RS_TRY(scan_u32_to_u64(ctx, W, cum, N));
  mean_kernel<T><<<1, 1024, 0, ctx->stream>>>(beta, N, scal);
  RS_LAUNCH_CHECK(ctx);
  double bh = 0.0;
  RS_CUDA_TRY(cudaMemcpyAsync(&bh, scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (!(bh > 0.0) || !std::isfinite(bh)) return rs_fail(RS_ENONFINITE, "rs_svrg_solve: mean smoothness is %g", bh);
  double eta = p->eta;
  if (p->eta_mult > 0.0) eta = p->eta_mult / bh;
  else if (!(eta > 0.0)) eta = 0.1 / bh;
  int64_t m = p->m > 0 ? p->m : (int64_t)std::ceil(bh / lam);
  if (m < 1) m = 1;
  if (eta_used) *eta_used = eta;
  if (m_used) *m_used = m;
  T* wa = static_cast<T*>(rs_scratch(ctx, SCR_WBAR, d * sizeof(T)));
  T* wb = static_cast<T*>(rs_scratch(ctx, SCR_WNEXT, d * sizeof(T)));
  T* mu = static_cast<T*>(rs_scratch(ctx, SCR_MU, d * sizeof(T)));
  // two sets of per-epoch data: the next epoch's index stream and R matrices are prepared on a
  // second stream (on SMs the inner loop leaves idle) while the current epoch runs
  const int64_t nblk = (m + kChainBlk - 1) / kChainBlk;
  uint32_t* idx2 = static_cast<uint32_t*>(rs_scratch(ctx, SCR_IDX, 2 * m * sizeof(uint32_t)));
  T* inq2 = static_cast<T*>(rs_scratch(ctx, SCR_INVNQ, 2 * m * sizeof(T)));
  T* Rt2 = static_cast<T*>(rs_scratch(ctx, SCR_R, 2 * (size_t)nblk * kChainBlk * kChainBlk * sizeof(T)));
  T* cv2 = static_cast<T*>(rs_scratch(ctx, SCR_C, 2 * (size_t)nblk * kChainBlk * sizeof(T)));
  T* tmp = static_cast<T*>(rs_scratch(ctx, SCR_TMPV, 2 * d * sizeof(T)));
  if (!wa || !wb || !mu || !idx2 || !inq2 || !Rt2 || !cv2 || !tmp) return RS_ENOMEM;
  SideStream sd;
  sd.main = ctx->stream;
  RS_CUDA_TRY(cudaStreamCreateWithFlags(&sd.side, cudaStreamNonBlocking));
  sd.ctx = ctx;
  for (int q = 0; q < 2; ++q) {
    RS_CUDA_TRY(cudaEventCreateWithFlags(&sd.ready[q], cudaEventDisableTiming));
    RS_CUDA_TRY(cudaEventCreateWithFlags(&sd.used[q], cudaEventDisableTiming));
  }
  RS_CUDA_TRY(cudaEventCreateWithFlags(&sd.start, cudaEventDisableTiming));
  auto set_idx = [&](int q) { return idx2 + (int64_t)q * m; };
  auto set_inq = [&](int q) { return inq2 + (int64_t)q * m; };
  auto set_rt = [&](int q) { return Rt2 + (int64_t)q * nblk * kChainBlk * kChainBlk; };
  auto set_cv = [&](int q) { return cv2 + (int64_t)q * nblk * kChainBlk; };
  // index stream and R of epoch s into set s & 1, on the second stream
  auto prepare = [&](int s) -> int {
    const int q = s & 1;
    ctx->stream = sd.side;
    int rc = index_stream_dispatch(ctx, W, cum, N, p->seed, (int64_t)p->epoch0 + s, 0, m, p->sampling, dt, set_idx(q),
                                   set_inq(q));
    if (rc == RS_OK) rc = epoch_prep_r_t<S, T>(ctx, Z, n, lam, set_idx(q), set_inq(q), m, eta, set_rt(q), set_cv(q));
    ctx->stream = sd.main;
    if (rc != RS_OK) return rc;
    RS_CUDA_TRY(cudaEventRecord(sd.ready[q], sd.side));
    return RS_OK;
  };
  const bool refine = p->refine && X;
  if (w0) RS_CUDA_TRY(cudaMemcpyAsync(wa, w0, d * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
  else RS_CUDA_TRY(cudaMemsetAsync(wa, 0, d * sizeof(T), ctx->stream));
  const int nep = p->epochs;
  std::vector<cudaEvent_t> ev;
  if (hist && hist->epoch_ms) {
    ev.resize(nep + 1);
    for (auto& e : ev) RS_CUDA_TRY(cudaEventCreate(&e));
    RS_CUDA_TRY(cudaEventRecord(ev[0], ctx->stream));
  }
  double* norms = scal + 4;
  // the second stream starts after the sampling table (built on the main stream) is complete
  RS_CUDA_TRY(cudaEventRecord(sd.start, ctx->stream));
  RS_CUDA_TRY(cudaStreamWaitEvent(sd.side, sd.start, 0));
  if (nep > 0) RS_TRY(prepare(0));
  for (int s = 0; s < nep; ++s) {
    const int q = s & 1;
    const bool want_norm = hist && hist->mu_norm2;
    if (refine) {
      T* u = tmp;
      T* g = tmp + d;
      RS_TRY(map_output_dispatch(ctx, V, sigma2, d, k, lam_m, dt, wa, u));                   // u = M w
      RS_TRY(full_gradient_t<SX, T>(ctx, X, y, X->n, lam, u, g, nullptr));                   // X^T (X u - y) / n
      add_ridge_kernel<T><<<blocks_for(ctx, d), 256, 0, ctx->stream>>>(g, u, d, lam, g);     // + lam u
      RS_LAUNCH_CHECK(ctx);
      RS_TRY(map_output_dispatch(ctx, V, sigma2, d, k, lam_m, dt, g, mu));                    // mu = M (...)
      if (want_norm) {
        norm2_kernel<T><<<1, 256, 0, ctx->stream>>>(mu, d, norms + s);
        RS_LAUNCH_CHECK(ctx);
      }
    } else {
      if constexpr (!IsFp8<S>::value)
        RS_TRY(full_gradient_t<S, T>(ctx, Z, y, n, lam, wa, mu, want_norm ? norms + s : nullptr));
    }
    if (opt && opt->mc) {   // proximal centre: mu -= kappa M c
      sub_vec_kernel<T><<<blocks_for(ctx, d), 256, 0, ctx->stream>>>(mu, opt->mc, d);
      RS_LAUNCH_CHECK(ctx);
      if (want_norm) {
        norm2_kernel<T><<<1, 256, 0, ctx->stream>>>(mu, d, norms + s);
        RS_LAUNCH_CHECK(ctx);
      }
    }
    RS_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, sd.ready[q], 0));
    RS_TRY(epoch_finish_t<S, T>(ctx, Z, set_idx(q), m, eta, set_rt(q), set_cv(q), wa, mu, p->average, wb));
    RS_CUDA_TRY(cudaEventRecord(sd.used[q], ctx->stream));
    if (s + 1 < nep) {
      // set q ^ 1 was last read by epoch s - 1
      if (s >= 1) RS_CUDA_TRY(cudaStreamWaitEvent(sd.side, sd.used[q ^ 1], 0));
      RS_TRY(prepare(s + 1));
    }
    std::swap(wa, wb);
    if (hist && hist->snapshots && s < hist->capacity)
      RS_TRY(map_output_dispatch(ctx, V, sigma2, d, k, lam_m, dt, wa, static_cast<T*>(hist->snapshots) + (int64_t)s * d));
    if (!ev.empty()) RS_CUDA_TRY(cudaEventRecord(ev[s + 1], ctx->stream));
  }
  RS_TRY(map_output_dispatch(ctx, V, sigma2, d, k, lam_m, dt, wa, w_out));
  if (opt && opt->wt_out) RS_CUDA_TRY(cudaMemcpyAsync(opt->wt_out, wa, d * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
  // the status word was cleared by rs_sampling_weights above; epochs may have set the timeout bit
  finite_check_kernel<T><<<blocks_for(ctx, d), 256, 0, ctx->stream>>>(w_out, d, 1e30, ctx->d_status);
  RS_LAUNCH_CHECK(ctx);
  int st = 0;
  RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (hist) {
    hist->epochs_run = nep;
    if (hist->mu_norm2 && nep > 0)
      RS_CUDA_TRY(cudaMemcpy(hist->mu_norm2, norms, std::min(nep, hist->capacity) * sizeof(double),
                             cudaMemcpyDeviceToHost));
    if (!ev.empty()) {
      for (int s = 0; s < nep && s < hist->capacity; ++s) RS_CUDA_TRY(cudaEventElapsedTime(&hist->epoch_ms[s], ev[0], ev[s + 1]));
      for (auto& e : ev) cudaEventDestroy(e);
    }
  }
  if (st & STATUS_TIMEOUT) return rs_fail(RS_ETIMEOUT, "rs_svrg_solve: a bounded wait of the inner-loop chain gave up");
  if (st & 1) return rs_fail(RS_ENONFINITE, "rs_svrg_solve: the iterate became non-finite (step size too large?)");
  if (st & 8) return rs_fail(RS_EDIVERGED, "rs_svrg_solve: the iterate diverged (step size too large?)");
  return RS_OK;
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

template <typename S, typename T>
static int solve_t(rs_ctx* ctx, const rs_matrix* Xin, const void* yin, const rs_sketch_params* sp,
                   const rs_svrg_params* p, void* w_out, rs_history* hist) {
  const int64_t n = Xin->n, d = Xin->d, k = sp->k, N = n + d;
  rs_matrix X = *Xin;
  const size_t es = sizeof(T), ss = sizeof(S);
  if (is_host_ptr(Xin->data)) {
    void* xd = rs_scratch(ctx, SCR_XDEV, (size_t)n * Xin->ld * ss);
    if (!xd) return RS_ENOMEM;
    RS_CUDA_TRY(cudaMemcpyAsync(xd, Xin->data, (size_t)n * Xin->ld * ss, cudaMemcpyHostToDevice, ctx->stream));
    X.data = xd;
  }
  const T* y = static_cast<const T*>(yin);
  if (is_host_ptr(yin)) {
    T* yd = static_cast<T*>(rs_scratch(ctx, SCR_YDEV, n * es));
    if (!yd) return RS_ENOMEM;
    RS_CUDA_TRY(cudaMemcpyAsync(yd, yin, n * es, cudaMemcpyHostToDevice, ctx->stream));
    y = yd;
  }
  const bool host_out = is_host_ptr(w_out);
  T* wdev = static_cast<T*>(host_out ? rs_scratch(ctx, SCR_WOUT, d * es) : w_out);
  T* V = static_cast<T*>(rs_scratch(ctx, SCR_V, d * k * es));
  double* sg = static_cast<double*>(rs_scratch(ctx, SCR_SIGMA, k * sizeof(double)));
  const int64_t ldz = (d * (int64_t)ss + 15) / 16 * 16 / (int64_t)ss;
  S* Zbuf = static_cast<S*>(rs_scratch(ctx, SCR_Z, (size_t)N * ldz * ss));
  T* beta = static_cast<T*>(rs_scratch(ctx, SCR_BETA, N * es));
  if (!wdev || !V || !sg || !Zbuf || !beta) return RS_ENOMEM;
  RS_TRY(sketch_dispatch(ctx, &X, sp, V, sg));
  rs_matrix Zm = {Zbuf, nullptr, N, d, ldz, X.dtype, 0};
  RS_TRY(precondition_dispatch(ctx, &X, V, sg, k, p->lambda, &Zm, beta, nullptr));
  RS_TRY(svrg_solve_t<S, T, S>(ctx, &Zm, &X, y, beta, V, sg, k, p, nullptr, wdev, hist, nullptr, nullptr));
  if (host_out) {
    RS_CUDA_TRY(cudaMemcpyAsync(w_out, wdev, d * es, cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return RS_OK;
}

int trace_dispatch(rs_ctx* ctx, const rs_matrix* X, double* out);   // dense.cu
extern "C" int rs_propose(rs_ctx* ctx, const float* theta, const rs_mlp_norm* norm, const double* sigma2,
                          double lambda, int64_t n, int64_t d, double trace_c, int32_t* k, double* eta_mult,
                          int64_t* m, int32_t* used_fallback);

// Alg. 3 with proposed parameters: rank-64 sketch, tr(C), rs_propose, components from the leading
// k Ritz pairs (stored in ZS), SVRG with eta = eta_mult / beta^ and the proposed m.
template <typename S, typename T, typename ZS>
static int solve_proposed_t(rs_ctx* ctx, const rs_matrix* Xin, const void* yin, const rs_sketch_params* sp,
                            const rs_svrg_params* p, const float* theta, const rs_mlp_norm* norm, void* w_out,
                            rs_history* hist, int32_t* k_out, double* eta_out, int64_t* m_out, int32_t* fb_out) {
  const int64_t n = Xin->n, d = Xin->d, N = n + d;
  // sketch rank: 64 (the network's input) unless the caller fixes a larger preconditioner rank
  const int64_t K = sp->k > 64 ? (int64_t)sp->k : 64;
  rs_matrix X = *Xin;
  const size_t es = sizeof(T), ss = sizeof(S), zs = sizeof(ZS);
  if (is_host_ptr(Xin->data)) {
    void* xd = rs_scratch(ctx, SCR_XDEV, (size_t)n * Xin->ld * ss);
    if (!xd) return RS_ENOMEM;
    RS_CUDA_TRY(cudaMemcpyAsync(xd, Xin->data, (size_t)n * Xin->ld * ss, cudaMemcpyHostToDevice, ctx->stream));
    X.data = xd;
  }
  const T* y = static_cast<const T*>(yin);
  if (is_host_ptr(yin)) {
    T* yd = static_cast<T*>(rs_scratch(ctx, SCR_YDEV, n * es));
    if (!yd) return RS_ENOMEM;
    RS_CUDA_TRY(cudaMemcpyAsync(yd, yin, n * es, cudaMemcpyHostToDevice, ctx->stream));
    y = yd;
  }
  const bool host_out = is_host_ptr(w_out);
  T* wdev = static_cast<T*>(host_out ? rs_scratch(ctx, SCR_WOUT, d * es) : w_out);
  T* V = static_cast<T*>(rs_scratch(ctx, SCR_V, d * K * es));
  double* sg = static_cast<double*>(rs_scratch(ctx, SCR_SIGMA, K * sizeof(double)));
  if (!wdev || !V || !sg) return RS_ENOMEM;
  rs_sketch_params s64 = *sp;
  s64.k = (int32_t)K;
  RS_TRY(sketch_dispatch(ctx, &X, &s64, V, sg));
  double trc = 0.0, s2h[64];
  RS_TRY(trace_dispatch(ctx, &X, &trc));   // synchronises
  RS_CUDA_TRY(cudaMemcpy(s2h, sg, sizeof(s2h), cudaMemcpyDeviceToHost));
  int32_t k = 0, fb = 0;
  double em = 0.0;
  int64_t m = 0;
  {
    // rs_propose is a public entry (it opens a new call generation); it does not touch X, so the
    // bfloat16 parts of X formed by the sketch stay valid for the preconditioner below
    const uint64_t gen = ctx->call_gen;
    RS_TRY(rs_propose(ctx, theta, norm, s2h, p->lambda, n, d, trc, &k, &em, &m, &fb));
    ctx->call_gen = gen;
  }
  if (K > 64) {
    // fixed rank: only eta and m are proposed.  The network's m is for its own rank k; Thm 1 sets the
    // epoch length in proportion to kappa~(k), so it is carried over to the fixed rank K by the
    // ratio kappa~(K) / kappa~(k) of the sketch's own estimates
    if (!fb) {
      std::vector<double> s2all((size_t)K);
      RS_CUDA_TRY(cudaMemcpy(s2all.data(), sg, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost));
      auto kt = [&](int64_t kk) {
        double head = 0.0;
        for (int64_t i = 0; i < kk; ++i) head += s2all[(size_t)i];
        return ((double)kk * s2all[(size_t)kk - 1] + (trc - head)) / p->lambda;
      };
      const double kn = kt(k), kf = kt(K);
      if (kn > 0.0 && kf > 0.0) m = std::max<int64_t>(1, std::llround((double)m * kf / kn));
    }
    k = (int32_t)K;
  }
  T* Vk = static_cast<T*>(rs_scratch(ctx, SCR_VK, d * k * es));
  const int64_t ldz = (d * (int64_t)zs + 15) / 16 * 16 / (int64_t)zs;
  ZS* Zbuf = static_cast<ZS*>(rs_scratch(ctx, SCR_Z, (size_t)N * ldz * zs));
  T* beta = static_cast<T*>(rs_scratch(ctx, SCR_BETA, N * es));
  if (!Vk || !Zbuf || !beta) return RS_ENOMEM;
  // leading k columns of the rank-64 Ritz basis (row-major d x 64 -> d x k)
  RS_CUDA_TRY(cudaMemcpy2DAsync(Vk, k * es, V, K * es, k * es, d, cudaMemcpyDeviceToDevice, ctx->stream));
  const int32_t zdt = std::is_same<ZS, __nv_bfloat16>::value ? RS_BF16 : X.dtype;
  rs_matrix Zm = {Zbuf, nullptr, N, d, ldz, zdt, 0};
  RS_TRY(precondition_dispatch(ctx, &X, Vk, sg, k, p->lambda, &Zm, beta, nullptr));
  rs_svrg_params q = *p;
  q.eta = 0.0;
  q.eta_mult = em;
  q.m = m;
  if (!std::is_same<ZS, S>::value) q.refine = 1;
  RS_TRY(svrg_solve_t<ZS, T, S>(ctx, &Zm, &X, y, beta, Vk, sg, k, &q, nullptr, wdev, hist, nullptr, nullptr));
  if (host_out) {
    RS_CUDA_TRY(cudaMemcpyAsync(w_out, wdev, d * es, cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  if (k_out) *k_out = k;
  if (eta_out) *eta_out = em;
  if (m_out) *m_out = m;
  if (fb_out) *fb_out = fb;
  return RS_OK;
}

// ====================================================================== C ABI

extern "C" {

int rs_full_gradient(rs_ctx* ctx, const rs_matrix* Z, const void* y, int64_t n, double lambda, const void* w,
                     void* mu) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_components(Z, n));
  RS_CHECK_ARG(y && w && mu, "rs_full_gradient: null argument");
  RS_CHECK_ARG(lambda > 0.0, "rs_full_gradient: lambda must be positive");
  if (Z->dtype == RS_F64)
    return full_gradient_t<double, double>(ctx, Z, static_cast<const double*>(y), n, lambda,
                                           static_cast<const double*>(w), static_cast<double*>(mu), nullptr);
  if (Z->dtype == RS_BF16)
    return full_gradient_t<__nv_bfloat16, float>(ctx, Z, static_cast<const float*>(y), n, lambda,
                                                 static_cast<const float*>(w), static_cast<float*>(mu), nullptr);
  return full_gradient_t<float, float>(ctx, Z, static_cast<const float*>(y), n, lambda, static_cast<const float*>(w),
                                       static_cast<float*>(mu), nullptr);
}

int rs_svrg_epoch(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lambda, const uint32_t* idx, const void* inv_nq,
                  int64_t m, double eta, const void* w_bar, const void* mu, int32_t average, void* w_next) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_components(Z, n, true));
  RS_CHECK_ARG(idx && inv_nq && w_bar && mu && w_next, "rs_svrg_epoch: null argument");
  RS_CHECK_ARG(m >= 1 && m < (1LL << 31), "rs_svrg_epoch: m out of range");
  RS_CHECK_ARG(w_next != w_bar, "rs_svrg_epoch: w_next must not alias w_bar");
  if (Z->dtype == RS_FP8E4M3)
    return svrg_epoch_t<__nv_fp8_e4m3, float>(ctx, Z, n, lambda, idx, static_cast<const float*>(inv_nq), m, eta,
                                              static_cast<const float*>(w_bar), static_cast<const float*>(mu), average,
                                              static_cast<float*>(w_next));
  if (Z->dtype == RS_F64)
    return svrg_epoch_t<double, double>(ctx, Z, n, lambda, idx, static_cast<const double*>(inv_nq), m, eta,
                                        static_cast<const double*>(w_bar), static_cast<const double*>(mu), average,
                                        static_cast<double*>(w_next));
  if (Z->dtype == RS_BF16)
    return svrg_epoch_t<__nv_bfloat16, float>(ctx, Z, n, lambda, idx, static_cast<const float*>(inv_nq), m, eta,
                                              static_cast<const float*>(w_bar), static_cast<const float*>(mu),
                                              average, static_cast<float*>(w_next));
  return svrg_epoch_t<float, float>(ctx, Z, n, lambda, idx, static_cast<const float*>(inv_nq), m, eta,
                                    static_cast<const float*>(w_bar), static_cast<const float*>(mu), average,
                                    static_cast<float*>(w_next));
}

int rs_svrg_solve(rs_ctx* ctx, const rs_matrix* Z, const rs_matrix* X, const void* y, const void* beta, const void* V,
                  const double* sigma2, int64_t k, const rs_svrg_params* p, const void* w0, void* w_out,
                  rs_history* hist, double* eta_used, int64_t* m_used) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(Z && p, "rs_svrg_solve: null argument");
  const int64_t n = Z->n - Z->d;
  RS_TRY(check_components(Z, n, true));
  RS_CHECK_ARG(y && V && sigma2 && w_out, "rs_svrg_solve: null argument");
  RS_CHECK_ARG(k >= 1 && k <= Z->d, "rs_svrg_solve: k must be in [1, d]");
  RS_CHECK_ARG(p->lambda > 0.0, "rs_svrg_solve: lambda must be positive");
  RS_CHECK_ARG(p->epochs >= 0 && p->epoch0 >= 0, "rs_svrg_solve: bad epoch counts");
  RS_CHECK_ARG(p->sampling == RS_SAMPLE_IMPORTANCE || p->sampling == RS_SAMPLE_UNIFORM, "rs_svrg_solve: bad sampling");
  if (p->refine) {
    RS_CHECK_ARG(X != nullptr, "rs_svrg_solve: refinement needs the stored data X");
    RS_TRY(check_matrix(X, "rs_svrg_solve X"));
    RS_CHECK_ARG(X->n == n && X->d == Z->d, "rs_svrg_solve: X must be n x d");
    RS_CHECK_ARG(X->dtype == Z->dtype || (Z->dtype == RS_BF16 && X->dtype == RS_F32) ||
                     (Z->dtype == RS_FP8E4M3 && (X->dtype == RS_F32 || X->dtype == RS_BF16)),
                 "rs_svrg_solve: X must be stored like Z (or in RS_F32 for RS_BF16 components, RS_F32 or RS_BF16 "
                 "for RS_FP8E4M3 components)");
  }
  if (Z->dtype == RS_FP8E4M3) {
    RS_CHECK_ARG(p->refine && X && beta, "rs_svrg_solve: FP8 components need refine, X and beta");
    if (X->dtype == RS_F32)
      return svrg_solve_t<__nv_fp8_e4m3, float, float>(
          ctx, Z, X, static_cast<const float*>(y), static_cast<const float*>(beta), static_cast<const float*>(V),
          sigma2, k, p, static_cast<const float*>(w0), static_cast<float*>(w_out), hist, eta_used, m_used);
    return svrg_solve_t<__nv_fp8_e4m3, float, __nv_bfloat16>(
        ctx, Z, X, static_cast<const float*>(y), static_cast<const float*>(beta), static_cast<const float*>(V), sigma2,
        k, p, static_cast<const float*>(w0), static_cast<float*>(w_out), hist, eta_used, m_used);
  }
  if (Z->dtype == RS_F64)
    return svrg_solve_t<double, double, double>(ctx, Z, X, static_cast<const double*>(y),
                                                static_cast<const double*>(beta), static_cast<const double*>(V), sigma2,
                                                k, p, static_cast<const double*>(w0), static_cast<double*>(w_out), hist,
                                                eta_used, m_used);
  if (Z->dtype == RS_BF16 && p->refine && X->dtype == RS_F32)
    return svrg_solve_t<__nv_bfloat16, float, float>(
        ctx, Z, X, static_cast<const float*>(y), static_cast<const float*>(beta), static_cast<const float*>(V), sigma2,
        k, p, static_cast<const float*>(w0), static_cast<float*>(w_out), hist, eta_used, m_used);
  if (Z->dtype == RS_BF16)
    return svrg_solve_t<__nv_bfloat16, float, __nv_bfloat16>(
        ctx, Z, X, static_cast<const float*>(y), static_cast<const float*>(beta), static_cast<const float*>(V), sigma2,
        k, p, static_cast<const float*>(w0), static_cast<float*>(w_out), hist, eta_used, m_used);
  return svrg_solve_t<float, float, float>(ctx, Z, X, static_cast<const float*>(y), static_cast<const float*>(beta),
                                           static_cast<const float*>(V), sigma2, k, p, static_cast<const float*>(w0),
                                           static_cast<float*>(w_out), hist, eta_used, m_used);
}

}  // extern "C"

// ---------------------------------------------------------------- accelerated SVRG (Catalyst)
namespace {

// beta1[i] = beta0[i] for i < n, beta0[i] f for the regulariser rows (their weight lam -> lam + kappa)
template <typename T>
__global__ void scale_tail_kernel(const T* b0, T* b1, int64_t N, int64_t n, double f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    b1[i] = i < n ? b0[i] : (T)((double)b0[i] * f);
}
// c = x + b (x - x_prev); x_prev = x; v *= s for the centre term
template <typename T>
__global__ void extrapolate_kernel(const T* x, T* x_prev, T* c, int64_t d, double b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const T xi = x[i];
    c[i] = xi + (T)b * (xi - x_prev[i]);
    x_prev[i] = xi;
  }
}
template <typename T>
__global__ void scale_vec_kernel(T* v, int64_t d, double s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (T)((double)v[i] * s);
}

// Catalyst (Lin, Mairal, Harchaoui 2015) around the epochs of Alg. 1: outer iteration t solves the
// proximal problem L(w) + kappa/2 ||w - c_{t-1}||^2 (regularisation lam + kappa; in the component
// form only the regulariser rows change: weight (lam + kappa)(n + d), label kappa c_j / (lam + kappa),
// which shifts every snapshot gradient by -kappa M c) with p->epochs epochs warm-started at the
// previous outer iterate, then extrapolates c_t = x_t + b_t (x_t - x_{t-1}).
template <typename S, typename T, typename SX>
int catalyst_t(rs_ctx* ctx, const rs_matrix* Z, const rs_matrix* X, const T* y, const T* beta_in, const T* V,
               const double* sigma2, int64_t k, const rs_svrg_params* p, const rs_catalyst_params* cp, T* w_out,
               rs_history* hist, double* kappa_used) {
  const int64_t N = Z->n, d = Z->d, n = N - d;
  const int32_t dt = sizeof(T) == 8 ? RS_F64 : RS_F32;
  const double lam = p->lambda;
  T* b0 = const_cast<T*>(beta_in);
  if (!b0) {
    if constexpr (IsFp8<S>::value) {
      return rs_fail(RS_EINVAL, "rs_catalyst_solve: FP8 components need beta");
    } else {
      b0 = static_cast<T*>(rs_scratch(ctx, SCR_CATB, N * sizeof(T)));
      if (!b0) return RS_ENOMEM;
      row_beta_only_kernel<S, T><<<blocks_for(ctx, N * 32), 256, 0, ctx->stream>>>(static_cast<const S*>(Z->data), N,
                                                                                    n, d, Z->ld, lam, b0);
      RS_LAUNCH_CHECK(ctx);
    }
  }
  double kappa = cp->kappa;
  if (!(kappa > 0.0)) {   // the Catalyst choice for SVRG: kappa = L / N - mu with L the mean smoothness
    double* sc = static_cast<double*>(rs_scratch(ctx, SCR_CATS, sizeof(double)));
    if (!sc) return RS_ENOMEM;
    mean_kernel<T><<<1, 1024, 0, ctx->stream>>>(b0, N, sc);
    RS_LAUNCH_CHECK(ctx);
    double bh = 0.0;
    RS_CUDA_TRY(cudaMemcpyAsync(&bh, sc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    kappa = std::max(0.0, bh / (double)N - lam);
  }
  if (kappa_used) *kappa_used = kappa;
  T* b1 = static_cast<T*>(rs_scratch(ctx, SCR_CATB2, N * sizeof(T)));
  T* vec = static_cast<T*>(rs_scratch(ctx, SCR_CATV, 6 * d * sizeof(T)));
  if (!b1 || !vec) return RS_ENOMEM;
  T *wt = vec, *wt2 = vec + d, *x = vec + 2 * d, *xprev = vec + 3 * d, *c = vec + 4 * d, *mc = vec + 5 * d;
  scale_tail_kernel<T><<<blocks_for(ctx, N), 256, 0, ctx->stream>>>(b0, b1, N, n, (lam + kappa) / lam);
  RS_LAUNCH_CHECK(ctx);
  RS_CUDA_TRY(cudaMemsetAsync(vec, 0, 6 * d * sizeof(T), ctx->stream));
  const double q = lam / (lam + kappa);
  double alpha = std::sqrt(q);
  std::vector<cudaEvent_t> ev;
  if (hist && hist->epoch_ms) {
    ev.resize(cp->outer + 1);
    for (auto& e : ev) RS_CUDA_TRY(cudaEventCreate(&e));
    RS_CUDA_TRY(cudaEventRecord(ev[0], ctx->stream));
  }
  int rc = RS_OK;
  for (int t = 0; t < cp->outer && rc == RS_OK; ++t) {
    rs_svrg_params p2 = *p;
    p2.lambda = lam + kappa;
    p2.epoch0 = p->epoch0 + t * p->epochs;
    const T* mcp = nullptr;
    if (kappa > 0.0) {
      RS_TRY(map_output_dispatch(ctx, V, sigma2, d, k, lam, dt, c, mc));   // M c
      scale_vec_kernel<T><<<blocks_for(ctx, d), 256, 0, ctx->stream>>>(mc, d, kappa);
      RS_LAUNCH_CHECK(ctx);
      mcp = mc;
    }
    CenterOpt<T> opt{lam, mcp, wt2};
    rc = svrg_solve_t<S, T, SX>(ctx, Z, X, y, b1, V, sigma2, k, &p2, t == 0 ? nullptr : wt, x, nullptr, nullptr,
                                nullptr, &opt);
    if (rc != RS_OK) break;
    std::swap(wt, wt2);
    const double a_prev = alpha;
    const double bq = alpha * alpha - q;
    alpha = 0.5 * (-bq + std::sqrt(bq * bq + 4.0 * a_prev * a_prev));
    const double b = a_prev * (1.0 - a_prev) / (a_prev * a_prev + alpha);
    extrapolate_kernel<T><<<blocks_for(ctx, d), 256, 0, ctx->stream>>>(x, xprev, c, d, b);
    RS_LAUNCH_CHECK(ctx);
    if (hist && hist->snapshots && t < hist->capacity)
      RS_CUDA_TRY(cudaMemcpyAsync(static_cast<T*>(hist->snapshots) + (int64_t)t * d, x, d * sizeof(T),
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    if (!ev.empty()) RS_CUDA_TRY(cudaEventRecord(ev[t + 1], ctx->stream));
  }
  if (rc == RS_OK) RS_CUDA_TRY(cudaMemcpyAsync(w_out, x, d * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (hist) {
    hist->epochs_run = cp->outer;
    if (!ev.empty()) {
      for (int t = 0; t < cp->outer && t < hist->capacity; ++t)
        RS_CUDA_TRY(cudaEventElapsedTime(&hist->epoch_ms[t], ev[0], ev[t + 1]));
      for (auto& e : ev) cudaEventDestroy(e);
    }
  }
  return rc;
}

}  // namespace

extern "C" {

int rs_catalyst_solve(rs_ctx* ctx, const rs_matrix* Z, const rs_matrix* X, const void* y, const void* beta,
                      const void* V, const double* sigma2, int64_t k, const rs_svrg_params* p,
                      const rs_catalyst_params* cp, void* w_out, rs_history* hist, double* kappa_used) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(Z && p && cp, "rs_catalyst_solve: null argument");
  const int64_t n = Z->n - Z->d;
  RS_TRY(check_components(Z, n, true));
  RS_CHECK_ARG(y && V && sigma2 && w_out, "rs_catalyst_solve: null argument");
  RS_CHECK_ARG(k >= 1 && k <= Z->d, "rs_catalyst_solve: k must be in [1, d]");
  RS_CHECK_ARG(p->lambda > 0.0 && std::isfinite(cp->kappa), "rs_catalyst_solve: need lambda > 0 and a finite kappa");
  RS_CHECK_ARG(cp->outer >= 1 && p->epochs >= 1 && p->epoch0 >= 0, "rs_catalyst_solve: need outer >= 1, epochs >= 1");
  RS_CHECK_ARG(p->sampling == RS_SAMPLE_IMPORTANCE || p->sampling == RS_SAMPLE_UNIFORM, "rs_catalyst_solve: bad sampling");
  if (p->refine) {
    RS_CHECK_ARG(X != nullptr, "rs_catalyst_solve: refinement needs the stored data X");
    RS_TRY(check_matrix(X, "rs_catalyst_solve X"));
    RS_CHECK_ARG(X->n == n && X->d == Z->d, "rs_catalyst_solve: X must be n x d");
    RS_CHECK_ARG(X->dtype == Z->dtype || (Z->dtype == RS_BF16 && X->dtype == RS_F32) ||
                     (Z->dtype == RS_FP8E4M3 && (X->dtype == RS_F32 || X->dtype == RS_BF16)),
                 "rs_catalyst_solve: X must be stored like Z (as for rs_svrg_solve)");
  }
  const float* yf = static_cast<const float*>(y);
  const float* bf = static_cast<const float*>(beta);
  const float* Vf = static_cast<const float*>(V);
  float* wf = static_cast<float*>(w_out);
  if (Z->dtype == RS_FP8E4M3) {
    RS_CHECK_ARG(p->refine && X && beta, "rs_catalyst_solve: FP8 components need refine, X and beta");
    if (X->dtype == RS_F32)
      return catalyst_t<__nv_fp8_e4m3, float, float>(ctx, Z, X, yf, bf, Vf, sigma2, k, p, cp, wf, hist, kappa_used);
    return catalyst_t<__nv_fp8_e4m3, float, __nv_bfloat16>(ctx, Z, X, yf, bf, Vf, sigma2, k, p, cp, wf, hist,
                                                           kappa_used);
  }
  if (Z->dtype == RS_F64)
    return catalyst_t<double, double, double>(ctx, Z, X, static_cast<const double*>(y), static_cast<const double*>(beta),
                                              static_cast<const double*>(V), sigma2, k, p, cp,
                                              static_cast<double*>(w_out), hist, kappa_used);
  if (Z->dtype == RS_BF16 && p->refine && X->dtype == RS_F32)
    return catalyst_t<__nv_bfloat16, float, float>(ctx, Z, X, yf, bf, Vf, sigma2, k, p, cp, wf, hist, kappa_used);
  if (Z->dtype == RS_BF16)
    return catalyst_t<__nv_bfloat16, float, __nv_bfloat16>(ctx, Z, X, yf, bf, Vf, sigma2, k, p, cp, wf, hist,
                                                           kappa_used);
  return catalyst_t<float, float, float>(ctx, Z, X, yf, bf, Vf, sigma2, k, p, cp, wf, hist, kappa_used);
}

int rs_solve(rs_ctx* ctx, const rs_matrix* X, const void* y, const rs_sketch_params* sp, const rs_svrg_params* p,
             void* w_out, rs_history* hist) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(X && X->data && y && sp && p && w_out, "rs_solve: null argument");
  RS_CHECK_ARG(X->n >= 1 && X->d >= 1 && X->ld >= X->d, "rs_solve: bad shape");
  RS_CHECK_ARG(X->dtype == RS_F64 || X->dtype == RS_F32 || X->dtype == RS_BF16,
               "rs_solve: dtype must be RS_F64, RS_F32 or RS_BF16");
  RS_CHECK_ARG((X->ld * (int64_t)dtype_size(X->dtype)) % 16 == 0, "rs_solve: row stride must be a multiple of 16 bytes");
  RS_CHECK_ARG(sp->k >= 1 && sp->k <= X->d && sp->k <= 256, "rs_solve: k must be in [1, min(d, 256)]");
  RS_CHECK_ARG(p->lambda > 0.0 && p->epochs >= 0, "rs_solve: bad SVRG parameters");
  if (X->dtype == RS_F64) return solve_t<double, double>(ctx, X, y, sp, p, w_out, hist);
  if (X->dtype == RS_BF16) return solve_t<__nv_bfloat16, float>(ctx, X, y, sp, p, w_out, hist);
  return solve_t<float, float>(ctx, X, y, sp, p, w_out, hist);
}

int rs_solve_proposed(rs_ctx* ctx, const rs_matrix* X, const void* y, const rs_sketch_params* sp,
                      const rs_svrg_params* p, const float* theta, const rs_mlp_norm* norm, int32_t z_dtype,
                      void* w_out, rs_history* hist, int32_t* k, double* eta_mult, int64_t* m, int32_t* used_fallback) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(X && X->data && y && sp && p && w_out, "rs_solve_proposed: null argument");
  RS_CHECK_ARG(X->n >= 1 && X->d >= 64 && X->ld >= X->d, "rs_solve_proposed: need d >= 64 (rank-64 sketch)");
  RS_CHECK_ARG(sp->k <= 64 || sp->k <= X->d, "rs_solve_proposed: a fixed rank k > 64 needs k <= d");
  RS_CHECK_ARG((X->ld * (int64_t)dtype_size(X->dtype)) % 16 == 0,
               "rs_solve_proposed: row stride must be a multiple of 16 bytes");
  RS_CHECK_ARG(p->lambda > 0.0 && p->epochs >= 0, "rs_solve_proposed: bad SVRG parameters");
  RS_CHECK_ARG(z_dtype == X->dtype || (z_dtype == RS_BF16 && X->dtype == RS_F32),
               "rs_solve_proposed: components must be stored like X or in RS_BF16 for RS_F32 data");
  if (X->dtype == RS_F64)
    return solve_proposed_t<double, double, double>(ctx, X, y, sp, p, theta, norm, w_out, hist, k, eta_mult, m,
                                                    used_fallback);
  if (X->dtype == RS_BF16) {
    RS_CHECK_ARG(p->refine, "rs_solve_proposed: RS_BF16 data needs refine = 1");
    return solve_proposed_t<__nv_bfloat16, float, __nv_bfloat16>(ctx, X, y, sp, p, theta, norm, w_out, hist, k,
                                                                  eta_mult, m, used_fallback);
  }
  RS_CHECK_ARG(X->dtype == RS_F32, "rs_solve_proposed: dtype must be RS_F64, RS_F32 or RS_BF16");
  if (z_dtype == RS_BF16)
    return solve_proposed_t<float, float, __nv_bfloat16>(ctx, X, y, sp, p, theta, norm, w_out, hist, k, eta_mult, m,
                                                         used_fallback);
  return solve_proposed_t<float, float, float>(ctx, X, y, sp, p, theta, norm, w_out, hist, k, eta_mult, m,
                                               used_fallback);
}

}  // extern "C"

// ====================================================================== autotuning
namespace {

// Ring stages of the column-owner full-gradient kernel for float / bf16 rows: every stage count
// that fits is timed on one pass over Z (one warm-up, three timed passes); the fastest is kept.
template <typename S>
int tune_fullgrad_t(rs_ctx* ctx, const rs_matrix* Z, int64_t n, TuneEntry* best, int* tried) {
  const int64_t d = Z->d;
  float* vec = static_cast<float*>(rs_scratch(ctx, SCR_CATV, (size_t)(n + 2 * d) * sizeof(float)));
  if (!vec) return RS_ENOMEM;
  RS_CUDA_TRY(cudaMemsetAsync(vec, 0, (size_t)(n + 2 * d) * sizeof(float), ctx->stream));
  const float* y = vec;
  const float* w = vec + n;
  float* mu = vec + n + d;
  cudaEvent_t e0, e1;
  RS_CUDA_TRY(cudaEventCreate(&e0));
  RS_CUDA_TRY(cudaEventCreate(&e1));
  best->kind = 0;
  int rc = RS_OK;
  for (int st : {2, 3, 4, 6, 8}) {
    TuneEntry probe;
    probe.kind = TUNE_FULLGRAD;
    probe.dtype = dtype_code<S>();
    probe.d = d;
    probe.a = st;
    tune_put(ctx, probe);   // the dispatch reads the stage cap from the cache
    for (int rep = 0; rep < 4 && rc == RS_OK; ++rep) {
      if (rep == 1) RS_CUDA_TRY(cudaEventRecord(e0, ctx->stream));
      rc = full_gradient_t<S, float>(ctx, Z, y, n, 1.0, w, mu, nullptr);
    }
    if (rc != RS_OK) break;
    RS_CUDA_TRY(cudaEventRecord(e1, ctx->stream));
    RS_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.0f;
    RS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 3.0f;
    ++*tried;
    if (!best->kind || ms < best->ms) {
      *best = probe;
      best->ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" int rs_autotune(rs_ctx* ctx, const rs_matrix* Z, int64_t n, rs_tune_report* rep) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(Z && rep, "rs_autotune: null argument");
  RS_TRY(check_components(Z, n, true));
  const int64_t N = Z->n, d = Z->d;
  *rep = rs_tune_report{};
  const TuneEntry* ct = tune_find(ctx, TUNE_CHAIN, Z->dtype, d);
  const bool fg_applies = Z->dtype == RS_F32 || Z->dtype == RS_BF16;
  const TuneEntry* ft = fg_applies ? tune_find(ctx, TUNE_FULLGRAD, Z->dtype, d) : nullptr;
  int tried = 0;
  if (!ct) {
    // probe: 8192 steps drawn uniformly over the N components
    constexpr int64_t kProbe = 8192;
    uint32_t* idx = static_cast<uint32_t*>(rs_scratch(ctx, SCR_IDX, kProbe * sizeof(uint32_t)));
    void* inq = rs_scratch(ctx, SCR_INVNQ, kProbe * sizeof(double));
    if (!idx || !inq) return RS_ENOMEM;
    const int32_t dt = Z->dtype == RS_F64 ? RS_F64 : RS_F32;
    RS_TRY(index_stream_dispatch(ctx, nullptr, nullptr, N, 0x5EEDull, 0, 0, kProbe, RS_SAMPLE_UNIFORM, dt, idx, inq));
    TuneEntry best;
    int rc;
    if (Z->dtype == RS_F64) rc = tune_chain_t<double, double>(ctx, Z, idx, kProbe, &best, &tried);
    else if (Z->dtype == RS_BF16) rc = tune_chain_t<__nv_bfloat16, float>(ctx, Z, idx, kProbe, &best, &tried);
    else if (Z->dtype == RS_FP8E4M3) rc = tune_chain_t<__nv_fp8_e4m3, float>(ctx, Z, idx, kProbe, &best, &tried);
    else rc = tune_chain_t<float, float>(ctx, Z, idx, kProbe, &best, &tried);
    RS_TRY(rc);
    tune_put(ctx, best);
    ct = tune_find(ctx, TUNE_CHAIN, Z->dtype, d);
  }
  if (fg_applies && !ft) {
    TuneEntry best;
    const int rc = Z->dtype == RS_BF16 ? tune_fullgrad_t<__nv_bfloat16>(ctx, Z, n, &best, &tried)
                                       : tune_fullgrad_t<float>(ctx, Z, n, &best, &tried);
    RS_TRY(rc);
    if (best.kind) tune_put(ctx, best);
    ft = tune_find(ctx, TUNE_FULLGRAD, Z->dtype, d);
  }
  rep->chain_cluster = ct->a;
  rep->chain_threads = ct->b;
  rep->chain_stages = ct->c;
  rep->chain_ms = ct->ms;
  if (ft) {
    rep->fullgrad_stages = ft->a;
    rep->fullgrad_ms = ft->ms;
  }
  rep->candidates = tried;
  rep->cached = tried == 0;
  return RS_OK;
}

// ====================================================================== allocation-free variant
//
// Some callers cannot call cudaMalloc: applications whose device memory is owned end to end by
// their own pool or arena (an allocation outside it either fails once the pool has reserved the
// device or breaks the pool's accounting), and latency-critical services that must stay off the
// driver's allocation path (cudaMalloc and cudaFree can synchronise the device).  For them
// rs_full_gradient_static runs the same full-gradient pass as rs_full_gradient, with the
// per-block partial sums in a fixed array in this library's device data instead of context
// scratch, and without a context.

#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = size_t(2) << 20;   // 2 MiB, held by every device that loads the library
static __device__ __align__(256) unsigned char g_fullgrad_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_static_scratch[kMaxDevices];   // device address of g_fullgrad_scratch, per device
int g_static_sms[kMaxDevices];
std::mutex g_static_mu;

// Once per device, with that device current: resolve the array's device address (the host-side
// symbol is only a stand-in and must never be handed to a kernel).
int static_scratch_setup(int dev, void** scratch, int* sms) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fullgrad_scratch);
    if (e != cudaSuccess) return rs_fail(RS_ECUDA, "rs_full_gradient_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int s = 0;
    e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return rs_fail(RS_ECUDA, "rs_full_gradient_static: %s", cudaGetErrorString(e));
    g_static_sms[dev] = s;
    g_static_scratch[dev] = p;
  }
  *scratch = g_static_scratch[dev];
  *sms = g_static_sms[dev];
  return RS_OK;
}

template <typename T>
int full_gradient_static_t(cudaStream_t stream, const rs_matrix* Z, const T* y, int64_t n, double lam, const T* w,
                           T* mu, void* scratch, int sms) {
  const int64_t N = Z->n, d = Z->d;
  constexpr int E = Vec<T>::N;
  const int64_t vecs = (d + E - 1) / E;
  const int vpl = (int)((vecs + 31) / 32);
  if (vpl > 8)
    return rs_fail(RS_EINVAL, "rs_full_gradient_static: d = %lld exceeds this entry point's %d-column maximum",
                   (long long)d, 32 * 8 * E);
  int64_t blocks = (int64_t)sms * 2;
  const int64_t fit = (int64_t)(kStaticScratchBytes / ((size_t)d * sizeof(T)));
  if (blocks > fit) blocks = fit;
  if (blocks < 1) return rs_fail(RS_EINVAL, "rs_full_gradient_static: d = %lld does not fit the 2 MiB scratch", (long long)d);
  T* part = static_cast<T*>(scratch);   // every block overwrites its own d partial sums: no clearing needed
  const int threads = 256;
  const size_t shm = (size_t)(threads / 32) * d * sizeof(T);   // at most 32 KiB: no attribute change needed
  const T* Zd = static_cast<const T*>(Z->data);
  if (vpl <= 1) fullgrad_kernel<T, 1><<<(unsigned)blocks, threads, shm, stream>>>(Zd, N, n, d, Z->ld, y, (T)lam, w, part);
  else if (vpl <= 2) fullgrad_kernel<T, 2><<<(unsigned)blocks, threads, shm, stream>>>(Zd, N, n, d, Z->ld, y, (T)lam, w, part);
  else if (vpl <= 4) fullgrad_kernel<T, 4><<<(unsigned)blocks, threads, shm, stream>>>(Zd, N, n, d, Z->ld, y, (T)lam, w, part);
  else fullgrad_kernel<T, 8><<<(unsigned)blocks, threads, shm, stream>>>(Zd, N, n, d, Z->ld, y, (T)lam, w, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rs_fail(RS_ECUDA, "rs_full_gradient_static: %s", cudaGetErrorString(e));
  fullgrad_reduce_kernel<T><<<(unsigned)((d + 31) / 32), 256, 0, stream>>>(part, (int)blocks, d, mu);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rs_fail(RS_ECUDA, "rs_full_gradient_static: %s", cudaGetErrorString(e));
  return RS_OK;
}

}  // namespace

extern "C" int rs_full_gradient_static(void* cuda_stream, const rs_matrix* Z, const void* y, int64_t n, double lambda,
                                       const void* w, void* mu) {
  RS_CHECK_ARG(Z && y && w && mu, "rs_full_gradient_static: null argument");
  RS_TRY(check_components(Z, n));
  // only float and double rows have a kernel here; a BF16 (or FP8) Z would be read at the wrong
  // element size, so it is refused before anything is launched
  RS_CHECK_ARG(Z->dtype == RS_F64 || Z->dtype == RS_F32,
               "rs_full_gradient_static: Z must be RS_F64 or RS_F32 (RS_BF16 / RS_FP8E4M3 rows: use rs_full_gradient)");
  RS_CHECK_ARG(lambda > 0.0, "rs_full_gradient_static: lambda must be positive");
  int dev = 0;
  RS_CUDA_TRY(cudaGetDevice(&dev));
  RS_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "rs_full_gradient_static: device %d out of range", dev);
  void* scratch = nullptr;
  int sms = 0;
  RS_TRY(static_scratch_setup(dev, &scratch, &sms));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (Z->dtype == RS_F64)
    return full_gradient_static_t<double>(s, Z, static_cast<const double*>(y), n, lambda, static_cast<const double*>(w),
                                          static_cast<double*>(mu), scratch, sms);
  return full_gradient_static_t<float>(s, Z, static_cast<const float*>(y), n, lambda, static_cast<const float*>(w),
                                       static_cast<float*>(mu), scratch, sms);
}
