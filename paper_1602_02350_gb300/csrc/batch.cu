// Batched solves: many problems, each at several lambda and SVRG settings ("chains"), with one
// sketch per problem, one set of components per (problem, lambda), per-epoch snapshot gradients
// that read each problem's stored data once for all of its chains, and batched launches for the
// index streams, the block preparation and the inner loops (one thread-block cluster per chain).
// Epoch 1 runs eagerly (it also sizes every scratch buffer); epochs 2..S are captured in one CUDA
// graph and launched once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "common.cuh"

int sketch_dispatch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* V, double* sigma2);
int precondition_dispatch(rs_ctx* ctx, const rs_matrix* X, const void* V, const double* sigma2, int64_t k, double lam,
                          rs_matrix* Xt, void* beta, double* beta_hat);
int sampling_weights_dispatch(rs_ctx* ctx, const void* beta, int32_t dtype, int64_t N, uint32_t* W);
int scan_u32_to_u64(rs_ctx* ctx, const uint32_t* in, uint64_t* out, int64_t N);
extern "C" int rs_full_gradient(rs_ctx* ctx, const rs_matrix* Z, const void* y, int64_t n, double lambda,
                                const void* w, void* mu);

namespace {

// y = M x with M = I - V diag(a) V^T (a = 1 - D'), x = xg_scale xg[c * xg_ld] + xf_scale xf[c]
struct MapJob {
  const float* V;
  const float* a;
  int64_t d;
  int32_t k, check;          // check: flag non-finite outputs in the status word
  const double* xg;
  int64_t xg_ld;
  double xg_scale;
  const float* xf;
  double xf_scale;
  float* y;
  int64_t y_ld, y_epoch_stride;
  float* y2;                 // optional second copy (unit stride)
};

__device__ __forceinline__ double map_input(const MapJob& J, int64_t c) {
  double x = 0.0;
  if (J.xg) x = J.xg_scale * J.xg[c * J.xg_ld];
  if (J.xf) x += J.xf_scale * (double)J.xf[c];
  return x;
}

// one block per job: t = V^T x, then y = x - V (a .* t), in float (as the one-problem solver's maps;
// double arithmetic is slow on this GPU).  x (formed in double from its parts, stored as float) is
// staged in shared memory; t by (column, row group) partial sums combined in group order; y with a
// warp per eight rows, lanes along the row (coalesced reads of V), one shuffle sum per row.
constexpr int kMapMaxD = 4096;
__global__ void __launch_bounds__(256) bmap_kernel(const MapJob* __restrict__ jobs, int64_t epoch, int* status) {
  __shared__ float xs[kMapMaxD];
  __shared__ float part[256];
  __shared__ float tv[256];
  const MapJob J = jobs[blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int k = J.k;
  const int64_t d = J.d;
  for (int64_t c = tid; c < d; c += nt) xs[c] = (float)map_input(J, c);
  __syncthreads();
  const int G = nt / k;   // row groups (k <= 256)
  const int j = tid % k, g = tid / k;
  if (g < G) {
    float s0 = 0.0f, s1 = 0.0f;
    int64_t c = g;
    for (; c + G < d; c += 2 * (int64_t)G) {
      s0 = fmaf(J.V[c * k + j], xs[c], s0);
      s1 = fmaf(J.V[(c + G) * k + j], xs[c + G], s1);
    }
    if (c < d) s0 = fmaf(J.V[c * k + j], xs[c], s0);
    part[g * k + j] = s0 + s1;
  }
  __syncthreads();
  if (tid < k) {
    float t = 0.0f;
    for (int q = 0; q < G; ++q) t += part[q * k + tid];   // fixed order
    tv[tid] = t * J.a[tid];
  }
  __syncthreads();
  bool bad = false;
  float* y = J.y + epoch * J.y_epoch_stride;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int64_t c0 = (int64_t)warp * 8; c0 < d; c0 += (int64_t)nw * 8) {
    float sr[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      sr[r] = 0.0f;
      const int64_t c = c0 + r;
      if (c < d)
        for (int q = lane; q < k; q += 32) sr[r] = fmaf(J.V[c * k + q], tv[q], sr[r]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) sr[r] = warp_sum(sr[r]);
    if (lane < 8 && c0 + lane < d) {
      float sl = sr[0];
#pragma unroll
      for (int r = 1; r < 8; ++r)
        if (lane == r) sl = sr[r];
      const int64_t c = c0 + lane;
      const float out = xs[c] - sl;
      y[c * J.y_ld] = out;
      if (J.y2) J.y2[c] = out;
      if (J.check && !isfinite(out)) bad = true;
    }
  }
  if (bad) atomicOr(status, STATUS_NONFINITE);
}

__global__ void adiag_f_kernel(const double* sigma2, int k, double lam, float* a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) a[j] = (float)(1.0 - sqrt((sigma2[k - 1] + lam) / (sigma2[j] + lam)));
}

// R[i][r] -= y[i]
__global__ void sub_labels_kernel(float* R, int64_t n, int r, const float* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x)
    R[e] -= y[e / r];
}

// Skinny products of a problem's stored data with its chains' vectors (R <= RMAX columns; U and
// Rm carry RMAX columns, the ones beyond R ignored), each one streaming pass over X at full load
// width (16 bytes per lane):  Rm = X U - y 1^T  and  G = X^T Rm / n.
// CPL consecutive columns of one row widened to float (vector loads when the row holds them all;
// rows are 16-byte aligned by the C ABI's contract, c is a multiple of CPL)
template <int CPL>
__device__ __forceinline__ void ld_cols(const __nv_bfloat16* p, int64_t c, int64_t d, float* v) {
  if (c + CPL <= d) {
    uint32_t w[CPL / 2];
    if constexpr (CPL == 8) {
      const uint4 q = *reinterpret_cast<const uint4*>(p + c);
      w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
    } else if constexpr (CPL == 4) {
      const uint2 q = *reinterpret_cast<const uint2*>(p + c);
      w[0] = q.x; w[1] = q.y;
    } else {
      w[0] = *reinterpret_cast<const uint32_t*>(p + c);
    }
#pragma unroll
    for (int k = 0; k < CPL / 2; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);
      v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  } else {
#pragma unroll
    for (int e = 0; e < CPL; ++e) v[e] = c + e < d ? __bfloat162float(p[c + e]) : 0.0f;
  }
}
template <int CPL>
__device__ __forceinline__ void ld_cols(const float* p, int64_t c, int64_t d, float* v) {
  if (c + CPL <= d) {
#pragma unroll
    for (int k = 0; k < CPL; k += 4) {
      if constexpr (CPL >= 4) {
        const float4 q = *reinterpret_cast<const float4*>(p + c + k);
        v[k] = q.x; v[k + 1] = q.y; v[k + 2] = q.z; v[k + 3] = q.w;
      } else {
        const float2 q = *reinterpret_cast<const float2*>(p + c);
        v[0] = q.x; v[1] = q.y;
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < CPL; ++e) v[e] = c + e < d ? p[c + e] : 0.0f;
  }
}

// Sum of v[k] over the 32 lanes for k = 0..31, scattered: lane L returns the sum for k = L
// (31 shuffles instead of 32 x 5)
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int o = 16 >> s;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = upper ? v[k] : v[k + o];
      const float keep = upper ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// Rm[i][r] = x_i . U[:, r] - y_i (zero for r >= R).  A warp takes RW = 32 / RMAX rows at a time; a
// lane loads CPL consecutive columns of each.  USM: U is staged in shared memory with 4 floats of
// padding after every CPL rows, so the quarter-warp's 16-byte reads fall on distinct banks.
template <typename S, int RMAX, bool USM>
__global__ void __launch_bounds__(256) skinny_xu_kernel(const S* __restrict__ X, int64_t n, int64_t d, int64_t ld,
                                                        const float* __restrict__ U, int R, const float* __restrict__ y,
                                                        float* __restrict__ Rm) {
  constexpr int RW = 32 / RMAX;
  constexpr int CPL = 16 / (int)sizeof(S);
  constexpr int USTR = CPL * RMAX + 4;   // floats per CPL rows of U in shared memory
  extern __shared__ float4 us4[];
  float* us = reinterpret_cast<float*>(us4);
  const int64_t ng = (d + CPL - 1) / CPL;
  if (USM) {
    for (int64_t e = threadIdx.x; e < ng * CPL * RMAX; e += blockDim.x) {
      const int64_t cc = e / RMAX;
      const int r = (int)(e % RMAX);
      us[(cc / CPL) * USTR + (cc % CPL) * RMAX + r] = cc < d ? U[cc * RMAX + r] : 0.0f;
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i0 = ((int64_t)blockIdx.x * nw + warp) * RW; i0 < n; i0 += (int64_t)gridDim.x * nw * RW) {
    float acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0f;
    // two column groups per step, all of their loads issued before the arithmetic (more bytes in
    // flight per warp); the second group of the last step may lie beyond the row
    for (int64_t g0 = lane; g0 < ng; g0 += 64) {
      float xv[2][RW][CPL];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t c = (g0 + 32 * h) * CPL;
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
          if (i0 + rr < n && c < d) ld_cols<CPL>(X + (i0 + rr) * ld, c, d, xv[h][rr]);
          else
#pragma unroll
            for (int e = 0; e < CPL; ++e) xv[h][rr][e] = 0.0f;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t g = g0 + 32 * h, c = g * CPL;
        if (g >= ng) break;
        const float4* u4 = USM ? reinterpret_cast<const float4*>(us + g * USTR)
                               : reinterpret_cast<const float4*>(U + c * RMAX);
#pragma unroll
        for (int e = 0; e < CPL; ++e) {
          if (!USM && c + e >= d) break;
#pragma unroll
          for (int q = 0; q < RMAX / 4; ++q) {
            const float4 u = u4[e * (RMAX / 4) + q];
#pragma unroll
            for (int rr = 0; rr < RW; ++rr) {
              acc[rr * RMAX + 4 * q] = fmaf(xv[h][rr][e], u.x, acc[rr * RMAX + 4 * q]);
              acc[rr * RMAX + 4 * q + 1] = fmaf(xv[h][rr][e], u.y, acc[rr * RMAX + 4 * q + 1]);
              acc[rr * RMAX + 4 * q + 2] = fmaf(xv[h][rr][e], u.z, acc[rr * RMAX + 4 * q + 2]);
              acc[rr * RMAX + 4 * q + 3] = fmaf(xv[h][rr][e], u.w, acc[rr * RMAX + 4 * q + 3]);
            }
          }
        }
      }
    }
    const float v = warp_reduce_scatter32(acc, lane);
    const int64_t i = i0 + lane / RMAX;
    const int r = lane % RMAX;
    if (i < n) Rm[i * RMAX + r] = r < R ? v - y[i] : 0.0f;
  }
}

// part[chunk][c][r] = sum over the chunk's rows of X[i][c] Rm[i][r] (r < R), per 32 CPL columns
// (CPL = 64 / RMAX per lane, 64 accumulators).
// The same transposed pass fed by bulk copies: a producer warp streams tiles of 16 row slices
// (32 CPL columns each) and the matching 16 rows of Rm into an 8-stage shared-memory ring
// (cp.async.bulk, bytes counted on mbarriers, bounded waits); 8 consumer warps take two rows of
// each tile, then the warps' sums are added in warp order (the ring's memory is reused).
constexpr int kXtrRows = 16, kXtrStages = 8;
constexpr long long kXtrWait = 2000000000LL;
template <typename S, int RMAX>
constexpr size_t xtr_bulk_smem() {
  constexpr size_t ring = (size_t)kXtrStages * kXtrRows * (32 * (64 / RMAX) * sizeof(S) + RMAX * sizeof(float));
  constexpr size_t red = (size_t)8 * 64 * 32 * sizeof(float);
  return ring > red ? ring : red;
}
template <typename S, int RMAX>
__global__ void __launch_bounds__(288) skinny_xtr_bulk_kernel(const S* __restrict__ X, int64_t n, int64_t d, int64_t ld,
                                                              const float* __restrict__ Rm, int R,
                                                              int64_t rows_per_chunk, float* __restrict__ part,
                                                              int* status) {
  constexpr int CPL = 64 / RMAX;
  constexpr int CPW = 32 * CPL;
  constexpr uint32_t XROW = CPW * sizeof(S);
  constexpr uint32_t XST = kXtrRows * XROW;
  constexpr uint32_t ST = XST + kXtrRows * RMAX * sizeof(float);
  extern __shared__ __align__(128) unsigned char xb_sh[];
  __shared__ uint64_t full[kXtrStages], empty[kXtrStages];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cb0 = (int64_t)blockIdx.y * CPW;
  const int64_t i0 = (int64_t)blockIdx.x * rows_per_chunk, i1 = min64(n, i0 + rows_per_chunk);
  const int64_t ntile = i1 > i0 ? (i1 - i0 + kXtrRows - 1) / kXtrRows : 0;
  // whole 16-byte units: a row slice is read up to the next 16-byte boundary, which lies inside
  // the row stride; staged columns >= d only reach accumulators that are never written
  const uint32_t xbytes = (uint32_t)((min64(CPW, d - cb0) * (int64_t)sizeof(S) + 15) / 16 * 16);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kXtrStages; ++s) {
      mbar_init_cta(&full[s], 1);
      mbar_init_cta(&empty[s], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  float acc[CPL][RMAX];
#pragma unroll
  for (int e = 0; e < CPL; ++e)
#pragma unroll
    for (int r = 0; r < RMAX; ++r) acc[e][r] = 0.0f;
  if (warp == 8) {
    if (lane == 0) {   // producer
      int64_t last_use[kXtrStages];
      for (int s = 0; s < kXtrStages; ++s) last_use[s] = -1;
      for (int64_t t = 0; t < ntile; ++t) {
        const int s = (int)(t % kXtrStages);
        const int64_t u = t / kXtrStages;
        if (u >= 1 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kXtrWait)) {
          atomicOr(status, STATUS_TIMEOUT);
          break;
        }
        const int64_t r0 = i0 + t * kXtrRows;
        const int rows = (int)min64(kXtrRows, i1 - r0);
        unsigned char* st = xb_sh + (size_t)s * ST;
        mbar_expect_tx_cta(&full[s], (uint32_t)rows * xbytes + (uint32_t)rows * RMAX * (uint32_t)sizeof(float));
        for (int r = 0; r < rows; ++r) bulk_copy_g2s(st + r * XROW, X + (r0 + r) * ld + cb0, xbytes, &full[s]);
        bulk_copy_g2s(st + XST, Rm + r0 * RMAX, (uint32_t)rows * RMAX * (uint32_t)sizeof(float), &full[s]);
        last_use[s] = u;
      }
      for (int s = 0; s < kXtrStages; ++s)   // every issued copy lands before the ring is reused
        if (last_use[s] >= 0 && !mbar_wait_bounded(&full[s], (uint32_t)(last_use[s] & 1), kXtrWait))
          atomicOr(status, STATUS_TIMEOUT);
    }
  } else {   // consumers: warp w takes rows 2w and 2w + 1 of each tile
    for (int64_t t = 0; t < ntile; ++t) {
      const int s = (int)(t % kXtrStages);
      const int64_t u = t / kXtrStages;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(u & 1), kXtrWait)) {
        if (lane == 0) atomicOr(status, STATUS_TIMEOUT);
        break;
      }
      const int rows = (int)min64(kXtrRows, i1 - (i0 + t * kXtrRows));
      const unsigned char* st = xb_sh + (size_t)s * ST;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = 2 * warp + h;
        if (rr < rows) {
          float xv[CPL];
          const S* xs = reinterpret_cast<const S*>(st + rr * XROW) + lane * CPL;
          if constexpr (sizeof(S) == 2) {
            uint32_t w[CPL / 2];
            if constexpr (CPL == 8) {
              const uint4 q = *reinterpret_cast<const uint4*>(xs);
              w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
            } else if constexpr (CPL == 4) {
              const uint2 q = *reinterpret_cast<const uint2*>(xs);
              w[0] = q.x; w[1] = q.y;
            } else {
              w[0] = *reinterpret_cast<const uint32_t*>(xs);
            }
#pragma unroll
            for (int k = 0; k < CPL / 2; ++k) {
              xv[2 * k] = __uint_as_float(w[k] << 16);
              xv[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
            }
          } else {
#pragma unroll
            for (int e = 0; e < CPL; ++e) xv[e] = (float)xs[e];
          }
          const float4* rq4 = reinterpret_cast<const float4*>(st + XST + rr * RMAX * sizeof(float));
#pragma unroll
          for (int q = 0; q < RMAX / 4; ++q) {
            const float4 rq = rq4[q];
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
              acc[e][4 * q] = fmaf(xv[e], rq.x, acc[e][4 * q]);
              acc[e][4 * q + 1] = fmaf(xv[e], rq.y, acc[e][4 * q + 1]);
              acc[e][4 * q + 2] = fmaf(xv[e], rq.z, acc[e][4 * q + 2]);
              acc[e][4 * q + 3] = fmaf(xv[e], rq.w, acc[e][4 * q + 3]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&empty[s]);
    }
  }
  __syncthreads();
  float* red = reinterpret_cast<float*>(xb_sh);   // [8][CPL * RMAX][32]
  if (warp < 8) {
#pragma unroll
    for (int e = 0; e < CPL; ++e)
#pragma unroll
      for (int r = 0; r < RMAX; ++r) red[((warp * CPL + e) * RMAX + r) * 32 + lane] = acc[e][r];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < CPL * RMAX * 32; k += blockDim.x) {
    float sum = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += red[w * CPL * RMAX * 32 + k];
    const int L = k % 32, er = k / 32, e = er / RMAX, r = er % RMAX;
    const int64_t col = cb0 + L * CPL + e;
    if (col < d && r < R) part[((int64_t)blockIdx.x * d + col) * R + r] = sum;
  }
}

// G[c][r] = (1/n) sum over chunks of the partials, in chunk order, in double
__global__ void skinny_reduce_kernel(const float* __restrict__ part, int nchunks, int64_t dr, double inv_n,
                                     double* __restrict__ G) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < dr; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nchunks; ++q) s += (double)part[(int64_t)q * dr + e];
    G[e] = s * inv_n;
  }
}

int blocks_cap(rs_ctx* ctx, int64_t work) {
  int64_t g = (work + 255) / 256;
  g = std::min<int64_t>(g, (int64_t)ctx->num_sms * 8);
  return (int)std::max<int64_t>(g, 1);
}

// bump allocator over one device buffer (256-byte aligned pieces)
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <typename U> U* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    U* p = base ? reinterpret_cast<U*>(base + off) : nullptr;
    off += count * sizeof(U);
    return p;
  }
};

struct Pair {        // one (problem, lambda): components and sampling table
  int p;
  double lam;
  void* Z;
  int64_t ldz;
  float* beta;
  uint32_t* W;
  uint64_t* cum;
  float* a;
  double bh;
};

// Side streams (non-blocking) and fork/join events for work that runs side by side; released on
// scope exit (a stream with work still queued is released once that work completes).
struct SideStreams {
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  int open(int count) {
    if (count <= 0) return RS_OK;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
      return rs_fail(RS_ECUDA, "side streams: event creation failed");
    for (int i = 0; i < count; ++i) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return rs_fail(RS_ECUDA, "side streams: stream creation failed");
      s.push_back(st);
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        return rs_fail(RS_ECUDA, "side streams: event creation failed");
      join.push_back(ev);
    }
    return RS_OK;
  }
  ~SideStreams() {
    for (auto e : join) cudaEventDestroy(e);
    for (auto st : s) cudaStreamDestroy(st);
    if (fork) cudaEventDestroy(fork);
  }
};

struct ProbWs {
  float* V;
  double* s2;
  float* U;          // d x R (refined snapshot gradient)
  float* Rm;         // n x R
  double* G;         // d x R
  int R;
  int Rp;            // column stride of U and Rm: R padded to 8, 16 or 32 (R itself beyond 32)
  int64_t k;
};

struct ChainWs {
  int pair, r;       // r: column of this chain in its problem's U / G
  int64_t m, nblk;
  double eta;
  float *wa, *wb, *mu, *u, *inq, *Rt, *cv, *Kt, *hn;
  uint32_t* idx;
};

template <typename S>
int solve_batched_body(rs_ctx* ctx, const rs_problem* P, int np, const rs_chain* C, int nc, const rs_batch_params* bp,
                       float* epoch_ms) {
  const int32_t dt = P[0].X.dtype;
  const int S_ep = bp->epochs;
  const bool refine = bp->refine != 0;
  // ---- (problem, lambda) pairs and per-problem chain columns
  std::vector<Pair> pairs;
  std::map<std::pair<int, uint64_t>, int> pair_of;
  std::vector<ChainWs> cw(nc);
  std::vector<ProbWs> pw(np);
  for (int p = 0; p < np; ++p) {
    pw[p].R = 0;
    pw[p].k = P[p].k > 0 ? P[p].k : std::max<int64_t>(1, P[p].X.d / 16);
  }
  for (int c = 0; c < nc; ++c) {
    uint64_t bits;
    std::memcpy(&bits, &C[c].lambda, sizeof(bits));
    auto key = std::make_pair((int)C[c].problem, bits);
    auto it = pair_of.find(key);
    if (it == pair_of.end()) {
      Pair q{};
      q.p = C[c].problem;
      q.lam = C[c].lambda;
      pairs.push_back(q);
      it = pair_of.emplace(key, (int)pairs.size() - 1).first;
    }
    cw[c].pair = it->second;
    cw[c].r = pw[C[c].problem].R++;
    const int64_t n = P[C[c].problem].X.n;
    cw[c].m = C[c].m > 0 ? C[c].m : 2 * n;
    if (cw[c].m >= (1LL << 31)) return rs_fail(RS_EINVAL, "rs_solve_batched: chain %d: m too large", c);
    cw[c].nblk = (cw[c].m + kChainBlk - 1) / kChainBlk;
  }
  // ---- workspace: two passes of the carver (sizes, then pointers)
  Carver cv;
  std::vector<int> order(nc);   // chains sorted by d (each batched inner-loop launch shares d)
  for (int c = 0; c < nc; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return P[C[a].problem].X.d < P[C[b].problem].X.d; });
  const size_t es = sizeof(S);
  ChainJob<S, float>* jobs_dev = nullptr;
  IdxJob* idx_dev = nullptr;
  MapJob *umap_dev = nullptr, *mumap_dev = nullptr, *snap_dev = nullptr, *final_dev = nullptr;
  int64_t *blk_off_dev = nullptr, *idx_off_dev = nullptr;
  int nsnap = 0;
  for (int c = 0; c < nc; ++c) nsnap += C[c].snapshots != nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    cv.off = 0;
    for (int p = 0; p < np; ++p) {
      const int64_t n = P[p].X.n, d = P[p].X.d, k = pw[p].k, R = std::max(1, pw[p].R);
      pw[p].Rp = R <= 8 ? 8 : (R <= 16 ? 16 : (R <= 32 ? 32 : (int)R));
      const int64_t Rp = pw[p].Rp;
      pw[p].V = cv.take<float>(d * k);
      pw[p].s2 = cv.take<double>(k);
      pw[p].U = refine ? cv.take<float>(d * Rp) : nullptr;
      pw[p].Rm = refine ? cv.take<float>(n * Rp) : nullptr;
      pw[p].G = refine ? cv.take<double>(d * R) : nullptr;
    }
    for (auto& q : pairs) {
      const int64_t n = P[q.p].X.n, d = P[q.p].X.d, N = n + d;
      q.ldz = (d * (int64_t)es + 15) / 16 * 16 / (int64_t)es;
      q.Z = cv.take<S>(N * q.ldz);
      q.beta = cv.take<float>(N);
      q.W = cv.take<uint32_t>(N);
      q.cum = cv.take<uint64_t>(N);
      q.a = cv.take<float>(pw[q.p].k);
    }
    for (int c = 0; c < nc; ++c) {
      const int64_t d = P[C[c].problem].X.d;
      cw[c].wa = cv.take<float>(d);
      cw[c].wb = cv.take<float>(d);
      cw[c].mu = cv.take<float>(d);
      cw[c].u = cv.take<float>(d);
      cw[c].idx = cv.take<uint32_t>(cw[c].m);
      cw[c].inq = cv.take<float>(cw[c].m);
      cw[c].Rt = cv.take<float>(cw[c].nblk * kChainBlk * kChainBlk);
      cw[c].cv = cv.take<float>(cw[c].nblk * kChainBlk);
      cw[c].Kt = cv.take<float>(cw[c].nblk * kChainBlk * kChainBlk);   // look-ahead cross Gram matrices
      cw[c].hn = cv.take<float>(cw[c].nblk * kChainBlk);
    }
    jobs_dev = cv.take<ChainJob<S, float>>(2 * (size_t)nc);
    idx_dev = cv.take<IdxJob>(nc);
    umap_dev = cv.take<MapJob>(2 * (size_t)nc);
    mumap_dev = cv.take<MapJob>(nc);
    snap_dev = cv.take<MapJob>(2 * (size_t)std::max(1, nsnap));
    final_dev = cv.take<MapJob>(nc);
    blk_off_dev = cv.take<int64_t>(nc + 1);
    idx_off_dev = cv.take<int64_t>(nc + 1);
    if (pass == 0) {
      cv.base = static_cast<char*>(rs_scratch(ctx, SCR_BATCH, cv.off + 256));
      if (!cv.base) return rs_fail(RS_ENOMEM, "rs_solve_batched: %.2f GB workspace does not fit", cv.off * 1e-9);
    }
  }
  // ---- setup: sketches, components, sampling tables (eager, synchronising)
  for (int p = 0; p < np; ++p) {
    rs_sketch_params sp{};
    sp.kind = bp->sketch_kind;
    sp.k = (int32_t)pw[p].k;
    sp.s = 0;
    sp.q_blocks = std::max(1, bp->q_blocks);
    sp.seed = bp->sketch_seed + (uint64_t)p;
    RS_TRY(sketch_dispatch(ctx, &P[p].X, &sp, pw[p].V, pw[p].s2));
  }
  for (auto& q : pairs) {
    const rs_matrix& X = P[q.p].X;
    const int64_t N = X.n + X.d;
    rs_matrix Zm = {q.Z, nullptr, N, X.d, q.ldz, dt, 0};
    RS_TRY(precondition_dispatch(ctx, &X, pw[q.p].V, pw[q.p].s2, pw[q.p].k, q.lam, &Zm, q.beta, &q.bh));
    if (!(q.bh > 0.0) || !std::isfinite(q.bh)) return rs_fail(RS_ENONFINITE, "rs_solve_batched: mean smoothness %g", q.bh);
    RS_TRY(sampling_weights_dispatch(ctx, q.beta, RS_F32, N, q.W));
    RS_TRY(scan_u32_to_u64(ctx, q.W, q.cum, N));
    adiag_f_kernel<<<(unsigned)((pw[q.p].k + 255) / 256), 256, 0, ctx->stream>>>(pw[q.p].s2, (int)pw[q.p].k, q.lam,
                                                                                 q.a);
    RS_LAUNCH_CHECK(ctx);
  }
  for (int p = 0; p < np; ++p)
    if (refine) RS_CUDA_TRY(cudaMemsetAsync(pw[p].U, 0, (size_t)P[p].X.d * pw[p].Rp * sizeof(float), ctx->stream));
  for (int c = 0; c < nc; ++c) {
    cw[c].eta = (C[c].eta_mult > 0.0 ? C[c].eta_mult : 1.0) / pairs[cw[c].pair].bh;
    RS_CUDA_TRY(cudaMemsetAsync(cw[c].wa, 0, P[C[c].problem].X.d * sizeof(float), ctx->stream));
  }
  // ---- job tables (host), copied once
  std::vector<ChainJob<S, float>> jobs(2 * (size_t)nc);
  std::vector<IdxJob> ij(nc);
  std::vector<MapJob> um(2 * (size_t)nc), mm(nc), sm(2 * (size_t)std::max(1, nsnap)), fm(nc);
  std::vector<int64_t> blk_off(nc + 1, 0), idx_off(nc + 1, 0);
  int si = 0;
  for (int o = 0; o < nc; ++o) {
    const int c = order[o];
    const Pair& q = pairs[cw[c].pair];
    const rs_problem& pr = P[C[c].problem];
    const ProbWs& W = pw[C[c].problem];
    const int64_t n = pr.X.n, d = pr.X.d;
    for (int par = 0; par < 2; ++par) {
      ChainJob<S, float>& J = jobs[par * (size_t)nc + o];
      J.Z = static_cast<const S*>(q.Z);
      J.N = n + d;
      J.ld = q.ldz;
      J.d = d;
      J.n = n;
      J.m = cw[c].m;
      J.idx = cw[c].idx;
      J.inv_nq = cw[c].inq;
      J.lam = q.lam;
      J.eta = cw[c].eta;
      J.mu = cw[c].mu;
      J.wbar = par ? cw[c].wb : cw[c].wa;
      J.wnext = par ? cw[c].wa : cw[c].wb;
      J.Rt = cw[c].Rt;
      J.cvec = cw[c].cv;
      J.Kt = cw[c].Kt;
      J.hn = cw[c].hn;
      J.average = bp->average;
      J.reserved = 0;
      MapJob u{};
      u.V = W.V;
      u.a = q.a;
      u.d = d;
      u.k = (int32_t)W.k;
      u.xf = par ? cw[c].wb : cw[c].wa;
      u.xf_scale = 1.0;
      u.y = refine ? W.U + cw[c].r : cw[c].u;
      u.y_ld = refine ? W.Rp : 1;
      u.y2 = refine ? cw[c].u : nullptr;
      um[par * (size_t)nc + o] = u;
      if (C[c].snapshots) {
        MapJob sj = u;
        sj.xf = par ? cw[c].wa : cw[c].wb;   // the new snapshot wnext
        sj.y = C[c].snapshots;
        sj.y_ld = 1;
        sj.y_epoch_stride = d;
        sj.y2 = nullptr;
        sm[par * (size_t)std::max(1, nsnap) + si] = sj;
      }
    }
    if (C[c].snapshots) ++si;
    MapJob mj{};
    mj.V = W.V;
    mj.a = q.a;
    mj.d = d;
    mj.k = (int32_t)W.k;
    mj.xg = refine ? W.G + cw[c].r : nullptr;
    mj.xg_ld = W.R;
    mj.xg_scale = 1.0;
    mj.xf = cw[c].u;
    mj.xf_scale = q.lam;
    mj.y = cw[c].mu;
    mj.y_ld = 1;
    mm[o] = mj;
    MapJob fj = um[o];
    fj.xf = (S_ep & 1) ? cw[c].wb : cw[c].wa;   // the snapshot after S epochs
    fj.y = C[c].w_out;
    fj.y_ld = 1;
    fj.y2 = nullptr;
    fj.check = 1;
    fm[o] = fj;
    IdxJob x{};
    x.W = q.W;
    x.cum = q.cum;
    x.N = n + d;
    x.m = cw[c].m;
    x.seed = C[c].seed;
    x.idx = cw[c].idx;
    x.inv_nq = cw[c].inq;
    ij[o] = x;
    blk_off[o + 1] = blk_off[o] + cw[c].nblk;
    idx_off[o + 1] = idx_off[o] + cw[c].m;
  }
  RS_CUDA_TRY(cudaMemcpyAsync(jobs_dev, jobs.data(), jobs.size() * sizeof(jobs[0]), cudaMemcpyHostToDevice, ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(idx_dev, ij.data(), ij.size() * sizeof(IdxJob), cudaMemcpyHostToDevice, ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(umap_dev, um.data(), um.size() * sizeof(MapJob), cudaMemcpyHostToDevice, ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(mumap_dev, mm.data(), mm.size() * sizeof(MapJob), cudaMemcpyHostToDevice, ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(snap_dev, sm.data(), sm.size() * sizeof(MapJob), cudaMemcpyHostToDevice, ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(final_dev, fm.data(), fm.size() * sizeof(MapJob), cudaMemcpyHostToDevice, ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(blk_off_dev, blk_off.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                              ctx->stream));
  RS_CUDA_TRY(cudaMemcpyAsync(idx_off_dev, idx_off.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                              ctx->stream));
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  // groups of consecutive (sorted) chains with the same d
  std::vector<std::pair<int, int>> groups;   // (first, count)
  for (int o = 0; o < nc;) {
    int e = o;
    const int64_t d = P[C[order[o]].problem].X.d;
    while (e < nc && P[C[order[e]].problem].X.d == d) ++e;
    groups.emplace_back(o, e - o);
    o = e;
  }
  const int64_t total_blocks = blk_off[nc], total_steps = idx_off[nc];
  SideStreams side;
  RS_TRY(side.open(std::min<int>((int)groups.size() - 1, 7)));

  auto run_epoch = [&](int s) -> int {
    const int par = s & 1;
    if (refine) {
      bmap_kernel<<<nc, 256, 0, ctx->stream>>>(umap_dev + par * (size_t)nc, 0, ctx->d_status);
      RS_LAUNCH_CHECK(ctx);
      for (int p = 0; p < np; ++p) {
        if (pw[p].R == 0) continue;
        const rs_matrix& X = P[p].X;
        const int64_t n = X.n, d = X.d, R = pw[p].R;
        const S* Xd = static_cast<const S*>(X.data);
        if (R <= 32) {
          // two streaming passes over X with the R columns in registers
          const int rmax = pw[p].Rp;
          constexpr int CPLU = 16 / (int)sizeof(S);
          const int64_t ng = (d + CPLU - 1) / CPLU;
          const size_t ushm = (size_t)ng * (CPLU * rmax + 4) * sizeof(float);
          const bool usm = ushm <= 100 * 1024;
          const int xu_blocks = ctx->num_sms * 2;
          // bfloat16 data: R = X U on the tensor cores (U split in three bfloat16 parts), then - y
          int rc_xu = RS_EUNSUPPORTED;
          if constexpr (std::is_same<S, __nv_bfloat16>::value)
            if (umma_enabled()) rc_xu = umma_gemm_xw(ctx, &X, pw[p].U, rmax, nullptr, pw[p].Rm, rmax, false);
          if (rc_xu != RS_OK && rc_xu != RS_EUNSUPPORTED) return rc_xu;
          if (rc_xu == RS_OK) {
            sub_labels_kernel<<<blocks_cap(ctx, n * rmax), 256, 0, ctx->stream>>>(pw[p].Rm, n, rmax, P[p].y);
          } else {
#define RS_XU(RM)                                                                                                    \
  do {                                                                                                               \
    if (usm) {                                                                                                       \
      RS_CUDA_TRY(cudaFuncSetAttribute(skinny_xu_kernel<S, RM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                       (int)ushm));                                                                  \
      skinny_xu_kernel<S, RM, true><<<xu_blocks, 256, ushm, ctx->stream>>>(Xd, n, d, X.ld, pw[p].U, (int)R, P[p].y,  \
                                                                           pw[p].Rm);                                \
    } else {                                                                                                         \
      skinny_xu_kernel<S, RM, false><<<xu_blocks, 256, 0, ctx->stream>>>(Xd, n, d, X.ld, pw[p].U, (int)R, P[p].y,    \
                                                                         pw[p].Rm);                                  \
    }                                                                                                                \
  } while (0)
          if (rmax == 8) RS_XU(8);
          else if (rmax == 16) RS_XU(16);
          else RS_XU(32);
#undef RS_XU
          }
          RS_LAUNCH_CHECK(ctx);
          const int cpw = 32 * (64 / rmax);   // columns per block of the transposed product
          const int cb = (int)((d + cpw - 1) / cpw);
          // row chunks: about two CTAs per SM in all, whole tiles of 16 rows
          const int nch = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 2 / cb, (n + 255) / 256));
          const int64_t rpc = ((n + nch - 1) / nch + 15) / 16 * 16;
          float* part = static_cast<float*>(rs_scratch(ctx, SCR_BPART, (size_t)nch * d * R * sizeof(float)));
          if (!part) return RS_ENOMEM;
          dim3 g2((unsigned)nch, (unsigned)cb);
#define RS_XTR(RM)                                                                                                 \
  do {                                                                                                             \
    constexpr size_t rshm = xtr_bulk_smem<S, RM>();                                                               \
    RS_CUDA_TRY(cudaFuncSetAttribute(skinny_xtr_bulk_kernel<S, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                     (int)rshm));                                                                  \
    skinny_xtr_bulk_kernel<S, RM><<<g2, 288, rshm, ctx->stream>>>(Xd, n, d, X.ld, pw[p].Rm, (int)R, rpc, part,    \
                                                                   ctx->d_status);                                 \
  } while (0)
          if (rmax == 8) RS_XTR(8);
          else if (rmax == 16) RS_XTR(16);
          else RS_XTR(32);
#undef RS_XTR
          RS_LAUNCH_CHECK(ctx);
          skinny_reduce_kernel<<<blocks_cap(ctx, d * R), 256, 0, ctx->stream>>>(part, nch, d * R, 1.0 / (double)n,
                                                                                pw[p].G);
          RS_LAUNCH_CHECK(ctx);
        } else {
          RS_TRY(launch_gemm<float, S, float>(ctx, n, R, d, 1.0, Xd, X.ld, 1, pw[p].U, R, 1, 0.0, nullptr, 0, pw[p].Rm,
                                              R, nullptr));
          sub_labels_kernel<<<blocks_cap(ctx, n * R), 256, 0, ctx->stream>>>(pw[p].Rm, n, (int)R, P[p].y);
          RS_LAUNCH_CHECK(ctx);
          RS_TRY(launch_gram<S, float>(ctx, n, d, R, Xd, X.ld, pw[p].Rm, R, 1.0 / (double)n, pw[p].G));
        }
      }
      bmap_kernel<<<nc, 256, 0, ctx->stream>>>(mumap_dev, 0, ctx->d_status);
      RS_LAUNCH_CHECK(ctx);
    } else {
      for (int o = 0; o < nc; ++o) {
        const int c = order[o];
        const Pair& q = pairs[cw[c].pair];
        const rs_matrix& X = P[q.p].X;
        rs_matrix Zm = {q.Z, nullptr, X.n + X.d, X.d, q.ldz, dt, 0};
        RS_TRY(rs_full_gradient(ctx, &Zm, P[q.p].y, X.n, q.lam, par ? cw[c].wb : cw[c].wa, cw[c].mu));
      }
    }
    RS_TRY(index_stream_batched(ctx, idx_dev, idx_off_dev, nc, total_steps, (uint32_t)s));
    RS_TRY(epoch_prep_batched<S, float>(ctx, jobs_dev + par * (size_t)nc, blk_off_dev, nc, total_blocks));
    // the width groups' inner loops run side by side: group 0 on the solver's stream, the others
    // on side streams forked from and joined back into it
    const int nside = std::min<int>((int)groups.size() - 1, (int)side.s.size());
    if (nside > 0) {
      RS_CUDA_TRY(cudaEventRecord(side.fork, ctx->stream));
      for (int i = 0; i < nside; ++i) RS_CUDA_TRY(cudaStreamWaitEvent(side.s[i], side.fork, 0));
    }
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const auto& g = groups[gi];
      cudaStream_t main_stream = ctx->stream;
      if (nside > 0 && gi > 0) ctx->stream = side.s[(gi - 1) % nside];
      const int grc = epoch_chain_batched<S, float>(ctx, jobs_dev + par * (size_t)nc + g.first, g.second,
                                                    P[C[order[g.first]].problem].X.d);
      ctx->stream = main_stream;
      if (grc != RS_OK) return grc;
    }
    for (int i = 0; i < nside; ++i) {
      RS_CUDA_TRY(cudaEventRecord(side.join[i], side.s[i]));
      RS_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, side.join[i], 0));
    }
    if (nsnap) {
      bmap_kernel<<<nsnap, 256, 0, ctx->stream>>>(snap_dev + par * (size_t)std::max(1, nsnap), s, ctx->d_status);
      RS_LAUNCH_CHECK(ctx);
    }
    return RS_OK;
  };

  std::vector<cudaEvent_t> ev;
  if (epoch_ms) {
    ev.resize(S_ep + 1);
    for (auto& e : ev) RS_CUDA_TRY(cudaEventCreate(&e));
    RS_CUDA_TRY(cudaEventRecord(ev[0], ctx->stream));
  }
  int rc = run_epoch(0);
  if (rc == RS_OK && !ev.empty()) rc = cudaEventRecord(ev[1], ctx->stream) == cudaSuccess ? RS_OK : RS_ECUDA;
  if (rc == RS_OK && S_ep > 1) {
    if (bp->use_graph) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      RS_CUDA_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
      for (int s = 1; s < S_ep && rc == RS_OK; ++s) {
        rc = run_epoch(s);
        // inside a capture only an external event-record node records the event when the graph runs
        if (rc == RS_OK && !ev.empty() &&
            cudaEventRecordWithFlags(ev[s + 1], ctx->stream, cudaEventRecordExternal) != cudaSuccess)
          rc = rs_fail(RS_ECUDA, "rs_solve_batched: event record in capture failed");
      }
      const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
      if (rc == RS_OK && ce != cudaSuccess) rc = rs_fail(RS_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
      if (rc == RS_OK) {
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        if (ie != cudaSuccess) rc = rs_fail(RS_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
      }
      if (rc == RS_OK) {
        const cudaError_t le = cudaGraphLaunch(exec, ctx->stream);
        if (le != cudaSuccess) rc = rs_fail(RS_ECUDA, "graph launch: %s", cudaGetErrorString(le));
      }
      if (rc == RS_OK) RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
    } else {
      for (int s = 1; s < S_ep && rc == RS_OK; ++s) {
        rc = run_epoch(s);
        if (rc == RS_OK && !ev.empty()) RS_CUDA_TRY(cudaEventRecord(ev[s + 1], ctx->stream));
      }
    }
  }
  if (rc == RS_OK) {
    bmap_kernel<<<nc, 256, 0, ctx->stream>>>(final_dev, 0, ctx->d_status);
    rc = cudaGetLastError() == cudaSuccess ? RS_OK : rs_fail(RS_ECUDA, "final map launch failed");
    ctx->launches++;
  }
  int st = 0;
  if (rc == RS_OK) {
    RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (!ev.empty())
      for (int s = 0; s < S_ep; ++s)
        if (cudaEventElapsedTime(&epoch_ms[s], ev[0], ev[s + 1]) != cudaSuccess) {
          cudaGetLastError();
          epoch_ms[s] = -1.0f;
        }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc != RS_OK) return rc;
  if (st & STATUS_TIMEOUT) return rs_fail(RS_ETIMEOUT, "rs_solve_batched: a bounded wait of an inner-loop chain gave up");
  if (st & STATUS_NONFINITE) return rs_fail(RS_ENONFINITE, "rs_solve_batched: an iterate became non-finite");
  return RS_OK;
}

// The work runs on a private non-blocking stream ordered after the context's stream (the legacy
// default stream cannot be captured into a graph); the context's stream waits for it at the end.
template <typename S>
int solve_batched_t(rs_ctx* ctx, const rs_problem* P, int np, const rs_chain* C, int nc, const rs_batch_params* bp,
                    float* epoch_ms) {
  cudaStream_t user = ctx->stream, own = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RS_CUDA_TRY(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
  int rc = RS_OK;
  if (cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(e0, user) != cudaSuccess ||
      cudaStreamWaitEvent(own, e0, 0) != cudaSuccess)
    rc = rs_fail(RS_ECUDA, "rs_solve_batched: stream setup failed");
  if (rc == RS_OK) {
    ctx->stream = own;
    rc = solve_batched_body<S>(ctx, P, np, C, nc, bp, epoch_ms);
    ctx->stream = user;
  }
  if (e1 && cudaEventRecord(e1, own) == cudaSuccess) cudaStreamWaitEvent(user, e1, 0);
  cudaStreamSynchronize(own);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(own);
  return rc;
}

}  // namespace

extern "C" int rs_solve_batched(rs_ctx* ctx, const rs_problem* probs, int32_t nprob, const rs_chain* chains,
                                int32_t nchain, const rs_batch_params* p, float* epoch_ms) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(probs && chains && p && nprob >= 1 && nchain >= 1, "rs_solve_batched: null argument or empty batch");
  RS_CHECK_ARG(p->epochs >= 1, "rs_solve_batched: epochs must be >= 1");
  RS_CHECK_ARG(p->sketch_kind == RS_SKETCH_GAUSSIAN || p->sketch_kind == RS_SKETCH_COUNTSKETCH,
               "rs_solve_batched: bad sketch kind");
  const int32_t dt = probs[0].X.dtype;
  RS_CHECK_ARG(dt == RS_F32 || dt == RS_BF16, "rs_solve_batched: data must be RS_F32 or RS_BF16");
  RS_CHECK_ARG(dt == RS_F32 || p->refine, "rs_solve_batched: RS_BF16 data needs refine = 1");
  for (int i = 0; i < nprob; ++i) {
    RS_TRY(check_matrix(&probs[i].X, "rs_solve_batched X"));
    RS_CHECK_ARG(probs[i].X.dtype == dt, "rs_solve_batched: all problems must share the dtype");
    RS_CHECK_ARG(probs[i].y, "rs_solve_batched: problem %d has no labels", i);
    const int64_t d = probs[i].X.d;
    const int64_t k = probs[i].k > 0 ? probs[i].k : std::max<int64_t>(1, d / 16);
    RS_CHECK_ARG(k <= d && k <= 256, "rs_solve_batched: problem %d: k must be in [1, min(d, 256)]", i);
    RS_CHECK_ARG(d <= 4096, "rs_solve_batched: problem %d: d > 4096 is not supported", i);
  }
  for (int c = 0; c < nchain; ++c) {
    RS_CHECK_ARG(chains[c].problem >= 0 && chains[c].problem < nprob, "rs_solve_batched: chain %d: bad problem", c);
    RS_CHECK_ARG(chains[c].lambda > 0.0, "rs_solve_batched: chain %d: lambda must be positive", c);
    RS_CHECK_ARG(chains[c].w_out, "rs_solve_batched: chain %d: null w_out", c);
  }
  if (dt == RS_BF16) return solve_batched_t<__nv_bfloat16>(ctx, probs, nprob, chains, nchain, p, epoch_ms);
  return solve_batched_t<float>(ctx, probs, nprob, chains, nchain, p, epoch_ms);
}
