// Internal definitions shared by the library's translation units (never by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <cstdarg>
#include <type_traits>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rs.h"

// ------------------------------------------------------------------ context

struct ScratchSlot {
  void* ptr = nullptr;
  size_t bytes = 0;
};

enum ScratchId {
  SCR_OMEGA = 0, SCR_SX, SCR_Y, SCR_Q, SCR_GRAM, SCR_B, SCR_PART, SCR_PART2,
  SCR_P, SCR_ADIAG, SCR_W, SCR_CUM, SCR_IDX, SCR_INVNQ, SCR_R, SCR_C, SCR_MU, SCR_WBAR,
  SCR_WNEXT, SCR_BETA, SCR_Z, SCR_XDEV, SCR_YDEV, SCR_V, SCR_S2, SCR_WOUT, SCR_BUCKET,
  SCR_SIGN, SCR_CSR, SCR_CNT, SCR_RED, SCR_EIG, SCR_MISC, SCR_STATUS, SCR_TMPV, SCR_SIGMA, SCR_LINV,
  SCR_MLP_PART, SCR_MLP_IO, SCR_BATCH, SCR_VK, SCR_KT, SCR_HN, SCR_UMMA, SCR_Z8, SCR_BPART, SCR_RPART, SCR_XPART, SCR_ROWSQ, SCR_SKPART, SCR_RITZ, SCR_CATB, SCR_CATB2, SCR_CATS, SCR_CATV, SCR_LINVD, SCR_JAC2, SCR_MAPPART, SCR_COUNT
};

// Launch choices measured by rs_autotune for one (kernel, storage type, width): chain = cluster
// size, threads per block and ring stages; fullgrad = ring stages of the column-owner kernel.
enum { TUNE_CHAIN = 1, TUNE_FULLGRAD = 2 };
struct TuneEntry {
  int32_t kind = 0, dtype = -1;
  int64_t d = 0;
  int32_t a = 0, b = 0, c = 0;
  float ms = 0.0f;
};
constexpr int kTuneSlots = 32;

struct rs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t launches = 0;
  ScratchSlot slots[SCR_COUNT];
  int* d_status = nullptr;     // device status word (bit flags, see STATUS_*)
  // public calls entered (rs_enter); the bfloat16 parts of a float X kept in SCR_XPART are reused
  // only within the call that formed them (X cannot change during one call)
  uint64_t call_gen = 0;
  const void* xp_src = nullptr;
  int64_t xp_n = 0, xp_d = 0, xp_ld = 0;
  uint64_t xp_gen = ~uint64_t(0);
  TuneEntry tune[kTuneSlots];   // autotuner cache (rs_autotune); empty slots have kind 0
  int ntune = 0;
};

// The cached choice for (kind, dtype, d), or nullptr.
inline const TuneEntry* tune_find(const rs_ctx* ctx, int kind, int dtype, int64_t d) {
  for (int i = 0; i < ctx->ntune; ++i)
    if (ctx->tune[i].kind == kind && ctx->tune[i].dtype == dtype && ctx->tune[i].d == d) return &ctx->tune[i];
  return nullptr;
}
inline void tune_put(rs_ctx* ctx, const TuneEntry& e) {
  for (int i = 0; i < ctx->ntune; ++i)
    if (ctx->tune[i].kind == e.kind && ctx->tune[i].dtype == e.dtype && ctx->tune[i].d == e.d) {
      ctx->tune[i] = e;
      return;
    }
  if (ctx->ntune < kTuneSlots) ctx->tune[ctx->ntune++] = e;
  else ctx->tune[kTuneSlots - 1] = e;   // a full cache replaces its last entry
}
template <typename S> constexpr int32_t dtype_code() {
  return std::is_same<S, double>::value ? RS_F64
         : std::is_same<S, float>::value ? RS_F32
         : std::is_same<S, __nv_bfloat16>::value ? RS_BF16 : RS_FP8E4M3;
}

enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

// thread-local error message
void rs_set_error(const char* fmt, ...);
int rs_fail(int code, const char* fmt, ...);
void* rs_scratch(rs_ctx* ctx, int slot, size_t bytes);   // nullptr on failure (error set)

#define RS_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess)                                                             \
      return rs_fail(RS_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
  } while (0)

#define RS_TRY(...)                 \
  do {                              \
    int _s = (__VA_ARGS__);         \
    if (_s != RS_OK) return _s;     \
  } while (0)

#define RS_LAUNCH_CHECK(ctx)                                                           \
  do {                                                                                 \
    (ctx)->launches++;                                                                 \
    cudaError_t _e = cudaGetLastError();                                               \
    if (_e != cudaSuccess)                                                             \
      return rs_fail(RS_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(_e), __FILE__, __LINE__); \
  } while (0)

#define RS_CHECK_ARG(cond, ...)                          \
  do {                                                   \
    if (!(cond)) return rs_fail(RS_EINVAL, __VA_ARGS__); \
  } while (0)

// Ensure the ctx's device is current for this host thread.
int rs_enter(rs_ctx* ctx);

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline size_t dtype_size(int dt) {
  switch (dt) {
    case RS_F64: return 8;
    case RS_F32: return 4;
    case RS_BF16: return 2;
    case RS_FP8E4M3: return 1;
  }
  return 0;
}

int check_matrix(const rs_matrix* X, const char* name);

inline int grid_cap(const rs_ctx* ctx, int per_sm) { return ctx->num_sms * per_sm; }

// ---------------------------------------------------------- Philox4x32-10

struct U32x4 {
  uint32_t x, y, z, w;
};

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ U32x4 philox4x32_10(U32x4 c, uint64_t seed) {
  uint32_t k0 = static_cast<uint32_t>(seed);
  uint32_t k1 = static_cast<uint32_t>(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = U32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

enum { TAG_GAUSS = 1, TAG_COUNTSKETCH = 2, TAG_SAMPLE = 3 };

// uniform (2*(w>>9)+1) 2^-24 on (0,1): exact in float
__device__ __forceinline__ float u24f(uint32_t w) { return static_cast<float>(2u * (w >> 9) + 1u) * 0x1p-24f; }
__device__ __forceinline__ double u24d(uint32_t w) { return static_cast<double>(2u * (w >> 9) + 1u) * 0x1p-24; }

__device__ __forceinline__ void box_muller(float ua, float ub, float& z0, float& z1) {
  const float rho = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  z0 = rho * c;
  z1 = rho * s;
}
__device__ __forceinline__ void box_muller(double ua, double ub, double& z0, double& z1) {
  const double rho = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  z0 = rho * c;
  z1 = rho * s;
}

// ----------------------------------------------------------- small helpers

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return static_cast<double>(v); }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return static_cast<double>(__bfloat162float(v)); }

// element conversion without a round trip through double
template <typename T, typename S> __device__ __forceinline__ T cvt(S v) { return static_cast<T>(v); }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return static_cast<double>(__bfloat162float(v));
}
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }
// FP8-e4m3 codes (components stored with a per-row scale: value = code * scale)
template <> __device__ __forceinline__ float cvt<float, __nv_fp8_e4m3>(__nv_fp8_e4m3 v) { return static_cast<float>(v); }
template <> __device__ __forceinline__ double cvt<double, __nv_fp8_e4m3>(__nv_fp8_e4m3 v) {
  return static_cast<double>(static_cast<float>(v));
}
using fp8_t = __nv_fp8_e4m3;
template <typename S> struct IsFp8 { static constexpr bool value = false; };
template <> struct IsFp8<__nv_fp8_e4m3> { static constexpr bool value = true; };

template <typename T> struct Vec;        // 16-byte vector of T
template <> struct Vec<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int N = 2; };

__device__ __forceinline__ void vec_to_arr(const float4& v, float* a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ void vec_to_arr(const double2& v, double* a) { a[0] = v.x; a[1] = v.y; }

// ------------------------------------------ mbarrier and bulk-copy primitives (CTA scope)

__device__ __forceinline__ uint32_t cta_smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init_cta(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(cta_smem_addr(bar)), "r"(count) : "memory");
}
// arrive once and add tx_bytes to the transaction count of the current phase
__device__ __forceinline__ void mbar_expect_tx_cta(uint64_t* bar, uint32_t tx_bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                   cta_smem_addr(bar)),
               "r"(tx_bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_cta(uint64_t* bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(cta_smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test_parity_cta(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(cta_smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of the given parity to complete, at most `budget` clock cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_test_parity_cta(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) that completes
// its bytes on the mbarrier
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   cta_smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(cta_smem_addr(bar))
               : "memory");
}

// Internal launch helpers implemented in dense.cu, used by several entry points.
template <typename T> struct NoDeduce { using type = T; };   // keeps a parameter out of type deduction
// A, C and C0 may be stored in other types than the compute type T (bfloat16 data).
template <typename T, typename TA = T, typename TC = T, typename TC0 = TC>
int launch_gemm(rs_ctx* ctx, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t sAm,
                int64_t sAk, const T* B, int64_t sBk, int64_t sBn, double beta, const typename NoDeduce<TC0>::type* C0,
                int64_t ldc0, TC* C, int64_t ldc, const T* col_scale);

// Gram / transposed product with split-K over the long dimension and double accumulation:
// G (Ma x Nb, double, row-major) = alpha * sum_r A[r][i] B[r][j], A: rows x Ma (lda), B: rows x Nb (ldb).
template <typename TA, typename TB = TA>
int launch_gram(rs_ctx* ctx, int64_t rows, int64_t Ma, int64_t Nb, const TA* A, int64_t lda, const TB* B,
                int64_t ldb, double alpha, double* G);

int run_sym_eig(rs_ctx* ctx, const double* G, int64_t k, int32_t prec, double* evals, double* W);

// tcgen05 product (umma.cu): C = X W diag(col_scale), X M x K bfloat16 or float rows (float rows are
// split into three bfloat16 parts first), W K x N float (N <= 256), C float; RS_EUNSUPPORTED when
// the tensor path cannot run (caller falls back).
bool umma_enabled();
// sync_check = false: no status reset and no synchronisation (usable inside a stream capture; the
// caller checks the status word afterwards).
int umma_gemm_xw(rs_ctx* ctx, const rs_matrix* X, const float* W, int64_t N, const float* col_scale, float* C,
                 int64_t ldc, bool sync_check = true);
// Y (d x k float) = X^T Pi on tensor cores for bfloat16 X (umma.cu), Pi the Gaussian test matrix of
// Alg. 2 with its entries rounded to bfloat16; RS_EUNSUPPORTED when the tensor path cannot run.
int umma_sketch(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t k, float* Y);
// Z (bfloat16) = X - P V^T (umma.cu) for bfloat16 X (k <= 128) or float X whose bfloat16 parts the
// same call has formed for X V (k <= 64), P n x k and V d x k float with row stride k;
// RS_EUNSUPPORTED when the tensor path cannot run.
// rowsq (optional, n floats) receives the squared norm of each stored (rounded) row of Z.
int umma_resid(rs_ctx* ctx, const rs_matrix* X, const float* P, const float* V, int64_t k, rs_matrix* Z,
               float* rowsq = nullptr);

// ------------------------------------------------ batched inner loops (many chains per launch)

// One chain of the inner loop of Alg. 1: components Z (storage S, N = n + d rows), the epoch's
// index stream and 1/(N q) factors, step size, snapshot gradient mu, snapshot wbar, output
// wnext, and its per-block workspace (Rt: blocks x 64 x 64, cvec: blocks x 64).
template <typename S, typename T>
struct ChainJob {
  const S* Z;
  int64_t N, ld, d, n, m;
  const uint32_t* idx;
  const T* inv_nq;
  double lam, eta;
  const T* mu;
  const T* wbar;
  T* wnext;
  T* Rt;
  T* cvec;
  T* Kt;        // look-ahead: blocks x 64 x 64 cross Gram matrices (next block's rows . this block's)
  T* hn;        // look-ahead: blocks x 64, next block's rows . mu
  int32_t average, reserved;
};

// Tensor-core (tcgen05) preparation of the blocked inner loop for bfloat16 components (umma.cu):
// R and c of every block of steps, as the CUDA-core preparation computes them.  jobs == nullptr:
// the single chain `one` over total_blocks blocks; otherwise CTA g serves the job j with
// blk_off[j] <= g < blk_off[j + 1] (device arrays, every Z 16-byte aligned with ld % 8 == 0).
// RS_EUNSUPPORTED when the tensor path is disabled or cannot run.
int umma_prep(rs_ctx* ctx, const ChainJob<__nv_bfloat16, float>& one, const ChainJob<__nv_bfloat16, float>* jobs,
              const int64_t* blk_off, int nj, int64_t total_blocks);

// Index stream of one chain (float factors): sampling table W / cum over N components.
struct IdxJob {
  const uint32_t* W;
  const uint64_t* cum;
  int64_t N, m;
  uint64_t seed;
  uint32_t* idx;
  float* inv_nq;
  int32_t uniform, reserved;
};

constexpr int kChainBlk = 64;   // steps per block of the blocked inner loop

// All jobs' index streams for one epoch; off (device, nj + 1) holds the prefix sums of m.
int index_stream_batched(rs_ctx* ctx, const IdxJob* jobs, const int64_t* off, int nj, int64_t total, uint32_t epoch);
// Per-block preparation for all jobs; blk_off (device, nj + 1): prefix sums of the block counts.
template <typename S, typename T>
int epoch_prep_batched(rs_ctx* ctx, const ChainJob<S, T>* jobs, const int64_t* blk_off, int nj, int64_t total_blocks);
// The chains of nj jobs that share d, one thread-block cluster each, in one launch.
template <typename S, typename T>
int epoch_chain_batched(rs_ctx* ctx, const ChainJob<S, T>* jobs, int nj, int64_t d);

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
