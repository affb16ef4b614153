// Tensor-core (tcgen05) product of bfloat16 or float data with a float matrix: C = X W diag(s), X
// (M x K, row-major), W (K x N, float), C (M x N, float).  This is the X V contraction of the
// preconditioner (Eq. (11)) and the X Q product of the Rayleigh-Ritz step (Alg. 2).  W is split
// into three bfloat16 parts, W = W0 + W1 + W2 (W1 = bf16(W - W0), ...), so the accumulating
// products reproduce the float W to about 2^-24 relative; bfloat16 X is exact, float X is split
// the same way into X0 + X1 + X2 and the six products X_a W_b with a + b <= 2 are accumulated
// (the dropped ones are below 2^-27).  Accumulation is FP32 in tensor memory.
//
// One CTA per 128 x 128 output tile, 128 threads: warp 0 allocates 128 tensor-memory columns and
// (lane 0) produces: TMA (cp.async.bulk.tensor, 128-byte swizzle) loads of the 128 x 64 X tile and
// the three 128 x 64 W-part tiles into a 3-stage ring whose full/empty mbarriers count the copied
// bytes and the completed MMAs; warp 1 lane 0 issues tcgen05.mma (M = 128, N = 128, K = 16, kind
// f16 with bfloat16 operands) and commits each stage back to its empty barrier; after the last
// stage all four warps read their 32 accumulator lanes with tcgen05.ld, scale the columns and
// store.  Every wait is bounded: on timeout the status word is flagged, no further copies or MMAs
// are issued, and the CTA still waits (bounded) for what it issued before freeing tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int UM = 128, UK = 64, NSPLIT = 3;
constexpr uint32_t A_BYTES = UM * UK * 2;               // 16 KB per X part
// NA = 1: bfloat16 X; NA = 3: float X split into three bfloat16 parts.  UN = 64 or 128 output
// columns per tile (W part tiles of UN x 64); as many ring stages as fit in 217 KB, at most 4.
template <int NA, int UN> __host__ __device__ constexpr uint32_t xw_stage_bytes() {
  return NA * A_BYTES + NSPLIT * (uint32_t)(UN * UK * 2);
}
template <int NA, int UN> __host__ __device__ constexpr int xw_stages() {
  return (int)(216u * 1024u / xw_stage_bytes<NA, UN>()) < 4 ? (int)(216u * 1024u / xw_stage_bytes<NA, UN>()) : 4;
}
constexpr long long kUmmaWait = 2000000000LL;

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  // K-major, 128-byte swizzle: start >> 4, leading offset (unused, 16 B), stride 1024 B between
  // 8-row groups, descriptor version 1, layout SWIZZLE_128B (2)
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: f32 accumulate, bf16 A and B, both K-major, N = UN, M = 128
template <int UN> __host__ __device__ constexpr uint32_t xw_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          cta_smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(cta_smem_addr(bar))
      : "memory");
}

template <int NA, int UN>
__global__ void __launch_bounds__(128, 1) umma_xw_kernel(const __grid_constant__ CUtensorMap tmX,
                                                         const __grid_constant__ CUtensorMap tmW, int64_t M, int K,
                                                         int N, int kp, const float* __restrict__ col_scale,
                                                         float* __restrict__ C, int64_t ldc, int* status) {
  constexpr int UST = xw_stages<NA, UN>();
  constexpr uint32_t STAGE_BYTES = xw_stage_bytes<NA, UN>();
  constexpr uint32_t B_BYTES = UN * UK * 2;
  constexpr uint32_t kIdesc = xw_idesc<UN>();
  extern __shared__ unsigned char um_raw[];
  // the swizzled tiles need 1024-byte alignment
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(um_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[UST], empty[UST], done;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * UM;
  const int n0 = blockIdx.y * UN;
  const int KB = (K + UK - 1) / UK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < UST; ++s) {
      mbar_init_cta(&full[s], 1);
      mbar_init_cta(&empty[s], 1);
    }
    mbar_init_cta(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cta_smem_addr(&tmem_holder)),
                 "r"(UN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;

  if (threadIdx.x == 0) {   // producer
    int issued_last[UST];
    for (int s = 0; s < UST; ++s) issued_last[s] = -1;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % UST, u = kb / UST;
      if (u >= 1 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kUmmaWait)) {
        atomicOr(status, STATUS_TIMEOUT);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      unsigned char* st = base + (size_t)s * STAGE_BYTES;
      mbar_expect_tx_cta(&full[s], STAGE_BYTES);
      for (int a = 0; a < NA; ++a) tma_load_2d(st + a * A_BYTES, &tmX, kb * UK, (int)(a * M + m0), &full[s]);
      for (int p = 0; p < NSPLIT; ++p)
        tma_load_2d(st + NA * A_BYTES + p * B_BYTES, &tmW, kb * UK, p * kp + n0, &full[s]);
      issued_last[s] = u;
    }
    for (int s = 0; s < UST; ++s)   // every issued copy lands before the CTA moves on
      if (issued_last[s] >= 0 && !mbar_wait_bounded(&full[s], (uint32_t)(issued_last[s] & 1), kUmmaWait))
        atomicOr(status, STATUS_TIMEOUT);
  } else if (threadIdx.x == 32) {   // MMA issuer
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % UST, u = kb / UST;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(u & 1), kUmmaWait)) {
        atomicOr(status, STATUS_TIMEOUT);
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = cta_smem_addr(base + (size_t)s * STAGE_BYTES);
      // products X_a W_b with a + b <= 2 (NA = 1: a = 0)
      constexpr int NPROD = NA == 1 ? 3 : 6;
#pragma unroll
      for (int kk = 0; kk < UK / 16; ++kk) {
#pragma unroll
        for (int q = 0; q < NPROD; ++q) {
          const int a = q < 3 ? 0 : (q < 5 ? 1 : 2);
          const int p = q < 3 ? q : (q < 5 ? q - 3 : 0);
          const uint64_t da = smem_desc_sw128(sa + a * A_BYTES + kk * 32);
          const uint64_t db = smem_desc_sw128(sa + NA * A_BYTES + p * B_BYTES + kk * 32);
          const uint32_t accum = (kb | kk | q) != 0;
          asm volatile(
              "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(kIdesc), "r"(accum)
              : "memory");
        }
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       cta_smem_addr(&empty[s]))
                   : "memory");
    }
    // completion of every MMA issued above
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     cta_smem_addr(&done))
                 : "memory");
  }
  __syncwarp();
  // epilogue: warp w owns accumulator lanes 32w..32w+31 (output rows m0 + 32w + lane)
  bool ok = mbar_wait_bounded(&done, 0u, kUmmaWait);
  if (!ok && lane == 0) atomicOr(status, STATUS_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok && !abort_flag);   // tcgen05.ld is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const int64_t row = m0 + warp * 32 + lane;
  if (ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < UN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) C[row * ldc + col] = __uint_as_float(v[j]) * (col_scale ? col_scale[col] : 1.0f);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UN) : "memory");
  }
}

// ------------------------------------------------------------------ range sketch Y = X^T Pi
// The first Krylov block of Alg. 2, Y = X^T Pi (d x k), for bfloat16 X: a contraction over the n
// rows.  D[c][j] = sum_i X[i][c] Pi[i][j]: the MMA's M dimension is 128 columns c of X, its K
// dimension the rows i and its N dimension the k columns of Pi.  X tiles arrive by TMA as they
// are stored (rows of 64 columns, 128-byte swizzle), which makes A the MN-major operand; Pi is
// read from its transposed bfloat16 copy Pi^T (k x n), which makes B K-major.  One CTA covers
// NT tiles of 128 columns of X and a contiguous range of rows (split K), 128 threads: warp 0
// lane 0 produces (TMA, ring of stages holding NT x 2 X boxes and one Pi^T box), warp 1 lane 0
// issues tcgen05.mma (M = 128, N = kp, K = 16) into NT tensor-memory accumulators, and all four
// warps read their 32 lanes (columns c) at the end and write the CTA's partial d x k block;
// sketch_reduce_kernel adds the partials of the row ranges in order.  Bounded waits.
constexpr int SK_ROWS = 64;                                   // rows of X per stage (K chunk)
constexpr uint32_t SK_XBOX = SK_ROWS * 128;                   // one 64 x 64 bfloat16 box of X
template <int NT> __host__ __device__ constexpr uint32_t sk_stage_bytes(int kp) {
  return (uint32_t)NT * 2 * SK_XBOX + (uint32_t)kp * 128;
}

// instruction descriptor: f32 accumulate, bf16 A and B, A MN-major (bit 15), B K-major, N, M = 128
__host__ __device__ constexpr uint32_t sk_idesc(int kp) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(kp >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

// MN-major, 128-byte swizzle: rows of the tile are K (64 elements of M or N each, 128 bytes), 8-row
// groups 1024 bytes apart (stride dimension), the two 64-wide halves of M = 128 `half` bytes apart
// (leading dimension)
__device__ __forceinline__ uint64_t smem_desc_mn_sw128(uint32_t saddr, uint32_t half) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((half >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <int NT>
__global__ void __launch_bounds__(128, 1) umma_sketch_kernel(const __grid_constant__ CUtensorMap tmX,
                                                             const __grid_constant__ CUtensorMap tmP, int64_t n,
                                                             int64_t d, int k, int kp, int stages,
                                                             int64_t chunks_per_cta, float* __restrict__ part,
                                                             int* status) {
  extern __shared__ unsigned char sk_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sk_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[4], empty[4], done;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  const uint32_t stage_bytes = sk_stage_bytes<NT>(kp);
  const uint32_t idesc = sk_idesc(kp);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.x * (NT * UM);
  const int64_t nchunks = (n + SK_ROWS - 1) / SK_ROWS;
  const int64_t q0 = (int64_t)blockIdx.y * chunks_per_cta;
  const int64_t q1 = min64(nchunks, q0 + chunks_per_cta);
  const int KB = (int)max64(0, q1 - q0);
  uint32_t tcols = 32;
  while (tcols < (uint32_t)(NT * kp)) tcols <<= 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init_cta(&full[s], 1);
      mbar_init_cta(&empty[s], 1);
    }
    mbar_init_cta(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cta_smem_addr(&tmem_holder)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;

  if (threadIdx.x == 0) {   // producer
    int issued_last[4] = {-1, -1, -1, -1};
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % stages, u = kb / stages;
      if (u >= 1 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kUmmaWait)) {
        atomicOr(status, STATUS_TIMEOUT);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      unsigned char* st = base + (size_t)s * stage_bytes;
      const int row = (int)((q0 + kb) * SK_ROWS);
      mbar_expect_tx_cta(&full[s], stage_bytes);
      for (int h = 0; h < NT * 2; ++h)   // boxes of 64 columns: tile t = h / 2, half h % 2
        tma_load_2d(st + h * SK_XBOX, &tmX, (int)(c0 + 64 * h), row, &full[s]);
      tma_load_2d(st + NT * 2 * SK_XBOX, &tmP, row, 0, &full[s]);
      issued_last[s] = u;
    }
    for (int s = 0; s < stages; ++s)
      if (issued_last[s] >= 0 && !mbar_wait_bounded(&full[s], (uint32_t)(issued_last[s] & 1), kUmmaWait))
        atomicOr(status, STATUS_TIMEOUT);
  } else if (threadIdx.x == 32) {   // MMA issuer
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % stages, u = kb / stages;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(u & 1), kUmmaWait)) {
        atomicOr(status, STATUS_TIMEOUT);
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = cta_smem_addr(base + (size_t)s * stage_bytes);
      const uint32_t sb = sa + NT * 2 * SK_XBOX;
#pragma unroll
      for (int kk = 0; kk < SK_ROWS / 16; ++kk) {
        const uint64_t db = smem_desc_sw128(sb + kk * 32);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          // 16 rows of the tile: 16 x 128 bytes into its first 64-column box; the second box is
          // SK_XBOX bytes further on
          const uint64_t da = smem_desc_mn_sw128(sa + t * 2 * SK_XBOX + kk * 16 * 128, SK_XBOX);
          const uint32_t accum = (kb | kk) != 0;
          asm volatile(
              "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem + (uint32_t)(t * kp)),
              "l"(da), "l"(db), "r"(idesc), "r"(accum)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       cta_smem_addr(&empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     cta_smem_addr(&done))
                 : "memory");
  }
  __syncwarp();
  // epilogue: warp w owns accumulator lanes 32w..32w+31, i.e. columns c0 + 128 t + 32 w + lane of X
  bool ok = KB == 0 || mbar_wait_bounded(&done, 0u, kUmmaWait);
  if (!ok && lane == 0) atomicOr(status, STATUS_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok && !abort_flag);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  float* pout = part + (int64_t)blockIdx.y * d * k;
  for (int t = 0; t < NT; ++t) {
    const int64_t c = c0 + (int64_t)t * UM + warp * 32 + lane;
    for (int j0 = 0; j0 < kp; j0 += 32) {
      uint32_t v[32];
      if (ok && KB > 0) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * kp + j0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0u;   // an empty row range contributes zeros
      }
      if (c < d) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j0 + j < k) pout[c * k + j0 + j] = __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

// Y[e] = sum over the row ranges r = 0..R-1 of part[r][e], added in increasing r
__global__ void sketch_reduce_kernel(const float* __restrict__ part, int R, int64_t count, float* __restrict__ Y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int r = 0; r < R; ++r) s += part[(int64_t)r * count + e];
    Y[e] = s;
  }
}

// ------------------------------------------------------------------ block preparation
// R = (I + eta K L)^{-1} K and c = -eta R (j . h) of one block of 64 inner steps (the blocked form
// of the inner loop of Alg. 1; K = diag(kappa) the importance weights of the sampled rows, L the
// strictly lower part of their Gram matrix G, h_l = mu^T z_l) for bfloat16 components.  The Gram
// matrix is a dense contraction over d: the CTA gathers the 64 sampled rows chunk by chunk (64
// columns, 128 bytes per row) into a 128-row tile in the 128-byte-swizzled K-major layout with
// 16-byte cp.async copies, rows 64..66 hold mu split into three bfloat16 parts (mu = m0 + m1 + m2
// to about 2^-24 relative), rows 67..127 are zero, and one thread issues tcgen05.mma (M = 128,
// N = 64: D = tile x rows 0..63^T, FP32 accumulation in tensor memory).  Products of bfloat16
// values are exact in FP32, so G matches the CUDA-core Gram matrix up to summation order.  After
// the last chunk warps 0-1 read G (accumulator lanes 0..63) and warp 2 the mu rows (lanes 64..66)
// into shared memory; then each of the 64 threads of warps 0-1 forward-substitutes one column of
// R (r_l = kappa_l (delta_lc - eta sum_{l'<l} G_ll' r_l')) in registers, and warp 2 the vector
// R (j . h) the same way (right-hand side kappa_l l h_l), with no block-wide barrier inside.
constexpr int PST = 3;                       // ring stages (64 columns each)
constexpr uint32_t P_STAGE = 128 * 128;      // 128 rows x 128 bytes
constexpr int GLD = 68;                      // Gram row stride in floats (16-byte rows)
constexpr uint32_t kPrepIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(cta_smem_addr(smem)), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}

// r_l = kap_l (rhs_l - et sum_{l' < l} G[l][l'] r_l') for l = 0..63; rhs = e_c for c >= 0, else v
__device__ __forceinline__ void block_fwd_subst(const float* __restrict__ G, const float* __restrict__ kap,
                                                const float* __restrict__ v, int c, float et, float (&r)[64]) {
#pragma unroll
  for (int l = 0; l < 64; ++l) {
    const float* Gl = G + l * GLD;
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
    for (int q = 0; q < l / 4; ++q) {
      const float4 g = *reinterpret_cast<const float4*>(Gl + 4 * q);
      s0 = fmaf(g.x, r[4 * q], s0);
      s1 = fmaf(g.y, r[4 * q + 1], s1);
      s2 = fmaf(g.z, r[4 * q + 2], s2);
      s3 = fmaf(g.w, r[4 * q + 3], s3);
    }
#pragma unroll
    for (int e = (l / 4) * 4; e < l; ++e) s0 = fmaf(Gl[e], r[e], s0);
    const float s = (s0 + s1) + (s2 + s3);
    const float rhs = c >= 0 ? (l == c ? 1.0f : 0.0f) : v[l];
    r[l] = kap[l] * fmaf(-et, s, rhs);
  }
}

// Grid: one CTA per block of steps.  jobs == nullptr: every CTA belongs to `one`; otherwise CTA g
// belongs to job j with blk_off[j] <= g < blk_off[j + 1].
__global__ void __launch_bounds__(128, 4) umma_prep_kernel(const __grid_constant__ ChainJob<__nv_bfloat16, float> one,
                                                           const ChainJob<__nv_bfloat16, float>* __restrict__ jobs,
                                                           const int64_t* __restrict__ blk_off, int nj, int* status) {
  extern __shared__ unsigned char up_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(up_raw) + 1023) & ~uintptr_t(1023));
  float* G = reinterpret_cast<float*>(base);   // [64][GLD], over the ring once every MMA has completed
  __shared__ uint64_t empty[PST], done;
  __shared__ uint32_t tmem_holder;
  __shared__ float kap[64], vv[64], hpart[3][64];
  __shared__ int64_t rowid[64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int64_t b = blockIdx.x;
  const ChainJob<__nv_bfloat16, float>* Jp = &one;
  if (jobs) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (blk_off[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    Jp = jobs + lo;
    b -= blk_off[lo];
  }
  const __nv_bfloat16* __restrict__ Z = Jp->Z;
  const int64_t N = Jp->N, ld = Jp->ld, d = Jp->d, n = Jp->n, m = Jp->m;
  const float* __restrict__ mu = Jp->mu;
  const float et = (float)Jp->eta;
  const int64_t t0 = b * 64;
  const int Bb = (int)min64(64, m - t0);
  if (tid < 64) {
    if (tid < Bb) {
      const uint32_t i = min(Jp->idx[t0 + tid], (uint32_t)(N - 1));   // indices are < N by contract
      rowid[tid] = i;
      const float Nn = (float)((double)N / (double)n), lN = (float)(Jp->lam * (double)N);
      kap[tid] = (i < (uint64_t)n ? Nn : lN) * Jp->inv_nq[t0 + tid];
    } else {
      rowid[tid] = -1;
      kap[tid] = 0.0f;
    }
  }
  if (tid == 0) {
    for (int s = 0; s < PST; ++s) mbar_init_cta(&empty[s], 1);
    mbar_init_cta(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cta_smem_addr(&tmem_holder)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // rows 64..127 of every stage start at zero (rows 64..66 take mu's parts per chunk)
  for (int e = tid; e < PST * 64 * 8; e += 128) {
    const int s = e / 512, r = 64 + (e % 512) / 8, q = e % 8;
    *reinterpret_cast<uint4*>(base + s * P_STAGE + r * 128 + q * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;
  const int nch = (int)((d + 63) / 64);
  auto fill = [&](int kc, int s) {
    unsigned char* st = base + s * P_STAGE;
    const int64_t c0 = (int64_t)kc * 64;
    for (int e = tid; e < 64 * 8; e += 128) {
      const int r = e >> 3, q = e & 7;
      const int64_t col = c0 + q * 8;
      const int64_t rid = rowid[r];
      const void* src = Z;
      int bytes = 0;
      if (rid >= 0 && col < d) {
        src = Z + rid * ld + col;
        bytes = (int)min64(8, d - col) * 2;
      }
      cp_async16_zfill(st + r * 128 + ((q ^ (r & 7)) << 4), src, bytes);
    }
    if (mu && tid < 8) {
      const int q = tid;
      const int64_t col = c0 + q * 8;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = col + i < d ? mu[col + i] : 0.0f;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __nv_bfloat16 lo = __float2bfloat16_rn(v[2 * i]), hi = __float2bfloat16_rn(v[2 * i + 1]);
          v[2 * i] -= __bfloat162float(lo);
          v[2 * i + 1] -= __bfloat162float(hi);
          w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        const int r = 64 + p;
        *reinterpret_cast<uint4*>(st + r * 128 + ((q ^ (r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int kc = 0; kc < PST - 1; ++kc) {
    if (kc < nch) fill(kc, kc);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int kc = 0; kc < nch; ++kc) {
    const int kn = kc + PST - 1;
    if (kn < nch) {
      const int s = kn % PST;
      // the stage was last read by the MMAs of chunk kn - PST
      if (kn >= PST && !mbar_wait_bounded(&empty[s], (uint32_t)(((kn - PST) / PST) & 1), kUmmaWait))
        atomicOr(status, STATUS_TIMEOUT);
      fill(kn, s);
    } else {
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PST - 1) : "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // generic-proxy writes -> tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = cta_smem_addr(base + (kc % PST) * P_STAGE);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = smem_desc_sw128(sa + kk * 32);
        const uint32_t accum = (kc | kk) != 0;
        asm volatile(
            "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
            "l"(da), "l"(da), "r"(kPrepIdesc), "r"(accum)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       cta_smem_addr(&empty[kc % PST]))
                   : "memory");
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (tid == 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     cta_smem_addr(&done))
                 : "memory");
  __syncwarp();
  bool ok = mbar_wait_bounded(&done, 0u, kUmmaWait);
  if (!ok && lane == 0) atomicOr(status, STATUS_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();   // every warp is past its wait before G overwrites the ring
  if (warp < 3 && ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (warp < 2) {
        float* gr = G + (warp * 32 + lane) * GLD + c0;
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4*>(gr + j) =
              make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                          __uint_as_float(v[j + 3]));
      } else if (lane < 3) {
#pragma unroll
        for (int j = 0; j < 32; ++j) hpart[lane][c0 + j] = __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(64) : "memory");
  }
  if (tid < 64) vv[tid] = mu ? (float)tid * ((hpart[1][tid] + hpart[2][tid]) + hpart[0][tid]) : 0.0f;
  __syncthreads();
  if (warp < 3) {
    float r[64];
    block_fwd_subst(G, kap, vv, warp < 2 ? tid : -1, et, r);
    if (warp < 2) {   // column tid of R is row tid of Rt
      float* out = Jp->Rt + (b * 64 + tid) * 64;
#pragma unroll
      for (int j = 0; j < 64; j += 4) *reinterpret_cast<float4*>(out + j) = make_float4(r[j], r[j + 1], r[j + 2], r[j + 3]);
    } else if (lane == 0) {
      float* out = Jp->cvec + b * 64;
#pragma unroll
      for (int j = 0; j < 64; ++j) out[j] = (mu && j < Bb) ? -et * r[j] : 0.0f;
    }
  }
}

// ------------------------------------------------------------------ components Z = X - P V^T
// The data rows of the preconditioned components (Eq. (11)): Z = X M = X - P V^T with P =
// X V diag(a) (n x k) and V (d x k), for bfloat16 X and Z.  P and V are split into three
// bfloat16 parts each (P = P0 + P1 + P2, V likewise) and the six products P_a V_b^T with
// a + b <= 2 accumulate in FP32 in tensor memory, which keeps the product to about 2^-24
// relative (the dropped terms are below 2^-27).
//
// One CTA per 128-row block, persistent over the 64-column output tiles, 192 threads: warp 0
// lane 0 loads (TMA, 128-byte swizzle) the block's P parts once and streams the V parts in K
// chunks of 64 through a ring of NB entries, and the 128 x 64 tiles of X into two buffers; warp 1
// lane 0 issues tcgen05.mma (M = 128, N = 64, K = 16) into one of two tensor-memory accumulators,
// so the next tile's products run while warps 2-5 drain the previous one: each of those threads
// owns one row of the tile, reads its 64 accumulator columns (tcgen05.ld) and its row of X,
// writes the bfloat16 rounding of X - P V^T over that row in place (same swizzled layout), and one
// thread stores the tile with a TMA bulk store, after which the buffer takes the next X tile.
// Every wait is bounded (status flag on timeout).
constexpr int RT_ROWS = 128, RT_COLS = 64;
constexpr uint32_t RT_A_TILE = 128 * 128;   // 128 rows x 64 bfloat16
constexpr uint32_t RT_B_TILE = 64 * 128;    // 64 rows x 64 bfloat16
constexpr uint32_t RT_X_TILE = 128 * 128;   // 128 rows x 64 bfloat16

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(cta_smem_addr(src))
               : "memory");
}

// XP = 1: bfloat16 X tiles; XP = 3: float X given as its three bfloat16 parts (rows a n .. a n + n - 1
// of the parts' map), summed in float in the epilogue (K chunks: KC = 1 only, two ring entries).
// NP = 3: P and V in three bfloat16 parts, six products (about 2^-24 relative); NP = 2 (k up to 256,
// where three parts of P no longer fit beside the ring): two parts each and the three products with
// a + b <= 1, about 2^-16 relative to |P| |V|^T, below half an ulp of the bfloat16 result for the
// data the components are formed from (|P V^T| within about 2^7 of |Z|).
template <int KC, int XP = 1, int NP = 3> __host__ __device__ constexpr int resid_ring() {
  return XP == 3 ? 2 : (KC == 1 ? 4 : 3);
}
template <int KC, int XP = 1, int NP = 3>
constexpr size_t resid_smem_bytes() {
  return (size_t)NP * KC * RT_A_TILE + (size_t)resid_ring<KC, XP, NP>() * NP * RT_B_TILE +
         2 * (size_t)XP * RT_X_TILE + 1024;
}

template <int KC, int XP = 1, int NP = 3>
__global__ void __launch_bounds__(192, 1) umma_resid_kernel(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB,
                                                            const __grid_constant__ CUtensorMap tmX,
                                                            const __grid_constant__ CUtensorMap tmZ, int64_t d,
                                                            int64_t np, int64_t dp, int64_t n_rows,
                                                            float* __restrict__ rowsq, int* status) {
  constexpr int NB = resid_ring<KC, XP, NP>();
  constexpr uint32_t A_BYTES = NP * KC * RT_A_TILE;
  constexpr uint32_t B_ENTRY = NP * RT_B_TILE;   // the NP V parts of one K chunk
  extern __shared__ unsigned char rt_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(rt_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* As = base;
  unsigned char* Bs = As + A_BYTES;
  unsigned char* XZ = Bs + NB * B_ENTRY;
  __shared__ uint64_t a_full, b_full[NB], b_empty[NB], x_full[2], x_empty[2], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_holder;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * RT_ROWS;
  const int ntiles = (int)((d + RT_COLS - 1) / RT_COLS);
  if (threadIdx.x == 0) {
    mbar_init_cta(&a_full, 1);
    for (int s = 0; s < NB; ++s) {
      mbar_init_cta(&b_full[s], 1);
      mbar_init_cta(&b_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init_cta(&x_full[s], 1);
      mbar_init_cta(&x_empty[s], 1);
      mbar_init_cta(&acc_full[s], 1);
      mbar_init_cta(&acc_empty[s], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cta_smem_addr(&tmem_holder)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;

  if (warp == 0) {
    if (lane == 0) {   // producer
      mbar_expect_tx_cta(&a_full, A_BYTES);
      for (int pa = 0; pa < NP; ++pa)
        for (int kc = 0; kc < KC; ++kc)
          tma_load_2d(As + (pa * KC + kc) * RT_A_TILE, &tmA, kc * 64, (int)(pa * np) + row0, &a_full);
      for (int t = 0; t < ntiles; ++t) {
        for (int kc = 0; kc < KC; ++kc) {
          const int c = t * KC + kc, e = c % NB, u = c / NB;
          if (u >= 1 && !mbar_wait_bounded(&b_empty[e], (uint32_t)((u - 1) & 1), kUmmaWait))
            atomicOr(status, STATUS_TIMEOUT);
          mbar_expect_tx_cta(&b_full[e], B_ENTRY);
          for (int pb = 0; pb < NP; ++pb)
            tma_load_2d(Bs + e * B_ENTRY + pb * RT_B_TILE, &tmB, kc * 64, (int)(pb * dp) + t * RT_COLS, &b_full[e]);
        }
        const int sx = t & 1, ux = t >> 1;
        if (ux >= 1 && !mbar_wait_bounded(&x_empty[sx], (uint32_t)((ux - 1) & 1), kUmmaWait))
          atomicOr(status, STATUS_TIMEOUT);
        mbar_expect_tx_cta(&x_full[sx], XP * RT_X_TILE);
        for (int a = 0; a < XP; ++a)
          tma_load_2d(XZ + (sx * XP + a) * RT_X_TILE, &tmX, t * RT_COLS, (int)(a * n_rows) + row0, &x_full[sx]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      if (!mbar_wait_bounded(&a_full, 0u, kUmmaWait)) atomicOr(status, STATUS_TIMEOUT);
      const uint32_t sa = cta_smem_addr(As);
      for (int t = 0; t < ntiles; ++t) {
        const int ab = t & 1, ua = t >> 1;
        if (ua >= 1 && !mbar_wait_bounded(&acc_empty[ab], (uint32_t)((ua - 1) & 1), kUmmaWait))
          atomicOr(status, STATUS_TIMEOUT);
        const uint32_t dt = tmem + (uint32_t)(ab * RT_COLS);
        for (int kc = 0; kc < KC; ++kc) {
          const int c = t * KC + kc, e = c % NB, u = c / NB;
          if (!mbar_wait_bounded(&b_full[e], (uint32_t)(u & 1), kUmmaWait)) atomicOr(status, STATUS_TIMEOUT);
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t sbb = cta_smem_addr(Bs + e * B_ENTRY);
          constexpr int NPROD = NP == 3 ? 6 : 3;
#pragma unroll
          for (int q = 0; q < NPROD; ++q) {
            // NP = 3: (0,0) (0,1) (0,2) (1,0) (1,1) (2,0); NP = 2: (0,0) (0,1) (1,0)
            const int pa = NP == 3 ? (q < 3 ? 0 : (q < 5 ? 1 : 2)) : (q < 2 ? 0 : 1);
            const int pb = NP == 3 ? (q < 3 ? q : (q < 5 ? q - 3 : 0)) : (q < 2 ? q : 0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t da = smem_desc_sw128(sa + (pa * KC + kc) * RT_A_TILE + kk * 32);
              const uint64_t db = smem_desc_sw128(sbb + pb * RT_B_TILE + kk * 32);
              const uint32_t accum = (kc | q | kk) != 0;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                  "l"(da), "l"(db), "r"(kPrepIdesc), "r"(accum)
                  : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           cta_smem_addr(&b_empty[e]))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         cta_smem_addr(&acc_full[ab]))
                     : "memory");
      }
    }
  } else {   // epilogue: warps 2..5, thread = row r of the tile (tensor-memory lane r)
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const bool lead = warp == 2 && lane == 0;
    float sq = 0.0f;   // squared norm of this row of the stored (rounded) components
    for (int t = 0; t < ntiles; ++t) {
      const int ab = t & 1, ua = t >> 1;
      bool ok = mbar_wait_bounded(&acc_full[ab], (uint32_t)(ua & 1), kUmmaWait);
      ok = mbar_wait_bounded(&x_full[ab], (uint32_t)(ua & 1), kUmmaWait) && ok;
      if (!ok) atomicOr(status, STATUS_TIMEOUT);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      uint32_t v[64];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * RT_COLS + 32 * h);
        uint32_t* w = v + 32 * h;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
              "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15]),
              "=r"(w[16]), "=r"(w[17]), "=r"(w[18]), "=r"(w[19]), "=r"(w[20]), "=r"(w[21]), "=r"(w[22]), "=r"(w[23]),
              "=r"(w[24]), "=r"(w[25]), "=r"(w[26]), "=r"(w[27]), "=r"(w[28]), "=r"(w[29]), "=r"(w[30]), "=r"(w[31])
            : "r"(taddr)
            : "memory");
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&acc_empty[ab]);
      unsigned char* xr = XZ + ab * XP * RT_X_TILE + r * 128;
#pragma unroll
      for (int u8 = 0; u8 < 8; ++u8) {
        const int off = (u8 ^ (r & 7)) << 4;
        float xv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) xv[e] = 0.0f;
        // float X: x = x0 + x1 + x2 (the first two parts add exactly), summed from the smallest part
#pragma unroll
        for (int a = XP - 1; a >= 0; --a) {
          const uint4 xw = *reinterpret_cast<const uint4*>(xr + a * RT_X_TILE + off);
          const uint32_t xs4[4] = {xw.x, xw.y, xw.z, xw.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xv[2 * e] += __uint_as_float(xs4[e] << 16);
            xv[2 * e + 1] += __uint_as_float(xs4[e] & 0xFFFF0000u);
          }
        }
        uint32_t zw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat16 z0 = __float2bfloat16_rn(xv[2 * e] - __uint_as_float(v[8 * u8 + 2 * e]));
          const __nv_bfloat16 z1 = __float2bfloat16_rn(xv[2 * e + 1] - __uint_as_float(v[8 * u8 + 2 * e + 1]));
          zw[e] = (uint32_t)__bfloat16_as_ushort(z0) | ((uint32_t)__bfloat16_as_ushort(z1) << 16);
          const float f0 = __bfloat162float(z0), f1 = __bfloat162float(z1);
          sq = fmaf(f0, f0, sq);
          sq = fmaf(f1, f1, sq);
        }
        *reinterpret_cast<uint4*>(xr + off) = make_uint4(zw[0], zw[1], zw[2], zw[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("bar.sync 1, 128;\n" ::: "memory");
      if (lead) {
        tma_store_2d(&tmZ, XZ + ab * XP * RT_X_TILE, t * RT_COLS, row0);
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        // the buffer takes the next X tile once the store has read it
        asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
        mbar_arrive_cta(&x_empty[ab]);
      }
    }
    if (lead) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    // columns beyond d entered as zeros (TMA fills out-of-range X with zeros, and the MMA products
    // there vanish), so sq is the full squared norm of the stored row
    if (rowsq && row0 + r < n_rows) rowsq[row0 + r] = sq;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128) : "memory");
  }
}

// Float rows (16-byte aligned, row stride lds) -> three bfloat16 parts (3 x rows x kp, kp a multiple
// of 8), part p = bf16(x - part 0 - .. - part p-1), zero beyond k; 8 elements per thread
__global__ void split3_x_kernel(const float* __restrict__ src, int64_t rows, int64_t k, int64_t lds, int64_t kp,
                                __nv_bfloat16* __restrict__ out) {
  const int64_t units = kp / 8, total = rows * units;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / units, c0 = (e % units) * 8;
    float v[8];
    const float* r = src + i * lds + c0;
    if (c0 + 8 <= k) {
      const float4 a = *reinterpret_cast<const float4*>(r), b = *reinterpret_cast<const float4*>(r + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = c0 + q < k ? r[q] : 0.0f;
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 lo = __float2bfloat16_rn(v[2 * q]), hi = __float2bfloat16_rn(v[2 * q + 1]);
        v[2 * q] -= __bfloat162float(lo);
        v[2 * q + 1] -= __bfloat162float(hi);
        w[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      }
      *reinterpret_cast<uint4*>(out + (int64_t)p * rows * kp + i * kp + c0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// src (rows x k float, row stride lds) -> out (3 x rows_pad x kp bfloat16): part p holds
// bf16(src - part 0 - .. - part p-1), zero beyond rows and k
__global__ void split3_rows_kernel(const float* __restrict__ src, int64_t rows, int k, int64_t lds, int64_t rows_pad,
                                   int kp, __nv_bfloat16* __restrict__ out) {
  const int64_t total = rows_pad * kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kp;
    const int c = (int)(e % kp);
    float r = (i < rows && c < k) ? src[i * lds + c] : 0.0f;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const __nv_bfloat16 h = __float2bfloat16_rn(r);
      out[(int64_t)p * total + e] = h;
      r -= __bfloat162float(h);
    }
  }
}

// W (K x N float, row-major) -> parts (NSPLIT x kp x ldp bfloat16): part p row j = column j of
// W_p, W = W0 + W1 + W2 with W_{p} = bf16(W - W_0 - .. - W_{p-1}); rows j >= N are zero
__global__ void split_transpose_kernel(const float* __restrict__ W, int K, int N, int kp, int ldp,
                                       __nv_bfloat16* __restrict__ out) {
  const int64_t total = (int64_t)kp * ldp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ldp), c = (int)(e % ldp);
    float r = (j < N && c < K) ? W[(int64_t)c * N + j] : 0.0f;
#pragma unroll
    for (int p = 0; p < NSPLIT; ++p) {
      const __nv_bfloat16 h = __float2bfloat16_rn(r);
      out[(int64_t)p * total + e] = h;
      r -= __bfloat162float(h);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

int make_map(CUtensorMap* map, const void* ptr, int64_t inner, int64_t rows, int64_t ld_elems, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return rs_fail(RS_EUNSUPPORTED, "tensor-map encoder unavailable");
  cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld_elems * 2};
  cuuint32_t box[2] = {(cuuint32_t)UK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), gdim, gstride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return rs_fail(RS_EUNSUPPORTED, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return RS_OK;
}

}  // namespace

// The tensor-core path is on unless RS_UMMA=0.
bool umma_enabled() {
  const char* env = std::getenv("RS_UMMA");
  return !(env && env[0] == '0');
}

// R and c of every block of steps of the given bfloat16 chains on tensor cores (on unless RS_UMMA=0
// or RS_UMMA_PREP=0).  RS_EUNSUPPORTED when it cannot run: the caller uses the CUDA-core path.
int umma_prep(rs_ctx* ctx, const ChainJob<__nv_bfloat16, float>& one, const ChainJob<__nv_bfloat16, float>* jobs,
              const int64_t* blk_off, int nj, int64_t total_blocks) {
  if (!umma_enabled()) return RS_EUNSUPPORTED;
  const char* env = std::getenv("RS_UMMA_PREP");
  if (env && env[0] == '0') return RS_EUNSUPPORTED;
  if (total_blocks < 1) return RS_OK;
  if (total_blocks > 0x7FFFFFFF) return RS_EUNSUPPORTED;
  if (!jobs && ((reinterpret_cast<uintptr_t>(one.Z) & 15) || (one.ld & 7) || one.n < 1)) return RS_EUNSUPPORTED;
  const size_t shm = (size_t)PST * P_STAGE + 1024;
  RS_CUDA_TRY(cudaFuncSetAttribute(umma_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  umma_prep_kernel<<<(unsigned)total_blocks, 128, shm, ctx->stream>>>(one, jobs, blk_off, nj, ctx->d_status);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

// Z (bfloat16 rows, n x d) = X - P V^T for bfloat16 X (k <= 128) or float X whose bfloat16 parts
// this call has formed (k <= 64), P (n x k float, row stride k), V (d x k float, row stride k), on
// tensor cores; rowsq (optional, n floats) receives the squared norms of the stored rows.  RS_EUNSUPPORTED when the tensor path is off or
// cannot run (the caller uses the CUDA-core product).
int umma_resid(rs_ctx* ctx, const rs_matrix* X, const float* P, const float* V, int64_t k, rs_matrix* Z,
               float* rowsq) {
  if (!umma_enabled() || !encode_fn()) return RS_EUNSUPPORTED;
  const char* env = std::getenv("RS_UMMA_RESID");
  if (env && env[0] == '0') return RS_EUNSUPPORTED;
  const int64_t n = X->n, d = X->d;
  if (k < 1 || k > 256 || n < 1 || d < 1 || n > 0x7FFFFF00LL / 3 || d > 0x7FFFFF00LL / 3) return RS_EUNSUPPORTED;
  const int kp = k <= 64 ? 64 : (k <= 128 ? 128 : 256);
  // float X: only with the three bfloat16 parts of this X formed earlier in the same call (the
  // tensor-core X V product leaves them in SCR_XPART), and k <= 64
  const bool f32 = X->dtype == RS_F32;
  const int64_t ldx = (d + 7) / 8 * 8;
  if (f32) {
    const bool cached = ctx->xp_gen == ctx->call_gen && ctx->xp_src == X->data && ctx->xp_n == n &&
                        ctx->xp_d == d && ctx->xp_ld == X->ld;
    if (!cached || kp != 64) return RS_EUNSUPPORTED;
  } else if (X->dtype != RS_BF16) {
    return RS_EUNSUPPORTED;
  }
  const int64_t np = (n + RT_ROWS - 1) / RT_ROWS * RT_ROWS, dp = (d + RT_COLS - 1) / RT_COLS * RT_COLS;
  __nv_bfloat16* parts = static_cast<__nv_bfloat16*>(
      rs_scratch(ctx, SCR_RPART, (size_t)3 * (np + dp) * kp * sizeof(__nv_bfloat16)));
  if (!parts) return RS_ENOMEM;
  __nv_bfloat16* vparts = parts + (size_t)3 * np * kp;
  const int sb = ctx->num_sms * 8;
  split3_rows_kernel<<<(unsigned)std::min<int64_t>((np * kp + 255) / 256, sb), 256, 0, ctx->stream>>>(
      P, n, (int)k, k, np, kp, parts);
  RS_LAUNCH_CHECK(ctx);
  split3_rows_kernel<<<(unsigned)std::min<int64_t>((dp * kp + 255) / 256, sb), 256, 0, ctx->stream>>>(
      V, d, (int)k, k, dp, kp, vparts);
  RS_LAUNCH_CHECK(ctx);
  CUtensorMap mA, mB, mX, mZ;
  RS_TRY(make_map(&mA, parts, kp, 3 * np, kp, RT_ROWS));
  RS_TRY(make_map(&mB, vparts, kp, 3 * dp, kp, RT_COLS));
  if (f32) RS_TRY(make_map(&mX, ctx->slots[SCR_XPART].ptr, d, 3 * n, ldx, RT_ROWS));
  else RS_TRY(make_map(&mX, X->data, d, n, X->ld, RT_ROWS));
  RS_TRY(make_map(&mZ, Z->data, d, n, Z->ld, RT_ROWS));
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  const unsigned grid = (unsigned)(np / RT_ROWS);
#define RS_RESID(KC_, XP_, NP_)                                                                               \
  do {                                                                                                        \
    constexpr size_t shm = resid_smem_bytes<KC_, XP_, NP_>();                                                 \
    RS_CUDA_TRY(cudaFuncSetAttribute(umma_resid_kernel<KC_, XP_, NP_>,                                        \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));                 \
    umma_resid_kernel<KC_, XP_, NP_><<<grid, 192, shm, ctx->stream>>>(mA, mB, mX, mZ, d, np, dp, n, rowsq,    \
                                                                       ctx->d_status);                        \
  } while (0)
  if (f32) RS_RESID(1, 3, 3);
  else if (kp == 64) RS_RESID(1, 1, 3);
  else if (kp == 128) RS_RESID(2, 1, 3);
  else RS_RESID(4, 1, 2);
#undef RS_RESID
  RS_LAUNCH_CHECK(ctx);
  int st = 0;
  RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (st & STATUS_TIMEOUT) return rs_fail(RS_ETIMEOUT, "tensor-core components: a bounded wait gave up");
  return RS_OK;
}

// C (M x N, float, ldc) = X (bfloat16 rows, M x K) W (K x N, float) diag(col_scale); N <= 256.
// RS_EUNSUPPORTED if the tensor-map encoder is unavailable (the caller then uses CUDA cores).
int umma_gemm_xw(rs_ctx* ctx, const rs_matrix* X, const float* W, int64_t N, const float* col_scale, float* C,
                 int64_t ldc, bool sync_check) {
  const int64_t M = X->n, K = X->d;
  if (N < 1 || N > 256 || K < 1) return RS_EUNSUPPORTED;
  if (X->dtype != RS_BF16 && X->dtype != RS_F32) return RS_EUNSUPPORTED;
  if (!encode_fn()) return RS_EUNSUPPORTED;
  const bool f32 = X->dtype == RS_F32;
  const int UN = N <= 64 ? 64 : 128;
  const int kp = (int)((N + UN - 1) / UN * UN);
  const int ldp = (int)((K + 7) / 8 * 8);        // 16-byte rows
  // float data: X = X0 + X1 + X2 in bfloat16 parts (about 2^-24 relative), at most 8 GB of parts
  const size_t xparts = f32 ? (size_t)NSPLIT * M * ldp * sizeof(__nv_bfloat16) : 0;
  if (f32 && (xparts > ((size_t)8 << 30) || 3 * M > 0x7FFFFF00LL)) return RS_EUNSUPPORTED;
  const size_t wparts = (size_t)NSPLIT * kp * ldp * sizeof(__nv_bfloat16);
  __nv_bfloat16* parts = static_cast<__nv_bfloat16*>(rs_scratch(ctx, SCR_UMMA, wparts));
  if (!parts) return RS_ENOMEM;
  split_transpose_kernel<<<(unsigned)std::min<int64_t>(((int64_t)kp * ldp + 255) / 256, ctx->num_sms * 8), 256, 0,
                           ctx->stream>>>(W, (int)K, (int)N, kp, ldp, parts);
  RS_LAUNCH_CHECK(ctx);
  CUtensorMap mx, mw;
  if (f32) {
    const bool cached = ctx->xp_gen == ctx->call_gen && ctx->xp_src == X->data && ctx->xp_n == M &&
                        ctx->xp_d == K && ctx->xp_ld == X->ld && ctx->slots[SCR_XPART].bytes >= xparts;
    __nv_bfloat16* xp = static_cast<__nv_bfloat16*>(rs_scratch(ctx, SCR_XPART, xparts));
    if (!xp) return RS_ENOMEM;
    if (!cached) {
      split3_x_kernel<<<(unsigned)std::min<int64_t>((M * (ldp / 8) + 255) / 256, ctx->num_sms * 8), 256, 0,
                        ctx->stream>>>(static_cast<const float*>(X->data), M, K, X->ld, ldp, xp);
      RS_LAUNCH_CHECK(ctx);
      ctx->xp_src = X->data;
      ctx->xp_n = M;
      ctx->xp_d = K;
      ctx->xp_ld = X->ld;
      ctx->xp_gen = ctx->call_gen;
    }
    RS_TRY(make_map(&mx, xp, K, 3 * M, ldp, UM));
  } else {
    RS_TRY(make_map(&mx, X->data, K, M, X->ld, UM));
  }
  RS_TRY(make_map(&mw, parts, K, (int64_t)NSPLIT * kp, ldp, UN));
  dim3 grid((unsigned)((M + UM - 1) / UM), (unsigned)(kp / UN));
  if ((M + UM - 1) / UM > 0x7FFFFFFF) return rs_fail(RS_EINVAL, "umma gemm: too many row tiles");
  if (sync_check) RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
#define RS_XW(NA_, UN_)                                                                                       \
  do {                                                                                                        \
    constexpr size_t shm = (size_t)xw_stages<NA_, UN_>() * xw_stage_bytes<NA_, UN_>() + 1024;                 \
    RS_CUDA_TRY(cudaFuncSetAttribute(umma_xw_kernel<NA_, UN_>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                     (int)shm));                                                              \
    umma_xw_kernel<NA_, UN_><<<grid, 128, shm, ctx->stream>>>(mx, mw, M, (int)K, (int)N, kp, col_scale, C, ldc, \
                                                               ctx->d_status);                                \
  } while (0)
  if (f32 && UN == 64) RS_XW(3, 64);
  else if (f32) RS_XW(3, 128);
  else if (UN == 64) RS_XW(1, 64);
  else RS_XW(1, 128);
#undef RS_XW
  RS_LAUNCH_CHECK(ctx);
  if (!sync_check) return RS_OK;   // inside a captured sequence: the caller reads the status word later
  int st = 0;
  RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (st & STATUS_TIMEOUT) return rs_fail(RS_ETIMEOUT, "tensor-core product: a bounded wait gave up");
  return RS_OK;
}

int gaussian_t_bf16_dispatch(rs_ctx* ctx, uint64_t seed, int64_t n, int64_t k, __nv_bfloat16* out, int64_t ld);

// Y (d x k float, row stride k) = X^T Pi for bfloat16 X on tensor cores, Pi the Gaussian test matrix
// of Alg. 2 rounded to bfloat16 (Pi^T formed once per call in scratch, k x n).  RS_EUNSUPPORTED when
// the tensor path is off or cannot run (the caller uses the CUDA-core sketch).
int umma_sketch(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t k, float* Y) {
  if (!umma_enabled() || !encode_fn()) return RS_EUNSUPPORTED;
  const char* env = std::getenv("RS_UMMA_SKETCH");
  if (env && env[0] == '0') return RS_EUNSUPPORTED;
  const int64_t n = X->n, d = X->d;
  if (X->dtype != RS_BF16 || k < 1 || k > 256 || n < 1 || d < 1 || n > 0x7FFFFF00LL || d > 0x7FFFFF00LL)
    return RS_EUNSUPPORTED;
  const int kp = (int)((k + 15) / 16 * 16);
  const int64_t ldp = (n + 7) / 8 * 8;                    // 16-byte rows of Pi^T
  __nv_bfloat16* PiT = static_cast<__nv_bfloat16*>(rs_scratch(ctx, SCR_OMEGA, (size_t)k * ldp * sizeof(__nv_bfloat16)));
  if (!PiT) return RS_ENOMEM;
  RS_TRY(gaussian_t_bf16_dispatch(ctx, seed, n, k, PiT, ldp));
  // NT column tiles per CTA (two when d allows, so each Pi^T tile feeds 256 columns), and enough
  // row ranges to fill the GPU once
  const int NT = d > UM ? 2 : 1;
  const int64_t dtiles = (d + NT * UM - 1) / (NT * UM);
  const int64_t nchunks = (n + SK_ROWS - 1) / SK_ROWS;
  int64_t R = std::max<int64_t>(1, std::min<int64_t>(nchunks, (ctx->num_sms + dtiles - 1) / dtiles));
  const int64_t per = (nchunks + R - 1) / R;
  R = (nchunks + per - 1) / per;
  if (R > 65535) return RS_EUNSUPPORTED;
  const uint32_t sb = NT == 2 ? sk_stage_bytes<2>(kp) : sk_stage_bytes<1>(kp);
  const int stages = (int)std::min<uint32_t>(4, (215u * 1024u) / sb);
  if (stages < 2) return RS_EUNSUPPORTED;
  float* part = static_cast<float*>(rs_scratch(ctx, SCR_SKPART, (size_t)R * d * k * sizeof(float)));
  if (!part) return RS_ENOMEM;
  CUtensorMap mx, mp;
  RS_TRY(make_map(&mx, X->data, d, n, X->ld, SK_ROWS));
  RS_TRY(make_map(&mp, PiT, n, k, ldp, (uint32_t)kp));
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  const size_t shm = (size_t)stages * sb + 1024;
  dim3 grid((unsigned)dtiles, (unsigned)R);
  if (NT == 2) {
    RS_CUDA_TRY(cudaFuncSetAttribute(umma_sketch_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    umma_sketch_kernel<2><<<grid, 128, shm, ctx->stream>>>(mx, mp, n, d, (int)k, kp, stages, per, part, ctx->d_status);
  } else {
    RS_CUDA_TRY(cudaFuncSetAttribute(umma_sketch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    umma_sketch_kernel<1><<<grid, 128, shm, ctx->stream>>>(mx, mp, n, d, (int)k, kp, stages, per, part, ctx->d_status);
  }
  RS_LAUNCH_CHECK(ctx);
  const int64_t count = d * k;
  sketch_reduce_kernel<<<(unsigned)std::min<int64_t>((count + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0,
                         ctx->stream>>>(part, (int)R, count, Y);
  RS_LAUNCH_CHECK(ctx);
  int st = 0;
  RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (st & STATUS_TIMEOUT) return rs_fail(RS_ETIMEOUT, "tensor-core range sketch: a bounded wait gave up");
  return RS_OK;
}
