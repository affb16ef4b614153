// The inner loop of Alg. 1 (m sequential variance-reduced steps of one epoch) on the GPU.
//
// Inside one block of B consecutive steps the recursion is, with delta = w - w_bar, z_j the
// component row sampled at step j of the block and kappa_j = gamma_{i_j} / (N q_{i_j}):
//   a_j              = kappa_j z_j^T delta_{before j}
//   delta_{after j}  = delta_{before j} - eta a_j z_j - eta mu
// Writing p_j = z_j^T delta_{t0} (delta at the block start) and h_j = z_j^T mu gives
//   a = R (p - eta (j h)),   R = (I + eta K L)^{-1} K,
// with L the strictly lower triangle of the block's Gram matrix Z_b Z_b^T and K = diag(kappa).
// R and c = -eta R (j h) depend only on the sampled rows and mu, so epoch_prep_kernel forms
// them for every block at once.  epoch_chain_kernel then runs the blocks in order on one
// thread-block cluster: per block, p = Z_b delta (one exchange of partial dot products through
// distributed shared memory), a = R p + c, and the rank-B update of delta and of the running
// sum of the iterates (for the epoch average).  Every iterate of the step-by-step recursion
// is represented exactly; only the rounding differs.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kBlk = kChainBlk;   // steps per block
constexpr int kCsMax = 16;   // largest cluster

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// sixteen FP8-e4m3 codes (one 16-byte load) widened to float and scaled
__device__ __forceinline__ void ld_widen(const __nv_fp8_e4m3* p, float* v, float sc) {
  const uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
  const __nv_fp8_e4m3* q = reinterpret_cast<const __nv_fp8_e4m3*>(&raw);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = static_cast<float>(q[k]) * sc;
}

// eight bfloat16 (one 16-byte load) widened to float: a bfloat16 is the upper half of a float
__device__ __forceinline__ void ld_widen8(const __nv_bfloat16* p, float* v) {
  const uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = __uint_as_float(w[k] << 16);
    v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
  }
}
__device__ __forceinline__ void ld_widen(const __nv_bfloat16* p, float* v, float) { ld_widen8(p, v); }

// ------------------------------------------------------------------ per-block preparation
// One thread block per block of steps.  Rows 0..B-1 of the staged tile are the sampled rows
// (zero beyond the last step), row B is mu, rows B+1..B+3 are zero.  Z is stored in S and
// widened to the compute type T while it is staged.  With LA (look-ahead) the rows of the next
// block follow as rows B+4..2B+3, and the block also writes the cross Gram matrix
// Kt[l][j] = z'_j . z_l (z' the next block's rows) and hn_j = z'_j . mu.
template <typename S, typename T, bool LA = false>
__device__ __forceinline__ void prep_body(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d, int64_t n,
                                          double lam, const uint32_t* __restrict__ idx, const T* __restrict__ inv_nq,
                                          int64_t m, double eta, const T* __restrict__ mu, T* __restrict__ Rt,
                                          T* __restrict__ cvec, T* __restrict__ Kt, T* __restrict__ hn, int64_t b,
                                          const float* __restrict__ rsc = nullptr) {
  constexpr int B = kBlk, RP0 = B + 4, RP = LA ? RP0 + B : RP0;
  constexpr int E = 16 / sizeof(T);
  constexpr int CH = 64;              // columns per staged chunk
  constexpr int TS = CH + E;          // tile row stride (16-byte multiple, skews banks)
  constexpr int NLT = (RP0 / 4) * (RP0 / 4 + 1) / 2;   // lower-triangular 4x4 tiles of the block Gram (153)
  constexpr int NXT = LA ? (B / 4) * (RP0 / 4) : 0;    // cross tiles next-block rows x (rows, mu) (272)
  extern __shared__ __align__(16) unsigned char pr_sh[];
  T* tile = reinterpret_cast<T*>(pr_sh);        // [2][RP][TS]
  T* G = tile + 2 * RP * TS;                    // [RP0][RP0 + 1]
  T* R = G + RP0 * (RP0 + 1);                   // [B][B + 1]   R[j][c]
  T* acc = R + B * (B + 1);                     // [B][B + 1]
  T* Gx = acc + B * (B + 1);                    // [B][RP0 + 1] (LA only)
  __shared__ T kap[B];
  __shared__ int64_t rowid[LA ? 2 * B : B];
  const int tid = threadIdx.x;
  const int64_t t0 = b * B;
  const int Bb = (int)min64(B, m - t0);
  const T Nn = (T)((double)N / (double)n), lN = (T)(lam * (double)N);
  if (tid < B) {
    if (tid < Bb) {
      const uint32_t i = min(idx[t0 + tid], (uint32_t)(N - 1));   // indices are < N by contract
      rowid[tid] = i;
      kap[tid] = (i < (uint64_t)n ? Nn : lN) * inv_nq[t0 + tid];
    } else {
      rowid[tid] = -1;
      kap[tid] = T(0);
    }
  } else if (LA && tid < 2 * B) {
    rowid[tid] = (t0 + tid < m) ? (int64_t)min(idx[t0 + tid], (uint32_t)(N - 1)) : -1;
  }
  __syncthreads();
  // staged row r: a sampled row of this block, mu, a zero row, or a sampled row of the next block
  auto row_of = [&](int r) -> int64_t {
    if (r < B) return r < Bb ? rowid[r] : -1;
    if (LA && r >= RP0) return rowid[B + r - RP0];
    return -1;
  };
  const int nch = (int)((d + CH - 1) / CH);
  auto stage = [&](int ch, int buf) {
    T* dst = tile + buf * RP * TS;
    const int64_t cbase = (int64_t)ch * CH;
    if constexpr (!std::is_same<S, T>::value) {
      // bfloat16 rows: synchronous 16-byte loads widened to float (the buffer being written was
      // last read before the previous chunk's closing barrier)
      constexpr int ES = 16 / sizeof(S);
      for (int e = tid; e < RP * (CH / ES); e += blockDim.x) {
        const int r = e / (CH / ES), q = e % (CH / ES);
        const int64_t col = cbase + q * ES;
        T v[ES];
#pragma unroll
        for (int i = 0; i < ES; ++i) v[i] = T(0);
        const int64_t rid = row_of(r);
        if (rid >= 0 && col < d) {
          const S* src = Z + rid * ld + col;
          const float sc = IsFp8<S>::value ? rsc[rid] : 1.0f;   // FP8 codes carry a per-row scale
          if (col + ES <= d) ld_widen(src, v, sc);
          else
            for (int i = 0; i < (int)(d - col); ++i) v[i] = cvt<T>(src[i]) * sc;
        } else if (r == B && mu) {
          for (int i = 0; i < ES; ++i)
            if (col + i < d) v[i] = mu[col + i];
        }
        using V = typename Vec<T>::type;
#pragma unroll
        for (int i = 0; i < ES; i += E) {
          V o;
          if constexpr (sizeof(T) == 4) o = V{v[i], v[i + 1], v[i + 2], v[i + 3]};
          else o = V{v[i], v[i + 1]};
          *reinterpret_cast<V*>(dst + r * TS + q * ES + i) = o;
        }
      }
      cp_async_commit();
      return;
    }
    for (int e = tid; e < RP * (CH / E); e += blockDim.x) {
      const int r = e / (CH / E), q = e % (CH / E);
      const int64_t col = cbase + q * E;
      const void* src = Z;
      int bytes = 0;
      if (col < d) {
        const int valid = (int)min64(E, d - col) * (int)sizeof(T);
        const int64_t rid = row_of(r);
        if (rid >= 0) { src = reinterpret_cast<const T*>(Z) + rid * ld + col; bytes = valid; }
        else if (r == B && mu) { src = mu + col; bytes = (reinterpret_cast<uintptr_t>(mu + col) & 15) ? 0 : valid; }
      }
      cp_async16(dst + r * TS + q * E, src, bytes);
    }
    cp_async_commit();
  };
  // mu may not be 16-byte aligned at every chunk: stage it with plain loads when it is not
  const bool mu_aligned = mu == nullptr || (reinterpret_cast<uintptr_t>(mu) & 15) == 0;
  // 4x4 tiles: thread tid takes tile tid and (look-ahead) tile tid + 256.  Tiles 0..152 are the
  // lower triangle of the RP0 x RP0 Gram matrix; tiles 153.. pair next-block rows with rows 0..RP0-1
  auto tile_of = [&](int id, int& I, int& J) {
    I = -1;
    J = -1;
    if (id < NLT) {
      int t = id, q = 0;
      while (q < RP0 / 4 && t > q) { t -= q + 1; ++q; }
      I = q;
      J = t;
    } else if (id < NLT + NXT) {
      I = RP0 / 4 + (id - NLT) / (RP0 / 4);
      J = (id - NLT) % (RP0 / 4);
    }
  };
  int TI, TJ, TI2 = -1, TJ2 = -1;
  tile_of(tid, TI, TJ);
  if (LA) tile_of(tid + 256, TI2, TJ2);
  T a4[4][4], b4[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) a4[i][j] = b4[i][j] = T(0);
  stage(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) stage(ch + 1, (ch + 1) & 1);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    T* tl = tile + (ch & 1) * RP * TS;
    if (!mu_aligned) {
      for (int c = tid; c < CH; c += blockDim.x) {
        const int64_t col = (int64_t)ch * CH + c;
        tl[B * TS + c] = col < d ? mu[col] : T(0);
      }
      __syncthreads();
    }
    if (TI >= 0) {
      using V = typename Vec<T>::type;
#pragma unroll 4
      for (int c = 0; c < CH; c += E) {
        T x[4][E], y[4][E];
#pragma unroll
        for (int i = 0; i < 4; ++i) vec_to_arr(*reinterpret_cast<const V*>(tl + (TI * 4 + i) * TS + c), x[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) vec_to_arr(*reinterpret_cast<const V*>(tl + (TJ * 4 + j) * TS + c), y[j]);
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a4[i][j] = fma(x[i][e], y[j][e], a4[i][j]);
      }
    }
    if (LA && TI2 >= 0) {
      using V = typename Vec<T>::type;
#pragma unroll 4
      for (int c = 0; c < CH; c += E) {
        T x[4][E], y[4][E];
#pragma unroll
        for (int i = 0; i < 4; ++i) vec_to_arr(*reinterpret_cast<const V*>(tl + (TI2 * 4 + i) * TS + c), x[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) vec_to_arr(*reinterpret_cast<const V*>(tl + (TJ2 * 4 + j) * TS + c), y[j]);
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) b4[i][j] = fma(x[i][e], y[j][e], b4[i][j]);
      }
    }
    __syncthreads();
  }
  auto store_tile = [&](int I, int J, T (&t4)[4][4]) {
    if (I < 0) return;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = I * 4 + i, gj = J * 4 + j;
        if (gi < RP0) {
          G[gi * (RP0 + 1) + gj] = t4[i][j];
          G[gj * (RP0 + 1) + gi] = t4[i][j];
        } else {
          Gx[(gi - RP0) * (RP0 + 1) + gj] = t4[i][j];
        }
      }
  };
  store_tile(TI, TJ, a4);
  if (LA) store_tile(TI2, TJ2, b4);
  for (int e = tid; e < B * (B + 1); e += blockDim.x) {
    R[e] = T(0);
    acc[e] = T(0);
  }
  __syncthreads();
  // R = (I + eta K L)^{-1} K row by row: row l is final once rows < l have been folded into acc
  const T et = (T)eta;
  const int cc = tid & (B - 1), jg = tid >> 6;      // column and row group of this thread
  for (int l = 0; l < Bb; ++l) {
    if (tid <= l) R[l * (B + 1) + tid] = (tid == l) ? kap[l] : -et * kap[l] * acc[l * (B + 1) + tid];
    __syncthreads();
    if (cc <= l) {
      const T rl = R[l * (B + 1) + cc];
      for (int j = l + 1 + jg; j < Bb; j += 4) acc[j * (B + 1) + cc] = fma(G[j * (RP0 + 1) + l], rl, acc[j * (B + 1) + cc]);
    }
    __syncthreads();
  }
  // c_j = -eta sum_{l <= j} R[j][l] l h_l with h_l = mu^T z_l = G[B][l]
  if (tid < B) {
    const int j = tid;
    T s = T(0);
    for (int l = 0; l <= j && l < Bb; ++l) s = fma(R[j * (B + 1) + l], (T)l * G[B * (RP0 + 1) + l], s);
    cvec[b * B + j] = j < Bb ? -et * s : T(0);
  }
  T* Rout = Rt + b * (int64_t)B * B;
  for (int e = tid; e < B * B; e += blockDim.x) {
    const int l = e / B, j = e % B;
    Rout[e] = R[j * (B + 1) + l];   // transposed: Rt[l][j] = R[j][l]
  }
  if constexpr (LA) {
    T* Kout = Kt + b * (int64_t)B * B;
    for (int e = tid; e < B * B; e += blockDim.x) {
      const int l = e / B, j = e % B;
      Kout[e] = Gx[j * (RP0 + 1) + l];   // Kt[l][j] = z'_j . z_l
    }
    if (tid < B) hn[b * B + tid] = Gx[tid * (RP0 + 1) + B];
  }
}

// dynamic shared memory of prep_body
template <typename T, bool LA>
constexpr size_t prep_smem_bytes() {
  constexpr int B = kBlk, RP0 = B + 4, RP = LA ? RP0 + B : RP0, E = 16 / sizeof(T);
  return (size_t)(2 * RP * (64 + E) + RP0 * (RP0 + 1) + 2 * B * (B + 1) + (LA ? B * (RP0 + 1) : 0)) * sizeof(T);
}

template <typename S, typename T>
__global__ void __launch_bounds__(256) epoch_prep_kernel(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                                         int64_t n, double lam, const uint32_t* __restrict__ idx,
                                                         const T* __restrict__ inv_nq, int64_t m, double eta,
                                                         const T* __restrict__ mu, T* __restrict__ Rt,
                                                         T* __restrict__ cvec, const float* __restrict__ rsc) {
  prep_body<S, T>(Z, N, ld, d, n, lam, idx, inv_nq, m, eta, mu, Rt, cvec, nullptr, nullptr, blockIdx.x, rsc);
}

template <typename S, typename T>
__global__ void __launch_bounds__(256) epoch_prep_la_kernel(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                                            int64_t n, double lam, const uint32_t* __restrict__ idx,
                                                            const T* __restrict__ inv_nq, int64_t m, double eta,
                                                            const T* __restrict__ mu, T* __restrict__ Rt,
                                                            T* __restrict__ cvec, T* __restrict__ Kt,
                                                            T* __restrict__ hn) {
  prep_body<S, T, true>(Z, N, ld, d, n, lam, idx, inv_nq, m, eta, mu, Rt, cvec, Kt, hn, blockIdx.x);
}

// all jobs' blocks in one grid: block g belongs to job j with blk_off[j] <= g < blk_off[j + 1]
template <typename S, typename T, bool LA>
__global__ void __launch_bounds__(256) epoch_prep_batched_kernel(const ChainJob<S, T>* __restrict__ jobs,
                                                                 const int64_t* __restrict__ blk_off, int nj) {
  const int64_t g = blockIdx.x;
  int lo = 0, hi = nj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blk_off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  const ChainJob<S, T> J = jobs[lo];
  prep_body<S, T, LA>(J.Z, J.N, J.ld, J.d, J.n, J.lam, J.idx, J.inv_nq, J.m, J.eta, J.mu, J.Rt, J.cvec, J.Kt, J.hn,
                      g - blk_off[lo]);
}

// ------------------------------------------------------------------ sequential chain
// One cluster of CS blocks; block r owns columns [r CW, (r+1) CW) of delta (CW = 32 QN).
// Per block of steps each block pushes its partial dot products straight from registers into
// every block's receive buffer with st.async, which signals the receiver's local mbarrier; the
// receivers sum the CS partials in rank order, so every block derives bit-identical a_j.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm(uint64_t* bar, uint32_t tx_bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(tx_bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 16-byte remote store into another block's shared memory that completes tx bytes on its mbarrier
__device__ __forceinline__ void st_async16(uint32_t raddr, uint32_t rbar, const uint32_t* v) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];\n" ::"r"(raddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(rbar)
               : "memory");
}

constexpr long long kWaitCycles = 4000000000LL;   // about two seconds: a wait this long is a fault

// Row padding of the staged slices when TPC lanes share a column: at least CPW elements and 16 bytes.
__host__ __device__ constexpr int chain_zpad(int tpc, int cpw, int esize) {
  return tpc > 1 ? (cpw * esize >= 16 ? cpw : 16 / esize) : 0;
}

template <typename S, typename T, int STAGES, int QN, int NT>
__device__ __forceinline__ void chain_body(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                           const uint32_t* __restrict__ idx, int64_t m, const T* __restrict__ Rt,
                                           const T* __restrict__ cvec, double eta, const T* __restrict__ mu,
                                           const T* __restrict__ wbar, int average, T* __restrict__ wnext,
                                           int* status, const float* __restrict__ rsc) {
  constexpr int B = kBlk;
  constexpr int ES = 16 / sizeof(S);
  constexpr int CW = 32 * QN;               // columns owned by this block
  constexpr int NCH = CW / ES;              // 16-byte chunks per row slice
  constexpr int CPL = NCH >= 32 ? NCH / 32 : 1;   // chunks per lane
  constexpr int NW = NT / 32;                 // warps
  constexpr int RPW = B / NW;                 // rows of the block per warp
  constexpr int H = NT / B;                   // threads per row of R p
  constexpr int W16 = RPW * (int)sizeof(T) / 16;    // 16-byte pieces of one warp's partials
  static_assert(RPW * sizeof(T) % 16 == 0, "partial dots travel in 16-byte pieces");
  static_assert(H == 4 || H == 8, "R p is split over 4 or 8 threads per row");
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char ch_sh[];
  // Layout: lane L of warp w owns the 16-byte chunks q = L + 32 v (v < CPL) of this block's column
  // slice, for the RPW rows RPW w .. RPW w + RPW - 1 of the block of steps.  It loads each of those
  // chunks once with a 16-byte shared-memory load, uses them for its part of the dot products and
  // keeps them in registers for the rank-B update, whose per-warp partial sums over the warp's rows
  // are added across the warps through shared memory (fixed warp order).
  constexpr int ZS = CW;                                   // row stride of the staged slices (in S)
  S* Zs = reinterpret_cast<S*>(ch_sh);                     // [STAGES][B][ZS]
  T* recv = reinterpret_cast<T*>(Zs + (size_t)STAGES * B * ZS);   // [2][kCsMax][B] partial dots from each rank
  // running sum of the iterates (epoch average) as a compensated (Kahan) pair in T: on GB300 a
  // double add sits on the critical path of every block with a long latency
  T* Ssum = recv + 2 * kCsMax * B;                         // [CW]
  T* Scmp = Ssum + CW;                                     // [CW] compensation
  T* dl = Scmp + CW;                                       // [CW]
  T* mus = dl + CW;                                        // [CW]
  T* pv = mus + CW;                                        // [B]
  T* av = pv + B;                                          // [B]   a_j, then (B_b - j) a_j in avw
  T* avw = av + B;                                         // [B]
  T* redu = avw + B;                                       // [NW][CW] per-warp partial sums of the update
  T* redw = redu + NW * CW;                                // [NW][CW] the same with the running-sum weights
  uint32_t* srow = reinterpret_cast<uint32_t*>(redw + NW * CW);   // [STAGES][B]
  float* sscale = reinterpret_cast<float*>(srow + STAGES * B);   // [STAGES][B] row scales (FP8 codes)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sscale + STAGES * B);   // [2]
  constexpr bool F8 = IsFp8<S>::value;
  __shared__ int aborted;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool lane_on = lane < NCH;
  const int64_t c0 = (int64_t)rank * CW;
  const int cwid = (int)max64(0, min64(CW, d - c0));
  const int64_t nblk = (m + B - 1) / B;
  const T et = (T)eta;
  const uint32_t tx_per_block = (uint32_t)(CS * B * sizeof(T));

  for (int c = tid; c < CW; c += NT) {
    dl[c] = T(0);
    Ssum[c] = T(0);
    Scmp[c] = T(0);
    mus[c] = c < cwid ? mu[c0 + c] : T(0);
  }
  auto fetch_rows = [&](int64_t blk) -> uint32_t {
    const int64_t t = blk * B + tid;
    return (tid < B && t < m) ? (uint32_t)min64((int64_t)idx[t], N - 1) : 0xFFFFFFFFu;
  };
  for (int s = 0; s < STAGES; ++s)
    if (tid < B) {
      const uint32_t row = fetch_rows(s);
      srow[s * B + tid] = row;
      if (F8) sscale[s * B + tid] = row != 0xFFFFFFFFu ? rsc[row] : 1.0f;
    }
  uint32_t pend_row = fetch_rows(STAGES);
  if (tid == 0) {
    aborted = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    mbar_arm(&mbar[0], tx_per_block);
    if (nblk > 1) mbar_arm(&mbar[1], tx_per_block);
  }
  __syncthreads();

  // rows beyond the last step and columns beyond d are zero-filled (source size 0); each thread
  // copies exactly the chunks it reads later
  auto load_block = [&](int64_t blk) {
    const int slot = (int)(blk % STAGES);
    S* zdst = Zs + (size_t)slot * B * ZS;
    const uint32_t* rows = srow + slot * B;
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int j = RPW * warp + r;
      const uint32_t row = rows[j];
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int q = lane + 32 * v;
        if (!lane_on) continue;
        const int col = q * ES;
        int bytes = 0;
        const S* src = Z;
        if (row != 0xFFFFFFFFu && col < cwid) {
          bytes = min(ES, cwid - col) * (int)sizeof(S);
          src = Z + (int64_t)row * ld + c0 + col;
        }
        cp_async16(zdst + j * ZS + col, src, bytes);
      }
    }
  };

#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nblk) load_block(s);
    cp_async_commit();
  }
  cluster.sync();   // every block's mbarriers are initialised before any remote store

  // remote addresses this lane pushes to: receiver = lane (lanes >= CS idle)
  const int dst = lane < CS ? lane : 0;
  const uint32_t recv_remote = map_rank(smem_u32(recv), dst);
  const uint32_t bar_remote0 = map_rank(smem_u32(&mbar[0]), dst);
  const uint32_t bar_remote1 = map_rank(smem_u32(&mbar[1]), dst);

  for (int64_t blk = 0; blk < nblk; ++blk) {
    // row indices are read one block ahead of when they enter the ring, so the load's latency is
    // hidden behind a whole block of steps
    const uint32_t next_row = pend_row;
    pend_row = fetch_rows(blk + STAGES + 1);
    float next_scale = 1.0f;
    if (F8 && tid < B && next_row != 0xFFFFFFFFu) next_scale = rsc[next_row];
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    if (blk + STAGES - 1 < nblk) load_block(blk + STAGES - 1);
    cp_async_commit();
    const int slot = (int)(blk % STAGES);
    const int par = (int)(blk & 1);
    const float myscale = (F8 && tid < B) ? sscale[slot * B + tid] : 1.0f;   // row tid of this block
    const int Bb = (int)min64(B, m - blk * B);
    const S* zs = Zs + (size_t)slot * B * ZS;
    // this block's R entries and c_j go straight from L2 into registers: issued here, used after the
    // exchange, so their latency is hidden behind the dot products (issuing them one block earlier,
    // during the update, measured slower: the loads then compete with the update's shared-memory
    // traffic).  Thread (j, h) with j = tid / H takes the terms l = h, h + H, ... of row j of R p.
    constexpr int RPT = B / H;   // R entries per thread
    T rreg[RPT];
    T creg = T(0);
    const int jr = tid / H, hr = tid % H;
    {
      const T* rsrc = Rt + blk * (int64_t)B * B + jr;
#pragma unroll
      for (int t = 0; t < RPT; ++t) {
        const int l = hr + H * t;
        rreg[t] = l <= jr ? __ldg(rsrc + l * B) : T(0);
      }
      if (hr == 0) creg = __ldg(cvec + blk * B + jr);
    }
    // the warp's rows of the staged slice, 16 bytes per chunk, kept for the update
    uint4 zr[RPW][CPL];
    T part[RPW];
    {
      T dv[CPL][ES];
#pragma unroll
      for (int v = 0; v < CPL; ++v)
#pragma unroll
        for (int e = 0; e < ES; ++e) dv[v][e] = lane_on ? dl[(lane + 32 * v) * ES + e] : T(0);
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const S* zrow = zs + (RPW * warp + r) * ZS;
        T sacc = T(0);
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          zr[r][v] = lane_on ? *reinterpret_cast<const uint4*>(zrow + (lane + 32 * v) * ES) : make_uint4(0u, 0u, 0u, 0u);
          const S* sv = reinterpret_cast<const S*>(&zr[r][v]);
#pragma unroll
          for (int e = 0; e < ES; ++e) sacc = fma(cvt<T>(sv[e]), dv[v][e], sacc);
        }
        part[r] = sacc;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < RPW; ++r) part[r] += __shfl_xor_sync(0xffffffffu, part[r], o);
    if (lane < CS) {
      uint32_t pw[RPW * sizeof(T) / 4];
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        if constexpr (sizeof(T) == 8) {
          pw[2 * r] = (uint32_t)__double2loint(part[r]);
          pw[2 * r + 1] = (uint32_t)__double2hiint(part[r]);
        } else {
          pw[r] = __float_as_uint(part[r]);
        }
      }
      const uint32_t base = recv_remote + (uint32_t)(((par * kCsMax + rank) * B + RPW * warp) * sizeof(T));
      const uint32_t rbar = par ? bar_remote1 : bar_remote0;
#pragma unroll
      for (int h = 0; h < W16; ++h) st_async16(base + 16 * h, rbar, pw + 4 * h);
    }
    // wait for the CS partial vectors of this block (bounded), then p = sum over ranks
    if (!aborted) {
      const long long t0c = clock64();
      while (!mbar_try_wait(&mbar[par], (uint32_t)((blk >> 1) & 1))) {
        if (clock64() - t0c > kWaitCycles) {
          atomicOr(status, STATUS_TIMEOUT);
          aborted = 1;
          break;
        }
      }
    }
    if (tid < B) {
      const T* rv = recv + (size_t)par * kCsMax * B + tid;
      T sp = T(0);
      for (int r = 0; r < CS; ++r) sp += rv[r * B];   // rank order: identical in every block
      pv[tid] = F8 ? sp * myscale : sp;
    }
    __syncthreads();
    if (tid == 0 && blk + 2 < nblk) mbar_arm(&mbar[par], tx_per_block);   // next use: block blk + 2
    // a = R p + c: the H threads of row j (adjacent lanes) sum their terms and combine by shuffles
    // in a fixed order; R is lower triangular, so the terms beyond the diagonal are zero
    {
      T s0 = T(0), s1 = T(0);
#pragma unroll
      for (int t = 0; t < RPT; t += 2) {
        s0 = fma(rreg[t], pv[hr + H * t], s0);
        if (t + 1 < RPT) s1 = fma(rreg[t + 1], pv[hr + H * (t + 1)], s1);
      }
      T sa = s0 + s1;
#pragma unroll
      for (int o = 1; o < H; o <<= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
      if (hr == 0) {
        sa += creg;
        // FP8 codes: the update multiplies stored codes, so a_j carries row j's scale (the slot's
        // scales are replaced only after the barrier below)
        const T a = F8 ? sa * (T)sscale[slot * B + jr] : sa;
        av[jr] = a;
        avw[jr] = (T)(Bb - jr) * a;   // weight B_b - j of the running-sum term
      }
    }
    __syncthreads();
    if (tid < B) {
      srow[slot * B + tid] = next_row;    // this slot now holds block blk + STAGES
      if (F8) sscale[slot * B + tid] = next_scale;
    }
    // rank-B update of this warp's rows: u_c = sum_j a_j z_jc, w_c = sum_j (B_b - j) a_j z_jc
    {
      T u[CPL][ES], w[CPL][ES];
#pragma unroll
      for (int v = 0; v < CPL; ++v)
#pragma unroll
        for (int e = 0; e < ES; ++e) u[v][e] = w[v][e] = T(0);
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int j = RPW * warp + r;
        const T a = av[j], aw = avw[j];
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          const S* sv = reinterpret_cast<const S*>(&zr[r][v]);
#pragma unroll
          for (int e = 0; e < ES; ++e) {
            const T z = cvt<T>(sv[e]);
            u[v][e] = fma(a, z, u[v][e]);
            w[v][e] = fma(aw, z, w[v][e]);
          }
        }
      }
      if (lane_on) {
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          T* du = redu + warp * CW + (lane + 32 * v) * ES;
          T* dw = redw + warp * CW + (lane + 32 * v) * ES;
#pragma unroll
          for (int e = 0; e < ES; e += 16 / (int)sizeof(T)) {
            if constexpr (sizeof(T) == 4) {
              *reinterpret_cast<float4*>(du + e) = make_float4(u[v][e], u[v][e + 1], u[v][e + 2], u[v][e + 3]);
              *reinterpret_cast<float4*>(dw + e) = make_float4(w[v][e], w[v][e + 1], w[v][e + 2], w[v][e + 3]);
            } else {
              *reinterpret_cast<double2*>(du + e) = make_double2(u[v][e], u[v][e + 1]);
              *reinterpret_cast<double2*>(dw + e) = make_double2(w[v][e], w[v][e + 1]);
            }
          }
        }
      }
    }
    __syncthreads();
    for (int c = tid; c < CW; c += NT) {
      T uu = T(0), ww = T(0);
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) {   // fixed warp order
        uu += redu[w2 * CW + c];
        ww += redw[w2 * CW + c];
      }
      const T bbT = (T)Bb;
      const T tri = (T)((Bb * (Bb + 1)) / 2);   // exact
      const T dold = dl[c];
      const T x = bbT * dold - et * (mus[c] * tri + ww);
      const T yk = x - Scmp[c];
      const T tk = Ssum[c] + yk;
      Scmp[c] = (tk - Ssum[c]) - yk;
      Ssum[c] = tk;
      dl[c] = dold - et * (bbT * mus[c] + uu);
    }
  }
  cp_async_wait<0>();
  cluster.sync();   // no block leaves while remote stores to it could still be in flight
  for (int c = tid; c < cwid; c += NT) {
    const double v = average ? ((double)Ssum[c] - (double)Scmp[c]) / (double)m : (double)dl[c];
    wnext[c0 + c] = (T)((double)wbar[c0 + c] + v);
  }
}

template <typename S, typename T, int STAGES, int QN, int NT>
__global__ void __launch_bounds__(NT) epoch_chain_kernel(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                                          const uint32_t* __restrict__ idx, int64_t m,
                                                          const T* __restrict__ Rt, const T* __restrict__ cvec,
                                                          double eta, const T* __restrict__ mu,
                                                          const T* __restrict__ wbar, int average,
                                                          T* __restrict__ wnext, int* status, const float* rsc) {
  chain_body<S, T, STAGES, QN, NT>(Z, N, ld, d, idx, m, Rt, cvec, eta, mu, wbar, average, wnext, status, rsc);
}

// one cluster per job (the cluster's blocks are consecutive in x)
template <typename S, typename T, int STAGES, int QN, int NT>
__global__ void __launch_bounds__(NT) epoch_chain_batched_kernel(const ChainJob<S, T>* __restrict__ jobs,
                                                                  int* status) {
  const int cs = (int)cg::this_cluster().num_blocks();
  const ChainJob<S, T> J = jobs[blockIdx.x / cs];
  chain_body<S, T, STAGES, QN, NT>(J.Z, J.N, J.ld, J.d, J.idx, J.m, J.Rt, J.cvec, J.eta, J.mu, J.wbar, J.average,
                                   J.wnext, status, nullptr);
}

// ------------------------------------------------------------------ look-ahead chain
// The same recursion with the cluster exchange taken off the critical path.  With delta_b the
// state at the start of block b, q = Z_{b+1} delta_b and K = Z_{b+1} Z_b^T (from the look-ahead
// preparation),
//   p_{b+1} = q - eta K a_b - B_b eta (Z_{b+1} mu),
// so the partial dot products of q are pushed to every rank at the start of block b and travel
// while the block forms a_b = R_b p_b + c_b and updates delta; p_0 = 0 because delta_0 = 0.
// Per block: Z rows in a ring of ZST stages (blocks b and b+1 resident, b+2.. in flight), and
// R_b, K_b, c_b, hn_b in a two-slot ring.
template <typename S, typename T, int ZST, int QN, int NT>
__device__ __forceinline__ void chain_la_body(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                              const uint32_t* __restrict__ idx, int64_t m, const T* __restrict__ Rt,
                                              const T* __restrict__ cvec, const T* __restrict__ Kt,
                                              const T* __restrict__ hn, double eta, const T* __restrict__ mu,
                                              const T* __restrict__ wbar, int average, T* __restrict__ wnext,
                                              int* status) {
  constexpr int B = kBlk;
  constexpr int E = 16 / sizeof(T);
  constexpr int ES = 16 / sizeof(S);
  constexpr int CW = 32 * QN;
  constexpr int NCH = CW / ES;
  constexpr int NW = NT / 32;
  constexpr int RPW = B / NW;
  constexpr int H = NT / B;
  constexpr int TPC = NT / CW > 0 ? NT / CW : 1;
  constexpr int JPT = B / TPC;
  constexpr int CPW = 32 / TPC;
  constexpr int W16 = RPW * (int)sizeof(T) / 16;
  constexpr int ZS = CW + chain_zpad(TPC, CPW, (int)sizeof(S));
  constexpr int AUX = 2 * B * B + 2 * B;   // one slot: R (l, j), K (l, j), c, hn
  static_assert(ZST >= 3, "blocks b and b+1 resident plus one in flight");
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char ch_sh[];
  S* Zs = reinterpret_cast<S*>(ch_sh);                                 // [ZST][B][ZS]
  T* aux = reinterpret_cast<T*>(Zs + (size_t)ZST * B * ZS);           // [2][AUX]
  T* recv = aux + 2 * AUX;                                             // [2][kCsMax][B]
  T* Ssum = recv + 2 * kCsMax * B;                                     // [CW] compensated running sum
  T* Scmp = Ssum + CW;                                                 // [CW]
  T* dl = Scmp + CW;                                                   // [CW]
  T* mus = dl + CW;                                                    // [CW]
  T* pv = mus + CW;                                                    // [B]
  T* av = pv + B;                                                      // [B]
  T* part4 = av + B;                                                   // [H][B]
  uint32_t* srow = reinterpret_cast<uint32_t*>(part4 + H * B);         // [ZST][B]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(srow + ZST * B);        // [2]
  __shared__ int aborted;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)rank * CW;
  const int cwid = (int)max64(0, min64(CW, d - c0));
  const int64_t nblk = (m + B - 1) / B;
  const T et = (T)eta;
  const uint32_t tx_per_block = (uint32_t)(CS * B * sizeof(T));

  for (int c = tid; c < CW; c += NT) {
    dl[c] = T(0);
    Ssum[c] = T(0);
    Scmp[c] = T(0);
    mus[c] = c < cwid ? mu[c0 + c] : T(0);
  }
  if (tid < B) pv[tid] = T(0);
  auto fetch_rows = [&](int64_t blk) -> uint32_t {
    const int64_t t = blk * B + tid;
    return (tid < B && t < m) ? (uint32_t)min64((int64_t)idx[t], N - 1) : 0xFFFFFFFFu;
  };
  for (int s = 0; s < ZST; ++s)
    if (tid < B) srow[s * B + tid] = fetch_rows(s);
  uint32_t pend_row = fetch_rows(ZST);
  if (tid == 0) {
    aborted = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (nblk > 1) mbar_arm(&mbar[1], tx_per_block);   // exchange for block 1
    if (nblk > 2) mbar_arm(&mbar[0], tx_per_block);   // exchange for block 2
  }
  __syncthreads();

  auto load_z = [&](int64_t blk) {
    const int slot = (int)(blk % ZST);
    S* zdst = Zs + (size_t)slot * B * ZS;
    const uint32_t* rows = srow + slot * B;
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int j = warp + NW * r;
      const uint32_t row = rows[j];
      for (int q = lane; q < NCH; q += 32) {
        const int col = q * ES;
        int bytes = 0;
        const S* src = Z;
        if (row != 0xFFFFFFFFu && col < cwid) {
          bytes = min(ES, cwid - col) * (int)sizeof(S);
          src = Z + (int64_t)row * ld + c0 + col;
        }
        cp_async16(zdst + j * ZS + col, src, bytes);
      }
    }
  };
  auto load_aux = [&](int64_t blk) {
    T* dst = aux + (size_t)(blk & 1) * AUX;
    for (int e = tid; e < AUX / E; e += NT) {
      const int o = e * E;
      const T* src;
      if (o < B * B) src = Rt + blk * (int64_t)B * B + o;
      else if (o < 2 * B * B) src = Kt + blk * (int64_t)B * B + (o - B * B);
      else if (o < 2 * B * B + B) src = cvec + blk * B + (o - 2 * B * B);
      else src = hn + blk * B + (o - 2 * B * B - B);
      cp_async16(dst + o, src, 16);
    }
  };

  for (int s = 0; s < ZST - 1; ++s)
    if (s < nblk) load_z(s);
  load_aux(0);
  cp_async_commit();
  cluster.sync();   // every block's mbarriers are initialised before any remote store

  const int dst = lane < CS ? lane : 0;
  const uint32_t recv_remote = map_rank(smem_u32(recv), dst);
  const uint32_t bar_remote0 = map_rank(smem_u32(&mbar[0]), dst);
  const uint32_t bar_remote1 = map_rank(smem_u32(&mbar[1]), dst);

  for (int64_t blk = 0; blk < nblk; ++blk) {
    cp_async_wait<0>();
    __syncthreads();
    if (blk + ZST - 1 < nblk) load_z(blk + ZST - 1);
    if (blk + 1 < nblk) load_aux(blk + 1);
    cp_async_commit();
    {
      const uint32_t nr = pend_row;
      pend_row = fetch_rows(blk + ZST + 1);
      if (tid < B) srow[(int)((blk + ZST) % ZST) * B + tid] = nr;   // that slot's block was issued long ago
    }
    const int Bb = (int)min64(B, m - blk * B);
    const bool has_next = blk + 1 < nblk;
    const T* A = aux + (size_t)(blk & 1) * AUX;
    const T* Rs = A;
    const T* Ks = A + B * B;
    const T* Cs = A + 2 * B * B;
    const T* Hs = Cs + B;
    // (A) partial dots of the next block's rows with delta_b, pushed to every rank
    if (has_next) {
      const S* zsn = Zs + (size_t)((blk + 1) % ZST) * B * ZS;
      T dv[QN];
#pragma unroll
      for (int q = 0; q < QN; ++q) dv[q] = dl[lane + 32 * q];
      T part[RPW];
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const S* zr = zsn + (RPW * warp + r) * ZS + lane;
        T sacc = T(0);
#pragma unroll
        for (int q = 0; q < QN; ++q) sacc = fma(cvt<T>(zr[32 * q]), dv[q], sacc);
        part[r] = sacc;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < RPW; ++r) part[r] += __shfl_xor_sync(0xffffffffu, part[r], o);
      if (lane < CS) {
        uint32_t pw[RPW * sizeof(T) / 4];
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          if constexpr (sizeof(T) == 8) {
            pw[2 * r] = (uint32_t)__double2loint(part[r]);
            pw[2 * r + 1] = (uint32_t)__double2hiint(part[r]);
          } else {
            pw[r] = __float_as_uint(part[r]);
          }
        }
        const int par = (int)((blk + 1) & 1);
        const uint32_t base = recv_remote + (uint32_t)(((par * kCsMax + rank) * B + RPW * warp) * sizeof(T));
        const uint32_t rbar = par ? bar_remote1 : bar_remote0;
#pragma unroll
        for (int h = 0; h < W16; ++h) st_async16(base + 16 * h, rbar, pw + 4 * h);
      }
    }
    // (B) a_b = R_b p_b + c_b: thread (j, h) sums the terms l = h, h + H, ... <= j
    {
      const int j = tid & (B - 1), h = tid >> 6;
      const T* rs = Rs + j;
      T s0 = T(0), s1 = T(0);
      const int lend = j + 1;
      int l = h;
      for (; l + H < lend; l += 2 * H) {
        s0 = fma(rs[l * B], pv[l], s0);
        s1 = fma(rs[(l + H) * B], pv[l + H], s1);
      }
      if (l < lend) s0 = fma(rs[l * B], pv[l], s0);
      part4[h * B + j] = s0 + s1;
    }
    __syncthreads();
    if (tid < B) {
      T sa = Cs[tid];
#pragma unroll
      for (int hh = 0; hh < H; ++hh) sa += part4[hh * B + tid];   // fixed order
      av[tid] = sa;
    }
    __syncthreads();
    // (C) rank-B update of delta and of the running sum with this block's rows
    {
      const S* zs = Zs + (size_t)(blk % ZST) * B * ZS;
      const int c = warp * CPW + (lane % CPW), g = lane / CPW;
      T u = T(0), w = T(0);
      T wt = (T)(Bb - g);
#pragma unroll 8
      for (int jj = 0; jj < JPT; ++jj) {
        const int j = g + TPC * jj;
        const T az = av[j] * cvt<T>(zs[j * ZS + c]);
        u += az;
        w = fma(wt, az, w);
        wt -= T(TPC);
      }
#pragma unroll
      for (int o = CPW; o < 32; o <<= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
      }
      if (g == 0) {
        const T bbT = (T)Bb;
        const T tri = (T)((Bb * (Bb + 1)) / 2);   // exact
        const T dold = dl[c];
        const T x = bbT * dold - et * (mus[c] * tri + w);
        const T yk = x - Scmp[c];
        const T tk = Ssum[c] + yk;
        Scmp[c] = (tk - Ssum[c]) - yk;
        Ssum[c] = tk;
        dl[c] = dold - et * (bbT * mus[c] + u);
      }
    }
    // (E) K a_b: thread (j, h) sums the terms l = h, h + H, ... (K is full)
    if (has_next) {
      const int j = tid & (B - 1), h = tid >> 6;
      const T* ks = Ks + j;
      T s0 = T(0), s1 = T(0);
#pragma unroll 4
      for (int l = h; l < B; l += 2 * H) {
        s0 = fma(ks[l * B], av[l], s0);
        s1 = fma(ks[(l + H) * B], av[l + H], s1);
      }
      part4[h * B + j] = s0 + s1;
    }
    // (D) the next block's partial dots from every rank (bounded wait)
    if (has_next && !aborted) {
      const long long t0c = clock64();
      while (!mbar_try_wait(&mbar[(blk + 1) & 1], (uint32_t)((blk >> 1) & 1))) {
        if (clock64() - t0c > kWaitCycles) {
          atomicOr(status, STATUS_TIMEOUT);
          aborted = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (has_next && tid < B) {
      const T* rv = recv + (size_t)((blk + 1) & 1) * kCsMax * B + tid;
      T q = T(0);
      for (int r = 0; r < CS; ++r) q += rv[r * B];   // rank order: identical in every block
      T kx = T(0);
#pragma unroll
      for (int hh = 0; hh < H; ++hh) kx += part4[hh * B + tid];
      pv[tid] = q - et * kx - et * (T)Bb * Hs[tid];
    }
    if (tid == 0 && blk + 3 < nblk) mbar_arm(&mbar[(blk + 1) & 1], tx_per_block);   // that slot's next use
  }
  cp_async_wait<0>();
  cluster.sync();   // no block leaves while remote stores to it could still be in flight
  for (int c = tid; c < cwid; c += NT) {
    const double v = average ? ((double)Ssum[c] - (double)Scmp[c]) / (double)m : (double)dl[c];
    wnext[c0 + c] = (T)((double)wbar[c0 + c] + v);
  }
}

template <typename S, typename T, int ZST, int QN, int NT>
__global__ void __launch_bounds__(NT) epoch_chain_la_kernel(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                                             const uint32_t* __restrict__ idx, int64_t m,
                                                             const T* __restrict__ Rt, const T* __restrict__ cvec,
                                                             const T* __restrict__ Kt, const T* __restrict__ hn,
                                                             double eta, const T* __restrict__ mu,
                                                             const T* __restrict__ wbar, int average,
                                                             T* __restrict__ wnext, int* status) {
  chain_la_body<S, T, ZST, QN, NT>(Z, N, ld, d, idx, m, Rt, cvec, Kt, hn, eta, mu, wbar, average, wnext, status);
}

template <typename S, typename T, int ZST, int QN, int NT>
__global__ void __launch_bounds__(NT) epoch_chain_la_batched_kernel(const ChainJob<S, T>* __restrict__ jobs,
                                                                     int* status) {
  const int cs = (int)cg::this_cluster().num_blocks();
  const ChainJob<S, T> J = jobs[blockIdx.x / cs];
  chain_la_body<S, T, ZST, QN, NT>(J.Z, J.N, J.ld, J.d, J.idx, J.m, J.Rt, J.cvec, J.Kt, J.hn, J.eta, J.mu, J.wbar,
                                   J.average, J.wnext, status);
}

struct ChainPlan {
  int cs = 0, qn = 0, stages = 0, nt = 0;
  size_t shm = 0;
};

template <typename S, typename T>
size_t chain_smem(int qn, int stages, int nt) {
  const int CW = 32 * qn;
  const int NW = nt / 32;
  return (size_t)stages * kBlk * CW * sizeof(S) + 2 * (size_t)kCsMax * kBlk * sizeof(T) + 4 * (size_t)CW * sizeof(T) +
         3 * (size_t)kBlk * sizeof(T) + 2 * (size_t)NW * CW * sizeof(T) + (size_t)stages * kBlk * sizeof(uint32_t) +
         (size_t)stages * kBlk * sizeof(float) + 2 * sizeof(uint64_t) + 64;
}

// Cluster size: enough blocks that each owns at most 64 columns, up to 16 blocks (then up to
// 256 columns each).  RS_CHAIN_CLUSTER overrides the cluster size (1, 2, 4, 8 or 16).
int choose_cluster(int64_t d) {
  const char* env = std::getenv("RS_CHAIN_CLUSTER");
  if (env) return std::atoi(env);
  int cs = 1;
  while (cs < kCsMax && (d + cs - 1) / cs > 64) cs *= 2;
  return cs;
}

// Threads per block of the chain: 512 by default, RS_CHAIN_THREADS = 256 or 512 overrides.
int choose_threads() {
  const char* env = std::getenv("RS_CHAIN_THREADS");
  const int nt = env ? std::atoi(env) : 512;
  return (nt == 256 || nt == 512) ? nt : 512;
}

template <typename S, typename T>
ChainPlan plan_chain(int64_t d, int cs, size_t cap = 200 * 1024, int nt_pick = 0, int max_st = 4) {
  ChainPlan p;
  const int nt = nt_pick ? nt_pick : choose_threads();
  if (cs < 1 || cs > kCsMax || (cs & (cs - 1))) return p;
  const int64_t per = (d + cs - 1) / cs;
  int qn = per <= 64 ? 2 : (per <= 128 ? 4 : (per <= 256 ? 8 : 0));
  if (!qn) return p;
  for (int st = max_st; st >= 2; --st) {
    const size_t shm = chain_smem<S, T>(qn, st, nt);
    if (shm <= cap) {
      p.nt = nt;
      p.cs = cs;
      p.qn = qn;
      p.stages = st;
      p.shm = shm;
      return p;
    }
  }
  return p;
}

template <typename S, typename T, int ST, int QN, int NT>
int launch_chain(rs_ctx* ctx, const ChainPlan& pl, const S* Z, int64_t N, int64_t ld, int64_t d,
                 const uint32_t* idx, int64_t m, const T* Rt, const T* cv, double eta, const T* mu, const T* wbar,
                 int average, T* wnext, const float* rsc) {
  auto kern = epoch_chain_kernel<S, T, ST, QN, NT>;
  RS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.shm));
  if (pl.cs > 8) RS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.cs, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = pl.shm;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return RS_EUNSUPPORTED;   // this cluster shape cannot be placed on the device: caller tries a smaller one
  }
  RS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, Z, N, ld, d, idx, m, Rt, cv, eta, mu, wbar, average, wnext,
                                 ctx->d_status, rsc));
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

// look-ahead chain: shared memory, plan (ZST = 4 or 3 stages within 200 KB, 512 threads)
template <typename S, typename T>
size_t chain_la_smem(int qn, int zst, int nt) {
  const int CW = 32 * qn;
  const int TPC = std::max(1, nt / CW);
  const int ZS = CW + chain_zpad(TPC, 32 / TPC, (int)sizeof(S));
  return (size_t)zst * kBlk * ZS * sizeof(S) + 2 * (size_t)(2 * kBlk * kBlk + 2 * kBlk) * sizeof(T) +
         2 * (size_t)kCsMax * kBlk * sizeof(T) + 2 * (size_t)CW * sizeof(T) + 2 * (size_t)CW * sizeof(T) +
         (2 + nt / kBlk) * (size_t)kBlk * sizeof(T) + (size_t)zst * kBlk * sizeof(uint32_t) + 2 * sizeof(uint64_t) +
         64;
}

template <typename S, typename T>
ChainPlan plan_chain_la(int64_t d, int cs) {
  ChainPlan p;
  const int nt = 512;
  if (cs < 1 || cs > kCsMax || (cs & (cs - 1))) return p;
  const int64_t per = (d + cs - 1) / cs;
  const int qn = per <= 64 ? 2 : (per <= 128 ? 4 : (per <= 256 ? 8 : 0));
  if (!qn) return p;
  for (int st = 4; st >= 3; --st) {
    const size_t shm = chain_la_smem<S, T>(qn, st, nt);
    if (shm <= 200 * 1024) {
      p.nt = nt;
      p.cs = cs;
      p.qn = qn;
      p.stages = st;
      p.shm = shm;
      return p;
    }
  }
  return p;
}

// The look-ahead variant (float arithmetic only) runs when RS_CHAIN_LOOKAHEAD=1.  Measured on
// GB300 it is slower than the plain chain (the cross Gram matrices double the preparation work and
// the second matrix-vector product lengthens each block), so it is off by default.
template <typename T>
bool use_lookahead() {
  if (sizeof(T) != 4) return false;
  const char* env = std::getenv("RS_CHAIN_LOOKAHEAD");
  return env && env[0] == '1';
}

template <typename K>
int config_cluster_launch(rs_ctx* ctx, K kern, const ChainPlan& pl, int nclusters, cudaLaunchConfig_t& cfg,
                          cudaLaunchAttribute* attr) {
  RS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.shm));
  if (pl.cs > 8) RS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cfg = {};
  cfg.gridDim = dim3((unsigned)(pl.cs * nclusters), 1, 1);
  cfg.blockDim = dim3(pl.nt, 1, 1);
  cfg.dynamicSmemBytes = pl.shm;
  cfg.stream = ctx->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return RS_EUNSUPPORTED;
  }
  return RS_OK;
}

template <typename S, typename T, int ZST, int QN>
int launch_chain_la(rs_ctx* ctx, const ChainPlan& pl, const S* Z, int64_t N, int64_t ld, int64_t d,
                    const uint32_t* idx, int64_t m, const T* Rt, const T* cv, const T* Kt, const T* hn, double eta,
                    const T* mu, const T* wbar, int average, T* wnext) {
  auto kern = epoch_chain_la_kernel<S, T, ZST, QN, 512>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  const int rc = config_cluster_launch(ctx, kern, pl, 1, cfg, attr);
  if (rc != RS_OK) return rc;
  RS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, Z, N, ld, d, idx, m, Rt, cv, Kt, hn, eta, mu, wbar, average, wnext,
                                 ctx->d_status));
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

template <typename S, typename T, int ZST, int QN>
int launch_chain_la_batched(rs_ctx* ctx, const ChainPlan& pl, const ChainJob<S, T>* jobs, int nj) {
  auto kern = epoch_chain_la_batched_kernel<S, T, ZST, QN, 512>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  const int rc = config_cluster_launch(ctx, kern, pl, nj, cfg, attr);
  if (rc != RS_OK) return rc;
  RS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, jobs, ctx->d_status));
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

}  // namespace

// The tensor-core preparation for bfloat16 components (RS_OK when it ran, RS_EUNSUPPORTED when
// the CUDA-core kernel has to run instead).
template <typename S, typename T>
int try_umma_prep(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lam, const uint32_t* idx, const T* inv_nq,
                  int64_t m, double eta, const T* mu, T* Rt, T* cv) {
  if constexpr (std::is_same<S, __nv_bfloat16>::value && std::is_same<T, float>::value) {
    ChainJob<S, T> one{};
    one.Z = static_cast<const S*>(Z->data);
    one.N = Z->n;
    one.ld = Z->ld;
    one.d = Z->d;
    one.n = n;
    one.m = m;
    one.idx = idx;
    one.inv_nq = inv_nq;
    one.lam = lam;
    one.eta = eta;
    one.mu = mu;
    one.Rt = Rt;
    one.cvec = cv;
    return umma_prep(ctx, one, nullptr, nullptr, 0, (m + kBlk - 1) / kBlk);
  } else {
    return RS_EUNSUPPORTED;
  }
}

template <typename S, typename T>
int svrg_epoch_t(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lam, const uint32_t* idx, const T* inv_nq,
                 int64_t m, double eta, const T* wbar, const T* mu, int average, T* wnext) {
  const int64_t N = Z->n, d = Z->d;
  const S* Zd = static_cast<const S*>(Z->data);
  const int64_t nblk = (m + kBlk - 1) / kBlk;
  T* Rt = static_cast<T*>(rs_scratch(ctx, SCR_R, (size_t)nblk * kBlk * kBlk * sizeof(T)));
  T* cv = static_cast<T*>(rs_scratch(ctx, SCR_C, (size_t)nblk * kBlk * sizeof(T)));
  if (!Rt || !cv) return RS_ENOMEM;
  const bool la = use_lookahead<T>() && !IsFp8<S>::value;
  if constexpr (sizeof(T) == 4 && !IsFp8<S>::value) {
    if (la) {
      T* Kt = static_cast<T*>(rs_scratch(ctx, SCR_KT, (size_t)nblk * kBlk * kBlk * sizeof(T)));
      T* hn = static_cast<T*>(rs_scratch(ctx, SCR_HN, (size_t)nblk * kBlk * sizeof(T)));
      if (!Kt || !hn) return RS_ENOMEM;
      constexpr size_t pshm = prep_smem_bytes<T, true>();
      RS_CUDA_TRY(cudaFuncSetAttribute(epoch_prep_la_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pshm));
      epoch_prep_la_kernel<S, T><<<(unsigned)nblk, 256, pshm, ctx->stream>>>(Zd, N, Z->ld, d, n, lam, idx, inv_nq, m,
                                                                             eta, mu, Rt, cv, Kt, hn);
      RS_LAUNCH_CHECK(ctx);
      for (int cs = choose_cluster(d); cs >= 1; cs /= 2) {
        const ChainPlan pl = plan_chain_la<S, T>(d, cs);
        if (!pl.cs) continue;
        int rc = RS_EUNSUPPORTED;
#define RS_CHAIN_LA(ST, QN)                                                                                          \
  if (pl.stages == ST && pl.qn == QN)                                                                                \
    rc = launch_chain_la<S, T, ST, QN>(ctx, pl, Zd, N, Z->ld, d, idx, m, Rt, cv, Kt, hn, eta, mu, wbar, average, wnext);
        RS_CHAIN_LA(4, 2) RS_CHAIN_LA(4, 4) RS_CHAIN_LA(4, 8) RS_CHAIN_LA(3, 2) RS_CHAIN_LA(3, 4) RS_CHAIN_LA(3, 8)
#undef RS_CHAIN_LA
        if (rc != RS_EUNSUPPORTED) return rc;
      }
      // no look-ahead layout fits: the plain chain below uses the same R and c
    }
  }
  if (!la) {
    const int urc = try_umma_prep<S, T>(ctx, Z, n, lam, idx, inv_nq, m, eta, mu, Rt, cv);
    if (urc != RS_OK && urc != RS_EUNSUPPORTED) return urc;
    if (urc == RS_EUNSUPPORTED) {
      constexpr size_t pshm = prep_smem_bytes<T, false>();
      RS_CUDA_TRY(
          cudaFuncSetAttribute(epoch_prep_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pshm));
      epoch_prep_kernel<S, T><<<(unsigned)nblk, 256, pshm, ctx->stream>>>(Zd, N, Z->ld, d, n, lam, idx, inv_nq, m,
                                                                          eta, mu, Rt, cv, Z->row_scale);
      RS_LAUNCH_CHECK(ctx);
    }
  }
  const TuneEntry* te = tune_find(ctx, TUNE_CHAIN, dtype_code<S>(), d);   // rs_autotune's choice, if any
  for (int cs = te ? te->a : choose_cluster(d); cs >= 1; cs /= 2) {
    const ChainPlan pl = plan_chain<S, T>(d, cs, 200 * 1024, te ? te->b : 0, te ? te->c : 4);
    if (!pl.cs) continue;
    int rc = RS_EUNSUPPORTED;
#define RS_CHAIN(ST, QN)                                                                                          \
  if (pl.stages == ST && pl.qn == QN && pl.nt == 256)                                                             \
    rc = launch_chain<S, T, ST, QN, 256>(ctx, pl, Zd, N, Z->ld, d, idx, m, Rt, cv, eta, mu, wbar, average, wnext,   \
                                         Z->row_scale);                                                           \
  if (pl.stages == ST && pl.qn == QN && pl.nt == 512)                                                             \
    rc = launch_chain<S, T, ST, QN, 512>(ctx, pl, Zd, N, Z->ld, d, idx, m, Rt, cv, eta, mu, wbar, average, wnext, \
                                         Z->row_scale);
    RS_CHAIN(4, 2) RS_CHAIN(4, 4) RS_CHAIN(4, 8) RS_CHAIN(3, 2) RS_CHAIN(3, 4) RS_CHAIN(3, 8)
    RS_CHAIN(2, 2) RS_CHAIN(2, 4) RS_CHAIN(2, 8)
#undef RS_CHAIN
    if (rc != RS_EUNSUPPORTED) return rc;
  }
  return rs_fail(RS_EUNSUPPORTED, "rs_svrg_epoch: no thread-block cluster layout fits d = %lld", (long long)d);
}

// ------------------------------------------------------------------ split preparation
// R of every block depends only on the sampled rows and the step size, c also on mu.  The
// one-problem solver therefore prepares the next epoch's R (epoch_prep_kernel with mu = null,
// on a second stream, on SMs the inner loop leaves idle) while the current epoch runs, and forms
// c after the snapshot gradient: h_l = z_l^T mu for the block's rows, c_j = -eta sum_{l<=j} R_jl l h_l.
namespace {

template <typename S, typename T>
__global__ void __launch_bounds__(512) epoch_c_kernel(const S* __restrict__ Z, int64_t N, int64_t ld, int64_t d,
                                                      const uint32_t* __restrict__ idx, int64_t m, double eta,
                                                      const T* __restrict__ mu, const T* __restrict__ Rt,
                                                      T* __restrict__ cvec, const float* __restrict__ rsc) {
  constexpr int B = kBlk;
  constexpr int EU = 16 / (int)sizeof(S);   // elements per 16-byte unit of a row
  extern __shared__ float4 ec_sh4[];
  T* mus = reinterpret_cast<T*>(ec_sh4);    // mu, zero-padded to whole units
  __shared__ T h[B];
  const int64_t b = blockIdx.x, t0 = b * B;
  const int Bb = (int)min64(B, m - t0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t nu = (d + EU - 1) / EU;
  for (int64_t e = threadIdx.x; e < nu * EU; e += blockDim.x) mus[e] = e < d ? mu[e] : T(0);
  __syncthreads();
  // h_l = z_l^T mu: a warp takes two rows at a time, 16-byte loads of both issued together
  for (int l0 = warp; l0 < B; l0 += 2 * nw) {
    int64_t ri[2];
    const S* row[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int l = l0 + k * nw;
      ri[k] = l < Bb ? min64((int64_t)idx[t0 + l], N - 1) : -1;
      row[k] = ri[k] >= 0 ? Z + ri[k] * ld : nullptr;
    }
    T s[2] = {T(0), T(0)};
    for (int64_t u = lane; u < nu; u += 32) {
      const int64_t c0 = u * EU;
      S v[2][EU];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!row[k]) {
#pragma unroll
          for (int e = 0; e < EU; ++e) v[k][e] = S(0.0f);
        } else if (c0 + EU <= d) {
          *reinterpret_cast<uint4*>(v[k]) = *reinterpret_cast<const uint4*>(row[k] + c0);
        } else {
#pragma unroll
          for (int e = 0; e < EU; ++e) v[k][e] = c0 + e < d ? row[k][c0 + e] : S(0.0f);
        }
      }
#pragma unroll
      for (int e = 0; e < EU; ++e) {
        const T me = mus[c0 + e];
        s[0] = fma(cvt<T>(v[0][e]), me, s[0]);
        s[1] = fma(cvt<T>(v[1][e]), me, s[1]);
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      T t = warp_sum(s[k]);
      const int l = l0 + k * nw;
      if (IsFp8<S>::value && ri[k] >= 0) t *= (T)rsc[ri[k]];
      if (lane == 0 && l < B) h[l] = ri[k] >= 0 ? t : T(0);
    }
  }
  __syncthreads();
  if (threadIdx.x < B) {
    const int j = threadIdx.x;
    const T* R = Rt + b * (int64_t)B * B;   // R[j][l] = Rt[l][j]
    T s = T(0);
    for (int l = 0; l <= j && l < Bb; ++l) s = fma(R[l * B + j], (T)l * h[l], s);
    cvec[b * B + j] = j < Bb ? -(T)eta * s : T(0);
  }
}

}  // namespace

// R (and zero c) of every block of an epoch, without mu, on the context's stream.
template <typename S, typename T>
int epoch_prep_r_t(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lam, const uint32_t* idx, const T* inv_nq,
                   int64_t m, double eta, T* Rt, T* cv) {
  const S* Zd = static_cast<const S*>(Z->data);
  const int64_t nblk = (m + kBlk - 1) / kBlk;
  const int urc = try_umma_prep<S, T>(ctx, Z, n, lam, idx, inv_nq, m, eta, (const T*)nullptr, Rt, cv);
  if (urc != RS_EUNSUPPORTED) return urc;
  constexpr size_t pshm = prep_smem_bytes<T, false>();
  RS_CUDA_TRY(cudaFuncSetAttribute(epoch_prep_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pshm));
  epoch_prep_kernel<S, T><<<(unsigned)nblk, 256, pshm, ctx->stream>>>(Zd, Z->n, Z->ld, Z->d, n, lam, idx, inv_nq, m,
                                                                      eta, nullptr, Rt, cv, Z->row_scale);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

// c of every block from mu and the prepared R, then the inner-loop chain.
template <typename S, typename T>
int epoch_finish_t(rs_ctx* ctx, const rs_matrix* Z, const uint32_t* idx, int64_t m, double eta, const T* Rt, T* cv,
                   const T* wbar, const T* mu, int average, T* wnext) {
  const S* Zd = static_cast<const S*>(Z->data);
  const int64_t N = Z->n, d = Z->d;
  const int64_t nblk = (m + kBlk - 1) / kBlk;
  constexpr int EU = 16 / (int)sizeof(S);
  const size_t cshm = (size_t)((d + EU - 1) / EU) * EU * sizeof(T);
  if (cshm > 48 * 1024)
    RS_CUDA_TRY(cudaFuncSetAttribute(epoch_c_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cshm));
  epoch_c_kernel<S, T><<<(unsigned)nblk, 512, cshm, ctx->stream>>>(Zd, N, Z->ld, d, idx, m, eta, mu, Rt, cv,
                                                                    Z->row_scale);
  RS_LAUNCH_CHECK(ctx);
  const TuneEntry* te = tune_find(ctx, TUNE_CHAIN, dtype_code<S>(), d);   // rs_autotune's choice, if any
  for (int cs = te ? te->a : choose_cluster(d); cs >= 1; cs /= 2) {
    const ChainPlan pl = plan_chain<S, T>(d, cs, 200 * 1024, te ? te->b : 0, te ? te->c : 4);
    if (!pl.cs) continue;
    int rc = RS_EUNSUPPORTED;
#define RS_CHAIN(ST, QN)                                                                                          \
  if (pl.stages == ST && pl.qn == QN && pl.nt == 256)                                                             \
    rc = launch_chain<S, T, ST, QN, 256>(ctx, pl, Zd, N, Z->ld, d, idx, m, Rt, cv, eta, mu, wbar, average, wnext,   \
                                         Z->row_scale);                                                           \
  if (pl.stages == ST && pl.qn == QN && pl.nt == 512)                                                             \
    rc = launch_chain<S, T, ST, QN, 512>(ctx, pl, Zd, N, Z->ld, d, idx, m, Rt, cv, eta, mu, wbar, average, wnext, \
                                         Z->row_scale);
    RS_CHAIN(4, 2) RS_CHAIN(4, 4) RS_CHAIN(4, 8) RS_CHAIN(3, 2) RS_CHAIN(3, 4) RS_CHAIN(3, 8)
    RS_CHAIN(2, 2) RS_CHAIN(2, 4) RS_CHAIN(2, 8)
#undef RS_CHAIN
    if (rc != RS_EUNSUPPORTED) return rc;
  }
  return rs_fail(RS_EUNSUPPORTED, "svrg epoch: no thread-block cluster layout fits d = %lld", (long long)d);
}

#define RS_SPLIT_INST(S, T)                                                                                      \
  template int epoch_prep_r_t<S, T>(rs_ctx*, const rs_matrix*, int64_t, double, const uint32_t*, const T*, int64_t, \
                                    double, T*, T*);                                                             \
  template int epoch_finish_t<S, T>(rs_ctx*, const rs_matrix*, const uint32_t*, int64_t, double, const T*, T*,     \
                                    const T*, const T*, int, T*);
RS_SPLIT_INST(float, float)
RS_SPLIT_INST(double, double)
RS_SPLIT_INST(__nv_bfloat16, float)
RS_SPLIT_INST(__nv_fp8_e4m3, float)
#undef RS_SPLIT_INST

// ------------------------------------------------------------------ batched launches

namespace {

// Cluster size of a chain in a batched launch: the fewest blocks (of at most 256 columns each)
// so that many chains run side by side; RS_BATCH_CLUSTER overrides (1, 2, 4, 8 or 16).
int choose_batch_cluster(int64_t d) {
  const char* env = std::getenv("RS_BATCH_CLUSTER");
  if (env) return std::atoi(env);
  int cs = 1;
  while (cs < kCsMax && (d + cs - 1) / cs > 256) cs *= 2;
  return cs;
}

template <typename S, typename T, int ST, int QN, int NT>
int launch_chain_batched(rs_ctx* ctx, const ChainPlan& pl, const ChainJob<S, T>* jobs, int nj) {
  auto kern = epoch_chain_batched_kernel<S, T, ST, QN, NT>;
  RS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.shm));
  if (pl.cs > 8) RS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(pl.cs * nj), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = pl.shm;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return RS_EUNSUPPORTED;
  }
  RS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, jobs, ctx->d_status));
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

}  // namespace

template <typename S, typename T>
int epoch_prep_batched(rs_ctx* ctx, const ChainJob<S, T>* jobs, const int64_t* blk_off, int nj, int64_t total_blocks) {
  if (nj < 1 || total_blocks < 1) return RS_OK;
  if (total_blocks > 0x7FFFFFFF) return rs_fail(RS_EINVAL, "batched epoch: too many blocks of steps");
  if (use_lookahead<T>()) {
    constexpr size_t pshm = prep_smem_bytes<T, true>();
    RS_CUDA_TRY(cudaFuncSetAttribute(epoch_prep_batched_kernel<S, T, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pshm));
    epoch_prep_batched_kernel<S, T, true><<<(unsigned)total_blocks, 256, pshm, ctx->stream>>>(jobs, blk_off, nj);
  } else {
    if constexpr (std::is_same<S, __nv_bfloat16>::value && std::is_same<T, float>::value) {
      const int urc = umma_prep(ctx, ChainJob<S, T>{}, jobs, blk_off, nj, total_blocks);
      if (urc != RS_EUNSUPPORTED) return urc;
    }
    constexpr size_t pshm = prep_smem_bytes<T, false>();
    RS_CUDA_TRY(cudaFuncSetAttribute(epoch_prep_batched_kernel<S, T, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pshm));
    epoch_prep_batched_kernel<S, T, false><<<(unsigned)total_blocks, 256, pshm, ctx->stream>>>(jobs, blk_off, nj);
  }
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

template <typename S, typename T>
int epoch_chain_batched(rs_ctx* ctx, const ChainJob<S, T>* jobs, int nj, int64_t d) {
  if (nj < 1) return RS_OK;
  if (use_lookahead<T>()) {
    const int64_t maxc = sizeof(S) == 2 ? 256 : 128;
    int cs = 1;
    while (cs < kCsMax && (d + cs - 1) / cs > maxc) cs *= 2;
    const ChainPlan pl = plan_chain_la<S, T>(d, cs);
    int rc = RS_EUNSUPPORTED;
    if (pl.cs) {
#define RS_CHAIN_LA(ST, QN) \
  if (pl.stages == ST && pl.qn == QN) rc = launch_chain_la_batched<S, T, ST, QN>(ctx, pl, jobs, nj);
      RS_CHAIN_LA(4, 2) RS_CHAIN_LA(4, 4) RS_CHAIN_LA(4, 8) RS_CHAIN_LA(3, 2) RS_CHAIN_LA(3, 4) RS_CHAIN_LA(3, 8)
#undef RS_CHAIN_LA
    }
    if (rc != RS_EUNSUPPORTED) return rc;
  }
  // many chains side by side: a ring small enough for two chain blocks per SM (the inner loop is
  // latency-bound, so two interleave), unless RS_BATCH_CHAIN_SMEM (KB; 0 = no limit) says otherwise
  size_t cap = 110 * 1024;
  if (const char* env = std::getenv("RS_BATCH_CHAIN_SMEM")) cap = std::atoi(env) > 0 ? (size_t)std::atoi(env) * 1024 : 0;
  for (int cs = choose_batch_cluster(d); cs >= 1; cs /= 2) {
    ChainPlan pl = cap ? plan_chain<S, T>(d, cs, cap) : ChainPlan{};
    if (!pl.cs) pl = plan_chain<S, T>(d, cs);
    if (!pl.cs) continue;
    int rc = RS_EUNSUPPORTED;
#define RS_CHAIN(ST, QN)                                                                  \
  if (pl.stages == ST && pl.qn == QN && pl.nt == 256)                                     \
    rc = launch_chain_batched<S, T, ST, QN, 256>(ctx, pl, jobs, nj);                      \
  if (pl.stages == ST && pl.qn == QN && pl.nt == 512)                                     \
    rc = launch_chain_batched<S, T, ST, QN, 512>(ctx, pl, jobs, nj);
    RS_CHAIN(4, 2) RS_CHAIN(4, 4) RS_CHAIN(4, 8) RS_CHAIN(3, 2) RS_CHAIN(3, 4) RS_CHAIN(3, 8)
    RS_CHAIN(2, 2) RS_CHAIN(2, 4) RS_CHAIN(2, 8)
#undef RS_CHAIN
    if (rc != RS_EUNSUPPORTED) return rc;
  }
  return rs_fail(RS_EUNSUPPORTED, "batched epoch: no thread-block cluster layout fits d = %lld", (long long)d);
}

template int epoch_prep_batched<float, float>(rs_ctx*, const ChainJob<float, float>*, const int64_t*, int, int64_t);
template int epoch_prep_batched<__nv_bfloat16, float>(rs_ctx*, const ChainJob<__nv_bfloat16, float>*, const int64_t*,
                                                      int, int64_t);
template int epoch_chain_batched<float, float>(rs_ctx*, const ChainJob<float, float>*, int, int64_t);
template int epoch_chain_batched<__nv_bfloat16, float>(rs_ctx*, const ChainJob<__nv_bfloat16, float>*, int, int64_t);

// ------------------------------------------------------------------ autotuning of the chain
// Times the inner-loop chain on the components Z for every launch layout that fits (cluster size,
// threads per block, ring stages) on a probe of m steps with the given index stream, and returns
// the fastest.  The block matrices are zero for the probe: the chain's work does not depend on the
// values, and zero keeps every iterate finite.
template <typename S, typename T>
int tune_chain_t(rs_ctx* ctx, const rs_matrix* Z, const uint32_t* idx, int64_t m, TuneEntry* best, int* tried) {
  const int64_t N = Z->n, d = Z->d;
  const S* Zd = static_cast<const S*>(Z->data);
  const int64_t nblk = (m + kBlk - 1) / kBlk;
  T* Rt = static_cast<T*>(rs_scratch(ctx, SCR_R, (size_t)nblk * kBlk * kBlk * sizeof(T)));
  T* cv = static_cast<T*>(rs_scratch(ctx, SCR_C, (size_t)nblk * kBlk * sizeof(T)));
  T* vec = static_cast<T*>(rs_scratch(ctx, SCR_TMPV, 3 * d * sizeof(T)));
  if (!Rt || !cv || !vec) return RS_ENOMEM;
  RS_CUDA_TRY(cudaMemsetAsync(Rt, 0, (size_t)nblk * kBlk * kBlk * sizeof(T), ctx->stream));
  RS_CUDA_TRY(cudaMemsetAsync(cv, 0, (size_t)nblk * kBlk * sizeof(T), ctx->stream));
  RS_CUDA_TRY(cudaMemsetAsync(vec, 0, 3 * d * sizeof(T), ctx->stream));
  const T *mu = vec, *wbar = vec + d;
  T* wnext = vec + 2 * d;
  cudaEvent_t e0, e1;
  RS_CUDA_TRY(cudaEventCreate(&e0));
  RS_CUDA_TRY(cudaEventCreate(&e1));
  best->kind = 0;
  int rc_all = RS_OK;
  for (int cs = 1; cs <= kCsMax && rc_all == RS_OK; cs *= 2) {
    if ((d + cs - 1) / cs > 256) continue;
    for (int nt : {256, 512}) {
      int last_st = 0;
      for (int st = 4; st >= 2; --st) {
        const ChainPlan pl = plan_chain<S, T>(d, cs, 200 * 1024, nt, st);
        if (!pl.cs || pl.stages == last_st) continue;
        last_st = pl.stages;
        float ms_sum = 0.0f;
        int rc = RS_OK;
        for (int rep = 0; rep < 4 && rc == RS_OK; ++rep) {   // one warm-up, three timed
          if (rep == 1) RS_CUDA_TRY(cudaEventRecord(e0, ctx->stream));
          rc = RS_EUNSUPPORTED;
#define RS_TCHAIN(ST, QN, NT)                                                                                      \
  if (pl.stages == ST && pl.qn == QN && pl.nt == NT)                                                               \
    rc = launch_chain<S, T, ST, QN, NT>(ctx, pl, Zd, N, Z->ld, d, idx, m, Rt, cv, 0.0, mu, wbar, 1, wnext,          \
                                        Z->row_scale);
          RS_TCHAIN(4, 2, 256) RS_TCHAIN(4, 4, 256) RS_TCHAIN(4, 8, 256) RS_TCHAIN(3, 2, 256) RS_TCHAIN(3, 4, 256)
          RS_TCHAIN(3, 8, 256) RS_TCHAIN(2, 2, 256) RS_TCHAIN(2, 4, 256) RS_TCHAIN(2, 8, 256)
          RS_TCHAIN(4, 2, 512) RS_TCHAIN(4, 4, 512) RS_TCHAIN(4, 8, 512) RS_TCHAIN(3, 2, 512) RS_TCHAIN(3, 4, 512)
          RS_TCHAIN(3, 8, 512) RS_TCHAIN(2, 2, 512) RS_TCHAIN(2, 4, 512) RS_TCHAIN(2, 8, 512)
#undef RS_TCHAIN
        }
        if (rc == RS_EUNSUPPORTED) continue;   // this cluster shape cannot be placed
        if (rc != RS_OK) {
          rc_all = rc;
          break;
        }
        RS_CUDA_TRY(cudaEventRecord(e1, ctx->stream));
        RS_CUDA_TRY(cudaEventSynchronize(e1));
        RS_CUDA_TRY(cudaEventElapsedTime(&ms_sum, e0, e1));
        ++*tried;
        const float ms = ms_sum / 3.0f;
        if (!best->kind || ms < best->ms) {
          best->kind = TUNE_CHAIN;
          best->dtype = dtype_code<S>();
          best->d = d;
          best->a = pl.cs;
          best->b = pl.nt;
          best->c = pl.stages;
          best->ms = ms;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc_all != RS_OK) return rc_all;
  if (!best->kind) return rs_fail(RS_EUNSUPPORTED, "rs_autotune: no chain layout fits d = %lld", (long long)d);
  return RS_OK;
}
template int tune_chain_t<float, float>(rs_ctx*, const rs_matrix*, const uint32_t*, int64_t, TuneEntry*, int*);
template int tune_chain_t<double, double>(rs_ctx*, const rs_matrix*, const uint32_t*, int64_t, TuneEntry*, int*);
template int tune_chain_t<__nv_bfloat16, float>(rs_ctx*, const rs_matrix*, const uint32_t*, int64_t, TuneEntry*, int*);
template int tune_chain_t<__nv_fp8_e4m3, float>(rs_ctx*, const rs_matrix*, const uint32_t*, int64_t, TuneEntry*, int*);

template int svrg_epoch_t<float, float>(rs_ctx*, const rs_matrix*, int64_t, double, const uint32_t*, const float*,
                                        int64_t, double, const float*, const float*, int, float*);
template int svrg_epoch_t<double, double>(rs_ctx*, const rs_matrix*, int64_t, double, const uint32_t*, const double*,
                                          int64_t, double, const double*, const double*, int, double*);
template int svrg_epoch_t<__nv_bfloat16, float>(rs_ctx*, const rs_matrix*, int64_t, double, const uint32_t*,
                                                const float*, int64_t, double, const float*, const float*, int, float*);
template int svrg_epoch_t<__nv_fp8_e4m3, float>(rs_ctx*, const rs_matrix*, int64_t, double, const uint32_t*,
                                                const float*, int64_t, double, const float*, const float*, int, float*);
