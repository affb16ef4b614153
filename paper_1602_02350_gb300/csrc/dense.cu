// Dense linear algebra of the sketch (Alg. 2) and the preconditioner (Eq. (11)):
// CUDA-core GEMM and split-K Gram kernels, Cholesky-QR, cyclic Jacobi, Rayleigh-Ritz,
// the data transform Z = [X M; M], smoothness constants, the output map w = M w~ and
// the double-precision objective of Eq. (1).
#include <type_traits>

#include "common.cuh"

int countsketch_dispatch(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t s, void* SX, int64_t ld_sx,
                         int32_t* bucket_out, void* sign_out);
int gaussian_dispatch(rs_ctx* ctx, uint64_t seed, int64_t row0, int64_t rows, int64_t cols, int32_t dtype, void* out,
                      int64_t ld);

namespace {

// ------------------------------------------------------------------ GEMM (CUDA cores)
// C[m][n] = alpha * col_scale[n] * sum_k A(m,k) B(k,n) + beta * C0[m][n]
// A(m,k) = A[m*sAm + k*sAk], B(k,n) = B[k*sBk + n*sBn].  64x64 tile, 16-deep k steps, 4x4 per thread.
template <typename T, typename TA, typename TC, typename TC0, bool A_KCONTIG, bool B_NCONTIG>
__global__ void __launch_bounds__(256) gemm_kernel(int64_t M, int64_t N, int64_t K, T alpha, const TA* __restrict__ A,
                                                   int64_t sAm, int64_t sAk, const T* __restrict__ B, int64_t sBk,
                                                   int64_t sBn, T beta, const TC0* C0, int64_t ldc0, TC* C, int64_t ldc,
                                                   const T* __restrict__ col_scale) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid * 4 + q;
      int mm, kk;
      if (A_KCONTIG) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? cvt<T>(A[gm * sAm + gk * sAk]) : T(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid * 4 + q;
      int kk, nn;
      if (B_NCONTIG) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? B[gk * sBk + gn * sBn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      T v = alpha * acc[i][j];
      if (col_scale) v *= col_scale[gn];
      if (C0) v = fma(beta, cvt<T>(C0[gm * ldc0 + gn]), v);
      C[gm * ldc + gn] = cvt<TC>(v);
    }
  }
}

// ------------------------------------------------------------------ split-K Gram
// part[chunk][i][j] = sum over rows r of the chunk of A[r][i] B[r][j]  (TACC accumulation)
template <typename TA, typename TB, typename TACC>
__global__ void __launch_bounds__(256) gram_kernel(int64_t rows, int64_t Ma, int64_t Nb, const TA* __restrict__ A,
                                                   int64_t lda, const TB* __restrict__ B, int64_t ldb,
                                                   int64_t rows_per_chunk, double* part) {
  constexpr int BT = 64, BK = 16;
  __shared__ TACC As[BK][BT + 4];
  __shared__ TACC Bs[BK][BT + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * BT, j0 = (int64_t)blockIdx.x * BT;
  const int64_t chunk = blockIdx.z;
  const int64_t r0 = chunk * rows_per_chunk, r1 = min(rows, r0 + rows_per_chunk);
  TACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = TACC(0);
  for (int64_t rr = r0; rr < r1; rr += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid * 4 + q;
      const int kk = e / BT, ii = e % BT;
      const int64_t r = rr + kk;
      As[kk][ii] = (r < r1 && i0 + ii < Ma) ? cvt<TACC>(A[r * lda + i0 + ii]) : TACC(0);
      Bs[kk][ii] = (r < r1 && j0 + ii < Nb) ? cvt<TACC>(B[r * ldb + j0 + ii]) : TACC(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TACC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* out = part + chunk * Ma * Nb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = i0 + ty * 4 + i;
    if (gi >= Ma) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gj = j0 + tx * 4 + j;
      if (gj < Nb) out[gi * Nb + gj] = (double)acc[i][j];
    }
  }
}

// The same split-K product for float accumulation with 16-byte loads: a 64 x 64 output tile per
// CTA, 32 rows per step staged in shared memory (double-buffered: the next step's tiles are loaded
// into registers while this step's products run).  Rows of A and B must be 16-byte aligned (the
// caller checks); a 16-byte unit that crosses the matrix edge is read element by element.
template <typename TA>
__device__ __forceinline__ void gram_unit_load(const TA* __restrict__ M, int64_t ld, int64_t r, int64_t r1, int64_t c,
                                               int64_t ncol, float* v) {
  constexpr int E = 16 / (int)sizeof(TA);
  if (r >= r1 || c >= ncol) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = 0.0f;
    return;
  }
  const TA* p = M + r * ld + c;
  if (c + E <= ncol) {
    if constexpr (sizeof(TA) == 2) {
      const uint4 q = *reinterpret_cast<const uint4*>(p);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
      }
    } else {
      const float4 q = *reinterpret_cast<const float4*>(p);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = c + e < ncol ? cvt<float>(p[e]) : 0.0f;
  }
}

template <typename TA>
__global__ void __launch_bounds__(256) gram_vec_kernel(int64_t rows, int64_t Ma, int64_t Nb, const TA* __restrict__ A,
                                                       int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                       int64_t rows_per_chunk, double* part) {
  constexpr int BT = 64, BK = 32, LDS = BT + 4;
  constexpr int EA = 16 / (int)sizeof(TA), UA = BK * BT / EA / 256;   // A units per thread (1 or 2)
  constexpr int UB = BK * BT / 4 / 256;                                 // B units per thread (2)
  __shared__ __align__(16) float As[2][BK][LDS];
  __shared__ __align__(16) float Bs[2][BK][LDS];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * BT, j0 = (int64_t)blockIdx.x * BT;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_chunk, r1 = min64(rows, r0 + rows_per_chunk);
  float va[UA][EA], vb[UB][4];
  auto load = [&](int64_t rr) {
#pragma unroll
    for (int q = 0; q < UA; ++q) {
      const int u = tid + 256 * q, kk = u / (BT / EA), cc = (u % (BT / EA)) * EA;
      gram_unit_load<TA>(A, lda, rr + kk, r1, i0 + cc, Ma, va[q]);
    }
#pragma unroll
    for (int q = 0; q < UB; ++q) {
      const int u = tid + 256 * q, kk = u / (BT / 4), cc = (u % (BT / 4)) * 4;
      gram_unit_load<float>(B, ldb, rr + kk, r1, j0 + cc, Nb, vb[q]);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < UA; ++q) {
      const int u = tid + 256 * q, kk = u / (BT / EA), cc = (u % (BT / EA)) * EA;
#pragma unroll
      for (int e = 0; e < EA; e += 4)
        *reinterpret_cast<float4*>(&As[buf][kk][cc + e]) = make_float4(va[q][e], va[q][e + 1], va[q][e + 2], va[q][e + 3]);
    }
#pragma unroll
    for (int q = 0; q < UB; ++q) {
      const int u = tid + 256 * q, kk = u / (BT / 4), cc = (u % (BT / 4)) * 4;
      *reinterpret_cast<float4*>(&Bs[buf][kk][cc]) = make_float4(vb[q][0], vb[q][1], vb[q][2], vb[q][3]);
    }
  };
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  int buf = 0;
  if (r0 < r1) {
    load(r0);
    store(0);
  }
  __syncthreads();
  for (int64_t rr = r0; rr < r1; rr += BK) {
    const bool more = rr + BK < r1;
    if (more) load(rr + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  double* out = part + (int64_t)blockIdx.z * Ma * Nb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = i0 + ty * 4 + i;
    if (gi >= Ma) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gj = j0 + tx * 4 + j;
      if (gj < Nb) out[gi * Nb + gj] = (double)acc[i][j];
    }
  }
}

// G[e] = alpha * sum over the chunks of part[c][e]: 32 entries per block, the chunks split over
// 8 warps (two interleaved partial sums each), then the warps' sums in warp order (deterministic;
// short dependent chains of double adds, which are slow on this GPU)
__global__ void __launch_bounds__(256) reduce_chunks_kernel(const double* part, int64_t nchunks, int64_t count,
                                                            double alpha, double* G) {
  __shared__ double sh[8][33];
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0;
  if (e < count) {
    int64_t c = g;
    for (; c + 8 < nchunks; c += 16) {
      s0 += part[c * count + e];
      s1 += part[(c + 8) * count + e];
    }
    for (; c < nchunks; c += 8) s0 += part[c * count + e];
  }
  sh[g][lane] = s0 + s1;
  __syncthreads();
  if (g == 0 && e < count) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sh[w][lane];
    G[e] = alpha * t;
  }
}

template <typename T>
__global__ void convert_from_double_kernel(const double* in, int64_t count, T* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)in[e];
}

// ------------------------------------------------------------------ Cholesky-QR
// Lower Cholesky factor L of the k x k double matrix G (G = L L^T, right-looking, one block) and
// its inverse L^{-1} (column c by forward substitution, one thread per column), computed in C and
// written as T.  L and the inverse live in shared memory when they fit (buf = nullptr), else in buf.
template <typename T, typename C>
__global__ void chol_inv_kernel(const double* G, int k, C* buf, T* Linv_out, int* status) {
  extern __shared__ __align__(16) unsigned char ci_raw[];
  C* ci_sh = reinterpret_cast<C*>(ci_raw);
  // rows padded to k + 1: column accesses by consecutive threads spread over the banks
  const int LD = k + 1;
  C* L = buf ? buf : ci_sh;
  C* Xi = L + (size_t)k * LD;
  C* dinv = Xi + (size_t)k * LD;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < k * k; e += nt) {
    const int r = e / k, c = e % k;
    L[r * LD + c] = (C)G[e];
    Xi[r * LD + c] = C(0);
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      C v = L[j * LD + j];
      if (!(v > C(0)) || !isfinite(v)) {
        atomicOr(status, 4);
        v = C(1);
      }
      const C r = sqrt(v);
      L[j * LD + j] = r;
      dinv[j] = C(1) / r;
    }
    __syncthreads();
    const C rj = dinv[j];
    for (int i = j + 1 + tid; i < k; i += nt) L[i * LD + j] *= rj;
    __syncthreads();
    const int w = k - j - 1;
    for (int e = tid; e < w * w; e += nt) {
      const int i = j + 1 + e / w, l = j + 1 + e % w;
      if (l <= i) L[i * LD + l] -= L[i * LD + j] * L[l * LD + j];
    }
    __syncthreads();
  }
  // column c of L^{-1} by forward substitution, four interleaved partial sums
  for (int c = tid; c < k; c += nt) {
    Xi[c * LD + c] = dinv[c];
    for (int i = c + 1; i < k; ++i) {
      C s0 = C(0), s1 = C(0), s2 = C(0), s3 = C(0);
      int p = c;
      for (; p + 3 < i; p += 4) {
        s0 = fma(L[i * LD + p], Xi[p * LD + c], s0);
        s1 = fma(L[i * LD + p + 1], Xi[(p + 1) * LD + c], s1);
        s2 = fma(L[i * LD + p + 2], Xi[(p + 2) * LD + c], s2);
        s3 = fma(L[i * LD + p + 3], Xi[(p + 3) * LD + c], s3);
      }
      for (; p < i; ++p) s0 = fma(L[i * LD + p], Xi[p * LD + c], s0);
      Xi[i * LD + c] = -((s0 + s1) + (s2 + s3)) * dinv[i];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) Linv_out[e] = (T)Xi[(e / k) * LD + e % k];
}

// The same factorisation for k up to a few hundred with the packed lower triangle of L in shared
// memory (row i at i (i + 1) / 2), overwritten in place by L^{-1}.  Cholesky by columns (pivot, the
// column scaled into a contiguous buffer, rank-1 update of the trailing triangle by warp rows);
// then the inverse by columns from the last (x = L[j+1:, j] from the buffer, x <- -L^{-1}[j+1:, j+1:]
// x / l_jj by one warp per row with shuffle sums).  Linv_out: Tout, k x k row-major, zero above the
// diagonal.  status bit 4 on a non-positive pivot (replaced by 1).
template <typename C, typename Tout>
__global__ void __launch_bounds__(1024) chol_inv_packed_kernel(const double* __restrict__ G, int k,
                                                               Tout* __restrict__ Linv_out, int* status) {
  extern __shared__ __align__(16) unsigned char cp_raw[];
  C* L = reinterpret_cast<C*>(cp_raw);
  C* col = L + (size_t)k * (k + 1) / 2;   // [k]
  __shared__ C piv;
  const int tid = threadIdx.x, nt = blockDim.x, nw = nt >> 5, wid = tid >> 5, ln = tid & 31;
  auto row = [](int i) { return i * (i + 1) / 2; };
  for (int i = wid; i < k; i += nw)
    for (int j = ln; j <= i; j += 32) L[row(i) + j] = (C)G[(size_t)i * k + j];
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      C v = L[row(j) + j];
      if (!(v > C(0)) || !isfinite(v)) {
        atomicOr(status, 4);
        v = C(1);
      }
      const C r = sqrt(v);
      L[row(j) + j] = r;
      piv = C(1) / r;
    }
    __syncthreads();
    const C rj = piv;
    for (int i = j + 1 + tid; i < k; i += nt) {
      const C v = L[row(i) + j] * rj;
      L[row(i) + j] = v;
      col[i] = v;
    }
    __syncthreads();
    for (int i = j + 1 + wid; i < k; i += nw) {
      const C lij = col[i];
      C* Li = L + row(i);
      for (int l = j + 1 + ln; l <= i; l += 32) Li[l] = fma(-lij, col[l], Li[l]);
    }
    __syncthreads();
  }
  for (int j = k - 1; j >= 0; --j) {
    for (int i = j + 1 + tid; i < k; i += nt) col[i] = L[row(i) + j];
    if (tid == 0) L[row(j) + j] = C(1) / L[row(j) + j];
    __syncthreads();
    const C ajj = -L[row(j) + j];
    for (int i = j + 1 + wid; i < k; i += nw) {
      const C* Li = L + row(i);
      C acc = C(0);
      for (int l = j + 1 + ln; l <= i; l += 32) acc = fma(Li[l], col[l], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (ln == 0) L[row(i) + j] = ajj * acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e % k;
    Linv_out[e] = j <= i ? (Tout)L[row(i) + j] : Tout(0);
  }
}

constexpr size_t kCholPackedMax = 200 * 1024;
template <typename C> size_t chol_packed_bytes(int64_t k) { return ((size_t)k * (k + 1) / 2 + (size_t)k) * sizeof(C); }

// ------------------------------------------------------------------ Jacobi eigensolver
// Cyclic Jacobi with round-robin pairing: each round rotates k/2 disjoint (p,q) planes at once.
// A plane is rotated only if |a_pq| exceeds both tol sqrt|a_pp a_qq| and an absolute floor of a
// few rounding units of ||G||_F; a sweep without rotations ends the iteration.  A and W are in
// shared memory (SMEM) or in global scratch for large k.
template <typename TW, bool SMEM>
__global__ void jacobi_kernel(const double* G, int k, TW* Ag, TW* Wg, double tol, double floor_ulps, int max_sweeps,
                              double* evals, double* Wout) {
  extern __shared__ unsigned char jsh[];
  const int K = (k + 1) & ~1;   // even number of players; index k is a dummy when k is odd
  // rows padded to k + 1 elements: the column updates (consecutive threads on consecutive rows)
  // then fall on distinct shared-memory banks
  const int LD = k + 1;
  TW* A = SMEM ? reinterpret_cast<TW*>(jsh) : Ag;
  TW* W = SMEM ? reinterpret_cast<TW*>(jsh) + (size_t)k * LD : Wg;
  __shared__ int pp[128], qq[128];
  __shared__ TW cc[128], ss[128];
  __shared__ double red[32];
  __shared__ int rotations;
  const int tid = threadIdx.x, nt = blockDim.x;
  double fro = 0.0;
  for (int e = tid; e < k * k; e += nt) {
    const int r = e / k, c = e % k;
    A[r * LD + c] = (TW)G[e];
    W[r * LD + c] = (r == c) ? TW(1) : TW(0);
    fro = fma(G[e], G[e], fro);
  }
  fro = warp_sum(fro);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int w = 0; w < nt / 32; ++w) f += red[w];
    red[0] = sqrt(f);
  }
  __syncthreads();
  const TW abs_floor = (TW)(floor_ulps * red[0] * (sizeof(TW) == 8 ? 0x1p-53 : 0x1p-24));
  const TW rel = (TW)tol;
  const int jt = tid % k, it0 = tid / k, istep = nt / k;   // nt >= 4 k by launch configuration
  const bool active = tid < istep * k;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotations = 0;
    __syncthreads();
    for (int r = 0; r < K - 1; ++r) {
      for (int i = tid; i < K / 2; i += nt) {
        auto pos = [&](int j) {   // round-robin seat of player j in round r (j - 1 + r < 2 (K - 1))
          if (j == 0) return 0;
          const int v = j - 1 + r;
          return (v >= K - 1 ? v - (K - 1) : v) + 1;
        };
        int p = pos(i), q = pos(K - 1 - i);
        if (p > q) { int t = p; p = q; q = t; }
        TW c = TW(1), s = TW(0);
        if (q < k) {
          const TW apq = A[p * LD + q];
          const TW app = A[p * LD + p], aqq = A[q * LD + q];
          // below a few rounding units of the larger diagonal entry a rotation only stirs
          // rounding noise (graded spectra would otherwise rotate until the sweep limit)
          const TW noise = TW(4) * (sizeof(TW) == 8 ? TW(0x1p-53) : TW(0x1p-24)) * fmax(fabs(app), fabs(aqq));
          const TW thr = fmax(fmax(rel * sqrt(fabs(app * aqq)), abs_floor), noise);
          if (fabs(apq) > thr) {
            const TW theta = (aqq - app) / (TW(2) * apq);
            const TW t = (theta >= TW(0) ? TW(1) : TW(-1)) / (fabs(theta) + sqrt(theta * theta + TW(1)));
            c = TW(1) / sqrt(t * t + TW(1));
            s = t * c;
            rotations = 1;   // any rotation in this sweep (every writer stores the same value)
          }
        }
        pp[i] = p; qq[i] = q; cc[i] = c; ss[i] = s;
      }
      __syncthreads();
      // rows: A <- J^T A   (thread owns column j = jt of pairs it0, it0 + istep, ...)
      if (active)
        for (int i = it0; i < K / 2; i += istep) {
          const int p = pp[i], q = qq[i];
          const TW c = cc[i], s = ss[i];
          if (q >= k || s == TW(0)) continue;
          const int j = jt;
          const TW ap = A[p * LD + j], aq = A[q * LD + j];
          A[p * LD + j] = c * ap - s * aq;
          A[q * LD + j] = s * ap + c * aq;
        }
      __syncthreads();
      // columns: A <- A J, W <- W J   (thread owns row j = jt)
      if (active)
        for (int i = it0; i < K / 2; i += istep) {
        const int j = jt;
        const int p = pp[i], q = qq[i];
        const TW c = cc[i], s = ss[i];
        if (q >= k || s == TW(0)) continue;
        const TW ap = A[j * LD + p], aq = A[j * LD + q];
        A[j * LD + p] = c * ap - s * aq;
        A[j * LD + q] = s * ap + c * aq;
        const TW wp = W[j * LD + p], wq = W[j * LD + q];
        W[j * LD + p] = c * wp - s * wq;
        W[j * LD + q] = s * wp + c * wq;
      }
      __syncthreads();
    }
    const int done = rotations == 0;   // read after the round's final barrier
    __syncthreads();
    if (done) break;
  }
  // sort descending (stable in index) and write out
  for (int i = tid; i < k; i += nt) {
    const TW ev = A[i * LD + i];
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const TW ej = A[j * LD + j];
      rank += (ej > ev) || (ej == ev && j < i);
    }
    evals[rank] = (double)ev;
    for (int r = 0; r < k; ++r) Wout[r * k + rank] = (double)W[r * LD + i];
  }
}

// Cyclic Jacobi in float on the packed lower triangle of A (k (k+1) / 2 floats in shared memory, so
// k up to 320 fits one CTA), with the same round-robin pairing and rotation thresholds as
// jacobi_kernel.  A round is one pass: the K/2 disjoint rotations are chosen (first barrier), then
// every 2 x 2 block A[(p_a, q_a), (p_b, q_b)] with a >= b is rotated from both sides by one thread
// (second barrier): the diagonal blocks take the closed form a_pp - t a_pq, a_qq + t a_pq, 0 and
// the others R_a M R_b^T.  The eigenvectors are not formed here: every round's rotations (p, q, c, s)
// are logged to global memory and jacobi_apply_kernel replays them onto the identity afterwards,
// many rows in parallel.  evals0 receives the diagonal (unsorted), *nsweeps the sweeps run.
__device__ __forceinline__ int tri_idx(int i, int j) {   // packed lower triangle, any order of (i, j)
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

__global__ void __launch_bounds__(1024) jacobi_packed_kernel(const double* __restrict__ G, int k, float tol,
                                                             double floor_ulps, int max_sweeps,
                                                             float4* __restrict__ rot_log, int* __restrict__ nsweeps,
                                                             double* __restrict__ evals0) {
  extern __shared__ float jp_sh[];
  float* A = jp_sh;
  const int K = (k + 1) & ~1;
  const int P = K / 2;
  __shared__ int pp[160], qq[160];
  __shared__ float cc[160], ss[160], tt[160];
  __shared__ double red[32];
  __shared__ int rotations;
  // pairs that rotate in the current round (compacted; their order does not matter, every 2 x 2 block
  // is updated exactly once from its old values), double-buffered counts
  __shared__ int act[160], isact[160], nact[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  double fro = 0.0;
  for (int e = tid; e < k * (k + 1) / 2; e += nt) {
    int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    const int j = e - i * (i + 1) / 2;
    const double g = G[(size_t)i * k + j];
    A[e] = (float)g;
    fro = fma(i == j ? g : 2.0 * g, g, fro);   // off-diagonal entries count twice in ||G||_F^2
  }
  fro = warp_sum(fro);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int w = 0; w < nt / 32; ++w) f += red[w];
    red[0] = sqrt(f);
  }
  __syncthreads();
  const float abs_floor = (float)(floor_ulps * red[0] * 0x1p-24);
  if (tid == 0) nact[0] = nact[1] = 0;
  int sweep = 0;
  int rnd = 0;   // rounds run so far (selects the count buffer)
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotations = 0;
    __syncthreads();
    for (int r = 0; r < K - 1; ++r, ++rnd) {
      float4* log_r = rot_log + ((size_t)sweep * (K - 1) + r) * P;
      const int cb_now = rnd & 1;
      if (tid == 0) nact[cb_now ^ 1] = 0;   // the next round's count (the previous round read it)
      for (int i = tid; i < P; i += nt) {
        auto pos = [&](int j) {   // round-robin seat of player j in round r
          if (j == 0) return 0;
          const int v = j - 1 + r;
          return (v >= K - 1 ? v - (K - 1) : v) + 1;
        };
        int p = pos(i), q = pos(K - 1 - i);
        if (p > q) { const int t2 = p; p = q; q = t2; }
        float c = 1.0f, sn = 0.0f, t = 0.0f;
        if (q < k) {
          const float apq = A[tri_idx(q, p)], app = A[tri_idx(p, p)], aqq = A[tri_idx(q, q)];
          const float noise = 4.0f * 0x1p-24f * fmaxf(fabsf(app), fabsf(aqq));
          const float thr = fmaxf(fmaxf(tol * sqrtf(fabsf(app * aqq)), abs_floor), noise);
          if (fabsf(apq) > thr) {
            const float theta = (aqq - app) / (2.0f * apq);
            t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
            c = 1.0f / sqrtf(t * t + 1.0f);
            sn = t * c;
            rotations = 1;
          }
        }
        pp[i] = p; qq[i] = q; cc[i] = c; ss[i] = sn; tt[i] = t;
        isact[i] = sn != 0.0f;
        if (sn != 0.0f) act[atomicAdd(&nact[cb_now], 1)] = i;
        log_r[i] = make_float4(__int_as_float(p), __int_as_float(q), c, sn);
      }
      __syncthreads();
      const int na = nact[cb_now];
      if (na == 0) continue;   // nothing rotates in this round (uniform: read after the barrier)
      // every 2 x 2 block (a, b), b <= a, of the round's planes, rotated from both sides from its old values
      auto upd = [&](int a, int b) {
        const int pa = pp[a], qa = qq[a], pb = pp[b], qb = qq[b];
        if (qa >= k || qb >= k) {
          // a dummy player (odd k): only the real rotation acts; rows/columns of the dummy do not exist
          if (a == b || (qa >= k && qb >= k)) return;
        }
        const float sa = ss[a], sb = ss[b];
        if (sa == 0.0f && sb == 0.0f) return;
        if (a == b) {
          const int ipq = tri_idx(qa, pa);
          const float apq = A[ipq], t = tt[a];
          A[tri_idx(pa, pa)] -= t * apq;
          A[tri_idx(qa, qa)] += t * apq;
          A[ipq] = 0.0f;
          return;
        }
        const float ca = cc[a], cb = cc[b];
        // M = [A(pa, pb) A(pa, qb); A(qa, pb) A(qa, qb)], rows of a dummy player are absent
        const bool ra = qa < k, rb = qb < k;
        const int i00 = tri_idx(pa, pb);
        const int i01 = rb ? tri_idx(pa, qb) : -1;
        const int i10 = ra ? tri_idx(qa, pb) : -1;
        const int i11 = (ra && rb) ? tri_idx(qa, qb) : -1;
        const float m00 = A[i00], m01 = rb ? A[i01] : 0.0f, m10 = ra ? A[i10] : 0.0f, m11 = (ra && rb) ? A[i11] : 0.0f;
        // rows (R_a): p' = c p - s q, q' = s p + c q
        const float r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;
        const float r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
        // columns (R_b)
        A[i00] = cb * r00 - sb * r01;
        if (rb) A[i01] = sb * r00 + cb * r01;
        if (ra) A[i10] = cb * r10 - sb * r11;
        if (ra && rb) A[i11] = sb * r10 + cb * r11;
      };
      if (2 * na <= P) {
        // few rotating pairs: only the blocks of a row or column of one of them
        for (int bi = tid; bi < na * P; bi += nt) {
          const int a = act[bi / P], b = bi % P;
          if (isact[b] && b > a) continue;   // both rotate: the block is taken from b's list
          upd(a, b);
        }
      } else {
        // every block: warp w takes the rows a = w, w + 32, ... of the triangle (equal numbers of
        // 32-wide column passes per warp), lanes the columns b <= a.  A lane's columns b = lane + 32 t
        // are the same for every row, so their planes and rotations are read once per round into
        // registers, and each row's once per row: the block update is then shared-memory traffic on
        // A alone.
        const int nw = nt >> 5, wid = tid >> 5, ln = tid & 31;
        constexpr int TB = 5;   // P <= 160
        int pbv[TB], qbv[TB];
        float cbv[TB], sbv[TB];
#pragma unroll
        for (int t = 0; t < TB; ++t) {
          const int b = ln + 32 * t;
          const bool in = b < P;
          pbv[t] = in ? pp[b] : 0;
          qbv[t] = in ? qq[b] : 0;
          cbv[t] = in ? cc[b] : 1.0f;
          sbv[t] = in ? ss[b] : 0.0f;
        }
        for (int a = wid; a < P; a += nw) {
          const int pa = pp[a], qa = qq[a];
          const float ca = cc[a], sa = ss[a], ta = tt[a];
          const bool ra = qa < k;
#pragma unroll
          for (int t = 0; t < TB; ++t) {
            const int b = ln + 32 * t;
            if (b > a) break;
            const int pb = pbv[t], qb = qbv[t];
            const float cb = cbv[t], sb = sbv[t];
            if ((!ra || qb >= k) && (a == b || (!ra && qb >= k))) continue;   // dummy player (odd k)
            if (sa == 0.0f && sb == 0.0f) continue;
            if (a == b) {
              const int ipq = tri_idx(qa, pa);
              const float apq = A[ipq];
              A[tri_idx(pa, pa)] -= ta * apq;
              A[tri_idx(qa, qa)] += ta * apq;
              A[ipq] = 0.0f;
              continue;
            }
            const bool rb = qb < k;
            const int i00 = tri_idx(pa, pb);
            const int i01 = rb ? tri_idx(pa, qb) : -1;
            const int i10 = ra ? tri_idx(qa, pb) : -1;
            const int i11 = (ra && rb) ? tri_idx(qa, qb) : -1;
            const float m00 = A[i00], m01 = rb ? A[i01] : 0.0f, m10 = ra ? A[i10] : 0.0f,
                        m11 = (ra && rb) ? A[i11] : 0.0f;
            const float r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;
            const float r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
            A[i00] = cb * r00 - sb * r01;
            if (rb) A[i01] = sb * r00 + cb * r01;
            if (ra) A[i10] = cb * r10 - sb * r11;
            if (ra && rb) A[i11] = sb * r10 + cb * r11;
          }
        }
      }
      __syncthreads();
    }
    const int done = rotations == 0;
    __syncthreads();
    if (done) {
      ++sweep;
      break;
    }
  }
  if (tid == 0) *nsweeps = sweep;
  for (int i = tid; i < k; i += nt) evals0[i] = (double)A[tri_idx(i, i)];
}

// W = product of the logged Jacobi rotations applied to the identity, in the logged order: row j
// of W takes (w_p, w_q) <- (c w_p - s w_q, s w_p + c w_q) for every rotation.  CTA = 8 rows of W in
// shared memory; thread (row, pair) applies one rotation of each round, rounds separated by a
// barrier (the rotations of a round act on disjoint columns).  Wout: double, k x k row-major.
constexpr int kJaRows = 8;
__global__ void __launch_bounds__(1024) jacobi_apply_kernel(const float4* __restrict__ rot_log,
                                                            const int* __restrict__ nsweeps, int k,
                                                            double* __restrict__ Wout) {
  extern __shared__ float ja_sh[];
  const int K = (k + 1) & ~1, P = K / 2, LDW = k + 1;
  const int row0 = blockIdx.x * kJaRows;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < kJaRows * LDW; e += nt) {
    const int rr = e / LDW, c = e % LDW;
    ja_sh[e] = (row0 + rr == c) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int rr = tid / P, a = tid % P;
  const bool active = rr < kJaRows && row0 + rr < k;
  const int64_t rounds = (int64_t)(*nsweeps) * (K - 1);
  float* wrow = ja_sh + rr * LDW;
  float4 cur = (active && rounds > 0) ? rot_log[a] : make_float4(0.f, 0.f, 1.f, 0.f);
  for (int64_t r = 0; r < rounds; ++r) {
    const float4 nxt = (active && r + 1 < rounds) ? rot_log[(r + 1) * P + a] : make_float4(0.f, 0.f, 1.f, 0.f);
    if (active && cur.w != 0.0f) {
      const int p = __float_as_int(cur.x), q = __float_as_int(cur.y);
      if (q < k) {
        const float wp = wrow[p], wq = wrow[q];
        wrow[p] = cur.z * wp - cur.w * wq;
        wrow[q] = cur.w * wp + cur.z * wq;
      }
    }
    cur = nxt;
    __syncthreads();
  }
  for (int e = tid; e < kJaRows * k; e += nt) {
    const int r2 = e / k, c = e % k;
    if (row0 + r2 < k) Wout[(size_t)(row0 + r2) * k + c] = (double)ja_sh[r2 * LDW + c];
  }
}

// Rayleigh quotients lambda_j = w_j^T G w_j / w_j^T w_j in double (one block per vector): turns
// float Jacobi eigenvectors (orthonormal to ~1e-6) into eigenvalues accurate to ~1e-12.
__global__ void rayleigh_kernel(const double* G, int k, const double* W, double* lam) {
  __shared__ double sh[2][32];
  const int j = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    double gw = 0.0;
    for (int c = 0; c < k; ++c) gw = fma(G[r * k + c], W[c * k + j], gw);
    const double wr = W[r * k + j];
    num = fma(wr, gw, num);
    den = fma(wr, wr, den);
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = num; sh[1][threadIdx.x >> 5] = den; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) { a += sh[0][w2]; b += sh[1][w2]; }
    lam[j] = a / b;
  }
}

// sort (lam, columns of W) descending by lam, stable in the column index
__global__ void sort_eig_kernel(const double* lam, const double* W, int k, double* evals, double* Wout) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double ev = lam[i];
    int rank = 0;
    for (int j = 0; j < k; ++j) rank += (lam[j] > ev) || (lam[j] == ev && j < i);
    evals[rank] = ev;
    for (int r = 0; r < k; ++r) Wout[r * k + rank] = W[r * k + i];
  }
}

// ------------------------------------------------------------------ preconditioner pieces
template <typename T>
__global__ void adiag_kernel(const double* sigma2, int k, double lam, T* a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) a[j] = (T)(1.0 - sqrt((sigma2[k - 1] + lam) / (sigma2[j] + lam)));
}

template <typename T>
__global__ void scale_cols_kernel(const T* V, int64_t d, int k, const T* a, T* Va) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d * k; e += (int64_t)gridDim.x * blockDim.x)
    Va[e] = V[e] * a[e % k];
}

template <typename T>
__global__ void identity_rows_kernel(T* Z, int64_t d, int64_t ld) {   // T: storage type
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d * d; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d, c = e % d;
    Z[r * ld + c] = cvt<T>((r == c) ? 1.0f : 0.0f);
  }
}

// beta_i = gamma_i ||z_i||^2; warp per row; per-block partial sums of beta for beta_hat
template <typename S, typename T>
__global__ void row_beta_kernel(const S* Z, int64_t N, int64_t n, int64_t d, int64_t ld, double lam, T* beta,
                                double* part) {
  // a warp takes two rows at a time; lanes read 16-byte units (rows are 16-byte aligned)
  constexpr int EU = 16 / (int)sizeof(S);
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double acc_blk = 0.0;
  const double gd = (double)N / (double)n, gr = lam * (double)N;
  const int64_t nu = (d + EU - 1) / EU;
  for (int64_t i0 = ((int64_t)blockIdx.x * nw + warp) * 2; i0 < N; i0 += (int64_t)gridDim.x * nw * 2) {
    T s[2] = {T(0), T(0)};
    for (int64_t u = lane; u < nu; u += 32) {
      const int64_t c0 = u * EU;
      S v[2][EU];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int64_t i = i0 + k;
        if (i >= N) {
#pragma unroll
          for (int e = 0; e < EU; ++e) v[k][e] = S(0.0f);
        } else if (c0 + EU <= d) {
          *reinterpret_cast<uint4*>(v[k]) = *reinterpret_cast<const uint4*>(Z + i * ld + c0);
        } else {
#pragma unroll
          for (int e = 0; e < EU; ++e) v[k][e] = c0 + e < d ? Z[i * ld + c0 + e] : S(0.0f);
        }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int e = 0; e < EU; ++e) {
          const T x = cvt<T>(v[k][e]);
          s[k] = fma(x, x, s[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t i = i0 + k;
      const T t = warp_sum(s[k]);
      if (i < N && lane == 0) {
        const double b = (i < n ? gd : gr) * (double)t;
        beta[i] = (T)b;
        acc_blk += b;
      }
    }
  }
  if (lane == 0) sh[warp] = acc_blk;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// beta_i with the data rows' squared norms already formed (rowsq, by the tensor-core components
// kernel): a thread per data row, a warp per regulariser row (read from Z), and the block's sum
// of beta in double for the mean.
template <typename S, typename T>
__global__ void row_beta_sq_kernel(const float* __restrict__ rowsq, const S* Z, int64_t N, int64_t n, int64_t d,
                                   int64_t ld, double lam, T* beta, double* part) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double gd = (double)N / (double)n, gr = lam * (double)N;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double b = gd * (double)rowsq[i];
    beta[i] = (T)b;
    acc += b;
  }
  for (int64_t i = n + (int64_t)blockIdx.x * nw + warp; i < N; i += (int64_t)gridDim.x * nw) {
    T s = T(0);
    for (int64_t c = lane; c < d; c += 32) {
      const T v = cvt<T>(Z[i * ld + c]);
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      const double b = gr * (double)s;
      beta[i] = (T)b;
      acc += b;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// out = scale * sum of part[0..np): lane-strided partial sums, then a fixed shuffle tree
__global__ void sum_parts_kernel(const double* part, int np, double scale, double* out) {
  double s = 0.0;
  for (int p = threadIdx.x; p < np; p += 32) s += part[p];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = s * scale;
}

// w[c] = wt[c] - sum_j V[c][j] a_j t_j with t = V^T wt (double)
template <typename T>
__global__ void map_output_kernel(const T* V, int64_t d, int k, const T* a, const double* t, const T* wt, T* w) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d; c += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += (double)V[c * k + j] * (double)a[j] * t[j];
    w[c] = (T)((double)wt[c] - s);
  }
}

// ------------------------------------------------------------------ objective (double)
template <typename TS, typename T>
__global__ void objective_kernel(const TS* X, int64_t n, int64_t d, int64_t ld, const T* y, const T* w, const T* wr,
                                 double* part) {
  __shared__ double sh[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double r2 = 0.0, e2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < n; i += (int64_t)gridDim.x * nw) {
    double sw = 0.0, se = 0.0;
    for (int64_t c = lane; c < d; c += 32) {
      const double x = cvt<double>(X[i * ld + c]);
      const double wc = (double)w[c];
      sw = fma(x, wc, sw);
      if (wr) se = fma(x, wc - (double)wr[c], se);
    }
    sw = warp_sum(sw);
    se = warp_sum(se);
    const double r = sw - (double)y[i];
    r2 = fma(r, r, r2);
    e2 = fma(se, se, e2);
  }
  if (lane == 0) { sh[0][warp] = r2; sh[1][warp] = e2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) { a += sh[0][w2]; b += sh[1][w2]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

template <typename T>
__global__ void objective_finish_kernel(const double* part, int np, int64_t n, int64_t d, double lam, const T* w,
                                        const T* wr, double* out) {
  __shared__ double sh[2][32];
  double ww = 0.0, ee = 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
    const double wc = (double)w[c];
    ww = fma(wc, wc, ww);
    if (wr) {
      const double e = wc - (double)wr[c];
      ee = fma(e, e, ee);
    }
  }
  ww = warp_sum(ww);
  ee = warp_sum(ee);
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = ww; sh[1][threadIdx.x >> 5] = ee; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, r2 = 0.0, e2 = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) { a += sh[0][w2]; b += sh[1][w2]; }
    for (int p = 0; p < np; ++p) { r2 += part[2 * p]; e2 += part[2 * p + 1]; }
    out[0] = 0.5 * r2 / (double)n + 0.5 * lam * a;
    out[1] = wr ? 0.5 * e2 / (double)n + 0.5 * lam * b : 0.0;
  }
}

// ||X||_F^2: each lane sums its part of a row in float (a few dozen terms), the row and block sums
// are accumulated in double; per-block partials are summed in block order by trace_finish
template <typename TS>
__global__ void sumsq_kernel(const TS* X, int64_t n, int64_t d, int64_t ld, double* part) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < n; i += (int64_t)gridDim.x * nw) {
    if constexpr (sizeof(TS) == 8) {
      for (int64_t c = lane; c < d; c += 32) {
        const double x = cvt<double>(X[i * ld + c]);
        a = fma(x, x, a);
      }
    } else {
      float r = 0.0f;
      for (int64_t c = lane; c < d; c += 32) {
        const float x = cvt<float>(X[i * ld + c]);
        r = fmaf(x, x, r);
      }
      a += (double)r;
    }
  }
  a = warp_sum(a);
  if (lane == 0) sh[warp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) t += sh[w2];
    part[blockIdx.x] = t;
  }
}

__global__ void trace_finish_kernel(const double* part, int np, double inv_n, double* out) {
  // lane-strided partial sums, then a fixed shuffle tree (one warp)
  double t = 0.0;
  for (int p = threadIdx.x; p < np; p += 32) t += part[p];
  t = warp_sum(t);
  if (threadIdx.x == 0) *out = t * inv_n;
}

// w = M x = x - V diag(a) V^T x in one block (a_j = 1 - D'_j from sigma2): partial sums of V^T x by
// (column, row-group), a fixed-order combine, then each thread forms its entries of w.  A is the
// accumulation type (double for double data).
template <typename T, typename A>
__global__ void __launch_bounds__(1024) map_fused_kernel(const T* __restrict__ V, const double* __restrict__ sigma2,
                                                         int64_t d, int k, double lam, const T* __restrict__ x,
                                                         T* __restrict__ y) {
  __shared__ A part[1024];
  __shared__ A tv[256];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int G = nt / k;                    // row groups (k <= 256 so G >= 4)
  const int j = tid % k, g = tid / k;
  if (g < G) {
    A s = A(0);
    for (int64_t c = g; c < d; c += G) s += (A)V[c * k + j] * (A)x[c];
    part[g * k + j] = s;
  }
  __syncthreads();
  if (tid < k) {
    A t = A(0);
    for (int q = 0; q < G; ++q) t += part[q * k + tid];   // fixed order
    const double a = 1.0 - sqrt((sigma2[k - 1] + lam) / (sigma2[tid] + lam));
    tv[tid] = (A)a * t;
  }
  __syncthreads();
  for (int64_t c = tid; c < d; c += nt) {
    const T* v = V + c * k;
    A s0 = A(0), s1 = A(0);
    int q = 0;
    for (; q + 1 < k; q += 2) {
      s0 += (A)v[q] * tv[q];
      s1 += (A)v[q + 1] * tv[q + 1];
    }
    if (q < k) s0 += (A)v[q] * tv[q];
    y[c] = (T)((A)x[c] - (s0 + s1));
  }
}

// The same map over many blocks for larger d: t_j = sum_c V_cj x_c as partial sums over row ranges
// (block b takes rows [b R, b R + R), thread j column j), a one-block combine in range order that
// also applies a_j, then y_c = x_c - sum_j V_cj (a t)_j with one warp per row (lanes over j, fixed
// shuffle tree).
template <typename T>
__global__ void __launch_bounds__(256) map_tpart_kernel(const T* __restrict__ V, int64_t d, int k, int64_t R,
                                                        const T* __restrict__ x, T* __restrict__ part) {
  const int64_t c0 = blockIdx.x * R, c1 = min64(d, c0 + R);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    T s0 = T(0), s1 = T(0);
    int64_t c = c0;
    for (; c + 1 < c1; c += 2) {
      s0 = fma(V[c * k + j], x[c], s0);
      s1 = fma(V[(c + 1) * k + j], x[c + 1], s1);
    }
    if (c < c1) s0 = fma(V[c * k + j], x[c], s0);
    part[(int64_t)blockIdx.x * k + j] = s0 + s1;
  }
}

template <typename T>
__global__ void map_tsum_kernel(const T* __restrict__ part, int P, int k, const double* __restrict__ sigma2,
                                double lam, T* __restrict__ tv) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    T t = T(0);
    for (int p = 0; p < P; ++p) t += part[(int64_t)p * k + j];   // range order
    tv[j] = (T)(1.0 - sqrt((sigma2[k - 1] + lam) / (sigma2[j] + lam))) * t;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) map_apply_kernel(const T* __restrict__ V, int64_t d, int k,
                                                        const T* __restrict__ tv, const T* __restrict__ x,
                                                        T* __restrict__ y) {
  __shared__ T ts[256];
  for (int j = threadIdx.x; j < k; j += blockDim.x) ts[j] = tv[j];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= d) return;
  const T* v = V + c * k;
  T s = T(0);
  for (int j = lane; j < k; j += 32) s = fma(v[j], ts[j], s);
  s = warp_sum(s);
  if (lane == 0) y[c] = x[c] - s;
}

// mean of a float vector in double (one block)
__global__ void mean_f_kernel(const float* v, int64_t N, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += (double)v[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t / (double)N;
  }
}

// FP8-e4m3 components with per-row scales: s_i = max_c |z_ic| / 448 (1 for a zero row), code_ic =
// e4m3(z_ic / s_i) (round to nearest, saturating), and beta_i = gamma_i s_i^2 sum_c code_ic^2 from the
// stored values.  One warp per row of the bfloat16 staging copy.
__global__ void quantize_fp8_rows_kernel(const __nv_bfloat16* __restrict__ Zb, int64_t N, int64_t n, int64_t d,
                                         int64_t ldb, double lam, __nv_fp8_e4m3* __restrict__ Zq, int64_t ldq,
                                         float* __restrict__ scale, float* __restrict__ beta) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double gd = (double)N / (double)n, gr = lam * (double)N;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < N; i += (int64_t)gridDim.x * nw) {
    const __nv_bfloat16* row = Zb + i * ldb;
    float mx = 0.0f;
    for (int64_t c = lane; c < d; c += 32) mx = fmaxf(mx, fabsf(__bfloat162float(row[c])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float sc = mx > 0.0f ? mx / 448.0f : 1.0f;
    const float inv = 1.0f / sc;
    float ss = 0.0f;
    for (int64_t c = lane; c < d; c += 32) {
      const __nv_fp8_e4m3 q(__bfloat162float(row[c]) * inv);
      Zq[i * ldq + c] = q;
      const float v = static_cast<float>(q);
      ss = fmaf(v, v, ss);
    }
    ss = warp_sum(ss);
    if (lane == 0) {
      scale[i] = sc;
      beta[i] = (float)((i < n ? gd : gr) * (double)sc * (double)sc * (double)ss);
    }
  }
}

int blocks_for(rs_ctx* ctx, int64_t work, int threads = 256) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ====================================================================== launchers

template <typename T, typename TA, typename TC, typename TC0>
int launch_gemm(rs_ctx* ctx, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t sAm, int64_t sAk,
                const T* B, int64_t sBk, int64_t sBn, double beta, const typename NoDeduce<TC0>::type* C0, int64_t ldc0,
                TC* C, int64_t ldc, const T* col_scale) {
  if (M <= 0 || N <= 0) return RS_OK;
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
  if (grid.y > 65535) return rs_fail(RS_EINVAL, "gemm: M = %lld too large", (long long)M);
  const bool ak = (sAk == 1), bn = (sBn == 1);
  if (ak && bn)
    gemm_kernel<T, TA, TC, TC0, true, true><<<grid, 256, 0, ctx->stream>>>(M, N, K, (T)alpha, A, sAm, sAk, B, sBk, sBn, (T)beta,
                                                              C0, ldc0, C, ldc, col_scale);
  else if (ak)
    gemm_kernel<T, TA, TC, TC0, true, false><<<grid, 256, 0, ctx->stream>>>(M, N, K, (T)alpha, A, sAm, sAk, B, sBk, sBn, (T)beta,
                                                               C0, ldc0, C, ldc, col_scale);
  else if (bn)
    gemm_kernel<T, TA, TC, TC0, false, true><<<grid, 256, 0, ctx->stream>>>(M, N, K, (T)alpha, A, sAm, sAk, B, sBk, sBn, (T)beta,
                                                               C0, ldc0, C, ldc, col_scale);
  else
    gemm_kernel<T, TA, TC, TC0, false, false><<<grid, 256, 0, ctx->stream>>>(M, N, K, (T)alpha, A, sAm, sAk, B, sBk, sBn,
                                                                (T)beta, C0, ldc0, C, ldc, col_scale);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}
#define RS_GEMM_INST(T, TA, TC, TC0)                                                                               \
  template int launch_gemm<T, TA, TC, TC0>(rs_ctx*, int64_t, int64_t, int64_t, double, const TA*, int64_t, int64_t,   \
                                           const T*, int64_t, int64_t, double, const typename NoDeduce<TC0>::type*,    \
                                           int64_t, TC*, int64_t, const T*);
RS_GEMM_INST(float, float, float, float)
RS_GEMM_INST(double, double, double, double)
RS_GEMM_INST(float, __nv_bfloat16, float, float)
RS_GEMM_INST(float, float, __nv_bfloat16, __nv_bfloat16)
RS_GEMM_INST(float, float, __nv_bfloat16, float)
RS_GEMM_INST(double, float, float, float)
#undef RS_GEMM_INST

template <typename TA, typename TB>
int launch_gram(rs_ctx* ctx, int64_t rows, int64_t Ma, int64_t Nb, const TA* A, int64_t lda, const TB* B, int64_t ldb,
                double alpha, double* G) {
  using TACC = typename std::conditional<sizeof(TA) == 8, double, float>::type;
  const int64_t tiles = ((Ma + 63) / 64) * ((Nb + 63) / 64);
  // enough row chunks to fill the GPU; at most 512 rows per chunk in float
  int64_t target = std::max<int64_t>(1, (int64_t)ctx->num_sms * 4 / tiles);
  int64_t rpc = std::max<int64_t>(64, (rows + target - 1) / target);
  if (sizeof(TACC) == 4) rpc = std::min<int64_t>(rpc, 512);
  rpc = (rpc + 15) / 16 * 16;
  const int64_t nchunks = (rows + rpc - 1) / rpc;
  double* part = static_cast<double*>(rs_scratch(ctx, SCR_PART, nchunks * Ma * Nb * sizeof(double)));
  if (!part) return RS_ENOMEM;
  if (nchunks > 65535) return rs_fail(RS_EINVAL, "gram: too many row chunks");
  dim3 grid((unsigned)((Nb + 63) / 64), (unsigned)((Ma + 63) / 64), (unsigned)nchunks);
  bool vec = false;
  if constexpr (std::is_same<TACC, float>::value && std::is_same<TB, float>::value)
    vec = (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0 &&
          (lda * (int64_t)sizeof(TA)) % 16 == 0 && (ldb * (int64_t)sizeof(TB)) % 16 == 0;
  if (vec) {
    if constexpr (std::is_same<TACC, float>::value && std::is_same<TB, float>::value)
      gram_vec_kernel<TA><<<grid, 256, 0, ctx->stream>>>(rows, Ma, Nb, A, lda, B, ldb, rpc, part);
  } else {
    gram_kernel<TA, TB, TACC><<<grid, 256, 0, ctx->stream>>>(rows, Ma, Nb, A, lda, B, ldb, rpc, part);
  }
  RS_LAUNCH_CHECK(ctx);
  const int64_t rblocks = (Ma * Nb + 31) / 32;
  if (rblocks > 0x7FFFFFFF) return rs_fail(RS_EINVAL, "gram: output too large");
  reduce_chunks_kernel<<<(unsigned)rblocks, 256, 0, ctx->stream>>>(part, nchunks, Ma * Nb, alpha, G);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}
#define RS_GRAM_INST(TA, TB)                                                                                     \
  template int launch_gram<TA, TB>(rs_ctx*, int64_t, int64_t, int64_t, const TA*, int64_t, const TB*, int64_t,    \
                                   double, double*);
RS_GRAM_INST(float, float)
RS_GRAM_INST(double, double)
RS_GRAM_INST(__nv_bfloat16, float)
RS_GRAM_INST(__nv_bfloat16, __nv_bfloat16)
#undef RS_GRAM_INST

template <typename T>
static int to_T(rs_ctx* ctx, const double* in, int64_t count, T* out) {
  convert_from_double_kernel<T><<<blocks_for(ctx, count), 256, 0, ctx->stream>>>(in, count, out);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

namespace {

// E = S - I (k x k, double)
__global__ void minus_identity_kernel(const double* __restrict__ S, int k, double* __restrict__ E) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x)
    E[e] = S[e] - (e / k == e % k ? 1.0 : 0.0);
}
// T = I - E / 2 + 3 E^2 / 8: the inverse square root of S = I + E to O(|E|^3)
__global__ void inv_sqrt_series_kernel(const double* __restrict__ E, const double* __restrict__ E2, int k,
                                       double* __restrict__ T) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x)
    T[e] = (e / k == e % k ? 1.0 : 0.0) - 0.5 * E[e] + 0.375 * E2[e];
}
// G <- (G + G^T) / 2
__global__ void symmetrize_kernel(double* G, int k) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e % k;
    if (i < j) {
      const double v = 0.5 * (G[i * k + j] + G[j * k + i]);
      G[i * k + j] = v;
      G[j * k + i] = v;
    }
  }
}

}  // namespace

int run_sym_eig(rs_ctx* ctx, const double* G, int64_t k, int32_t prec, double* evals, double* W) {
  if (k < 1 || k > 256) return rs_fail(RS_EINVAL, "sym_eig: k = %lld outside [1, 256]", (long long)k);
  const size_t es = prec == RS_F64 ? 8 : 4;
  const size_t bytes = 2 * (size_t)k * (k + 1) * es;   // rows padded to k + 1
  const bool smem = bytes <= 200 * 1024;
  void* g = nullptr;
  if (!smem) {
    g = rs_scratch(ctx, SCR_EIG, bytes);
    if (!g) return RS_ENOMEM;
  }
  const int threads = k <= 16 ? 256 : 1024;   // at least 4 k threads (one column per thread per pair group)
  const size_t shm = smem ? bytes : 0;
  if (prec == RS_F64) {
    double* Ag = static_cast<double*>(g);
    if (smem) {
      RS_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)shm));
      jacobi_kernel<double, true><<<1, threads, shm, ctx->stream>>>(G, (int)k, nullptr, nullptr, 1e-15, 8.0, 30,
                                                                    evals, W);
    } else {
      jacobi_kernel<double, false><<<1, threads, 0, ctx->stream>>>(G, (int)k, Ag, Ag + k * (k + 1), 1e-15, 8.0, 30, evals,
                                                                   W);
    }
  } else {
    // float iterations, then double Rayleigh quotients of the float eigenvectors and a re-sort
    double* tmp = static_cast<double*>(rs_scratch(ctx, SCR_RED, (size_t)(k * k + 2 * k) * sizeof(double)));
    if (!tmp) return RS_ENOMEM;
    double* Wt = tmp;
    double* lam0 = tmp + k * k;
    double* lam1 = lam0 + k;
    const char* env = std::getenv("RS_JACOBI_PACKED");
    if (k >= 2 && !(env && env[0] == '0')) {
      // packed one-pass rounds with a rotation log, eigenvectors replayed in parallel afterwards
      constexpr int kMaxSweeps = 30;
      const int K = (int)((k + 1) & ~int64_t(1)), P = K / 2;
      const size_t log_bytes = (size_t)kMaxSweeps * (K - 1) * P * sizeof(float4);
      unsigned char* lg = static_cast<unsigned char*>(rs_scratch(ctx, SCR_EIG, log_bytes + 256));
      if (!lg) return RS_ENOMEM;
      float4* rot_log = reinterpret_cast<float4*>(lg);
      int* nsw = reinterpret_cast<int*>(lg + log_bytes);
      const size_t pshm = (size_t)k * (k + 1) / 2 * sizeof(float);
      const size_t ashm = (size_t)kJaRows * (k + 1) * sizeof(float);
      RS_CUDA_TRY(cudaFuncSetAttribute(jacobi_packed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pshm));
      // pass 1: float Jacobi on G.  Its absolute floor (a few rounding units of ||G||) stops it from
      // stirring rounding noise, but also leaves the small eigenvalues of a graded spectrum with only
      // absolute accuracy.
      jacobi_packed_kernel<<<1, 1024, pshm, ctx->stream>>>(G, (int)k, 1e-6f, 8.0, kMaxSweeps, rot_log, nsw, lam0);
      RS_LAUNCH_CHECK(ctx);
      jacobi_apply_kernel<<<(unsigned)((k + kJaRows - 1) / kJaRows), kJaRows * P, ashm, ctx->stream>>>(rot_log, nsw,
                                                                                                       (int)k, Wt);
      RS_LAUNCH_CHECK(ctx);
      // pass 2: H = W1^T G W1 formed in double is diagonal up to the first pass's rounding, so each
      // entry in float keeps its own relative accuracy; Jacobi on H with the relative criterion alone
      // (no absolute floor) then resolves the small eigenvalues to relative accuracy, and W = W1 W2.
      double* aux = static_cast<double*>(rs_scratch(ctx, SCR_JAC2, (size_t)3 * k * k * sizeof(double)));
      if (!aux) return RS_ENOMEM;
      double* Hd = aux;
      double* Tm = aux + k * k;
      double* W2 = aux + 2 * k * k;
      RS_TRY(launch_gemm<double>(ctx, k, k, k, 1.0, G, k, 1, Wt, k, 1, 0.0, nullptr, 0, Tm, k, nullptr));    // G W1
      RS_TRY(launch_gemm<double>(ctx, k, k, k, 1.0, Wt, 1, k, Tm, k, 1, 0.0, nullptr, 0, Hd, k, nullptr));   // W1^T (G W1)
      symmetrize_kernel<<<(unsigned)std::min<int64_t>((k * k + 255) / 256, 1024), 256, 0, ctx->stream>>>(Hd, (int)k);
      RS_LAUNCH_CHECK(ctx);
      jacobi_packed_kernel<<<1, 1024, pshm, ctx->stream>>>(Hd, (int)k, 1e-6f, 0.0, kMaxSweeps, rot_log, nsw, lam0);
      RS_LAUNCH_CHECK(ctx);
      jacobi_apply_kernel<<<(unsigned)((k + kJaRows - 1) / kJaRows), kJaRows * P, ashm, ctx->stream>>>(rot_log, nsw,
                                                                                                       (int)k, W2);
      RS_LAUNCH_CHECK(ctx);
      RS_TRY(launch_gemm<double>(ctx, k, k, k, 1.0, Wt, k, 1, W2, k, 1, 0.0, nullptr, 0, Tm, k, nullptr));   // W1 W2
      RS_CUDA_TRY(cudaMemcpyAsync(Wt, Tm, (size_t)k * k * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
      rayleigh_kernel<<<(unsigned)k, 128, 0, ctx->stream>>>(G, (int)k, Wt, lam1);
      RS_LAUNCH_CHECK(ctx);
      sort_eig_kernel<<<1, 256, 0, ctx->stream>>>(lam1, Wt, (int)k, evals, W);
      RS_LAUNCH_CHECK(ctx);
      return RS_OK;
    }
    float* Ag = static_cast<float*>(g);
    if (smem) {
      RS_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)shm));
      jacobi_kernel<float, true><<<1, threads, shm, ctx->stream>>>(G, (int)k, nullptr, nullptr, 1e-6, 8.0, 30, lam0,
                                                                   Wt);
    } else {
      jacobi_kernel<float, false><<<1, threads, 0, ctx->stream>>>(G, (int)k, Ag, Ag + k * (k + 1), 1e-6, 8.0, 30, lam0, Wt);
    }
    RS_LAUNCH_CHECK(ctx);
    rayleigh_kernel<<<(unsigned)k, 128, 0, ctx->stream>>>(G, (int)k, Wt, lam1);
    RS_LAUNCH_CHECK(ctx);
    sort_eig_kernel<<<1, 256, 0, ctx->stream>>>(lam1, Wt, (int)k, evals, W);
  }
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

// ---------------------------------------------------------------------- Alg. 2 pieces

static int read_status(rs_ctx* ctx, int* st);

template <typename T>
static int orthonormalize_t(rs_ctx* ctx, const T* Y, int64_t d, int64_t k, T* Q) {
  double* G = static_cast<double*>(rs_scratch(ctx, SCR_GRAM, k * k * sizeof(double)));
  T* tmp = static_cast<T*>(rs_scratch(ctx, SCR_TMPV, d * k * sizeof(T)));
  T* Linv = static_cast<T*>(rs_scratch(ctx, SCR_LINV, k * k * sizeof(T)));
  if (!G || !tmp || !Linv) return RS_ENOMEM;
  const size_t bytes = (2 * (size_t)k * (k + 1) + k) * sizeof(double);   // L, L^{-1} (rows k + 1), 1/diag
  const bool smem = bytes <= 160 * 1024;
  double* buf = nullptr;
  if (!smem) {
    buf = static_cast<double*>(rs_scratch(ctx, SCR_EIG, bytes));
    if (!buf) return RS_ENOMEM;
  }
  const size_t shm = smem ? bytes : 0;
  RS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_kernel<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  RS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_kernel<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const T* src = Y;
  for (int pass = 0; pass < 2; ++pass) {
    T* dst = pass == 0 ? tmp : Q;
    RS_TRY(launch_gram<T>(ctx, d, k, k, src, k, src, k, 1.0, G));
    // the first factorisation sees cond(Y)^2 and runs in double; the second one factors the Gram
    // matrix of an already orthonormal-to-rounding basis (condition ~1) in the storage type
    // (double work is slow on this GPU)
    if (pass == 0 && sizeof(T) == 4) {
      // float Y: Y L^{-T} is also formed in double.  A float product would perturb span(Y) by about
      // 2^-24 cond(Y)^2 (its rounding relative to |Y| |L^{-1}|, divided by the smallest singular value
      // of Y), which for graded spectra scrambles the weakest directions of the sketch and with them
      // the smallest Ritz values; in double the perturbation is 2^-53 cond(Y)^2.  L itself only sets
      // how orthonormal this first basis comes out (span(Y L^{-T}) = span(Y) for any invertible L),
      // so it is factored in float on chip when its packed triangle fits (the second pass restores
      // orthonormality), and in double when the float pivots break down (cond(Y)^2 near 2^24).
      double* Ld = static_cast<double*>(rs_scratch(ctx, SCR_LINVD, k * k * sizeof(double)));
      if (!Ld) return RS_ENOMEM;
      bool done = false;
      if (chol_packed_bytes<float>(k) <= kCholPackedMax) {
        const size_t ps = chol_packed_bytes<float>(k);
        int st0 = 0, st = 0;
        RS_TRY(read_status(ctx, &st0));   // the status word accumulates over the whole sketch
        RS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_packed_kernel<float, double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps));
        chol_inv_packed_kernel<float, double><<<1, 1024, ps, ctx->stream>>>(G, (int)k, Ld, ctx->d_status);
        RS_LAUNCH_CHECK(ctx);
        RS_TRY(read_status(ctx, &st));
        done = (st & 4) == 0 || (st0 & 4) != 0;
        if (!done) RS_CUDA_TRY(cudaMemcpy(ctx->d_status, &st0, sizeof(int), cudaMemcpyHostToDevice));   // retry in double
      }
      if (!done) {
        RS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shm));
        chol_inv_kernel<double, double><<<1, 256, shm, ctx->stream>>>(G, (int)k, buf, Ld, ctx->d_status);
        RS_LAUNCH_CHECK(ctx);
      }
      RS_TRY(launch_gemm<double, T, T, T>(ctx, d, k, k, 1.0, src, k, 1, Ld, 1, k, 0.0, nullptr, 0, dst, k, nullptr));
      src = dst;
      continue;
    }
    if (pass == 0) {
      if (chol_packed_bytes<double>(k) <= kCholPackedMax) {
        RS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_packed_kernel<double, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_packed_bytes<double>(k)));
        chol_inv_packed_kernel<double, T><<<1, 1024, chol_packed_bytes<double>(k), ctx->stream>>>(G, (int)k, Linv,
                                                                                                 ctx->d_status);
      } else {
        chol_inv_kernel<T, double><<<1, 256, shm, ctx->stream>>>(G, (int)k, buf, Linv, ctx->d_status);
      }
    } else if (chol_packed_bytes<T>(k) <= kCholPackedMax) {
      RS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_packed_kernel<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)chol_packed_bytes<T>(k)));
      chol_inv_packed_kernel<T, T><<<1, 1024, chol_packed_bytes<T>(k), ctx->stream>>>(G, (int)k, Linv, ctx->d_status);
    } else {
      chol_inv_kernel<T, T><<<1, 256, shm, ctx->stream>>>(G, (int)k, reinterpret_cast<T*>(buf), Linv, ctx->d_status);
    }
    RS_LAUNCH_CHECK(ctx);
    // Q = Y L^{-T}: B(p, j) = Linv[j][p]
    RS_TRY(launch_gemm<T>(ctx, d, k, k, 1.0, src, k, 1, Linv, 1, k, 0.0, nullptr, 0, dst, k, nullptr));
    src = dst;
  }
  return RS_OK;
}

static int read_status(rs_ctx* ctx, int* st) {
  RS_CUDA_TRY(cudaMemcpyAsync(st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return RS_OK;
}

template <typename S, typename T>
static int range_sketch_t(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, T* Y) {
  const int64_t n = X->n, d = X->d, k = p->k;
  const int32_t dt = sizeof(T) == 8 ? RS_F64 : RS_F32;
  double* Gd = static_cast<double*>(rs_scratch(ctx, SCR_GRAM, d * k * sizeof(double)));
  if (!Gd) return RS_ENOMEM;
  if (p->kind == RS_SKETCH_GAUSSIAN) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value && std::is_same<T, float>::value) {
      // bfloat16 data: the contraction on tensor cores with the test matrix rounded to bfloat16
      const int rc = umma_sketch(ctx, X, p->seed, k, Y);
      if (rc != RS_EUNSUPPORTED) return rc;
    }
    T* Om = static_cast<T*>(rs_scratch(ctx, SCR_OMEGA, n * k * sizeof(T)));
    if (!Om) return RS_ENOMEM;
    RS_TRY(gaussian_dispatch(ctx, p->seed, 0, n, k, dt, Om, k));
    RS_TRY(launch_gram<S, T>(ctx, n, d, k, static_cast<const S*>(X->data), X->ld, Om, k, 1.0, Gd));
  } else {
    const int64_t s = p->s > 0 ? p->s : std::min<int64_t>(n, 64 * k);
    T* SX = static_cast<T*>(rs_scratch(ctx, SCR_SX, s * d * sizeof(T)));
    T* Gp = static_cast<T*>(rs_scratch(ctx, SCR_OMEGA, s * k * sizeof(T)));
    if (!SX || !Gp) return RS_ENOMEM;
    RS_TRY(countsketch_dispatch(ctx, X, p->seed, s, SX, d, nullptr, nullptr));
    RS_TRY(gaussian_dispatch(ctx, p->seed, 0, s, k, dt, Gp, k));
    RS_TRY(launch_gram<T>(ctx, s, d, k, SX, d, Gp, k, 1.0, Gd));
  }
  return to_T<T>(ctx, Gd, d * k, Y);
}

template <typename S, typename T>
static int ritz_t(rs_ctx* ctx, const rs_matrix* X, const T* Q, int64_t kq, int64_t k, T* V, double* sigma2) {
  const int64_t n = X->n, d = X->d;
  T* B = static_cast<T*>(rs_scratch(ctx, SCR_B, n * kq * sizeof(T)));
  double* G = static_cast<double*>(rs_scratch(ctx, SCR_GRAM, kq * kq * sizeof(double)));
  double* ev = static_cast<double*>(rs_scratch(ctx, SCR_S2, kq * sizeof(double)));
  double* Wd = static_cast<double*>(rs_scratch(ctx, SCR_W, kq * kq * sizeof(double)));
  T* Wt = static_cast<T*>(rs_scratch(ctx, SCR_ADIAG, kq * kq * sizeof(T)));
  if (!B || !G || !ev || !Wd || !Wt) return RS_ENOMEM;
  // B = X Q (n x kq), G = B^T B / n   (bfloat16 or float data: X Q on the tensor cores)
  int rc_b = RS_EUNSUPPORTED;
  if constexpr ((std::is_same<S, __nv_bfloat16>::value || std::is_same<S, float>::value) &&
                std::is_same<T, float>::value)
    if (umma_enabled()) rc_b = umma_gemm_xw(ctx, X, Q, kq, nullptr, B, kq);
  if (rc_b == RS_EUNSUPPORTED)
    RS_TRY(launch_gemm<T, S, T>(ctx, n, kq, d, 1.0, static_cast<const S*>(X->data), X->ld, 1, Q, kq, 1, 0.0, nullptr, 0,
                                B, kq, nullptr));
  else if (rc_b != RS_OK)
    return rc_b;
  RS_TRY(launch_gram<T>(ctx, n, kq, kq, B, kq, B, kq, 1.0 / (double)n, G));
  if constexpr (sizeof(T) == 4) {
    // Q in float is orthonormal only to the rounding of its last Cholesky-QR factorisation, S = Q^T Q =
    // I + E with |E| ~ k 2^-24, and an unaccounted E would move the smallest Ritz values by about
    // |E| sigma_1^2.  Rayleigh-Ritz is therefore taken in the metric of the basis as stored: with
    // T = S^{-1/2} (series to O(|E|^3), all in double) the Ritz pairs of C on span(Q) are the eigenpairs
    // of T G T, and V = Q T W.
    double* Sd = static_cast<double*>(rs_scratch(ctx, SCR_RITZ, (size_t)5 * kq * kq * sizeof(double)));
    if (!Sd) return RS_ENOMEM;
    double* Ed = Sd + kq * kq;
    double* E2 = Ed + kq * kq;
    double* Td = E2 + kq * kq;
    double* Hd = Td + kq * kq;
    const unsigned sb = (unsigned)std::min<int64_t>((kq * kq + 255) / 256, 1024);
    RS_TRY(launch_gram<T>(ctx, d, kq, kq, Q, kq, Q, kq, 1.0, Sd));
    minus_identity_kernel<<<sb, 256, 0, ctx->stream>>>(Sd, (int)kq, Ed);
    RS_LAUNCH_CHECK(ctx);
    RS_TRY(launch_gemm<double>(ctx, kq, kq, kq, 1.0, Ed, kq, 1, Ed, kq, 1, 0.0, nullptr, 0, E2, kq, nullptr));
    inv_sqrt_series_kernel<<<sb, 256, 0, ctx->stream>>>(Ed, E2, (int)kq, Td);
    RS_LAUNCH_CHECK(ctx);
    RS_TRY(launch_gemm<double>(ctx, kq, kq, kq, 1.0, G, kq, 1, Td, kq, 1, 0.0, nullptr, 0, Hd, kq, nullptr));   // G T
    RS_TRY(launch_gemm<double>(ctx, kq, kq, kq, 1.0, Td, kq, 1, Hd, kq, 1, 0.0, nullptr, 0, G, kq, nullptr));   // T G T
    symmetrize_kernel<<<sb, 256, 0, ctx->stream>>>(G, (int)kq);
    RS_LAUNCH_CHECK(ctx);
    RS_TRY(run_sym_eig(ctx, G, kq, RS_F32, ev, Wd));
    RS_TRY(launch_gemm<double>(ctx, kq, kq, kq, 1.0, Td, kq, 1, Wd, kq, 1, 0.0, nullptr, 0, Hd, kq, nullptr));  // T W
    RS_TRY(to_T<T>(ctx, Hd, kq * kq, Wt));
  } else {
    RS_TRY(run_sym_eig(ctx, G, kq, RS_F64, ev, Wd));
    RS_TRY(to_T<T>(ctx, Wd, kq * kq, Wt));
  }
  // V = Q W[:, :k]
  RS_TRY(launch_gemm<T>(ctx, d, k, kq, 1.0, Q, kq, 1, Wt, kq, 1, 0.0, nullptr, 0, V, k, nullptr));
  RS_CUDA_TRY(cudaMemcpyAsync(sigma2, ev, k * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return RS_OK;
}

template <typename S, typename T>
static int sketch_t(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, T* V, double* sigma2) {
  const int64_t n = X->n, d = X->d, k = p->k;
  const int64_t q = std::max(1, p->q_blocks);
  const int64_t kq = k * q;
  if (kq > std::min<int64_t>(d, 256)) return rs_fail(RS_EINVAL, "rs_sketch: k * q_blocks = %lld exceeds min(d, 256)", (long long)kq);
  // The Krylov space K = [A Pi, C A Pi, ..., C^{q-1} A Pi] of Alg. 2 (C = A A^T) is built block by
  // block: Q_0 = orth(A Pi); Y_j = C Q_{j-1} with the earlier blocks projected out (twice), Q_j =
  // orth(Y_j).  [Q_0 .. Q_{q-1}] is then an orthonormal basis of K without forming the badly scaled
  // powers C^j A Pi explicitly.
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  T* Yk = static_cast<T*>(rs_scratch(ctx, SCR_Y, d * k * sizeof(T)));
  T* Qall = static_cast<T*>(rs_scratch(ctx, SCR_Q, 2 * d * kq * sizeof(T)));
  if (!Yk || !Qall) return RS_ENOMEM;
  T* Qb = Qall;              // q blocks, each d x k contiguous
  T* Qm = Qall + d * kq;     // d x kq row-major basis
  RS_TRY(range_sketch_t<S, T>(ctx, X, p, Yk));
  RS_TRY(orthonormalize_t<T>(ctx, Yk, d, k, Qb));
  if (q > 1) {
    T* B = static_cast<T*>(rs_scratch(ctx, SCR_B, n * k * sizeof(T)));
    double* Gd = static_cast<double*>(rs_scratch(ctx, SCR_GRAM, d * k * sizeof(double)));
    double* Pd = static_cast<double*>(rs_scratch(ctx, SCR_MISC, k * k * sizeof(double)));
    T* Pt = static_cast<T*>(rs_scratch(ctx, SCR_ADIAG, k * k * sizeof(T)));
    if (!B || !Gd || !Pd || !Pt) return RS_ENOMEM;
    for (int64_t j = 1; j < q; ++j) {
      const T* Qprev = Qb + (j - 1) * d * k;
      RS_TRY(launch_gemm<T, S, T>(ctx, n, k, d, 1.0, static_cast<const S*>(X->data), X->ld, 1, Qprev, k, 1, 0.0, nullptr,
                            0, B, k, nullptr));
      RS_TRY(launch_gram<S, T>(ctx, n, d, k, static_cast<const S*>(X->data), X->ld, B, k, 1.0 / (double)n, Gd));
      RS_TRY(to_T<T>(ctx, Gd, d * k, Yk));
      for (int pass = 0; pass < 2; ++pass)
        for (int64_t i = 0; i < j; ++i) {
          const T* Qi = Qb + i * d * k;
          RS_TRY(launch_gram<T>(ctx, d, k, k, Qi, k, Yk, k, 1.0, Pd));   // Q_i^T Y_j
          RS_TRY(to_T<T>(ctx, Pd, k * k, Pt));
          RS_TRY(launch_gemm<T>(ctx, d, k, k, -1.0, Qi, k, 1, Pt, k, 1, 1.0, Yk, k, Yk, k, nullptr));
        }
      RS_TRY(orthonormalize_t<T>(ctx, Yk, d, k, Qb + j * d * k));
    }
  }
  for (int64_t j = 0; j < q; ++j)
    RS_CUDA_TRY(cudaMemcpy2DAsync(Qm + j * k, kq * sizeof(T), Qb + j * d * k, k * sizeof(T), k * sizeof(T), d,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  RS_TRY(ritz_t<S, T>(ctx, X, Qm, kq, k, V, sigma2));
  int st = 0;
  RS_TRY(read_status(ctx, &st));
  if (st & 4) return rs_fail(RS_EINVAL, "rs_sketch: the sketch is rank deficient to working precision");
  return RS_OK;
}

// ---------------------------------------------------------------------- preconditioner

// X stored in S, components Z stored in SZ (S, or bfloat16 for float data), compute type T
template <typename S, typename T, typename SZ = S>
static int precondition_t(rs_ctx* ctx, const rs_matrix* X, const T* V, const double* sigma2, int64_t k, double lam,
                          rs_matrix* Xt, T* beta, double* beta_hat) {
  const int64_t n = X->n, d = X->d, N = n + d;
  SZ* Z = static_cast<SZ*>(const_cast<void*>(Xt->data));
  const int64_t ldz = Xt->ld;
  T* a = static_cast<T*>(rs_scratch(ctx, SCR_ADIAG, k * sizeof(T)));
  T* P = static_cast<T*>(rs_scratch(ctx, SCR_P, n * k * sizeof(T)));
  T* Va = static_cast<T*>(rs_scratch(ctx, SCR_TMPV, d * k * sizeof(T)));
  if (!a || !P || !Va) return RS_ENOMEM;
  adiag_kernel<T><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(sigma2, (int)k, lam, a);
  RS_LAUNCH_CHECK(ctx);
  const S* Xd = static_cast<const S*>(X->data);
  // P = X V diag(a);  Z[0:n] = X - P V^T   (bfloat16 or float data: X V on the tensor cores)
  int rc_p = RS_EUNSUPPORTED;
  if constexpr ((std::is_same<S, __nv_bfloat16>::value || std::is_same<S, float>::value) &&
                std::is_same<T, float>::value)
    if (umma_enabled()) rc_p = umma_gemm_xw(ctx, X, V, k, a, P, k);
  if (rc_p == RS_EUNSUPPORTED)
    RS_TRY(launch_gemm<T, S, T>(ctx, n, k, d, 1.0, Xd, X->ld, 1, V, k, 1, 0.0, nullptr, 0, P, k, a));
  else if (rc_p != RS_OK)
    return rc_p;
  int rc_z = RS_EUNSUPPORTED;
  float* rowsq = nullptr;   // squared norms of the data rows of Z, formed by the tensor-core kernel
  if constexpr ((std::is_same<S, __nv_bfloat16>::value || std::is_same<S, float>::value) &&
                std::is_same<SZ, __nv_bfloat16>::value && std::is_same<T, float>::value)
    if (rc_p == RS_OK) {
      rowsq = static_cast<float*>(rs_scratch(ctx, SCR_ROWSQ, n * sizeof(float)));
      if (!rowsq) return RS_ENOMEM;
      rc_z = umma_resid(ctx, X, P, V, k, Xt, rowsq);
    }
  if (rc_z == RS_EUNSUPPORTED)
    RS_TRY(launch_gemm<T, T, SZ, S>(ctx, n, d, k, -1.0, P, k, 1, V, 1, k, 1.0, Xd, X->ld, Z, ldz, nullptr));
  else if (rc_z != RS_OK)
    return rc_z;
  // Z[n:n+d] = I - V diag(a) V^T   (the rows b_j = M e_j)
  scale_cols_kernel<T><<<blocks_for(ctx, d * k), 256, 0, ctx->stream>>>(V, d, (int)k, a, Va);
  RS_LAUNCH_CHECK(ctx);
  SZ* Zb = Z + n * ldz;
  identity_rows_kernel<SZ><<<blocks_for(ctx, d * d), 256, 0, ctx->stream>>>(Zb, d, ldz);
  RS_LAUNCH_CHECK(ctx);
  RS_TRY(launch_gemm<T, T, SZ>(ctx, d, d, k, -1.0, Va, k, 1, V, 1, k, 1.0, Zb, ldz, Zb, ldz, nullptr));
  // smoothness constants
  const int blocks = blocks_for(ctx, N * 32);
  double* part = static_cast<double*>(rs_scratch(ctx, SCR_MISC, (blocks + 1) * sizeof(double)));
  if (!part) return RS_ENOMEM;
  if (rc_z == RS_OK && rowsq)
    row_beta_sq_kernel<SZ, T><<<blocks, 256, 0, ctx->stream>>>(rowsq, Z, N, n, d, ldz, lam, beta, part);
  else
    row_beta_kernel<SZ, T><<<blocks, 256, 0, ctx->stream>>>(Z, N, n, d, ldz, lam, beta, part);
  RS_LAUNCH_CHECK(ctx);
  if (beta_hat) {
    sum_parts_kernel<<<1, 32, 0, ctx->stream>>>(part, blocks, 1.0 / (double)N, part + blocks);
    RS_LAUNCH_CHECK(ctx);
    RS_CUDA_TRY(cudaMemcpyAsync(beta_hat, part + blocks, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return RS_OK;
}

template <typename T>
static int map_output_t(rs_ctx* ctx, const T* V, const double* sigma2, int64_t d, int64_t k, double lam, const T* wt,
                        T* w) {
  if (k <= 256 && d * k <= 65536) {   // one launch
    map_fused_kernel<T, T><<<1, 1024, 0, ctx->stream>>>(V, sigma2, d, (int)k, lam, wt, w);
    RS_LAUNCH_CHECK(ctx);
    return RS_OK;
  }
  if (k <= 256) {   // larger d: many blocks (the one-block kernel is latency-bound on a few MB of V)
    const int64_t R = 32;
    const int P = (int)((d + R - 1) / R);
    T* part = static_cast<T*>(rs_scratch(ctx, SCR_MAPPART, ((size_t)P * k + k) * sizeof(T)));
    if (!part) return RS_ENOMEM;
    T* tv = part + (size_t)P * k;
    map_tpart_kernel<T><<<(unsigned)P, 256, 0, ctx->stream>>>(V, d, (int)k, R, wt, part);
    RS_LAUNCH_CHECK(ctx);
    map_tsum_kernel<T><<<1, 256, 0, ctx->stream>>>(part, P, (int)k, sigma2, lam, tv);
    RS_LAUNCH_CHECK(ctx);
    map_apply_kernel<T><<<(unsigned)((d + 7) / 8), 256, 0, ctx->stream>>>(V, d, (int)k, tv, wt, w);
    RS_LAUNCH_CHECK(ctx);
    return RS_OK;
  }
  T* a = static_cast<T*>(rs_scratch(ctx, SCR_ADIAG, k * sizeof(T)));
  double* tv = static_cast<double*>(rs_scratch(ctx, SCR_RED, k * sizeof(double)));
  if (!a || !tv) return RS_ENOMEM;
  adiag_kernel<T><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(sigma2, (int)k, lam, a);
  RS_LAUNCH_CHECK(ctx);
  RS_TRY(launch_gram<T>(ctx, d, k, 1, V, k, wt, 1, 1.0, tv));
  map_output_kernel<T><<<blocks_for(ctx, d), 256, 0, ctx->stream>>>(V, d, (int)k, a, tv, wt, w);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int map_output_dispatch(rs_ctx* ctx, const void* V, const double* sigma2, int64_t d, int64_t k, double lam,
                        int32_t dtype, const void* wt, void* w) {
  if (dtype == RS_F64)
    return map_output_t<double>(ctx, static_cast<const double*>(V), sigma2, d, k, lam,
                                static_cast<const double*>(wt), static_cast<double*>(w));
  return map_output_t<float>(ctx, static_cast<const float*>(V), sigma2, d, k, lam, static_cast<const float*>(wt),
                             static_cast<float*>(w));
}

int sketch_dispatch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* V, double* sigma2) {
  if (X->dtype == RS_F64) return sketch_t<double, double>(ctx, X, p, static_cast<double*>(V), sigma2);
  if (X->dtype == RS_F32) return sketch_t<float, float>(ctx, X, p, static_cast<float*>(V), sigma2);
  if (X->dtype == RS_BF16) return sketch_t<__nv_bfloat16, float>(ctx, X, p, static_cast<float*>(V), sigma2);
  return rs_fail(RS_EUNSUPPORTED, "rs_sketch: dtype %d not supported by this build", X->dtype);
}

int precondition_dispatch(rs_ctx* ctx, const rs_matrix* X, const void* V, const double* sigma2, int64_t k, double lam,
                          rs_matrix* Xt, void* beta, double* beta_hat) {
  if (Xt->dtype == RS_FP8E4M3) {
    // bfloat16 components in scratch, then per-row scaled FP8 codes and beta from the stored values
    const int64_t n = X->n, d = X->d, N = n + d;
    const int64_t ldb = (d + 7) / 8 * 8;
    __nv_bfloat16* Zb = static_cast<__nv_bfloat16*>(rs_scratch(ctx, SCR_Z8, (size_t)N * ldb * sizeof(__nv_bfloat16)));
    if (!Zb) return RS_ENOMEM;
    rs_matrix Zm = {Zb, nullptr, N, d, ldb, RS_BF16, 0};
    int rc;
    if (X->dtype == RS_F32)
      rc = precondition_t<float, float, __nv_bfloat16>(ctx, X, static_cast<const float*>(V), sigma2, k, lam, &Zm,
                                                       static_cast<float*>(beta), nullptr);
    else if (X->dtype == RS_BF16)
      rc = precondition_t<__nv_bfloat16, float>(ctx, X, static_cast<const float*>(V), sigma2, k, lam, &Zm,
                                                static_cast<float*>(beta), nullptr);
    else
      return rs_fail(RS_EUNSUPPORTED, "rs_precondition: FP8 components need RS_F32 or RS_BF16 data");
    if (rc != RS_OK) return rc;
    quantize_fp8_rows_kernel<<<blocks_for(ctx, N * 32), 256, 0, ctx->stream>>>(
        Zb, N, n, d, ldb, lam, static_cast<__nv_fp8_e4m3*>(const_cast<void*>(Xt->data)), Xt->ld,
        const_cast<float*>(Xt->row_scale), static_cast<float*>(beta));
    RS_LAUNCH_CHECK(ctx);
    if (beta_hat) {
      double* part = static_cast<double*>(rs_scratch(ctx, SCR_MISC, 2 * sizeof(double)));
      if (!part) return RS_ENOMEM;
      mean_f_kernel<<<1, 1024, 0, ctx->stream>>>(static_cast<const float*>(beta), N, part);
      RS_LAUNCH_CHECK(ctx);
      RS_CUDA_TRY(cudaMemcpyAsync(beta_hat, part, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return RS_OK;
  }
  if (X->dtype == RS_F64)
    return precondition_t<double, double>(ctx, X, static_cast<const double*>(V), sigma2, k, lam, Xt,
                                  static_cast<double*>(beta), beta_hat);
  if (X->dtype == RS_F32 && Xt->dtype == RS_BF16)
    return precondition_t<float, float, __nv_bfloat16>(ctx, X, static_cast<const float*>(V), sigma2, k, lam, Xt,
                                                       static_cast<float*>(beta), beta_hat);
  if (X->dtype == RS_F32)
    return precondition_t<float, float>(ctx, X, static_cast<const float*>(V), sigma2, k, lam, Xt,
                                        static_cast<float*>(beta), beta_hat);
  if (X->dtype == RS_BF16)
    return precondition_t<__nv_bfloat16, float>(ctx, X, static_cast<const float*>(V), sigma2, k, lam, Xt,
                                                static_cast<float*>(beta), beta_hat);
  return rs_fail(RS_EUNSUPPORTED, "rs_precondition: dtype %d not supported by this build", X->dtype);
}

int objective_dispatch(rs_ctx* ctx, const rs_matrix* X, const void* y, double lam, const void* w, const void* wr,
                       double* out) {
  const int64_t n = X->n, d = X->d;
  const int blocks = blocks_for(ctx, n * 32);
  double* part = static_cast<double*>(rs_scratch(ctx, SCR_MISC, (2 * blocks + 2) * sizeof(double)));
  if (!part) return RS_ENOMEM;
  double* res = part + 2 * blocks;
  if (X->dtype == RS_F64) {
    objective_kernel<double, double><<<blocks, 256, 0, ctx->stream>>>(
        static_cast<const double*>(X->data), n, d, X->ld, static_cast<const double*>(y),
        static_cast<const double*>(w), static_cast<const double*>(wr), part);
    RS_LAUNCH_CHECK(ctx);
    objective_finish_kernel<double><<<1, 256, 0, ctx->stream>>>(part, blocks, n, d, lam, static_cast<const double*>(w),
                                                                static_cast<const double*>(wr), res);
  } else if (X->dtype == RS_F32) {
    objective_kernel<float, float><<<blocks, 256, 0, ctx->stream>>>(
        static_cast<const float*>(X->data), n, d, X->ld, static_cast<const float*>(y), static_cast<const float*>(w),
        static_cast<const float*>(wr), part);
    RS_LAUNCH_CHECK(ctx);
    objective_finish_kernel<float><<<1, 256, 0, ctx->stream>>>(part, blocks, n, d, lam, static_cast<const float*>(w),
                                                               static_cast<const float*>(wr), res);
  } else if (X->dtype == RS_BF16) {
    objective_kernel<__nv_bfloat16, float><<<blocks, 256, 0, ctx->stream>>>(
        static_cast<const __nv_bfloat16*>(X->data), n, d, X->ld, static_cast<const float*>(y),
        static_cast<const float*>(w), static_cast<const float*>(wr), part);
    RS_LAUNCH_CHECK(ctx);
    objective_finish_kernel<float><<<1, 256, 0, ctx->stream>>>(part, blocks, n, d, lam, static_cast<const float*>(w),
                                                               static_cast<const float*>(wr), res);
  } else {
    return rs_fail(RS_EUNSUPPORTED, "rs_objective: dtype %d", X->dtype);
  }
  RS_LAUNCH_CHECK(ctx);
  RS_CUDA_TRY(cudaMemcpyAsync(out, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return RS_OK;
}

int trace_dispatch(rs_ctx* ctx, const rs_matrix* X, double* out) {
  const int64_t n = X->n, d = X->d;
  const int blocks = blocks_for(ctx, n * 32);
  double* part = static_cast<double*>(rs_scratch(ctx, SCR_MISC, (blocks + 1) * sizeof(double)));
  if (!part) return RS_ENOMEM;
  if (X->dtype == RS_F64)
    sumsq_kernel<double><<<blocks, 256, 0, ctx->stream>>>(static_cast<const double*>(X->data), n, d, X->ld, part);
  else if (X->dtype == RS_F32)
    sumsq_kernel<float><<<blocks, 256, 0, ctx->stream>>>(static_cast<const float*>(X->data), n, d, X->ld, part);
  else if (X->dtype == RS_BF16)
    sumsq_kernel<__nv_bfloat16><<<blocks, 256, 0, ctx->stream>>>(static_cast<const __nv_bfloat16*>(X->data), n, d,
                                                                 X->ld, part);
  else
    return rs_fail(RS_EUNSUPPORTED, "rs_trace_c: dtype %d", X->dtype);
  RS_LAUNCH_CHECK(ctx);
  trace_finish_kernel<<<1, 32, 0, ctx->stream>>>(part, blocks, 1.0 / (double)n, part + blocks);
  RS_LAUNCH_CHECK(ctx);
  RS_CUDA_TRY(cudaMemcpyAsync(out, part + blocks, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return RS_OK;
}

// ====================================================================== C ABI

extern "C" {

int rs_range_sketch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* Y) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_range_sketch X"));
  RS_CHECK_ARG(p && Y, "rs_range_sketch: null argument");
  RS_CHECK_ARG(p->k >= 1 && p->k <= X->d && p->k <= 256, "rs_range_sketch: k must be in [1, min(d, 256)]");
  RS_CHECK_ARG(p->kind == RS_SKETCH_GAUSSIAN || p->kind == RS_SKETCH_COUNTSKETCH, "rs_range_sketch: bad kind");
  if (X->dtype == RS_F64) return range_sketch_t<double, double>(ctx, X, p, static_cast<double*>(Y));
  if (X->dtype == RS_F32) return range_sketch_t<float, float>(ctx, X, p, static_cast<float*>(Y));
  if (X->dtype == RS_BF16) return range_sketch_t<__nv_bfloat16, float>(ctx, X, p, static_cast<float*>(Y));
  return rs_fail(RS_EUNSUPPORTED, "rs_range_sketch: dtype %d", X->dtype);
}

int rs_orthonormalize(rs_ctx* ctx, const void* Y, int64_t d, int64_t k, int32_t dtype, void* Q) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(Y && Q && d >= 1 && k >= 1 && k <= d && k <= 256, "rs_orthonormalize: bad arguments");
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  int rc;
  if (dtype == RS_F64) rc = orthonormalize_t<double>(ctx, static_cast<const double*>(Y), d, k, static_cast<double*>(Q));
  else if (dtype == RS_F32) rc = orthonormalize_t<float>(ctx, static_cast<const float*>(Y), d, k, static_cast<float*>(Q));
  else return rs_fail(RS_EUNSUPPORTED, "rs_orthonormalize: dtype %d", dtype);
  if (rc != RS_OK) return rc;
  int st = 0;
  RS_TRY(read_status(ctx, &st));
  if (st & 4) return rs_fail(RS_EINVAL, "rs_orthonormalize: Y is rank deficient to working precision");
  return RS_OK;
}

int rs_sym_eig(rs_ctx* ctx, const double* G, int64_t k, int32_t prec, double* evals, double* W) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(G && evals && W, "rs_sym_eig: null argument");
  RS_CHECK_ARG(prec == RS_F64 || prec == RS_F32, "rs_sym_eig: prec must be RS_F64 or RS_F32");
  return run_sym_eig(ctx, G, k, prec, evals, W);
}

int rs_ritz(rs_ctx* ctx, const rs_matrix* X, const void* Q, int64_t k, void* V, double* sigma2) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_ritz X"));
  RS_CHECK_ARG(Q && V && sigma2 && k >= 1 && k <= X->d && k <= 256, "rs_ritz: bad arguments");
  if (X->dtype == RS_F64)
    return ritz_t<double, double>(ctx, X, static_cast<const double*>(Q), k, k, static_cast<double*>(V), sigma2);
  if (X->dtype == RS_F32)
    return ritz_t<float, float>(ctx, X, static_cast<const float*>(Q), k, k, static_cast<float*>(V), sigma2);
  if (X->dtype == RS_BF16)
    return ritz_t<__nv_bfloat16, float>(ctx, X, static_cast<const float*>(Q), k, k, static_cast<float*>(V), sigma2);
  return rs_fail(RS_EUNSUPPORTED, "rs_ritz: dtype %d", X->dtype);
}

int rs_sketch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* V, double* sigma2) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_sketch X"));
  RS_CHECK_ARG(p && V && sigma2, "rs_sketch: null argument");
  RS_CHECK_ARG(p->k >= 1 && p->k <= X->d && p->k <= 256, "rs_sketch: k must be in [1, min(d, 256)]");
  RS_CHECK_ARG(p->kind == RS_SKETCH_GAUSSIAN || p->kind == RS_SKETCH_COUNTSKETCH, "rs_sketch: bad kind");
  return sketch_dispatch(ctx, X, p, V, sigma2);
}

int rs_precondition(rs_ctx* ctx, const rs_matrix* X, const void* V, const double* sigma2, int64_t k, double lambda,
                    rs_matrix* Xt, void* beta, double* beta_hat) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_precondition X"));
  RS_TRY(check_matrix(Xt, "rs_precondition Xt"));
  RS_CHECK_ARG(V && sigma2 && beta, "rs_precondition: null argument");
  RS_CHECK_ARG(k >= 1 && k <= X->d, "rs_precondition: k must be in [1, d]");
  RS_CHECK_ARG(lambda > 0.0, "rs_precondition: lambda must be positive");
  RS_CHECK_ARG(Xt->n == X->n + X->d && Xt->d == X->d, "rs_precondition: Xt must be (n + d) x d");
  RS_CHECK_ARG(Xt->dtype == X->dtype || (X->dtype == RS_F32 && Xt->dtype == RS_BF16) ||
                   (Xt->dtype == RS_FP8E4M3 && (X->dtype == RS_F32 || X->dtype == RS_BF16)),
               "rs_precondition: Xt dtype must equal X dtype (or be RS_BF16 for RS_F32 data, or RS_FP8E4M3)");
  return precondition_dispatch(ctx, X, V, sigma2, k, lambda, Xt, beta, beta_hat);
}

int rs_map_output(rs_ctx* ctx, const void* V, const double* sigma2, int64_t d, int64_t k, double lambda, int32_t dtype,
                  const void* w_tilde, void* w) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(V && sigma2 && w_tilde && w && d >= 1 && k >= 1 && k <= d, "rs_map_output: bad arguments");
  RS_CHECK_ARG(dtype == RS_F64 || dtype == RS_F32, "rs_map_output: dtype must be RS_F64 or RS_F32");
  return map_output_dispatch(ctx, V, sigma2, d, k, lambda, dtype, w_tilde, w);
}

int rs_objective(rs_ctx* ctx, const rs_matrix* X, const void* y, double lambda, const void* w, const void* w_ref,
                 double* out) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_objective X"));
  RS_CHECK_ARG(y && w && out, "rs_objective: null argument");
  return objective_dispatch(ctx, X, y, lambda, w, w_ref, out);
}

int rs_trace_c(rs_ctx* ctx, const rs_matrix* X, double* out) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_trace_c X"));
  RS_CHECK_ARG(out, "rs_trace_c: null argument");
  return trace_dispatch(ctx, X, out);
}

}  // extern "C"
