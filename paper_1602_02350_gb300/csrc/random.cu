// Random streams of the method: Philox words, the Gaussian test matrix of Alg. 2, the
// CountSketch (deterministic bucket gather), integer sampling weights, their prefix sums,
// and the importance-sampled index stream of Alg. 1.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void philox_words_kernel(uint64_t seed, uint32_t c2, uint32_t c3, int64_t count, uint32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    U32x4 w = philox4x32_10(U32x4{(uint32_t)i, (uint32_t)((uint64_t)i >> 32), c2, c3}, seed);
    reinterpret_cast<uint4*>(out)[i] = make_uint4(w.x, w.y, w.z, w.w);
  }
}

template <typename T>
__device__ __forceinline__ void gauss4(uint64_t seed, int64_t i, uint32_t g, T* z) {
  U32x4 w = philox4x32_10(U32x4{(uint32_t)i, (uint32_t)((uint64_t)i >> 32), g, TAG_GAUSS}, seed);
  if constexpr (sizeof(T) == 8) {
    box_muller(u24d(w.x), u24d(w.y), z[0], z[1]);
    box_muller(u24d(w.z), u24d(w.w), z[2], z[3]);
  } else {
    box_muller(u24f(w.x), u24f(w.y), z[0], z[1]);
    box_muller(u24f(w.z), u24f(w.w), z[2], z[3]);
  }
}

template <typename T>
__global__ void gaussian_kernel(uint64_t seed, int64_t row0, int64_t rows, int64_t cols, T* out, int64_t ld) {
  const int64_t groups = (cols + 3) / 4;
  const int64_t total = rows * groups;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / groups;
    const uint32_t g = (uint32_t)(e % groups);
    T z[4];
    gauss4<T>(seed, row0 + r, g, z);
    T* dst = out + r * ld + 4 * (int64_t)g;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * (int64_t)g + q < cols) dst[q] = z[q];
  }
}

// Transposed bfloat16 test matrix for the tensor-core range sketch: out[j * ld + i] = bf16(Pi(i, j))
// for j < k, i < n (the float Box-Muller value of entry (i, j), rounded to nearest).  Consecutive
// threads take consecutive rows i of one group of four columns, so each of the four stores is
// coalesced along a row of the output.
__global__ void gaussian_t_bf16_kernel(uint64_t seed, int64_t n, int64_t k, __nv_bfloat16* out, int64_t ld) {
  const int64_t groups = (k + 3) / 4;
  const int64_t total = n * groups;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;
    const uint32_t g = (uint32_t)(e / n);
    float z[4];
    gauss4<float>(seed, i, g, z);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * (int64_t)g + q < k) out[(4 * (int64_t)g + q) * ld + i] = __float2bfloat16_rn(z[q]);
  }
}

// ---------------------------------------------------------------- CountSketch

template <typename T>
__global__ void cs_hash_kernel(uint64_t seed, int64_t n, int64_t s, int32_t* bucket, T* sign) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    U32x4 w = philox4x32_10(U32x4{(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, TAG_COUNTSKETCH}, seed);
    bucket[i] = (int32_t)(((uint64_t)w.x * (uint64_t)s) >> 32);
    sign[i] = (w.y >> 31) ? T(-1) : T(1);
  }
}

// cnt[h * nchunks + c] = number of rows of chunk c (rows [c R, (c+1) R)) in bucket h
__global__ void cs_chunk_count_kernel(const int32_t* bucket, int64_t n, int64_t s, int64_t R, int64_t nchunks,
                                      uint32_t* cnt) {
  extern __shared__ uint32_t sh_cnt[];
  const int64_t c = blockIdx.x;
  for (int64_t h = threadIdx.x; h < s; h += blockDim.x) sh_cnt[h] = 0;
  __syncthreads();
  const int64_t r0 = c * R, r1 = min(n, r0 + R);
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) atomicAdd(&sh_cnt[bucket[i]], 1u);
  __syncthreads();
  for (int64_t h = threadIdx.x; h < s; h += blockDim.x) cnt[h * nchunks + c] = sh_cnt[h];
}

// One warp per chunk walks its rows in order and writes each row index to its stable
// position base[h * nchunks + c] + (rows of bucket h earlier in the chunk).
__global__ void cs_place_kernel(const int32_t* bucket, int64_t n, int64_t s, int64_t R, int64_t nchunks,
                                const uint64_t* incl, const uint32_t* cnt, int32_t* perm) {
  extern __shared__ uint32_t sh_run[];
  const int64_t c = blockIdx.x;
  for (int64_t h = threadIdx.x; h < s; h += blockDim.x) sh_run[h] = 0;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const int64_t r0 = c * R, r1 = min(n, r0 + R);
  for (int64_t g = r0; g < r1; g += 32) {
    const int64_t i = g + lane;
    const bool valid = i < r1;
    const int h = valid ? bucket[i] : -1 - lane;   // distinct dummy keys for invalid lanes
    const unsigned same = __match_any_sync(0xffffffffu, h);
    const unsigned lt = same & ((1u << lane) - 1u);
    uint32_t base_run = 0;
    if (valid) base_run = sh_run[h];
    __syncwarp();
    if (valid) {
      const int64_t slot = h * nchunks + c;
      const uint64_t start = incl[slot] - cnt[slot];   // exclusive prefix
      perm[start + base_run + __popc(lt)] = (int32_t)i;
      // the highest lane of each group advances the running count
      if ((same >> lane) == 1u) sh_run[h] = base_run + __popc(same);
    }
    __syncwarp();
  }
}

// Float rows (16-byte aligned) with float sums: one warp per bucket, 1024 columns per pass, each
// lane holding 8 float4 accumulators, so the 8 16-byte loads of a row are in flight together.
__global__ void cs_gather_f32_kernel(const float* __restrict__ X, int64_t ld, int64_t d, int64_t s, int64_t nchunks,
                                     const uint64_t* __restrict__ incl, const uint32_t* __restrict__ cnt,
                                     const int32_t* __restrict__ perm, const float* __restrict__ sign,
                                     float* __restrict__ SX, int64_t ld_sx) {
  const int warps = blockDim.x / 32;
  const int lane = threadIdx.x & 31;
  for (int64_t h = blockIdx.x * (int64_t)warps + threadIdx.x / 32; h < s; h += (int64_t)gridDim.x * warps) {
    const int64_t first = h * nchunks, last = h * nchunks + nchunks - 1;
    const uint64_t start = incl[first] - cnt[first];
    const uint64_t end = incl[last];
    for (int64_t c0 = 0; c0 < d; c0 += 1024) {
      float4 acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      for (uint64_t p = start; p < end; ++p) {
        const int64_t i = perm[p];
        const float sg = sign[i];
        const float* row = X + i * ld;
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t col = c0 + (q * 32 + lane) * 4;
          if (col + 4 <= d) {
            v[q] = *reinterpret_cast<const float4*>(row + col);
          } else {
            v[q].x = col < d ? row[col] : 0.0f;
            v[q].y = col + 1 < d ? row[col + 1] : 0.0f;
            v[q].z = col + 2 < d ? row[col + 2] : 0.0f;
            v[q].w = col + 3 < d ? row[col + 3] : 0.0f;
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          acc[q].x += sg * v[q].x;
          acc[q].y += sg * v[q].y;
          acc[q].z += sg * v[q].z;
          acc[q].w += sg * v[q].w;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t col = c0 + (q * 32 + lane) * 4;
        const float a[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (col + e < d) SX[h * ld_sx + col + e] = a[e];
      }
    }
  }
}

// One warp per bucket: SX[h] = sum over its rows (in increasing row index) of sign * x.
template <typename T, typename TS>
__global__ void cs_gather_kernel(const TS* X, int64_t ld, int64_t d, int64_t s, int64_t nchunks,
                                 const uint64_t* incl, const uint32_t* cnt, const int32_t* perm, const T* sign,
                                 T* SX, int64_t ld_sx) {
  const int warps = blockDim.x / 32;
  const int lane = threadIdx.x & 31;
  for (int64_t h = blockIdx.x * (int64_t)warps + threadIdx.x / 32; h < s; h += (int64_t)gridDim.x * warps) {
    const int64_t first = h * nchunks, last = h * nchunks + nchunks - 1;
    const uint64_t start = incl[first] - cnt[first];
    const uint64_t end = incl[last];
    for (int64_t c0 = 0; c0 < d; c0 += 32 * 4) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (uint64_t p = start; p < end; ++p) {
        const int64_t i = perm[p];
        const T sg = sign[i];
        const TS* row = X + i * ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t col = c0 + q * 32 + lane;
          if (col < d) acc[q] += sg * cvt<T>(row[col]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t col = c0 + q * 32 + lane;
        if (col < d) SX[h * ld_sx + col] = acc[q];
      }
    }
  }
}

// ------------------------------------------------------------------- scans

// inclusive scan of uint32 -> uint64, 1024 elements per block; block totals to bsum
__global__ void scan_block_kernel(const uint32_t* in, uint64_t* out, int64_t N, uint64_t* bsum) {
  __shared__ uint64_t sh[1024];
  __shared__ uint64_t warp_tot[32];
  const int64_t base = blockIdx.x * 1024LL;
  const int t = threadIdx.x;   // 256 threads x 4 elements
  uint64_t v[4];
  uint64_t run = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + 4 * t + q;
    run += (i < N) ? (uint64_t)in[i] : 0ull;
    v[q] = run;
  }
  // warp-inclusive scan of thread totals
  const int lane = t & 31, w = t >> 5;
  uint64_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t z = lane < 8 ? warp_tot[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    if (lane < 8) warp_tot[lane] = z;
  }
  __syncthreads();
  const uint64_t prefix = (x - run) + (w > 0 ? warp_tot[w - 1] : 0ull);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + 4 * t + q;
    if (i < N) out[i] = v[q] + prefix;
  }
  if (t == 255 && bsum) bsum[blockIdx.x] = x + (w > 0 ? warp_tot[w - 1] : 0ull);
  (void)sh;
}

// exclusive-in-place scan of the block totals by one block (nb <= 16384)
__global__ void scan_totals_kernel(uint64_t* bsum, int64_t nb) {
  __shared__ uint64_t part[1024];
  const int t = threadIdx.x;  // 1024 threads, 16 per thread
  const int per = (int)((nb + 1023) / 1024);
  uint64_t s = 0;
  for (int q = 0; q < per; ++q) {
    const int64_t i = (int64_t)t * per + q;
    if (i < nb) s += bsum[i];
  }
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    uint64_t y = (t >= o) ? part[t - o] : 0ull;
    __syncthreads();
    part[t] += y;
    __syncthreads();
  }
  uint64_t run = (t > 0) ? part[t - 1] : 0ull;
  for (int q = 0; q < per; ++q) {
    const int64_t i = (int64_t)t * per + q;
    if (i < nb) {
      const uint64_t v = bsum[i];
      bsum[i] = run;
      run += v;
    }
  }
}

__global__ void scan_add_kernel(uint64_t* out, int64_t N, const uint64_t* boff) {
  const int64_t i = blockIdx.x * 1024LL + threadIdx.x * 4;
  const uint64_t o = boff[blockIdx.x];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (i + q < N) out[i + q] += o;
}

// ------------------------------------------------------------ sampling weights

template <typename T>
__global__ void max_abs_kernel(const T* beta, int64_t N, double* part, int* status) {
  __shared__ double sh[32];
  double m = 0.0;
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double b = to_d(beta[i]);
    if (!(b >= 0.0) || isinf(b)) bad = true;   // NaN fails b >= 0
    else m = fmax(m, b);
  }
  if (bad) atomicOr(status, STATUS_NONFINITE);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) part[blockIdx.x] = m;
  }
}

template <typename T>
__global__ void quantize_kernel(const T* beta, int64_t N, const double* part, int nparts, uint32_t* W) {
  __shared__ double bmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int p = 0; p < nparts; ++p) m = fmax(m, part[p]);
    bmax = m;
  }
  __syncthreads();
  const double mx = bmax;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t w = 1;
    if (mx > 0.0) {
      const double q = __ddiv_rn(to_d(beta[i]), mx);
      const double f = floor(ldexp(q, 24));
      w = f >= 1.0 ? (uint32_t)f : 1u;
    }
    W[i] = w;
  }
}

// Step tt of an epoch: component index (Philox counter (tt, epoch, tag 3)) and 1/(N q_i)
template <typename T>
__device__ __forceinline__ void draw_index(const uint32_t* W, const uint64_t* cum, int64_t N, uint64_t seed,
                                           uint32_t epoch, uint64_t tt, int uniform, uint32_t& i, T& c) {
  U32x4 w = philox4x32_10(U32x4{(uint32_t)tt, (uint32_t)(tt >> 32), epoch, TAG_SAMPLE}, seed);
  if (uniform) {
    i = (uint32_t)(((uint64_t)w.x * (uint64_t)N) >> 32);
    c = T(1);
  } else {
    const uint64_t total = cum[N - 1];
    const uint64_t u = ((uint64_t)w.y << 32) | (uint64_t)w.x;
    const uint64_t r = __umul64hi(u, total);
    int64_t lo = 0, hi = N - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cum[mid] > r) hi = mid;
      else lo = mid + 1;
    }
    i = (uint32_t)lo;
    c = (T)((double)total / ((double)N * (double)W[lo]));
  }
}

template <typename T>
__global__ void index_stream_kernel(const uint32_t* W, const uint64_t* cum, int64_t N, uint64_t seed, uint32_t epoch,
                                    int64_t t0, int64_t m, int uniform, uint32_t* idx, T* inv_nq) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t i;
    T c;
    draw_index<T>(W, cum, N, seed, epoch, (uint64_t)(t0 + t), uniform, i, c);
    idx[t] = i;
    inv_nq[t] = c;
  }
}

// every job's stream: global step t belongs to the job j with off[j] <= t < off[j + 1]
__global__ void index_stream_batched_kernel(const IdxJob* __restrict__ jobs, const int64_t* __restrict__ off, int nj,
                                            int64_t total, uint32_t epoch) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const IdxJob& J = jobs[lo];
    const int64_t tl = t - off[lo];
    uint32_t i;
    float c;
    draw_index<float>(J.W, J.cum, J.N, J.seed, epoch, (uint64_t)tl, J.uniform, i, c);
    J.idx[tl] = i;
    J.inv_nq[tl] = c;
  }
}

int grid_for(rs_ctx* ctx, int64_t work, int threads = kThreads) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// inclusive uint32 -> uint64 scan (also used by the CountSketch); scratch slot SCR_RED
int scan_u32_to_u64(rs_ctx* ctx, const uint32_t* in, uint64_t* out, int64_t N) {
  const int64_t nb = (N + 1023) / 1024;
  if (nb > 16384) return rs_fail(RS_EINVAL, "scan: %lld elements exceed the 2^24 limit", (long long)N);
  uint64_t* bsum = static_cast<uint64_t*>(rs_scratch(ctx, SCR_RED, nb * sizeof(uint64_t)));
  if (!bsum) return RS_ENOMEM;
  scan_block_kernel<<<(unsigned)nb, 256, 0, ctx->stream>>>(in, out, N, bsum);
  RS_LAUNCH_CHECK(ctx);
  if (nb > 1) {
    scan_totals_kernel<<<1, 1024, 0, ctx->stream>>>(bsum, nb);
    RS_LAUNCH_CHECK(ctx);
    scan_add_kernel<<<(unsigned)nb, 256, 0, ctx->stream>>>(out, N, bsum);
    RS_LAUNCH_CHECK(ctx);
  }
  return RS_OK;
}

template <typename T>
static int sampling_weights_t(rs_ctx* ctx, const T* beta, int64_t N, uint32_t* W) {
  const int g = grid_for(ctx, N);
  double* part = static_cast<double*>(rs_scratch(ctx, SCR_MISC, g * sizeof(double)));
  if (!part) return RS_ENOMEM;
  RS_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  max_abs_kernel<T><<<g, kThreads, 0, ctx->stream>>>(beta, N, part, ctx->d_status);
  RS_LAUNCH_CHECK(ctx);
  quantize_kernel<T><<<g, kThreads, 0, ctx->stream>>>(beta, N, part, g, W);
  RS_LAUNCH_CHECK(ctx);
  int st = 0;
  RS_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (st & STATUS_NONFINITE) return rs_fail(RS_ENONFINITE, "rs_sampling_weights: NaN, Inf or negative beta");
  return RS_OK;
}

template <typename T>
static int countsketch_t(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t s, T* SX, int64_t ld_sx,
                         int32_t* bucket_out, T* sign_out) {
  const int64_t n = X->n, d = X->d;
  int32_t* bucket = bucket_out ? bucket_out : static_cast<int32_t*>(rs_scratch(ctx, SCR_BUCKET, n * 4));
  T* sign = sign_out ? sign_out : static_cast<T*>(rs_scratch(ctx, SCR_SIGN, n * sizeof(T)));
  if (!bucket || !sign) return RS_ENOMEM;
  // rows per chunk of the stable placement: one warp walks a chunk in order, so shorter chunks
  // shorten that serial walk (more counters to scan, which is cheap)
  const int64_t R = 1024;
  const int64_t nchunks = (n + R - 1) / R;
  const int64_t slots = s * nchunks;
  uint32_t* cnt = static_cast<uint32_t*>(rs_scratch(ctx, SCR_CNT, slots * 4));
  uint64_t* incl = static_cast<uint64_t*>(rs_scratch(ctx, SCR_CSR, slots * 8 + n * 4 + 16));
  if (!cnt || !incl) return RS_ENOMEM;
  int32_t* perm = reinterpret_cast<int32_t*>(incl + slots);
  cs_hash_kernel<T><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(seed, n, s, bucket, sign);
  RS_LAUNCH_CHECK(ctx);
  const size_t shm = s * sizeof(uint32_t);
  if (shm > 200 * 1024) return rs_fail(RS_EINVAL, "rs_countsketch: s = %lld buckets exceed the on-chip table", (long long)s);
  RS_CUDA_TRY(cudaFuncSetAttribute(cs_chunk_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  RS_CUDA_TRY(cudaFuncSetAttribute(cs_place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  cs_chunk_count_kernel<<<(unsigned)nchunks, 1024, shm, ctx->stream>>>(bucket, n, s, R, nchunks, cnt);
  RS_LAUNCH_CHECK(ctx);
  RS_TRY(scan_u32_to_u64(ctx, cnt, incl, slots));
  cs_place_kernel<<<(unsigned)nchunks, 256, shm, ctx->stream>>>(bucket, n, s, R, nchunks, incl, cnt, perm);
  RS_LAUNCH_CHECK(ctx);
  const int warps = 8;
  const int64_t g = std::min<int64_t>((s + warps - 1) / warps, (int64_t)ctx->num_sms * 16);
  switch (X->dtype) {
    case RS_F64:
      cs_gather_kernel<T, double><<<(unsigned)g, 32 * warps, 0, ctx->stream>>>(
          static_cast<const double*>(X->data), X->ld, d, s, nchunks, incl, cnt, perm, sign, SX, ld_sx);
      break;
    case RS_F32:
      if constexpr (std::is_same<T, float>::value)
        cs_gather_f32_kernel<<<(unsigned)g, 32 * warps, 0, ctx->stream>>>(
            static_cast<const float*>(X->data), X->ld, d, s, nchunks, incl, cnt, perm, sign, SX, ld_sx);
      else
        cs_gather_kernel<T, float><<<(unsigned)g, 32 * warps, 0, ctx->stream>>>(
            static_cast<const float*>(X->data), X->ld, d, s, nchunks, incl, cnt, perm, sign, SX, ld_sx);
      break;
    case RS_BF16:
      cs_gather_kernel<T, __nv_bfloat16><<<(unsigned)g, 32 * warps, 0, ctx->stream>>>(
          static_cast<const __nv_bfloat16*>(X->data), X->ld, d, s, nchunks, incl, cnt, perm, sign, SX, ld_sx);
      break;
    default:
      return rs_fail(RS_EUNSUPPORTED, "rs_countsketch: dtype %d", X->dtype);
  }
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int countsketch_dispatch(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t s, void* SX, int64_t ld_sx,
                         int32_t* bucket_out, void* sign_out) {
  if (X->dtype == RS_F64)
    return countsketch_t<double>(ctx, X, seed, s, static_cast<double*>(SX), ld_sx, bucket_out,
                                 static_cast<double*>(sign_out));
  return countsketch_t<float>(ctx, X, seed, s, static_cast<float*>(SX), ld_sx, bucket_out,
                              static_cast<float*>(sign_out));
}

int gaussian_t_bf16_dispatch(rs_ctx* ctx, uint64_t seed, int64_t n, int64_t k, __nv_bfloat16* out, int64_t ld) {
  const int64_t work = n * ((k + 3) / 4);
  gaussian_t_bf16_kernel<<<grid_for(ctx, work), kThreads, 0, ctx->stream>>>(seed, n, k, out, ld);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int gaussian_dispatch(rs_ctx* ctx, uint64_t seed, int64_t row0, int64_t rows, int64_t cols, int32_t dtype, void* out,
                      int64_t ld) {
  const int64_t work = rows * ((cols + 3) / 4);
  if (dtype == RS_F64)
    gaussian_kernel<double><<<grid_for(ctx, work), kThreads, 0, ctx->stream>>>(seed, row0, rows, cols,
                                                                                 static_cast<double*>(out), ld);
  else if (dtype == RS_F32)
    gaussian_kernel<float><<<grid_for(ctx, work), kThreads, 0, ctx->stream>>>(seed, row0, rows, cols,
                                                                               static_cast<float*>(out), ld);
  else
    return rs_fail(RS_EUNSUPPORTED, "rs_gaussian: dtype %d", dtype);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int index_stream_dispatch(rs_ctx* ctx, const uint32_t* W, const uint64_t* cum, int64_t N, uint64_t seed,
                          int64_t epoch, int64_t t0, int64_t m, int32_t sampling, int32_t dtype, uint32_t* idx,
                          void* inv_nq) {
  const int g = grid_for(ctx, m);
  const int uni = sampling == RS_SAMPLE_UNIFORM;
  if (dtype == RS_F64)
    index_stream_kernel<double><<<g, kThreads, 0, ctx->stream>>>(W, cum, N, seed, (uint32_t)epoch, t0, m, uni, idx,
                                                                  static_cast<double*>(inv_nq));
  else
    index_stream_kernel<float><<<g, kThreads, 0, ctx->stream>>>(W, cum, N, seed, (uint32_t)epoch, t0, m, uni, idx,
                                                                 static_cast<float*>(inv_nq));
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int index_stream_batched(rs_ctx* ctx, const IdxJob* jobs, const int64_t* off, int nj, int64_t total, uint32_t epoch) {
  if (nj < 1 || total < 1) return RS_OK;
  index_stream_batched_kernel<<<grid_for(ctx, total), kThreads, 0, ctx->stream>>>(jobs, off, nj, total, epoch);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int sampling_weights_dispatch(rs_ctx* ctx, const void* beta, int32_t dtype, int64_t N, uint32_t* W) {
  if (dtype == RS_F64) return sampling_weights_t<double>(ctx, static_cast<const double*>(beta), N, W);
  if (dtype == RS_F32) return sampling_weights_t<float>(ctx, static_cast<const float*>(beta), N, W);
  return rs_fail(RS_EUNSUPPORTED, "rs_sampling_weights: dtype %d", dtype);
}

extern "C" {

int rs_philox_words(rs_ctx* ctx, uint64_t seed, uint32_t c2, uint32_t c3, int64_t count, uint32_t* out) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(count >= 0, "rs_philox_words: count < 0");
  RS_CHECK_ARG(out && aligned16(out), "rs_philox_words: out must be a 16-byte aligned device pointer");
  if (count == 0) return RS_OK;
  philox_words_kernel<<<grid_for(ctx, count), kThreads, 0, ctx->stream>>>(seed, c2, c3, count, out);
  RS_LAUNCH_CHECK(ctx);
  return RS_OK;
}

int rs_gaussian(rs_ctx* ctx, uint64_t seed, int64_t row0, int64_t rows, int64_t cols, int32_t dtype, void* out,
                int64_t ld) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(rows >= 0 && cols >= 0 && row0 >= 0 && ld >= cols, "rs_gaussian: bad shape");
  RS_CHECK_ARG(out != nullptr || rows * cols == 0, "rs_gaussian: null output");
  if (rows == 0 || cols == 0) return RS_OK;
  return gaussian_dispatch(ctx, seed, row0, rows, cols, dtype, out, ld);
}

int rs_countsketch(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t s, void* SX, int64_t ld_sx,
                   int32_t* bucket_out, void* sign_out) {
  RS_TRY(rs_enter(ctx));
  RS_TRY(check_matrix(X, "rs_countsketch X"));
  RS_CHECK_ARG(s >= 1 && s <= (1 << 20), "rs_countsketch: s out of range");
  RS_CHECK_ARG(SX && ld_sx >= X->d, "rs_countsketch: bad output");
  return countsketch_dispatch(ctx, X, seed, s, SX, ld_sx, bucket_out, sign_out);
}

int rs_sampling_weights(rs_ctx* ctx, const void* beta, int32_t dtype, int64_t N, uint32_t* W) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(beta && W && N >= 1, "rs_sampling_weights: bad arguments");
  return sampling_weights_dispatch(ctx, beta, dtype, N, W);
}

int rs_sampling_table(rs_ctx* ctx, const uint32_t* W, int64_t N, uint64_t* cum) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(W && cum && N >= 1, "rs_sampling_table: bad arguments");
  return scan_u32_to_u64(ctx, W, cum, N);
}

int rs_index_stream(rs_ctx* ctx, const uint32_t* W, const uint64_t* cum, int64_t N, uint64_t seed, int64_t epoch,
                    int64_t t0, int64_t m, int32_t sampling, int32_t dtype, uint32_t* idx, void* inv_nq) {
  RS_TRY(rs_enter(ctx));
  RS_CHECK_ARG(N >= 1 && N < (1LL << 32) && m >= 0 && t0 >= 0 && epoch >= 0 && epoch < (1LL << 32),
               "rs_index_stream: bad sizes");
  RS_CHECK_ARG(sampling == RS_SAMPLE_UNIFORM || (W && cum), "rs_index_stream: importance sampling needs W and cum");
  RS_CHECK_ARG(idx && inv_nq, "rs_index_stream: null output");
  RS_CHECK_ARG(dtype == RS_F64 || dtype == RS_F32, "rs_index_stream: dtype must be RS_F64 or RS_F32");
  if (m == 0) return RS_OK;
  return index_stream_dispatch(ctx, W, cum, N, seed, epoch, t0, m, sampling, dtype, idx, inv_nq);
}

}  // extern "C"
