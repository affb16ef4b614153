/*
 * rs.h -- C ABI of the GB300 (sm_103a) library for ridge regression by sketched
 * preconditioned SVRG (Gonen, Orabona, Shalev-Shwartz, "Solving Ridge Regression
 * using Sketched Preconditioned SVRG").
 *
 * Problem (Eq. (1)):  min_w  L(w) = (1/n) sum_i 1/2 (w^T x_i - y_i)^2 + (lam/2) ||w||^2.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major; row i of X is the example x_i.  ``ld`` is the row
 *     stride in elements; ld * sizeof(element) and the base address must be
 *     multiples of 16 bytes (vectorised and asynchronous copies), else RS_EINVAL.
 *   - Every array argument is a caller-owned DEVICE pointer unless its comment
 *     says "host".  The library never frees caller memory.
 *   - "T" below is the compute type of the call: double when the data matrix is
 *     RS_F64, float otherwise.  Vectors and small matrices (y, w, mu, V, Q, ...)
 *     are T unless stated.
 *   - Calls are ordered on the context's CUDA stream and return without a host
 *     synchronisation unless stated; a status of RS_OK means the work was
 *     enqueued.  rs_svrg_solve, rs_solve and rs_objective synchronise.
 *   - On a non-zero status nothing is guaranteed about outputs; the message is
 *     available from rs_last_error() (per host thread).  No C++ exception
 *     crosses this boundary, and there is no CPU fallback: without a CUDA
 *     device every compute call returns RS_ECUDA.
 *   - The context owns scratch memory (grown on demand with cudaMalloc, kept
 *     until rs_destroy) and a device status word that kernels use to report
 *     non-finite data.
 *   - Random draws come from the counter-based Philox4x32-10 generator (Salmon
 *     et al., SC'11), key = the 64-bit seed, counter words
 *       Gaussian entry (i, 4g+r):  (lo32(i), hi32(i), g, 1)
 *       CountSketch row i:         (lo32(i), hi32(i), 0, 2)
 *       SVRG step t of epoch e:    (lo32(t), hi32(t), e, 3)
 *     so results are reproducible bit for bit for a given seed.
 */
#ifndef RS_H
#define RS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RS_ABI_VERSION 1

/* status codes */
enum {
  RS_OK = 0,
  RS_EINVAL = 1,          /* bad shape, stride, alignment, parameter */
  RS_ENOMEM = 2,          /* scratch allocation failed */
  RS_ECUDA = 3,           /* CUDA runtime error (message has the CUDA error string) */
  RS_ENONFINITE = 4,      /* NaN or Inf met in the data or an iterate */
  RS_ETIMEOUT = 5,        /* a bounded device-side wait gave up */
  RS_EDIVERGED = 6,       /* SVRG iterate grew without bound (step size too large) */
  RS_ENOTCONVERGED = 7,   /* tolerance not met within the epoch budget (w_out still written) */
  RS_EUNSUPPORTED = 8     /* valid request this build does not implement */
};

typedef enum { RS_F64 = 0, RS_F32 = 1, RS_BF16 = 2, RS_FP8E4M3 = 3 } rs_dtype;

typedef struct rs_ctx rs_ctx;

/* Dense row-major matrix in device memory. */
typedef struct {
  const void* data;        /* n rows of ld elements of type dtype */
  const float* row_scale;  /* RS_FP8E4M3 only: n per-row scales (value = code * scale); else NULL */
  int64_t n, d, ld;        /* rows, columns, row stride (elements) */
  int32_t dtype;           /* rs_dtype */
  int32_t reserved;
} rs_matrix;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device ``device`` issuing work on ``cuda_stream``
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the handle. */
int rs_create(rs_ctx** ctx, int device, void* cuda_stream);
/* Free the context and its scratch memory (synchronises its stream). */
int rs_destroy(rs_ctx* ctx);
/* Change the stream later calls are ordered on. */
int rs_set_stream(rs_ctx* ctx, void* cuda_stream);
/* Message of the last non-zero status returned on this host thread ("" if none). */
const char* rs_last_error(void);
/* RS_ABI_VERSION of the loaded library. */
int rs_abi_version(void);
/* Number of kernel launches this context has issued since creation. */
int64_t rs_launch_count(const rs_ctx* ctx);

/* ------------------------------------------------------- random streams */

/* Raw Philox4x32-10 words: out[4*i + w] = word w of counter (lo32(i), hi32(i), c2, c3)
 * with key ``seed``, i = 0..count-1.  out: 4*count uint32. */
int rs_philox_words(rs_ctx* ctx, uint64_t seed, uint32_t c2, uint32_t c3, int64_t count,
                    uint32_t* out);

/* Gaussian test matrix of Alg. 2: out[r*ld + j] = Pi(row0 + r, j), N(0,1), for
 * r < rows, j < cols.  Entry (i, 4g+r) is Box-Muller on the words of counter
 * (i, g, tag 1): words (0,1) -> r = 0,1 and (2,3) -> r = 2,3, each word mapped to
 * the uniform (2*(w>>9)+1) 2^-24.  dtype RS_F64 evaluates log/sqrt/sincospi in
 * double, RS_F32 in float (within a few float ulps of the double values). */
int rs_gaussian(rs_ctx* ctx, uint64_t seed, int64_t row0, int64_t rows, int64_t cols,
                int32_t dtype, void* out, int64_t ld);

/* CountSketch S X (s x d, T, row stride ld_sx): row h is the sum of sigma(i) x_i over
 * the rows i with h(i) = h, added in increasing i (deterministic).
 * h(i) = floor(w0 * s / 2^32), sigma(i) = -1 iff bit 31 of w1, words of counter
 * (i, 0, tag 2).  bucket_out (int32, n) and sign_out (T, n) may be NULL. */
int rs_countsketch(rs_ctx* ctx, const rs_matrix* X, uint64_t seed, int64_t s, void* SX,
                   int64_t ld_sx, int32_t* bucket_out, void* sign_out);

/* ------------------------------------------------------------- sketch (Alg. 2) */

enum { RS_SKETCH_GAUSSIAN = 0, RS_SKETCH_COUNTSKETCH = 1 };

typedef struct {
  int32_t kind;        /* RS_SKETCH_GAUSSIAN: Pi ~ N(0,1)^{n x k};
                          RS_SKETCH_COUNTSKETCH: Pi = S^T G', S an s x n CountSketch, G' ~ N(0,1)^{s x k} */
  int32_t k;           /* rank, 1 <= k <= min(d, 256) */
  int64_t s;           /* CountSketch rows (kind 1); 0 = min(n, 64 k) */
  int32_t q_blocks;    /* Krylov blocks q of Alg. 2 (>= 1; 1 = single-pass range sketch) */
  int32_t reserved;
  uint64_t seed;
} rs_sketch_params;

/* First Krylov block of Alg. 2 without its n^{-1/2}: Y = X^T Pi (d x k, T, row-major). */
int rs_range_sketch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* Y);

/* Orthonormalise the k columns of Y (d x k, T) (Alg. 2, "orthonormalize"): Cholesky-QR
 * applied twice, Gram matrices accumulated and factored in double.  Q (d x k, T) spans Y
 * with Q^T Y upper triangular with positive diagonal.  RS_EINVAL if Y is rank deficient
 * to working precision. */
int rs_orthonormalize(rs_ctx* ctx, const void* Y, int64_t d, int64_t k, int32_t dtype, void* Q);

/* Symmetric eigen-decomposition G = W diag(evals) W^T of a k x k matrix (double, row-major)
 * by cyclic Jacobi on one thread block.  evals descending (double, k); W (double, k x k,
 * column j = eigenvector j).  prec RS_F64 iterates in double, RS_F32 in float. */
int rs_sym_eig(rs_ctx* ctx, const double* G, int64_t k, int32_t prec, double* evals, double* W);

/* Rayleigh-Ritz (Alg. 2, last two steps) for Q (d x k, T, orthonormal columns):
 * G = (X Q)^T (X Q) / n (accumulated in double), G = W diag(sigma2) W^T,
 * V = Q W (d x k, T), sigma2 (double, k) descending: the Ritz pairs of C = X^T X / n. */
int rs_ritz(rs_ctx* ctx, const rs_matrix* X, const void* Q, int64_t k, void* V, double* sigma2);

/* Alg. 2 composed: range sketch, q-1 products with C, orthonormalisation, Rayleigh-Ritz.
 * V (d x k, T): approximate leading eigenvectors of C; sigma2 (double, k) descending. */
int rs_sketch(rs_ctx* ctx, const rs_matrix* X, const rs_sketch_params* p, void* V, double* sigma2);

/* --------------------------------------------------- preconditioner (Eq. (11)) */

/* Apply the sketched preconditioner of Eq. (11) without its scalar c = (sigma2_k + lam)^{-1/2}:
 *   M = I - V (I - D') V^T,   D'_j = sqrt((sigma2_k + lam) / (sigma2_j + lam)),
 * and write the N = n + d components of Sec. 5.1 as the rows of Z (Xt):
 *   rows 0..n-1:   z_i = M x_i            (x~_i of Alg. 3),
 *   rows n..n+d-1: z_{n+j} = M e_j        (b_j of Alg. 3; M is symmetric).
 * Xt->data is written (cast away const); Xt->n must be n + d, Xt->d = d, Xt->dtype equal
 * to X->dtype (RS_F64, RS_F32 or RS_BF16), or RS_BF16 for RS_F32 data (each component is
 * formed in float and rounded once), or RS_FP8E4M3 for RS_F32 / RS_BF16 data: one scale per row,
 * s_i = max_c |z_ic| / 448, written to Xt->row_scale (float, n + d), codes e4m3(z_ic / s_i) rounded
 * to nearest; beta is then computed from the stored values.
 * beta (T, n + d): smoothness beta_i = gamma_i ||z_i||^2 with gamma_i = (n+d)/n for data
 * rows and lam (n+d) for regulariser rows (Alg. 3).  beta_hat (host, nullable): mean beta. */
int rs_precondition(rs_ctx* ctx, const rs_matrix* X, const void* V, const double* sigma2, int64_t k,
                    double lambda, rs_matrix* Xt, void* beta, double* beta_hat);

/* w = M w~ (d, T): map an iterate of the preconditioned problem back (Eq. (4)). */
int rs_map_output(rs_ctx* ctx, const void* V, const double* sigma2, int64_t d, int64_t k,
                  double lambda, int32_t dtype, const void* w_tilde, void* w);

/* ------------------------------------------------------ sampling (Alg. 1) */

/* Integer sampling weights W_i = max(1, floor(2^24 beta_i / max_j beta_j)) (uint32, N),
 * computed with one double division per entry, so equal beta gives equal W on any
 * machine.  RS_ENONFINITE if a beta is NaN/Inf or negative. */
int rs_sampling_weights(rs_ctx* ctx, const void* beta, int32_t dtype, int64_t N, uint32_t* W);

/* Inclusive prefix sums cum[i] = W_0 + ... + W_i (uint64, N); q_i = W_i / cum[N-1]. */
int rs_sampling_table(rs_ctx* ctx, const uint32_t* W, int64_t N, uint64_t* cum);

enum { RS_SAMPLE_IMPORTANCE = 0, RS_SAMPLE_UNIFORM = 1 };

/* Index stream of Alg. 1 for steps t = t0..t0+m-1 of epoch ``epoch``: with u the 64-bit
 * word w1 2^32 + w0 of counter (t, epoch, tag 3) and T = cum[N-1],
 *   IMPORTANCE: r = floor(u T / 2^64), idx = smallest i with cum[i] > r,
 *   UNIFORM:    idx = floor(w0 N / 2^32)   (W and cum may be NULL),
 * and inv_nq[t] = 1 / (N q_idx) (T dtype) with q_i = W_i / T (1/(N q) = 1 for UNIFORM).
 * idx: uint32 (m), inv_nq: dtype (m). */
int rs_index_stream(rs_ctx* ctx, const uint32_t* W, const uint64_t* cum, int64_t N, uint64_t seed,
                    int64_t epoch, int64_t t0, int64_t m, int32_t sampling, int32_t dtype,
                    uint32_t* idx, void* inv_nq);

/* --------------------------------------------------------- SVRG (Alg. 1) */

/* Full gradient of the preconditioned objective (Alg. 1, v_bar = grad F(w_bar)) over the
 * N = n + d rows z_i of Z (layout of rs_precondition):
 *   mu = (1/N) sum_i gamma_i (z_i^T w - y_i) z_i,  y_i = 0 for i >= n,
 * which equals X~^T (X~ w - y)/n + lam M^T M w.  One streaming pass over Z; deterministic. */
int rs_full_gradient(rs_ctx* ctx, const rs_matrix* Z, const void* y, int64_t n, double lambda,
                     const void* w, void* mu);

/* Allocation-free rs_full_gradient (the paper has no counterpart; this is a service to callers).
 * Some callers cannot call cudaMalloc: applications whose device memory is owned end to end by
 * their own pool or arena (an allocation outside it fails once the pool has reserved the device,
 * or breaks its accounting) and latency-critical services that must stay off the driver's
 * allocation path (cudaMalloc/cudaFree can synchronise the device).  This entry point takes no
 * context and allocates nothing: its per-block partial sums live in a 2 MiB array in the
 * library's device data, which every GPU that loads the library holds until the process exits.
 * Same arguments and result as rs_full_gradient (mu is written on ``cuda_stream``, a
 * cudaStream_t, NULL = legacy default stream, on the caller's current device); the same kernels
 * run, so results match rs_full_gradient.
 *   - Z must be RS_F32 or RS_F64 (y, w, mu of the same type); RS_BF16 and RS_FP8E4M3 rows return
 *     RS_EINVAL before anything is launched (rs_full_gradient takes them).
 *   - Limit: d <= 1024 for RS_F32 and d <= 512 for RS_F64 rows; larger d returns RS_EINVAL.
 *   - The first call on each device resolves the array's device address (once per device, with
 *     that device current); make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents; nothing in it needs
 *     to start at zero (each call overwrites every partial it reads).  Calls that overlap on the
 *     GPU (different streams, or different host threads without ordering) race on the array. */
int rs_full_gradient_static(void* cuda_stream, const rs_matrix* Z, const void* y, int64_t n, double lambda,
                            const void* w, void* mu);

/* One outer iteration of Alg. 1 for a given index stream (idx, inv_nq from rs_index_stream):
 *   w_0 = w_bar;  w_t = w_{t-1} - eta ((grad f_i(w_{t-1}) - grad f_i(w_bar)) inv_nq[t] + mu);
 *   w_next = (1/m) sum_{t=1..m} w_t  (average != 0)  or  w_m  (average == 0),
 * with grad f_i(w) - grad f_i(w_bar) = gamma_i (z_i^T (w - w_bar)) z_i.  The m sequential
 * steps are evaluated in blocks of 64 with the block's Gram matrix, which gives the same
 * iterates as the step-by-step recursion up to rounding.  w_next must not alias w_bar. */
int rs_svrg_epoch(rs_ctx* ctx, const rs_matrix* Z, int64_t n, double lambda, const uint32_t* idx,
                  const void* inv_nq, int64_t m, double eta, const void* w_bar, const void* mu,
                  int32_t average, void* w_next);

typedef struct {
  double lambda;
  double eta;          /* <= 0: Thm 2 value 0.1 / beta_hat; eta_mult > 0 overrides */
  double eta_mult;     /* > 0: eta = eta_mult / beta_hat */
  int64_t m;           /* inner steps per epoch; <= 0: Thm 2 value ceil(beta_hat / lam) */
  int32_t epochs;      /* outer iterations S */
  int32_t epoch0;      /* first epoch number (resume at an epoch boundary) */
  int32_t sampling;    /* RS_SAMPLE_IMPORTANCE (q_i ~ beta_i) or RS_SAMPLE_UNIFORM */
  int32_t average;     /* 1: epoch output is the average of w_1..w_m (Alg. 1); 0: w_m */
  uint64_t seed;
  int32_t refine;      /* 1: form each snapshot's full gradient on the stored data X,
                          mu = M (X^T (X M w~ - y)/n + lam M w~), instead of on Z; the fixed point
                          is then exact for X as stored even when Z is a rounded (BF16) copy */
  int32_t reserved;
} rs_svrg_params;

typedef struct {
  int32_t capacity;      /* number of epochs the buffers below hold */
  int32_t epochs_run;    /* written */
  void* snapshots;       /* device, nullable: capacity x d (T), w_bar_s in ORIGINAL coordinates (M w~) */
  double* mu_norm2;      /* host, nullable: ||mu||^2 at the start of each epoch */
  float* epoch_ms;       /* host, nullable: cumulative device time at the end of each epoch */
} rs_history;

/* Alg. 1 on the components Z (rs_precondition layout, N = n + d rows; RS_F64, RS_F32, RS_BF16 or
 * RS_FP8E4M3 storage; FP8 components need p->refine, X and beta) for p->epochs epochs, starting from w0 (preconditioned coordinates, nullable = 0).
 * X (n x d, stored like Z, or RS_F32 for RS_BF16 components) is the stored data, required
 * when p->refine is set, else
 * nullable.  beta (T, N; nullable = recomputed from Z) sets the sampling weights.  V/sigma2/k
 * give M for the output map: w_out = M w~_S (original coordinates, Alg. 3 read as
 * w = P^{-1/2} w~).  eta_used / m_used (host, nullable) receive the resolved step size and
 * epoch length.  Synchronises.  RS_ENONFINITE / RS_EDIVERGED if an iterate becomes
 * non-finite, RS_ETIMEOUT if a bounded device wait of the inner loop gave up. */
int rs_svrg_solve(rs_ctx* ctx, const rs_matrix* Z, const rs_matrix* X, const void* y, const void* beta, const void* V,
                  const double* sigma2, int64_t k, const rs_svrg_params* p, const void* w0,
                  void* w_out, rs_history* hist, double* eta_used, int64_t* m_used);

/* Accelerated SVRG (the accelerated variant Thm 1 refers to; the paper names it in Sec. 1 without
 * fixing a scheme): Catalyst (Lin, Mairal and Harchaoui, NIPS 2015) around Alg. 1 on the same
 * components.  Outer iteration t = 1..outer minimises the proximal problem
 *   L(w) + (kappa/2) ||w - c_{t-1}||^2
 * with p->epochs epochs of Alg. 1 (as rs_svrg_solve with p; epoch numbers continue from p->epoch0
 * across the outer iterations, so every epoch draws its own index stream) warm-started at the
 * previous outer iterate.  In the component form only the regulariser rows change: their weight
 * becomes (lambda + kappa)(n + d) and their label kappa c_j / (lambda + kappa), i.e. every snapshot
 * gradient is shifted by -kappa M c and the smoothness constants of those rows scale by
 * (lambda + kappa) / lambda (eta and the importance weights follow).  Then
 *   alpha_t^2 = (1 - alpha_t) alpha_{t-1}^2 + q alpha_t,  q = lambda / (lambda + kappa),  alpha_0 = sqrt(q),
 *   c_t = x_t + alpha_{t-1} (1 - alpha_{t-1}) / (alpha_{t-1}^2 + alpha_t) (x_t - x_{t-1}),
 * with x_t = M w~_t in original coordinates; w_out = x_outer.
 * cp->kappa <= 0 selects kappa = max(0, beta^ / (n + d) - lambda) (beta^ the mean smoothness of the
 * original components; Catalyst's choice for SVRG).  beta: smoothness constants for lambda as
 * rs_precondition writes them (nullable except for FP8 components: then recomputed from Z).
 * hist (nullable): capacity >= outer; snapshots receives x_t, epoch_ms the cumulative time at the end
 * of each outer iteration.  kappa_used (host, nullable).  Synchronises.  Errors as rs_svrg_solve;
 * RS_EINVAL for outer < 1 or epochs < 1. */
typedef struct {
  double kappa;        /* proximal weight (<= 0: the default above) */
  int32_t outer;       /* outer iterations */
  int32_t reserved;
} rs_catalyst_params;

int rs_catalyst_solve(rs_ctx* ctx, const rs_matrix* Z, const rs_matrix* X, const void* y, const void* beta,
                      const void* V, const double* sigma2, int64_t k, const rs_svrg_params* p,
                      const rs_catalyst_params* cp, void* w_out, rs_history* hist, double* kappa_used);

/* Autotuning of the launch layouts (no counterpart in the paper).  For components Z (storage type,
 * width d) this times, on this GPU, every layout that fits for
 *   - the inner-loop chain of Alg. 1: thread-block cluster size (1..16 blocks, each owning at most
 *     256 columns), threads per block (256 or 512) and ring stages (2..4), on a probe epoch of 8192
 *     uniformly drawn steps (one warm-up and three timed launches each);
 *   - the full-gradient pass for RS_F32 / RS_BF16 rows: the ring stages of its bulk-copy pipeline
 *     (2, 3, 4, 6, 8 within the shared-memory budget), one pass each (warm-up + three timed);
 * keeps the fastest of each in the context, and later calls on this context with components of the
 * same storage type and width use them (rs_svrg_epoch, rs_svrg_solve, rs_solve, rs_full_gradient,
 * rs_catalyst_solve).  A second call for the same shape times nothing (report->cached = 1).
 * Synchronises.  report (host): the chosen layout and its time per probe launch / pass. */
typedef struct {
  int32_t chain_cluster, chain_threads, chain_stages;
  float chain_ms;           /* per launch of the 8192-step probe */
  int32_t fullgrad_stages;  /* 0 when the storage type has no tunable full-gradient kernel */
  float fullgrad_ms;        /* per pass */
  int32_t candidates;       /* layouts timed by this call */
  int32_t cached;           /* 1: both choices were already in the context */
} rs_tune_report;

int rs_autotune(rs_ctx* ctx, const rs_matrix* Z, int64_t n, rs_tune_report* report);

/* Alg. 3 end to end: sketch (Alg. 2), preconditioner and transformed components (Eq. (11),
 * Sec. 5.1), SVRG (Alg. 1), w_out = M w~ (Eq. (4)).  X may be RS_F64, RS_F32 or RS_BF16 (the
 * components are stored in the same type; with RS_BF16 set p->refine).  X->data, y and w_out may be HOST
 * pointers (detected): the data is then copied to scratch memory and the result back inside
 * the call.  Scratch holds (n + d) x d elements for the components.  Synchronises. */
int rs_solve(rs_ctx* ctx, const rs_matrix* X, const void* y, const rs_sketch_params* sp,
             const rs_svrg_params* p, void* w_out, rs_history* hist);

/* ----------------------------------------------------- accuracy (Eq. (1)) */

/* out[0] = L(w) of Eq. (1); out[1] = 1/2 e^T (C + lam I) e = (1/2n)||X e||^2 + (lam/2)||e||^2
 * with e = w - w_ref, which is L(w) - L(w_ref) when w_ref minimises L (out[1] = 0 if w_ref
 * is NULL).  Accumulated in double.  out: host, 2 doubles.  Synchronises. */
int rs_objective(rs_ctx* ctx, const rs_matrix* X, const void* y, double lambda, const void* w,
                 const void* w_ref, double* out);

/* ------------------------------------------------------- batched solves
 *
 * Many ridge problems, each at several lambda (a regularisation path) and/or several SVRG
 * settings, solved together: one Alg. 2 sketch per problem shared by all its chains, one set of
 * components Z (Eq. (11), Sec. 5.1) per (problem, lambda), and per epoch one pass over each
 * problem's stored data for the snapshot gradients of all its chains (refined form:
 * U = [M_c w~_c], R = X U - y 1^T, G = X^T R / n, mu_c = M_c (G e_c + lam_c M_c w~_c)), one launch
 * for every chain's index stream, one for every chain's block preparation, and one per distinct
 * d for the inner loops themselves (one thread-block cluster per chain).  Epochs 2..S are
 * captured in one CUDA graph and launched once.  The paper solves one problem at a time;
 * batching is this library's extension. */

typedef struct {
  rs_matrix X;        /* n x d data, RS_F32 or RS_BF16 (all problems of a call share the dtype) */
  const float* y;     /* n labels */
  int32_t k;          /* sketch rank, 1 <= k <= min(d, 256); 0 = max(1, d / 16) */
  int32_t reserved;
} rs_problem;

typedef struct {
  int32_t problem;    /* index into the problem array */
  int32_t reserved;
  double lambda;      /* > 0 */
  double eta_mult;    /* eta = eta_mult / beta^, beta^ the mean smoothness of this chain's
                         components; <= 0 selects 1 */
  int64_t m;          /* epoch length; <= 0 selects 2 n */
  uint64_t seed;      /* SVRG index stream seed (Philox key) */
  float* w_out;       /* d floats (device): w = M w~_S in original coordinates */
  float* snapshots;   /* nullable: epochs x d floats (device), w after each epoch */
} rs_chain;

typedef struct {
  int32_t epochs;       /* S >= 1 */
  int32_t sketch_kind;  /* RS_SKETCH_GAUSSIAN or RS_SKETCH_COUNTSKETCH */
  int32_t q_blocks;     /* Krylov blocks of Alg. 2 (>= 1) */
  int32_t refine;       /* 1: snapshot gradients on the stored data (required for RS_BF16);
                           0: one pass over each chain's components Z */
  int32_t use_graph;    /* 1: capture epochs 2..S in a CUDA graph */
  int32_t average;      /* epoch output = average of the iterates (Alg. 1) */
  uint64_t sketch_seed; /* problem p is sketched with seed sketch_seed + p */
} rs_batch_params;

/* Solve every chain (host array of nchain descriptors; each chain's problem, lambda, step size,
 * epoch length, seed and outputs).  Chains with the same (problem, lambda) share their
 * components.  epoch_ms (host, nullable, epochs floats): time from the start of the first epoch
 * to the end of epoch s.  Synchronises.  RS_ENOMEM if the workspace (components of every
 * (problem, lambda) pair plus per-chain buffers) does not fit; RS_ENONFINITE / RS_ETIMEOUT as
 * rs_svrg_solve. */
int rs_solve_batched(rs_ctx* ctx, const rs_problem* probs, int32_t nprob, const rs_chain* chains, int32_t nchain,
                     const rs_batch_params* p, float* epoch_ms);

/* tr(C) = ||X||_F^2 / n (Eq. (2)), accumulated in double; the tail sum of the spectrum in the
 * runtime model of Thm 1 is tr(C) minus the leading sketched eigenvalues.  out: host, 1
 * double.  Synchronises. */
int rs_trace_c(rs_ctx* ctx, const rs_matrix* X, double* out);

/* ------------------------------------------------------- speed-up diagnostic
 *
 * The ratio after Thm 1 (Sec. 2; plotted against k in Fig. 1): preconditioned SVRG is faster than
 * plain SVRG by about
 *   ratio(k) = sum_{i=1..d} lambda_i / (k lambda_k + sum_{i>k} lambda_i),
 * and by sqrt(ratio(k)) with acceleration, lambda_i the eigenvalues of C = X^T X / n.  From a sketch
 * it is evaluated with sum_i lambda_i = tr(C) (rs_trace_c), lambda_i = sigma2[i-1] for i <= k and
 * the tail sum tr(C) - sum_{i<=k} sigma2[i-1] (left-to-right prefix sum in double).
 * sigma2: device, kmax doubles, descending (the Ritz values of rs_sketch of rank >= kmax).
 * ratio (device, kmax doubles): ratio[k-1] = ratio(k); ratio_accel (device, nullable): its square
 * roots.  A non-positive denominator gives NaN.  RS_EINVAL unless 1 <= kmax <= 65536 and tr(C) is
 * finite and positive.  Enqueued on the context's stream. */
int rs_speedup_ratio(rs_ctx* ctx, const double* sigma2, int64_t kmax, double trace_c, double* ratio,
                     double* ratio_accel);

/* Check of the bounded device-side waits (no counterpart in the paper).  Every wait in this
 * library's kernels (mbarrier phases of the copy/MMA pipelines, the cluster exchange of the inner
 * loop) gives up after a budget of clock cycles, sets a bit in the context's status word and lets
 * the kernel return, so the call reports RS_ETIMEOUT and the context stays usable.  This entry runs
 * one such wait on an mbarrier expecting one arrival: with complete != 0 the arrival is made and the
 * call returns RS_OK; with complete == 0 nothing arrives, the wait gives up after budget_cycles
 * (1 .. 4e9, about two seconds at most) and the call returns RS_ETIMEOUT.  Synchronises. */
int rs_wait_probe(rs_ctx* ctx, int64_t budget_cycles, int32_t complete);

/* ------------------------------------------------------- parameter proposal
 *
 * The paper sets the SVRG parameters from theory (Sec. 3, the SVRG theorem of Xiao and Zhang:
 * eta = 0.1 / beta^, m = ceil(kappa^_F)) and leaves the sketch rank k to the user (Thm 1 gives
 * the runtime it trades off).  The library adds a small network that proposes (k, eta, m) from
 * the sketched spectrum; the theory setting is its fallback.  Nothing below has a counterpart
 * in the paper except those defaults.
 *
 * Network: x (67 inputs) -> ReLU(W1 x + b1) (128) -> ReLU(W2 . + b2) (128) -> W3 . + b3 (3).
 * Parameters theta: one float vector of RS_MLP_NPARAM entries, W1 (128 x 67), b1, W2
 * (128 x 128), b2, W3 (3 x 128), b3, each row-major, in that order.
 * Inputs: log of the 64 leading sketched singular values (sqrt of sigma~_i^2), log lambda,
 * log n, log d.  Outputs: log2 k, ln eta_mult, log2(m / n), where eta = eta_mult / beta^ and
 * beta^ is the mean smoothness rs_precondition reports. */

#define RS_MLP_IN 67
#define RS_MLP_HIDDEN 128
#define RS_MLP_OUT 3
#define RS_MLP_NPARAM (RS_MLP_HIDDEN * RS_MLP_IN + RS_MLP_HIDDEN + RS_MLP_HIDDEN * RS_MLP_HIDDEN + RS_MLP_HIDDEN + \
                       RS_MLP_OUT * RS_MLP_HIDDEN + RS_MLP_OUT)

/* out (float, B x 3) = network(theta, X) for the B rows of X (float, B x 67, row-major). */
int rs_mlp_forward(rs_ctx* ctx, const float* theta, const float* X, int64_t B, float* out);

typedef struct {
  float lr, beta1, beta2, eps;   /* Adam (Kingma and Ba, ICLR 2015) */
  int32_t step;                  /* t >= 1 of this update (bias corrections 1 - beta^t) */
  int32_t reserved;
} rs_adam_params;

/* One training step on the batch (X: float B x 67, T: float B x 3 targets, 1 <= B):
 * loss = (1/B) sum_s ||network(theta, x_s) - t_s||^2, its gradient g by backpropagation
 * (ReLU derivative 0 at 0), then Adam on theta with moment vectors adam_m, adam_v (float,
 * RS_MLP_NPARAM each, caller-initialised, zero at t = 1).  grad_out (float, RS_MLP_NPARAM;
 * nullable) receives g; loss_out (device float; nullable) the loss before the update.
 * Deterministic: per-block gradient partials are summed in a fixed order. */
int rs_mlp_train_step(rs_ctx* ctx, float* theta, float* adam_m, float* adam_v, const float* X, const float* T,
                      int64_t B, const rs_adam_params* p, float* grad_out, float* loss_out);

/* Affine normalisation stored with trained weights: the network sees (x - in_mean) / in_std
 * and its raw output o gives o * out_std + out_mean. */
typedef struct {
  float in_mean[RS_MLP_IN], in_std[RS_MLP_IN], out_mean[RS_MLP_OUT], out_std[RS_MLP_OUT];
} rs_mlp_norm;

/* Propose (k, eta_mult, m) for a problem with sketched eigenvalues sigma2 (host double, 64,
 * descending: the first 64 of an Alg. 2 sketch of rank >= 64), regularisation lambda, size n x d
 * and trace_c = tr(C) = ||X||_F^2 / n.  With theta (device) and norm (host) the network runs
 * on the GPU on the inputs 0.5 log(sigma2_i / sigma2_0) (i < 64), log(lambda / sigma2_0), log n,
 * log d (invariant to the scale of X), normalised by norm and clipped to +-3; its proposal is
 * k = round(2^o0) (clamped to [1, min(64, d)]), eta_mult = e^o1,
 * m = round(n 2^o2).  The theory setting is used instead (*used_fallback = 1) when theta is
 * NULL or an output is non-finite or outside eta_mult in [0.01, 8], m / n in [2^-8, 2^6]:
 * k minimises n d k + (kappa~(k) + n + d) d with kappa~(k) = (k sigma_k^2 + tr(C)
 * - sum_{i<=k} sigma_i^2) / lambda (Thm 1), eta_mult = 0.1 and m = ceil(kappa~(k) + d)
 * (= beta^ / lambda for exact eigenvectors).  Outputs are host pointers.  Synchronises. */
int rs_propose(rs_ctx* ctx, const float* theta, const rs_mlp_norm* norm, const double* sigma2, double lambda,
               int64_t n, int64_t d, double trace_c, int32_t* k, double* eta_mult, int64_t* m,
               int32_t* used_fallback);

/* Alg. 3 with proposed parameters, end to end: a rank-64 sketch of X (Alg. 2 with sp; sp->k <= 64
 * is replaced by 64; d >= 64), tr(C), rs_propose (theta / norm as there; NULL = theory setting),
 * the components of Eq. (11) / Sec. 5.1 from the leading k Ritz pairs, stored as z_dtype
 * (X->dtype, or RS_BF16 for RS_F32 data: then the snapshot gradients are refined on X), and
 * p->epochs epochs of Alg. 1 with eta = eta_mult / beta^ and the proposed m (p->eta, p->eta_mult
 * and p->m are ignored).  With sp->k > 64 the caller fixes the rank instead: the sketch has rank
 * sp->k (<= d), its first 64 Ritz values are the network's input, the preconditioner keeps all
 * sp->k pairs and only eta_mult and m are proposed, m carried from the network's rank k_net to
 * sp->k as m kappa~(sp->k) / kappa~(k_net) with kappa~ as in rs_propose from the sketch's Ritz
 * values (*k returns sp->k).  X, y and w_out may be
 * host pointers as in rs_solve.  k, eta_mult, m, used_fallback (host, nullable) receive the
 * parameters used.  Synchronises. */
int rs_solve_proposed(rs_ctx* ctx, const rs_matrix* X, const void* y, const rs_sketch_params* sp,
                      const rs_svrg_params* p, const float* theta, const rs_mlp_norm* norm, int32_t z_dtype,
                      void* w_out, rs_history* hist, int32_t* k, double* eta_mult, int64_t* m,
                      int32_t* used_fallback);

#ifdef __cplusplus
}
#endif

#endif /* RS_H */
