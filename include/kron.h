/*
 * kron.h - C ABI of the GB300 (sm_103a) Kronecker-regression library.
 *
 * The library computes the hot path of FastKroneckerRegression (Alg. 2 of
 * "Subquadratic Kronecker Regression with Applications to Tensor Decomposition"):
 * leverage-score row sampling of K = A(1) (x) ... (x) A(N) followed by Richardson
 * iteration on the sampled system, preconditioned by the unsampled normal matrix;
 * and its block-design extension FastFactorMatrixUpdate (Alg. 3) inside TuckerALS
 * (Alg. 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Layout: row-major matrices, C-order tensors (last index fastest). Row
 *    (i1..iN) of K is b[((i1*I2 + i2)*I3 + ...)*IN + iN]; the unknown x and the
 *    Tucker core G are indexed the same way over (r1..rN). This is the ordering
 *    under which K = A(1) (x) ... (x) A(N) multiplies vec(X) in Alg. 1.
 *  - Pointers are DEVICE pointers owned by the caller unless a comment says "host".
 *    (kr_opts.host_io = 1 switches the factor, right-hand-side and solution
 *    pointers of the solver entry points to host memory; the library then copies
 *    them in and out inside the call.)
 *  - Every call is enqueued on the context's stream and returns when its outputs
 *    are complete (the call synchronises the stream before returning).
 *  - Errors: a kr_status code; kr_last_error() gives a message. Nothing is thrown
 *    across the ABI. Device-side problems (non-finite values, divergence) are
 *    reported through status codes, never by trapping the GPU.
 *  - Limits: 1 <= N <= KR_MAX_MODES, 1 <= R_n <= I_n, R_n <= 64, I_n <= 65535,
 *    prod(I_n) < 2^32, number of draws s < 2^31.
 *  - The calls are synchronous. There are no _async variants: every call reads its
 *    report (iteration count, distinct rows, objective) back to the host before it
 *    returns, and the part of a solve that repeats (the Richardson loop) is already run
 *    by the library as one CUDA graph with the stopping rule on the device.
 *  - Determinism: every path is deterministic. Sums over blocks, tiles and draws run in
 *    a fixed order, and the only atomics are integer additions, which commute. Equal
 *    inputs, seed and call id give bit-identical outputs on the same device.
 */
#ifndef KRON_H
#define KRON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KR_API __attribute__((visibility("default")))
#else
#define KR_API
#endif

#define KR_MAX_MODES 8
#define KR_MAX_RANK 64

typedef enum {
  KR_OK = 0,
  KR_EINVAL = 1,      /* invalid argument (shape, range, null pointer) */
  KR_ENOMEM = 2,      /* device allocation failed */
  KR_ECUDA = 3,       /* a CUDA runtime call failed */
  KR_ENONFINITE = 4,  /* NaN/Inf met in an input or an iterate */
  KR_ERANK = 5,       /* a factor matrix is numerically rank deficient */
  KR_ENOTCONV = 6,    /* max_iter reached before the stopping rule held */
  KR_EDIVERGED = 7,   /* the Richardson step grew 3 times in a row */
  KR_ETIMEOUT = 8,    /* a bounded device wait ran out: the tensor-core mode product's pipeline
                         waits (TMA, MMA and epilogue mbarriers) give up after about 2 s, free
                         their tensor memory and report it; the context stays usable */
  KR_ENOTIMPL = 9     /* shape outside what this build supports */
} kr_status;

typedef struct kr_ctx kr_ctx;
typedef struct kr_sketch kr_sketch;

/* N factor matrices A[n] of shape I[n] x R[n] (row-major, FP32). */
typedef struct {
  int32_t N;
  int64_t I[KR_MAX_MODES];
  int32_t R[KR_MAX_MODES];
  const float* A[KR_MAX_MODES];
} kr_factors;

/* Options of the solvers (zero-initialise, then set what is needed). */
typedef struct {
  double eps;            /* approximation parameter, 0 < eps < 1 (Alg. 2 input) */
  double delta;          /* failure probability (recorded; the default sample count does not use it) */
  double lambda;         /* L2 regularisation (kron_ridge, tucker_als_sweep); >= 0 */
  double sample_scale;   /* c in s = ceil(c * R * ln(R) / eps); <= 0 selects 4 */
  int64_t num_samples;   /* > 0 overrides the sample count s */
  int32_t max_iter;      /* Richardson iteration cap; <= 0 selects 100 */
  double tol;            /* stop when ||step|| <= tol * ||x||; <= 0 selects 1e-7 */
  double step;           /* Richardson step; <= 0 selects the paper's 1 - sqrt(eps) */
  int32_t precision;     /* contraction format of the sampled products (slab passes of Alg. 2):
                            0: FP32-accurate (3xTF32 tensor-core products, FP32 residuals);
                            1: BF16 tensor-core products, 2: FP8 e4m3 with one scale per row of
                            the non-contracted index (both FP32 accumulation, FP32 residuals).
                            With 1 or 2 the Richardson loop runs its steps in that format until
                            its step falls below max(tol, 2^-7) (BF16) or max(tol, 2^-4) (e4m3)
                            or the stopping rule holds, then continues with FP32-accurate steps
                            from that point until the stopping rule holds (iterative refinement:
                            the fixed point is the FP32 path's); the final objective check is
                            always FP32/FP64. e4m3 needs R_{N-1} % 32 == 0 and BF16
                            R_{N-1} % 16 == 0 (else the next finer format); the per-cell path
                            (KR_OPT_SLAB_PASS 0) and the Alg. 3 factor steps ignore it. */
  int32_t host_io;       /* 1: factors, b / X and x / A / G are host pointers */
  uint64_t seed;         /* Philox key */
  uint64_t call_id;      /* Philox counter word 3 (distinguishes sketches drawn with one seed) */
  int32_t partition_T;   /* modes in the partition T of Thm 4.4 (bit n = mode n): 0 or -1 select the
                            last mode, the only partition this build evaluates; any other mask gives
                            KR_ENOTIMPL */
  int32_t deterministic; /* accepted for every value: all paths are deterministic (see above) */
  int32_t stop_rule;     /* 0: stop when ||step|| <= tol ||x|| ("until convergence" read as a
                            relative step). 1: the (1+eps)-aware rule: stop once the Lemma 4.2 bound
                            on the sampled objective's excess after the step,
                            rho^2 g^T M+ g / (1 - sqrt(eps)) with rho = 2 sqrt(eps) - eps, is at most
                            theta * eps times the lower bound f~(x) - g^T M+ g / (1 - sqrt(eps)) of
                            the sampled minimum (the O(log 1/eps) iterations of the proof of
                            Thm 4.5); the relative-step rule stays in force as a backstop. Applies to
                            kron_regress / kron_ridge / kron_ridge_batched and the core steps of
                            tucker_als_sweep, and to the factor steps (tucker_factor_update and the
                            sweep's) with two other modes on the slab path: there each row's rule is
                            the same bound on its penalised objective (sampled term plus
                            lambda ||(G+)^T z||^2 + w ||(I - G+ G) z||^2), and the loop ends once every
                            row's rule holds (report converged = 3). */
  double theta;          /* fraction of eps of stop_rule 1; <= 0 selects 0.01 */
} kr_opts;

/* Host-side report filled by the solvers (may be NULL). */
typedef struct {
  int32_t iters;             /* Richardson iterations taken (last problem / last step) */
  int32_t converged;         /* 1: ||step|| <= tol ||x||; 2: stalled at the FP32 rounding floor
                                (no new minimum step for 8 iterations, smallest relative step
                                within 100 tol); 3: the (1+eps)-aware rule held (stop_rule 1);
                                0: not converged */
  int64_t s;                 /* draws */
  int64_t distinct;          /* distinct sampled rows */
  double obj_sampled;        /* ||S(Kx - b)||^2 + lambda ||x||^2 at the returned x, FP64 accumulation */
  double rel_update;         /* last ||step|| / ||x|| */
  float t_ms[8];             /* leverage, sample, group+gather, rhs, iterate, final check, copies, total */
  int32_t iters_reduced;     /* of iters, the steps whose sampled products ran in reduced precision */
  int32_t precision_used;    /* contraction format of those steps (kr_opts.precision after the
                                shape fallback: 0 when every step ran FP32-accurate) */
} kr_report;

/* ---------------------------------------------------------------- context */

/* Create a context bound to the current CUDA device and the given stream
 * (cudaStream_t, may be NULL for the legacy default stream). The context owns its
 * workspace. workspace_bytes > 0 reserves that much device memory now (KR_ENOMEM if it
 * cannot); 0 reserves nothing. Either way the workspace grows on demand when a call
 * needs more, and kr_destroy frees it. The context also creates a non-blocking stream of
 * its own (loop bodies captured into graphs are recorded there) and 1 KB of device state
 * for the asynchronous solves, so that a solve captured into a caller's graph allocates
 * nothing (KR_ENOMEM if either fails). */
KR_API kr_status kr_create(kr_ctx** ctx, void* cuda_stream, size_t workspace_bytes);
KR_API void kr_destroy(kr_ctx* ctx);
KR_API kr_status kr_set_stream(kr_ctx* ctx, void* cuda_stream);
/* Message of the last failed call on this context (static storage, valid until
 * the next call on the context). */
KR_API const char* kr_last_error(const kr_ctx* ctx);
/* Number of kernels this context has launched so far (instrumentation). */
KR_API int64_t kr_launch_count(const kr_ctx* ctx);

/* Launches of the tcgen05 tensor-core kernel (the 3xTF32 mode product, KR_OPT_TENSOR_CORES)
 * on this context so far; counted in kr_launch_count too. */
KR_API int64_t kr_tc_launch_count(const kr_ctx* ctx);

/* CUDA graphs launched on this context so far: the device-side Richardson loops, and the
 * sweeps after the first of tucker_als_exact_sweep (captured together as one graph). */
KR_API int64_t kr_graph_count(const kr_ctx* ctx);

/* The autotuner's choices (KR_OPT_AUTOTUNE) as text, one shape class per line:
 * "N I_{N-1} R_{N-1} I_N R_N log2s budget ms@2048 ms@4096 ms@8192 ms@16384 ms@32768".
 * Writes at most cap bytes (NUL-terminated when cap > 0); returns the length of the full text. */
KR_API int64_t kr_autotune_report(kr_ctx* ctx, char* buf, int64_t cap);

/* Per-kernel timing (instrumentation, off by default). When enabled, the library
 * records a CUDA event pair on its stream around every launch of the kernel kinds
 * below; kr_timing_read synchronises the stream and returns, for one kind, the summed
 * event time (ms) and the number of launches since the last reset. */
enum {
  KR_K_RESID = 0,      /* sampled residual + transpose accumulation (a7 + a8) */
  KR_K_MODEPROD = 1,   /* mode-n products (KronMatMul, preconditioner) */
  KR_K_SAMPLE = 2,     /* Philox sampling of the row keys (a3; with the dense grouping also its
                          per-key counts and key bitmap, a4, in the same kernel) */
  KR_K_SCATTER = 3,    /* grouping of the row keys: radix sort or key-bitmap ranks (a4) */
  KR_K_DEDUP = 4,      /* merge of repeated rows + gather of b (a4 + a5) */
  KR_K_TABLES = 5,     /* Gram, Cholesky, leverage, CDF, eigen, guide tables, probability ranks (a1 + a2) */
  KR_K_VECTOR = 6,     /* Richardson update, reductions (a10) */
  KR_K_SLAB = 7,       /* fused slab pass: last-two-mode products + sampled residual (a6-a8) */
  KR_K_KINDS = 8
};
/* Context options. The defaults suit every input; the switches exist for A/B timing
 * and for tests that run both formulations of the sampled products.
 *  KR_OPT_SLAB_PASS (default 1): 1 evaluates the sampled products of one Richardson
 *    step (Thm 4.4 with T = the last mode) with the fused slab pass wherever the shape
 *    allows it (N >= 2, R[N-2] <= 64, R[N-1] <= 64, a single right-hand side); 0 always
 *    uses the per-cell residual pass between two full mode products.
 *  KR_OPT_SLAB_TILE_ENTRIES (default 16384, range [256, 2^22]): entry budget of one
 *    tile of the slab pass.
 *  KR_OPT_DEVICE_LOOP (default 1): 1 runs the Richardson steps after the first as one CUDA
 *    graph (a conditional loop whose body is one step and a device-side evaluation of the
 *    stopping rule), 0 returns to the host after every step. Both apply the same rule to
 *    the same device-side sums, so they give identical results. Per-kernel timing
 *    (kr_timing_enable) always uses the host loop.
 *  KR_OPT_BATCH_WORKERS (default 4, range [1, 32]): problems of kron_ridge_batched solved
 *    concurrently, each by a worker context with its own stream and workspace (created on
 *    first use, kept until kr_destroy). 1 solves them one after another on ctx's stream.
 *    Every problem's result is the same whatever the number of workers.
 *  KR_OPT_GROUPING (default 0): how the draws of a sketch are grouped into merged rows.
 *    1 sorts the row keys (stable LSD radix sort) and merges the runs of equal keys; 2 sets
 *    one bit per draw in a bitmap of the key space (prod I_n keys, times the factor rows of an
 *    Alg. 3 step; at most 2^32; 8 bytes of workspace per 32 keys), ranks the set bits and
 *    counts the draws per rank with integer atomics; 3 ranks the same bitmap but every draw
 *    adds one to a dense per-key counter (4 bytes per key, kept by the context, all zero
 *    between calls) and only a key's first draw sets its bit, so no key is written per draw;
 *    0 takes 3 when the key space is at most 64 times the draw count and its counters fit in
 *    4 GB, else 2 when the first holds, else 1. All give identical sketches.
 *  KR_OPT_HOST_GATHER (default 1): host-buffer solves (kr_opts.host_io) with b in
 *    page-locked host memory (cudaHostAlloc / cudaHostRegister, mapped into the device's
 *    address space) gather the sampled entries b~ = S b in place, reading s of the prod I
 *    entries of b; 0 copies all of b to the device first (on a second stream, overlapped
 *    with the tables, draws and grouping). Other host memory is always copied. Both give
 *    identical results.
 *  KR_OPT_JL_K (default 0, range [0, 64]): 0 samples by the exact statistical leverage scores;
 *    k > 0 by JL-approximate ones (the approximate scores of Alg. 2's first steps, App. B's
 *    Johnson-Lindenstrauss lemma): l~_i = ||a_i^T L^-T Pi||^2 / k with L the FP64 Cholesky factor
 *    of A(n)^T A(n) and Pi an R_n x k matrix of signs, entry (r, j) from the low bit of word w0 of
 *    Philox4x32-10 under key (KR_OPT_JL_SEED lo, hi) at counter (r k + j, 0, n, 0) (0: +1, 1: -1),
 *    n the factor's position in the call. E[l~_i] = l_i. Applies to every table build
 *    (kron_leverage, the solvers, the Tucker steps); the weights use the same scores, so the
 *    sketch stays unbiased.
 *  KR_OPT_JL_SEED (default 0): the Philox key of the JL sign matrices.
 *  KR_OPT_TENSOR_CORES (default 1): 1 runs the mode products of KronMatMul (Lemma 4.3) whose
 *    contracted index is the last, contiguous one (M x K times K x J with M >= 1024 rows,
 *    K >= 32 and a multiple of 4, J <= 256, the input 16-byte aligned) on the tcgen05 tensor
 *    cores in 3xTF32 (FP32 accuracy: operands split into TF32 hi and lo parts, FP32
 *    accumulation); 0 keeps every mode product on the CUDA cores.
 *  KR_OPT_BATCH_MODE (default 0): how kron_ridge_batched runs its problems. 0: on
 *    KR_OPT_BATCH_WORKERS worker contexts, each solving one problem after another. 1 (fused):
 *    one context and host thread per problem set up every problem concurrently on its own
 *    stream; the problems' Richardson loops (device-side conditional loops) then run as
 *    concurrent nodes of ONE CUDA graph, launched once for the whole batch, and each problem
 *    finishes with its final check. Results are bit-identical to the per-problem solves with
 *    the same options. The fused mode groups draws by ranks in a key bitmap (KR_OPT_GROUPING
 *    0 selects 2 there: no per-context dense counters) and keeps nprob contexts with their
 *    workspaces until kr_destroy.
 *  KR_OPT_AUTOTUNE (default 0): 1 chooses the slab pass's tile entry budget by measurement:
 *    the first solve of a shape class (N, I_{N-1}, R_{N-1}, I_N, R_N, floor(log2 s)) times one
 *    slab pass at each budget in {2048, 4096, 8192, 16384, 32768} and keeps the fastest for the
 *    class; kr_autotune_report lists the choices. A batch's contexts share the table.
 * Returns KR_EINVAL for an unknown key or a value out of range. */
enum {
  KR_OPT_SLAB_PASS = 1,
  KR_OPT_SLAB_TILE_ENTRIES = 2,
  KR_OPT_DEVICE_LOOP = 3,
  KR_OPT_BATCH_WORKERS = 4,
  KR_OPT_GROUPING = 5,
  KR_OPT_HOST_GATHER = 6,
  KR_OPT_JL_K = 7,
  KR_OPT_JL_SEED = 8,
  KR_OPT_TENSOR_CORES = 9,
  KR_OPT_BATCH_MODE = 10,
  KR_OPT_AUTOTUNE = 11
};
KR_API kr_status kr_set_option(kr_ctx* ctx, int32_t key, int64_t value);

KR_API kr_status kr_timing_enable(kr_ctx* ctx, int32_t on);
KR_API kr_status kr_timing_read(kr_ctx* ctx, int32_t kind, double* total_ms, int64_t* launches);
KR_API kr_status kr_timing_reset(kr_ctx* ctx);

/* The library's default sample count (Alg. 2's s with the experiments' scaled constant):
 * s = ceil(c R ln(R) / eps) with the natural logarithm, at least 1 (1 when R <= 1); c <= 0
 * selects 4. The solvers use it when kr_opts.num_samples is 0 (with R = prod R_n, or
 * prod_{m != n} R_m for an Alg. 3 row). Returns -1 for eps outside (0, 1) or R < 1. */
KR_API int64_t kron_sample_count(int64_t R, double eps, double c);

/* ---------------------------------------------------------------- a1 + a2 */

/* Statistical leverage scores and sampling tables of each factor
 * (§3 eq. ridge leverage via SVD at lambda = 0; Lemma 4.1: the scores of K are the
 * products of these; proof of Thm 4.5: one CDF per factor).
 *  lev[n]  (device, I[n] doubles, may be NULL): l_i = a_i^T (A^T A)^-1 a_i, computed
 *          from an FP64 Gram matrix and its FP64 Cholesky factor.
 *  cdf[n]  (device, I[n] doubles, may be NULL): cdf[i] = fl(prefix_i / total),
 *          left-to-right FP64 prefix; entries from the last positive-mass row on are 1.0.
 *  prob[n] (device, I[n] doubles, may be NULL): l_i / total.
 *  rank    (host, N ints, may be NULL): numerical rank of each factor
 *          (= R[n] unless a Cholesky pivot falls below R * 2^-52 * max diagonal).
 * Returns KR_ERANK if a factor is rank deficient (outputs for that factor undefined). */
KR_API kr_status kron_leverage(kr_ctx* ctx, const kr_factors* f, double* const lev[],
                        double* const cdf[], double* const prob[], int32_t* rank);

/* ---------------------------------------------------------------- a3 */

/* SampleRows on K from the product distribution (§3 Def. of leverage score
 * sampling; the row-sampling step of Alg. 2; coordinates drawn
 * independently per factor, proof of Thm 4.5).
 * Draw t, coordinate m (position in this call's mode list) uses the uniform
 * u = (((wa << 32) | wb) >> 11) * 2^-53 from Philox4x32-10 (Salmon et al. 2011) with
 * key (seed lo, seed hi) and counter (t lo, t hi, (m / 2) + 256 * row, call_id lo),
 * words (w0, w1) for even m and (w2, w3) for odd m; the index is the smallest i
 * with u < cdf[m][i] (bit-exact against any implementation of the same rule).
 *  N, I   : number of modes in the list and their sizes (I is host).
 *  cdf[m] : device tables as produced by kron_leverage.
 *  prob[m]: device probabilities (needed only when w != NULL).
 *  idx    : device s x N int32 (row t = draw t), may be NULL.
 *  w      : device s floats, w_t = 1 / sqrt(s * prod_m prob[m][idx[t][m]]), may be NULL. */
KR_API kr_status kron_sample(kr_ctx* ctx, int32_t N, const int64_t* I, const double* const cdf[],
                      const double* const prob[], int64_t s, uint64_t seed, uint64_t call_id,
                      int32_t row, int32_t* idx, float* w);

/* Allocation-free twin of kron_sample, for callers that must not allocate device
 * memory: code that runs under a memory manager owning every byte of the GPU (a
 * caching allocator with a fixed budget, where an extra cudaMalloc would fail or
 * fragment its pool), and latency-critical paths that cannot afford cudaMalloc's
 * device-wide synchronisation. The paper has no counterpart: this is a deployment
 * entry point, not a step of the method.
 * Inputs, outputs and the drawing rule are exactly those of kron_sample (outputs are
 * identical). The one piece of scratch, the integer sampling thresholds
 * ceil(cdf * 2^53), lives in a static device array of KR_NOALLOC_MAX_ROWS 64-bit
 * entries (128 KB) that every GPU loading this library holds until the process exits.
 * The call makes no device allocation and does not grow the context's workspace.
 *  - sum over m of I[m] must not exceed KR_NOALLOC_MAX_ROWS; larger tables are
 *    rejected with KR_EINVAL and a message naming the limit.
 *  - The first call on a device looks up the array's device address (with the
 *    context's device current); make that first call before any stream capture.
 *  - Each call writes every threshold entry it reads before reading it, so nothing
 *    left by an earlier call is used. All calls share the one array: calls whose work
 *    overlaps on the GPU (other streams or host threads) race on it, so the caller
 *    must keep them from overlapping. */
#define KR_NOALLOC_MAX_ROWS 16384
KR_API kr_status kron_sample_noalloc(kr_ctx* ctx, int32_t N, const int64_t* I, const double* const cdf[],
                                     const double* const prob[], int64_t s, uint64_t seed,
                                     uint64_t call_id, int32_t row, int32_t* idx, float* w);

/* ---------------------------------------------------------------- a3 + a4 + a5 */

/* Draw s rows of K (as kron_sample) and group them (Thm 4.4 proof: the support of S
 * split into cells = (i_1..i_{N-1}) and the last coordinate i_N), merging repeated
 * rows into a multiplicity c_j with weight omega_j = c_j / (s prod_n p_n(i_n))
 * (the same sketched objective as c_j rows of weight 1/(s p)); gather
 * b~_j = b[key_j] (Alg. 2, "b~ = S b" up to the factor sqrt(omega_j)).
 * b (device, prod I floats) may be NULL (no gather). The sketch lives in device
 * memory owned by the returned handle; free it with kron_sketch_free. */
KR_API kr_status kron_sketch(kr_ctx* ctx, const kr_factors* f, const double* const cdf[],
                      const double* const prob[], const float* b, int64_t s, uint64_t seed,
                      uint64_t call_id, int32_t row, kr_sketch** out);
/* Number of distinct rows of a sketch. */
KR_API int64_t kron_sketch_distinct(const kr_sketch* sk);
/* Copy the sketch out in increasing linear-row order (device outputs; any may be NULL):
 * keys (int64 linear row index), counts (int32), omega (float), btilde (float). */
KR_API kr_status kron_sketch_export(kr_ctx* ctx, const kr_sketch* sk, int64_t* keys, int32_t* counts,
                             float* omega, float* btilde);
/* g = K~^T Omega (b~ - K~ x) for the sketch's rows (Thm 4.4 sampled products, Alg. 2
 * Richardson gradient without the lambda term); obj (host, may be NULL) receives
 * sum_j omega_j (b~_j - (Kx)_j)^2 accumulated in FP64. x, g: device R floats. */
KR_API kr_status kron_sketch_residual(kr_ctx* ctx, const kr_sketch* sk, const kr_factors* f,
                               const float* x, float* g, double* obj);
KR_API void kron_sketch_free(kr_sketch* sk);

/* ---------------------------------------------------------------- a7/a8 building block, a9 */

/* KronMatMul (Lemma 4.3): y = (B(1) (x) ... (x) B(N)) x for matrices B(n) of shape
 * J[n] x K[n] (row-major; trans[n] = 1 means the stored array is K[n] x J[n] and its
 * transpose is used). x: prod K floats, y: prod J floats (device). */
KR_API kr_status kron_matmul(kr_ctx* ctx, int32_t N, const int64_t* J, const int64_t* K,
                      const float* const B[], const int32_t* trans, const float* x, float* y);

/* Preconditioner of Alg. 2: d = M^+ g with M^+ = (V1 (x)...(x) VN) D (V1 (x)...(x) VN)^T,
 * D = (S1^2 (x)...(x) SN^2 + lambda I)^+ (for lambda = 0: (A1^T A1)^-1 (x) ... (x) (AN^T AN)^-1
 * from FP64 Cholesky inverses). g, d: device R floats. */
KR_API kr_status kron_precond(kr_ctx* ctx, const kr_factors* f, double lambda, const float* g, float* d);

/* Full objective ||Kx - b||^2 + lambda ||x||^2 (Thm 4.5's guarantee), FP64 accumulation
 * over all prod I rows; result on the host. */
KR_API kr_status kron_objective(kr_ctx* ctx, const kr_factors* f, const float* b, const float* x,
                         double lambda, double* obj);

/* ---------------------------------------------------------------- solvers */

/* Alg. 2 FastKroneckerRegression with lambda = 0 (opts->lambda is ignored):
 * x ~ argmin ||Kx - b||^2 over x in R^{R_1...R_N}. b: prod I floats; x: prod R floats
 * (output; the iteration starts from 0). Returns KR_ENOTCONV (with x written) if
 * max_iter is reached. */
KR_API kr_status kron_regress(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts,
                       float* x, kr_report* report);

/* Alg. 2 with lambda = opts->lambda > 0 (ridge; sampling by statistical scores, the
 * sqrt(lambda) I block is never sampled, Cor. 3.3 / Lemma 3.2). */
KR_API kr_status kron_ridge(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts,
                     float* x, kr_report* report);

/* The report of an asynchronous solve, written in DEVICE memory when the solve completes. */
typedef struct {
  int32_t status;          /* the solve's kr_status: KR_OK, KR_ENOTCONV (x written), KR_ENONFINITE,
                              KR_EDIVERGED, or KR_ERANK (a factor numerically rank deficient) */
  int32_t iters;           /* Richardson iterations (both phases of a reduced-precision solve) */
  int32_t converged;       /* as kr_report.converged */
  int32_t iters_reduced;   /* as kr_report.iters_reduced */
  int32_t precision_used;  /* as kr_report.precision_used */
  int32_t reserved;
  int64_t s;               /* draws */
  int64_t distinct;        /* distinct sampled rows */
  double obj_sampled;      /* as kr_report.obj_sampled (FP64) */
  double rel_update;       /* as kr_report.rel_update */
} kr_dev_report;

/* kron_regress / kron_ridge enqueued on the context's stream without waiting: the call
 * returns once the work is enqueued, and *report (device memory, 56 bytes) holds the
 * outcome when the stream reaches the end of the solve. Device pointers only (host_io 0;
 * else KR_EINVAL); argument errors are returned at once, errors of the solve itself in
 * report->status. If the stream is being captured (cudaStreamBeginCapture, any mode), the
 * whole solve is captured into the caller's graph, its Richardson loop (and the FP32
 * refinement of a reduced-precision solve) as conditional WHILE nodes, so one graph launch
 * replays the whole solve; otherwise the kernels are enqueued and each loop is launched as
 * a graph of its own, nothing is read back, and the stream is synchronised only when a
 * buffer of the context has to grow. Inside a capture a buffer cannot grow (KR_ENOTIMPL,
 * with part of the solve captured: discard the graph): run the same or a larger solve once
 * before capturing. A captured graph uses the context's workspace, so it stays valid while
 * the context lives and its workspace does not grow, and instances of it must not run
 * concurrently with each other or with other calls on the context. The results equal the
 * synchronous solve's bit for bit, except that with lambda > 0 the preconditioner is always
 * applied in FP64 (the synchronous solve reads the factors' spectra on the host to decide).
 * The autotuner (KR_OPT_AUTOTUNE) uses its recorded choice for the shape class, else the
 * context's tile budget; kr_launch_count counts a loop's kernels once. */
KR_API kr_status kron_regress_async(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts,
                                    float* x, kr_dev_report* report);
KR_API kr_status kron_ridge_async(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts,
                                  float* x, kr_dev_report* report);

/* nprob independent ridge problems (host arrays of descriptors and pointers); each
 * uses opts with call_id + problem index. reports: host array of nprob (may be NULL).
 * The problems run concurrently on KR_OPT_BATCH_WORKERS worker contexts (host threads,
 * one stream each), after the work already enqueued on ctx's stream; the call returns
 * when all are done. Returns the first hard error (lowest problem index, its message in
 * kr_last_error), else KR_ENOTCONV if any problem did not converge, else KR_OK. */
KR_API kr_status kron_ridge_batched(kr_ctx* ctx, int32_t nprob, const kr_factors* probs,
                             const float* const b[], const kr_opts* opts, float* const x[],
                             kr_report* reports);

/* Alg. 3 FastFactorMatrixUpdate for mode n (App. C): every row i of X_(n) solves the
 * penalised sketched problem in z = G_(n)^T y (Lemmas 5.1, 5.2) with its own sketch
 * (Philox counter row i) over the modes m != n, Richardson-iterated with the Woodbury
 * form of the unsampled preconditioner (standard sign), and row i of A[n] becomes
 * (G_(n)^T)^+ z. The I[n] rows are solved together as one batch; the stopping rule
 * is applied to the largest per-row relative step. opts->lambda is the L2 weight,
 * w = (1 + 12/eps) prod_{m != n} sigma_max(A(m))^2. X: prod I floats; A[m]: I[m] x R[m];
 * G: prod R floats (C-order); A[n] is overwritten. Needs R[n] <= prod_{m != n} R[m]
 * (else KR_EINVAL), prod_{m != n} R[m] <= 24576 (else KR_ENOTIMPL) and a full-row-rank
 * G_(n) (else KR_ERANK). The terms of the update that cancel in the row space of
 * G_(n)^T (w z and G+ (w G z)) and the output rows are formed in FP64. With one or two
 * other modes the Woodbury preconditioner is FP64 as well (FP64 eigen-decompositions of
 * the other modes' Gram matrices; w multiplies any error of its base inverse); with more
 * it is FP32. The sampled terms and the iterate z are FP32. */
KR_API kr_status tucker_factor_update(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R,
                                      const float* X, float* const A[], const float* G, int32_t n,
                                      const kr_opts* opts, kr_report* report);

/* TuckerALS (Alg. 1) with sampled factor updates (Alg. 3, fresh sketch per factor row,
 * Woodbury preconditioner) and sampled core updates (Alg. 2 with b = vec X).
 * X: prod I floats; A[n]: I[n] x R[n] floats (in/out); G: prod R floats (in/out).
 * Sweep k, step n (0..N-1 factor steps, N core step) draws with call id
 * opts->call_id + k*(N+1) + n; factor row i uses counter row i. A step that stops at
 * max_iter does not end the sweeps. The first sweep runs from the host; with
 * KR_OPT_DEVICE_LOOP 1 (the default, and no timing) the sweeps after it are captured into ONE
 * CUDA graph launched once (kr_graph_count counts it): each step's Richardson loop is a
 * conditional WHILE node (a reduced-precision core step's FP32 refinement a second one,
 * entered on the device), the Woodbury weight w is computed on the device in the host's
 * order, and the rank, pivot and capacitance checks are device flags read after the graph
 * (KR_ERANK then names the check, not the step; the later steps have run on the failed
 * state). Inside the graph a core step with lambda > 0 applies its preconditioner in FP64
 * (the host sweep does so only for badly conditioned factors); otherwise the results are
 * bit-identical to the host sweeps. If the graph cannot be built (a buffer would have to
 * grow, the stream is the legacy default stream, ...) nothing of it runs and the sweeps
 * continue from the host; kr_last_error says why. report: the last core step's report, with
 * iters the total over all steps and the phase times of graph-run steps 0. */
KR_API kr_status tucker_als_sweep(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R,
                           const float* X, float* const A[], float* G, const kr_opts* opts,
                           int32_t sweeps, kr_report* report);

/* Exact TuckerALS (Alg. 1 with the exact factor and core updates of App. C, by KronMatMul):
 * the baseline of the sampled sweep. Per sweep, for n = 0..N-1 the factor update
 *   A(n)^T = (G_(n) (K^T K) G_(n)^T + lambda I)^-1 G_(n) Z_(n)^T,  K = (x)_{m != n} A(m),
 *   Z = X x_{m != n} A(m)^T  (one pass over X; H and its Cholesky solves in FP64),
 * then the core update G = (K^T K + lambda I)^-1 K^T vec X with K = (x)_m A(m) (Alg. 2's
 * preconditioner, applied exactly). X: prod I floats; A[n]: I[n] x R[n] (in/out); G: prod R
 * (in/out), all device. rre (host, sweeps doubles, may be NULL) receives the relative
 * reconstruction error ||X - G x_1 A(1) ... x_N A(N)||^2 / ||X||^2 after each sweep.
 * With lambda = 0 every R[n] must not exceed the product of the other ranks (else the factor
 * system G_(n) (K^T K) G_(n)^T is singular: KR_EINVAL). Returns KR_ERANK if a factor system
 * is not positive definite (a rank-deficient core unfolding or factor; checked on the device
 * and reported after the last sweep). The first sweep runs from the host; with
 * KR_OPT_DEVICE_LOOP 1 (the default) every later sweep (its N factor updates, the core update
 * and its RRE terms) is captured into ONE CUDA graph launched once (kr_graph_count counts it),
 * with results bit-identical to running the same sweeps from the host. */
KR_API kr_status tucker_als_exact_sweep(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X,
                                        float* const A[], float* G, double lambda, int32_t sweeps, double* rre);

/* Relative reconstruction error of a Tucker decomposition (the paper's RRE, App. D):
 * ||X - G x_1 A(1) ... x_N A(N)||^2 / ||X||^2, evaluated as
 * (||X||^2 - 2 <X x_m A(m)^T, G> + <G, G x_m A(m)^T A(m)>) / ||X||^2 with FP64 sums (one pass
 * over X; the reconstruction is never formed). rre is a host double. */
KR_API kr_status tucker_rre(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X,
                            const float* const A[], const float* G, double* rre);

#ifdef __cplusplus
}
#endif
#endif /* KRON_H */
