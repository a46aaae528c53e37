// Internal definitions shared by the translation units of libkron.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/kron.h"

#define KR_WARP 32

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from that paper's definition: a round
// maps (x0, x1, x2, x3) to (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)) with
// M0 = 0xD2511F53, M1 = 0xCD9E8D57, and the key is bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ------------------------------------------------------------------ context

struct kr_shared_loop;  // a fused batch's rendezvous: the problems' device loops in one graph
struct kr_tune_table;   // the autotuner's measured choices, per shape class

struct kr_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  int cc_major = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t launches = 0;
  // grow-on-demand device workspace
  char* ws = nullptr;
  size_t ws_size = 0;
  // split-K partial sums of the mode products (grown on demand)
  float* split_buf = nullptr;
  size_t split_size = 0;
  // pinned host buffer for small read-backs
  char* hbuf = nullptr;
  size_t hbuf_size = 0;
  // dense per-key draw counters of the rank grouping (grown on demand; all zero between
  // sketch builds, dcnt_clean false while a build that uses them is in flight on the host)
  uint32_t* dcnt = nullptr;
  size_t dcnt_size = 0;
  bool dcnt_clean = false;
  // options (kr_set_option)
  int slab_pass = 1;
  uint32_t slab_tile_entries = 16384;
  int device_loop = 1;  // Richardson iterations 2.. as one CUDA graph with a conditional loop
  int batch_workers = 4;  // kron_ridge_batched: problems solved concurrently (worker contexts)
  int grouping = 0;       // draws grouped by: 0 automatic, 1 radix sort, 2 ranks in a key bitmap
  int host_gather = 1;    // host-buffer solves: gather b~ from page-locked b in place (no copy of b)
  int jl_k = 0;           // JL-approximate leverage scores with this many sign columns (0: exact scores)
  uint64_t jl_seed = 0;   // Philox key of the JL sign matrices
  int tensor_cores = 1;   // contiguous-index mode products on tcgen05 (3xTF32) where eligible
  int batch_mode = 0;     // kron_ridge_batched: 0 worker contexts, 1 fused (one graph for all loops)
  int autotune = 0;       // slab-pass tile budget chosen by measurement per shape class
  kr_shared_loop* shared_loop = nullptr;  // set on the per-problem contexts of a fused batch
  kr_tune_table* tune = nullptr;          // the autotuner's table (owned when tune_owned)
  bool tune_owned = false;
  cudaEvent_t loop_ev = nullptr;          // end of this context's work before a shared round (owned)
  cudaEvent_t tune_ev[2] = {};            // the autotuner's timing pair (owned)
  // split B planes of the tensor-core mode product (grow-on-demand) and its device error word
  float* tc_buf = nullptr;
  size_t tc_size = 0;
  int* tc_err = nullptr;
  int64_t tc_launches = 0;
  int tc_attr = 0;  // dynamic shared memory the tensor-core kernel has been allowed
  int64_t graphs = 0;  // CUDA graphs this context launched (device loops, sweeps)
  // Set while tucker_als_sweep captures sweeps into one graph: the steps read nothing back
  // on the host, keep their checks on the device (gm.err bits, gm.status slots, gm.w slots),
  // and put each Richardson loop into the capture as a conditional WHILE node.
  struct GraphMode {
    bool on = false;
    bool capturing = true;   // loops go into the ongoing capture; else each is its own graph,
                             // launched without waiting (an asynchronous solve outside capture)
    void* report = nullptr;  // kr_dev_report of an asynchronous solve (device)
    void* mem = nullptr;     // one device allocation holding the arrays below (owned)
    int* err = nullptr;      // OR of KR_GM_* bits
    int* status = nullptr;   // {StepCheck, iteration count} per loop, in capture order
    double* w = nullptr;     // one Woodbury penalty per factor step, in capture order
    double* obj = nullptr;   // the last core step's sampled {residual, ||x||^2}
    void* last = nullptr;    // the last core step's Richardson state
    unsigned long long* distinct = nullptr;  // the last sketch's distinct rows
    int nstatus = 0, nw = 0, slot = 0, wslot = 0;
    std::vector<int64_t> body_launches;  // kernels per iteration of each captured loop
    std::vector<int> base_slot;          // loop whose count a resumed loop continues, or -1
    std::vector<int> owner;              // each loop's step: factor mode n, or -1 for a core step
    int cur_owner = -1;                  // the step being captured
    int64_t last_s = 0;                  // the last core step's sample count
    int last_prec = 0;                   // and the precision of its first phase
  } gm;
  cudaStream_t side_stream = nullptr;  // captures a loop body inside an ongoing capture (owned)
  void* gm_async = nullptr;  // an asynchronous solve's device state (GraphMode arrays; owned)
  // worker contexts of kron_ridge_batched, each with its own stream and workspace (owned)
  std::vector<kr_ctx*> workers;
  std::vector<cudaStream_t> worker_streams;
  // host-buffer solves: b is copied in on its own stream while the solve stream builds the
  // tables and draws; the gather waits for b_ready (created on first use, owned)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t b_ready = nullptr;
  // device copies of a host-buffer solve's factors, b and x (grow-on-demand, kept)
  char* io = nullptr;
  size_t io_size = 0;
  // set during a host-buffer solve: the event the gather of b waits for (nullptr: none)
  cudaEvent_t b_wait = nullptr;
  cudaEvent_t ev[10] = {};
  cudaEvent_t pev[2] = {};  // completion of the two in-flight Richardson norm read-backs
  // per-kernel timing (instrumentation)
  bool timing = false;
  struct Timed {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> pool;
  double t_ms[KR_K_KINDS] = {};
  int64_t t_n[KR_K_KINDS] = {};
};

cudaEvent_t kr_timing_event(kr_ctx* ctx);

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it). The
// limit is a per-function setting shared by every context and host thread, so the
// query-and-raise is serialised process-wide; a launch sized for an earlier, larger limit
// stays valid.
kr_status kr_func_smem(kr_ctx* ctx, const void* func, size_t bytes);
template <class F>
kr_status kr_smem_attr(kr_ctx* ctx, F* func, size_t bytes) {
  return kr_func_smem(ctx, reinterpret_cast<const void*>(func), bytes);
}
int kr_kind_of(const char* kernel_name);

kr_status kr_fail(kr_ctx* ctx, kr_status st, const char* fmt, ...);
kr_status kr_fail_cuda(kr_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);

#define KR_TRY(expr)                         \
  do {                                       \
    kr_status _st = (expr);                  \
    if (_st != KR_OK) return _st;            \
  } while (0)

#define KR_CUDA(ctx, expr)                                                         \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) return kr_fail_cuda((ctx), _e, #expr, __FILE__, __LINE__); \
  } while (0)

// Launch and count; checks the launch error. With timing enabled, an event pair
// brackets the launch on the same stream (kind from the kernel's name).
#define KR_LAUNCH(ctx, kernel, grid, block, smem, ...)                                   \
  do {                                                                                   \
    cudaEvent_t _ea = nullptr, _eb = nullptr;                                            \
    if ((ctx)->timing) {                                                                 \
      _ea = kr_timing_event(ctx);                                                        \
      _eb = kr_timing_event(ctx);                                                        \
      cudaEventRecord(_ea, (ctx)->stream);                                               \
    }                                                                                    \
    kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);                     \
    (ctx)->launches++;                                                                   \
    cudaError_t _e = cudaGetLastError();                                                 \
    if (_e != cudaSuccess) return kr_fail_cuda((ctx), _e, #kernel, __FILE__, __LINE__);  \
    if ((ctx)->timing) {                                                                 \
      cudaEventRecord(_eb, (ctx)->stream);                                               \
      (ctx)->pending.push_back({kr_kind_of(#kernel), _ea, _eb});                         \
    }                                                                                    \
  } while (0)

// Programmatic dependent launch: a kernel launched with KR_LAUNCH_PDL may start (and run
// its prologue) while the previous kernel on the stream finishes. Every such kernel calls
// kr_pdl_wait() before it reads anything the previous kernels wrote (and before it
// completes), and may call kr_pdl_trigger() once all its blocks have started, so that the
// next kernel's blocks are scheduled as this one's retire. Without the launch attribute
// both are no-ops.
__device__ __forceinline__ void kr_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void kr_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t kr_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                          Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#define KR_LAUNCH_PDL(ctx, kernel, grid, block, smem, ...)                                  \
  do {                                                                                      \
    cudaEvent_t _ea = nullptr, _eb = nullptr;                                               \
    if ((ctx)->timing) {                                                                    \
      _ea = kr_timing_event(ctx);                                                           \
      _eb = kr_timing_event(ctx);                                                           \
      cudaEventRecord(_ea, (ctx)->stream);                                                  \
    }                                                                                       \
    cudaError_t _e = kr_launch_pdl(kernel, dim3(grid), dim3(block), (smem), (ctx)->stream, __VA_ARGS__); \
    (ctx)->launches++;                                                                      \
    if (_e == cudaSuccess) _e = cudaGetLastError();                                         \
    if (_e != cudaSuccess) return kr_fail_cuda((ctx), _e, #kernel, __FILE__, __LINE__);     \
    if ((ctx)->timing) {                                                                    \
      cudaEventRecord(_eb, (ctx)->stream);                                                  \
      (ctx)->pending.push_back({kr_kind_of(#kernel), _ea, _eb});                            \
    }                                                                                       \
  } while (0)

// Ensures the workspace holds at least `bytes` (synchronises when it grows).
kr_status kr_ws_reserve(kr_ctx* ctx, size_t bytes);
// The same for the device copies of a host-buffer solve's inputs and output.
kr_status kr_io_reserve(kr_ctx* ctx, size_t bytes);
kr_status kr_hbuf_reserve(kr_ctx* ctx, size_t bytes);
kr_status kr_split_reserve(kr_ctx* ctx, size_t bytes);

// Bump allocator over a reserved region.
struct Carve {
  char* base;
  size_t cap;
  size_t off = 0;
  Carve(char* b, size_t c) : base(b), cap(c) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};
// Size accounting twin of Carve.
struct Need {
  size_t off = 0;
  template <class T>
  void add(size_t count) {
    off = (off + 255) & ~size_t(255);
    off += count * sizeof(T);
  }
};

// ------------------------------------------------------------------ shapes

struct Modes {
  int N;
  int I[KR_MAX_MODES];
  int R[KR_MAX_MODES];
  const float* A[KR_MAX_MODES];
};

kr_status kr_check_factors(kr_ctx* ctx, const kr_factors* f, Modes* m);
// s = ceil(c R ln R / eps), at least 1 (c <= 0 selects 4); -1 for eps outside (0, 1) or R < 1.
int64_t kr_sample_count(int64_t R, double eps, double c);
int64_t kr_prod_I(const Modes& m);
int64_t kr_prod_R(const Modes& m);

// Per-mode device tables derived from the factors (a1 + a2).
struct FactorTables {
  int N = 0;
  int I[KR_MAX_MODES] = {};
  int R[KR_MAX_MODES] = {};
  double* lev[KR_MAX_MODES] = {};    // I[n]
  double* cdf[KR_MAX_MODES] = {};    // I[n]
  double* prob[KR_MAX_MODES] = {};   // I[n]
  uint64_t* thr[KR_MAX_MODES] = {};  // I[n]: integer thresholds ceil(cdf * 2^53)
  float* invp[KR_MAX_MODES] = {};    // I[n]: 1 / p (FP32; 0 for zero-mass rows)
  float* ginv[KR_MAX_MODES] = {};    // R x R: (A^T A)^-1 (FP32, from FP64 Cholesky)
  float* V[KR_MAX_MODES] = {};       // R x R: eigenvectors of A^T A (columns, FP32)
  float* sig2[KR_MAX_MODES] = {};    // R: eigenvalues of A^T A (FP32)
  double* gram[KR_MAX_MODES] = {};   // R x R FP64
  double* linv[KR_MAX_MODES] = {};   // R x R FP64: inverse of the Cholesky factor of the Gram
  double* V64[KR_MAX_MODES] = {};    // R x R: eigenvectors of A^T A (columns, FP64; with the eigen-decomposition)
  double* sig64[KR_MAX_MODES] = {};  // R: eigenvalues of A^T A (FP64)
  double sig_max[KR_MAX_MODES] = {}; // host copies of each mode's largest and smallest eigenvalue
  double sig_min[KR_MAX_MODES] = {}; // (read back with the rank check when the eigen-decomposition is built)
  int rank[KR_MAX_MODES] = {};
  int* flags = nullptr;              // device: per mode, nonzero when its Cholesky met a non-positive pivot
};

// Computes Gram, Cholesky, leverage scores, CDF, thresholds, inverse probabilities,
// and (if want_eig) the eigen-decomposition of each factor Gram matrix. Buffers are
// carved from `cv` (which must be large enough: see kr_tables_need).
void kr_tables_need(const Modes& m, bool want_eig, Need& nd);
// FP64 eigen-decompositions G = V diag(sig2) V^T of nmat FP64 Gram matrices (R[n] <= 64;
// V row-major with the eigenvectors as columns), by cyclic Jacobi.
kr_status kr_eig64(kr_ctx* ctx, int nmat, const int* R, const double* const* gram, double* const* V,
                   double* const* sig2);
kr_status kr_tables_build(kr_ctx* ctx, const Modes& m, bool want_eig, Carve& cv, FactorTables& t,
                          bool check_rank = true);

// ------------------------------------------------------------------ mode products

// out[p, j, q] = sum_k B[j, k] * in[p, k, q], B stored J x K (trans = 0) or K x J (trans = 1).
// Tensor-core (tcgen05, 3xTF32) product Y[m, j] = sum_k X[m, k] B[j, k] (B stored K x J
// when trans), Y rows ldy floats apart; KR_ENOTIMPL when the shape or the build does not
// qualify (the caller then uses the CUDA-core kernel). kr_tc_check reads the kernel's
// error word (synchronises the stream): KR_ETIMEOUT when one of its bounded waits ran out.
bool kr_tc_eligible(const kr_ctx* ctx, const float* X, int64_t M, int K, int J);
kr_status kr_gemm_tc(kr_ctx* ctx, const float* X, int64_t M, int K, const float* B, int J, int trans, float* Y,
                     int64_t ldy);
kr_status kr_tc_check(kr_ctx* ctx);
kr_status kr_mode_product(kr_ctx* ctx, const float* in, float* out, int64_t P, int K, int64_t Q, int J,
                          const float* B, int trans);
// KronMatMul along the modes with B[n] != nullptr (identity elsewhere); intermediates
// in tmp0/tmp1 (each must hold the largest intermediate), result in `out` (may be `in`).
kr_status kr_kron_apply2(kr_ctx* ctx, int N, const int* dimsIn, const int* dimsOut, const float* const* B,
                         const int* trans, const float* in, float* out, float* tmp0, float* tmp1);
// x[i] /= prod_n sig2_n[r_n] + shift (trailing dims of t; a leading batch axis allowed).
kr_status kr_diag_scale(kr_ctx* ctx, const FactorTables& t, double shift, float* x, int64_t total);
// d = M+ g (Alg. 2 preconditioner) from the factor tables; tmp0/tmp1 hold R floats each.
kr_status kr_precond_apply(kr_ctx* ctx, const FactorTables& t, double lambda, const float* g, float* d, float* tmp0,
                           float* tmp1);

// ------------------------------------------------------------------ sketch

struct kr_sketch {
  int N = 0;
  int I[KR_MAX_MODES] = {};
  int64_t s = 0;       // all draws (nrow * s_row)
  int64_t s_row = 0;   // draws per row batch
  int nrow = 1;        // row batches (Tucker factor rows; 1 for a plain solve)
  int64_t ncell_inner = 0;  // prod_{n < N-1} I[n]
  int64_t xI = 1, xPafter = 1;  // gather map from a batch row into X (see k_dedup)
  int64_t ncell = 0;   // nrow * ncell_inner
  int IT = 0;          // I[N-1]
  int64_t distinct = 0;
  // device arrays (owned)
  bool want_desc = true;  // build perm/desc (the per-cell residual pass); the slab pass does not use them
  uint32_t* cell_start = nullptr;  // ncell: first entry of the cell (entries of consecutive cells back to back)
  uint32_t* cell_nd = nullptr;     // ncell: distinct entries of the cell
  uint32_t* ent = nullptr;         // s (first `distinct` used): packed (i_T | count << 16) at cell_start[c] + k
  float* bt = nullptr;             // s: b~ at the same positions
  float* cell_w = nullptr;         // ncell: prod_{n<N-1} (1/p_n(i_n)) / s
  float* invpT = nullptr;          // IT: 1/p_{N-1}(i)
  uint32_t* perm = nullptr;        // ncell: cells by decreasing distinct-row count (work balance)
  uint4* desc = nullptr;           // ncell, in perm order: {cell, start, distinct, weight bits}
  char* mem = nullptr;
};

// Sketch construction: check the shape, set dimensions, account/carve the sketch's own
// arrays, then fill them (sampling, grouping, merging, gather) using scratch from `cv`.
kr_status kr_sketch_check(kr_ctx* ctx, const Modes& m, int64_t s);
void kr_sketch_setup(kr_sketch* sk, const Modes& m, int64_t s);
void kr_sketch_setup_rows(kr_sketch* sk, const Modes& m, int64_t s_row, int nrow, int64_t xI, int64_t xPafter);
void kr_sketch_own_need(const kr_sketch* sk, Need& nd);
void kr_sketch_layout(kr_sketch* sk, Carve& cv);
void kr_sketch_scratch_need(const kr_ctx* ctx, int64_t s, int64_t ncell, int64_t IT, Need& nd);
// Grouping of the draws: by ranks in a bitmap of the key space (ncell * IT keys) or by
// radix sort (KR_OPT_GROUPING; automatic: ranks when the key space is at most 64 s).
bool kr_group_by_rank(const kr_ctx* ctx, int64_t s, int64_t keyspace);
// With defer_distinct the distinct-row count is copied to the context's pinned buffer at
// KR_HBUF_DISTINCT without a synchronisation (sk->distinct = -1 until the caller reads it
// after its next stream synchronisation).
constexpr size_t KR_HBUF_DISTINCT = 2048;
kr_status kr_sketch_fill(kr_ctx* ctx, const Modes& m, const FactorTables& t, const float* b, uint64_t seed,
                         uint64_t call_id, int row, kr_sketch* sk, Carve& cv, bool defer_distinct = false);
// Residual/gradient pass: W[c, :] = sum_j omega_j (b~_j - <a_T, Y[c]>) a_T; obj partials.
kr_status kr_sketch_resid(kr_ctx* ctx, const kr_sketch* sk, const float* AT, int RT, const float* Y,
                          float* W, double* obj_partial, int nblocks, int* used);
int kr_resid_blocks(kr_ctx* ctx);

// Exclusive scan of n u32 values (in may equal out); scratch carved from cv.
void kr_scan_need(int64_t n, Need& nd);
kr_status kr_scan_u32(kr_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, Carve& cv);
// Stable LSD radix sort of n keys on their low nbits bits; *sorted is keys or alt.
void kr_radix_need(int64_t n, Need& nd);
kr_status kr_radix_sort_u32(kr_ctx* ctx, uint32_t* keys, uint32_t* alt, int64_t n, int nbits, uint32_t** sorted,
                            Carve& cv);
// perm = cells ordered by decreasing floor(log2(distinct rows)), stable (deterministic).
void kr_perm_need(int64_t ncell, Need& nd);
kr_status kr_balance_perm(kr_ctx* ctx, const uint32_t* nd, int64_t ncell, uint32_t* perm, Carve& cv);

// ------------------------------------------------------------------ fused slab pass

// Tiles of the fused slab pass: runs of consecutive non-empty cells of one slab (the
// cells sharing i_1..i_{N-2}), at most `cb` cells and about `et` entries each.
struct kr_tiles {
  int64_t P = 0;       // slabs: prod_{n < N-2} I[n] (1 for N = 2)
  int I2 = 0, R2 = 0;  // mode N-2 (second to last)
  int IT = 0, RT = 0;  // mode N-1 (the gathered one)
  int cb = 0;          // cells per tile at most
  uint32_t et = 0;     // entry budget of a tile
  int64_t ntmax = 0;   // tile capacity (upper bound of the device-side tile count)
  uint4* act = nullptr;          // ncell: {cell, first entry, entries, weight bits} of non-empty cells
  uint4* tile = nullptr;         // ntmax: {first non-empty cell, cells, slab, entries}
  uint32_t* cost = nullptr;      // ntmax: work estimate (0 past the last tile)
  uint32_t* order = nullptr;     // ntmax: processing order (heaviest first)
  uint4* tsort = nullptr;        // ntmax: descriptors in processing order (packed, see kr_slab.cu)
  uint2* slab = nullptr;         // P: {first tile, tiles}
  uint32_t* tstart = nullptr;    // P + 1: first tile of every slab (tiles are in slab order)
  // backward fold of the last prefix mode (k_tile_reduce): groups p' of Iq slabs, Rq rows
  int64_t Pq = 1;
  int Iq = 1, Rq = 1, nc = 1;
  int nout = 1;                  // weight matrices of the fold (2: a second output, see kr_tile_reduce)
  float* zred = nullptr;         // nc x nout x Pq x Rq x R2 x RT chunk partials (nc > 1)
  uint32_t* meta = nullptr;      // [0] tiles, [1] non-empty cells, [2] work counter (zero between passes)
  float* zpart = nullptr;        // ntmax x R2 x RT: contributions of tiles of multi-tile slabs
  double* objpart = nullptr;     // ntmax: per-tile sampled objective (FP64; zero past the last)
};

// Whether the sketch/shape admits the slab pass (N >= 2, R[N-2] <= 64, R[N-1] <= 64,
// shared memory for two teams; a single right-hand side unless `rows`, where each row of a
// batched-row sketch is its own group of slabs with its own X1).
bool kr_slab_eligible(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, bool rows = false);
void kr_tiles_setup(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, kr_tiles* tl);
void kr_tiles_own_need(const kr_tiles* tl, int64_t ncell, Need& nd);
void kr_tiles_layout(kr_tiles* tl, int64_t ncell, Carve& cv);
void kr_tiles_scratch_need(const kr_tiles* tl, int64_t ncell, Need& nd);
// Builds the tiles from a filled sketch (scratch from cv).
kr_status kr_tiles_build(kr_ctx* ctx, const kr_sketch* sk, kr_tiles* tl, Carve& cv);
// One fused pass from X1 (P x R2 x RT): every tile's contribution to its slab's
// Z[p] = sum_i A(N-2)[i]^T W[p, i] goes to tl->zpart (see kr_slab.cu); with want_obj the
// per-tile objective partials go to tl->objpart (tl->ntmax doubles).
// rearm: zero the tile counter first (needed when no tile reduction followed the last pass).
// flags: KR_SLAB_ZERO_X when X1 is zero (the first Richardson step; X1 is not read),
// KR_SLAB_OBJ_ONLY when only the objective partials are wanted (no tile Z is written).
enum { KR_SLAB_ZERO_X = 1, KR_SLAB_OBJ_ONLY = 2 };
kr_status kr_slab_pass(kr_ctx* ctx, const kr_sketch* sk, kr_tiles* tl, const float* A2, const float* AT,
                       const float* X1, bool want_obj, bool rearm, int prec = 0, int flags = 0);
// The contraction format a slab pass asked for `prec` (0 FP32-accurate 3xTF32, 1 BF16,
// 2 e4m3 with per-row scales) runs at for these ranks (falls back to the next finer one).
int kr_slab_precision(int R2, int RT, int prec);
// W[p', r, :] = sum over the tiles of the slabs p' * Iq + i of Aq[i, r] zpart[t, :]
// (Aq = A(N-3) for N >= 3, nullptr for N = 2): Pq x Rq x R2 x RT floats. With Aq2 the same
// sum with the weights Aq2 goes to W2 (one pass over the tiles for both). With opart the
// tiles' objective partials of the pass (tl->objpart, written by a want_obj pass) are summed
// in tile order per chunk: opart[c * Pq + p'] (tl->nc * tl->Pq doubles).
kr_status kr_tile_reduce(kr_ctx* ctx, kr_tiles* tl, const float* Aq, float* W, double* opart = nullptr,
                         const float* Aq2 = nullptr, float* W2 = nullptr);

// ------------------------------------------------------------------ solvers

struct SolveCfg {
  double lambda, eps, alpha, tol;
  int max_iter;
  int64_t s;
  int stop_rule = 0;     // 1: the (1+eps)-aware rule (kr_opts.stop_rule)
  double theta = 0.01;   // its fraction of eps
  int prec = 0;          // kr_opts.precision: slab-pass contractions of the first phase
};

enum StepCheck { STEP_CONTINUE, STEP_CONVERGED, STEP_FLOOR, STEP_DIVERGED, STEP_NONFINITE, STEP_MAXITER, STEP_EPS };
// Runs the steps of a Richardson loop as one CUDA graph: a conditional WHILE node whose
// body is one captured step, body(hnd, 1); the body's last kernel clears the condition.
// Launches the graph once on ctx->stream, waits for it to end, and returns the launches of one
// captured step in *per_step; false when graphs are unavailable (nothing ran, the caller
// continues with its host loop).
bool kr_graph_while(kr_ctx* ctx, const std::function<kr_status(cudaGraphConditionalHandle, int)>& body,
                    int64_t* per_step);
// Inside an ongoing capture of ctx->stream: a condition handle of the capture's graph whose
// value is dflt at every launch (1: the loop runs at least once; 0: a kernel captured before
// the loop decides), and a conditional WHILE node after the captured work with body(hnd, 1)
// captured into it (its last kernel sets the condition). *per_body = kernels per iteration.
kr_status kr_gm_handle(kr_ctx* ctx, unsigned dflt, cudaGraphConditionalHandle* hnd);
kr_status kr_capture_while(kr_ctx* ctx, cudaGraphConditionalHandle hnd,
                           const std::function<kr_status(cudaGraphConditionalHandle, int)>& body, int64_t* per_body);
// Graph-mode bookkeeping (kr_ctx::gm): bits of the device error word; a kernel that ORs a
// table build's pivot flags (or a capacitance flag) into it; one that stores a loop's final
// {status, iteration count} in the next slot (*slot_out = its index; base_slot: the loop a
// resumed loop continues, whose count is subtracted when launches are tallied).
enum { KR_GM_FACTOR_RANK = 1, KR_GM_CORE_UNFOLD_RANK = 2, KR_GM_CAPACITANCE = 4 };
constexpr size_t KR_GM_ASYNC_BYTES = 1024;  // kr_ctx::gm_async
kr_status kr_gm_flags(kr_ctx* ctx, const int* flags, int n, int bit);
// Runs fn, which adds loops (kr_gm_handle / kr_capture_while), where they belong: into the
// ongoing capture, or (an asynchronous solve outside capture) captured on its own and
// launched on the stream as one graph without waiting.
kr_status kr_gm_section(kr_ctx* ctx, const std::function<kr_status()>& fn);
// After a captured sweep ran (stream synchronised): the last core step's report fields
// (converged, rel_update, obj_sampled, distinct, s, precision_used) from the device copies.
kr_status kr_gm_core_report(kr_ctx* ctx, double lambda, kr_report* rep);
// Bytes of the device copy of a core step's Richardson state.
size_t kr_gm_state_bytes();
kr_status kr_gm_status(kr_ctx* ctx, const int* status, const int* it, int64_t per_body, int base_slot,
                       int* slot_out);
// A fused batch's problems each add their device loop (body captured on their own stream) as
// one more conditional WHILE node of a shared graph; the last active problem to arrive
// launches the graph on the batch's stream, after every member's earlier work, and waits for
// it. Returns false when the round could not run (the caller continues with its host loop).
bool kr_shared_loop_run(kr_shared_loop* sl, kr_ctx* ctx,
                        const std::function<kr_status(cudaGraphConditionalHandle, int)>& body, int64_t* per_step);
// A problem that will add no further loop (its solve returned) leaves the rendezvous.
void kr_shared_loop_leave(kr_shared_loop* sl);
kr_shared_loop* kr_shared_loop_new(cudaStream_t stream, int members);
void kr_shared_loop_delete(kr_shared_loop* sl);
// Autotuner table: the slab tile budget measured best for a shape class, or 0 if unknown.
uint32_t kr_tune_lookup(kr_ctx* ctx, const int64_t* key);
void kr_tune_record(kr_ctx* ctx, const int64_t* key, uint32_t et, const float* ms, int nc);
void kr_tune_free(kr_ctx* ctx);
// Stopping rule of the Richardson loops ("until convergence" in Alg. 2 and Alg. 3):
// converged when ||step|| <= tol ||x||; stalled at the FP32 rounding floor when no new
// minimum step was seen for 8 iterations and the smallest relative step is within
// 100 tol; diverged when the step grew 3 times in a row and exceeds 16x its minimum.
// h = {||step||^2, ||x||^2, non-finite flag}; rel_override >= 0 replaces ||step||/||x||
// (the batched factor step passes its largest per-row ratio).
__host__ __device__ inline StepCheck step_check(const double* h, double tol, double* prev_step, double* min_step,
                                         double* min_rel, int* grow,
                     int* since_min, double* rel_out, double rel_override) {
  const double step = sqrt(h[0]), xn = sqrt(h[1]);
  if (h[2] != 0.0 || !isfinite(step) || !isfinite(xn)) return STEP_NONFINITE;
  double rel = xn > 0.0 ? step / xn : (step == 0.0 ? 0.0 : INFINITY);
  if (rel_override >= 0.0) rel = rel_override;
  *rel_out = rel;
  if (rel <= tol) return STEP_CONVERGED;
  if (step < *min_step) {
    *min_step = step;
    *since_min = 0;
  } else {
    ++*since_min;
  }
  if (rel < *min_rel) *min_rel = rel;
  *grow = (step > *prev_step) ? *grow + 1 : 0;
  *prev_step = step;
  if (*grow >= 3 && step > 16.0 * *min_step) return STEP_DIVERGED;
  if (*since_min >= 8 && *min_rel <= 100.0 * tol) return STEP_FLOOR;
  return STEP_CONTINUE;
}

// Alg. 2 on device-resident factors and b; x (R floats) is written.
kr_status kr_solve_device(kr_ctx* ctx, const Modes& m, const float* b, const SolveCfg& cfg, uint64_t seed,
                          uint64_t call_id, float* x_out, kr_report* rep);
