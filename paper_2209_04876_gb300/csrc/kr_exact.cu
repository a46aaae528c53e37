// Exact Tucker ALS by KronMatMul (App. C, the exact factor and core updates of Alg. 1), the
// baseline the sampled sweep (Alg. 3 factor steps, Alg. 2 core step) is measured against,
// and the relative reconstruction error of a Tucker decomposition (App. D's RRE).
//
// Factor update of mode n, for all rows at once: with K = (x)_{m != n} A(m) and G_(n) the
// mode-n unfolding of the core (columns in C-order over the other modes),
//   A(n)^T = H^-1 G_(n) Z_(n)^T,   H = G_(n) (K^T K) G_(n)^T + lambda I,   Z = X x_{m != n} A(m)^T,
// where K^T K = (x)_{m != n} A(m)^T A(m) is applied to the core as mode products
// (W = G x_{m != n} Gram_m, H = G_(n) W_(n)^T + lambda I). Z is the one pass over X (KronMatMul,
// Lemma 4.3); H, its Cholesky factor and the solves are FP64.
// Core update: G = (K^T K + lambda I)^-1 K^T vec X with K = (x)_m A(m): g = X x_m A(m)^T, then
// the Kronecker preconditioner of Alg. 2 (exact here: M^-1 g).
// RRE = ||X - G x_1 A(1) ... x_N A(N)||^2 / ||X||^2 = (||X||^2 - 2 <g, G> + <G, G x_m Gram_m>) / ||X||^2,
// with g = X x_m A(m)^T at the same factors (one pass over X, no reconstruction).
#include <math.h>

#include <string>

#include "kr_internal.cuh"

namespace {

constexpr int EX_THREADS = 256;

// out[r, i] = sum_{p, q} F[p, r, q] Z[p, i, q] over p < P, q < Q (F has Rn in the middle, Z has Ni),
// FP64 accumulation; FT = float or double. One thread per (r, i).
template <class FT, class ZT>
__global__ void k_unfold_contract(const FT* __restrict__ F, const ZT* __restrict__ Z, int64_t P, int Rn, int Ni,
                                  int64_t Q, double* __restrict__ out) {
  const int64_t tot = (int64_t)Rn * Ni;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Ni), i = (int)(e % Ni);
    double acc = 0.0;
    for (int64_t p = 0; p < P; ++p) {
      const FT* f = F + (p * Rn + r) * Q;
      const ZT* z = Z + (p * Ni + i) * Q;
      for (int64_t q = 0; q < Q; ++q) acc = fma((double)f[q], (double)z[q], acc);
    }
    out[e] = acc;
  }
}

// out[p, j, q] = sum_k S[j, k] in[p, k, q] for a symmetric R x R FP64 matrix S (a Gram matrix).
template <class IT>
__global__ void k_mode_sym64(const IT* __restrict__ in, double* __restrict__ out, int64_t P, int R, int64_t Q,
                             const double* __restrict__ S) {
  const int64_t tot = P * R * Q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e % Q;
    const int64_t pj = e / Q;
    const int j = (int)(pj % R);
    const int64_t p = pj / R;
    const IT* col = in + p * R * Q + q;
    double acc = 0.0;
    for (int k = 0; k < R; ++k) acc = fma(S[(int64_t)j * R + k], (double)col[(int64_t)k * Q], acc);
    out[e] = acc;
  }
}

// Every block factors H + lambda I (Rn x Rn, FP64, Cholesky in shared memory) and solves
// (H + lambda I) a_i = rhs[:, i] for its share of the columns i < Ni; a_i becomes row i of A
// (Ni x Rn, FP32). flag[0] = 1 if a pivot is not positive.
__global__ void __launch_bounds__(EX_THREADS) k_chol_rows(const double* __restrict__ H, double lambda, int Rn,
                                                           const double* __restrict__ rhs, int Ni, float* __restrict__ A,
                                                           int* __restrict__ flag) {
  __shared__ double L[KR_MAX_RANK * (KR_MAX_RANK + 1)];
  constexpr int LD = KR_MAX_RANK + 1;
  for (int e = threadIdx.x; e < Rn * Rn; e += blockDim.x) {
    const int r = e / Rn, c = e % Rn;
    L[r * LD + c] = H[e] + (r == c ? lambda : 0.0);
  }
  __syncthreads();
  // right-looking Cholesky: column k, then the trailing update
  for (int k = 0; k < Rn; ++k) {
    if (threadIdx.x == 0) {
      const double d = L[k * LD + k];
      if (!(d > 0.0)) flag[0] = 1;
      L[k * LD + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double dk = L[k * LD + k];
    for (int r = k + 1 + threadIdx.x; r < Rn; r += blockDim.x) L[r * LD + k] /= dk;
    __syncthreads();
    for (int e = threadIdx.x; e < (Rn - k - 1) * (Rn - k - 1); e += blockDim.x) {
      const int r = k + 1 + e / (Rn - k - 1), c = k + 1 + e % (Rn - k - 1);
      if (c <= r) L[r * LD + c] -= L[r * LD + k] * L[c * LD + k];
    }
    __syncthreads();
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ni; i += gridDim.x * blockDim.x) {
    double y[KR_MAX_RANK];
    for (int r = 0; r < Rn; ++r) {  // L y = b
      double v = rhs[(int64_t)r * Ni + i];
      for (int c = 0; c < r; ++c) v -= L[r * LD + c] * y[c];
      y[r] = v / L[r * LD + r];
    }
    for (int r = Rn - 1; r >= 0; --r) {  // L^T a = y
      double v = y[r];
      for (int c = r + 1; c < Rn; ++c) v -= L[c * LD + r] * y[c];
      y[r] = v / L[r * LD + r];
    }
    for (int r = 0; r < Rn; ++r) A[(int64_t)i * Rn + r] = (float)y[r];
  }
}

// Per-block FP64 partial sums of a . b (a FP32; b FP32 or FP64).
template <class BT>
__global__ void __launch_bounds__(EX_THREADS) k_dot_part(const float* __restrict__ a, const BT* __restrict__ b,
                                                          int64_t n, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)a[i], (double)b[i], s);
  __shared__ double red[EX_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < EX_THREADS / 32; ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

// out[0] = sum of n partials (one block, fixed order).
__global__ void __launch_bounds__(EX_THREADS) k_sum_part(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[EX_THREADS];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

int ex_grid(kr_ctx* ctx, int64_t work) {
  int64_t g = (work + EX_THREADS - 1) / EX_THREADS;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// Largest tensor of X x_{m in S} A(m)^T when the modes of S are applied in increasing order.
int64_t ex_max_intermediate(const Modes& m, int skip) {
  int64_t cur = kr_prod_I(m), mx = cur;
  for (int n = 0; n < m.N; ++n) {
    if (n == skip) continue;
    cur = cur / m.I[n] * m.R[n];
    if (cur > mx) mx = cur;
  }
  return mx;
}

struct ExBufs {
  float* t0;
  float* t1;
  float* Z;       // I_n x R_{!=n} (largest n) / g (R)
  double* rhs;    // R_n x I_n
  double* W0;     // R doubles
  double* W1;     // R doubles
  double* H;      // R_n x R_n
  double* part;   // partial sums
  double* red;    // 4 doubles
  int* flag;
};

// X x_{m != skip} A(m)^T (skip = -1: every mode) into out.
kr_status ex_project(kr_ctx* ctx, const Modes& m, const float* X, int skip, const ExBufs& b, float* out) {
  int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  for (int n = 0; n < m.N; ++n) {
    din[n] = m.I[n];
    dout[n] = n == skip ? m.I[n] : m.R[n];
    B[n] = n == skip ? nullptr : m.A[n];
    tr[n] = 1;
  }
  return kr_kron_apply2(ctx, m.N, din, dout, B, tr, X, out, b.t0, b.t1);
}

// W = G x_{m != skip} Gram_m (FP64, R entries); returns the buffer holding it.
kr_status ex_gram_apply(kr_ctx* ctx, const Modes& m, const FactorTables& t, const float* G, int skip, const ExBufs& b,
                        const double** W) {
  const int64_t R = kr_prod_R(m);
  const double* src = nullptr;
  double* dst = b.W0;
  int64_t P = 1;
  bool first = true;
  for (int n = 0; n < m.N; ++n) {
    const int64_t Q = R / P / m.R[n];
    if (n != skip) {
      if (first)
        KR_LAUNCH(ctx, k_mode_sym64<float>, ex_grid(ctx, R), EX_THREADS, 0, G, dst, P, m.R[n], Q, (const double*)t.gram[n]);
      else
        KR_LAUNCH(ctx, k_mode_sym64<double>, ex_grid(ctx, R), EX_THREADS, 0, src, dst, P, m.R[n], Q,
                  (const double*)t.gram[n]);
      first = false;
      src = dst;
      dst = (dst == b.W0) ? b.W1 : b.W0;
    }
    P *= m.R[n];
  }
  if (first) {  // no other mode: W = G (not reached for N >= 2)
    return kr_fail(ctx, KR_EINVAL, "tucker exact: at least two modes");
  }
  *W = src;
  return KR_OK;
}

kr_status ex_need(const Modes& m, Need& nd) {
  int64_t mx = 0, zmax = 0;
  int rimax = 0;
  const int64_t R = kr_prod_R(m);
  for (int n = -1; n < m.N; ++n) {
    const int64_t v = ex_max_intermediate(m, n);
    if (v > mx) mx = v;
    if (n >= 0) {
      const int64_t z = R / m.R[n] * m.I[n];
      if (z > zmax) zmax = z;
      const int ri = m.R[n] * m.I[n];
      if (ri > rimax) rimax = ri;
    }
  }
  if (R > zmax) zmax = R;
  nd.add<float>(mx);
  nd.add<float>(mx);
  nd.add<float>(zmax);
  nd.add<double>(rimax);
  nd.add<double>(R);
  nd.add<double>(R);
  nd.add<double>((size_t)KR_MAX_RANK * KR_MAX_RANK);
  nd.add<double>(4096);
  nd.add<double>(8);
  nd.add<int>(4);
  kr_tables_need(m, true, nd);
  return KR_OK;
}

ExBufs ex_carve(const Modes& m, Carve& cv) {
  int64_t mx = 0, zmax = 0;
  int rimax = 0;
  const int64_t R = kr_prod_R(m);
  for (int n = -1; n < m.N; ++n) {
    const int64_t v = ex_max_intermediate(m, n);
    if (v > mx) mx = v;
    if (n >= 0) {
      const int64_t z = R / m.R[n] * m.I[n];
      if (z > zmax) zmax = z;
      const int ri = m.R[n] * m.I[n];
      if (ri > rimax) rimax = ri;
    }
  }
  if (R > zmax) zmax = R;
  ExBufs b;
  b.t0 = cv.take<float>(mx);
  b.t1 = cv.take<float>(mx);
  b.Z = cv.take<float>(zmax);
  b.rhs = cv.take<double>(rimax);
  b.W0 = cv.take<double>(R);
  b.W1 = cv.take<double>(R);
  b.H = cv.take<double>((size_t)KR_MAX_RANK * KR_MAX_RANK);
  b.part = cv.take<double>(4096);
  b.red = cv.take<double>(8);
  b.flag = cv.take<int>(4);
  return b;
}

// sum a . b (FP64) into red[k].
template <class BT>
kr_status ex_dot(kr_ctx* ctx, const float* a, const BT* bv, int64_t n, const ExBufs& b, int k) {
  int g = ex_grid(ctx, n);
  if (g > 4096) g = 4096;
  KR_LAUNCH(ctx, k_dot_part<BT>, g, EX_THREADS, 0, a, bv, n, b.part);
  KR_LAUNCH(ctx, k_sum_part, 1, EX_THREADS, 0, (const double*)b.part, g, b.red + k);
  return KR_OK;
}

// red[0] = ||X||^2, red[1] = <g, G>, red[2] = <G, G x_m Gram_m> for the current factors.
// The three terms nearly cancel (an RRE of 1e-4 comes from terms of order 1), so g is
// projected on the CUDA cores: the tensor-core product's rounding is biased (its FP32
// accumulation truncates, error of one sign about 1e-6 of the product), which the cancellation
// would turn into a percent-level RRE error, while the CUDA-core sum's errors are unbiased and
// average out over the R terms of <g, G>.
kr_status ex_rre_terms(kr_ctx* ctx, const Modes& m, const float* X, const float* G, const FactorTables& t,
                       const ExBufs& b, bool have_g) {
  const int64_t R = kr_prod_R(m);
  KR_TRY(ex_dot<float>(ctx, X, X, kr_prod_I(m), b, 0));
  if (!have_g || ctx->tensor_cores) {
    const int tc = ctx->tensor_cores;
    ctx->tensor_cores = 0;
    const kr_status st = ex_project(ctx, m, X, -1, b, b.Z);
    ctx->tensor_cores = tc;
    KR_TRY(st);
  }
  KR_TRY(ex_dot<float>(ctx, b.Z, G, R, b, 1));
  const double* W = nullptr;
  KR_TRY(ex_gram_apply(ctx, m, t, G, -1, b, &W));
  KR_TRY(ex_dot<double>(ctx, G, W, R, b, 2));
  return KR_OK;
}

// OR of a table build's per-mode pivot flags into the sweep's flag.
__global__ void k_flags_or(const int* __restrict__ f, int n, int* __restrict__ out) {
  if (threadIdx.x == 0) {
    int v = 0;
    for (int i = 0; i < n; ++i) v |= f[i];
    if (v) atomicOr(out, 1);
  }
}

double ex_rre_from(const double* h) { return h[0] > 0.0 ? (h[0] - 2.0 * h[1] + h[2]) / h[0] : 0.0; }

kr_status ex_args(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X, const float* const A[],
                  const float* G, Modes* m) {
  if (!I || !R || !X || !A || !G) return kr_fail(ctx, KR_EINVAL, "tucker: null argument");
  if (N < 2 || N > KR_MAX_MODES) return kr_fail(ctx, KR_EINVAL, "tucker: N=%d outside [2,%d]", N, KR_MAX_MODES);
  kr_factors f = {};
  f.N = N;
  for (int n = 0; n < N; ++n) {
    f.I[n] = I[n];
    f.R[n] = R[n];
    f.A[n] = A[n];
  }
  return kr_check_factors(ctx, &f, m);
}

}  // namespace

extern "C" kr_status tucker_als_exact_sweep(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X,
                                            float* const A[], float* G, double lambda, int32_t sweeps, double* rre) {
  if (!ctx) return KR_EINVAL;
  Modes m;
  KR_TRY(ex_args(ctx, N, I, R, X, (const float* const*)A, G, &m));
  if (sweeps < 0) return kr_fail(ctx, KR_EINVAL, "tucker_als_exact_sweep: sweeps < 0");
  if (!(lambda >= 0.0) || !isfinite(lambda)) return kr_fail(ctx, KR_EINVAL, "tucker_als_exact_sweep: lambda must be >= 0");
  if (lambda == 0.0) {
    const int64_t Rt = kr_prod_R(m);
    for (int n = 0; n < N; ++n)
      if ((int64_t)m.R[n] * m.R[n] > Rt)
        return kr_fail(ctx, KR_EINVAL,
                       "tucker_als_exact_sweep: lambda = 0 needs R[n] <= prod of the other ranks (mode %d: %d > %lld)", n,
                       m.R[n], (long long)(Rt / m.R[n]));
  }
  const size_t nrre = 3 * (size_t)(sweeps > 0 ? sweeps : 1);  // the RRE terms of every sweep
  Need nd;
  nd.add<double>(nrre);
  KR_TRY(ex_need(m, nd));
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  KR_TRY(kr_hbuf_reserve(ctx, 4096 + sizeof(double) * nrre));
  Carve cv(ctx->ws, ctx->ws_size);
  double* rre_dev = cv.take<double>(nrre);
  ExBufs b = ex_carve(m, cv);
  const Carve tables_cv = cv;
  KR_CUDA(ctx, cudaMemsetAsync(b.flag, 0, sizeof(int), ctx->stream));
  // One sweep: the N factor updates, the core update, and the sweep's RRE terms into
  // rre_dev[3 k..]. Nothing in it reads device data on the host (rank-deficient factors are
  // flagged on the device), so the sweeps after the first, which sizes every buffer and sets
  // every kernel attribute, can be captured into one graph.
  auto one_sweep = [&](int k) -> kr_status {
    for (int n = 0; n < N; ++n) {
      Carve tc = tables_cv;
      FactorTables t;
      KR_TRY(kr_tables_build(ctx, m, false, tc, t, false));  // FP64 Gram matrices of the current factors
      // Z = X x_{m != n} A(m)^T (I_n in mode n), rhs = G_(n) Z_(n)^T (R_n x I_n)
      KR_TRY(ex_project(ctx, m, X, n, b, b.Z));
      int64_t P = 1, Q = 1;
      for (int j = 0; j < n; ++j) P *= m.R[j];
      for (int j = n + 1; j < N; ++j) Q *= m.R[j];
      KR_LAUNCH(ctx, (k_unfold_contract<float, float>), ex_grid(ctx, (int64_t)m.R[n] * m.I[n]), EX_THREADS, 0,
                (const float*)G, (const float*)b.Z, P, m.R[n], m.I[n], Q, b.rhs);
      // H = G_(n) (G x_{m != n} Gram_m)_(n)^T, then A(n) rows from the FP64 Cholesky solves
      const double* W = nullptr;
      KR_TRY(ex_gram_apply(ctx, m, t, G, n, b, &W));
      KR_LAUNCH(ctx, (k_unfold_contract<float, double>), ex_grid(ctx, (int64_t)m.R[n] * m.R[n]), EX_THREADS, 0,
                (const float*)G, W, P, m.R[n], m.R[n], Q, b.H);
      const int gsolve = ex_grid(ctx, m.I[n]);
      KR_LAUNCH(ctx, k_chol_rows, gsolve, EX_THREADS, 0, (const double*)b.H, lambda, m.R[n], (const double*)b.rhs,
                m.I[n], A[n], b.flag);
    }
    // core: g = X x_m A(m)^T, G = (K^T K + lambda I)^-1 g (Alg. 2's preconditioner, exact)
    Carve tc = tables_cv;
    FactorTables t;
    KR_TRY(kr_tables_build(ctx, m, lambda > 0.0, tc, t, false));
    KR_LAUNCH(ctx, k_flags_or, 1, 32, 0, (const int*)t.flags, N, b.flag);
    KR_TRY(ex_project(ctx, m, X, -1, b, b.Z));
    KR_TRY(kr_precond_apply(ctx, t, lambda, b.Z, G, b.t0, b.t1));
    if (rre) {
      KR_TRY(ex_rre_terms(ctx, m, X, G, t, b, true));
      KR_CUDA(ctx, cudaMemcpyAsync(rre_dev + 3 * k, b.red, 3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return KR_OK;
  };
  int done = 0;
  if (sweeps > 0) {
    KR_TRY(one_sweep(0));
    done = 1;
  }
  if (sweeps > 1 && ctx->device_loop && !ctx->timing) {
    // sweeps 2.. captured into ONE CUDA graph, launched once
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t l0 = ctx->launches;
    std::string why;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) why = std::string("begin capture: ") + cudaGetErrorString(e);
    if (why.empty()) {
      kr_status cs = KR_OK;
      for (int k = 1; k < sweeps && cs == KR_OK; ++k) cs = one_sweep(k);
      if (cs != KR_OK) why = "capture: " + ctx->err;
      e = cudaStreamEndCapture(ctx->stream, &graph);
      if (e != cudaSuccess && why.empty()) why = std::string("end capture: ") + cudaGetErrorString(e);
    }
    if (why.empty() && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
      why = std::string("instantiate: ") + cudaGetErrorString(e);
    if (why.empty() && (e = cudaGraphLaunch(exec, ctx->stream)) != cudaSuccess)
      why = std::string("launch: ") + cudaGetErrorString(e);
    if (why.empty() && (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
      why = std::string("run: ") + cudaGetErrorString(e);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (why.empty()) {
      done = sweeps;
      ctx->graphs++;
    } else {
      cudaGetLastError();  // graphs unavailable: the remaining sweeps run from the host
      ctx->launches = l0;
      ctx->err = "tucker_als_exact_sweep: sweeps 2.. ran from the host (" + why + ")";
    }
  }
  for (int k = done; k < sweeps; ++k) KR_TRY(one_sweep(k));
  double* hr = reinterpret_cast<double*>(ctx->hbuf + 64);
  if (rre && sweeps > 0)
    KR_CUDA(ctx, cudaMemcpyAsync(hr, rre_dev, sizeof(double) * 3 * (size_t)sweeps, cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaMemcpyAsync(ctx->hbuf, b.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rre)
    for (int k = 0; k < sweeps; ++k) rre[k] = ex_rre_from(hr + 3 * k);
  if (*(const int*)ctx->hbuf)
    return kr_fail(ctx, KR_ERANK, "tucker_als_exact_sweep: a factor system is not positive definite or a factor is "
                                  "rank deficient");
  return kr_tc_check(ctx);
}

extern "C" kr_status tucker_rre(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X,
                                const float* const A[], const float* G, double* rre) {
  if (!ctx) return KR_EINVAL;
  if (!rre) return kr_fail(ctx, KR_EINVAL, "tucker_rre: null output");
  Modes m;
  KR_TRY(ex_args(ctx, N, I, R, X, A, G, &m));
  Need nd;
  KR_TRY(ex_need(m, nd));
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  Carve cv(ctx->ws, ctx->ws_size);
  ExBufs b = ex_carve(m, cv);
  FactorTables t;
  KR_TRY(kr_tables_build(ctx, m, false, cv, t, false));
  KR_TRY(ex_rre_terms(ctx, m, X, G, t, b, false));
  KR_CUDA(ctx, cudaMemcpyAsync(ctx->hbuf, b.red, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *rre = ex_rre_from((const double*)ctx->hbuf);
  return KR_OK;
}
