// a1 + a2: factor Gram matrices, Cholesky, leverage scores, sampling tables,
// eigen-decompositions for the preconditioner.
//
// Leverage scores follow §3 (statistical scores l_i = a_i^T (A^T A)^-1 a_i, the
// lambda = 0 case of the ridge-score definition); the sampling distribution of K
// is their product (Lemma 4.1) and is drawn one coordinate at a time from one CDF
// per factor (proof of Thm 4.5). The preconditioner of Alg. 2 needs
// (A^T A)^-1 per factor when lambda = 0 and the eigen-decomposition
// A^T A = V S^2 V^T when lambda > 0.
//
// Precision: Gram, Cholesky, triangular inverse, scores and CDF in FP64 (exact
// FP32 x FP32 products, FP64 sums). The eigen-decomposition of the lambda > 0
// preconditioner is an FP64 Jacobi of the FP64 Gram, rounded to FP32 for the
// application: the preconditioner has to be a spectral approximation of the normal matrix
// (Lemma 4.2), and an FP32 Jacobi's eigenvalues carry absolute errors of about
// u32 ||G||, which for nearly rank-one factors (the paper's synthetic workload, cond(G)
// near 1e8) exceed the small eigenvalues themselves. The Alg. 3 factor step's Woodbury
// base (K^T K + w I)^-1 with w >> ||K^T K|| takes the same FP64 Jacobi (kr_eig64): there
// an orthogonality error e of V perturbs K^T K by about w e.
#include <math.h>

#include "kr_internal.cuh"

namespace {

constexpr int GRAM_ROWS = 16;
constexpr int MAXR = KR_MAX_RANK;
constexpr int LD = MAXR + 1;

struct ModePtrs {
  int N;
  int I[KR_MAX_MODES];
  int R[KR_MAX_MODES];
  const float* A[KR_MAX_MODES];
  double* part[KR_MAX_MODES];
  double* gram[KR_MAX_MODES];
  double* linv[KR_MAX_MODES];
  double* lev[KR_MAX_MODES];
  double* cdf[KR_MAX_MODES];
  double* prob[KR_MAX_MODES];
  uint64_t* thr[KR_MAX_MODES];
  float* invp[KR_MAX_MODES];
  float* ginv[KR_MAX_MODES];
  float* V[KR_MAX_MODES];
  float* sig2[KR_MAX_MODES];
  int* flags;  // per mode: 1 = rank deficient
};

// Partial Gram over GRAM_ROWS rows per block (upper triangle, FP64 accumulation).
__global__ void k_gram_partial(ModePtrs mp) {
  const int n = blockIdx.y;
  const int I = mp.I[n], R = mp.R[n];
  const int r0 = blockIdx.x * GRAM_ROWS;
  if (r0 >= I) return;
  const int rows = min(GRAM_ROWS, I - r0);
  __shared__ double a[GRAM_ROWS][LD];
  const float* A = mp.A[n];
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x) {
    int rr = e / R, c = e % R;
    a[rr][c] = (double)A[(int64_t)(r0 + rr) * R + c];
  }
  __syncthreads();
  double* out = mp.part[n] + (int64_t)blockIdx.x * R * R;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    int i = e / R, j = e % R;
    if (i > j) continue;
    double acc = 0.0;
    for (int rr = 0; rr < rows; ++rr) acc = fma(a[rr][i], a[rr][j], acc);
    out[e] = acc;
  }
}

// Deterministic reduction of the partials (block order), mirrored to full symmetric.
// One thread per upper-triangle entry; loads are issued in batches ahead of the sum.
__global__ void k_gram_reduce(ModePtrs mp) {
  const int n = blockIdx.y;
  const int I = mp.I[n], R = mp.R[n];
  const int nchunk = (I + GRAM_ROWS - 1) / GRAM_ROWS;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * R) return;
  const int i = e / R, j = e % R;
  if (i > j) return;
  const double* part = mp.part[n] + e;
  double acc = 0.0;
  for (int c0 = 0; c0 < nchunk; c0 += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (c0 + u < nchunk) ? part[(int64_t)(c0 + u) * R * R] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c0 + u < nchunk) acc += v[u];
  }
  mp.gram[n][i * R + j] = acc;
  mp.gram[n][j * R + i] = acc;
}

// 1/sqrt(d) for d > 0 in FP64: an FP32 estimate of the reduced argument refined by two
// Newton steps y <- y (3 - d y^2) / 2 (each doubles the correct bits: 24 -> 48 -> 96, so
// the result is within an ulp or two). FP64 square root and division are long dependent
// sequences on this part; the Newton form keeps the pivot chain of the Cholesky short.
__device__ __forceinline__ double rsqrt_fp64(double d) {
  const int e = (int)((__double_as_longlong(d) >> 52) & 0x7FF) - 1023;
  if (e < -1000 || e > 1000) return 1.0 / sqrt(d);
  const int h = e >> 1;  // d = m * 4^h with m in [1, 4)
  const double m = d * __longlong_as_double((long long)(1023 - 2 * h) << 52);
  double y = (double)rsqrtf((float)m) * __longlong_as_double((long long)(1023 - h) << 52);
  const double hd = 0.5 * d;
  y = y * fma(-hd, y * y, 1.5);
  y = y * fma(-hd, y * y, 1.5);
  return y;
}

// One block per mode: the Cholesky factor G = L L^T in FP64, written (lower triangle, R x R)
// over the mode's Gram partials (mp.part, no longer needed once the Gram matrix is formed),
// and the pivot flag. L^-1 and (A^T A)^-1 follow in k_trinv and k_ginv, spread over blocks.
__global__ void k_cholesky(ModePtrs mp) {
  const int n = blockIdx.x;
  const int R = mp.R[n];
  extern __shared__ double sm[];
  double* L = sm;  // R x LD
  __shared__ int bad;
  __shared__ double maxdiag;
  __shared__ double pinv;
  const int tid = threadIdx.x;
  for (int e = tid; e < R * R; e += blockDim.x) L[(e / R) * LD + e % R] = mp.gram[n][e];
  if (tid == 0) {
    bad = 0;
    double md = 0.0;
    for (int i = 0; i < R; ++i) md = fmax(md, mp.gram[n][i * R + i]);
    maxdiag = md;
  }
  __syncthreads();
  const double tol = maxdiag * (double)R * 1e-15;
  for (int k = 0; k < R; ++k) {
    if (tid == 0) {  // the pivot: one reciprocal square root per step
      double d = L[k * LD + k];
      if (!(d > tol)) {  // also catches NaN
        bad = 1;
        d = 1.0;
      }
      const double y = rsqrt_fp64(d);
      L[k * LD + k] = d * y;
      pinv = y;
    }
    __syncthreads();
    const double inv = pinv;
    for (int i = k + 1 + tid; i < R; i += blockDim.x) L[i * LD + k] *= inv;
    __syncthreads();
    const int m = R - k - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) L[i * LD + j] = fma(-L[i * LD + k], L[j * LD + k], L[i * LD + j]);
    }
    __syncthreads();
  }
  double* Lout = mp.part[n];
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int i = e / R, j = e % R;
    Lout[e] = j <= i ? L[i * LD + j] : 0.0;
  }
  if (tid == 0) mp.flags[n] = bad;
}

// Column j of L^-1 (block (j, mode); one warp), by forward substitution in FP64:
// x_j = 1 / L_jj, x_i = -(sum_{j <= k < i} L_ik x_k) / L_ii for i > j, 0 above the diagonal.
__global__ void __launch_bounds__(32) k_trinv(ModePtrs mp) {
  const int n = blockIdx.y, j = blockIdx.x, R = mp.R[n];
  if (j >= R) return;
  __shared__ double Ls[MAXR * LD];
  __shared__ double x[MAXR], rd[MAXR];
  const double* L = mp.part[n];
  const int lane = threadIdx.x;
  for (int e = lane; e < R * R; e += 32) {
    const int i = e / R, k = e % R;
    if (i >= j && k >= j && k <= i) Ls[i * LD + k] = L[e];
  }
  for (int i = lane; i < R; i += 32) {
    rd[i] = i >= j ? 1.0 / L[i * R + i] : 0.0;
    x[i] = 0.0;
  }
  __syncwarp();
  if (lane == 0) x[j] = rd[j];
  __syncwarp();
  for (int i = j + 1; i < R; ++i) {
    double acc = 0.0;
    for (int k = j + lane; k < i; k += 32) acc = fma(Ls[i * LD + k], x[k], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) x[i] = -acc * rd[i];
    __syncwarp();
  }
  for (int i = lane; i < R; i += 32) mp.linv[n][i * R + j] = x[i];
}

// Row i of (A^T A)^-1 = X^T X with X = L^-1, in FP32 (a preconditioner only needs a
// spectral approximation): block (i, mode).
__global__ void __launch_bounds__(64) k_ginv(ModePtrs mp) {
  const int n = blockIdx.y, i = blockIdx.x, R = mp.R[n];
  if (i >= R) return;
  const double* X = mp.linv[n];
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    const int k0 = i > j ? i : j;
    float acc = 0.f;
    for (int k = k0; k < R; ++k) acc = fmaf((float)X[k * R + i], (float)X[k * R + j], acc);
    mp.ginv[n][i * R + j] = acc;
  }
}

// l_i = ||L^-1 a_i||^2 in FP64: LEV_ROWS rows per block, one warp per row, a lane per
// component of L^-1 a_i, the squares summed over the warp in a fixed tree order.
constexpr int LEV_ROWS = 8;
__global__ void __launch_bounds__(LEV_ROWS * 32) k_leverage(ModePtrs mp) {
  const int n = blockIdx.y;
  const int I = mp.I[n], R = mp.R[n];
  const int r0 = blockIdx.x * LEV_ROWS;
  if (r0 >= I) return;
  extern __shared__ double sm[];
  double* X = sm;              // R x LD
  double* a = sm + MAXR * LD;  // LEV_ROWS x LD
  const int rows = min(LEV_ROWS, I - r0);
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) X[(e / R) * LD + (e % R)] = mp.linv[n][e];
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x)
    a[(e / R) * LD + (e % R)] = (double)mp.A[n][(int64_t)(r0 + e / R) * R + (e % R)];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= rows) return;
  double acc = 0.0;
  for (int k = lane; k < R; k += 32) {
    double v = 0.0;
    for (int m = 0; m <= k; ++m) v = fma(X[k * LD + m], a[w * LD + m], v);
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) mp.lev[n][r0 + w] = acc;
}

// JL-approximate scores (the approximate leverage scores of Alg. 2's first steps, with App. B's
// Johnson-Lindenstrauss lemma): l~_i = ||a_i^T B||^2 / k with B = L^-T Pi (R x k), L the Cholesky
// factor of the Gram matrix and Pi an R x k matrix of signs, entry (r, j) from the low bit of
// word w0 of Philox4x32-10 under the JL key at counter (r k + j, 0, mode, 0) (0: +1, 1: -1).
// E[l~_i] = l_i. The cost per row is R k instead of about R^2 / 2.
constexpr int JL_MAXK = 64;
// Per-mode device pointers passed to a kernel by value (inside its parameter block): a
// kernel must never receive a host array of device pointers, which would outlive neither the
// host frame that holds it nor a device without access to host memory.
struct PtrSet {
  double* p[KR_MAX_MODES];
};

__global__ void k_jl_basis(ModePtrs mp, int k, uint32_t s0, uint32_t s1, PtrSet B) {
  const int n = blockIdx.y;
  const int R = mp.R[n];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * k; e += gridDim.x * blockDim.x) {
    const int c = e / k, j = e - c * k;
    double acc = 0.0;
    for (int r = c; r < R; ++r) {  // (L^-1)^T: L^-1 is lower triangular
      const uint4 w = philox4x32_10(make_uint4((uint32_t)(r * k + j), 0u, (uint32_t)n, 0u), s0, s1);
      const double sg = (w.x & 1u) ? -1.0 : 1.0;
      acc = fma(mp.linv[n][r * R + c], sg, acc);
    }
    B.p[n][e] = acc;
  }
}

// l~_i for LEV_ROWS rows per block, one warp per row, lanes over the k columns of B.
__global__ void __launch_bounds__(LEV_ROWS * 32) k_leverage_jl(ModePtrs mp, int k, PtrSet B) {
  const int n = blockIdx.y;
  const int I = mp.I[n], R = mp.R[n];
  const int r0 = blockIdx.x * LEV_ROWS;
  if (r0 >= I) return;
  extern __shared__ double sm[];
  double* Bs = sm;                 // R x k
  double* a = sm + MAXR * JL_MAXK;  // LEV_ROWS x LD
  const int rows = min(LEV_ROWS, I - r0);
  for (int e = threadIdx.x; e < R * k; e += blockDim.x) Bs[e] = B.p[n][e];
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x)
    a[(e / R) * LD + (e % R)] = (double)mp.A[n][(int64_t)(r0 + e / R) * R + (e % R)];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= rows) return;
  double acc = 0.0;
  for (int j = lane; j < k; j += 32) {
    double v = 0.0;
    for (int c = 0; c < R; ++c) v = fma(a[w * LD + c], Bs[c * k + j], v);
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) mp.lev[n][r0 + w] = acc / (double)k;
}

// One block per mode: left-to-right FP64 prefix of the scores (the convention of the
// sampling tables), normalised CDF, integer thresholds, probabilities and FP32 inverse
// probabilities. The prefix is one dependent chain of additions: the scores are staged in
// shared memory and one thread adds them from registers in batches, so the chain holds
// nothing but the additions; the index of the last positive score is a parallel max.
constexpr int CDF_THREADS = 256;
constexpr int CDF_CHUNK = 4096;
__global__ void __launch_bounds__(CDF_THREADS) k_cdf(ModePtrs mp) {
  const int n = blockIdx.x;
  const int I = mp.I[n];
  double* cdf = mp.cdf[n];
  const double* lev = mp.lev[n];
  __shared__ double chunk[CDF_CHUNK];
  __shared__ double total;
  __shared__ int last;
  if (threadIdx.x == 0) last = -1;
  __syncthreads();
  {
    int lp = -1;
    for (int i = threadIdx.x; i < I; i += blockDim.x)
      if (lev[i] > 0.0) lp = i;
    if (lp >= 0) atomicMax(&last, lp);
  }
  double acc = 0.0;  // thread 0 only
  for (int c0 = 0; c0 < I; c0 += CDF_CHUNK) {
    const int cn = min(CDF_CHUNK, I - c0);
    for (int i = threadIdx.x; i < cn; i += blockDim.x) chunk[i] = lev[c0 + i];
    __syncthreads();
    if (threadIdx.x == 0) {
      int i = 0;
      for (; i + 16 <= cn; i += 16) {
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = chunk[i + u];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          acc = __dadd_rn(acc, v[u]);
          v[u] = acc;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) chunk[i + u] = v[u];
      }
      for (; i < cn; ++i) {
        acc = __dadd_rn(acc, chunk[i]);
        chunk[i] = acc;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) cdf[c0 + i] = chunk[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) total = acc;
  __syncthreads();
  const double T = total;
  const int lpos = last;
  for (int i = threadIdx.x; i < I; i += blockDim.x) {
    double c = (lpos >= 0 && i >= lpos) ? 1.0 : __ddiv_rn(cdf[i], T);
    cdf[i] = c;
    double l = lev[i];
    mp.prob[n][i] = __ddiv_rn(l, T);
    mp.invp[n][i] = l > 0.0 ? (float)__ddiv_rn(T, l) : 0.f;
    // u < c  <=>  U < ceil(c * 2^53) for the 53-bit integer U with u = U * 2^-53; the last
    // threshold is 2^53 whatever the scores were (all zero or not finite for a factor that
    // failed its rank check on the device), so the sampler's search stays in the table
    mp.thr[n][i] = i == I - 1 ? (uint64_t(1) << 53) : (uint64_t)ceil(c * 9007199254740992.0);
  }
}

// Cyclic Jacobi eigen-decomposition (FP32) of each Gram matrix, one block per mode,
// parallel (round-robin) ordering of disjoint rotations.
// Cyclic Jacobi eigen-decomposition of the Gram matrices (one block per matrix, round-robin
// pairs), in T = float (the Alg. 2 preconditioner) or T = double (the Woodbury base of the
// Alg. 3 factor step, where the penalty w multiplies any non-orthogonality of V).
template <class T>
struct JacobiArgs {
  int R[KR_MAX_MODES];
  const double* gram[KR_MAX_MODES];
  T* V[KR_MAX_MODES];
  T* sig2[KR_MAX_MODES];
};
__device__ __forceinline__ float jac_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jac_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float jac_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double jac_abs(double x) { return fabs(x); }
__device__ __forceinline__ float jac_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double jac_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float jac_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double jac_max(double a, double b) { return fmax(a, b); }

template <class T>
__global__ void k_jacobi(JacobiArgs<T> ja) {
  const int n = blockIdx.x;
  const int R = ja.R[n];
  const int m = (R + 1) & ~1;
  extern __shared__ __align__(16) unsigned char jac_raw[];
  T* A = reinterpret_cast<T*>(jac_raw);  // (MAXR+1) x LD
  T* V = A + (MAXR + 1) * LD;
  __shared__ T cs[MAXR / 2 + 1], sn[MAXR / 2 + 1];
  __shared__ int pp[MAXR / 2 + 1], qq[MAXR / 2 + 1];
  __shared__ T red[2];
  const int tid = threadIdx.x;
  const T one = T(1), zero = T(0);
  for (int e = tid; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    A[i * LD + j] = (i < R && j < R) ? (T)ja.gram[n][i * R + j] : zero;
    V[i * LD + j] = (i == j) ? one : zero;
  }
  __syncthreads();
  // converged when the off-diagonal squares are below 1e-14 (FP32) / 1e-26 (FP64) of the diagonal's
  // (FP64: an off-diagonal norm ~3e-13 of the matrix's, above the rounding floor of about
  // R * 1e-16 that a stricter test would never reach)
  const T conv = sizeof(T) == 4 ? T(1e-14f) : T(1e-26);
  const int max_sweeps = sizeof(T) == 4 ? 20 : 40;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < m - 1; ++r) {
      if (tid < m / 2) {
        int k = tid;
        // players 1..m-1 rotate around player 0
        int p = (k == 0) ? 0 : 1 + ((k - 1 + r) % (m - 1));
        int q = 1 + ((m - 2 - k + r) % (m - 1));
        if (p > q) { int t = p; p = q; q = t; }
        T apq = A[p * LD + q], app = A[p * LD + p], aqq = A[q * LD + q];
        T c = one, s = zero;
        if (jac_abs(apq) > T(1e-30f) * (jac_abs(app) + jac_abs(aqq)) && apq != zero) {
          T tau = (aqq - app) / (T(2) * apq);
          T t = (tau >= zero ? one : -one) / (jac_abs(tau) + jac_sqrt(one + tau * tau));
          c = jac_rsqrt(one + t * t);
          s = t * c;
        }
        cs[k] = c; sn[k] = s; pp[k] = p; qq[k] = q;
      }
      __syncthreads();
      for (int w = tid; w < (m / 2) * m; w += blockDim.x) {  // rows: A <- J^T A
        int k = w / m, j = w % m;
        T c = cs[k], s = sn[k];
        if (s == zero) continue;
        int p = pp[k], q = qq[k];
        T ap = A[p * LD + j], aq = A[q * LD + j];
        A[p * LD + j] = c * ap - s * aq;
        A[q * LD + j] = s * ap + c * aq;
      }
      __syncthreads();
      for (int w = tid; w < (m / 2) * m; w += blockDim.x) {  // columns: A <- A J, V <- V J
        int k = w / m, i = w % m;
        T c = cs[k], s = sn[k];
        if (s == zero) continue;
        int p = pp[k], q = qq[k];
        T ap = A[i * LD + p], aq = A[i * LD + q];
        A[i * LD + p] = c * ap - s * aq;
        A[i * LD + q] = s * ap + c * aq;
        T vp = V[i * LD + p], vq = V[i * LD + q];
        V[i * LD + p] = c * vp - s * vq;
        V[i * LD + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    if (tid == 0) {
      T off = zero, dg = zero;
      for (int i = 0; i < R; ++i)
        for (int j = 0; j < R; ++j) {
          T v = A[i * LD + j];
          if (i == j) dg += v * v; else off += v * v;
        }
      red[0] = off; red[1] = dg;
    }
    __syncthreads();
    bool done = red[0] <= conv * red[1];
    __syncthreads();
    if (done) break;
  }
  for (int e = tid; e < R * R; e += blockDim.x) ja.V[n][e] = V[(e / R) * LD + (e % R)];
  for (int i = tid; i < R; i += blockDim.x) ja.sig2[n][i] = jac_max(A[i * LD + i], zero);
}

// FP32 copies of the FP64 eigenpairs, all modes in one grid (mode n's R x R vectors then
// its R values, in mode order).
__global__ void k_eig_to_f32(ModePtrs mp, PtrSet V64, PtrSet s64) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  for (int n = 0; n < mp.N; ++n) {
    const int R = mp.R[n], rr = R * R;
    if (e < rr) {
      mp.V[n][e] = (float)V64.p[n][e];
      return;
    }
    e -= rr;
    if (e < R) {
      mp.sig2[n][e] = (float)s64.p[n][e];
      return;
    }
    e -= R;
  }
}

}  // namespace

kr_status kr_eig64(kr_ctx* ctx, int nmat, const int* R, const double* const* gram, double* const* V,
                   double* const* sig2) {
  if (nmat < 1 || nmat > KR_MAX_MODES) return kr_fail(ctx, KR_EINVAL, "eig64: %d matrices", nmat);
  JacobiArgs<double> ja = {};
  for (int n = 0; n < nmat; ++n) {
    if (R[n] < 1 || R[n] > MAXR) return kr_fail(ctx, KR_EINVAL, "eig64: R=%d", R[n]);
    ja.R[n] = R[n];
    ja.gram[n] = gram[n];
    ja.V[n] = V[n];
    ja.sig2[n] = sig2[n];
  }
  const size_t smem = 2 * (MAXR + 1) * LD * sizeof(double);
  KR_TRY(kr_smem_attr(ctx, k_jacobi<double>, smem));
  KR_LAUNCH(ctx, k_jacobi<double>, nmat, 256, smem, ja);
  return KR_OK;
}

void kr_tables_need(const Modes& m, bool want_eig, Need& nd) {
  for (int n = 0; n < m.N; ++n) {
    int I = m.I[n], R = m.R[n];
    nd.add<double>((size_t)((I + GRAM_ROWS - 1) / GRAM_ROWS) * R * R);
    nd.add<double>((size_t)R * R);  // gram
    nd.add<double>((size_t)R * R);  // linv
    nd.add<double>(I);
    nd.add<double>(I);
    nd.add<double>(I);
    nd.add<uint64_t>(I);
    nd.add<float>(I);
    nd.add<float>((size_t)R * R);
    nd.add<double>((size_t)R * JL_MAXK);  // JL basis L^-T Pi
    if (want_eig) {
      nd.add<float>((size_t)R * R);
      nd.add<float>(R);
      nd.add<double>((size_t)R * R);  // FP64 eigenvectors
      nd.add<double>(R);              // FP64 eigenvalues
    }
  }
  nd.add<int>(KR_MAX_MODES);
}

kr_status kr_tables_build(kr_ctx* ctx, const Modes& m, bool want_eig, Carve& cv, FactorTables& t, bool check_rank) {
  double* V64[KR_MAX_MODES] = {};
  double* s64[KR_MAX_MODES] = {};
  double* jlB[KR_MAX_MODES] = {};
  ModePtrs mp = {};
  mp.N = m.N;
  t.N = m.N;
  int maxI = 0;
  for (int n = 0; n < m.N; ++n) {
    int I = m.I[n], R = m.R[n];
    mp.I[n] = I; mp.R[n] = R; mp.A[n] = m.A[n];
    t.I[n] = I; t.R[n] = R;
    mp.part[n] = cv.take<double>((size_t)((I + GRAM_ROWS - 1) / GRAM_ROWS) * R * R);
    mp.gram[n] = t.gram[n] = cv.take<double>((size_t)R * R);
    mp.linv[n] = t.linv[n] = cv.take<double>((size_t)R * R);
    mp.lev[n] = t.lev[n] = cv.take<double>(I);
    mp.cdf[n] = t.cdf[n] = cv.take<double>(I);
    mp.prob[n] = t.prob[n] = cv.take<double>(I);
    mp.thr[n] = t.thr[n] = cv.take<uint64_t>(I);
    mp.invp[n] = t.invp[n] = cv.take<float>(I);
    mp.ginv[n] = t.ginv[n] = cv.take<float>((size_t)R * R);
    jlB[n] = cv.take<double>((size_t)R * JL_MAXK);
    if (want_eig) {
      mp.V[n] = t.V[n] = cv.take<float>((size_t)R * R);
      mp.sig2[n] = t.sig2[n] = cv.take<float>(R);
      V64[n] = t.V64[n] = cv.take<double>((size_t)R * R);
      s64[n] = t.sig64[n] = cv.take<double>(R);
    }
    maxI = I > maxI ? I : maxI;
  }
  mp.flags = t.flags = cv.take<int>(KR_MAX_MODES);
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "tables: workspace too small");

  const size_t chol_smem = (size_t)MAXR * LD * sizeof(double);
  const size_t lev_smem = (MAXR * LD + LEV_ROWS * LD) * sizeof(double);
  KR_TRY(kr_smem_attr(ctx, k_cholesky, chol_smem));
  KR_TRY(kr_smem_attr(ctx, k_leverage, lev_smem));
  dim3 gg((maxI + GRAM_ROWS - 1) / GRAM_ROWS, m.N);
  KR_LAUNCH(ctx, k_gram_partial, gg, 256, 0, mp);
  int maxR = 0;
  for (int n = 0; n < m.N; ++n) maxR = m.R[n] > maxR ? m.R[n] : maxR;
  KR_LAUNCH(ctx, k_gram_reduce, dim3((maxR * maxR + 255) / 256, m.N), 256, 0, mp);
  KR_LAUNCH(ctx, k_cholesky, m.N, 256, chol_smem, mp);
  KR_LAUNCH(ctx, k_trinv, dim3(maxR, m.N), 32, 0, mp);
  KR_LAUNCH(ctx, k_ginv, dim3(maxR, m.N), 64, 0, mp);
  dim3 gl((maxI + LEV_ROWS - 1) / LEV_ROWS, m.N);
  if (ctx->jl_k > 0) {
    const int k = ctx->jl_k;
    const size_t jl_smem = ((size_t)MAXR * JL_MAXK + LEV_ROWS * LD) * sizeof(double);
    KR_TRY(kr_smem_attr(ctx, k_leverage_jl, jl_smem));
    PtrSet jls = {};
    for (int n = 0; n < m.N; ++n) jls.p[n] = jlB[n];
    KR_LAUNCH(ctx, k_jl_basis, dim3((maxR * k + 255) / 256, m.N), 256, 0, mp, k, (uint32_t)ctx->jl_seed,
              (uint32_t)(ctx->jl_seed >> 32), jls);
    KR_LAUNCH(ctx, k_leverage_jl, gl, LEV_ROWS * 32, jl_smem, mp, k, jls);
  } else {
    KR_LAUNCH(ctx, k_leverage, gl, LEV_ROWS * 32, lev_smem, mp);
  }
  KR_LAUNCH(ctx, k_cdf, m.N, CDF_THREADS, 0, mp);
  if (want_eig) {
    KR_TRY(kr_eig64(ctx, m.N, m.R, mp.gram, V64, s64));
    int tot = 0;
    for (int n = 0; n < m.N; ++n) tot += m.R[n] * (m.R[n] + 1);
    PtrSet vs = {}, ss = {};
    for (int n = 0; n < m.N; ++n) {
      vs.p[n] = V64[n];
      ss.p[n] = s64[n];
    }
    KR_LAUNCH(ctx, k_eig_to_f32, (tot + 255) / 256, 256, 0, mp, vs, ss);
  }
  if (check_rank) {
    int ntot = 0;
    if (want_eig)
      for (int n = 0; n < m.N; ++n) ntot += m.R[n];
    KR_TRY(kr_hbuf_reserve(ctx, 4096 + sizeof(double) * (size_t)ntot));
    int* hf = (int*)ctx->hbuf;
    double* hs = reinterpret_cast<double*>(ctx->hbuf + 4096);  // eigenvalues past the small read-back area
    KR_CUDA(ctx, cudaMemcpyAsync(hf, mp.flags, sizeof(int) * m.N, cudaMemcpyDeviceToHost, ctx->stream));
    if (want_eig) {
      int off = 0;
      for (int n = 0; n < m.N; ++n) {
        KR_CUDA(ctx, cudaMemcpyAsync(hs + off, s64[n], sizeof(double) * m.R[n], cudaMemcpyDeviceToHost, ctx->stream));
        off += m.R[n];
      }
    }
    KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (want_eig) {
      int off = 0;
      for (int n = 0; n < m.N; ++n) {
        double lo = INFINITY, hi = 0.0;
        for (int r = 0; r < m.R[n]; ++r) {
          lo = fmin(lo, hs[off + r]);
          hi = fmax(hi, hs[off + r]);
        }
        t.sig_min[n] = fmax(lo, 0.0);
        t.sig_max[n] = hi;
        off += m.R[n];
      }
    }
    for (int n = 0; n < m.N; ++n) {
      t.rank[n] = hf[n] ? -1 : m.R[n];
      if (hf[n]) return kr_fail(ctx, KR_ERANK, "factor %d is numerically rank deficient (Cholesky pivot)", n);
    }
  }
  return KR_OK;
}

extern "C" kr_status kron_leverage(kr_ctx* ctx, const kr_factors* f, double* const lev[], double* const cdf[],
                                   double* const prob[], int32_t* rank) {
  if (!ctx) return KR_EINVAL;
  Modes m;
  KR_TRY(kr_check_factors(ctx, f, &m));
  Need nd;
  kr_tables_need(m, false, nd);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  Carve cv(ctx->ws, ctx->ws_size);
  FactorTables t;
  kr_status st = kr_tables_build(ctx, m, false, cv, t, true);
  if (rank)
    for (int n = 0; n < m.N; ++n) rank[n] = t.rank[n] < 0 ? -1 : m.R[n];
  if (st != KR_OK && st != KR_ERANK) return st;
  for (int n = 0; n < m.N; ++n) {
    size_t bytes = sizeof(double) * m.I[n];
    if (lev && lev[n]) KR_CUDA(ctx, cudaMemcpyAsync(lev[n], t.lev[n], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (cdf && cdf[n]) KR_CUDA(ctx, cudaMemcpyAsync(cdf[n], t.cdf[n], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (prob && prob[n]) KR_CUDA(ctx, cudaMemcpyAsync(prob[n], t.prob[n], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return st;
}
