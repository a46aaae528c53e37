// Alg. 3 FastFactorMatrixUpdate, batched over the rows of one factor, and Alg. 1
// TuckerALS (sampled factor steps, then a sampled core step).
//
// Factor step for mode n (App. C): with K = (x)_{m != n} A(m), G = G_(n) (R_n x R_{!=n},
// columns in C-order over the other modes), G+ = pinv(G) and the penalty
// w = (1 + 12/eps) prod_{m != n} sigma_max(A(m))^2, each row i of X_(n) solves
//   min_z ||S_i (K z - b_i)||^2 + lambda ||(G^T)^+ z||^2 + w ||N z||^2,  N = I - G+ G,
// by the Richardson iteration of Alg. 3,
//   z <- z - (1 - sqrt(eps)) M^-1 ((K~^T K~ + w I) z + lambda G+ (G+)^T z - w G+ G z - K~^T b~),
// with a fresh sketch S_i per row, and returns a_i = (G+)^T z. The preconditioner is the
// unsampled M = K^T K + w I + G+ (lambda (G+)^T - w G), inverted with the Woodbury
// identity (standard sign)
//   M^-1 = A^-1 - A^-1 U (I + V A^-1 U)^-1 V A^-1,  A = K^T K + w I, U = G+, V = lambda (G+)^T - w G,
// where A^-1 = (x)V_m (S_m^2 (x)... + w)^-1 (x)V_m^T from the factor eigen-decompositions.
//
// All rows of the factor run together: the sketch keys draws by (row, cell), b~ is
// gathered from X_(n), and the sampled products run in the slab pass (two other modes)
// or between batched mode products. With one or two other modes, everything after the
// sampled products is one kernel per row (k_factor_rows) in FP64: the Woodbury pieces
// come from FP64 eigen-decompositions, because w multiplies any error of A^-1 and the
// capacitance I + V A^-1 U cancels to about 1/((1 + 12/eps) cond(K^T K)) of the terms that
// form it. With more other modes the batched FP32 mode-product chain applies M^-1 (the
// capacitance still in FP64). The Richardson iterations after the first run as one CUDA
// graph with the stopping rule on the device.
#include <math.h>
#include <stdio.h>

#include "kr_internal.cuh"

namespace {

struct Dims {
  int N;
  int R[KR_MAX_MODES];
};

// G (C-order over R) -> Gn (R_n x Rne) and Gt = Gn^T (Rne x R_n).
__global__ void k_unfold(const float* __restrict__ G, Dims d, int n, int64_t Rtot, int Rne, float* __restrict__ Gn,
                         float* __restrict__ Gt) {
  const int Rn = d.R[n];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Rtot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e;
    int idx[KR_MAX_MODES];
    for (int m = d.N - 1; m >= 0; --m) {
      idx[m] = (int)(rem % d.R[m]);
      rem /= d.R[m];
    }
    int64_t k = 0;
    for (int m = 0; m < d.N; ++m)
      if (m != n) k = k * d.R[m] + idx[m];
    const float v = G[e];
    Gn[(int64_t)idx[n] * Rne + k] = v;
    Gt[k * Rn + idx[n]] = v;
  }
}

// out = ca * a + cb * b
__global__ void k_lin2(float* __restrict__ out, const float* __restrict__ a, float ca, const float* __restrict__ b,
                       float cb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = ca * a[i] + cb * b[i];
}

// Hinv = L^-T L^-1 = (G_(n) G_(n)^T)^-1 in FP64 from the inverse Cholesky factor (one block).
__global__ void k_hinv(const double* __restrict__ linv, int Rn, double* __restrict__ hinv) {
  for (int e = threadIdx.x; e < Rn * Rn; e += blockDim.x) {
    const int i = e / Rn, j = e % Rn;
    double acc = 0.0;
    for (int k = i > j ? i : j; k < Rn; ++k) acc = fma(linv[k * Rn + i], linv[k * Rn + j], acc);
    hinv[e] = acc;
  }
}

// G+ = G_(n)^T Hinv in FP64 (Rne x R_n), and its FP32 copy for the preconditioner.
__global__ void k_gp64(const float* __restrict__ Gt, const double* __restrict__ hinv, int Rn, int64_t Rne,
                       double* __restrict__ gp64, float* __restrict__ gp32) {
  const int64_t tot = Rne * Rn;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / Rn;
    const int a = (int)(e % Rn);
    double acc = 0.0;
    for (int b = 0; b < Rn; ++b) acc = fma((double)Gt[k * Rn + b], hinv[b * Rn + a], acc);
    gp64[e] = acc;
    gp32[e] = (float)acc;
  }
}

// Per row i (one block): the deterministic part of Alg. 3's gradient in FP64,
//   grad = w z + G+ (lambda (G+)^T z - w G z) - gsk,
// where w z and G+ (w G z) cancel in the row space of G^T (exactly, for exact G+), so the
// combination is formed in FP64 from the FP32 iterate. With out_a != null the block
// instead writes the factor row a_i = (G+)^T z_i.
constexpr int PEN_MAXRN = KR_MAX_RANK;
__global__ void __launch_bounds__(256) k_penalty_rows(const float* __restrict__ Z, const float* __restrict__ Gn,
                                                      const double* __restrict__ gp64, const float* __restrict__ gsk,
                                                      int Rn, int Rne, double lambda, double w_arg,
                                                      float* __restrict__ grad, float* __restrict__ out_a,
                                                      double* __restrict__ grad64, const double* __restrict__ wp) {
  extern __shared__ double zs[];  // Rne
  const double w = wp ? *wp : w_arg;  // the penalty on the device (graph sweeps) or by value
  __shared__ double tv[PEN_MAXRN], uv[PEN_MAXRN];
  const int64_t row = blockIdx.x;
  const float* z = Z + row * Rne;
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) zs[k] = (double)z[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a = warp; a < Rn; a += nw) {
    double t = 0.0, u = 0.0;
    for (int k = lane; k < Rne; k += 32) {
      t = fma((double)Gn[(int64_t)a * Rne + k], zs[k], t);
      u = fma(gp64[(int64_t)k * Rn + a], zs[k], u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, off);
      u += __shfl_xor_sync(0xffffffffu, u, off);
    }
    if (lane == 0) {
      tv[a] = t;
      uv[a] = u;
    }
  }
  __syncthreads();
  if (out_a) {
    for (int a = threadIdx.x; a < Rn; a += blockDim.x) out_a[row * Rn + a] = (float)uv[a];
    return;
  }
  for (int a = threadIdx.x; a < Rn; a += blockDim.x) tv[a] = lambda * uv[a] - w * tv[a];
  __syncthreads();
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) {
    double c = 0.0;
    for (int a = 0; a < Rn; ++a) c = fma(gp64[(int64_t)k * Rn + a], tv[a], c);
    const double gv = w * zs[k] + c - (double)gsk[row * Rne + k];
    if (grad64)
      grad64[row * Rne + k] = gv;
    else
      grad[row * Rne + k] = (float)gv;
  }
}

// Vw[a][k] = lambda * Gp[k][a] - w * Gn[a][k]  (R_n x Rne);  GpT[a][k] = Gp[k][a]
__global__ void k_vw(const float* __restrict__ Gp, const float* __restrict__ Gn, int Rn, int Rne, float lambda,
                     float w_arg, float* __restrict__ Vw, float* __restrict__ GpT, const double* __restrict__ wp) {
  const float w = wp ? (float)*wp : w_arg;
  const int64_t tot = (int64_t)Rn * Rne;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / Rne), k = (int)(e % Rne);
    const float gp = Gp[(int64_t)k * Rn + a];
    GpT[e] = gp;
    Vw[e] = lambda * gp - w * Gn[e];
  }
}

// C[a][b] = delta_ab + sum_k Vw[a][k] AinvUt[b][k], FP64 accumulation; block per (a, b).
__global__ void k_capacitance(const float* __restrict__ Vw, const float* __restrict__ AinvUt, int Rn, int Rne,
                              double* __restrict__ C) {
  const int a = blockIdx.x / Rn, b = blockIdx.x % Rn;
  double acc = 0.0;
  for (int k = threadIdx.x; k < Rne; k += blockDim.x)
    acc += (double)Vw[(int64_t)a * Rne + k] * (double)AinvUt[(int64_t)b * Rne + k];
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    C[blockIdx.x] = t + (a == b ? 1.0 : 0.0);
  }
}

// Gauss-Jordan inverse with partial pivoting in FP64 (one block, n <= 64).
__global__ void k_gauss_jordan(const double* __restrict__ C, int n, float* __restrict__ Cinv, int* __restrict__ bad,
                               double* __restrict__ Cinv64) {
  extern __shared__ double aug[];  // n x 2n
  const int w2 = 2 * n;
  __shared__ int piv;
  __shared__ double pv;
  for (int e = threadIdx.x; e < n * w2; e += blockDim.x) {
    const int i = e / w2, j = e % w2;
    aug[e] = j < n ? C[i * n + j] : (j - n == i ? 1.0 : 0.0);
  }
  if (threadIdx.x == 0) *bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(aug[k * w2 + k]);
      for (int i = k + 1; i < n; ++i) {
        double v = fabs(aug[i * w2 + k]);
        if (v > best) { best = v; p = i; }
      }
      piv = p;
      pv = aug[p * w2 + k];
      if (!(best > 0.0)) *bad = 1;
    }
    __syncthreads();
    const int p = piv;
    const double pivot = pv != 0.0 ? pv : 1.0;
    if (p != k)
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        double t = aug[k * w2 + j];
        aug[k * w2 + j] = aug[p * w2 + j];
        aug[p * w2 + j] = t;
      }
    __syncthreads();
    for (int j = threadIdx.x; j < w2; j += blockDim.x) aug[k * w2 + j] /= pivot;
    __syncthreads();
    for (int e = threadIdx.x; e < n * w2; e += blockDim.x) {
      const int i = e / w2, j = e % w2;
      if (i == k) continue;
      const double f = aug[i * w2 + k];
      if (j != k) aug[e] -= f * aug[k * w2 + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) aug[i * w2 + k] = 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const double v = aug[(e / n) * w2 + n + (e % n)];
    Cinv[e] = (float)v;
    if (Cinv64) Cinv64[e] = v;
  }
}

// z <- z - alpha d, one block per row; rowstat[r] = {||step||^2, ||z||^2, non-finite}.
// The sums inside the block are FP32 fixed-order trees (FP64 issues at a small fraction of
// the FP32 rate here; a stopping-rule norm needs no more than FP32's relative precision);
// rowstat holds them in FP64 for the sums over rows.
__global__ void k_row_update(float* __restrict__ z, const float* __restrict__ d, float alpha, int L,
                             double* __restrict__ rowstat) {
  const int64_t base = (int64_t)blockIdx.x * L;
  float s1 = 0.f, s2 = 0.f, bad = 0.f;
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const float st = alpha * d[base + k];
    const float zn = z[base + k] - st;
    z[base + k] = zn;
    s1 = fmaf(st, st, s1);
    s2 = fmaf(zn, zn, s2);
    if (!isfinite(zn)) bad = 1.f;
  }
  __shared__ float red[3][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    bad = fmaxf(bad, __shfl_xor_sync(0xffffffffu, bad, off));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
    red[2][threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
      c = fmaxf(c, red[2][k]);
    }
    rowstat[3 * (int64_t)blockIdx.x + 0] = (double)a;
    rowstat[3 * (int64_t)blockIdx.x + 1] = (double)b;
    rowstat[3 * (int64_t)blockIdx.x + 2] = (double)c;
  }
}

// The Woodbury base A^-1 = (K^T K + w I)^-1 = (V1 (x) V2)(S1^2 (x) S2^2 + w)^-1 (V1 (x) V2)^T on
// one R1 x R2 block in FP64, from FP64 eigen-decompositions of the other modes' Gram
// matrices. With w >> ||K^T K|| every piece of the Woodbury form is kept in FP64: the
// capacitance I + V A^-1 U cancels to about 1/((1 + 12/eps) cond(K^T K)) of its terms, and an
// error e in A^-1 (or in V's orthogonality) acts like a perturbation w e of K^T K, which
// left in FP32 slows Richardson from ~16 to hundreds of iterations once the factors lose
// their orthonormality. One other mode: R1 = 1 and V1 = S1 = 1 (V1 == nullptr).
struct WbBase {
  int R1, R2;
  const double* V1;  // R1 x R1 eigenvectors (columns), nullptr for R1 = 1
  const double* V2;  // R2 x R2
  const double* s1;  // R1 eigenvalues (nullptr for R1 = 1)
  const double* s2;  // R2
  double w;
  const double* wp;  // when set, the penalty is read here (computed on the device) instead of w
};

// M (R1 x R2, shared memory) <- A^-1 M; T is shared scratch of the same size. Called by
// every thread of the block (it synchronises).
__device__ void base_apply_block64(const WbBase& b, double* M, double* T) {
  const int R1 = b.R1, R2 = b.R2, n = R1 * R2;
  const double bw = b.wp ? *b.wp : b.w;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {  // T = V1^T M
    const int j = e / R2, l = e - j * R2;
    double acc = 0.0;
    if (b.V1)
      for (int k = 0; k < R1; ++k) acc = fma(b.V1[k * R1 + j], M[k * R2 + l], acc);
    else
      acc = M[e];
    T[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {  // M = (T V2) / (s1 s2 + w)
    const int j = e / R2, l = e - j * R2;
    double acc = 0.0;
    for (int r = 0; r < R2; ++r) acc = fma(T[j * R2 + r], b.V2[r * R2 + l], acc);
    const double d = (b.s1 ? b.s1[j] * b.s2[l] : b.s2[l]) + bw;
    M[e] = d > 0.0 ? acc / d : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {  // T = V1 M
    const int j = e / R2, l = e - j * R2;
    double acc = 0.0;
    if (b.V1)
      for (int k = 0; k < R1; ++k) acc = fma(b.V1[j * R1 + k], M[k * R2 + l], acc);
    else
      acc = M[e];
    T[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {  // M = T V2^T
    const int j = e / R2, r = e - j * R2;
    double acc = 0.0;
    for (int l = 0; l < R2; ++l) acc = fma(T[j * R2 + l], b.V2[r * R2 + l], acc);
    M[e] = acc;
  }
  __syncthreads();
}

// AinvU[a] = A^-1 (column a of G+), one block per column (FP64).
__global__ void __launch_bounds__(256) k_base_cols64(WbBase b, const double* __restrict__ gp64, int Rn, int Rne,
                                                     double* __restrict__ AinvU) {
  extern __shared__ double bc_smem[];
  double* M = bc_smem;
  double* T = bc_smem + Rne;
  const int a = blockIdx.x;
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) M[k] = gp64[(int64_t)k * Rn + a];
  __syncthreads();
  base_apply_block64(b, M, T);
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) AinvU[(int64_t)a * Rne + k] = M[k];
}

// Vw[a][k] = lambda G+[k][a] - w G_(n)[a][k]  (R_n x Rne, FP64)
__global__ void k_vw64(const double* __restrict__ gp64, const float* __restrict__ Gn, int Rn, int Rne, double lambda,
                       double w_arg, double* __restrict__ Vw, const double* __restrict__ wp) {
  const double w = wp ? *wp : w_arg;
  const int64_t tot = (int64_t)Rn * Rne;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / Rne), k = (int)(e % Rne);
    Vw[e] = lambda * gp64[(int64_t)k * Rn + a] - w * (double)Gn[e];
  }
}

// C[a][b] = delta_ab + sum_k Vw[a][k] AinvU[b][k] from FP64 inputs; block per (a, b).
__global__ void k_capacitance64(const double* __restrict__ Vw, const double* __restrict__ AinvU, int Rn, int Rne,
                                double* __restrict__ C) {
  const int a = blockIdx.x / Rn, b = blockIdx.x % Rn;
  double acc = 0.0;
  for (int k = threadIdx.x; k < Rne; k += blockDim.x)
    acc = fma(Vw[(int64_t)a * Rne + k], AinvU[(int64_t)b * Rne + k], acc);
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    C[blockIdx.x] = t + (a == b ? 1.0 : 0.0);
  }
}

// One Richardson step of every row of a factor step with at most two other modes (one
// block per row), all in FP64 up to the FP32 iterate: the gradient combination of
// k_penalty_rows, the Woodbury preconditioner
//   D = A^-1 g,   d = D - (A^-1 U) C^-1 V D,
// then z <- z - alpha d and the row statistics of k_row_update. Shared memory: z, and
// two R1 x R2 buffers, in FP64.
constexpr int FR_MAX_RNE = 4096;
struct RowStep {
  WbBase b;
  int Rn, Rne;
  const float* Gn;
  const double* gp64;
  const double* Vw;     // Rn x Rne: lambda (G+)^T - w G
  const double* AinvU;  // Rn x Rne: A^-1 applied to the columns of G+
  const double* Cinv;   // Rn x Rn
  double lambda, w, alpha;
  const double* wp;  // when set, the penalty is read here instead of w
  // the (1+eps)-aware rule: per row, q = g^T M+ g and the penalty part of the row's objective
  // at z before the step, lambda ||(G+)^T z||^2 + w ||(I - G+ G) z||^2 (null: not wanted)
  double* rowq;
  double* rowpen;
};
__global__ void __launch_bounds__(256) k_factor_rows(RowStep p, float* __restrict__ Z, const float* __restrict__ gsk,
                                                     double* __restrict__ rowstat) {
  extern __shared__ double fr_smem[];
  const int Rn = p.Rn, Rne = p.Rne;
  const bool eps = p.rowq != nullptr;
  double* zs = fr_smem;     // Rne
  double* M = zs + Rne;     // Rne
  double* T = M + Rne;      // Rne
  double* G4 = T + Rne;     // Rne: the gradient (eps rule only)
  __shared__ double tv[PEN_MAXRN], uv[PEN_MAXRN], gz[PEN_MAXRN];
  __shared__ float red[3][8];
  __shared__ double dred[2][8];
  const int64_t row = blockIdx.x;
  float* z = Z + row * Rne;
  const float* g_sk = gsk + row * Rne;
  const double pw = p.wp ? *p.wp : p.w;
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) zs[k] = (double)z[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // gradient: w z + G+ (lambda (G+)^T z - w G z) - gsk
  for (int a = warp; a < Rn; a += nw) {
    double t = 0.0, u = 0.0;
    for (int k = lane; k < Rne; k += 32) {
      t = fma((double)p.Gn[(int64_t)a * Rne + k], zs[k], t);
      u = fma(p.gp64[(int64_t)k * Rn + a], zs[k], u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, off);
      u += __shfl_xor_sync(0xffffffffu, u, off);
    }
    if (lane == 0) {
      tv[a] = t;
      uv[a] = u;
      gz[a] = t;
    }
  }
  __syncthreads();
  double pen = 0.0;  // this thread's part of the penalty terms (eps rule)
  if (eps)
    for (int a = threadIdx.x; a < Rn; a += blockDim.x) pen = fma(p.lambda * uv[a], uv[a], pen);
  __syncthreads();
  for (int a = threadIdx.x; a < Rn; a += blockDim.x) tv[a] = p.lambda * uv[a] - pw * tv[a];
  __syncthreads();
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) {
    double c = 0.0;
    for (int a = 0; a < Rn; ++a) c = fma(p.gp64[(int64_t)k * Rn + a], tv[a], c);
    M[k] = pw * zs[k] + c - (double)g_sk[k];
    if (eps) {  // (I - G+ G) z at k
      double gg = 0.0;
      for (int a = 0; a < Rn; ++a) gg = fma(p.gp64[(int64_t)k * Rn + a], gz[a], gg);
      const double nz = zs[k] - gg;
      pen = fma(pw * nz, nz, pen);
      G4[k] = M[k];
    }
  }
  __syncthreads();
  base_apply_block64(p.b, M, T);  // D = A^-1 g
  // Woodbury correction: u1 = V D (tv), u2 = C^-1 u1 (uv), d = D - (A^-1 U) u2
  for (int a = warp; a < Rn; a += nw) {
    double acc = 0.0;
    for (int k = lane; k < Rne; k += 32) acc = fma(p.Vw[(int64_t)a * Rne + k], M[k], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) tv[a] = acc;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < Rn; a += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < Rn; ++b) acc = fma(p.Cinv[a * Rn + b], tv[b], acc);
    uv[a] = acc;
  }
  __syncthreads();
  float s_1 = 0.f, s_2 = 0.f, bad = 0.f;
  double q = 0.0;  // this thread's part of g^T M+ g (eps rule)
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) {
    double gr = 0.0;
    for (int a = 0; a < Rn; ++a) gr = fma(p.AinvU[(int64_t)a * Rne + k], uv[a], gr);
    if (eps) q = fma(G4[k], M[k] - gr, q);
    const float st = (float)(p.alpha * (M[k] - gr));
    const float zn = (float)zs[k] - st;
    z[k] = zn;
    s_1 = fmaf(st, st, s_1);
    s_2 = fmaf(zn, zn, s_2);
    if (!isfinite(zn)) bad = 1.f;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s_1 += __shfl_xor_sync(0xffffffffu, s_1, off);
    s_2 += __shfl_xor_sync(0xffffffffu, s_2, off);
    bad = fmaxf(bad, __shfl_xor_sync(0xffffffffu, bad, off));
  }
  if (eps) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      q += __shfl_xor_sync(0xffffffffu, q, off);
      pen += __shfl_xor_sync(0xffffffffu, pen, off);
    }
  }
  if (lane == 0) {
    red[0][warp] = s_1;
    red[1][warp] = s_2;
    red[2][warp] = bad;
    dred[0][warp] = q;
    dred[1][warp] = pen;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, c = 0.f;
    double qs = 0.0, ps = 0.0;
    for (int k = 0; k < nw; ++k) {
      a += red[0][k];
      b += red[1][k];
      c = fmaxf(c, red[2][k]);
      qs += dred[0][k];
      ps += dred[1][k];
    }
    rowstat[3 * row + 0] = (double)a;
    rowstat[3 * row + 1] = (double)b;
    rowstat[3 * row + 2] = (double)c;
    if (eps) {
      p.rowq[row] = qs;
      p.rowpen[row] = ps;
    }
  }
}

// State of a factor step's Richardson loop on the device (the stopping rule's history).
struct FactorLoop {
  double h[4];
  double prev_step, min_step, min_rel, rel;
  int grow, since_min, it, status;
};

__global__ void k_factor_loop_init(FactorLoop* st) {
  st->prev_step = INFINITY;
  st->min_step = INFINITY;
  st->min_rel = INFINITY;
  st->rel = INFINITY;
  st->grow = 0;
  st->since_min = 0;
  st->it = 0;
  st->status = STEP_CONTINUE;
}

// out = {sum ||step||^2, sum ||z||^2, any non-finite, max_r ||step_r|| / ||z_r||} (one block).
// With st, thread 0 then applies the stopping rule (the same function as the host loop,
// on the largest per-row ratio), counts the iteration, stops at max_iter, and inside a
// graph sets the loop condition.
// The (1+eps)-aware rule of the rows (on): row i's objective before the step is its slab's
// tile objective partials (the sampled term, tiles [tstart[i], tstart[i + 1])) plus pen[i],
// and the rule holds for it when rho^2 q_i / c1 <= theta eps (f_i - q_i / c1) (Lemma 4.2 and
// the proof of Thm 4.5, with the bounds of the penalised sampled matrix).
struct RowsEps {
  int on;
  const double* q;
  const double* pen;
  const double* objpart;
  const uint32_t* tstart;
  double rho2_c1, inv_c1, theta_eps;
};

__global__ void k_rows_reduce(const double* __restrict__ rowstat, int nrow, double* __restrict__ out,
                              FactorLoop* __restrict__ st, double tol, int max_iter, cudaGraphConditionalHandle hnd,
                              int use_hnd, RowsEps re) {
  double s1 = 0, s2 = 0, bad = 0, mx = 0, fail = 0;
  for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
    const double a = rowstat[3 * r], b = rowstat[3 * r + 1];
    s1 += a;
    s2 += b;
    bad = fmax(bad, rowstat[3 * r + 2]);
    const double rel = b > 0.0 ? sqrt(a / b) : (a > 0.0 ? INFINITY : 0.0);
    mx = fmax(mx, rel);
    if (re.on) {
      double f = re.pen[r];
      for (uint32_t t = re.tstart[r]; t < re.tstart[r + 1]; ++t) f += re.objpart[t];
      const double q = re.q[r];
      const bool ok = isfinite(f) && isfinite(q) && re.rho2_c1 * q <= re.theta_eps * fmax(f - q * re.inv_c1, 0.0);
      if (!ok) fail = 1.0;
    }
  }
  __shared__ double red[5][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, off));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    fail = fmax(fail, __shfl_xor_sync(0xffffffffu, fail, off));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
    red[2][threadIdx.x >> 5] = bad;
    red[3][threadIdx.x >> 5] = mx;
    red[4][threadIdx.x >> 5] = fail;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0, d = 0, e = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
      c = fmax(c, red[2][k]);
      d = fmax(d, red[3][k]);
      e = fmax(e, red[4][k]);
    }
    out[0] = a;
    out[1] = b;
    out[2] = c;
    out[3] = d;
    if (st) {
      const double hv[4] = {a, b, c, d};
      for (int k = 0; k < 4; ++k) st->h[k] = hv[k];
      st->it += 1;
      int status = STEP_CONTINUE;
      if (re.on && e == 0.0 && c == 0.0) status = STEP_EPS;  // every row's rule holds
      if (status == STEP_CONTINUE)
        status = step_check(hv, tol, &st->prev_step, &st->min_step, &st->min_rel, &st->grow, &st->since_min,
                            &st->rel, d);
      if (status == STEP_CONTINUE && st->it >= max_iter) status = STEP_MAXITER;
      st->status = status;
      if (use_hnd) cudaGraphSetConditional(hnd, status == STEP_CONTINUE ? 1u : 0u);
    }
  }
}

// ------------------------------------------------------------------ FP64 Woodbury chain
//
// Factor steps with three or more other modes (or more unknowns per row than the fused row
// kernel takes) apply the Woodbury preconditioner as a batched chain over the rows:
//   D = A^-1 grad,  A^-1 = (x)V_m (S^2 + w)^-1 (x)V_m^T   (mode products, all rows at once)
//   d = D - (A^-1 U) C^-1 V D                              (per row)
// in FP64 throughout (the reasons of WbBase hold for any number of modes: w multiplies every
// error of A^-1), up to the FP32 iterate z.

// out[p, j, q] = sum_k B'[j, k] in[p, k, q], B' = V (trans = 0) or V^T (trans = 1), V R x R.
__global__ void k_mode_sq64(const double* __restrict__ in, double* __restrict__ out, int64_t P, int R, int64_t Q,
                            const double* __restrict__ V, int trans) {
  const int64_t tot = P * R * Q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e % Q;
    const int64_t pj = e / Q;
    const int j = (int)(pj % R);
    const int64_t p = pj / R;
    const double* col = in + p * R * Q + q;
    double acc = 0.0;
    for (int k = 0; k < R; ++k) acc = fma(trans ? V[(int64_t)k * R + j] : V[(int64_t)j * R + k], col[(int64_t)k * Q], acc);
    out[e] = acc;
  }
}

struct Diag64 {
  int No;
  int R[KR_MAX_MODES];
  const double* s[KR_MAX_MODES];
  const double* wp;  // when set, the penalty is read here instead of the w argument
};

// x[b, r] /= prod_m s_m[r_m] + w over the trailing Rne entries of every batch row b.
__global__ void k_diag_w64(double* __restrict__ x, int64_t total, int64_t Rne, Diag64 d, double w_arg) {
  const double w = d.wp ? *d.wp : w_arg;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = i % Rne;
    double prod = 1.0;
    for (int m = d.No - 1; m >= 0; --m) {
      const int r = (int)(rem % d.R[m]);
      rem /= d.R[m];
      prod *= d.s[m][r];
    }
    const double dv = prod + w;
    x[i] = dv > 0.0 ? x[i] / dv : 0.0;
  }
}

// out[c][r] = in[r][c] (rows x cols, FP64).
__global__ void k_transpose64(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
  const int64_t tot = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    out[c * rows + r] = in[e];
  }
}

// One block per row i: u = V D_i (R_n), v = C^-1 u, d = D_i - (A^-1 U)^T v, then z_i <- z_i - alpha d
// with the row statistics of k_row_update (FP32 step norms).
__global__ void __launch_bounds__(256) k_wb_rows64(const double* __restrict__ D, const double* __restrict__ Vw,
                                                   const double* __restrict__ Cinv, const double* __restrict__ AinvU,
                                                   int Rn, int Rne, float* __restrict__ Z, float alpha,
                                                   double* __restrict__ rowstat) {
  __shared__ double uv[KR_MAX_RANK], vv[KR_MAX_RANK];
  const int64_t row = blockIdx.x;
  const double* Di = D + row * Rne;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a = warp; a < Rn; a += nw) {
    double t = 0.0;
    for (int k = lane; k < Rne; k += 32) t = fma(Vw[(int64_t)a * Rne + k], Di[k], t);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) uv[a] = t;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < Rn; a += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < Rn; ++b) t = fma(Cinv[(int64_t)a * Rn + b], uv[b], t);
    vv[a] = t;
  }
  __syncthreads();
  float s1 = 0.f, s2 = 0.f, bad = 0.f;
  float* z = Z + row * Rne;
  for (int k = threadIdx.x; k < Rne; k += blockDim.x) {
    double c = Di[k];
    for (int a = 0; a < Rn; ++a) c = fma(-AinvU[(int64_t)a * Rne + k], vv[a], c);
    const float st = alpha * (float)c;
    const float zn = z[k] - st;
    z[k] = zn;
    s1 = fmaf(st, st, s1);
    s2 = fmaf(zn, zn, s2);
    if (!isfinite(zn)) bad = 1.f;
  }
  __shared__ float red[3][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    bad = fmaxf(bad, __shfl_xor_sync(0xffffffffu, bad, off));
  }
  if (lane == 0) {
    red[0][warp] = s1;
    red[1][warp] = s2;
    red[2][warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int k = 0; k < nw; ++k) {
      a += red[0][k];
      b += red[1][k];
      c = fmaxf(c, red[2][k]);
    }
    rowstat[3 * row + 0] = (double)a;
    rowstat[3 * row + 1] = (double)b;
    rowstat[3 * row + 2] = (double)c;
  }
}

int grid_of(kr_ctx* ctx, int64_t work) {
  int64_t g = (work + 255) / 256;
  if (g > ctx->num_sms * 8) g = ctx->num_sms * 8;
  return g < 1 ? 1 : (int)g;
}

// Batched A^-1 = (x)V (S^2 + w)^-1 (x)V^T over the other modes for `nrow` vectors.
kr_status base_apply(kr_ctx* ctx, const FactorTables& to, int nrow, double w, const float* in, float* out, float* t0,
                     float* t1) {
  const int No = to.N;
  int dims[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  int tr[KR_MAX_MODES];
  dims[0] = nrow;
  B[0] = nullptr;
  tr[0] = 0;
  int64_t Rne = 1;
  for (int m = 0; m < No; ++m) {
    dims[m + 1] = to.R[m];
    B[m + 1] = to.V[m];
    tr[m + 1] = 1;
    Rne *= to.R[m];
  }
  KR_TRY(kr_kron_apply2(ctx, No + 1, dims, dims, B, tr, in, out, t0, t1));
  KR_TRY(kr_diag_scale(ctx, to, w, out, Rne * nrow));
  for (int m = 0; m < No; ++m) tr[m + 1] = 0;
  return kr_kron_apply2(ctx, No + 1, dims, dims, B, tr, out, out, t0, t1);
}

// Batched FP64 A^-1 = (x)V (S^2 + w)^-1 (x)V^T over the No other modes for `nrow` rows of Rne
// entries: out = A^-1 in (tmp: nrow * Rne doubles; in aliases neither out nor tmp).
kr_status base_apply64(kr_ctx* ctx, int No, const int* Ro, double* const* V64, double* const* s64, int nrow, double w,
                       const double* in, double* out, double* tmp, const double* wp = nullptr) {
  int64_t Rne = 1;
  for (int m = 0; m < No; ++m) Rne *= Ro[m];
  const int64_t tot = Rne * nrow;
  const int grid = grid_of(ctx, tot);
  const double* src = in;
  int k = 0;
  for (int pass = 0; pass < 2; ++pass) {  // V^T along every mode, the diagonal, then V
    int64_t P = nrow, Q = Rne;
    for (int m = 0; m < No; ++m) {
      Q /= Ro[m];
      double* dst = (k & 1) ? out : tmp;  // 2 No products: the last lands in out
      ++k;
      KR_LAUNCH(ctx, k_mode_sq64, grid, 256, 0, src, dst, P, Ro[m], Q, (const double*)V64[m], pass == 0 ? 1 : 0);
      src = dst;
      P *= Ro[m];
    }
    if (pass == 0) {
      Diag64 dd = {};
      dd.No = No;
      dd.wp = wp;
      for (int m = 0; m < No; ++m) {
        dd.R[m] = Ro[m];
        dd.s[m] = s64[m];
      }
      KR_LAUNCH(ctx, k_diag_w64, grid, 256, 0, const_cast<double*>(src), tot, Rne, dd, w);
    }
  }
  return KR_OK;
}

// The other modes' FP32 eigenvalue arrays sigma^2 (for the penalty w on the device).
struct SigMax {
  int n;
  int R[KR_MAX_MODES];
  const float* s[KR_MAX_MODES];
};

// *w = (1 + 12/eps) prod_k max_i s[k][i]: the host formula, in the same order and precision
// (FP32 maxima from 0, FP64 products), so the graph sweep's w is bit-identical.
__global__ void k_penalty_w(SigMax sm, double eps, double* __restrict__ w) {
  if (threadIdx.x != 0) return;
  double v = 1.0 + 12.0 / eps;
  for (int k = 0; k < sm.n; ++k) {
    float mxv = 0.f;
    for (int i = 0; i < sm.R[k]; ++i) mxv = sm.s[k][i] > mxv ? sm.s[k][i] : mxv;
    v *= (double)mxv;
  }
  *w = v;
}

struct FactorStep {
  int n;
  int No;
  int Rn;
  int64_t Rne;
  int In;
};

}  // namespace

// One Alg. 3 factor update of mode n (A[n] overwritten). Returns the iteration count.
kr_status kr_factor_step(kr_ctx* ctx, const Modes& m, const float* X, const float* G, int n, const SolveCfg& cfg,
                         uint64_t seed, uint64_t call_id, float* An_out, kr_report* rep) {
  const int N = m.N;
  const int No = N - 1;
  const int Rn = m.R[n], In = m.I[n];
  Modes mo;
  mo.N = No;
  int64_t Rne = 1, Pafter = 1;
  for (int k = 0, j = 0; k < N; ++k) {
    if (k == n) continue;
    mo.I[j] = m.I[k];
    mo.R[j] = m.R[k];
    mo.A[j] = m.A[k];
    Rne *= m.R[k];
    ++j;
  }
  for (int k = n + 1; k < N; ++k) Pafter *= m.I[k];
  if (Rn > Rne)
    return kr_fail(ctx, KR_EINVAL, "factor step %d: R_n=%d exceeds prod of the other ranks (%lld): G_(n) cannot have full row rank",
                   n, Rn, (long long)Rne);
  if (Rne > 24576)
    return kr_fail(ctx, KR_ENOTIMPL, "factor step %d: prod of the other ranks %lld > 24576", n, (long long)Rne);
  KR_TRY(kr_sketch_check(ctx, mo, cfg.s * In));
  kr_sketch sk;
  kr_sketch_setup_rows(&sk, mo, cfg.s, In, In, Pafter);
  const int RT = mo.R[No - 1];
  const int64_t cells = sk.ncell;
  // two other modes: the sampled products of every row by the fused slab pass (each row is
  // its own group of slabs, its z block the slab's X1), else the per-cell pass between two
  // batched mode products
  const bool slab = ctx->slab_pass && No == 2 && kr_slab_eligible(ctx, mo, &sk, true);
  kr_tiles tl;
  if (slab) kr_tiles_setup(ctx, mo, &sk, &tl);
  // largest batched intermediate: forward (In, I_o..., R_T) or the precond (In, Rne); also Rn x Rne batches
  int64_t mx = (int64_t)In * Rne;
  {
    int64_t cur = (int64_t)In * Rne;
    for (int k = 0; k < No - 1; ++k) {
      cur = cur / mo.R[k] * mo.I[k];
      if (cur > mx) mx = cur;
    }
  }
  if ((int64_t)Rn * Rne > mx) mx = (int64_t)Rn * Rne;
  Modes mg;  // G_(n)^T as a one-mode "factor" for its Gram / Cholesky / inverse
  mg.N = 1;
  mg.I[0] = (int)Rne;
  mg.R[0] = Rn;
  Need nd;
  kr_tables_need(m, true, nd);
  kr_tables_need(mg, false, nd);
  kr_sketch_own_need(&sk, nd);
  const int64_t ZL = (int64_t)In * Rne;
  for (int k = 0; k < 5; ++k) nd.add<float>(ZL);      // Z, Gb, Gr, D, spare
  nd.add<float>(cells * RT);                          // Y
  nd.add<float>(cells * RT);                          // W
  nd.add<float>(mx);                                  // t0
  nd.add<float>(mx);                                  // t1
  for (int k = 0; k < 3; ++k) nd.add<float>((int64_t)In * Rn);  // U1, U2, S3
  for (int k = 0; k < 6; ++k) nd.add<float>((int64_t)Rn * Rne);  // Gn, Gt, Gp, GpT, Vw, AinvUt
  nd.add<double>((int64_t)Rn * Rn);                   // Hinv (FP64)
  nd.add<double>((int64_t)Rn * Rne);                  // G+ (FP64)
  nd.add<double>((int64_t)Rn * Rn);                   // C
  nd.add<float>((int64_t)Rn * Rn);                    // Cinv
  nd.add<double>(3 * (int64_t)In + 8);                // row stats, reductions
  nd.add<double>(2 * (int64_t)In);                    // per-row q and penalty terms (eps rule)
  nd.add<int>(8);
  nd.add<double>(1024);                               // resid partials
  nd.add<FactorLoop>(1);                              // stopping-rule state
  // one or two other modes: the gradient, the FP64 Woodbury preconditioner and the update
  // of every row in one kernel (k_factor_rows); more: the batched FP32 mode-product chain
  const bool fused_rows = No <= 2 && Rne <= FR_MAX_RNE && Rn <= PEN_MAXRN;
  nd.add<double>((int64_t)Rn * Rne);  // A^-1 U
  nd.add<double>((int64_t)Rn * Rne);  // V
  nd.add<double>((int64_t)Rn * Rn);   // C^-1
  if (!fused_rows) {
    nd.add<double>((int64_t)Rn * Rne);  // (G+)^T
    for (int k = 0; k < 3; ++k) nd.add<double>(ZL);  // gradient, A^-1 gradient, scratch (FP64 chain)
  }
  if (slab) kr_tiles_own_need(&tl, cells, nd);
  {
    Need sc = nd;  // the tile construction reuses the sketch build's scratch
    kr_sketch_scratch_need(ctx, sk.s, cells, sk.IT, nd);
    if (slab) {
      kr_tiles_scratch_need(&tl, cells, sc);
      if (sc.off > nd.off) nd.off = sc.off;
    }
  }
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  // inside a captured sweep (ctx->gm.on) nothing is read back: rank and capacitance checks
  // go to the device error word, the penalty w is computed on the device, and the loop is a
  // conditional node of the sweep's graph
  const bool gm = ctx->gm.on;
  Carve cv(ctx->ws, ctx->ws_size);
  FactorTables ta;
  KR_TRY(kr_tables_build(ctx, m, true, cv, ta, !gm));
  if (gm) KR_TRY(kr_gm_flags(ctx, ta.flags, N, KR_GM_FACTOR_RANK));
  FactorTables to;  // the other modes' tables
  to.N = No;
  for (int k = 0, j = 0; k < N; ++k) {
    if (k == n) continue;
    to.I[j] = ta.I[k];
    to.R[j] = ta.R[k];
    to.thr[j] = ta.thr[k];
    to.invp[j] = ta.invp[k];
    to.prob[j] = ta.prob[k];
    to.V[j] = ta.V[k];
    to.sig2[j] = ta.sig2[k];
    to.ginv[j] = ta.ginv[k];
    ++j;
  }
  // G_(n), its transpose, and G+ = G_(n)^T (G_(n) G_(n)^T)^-1
  float* Gn = cv.take<float>((int64_t)Rn * Rne);
  float* Gt = cv.take<float>((int64_t)Rn * Rne);
  float* Gp = cv.take<float>((int64_t)Rn * Rne);
  float* GpT = cv.take<float>((int64_t)Rn * Rne);
  float* Vw = cv.take<float>((int64_t)Rn * Rne);
  float* AinvUt = cv.take<float>((int64_t)Rn * Rne);
  Dims dg;
  dg.N = N;
  for (int k = 0; k < N; ++k) dg.R[k] = m.R[k];
  const int64_t Rtot = Rne * Rn;
  KR_LAUNCH(ctx, k_unfold, grid_of(ctx, Rtot), 256, 0, G, dg, n, Rtot, (int)Rne, Gn, Gt);
  mg.A[0] = Gt;
  FactorTables tg;
  {
    kr_status st = kr_tables_build(ctx, mg, false, cv, tg, !gm);
    if (st == KR_ERANK) return kr_fail(ctx, KR_ERANK, "factor step %d: the core unfolding G_(n) is rank deficient", n);
    KR_TRY(st);
    if (gm) KR_TRY(kr_gm_flags(ctx, tg.flags, 1, KR_GM_CORE_UNFOLD_RANK));
  }
  KR_TRY(kr_smem_attr(ctx, k_penalty_rows, sizeof(double) * Rne));
  // G+ = G_(n)^T (G_(n) G_(n)^T)^-1 in FP64 (and FP32 for the preconditioner)
  double* hinv = cv.take<double>((int64_t)Rn * Rn);
  double* gp64 = cv.take<double>((int64_t)Rn * Rne);
  KR_LAUNCH(ctx, k_hinv, 1, 256, 0, tg.linv[0], Rn, hinv);
  KR_LAUNCH(ctx, k_gp64, grid_of(ctx, Rtot), 256, 0, Gt, hinv, Rn, Rne, gp64, Gp);
  // w = (1 + 12/eps) prod_{m != n} sigma_max^2 (eigenvalues of the other Gram matrices)
  double w = 1.0 + 12.0 / cfg.eps;
  const double* wdev = nullptr;
  if (gm) {
    if (ctx->gm.wslot >= ctx->gm.nw) return kr_fail(ctx, KR_EINVAL, "graph sweep: more factor steps than penalty slots");
    double* wd = ctx->gm.w + ctx->gm.wslot++;
    SigMax sm = {};
    sm.n = No;
    for (int k = 0; k < No; ++k) {
      sm.s[k] = to.sig2[k];
      sm.R[k] = to.R[k];
    }
    KR_LAUNCH(ctx, k_penalty_w, 1, 32, 0, sm, cfg.eps, wd);
    wdev = wd;
  } else {
    float* hs = (float*)ctx->hbuf;
    for (int k = 0; k < No; ++k)
      KR_CUDA(ctx, cudaMemcpyAsync(hs + 64 * k, to.sig2[k], sizeof(float) * to.R[k], cudaMemcpyDeviceToHost, ctx->stream));
    KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < No; ++k) {
      float mxv = 0.f;
      const float* hsk = (const float*)ctx->hbuf + 64 * k;
      for (int i = 0; i < to.R[k]; ++i) mxv = hsk[i] > mxv ? hsk[i] : mxv;
      w *= (double)mxv;
    }
  }
  const float wf = (float)w, lf = (float)cfg.lambda;
  KR_LAUNCH(ctx, k_vw, grid_of(ctx, Rtot), 256, 0, Gp, Gn, Rn, (int)Rne, lf, wf, Vw, GpT, wdev);
  // iteration buffers
  kr_sketch_layout(&sk, cv);
  float* Z = cv.take<float>(ZL);
  float* Gb = cv.take<float>(ZL);
  float* Gr = cv.take<float>(ZL);
  float* D = cv.take<float>(ZL);
  float* spare = cv.take<float>(ZL);  // keeps the layout of the size accounting
  float* Y = cv.take<float>(cells * RT);
  float* W = cv.take<float>(cells * RT);
  float* t0 = cv.take<float>(mx);
  float* t1 = cv.take<float>(mx);
  float* U1 = cv.take<float>((int64_t)In * Rn);
  float* U2 = cv.take<float>((int64_t)In * Rn);
  float* S3 = cv.take<float>((int64_t)In * Rn);  // keeps the layout of the size accounting
  (void)S3;
  double* C = cv.take<double>((int64_t)Rn * Rn);
  float* Cinv = cv.take<float>((int64_t)Rn * Rn);
  double* rowstat = cv.take<double>(3 * (int64_t)In + 8);
  double* roweps = cv.take<double>(2 * (int64_t)In);
  double* red = rowstat + 3 * (int64_t)In;
  int* flag = cv.take<int>(8);
  double* rpart = cv.take<double>(1024);
  FactorLoop* dloop = cv.take<FactorLoop>(1);
  RowStep rs = {};
  double* V64[KR_MAX_MODES] = {};
  double* s64[KR_MAX_MODES] = {};
  double *AinvU64 = nullptr, *Vw64 = nullptr, *Cinv64 = nullptr;
  double *GpT64 = nullptr, *G64 = nullptr, *D64 = nullptr, *T64 = nullptr;
  AinvU64 = cv.take<double>((int64_t)Rn * Rne);
  Vw64 = cv.take<double>((int64_t)Rn * Rne);
  Cinv64 = cv.take<double>((int64_t)Rn * Rn);
  if (!fused_rows) {
    GpT64 = cv.take<double>((int64_t)Rn * Rne);
    G64 = cv.take<double>(ZL);
    D64 = cv.take<double>(ZL);
    T64 = cv.take<double>(ZL);
  }
  // the other modes' FP64 eigen-decompositions (built with the tables): the Woodbury base
  int Ro[KR_MAX_MODES];
  for (int k = 0, j = 0; k < N; ++k) {
    if (k == n) continue;
    Ro[j] = m.R[k];
    V64[j] = ta.V64[k];
    s64[j] = ta.sig64[k];
    ++j;
  }
  if (slab) kr_tiles_layout(&tl, cells, cv);
  (void)spare;
  // The (1+eps)-aware rule (kr_opts.stop_rule 1) for the rows: on the slab path (each row
  // its own slab, whose tiles give the row's sampled objective) with the fused row kernel
  // (which forms q and the penalty terms); otherwise the relative-step rule.
  const bool eps_rows = cfg.stop_rule == 1 && slab && fused_rows;
  const size_t fr_smem = (size_t)(eps_rows ? 32 : 24) * Rne;
  RowsEps reps = {};
  if (eps_rows) {
    const double se = sqrt(cfg.eps), c1 = 1.0 - se;
    const double rho = fmax(fabs(1.0 - cfg.alpha * (1.0 - se)), fabs(1.0 - cfg.alpha * (1.0 + se)));
    reps.on = 1;
    reps.q = roweps;
    reps.pen = roweps + In;
    reps.objpart = tl.objpart;
    reps.tstart = tl.tstart;
    reps.rho2_c1 = rho * rho / c1;
    reps.inv_c1 = 1.0 / c1;
    reps.theta_eps = cfg.theta * cfg.eps;
  }
  const size_t gj_smem = (size_t)Rn * 2 * Rn * sizeof(double);
  KR_TRY(kr_smem_attr(ctx, k_gauss_jordan, gj_smem));
  if (fused_rows) {
    // FP64 Woodbury pieces: A^-1 U, V, the capacitance and its inverse
    rs.b.R1 = No == 2 ? Ro[0] : 1;
    rs.b.R2 = Ro[No - 1];
    rs.b.V1 = No == 2 ? V64[0] : nullptr;
    rs.b.V2 = V64[No - 1];
    rs.b.s1 = No == 2 ? s64[0] : nullptr;
    rs.b.s2 = s64[No - 1];
    rs.b.w = w;
    rs.b.wp = wdev;
    rs.Rn = Rn;
    rs.Rne = (int)Rne;
    rs.Gn = Gn;
    rs.gp64 = gp64;
    rs.Vw = Vw64;
    rs.AinvU = AinvU64;
    rs.Cinv = Cinv64;
    rs.lambda = cfg.lambda;
    rs.w = w;
    rs.wp = wdev;
    rs.alpha = cfg.alpha;
    KR_LAUNCH(ctx, k_vw64, grid_of(ctx, Rtot), 256, 0, gp64, Gn, Rn, (int)Rne, cfg.lambda, w, Vw64, wdev);
    KR_TRY(kr_smem_attr(ctx, k_base_cols64, (size_t)16 * Rne));
    KR_LAUNCH(ctx, k_base_cols64, Rn, 256, (size_t)16 * Rne, rs.b, gp64, Rn, (int)Rne, AinvU64);
    KR_LAUNCH(ctx, k_capacitance64, Rn * Rn, 256, 0, Vw64, AinvU64, Rn, (int)Rne, C);
    KR_LAUNCH(ctx, k_gauss_jordan, 1, 256, gj_smem, C, Rn, Cinv, flag, Cinv64);
    if (gm) KR_TRY(kr_gm_flags(ctx, flag, 1, KR_GM_CAPACITANCE));
    if (eps_rows) {
      rs.rowq = roweps;
      rs.rowpen = roweps + In;
    }
    KR_TRY(kr_smem_attr(ctx, k_factor_rows, fr_smem));
  } else {
    // FP64 chain: A^-1 U (A^-1 applied to each column of G+, batched), V, the capacitance
    // and its inverse
    KR_LAUNCH(ctx, k_transpose64, grid_of(ctx, Rtot), 256, 0, (const double*)gp64, (int)Rne, Rn, GpT64);
    KR_TRY(base_apply64(ctx, No, Ro, V64, s64, Rn, w, GpT64, AinvU64, T64, wdev));
    KR_LAUNCH(ctx, k_vw64, grid_of(ctx, Rtot), 256, 0, gp64, Gn, Rn, (int)Rne, cfg.lambda, w, Vw64, wdev);
    KR_LAUNCH(ctx, k_capacitance64, Rn * Rn, 256, 0, Vw64, AinvU64, Rn, (int)Rne, C);
    KR_LAUNCH(ctx, k_gauss_jordan, 1, 256, gj_smem, C, Rn, Cinv, flag, Cinv64);
    if (gm) KR_TRY(kr_gm_flags(ctx, flag, 1, KR_GM_CAPACITANCE));
  }
  // batched sketch: row i of X_(n), fresh draws per row (counter row = i)
  {
    Carve sc = cv;
    KR_TRY(kr_sketch_fill(ctx, mo, to, X, seed, call_id, 0, &sk, sc, gm));
  }
  if (slab) KR_TRY(kr_tiles_build(ctx, &sk, &tl, cv));
  KR_CUDA(ctx, cudaMemsetAsync(Z, 0, sizeof(float) * ZL, ctx->stream));
  // mode-product plans over the batch axis
  int dfw_in[KR_MAX_MODES], dfw_out[KR_MAX_MODES], trf[KR_MAX_MODES], trb[KR_MAX_MODES];
  const float* Bf[KR_MAX_MODES];
  dfw_in[0] = dfw_out[0] = In;
  Bf[0] = nullptr;
  trf[0] = trb[0] = 0;
  for (int k = 0; k < No; ++k) {
    dfw_in[k + 1] = mo.R[k];
    dfw_out[k + 1] = (k < No - 1) ? mo.I[k] : mo.R[k];
    Bf[k + 1] = (k < No - 1) ? mo.A[k] : nullptr;
    trf[k + 1] = 0;
    trb[k + 1] = 1;
  }
  const int nblk = kr_resid_blocks(ctx);
  FactorLoop* hl = reinterpret_cast<FactorLoop*>(ctx->hbuf);
  int* hflag = reinterpret_cast<int*>(static_cast<char*>(ctx->hbuf) + 512);
  KR_LAUNCH(ctx, k_factor_loop_init, 1, 1, 0, dloop);
  // One Richardson iteration of every row, then the stopping rule on the device (inside
  // the graph it also sets the loop condition).
  bool z_zero = false;  // z is zero (the first iteration from the host)
  auto one_iter = [&](cudaGraphConditionalHandle hnd, int use_hnd) -> kr_status {
    int used = 0;
    // sampled part: Gb = K~^T Omega (b~ - K~ z) per row
    if (slab) {
      KR_TRY(kr_slab_pass(ctx, &sk, &tl, mo.A[0], mo.A[1], Z, eps_rows, false, 0, z_zero ? KR_SLAB_ZERO_X : 0));
      KR_TRY(kr_tile_reduce(ctx, &tl, nullptr, Gb));
    } else {
      KR_TRY(kr_kron_apply2(ctx, No + 1, dfw_in, dfw_out, Bf, trf, Z, Y, t0, t1));
      KR_TRY(kr_sketch_resid(ctx, &sk, mo.A[No - 1], RT, Y, W, rpart, nblk, &used));
      KR_TRY(kr_kron_apply2(ctx, No + 1, dfw_out, dfw_in, Bf, trb, W, Gb, t0, t1));
    }
    if (fused_rows) {
      KR_LAUNCH(ctx, k_factor_rows, In, 256, fr_smem, rs, Z, Gb, rowstat);
    } else {
      // grad = w z + G+ (lambda (G+)^T z - w G z) - Gb  (FP64, one block per row)
      KR_LAUNCH(ctx, k_penalty_rows, In, 256, sizeof(double) * Rne, Z, Gn, gp64, Gb, Rn, (int)Rne, cfg.lambda, w,
                (float*)nullptr, (float*)nullptr, G64, wdev);
      // d = M^-1 grad (Woodbury, FP64), z <- z - alpha d
      KR_TRY(base_apply64(ctx, No, Ro, V64, s64, In, w, G64, D64, T64, wdev));
      KR_LAUNCH(ctx, k_wb_rows64, In, 256, 0, (const double*)D64, (const double*)Vw64, (const double*)Cinv64,
                (const double*)AinvU64, Rn, (int)Rne, Z, (float)cfg.alpha, rowstat);
    }
    // stopping rule on the largest per-row relative step
    KR_LAUNCH(ctx, k_rows_reduce, 1, 256, 0, rowstat, In, red, dloop, cfg.tol, cfg.max_iter, hnd, use_hnd, reps);
    return KR_OK;
  };
  auto read_state = [&]() -> kr_status {
    KR_CUDA(ctx, cudaMemcpyAsync(hl, dloop, sizeof(FactorLoop), cudaMemcpyDeviceToHost, ctx->stream));
    KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return KR_OK;
  };
  if (gm) {
    // the first iteration (z = 0) ahead of the WHILE node, as the host loop runs it, its check
    // setting the node's condition; the rest inside the node; then the new factor rows
    // a_i = (G+)^T z_i
    cudaGraphConditionalHandle h = 0;
    int64_t pb = 0;
    KR_TRY(kr_gm_handle(ctx, 0, &h));
    z_zero = true;
    const kr_status s1 = one_iter(h, 1);
    z_zero = false;
    KR_TRY(s1);
    KR_TRY(kr_capture_while(ctx, h, one_iter, &pb));
    KR_TRY(kr_gm_status(ctx, &dloop->status, &dloop->it, pb, -1, nullptr));
    KR_LAUNCH(ctx, k_penalty_rows, In, 256, sizeof(double) * Rne, Z, Gn, gp64, Gb, Rn, (int)Rne, cfg.lambda, w, Gr,
              An_out, (double*)nullptr, wdev);
    return KR_OK;
  }
  // The first iteration runs from the host (with the capacitance check; z = 0, so the
  // slab pass skips its forward product); iterations 2.. as one graph (KR_OPT_DEVICE_LOOP)
  // or from the host.
  z_zero = true;
  const kr_status st1 = one_iter(0, 0);
  z_zero = false;
  KR_TRY(st1);
  KR_CUDA(ctx, cudaMemcpyAsync(hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KR_TRY(read_state());
  if (*hflag != 0) return kr_fail(ctx, KR_ERANK, "factor step %d: the Woodbury capacitance matrix is singular", n);
  if (hl->status == STEP_CONTINUE && ctx->device_loop && !ctx->timing) {
    int64_t per_step = 0;
    const int it0 = hl->it;
    if (kr_graph_while(ctx, one_iter, &per_step)) {
      KR_TRY(read_state());
      ctx->launches += per_step * (hl->it - it0);
    }
  }
  while (hl->status == STEP_CONTINUE) {
    KR_TRY(one_iter(0, 0));
    KR_TRY(read_state());
  }
  const int it = hl->it;
  const double rel = hl->rel;
  const int converged = hl->status == STEP_CONVERGED ? 1 : hl->status == STEP_FLOOR ? 2 : hl->status == STEP_EPS ? 3 : 0;
  kr_status st = KR_OK;
  if (hl->status == STEP_NONFINITE)
    st = kr_fail(ctx, KR_ENONFINITE, "factor step %d: iterate became non-finite at iteration %d", n, it);
  if (hl->status == STEP_DIVERGED)
    st = kr_fail(ctx, KR_EDIVERGED, "factor step %d: Richardson step grew 3 times past 16x its minimum", n);
  // a_i = (G+)^T z_i  (the new factor rows, FP64 accumulation)
  KR_LAUNCH(ctx, k_penalty_rows, In, 256, sizeof(double) * Rne, Z, Gn, gp64, Gb, Rn, (int)Rne, cfg.lambda, w, Gr,
            An_out, (double*)nullptr, wdev);
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rep) {
    rep->iters = it;
    rep->converged = converged;
    rep->s = cfg.s;
    rep->distinct = sk.distinct;
    rep->rel_update = rel;
  }
  if (st != KR_OK) return st;
  if (!converged) return kr_fail(ctx, KR_ENOTCONV, "factor step %d: no convergence in %d iterations", n, cfg.max_iter);
  return KR_OK;
}

namespace {

kr_status tucker_args(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X, float* const A[],
                      const float* G, const kr_opts* o, Modes* m) {
  if (!o || !I || !R || !X || !A || !G) return kr_fail(ctx, KR_EINVAL, "tucker: null argument");
  if (N < 2 || N > KR_MAX_MODES) return kr_fail(ctx, KR_EINVAL, "tucker: N=%d outside [2,%d]", N, KR_MAX_MODES);
  if (!(o->eps > 0.0 && o->eps < 1.0)) return kr_fail(ctx, KR_EINVAL, "tucker: eps outside (0,1)");
  if (o->precision < 0 || o->precision > 2)
    return kr_fail(ctx, KR_EINVAL, "tucker: precision=%d (0 FP32, 1 BF16, 2 FP8 e4m3)", o->precision);
  if (!(o->lambda >= 0.0) || !isfinite(o->lambda)) return kr_fail(ctx, KR_EINVAL, "tucker: lambda must be >= 0");
  if (o->host_io) return kr_fail(ctx, KR_ENOTIMPL, "tucker: host_io is not supported; pass device pointers");
  kr_factors f = {};
  f.N = N;
  for (int n = 0; n < N; ++n) {
    f.I[n] = I[n];
    f.R[n] = R[n];
    f.A[n] = A[n];
  }
  return kr_check_factors(ctx, &f, m);
}

SolveCfg cfg_from(const kr_opts* o, int64_t Rsz) {
  SolveCfg c;
  c.lambda = o->lambda;
  c.eps = o->eps;
  c.alpha = o->step > 0 ? o->step : 1.0 - sqrt(o->eps);
  c.tol = o->tol > 0 ? o->tol : 1e-7;
  c.max_iter = o->max_iter > 0 ? o->max_iter : 100;
  c.s = o->num_samples > 0 ? o->num_samples : kr_sample_count(Rsz, o->eps, o->sample_scale);
  c.stop_rule = o->stop_rule == 1 ? 1 : 0;  // used by the core steps (Alg. 2 solves)
  c.theta = o->theta > 0 ? o->theta : 0.01;
  c.prec = o->precision;  // the core steps' slab passes (the factor steps run FP32)
  return c;
}

}  // namespace

extern "C" kr_status tucker_factor_update(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X,
                                          float* const A[], const float* G, int32_t n, const kr_opts* opts,
                                          kr_report* report) {
  if (!ctx) return KR_EINVAL;
  Modes m;
  KR_TRY(tucker_args(ctx, N, I, R, X, A, G, opts, &m));
  if (n < 0 || n >= N) return kr_fail(ctx, KR_EINVAL, "tucker_factor_update: mode %d outside [0,%d)", n, N);
  int64_t Rne = 1;
  for (int k = 0; k < N; ++k)
    if (k != n) Rne *= R[k];
  SolveCfg cfg = cfg_from(opts, Rne);
  if (report) *report = kr_report{};
  return kr_factor_step(ctx, m, X, G, n, cfg, opts->seed, opts->call_id, A[n], report);
}

namespace {

// Sweeps k0..k1-1 of the sampled TuckerALS captured into ONE CUDA graph (ctx->gm.on while
// capturing): the factor steps' and core steps' Richardson loops become conditional WHILE
// nodes, their checks device words. *ran is false when the graph could not be built or
// launched (nothing ran; ctx->err says why and the caller continues from the host).
kr_status graph_sweeps(kr_ctx* ctx, const Modes& m, const float* X, float* G, const kr_opts* opts, int k0, int k1,
                       const std::function<kr_status(int, int)>& step, kr_report* r, int* total_iters, bool* ran) {
  *ran = false;
  const int N = m.N;
  const int nloops = (k1 - k0) * (N + 2);  // a core step's loop and its FP32 refinement
  const int nw = (k1 - k0) * N;
  const size_t off_status = 16, off_w = off_status + 8 * (size_t)nloops, off_obj = off_w + 8 * (size_t)nw;
  const size_t off_last = off_obj + 16, off_dist = off_last + ((kr_gm_state_bytes() + 15) / 16) * 16;
  const size_t bytes = off_dist + 16;
  KR_TRY(kr_hbuf_reserve(ctx, 4096 + 8 * (size_t)nloops));
  if (!ctx->side_stream) KR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "tucker_als_sweep: sweeps 2.. ran from the host (no memory for the graph's state)";
    return KR_OK;
  }
  char* b = static_cast<char*>(mem);
  kr_ctx::GraphMode& g = ctx->gm;
  g.mem = mem;
  g.err = reinterpret_cast<int*>(b);
  g.status = reinterpret_cast<int*>(b + off_status);
  g.w = reinterpret_cast<double*>(b + off_w);
  g.obj = reinterpret_cast<double*>(b + off_obj);
  g.last = b + off_last;
  g.distinct = reinterpret_cast<unsigned long long*>(b + off_dist);
  g.nstatus = nloops;
  g.nw = nw;
  g.slot = g.wslot = 0;
  g.body_launches.clear();
  g.base_slot.clear();
  g.owner.clear();
  auto release = [&]() {
    cudaFree(g.mem);
    g = kr_ctx::GraphMode();
  };
  {
    const cudaError_t e = cudaMemsetAsync(mem, 0, bytes, ctx->stream);
    if (e != cudaSuccess) {
      release();
      return kr_fail_cuda(ctx, e, "graph sweep: state reset", __FILE__, __LINE__);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const int64_t l0 = ctx->launches;
  std::string why;
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) why = std::string("begin capture: ") + cudaGetErrorString(e);
  if (why.empty()) {
    g.on = true;
    kr_status cs = KR_OK;
    for (int k = k0; k < k1 && cs == KR_OK; ++k)
      for (int n = 0; n <= N && cs == KR_OK; ++n) {
        g.cur_owner = n < N ? n : -1;
        cs = step(k, n);
      }
    g.on = false;
    if (cs != KR_OK) why = "capture: " + ctx->err;
    e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e != cudaSuccess && why.empty()) why = std::string("end capture: ") + cudaGetErrorString(e);
  }
  if (why.empty() && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
    why = std::string("instantiate: ") + cudaGetErrorString(e);
  if (why.empty() && (e = cudaGraphLaunch(exec, ctx->stream)) != cudaSuccess)
    why = std::string("launch: ") + cudaGetErrorString(e);
  if (!why.empty()) {
    // nothing ran: the captured counter reset did not happen either
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    ctx->launches = l0;
    ctx->dcnt_clean = false;
    cudaStreamSynchronize(ctx->stream);
    release();
    ctx->err = "tucker_als_sweep: sweeps 2.. ran from the host (" + why + ")";
    return KR_OK;
  }
  *ran = true;
  ctx->graphs++;
  e = cudaStreamSynchronize(ctx->stream);
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    release();
    return kr_fail_cuda(ctx, e, "graph sweep: run", __FILE__, __LINE__);
  }
  // the checks: the error word, then every loop's final status (a resumed loop's base is
  // superseded by it), in capture order
  int* h = reinterpret_cast<int*>(ctx->hbuf);
  kr_status st = KR_OK;
  if (cudaMemcpy(h, mem, off_w, cudaMemcpyDeviceToHost) != cudaSuccess) {
    release();
    return kr_fail(ctx, KR_ECUDA, "graph sweep: reading its checks: %s", cudaGetErrorString(cudaGetLastError()));
  }
  const int err = h[0];
  const int* stat = h + off_status / sizeof(int);
  const int nl = g.slot;
  std::vector<char> superseded((size_t)nl, 0);
  for (int i = 0; i < nl; ++i)
    if (g.base_slot[(size_t)i] >= 0) superseded[(size_t)g.base_slot[(size_t)i]] = 1;
  for (int i = 0; i < nl; ++i) {
    const int base = g.base_slot[(size_t)i];
    // a first loop's first iteration ran ahead of its node; a resumed loop's all ran inside
    const int runs = stat[2 * i + 1] - (base >= 0 ? stat[2 * base + 1] : 1);
    ctx->launches += g.body_launches[(size_t)i] * (runs > 0 ? runs : 0);
    if (superseded[(size_t)i]) continue;
    *total_iters += stat[2 * i + 1];
    const int status = stat[2 * i];
    const int who = g.owner[(size_t)i];
    char what[64];
    if (who >= 0) snprintf(what, sizeof(what), "factor step %d", who);
    else snprintf(what, sizeof(what), "core step");
    if (st != KR_OK) continue;
    if (status == STEP_NONFINITE)
      st = kr_fail(ctx, KR_ENONFINITE, "tucker_als_sweep (graph): %s: iterate became non-finite", what);
    else if (status == STEP_DIVERGED)
      st = kr_fail(ctx, KR_EDIVERGED, "tucker_als_sweep (graph): %s: Richardson step diverged", what);
  }
  if (err & KR_GM_FACTOR_RANK)
    st = kr_fail(ctx, KR_ERANK, "tucker_als_sweep (graph): a factor is numerically rank deficient (Cholesky pivot)");
  else if (err & KR_GM_CORE_UNFOLD_RANK)
    st = kr_fail(ctx, KR_ERANK, "tucker_als_sweep (graph): a core unfolding G_(n) is rank deficient");
  else if (err & KR_GM_CAPACITANCE)
    st = kr_fail(ctx, KR_ERANK, "tucker_als_sweep (graph): a Woodbury capacitance matrix is singular");
  if (st == KR_OK) {
    st = kr_gm_core_report(ctx, opts->lambda, r);
    // the last core step's reduced-precision phase, when it had one
    r->iters_reduced = 0;
    for (int i = nl - 1; i >= 0; --i)
      if (g.owner[(size_t)i] < 0) {
        const int base = g.base_slot[(size_t)i];
        if (base >= 0) r->iters_reduced = stat[2 * base + 1];
        break;
      }
    for (int i = 0; i < 6; ++i) r->t_ms[i] = 0.f;  // phases are not timed inside the graph
  }
  (void)X;
  (void)G;
  release();
  return st;
}

}  // namespace

extern "C" kr_status tucker_als_sweep(kr_ctx* ctx, int32_t N, const int64_t* I, const int32_t* R, const float* X,
                                      float* const A[], float* G, const kr_opts* opts, int32_t sweeps,
                                      kr_report* report) {
  if (!ctx) return KR_EINVAL;
  Modes m;
  KR_TRY(tucker_args(ctx, N, I, R, X, A, G, opts, &m));
  if (sweeps < 0) return kr_fail(ctx, KR_EINVAL, "tucker_als_sweep: sweeps < 0");
  if (report) *report = kr_report{};
  cudaEvent_t e0 = ctx->ev[8], e1 = ctx->ev[9];
  KR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
  int total_iters = 0;
  kr_report r = {};
  // step n < N of sweep k: the factor update of mode n; n = N: the core step, Alg. 2 with
  // b = vec X, K = A(1) (x) ... (x) A(N). A step that stops at max_iter does not end the sweep.
  auto step = [&](int k, int n) -> kr_status {
    const uint64_t cid = opts->call_id + (uint64_t)k * (N + 1) + n;
    kr_status st;
    if (n < N) {
      int64_t Rne = 1;
      for (int j = 0; j < N; ++j)
        if (j != n) Rne *= R[j];
      SolveCfg cfg = cfg_from(opts, Rne);
      st = kr_factor_step(ctx, m, X, G, n, cfg, opts->seed, cid, A[n], &r);
    } else {
      SolveCfg cfg = cfg_from(opts, kr_prod_R(m));
      st = kr_solve_device(ctx, m, X, cfg, opts->seed, cid, G, &r);
    }
    if (!ctx->gm.on) total_iters += r.iters;
    return st == KR_ENOTCONV ? KR_OK : st;
  };
  int done = 0;
  if (sweeps > 0) {
    for (int n = 0; n <= N; ++n) KR_TRY(step(0, n));
    done = 1;
  }
  if (sweeps > 1 && ctx->device_loop && !ctx->timing) {
    // sweeps 2.. as one CUDA graph (the first sized every buffer and tuned every shape)
    bool ran = false;
    KR_TRY(graph_sweeps(ctx, m, X, G, opts, 1, sweeps, step, &r, &total_iters, &ran));
    if (ran) done = sweeps;
  }
  for (int k = done; k < sweeps; ++k)
    for (int n = 0; n <= N; ++n) KR_TRY(step(k, n));
  KR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (report) {
    *report = r;
    report->iters = total_iters;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    report->t_ms[7] = ms;
  }
  return KR_OK;
}
