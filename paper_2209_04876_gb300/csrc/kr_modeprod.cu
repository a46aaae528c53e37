// Mode-n products, KronMatMul (Lemma 4.3) and the Kronecker preconditioner of Alg. 2.
//
// One mode product maps a tensor viewed as (P, K, Q) to (P, J, Q):
//   out[p, j, q] = sum_k B[j, k] in[p, k, q]
// i.e. the n-mode product of §2 with P = prod of the leading dimensions and
// Q = prod of the trailing ones. KronMatMul applies one such product per mode
// (the recursion in the proof of Lemma 4.3, unrolled). The preconditioner
// M+ = (V1 (x)...(x) VN) D (V1 (x)...(x) VN)^T of Alg. 2 is N products with V^T, a
// diagonal scaling, and N products with V (square Kronecker mat-vec theorem, App. B);
// for lambda = 0 it is N products with the (A^T A)^-1 factors.
//
// The kernel is an FP32 CUDA-core tiled GEMM over (J) x (P*Q) with the K reduction
// staged through shared memory; FP32 accumulation.
#include "kr_internal.cuh"

namespace {

constexpr int TN = 64, TK = 16;

// Tile: TJ rows of B (output index j) x 64 output columns n = p*Q + q, K staged in
// chunks of 16 through shared memory. Each thread owns (TJ/16) x 4 outputs. The
// (p, q) split of the columns a thread loads and stores is computed once, outside the
// K loop.
template <int TJ>
__global__ void __launch_bounds__(256) k_mode_product(const float* __restrict__ in, float* __restrict__ out, int64_t P,
                                                       int K, int64_t Q, int J, const float* __restrict__ B, int trans) {
  constexpr int RJ = TJ / 16;  // rows per thread
  __shared__ __align__(16) float Bs[TK][TJ + 4];
  __shared__ __align__(16) float Xs[TK][TN + 4];
  kr_pdl_trigger();
  kr_pdl_wait();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int j0 = blockIdx.y * TJ;
  const int64_t n0 = (int64_t)blockIdx.x * TN;
  const int64_t NN = P * Q;
  // input loads: every thread loads column nn = tid % 64 for k rows (tid / 64) + 4 i
  const int ld_nn = threadIdx.x & (TN - 1);
  const int ld_kk = threadIdx.x >> 6;  // 0..3
  int64_t in_base = -1;
  {
    const int64_t n = n0 + ld_nn;
    if (n < NN) {
      const int64_t p = n / Q, q = n - p * Q;
      in_base = p * K * Q + q;
    }
  }
  // output columns of this thread
  int64_t out_base[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t n = n0 + tx * 4 + c;
    out_base[c] = -1;
    if (n < NN) {
      const int64_t p = n / Q, q = n - p * Q;
      out_base[c] = p * (int64_t)J * Q + q;
    }
  }
  float acc[RJ][4];
#pragma unroll
  for (int a = 0; a < RJ; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TJ; e += 256) {
      int kk, jj;
      if (trans) { jj = e % TJ; kk = e / TJ; } else { kk = e % TK; jj = e / TK; }
      const int j = j0 + jj, k = k0 + kk;
      float v = 0.f;
      if (j < J && k < K) v = trans ? B[(int64_t)k * J + j] : B[(int64_t)j * K + k];
      Bs[kk][jj] = v;
    }
#pragma unroll
    for (int i = 0; i < TK / 4; ++i) {
      const int kk = ld_kk + 4 * i;
      const int k = k0 + kk;
      Xs[kk][ld_nn] = (in_base >= 0 && k < K) ? in[in_base + (int64_t)k * Q] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float bj[RJ], xn[4];
      if (RJ == 4) {
        const float4 t = *reinterpret_cast<const float4*>(&Bs[kk][ty * 4]);
        bj[0] = t.x; bj[1] = t.y; bj[2] = t.z; bj[3] = t.w;
      } else {
        const float2 t = *reinterpret_cast<const float2*>(&Bs[kk][ty * 2]);
        bj[0] = t.x; bj[1] = t.y;
      }
      {
        const float4 t = *reinterpret_cast<const float4*>(&Xs[kk][tx * 4]);
        xn[0] = t.x; xn[1] = t.y; xn[2] = t.z; xn[3] = t.w;
      }
#pragma unroll
      for (int a = 0; a < RJ; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(bj[a], xn[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RJ; ++a) {
    const int j = j0 + ty * RJ + a;
    if (j >= J) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (out_base[c] >= 0) out[out_base[c] + (int64_t)j * Q] = acc[a][c];
  }
}

// Register-blocked SGEMM form of the mode product for Q % 4 == 0 (then four consecutive
// output columns n = p*Q + q share p and are contiguous in memory). Tile BM rows of B x
// 128 columns, K staged 32 at a time with the next stage prefetched into registers; each
// thread owns BM/16 rows x 8 columns (columns tx*4..+3 and 64+tx*4..+3, so the quarter-warp
// shared-memory reads are conflict-free), float4 loads of the input and float4 stores.
constexpr int SG_BN = 128, SG_BK = 32;

// Split K: block z covers K rows [z * kchunk, min(K, (z+1) * kchunk)) and writes its
// partial sum to out + z * zstride (zstride = 0 when gridDim.z == 1).
template <int BM>
__global__ void __launch_bounds__(256, 2) k_mode_product_q4(const float* __restrict__ in, float* __restrict__ out,
                                                         int64_t P, int K, int64_t Q, int J, const float* __restrict__ B,
                                                         int trans, int kchunk, int64_t zstride) {
  constexpr int RM = BM / 16;
  __shared__ __align__(16) float Bs[SG_BK][BM + 4];
  __shared__ __align__(16) float Xs[SG_BK][SG_BN + 4];
  kr_pdl_trigger();
  kr_pdl_wait();  // `in` is the previous kernel's output
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int j0 = blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * SG_BN;
  const int64_t NN = P * Q;
  // input: thread loads float4 column group nl = tid % 32 for k rows tid/32 + 8 i
  const int nl = (tid & 31) * 4;
  const int kl = tid >> 5;
  int64_t in_base = -1;
  {
    const int64_t n = n0 + nl;
    if (n < NN) {
      const int64_t p = n / Q, q = n - p * Q;
      in_base = p * K * Q + q;
    }
  }
  const int kend = min(K, (int)(blockIdx.z + 1) * kchunk);
  float4 xr[4];
  constexpr int NB = BM * SG_BK / 256;  // B-tile entries per thread
  // 32-row tiles prefetch the small B tile with the input tile (all loads of a stage in
  // flight together); 64-row tiles have no registers to spare and read it at the store
  constexpr bool PRE_B = BM <= 32;
  float br[PRE_B ? NB : 1];
  auto b_entry = [&](int i, int k0) -> float {
    const int e = tid + 256 * i;
    int jj, kk;
    if (trans) { jj = e % BM; kk = e / BM; } else { kk = e % SG_BK; jj = e / SG_BK; }
    const int j = j0 + jj, k = k0 + kk;
    return (j < J && k < kend) ? (trans ? __ldg(&B[(int64_t)k * J + j]) : __ldg(&B[(int64_t)j * K + k])) : 0.f;
  };
  auto b_slot = [&](int i, int& jj, int& kk) {
    const int e = tid + 256 * i;
    if (trans) { jj = e % BM; kk = e / BM; } else { kk = e % SG_BK; jj = e / SG_BK; }
  };
  auto load_stage = [&](int k0) {  // input tile into registers (prefetch)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + kl + 8 * i;
      xr[i] = (in_base >= 0 && k < kend) ? __ldg(reinterpret_cast<const float4*>(in + in_base + (int64_t)k * Q))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (PRE_B) {
#pragma unroll
      for (int i = 0; i < NB; ++i) br[i] = b_entry(i, k0);
    }
  };
  auto store_stage = [&](int k0) {  // registers -> shared; the B tile from registers or L1/L2
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<float4*>(&Xs[kl + 8 * i][nl]) = xr[i];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      int jj, kk;
      b_slot(i, jj, kk);
      if constexpr (PRE_B) Bs[kk][jj] = br[i];
      else Bs[kk][jj] = b_entry(i, k0);
    }
  };
  float acc[RM][8];
#pragma unroll
  for (int a = 0; a < RM; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  out += (int64_t)blockIdx.z * zstride;
  load_stage(kb);
  for (int k0 = kb; k0 < ke; k0 += SG_BK) {
    store_stage(k0);
    __syncthreads();
    if (k0 + SG_BK < ke) load_stage(k0 + SG_BK);  // in flight during the compute below
#pragma unroll 8
    for (int kk = 0; kk < SG_BK; ++kk) {
      float av[RM], xv[8];
#pragma unroll
      for (int a = 0; a < RM; a += 2) {
        const float2 t = *reinterpret_cast<const float2*>(&Bs[kk][ty * RM + a]);
        av[a] = t.x;
        av[a + 1] = t.y;
      }
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[kk][tx * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[kk][64 + tx * 4]);
      xv[0] = x0.x; xv[1] = x0.y; xv[2] = x0.z; xv[3] = x0.w;
      xv[4] = x1.x; xv[5] = x1.y; xv[6] = x1.z; xv[7] = x1.w;
#pragma unroll
      for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(av[a], xv[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t n = n0 + h * 64 + tx * 4;
    if (n >= NN) continue;
    const int64_t p = n / Q, q = n - p * Q;
    const int64_t ob = p * (int64_t)J * Q + q;
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      const int j = j0 + ty * RM + a;
      if (j >= J) continue;
      *reinterpret_cast<float4*>(out + ob + (int64_t)j * Q) =
          make_float4(acc[a][4 * h + 0], acc[a][4 * h + 1], acc[a][4 * h + 2], acc[a][4 * h + 3]);
    }
  }
}

// out[i] = sum_z part[z * n + i] in increasing z (deterministic split-K reduction).
__global__ void k_splitk_reduce(const float* __restrict__ part, int S, int64_t n, float* __restrict__ out) {
  kr_pdl_trigger();
  kr_pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int z = 0; z < S; ++z) acc += part[(int64_t)z * n + i];
    out[i] = acc;
  }
}

struct DiagArgs {
  int N;
  int R[KR_MAX_MODES];
  const float* sig2[KR_MAX_MODES];
};

// x[r] *= 1 / (prod_n sig2_n[r_n] + lambda)  (pseudo-inverse: 0 where the sum is 0)
__global__ void k_diag_scale(float* __restrict__ x, int64_t total, DiagArgs da, float lambda) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = i;
    float prod = 1.f;
    for (int n = da.N - 1; n >= 0; --n) {
      int r = (int)(rem % da.R[n]);
      rem /= da.R[n];
      prod *= da.sig2[n][r];
    }
    float d = prod + lambda;
    x[i] = d > 0.f ? x[i] / d : 0.f;
  }
}

}  // namespace

kr_status kr_mode_product(kr_ctx* ctx, const float* in, float* out, int64_t P, int K, int64_t Q, int J, const float* B,
                          int trans) {
  const int64_t NN = P * Q;
  if (NN == 0 || J == 0) return KR_OK;
  if (Q == 1 && kr_tc_eligible(ctx, in, P, K, J)) {  // contiguous contraction: tcgen05, 3xTF32
    const kr_status st = kr_gemm_tc(ctx, in, P, K, B, J, trans, out, J);
    if (st != KR_ENOTIMPL) return st;
  }
  const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  if (Q % 4 == 0 && aligned) {
    // 64-row tiles unless they leave SMs idle (then 32-row tiles double the blocks)
    int BM = J <= 32 ? 32 : 64;
    if (BM == 64 && ((NN + SG_BN - 1) / SG_BN) * ((J + 63) / 64) < ctx->num_sms) BM = 32;
    dim3 grid((unsigned)((NN + SG_BN - 1) / SG_BN), (unsigned)((J + BM - 1) / BM), 1);
    // split K when the output alone gives too few blocks to fill the GPU
    int S = 1, kchunk = K;
    const int64_t blocks = (int64_t)grid.x * grid.y;
    const int64_t outn = NN * J;
    if (K >= 4 * SG_BK && blocks < 2 * ctx->num_sms) {
      int64_t want = (2 * ctx->num_sms + blocks - 1) / blocks;
      int64_t maxs = K / SG_BK;
      S = (int)(want < maxs ? want : maxs);
      if ((int64_t)S * outn > (int64_t(1) << 24)) S = (int)((int64_t(1) << 24) / outn);
      if (S < 1) S = 1;
      kchunk = ((K + S - 1) / S + SG_BK - 1) / SG_BK * SG_BK;
      S = (K + kchunk - 1) / kchunk;
    }
    float* dst = out;
    if (S > 1) {
      KR_TRY(kr_split_reserve(ctx, (size_t)S * outn * sizeof(float)));
      dst = ctx->split_buf;
    }
    grid.z = (unsigned)S;
    if (BM == 32)
      KR_LAUNCH_PDL(ctx, k_mode_product_q4<32>, grid, 256, 0, in, dst, P, K, Q, J, B, trans, kchunk, S > 1 ? outn : 0);
    else
      KR_LAUNCH_PDL(ctx, k_mode_product_q4<64>, grid, 256, 0, in, dst, P, K, Q, J, B, trans, kchunk, S > 1 ? outn : 0);
    if (S > 1) {
      int rg = (int)((outn + 255) / 256);
      if (rg > ctx->num_sms * 8) rg = ctx->num_sms * 8;
      KR_LAUNCH_PDL(ctx, k_splitk_reduce, rg, 256, 0, dst, S, outn, out);
    }
    return KR_OK;
  }
  if (J <= 32) {
    dim3 grid((unsigned)((NN + TN - 1) / TN), (unsigned)((J + 31) / 32));
    KR_LAUNCH_PDL(ctx, k_mode_product<32>, grid, 256, 0, in, out, P, K, Q, J, B, trans);
  } else {
    dim3 grid((unsigned)((NN + TN - 1) / TN), (unsigned)((J + 63) / 64));
    KR_LAUNCH_PDL(ctx, k_mode_product<64>, grid, 256, 0, in, out, P, K, Q, J, B, trans);
  }
  return KR_OK;
}

// Applies B_n (dimsOut[n] x dimsIn[n], or its stored transpose) along every mode n
// with B[n] != nullptr. Intermediates alternate between tmp0 and tmp1, the last
// product writes `out`; no product reads and writes the same buffer, so `in` may be
// `out`. tmp0/tmp1 must hold the largest intermediate.
kr_status kr_kron_apply2(kr_ctx* ctx, int N, const int* dimsIn, const int* dimsOut, const float* const* B,
                         const int* trans, const float* in, float* out, float* tmp0, float* tmp1) {
  int cur[KR_MAX_MODES];
  int active = 0;
  int64_t tot = 1;
  for (int n = 0; n < N; ++n) {
    cur[n] = dimsIn[n];
    tot *= dimsIn[n];
    if (B[n]) ++active;
  }
  if (active == 0) {
    if (out != in) KR_CUDA(ctx, cudaMemcpyAsync(out, in, sizeof(float) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
    return KR_OK;
  }
  const float* src = in;
  if (active == 1 && in == out) {
    KR_CUDA(ctx, cudaMemcpyAsync(tmp0, in, sizeof(float) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
    src = tmp0;
  }
  // Mode products commute. When the last mode shrinks and its product qualifies for the
  // tensor cores (contiguous contraction over the whole input), it goes first: the pass over
  // the largest tensor then runs on tcgen05 and every later product sees the reduced tensor.
  int order[KR_MAX_MODES];
  for (int n = 0; n < N; ++n) order[n] = n;
  if (N > 1 && B[N - 1] && dimsOut[N - 1] < dimsIn[N - 1] && kr_tc_eligible(ctx, src, tot / dimsIn[N - 1],
                                                                               dimsIn[N - 1], dimsOut[N - 1])) {
    for (int n = N - 1; n > 0; --n) order[n] = order[n - 1];
    order[0] = N - 1;
  }
  int a = 0;
  for (int o = 0; o < N; ++o) {
    const int n = order[o];
    if (!B[n]) continue;
    int64_t P = 1, Q = 1;
    for (int m = 0; m < n; ++m) P *= cur[m];
    for (int m = n + 1; m < N; ++m) Q *= cur[m];
    float* dst = (a == active - 1) ? out : (src == tmp0 ? tmp1 : tmp0);
    KR_TRY(kr_mode_product(ctx, src, dst, P, cur[n], Q, dimsOut[n], B[n], trans ? trans[n] : 0));
    cur[n] = dimsOut[n];
    src = dst;
    ++a;
  }
  return KR_OK;
}

kr_status kr_kron_apply(kr_ctx* ctx, int N, const int* dimsIn, const int* dimsOut, const float* const* B,
                        const int* trans, const float* in, float* out, float* tmp, int64_t tmp_elems) {
  return kr_kron_apply2(ctx, N, dimsIn, dimsOut, B, trans, in, out, tmp, tmp + tmp_elems);
}

// d = M+ g for Alg. 2's preconditioner built from tables t (tmp0, tmp1: R floats each).
kr_status kr_precond_apply(kr_ctx* ctx, const FactorTables& t, double lambda, const float* g, float* d, float* tmp0,
                           float* tmp1) {
  const int N = t.N;
  int dims[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  int tr[KR_MAX_MODES];
  int64_t R = 1;
  for (int n = 0; n < N; ++n) {
    dims[n] = t.R[n];
    R *= t.R[n];
  }
  if (lambda == 0.0) {
    for (int n = 0; n < N; ++n) {
      B[n] = t.ginv[n];
      tr[n] = 0;
    }
    return kr_kron_apply2(ctx, N, dims, dims, B, tr, g, d, tmp0, tmp1);
  }
  for (int n = 0; n < N; ++n) {
    B[n] = t.V[n];
    tr[n] = 1;  // V^T
  }
  KR_TRY(kr_kron_apply2(ctx, N, dims, dims, B, tr, g, d, tmp0, tmp1));
  DiagArgs da = {};
  da.N = N;
  for (int n = 0; n < N; ++n) {
    da.R[n] = t.R[n];
    da.sig2[n] = t.sig2[n];
  }
  int grid = (int)((R + 255) / 256);
  if (grid > ctx->num_sms * 8) grid = ctx->num_sms * 8;
  KR_LAUNCH(ctx, k_diag_scale, grid, 256, 0, d, R, da, (float)lambda);
  for (int n = 0; n < N; ++n) tr[n] = 0;  // V
  return kr_kron_apply2(ctx, N, dims, dims, B, tr, d, d, tmp0, tmp1);
}

// x[i] /= prod_n sig2_n[r_n] + shift over the trailing dims of t (a leading batch axis is
// allowed: total may be a multiple of prod R).
kr_status kr_diag_scale(kr_ctx* ctx, const FactorTables& t, double shift, float* x, int64_t total) {
  DiagArgs da = {};
  da.N = t.N;
  for (int n = 0; n < t.N; ++n) {
    da.R[n] = t.R[n];
    da.sig2[n] = t.sig2[n];
  }
  int grid = (int)((total + 255) / 256);
  if (grid > ctx->num_sms * 8) grid = ctx->num_sms * 8;
  if (grid < 1) grid = 1;
  KR_LAUNCH(ctx, k_diag_scale, grid, 256, 0, x, total, da, (float)shift);
  return KR_OK;
}

// ------------------------------------------------------------------ C ABI

extern "C" kr_status kron_matmul(kr_ctx* ctx, int32_t N, const int64_t* J, const int64_t* K, const float* const B[],
                                 const int32_t* trans, const float* x, float* y) {
  if (!ctx) return KR_EINVAL;
  if (N < 1 || N > KR_MAX_MODES || !J || !K || !B || !x || !y) return kr_fail(ctx, KR_EINVAL, "kron_matmul: bad arguments");
  int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
  int64_t cur = 1, mx = 1;
  for (int n = 0; n < N; ++n) {
    if (J[n] < 1 || K[n] < 1 || J[n] > (1 << 30) || K[n] > (1 << 30) || !B[n])
      return kr_fail(ctx, KR_EINVAL, "kron_matmul: bad mode %d", n);
    din[n] = (int)K[n];
    dout[n] = (int)J[n];
    tr[n] = trans ? trans[n] : 0;
    cur *= K[n];
  }
  mx = cur;
  for (int n = 0; n < N; ++n) {
    cur = cur / K[n] * J[n];
    if (cur > mx) mx = cur;
  }
  Need nd;
  nd.add<float>(mx);
  nd.add<float>(mx);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  Carve cv(ctx->ws, ctx->ws_size);
  float* t0 = cv.take<float>(mx);
  float* t1 = cv.take<float>(mx);
  KR_TRY(kr_kron_apply2(ctx, N, din, dout, B, tr, x, y, t0, t1));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return kr_tc_check(ctx);
}

extern "C" kr_status kron_precond(kr_ctx* ctx, const kr_factors* f, double lambda, const float* g, float* d) {
  if (!ctx) return KR_EINVAL;
  Modes m;
  KR_TRY(kr_check_factors(ctx, f, &m));
  if (!(lambda >= 0.0) || !g || !d) return kr_fail(ctx, KR_EINVAL, "kron_precond: bad lambda or null vector");
  int64_t R = kr_prod_R(m);
  Need nd;
  kr_tables_need(m, lambda > 0.0, nd);
  nd.add<float>(R);
  nd.add<float>(R);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  Carve cv(ctx->ws, ctx->ws_size);
  FactorTables t;
  KR_TRY(kr_tables_build(ctx, m, lambda > 0.0, cv, t, true));
  float* t0 = cv.take<float>(R);
  float* t1 = cv.take<float>(R);
  KR_TRY(kr_precond_apply(ctx, t, lambda, g, d, t0, t1));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return KR_OK;
}
