// a6-a12: sampled products, Richardson iteration (Alg. 2), final checks, solvers.
//
// One Richardson step of Alg. 2,
//   x <- x - (1 - sqrt(eps)) M+ (K~^T K~ x + lambda x - K~^T b~),
// is evaluated with the sampled products of Thm 4.4 (T = the last mode):
//   Y  = X x_1 A(1) ... x_{N-1} A(N-1)           (cells x R_N, mode products)
//   r_j = omega_j (b~_j - <A(N)[i_j], Y[cell_j]>)  (per distinct sampled row)
//   W[c] = sum_{j in c} r_j A(N)[i_j]             (cells x R_N)
//   g  = W x_1 A(1)^T ... x_{N-1} A(N-1)^T         (= K~^T Omega (b~ - K~ x))
//   x <- x + alpha M+ (g - lambda x)
// The residual is formed per row from b~ in FP32 (explicit-residual form), so the
// iteration itself refines the solution to FP32 working accuracy.
#include <math.h>

#include <atomic>
#include <thread>

#include <vector>

#include "kr_internal.cuh"

namespace {

// ------------------------------------------------------------------ sampled residual

struct ResidArgs {
  const uint32_t* cell_start;
  const uint32_t* cell_nd;
  const uint32_t* ent;
  const float* bt;
  const float* cell_w;
  const float* invpT;
  const uint32_t* perm;  // processing order of the cells (may be null: identity)
  const uint4* desc;     // per processed cell: {cell, start, distinct, weight bits}
  const float* AT;       // IT x RT
  int IT, RT;
  const float* Y;   // ncell x RT
  float* W;         // ncell x RT
  int64_t ncell;
  double* obj_partial;  // gridDim.x
};

// Lanes per cell and columns per lane for a padded R_N.
template <int RTP>
struct ResidShape {
  static constexpr int COLS = RTP >= 8 ? 8 : 4;
  static constexpr int G = RTP / COLS;  // lanes per cell
  static constexpr int CPW = 32 / G;    // cells per warp
  static constexpr int LDA = RTP + 4;   // shared-memory row stride of A_N (floats)
};
constexpr int RESID_D = 4;          // chunks of G rows in flight per lane group
constexpr int RESID_THREADS = 512;  // 16 warps share one copy of A_N in shared memory

// One lane group of G lanes per cell: lane g owns columns [g*COLS, (g+1)*COLS) of Y[c]
// and W[c]. The cell's (entry, b~) stream is read in chunks of G rows, lane g loading row
// g of a chunk (distinct addresses, coalesced within the group); a ring of RESID_D chunks
// per lane keeps RESID_D*G rows in flight. Each row is broadcast to the group with a
// shuffle, its dot product with y is reduced over the group, and the axpy into w reads
// the A_N row from shared memory again. Cells are taken in `perm` order (similar
// distinct-row counts share a warp).
template <int RTP, bool SMEM_A>
__global__ void __launch_bounds__(RESID_THREADS, 2) k_resid(ResidArgs a) {
  using S = ResidShape<RTP>;
  constexpr int COLS = S::COLS, G = S::G, CPW = S::CPW, LDA = S::LDA;
  extern __shared__ float4 sm4[];
  float* sA = reinterpret_cast<float*>(sm4);
  float* sInvp = sA + (SMEM_A ? (size_t)a.IT * LDA : 0);
  const int RT = a.RT;
  if (SMEM_A) {
    for (int e = threadIdx.x; e < a.IT * LDA; e += blockDim.x) {
      int i = e / LDA, r = e - i * LDA;
      sA[e] = r < RT ? a.AT[(int64_t)i * RT + r] : 0.f;
    }
  }
  for (int i = threadIdx.x; i < a.IT; i += blockDim.x) sInvp[i] = a.invpT[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = lane % G, slot = lane / G;
  const int gbase = slot * G;  // first lane of this group
  const int c0col = g * COLS;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  double obj = 0.0;
  // descriptor of this lane group's first cell; the next one is prefetched while the
  // current cell is processed
  uint4 dnext = make_uint4(0u, 0u, 0u, 0u);
  if (gw * CPW + slot < a.ncell) dnext = __ldg(&a.desc[gw * CPW + slot]);
  for (int64_t q0 = gw * CPW; q0 < a.ncell; q0 += warps * CPW) {
    const int64_t q = q0 + slot;
    const bool live = q < a.ncell;
    const uint4 dc = dnext;
    {
      const int64_t qn = q + warps * CPW;
      if (qn < a.ncell) dnext = __ldg(&a.desc[qn]);
    }
    const int64_t c = live ? (int64_t)dc.x : 0;
    const uint32_t n = live ? dc.z : 0u;
    const uint32_t base = live ? dc.y : 0u;
    const float cw = live ? __uint_as_float(dc.w) : 0.f;
    float y[COLS], w[COLS];
    if (live && (RT % 4) == 0 && c0col + COLS <= RT) {
      const float4* yr = reinterpret_cast<const float4*>(a.Y + c * RT + c0col);
#pragma unroll
      for (int v = 0; v < COLS / 4; ++v) {
        const float4 t = __ldg(&yr[v]);
        y[4 * v + 0] = t.x; y[4 * v + 1] = t.y; y[4 * v + 2] = t.z; y[4 * v + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        int r = c0col + k;
        y[k] = (live && r < RT) ? a.Y[c * RT + r] : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < COLS; ++k) w[k] = 0.f;
    float objc = 0.f;
    uint32_t nmax = n;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, off));
    const uint32_t nchunk = (nmax + G - 1) / G;
    uint32_t ring_e[RESID_D];
    float ring_b[RESID_D];
#pragma unroll
    for (int d = 0; d < RESID_D; ++d) {
      const uint32_t j = (uint32_t)d * G + g;
      const bool act = j < n;
      ring_e[d] = act ? __ldg(&a.ent[base + j]) : 0u;
      ring_b[d] = act ? __ldg(&a.bt[base + j]) : 0.f;
    }
    for (uint32_t k0 = 0; k0 < nchunk; k0 += RESID_D) {
#pragma unroll
      for (int d = 0; d < RESID_D; ++d) {
        const uint32_t e_mine = ring_e[d];
        const float b_mine = ring_b[d];
        {  // refill this slot with chunk k0 + d + RESID_D
          const uint32_t j = (k0 + d + RESID_D) * G + g;
          const bool act = j < n;
          ring_e[d] = act ? __ldg(&a.ent[base + j]) : 0u;
          ring_b[d] = act ? __ldg(&a.bt[base + j]) : 0.f;
        }
        if (k0 + d >= nchunk) continue;  // warp-uniform
#pragma unroll
        for (int sidx = 0; sidx < G; ++sidx) {
          const uint32_t e = __shfl_sync(0xffffffffu, e_mine, gbase + sidx);
          const float bj = __shfl_sync(0xffffffffu, b_mine, gbase + sidx);
          const int it = (int)(e & 0xFFFFu);
          float p = 0.f;
          if (SMEM_A) {
            const float4* row = reinterpret_cast<const float4*>(sA + (size_t)it * LDA + c0col);
#pragma unroll
            for (int v = 0; v < COLS / 4; ++v) {
              const float4 t = row[v];
              p = fmaf(t.x, y[4 * v + 0], p);
              p = fmaf(t.y, y[4 * v + 1], p);
              p = fmaf(t.z, y[4 * v + 2], p);
              p = fmaf(t.w, y[4 * v + 3], p);
            }
          } else {
#pragma unroll
            for (int k = 0; k < COLS; ++k) {
              int r = c0col + k;
              if (r < RT) p = fmaf(__ldg(&a.AT[(int64_t)it * RT + r]), y[k], p);
            }
          }
#pragma unroll
          for (int off = G / 2; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
          const float om = (float)(e >> 16) * cw * sInvp[it];  // 0 for rows past the cell (count 0)
          const float res = bj - p;
          const float rr = om * res;
          if (SMEM_A) {
            const float4* row = reinterpret_cast<const float4*>(sA + (size_t)it * LDA + c0col);
#pragma unroll
            for (int v = 0; v < COLS / 4; ++v) {
              const float4 t = row[v];
              w[4 * v + 0] = fmaf(rr, t.x, w[4 * v + 0]);
              w[4 * v + 1] = fmaf(rr, t.y, w[4 * v + 1]);
              w[4 * v + 2] = fmaf(rr, t.z, w[4 * v + 2]);
              w[4 * v + 3] = fmaf(rr, t.w, w[4 * v + 3]);
            }
          } else {
#pragma unroll
            for (int k = 0; k < COLS; ++k) {
              int r = c0col + k;
              if (r < RT) w[k] = fmaf(rr, __ldg(&a.AT[(int64_t)it * RT + r]), w[k]);
            }
          }
          objc = fmaf(rr, res, objc);
        }
      }
    }
    if (live) {
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        int r = c0col + k;
        if (r < RT) a.W[c * RT + r] = w[k];
      }
      if (g == 0) obj += (double)objc;
    }
  }
  // block reduction of the objective partial (FP64)
  __shared__ double red[RESID_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) obj += __shfl_xor_sync(0xffffffffu, obj, off);
  if (lane == 0) red[threadIdx.x >> 5] = obj;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    a.obj_partial[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------ vector kernels

// g <- g - lambda x (the lambda term of the Richardson gradient)
__global__ void k_sub_lambda_x(float* __restrict__ g, const float* __restrict__ x, float lambda, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    g[i] = fmaf(-lambda, x[i], g[i]);
}

// {||step||^2, ||x||^2, non-finite flag, g^T step} of the block's elements, written to
// part[4 * blockIdx.x + 0..3] in FP64. Inside the block the sums are FP32 fixed-order trees
// (per thread, warp shuffles, then one warp over the warp sums): FP64 arithmetic issues at
// a small fraction of the FP32 rate on this part, and a stopping-rule norm needs no more
// than FP32's relative precision (about 1e-6 after the tree). The blocks' partials are
// added in FP64. Called by all threads of a block of at most 1024 threads, once per kernel.
// The fourth sum, g^T step with g the gradient the step was taken from (lambda term
// included), gives q = g^T M+ g = g^T step / alpha for the (1+eps)-aware stopping rule; it
// is zero when the caller passes no gradient.
constexpr int KR_NPART = 4;
__device__ __forceinline__ void step_norms_block(float s1, float s2, float bad, float s3, double* __restrict__ part) {
  __shared__ float red[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    bad = fmaxf(bad, __shfl_xor_sync(0xffffffffu, bad, off));
    s3 += __shfl_xor_sync(0xffffffffu, s3, off);
  }
  if (lane == 0) {
    red[0][w] = s1;
    red[1][w] = s2;
    red[2][w] = bad;
    red[3][w] = s3;
  }
  __syncthreads();
  if (w == 0) {
    float a = lane < nw ? red[0][lane] : 0.f, b = lane < nw ? red[1][lane] : 0.f, c = lane < nw ? red[2][lane] : 0.f;
    float d = lane < nw ? red[3][lane] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      b += __shfl_xor_sync(0xffffffffu, b, off);
      c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, off));
      d += __shfl_xor_sync(0xffffffffu, d, off);
    }
    if (lane == 0) {
      part[KR_NPART * blockIdx.x + 0] = (double)a;
      part[KR_NPART * blockIdx.x + 1] = (double)b;
      part[KR_NPART * blockIdx.x + 2] = (double)c;
      part[KR_NPART * blockIdx.x + 3] = (double)d;
    }
  }
}

// The gradient a step was taken from, for the stopping rule's g^T step: entry e is
// g[e] - lam * x_old[e] (g = nullptr: not wanted).
struct StepGrad {
  const float* g;
  float lam;
};
__device__ __forceinline__ float step_grad(const StepGrad& sg, int64_t e, float xold) {
  return sg.g ? fmaf(-sg.lam, xold, __ldg(sg.g + e)) : 0.f;
}

// x <- x + alpha d, with the step norms (step_norms_block).
__global__ void __launch_bounds__(256) k_update_reduce(float* __restrict__ x, const float* __restrict__ d, float alpha,
                                                       int64_t n, double* __restrict__ part, StepGrad sg) {
  float s1 = 0.f, s2 = 0.f, bad = 0.f, s3 = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float st = alpha * d[i];
    const float xo = x[i];
    const float xn = xo + st;
    x[i] = xn;
    s1 = fmaf(st, st, s1);
    s2 = fmaf(xn, xn, s2);
    s3 = fmaf(step_grad(sg, i, xo), st, s3);
    if (!isfinite(xn)) bad = 1.f;
  }
  step_norms_block(s1, s2, bad, s3, part);
}

// Richardson state on the device: the stopping rule of Alg. 2 is evaluated on the device
// after every step, so a run of iterations needs no host round trip. The rule works on
// squared norms (no FP64 square root on the device; one divide for the ratio):
// ||step|| <= tol ||x||  <=>  h0 <= tol^2 h1, and the step comparisons of the guards
// compare squares. The host takes sqrt(h0 / h1) of the last step for the report.
struct RichState {
  double h[3];  // last {||step||^2, ||x||^2, non-finite flag}
  double prev_h0, min_h0, min_q;  // previous and smallest ||step||^2, smallest h0 / h1
  double f, q;  // last step: sampled objective at x before it, g^T M+ g (eps-aware rule only)
  int grow, since_min, it, status;  // status: StepCheck (0 = continue)
};

// The state fields the rule reads, fetched once per kernel right after its dependency
// wait (only the last block of a step writes the state, at its very end), so the check
// does not wait for them.
struct RichSnap {
  double prev_h0, min_h0, min_q;
  double xx;  // ||x||^2 before this step (the last step's h[1]; 0 before the first)
  int grow, since_min, it;
};
__device__ __forceinline__ RichSnap rich_load(const RichState* st) {
  RichSnap r;
  r.prev_h0 = __ldcg(&st->prev_h0);
  r.min_h0 = __ldcg(&st->min_h0);
  r.min_q = __ldcg(&st->min_q);
  r.xx = __ldcg(&st->h[1]);
  r.grow = __ldcg(&st->grow);
  r.since_min = __ldcg(&st->since_min);
  r.it = __ldcg(&st->it);
  return r;
}

// Stopping-rule arguments handed to the kernel that ends a step.
struct RichArgs {
  RichState* st;
  double tol;
  int max_iter;
  cudaGraphConditionalHandle hnd;
  int use_hnd;
  unsigned int* ticket;  // zero between steps
  // The (1+eps)-aware rule (eps_rule = 1): stop once
  //   rho^2 q / c1 <= theta eps max(f - q / c1, 0)
  // with f = sampled objective at x before the step (sum of `on` FP64 partials at op, plus
  // lambda ||x||^2), q = g^T M+ g = g^T step / alpha, c1 = 1 - sqrt(eps) and rho the
  // contraction factor of the step (Lemma 4.2: the excess after the step is at most
  // rho^2 q / c1, and f - q / c1 bounds the sampled minimum from below).
  int eps_rule;
  double rho2_c1, inv_c1, theta_eps, inv_alpha, lambda;
  const double* op;
  int on;
};

// The rule after one step: the same guards as step_check (converged, diverged: three
// growths in a row past 16x the smallest step, floor: no new smallest step for 8 steps
// with the ratio once within 100 tol), on squares.
__device__ int step_check_sq(const double* h, double tol, RichSnap& r) {
  const double h0 = h[0], h1 = h[1];
  if (h[2] != 0.0 || !isfinite(h0) || !isfinite(h1)) return STEP_NONFINITE;
  const double q = h1 > 0.0 ? h0 / h1 : (h0 == 0.0 ? 0.0 : INFINITY);
  if (q <= tol * tol) return STEP_CONVERGED;
  if (h0 < r.min_h0) {
    r.min_h0 = h0;
    r.since_min = 0;
  } else {
    ++r.since_min;
  }
  if (q < r.min_q) r.min_q = q;
  r.grow = (h0 > r.prev_h0) ? r.grow + 1 : 0;
  r.prev_h0 = h0;
  if (r.grow >= 3 && h0 > 256.0 * r.min_h0) return STEP_DIVERGED;
  if (r.since_min >= 8 && r.min_q <= 1e4 * tol * tol) return STEP_FLOOR;
  return STEP_CONTINUE;
}

// The stopping rule of Alg. 2 after one step, evaluated by the first warp of a block: the
// step's block partials (and, for the eps-aware rule, the objective partials) summed in
// FP64 (strided per lane, then warp shuffles: a fixed order), the rule applied to the state
// (snapshot `snap`, valid in thread 0), the iteration counted (max_iter ends the loop in
// any case) and, inside the graph, the loop condition set.
__device__ void rich_check_block(const double* __restrict__ part, int np, const RichArgs& ra, RichSnap snap) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0, f = 0.0;
  for (int k = lane; k < np; k += 32) {
    a += __ldcg(part + KR_NPART * k + 0);
    b += __ldcg(part + KR_NPART * k + 1);
    c = fmax(c, __ldcg(part + KR_NPART * k + 2));
    d += __ldcg(part + KR_NPART * k + 3);
  }
  if (ra.eps_rule)
    for (int k = lane; k < ra.on; k += 32) f += __ldcg(ra.op + k);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c = fmax(c, __shfl_xor_sync(0xffffffffu, c, off));
    d += __shfl_xor_sync(0xffffffffu, d, off);
    f += __shfl_xor_sync(0xffffffffu, f, off);
  }
  if (lane == 0) {
    RichState* st = ra.st;
    const double h[3] = {a, b, c};
    int status = STEP_CONTINUE;
    double fx = 0.0, q = 0.0;
    if (ra.eps_rule) {
      fx = f + ra.lambda * snap.xx;
      q = d * ra.inv_alpha;
      if (h[2] == 0.0 && isfinite(fx) && isfinite(q) && ra.rho2_c1 * q <= ra.theta_eps * fmax(fx - q * ra.inv_c1, 0.0))
        status = STEP_EPS;
    }
    if (status == STEP_CONTINUE) status = step_check_sq(h, ra.tol, snap);
    snap.it += 1;
    if (status == STEP_CONTINUE && snap.it >= ra.max_iter) status = STEP_MAXITER;
    st->h[0] = h[0];
    st->h[1] = h[1];
    st->h[2] = h[2];
    st->prev_h0 = snap.prev_h0;
    st->min_h0 = snap.min_h0;
    st->min_q = snap.min_q;
    st->f = fx;
    st->q = q;
    st->grow = snap.grow;
    st->since_min = snap.since_min;
    st->it = snap.it;
    st->status = status;
    if (ra.use_hnd) cudaGraphSetConditional(ra.hnd, status == STEP_CONTINUE ? 1u : 0u);
  }
}

// Between the reduced-precision phase and the FP32 refinement: the loop continues from the
// current x with a fresh stall / growth history (the iteration count carries on).
__global__ void k_rich_resume(RichState* st) {
  st->prev_h0 = st->min_h0 = st->min_q = INFINITY;
  st->grow = st->since_min = 0;
  st->status = STEP_CONTINUE;
}

// The refinement's entry inside a captured sweep: unless the first phase stopped at max_iter
// (which bounds both phases), the state is reset as k_rich_resume does and the loop runs.
__global__ void k_rich_resume_dev(RichState* st, cudaGraphConditionalHandle hnd) {
  const bool go = st->status != STEP_MAXITER;
  if (go) {
    st->prev_h0 = st->min_h0 = st->min_q = INFINITY;
    st->grow = st->since_min = 0;
    st->status = STEP_CONTINUE;
  }
  cudaGraphSetConditional(hnd, go ? 1u : 0u);
}

// x = 0 when *status == which (a non-finite first phase restarts the refinement from 0).
__global__ void k_zero_if_status(float* __restrict__ x, int64_t n, const int* __restrict__ status, int which) {
  if (*status != which) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = 0.f;
}

// An asynchronous solve's report, from the final state and objective (one thread). slots:
// the loops' {status, count}; refined: slot 0 was the reduced-precision phase.
__global__ void k_async_report(const RichState* st, const double* obj, const unsigned long long* distinct,
                               const int* err, const int* slots, int refined, double lambda, int64_t s, int prec,
                               kr_dev_report* out) {
  if (threadIdx.x != 0) return;
  kr_dev_report r = {};
  const int stt = st->status;
  r.iters = st->it;
  r.converged = stt == STEP_CONVERGED ? 1 : stt == STEP_FLOOR ? 2 : stt == STEP_EPS ? 3 : 0;
  r.status = *err             ? KR_ERANK
             : r.converged    ? KR_OK
             : stt == STEP_NONFINITE ? KR_ENONFINITE
             : stt == STEP_DIVERGED  ? KR_EDIVERGED
                                     : KR_ENOTCONV;
  r.iters_reduced = refined ? slots[1] : 0;
  r.precision_used = prec;
  r.s = s;
  r.distinct = (int64_t)*distinct;
  r.obj_sampled = obj[0] + lambda * obj[1];
  const double h0 = st->h[0], h1 = st->h[1];
  r.rel_update = h1 > 0.0 ? sqrt(h0) / sqrt(h1) : (h0 == 0.0 ? 0.0 : INFINITY);
  *out = r;
}

__global__ void k_rich_init(RichState* st) {
  st->h[0] = st->h[1] = st->h[2] = 0.0;
  st->prev_h0 = st->min_h0 = st->min_q = INFINITY;
  st->f = st->q = 0.0;
  st->grow = st->since_min = st->it = 0;
  st->status = STEP_CONTINUE;
}

// Sums the step's block partials, applies the stopping rule, counts the iteration (max_iter
// ends the loop in any case) and, inside the graph, sets the loop condition.
__global__ void __launch_bounds__(32) k_rich_check(const double* __restrict__ part, int np, RichArgs ra) {
  kr_pdl_wait();
  RichSnap snap = {};
  if (threadIdx.x == 0) snap = rich_load(ra.st);
  rich_check_block(part, np, ra, snap);
}

// ------------------------------------------------------------------ preconditioned step in FP64
//
// For badly conditioned ridge problems (u32 sqrt(cond(M)) above 1e-3, e.g. the paper's
// synthetic factors with entries 1 + N(0, 1e-6), cond(A^T A) near 1e8) the FP32 application of
// M+ = (V1 (x)...(x) VN) D (V1 (x)...(x) VN)^T loses the spectral approximation Lemma 4.2 needs.
// Then the step applies M+ in FP64 from the FP64 eigenpairs: g - lambda x widened to FP64, the
// N mode products with V^T, the diagonal, the N products with V, and the FP32 update of x
// with the step statistics of step_norms_block. The sampled products stay FP32.
struct Pc64Modes {
  int N;
  int R[KR_MAX_MODES];
  const double* V[KR_MAX_MODES];    // R x R, eigenvectors as columns
  const double* sig[KR_MAX_MODES];  // R eigenvalues
};

__global__ void k_grad64(const float* __restrict__ g, const float* __restrict__ x, float lam, int64_t n,
                         double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)g[i] - (double)lam * (double)x[i];
}

// out[p, j, q] = sum_k B[j, k] in[p, k, q] with B = V (trans = 0) or V^T (trans = 1), V R x R.
__global__ void k_mode64(const double* __restrict__ in, double* __restrict__ out, int64_t P, int R, int64_t Q,
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

// x[r] /= prod_n sig_n[r_n] + lambda (0 where that is 0), FP64.
__global__ void k_diag64(double* __restrict__ x, int64_t total, Pc64Modes pm, double lambda) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = i;
    double prod = 1.0;
    for (int n = pm.N - 1; n >= 0; --n) {
      const int r = (int)(rem % pm.R[n]);
      rem /= pm.R[n];
      prod *= pm.sig[n][r];
    }
    const double d = prod + lambda;
    x[i] = d > 0.0 ? x[i] / d : 0.0;
  }
}

// x <- x + alpha d (d FP64, x FP32) with the step statistics (step_norms_block).
__global__ void __launch_bounds__(256) k_update64(float* __restrict__ x, const double* __restrict__ d, float alpha,
                                                  int64_t n, double* __restrict__ part, StepGrad sg) {
  float s1 = 0.f, s2 = 0.f, bad = 0.f, s3 = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float st = (float)((double)alpha * d[i]);
    const float xo = x[i];
    const float xn = xo + st;
    x[i] = xn;
    s1 = fmaf(st, st, s1);
    s2 = fmaf(xn, xn, s2);
    s3 = fmaf(step_grad(sg, i, xo), st, s3);
    if (!isfinite(xn)) bad = 1.f;
  }
  step_norms_block(s1, s2, bad, s3, part);
}

// ------------------------------------------------------------------ preconditioned step, fused

// The preconditioner of Alg. 2 is a Kronecker product, M+ = B_1 (x) ... (x) B_N
// (B_n = G_n^-1 for lambda = 0; V_n^T, a diagonal, V_n for lambda > 0), so
// d = M+ (g - lambda x) splits into the first mode (mixing the R_1 slabs of the iterate)
// and the other modes (inside one slab of Q = R / R_1 entries). k_pc_mode0 applies the
// first-mode matrix, optionally forming g - lambda x on the way in and the update
// x <- x + alpha d with its norms on the way out; k_pc_slab applies the other modes to one
// slab in shared memory (for lambda > 0: V^T, the diagonal, then V), optionally with the
// update.
struct PcModes {
  int N;
  int R[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];   // per mode: R x R
  const float* B2[KR_MAX_MODES];  // lambda > 0: V applied after the diagonal
  const float* sig2[KR_MAX_MODES];
  int trans;                      // B applied transposed (V^T)
  float lambda;
};

// out[j, q] = sum_k B0'[j, k] (in[k, q] - lambda xl[k, q]); B0' = B0 or B0^T. A block
// takes a panel of PC_TQ columns q: the panel of the input and B0 are staged in shared
// memory. With x != nullptr the result is the step: x <- x + alpha out, norms reduced.
constexpr int PC_TQ = 32;
__global__ void __launch_bounds__(256) k_pc_mode0(const float* __restrict__ in, const float* __restrict__ xl,
                                                  float lambda, const float* __restrict__ B0, int trans, int R0,
                                                  int Q, float* __restrict__ out, float* __restrict__ x,
                                                  float alpha, double* __restrict__ part, StepGrad sg) {
  __shared__ float sB[KR_MAX_RANK * KR_MAX_RANK];
  __shared__ float sIn[KR_MAX_RANK * PC_TQ];
  for (int e = threadIdx.x; e < R0 * R0; e += blockDim.x) {
    const int j = e / R0, k = e - j * R0;
    sB[e] = trans ? __ldg(B0 + k * R0 + j) : __ldg(B0 + e);  // sB[j * R0 + k] = B0'[j, k]
  }
  float s1 = 0.f, s2 = 0.f, bad = 0.f, s3 = 0.f;
  for (int q0 = blockIdx.x * PC_TQ; q0 < Q; q0 += gridDim.x * PC_TQ) {
    const int tq = min(PC_TQ, Q - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < R0 * PC_TQ; e += blockDim.x) {
      const int k = e / PC_TQ, c = e - k * PC_TQ;
      float v = 0.f;
      if (c < tq) {
        const int64_t gi = (int64_t)k * Q + q0 + c;
        v = __ldg(in + gi);
        if (xl) v = fmaf(-lambda, __ldg(xl + gi), v);
      }
      sIn[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R0 * PC_TQ; e += blockDim.x) {
      const int j = e / PC_TQ, c = e - j * PC_TQ;
      if (c >= tq) continue;
      const float* brow = sB + j * R0;
      float acc = 0.f;
      for (int k = 0; k < R0; ++k) acc = fmaf(brow[k], sIn[k * PC_TQ + c], acc);
      const int64_t gi = (int64_t)j * Q + q0 + c;
      if (x) {
        const float st = alpha * acc;
        const float xo = x[gi];
        const float xn = xo + st;
        x[gi] = xn;
        s1 = fmaf(st, st, s1);
        s2 = fmaf(xn, xn, s2);
        s3 = fmaf(step_grad(sg, gi, xo), st, s3);
        if (!isfinite(xn)) bad = 1.f;
      } else {
        out[gi] = acc;
      }
    }
  }
  if (x) step_norms_block(s1, s2, bad, s3, part);
}

// In shared memory: t (P0 x R_m0 x ... x R_{N-1}, Q entries) <- B applied along modes
// m0..N-1 (B staged in sB transposed: mode m at offset boff[m], entry (k, j) = B'[j, k], so
// lanes with consecutive output rows j read consecutive words, and lanes sharing j
// broadcast). With R_m a multiple of 4 and aligned operands a thread forms four
// consecutive output rows from one 16-byte load of B per k, and lanes take consecutive
// trailing positions q.
__device__ void pc_modes_from(const PcModes& pm, const float* sB, const int* boff, float* t, float* u, int Q, int m0,
                              int P0) {
  float* src = t;
  float* dst = u;
  int P = P0;
  for (int m = m0; m < pm.N; ++m) {
    const int Rm = pm.R[m];
    const int Qm = Q / P / Rm;  // entries after mode m
    const float* Bm = sB + boff[m];
    // the vector path reads B and (for the last mode) writes dst 16 bytes at a time: both
    // addresses must be 16-byte aligned, which the caller's layout does not guarantee
    const bool vec = (Rm & 3) == 0 && (reinterpret_cast<uintptr_t>(Bm) & 15) == 0 &&
                     (Qm != 1 || (reinterpret_cast<uintptr_t>(dst) & 15) == 0);
    if (vec) {
      const int R4 = Rm >> 2;
      const int items = Q >> 2;
      for (int e = threadIdx.x; e < items; e += blockDim.x) {
        const int qq = e % Qm;
        const int rest = e / Qm;
        const int jq = rest % R4;
        const int p = rest / R4;
        const float* col = src + (size_t)p * Rm * Qm + qq;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < Rm; ++k) {
          const float v = col[k * Qm];
          const float4 bk = *reinterpret_cast<const float4*>(Bm + k * Rm + 4 * jq);
          acc.x = fmaf(bk.x, v, acc.x);
          acc.y = fmaf(bk.y, v, acc.y);
          acc.z = fmaf(bk.z, v, acc.z);
          acc.w = fmaf(bk.w, v, acc.w);
        }
        float* o = dst + (size_t)p * Rm * Qm + (4 * jq) * Qm + qq;
        if (Qm == 1) {
          *reinterpret_cast<float4*>(o) = acc;
        } else {
          o[0] = acc.x;
          o[Qm] = acc.y;
          o[2 * Qm] = acc.z;
          o[3 * Qm] = acc.w;
        }
      }
    } else {
      for (int e = threadIdx.x; e < Q; e += blockDim.x) {
        const int p = e / (Rm * Qm);
        const int rest = e - p * Rm * Qm;
        const int jj = rest / Qm;
        const int qq = rest - jj * Qm;
        const float* col = src + p * Rm * Qm + qq;
        const float* bcol = Bm + jj;
        float acc = 0.f;
        for (int k = 0; k < Rm; ++k) acc = fmaf(bcol[k * Rm], col[k * Qm], acc);
        dst[e] = acc;
      }
    }
    __syncthreads();
    float* tmp = src;
    src = dst;
    dst = tmp;
    P *= Rm;
  }
  if (src != t) {
    for (int e = threadIdx.x; e < Q; e += blockDim.x) t[e] = src[e];
    __syncthreads();
  }
}

// A whole slab of modes 1..N-1.
__device__ __forceinline__ void pc_slab_modes(const PcModes& pm, const float* sB, const int* boff, float* t, float* u,
                                              int Q) {
  pc_modes_from(pm, sB, boff, t, u, Q, 1, 1);
}

// The whole step in one kernel when the iterate fits in shared memory: block j stages
// in - lambda xl (all R_1 x Q entries), forms slab j of the first-mode product from row j
// of B0', applies the other modes (rest != 0; for lambda > 0 also the diagonal and the
// second set), then writes out[j] or takes the step (x != nullptr) with its norms.
__global__ void __launch_bounds__(1024) k_pc_fused(PcModes pm, const float* __restrict__ in,
                                                   const float* __restrict__ xl, float lambda,
                                                   const float* __restrict__ B0, int trans0, int rest, int R0, int Q,
                                                   float* __restrict__ out, float* __restrict__ x, float alpha,
                                                   double* __restrict__ part, RichArgs ra, StepGrad sg) {
  extern __shared__ float pc_smem[];
  float* full = pc_smem;          // R0 x Q
  float* t = full + (size_t)R0 * Q;
  float* u = t + Q;
  float* b0 = u + Q;              // row j of B0'
  float* sB = b0 + KR_MAX_RANK;   // other modes, transposed (as in k_pc_slab)
  const int j = blockIdx.x;
  int boff[KR_MAX_MODES], boff2[KR_MAX_MODES];
  int off = 0;
  if (rest) {
    for (int m = 1; m < pm.N; ++m) {
      const int Rm = pm.R[m];
      boff[m] = off;
      for (int e = threadIdx.x; e < Rm * Rm; e += blockDim.x) {
        const int k = e / Rm, jj = e - k * Rm;
        sB[off + e] = pm.trans ? __ldg(pm.B[m] + k * Rm + jj) : __ldg(pm.B[m] + jj * Rm + k);
      }
      off += Rm * Rm;
    }
    if (pm.lambda > 0.f) {
      for (int m = 1; m < pm.N; ++m) {
        const int Rm = pm.R[m];
        boff2[m] = off;
        for (int e = threadIdx.x; e < Rm * Rm; e += blockDim.x) {
          const int k = e / Rm, jj = e - k * Rm;
          sB[off + e] = __ldg(pm.B2[m] + jj * Rm + k);
        }
        off += Rm * Rm;
      }
    }
  }
  for (int k = threadIdx.x; k < R0; k += blockDim.x) b0[k] = trans0 ? __ldg(B0 + k * R0 + j) : __ldg(B0 + j * R0 + k);
  kr_pdl_trigger();
  kr_pdl_wait();  // the gradient (and x) come from the previous kernels
  RichSnap snap = {};
  if (threadIdx.x == 0 && x && ra.st) snap = rich_load(ra.st);
  const int64_t tot = (int64_t)R0 * Q;
  if ((Q & 3) == 0) {
    const float4* in4 = reinterpret_cast<const float4*>(in);
    const float4* xl4 = reinterpret_cast<const float4*>(xl);
    float4* f4 = reinterpret_cast<float4*>(full);
#pragma unroll 8
    for (int64_t e = threadIdx.x; e < tot / 4; e += blockDim.x) {
      float4 v = __ldg(in4 + e);
      if (xl) {
        const float4 w = __ldg(xl4 + e);
        v.x = fmaf(-lambda, w.x, v.x);
        v.y = fmaf(-lambda, w.y, v.y);
        v.z = fmaf(-lambda, w.z, v.z);
        v.w = fmaf(-lambda, w.w, v.w);
      }
      f4[e] = v;
    }
  } else {
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      float v = __ldg(in + e);
      if (xl) v = fmaf(-lambda, __ldg(xl + e), v);
      full[e] = v;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    float acc = 0.f;
    for (int k = 0; k < R0; ++k) acc = fmaf(b0[k], full[(int64_t)k * Q + q], acc);
    t[q] = acc;
  }
  __syncthreads();
  if (rest) {
    pc_slab_modes(pm, sB, boff, t, u, Q);
    if (pm.lambda > 0.f) {
      const float s0 = pm.sig2[0][j];
      for (int e = threadIdx.x; e < Q; e += blockDim.x) {
        int rem = e;
        float prod = 1.f;
        for (int m = pm.N - 1; m >= 1; --m) {
          const int q = rem / pm.R[m];
          prod *= pm.sig2[m][rem - q * pm.R[m]];
          rem = q;
        }
        prod *= s0;
        const float dv = prod + pm.lambda;
        t[e] = dv > 0.f ? t[e] / dv : 0.f;
      }
      __syncthreads();
      pc_slab_modes(pm, sB, boff2, t, u, Q);
    }
  }
  float s1 = 0.f, s2 = 0.f, bad = 0.f, s3 = 0.f;
  for (int e = threadIdx.x; e < Q; e += blockDim.x) {
    if (x) {
      const int64_t gi = (int64_t)j * Q + e;
      const float st = alpha * t[e];
      const float xo = x[gi];
      const float xn = xo + st;
      x[gi] = xn;
      s1 = fmaf(st, st, s1);
      s2 = fmaf(xn, xn, s2);
      s3 = fmaf(step_grad(sg, gi, xo), st, s3);
      if (!isfinite(xn)) bad = 1.f;
    } else {
      out[(int64_t)j * Q + e] = t[e];
    }
  }
  if (x) step_norms_block(s1, s2, bad, s3, part);
  if (x && ra.st) {  // the last block to finish evaluates the stopping rule
    __shared__ bool last;
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(ra.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      rich_check_block(part, gridDim.x, ra, snap);
      if (threadIdx.x == 0) *ra.ticket = 0u;
    }
  }
}

// One block per slab j of the first mode: the other modes (and, for lambda > 0, the
// diagonal and the second set of modes); with x != nullptr the step and its norms.
// Shared memory: the slab twice, then the matrices of modes 1..N-1 (both sets).
__global__ void __launch_bounds__(1024) k_pc_slab(PcModes pm, const float* __restrict__ in, int Q,
                                                  float* __restrict__ out, float* __restrict__ x, float alpha,
                                                  double* __restrict__ part, StepGrad sg) {
  extern __shared__ float pc_smem[];
  float* t = pc_smem;
  float* u = pc_smem + Q;
  float* sB = pc_smem + 2 * Q;
  int boff[KR_MAX_MODES], boff2[KR_MAX_MODES];
  int off = 0;
  for (int m = 1; m < pm.N; ++m) {
    const int Rm = pm.R[m];
    boff[m] = off;
    for (int e = threadIdx.x; e < Rm * Rm; e += blockDim.x) {  // e = k * Rm + j
      const int k = e / Rm, j = e - k * Rm;
      sB[off + e] = pm.trans ? __ldg(pm.B[m] + k * Rm + j) : __ldg(pm.B[m] + j * Rm + k);
    }
    off += Rm * Rm;
  }
  if (pm.lambda > 0.f) {
    for (int m = 1; m < pm.N; ++m) {
      const int Rm = pm.R[m];
      boff2[m] = off;
      for (int e = threadIdx.x; e < Rm * Rm; e += blockDim.x) {
        const int k = e / Rm, j = e - k * Rm;
        sB[off + e] = __ldg(pm.B2[m] + j * Rm + k);
      }
      off += Rm * Rm;
    }
  }
  const int j = blockIdx.x;
  for (int e = threadIdx.x; e < Q; e += blockDim.x) t[e] = in[(int64_t)j * Q + e];
  __syncthreads();
  pc_slab_modes(pm, sB, boff, t, u, Q);
  if (pm.lambda > 0.f) {
    const float s0 = pm.sig2[0][j];
    for (int e = threadIdx.x; e < Q; e += blockDim.x) {
      int rem = e;
      float prod = 1.f;
      for (int m = pm.N - 1; m >= 1; --m) {
        const int q = rem / pm.R[m];
        prod *= pm.sig2[m][rem - q * pm.R[m]];
        rem = q;
      }
      prod *= s0;
      const float dv = prod + pm.lambda;
      t[e] = dv > 0.f ? t[e] / dv : 0.f;
    }
    __syncthreads();
    pc_slab_modes(pm, sB, boff2, t, u, Q);
  }
  float s1 = 0.f, s2 = 0.f, bad = 0.f, s3 = 0.f;
  for (int e = threadIdx.x; e < Q; e += blockDim.x) {
    if (x) {
      const int64_t gi = (int64_t)j * Q + e;
      const float st = alpha * t[e];
      const float xo = x[gi];
      const float xn = xo + st;
      x[gi] = xn;
      s1 = fmaf(st, st, s1);
      s2 = fmaf(xn, xn, s2);
      s3 = fmaf(step_grad(sg, gi, xo), st, s3);
      if (!isfinite(xn)) bad = 1.f;
    } else {
      out[(int64_t)j * Q + e] = t[e];
    }
  }
  if (x) step_norms_block(s1, s2, bad, s3, part);
}

// The step when the first mode of the preconditioner has already been applied (for
// lambda = 0 the tile reduction folds G_1^-1 into its weights, so `in` holds
// G_1^-1 x_1 g): what remains acts inside each slab j of the first mode. Block (j, s)
// stages slab j, forms rows [s nr, (s+1) nr) of its mode-1 product (nr = R_1 / S), applies
// modes 2..N-1 to those rows, takes the step on them with the FP32 block norms, and the
// last block to finish evaluates the stopping rule. Shared memory: the slab, two buffers
// of the block's rows, the matrices of modes 1..N-1 (transposed).
__global__ void __launch_bounds__(256) k_pc_rows(PcModes pm, const float* __restrict__ in, int Q, int S,
                                                 float* __restrict__ x, float alpha, double* __restrict__ part,
                                                 RichArgs ra, StepGrad sg) {
  extern __shared__ float pc_smem[];
  const int R1 = pm.R[1], Q1 = Q / R1, nr = R1 / S, nq = nr * Q1;
  float* full = pc_smem;
  float* t = full + Q;
  float* u = t + nq;
  float* sB = u + nq;
  int boff[KR_MAX_MODES];
  int off = 0;
  for (int m = 1; m < pm.N; ++m) {
    const int Rm = pm.R[m];
    boff[m] = off;
    for (int e = threadIdx.x; e < Rm * Rm; e += blockDim.x) {  // e = k * Rm + jj
      const int k = e / Rm, jj = e - k * Rm;
      sB[off + e] = __ldg(pm.B[m] + jj * Rm + k);
    }
    off += Rm * Rm;
  }
  kr_pdl_trigger();
  kr_pdl_wait();  // `in` and x come from the previous kernels
  RichSnap snap = {};
  if (threadIdx.x == 0 && ra.st) snap = rich_load(ra.st);
  const int j = blockIdx.x / S, s = blockIdx.x - j * S;
  float* xr = x + (int64_t)j * Q + (int64_t)s * nq;
  // this thread's first four entries of x in flight with the slab (the update at the end
  // uses them; blocks of 256 threads)
  float xv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + k * 256;
    xv[k] = e < nq ? xr[e] : 0.f;
  }
  const float* src = in + (int64_t)j * Q;
  for (int e = threadIdx.x; e < Q; e += blockDim.x) full[e] = __ldg(src + e);
  __syncthreads();
  {  // mode 1, rows jj = s nr .. s nr + nr - 1
    const float* B1 = sB + boff[1];
    for (int e = threadIdx.x; e < nq; e += blockDim.x) {
      const int jr = e / Q1, q = e - jr * Q1, jj = s * nr + jr;
      float acc = 0.f;
      for (int k = 0; k < R1; ++k) acc = fmaf(B1[k * R1 + jj], full[k * Q1 + q], acc);
      t[e] = acc;
    }
  }
  __syncthreads();
  pc_modes_from(pm, sB, boff, t, u, nq, 2, nr);
  float s1 = 0.f, s2 = 0.f, bad = 0.f, s3 = 0.f;
  const int64_t r0 = (int64_t)j * Q + (int64_t)s * nq;  // first entry of the block's rows
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // the prefetched entries
    const int e = threadIdx.x + k * 256;
    if (e < nq) {
      const float st = alpha * t[e];
      const float xn = xv[k] + st;
      xr[e] = xn;
      s1 = fmaf(st, st, s1);
      s2 = fmaf(xn, xn, s2);
      s3 = fmaf(step_grad(sg, r0 + e, xv[k]), st, s3);
      if (!isfinite(xn)) bad = 1.f;
    }
  }
  for (int e = threadIdx.x + 4 * 256; e < nq; e += blockDim.x) {  // larger slabs: the rest
    const float st = alpha * t[e];
    const float xo = xr[e];
    const float xn = xo + st;
    xr[e] = xn;
    s1 = fmaf(st, st, s1);
    s2 = fmaf(xn, xn, s2);
    s3 = fmaf(step_grad(sg, r0 + e, xo), st, s3);
    if (!isfinite(xn)) bad = 1.f;
  }
  step_norms_block(s1, s2, bad, s3, part);
  if (ra.st) {  // the last block to finish evaluates the stopping rule
    __shared__ bool last;
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(ra.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      rich_check_block(part, gridDim.x, ra, snap);
      if (threadIdx.x == 0) *ra.ticket = 0u;
    }
  }
}

// Deterministic sum of per-block partials: out[k] = sum_b part[stride*b + k] (k < stride),
// the last component combined with max (flags) when maxlast. One block of 256 threads:
// fixed strided partial sums, then a fixed-order tree, so the result is reproducible.
__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ part, int nb, int stride,
                                                         int maxlast, double* __restrict__ out) {
  __shared__ double red[256];
  for (int k = 0; k < stride; ++k) {
    const bool mx = maxlast && k == stride - 1;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const double v = part[(int64_t)stride * b + k];
      acc = mx ? fmax(acc, v) : acc + v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
      if ((int)threadIdx.x < off) red[threadIdx.x] = mx ? fmax(red[threadIdx.x], red[threadIdx.x + off])
                                                       : red[threadIdx.x] + red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
    __syncthreads();
  }
}

__global__ void k_dot_self(const float* __restrict__ x, int64_t n, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[i] * x[i];
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}


// Full objective: per cell, all I_N rows: sum (<A_N[i], Y[c]> - b[c, i])^2 in FP64.
// Persistent blocks stage A_N once (rows padded to an odd stride: conflict-free reads by
// consecutive threads), then 8 cells' Y rows at a time; SMEM_A = false reads A_N through L1.
constexpr int FULL_CELLS = 8;
template <bool SMEM_A>
__global__ void __launch_bounds__(256) k_full_obj(const float* __restrict__ Y, const float* __restrict__ AT,
                                                  const float* __restrict__ b, int64_t ncell, int IT, int RT,
                                                  double* __restrict__ part) {
  extern __shared__ float fsm[];
  const int LD = RT + 1;
  float* As = fsm;                                     // IT x LD (SMEM_A)
  float* Ys = fsm + (SMEM_A ? (size_t)IT * LD : 0);   // FULL_CELLS x RT
  if (SMEM_A)
    for (int e = threadIdx.x; e < IT * RT; e += blockDim.x) As[(e / RT) * LD + (e % RT)] = AT[e];
  double acc = 0.0;
  for (int64_t c0 = (int64_t)blockIdx.x * FULL_CELLS; c0 < ncell; c0 += (int64_t)gridDim.x * FULL_CELLS) {
    const int nc = (int)min((int64_t)FULL_CELLS, ncell - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < nc * RT; e += blockDim.x) Ys[e] = Y[c0 * RT + e];
    __syncthreads();
    for (int e = threadIdx.x; e < nc * IT; e += blockDim.x) {
      const int cc = e / IT, i = e - cc * IT;
      float u = 0.f;
      for (int r = 0; r < RT; ++r)
        u = fmaf(SMEM_A ? As[i * LD + r] : __ldg(&AT[(int64_t)i * RT + r]), Ys[cc * RT + r], u);
      const double d = (double)u - (double)b[(c0 + cc) * IT + i];
      acc += d * d;
    }
  }
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

int grid_cap(kr_ctx* ctx, int64_t work, int block, int per_sm) {
  int64_t g = (work + block - 1) / block;
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int rt_pad(int RT) {
  if (RT <= 4) return 4;
  if (RT <= 8) return 8;
  if (RT <= 16) return 16;
  if (RT <= 32) return 32;
  return 64;
}

// Launches at most `grid` blocks (resident blocks per SM x SMs); *used = blocks launched.
template <int RTP>
kr_status launch_resid_t(kr_ctx* ctx, const ResidArgs& a, int grid, int* used) {
  size_t smemA = (size_t)a.IT * ResidShape<RTP>::LDA * sizeof(float);
  size_t smemI = (size_t)a.IT * sizeof(float);
  // grid = resident blocks per SM x SMs (a persistent, grid-stride sweep over the cells);
  // `grid` is the cap that sizes the objective partials
  int per_sm = 1;
  if (smemA + smemI <= ctx->smem_optin) {
    KR_TRY(kr_smem_attr(ctx, k_resid<RTP, true>, smemA + smemI));
    KR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid<RTP, true>, RESID_THREADS,
                                                               smemA + smemI));
    int g = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
    if (g > grid) g = grid;
    KR_LAUNCH(ctx, (k_resid<RTP, true>), g, RESID_THREADS, smemA + smemI, a);
    *used = g;
    return KR_OK;
  }
  KR_TRY(kr_smem_attr(ctx, k_resid<RTP, false>, smemI));
  KR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid<RTP, false>, RESID_THREADS, smemI));
  int g = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
  if (g > grid) g = grid;
  KR_LAUNCH(ctx, (k_resid<RTP, false>), g, RESID_THREADS, smemI, a);
  *used = g;
  return KR_OK;
  return KR_OK;
}

}  // namespace

int kr_resid_blocks(kr_ctx* ctx) { return ctx->num_sms * 4; }

kr_status kr_sketch_resid(kr_ctx* ctx, const kr_sketch* sk, const float* AT, int RT, const float* Y, float* W,
                          double* obj_partial, int nblocks, int* used) {
  ResidArgs a;
  a.cell_start = sk->cell_start;
  a.cell_nd = sk->cell_nd;
  a.ent = sk->ent;
  a.bt = sk->bt;
  a.cell_w = sk->cell_w;
  a.invpT = sk->invpT;
  a.perm = sk->perm;
  a.desc = sk->desc;
  a.AT = AT;
  a.IT = sk->IT;
  a.RT = RT;
  a.Y = Y;
  a.W = W;
  a.ncell = sk->ncell;
  a.obj_partial = obj_partial;
  switch (rt_pad(RT)) {
    case 4: return launch_resid_t<4>(ctx, a, nblocks, used);
    case 8: return launch_resid_t<8>(ctx, a, nblocks, used);
    case 16: return launch_resid_t<16>(ctx, a, nblocks, used);
    case 32: return launch_resid_t<32>(ctx, a, nblocks, used);
    default: return launch_resid_t<64>(ctx, a, nblocks, used);
  }
}

// ------------------------------------------------------------------ the solver

namespace {

struct IterBufs {
  float* x;      // R
  float* Y;      // ncell x RT
  float* W;      // ncell x RT
  float* g;      // R
  float* d;      // R
  float* t0;     // max intermediate
  float* t1;     // max intermediate
  double* part;  // step partials (KR_NPART per block)
  double* opart = nullptr;  // objective partials of the sampled pass (per-cell pass: per block; slab pass:
                            // per chunk of the tile reduction)
  double* red;   // 4 doubles
  RichState* rich = nullptr;  // device stopping-rule state
  // slab form (tl != nullptr): X1 and Z are P x R_{N-1} x R_N (N >= 3; x and g for N = 2)
  kr_tiles* tl = nullptr;
  float* X1 = nullptr;
  float* Z = nullptr;
  // N = 3, lambda = 0: A(1) G_1^-1, the weights of the tile reduction with the first mode
  // of the preconditioner folded in (then g holds G_1^-1 x_1 gradient)
  float* B1 = nullptr;
  // with B1 and the eps-aware rule: the gradient itself (a second output of the tile reduction)
  float* g2 = nullptr;
  bool x_zero = false;  // x is zero (a solve's first step): the slab pass skips its forward product
};

int64_t max_intermediate(const Modes& m) {
  // forward: dims R -> (I_0..I_{N-2}, R_{N-1}); backward: the reverse; precond: R
  int64_t mx = kr_prod_R(m);
  int64_t cur = mx;
  for (int n = 0; n < m.N - 1; ++n) {
    cur = cur / m.R[n] * m.I[n];
    if (cur > mx) mx = cur;
  }
  return mx;
}

// Forward sampled pass at x: Y, then the residual kernel (W and objective partials;
// *used = number of partials written).
kr_status forward_resid(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, const IterBufs& bf, int nblk, int* used) {
  const int N = m.N;
  int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    din[n] = m.R[n];
    dout[n] = (n < N - 1) ? m.I[n] : m.R[n];
    B[n] = (n < N - 1) ? m.A[n] : nullptr;
    tr[n] = 0;
  }
  KR_TRY(kr_kron_apply2(ctx, N, din, dout, B, tr, bf.x, bf.Y, bf.t0, bf.t1));
  return kr_sketch_resid(ctx, sk, m.A[N - 1], m.R[N - 1], bf.Y, bf.W, bf.opart ? bf.opart : bf.part, nblk, used);
}

kr_status backward(kr_ctx* ctx, const Modes& m, const IterBufs& bf) {
  const int N = m.N;
  int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    din[n] = (n < N - 1) ? m.I[n] : m.R[n];
    dout[n] = m.R[n];
    B[n] = (n < N - 1) ? m.A[n] : nullptr;
    tr[n] = 1;  // A^T from the stored I x R array
  }
  return kr_kron_apply2(ctx, N, din, dout, B, tr, bf.W, bf.g, bf.t0, bf.t1);
}

// Whether `func` can run with `dyn` bytes of dynamic shared memory next to its static
// shared memory; if so the kernel's dynamic limit is raised to at least `dyn`.
template <class F>
kr_status smem_fit(kr_ctx* ctx, F func, size_t dyn, bool* fits) {
  cudaFuncAttributes fa;
  KR_CUDA(ctx, cudaFuncGetAttributes(&fa, func));
  *fits = dyn + fa.sharedSizeBytes <= ctx->smem_optin;
  if (*fits) KR_TRY(kr_smem_attr(ctx, func, dyn));
  return KR_OK;
}

// One preconditioned Richardson step, x <- x + alpha M+ (g - lambda x); the last kernel
// writes the FP64 partials {||alpha d||^2, ||x||^2, non-finite flag} of its *nparts
// blocks to part (the caller adds them in block order). One kernel when the iterate fits
// in shared memory (two for lambda > 0), else the first mode and the slabs' other modes
// as two (three), else the per-mode sequence. tmp0..tmp2: R floats.
kr_status pc_step_core(kr_ctx* ctx, const FactorTables& t, double lambda, float* g, float* x, float alpha,
                       float* tmp0, float* tmp1, float* tmp2, int ublk, double* part, const RichArgs& ra,
                       int* nparts, bool* checked);

// With mode0_done (lambda = 0, N >= 2) g already holds G_1^-1 x_1 (gradient) and the
// step applies the other modes only (k_pc_rows); graw, if not null, is the gradient itself
// (for the eps-aware rule's g^T step).
kr_status pc_step(kr_ctx* ctx, const FactorTables& t, double lambda, float* g, float* x, float alpha, float* tmp0,
                  float* tmp1, float* tmp2, int ublk, double* part, const RichArgs& ra, bool mode0_done = false,
                  const float* graw = nullptr, double* pc64 = nullptr) {
  int np = 0;
  bool checked = false;
  if (pc64) {  // FP64 application of M+ (badly conditioned ridge problems); pc64: 2 R doubles
    const int N = t.N;
    int64_t R = 1;
    for (int n = 0; n < N; ++n) R *= t.R[n];
    Pc64Modes pm = {};
    pm.N = N;
    for (int n = 0; n < N; ++n) {
      pm.R[n] = t.R[n];
      pm.V[n] = t.V64[n];
      pm.sig[n] = t.sig64[n];
    }
    double* a = pc64;
    double* b = pc64 + R;
    const int grid = grid_cap(ctx, R, 256, 4);
    KR_LAUNCH(ctx, k_grad64, grid, 256, 0, (const float*)g, (const float*)x, (float)lambda, R, a);
    for (int pass = 0; pass < 2; ++pass) {  // V^T along every mode, then (after D) V
      if (pass == 1) KR_LAUNCH(ctx, k_diag64, grid, 256, 0, a, R, pm, lambda);
      int64_t P = 1;
      for (int n = 0; n < N; ++n) {
        const int64_t Q = R / P / t.R[n];
        KR_LAUNCH(ctx, k_mode64, grid, 256, 0, (const double*)a, b, P, t.R[n], Q, t.V64[n], pass == 0 ? 1 : 0);
        double* tmp = a;
        a = b;
        b = tmp;
        P *= t.R[n];
      }
    }
    const StepGrad sg = {ra.eps_rule ? g : nullptr, (float)lambda};
    KR_LAUNCH(ctx, k_update64, ublk, 256, 0, x, (const double*)a, alpha, R, part, sg);
    KR_LAUNCH(ctx, k_rich_check, 1, 32, 0, part, ublk, ra);
    return KR_OK;
  }
  if (mode0_done) {
    const int N = t.N;
    int64_t Q = 1;
    size_t nb = 0;
    for (int n = 1; n < N; ++n) {
      Q *= t.R[n];
      nb += (size_t)t.R[n] * t.R[n];
    }
    const int R1 = t.R[1];
    const int S = (R1 % 4 == 0) ? 4 : (R1 % 2 == 0 ? 2 : 1);
    const int64_t nq = Q / S;
    PcModes pm = {};
    pm.N = N;
    for (int n = 0; n < N; ++n) {
      pm.R[n] = t.R[n];
      pm.B[n] = t.ginv[n];
    }
    const size_t smem = ((size_t)Q + 2 * (size_t)nq + nb) * sizeof(float);
    bool fits = false;
    KR_TRY(smem_fit(ctx, k_pc_rows, smem, &fits));
    if (!fits) return kr_fail(ctx, KR_EINVAL, "preconditioned step: slab of %lld entries too large", (long long)Q);
    const StepGrad sg = {ra.eps_rule ? graw : nullptr, 0.f};
    KR_LAUNCH_PDL(ctx, k_pc_rows, t.R[0] * S, 256, smem, pm, (const float*)g, (int)Q, S, x, alpha, part, ra, sg);
    return KR_OK;
  }
  KR_TRY(pc_step_core(ctx, t, lambda, g, x, alpha, tmp0, tmp1, tmp2, ublk, part, ra, &np, &checked));
  if (!checked) KR_LAUNCH(ctx, k_rich_check, 1, 32, 0, part, np, ra);
  return KR_OK;
}

// The step itself; *checked when the last kernel also applied the stopping rule.
kr_status pc_step_core(kr_ctx* ctx, const FactorTables& t, double lambda, float* g, float* x, float alpha,
                       float* tmp0, float* tmp1, float* tmp2, int ublk, double* part, const RichArgs& ra,
                       int* nparts, bool* checked) {
  const int N = t.N;
  int64_t R = 1;
  for (int n = 0; n < N; ++n) R *= t.R[n];
  const int R0 = t.R[0];
  const int64_t Q = R / R0;
  size_t nb = 0;
  for (int n = 1; n < N; ++n) nb += (size_t)t.R[n] * t.R[n];
  if (lambda > 0.0) nb *= 2;
  const size_t smem = (2 * (size_t)Q + nb) * sizeof(float);
  // the gradient of the step for the eps-aware rule's g^T step: g - lambda x_old
  const StepGrad sg = {ra.eps_rule ? g : nullptr, (float)lambda};
  const StepGrad sg0 = {ra.eps_rule ? g : nullptr, 0.f};  // g already holds g - lambda x
  const StepGrad none_sg = {nullptr, 0.f};
  bool split = false;
  if (Q <= (int64_t(1) << 20)) KR_TRY(smem_fit(ctx, k_pc_slab, smem, &split));
  if (!split) {
    if (lambda > 0.0) KR_LAUNCH(ctx, k_sub_lambda_x, ublk, 256, 0, g, x, (float)lambda, R);
    KR_TRY(kr_precond_apply(ctx, t, lambda, g, tmp0, tmp1, tmp2));
    KR_LAUNCH(ctx, k_update_reduce, ublk, 256, 0, x, tmp0, alpha, R, part, sg0);
    *nparts = ublk;
    return KR_OK;
  }
  PcModes pm = {};
  pm.N = N;
  for (int n = 0; n < N; ++n) {
    pm.R[n] = t.R[n];
    pm.B[n] = lambda > 0.0 ? t.V[n] : t.ginv[n];
    pm.B2[n] = t.V[n];
    pm.sig2[n] = t.sig2[n];
  }
  pm.trans = lambda > 0.0 ? 1 : 0;
  pm.lambda = (float)lambda;

  int g0 = (int)((Q + PC_TQ - 1) / PC_TQ);
  if (g0 > ctx->num_sms * 4) g0 = ctx->num_sms * 4;
  const int sthreads = Q >= 1024 ? 1024 : (Q <= 256 ? 256 : (int)((Q + 31) / 32 * 32));
  const float* xl = lambda > 0.0 ? x : nullptr;
  const int Qi = (int)Q;
  const size_t fsmem = ((size_t)R + 2 * (size_t)Q + KR_MAX_RANK + nb) * sizeof(float);
  bool fused = false;
  KR_TRY(smem_fit(ctx, k_pc_fused, fsmem, &fused));
  if (fused) {
    if (lambda == 0.0) {
      KR_LAUNCH_PDL(ctx, k_pc_fused, R0, sthreads, fsmem, pm, g, (const float*)nullptr, 0.f, pm.B[0], 0,
                    N > 1 ? 1 : 0, R0, Qi, (float*)nullptr, x, alpha, part, ra, sg);
      *nparts = R0;
      *checked = true;
      return KR_OK;
    }
    RichArgs none = ra;
    none.st = nullptr;
    KR_LAUNCH_PDL(ctx, k_pc_fused, R0, sthreads, fsmem, pm, g, (const float*)x, (float)lambda, pm.B[0], 1, 1, R0,
                  Qi, tmp0, (float*)nullptr, 0.f, part, none, none_sg);
    KR_LAUNCH_PDL(ctx, k_pc_fused, R0, sthreads, fsmem, pm, (const float*)tmp0, (const float*)nullptr, 0.f,
                  pm.B2[0], 0, 0, R0, Qi, (float*)nullptr, x, alpha, part, ra, sg);
    *nparts = R0;
    *checked = true;
    return KR_OK;
  }
  if (lambda == 0.0 && N == 1) {
    KR_LAUNCH(ctx, k_pc_mode0, g0, 256, 0, g, xl, 0.f, pm.B[0], 0, R0, Qi, nullptr, x, alpha, part, sg);
    *nparts = g0;
    return KR_OK;
  }
  KR_LAUNCH(ctx, k_pc_mode0, g0, 256, 0, g, xl, (float)lambda, pm.B[0], pm.trans, R0, Qi, tmp0, nullptr, 0.f, part,
            none_sg);
  if (lambda == 0.0) {
    KR_LAUNCH(ctx, k_pc_slab, R0, sthreads, smem, pm, tmp0, Qi, nullptr, x, alpha, part, sg);
    *nparts = R0;
    return KR_OK;
  }
  KR_LAUNCH(ctx, k_pc_slab, R0, sthreads, smem, pm, tmp0, Qi, tmp1, nullptr, 0.f, part, none_sg);
  KR_LAUNCH(ctx, k_pc_mode0, g0, 256, 0, tmp1, nullptr, 0.f, pm.B2[0], 0, R0, Qi, nullptr, x, alpha, part, sg);
  *nparts = g0;
  return KR_OK;
}

// Largest intermediate of the prefix mode products of the slab form (modes < N-2).
int64_t slab_max_intermediate(const Modes& m) {
  int64_t cur = kr_prod_R(m), mx = cur;
  for (int n = 0; n < m.N - 2; ++n) {
    cur = cur / m.R[n] * m.I[n];
    if (cur > mx) mx = cur;
  }
  return mx;
}

// Slab form of the sampled pass: X1 = X x_1 A(1) ... x_{N-2} A(N-2), then the fused slab
// kernel (Z and the per-tile objective partials in bf.tl->objpart).
kr_status slab_forward(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, const IterBufs& bf, bool want_obj,
                       bool rearm, int prec = 0, int flags = 0) {
  const int N = m.N;
  const float* X1 = bf.x;
  if (bf.x_zero) flags |= KR_SLAB_ZERO_X;  // X1 = 0 as well: not formed
  if (N > 2 && !bf.x_zero) {
    int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
    const float* B[KR_MAX_MODES];
    for (int n = 0; n < N; ++n) {
      din[n] = m.R[n];
      dout[n] = (n < N - 2) ? m.I[n] : m.R[n];
      B[n] = (n < N - 2) ? m.A[n] : nullptr;
      tr[n] = 0;
    }
    KR_TRY(kr_kron_apply2(ctx, N, din, dout, B, tr, bf.x, bf.X1, bf.t0, bf.t1));
    X1 = bf.X1;
  }
  return kr_slab_pass(ctx, sk, bf.tl, m.A[N - 2], m.A[N - 1], X1, want_obj, rearm, prec, flags);
}

// g = Z x_1 A(1)^T ... x_{N-2} A(N-2)^T: the sum over the tiles folded with the last
// prefix mode (mode N-2 in the paper's 1-based count), then the earlier prefix modes.
kr_status slab_backward(kr_ctx* ctx, const Modes& m, const IterBufs& bf, double* opart) {
  const int N = m.N;
  if (N <= 3)
    return kr_tile_reduce(ctx, bf.tl, N == 3 ? (bf.B1 ? bf.B1 : m.A[0]) : nullptr, bf.g, opart,
                          bf.g2 ? m.A[0] : nullptr, bf.g2);
  KR_TRY(kr_tile_reduce(ctx, bf.tl, m.A[N - 3], bf.Z, opart));
  int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    din[n] = (n < N - 3) ? m.I[n] : m.R[n];
    dout[n] = m.R[n];
    B[n] = (n < N - 3) ? m.A[n] : nullptr;
    tr[n] = 1;
  }
  return kr_kron_apply2(ctx, N, din, dout, B, tr, bf.Z, bf.g, bf.t0, bf.t1);
}

// Sampled pass at x: g = K~^T Omega (b~ - K~ x) (if want_g) and the objective partials
// (*op, *on: FP64 values to be summed; with want_g only when want_obj).
kr_status sampled_pass(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, const IterBufs& bf, int nblk, bool want_g,
                       const double** op, int* on, bool want_obj = false, int prec = 0) {
  if (bf.tl) {
    KR_TRY(slab_forward(ctx, m, sk, bf, !want_g || want_obj, !want_g, prec, want_g ? 0 : KR_SLAB_OBJ_ONLY));
    if (!want_g) {
      *op = bf.tl->objpart;
      *on = (int)bf.tl->ntmax;
      return KR_OK;
    }
    // the tile reduction also sums the tiles' objective partials per chunk, in tile order
    *op = bf.opart;
    *on = (int)(bf.tl->nc * bf.tl->Pq);
    return slab_backward(ctx, m, bf, want_obj ? bf.opart : nullptr);
  }
  int used = 0;
  KR_TRY(forward_resid(ctx, m, sk, bf, nblk, &used));
  *op = bf.opart ? bf.opart : bf.part;
  *on = used;
  return want_g ? backward(ctx, m, bf) : KR_OK;
}

}  // namespace



bool kr_graph_while(kr_ctx* ctx, const std::function<kr_status(cudaGraphConditionalHandle, int)>& body,
                    int64_t* per_step) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle hnd = 0;
  bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
  ok = ok && cudaGraphConditionalHandleCreate(&hnd, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  ok = ok && cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
  *per_step = 0;
  if (ok && cudaStreamBeginCaptureToGraph(ctx->stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed) == cudaSuccess) {
    const int64_t l0 = ctx->launches;
    const kr_status cs = body(hnd, 1);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &captured);
    *per_step = ctx->launches - l0;
    ctx->launches = l0;
    ok = cs == KR_OK && ce == cudaSuccess;
  } else {
    ok = false;
  }
  ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (ok) ok = cudaGraphLaunch(exec, ctx->stream) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(ctx->stream) == cudaSuccess;  // the graph ends before it is destroyed
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (!ok) cudaGetLastError();  // graphs unavailable: the host loop takes over
  if (ok) ctx->graphs++;
  return ok;
}

kr_status kr_gm_handle(kr_ctx* ctx, unsigned dflt, cudaGraphConditionalHandle* hnd) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t graph = nullptr;
  KR_CUDA(ctx, cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return kr_fail(ctx, KR_EINVAL, "graph sweep: the stream is not capturing");
  KR_CUDA(ctx, cudaGraphConditionalHandleCreate(hnd, graph, dflt, cudaGraphCondAssignDefault));
  return KR_OK;
}

kr_status kr_capture_while(kr_ctx* ctx, cudaGraphConditionalHandle hnd,
                           const std::function<kr_status(cudaGraphConditionalHandle, int)>& body, int64_t* per_body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t ndeps = 0;
  KR_CUDA(ctx, cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &graph, &deps, &edges, &ndeps));
  if (cs != cudaStreamCaptureStatusActive) return kr_fail(ctx, KR_EINVAL, "graph sweep: the stream is not capturing");
  if (!ctx->side_stream) return kr_fail(ctx, KR_EINVAL, "graph sweep: no side stream for the loop bodies");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  // full dependencies on everything captured so far on the stream
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  KR_CUDA(ctx, cudaGraphAddNode(&node, graph, dv.empty() ? nullptr : dv.data(), nullptr, dv.size(), &cp));
  KR_CUDA(ctx, cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  const cudaStream_t main = ctx->stream;
  KR_CUDA(ctx, cudaStreamBeginCaptureToGraph(ctx->side_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
  const int64_t l0 = ctx->launches;
  ctx->stream = ctx->side_stream;
  const kr_status st = body(hnd, 1);
  ctx->stream = main;
  *per_body = ctx->launches - l0;
  ctx->launches = l0;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->side_stream, &captured);
  if (st != KR_OK) return st;
  if (ce != cudaSuccess) return kr_fail_cuda(ctx, ce, "graph sweep: end of a loop body's capture", __FILE__, __LINE__);
  return KR_OK;
}

kr_status kr_gm_section(kr_ctx* ctx, const std::function<kr_status()>& fn) {
  if (ctx->gm.capturing) return fn();
  KR_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
  const kr_status st = fn();
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
  if (st != KR_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != KR_OK) return st;
    return kr_fail_cuda(ctx, ce, "asynchronous solve: capture of a loop", __FILE__, __LINE__);
  }
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, ctx->stream);
  if (ex) cudaGraphExecDestroy(ex);  // an executable still running is freed when it completes
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return kr_fail_cuda(ctx, e, "asynchronous solve: launch of a loop graph", __FILE__, __LINE__);
  ctx->graphs++;
  return KR_OK;
}

namespace {
__global__ void k_gm_flags(const int* __restrict__ f, int n, int bit, int* __restrict__ err) {
  if (threadIdx.x == 0) {
    int v = 0;
    for (int i = 0; i < n; ++i) v |= f[i];
    if (v) atomicOr(err, bit);
  }
}
__global__ void k_gm_store(const int* __restrict__ status, const int* __restrict__ it, int* __restrict__ dst) {
  if (threadIdx.x == 0) {
    dst[0] = *status;
    dst[1] = *it;
  }
}
}  // namespace

kr_status kr_gm_flags(kr_ctx* ctx, const int* flags, int n, int bit) {
  KR_LAUNCH(ctx, k_gm_flags, 1, 32, 0, flags, n, bit, ctx->gm.err);
  return KR_OK;
}

kr_status kr_gm_status(kr_ctx* ctx, const int* status, const int* it, int64_t per_body, int base_slot,
                       int* slot_out) {
  if (ctx->gm.slot >= ctx->gm.nstatus) return kr_fail(ctx, KR_EINVAL, "graph sweep: more loops than status slots");
  KR_LAUNCH(ctx, k_gm_store, 1, 32, 0, status, it, ctx->gm.status + 2 * ctx->gm.slot);
  ctx->gm.body_launches.push_back(per_body);
  ctx->gm.base_slot.push_back(base_slot);
  ctx->gm.owner.push_back(ctx->gm.cur_owner);
  if (slot_out) *slot_out = ctx->gm.slot;
  ctx->gm.slot++;
  return KR_OK;
}

size_t kr_gm_state_bytes() { return sizeof(RichState); }
static_assert(64 + sizeof(RichState) <= KR_GM_ASYNC_BYTES, "an asynchronous solve's state must fit kr_ctx::gm_async");

kr_status kr_gm_core_report(kr_ctx* ctx, double lambda, kr_report* rep) {
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  char* h = static_cast<char*>(ctx->hbuf);
  RichState* hs = reinterpret_cast<RichState*>(h);
  double* obj = reinterpret_cast<double*>(h + 1024);
  unsigned long long* dist = reinterpret_cast<unsigned long long*>(h + 1040);
  KR_CUDA(ctx, cudaMemcpyAsync(hs, ctx->gm.last, sizeof(RichState), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaMemcpyAsync(obj, ctx->gm.obj, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaMemcpyAsync(dist, ctx->gm.distinct, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  rep->iters = hs->it;
  rep->converged = hs->status == STEP_CONVERGED ? 1 : hs->status == STEP_FLOOR ? 2 : hs->status == STEP_EPS ? 3 : 0;
  rep->rel_update = hs->h[1] > 0.0 ? sqrt(hs->h[0]) / sqrt(hs->h[1]) : (hs->h[0] == 0.0 ? 0.0 : INFINITY);
  rep->obj_sampled = obj[0] + lambda * obj[1];
  rep->distinct = (int64_t)*dist;
  rep->s = ctx->gm.last_s;
  rep->precision_used = ctx->gm.last_prec;
  return KR_OK;
}

// Core Alg. 2 solve on device-resident inputs. Timings go to rep->t_ms if rep != NULL.
kr_status kr_solve_device(kr_ctx* ctx, const Modes& m, const float* b, const SolveCfg& cfg, uint64_t seed,
                          uint64_t call_id, float* x_out, kr_report* rep) {
  const int N = m.N;
  const int64_t R = kr_prod_R(m);
  const int RT = m.R[N - 1];
  const int nblk = kr_resid_blocks(ctx);
  KR_TRY(kr_sketch_check(ctx, m, cfg.s));
  kr_sketch sk;
  kr_sketch_setup(&sk, m, cfg.s);
  const int64_t ncell = sk.ncell;
  const bool slab = ctx->slab_pass && kr_slab_eligible(ctx, m, &sk);
  sk.want_desc = !slab;
  kr_tiles tl;
  int64_t nyw = ncell * RT, nx1 = 0;  // floats of Y / W (per-cell form) or X1 / Z (slab form, N >= 3)
  int64_t mx = max_intermediate(m);
  // the autotuner's shape class and its candidate tile budgets (the tiles' arrays are sized
  // for the smallest, which needs the most tiles)
  static const uint32_t kTuneEt[5] = {2048, 4096, 8192, 16384, 32768};
  int64_t tkey[6] = {N, m.I[N > 1 ? N - 2 : 0], m.R[N > 1 ? N - 2 : 0], m.I[N - 1], RT, 0};
  for (int64_t v = cfg.s; v > 1; v >>= 1) ++tkey[5];
  // inside a captured sweep (ctx->gm.on) nothing is read back, timed or tuned: checks go to
  // the device error word, each loop is a conditional node, and an untuned class keeps the
  // context's tile budget
  const bool gm = ctx->gm.on;
  uint32_t tuned_et = (slab && ctx->autotune) ? kr_tune_lookup(ctx, tkey) : 0;
  const bool tune_now = slab && ctx->autotune && tuned_et == 0 && !gm;
  const bool use_tuned = ctx->autotune && (tuned_et != 0 || tune_now);
  if (slab) {
    const uint32_t et_keep = ctx->slab_tile_entries;
    if (use_tuned) ctx->slab_tile_entries = tune_now ? kTuneEt[0] : tuned_et;
    kr_tiles_setup(ctx, m, &sk, &tl);
    ctx->slab_tile_entries = et_keep;
    // folded first preconditioner mode with the eps-aware rule: the reduction also returns g
    if (N == 3 && cfg.lambda == 0.0 && cfg.stop_rule == 1) tl.nout = 2;
    nyw = 0;
    nx1 = N > 2 ? tl.P * m.R[N - 2] * RT : 0;
    mx = slab_max_intermediate(m);
  }
  Need nd;
  kr_tables_need(m, cfg.lambda > 0.0, nd);
  kr_sketch_own_need(&sk, nd);
  if (slab) kr_tiles_own_need(&tl, ncell, nd);
  nd.add<float>(nyw);  // Y
  nd.add<float>(nyw);  // W
  nd.add<float>(nx1);  // X1
  nd.add<float>(nx1);  // Z
  nd.add<float>(R);    // g
  nd.add<float>(R);    // d
  nd.add<float>(mx);   // t0
  nd.add<float>(mx);   // t1
  const size_t npart = (size_t)KR_NPART * (nblk > 1024 ? nblk : 1024);
  const bool eps_rule = cfg.stop_rule == 1;
  const size_t nopart = eps_rule ? (slab ? (size_t)(tl.nc * tl.Pq) : (size_t)nblk) : 0;
  nd.add<double>(npart);
  nd.add<double>(nopart);
  nd.add<double>(16);
  nd.add<RichState>(1);
  // the first preconditioner mode folded into the tile reduction (lambda = 0, N = 3)
  const bool fold0 = slab && N == 3 && cfg.lambda == 0.0;
  nd.add<float>(fold0 ? (size_t)m.I[0] * m.R[0] : 0);
  nd.add<float>(fold0 && eps_rule ? (size_t)R : 0);
  nd.add<double>(cfg.lambda > 0.0 ? 2 * (size_t)R : 0);  // FP64 preconditioner buffers (ill-conditioned ridge)
  {
    Need sc = nd;
    kr_sketch_scratch_need(ctx, cfg.s, ncell, m.I[m.N - 1], nd);
    if (slab) {
      kr_tiles_scratch_need(&tl, ncell, sc);
      if (sc.off > nd.off) nd.off = sc.off;
    }
  }
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  Carve cv(ctx->ws, ctx->ws_size);
  cudaEvent_t* ev = ctx->ev;
  auto mark = [&](int i) -> kr_status {
    if (!gm) KR_CUDA(ctx, cudaEventRecord(ev[i], ctx->stream));
    return KR_OK;
  };
  KR_TRY(mark(0));
  FactorTables t;
  KR_TRY(kr_tables_build(ctx, m, cfg.lambda > 0.0, cv, t, !gm));
  if (gm) KR_TRY(kr_gm_flags(ctx, t.flags, N, KR_GM_FACTOR_RANK));
  KR_TRY(mark(1));
  kr_sketch_layout(&sk, cv);
  IterBufs bf;
  if (slab) {
    kr_tiles_layout(&tl, ncell, cv);
    bf.tl = &tl;
  }
  bf.x = x_out;
  bf.Y = cv.take<float>(nyw);
  bf.W = cv.take<float>(nyw);
  bf.X1 = cv.take<float>(nx1);
  bf.Z = cv.take<float>(nx1);
  bf.g = cv.take<float>(R);
  bf.d = cv.take<float>(R);
  bf.t0 = cv.take<float>(mx);
  bf.t1 = cv.take<float>(mx);
  bf.part = cv.take<double>(npart);
  bf.opart = eps_rule ? cv.take<double>(nopart) : nullptr;
  bf.red = cv.take<double>(16);
  bf.rich = cv.take<RichState>(1);
  // The ridge preconditioner in FP64 when FP32 rounding of its application, about
  // u32 sqrt(cond(M)) relative in M's norm, would spoil the spectral approximation.
  double* pc64 = nullptr;
  if (cfg.lambda > 0.0) {
    double* buf = cv.take<double>(2 * (size_t)R);
    if (gm) {  // the factors' spectra, which decide it, are not read back
      pc64 = buf;
    } else {
      double hi = 1.0, lo = 1.0;
      for (int n = 0; n < N; ++n) {
        hi *= t.sig_max[n];
        lo *= t.sig_min[n];
      }
      const double cond = (hi + cfg.lambda) / (lo + cfg.lambda);
      if (ldexp(sqrt(cond), -24) > 1e-3) pc64 = buf;
    }
  }
  if (fold0) {  // B1 = A(1) G_1^-1 (G_1^-1 symmetric: row i of B1 = G_1^-1 applied to row i of A(1))
    bf.B1 = cv.take<float>((size_t)m.I[0] * m.R[0]);
    KR_TRY(kr_mode_product(ctx, m.A[0], bf.B1, m.I[0], m.R[0], 1, m.R[0], t.ginv[0], 0));
    if (eps_rule) bf.g2 = cv.take<float>(R);
  }
  {
    Carve sc = cv;
    KR_TRY(kr_sketch_fill(ctx, m, t, b, seed, call_id, 0, &sk, sc, true));
  }
  KR_CUDA(ctx, cudaMemsetAsync(bf.x, 0, sizeof(float) * R, ctx->stream));
  if (tune_now) {
    // one slab pass (its cost does not depend on x) timed at every candidate budget; the
    // fastest is kept for the shape class
    for (int i = 0; i < 2; ++i)
      if (!ctx->tune_ev[i]) KR_CUDA(ctx, cudaEventCreate(&ctx->tune_ev[i]));
    float ms[5];
    int best = 0;
    for (int c = 0; c < 5; ++c) {
      tl.et = kTuneEt[c];
      {
        Carve sc = cv;  // the final build below takes the same scratch
        KR_TRY(kr_tiles_build(ctx, &sk, &tl, sc));
      }
      KR_TRY(slab_forward(ctx, m, &sk, bf, false, true));  // warm
      // the fastest of three passes: other streams' work (a fused batch's other problems)
      // can only add time
      ms[c] = INFINITY;
      for (int rep = 0; rep < 3; ++rep) {
        KR_CUDA(ctx, cudaEventRecord(ctx->tune_ev[0], ctx->stream));
        KR_TRY(slab_forward(ctx, m, &sk, bf, false, true));
        KR_CUDA(ctx, cudaEventRecord(ctx->tune_ev[1], ctx->stream));
        KR_CUDA(ctx, cudaEventSynchronize(ctx->tune_ev[1]));
        float t = 0.f;
        KR_CUDA(ctx, cudaEventElapsedTime(&t, ctx->tune_ev[0], ctx->tune_ev[1]));
        ms[c] = fminf(ms[c], t);
      }
      if (ms[c] < ms[best]) best = c;
    }
    tuned_et = kTuneEt[best];
    kr_tune_record(ctx, tkey, tuned_et, ms, 5);
  }
  if (slab) {
    if (use_tuned) tl.et = tuned_et;
    KR_TRY(kr_tiles_build(ctx, &sk, &tl, cv));
  }
  KR_TRY(mark(2));
  KR_TRY(mark(3));
  double* h = (double*)ctx->hbuf;
  const int ublk = grid_cap(ctx, R, 256, 4);
  int it = 0, converged = 0;
  double rel = INFINITY;
  kr_status st = KR_OK;
  const double* op = nullptr;
  int on = 0;
  KR_LAUNCH(ctx, k_rich_init, 1, 1, 0, bf.rich);
  RichState* hs = reinterpret_cast<RichState*>(ctx->hbuf);
  // One Richardson step and the stopping rule on the device (inside the graph the check
  // also sets the loop condition).
  unsigned int* ticket = reinterpret_cast<unsigned int*>(bf.red + 8);
  KR_CUDA(ctx, cudaMemsetAsync(ticket, 0, sizeof(unsigned int), ctx->stream));
  // Constants of the (1+eps)-aware rule: with sampled-to-exact spectral bounds
  // (1 - sqrt(eps)) M <= H <= (1 + sqrt(eps)) M (proof of Thm 4.5), the step x - alpha M+ g
  // contracts the excess by rho^2 with rho = max(|1 - alpha (1 - sqrt(eps))|,
  // |1 - alpha (1 + sqrt(eps))|) (= 2 sqrt(eps) - eps at the paper's alpha = 1 - sqrt(eps);
  // Lemma 4.2), and g^T M+ g >= (1 - sqrt(eps)) times the excess.
  const double se = sqrt(cfg.eps), c1 = 1.0 - se;
  const double rho = fmax(fabs(1.0 - cfg.alpha * (1.0 - se)), fabs(1.0 - cfg.alpha * (1.0 + se)));
  // Reduced-precision contractions (kr_opts.precision) for the first phase of the loop, on
  // the slab path only; the phase ends at a step tolerance the format can reach.
  const int prec1 = (slab && cfg.prec > 0) ? kr_slab_precision(tl.R2, tl.RT, cfg.prec) : 0;
  int cur_prec = prec1;
  double cur_tol = prec1 == 0 ? cfg.tol : fmax(cfg.tol, prec1 == 1 ? 0.0078125 : 0.0625);
  auto one_step = [&](cudaGraphConditionalHandle hnd, int use_hnd) -> kr_status {
    KR_TRY(sampled_pass(ctx, m, &sk, bf, nblk, true, &op, &on, eps_rule, cur_prec));
    RichArgs ra = {};
    ra.st = bf.rich;
    ra.tol = cur_tol;
    ra.max_iter = cfg.max_iter;
    ra.hnd = hnd;
    ra.use_hnd = use_hnd;
    ra.ticket = ticket;
    ra.eps_rule = eps_rule ? 1 : 0;
    ra.rho2_c1 = rho * rho / c1;
    ra.inv_c1 = 1.0 / c1;
    ra.theta_eps = cfg.theta * cfg.eps;
    ra.inv_alpha = 1.0 / cfg.alpha;
    ra.lambda = cfg.lambda;
    ra.op = op;
    ra.on = on;
    return pc_step(ctx, t, cfg.lambda, bf.g, bf.x, (float)cfg.alpha, bf.d, bf.t0, bf.t1, ublk, bf.part, ra,
                   bf.B1 != nullptr, bf.g2, pc64);
  };
  auto read_state = [&]() -> kr_status {
    KR_CUDA(ctx, cudaMemcpyAsync(hs, bf.rich, sizeof(RichState), cudaMemcpyDeviceToHost, ctx->stream));
    KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return KR_OK;
  };
  bool from_zero = true;  // x = 0 before the first step
  auto run_loop = [&]() -> kr_status {
    // The first step runs from the host: it grows every buffer and sets every kernel
    // attribute the steps need, so the captured steps allocate nothing.
    bf.x_zero = from_zero;
    const kr_status st0 = one_step(0, 0);
    bf.x_zero = false;
    from_zero = false;
    KR_TRY(st0);
    KR_TRY(read_state());
    if (hs->status == STEP_CONTINUE && ctx->device_loop && !ctx->timing) {
      // Steps 2.. as one graph (in a fused batch: one node of the batch's shared graph);
      // k_rich_check clears the condition on convergence, failure or max_iter.
      int64_t per_step = 0;
      const int it0 = hs->it;
      const bool ran = ctx->shared_loop ? kr_shared_loop_run(ctx->shared_loop, ctx, one_step, &per_step)
                                        : kr_graph_while(ctx, one_step, &per_step);
      if (ran) {
        KR_TRY(read_state());
        ctx->launches += per_step * (hs->it - it0);
      }
    }
    while (hs->status == STEP_CONTINUE) {
      KR_TRY(one_step(0, 0));
      KR_TRY(read_state());
    }
    return KR_OK;
  };
  if (gm) {
    // the loop (and the FP32 refinement, entered on the device when the first phase did
    // not stop at max_iter) as conditional nodes of the sweep's graph or, for an
    // asynchronous solve outside capture, of graphs of their own
    int slot1 = -1;
    KR_TRY(kr_gm_section(ctx, [&]() -> kr_status {
      cudaGraphConditionalHandle h1 = 0;
      int64_t pb = 0;
      KR_TRY(kr_gm_handle(ctx, 0, &h1));
      // the first step from x = 0 ahead of the node, as the host loop runs it; its check
      // sets the node's condition
      bf.x_zero = true;
      const kr_status s1 = one_step(h1, 1);
      bf.x_zero = false;
      KR_TRY(s1);
      KR_TRY(kr_capture_while(ctx, h1, one_step, &pb));
      return kr_gm_status(ctx, &bf.rich->status, &bf.rich->it, pb, -1, &slot1);
    }));
    if (prec1 > 0) {
      KR_TRY(kr_gm_section(ctx, [&]() -> kr_status {
        cudaGraphConditionalHandle h2 = 0;
        int64_t pb = 0;
        KR_TRY(kr_gm_handle(ctx, 0, &h2));
        KR_LAUNCH(ctx, k_zero_if_status, grid_cap(ctx, R, 256, 4), 256, 0, bf.x, R, &bf.rich->status,
                  (int)STEP_NONFINITE);
        KR_LAUNCH(ctx, k_rich_resume_dev, 1, 1, 0, bf.rich, h2);
        cur_prec = 0;
        cur_tol = cfg.tol;
        KR_TRY(kr_capture_while(ctx, h2, one_step, &pb));
        return kr_gm_status(ctx, &bf.rich->status, &bf.rich->it, pb, slot1, nullptr);
      }));
    }
    // the sampled objective at the returned x and the final state, for the sweep's report
    KR_TRY(sampled_pass(ctx, m, &sk, bf, nblk, false, &op, &on));
    KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, op, on, 1, 0, bf.red);
    KR_LAUNCH(ctx, k_dot_self, ublk, 256, 0, bf.x, R, bf.part + 1024);
    KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, bf.part + 1024, ublk, 1, 0, bf.red + 1);
    KR_CUDA(ctx, cudaMemcpyAsync(ctx->gm.obj, bf.red, 2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    KR_CUDA(ctx, cudaMemcpyAsync(ctx->gm.last, bf.rich, sizeof(RichState), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->gm.last_s = cfg.s;
    ctx->gm.last_prec = prec1;
    if (ctx->gm.report)
      KR_LAUNCH(ctx, k_async_report, 1, 32, 0, (const RichState*)bf.rich, (const double*)bf.red,
                (const unsigned long long*)ctx->gm.distinct, (const int*)ctx->gm.err, (const int*)ctx->gm.status,
                prec1 > 0 ? 1 : 0, cfg.lambda, cfg.s, prec1, static_cast<kr_dev_report*>(ctx->gm.report));
    return KR_OK;
  }
  KR_TRY(run_loop());
  int iters_reduced = 0;
  if (prec1 > 0) {
    // FP32 refinement from where the reduced-precision steps stopped (from x = 0 if they
    // produced a non-finite iterate); max_iter bounds both phases together
    iters_reduced = hs->it;
    if (hs->status != STEP_MAXITER) {
      if (hs->status == STEP_NONFINITE) KR_CUDA(ctx, cudaMemsetAsync(bf.x, 0, sizeof(float) * R, ctx->stream));
      KR_LAUNCH(ctx, k_rich_resume, 1, 1, 0, bf.rich);
      cur_prec = 0;
      cur_tol = cfg.tol;
      KR_TRY(run_loop());
    }
  }
  it = hs->it;
  rel = hs->h[1] > 0.0 ? sqrt(hs->h[0]) / sqrt(hs->h[1]) : (hs->h[0] == 0.0 ? 0.0 : INFINITY);
  if (hs->status == STEP_NONFINITE) st = kr_fail(ctx, KR_ENONFINITE, "Richardson iterate became non-finite at iteration %d", it);
  if (hs->status == STEP_DIVERGED)
    st = kr_fail(ctx, KR_EDIVERGED, "Richardson step grew 3 times in a row past 16x its minimum (iteration %d)", it);
  if (hs->status == STEP_CONVERGED) converged = 1;
  if (hs->status == STEP_FLOOR) converged = 2;
  if (hs->status == STEP_EPS) converged = 3;
  KR_CUDA(ctx, cudaEventRecord(ev[4], ctx->stream));
  // final sampled objective at the returned x (FP64 accumulation)
  KR_TRY(sampled_pass(ctx, m, &sk, bf, nblk, false, &op, &on));
  KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, op, on, 1, 0, bf.red);
  KR_LAUNCH(ctx, k_dot_self, ublk, 256, 0, bf.x, R, bf.part + 1024);
  KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, bf.part + 1024, ublk, 1, 0, bf.red + 1);
  KR_CUDA(ctx, cudaMemcpyAsync(h, bf.red, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaEventRecord(ev[5], ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  sk.distinct = (int64_t)(*(const unsigned long long*)((const char*)ctx->hbuf + KR_HBUF_DISTINCT));
  if (rep) {
    rep->iters = it;
    rep->converged = converged;
    rep->s = cfg.s;
    rep->distinct = sk.distinct;
    rep->obj_sampled = h[0] + cfg.lambda * h[1];
    rep->rel_update = rel;
    float ms;
    cudaEventElapsedTime(&ms, ev[0], ev[1]); rep->t_ms[0] = ms;
    cudaEventElapsedTime(&ms, ev[1], ev[2]); rep->t_ms[1] = ms;  // sample + group + gather
    rep->t_ms[2] = 0.f;
    cudaEventElapsedTime(&ms, ev[2], ev[3]); rep->t_ms[3] = ms;
    cudaEventElapsedTime(&ms, ev[3], ev[4]); rep->t_ms[4] = ms;
    cudaEventElapsedTime(&ms, ev[4], ev[5]); rep->t_ms[5] = ms;
    cudaEventElapsedTime(&ms, ev[0], ev[5]); rep->t_ms[7] = ms;
    rep->iters_reduced = iters_reduced;
    rep->precision_used = prec1;
  }
  if (st != KR_OK) return st;
  if (!converged) return kr_fail(ctx, KR_ENOTCONV, "no convergence within %d iterations (rel step %.3e)", cfg.max_iter, rel);
  return KR_OK;
}

namespace {

int64_t default_samples(const kr_opts* o, int64_t R) {
  return o->num_samples > 0 ? o->num_samples : kr_sample_count(R, o->eps, o->sample_scale);
}

// The solvers' argument checks and configuration (shared by the synchronous and the
// asynchronous entry points).
kr_status solve_setup(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* o, float* x, double lambda,
                      Modes* mp, SolveCfg* cp) {
  if (!ctx) return KR_EINVAL;
  if (!o || !b || !x) return kr_fail(ctx, KR_EINVAL, "solver: null opts, b or x");
  Modes& m = *mp;
  KR_TRY(kr_check_factors(ctx, f, &m));
  if (!(o->eps > 0.0 && o->eps < 1.0)) return kr_fail(ctx, KR_EINVAL, "solver: eps=%g outside (0,1)", o->eps);
  if (o->precision < 0 || o->precision > 2)
    return kr_fail(ctx, KR_EINVAL, "solver: precision=%d (0 FP32, 1 BF16, 2 FP8 e4m3)", o->precision);
  if (o->partition_T != 0 && o->partition_T != -1 && o->partition_T != (1 << (m.N - 1)))
    return kr_fail(ctx, KR_ENOTIMPL, "solver: partition_T=0x%x (only the last mode, 0x%x, is built)", o->partition_T,
                   1 << (m.N - 1));
  {
    int cur = -1;
    KR_CUDA(ctx, cudaGetDevice(&cur));
    if (cur != ctx->device)
      return kr_fail(ctx, KR_EINVAL, "solver: current device %d is not the context's device %d", cur, ctx->device);
  }
  if (!(lambda >= 0.0) || !isfinite(lambda)) return kr_fail(ctx, KR_EINVAL, "solver: lambda must be finite and >= 0");
  SolveCfg& cfg = *cp;
  cfg.lambda = lambda;
  cfg.eps = o->eps;
  cfg.alpha = o->step > 0 ? o->step : 1.0 - sqrt(o->eps);
  cfg.tol = o->tol > 0 ? o->tol : 1e-7;
  cfg.max_iter = o->max_iter > 0 ? o->max_iter : 100;
  if (o->stop_rule != 0 && o->stop_rule != 1) return kr_fail(ctx, KR_EINVAL, "solver: stop_rule must be 0 or 1");
  cfg.stop_rule = o->stop_rule;
  cfg.theta = o->theta > 0 ? o->theta : 0.01;
  cfg.prec = o->precision;
  cfg.s = default_samples(o, kr_prod_R(m));
  return KR_OK;
}

kr_status solve_entry(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* o, float* x, kr_report* rep,
                      double lambda) {
  Modes m;
  SolveCfg cfg;
  KR_TRY(solve_setup(ctx, f, b, o, x, lambda, &m, &cfg));
  const int64_t R = kr_prod_R(m), I = kr_prod_I(m);
  if (rep) *rep = kr_report{};
  if (!o->host_io) return kr_solve_device(ctx, m, b, cfg, o->seed, o->call_id, x, rep);
  // host buffers: copy factors and b in, x out, inside the call
  cudaEvent_t e0 = ctx->ev[6], e1 = ctx->ev[7];
  // b in page-locked host memory is mapped into the device's address space: the gather reads
  // the s sampled entries in place (Alg. 2 reads b only at the sampled rows) instead of
  // copying all prod I entries, and no device copy of b is needed
  const float* b_mapped = nullptr;
  if (ctx->host_gather) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, b) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
      b_mapped = static_cast<const float*>(pa.devicePointer);
    else
      cudaGetLastError();  // not page-locked: copy it
  }
  size_t bytes = 0;
  for (int n = 0; n < m.N; ++n) bytes += ((size_t)m.I[n] * m.R[n] * 4 + 255) & ~size_t(255);
  bytes += ((size_t)R * 4 + 255) & ~size_t(255);
  if (!b_mapped) bytes += ((size_t)I * 4 + 255) & ~size_t(255);
  KR_TRY(kr_io_reserve(ctx, bytes));
  char* dev = ctx->io;
  KR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
  Carve cv(dev, bytes);
  Modes md = m;
  for (int n = 0; n < m.N; ++n) {
    float* a = cv.take<float>((size_t)m.I[n] * m.R[n]);
    KR_CUDA(ctx, cudaMemcpyAsync(a, m.A[n], sizeof(float) * m.I[n] * m.R[n], cudaMemcpyHostToDevice, ctx->stream));
    md.A[n] = a;
  }
  float* xd = cv.take<float>(R);
  float* bd = b_mapped ? nullptr : cv.take<float>(I);
  if (b_mapped) {
    kr_status st = kr_solve_device(ctx, md, b_mapped, cfg, o->seed, o->call_id, xd, rep);
    if (st == KR_OK || st == KR_ENOTCONV) {
      KR_CUDA(ctx, cudaMemcpyAsync(x, xd, sizeof(float) * R, cudaMemcpyDeviceToHost, ctx->stream));
    }
    KR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (rep) {
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      rep->t_ms[6] = ms - rep->t_ms[7];
      rep->t_ms[7] = ms;
    }
    return st;
  }
  // b on the copy stream, overlapping the tables, draws and sort of the solve stream; the
  // gather waits for it
  if (!ctx->copy_stream) {
    KR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    KR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->b_ready, cudaEventDisableTiming));
  }
  // after the factors: copies in one direction share the copy engine, and the solve stream's
  // first kernels need the factors, not b
  KR_CUDA(ctx, cudaEventRecord(ctx->b_ready, ctx->stream));
  KR_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->b_ready, 0));
  KR_CUDA(ctx, cudaMemcpyAsync(bd, b, sizeof(float) * I, cudaMemcpyHostToDevice, ctx->copy_stream));
  KR_CUDA(ctx, cudaEventRecord(ctx->b_ready, ctx->copy_stream));
  ctx->b_wait = ctx->b_ready;
  kr_status st = kr_solve_device(ctx, md, bd, cfg, o->seed, o->call_id, xd, rep);
  ctx->b_wait = nullptr;
  // the staging buffer is reused by the next call: order it after the copy in every case
  KR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->b_ready, 0));
  if (st == KR_OK || st == KR_ENOTCONV) {
    KR_CUDA(ctx, cudaMemcpyAsync(x, xd, sizeof(float) * R, cudaMemcpyDeviceToHost, ctx->stream));
  }
  KR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rep) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    rep->t_ms[6] = ms - rep->t_ms[7];
    rep->t_ms[7] = ms;
  }
  return st;
}

}  // namespace

extern "C" kr_status kron_regress(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts, float* x,
                                  kr_report* report) {
  return solve_entry(ctx, f, b, opts, x, report, 0.0);
}

extern "C" kr_status kron_ridge(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts, float* x,
                                kr_report* report) {
  if (!ctx) return KR_EINVAL;
  if (!opts || !(opts->lambda > 0.0)) return kr_fail(ctx, KR_EINVAL, "kron_ridge: opts->lambda must be > 0");
  return solve_entry(ctx, f, b, opts, x, report, opts->lambda);
}

namespace {

kr_status solve_async(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* o, float* x,
                      kr_dev_report* report, double lambda) {
  Modes m;
  SolveCfg cfg;
  KR_TRY(solve_setup(ctx, f, b, o, x, lambda, &m, &cfg));
  if (!report) return kr_fail(ctx, KR_EINVAL, "asynchronous solve: null report");
  if (o->host_io) return kr_fail(ctx, KR_EINVAL, "asynchronous solve: device pointers only (host_io must be 0)");
  if (ctx->gm.on) return kr_fail(ctx, KR_EINVAL, "asynchronous solve: the context is capturing a sweep");
  if (!ctx->gm_async || !ctx->side_stream) return kr_fail(ctx, KR_ENOMEM, "asynchronous solve: no device state");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  KR_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs == cudaStreamCaptureStatusInvalidated)
    return kr_fail(ctx, KR_EINVAL, "asynchronous solve: the stream's capture has been invalidated");
  if (cs == cudaStreamCaptureStatusNone && (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy))
    return kr_fail(ctx, KR_EINVAL, "asynchronous solve: the legacy default stream cannot run its loop graphs");
  // the device state: error word, two loop slots, objective, final state, distinct count
  char* d = static_cast<char*>(ctx->gm_async);
  kr_ctx::GraphMode& g = ctx->gm;
  g = kr_ctx::GraphMode();
  g.err = reinterpret_cast<int*>(d);
  g.status = reinterpret_cast<int*>(d + 16);
  g.obj = reinterpret_cast<double*>(d + 32);
  g.distinct = reinterpret_cast<unsigned long long*>(d + 48);
  g.last = d + 64;
  g.nstatus = 2;
  g.report = report;
  g.capturing = cs == cudaStreamCaptureStatusActive;
  g.on = true;
  const int timing = ctx->timing;
  ctx->timing = 0;  // nothing is timed or read back
  kr_status st = KR_OK;
  const cudaError_t e = cudaMemsetAsync(g.err, 0, 16, ctx->stream);
  if (e != cudaSuccess) st = kr_fail_cuda(ctx, e, "asynchronous solve: state reset", __FILE__, __LINE__);
  if (st == KR_OK) st = kr_solve_device(ctx, m, b, cfg, o->seed, o->call_id, x, nullptr);
  ctx->timing = timing;
  g = kr_ctx::GraphMode();
  return st;
}

}  // namespace

extern "C" kr_status kron_regress_async(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts,
                                        float* x, kr_dev_report* report) {
  return solve_async(ctx, f, b, opts, x, report, 0.0);
}

extern "C" kr_status kron_ridge_async(kr_ctx* ctx, const kr_factors* f, const float* b, const kr_opts* opts, float* x,
                                      kr_dev_report* report) {
  if (!ctx) return KR_EINVAL;
  if (!opts || !(opts->lambda > 0.0)) return kr_fail(ctx, KR_EINVAL, "kron_ridge_async: opts->lambda must be > 0");
  return solve_async(ctx, f, b, opts, x, report, opts->lambda);
}

// Worker contexts for concurrent problems: a context each, on its own non-blocking stream,
// created on first use and kept by `ctx`; options follow ctx's.
static kr_status kr_workers_reserve(kr_ctx* ctx, int n) {
  while ((int)ctx->workers.size() < n) {
    cudaStream_t s = nullptr;
    KR_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    kr_ctx* w = nullptr;
    const kr_status st = kr_create(&w, s, 0);
    if (st != KR_OK) {
      cudaStreamDestroy(s);
      return kr_fail(ctx, st, "kron_ridge_batched: worker context creation failed");
    }
    ctx->workers.push_back(w);
    ctx->worker_streams.push_back(s);
  }
  for (int i = 0; i < n; ++i) {
    kr_ctx* w = ctx->workers[i];
    w->slab_pass = ctx->slab_pass;
    w->slab_tile_entries = ctx->slab_tile_entries;
    w->device_loop = ctx->device_loop;
    w->grouping = ctx->grouping;
    w->host_gather = ctx->host_gather;
    w->jl_k = ctx->jl_k;
    w->jl_seed = ctx->jl_seed;
    w->tensor_cores = ctx->tensor_cores;
    w->autotune = ctx->autotune;
    if (ctx->autotune && !ctx->tune) kr_tune_lookup(ctx, nullptr);  // creates ctx's table
    if (w->tune_owned) kr_tune_free(w);
    w->tune = ctx->tune;  // one table for the batch
    w->shared_loop = nullptr;
    w->timing = false;
  }
  return KR_OK;
}

// Fused batch (KR_OPT_BATCH_MODE 1): a context and a host thread per problem. Every problem
// builds its tables, sketch and tiles concurrently on its own stream and takes its first
// Richardson step; the problems' remaining steps (device-side conditional loops) then run as
// the concurrent nodes of one CUDA graph, launched once on ctx's stream (kr_shared_loop_run),
// and every problem ends with its own final objective check. Each problem runs the kernels of
// its single solve in the same order, so its result is bit-identical to that solve's.
static kr_status batched_fused(kr_ctx* ctx, int32_t nprob, const kr_factors* probs, const float* const b[],
                               const kr_opts* opts, float* const x[], kr_report* reports) {
  KR_TRY(kr_workers_reserve(ctx, nprob));
  kr_shared_loop* sl = kr_shared_loop_new(ctx->stream, nprob);
  for (int p = 0; p < nprob; ++p) {
    kr_ctx* w = ctx->workers[p];
    w->shared_loop = sl;
    if (w->grouping == 0) w->grouping = 2;  // key bitmap: no 4 GB dense counters per context
  }
  KR_CUDA(ctx, cudaEventRecord(ctx->ev[9], ctx->stream));
  for (int p = 0; p < nprob; ++p) KR_CUDA(ctx, cudaStreamWaitEvent(ctx->worker_streams[p], ctx->ev[9], 0));
  std::vector<kr_status> st(nprob, KR_OK);
  std::vector<std::string> msg(nprob);
  std::vector<int64_t> l0(nprob);
  for (int p = 0; p < nprob; ++p) l0[p] = ctx->workers[p]->launches;
  auto run = [&](int p) {
    kr_ctx* w = ctx->workers[p];
    const cudaError_t de = cudaSetDevice(ctx->device);
    if (de != cudaSuccess) {
      st[p] = KR_ECUDA;
      msg[p] = std::string("kron_ridge_batched: cudaSetDevice failed in a worker: ") + cudaGetErrorString(de);
    } else {
      kr_opts o = *opts;
      o.call_id = opts->call_id + (uint64_t)p;
      st[p] = solve_entry(w, &probs[p], b[p], &o, x[p], reports ? &reports[p] : nullptr, opts->lambda);
      if (st[p] != KR_OK) msg[p] = w->err;
    }
    kr_shared_loop_leave(sl);  // in every case: the other problems do not wait for this one
  };
  std::vector<std::thread> pool;
  for (int p = 1; p < nprob; ++p) pool.emplace_back(run, p);
  run(0);
  for (auto& t : pool) t.join();
  kr_shared_loop_delete(sl);
  for (int p = 0; p < nprob; ++p) {
    ctx->workers[p]->shared_loop = nullptr;
    ctx->launches += ctx->workers[p]->launches - l0[p];
  }
  kr_status worst = KR_OK;
  for (int p = 0; p < nprob; ++p) {
    if (st[p] != KR_OK && st[p] != KR_ENOTCONV) {
      ctx->err = msg[p];
      return st[p];
    }
    if (st[p] == KR_ENOTCONV && worst == KR_OK) {
      worst = KR_ENOTCONV;
      ctx->err = msg[p];
    }
  }
  return worst;
}

extern "C" kr_status kron_ridge_batched(kr_ctx* ctx, int32_t nprob, const kr_factors* probs, const float* const b[],
                                        const kr_opts* opts, float* const x[], kr_report* reports) {
  if (!ctx) return KR_EINVAL;
  if (nprob < 0 || (nprob > 0 && (!probs || !b || !x || !opts)))
    return kr_fail(ctx, KR_EINVAL, "kron_ridge_batched: bad arguments");
  if (ctx->batch_mode == 1 && nprob > 1) return batched_fused(ctx, nprob, probs, b, opts, x, reports);
  const int W = nprob < ctx->batch_workers ? nprob : ctx->batch_workers;
  if (W <= 1) {  // one after another on ctx's stream
    kr_status worst = KR_OK;
    for (int p = 0; p < nprob; ++p) {
      kr_opts o = *opts;
      o.call_id = opts->call_id + (uint64_t)p;
      kr_status st = solve_entry(ctx, &probs[p], b[p], &o, x[p], reports ? &reports[p] : nullptr, opts->lambda);
      if (st != KR_OK && st != KR_ENOTCONV) return st;
      if (st != KR_OK) worst = st;
    }
    return worst;
  }
  KR_TRY(kr_workers_reserve(ctx, W));
  // the problems' inputs may come from work enqueued on ctx's stream
  KR_CUDA(ctx, cudaEventRecord(ctx->ev[9], ctx->stream));
  for (int i = 0; i < W; ++i) KR_CUDA(ctx, cudaStreamWaitEvent(ctx->worker_streams[i], ctx->ev[9], 0));
  std::vector<kr_status> st(nprob, KR_OK);
  std::vector<std::string> msg(nprob);
  std::atomic<int> next{0};
  std::vector<int64_t> l0(W);
  for (int i = 0; i < W; ++i) l0[i] = ctx->workers[i]->launches;
  auto run = [&](int wi) {
    kr_ctx* w = ctx->workers[wi];
    // a new host thread starts on device 0: make the context's device current first
    const cudaError_t de = cudaSetDevice(ctx->device);
    for (;;) {
      const int p = next.fetch_add(1);
      if (p >= nprob) break;
      if (de != cudaSuccess) {
        st[p] = KR_ECUDA;
        msg[p] = std::string("kron_ridge_batched: cudaSetDevice failed in a worker: ") + cudaGetErrorString(de);
        continue;
      }
      kr_opts o = *opts;
      o.call_id = opts->call_id + (uint64_t)p;
      st[p] = solve_entry(w, &probs[p], b[p], &o, x[p], reports ? &reports[p] : nullptr, opts->lambda);
      if (st[p] != KR_OK) msg[p] = w->err;
    }
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < W; ++i) pool.emplace_back(run, i);
  run(0);
  for (auto& t : pool) t.join();
  for (int i = 0; i < W; ++i) ctx->launches += ctx->workers[i]->launches - l0[i];
  kr_status worst = KR_OK;
  for (int p = 0; p < nprob; ++p) {
    if (st[p] != KR_OK && st[p] != KR_ENOTCONV) {
      ctx->err = msg[p];
      return st[p];
    }
    if (st[p] == KR_ENOTCONV && worst == KR_OK) {
      worst = KR_ENOTCONV;
      ctx->err = msg[p];
    }
  }
  return worst;
}

extern "C" kr_status kron_sketch_residual(kr_ctx* ctx, const kr_sketch* sk, const kr_factors* f, const float* x,
                                          float* g, double* obj) {
  if (!ctx || !sk || !x || !g) return KR_EINVAL;
  Modes m;
  KR_TRY(kr_check_factors(ctx, f, &m));
  if (m.N != sk->N) return kr_fail(ctx, KR_EINVAL, "kron_sketch_residual: N mismatch");
  for (int n = 0; n < m.N; ++n)
    if (m.I[n] != sk->I[n]) return kr_fail(ctx, KR_EINVAL, "kron_sketch_residual: I mismatch");
  const int nblk = kr_resid_blocks(ctx);
  const int64_t mx = max_intermediate(m);
  const int RT = m.R[m.N - 1];
  Need nd;
  nd.add<float>(sk->ncell * RT);
  nd.add<float>(sk->ncell * RT);
  nd.add<float>(mx);
  nd.add<float>(mx);
  nd.add<double>(nblk);
  nd.add<double>(4);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  Carve cv(ctx->ws, ctx->ws_size);
  IterBufs bf;
  bf.x = const_cast<float*>(x);
  bf.Y = cv.take<float>(sk->ncell * RT);
  bf.W = cv.take<float>(sk->ncell * RT);
  bf.t0 = cv.take<float>(mx);
  bf.t1 = cv.take<float>(mx);
  bf.part = cv.take<double>(nblk);
  bf.red = cv.take<double>(4);
  bf.g = g;
  bf.d = nullptr;
  int used = 0;
  KR_TRY(forward_resid(ctx, m, sk, bf, nblk, &used));
  KR_TRY(backward(ctx, m, bf));
  KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, bf.part, used, 1, 0, bf.red);
  KR_CUDA(ctx, cudaMemcpyAsync(ctx->hbuf, bf.red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (obj) *obj = *(double*)ctx->hbuf;
  return KR_OK;
}

extern "C" kr_status kron_objective(kr_ctx* ctx, const kr_factors* f, const float* b, const float* x, double lambda,
                                    double* obj) {
  if (!ctx) return KR_EINVAL;
  if (!b || !x || !obj) return kr_fail(ctx, KR_EINVAL, "kron_objective: null argument");
  Modes m;
  KR_TRY(kr_check_factors(ctx, f, &m));
  const int N = m.N;
  const int64_t R = kr_prod_R(m), mx = max_intermediate(m);
  int64_t ncell = 1;
  for (int n = 0; n < N - 1; ++n) ncell *= m.I[n];
  const int RT = m.R[N - 1];
  const int nblk = ctx->num_sms * 2;
  Need nd;
  nd.add<float>(ncell * RT);
  nd.add<float>(mx);
  nd.add<float>(mx);
  nd.add<double>(nblk + 1024);
  nd.add<double>(4);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  Carve cv(ctx->ws, ctx->ws_size);
  float* Y = cv.take<float>(ncell * RT);
  float* t0 = cv.take<float>(mx);
  float* t1 = cv.take<float>(mx);
  double* part = cv.take<double>(nblk + 1024);
  double* red = cv.take<double>(4);
  int din[KR_MAX_MODES], dout[KR_MAX_MODES], tr[KR_MAX_MODES];
  const float* B[KR_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    din[n] = m.R[n];
    dout[n] = (n < N - 1) ? m.I[n] : m.R[n];
    B[n] = (n < N - 1) ? m.A[n] : nullptr;
    tr[n] = 0;
  }
  KR_TRY(kr_kron_apply2(ctx, N, din, dout, B, tr, x, Y, t0, t1));
  {
    const size_t smA = (size_t)m.I[N - 1] * (RT + 1) * sizeof(float), smY = (size_t)FULL_CELLS * RT * sizeof(float);
    if (smA + smY <= ctx->smem_optin) {
      KR_TRY(kr_smem_attr(ctx, k_full_obj<true>, smA + smY));
      KR_LAUNCH(ctx, k_full_obj<true>, nblk, 256, smA + smY, Y, m.A[N - 1], b, ncell, m.I[N - 1], RT, part);
    } else {
      KR_LAUNCH(ctx, k_full_obj<false>, nblk, 256, smY, Y, m.A[N - 1], b, ncell, m.I[N - 1], RT, part);
    }
  }
  KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, part, nblk, 1, 0, red);
  const int ublk = grid_cap(ctx, R, 256, 4);
  KR_LAUNCH(ctx, k_dot_self, ublk, 256, 0, x, R, part + nblk);
  KR_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, part + nblk, ublk, 1, 0, red + 1);
  KR_CUDA(ctx, cudaMemcpyAsync(ctx->hbuf, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double* h = (double*)ctx->hbuf;
  *obj = h[0] + lambda * h[1];
  return KR_OK;
}
