// a6-a8 fused: the sampled products of one Richardson step of Alg. 2 (Thm 4.4 with
// T = the last mode), evaluated slab by slab.
//
// With x read as an R_1 x ... x R_N tensor, cells c = (i_1..i_{N-1}) and slabs
// p = (i_1..i_{N-2}), the step needs
//   X1 = X x_1 A(1) ... x_{N-2} A(N-2)                         (P x R_{N-1} x R_N)
//   Y[p, i]  = sum_r A(N-1)[i, r] X1[p, r, :]                    (one R_N row per cell)
//   r_j      = omega_j (b~_j - <A(N)[i_j], Y[c_j]>)              (per distinct sampled row)
//   W[p, i]  = sum_{j in cell (p, i)} r_j A(N)[i_j]
//   Z[p]     = sum_i A(N-1)[i, :]^T W[p, i]                      (R_{N-1} x R_N)
// and then g = Z x_1 A(1)^T ... x_{N-2} A(N-2)^T. Only cells holding sampled rows
// contribute, so Y and W exist only for those, and only inside one kernel: a tile (a
// run of non-empty cells of one slab) forms its Y rows in shared memory from X1[p],
// walks its entries, accumulates W in place of Y, and contracts W with the tile's rows
// of A(N-1) into the slab's Z. The two large mode products of the unfused form (to and
// from the cells x R_N intermediates) and their HBM round trips disappear.
//
// Loads that stream (the entry stream, b~) or that other tiles re-read from L2 (X1[p], rows
// of A(N-1)) bypass L1, which keeps the rows of A(N) the walk gathers when A(N) is not held
// in shared memory.
// A persistent CTA holds A(N) and 1/p_N in shared memory once and runs two teams of 256
// threads, each taking tiles from a global counter in decreasing-work order. Inside a
// tile, the entries (contiguous in cell order) are split into equal segments, one per
// lane group of G lanes; a group that starts inside a cell owned by an earlier group
// keeps that cell's partial W apart, and the partials are added to the owner's W in
// group order afterwards. Every sum has a fixed order, so the pass is deterministic.
// Slabs split over several tiles are completed by the last of their tiles to finish,
// which adds the tiles' contributions in tile order.
#include <cuda_bf16.h>

#include "kr_internal.cuh"

namespace {

constexpr int SLAB_TEAM = 256;
constexpr int SLAB_TEAMS = 2;
constexpr int SLAB_D = 4;  // chunks of G entries in flight per lane

template <int RTP>
struct SlabShape {
  static constexpr int COLS = RTP < 16 ? RTP : 16;  // columns of a row held by one lane
  static constexpr int G = RTP / COLS;              // lanes per group
  static constexpr int NQ = COLS / 4;               // float4 quads per lane
  static constexpr int NG = SLAB_TEAM / G;          // groups per team
  static constexpr int CB = (SLAB_TEAM >= 256 ? 128 : 64) >> (RTP >= 64 ? 1 : 0);  // cells per tile at most
  static constexpr int PF = SLAB_TEAM * COLS;       // floats of the partial buffer (NG x RTP)
};

int rt_pad(int RT) {
  int r = 4;
  while (r < RT) r <<= 1;
  return r;
}
int cb_for(int RTP) { return (SLAB_TEAM >= 256 ? 128 : 64) >> (RTP >= 64 ? 1 : 0); }

struct SlabArgs {
  const uint4* act;
  const uint4* tsort;  // per processing slot: {first cell, tile, slab, entries | (cells - 1) << 24 | multi << 31}
  uint32_t* meta;
  const uint32_t* ent;
  const float* bt;
  const float* invpT;
  const float* AT;  // IT x RT
  const float* A2;  // I2 x R2
  const float* X1;  // P x R2 x RT
  float* zpart;     // ntmax x R2 x RT
  double* objpart;  // ntmax
  int IT, RT, I2, R2, R2P, R2S;
  int mma, XS;  // Y and Z on tensor cores (3xTF32); row stride of the split X1[p] (floats)
  int64_t P;
  int a2vec, atvec;
  int zero_x;    // X1 is zero (the first Richardson step): Y = 0, the residual is b~
  int obj_only;  // only the objective is wanted: no W accumulation, no Z
  // shared-memory layout (bytes)
  uint32_t team_off, team_bytes, o_a2, o_x1, o_pf, o_act, o_cs, o_ctl;
};

__device__ __forceinline__ void team_sync(int team) {
  asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(SLAB_TEAM) : "memory");
}

// FP32-accurate products on the TF32 tensor path: x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi), and a.b ~ a_hi.b_hi + a_hi.b_lo + a_lo.b_hi (the dropped lo.lo term is
// below FP32 rounding), each an m16n8k8 TF32 MMA with FP32 accumulation.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_tf32x3(float* c, const uint32_t* ah, const uint32_t* al, const uint32_t* bh,
                                           const uint32_t* bl) {
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}

// Reduced-precision products (kr_opts.precision 1 and 2): one BF16 m16n8k16 MMA, or one
// FP8 (e4m3) m16n8k32 MMA whose operands are scaled per row of the non-contracted index
// (the scales factor out of the sum and multiply the FP32 result), FP32 accumulation.
// Pairs and quads pack the element with the smaller k index in the low bits.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// e4m3 pair with saturation to +-448: the first source goes to the high byte
__device__ __forceinline__ uint32_t cvt_e4m3x2(float hi, float lo) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t pack_e4m3(float x0, float x1, float x2, float x3) {
  return cvt_e4m3x2(x1, x0) | (cvt_e4m3x2(x3, x2) << 16);
}
__device__ __forceinline__ void mma_e4m3(float* c, const uint32_t* a, const uint32_t* b) {
  asm("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
constexpr float E4M3_MAX = 448.f;
// k steps of one MMA and the cell padding of the tile's Z product, per precision
template <int PREC>
struct PrecShape {
  static constexpr int KS = PREC == 0 ? 8 : (PREC == 1 ? 16 : 32);
};

// Row `it` of A(N), the lane's quads qd[v] (zero past R_N).
template <int RTP, bool SMEM_A>
__device__ __forceinline__ void load_arow(const SlabArgs& a, const float* sA, int it, const int* qd, float4* av) {
  constexpr int NQ = SlabShape<RTP>::NQ;
  if (SMEM_A) {
    const float4* row = reinterpret_cast<const float4*>(sA + (size_t)it * RTP);
#pragma unroll
    for (int v = 0; v < NQ; ++v) av[v] = row[qd[v]];
  } else if (a.atvec) {
    const float4* row = reinterpret_cast<const float4*>(a.AT + (size_t)it * a.RT);
#pragma unroll
    for (int v = 0; v < NQ; ++v) av[v] = 4 * qd[v] < a.RT ? __ldg(row + qd[v]) : make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    const float* row = a.AT + (size_t)it * a.RT;
#pragma unroll
    for (int v = 0; v < NQ; ++v) {
      const int c = 4 * qd[v];
      av[v].x = c + 0 < a.RT ? __ldg(row + c + 0) : 0.f;
      av[v].y = c + 1 < a.RT ? __ldg(row + c + 1) : 0.f;
      av[v].z = c + 2 < a.RT ? __ldg(row + c + 2) : 0.f;
      av[v].w = c + 3 < a.RT ? __ldg(row + c + 3) : 0.f;
    }
  }
}

// <A(N) row, y> over this lane's quads: one FMA chain per quad, chains added pairwise.
template <int NQ>
__device__ __forceinline__ float dot_quads(const float4* av, const float* y) {
  float c[NQ];
#pragma unroll
  for (int v = 0; v < NQ; ++v) {
    c[v] = av[v].x * y[4 * v];
    c[v] = fmaf(av[v].y, y[4 * v + 1], c[v]);
    c[v] = fmaf(av[v].z, y[4 * v + 2], c[v]);
    c[v] = fmaf(av[v].w, y[4 * v + 3], c[v]);
  }
  if (NQ == 4) return (c[0] + c[1]) + (c[2 % NQ] + c[3 % NQ]);
  if (NQ == 2) return c[0] + c[1 % NQ];
  return c[0];
}

template <int NQ>
__device__ __forceinline__ void axpy_quads(float rr, const float4* av, float* w) {
#pragma unroll
  for (int v = 0; v < NQ; ++v) {
    w[4 * v + 0] = fmaf(rr, av[v].x, w[4 * v + 0]);
    w[4 * v + 1] = fmaf(rr, av[v].y, w[4 * v + 1]);
    w[4 * v + 2] = fmaf(rr, av[v].z, w[4 * v + 2]);
    w[4 * v + 3] = fmaf(rr, av[v].w, w[4 * v + 3]);
  }
}

// Sum over the G lanes of a group (the mask names the group only, so the call may sit
// in control flow that is uniform per group but not per warp).
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned gmask) {
#pragma unroll
  for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(gmask, v, off);
  return v;
}

// One sampled row against the current cell: r = omega (b~ - <a, y>), w += r a (and the
// objective term r (b~ - <a, y>) when OBJ).
// zx: y is zero (the product is skipped; the residual is b~ exactly as with the product);
// wskip: the objective only (no W accumulation). Both are uniform over the kernel.
template <int RTP, bool SMEM_A, bool OBJ>
__device__ __forceinline__ void slab_entry(const SlabArgs& a, const float* sA, const float* sInvp, const int* qd,
                                           unsigned gmask, uint32_t e, float bj, float cw, const float* y, float* w,
                                           float& objc, bool zx, bool wskip) {
  using S = SlabShape<RTP>;
  const int it = (int)(e & 0xFFFFu);
  float4 av[S::NQ];
  load_arow<RTP, SMEM_A>(a, sA, it, qd, av);
  const float pr = zx ? 0.f : group_sum<S::G>(dot_quads<S::NQ>(av, y), gmask);
  const float om = (float)(e >> 16) * cw * sInvp[it];  // 0 past the segment (count 0)
  const float res = bj - pr;
  const float rr = om * res;
  if (!wskip) axpy_quads<S::NQ>(rr, av, w);
  if (OBJ) objc = fmaf(rr, res, objc);
}

// Cell k ends: its W goes to the cell's row (owned) or to the group's partial slot (the
// cell began in an earlier group's segment); the walk moves to cell k + 1.
template <int RTP, bool OBJ>
__device__ __forceinline__ void slab_next_cell(float* sYW, float* sPf, const uint32_t* sCS, const uint4* sAct,
                                               uint32_t e0, int q, const int* qd, int& k, uint32_t& nb, float& cw,
                                               bool& foreign, float* y, float* w, float& objc, double& objt) {
  using S = SlabShape<RTP>;
  float* dst = foreign ? (sPf + q * RTP) : (sYW + k * RTP);
#pragma unroll
  for (int v = 0; v < S::NQ; ++v)
    reinterpret_cast<float4*>(dst)[qd[v]] = make_float4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
  if (OBJ) {
    objt += (double)objc;
    objc = 0.f;
  }
  ++k;
  nb = sCS[k + 1] - e0;
  cw = __uint_as_float(sAct[k].w);
  foreign = false;
#pragma unroll
  for (int v = 0; v < S::NQ; ++v) {
    const float4 t4 = reinterpret_cast<const float4*>(sYW + k * RTP)[qd[v]];
    y[4 * v + 0] = t4.x;
    y[4 * v + 1] = t4.y;
    y[4 * v + 2] = t4.z;
    y[4 * v + 3] = t4.w;
  }
#pragma unroll
  for (int c = 0; c < S::COLS; ++c) w[c] = 0.f;
}

template <int RTP, bool SMEM_A, bool OBJ, int PREC>
__global__ void __launch_bounds__(SLAB_TEAM* SLAB_TEAMS, 1) k_slab(SlabArgs a) {
  using S = SlabShape<RTP>;
  constexpr int COLS = S::COLS, G = S::G, NQ = S::NQ, NG = S::NG;
  constexpr int XQ = RTP / 4;
  constexpr int NT8 = RTP >= 8 ? RTP / 8 : 1;   // n tiles of the tensor-core products
  constexpr int KS = PrecShape<PREC>::KS;       // k of one MMA: cells are padded to it
  const bool mma = RTP >= 8 && a.mma;
  extern __shared__ float4 slab_smem[];
  char* sm = reinterpret_cast<char*>(slab_smem);
  float* sA = reinterpret_cast<float*>(sm);
  float* sInvp = sA + (SMEM_A ? (size_t)a.IT * RTP : 0);
  const int RT = a.RT, R2 = a.R2, R2P = a.R2P, R2S = a.R2S;
  const int zn = R2 * RT;
  if (SMEM_A) {
    if (a.atvec && RT == RTP) {  // rows already padded: a straight float4 copy
      const float4* src = reinterpret_cast<const float4*>(a.AT);
      float4* dst = reinterpret_cast<float4*>(sA);
      const int n4 = a.IT * (RTP / 4);
#pragma unroll 8
      for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
    } else {
      for (int e = threadIdx.x; e < a.IT * RTP; e += blockDim.x) {
        const int i = e / RTP, r = e - i * RTP;
        sA[e] = r < RT ? __ldg(a.AT + (size_t)i * RT + r) : 0.f;
      }
    }
  }
  for (int i = threadIdx.x; i < a.IT; i += blockDim.x) sInvp[i] = __ldg(a.invpT + i);
  __syncthreads();
  kr_pdl_trigger();
  kr_pdl_wait();  // X1 and the work counter come from the previous kernels

  const int team = threadIdx.x / SLAB_TEAM, tt = threadIdx.x % SLAB_TEAM;
  char* tb = sm + a.team_off + (size_t)team * a.team_bytes;
  float* sYW = reinterpret_cast<float*>(tb);
  float* sA2 = reinterpret_cast<float*>(tb + a.o_a2);
  float* sX1 = reinterpret_cast<float*>(tb + a.o_x1);
  float* sPf = reinterpret_cast<float*>(tb + a.o_pf);
  uint4* sAct = reinterpret_cast<uint4*>(tb + a.o_act);
  uint32_t* sCS = reinterpret_cast<uint32_t*>(tb + a.o_cs);
  uint32_t* sCtl = reinterpret_cast<uint32_t*>(tb + a.o_ctl);
  double* sRed = reinterpret_cast<double*>(tb + a.o_ctl + 32);
  const uint32_t ntiles = a.meta[0];
  const int lane = threadIdx.x & 31, wt = tt >> 5;
  const int q = tt / G, g = tt % G;
  const int gbase = lane - g;
  // Quads of a row handled by this lane, rotated so that the 8 lanes of a quarter warp
  // touch 8 different bank quads whatever rows they read (G = 2, 4).
  const int rot = (lane & 7) >> (G == 1 ? 0 : 1);
  int qd[NQ];
#pragma unroll
  for (int v = 0; v < NQ; ++v) qd[v] = g * NQ + ((v + rot) & (NQ - 1));

  // The leader claims the next processing slot one tile ahead, so only the descriptor
  // load (one round trip) sits between two tiles.
  uint32_t nk = 0;
  if (tt == 0) nk = atomicAdd(&a.meta[2], 1u);
  for (;;) {
    if (tt == 0) {
      const uint4 d = nk < ntiles ? a.tsort[nk] : make_uint4(0u, 0xFFFFFFFFu, 0u, 0u);
      *reinterpret_cast<uint4*>(sCtl + 4) = d;
      if (nk < ntiles) nk = atomicAdd(&a.meta[2], 1u);
    }
    team_sync(team);
    const uint4 td = *reinterpret_cast<const uint4*>(sCtl + 4);
    const uint32_t t = td.y;
    if (t == 0xFFFFFFFFu) break;
    const int na = (int)((td.w >> 24) & 0x7Fu) + 1;
    const int64_t p = td.z;
    const uint32_t E = td.w & 0xFFFFFFu;
    // ---- tile metadata, rows of A(N-1), X1[p]
    if (tt < na) {
      const uint4 ac = a.act[td.x + tt];
      sAct[tt] = ac;
      sCS[tt] = ac.y;
      if (tt == na - 1) sCS[na] = ac.y + ac.z;
    }
    team_sync(team);
    // rows of A(N-1) of the tile's cells, loaded by the whole team with four loads in flight
    // per thread; with the tensor-core products, rows past the last cell up to the next
    // multiple of the MMA's k are the padding of the Z product's last k step: zero in both
    // operands (A(N-1) rows here, W rows of sYW below), so they add exactly nothing
    const int nrow = mma ? ((na + KS - 1) & ~(KS - 1)) : na;
    if (a.a2vec) {
      const int q4 = R2P / 4, n4 = nrow * q4;
      for (int i0 = tt; i0 < n4; i0 += 4 * SLAB_TEAM) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * SLAB_TEAM;
          const int row = i / q4, k4 = i - row * q4;
          v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i < n4 && row < na && 4 * k4 < R2) {
            const uint32_t i2 = sAct[row].x % (uint32_t)a.I2;
            v[u] = __ldcg(reinterpret_cast<const float4*>(a.A2 + (size_t)i2 * R2) + k4);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * SLAB_TEAM;
          const int row = i / q4, k4 = i - row * q4;
          if (i < n4) *reinterpret_cast<float4*>(sA2 + row * R2S + 4 * k4) = v[u];
        }
      }
    } else {
      const int n1 = nrow * R2P;
      for (int i0 = tt; i0 < n1; i0 += 4 * SLAB_TEAM) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * SLAB_TEAM;
          const int row = i / R2P, k2 = i - row * R2P;
          v[u] = 0.f;
          if (i < n1 && row < na && k2 < R2) v[u] = __ldcg(a.A2 + (size_t)(sAct[row].x % (uint32_t)a.I2) * R2 + k2);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * SLAB_TEAM;
          const int row = i / R2P, k2 = i - row * R2P;
          if (i < n1) sA2[row * R2S + k2] = v[u];
        }
      }
    }
    for (int i = tt; i < (nrow - na) * RTP; i += SLAB_TEAM) sYW[na * RTP + i] = 0.f;
    if (!a.zero_x) {  // X1[p], staged for the Y product
      const float* xp = a.X1 + p * zn;
      if (PREC == 1 && mma) {
        // X1[p]^T in BF16: row c holds column c of X1[p] (r contiguous), XS32 words a row
        uint16_t* xt = reinterpret_cast<uint16_t*>(sX1);
        const int xs2 = 2 * (R2P / 2 + 4);
        for (int i = tt; i < R2P * RTP; i += SLAB_TEAM) {
          const int r = i / RTP, c = i % RTP;
          const float v = (r < R2 && c < RT) ? __ldcg(xp + r * RT + c) : 0.f;
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          xt[c * xs2 + r] = *reinterpret_cast<const uint16_t*>(&h);
        }
      } else if (PREC == 2 && mma) {
        // X1[p]^T in e4m3 with one scale per column c of X1[p] (the MMA's n index)
        float* xsc = sPf + S::CB;
        if (tt < RTP) {
          float m = 0.f;
          if (tt < RT)
            for (int r = 0; r < R2; ++r) m = fmaxf(m, fabsf(__ldcg(xp + r * RT + tt)));
          xsc[tt] = m > 0.f ? m / E4M3_MAX : 1.f;
        }
        team_sync(team);
        uint8_t* xt = reinterpret_cast<uint8_t*>(sX1);
        const int xs4 = 4 * (R2P / 4 + 4);
        for (int i = tt; i < R2P * RTP / 2; i += SLAB_TEAM) {
          const int r = (2 * i) / RTP, c = (2 * i) % RTP;  // two columns c, c + 1 of row r
          const float v0 = (r < R2 && c < RT) ? __ldcg(xp + r * RT + c) / xsc[c] : 0.f;
          const float v1 = (r < R2 && c + 1 < RT) ? __ldcg(xp + r * RT + c + 1) / xsc[c + 1] : 0.f;
          const uint32_t q = cvt_e4m3x2(v1, v0);
          xt[c * xs4 + r] = (uint8_t)(q & 0xFFu);
          xt[(c + 1) * xs4 + r] = (uint8_t)(q >> 8);
        }
      } else {  // FP32 X1[p] (split once into TF32 hi / lo planes, rows of XS floats, for the MMAs)
        uint32_t* xh = reinterpret_cast<uint32_t*>(sX1);
        uint32_t* xl = xh + R2P * a.XS;
        const int nx = R2P * RTP;
        for (int i0 = tt; i0 < nx; i0 += 8 * SLAB_TEAM) {
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * SLAB_TEAM;
            const int r = i / RTP, c = i % RTP;
            v[u] = (i < nx && r < R2 && c < RT) ? __ldcg(xp + r * RT + c) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * SLAB_TEAM;
            const int r = i / RTP, c = i % RTP;
            if (i < nx) {
              if (mma) tf32_split(v[u], xh[r * a.XS + c], xl[r * a.XS + c]);
              else sX1[i] = v[u];
            }
          }
        }
      }
    }
    team_sync(team);
    if (PREC == 2 && mma) {  // e4m3 scale of each row of A(N-1) in the tile (1 for padding rows)
      if (tt < nrow) {
        float m = 0.f;
        if (tt < na)
          for (int k2 = 0; k2 < R2; ++k2) m = fmaxf(m, fabsf(sA2[tt * R2S + k2]));
        sPf[tt] = m > 0.f ? m / E4M3_MAX : 1.f;
      }
      team_sync(team);
    }
    // ---- Y rows of the tile's cells: sYW[k] = A(N-1)[i_k] X1[p] (0 when X1 is)
    if (a.zero_x) {
      for (int i = tt; i < na * RTP; i += SLAB_TEAM) sYW[i] = 0.f;
    } else if (PREC != 0 && mma) {
      // one 16-row block of cells per warp, all RTP columns: A = rows of A(N-1) (a0 (g, k0),
      // a1 (g + 8, k0), a2 (g, k1), a3 (g + 8, k1)), B = X1[p]^T rows (b0 at k0, b1 at k1 of
      // column n = g), C as in the TF32 form; BF16: k0 = 2q.., k1 = 2q + 8..; e4m3: k0 =
      // 4q.., k1 = 4q + 16.. (g = lane / 4, q = lane % 4)
      const int fr = lane >> 2, fc = lane & 3;
      const uint32_t* xt = reinterpret_cast<const uint32_t*>(sX1);
      const int xs = PREC == 1 ? R2P / 2 + 4 : R2P / 4 + 4;  // words per X1^T row
      const float* xsc = sPf + S::CB;
      const int nmt = (na + 15) >> 4;
      for (int mt = wt; mt < nmt; mt += SLAB_TEAM / 32) {
        float acc[NT8][4];
#pragma unroll
        for (int nt = 0; nt < NT8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        const float* ar0 = sA2 + (16 * mt + fr) * R2S;
        const float* ar1 = ar0 + 8 * R2S;
        float is0 = 1.f, is1 = 1.f;
        if (PREC == 2) {
          is0 = 1.f / sPf[16 * mt + fr];
          is1 = 1.f / sPf[16 * mt + fr + 8];
        }
        for (int ks = 0; ks < R2P / KS; ++ks) {
          uint32_t af[4];
          if (PREC == 1) {
            const int k0 = 16 * ks + 2 * fc;
            af[0] = pack_bf16(ar0[k0], ar0[k0 + 1]);
            af[1] = pack_bf16(ar1[k0], ar1[k0 + 1]);
            af[2] = pack_bf16(ar0[k0 + 8], ar0[k0 + 9]);
            af[3] = pack_bf16(ar1[k0 + 8], ar1[k0 + 9]);
          } else {
            const int k0 = 32 * ks + 4 * fc;
            af[0] = pack_e4m3(ar0[k0] * is0, ar0[k0 + 1] * is0, ar0[k0 + 2] * is0, ar0[k0 + 3] * is0);
            af[1] = pack_e4m3(ar1[k0] * is1, ar1[k0 + 1] * is1, ar1[k0 + 2] * is1, ar1[k0 + 3] * is1);
            af[2] = pack_e4m3(ar0[k0 + 16] * is0, ar0[k0 + 17] * is0, ar0[k0 + 18] * is0, ar0[k0 + 19] * is0);
            af[3] = pack_e4m3(ar1[k0 + 16] * is1, ar1[k0 + 17] * is1, ar1[k0 + 18] * is1, ar1[k0 + 19] * is1);
          }
#pragma unroll
          for (int nt = 0; nt < NT8; ++nt) {
            // one k step is 32 bytes (8 words) of an X1^T row in both formats; b1 is 16 bytes on
            const uint32_t* xr = xt + (8 * nt + fr) * xs + 8 * ks + fc;
            const uint32_t bf[2] = {xr[0], xr[4]};
            if (PREC == 1) mma_bf16(acc[nt], af, bf);
            else mma_e4m3(acc[nt], af, bf);
          }
        }
        const int r0 = 16 * mt + fr, r1 = r0 + 8;
#pragma unroll
        for (int nt = 0; nt < NT8; ++nt) {
          const int c0 = 8 * nt + 2 * fc;
          float s00 = 1.f, s01 = 1.f, s10 = 1.f, s11 = 1.f;
          if (PREC == 2) {
            const float sr0 = sPf[r0], sr1 = sPf[r1];
            s00 = sr0 * xsc[c0];
            s01 = sr0 * xsc[c0 + 1];
            s10 = sr1 * xsc[c0];
            s11 = sr1 * xsc[c0 + 1];
          }
          if (r0 < na) *reinterpret_cast<float2*>(sYW + r0 * RTP + c0) = make_float2(acc[nt][0] * s00, acc[nt][1] * s01);
          if (r1 < na) *reinterpret_cast<float2*>(sYW + r1 * RTP + c0) = make_float2(acc[nt][2] * s10, acc[nt][3] * s11);
        }
      }
    } else if (mma) {
      // one 16-row block of cells per warp, all RTP columns: m16n8k8 fragments (A = rows of
      // A(N-1): a0 (g, q), a1 (g + 8, q), a2 (g, q + 4), a3 (g + 8, q + 4); B = X1[p]: b0 (q, g),
      // b1 (q + 4, g); C: (g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1) with g = lane / 4,
      // q = lane % 4: fr and fc below)
      const int fr = lane >> 2, fc = lane & 3;
      const uint32_t* xh = reinterpret_cast<const uint32_t*>(sX1);
      const uint32_t* xl = xh + R2P * a.XS;
      const int nmt = (na + 15) >> 4;
      for (int mt = wt; mt < nmt; mt += SLAB_TEAM / 32) {
        float acc[NT8][4];
#pragma unroll
        for (int nt = 0; nt < NT8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        const float* ar0 = sA2 + (16 * mt + fr) * R2S + fc;
        const float* ar1 = ar0 + 8 * R2S;
        for (int ks = 0; ks < R2P / 8; ++ks) {
          uint32_t ah[4], al[4];
          tf32_split(ar0[8 * ks], ah[0], al[0]);
          tf32_split(ar1[8 * ks], ah[1], al[1]);
          tf32_split(ar0[8 * ks + 4], ah[2], al[2]);
          tf32_split(ar1[8 * ks + 4], ah[3], al[3]);
          const uint32_t* bh0 = xh + (8 * ks + fc) * a.XS + fr;
          const uint32_t* bl0 = xl + (8 * ks + fc) * a.XS + fr;
#pragma unroll
          for (int nt = 0; nt < NT8; ++nt) {
            const uint32_t bh[2] = {bh0[8 * nt], bh0[8 * nt + 4 * a.XS]};
            const uint32_t bl[2] = {bl0[8 * nt], bl0[8 * nt + 4 * a.XS]};
            mma_tf32x3(acc[nt], ah, al, bh, bl);
          }
        }
        const int r0 = 16 * mt + fr, r1 = r0 + 8;
#pragma unroll
        for (int nt = 0; nt < NT8; ++nt) {
          if (r0 < na) *reinterpret_cast<float2*>(sYW + r0 * RTP + 8 * nt + 2 * fc) = make_float2(acc[nt][0], acc[nt][1]);
          if (r1 < na) *reinterpret_cast<float2*>(sYW + r1 * RTP + 8 * nt + 2 * fc) = make_float2(acc[nt][2], acc[nt][3]);
        }
      }
    } else {
      const int ncq = (na + 3) >> 2;
      for (int w = tt; w < ncq * XQ; w += SLAB_TEAM) {
        const int cq = w / XQ, xq = w % XQ;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
        for (int k4 = 0; k4 < R2P / 4; ++k4) {
          float4 av[4], xv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4*>(sA2 + (4 * cq + i) * R2S + 4 * k4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) xv[kk] = *reinterpret_cast<const float4*>(sX1 + (4 * k4 + kk) * RTP + 4 * xq);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ak[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              acc[i][0] = fmaf(ak[kk], xv[kk].x, acc[i][0]);
              acc[i][1] = fmaf(ak[kk], xv[kk].y, acc[i][1]);
              acc[i][2] = fmaf(ak[kk], xv[kk].z, acc[i][2]);
              acc[i][3] = fmaf(ak[kk], xv[kk].w, acc[i][3]);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (4 * cq + i < na)
            *reinterpret_cast<float4*>(sYW + (4 * cq + i) * RTP + 4 * xq) =
                make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
    }
    team_sync(team);
    // ---- walk: group q takes entries [j0, j1) of the tile
    const uint32_t e0 = sCS[0];
    const uint32_t L = (E + NG - 1) / NG;
    const uint32_t j0 = (uint32_t)q * L;
    const uint32_t j1 = min(j0 + L, E);
    const bool has = j0 < E;
    int k = 0;
    if (has) {  // last cell starting at or before j0
      int lo = 0, hi = na - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sCS[mid] - e0 <= j0) lo = mid;
        else hi = mid - 1;
      }
      k = lo;
    }
    uint32_t nb = sCS[k + 1] - e0;
    bool foreign = has && (sCS[k] - e0 < j0);
    float cw = __uint_as_float(sAct[k].w);
    float y[COLS], w[COLS];
#pragma unroll
    for (int v = 0; v < NQ; ++v) {
      const float4 t4 = reinterpret_cast<const float4*>(sYW + k * RTP)[qd[v]];
      y[4 * v + 0] = t4.x;
      y[4 * v + 1] = t4.y;
      y[4 * v + 2] = t4.z;
      y[4 * v + 3] = t4.w;
    }
#pragma unroll
    for (int c = 0; c < COLS; ++c) w[c] = 0.f;
    float objc = 0.f;
    double objt = 0.0;
    team_sync(team);  // every group holds its first y before owners overwrite Y with W
    const uint32_t nchunk = (L + G - 1) / G;
    const bool zx = a.zero_x != 0, wskip = a.obj_only != 0;
    const uint32_t* ent = a.ent + e0;
    const float* bt = a.bt + e0;
    uint32_t re[SLAB_D];
    float rb[SLAB_D];
#pragma unroll
    for (int d = 0; d < SLAB_D; ++d) {
      const uint32_t j = j0 + (uint32_t)d * G + g;
      const bool on = j < j1;
      re[d] = on ? __ldcs(ent + j) : 0u;
      rb[d] = on ? __ldcs(bt + j) : 0.f;
    }
    for (uint32_t u0 = 0; u0 < nchunk; u0 += SLAB_D) {
#pragma unroll
      for (int d = 0; d < SLAB_D; ++d) {
        const uint32_t e_m = re[d];
        const float b_m = rb[d];
        {  // refill this slot SLAB_D chunks ahead
          const uint32_t j = j0 + (u0 + d + SLAB_D) * G + g;
          const bool on = j < j1;
          re[d] = on ? __ldcs(ent + j) : 0u;
          rb[d] = on ? __ldcs(bt + j) : 0.f;
        }
        if (u0 + d >= nchunk) continue;  // uniform over the team
#pragma unroll
        for (int sidx = 0; sidx < G; ++sidx) {
          const uint32_t j = j0 + (u0 + d) * G + sidx;
          const uint32_t e = G > 1 ? __shfl_sync(0xffffffffu, e_m, gbase + sidx) : e_m;
          const float bj = G > 1 ? __shfl_sync(0xffffffffu, b_m, gbase + sidx) : b_m;
          if (j < j1 && j == nb)
            slab_next_cell<RTP, OBJ>(sYW, sPf, sCS, sAct, e0, q, qd, k, nb, cw, foreign, y, w, objc, objt);
          slab_entry<RTP, SMEM_A, OBJ>(a, sA, sInvp, qd, 0xffffffffu, e, bj, cw, y, w, objc, zx, wskip);
        }
      }
    }
    // The last cell of the segment: a partial (it began in an earlier segment), complete
    // (stored now), or continuing into later segments (kept until their partials exist).
    const bool pending = has && !foreign && nb > j1;
    if (has && !pending) {
      float* dst = foreign ? (sPf + q * RTP) : (sYW + k * RTP);
#pragma unroll
      for (int v = 0; v < NQ; ++v)
        reinterpret_cast<float4*>(dst)[qd[v]] = make_float4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
    }
    if (OBJ && has) objt += (double)objc;
    if (OBJ) {  // objective of the tile: one lane per group
      double ov = (g == 0 && has) ? objt : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ov += __shfl_xor_sync(0xffffffffu, ov, off);
      if (lane == 0) sRed[wt] = ov;
    }
    team_sync(team);
    // ---- the owner of a cell continuing past its segment adds the later groups'
    //      partials in group order
    if (pending) {
      for (uint32_t q2 = (uint32_t)q + 1; q2 < (uint32_t)NG && q2 * L < nb; ++q2) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) {
          const float4 pq = reinterpret_cast<const float4*>(sPf + q2 * RTP)[qd[v]];
          w[4 * v + 0] += pq.x;
          w[4 * v + 1] += pq.y;
          w[4 * v + 2] += pq.z;
          w[4 * v + 3] += pq.w;
        }
      }
#pragma unroll
      for (int v = 0; v < NQ; ++v)
        reinterpret_cast<float4*>(sYW + k * RTP)[qd[v]] = make_float4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
    }
    if (OBJ && tt == 0) {
      double s = 0.0;
      for (int i = 0; i < SLAB_TEAM / 32; ++i) s += sRed[i];
      a.objpart[t] = s;
    }
    team_sync(team);
    if (a.obj_only) continue;  // the tiles' Z is not wanted
    // ---- Z contribution: sum_k A(N-1)[i_k]^T W[k]
    if (PREC != 0 && mma) {
      // one 16 x 8 block of Z per warp step over all cells (k): A = A(N-1)^T (m = r, k = cell),
      // B = W (k = cell, n = column); fragment positions as in the Y product. e4m3: one scale
      // per row r of A(N-1)^T and per column of W, over the tile's cells
      const int fr = lane >> 2, fc = lane & 3;
      float* usc = sPf;        // R2P scales of A(N-1)^T rows
      float* vsc = sPf + R2P;  // RTP scales of W columns
      if (PREC == 2) {
        if (tt < R2P + RTP) {
          const bool isu = tt < R2P;
          const int c = isu ? tt : tt - R2P;
          const float* src = isu ? sA2 + c : sYW + c;
          const int stride = isu ? R2S : RTP;
          float m = 0.f;
          for (int i = 0; i < na; ++i) m = fmaxf(m, fabsf(src[i * stride]));
          (isu ? usc : vsc)[c] = m > 0.f ? m / E4M3_MAX : 1.f;
        }
        team_sync(team);
      }
      const int nnt = NT8, nblk = (R2 / 16) * nnt, nks = (na + KS - 1) / KS;
      float* dst = a.zpart + (size_t)t * zn;
      for (int b = wt; b < nblk; b += SLAB_TEAM / 32) {
        const int mt = b / nnt, nt = b - mt * nnt;
        const int m0 = 16 * mt + fr, n0 = 8 * nt + fr;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        float iu0 = 1.f, iu1 = 1.f, iv = 1.f;
        if (PREC == 2) {
          iu0 = 1.f / usc[m0];
          iu1 = 1.f / usc[m0 + 8];
          iv = 1.f / vsc[n0];
        }
        for (int ks = 0; ks < nks; ++ks) {
          uint32_t af[4], bf[2];
          if (PREC == 1) {
            const int k0 = 16 * ks + 2 * fc;
            const float* a0 = sA2 + k0 * R2S + m0;
            const float* w0 = sYW + k0 * RTP + n0;
            af[0] = pack_bf16(a0[0], a0[R2S]);
            af[1] = pack_bf16(a0[8], a0[R2S + 8]);
            af[2] = pack_bf16(a0[8 * R2S], a0[9 * R2S]);
            af[3] = pack_bf16(a0[8 * R2S + 8], a0[9 * R2S + 8]);
            bf[0] = pack_bf16(w0[0], w0[RTP]);
            bf[1] = pack_bf16(w0[8 * RTP], w0[9 * RTP]);
            mma_bf16(acc, af, bf);
          } else {
            const int k0 = 32 * ks + 4 * fc;
            const float* a0 = sA2 + k0 * R2S + m0;
            const float* a2 = a0 + 16 * R2S;
            const float* w0 = sYW + k0 * RTP + n0;
            const float* w2 = w0 + 16 * RTP;
            af[0] = pack_e4m3(a0[0] * iu0, a0[R2S] * iu0, a0[2 * R2S] * iu0, a0[3 * R2S] * iu0);
            af[1] = pack_e4m3(a0[8] * iu1, a0[R2S + 8] * iu1, a0[2 * R2S + 8] * iu1, a0[3 * R2S + 8] * iu1);
            af[2] = pack_e4m3(a2[0] * iu0, a2[R2S] * iu0, a2[2 * R2S] * iu0, a2[3 * R2S] * iu0);
            af[3] = pack_e4m3(a2[8] * iu1, a2[R2S + 8] * iu1, a2[2 * R2S + 8] * iu1, a2[3 * R2S + 8] * iu1);
            bf[0] = pack_e4m3(w0[0] * iv, w0[RTP] * iv, w0[2 * RTP] * iv, w0[3 * RTP] * iv);
            bf[1] = pack_e4m3(w2[0] * iv, w2[RTP] * iv, w2[2 * RTP] * iv, w2[3 * RTP] * iv);
            mma_e4m3(acc, af, bf);
          }
        }
        const int r0 = 16 * mt + fr, c0 = 8 * nt + 2 * fc;
        float s00 = 1.f, s01 = 1.f, s10 = 1.f, s11 = 1.f;
        if (PREC == 2) {
          s00 = usc[r0] * vsc[c0];
          s01 = usc[r0] * vsc[c0 + 1];
          s10 = usc[r0 + 8] * vsc[c0];
          s11 = usc[r0 + 8] * vsc[c0 + 1];
        }
        float* z0 = dst + r0 * RT;
        float* z1 = z0 + 8 * RT;
        if (c0 < RT) {
          z0[c0] = acc[0] * s00;
          z1[c0] = acc[2] * s10;
        }
        if (c0 + 1 < RT) {
          z0[c0 + 1] = acc[1] * s01;
          z1[c0 + 1] = acc[3] * s11;
        }
      }
      continue;
    }
    if (mma) {
      // one 16 x 8 block of Z per warp step over all cells (k): A = A(N-1)^T (a0 at
      // (m = fr, k = fc): row k of the staged rows, column m), B = W (b0 at (k = fc, n = fr));
      // the cells past na up to the next multiple of 8 are zero in both operands
      const int fr = lane >> 2, fc = lane & 3;
      const int nnt = NT8, nblk = (R2 / 16) * nnt, nks = (na + 7) >> 3;
      float* dst = a.zpart + (size_t)t * zn;
      for (int b = wt; b < nblk; b += SLAB_TEAM / 32) {
        const int mt = b / nnt, nt = b - mt * nnt;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* ac = sA2 + fc * R2S + 16 * mt + fr;
        const float* wc = sYW + fc * RTP + 8 * nt + fr;
        for (int ks = 0; ks < nks; ++ks) {
          const float* a0 = ac + 8 * ks * R2S;
          const float* w0 = wc + 8 * ks * RTP;
          uint32_t ah[4], al[4], bh[2], bl[2];
          tf32_split(a0[0], ah[0], al[0]);
          tf32_split(a0[8], ah[1], al[1]);
          tf32_split(a0[4 * R2S], ah[2], al[2]);
          tf32_split(a0[4 * R2S + 8], ah[3], al[3]);
          tf32_split(w0[0], bh[0], bl[0]);
          tf32_split(w0[4 * RTP], bh[1], bl[1]);
          mma_tf32x3(acc, ah, al, bh, bl);
        }
        // scalar stores: rows of R_N floats need not keep pairs 8-byte aligned (odd R_N),
        // and the padding columns c >= R_N are dropped
        const int r0 = 16 * mt + fr, c0 = 8 * nt + 2 * fc;
        float* z0 = dst + r0 * RT;
        float* z1 = z0 + 8 * RT;
        if (c0 < RT) {
          z0[c0] = acc[0];
          z1[c0] = acc[2];
        }
        if (c0 + 1 < RT) {
          z0[c0 + 1] = acc[1];
          z1[c0 + 1] = acc[3];
        }
      }
      continue;
    }
    {  // SIMT form: cells split over ks thread sets
      const int ZQ = R2P / 4, ntt = ZQ * XQ;
      int ks = SLAB_TEAM / ntt;
      const int cap = S::PF / (R2P * RTP);
      if (ks > cap) ks = cap;
      if (ks < 1) ks = 1;
      for (int it = tt; it < ntt * ks; it += SLAB_TEAM) {
        const int part = it / ntt, wq = it % ntt, zq = wq / XQ, xq = wq % XQ;
        const int k_lo = part * na / ks, k_hi = (part + 1) * na / ks;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
        for (int kk = k_lo; kk < k_hi; ++kk) {
          const float4 av = *reinterpret_cast<const float4*>(sA2 + kk * R2S + 4 * zq);
          const float4 yv = *reinterpret_cast<const float4*>(sYW + kk * RTP + 4 * xq);
          const float ak[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][0] = fmaf(ak[i], yv.x, acc[i][0]);
            acc[i][1] = fmaf(ak[i], yv.y, acc[i][1]);
            acc[i][2] = fmaf(ak[i], yv.z, acc[i][2]);
            acc[i][3] = fmaf(ak[i], yv.w, acc[i][3]);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          *reinterpret_cast<float4*>(sPf + part * (R2P * RTP) + (4 * zq + i) * RTP + 4 * xq) =
              make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
      team_sync(team);
      // the k-split parts in order, to the tile's slot (k_tile_reduce adds the tiles)
      float* dst = a.zpart + (size_t)t * zn;
      for (int i = tt; i < zn; i += SLAB_TEAM) {
        const int r = i / RT, c = i - r * RT;
        float v = sPf[r * RTP + c];
        for (int part = 1; part < ks; ++part) v += sPf[part * (R2P * RTP) + r * RTP + c];
        dst[i] = v;
      }
    }
  }
}

// The backward product of the last prefix mode folded into the sum over tiles:
// W[p', r, :] = sum_i Aq[i, r] Z[p' Iq + i, :] with Z[p] = sum of the tiles of slab p
// (tiles of slab p: [tstart[p], tstart[p + 1]); Aq = A(N-2) for N >= 3; for N = 2 there
// is no prefix mode: Iq = Rq = 1, weight 1). The Iq slabs of a group are split into nc
// chunks of at most TR_MAXS slabs (blockIdx.y) and the columns into panels (blockIdx.x):
// a block forms Z of its slabs for its panel in shared memory (tiles in order), then
// part[c] = sum over its slabs of Aq rows x Z (slab order); k_tile_reduce2 adds the chunks
// in order.
constexpr int TR_MAXS = 64;  // slabs per chunk at most
constexpr int TR_QP = 64;    // columns per block
// Shared memory of k_tile_reduce1 (floats, rows of 16 bytes): tile starts (TR_MAXS + 1,
// padded to 68), Z of the chunk's slabs (per x TR_QP), Aq rows (per x Rq4), then as many
// staged tile rows (TR_QP each) as the 48 KB budget leaves, at most 256.
struct TileReduceSmem {
  int per, rq4, tb;
  size_t bytes;
};
TileReduceSmem tile_reduce_smem(int per, int Rq, int nout) {
  TileReduceSmem L;
  L.per = per;
  L.rq4 = (Rq + 3) & ~3;
  const size_t fixed = (68 + (size_t)per * TR_QP + (size_t)nout * per * L.rq4) * sizeof(float);
  const size_t budget = 48 * 1024;
  int tb = fixed < budget ? (int)((budget - fixed) / (TR_QP * sizeof(float))) : 0;
  L.tb = tb > 256 ? 256 : (tb < 16 ? 16 : tb);
  L.bytes = fixed + (size_t)L.tb * TR_QP * sizeof(float);
  return L;
}
// TWO: a second weight matrix Aq2 in the same pass (its sums to part2). With opart, block
// x = 0 of every (chunk, group) also adds the objective partials of the chunk's tiles in
// tile order: opart[c * Pq + pq].
template <bool TWO>
__global__ void __launch_bounds__(256) k_tile_reduce1(const uint32_t* __restrict__ tstart, int Iq,
                                                      const float* __restrict__ zpart, const float* __restrict__ Aq,
                                                      const float* __restrict__ Aq2, int Rq, int zn, int nc,
                                                      int64_t Pq, float* __restrict__ part,
                                                      float* __restrict__ part2, int64_t cstride,
                                                      uint32_t* __restrict__ counter, int TB,
                                                      const double* __restrict__ objpart,
                                                      double* __restrict__ opart) {
  extern __shared__ float4 tr_smem[];
  const int64_t pq = blockIdx.z;
  const int c = blockIdx.y;
  const int qb = blockIdx.x * TR_QP;
  const int per = (Iq + nc - 1) / nc;
  const int i0 = min(Iq, c * per), i1 = min(Iq, i0 + per), S = i1 - i0;
  const int Rq4 = (Rq + 3) & ~3;  // ranks padded with zeros to the 4-rank blocks below
  uint32_t* s_ts = reinterpret_cast<uint32_t*>(tr_smem);
  float* s_z = reinterpret_cast<float*>(tr_smem) + 68;  // [per][TR_QP]
  float* s_a = s_z + (size_t)per * TR_QP;                // [per][Rq4]
  float* s_a2 = s_a + (size_t)per * Rq4;                 // [per][Rq4] (TWO)
  float* s_t = s_a + (size_t)(TWO ? 2 : 1) * per * Rq4;  // [TB][TR_QP]
  for (int k = threadIdx.x; k <= S; k += blockDim.x) s_ts[k] = tstart[pq * Iq + i0 + k];
  for (int e = threadIdx.x; e < S * Rq4; e += blockDim.x) {
    const int i = e / Rq4, r = e - i * Rq4;
    s_a[e] = r < Rq ? (Aq ? __ldg(Aq + (size_t)(i0 + i) * Rq + r) : 1.f) : 0.f;
    if (TWO) s_a2[e] = r < Rq ? __ldg(Aq2 + (size_t)(i0 + i) * Rq + r) : 0.f;
  }
  for (int e = threadIdx.x; e < S * TR_QP; e += blockDim.x) s_z[e] = 0.f;
  kr_pdl_trigger();
  kr_pdl_wait();  // zpart: the slab pass has finished
  // ... and its work counter can be re-armed for the next pass
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  // Z of the chunk's slabs for this panel, tiles of one slab added in tile order. The
  // chunk's tiles are contiguous; a batch of tile rows is staged with independent loads
  // (16 bytes each where the row layout allows), then every (slab, column) adds the
  // batch's tiles of its slab.
  const uint32_t t0 = s_ts[0], t1 = s_ts[S];
  const bool vec = (zn & 3) == 0;
  for (uint32_t tb = t0; tb < t1; tb += (uint32_t)TB) {
    const int nt = (int)min((uint32_t)TB, t1 - tb);
    if (vec) {
      for (int e = threadIdx.x; e < nt * (TR_QP / 4); e += blockDim.x) {
        const int tl = e / (TR_QP / 4), c4 = e - tl * (TR_QP / 4), q = qb + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < zn) v = __ldg(reinterpret_cast<const float4*>(zpart + (size_t)(tb + tl) * zn + q));
        *reinterpret_cast<float4*>(s_t + tl * TR_QP + 4 * c4) = v;
      }
    } else {
      for (int e = threadIdx.x; e < nt * TR_QP; e += blockDim.x) {
        const int tl = e / TR_QP, qq = e - tl * TR_QP, q = qb + qq;
        s_t[tl * TR_QP + qq] = q < zn ? __ldg(zpart + (size_t)(tb + tl) * zn + q) : 0.f;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < S * TR_QP; e += blockDim.x) {
      const int i = e / TR_QP, qq = e - i * TR_QP;
      const uint32_t lo = max(s_ts[i], tb), hi = min(s_ts[i + 1], tb + (uint32_t)nt);
      if (lo >= hi) continue;
      float z = s_z[i * TR_QP + qq];
      for (uint32_t t = lo; t < hi; ++t) z += s_t[(t - tb) * TR_QP + qq];
      s_z[i * TR_QP + qq] = z;
    }
    __syncthreads();
  }
  // part[c][pq][r][q] = sum_i Aq[i0 + i, r] Z[i, q] in slab order; a thread forms 4 ranks x
  // 2 columns (one 16-byte load of Aq's row and one 8-byte load of Z per slab)
  float* out = part + (size_t)c * cstride + (size_t)pq * Rq * zn;
  float* out2 = TWO ? part2 + (size_t)c * cstride + (size_t)pq * Rq * zn : nullptr;
  const int R4 = (Rq + 3) >> 2;
  for (int e = threadIdx.x; e < R4 * (TR_QP / 2); e += blockDim.x) {
    const int r4 = e / (TR_QP / 2), q2 = e - r4 * (TR_QP / 2), r0 = 4 * r4, qq = 2 * q2, q = qb + qq;
    if (q >= zn) continue;
    float acc[4][2] = {};
    float acc2[4][2] = {};
    for (int i = 0; i < S; ++i) {
      const float4 av = *reinterpret_cast<const float4*>(s_a + i * Rq4 + r0);
      const float2 zv = *reinterpret_cast<const float2*>(s_z + i * TR_QP + qq);
      acc[0][0] = fmaf(av.x, zv.x, acc[0][0]);
      acc[0][1] = fmaf(av.x, zv.y, acc[0][1]);
      acc[1][0] = fmaf(av.y, zv.x, acc[1][0]);
      acc[1][1] = fmaf(av.y, zv.y, acc[1][1]);
      acc[2][0] = fmaf(av.z, zv.x, acc[2][0]);
      acc[2][1] = fmaf(av.z, zv.y, acc[2][1]);
      acc[3][0] = fmaf(av.w, zv.x, acc[3][0]);
      acc[3][1] = fmaf(av.w, zv.y, acc[3][1]);
      if (TWO) {
        const float4 bv = *reinterpret_cast<const float4*>(s_a2 + i * Rq4 + r0);
        acc2[0][0] = fmaf(bv.x, zv.x, acc2[0][0]);
        acc2[0][1] = fmaf(bv.x, zv.y, acc2[0][1]);
        acc2[1][0] = fmaf(bv.y, zv.x, acc2[1][0]);
        acc2[1][1] = fmaf(bv.y, zv.y, acc2[1][1]);
        acc2[2][0] = fmaf(bv.z, zv.x, acc2[2][0]);
        acc2[2][1] = fmaf(bv.z, zv.y, acc2[2][1]);
        acc2[3][0] = fmaf(bv.w, zv.x, acc2[3][0]);
        acc2[3][1] = fmaf(bv.w, zv.y, acc2[3][1]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (r0 + j >= Rq) break;
      out[(size_t)(r0 + j) * zn + q] = acc[j][0];
      if (q + 1 < zn) out[(size_t)(r0 + j) * zn + q + 1] = acc[j][1];
      if (TWO) {
        out2[(size_t)(r0 + j) * zn + q] = acc2[j][0];
        if (q + 1 < zn) out2[(size_t)(r0 + j) * zn + q + 1] = acc2[j][1];
      }
    }
  }
  if (opart && blockIdx.x == 0) {  // the chunk's tiles' objective: fixed strides, then a fixed tree
    __shared__ double s_o[256];
    double acc = 0.0;
    for (uint32_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) acc += __ldcg(objpart + t);
    s_o[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
      if ((int)threadIdx.x < off) s_o[threadIdx.x] += s_o[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) opart[(size_t)c * Pq + pq] = s_o[0];
  }
}

// W = sum over the nc chunks of part, in chunk order; four columns per thread when the
// length allows, the loads of a batch of chunks in flight together. Chunk c starts at
// part + c * cstride; with W2 each chunk holds two outputs back to back (W's total entries,
// then W2's).
__global__ void __launch_bounds__(128) k_tile_reduce2(const float* __restrict__ part, int nc, int64_t cstride,
                                                      int64_t total, float* __restrict__ W, float* __restrict__ W2) {
  kr_pdl_trigger();
  kr_pdl_wait();
  if ((total & 3) == 0) {
    const int64_t n4 = total >> 2, all4 = W2 ? 2 * n4 : n4, cs4 = cstride >> 2;
    const float4* p4 = reinterpret_cast<const float4*>(part);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < all4; e += (int64_t)gridDim.x * blockDim.x) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int c0 = 0; c0 < nc; c0 += 16) {
        float4 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = c0 + c < nc ? __ldg(p4 + (size_t)(c0 + c) * cs4 + e) : s;
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c0 + c < nc) {
            if (c0 + c == 0) {
              s = v[c];
            } else {
              s.x += v[c].x;
              s.y += v[c].y;
              s.z += v[c].z;
              s.w += v[c].w;
            }
          }
      }
      if (e < n4) reinterpret_cast<float4*>(W)[e] = s;
      else reinterpret_cast<float4*>(W2)[e - n4] = s;
    }
    return;
  }
  const int64_t all = W2 ? 2 * total : total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < all; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c0 = 0; c0 < nc; c0 += 16) {  // loads of a batch in flight together, added in order
      float v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = c0 + c < nc ? __ldg(part + (size_t)(c0 + c) * cstride + e) : 0.f;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c0 + c < nc) s = (c0 + c == 0) ? v[c] : s + v[c];
    }
    if (e < total) W[e] = s;
    else W2[e - total] = s;
  }
}

// tstart[P] = tiles (after the exclusive scan of the per-slab tile counts).
__global__ void k_tiles_counts(int64_t P, const uint2* __restrict__ slab, uint32_t* __restrict__ cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
    cnt[p] = slab[p].y;
}
__global__ void k_tiles_tail(int64_t P, const uint32_t* __restrict__ meta, uint32_t* __restrict__ tstart) {
  tstart[P] = meta[0];
}

// ------------------------------------------------------------------ tile construction

__global__ void k_tiles_flag(const uint32_t* __restrict__ nd, int64_t n, uint32_t* __restrict__ f) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    f[c] = nd[c] > 0 ? 1u : 0u;
}

// Non-empty cells in cell order: act[aidx[c]] = {c, start, nd, weight bits}.
__global__ void k_tiles_act(int64_t ncell, const uint32_t* __restrict__ nd, const uint32_t* __restrict__ start,
                            const float* __restrict__ cw, const uint32_t* __restrict__ aidx, uint4* __restrict__ act,
                            uint32_t* __restrict__ meta) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t n = nd[c];
    if (n > 0) act[aidx[c]] = make_uint4((uint32_t)c, start[c], n, __float_as_uint(cw[c]));
    if (c == ncell - 1) meta[1] = aidx[c] + (n > 0 ? 1u : 0u);
  }
}

// A tile starts at non-empty cell a when a is the first of its slab, when the tile has
// reached cb cells, or when floor(entries before a in the slab / et) changes.
__global__ void k_tiles_start(int64_t ncell, uint32_t I2, uint32_t cb, uint32_t et, const uint4* __restrict__ act,
                              const uint32_t* __restrict__ aidx, const uint32_t* __restrict__ start,
                              const uint32_t* __restrict__ meta, uint32_t* __restrict__ f) {
  const uint32_t nact = meta[1];
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < ncell; a += (int64_t)gridDim.x * blockDim.x) {
    if (a >= nact) {
      f[a] = 0u;
      continue;
    }
    const uint4 ac = act[a];
    const uint32_t cs = (ac.x / I2) * I2;  // first cell of the slab
    const uint32_t la = (uint32_t)a - aidx[cs];
    const uint32_t base = start[cs];
    bool s = la == 0 || la % cb == 0;
    if (!s) s = (ac.y - base) / et != (act[a - 1].y - base) / et;
    f[a] = s ? 1u : 0u;
  }
}

__global__ void k_tiles_first(int64_t ncell, uint32_t I2, const uint4* __restrict__ act, const uint32_t* __restrict__ f,
                              const uint32_t* __restrict__ tidx, uint4* __restrict__ tile, uint32_t* __restrict__ meta) {
  const uint32_t nact = meta[1];
  if (blockIdx.x == 0 && threadIdx.x == 0 && nact == 0) meta[0] = 0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nact; a += (int64_t)gridDim.x * blockDim.x) {
    if (f[a]) tile[tidx[a]] = make_uint4((uint32_t)a, 0u, act[a].x / I2, 0u);
    if (a == nact - 1) meta[0] = tidx[a] + f[a];
  }
}

__global__ void k_tiles_init_slab(int64_t P, uint2* __restrict__ slab) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
    slab[p] = make_uint2(0xFFFFFFFFu, 0u);
}

// Cell count, entry count and work estimate of every tile; first tile and tile count
// of every slab (integer atomics: the result does not depend on their order).
__global__ void k_tiles_fin(int64_t ntmax, uint32_t cellcost, const uint4* __restrict__ act, uint4* __restrict__ tile,
                            uint32_t* __restrict__ cost, uint2* __restrict__ slab, const uint32_t* __restrict__ meta) {
  const uint32_t nt = meta[0], nact = meta[1];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntmax; t += (int64_t)gridDim.x * blockDim.x) {
    if (t >= nt) {
      cost[t] = 0u;
      continue;
    }
    const uint32_t a0 = tile[t].x;
    const uint32_t a1 = (t + 1 < nt) ? tile[t + 1].x : nact;
    const uint32_t na = a1 - a0;
    const uint4 last = act[a1 - 1];
    const uint32_t E = last.y + last.z - act[a0].y;
    const uint32_t p = tile[t].z;
    tile[t].y = na;
    tile[t].w = E;
    cost[t] = E + cellcost * na;
    atomicMin(&slab[p].x, (uint32_t)t);
    atomicAdd(&slab[p].y, 1u);
  }
}

// Tile descriptors in processing order, with the tile index and a flag for slabs of
// more than one tile packed in.
__global__ void k_tiles_sort(int64_t ntmax, const uint32_t* __restrict__ order, const uint4* __restrict__ tile,
                             const uint2* __restrict__ slab, const uint32_t* __restrict__ meta,
                             uint4* __restrict__ tsort) {
  const uint32_t nt = meta[0];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = order[k];
    const uint4 d = tile[t];
    const uint32_t multi = slab[d.z].y > 1 ? 1u : 0u;
    tsort[k] = make_uint4(d.x, t, d.z, d.w | ((d.y - 1u) << 24) | (multi << 31));
  }
}

struct SlabLayout {
  int RTP, R2P, R2S, cb, mma, XS;
  bool smem_a;
  size_t bytes;
  uint32_t team_off, team_bytes, o_a2, o_x1, o_pf, o_act, o_cs, o_ctl;
};

size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

SlabLayout slab_layout(int IT, int RT, int R2, bool smem_a) {
  SlabLayout L = {};
  L.RTP = rt_pad(RT);
  L.R2P = (R2 + 3) / 4 * 4;
  L.R2S = L.R2P + 4;
  // Y and Z on the TF32 tensor path when the fragments tile the shapes exactly
  L.mma = (R2 % 16 == 0 && L.RTP >= 8) ? 1 : 0;
  L.XS = L.RTP + 8;  // row stride of the split X1[p] planes: conflict-free B fragment loads
  L.cb = cb_for(L.RTP);
  L.smem_a = smem_a;
  const int cols = L.RTP < 16 ? L.RTP : 16;
  size_t off = smem_a ? (size_t)IT * L.RTP * 4 : 0;
  off += (size_t)((IT + 3) / 4 * 4) * 4;
  L.team_off = (uint32_t)al16(off);
  size_t t = 0;
  t += (size_t)L.cb * L.RTP * 4;  // Y / W
  L.o_a2 = (uint32_t)t;
  t += al16((size_t)L.cb * L.R2S * 4);
  L.o_x1 = (uint32_t)t;
  t += al16(L.mma ? (size_t)2 * L.R2P * L.XS * 4 : (size_t)L.R2P * L.RTP * 4);
  L.o_pf = (uint32_t)t;
  t += (size_t)SLAB_TEAM * cols * 4;
  L.o_act = (uint32_t)t;
  t += (size_t)L.cb * 16;
  L.o_cs = (uint32_t)t;
  t += al16((size_t)(L.cb + 4) * 4);
  L.o_ctl = (uint32_t)t;
  t += 128;
  L.team_bytes = (uint32_t)al16(t);
  L.bytes = L.team_off + (size_t)SLAB_TEAMS * L.team_bytes;
  return L;
}

template <int RTP, bool SMEM_A, bool OBJ, int PREC>
kr_status launch_slab_t(kr_ctx* ctx, const SlabArgs& a, size_t smem) {
  KR_TRY(kr_smem_attr(ctx, k_slab<RTP, SMEM_A, OBJ, PREC>, smem));
  KR_LAUNCH_PDL(ctx, (k_slab<RTP, SMEM_A, OBJ, PREC>), ctx->num_sms, SLAB_TEAM * SLAB_TEAMS, smem, a);
  return KR_OK;
}

template <bool SMEM_A, bool OBJ, int PREC>
kr_status launch_slab_p(kr_ctx* ctx, int RTP, const SlabArgs& a, size_t smem) {
  switch (RTP) {
    case 4: return launch_slab_t<4, SMEM_A, OBJ, 0>(ctx, a, smem);  // no tensor-core products
    case 8: return launch_slab_t<8, SMEM_A, OBJ, PREC>(ctx, a, smem);
    case 16: return launch_slab_t<16, SMEM_A, OBJ, PREC>(ctx, a, smem);
    case 32: return launch_slab_t<32, SMEM_A, OBJ, PREC>(ctx, a, smem);
    case 64: return launch_slab_t<64, SMEM_A, OBJ, PREC>(ctx, a, smem);
    default: return kr_fail(ctx, KR_EINVAL, "slab pass: R_N padded to %d", RTP);
  }
}

// The objective pass (the final FP64 check) always runs the FP32-accurate products.
template <bool SMEM_A, bool OBJ>
kr_status launch_slab(kr_ctx* ctx, int RTP, int prec, const SlabArgs& a, size_t smem) {
  if (OBJ || prec == 0) return launch_slab_p<SMEM_A, OBJ, 0>(ctx, RTP, a, smem);
  if (prec == 1) return launch_slab_p<SMEM_A, false, 1>(ctx, RTP, a, smem);
  return launch_slab_p<SMEM_A, false, 2>(ctx, RTP, a, smem);
}

int grid_n(kr_ctx* ctx, int64_t n, int block = 256) {
  int64_t g = (n + block - 1) / block;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

bool kr_slab_eligible(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, bool rows) {
  if (m.N < 2 || (sk->nrow != 1 && !rows)) return false;
  const int RT = m.R[m.N - 1], R2 = m.R[m.N - 2];
  if (RT > 64 || R2 > 64 || m.I[m.N - 1] > 65535) return false;
  return slab_layout(m.I[m.N - 1], RT, R2, false).bytes <= ctx->smem_optin;
}

void kr_tiles_setup(kr_ctx* ctx, const Modes& m, const kr_sketch* sk, kr_tiles* tl) {
  const int N = m.N;
  tl->I2 = m.I[N - 2];
  tl->R2 = m.R[N - 2];
  tl->IT = m.I[N - 1];
  tl->RT = m.R[N - 1];
  // slabs: the cells without their last index (a batched-row sketch's row axis included)
  const int64_t P = sk->ncell / tl->I2;
  tl->P = P;
  tl->cb = cb_for(rt_pad(tl->RT));
  tl->et = ctx->slab_tile_entries;
  const int64_t ncell = sk->ncell;
  int64_t bound = P + (ncell + tl->cb - 1) / tl->cb + (sk->s + tl->et - 1) / tl->et;
  tl->ntmax = bound < ncell ? bound : ncell;
  if (tl->ntmax < 1) tl->ntmax = 1;
  if (N >= 3) {
    tl->Iq = m.I[N - 3];
    tl->Rq = m.R[N - 3];
  } else {
    tl->Iq = 1;
    tl->Rq = 1;
  }
  tl->Pq = P / tl->Iq;
  // chunks of about 16 slabs (at most 64 = TR_MAXS), at most 32 chunks unless the
  // 64-slab limit needs more
  int nc = tl->Iq / 16;
  nc = nc < 1 ? 1 : (nc > 32 ? 32 : nc);
  const int need = (tl->Iq + 63) / 64;
  tl->nc = nc > need ? nc : need;
}

void kr_tiles_own_need(const kr_tiles* tl, int64_t ncell, Need& nd) {
  nd.add<uint4>(ncell);
  nd.add<uint4>(tl->ntmax);
  nd.add<uint32_t>(tl->ntmax);
  nd.add<uint32_t>(tl->ntmax);
  nd.add<uint4>(tl->ntmax);
  nd.add<uint2>(tl->P);
  nd.add<uint32_t>(tl->P + 1);
  nd.add<float>(tl->nc > 1 ? (size_t)tl->nc * tl->nout * tl->Pq * tl->Rq * tl->R2 * tl->RT : 0);
  nd.add<uint32_t>(4);
  nd.add<float>((size_t)tl->ntmax * tl->R2 * tl->RT);
  nd.add<double>(tl->ntmax);
}

void kr_tiles_layout(kr_tiles* tl, int64_t ncell, Carve& cv) {
  tl->act = cv.take<uint4>(ncell);
  tl->tile = cv.take<uint4>(tl->ntmax);
  tl->cost = cv.take<uint32_t>(tl->ntmax);
  tl->order = cv.take<uint32_t>(tl->ntmax);
  tl->tsort = cv.take<uint4>(tl->ntmax);
  tl->slab = cv.take<uint2>(tl->P);
  tl->tstart = cv.take<uint32_t>(tl->P + 1);
  tl->zred = cv.take<float>(tl->nc > 1 ? (size_t)tl->nc * tl->nout * tl->Pq * tl->Rq * tl->R2 * tl->RT : 0);
  tl->meta = cv.take<uint32_t>(4);
  tl->zpart = cv.take<float>((size_t)tl->ntmax * tl->R2 * tl->RT);
  tl->objpart = cv.take<double>(tl->ntmax);
}

void kr_tiles_scratch_need(const kr_tiles* tl, int64_t ncell, Need& nd) {
  nd.add<uint32_t>(ncell);  // flags
  nd.add<uint32_t>(ncell);  // non-empty index
  nd.add<uint32_t>(ncell);  // tile index
  kr_scan_need(ncell, nd);
  kr_perm_need(tl->ntmax, nd);
}

kr_status kr_tiles_build(kr_ctx* ctx, const kr_sketch* sk, kr_tiles* tl, Carve& cv) {
  const int64_t ncell = sk->ncell;
  uint32_t* f = cv.take<uint32_t>(ncell);
  uint32_t* aidx = cv.take<uint32_t>(ncell);
  uint32_t* tidx = cv.take<uint32_t>(ncell);
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "slab tiles: workspace too small");
  KR_CUDA(ctx, cudaMemsetAsync(tl->meta, 0, 4 * sizeof(uint32_t), ctx->stream));
  KR_CUDA(ctx, cudaMemsetAsync(tl->objpart, 0, sizeof(double) * tl->ntmax, ctx->stream));
  KR_LAUNCH(ctx, k_tiles_flag, grid_n(ctx, ncell), 256, 0, sk->cell_nd, ncell, f);
  {
    Carve sc = cv;
    KR_TRY(kr_scan_u32(ctx, f, aidx, ncell, sc));
  }
  KR_LAUNCH(ctx, k_tiles_act, grid_n(ctx, ncell), 256, 0, ncell, sk->cell_nd, sk->cell_start, sk->cell_w, aidx,
            tl->act, tl->meta);
  KR_LAUNCH(ctx, k_tiles_start, grid_n(ctx, ncell), 256, 0, ncell, (uint32_t)tl->I2, (uint32_t)tl->cb, tl->et, tl->act,
            aidx, sk->cell_start, tl->meta, f);
  {
    Carve sc = cv;
    KR_TRY(kr_scan_u32(ctx, f, tidx, ncell, sc));
  }
  KR_LAUNCH(ctx, k_tiles_first, grid_n(ctx, ncell), 256, 0, ncell, (uint32_t)tl->I2, tl->act, f, tidx, tl->tile,
            tl->meta);
  KR_LAUNCH(ctx, k_tiles_init_slab, grid_n(ctx, tl->P), 256, 0, tl->P, tl->slab);
  KR_LAUNCH(ctx, k_tiles_fin, grid_n(ctx, tl->ntmax), 256, 0, tl->ntmax, (uint32_t)tl->R2, tl->act, tl->tile, tl->cost,
            tl->slab, tl->meta);
  {
    Carve sc = cv;
    KR_TRY(kr_balance_perm(ctx, tl->cost, tl->ntmax, tl->order, sc));
  }
  KR_LAUNCH(ctx, k_tiles_sort, grid_n(ctx, tl->ntmax), 256, 0, tl->ntmax, tl->order, tl->tile, tl->slab, tl->meta,
            tl->tsort);
  KR_LAUNCH(ctx, k_tiles_counts, grid_n(ctx, tl->P), 256, 0, tl->P, tl->slab, tl->tstart);
  {
    Carve sc = cv;
    KR_TRY(kr_scan_u32(ctx, tl->tstart, tl->tstart, tl->P, sc));
  }
  KR_LAUNCH(ctx, k_tiles_tail, 1, 1, 0, tl->P, tl->meta, tl->tstart);
  return KR_OK;
}

int kr_slab_precision(int R2, int RT, int prec) {
  // the tensor-core products need R_{N-1} in whole k steps: 32 for e4m3, 16 for BF16
  // (and the TF32 form: 16); otherwise the pass falls back to the next finer format
  if (rt_pad(RT) < 8 || R2 % 16 != 0) return 0;
  if (prec >= 2 && R2 % 32 != 0) prec = 1;
  return prec < 0 ? 0 : (prec > 2 ? 2 : prec);
}

kr_status kr_slab_pass(kr_ctx* ctx, const kr_sketch* sk, kr_tiles* tl, const float* A2, const float* AT,
                       const float* X1, bool want_obj, bool rearm, int prec, int flags) {
  SlabLayout L = slab_layout(tl->IT, tl->RT, tl->R2, true);
  if (L.bytes > ctx->smem_optin) L = slab_layout(tl->IT, tl->RT, tl->R2, false);
  if (L.bytes > ctx->smem_optin) return kr_fail(ctx, KR_ENOTIMPL, "slab pass: %zu bytes of shared memory", L.bytes);
  SlabArgs a = {};
  a.act = tl->act;
  a.tsort = tl->tsort;
  a.meta = tl->meta;
  a.ent = sk->ent;
  a.bt = sk->bt;
  a.invpT = sk->invpT;
  a.AT = AT;
  a.A2 = A2;
  a.X1 = X1;
  a.zpart = tl->zpart;
  a.objpart = tl->objpart;
  a.IT = tl->IT;
  a.RT = tl->RT;
  a.I2 = tl->I2;
  a.R2 = tl->R2;
  a.R2P = L.R2P;
  a.R2S = L.R2S;
  a.mma = L.mma;
  a.XS = L.XS;
  a.P = tl->P;
  a.a2vec = (tl->R2 % 4 == 0) && ((reinterpret_cast<uintptr_t>(A2) & 15) == 0);
  a.atvec = (tl->RT % 4 == 0) && ((reinterpret_cast<uintptr_t>(AT) & 15) == 0);
  a.zero_x = (flags & KR_SLAB_ZERO_X) ? 1 : 0;
  a.obj_only = (flags & KR_SLAB_OBJ_ONLY) && want_obj ? 1 : 0;
  a.team_off = L.team_off;
  a.team_bytes = L.team_bytes;
  a.o_a2 = L.o_a2;
  a.o_x1 = L.o_x1;
  a.o_pf = L.o_pf;
  a.o_act = L.o_act;
  a.o_cs = L.o_cs;
  a.o_ctl = L.o_ctl;
  if (rearm) KR_CUDA(ctx, cudaMemsetAsync(tl->meta + 2, 0, sizeof(uint32_t), ctx->stream));
  const int pr = kr_slab_precision(tl->R2, tl->RT, prec);
  kr_status st = L.smem_a ? (want_obj ? launch_slab<true, true>(ctx, L.RTP, pr, a, L.bytes)
                                      : launch_slab<true, false>(ctx, L.RTP, pr, a, L.bytes))
                         : (want_obj ? launch_slab<false, true>(ctx, L.RTP, pr, a, L.bytes)
                                     : launch_slab<false, false>(ctx, L.RTP, pr, a, L.bytes));
  return st;
}

kr_status kr_tile_reduce(kr_ctx* ctx, kr_tiles* tl, const float* Aq, float* W, double* opart, const float* Aq2,
                         float* W2) {
  const int zn = tl->R2 * tl->RT;
  const int nout = Aq2 ? 2 : 1;
  if (nout > tl->nout) return kr_fail(ctx, KR_EINVAL, "tile reduction: %d outputs, room for %d", nout, tl->nout);
  const dim3 grid((unsigned)((zn + TR_QP - 1) / TR_QP), (unsigned)tl->nc, (unsigned)tl->Pq);
  const int64_t total = tl->Pq * tl->Rq * zn;
  float* part = tl->nc > 1 ? tl->zred : W;
  float* part2 = tl->nc > 1 ? tl->zred + total : W2;
  const int64_t cstride = (int64_t)nout * total;
  const TileReduceSmem L = tile_reduce_smem((tl->Iq + tl->nc - 1) / tl->nc, tl->Rq, nout);
  if (nout == 2) {
    KR_TRY(kr_smem_attr(ctx, k_tile_reduce1<true>, L.bytes));
    KR_LAUNCH_PDL(ctx, k_tile_reduce1<true>, grid, 256, L.bytes, tl->tstart, tl->Iq, tl->zpart, Aq, Aq2, tl->Rq, zn,
                  tl->nc, tl->Pq, part, part2, cstride, tl->meta + 2, L.tb, (const double*)tl->objpart, opart);
  } else {
    KR_TRY(kr_smem_attr(ctx, k_tile_reduce1<false>, L.bytes));
    KR_LAUNCH_PDL(ctx, k_tile_reduce1<false>, grid, 256, L.bytes, tl->tstart, tl->Iq, tl->zpart, Aq, (const float*)nullptr,
                  tl->Rq, zn, tl->nc, tl->Pq, part, (float*)nullptr, cstride, tl->meta + 2, L.tb,
                  (const double*)tl->objpart, opart);
  }
  if (tl->nc > 1) {
    const int64_t work = ((total & 3) == 0 ? total / 4 : total) * nout;
    KR_LAUNCH_PDL(ctx, k_tile_reduce2, grid_n(ctx, work, 128), 128, 0, (const float*)tl->zred, tl->nc, cstride, total, W,
                  nout == 2 ? W2 : (float*)nullptr);
  }
  return KR_OK;
}
