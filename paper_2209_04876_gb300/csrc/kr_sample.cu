// a3 + a4 + a5: product-distribution sampling, grouping of the draws by cell,
// merging of repeated rows, and the gather b~ = S b.
//
// SampleRows (§3 Def. of leverage score sampling) on K with the product
// distribution of Lemma 4.1: every coordinate of a draw is sampled independently
// from its factor's CDF (proof of Thm 4.5). The uniform for draw t and coordinate m
// comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), implemented here
// from that paper's definition: round (x0,x1,x2,x3) -> (hi(M1 x2) ^ x1 ^ k0,
// lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)), key bumped by the Weyl constants.
// Counter (t lo, t hi, m/2 + 256*row, call id lo), key (seed lo, seed hi); words
// (w0,w1) serve even m and (w2,w3) odd m; U = ((wa << 32) | wb) >> 11 and the drawn
// index is the smallest i with U * 2^-53 < cdf[i], evaluated exactly in integers as
// U < ceil(cdf[i] * 2^53).
//
// Grouping (the sets S_1, S_2 and B_S of the proof of Thm 4.4 with T = {N}):
// cell = (i_1..i_{N-1}), the last coordinate i_N stays with the sample. A counting
// sort by cell (histogram, scan, scatter), then per cell a table over i_N merges
// repeated rows into multiplicities in increasing i_N order, and gathers b.
#include "kr_internal.cuh"

namespace {

struct SampleModes {
  int N;
  int I[KR_MAX_MODES];
  const uint64_t* thr[KR_MAX_MODES];
  const double* prob[KR_MAX_MODES];
  const float* invp[KR_MAX_MODES];
};

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

__device__ __forceinline__ uint64_t u53(uint32_t a, uint32_t b) {
  return ((uint64_t(a) << 32) | uint64_t(b)) >> 11;
}

// Smallest i with U < thr[i] (thr non-decreasing, thr[n-1] = 2^53 > U).
__device__ __forceinline__ int search_thr(const uint64_t* thr, int n, uint64_t U) {
  int base = 0, len = n;
  while (len > 1) {
    int half = len >> 1;
    base = (thr[base + half - 1] <= U) ? base + half : base;
    len -= half;
  }
  return base;
}

// Draws the multi-index of draw t into idx[0..N).
__device__ __forceinline__ void draw(const SampleModes& sm, const uint64_t* const* thr, uint64_t t,
                                     uint32_t k0, uint32_t k1, uint32_t row, uint32_t cid, int* idx) {
  for (int k = 0; 2 * k < sm.N; ++k) {
    uint4 w = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)k + 256u * row, cid), k0, k1);
    idx[2 * k] = search_thr(thr[2 * k], sm.I[2 * k], u53(w.x, w.y));
    if (2 * k + 1 < sm.N) idx[2 * k + 1] = search_thr(thr[2 * k + 1], sm.I[2 * k + 1], u53(w.z, w.w));
  }
}

// Thresholds to shared memory when they fit (sum I_n <= 4096 entries = 32 KB).
constexpr int THR_SMEM = 4096;

__device__ __forceinline__ void load_thr(const SampleModes& sm, uint64_t* buf, const uint64_t** thr) {
  int tot = 0;
  for (int n = 0; n < sm.N; ++n) tot += sm.I[n];
  if (tot <= THR_SMEM) {
    int off = 0;
    for (int n = 0; n < sm.N; ++n) {
      for (int i = threadIdx.x; i < sm.I[n]; i += blockDim.x) buf[off + i] = sm.thr[n][i];
      thr[n] = buf + off;
      off += sm.I[n];
    }
  } else {
    for (int n = 0; n < sm.N; ++n) thr[n] = sm.thr[n];
  }
  __syncthreads();
}

// kron_sample surface: indices (s x N) and weights 1/sqrt(s prod p).
__global__ void k_sample_idx(SampleModes sm, int64_t s, uint32_t k0, uint32_t k1, uint32_t row, uint32_t cid,
                             int32_t* __restrict__ idx_out, float* __restrict__ w_out) {
  __shared__ uint64_t buf[THR_SMEM];
  const uint64_t* thr[KR_MAX_MODES];
  load_thr(sm, buf, thr);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < s; t += (int64_t)gridDim.x * blockDim.x) {
    int idx[KR_MAX_MODES];
    draw(sm, thr, (uint64_t)t, k0, k1, row, cid, idx);
    if (idx_out)
      for (int n = 0; n < sm.N; ++n) idx_out[t * sm.N + n] = idx[n];
    if (w_out) {
      double p = (double)s;
      for (int n = 0; n < sm.N; ++n) p *= sm.prob[n][idx[n]];
      w_out[t] = (float)(1.0 / sqrt(p));
    }
  }
}

// Solver path: cell id and last coordinate packed in one key; histogram by cell.
// Draws come in nrow batches of s_row (one batch per Tucker factor row; nrow = 1 for a
// plain solve). Draw t of batch r uses Philox counter row row0 + r. The key is
// cell * IT + i_T with cell = r * ncell_inner + (i_1..i_{N-1}) (the linear row index of
// the batched system). The histogram atomic returns each draw's rank inside its cell
// (rank[t]), so the scatter needs no atomics. Templated on N so the per-draw indices
// and table pointers stay in registers.
template <int N>
__global__ void __launch_bounds__(256) k_sample_keys(SampleModes sm, int64_t s_row, int nrow, uint32_t k0,
                                                     uint32_t k1, uint32_t row0, uint32_t cid, int64_t ncell_inner,
                                                     uint32_t* __restrict__ keys, uint32_t* __restrict__ rank,
                                                     uint32_t* __restrict__ cell_cnt) {
  __shared__ uint64_t buf[THR_SMEM];
  const uint64_t* thr[N];
  int In[N];
  {
    int tot = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) tot += sm.I[n];
    int off = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      In[n] = sm.I[n];
      if (tot <= THR_SMEM) {
        for (int i = threadIdx.x; i < In[n]; i += blockDim.x) buf[off + i] = sm.thr[n][i];
        thr[n] = buf + off;
        off += In[n];
      } else {
        thr[n] = sm.thr[n];
      }
    }
    __syncthreads();
  }
  const uint32_t IT = (uint32_t)In[N - 1];
  const int64_t total = s_row * nrow;
  const uint32_t lane = threadIdx.x & 31;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < total; t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    const bool live = t < total;
    uint32_t cell = 0, key = 0;
    if (live) {
      uint32_t r = 0;
      int64_t tl = t;
      if (nrow > 1) {
        r = (uint32_t)((uint64_t)t / (uint64_t)s_row);
        tl = t - (int64_t)r * s_row;
      }
      int idx[N];
#pragma unroll
      for (int k = 0; 2 * k < N; ++k) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)tl, (uint32_t)((uint64_t)tl >> 32), (uint32_t)k + 256u * (row0 + r), cid), k0, k1);
        idx[2 * k] = search_thr(thr[2 * k], In[2 * k], u53(w.x, w.y));
        if (2 * k + 1 < N) idx[2 * k + 1] = search_thr(thr[2 * k + 1], In[2 * k + 1], u53(w.z, w.w));
      }
#pragma unroll
      for (int n = 0; n < N - 1; ++n) cell = cell * (uint32_t)In[n] + (uint32_t)idx[n];
      cell += r * (uint32_t)ncell_inner;
      key = cell * IT + (uint32_t)idx[N - 1];
      keys[t] = key;
    }
    // warp-aggregated histogram increment; the returned base gives each draw its rank
    const unsigned act = __ballot_sync(0xffffffffu, live);
    if (live) {
      const unsigned peers = __match_any_sync(act, cell);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(&cell_cnt[cell], (uint32_t)__popc(peers));
      base = __shfl_sync(peers, base, leader);
      rank[t] = base + __popc(peers & ((1u << lane) - 1u));
    }
  }
}

// Scatter i_T of every draw into its cell's slot range (position = cell start + rank).
__global__ void k_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rank, int64_t s, uint32_t IT,
                          const uint32_t* __restrict__ start, uint16_t* __restrict__ slot) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < s; t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = keys[t];
    const uint32_t cell = key / IT;
    slot[start[cell] + rank[t]] = (uint16_t)(key - cell * IT);
  }
}

// Per cell (one warp): count table over i_T in shared memory, then emit the distinct
// entries in increasing i_T order with their multiplicities, gather b, and the
// per-cell weight prod_{n<N-1} 1/p_n(i_n) / s.
constexpr int DEDUP_WARPS = 8;
constexpr int DEDUP_MAX_IT = 8192;

// Batched rows: cell c belongs to row c / ncell_inner; its entry (c, i) is the row-major
// index key = (c % ncell_inner) * IT + i over the sampled modes, and b is read at
// ((key / xPafter) * xI + row) * xPafter + key % xPafter (X_(n) row `row`; for a plain
// solve xI = xPafter = 1 and the index is the key itself).
__global__ void k_dedup(SampleModes sm, int64_t ncell, int64_t ncell_inner, int64_t xI, int64_t xPafter, uint32_t IT,
                        float inv_s, const uint32_t* __restrict__ start,
                        const uint32_t* __restrict__ cnt, const uint16_t* __restrict__ slot, const float* __restrict__ b,
                        uint32_t* __restrict__ ent, float* __restrict__ bt, uint32_t* __restrict__ nd,
                        float* __restrict__ cell_w) {
  extern __shared__ uint32_t tabs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* tab = tabs + (size_t)warp * IT;
  for (uint32_t i = lane; i < IT; i += 32) tab[i] = 0;
  __syncwarp();
  const uint32_t chunk = (IT + 31) / 32;
  const uint32_t lo = min(IT, lane * chunk), hi = min(IT, lo + chunk);
  for (int64_t c = (int64_t)blockIdx.x * DEDUP_WARPS + warp; c < ncell; c += (int64_t)gridDim.x * DEDUP_WARPS) {
    const uint32_t n = cnt[c], base = start[c];
    const uint32_t c32 = (uint32_t)c, nci = (uint32_t)ncell_inner;
    const uint32_t row32 = c32 / nci;
    const int64_t c_in = (int64_t)(c32 - row32 * nci), row = row32;
    if (lane == 0) {
      // weight of the cell: prod over the first N-1 coordinates of 1/p
      float w = inv_s;
      uint32_t rem = (uint32_t)c_in;
      for (int m = sm.N - 2; m >= 0; --m) {
        const uint32_t Im = (uint32_t)sm.I[m];
        const uint32_t q = rem / Im;
        w *= sm.invp[m][rem - q * Im];
        rem = q;
      }
      cell_w[c] = w;
    }
    if (n == 0) {
      if (lane == 0) nd[c] = 0;
      continue;
    }
    for (uint32_t j = lane; j < n; j += 32) atomicAdd(&tab[slot[base + j]], 1u);
    __syncwarp();
    uint32_t mine = 0;
    for (uint32_t i = lo; i < hi; ++i) {
      uint32_t v = tab[i];
      mine += (v + 65534u) / 65535u;  // entries needed (multiplicity stored in 16 bits)
    }
    uint32_t incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    uint32_t pos = base + incl - mine;
    const int64_t rowbase = c_in * (int64_t)IT;
    for (uint32_t i = lo; i < hi; ++i) {
      uint32_t v = tab[i];
      if (v == 0) continue;
      tab[i] = 0;
      float bv = 0.f;
      if (b) {
        const int64_t key = rowbase + i;
        const int64_t bi = (xPafter == 1 && xI == 1) ? key : ((key / xPafter) * xI + row) * xPafter + key % xPafter;
        bv = b[bi];
      }
      while (v > 0) {
        uint32_t take = v > 65535u ? 65535u : v;
        ent[pos] = i | (take << 16);
        bt[pos] = bv;
        ++pos;
        v -= take;
      }
    }
    uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) nd[c] = total;
    __syncwarp();
  }
}

// Compaction of the merged entries: cell c's nd[c] entries move from its draw-sized
// region at start[c] to position newstart[c] (exclusive scan of nd), so that the entries
// of consecutive cells lie back to back. One warp per cell; the copy goes to scratch and
// k_copy_back returns the first total[0] entries.
__global__ void k_compact(int64_t ncell, const uint32_t* __restrict__ start, const uint32_t* __restrict__ newstart,
                          const uint32_t* __restrict__ nd, const uint32_t* __restrict__ ent,
                          const float* __restrict__ bt, uint32_t* __restrict__ ent2, float* __restrict__ bt2) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell; c += warps) {
    const uint32_t n = nd[c], from = start[c], to = newstart[c];
    for (uint32_t k = lane; k < n; k += 32) {
      ent2[to + k] = ent[from + k];
      bt2[to + k] = bt[from + k];
    }
  }
}

__global__ void k_copy_back(const unsigned long long* __restrict__ total, const uint32_t* __restrict__ ent2,
                            const float* __restrict__ bt2, uint32_t* __restrict__ ent, float* __restrict__ bt) {
  const int64_t n = (int64_t)total[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ent[i] = ent2[i];
    bt[i] = bt2[i];
  }
}

// Sketch export: linear keys, counts, weights and b~ in increasing key order.
__global__ void k_export(int64_t ncell, uint32_t IT, const uint32_t* __restrict__ start, const uint32_t* __restrict__ nd,
                         const uint32_t* __restrict__ off, const uint32_t* __restrict__ ent, const float* __restrict__ bt,
                         const float* __restrict__ cell_w, const float* __restrict__ invpT, int64_t* keys,
                         int32_t* counts, float* omega, float* btilde) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    uint32_t n = nd[c], b0 = start[c], o = off[c];
    for (uint32_t k = 0; k < n; ++k) {
      uint32_t e = ent[b0 + k];
      uint32_t it = e & 0xFFFFu, ct = e >> 16;
      if (keys) keys[o + k] = c * (int64_t)IT + it;
      if (counts) counts[o + k] = (int32_t)ct;
      if (omega) omega[o + k] = (float)ct * cell_w[c] * invpT[it];
      if (btilde) btilde[o + k] = bt[b0 + k];
    }
  }
}

// Cell descriptors in processing order: one 16-byte load per cell in the residual pass.
__global__ void k_build_desc(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ start,
                             const uint32_t* __restrict__ nd, const float* __restrict__ cw, int64_t ncell,
                             uint4* __restrict__ desc) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ncell; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = perm[q];
    desc[q] = make_uint4(c, start[c], nd[c], __float_as_uint(cw[c]));
  }
}

__global__ void k_sum_u32(const uint32_t* __restrict__ v, int64_t n, unsigned long long* out) {
  unsigned long long acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) acc += v[i];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

SampleModes make_sample_modes(const Modes& m, const FactorTables& t) {
  SampleModes sm = {};
  sm.N = m.N;
  for (int n = 0; n < m.N; ++n) {
    sm.I[n] = m.I[n];
    sm.thr[n] = t.thr[n];
    sm.prob[n] = t.prob[n];
    sm.invp[n] = t.invp[n];
  }
  return sm;
}

int grid_for(kr_ctx* ctx, int64_t work, int block, int per_sm = 8) {
  int64_t g = (work + block - 1) / block;
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void kr_sketch_setup(kr_sketch* sk, const Modes& m, int64_t s) { kr_sketch_setup_rows(sk, m, s, 1, 1, 1); }

void kr_sketch_setup_rows(kr_sketch* sk, const Modes& m, int64_t s_row, int nrow, int64_t xI, int64_t xPafter) {
  sk->N = m.N;
  for (int n = 0; n < m.N; ++n) sk->I[n] = m.I[n];
  sk->s_row = s_row;
  sk->nrow = nrow;
  sk->s = s_row * nrow;
  int64_t ncell = 1;
  for (int n = 0; n < m.N - 1; ++n) ncell *= m.I[n];
  sk->ncell_inner = ncell;
  sk->ncell = ncell * nrow;
  sk->IT = m.I[m.N - 1];
  sk->xI = xI;
  sk->xPafter = xPafter;
}

void kr_sketch_own_need(const kr_sketch* sk, Need& nd) {
  nd.add<uint32_t>(sk->ncell);
  nd.add<uint32_t>(sk->ncell);
  nd.add<uint32_t>(sk->s);
  nd.add<float>(sk->s);
  nd.add<float>(sk->ncell);
  nd.add<float>(sk->IT);
  nd.add<uint32_t>(sk->ncell);
  nd.add<uint4>(sk->ncell);
}

void kr_sketch_layout(kr_sketch* sk, Carve& cv) {
  sk->cell_start = cv.take<uint32_t>(sk->ncell);
  sk->cell_nd = cv.take<uint32_t>(sk->ncell);
  sk->ent = cv.take<uint32_t>(sk->s);
  sk->bt = cv.take<float>(sk->s);
  sk->cell_w = cv.take<float>(sk->ncell);
  sk->invpT = cv.take<float>(sk->IT);
  sk->perm = cv.take<uint32_t>(sk->ncell);
  sk->desc = cv.take<uint4>(sk->ncell);
}

kr_status kr_sketch_check(kr_ctx* ctx, const Modes& m, int64_t s) {
  if (s < 1 || s >= (int64_t(1) << 31)) return kr_fail(ctx, KR_EINVAL, "sketch: s=%lld outside [1, 2^31)", (long long)s);
  if (m.I[m.N - 1] > DEDUP_MAX_IT)
    return kr_fail(ctx, KR_ENOTIMPL, "sketch: last mode size %d exceeds %d", m.I[m.N - 1], DEDUP_MAX_IT);
  return KR_OK;
}

// Second phase of the sketch build, with scratch carved from `cv`.
kr_status kr_sketch_fill(kr_ctx* ctx, const Modes& m, const FactorTables& t, const float* b, uint64_t seed,
                         uint64_t call_id, int row, kr_sketch* sk, Carve& cv) {
  const int N = m.N;
  const int64_t s = sk->s, ncell = sk->ncell;
  const uint32_t IT = (uint32_t)sk->IT;
  uint32_t* keys = cv.take<uint32_t>(s);
  uint32_t* cnt = cv.take<uint32_t>(ncell);
  uint32_t* rank = cv.take<uint32_t>(s);
  uint16_t* slot = cv.take<uint16_t>(s);
  unsigned long long* dsum = cv.take<unsigned long long>(1);
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "sketch: workspace too small");
  SampleModes sm = make_sample_modes(m, t);
  KR_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * ncell, ctx->stream));
  KR_CUDA(ctx, cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), ctx->stream));
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32), cid = (uint32_t)call_id;
  {
    const int gs = grid_for(ctx, s, 256);
#define KR_SAMPLE_KEYS(NN)                                                                                \
  case NN:                                                                                                \
    KR_LAUNCH(ctx, k_sample_keys<NN>, gs, 256, 0, sm, sk->s_row, sk->nrow, k0, k1, (uint32_t)row, cid,     \
              sk->ncell_inner, keys, rank, cnt);                                                          \
    break;
    switch (N) {
      KR_SAMPLE_KEYS(1)
      KR_SAMPLE_KEYS(2)
      KR_SAMPLE_KEYS(3)
      KR_SAMPLE_KEYS(4)
      KR_SAMPLE_KEYS(5)
      KR_SAMPLE_KEYS(6)
      KR_SAMPLE_KEYS(7)
      KR_SAMPLE_KEYS(8)
      default:
        return kr_fail(ctx, KR_EINVAL, "sketch: N=%d", N);
    }
#undef KR_SAMPLE_KEYS
  }
  {
    Carve sc = cv;  // scan scratch is transient
    KR_TRY(kr_scan_u32(ctx, cnt, sk->cell_start, ncell, sc));
  }
  KR_LAUNCH(ctx, k_scatter, grid_for(ctx, s, 256), 256, 0, keys, rank, s, IT, sk->cell_start, slot);
  const size_t dsmem = (size_t)DEDUP_WARPS * IT * sizeof(uint32_t);
  KR_CUDA(ctx, cudaFuncSetAttribute(k_dedup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
  KR_LAUNCH(ctx, k_dedup, grid_for(ctx, ncell, DEDUP_WARPS, 8), DEDUP_WARPS * 32, dsmem, sm, ncell, sk->ncell_inner,
            sk->xI, sk->xPafter, IT, (float)(1.0 / (double)sk->s_row), sk->cell_start, cnt, slot, b, sk->ent, sk->bt,
            sk->cell_nd, sk->cell_w);
  // entries back to back in cell order (the draw-sized regions leave gaps)
  {
    Carve sc = cv;
    KR_TRY(kr_scan_u32(ctx, sk->cell_nd, cnt, ncell, sc));
  }
  KR_LAUNCH(ctx, k_sum_u32, grid_for(ctx, ncell, 256, 2), 256, 0, sk->cell_nd, ncell, dsum);
  KR_LAUNCH(ctx, k_compact, grid_for(ctx, ncell, 8, 8), 256, 0, ncell, sk->cell_start, cnt, sk->cell_nd, sk->ent,
            sk->bt, keys, reinterpret_cast<float*>(rank));
  KR_LAUNCH(ctx, k_copy_back, grid_for(ctx, s, 256), 256, 0, dsum, keys, reinterpret_cast<const float*>(rank), sk->ent,
            sk->bt);
  KR_CUDA(ctx, cudaMemcpyAsync(sk->cell_start, cnt, sizeof(uint32_t) * ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  if (sk->want_desc) {
    Carve sc = cv;
    KR_TRY(kr_balance_perm(ctx, sk->cell_nd, ncell, sk->perm, sc));
    KR_LAUNCH(ctx, k_build_desc, grid_for(ctx, ncell, 256), 256, 0, sk->perm, sk->cell_start, sk->cell_nd,
              sk->cell_w, ncell, sk->desc);
  }
  KR_CUDA(ctx, cudaMemcpyAsync(sk->invpT, t.invp[N - 1], sizeof(float) * IT, cudaMemcpyDeviceToDevice, ctx->stream));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  KR_CUDA(ctx, cudaMemcpyAsync(ctx->hbuf, dsum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  sk->distinct = (int64_t)(*(unsigned long long*)ctx->hbuf);
  return KR_OK;
}

void kr_sketch_scratch_need(int64_t s, int64_t ncell, Need& nd) {
  nd.add<uint32_t>(s);
  nd.add<uint32_t>(ncell);
  nd.add<uint32_t>(s);
  nd.add<uint16_t>(s);
  nd.add<unsigned long long>(1);
  kr_scan_need(ncell, nd);
  kr_perm_need(ncell, nd);
}

// ------------------------------------------------------------------ C ABI

__global__ void k_thr_from_cdf(const double* cdf, uint64_t* thr, int n);
__global__ void k_invp_from_prob(const double* prob, float* invp, int n);

extern "C" kr_status kron_sample(kr_ctx* ctx, int32_t N, const int64_t* I, const double* const cdf[],
                                 const double* const prob[], int64_t s, uint64_t seed, uint64_t call_id, int32_t row,
                                 int32_t* idx, float* w) {
  if (!ctx) return KR_EINVAL;
  if (N < 1 || N > KR_MAX_MODES || !I || !cdf) return kr_fail(ctx, KR_EINVAL, "kron_sample: bad N or null arrays");
  if (s < 1 || s >= (int64_t(1) << 31)) return kr_fail(ctx, KR_EINVAL, "kron_sample: s outside [1, 2^31)");
  if (row < 0 || row >= (1 << 24)) return kr_fail(ctx, KR_EINVAL, "kron_sample: row outside [0, 2^24)");
  if (w && !prob) return kr_fail(ctx, KR_EINVAL, "kron_sample: weights need prob");
  Need nd;
  for (int n = 0; n < N; ++n) {
    if (I[n] < 1 || I[n] > 65535 || !cdf[n]) return kr_fail(ctx, KR_EINVAL, "kron_sample: bad I[%d] or cdf[%d]", n, n);
    nd.add<uint64_t>(I[n]);
  }
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  Carve cv(ctx->ws, ctx->ws_size);
  SampleModes sm = {};
  sm.N = N;
  for (int n = 0; n < N; ++n) {
    sm.I[n] = (int)I[n];
    uint64_t* thr = cv.take<uint64_t>(I[n]);
    sm.thr[n] = thr;
    sm.prob[n] = prob ? prob[n] : nullptr;
  }
  // thresholds from the caller's CDF tables
  for (int n = 0; n < N; ++n) {
    KR_LAUNCH(ctx, k_thr_from_cdf, grid_for(ctx, I[n], 256), 256, 0, cdf[n], const_cast<uint64_t*>(sm.thr[n]),
              (int)I[n]);
  }
  KR_LAUNCH(ctx, k_sample_idx, grid_for(ctx, s, 256), 256, 0, sm, s, (uint32_t)seed, (uint32_t)(seed >> 32),
            (uint32_t)row, (uint32_t)call_id, idx, w);
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return KR_OK;
}

__global__ void k_thr_from_cdf(const double* cdf, uint64_t* thr, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    thr[i] = (uint64_t)ceil(cdf[i] * 9007199254740992.0);
}

extern "C" kr_status kron_sketch(kr_ctx* ctx, const kr_factors* f, const double* const cdf[], const double* const prob[],
                                 const float* b, int64_t s, uint64_t seed, uint64_t call_id, int32_t row,
                                 kr_sketch** out) {
  if (!ctx || !out) return KR_EINVAL;
  *out = nullptr;
  Modes m;
  KR_TRY(kr_check_factors(ctx, f, &m));
  if (!cdf || !prob) return kr_fail(ctx, KR_EINVAL, "kron_sketch: cdf and prob are required");
  if (row < 0 || row >= (1 << 24)) return kr_fail(ctx, KR_EINVAL, "kron_sketch: row outside [0, 2^24)");
  int64_t ncell = 1;
  for (int n = 0; n < m.N - 1; ++n) ncell *= m.I[n];
  Need nd;
  for (int n = 0; n < m.N; ++n) {
    nd.add<uint64_t>(m.I[n]);
    nd.add<double>(m.I[n]);
    nd.add<float>(m.I[n]);
  }
  kr_sketch_scratch_need(s, ncell, nd);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  Carve cv(ctx->ws, ctx->ws_size);
  FactorTables t;
  t.N = m.N;
  for (int n = 0; n < m.N; ++n) {
    t.thr[n] = cv.take<uint64_t>(m.I[n]);
    t.prob[n] = const_cast<double*>(prob[n]);
    t.invp[n] = cv.take<float>(m.I[n]);
    KR_LAUNCH(ctx, k_thr_from_cdf, grid_for(ctx, m.I[n], 256), 256, 0, cdf[n], t.thr[n], m.I[n]);
    KR_LAUNCH(ctx, k_invp_from_prob, grid_for(ctx, m.I[n], 256), 256, 0, prob[n], t.invp[n], m.I[n]);
  }
  KR_TRY(kr_sketch_check(ctx, m, s));
  kr_sketch* sk = new kr_sketch();
  kr_sketch_setup(sk, m, s);
  Need own;
  kr_sketch_own_need(sk, own);
  cudaError_t e = cudaMalloc((void**)&sk->mem, own.off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete sk;
    return kr_fail(ctx, KR_ENOMEM, "kron_sketch: allocation of %zu bytes failed", own.off);
  }
  Carve oc(sk->mem, own.off);
  kr_sketch_layout(sk, oc);
  kr_status st = kr_sketch_fill(ctx, m, t, b, seed, call_id, row, sk, cv);
  if (st != KR_OK) {
    kron_sketch_free(sk);
    return st;
  }
  *out = sk;
  return KR_OK;
}

__global__ void k_invp_from_prob(const double* prob, float* invp, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double p = prob[i];
    invp[i] = p > 0.0 ? (float)(1.0 / p) : 0.f;
  }
}

extern "C" int64_t kron_sketch_distinct(const kr_sketch* sk) { return sk ? sk->distinct : 0; }

extern "C" kr_status kron_sketch_export(kr_ctx* ctx, const kr_sketch* sk, int64_t* keys, int32_t* counts, float* omega,
                                        float* btilde) {
  if (!ctx || !sk) return KR_EINVAL;
  Need nd;
  nd.add<uint32_t>(sk->ncell);
  kr_scan_need(sk->ncell, nd);
  KR_TRY(kr_ws_reserve(ctx, nd.off));
  Carve cv(ctx->ws, ctx->ws_size);
  uint32_t* off = cv.take<uint32_t>(sk->ncell);
  KR_TRY(kr_scan_u32(ctx, sk->cell_nd, off, sk->ncell, cv));
  KR_LAUNCH(ctx, k_export, grid_for(ctx, sk->ncell, 128), 128, 0, sk->ncell, (uint32_t)sk->IT, sk->cell_start,
            sk->cell_nd, off, sk->ent, sk->bt, sk->cell_w, sk->invpT, keys, counts, omega, btilde);
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return KR_OK;
}

extern "C" void kron_sketch_free(kr_sketch* sk) {
  if (!sk) return;
  if (sk->mem) {
    cudaDeviceSynchronize();
    cudaFree(sk->mem);
  }
  delete sk;
}

// ------------------------------------------------------------------ allocation-free sampling

#include <mutex>

// Scratch of kron_sample_noalloc: integer thresholds of the caller's CDF tables.
static __device__ __align__(256) uint64_t kr_noalloc_thr[KR_NOALLOC_MAX_ROWS];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex noalloc_mu;
uint64_t* noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of kr_noalloc_thr on the current device, looked up once per device.
kr_status noalloc_scratch(kr_ctx* ctx, uint64_t** out) {
  int dev = -1;
  KR_CUDA(ctx, cudaGetDevice(&dev));
  if (dev != ctx->device) return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: current device %d is not the context's device %d", dev, ctx->device);
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(noalloc_mu);
  if (!noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, kr_noalloc_thr);
    if (e != cudaSuccess || !p) return kr_fail_cuda(ctx, e, "cudaGetSymbolAddress(kr_noalloc_thr)", __FILE__, __LINE__);
    noalloc_ptr[dev] = static_cast<uint64_t*>(p);
  }
  *out = noalloc_ptr[dev];
  return KR_OK;
}
}  // namespace

extern "C" kr_status kron_sample_noalloc(kr_ctx* ctx, int32_t N, const int64_t* I, const double* const cdf[],
                                         const double* const prob[], int64_t s, uint64_t seed, uint64_t call_id,
                                         int32_t row, int32_t* idx, float* w) {
  if (!ctx) return KR_EINVAL;
  if (N < 1 || N > KR_MAX_MODES || !I || !cdf) return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: bad N or null arrays");
  if (s < 1 || s >= (int64_t(1) << 31)) return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: s outside [1, 2^31)");
  if (row < 0 || row >= (1 << 24)) return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: row outside [0, 2^24)");
  if (w && !prob) return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: weights need prob");
  int64_t total = 0;
  for (int n = 0; n < N; ++n) {
    if (I[n] < 1 || I[n] > 65535 || !cdf[n])
      return kr_fail(ctx, KR_EINVAL, "kron_sample_noalloc: bad I[%d] or cdf[%d]", n, n);
    total += I[n];
  }
  if (total > KR_NOALLOC_MAX_ROWS)
    return kr_fail(ctx, KR_EINVAL,
                   "kron_sample_noalloc: the tables hold %lld rows in total, above the static scratch limit "
                   "KR_NOALLOC_MAX_ROWS = %d (use kron_sample)",
                   (long long)total, KR_NOALLOC_MAX_ROWS);
  uint64_t* scratch = nullptr;
  KR_TRY(noalloc_scratch(ctx, &scratch));
  SampleModes sm = {};
  sm.N = N;
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    sm.I[n] = (int)I[n];
    sm.thr[n] = scratch + off;
    sm.prob[n] = prob ? prob[n] : nullptr;
    KR_LAUNCH(ctx, k_thr_from_cdf, grid_for(ctx, I[n], 256), 256, 0, cdf[n], scratch + off, (int)I[n]);
    off += I[n];
  }
  KR_LAUNCH(ctx, k_sample_idx, grid_for(ctx, s, 256), 256, 0, sm, s, (uint32_t)seed, (uint32_t)(seed >> 32),
            (uint32_t)row, (uint32_t)call_id, idx, w);
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return KR_OK;
}
