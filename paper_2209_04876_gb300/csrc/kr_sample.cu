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
// cell = (i_1..i_{N-1}), the last coordinate i_N stays with the sample. Every draw
// writes its row key cell * I_N + i_N. The distinct keys and their multiplicities, in
// increasing key order, come either from ranks in a bitmap of the key space (when it
// holds at most 64 keys per draw) or from a stable radix sort of the keys (kr_sort.cu)
// and its runs of equal keys; both give the merged entries (i_N, multiplicity) of each
// cell in increasing i_N order, with b gathered.
#include "kr_internal.cuh"

namespace {

struct SampleModes {
  int N;
  int I[KR_MAX_MODES];
  const uint64_t* thr[KR_MAX_MODES];
  const double* prob[KR_MAX_MODES];
  const float* invp[KR_MAX_MODES];
};

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

// Draws of 3 or 4 coordinates take one Philox call (counter word 2 = 256 row): its 128 bits,
// w.x most significant, cut from the top into N chunks of floor(128 / N) bits (42 or 32),
// each placed on the 53-bit threshold grid (U = chunk << (53 - bits)). Other N: one call per
// two coordinates, 53 bits each.
__device__ __forceinline__ void chunk_uniforms(uint4 w, int N, uint64_t* U) {
  if (N == 4) {
    U[0] = (uint64_t)w.x << 21;
    U[1] = (uint64_t)w.y << 21;
    U[2] = (uint64_t)w.z << 21;
    U[3] = (uint64_t)w.w << 21;
  } else {
    U[0] = (((uint64_t)w.x << 10) | (w.y >> 22)) << 11;
    U[1] = (((uint64_t)(w.y & 0x3FFFFFu) << 20) | (w.z >> 12)) << 11;
    U[2] = (((uint64_t)(w.z & 0xFFFu) << 30) | (w.w >> 2)) << 11;
  }
}

// Draws the multi-index of draw t into idx[0..N).
__device__ __forceinline__ void draw(const SampleModes& sm, const uint64_t* const* thr, uint64_t t,
                                     uint32_t k0, uint32_t k1, uint32_t row, uint32_t cid, int* idx) {
  if (sm.N == 3 || sm.N == 4) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 256u * row, cid), k0, k1);
    uint64_t U[4];
    chunk_uniforms(w, sm.N, U);
    for (int m = 0; m < sm.N; ++m) idx[m] = search_thr(thr[m], sm.I[m], U[m]);
    return;
  }
  for (int k = 0; 2 * k < sm.N; ++k) {
    uint4 w = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)k + 256u * row, cid), k0, k1);
    idx[2 * k] = search_thr(thr[2 * k], sm.I[2 * k], u53(w.x, w.y));
    if (2 * k + 1 < sm.N) idx[2 * k + 1] = search_thr(thr[2 * k + 1], sm.I[2 * k + 1], u53(w.z, w.w));
  }
}

// Thresholds to shared memory when they fit (sum I_n <= 4096 entries = 32 KB).
constexpr int THR_SMEM = 4096;
constexpr int GUIDE_MAX = 65536;  // guide entries per mode at most (I_n <= 65535)

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

// Guide table of one mode (Chen & Asau's indexed search): g[m] = smallest i with
// thr[i] > m * 2^shift, so the inverse-CDF search of U starts at g[U >> shift] and steps
// forward while thr[i] <= U. The result is the same index as the binary search.
__global__ void k_guide(const uint64_t* __restrict__ thr, int n, int shift, int M, uint16_t* __restrict__ g) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x)
    g[m] = (uint16_t)search_thr(thr, n, (uint64_t)m << shift);
}

struct DrawModes {
  int N;
  int I[KR_MAX_MODES];
  int shift[KR_MAX_MODES];  // 53 - log2(guide entries)
  int M[KR_MAX_MODES];      // guide entries
  const uint64_t* thr[KR_MAX_MODES];
  const uint16_t* guide[KR_MAX_MODES];
  const uint16_t* prk[KR_MAX_MODES];  // rows ranked by decreasing probability (dense counters; or null)
};

// Dense counters are addressed by each index's rank in its mode's decreasing-probability
// order (the key's bitmap bit and every output stay in the original key order). Draws
// concentrate on the most probable rows (high-leverage rows: a few per cent of a mode's
// rows can carry most of its mass), so this packs the busiest counters into a corner of
// the array and their atomic updates touch far fewer L2 sectors. Modes of at most PRK_MAX
// rows (a rank table of uint16 per mode).
constexpr int PRK_MAX = 4096;

struct ProbRanks {
  int I[KR_MAX_MODES];
  const double* prob[KR_MAX_MODES];
  uint16_t* out[KR_MAX_MODES];
};

// out[n][i] = #{ j : p_j > p_i, or p_j = p_i and j < i }: row i's place when mode n's rows
// are sorted by decreasing probability (ties by index). Block (n, c) ranks rows
// [256 c, 256 c + 256) of mode n.
// Probabilities are non-negative doubles, which order exactly as their bit patterns do as
// unsigned integers, so the comparisons run on the integer pipe.
__global__ void __launch_bounds__(256) k_prob_rank(ProbRanks pr) {
  __shared__ unsigned long long sp[PRK_MAX];
  const int n = blockIdx.x, I = pr.I[n];
  if (256 * (int)blockIdx.y >= I) return;
  for (int i = threadIdx.x; i < I; i += blockDim.x) sp[i] = (unsigned long long)__double_as_longlong(pr.prob[n][i]);
  __syncthreads();
  {
    const int i = 256 * blockIdx.y + threadIdx.x;
    if (i >= I) return;
    const unsigned long long pi = sp[i];
    int r = 0;
    for (int j = 0; j < I; ++j) {
      const unsigned long long pj = sp[j];
      r += (pj > pi || (pj == pi && j < i)) ? 1 : 0;
    }
    pr.out[n][i] = (uint16_t)r;
  }
}

// thr[I - 1] = 2^53 > U (both table builders set it), so the forward steps end in the table.
__device__ __forceinline__ int guided_search(const uint64_t* thr, const uint16_t* guide, int shift, uint64_t U) {
  int i = guide[U >> shift];
  while (thr[i] <= U) ++i;
  return i;
}

// Solver path: every draw's row key cell * IT + i_T (cell = r * ncell_inner +
// (i_1..i_{N-1}) for draw batch r, the linear row index of the batched system). Draws
// come in nrow batches of s_row (one per Tucker factor row; nrow = 1 for a plain solve);
// draw t of batch r uses Philox counter row row0 + r. With a key bitmap (grouping by
// rank, below) every draw also sets its key's bit there. With dense counts (dcnt: one
// counter per key of the key space, zero on entry) a draw adds one to its key's counter
// instead of writing the key, and only the first draw of a key (the counter was 0) sets
// its bit. Templated on N so the per-draw indices and table pointers stay in registers.
template <int N>
__global__ void __launch_bounds__(256) k_draw_keys(DrawModes dm, int64_t s_row, int nrow, uint32_t k0, uint32_t k1,
                                                   uint32_t row0, uint32_t cid, uint32_t ncell_inner,
                                                   uint32_t* __restrict__ keys, uint2* __restrict__ bm,
                                                   uint32_t* __restrict__ dcnt) {
  __shared__ uint64_t s_thr[THR_SMEM];
  __shared__ uint16_t s_guide[THR_SMEM];
  __shared__ uint16_t s_prk[THR_SMEM];
  const uint64_t* thr[N];
  const uint16_t* guide[N];
  const uint16_t* prk[N];
  int In[N], sh[N];
  {
    int ti = 0, tm = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      ti += dm.I[n];
      tm += dm.M[n];
    }
    const bool fit = ti <= THR_SMEM && tm <= THR_SMEM;
    int oi = 0, om = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      In[n] = dm.I[n];
      sh[n] = dm.shift[n];
      if (fit) {
        for (int i = threadIdx.x; i < In[n]; i += blockDim.x) s_thr[oi + i] = dm.thr[n][i];
        for (int i = threadIdx.x; i < dm.M[n]; i += blockDim.x) s_guide[om + i] = dm.guide[n][i];
        if (dm.prk[0])
          for (int i = threadIdx.x; i < In[n]; i += blockDim.x) s_prk[oi + i] = dm.prk[n][i];
        thr[n] = s_thr + oi;
        guide[n] = s_guide + om;
        prk[n] = s_prk + oi;
        oi += In[n];
        om += dm.M[n];
      } else {
        thr[n] = dm.thr[n];
        guide[n] = dm.guide[n];
        prk[n] = dm.prk[n];
      }
    }
    __syncthreads();
  }
  const uint32_t IT = (uint32_t)In[N - 1];
  const int64_t total = s_row * nrow;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t r = 0;
    int64_t tl = t;
    if (nrow > 1) {
      r = (uint32_t)((uint64_t)t / (uint64_t)s_row);
      tl = t - (int64_t)r * s_row;
    }
    int idx[N];
    if (N == 3 || N == 4) {  // one Philox call for the whole draw (chunk_uniforms)
      const uint4 w =
          philox4x32_10(make_uint4((uint32_t)tl, (uint32_t)((uint64_t)tl >> 32), 256u * (row0 + r), cid), k0, k1);
      uint64_t U[4];
      chunk_uniforms(w, N, U);
#pragma unroll
      for (int m = 0; m < N; ++m) idx[m] = guided_search(thr[m], guide[m], sh[m], U[m]);
    } else {
#pragma unroll
      for (int k = 0; 2 * k < N; ++k) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)tl, (uint32_t)((uint64_t)tl >> 32), (uint32_t)k + 256u * (row0 + r), cid), k0, k1);
        idx[2 * k] = guided_search(thr[2 * k], guide[2 * k], sh[2 * k], u53(w.x, w.y));
        if (2 * k + 1 < N)
          idx[2 * k + 1] = guided_search(thr[2 * k + 1], guide[2 * k + 1], sh[2 * k + 1], u53(w.z, w.w));
      }
    }
    uint32_t cell = 0;
#pragma unroll
    for (int n = 0; n < N - 1; ++n) cell = cell * (uint32_t)In[n] + (uint32_t)idx[n];
    cell += r * ncell_inner;
    const uint32_t key = cell * IT + (uint32_t)idx[N - 1];
    if (dcnt) {
      uint32_t ckey = key;  // the key's counter
      if (dm.prk[0]) {
        uint32_t pc = 0;
#pragma unroll
        for (int n = 0; n < N - 1; ++n) pc = pc * (uint32_t)In[n] + (uint32_t)prk[n][idx[n]];
        ckey = (pc + r * ncell_inner) * IT + (uint32_t)prk[N - 1][idx[N - 1]];
      }
      if (atomicAdd(dcnt + ckey, 1u) == 0u) atomicOr(&bm[key >> 5].x, 1u << (key & 31));
    } else {
      keys[t] = key;
      if (bm) atomicOr(&bm[key >> 5].x, 1u << (key & 31));
    }
  }
}

// ------------------------------------------------------------------ runs of equal keys
//
// Runs of equal sorted keys become the merged entries of the sketch in four passes that
// touch the keys twice: heads counted per tile of 4096 keys, the run starts written in
// order (the tile counts scanned), entries past one per run counted per tile of runs (a
// multiplicity above 65535 takes several entries; such runs are rare), then the entries
// emitted with b gathered.

constexpr int RLE_THREADS = 256;
constexpr int RLE_ITEMS = 16;
constexpr int RLE_TILE = RLE_THREADS * RLE_ITEMS;  // keys (or runs) per block

constexpr int RUN_ITEMS = 4;                          // runs per thread in the extras count and the emit
constexpr int RUN_TILE = RLE_THREADS * RUN_ITEMS;      // runs per block there

// Words of the run merge's per-tile arrays: head counts and their offsets per key tile,
// extras and their offsets per run tile.
int64_t rle_scratch_words(int64_t s) {
  return 2 * ((s + RLE_TILE - 1) / RLE_TILE) + 2 * ((s + RUN_TILE - 1) / RUN_TILE);
}

__device__ __forceinline__ uint32_t rle_block_sum(uint32_t v, uint32_t* sh) {  // sh: RLE_THREADS / 32 words
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < RLE_THREADS / 32; ++w) t += sh[w];
  __syncthreads();
  return t;
}

// Exclusive block scan (block of RLE_THREADS threads); sh: RLE_THREADS / 32 + 1 words.
__device__ __forceinline__ uint32_t rle_block_excl(uint32_t v, uint32_t* sh, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < RLE_THREADS / 32 ? sh[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += t;
    }
    if (lane < RLE_THREADS / 32) sh[lane] = wi - w;
    if (lane == RLE_THREADS / 32 - 1) sh[RLE_THREADS / 32] = wi;
  }
  __syncthreads();
  const uint32_t r = sh[warp] + incl - v;
  *total = sh[RLE_THREADS / 32];
  __syncthreads();
  return r;
}

// Run heads per tile of the sorted keys (a head starts a run of equal keys).
__global__ void __launch_bounds__(RLE_THREADS) k_rle_tcount(const uint32_t* __restrict__ k, int64_t n,
                                                            uint32_t* __restrict__ tcnt) {
  __shared__ uint32_t sh[RLE_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * RLE_TILE;
  uint32_t c = 0;
#pragma unroll 4
  for (int i = 0; i < RLE_ITEMS; ++i) {
    const int64_t e = base + (int64_t)i * RLE_THREADS + threadIdx.x;
    if (e < n && (e == 0 || __ldg(k + e) != __ldg(k + e - 1))) ++c;
  }
  const uint32_t t = rle_block_sum(c, sh);
  if (threadIdx.x == 0) tcnt[blockIdx.x] = t;
}

// Run starts: hp[d] = first key index of run d (toff: exclusive scan of the tile head
// counts). A thread flags 16 consecutive keys of the tile (staged in shared memory); the
// tile's starts are collected in shared memory and written out coalesced. The last tile
// sets hp[nd] = n and meta[0] = nd.
__global__ void __launch_bounds__(RLE_THREADS) k_rle_starts(const uint32_t* __restrict__ k, int64_t n,
                                                            const uint32_t* __restrict__ toff, int ntile,
                                                            uint32_t* __restrict__ hp, uint32_t* __restrict__ meta) {
  __shared__ uint32_t sh[RLE_THREADS / 32 + 1];
  __shared__ uint32_t buf[RLE_TILE + RLE_TILE / 32];
  __shared__ uint32_t first_head;
#define PADJ(j) ((j) + ((j) >> 5))
  const int64_t base = (int64_t)blockIdx.x * RLE_TILE;
  for (int i = 0; i < RLE_ITEMS; ++i) {
    const int j = i * RLE_THREADS + threadIdx.x;
    const int64_t e = base + j;
    buf[PADJ(j)] = e < n ? __ldg(k + e) : 0u;
  }
  if (threadIdx.x == 0) first_head = (base == 0 || __ldg(k + base) != __ldg(k + base - 1)) ? 1u : 0u;
  __syncthreads();
  uint32_t flags = 0;
  const int j0 = threadIdx.x * RLE_ITEMS;
#pragma unroll
  for (int i = 0; i < RLE_ITEMS; ++i) {
    const int j = j0 + i;
    if (base + j < n) {
      const bool head = j == 0 ? first_head != 0u : buf[PADJ(j)] != buf[PADJ(j - 1)];
      flags |= (head ? 1u : 0u) << i;
    }
  }
  uint32_t tot;
  uint32_t pos = rle_block_excl((uint32_t)__popc(flags), sh, &tot);  // ends with a barrier: buf is free
#pragma unroll
  for (int i = 0; i < RLE_ITEMS; ++i)
    if ((flags >> i) & 1u) buf[pos++] = (uint32_t)(base + j0 + i);
  __syncthreads();
  const uint32_t off = toff[blockIdx.x];
  for (uint32_t j = threadIdx.x; j < tot; j += RLE_THREADS) hp[off + j] = buf[j];
  if (blockIdx.x == ntile - 1 && threadIdx.x == 0) {
    hp[off + tot] = (uint32_t)n;
    meta[0] = off + tot;
  }
#undef PADJ
}

// Multiplicity of run d: from the run starts (sorted keys) or the counts (grouping by
// rank, RANKED).
template <bool RANKED>
__device__ __forceinline__ uint32_t run_len(const uint32_t* __restrict__ hp, int64_t d) {
  return RANKED ? hp[d] : hp[d + 1] - hp[d];
}

// Entries past one per run, per tile of runs: a multiplicity above 65535 takes
// ceil(len / 65535) entries.
template <bool RANKED>
__global__ void __launch_bounds__(RLE_THREADS) k_rle_ecount(const uint32_t* __restrict__ hp,
                                                            const uint32_t* __restrict__ meta,
                                                            uint32_t* __restrict__ ecnt) {
  __shared__ uint32_t sh[RLE_THREADS / 32];
  const uint32_t nd = meta[0];
  const int64_t base = (int64_t)blockIdx.x * RUN_TILE;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < RUN_ITEMS; ++i) {
    const int64_t d = base + (int64_t)i * RLE_THREADS + threadIdx.x;
    if (d < nd) c += (run_len<RANKED>(hp, d) - 1u) / 65535u;
  }
  const uint32_t t = rle_block_sum(c, sh);
  if (threadIdx.x == 0) ecnt[blockIdx.x] = t;
}

// Entries of run d at d + (entries past one of the runs before d): (i_T | multiplicity << 16)
// and b~ gathered from b. A batch row's entry (c, i) is the row-major index
// key = (c % ncell_inner) * IT + i over the sampled modes and b is read at
// ((key / xPafter) * xI + row) * xPafter + key % xPafter (X_(n) row `row`; for a plain solve
// xI = xPafter = 1 and the index is the key). Entries per cell are added to nd (one atomic
// per cell and warp). A tile of runs without long runs (ecnt = 0, nearly all) needs no
// local scan. RANKED (grouping by rank): keys[d] is run d's key and hp[d] its multiplicity.
template <bool RANKED>
__global__ void __launch_bounds__(RLE_THREADS) k_rle_emit(const uint32_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ hp,
                                                          const uint32_t* __restrict__ ecnt,
                                                          const uint32_t* __restrict__ eoff,
                                                          const uint32_t* __restrict__ meta, uint32_t IT,
                                                          uint32_t ncell_inner, int64_t xI, int64_t xPafter,
                                                          const float* __restrict__ b, uint32_t* __restrict__ ent,
                                                          float* __restrict__ bt, uint32_t* __restrict__ nd,
                                                          unsigned long long* __restrict__ total) {
  __shared__ uint32_t sh[RLE_THREADS / 32 + 1];
  const uint32_t ndist = meta[0];
  const int64_t base = (int64_t)blockIdx.x * RUN_TILE;
  if (base >= ndist) return;  // uniform over the block
  const bool longruns = ecnt[blockIdx.x] != 0u;
  uint32_t carry = eoff[blockIdx.x];
#pragma unroll
  for (int it = 0; it < RUN_ITEMS; ++it) {
    const int64_t d = base + (int64_t)it * RLE_THREADS + threadIdx.x;
    const bool live = d < ndist;
    uint32_t h0 = 0, cnt = 0, m = 0;
    if (live) {
      h0 = RANKED ? (uint32_t)d : hp[d];
      cnt = run_len<RANKED>(hp, d);
      m = (cnt + 65534u) / 65535u;
    }
    uint32_t before = 0, tot = 0;
    if (longruns) before = rle_block_excl(live ? m - 1u : 0u, sh, &tot);
    uint32_t cell = 0;
    if (live) {
      const uint32_t key = keys[h0];
      cell = key / IT;
      const uint32_t i = key - cell * IT;
      float bv = 0.f;
      if (b) {
        const uint32_t row = cell / ncell_inner;
        const int64_t rk = (int64_t)(cell - row * ncell_inner) * IT + i;
        const int64_t bi = (xPafter == 1 && xI == 1) ? rk : ((rk / xPafter) * xI + row) * xPafter + rk % xPafter;
        bv = b[bi];
      }
      uint32_t pos = (uint32_t)d + carry + before;
      if (d == ndist - 1) total[0] = (unsigned long long)pos + m;
      while (cnt > 0) {
        const uint32_t take = cnt > 65535u ? 65535u : cnt;
        ent[pos] = i | (take << 16);
        bt[pos] = bv;
        ++pos;
        cnt -= take;
      }
    }
    carry += tot;
    const unsigned act = __ballot_sync(0xffffffffu, live);
    if (live) {
      const unsigned peers = __match_any_sync(act, cell);
      const uint32_t sum = __reduce_add_sync(peers, m);
      if ((peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0u) atomicAdd(&nd[cell], sum);
    }
  }
}

// ------------------------------------------------------------------ grouping by rank
//
// When the key space ncell * IT is not much larger than the number of draws, one bit per
// possible key replaces the sort. The draws set their keys' bits; a scan of the bitmap's
// popcounts gives every set bit its rank (the distinct keys in increasing order: the runs
// of the sorted keys, in the same order), and every draw adds one to the count at its
// key's rank. Integer additions commute, so the counts are those of the runs whatever the
// order of the atomics, and the emit above writes the same entries as after a sort.
// Bitmap words are uint2 {bits, distinct keys before the word}.

constexpr int BM_ITEMS = 8;                      // bitmap words per thread in the rank scan
constexpr int BM_TILE = RLE_THREADS * BM_ITEMS;  // bitmap words per block
constexpr int BM_KEYCAP = 6144;                  // keys of a tile staged in shared memory

// Set bits per tile of bitmap words.
__global__ void __launch_bounds__(RLE_THREADS) k_bm_tcount(const uint2* __restrict__ bm, int64_t nw,
                                                           uint32_t* __restrict__ tcnt) {
  __shared__ uint32_t sh[RLE_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * BM_TILE;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < BM_ITEMS; ++i) {
    const int64_t w = base + (int64_t)i * RLE_THREADS + threadIdx.x;
    if (w < nw) c += (uint32_t)__popc(__ldg(&bm[w].x));
  }
  const uint32_t t = rle_block_sum(c, sh);
  if (threadIdx.x == 0) tcnt[blockIdx.x] = t;
}

// Ranks: bm[w].y = distinct keys before word w (toff: exclusive scan of the tile counts),
// dk[d] = the d-th distinct key, cnt[d] = 0 (the counts are added next by k_bm_count) or,
// with dense counts, cnt[d] = dcnt[dk[d]], after which that counter is reset to zero (so
// the dense counters are all zero again once every tile has run). A thread ranks BM_ITEMS
// consecutive words of the tile (staged in shared memory); the tile's keys are collected
// in shared memory and written out coalesced (a dense tile with more than BM_KEYCAP keys
// writes them directly). The last tile sets meta[0] = distinct keys.
// Where a key's dense counter lives (k_draw_keys): the key with each index replaced by its
// rank in its mode's decreasing-probability order (prk[0] null: the key itself).
struct CountMap {
  int N;
  uint32_t I[KR_MAX_MODES];
  uint32_t IT, ncell_inner;
  const uint16_t* prk[KR_MAX_MODES];
};
__device__ __forceinline__ uint32_t count_slot(const CountMap& cm, uint32_t key) {
  if (!cm.prk[0]) return key;
  const int N = cm.N;
  const uint32_t cell = key / cm.IT, iT = key - cell * cm.IT;
  const uint32_t r = cell / cm.ncell_inner;
  uint32_t inner = cell - r * cm.ncell_inner, pc = 0, mult = 1;
  for (int n = N - 2; n >= 0; --n) {
    const uint32_t q = inner / cm.I[n];
    pc += (uint32_t)cm.prk[n][inner - q * cm.I[n]] * mult;
    mult *= cm.I[n];
    inner = q;
  }
  return (pc + r * cm.ncell_inner) * cm.IT + (uint32_t)cm.prk[N - 1][iT];
}

__global__ void __launch_bounds__(RLE_THREADS) k_bm_rank(uint2* __restrict__ bm, int64_t nw,
                                                         const uint32_t* __restrict__ toff, int ntile,
                                                         uint32_t* __restrict__ dk, uint32_t* __restrict__ cnt,
                                                         uint32_t* __restrict__ meta, uint32_t* __restrict__ dcnt,
                                                         CountMap cm) {
  __shared__ uint32_t sh[RLE_THREADS / 32 + 1];
  __shared__ uint32_t bits[BM_TILE + BM_TILE / 32];
  __shared__ uint32_t pre[BM_TILE + BM_TILE / 32];
  __shared__ uint32_t skeys[BM_KEYCAP];
#define PADJ(j) ((j) + ((j) >> 5))
  const int64_t base = (int64_t)blockIdx.x * BM_TILE;
  for (int i = 0; i < BM_ITEMS; ++i) {
    const int j = i * RLE_THREADS + threadIdx.x;
    const int64_t w = base + j;
    bits[PADJ(j)] = w < nw ? bm[w].x : 0u;
  }
  __syncthreads();
  const int j0 = threadIdx.x * BM_ITEMS;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < BM_ITEMS; ++i) c += (uint32_t)__popc(bits[PADJ(j0 + i)]);
  uint32_t tot;
  uint32_t pos = rle_block_excl(c, sh, &tot);  // ends with a barrier
  const uint32_t off = toff[blockIdx.x];
  const bool staged = tot <= (uint32_t)BM_KEYCAP;  // uniform over the block
#pragma unroll
  for (int i = 0; i < BM_ITEMS; ++i) {
    const int j = j0 + i;
    uint32_t v = bits[PADJ(j)];
    pre[PADJ(j)] = off + pos;
    const uint32_t kb = (uint32_t)(base + j) << 5;  // key space <= 2^32: word index < 2^27
    while (v) {
      const uint32_t key = kb + (uint32_t)(__ffs(v) - 1);
      if (staged)
        skeys[pos] = key;
      else
        dk[off + pos] = key;
      ++pos;
      v &= v - 1u;
    }
  }
  __syncthreads();
  for (int i = 0; i < BM_ITEMS; ++i) {
    const int j = i * RLE_THREADS + threadIdx.x;
    const int64_t w = base + j;
    if (w < nw) bm[w].y = pre[PADJ(j)];
  }
  for (uint32_t j = threadIdx.x; j < tot; j += RLE_THREADS) {
    // (unstaged keys were written by other threads of the block before the barrier above)
    const uint32_t key = staged ? skeys[j] : dk[off + j];
    if (staged) dk[off + j] = key;
    if (dcnt) {
      const uint32_t slot = count_slot(cm, key);
      cnt[off + j] = dcnt[slot];
      dcnt[slot] = 0u;
    } else {
      cnt[off + j] = 0u;
    }
  }
  if (blockIdx.x == ntile - 1 && threadIdx.x == 0) meta[0] = off + tot;
#undef PADJ
}

// Multiplicities: every draw adds one at its key's rank (four draws in flight per thread).
__global__ void __launch_bounds__(256) k_bm_count(const uint32_t* __restrict__ keys, int64_t s,
                                                  const uint2* __restrict__ bm, uint32_t* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; t + 3 * stride < s; t += 4 * stride) {
    uint32_t k[4];
    uint2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = __ldg(keys + t + u * stride);
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldg(bm + (k[u] >> 5));
#pragma unroll
    for (int u = 0; u < 4; ++u) atomicAdd(cnt + v[u].y + (uint32_t)__popc(v[u].x & ((1u << (k[u] & 31)) - 1u)), 1u);
  }
  for (; t < s; t += stride) {
    const uint32_t k = __ldg(keys + t);
    const uint2 v = __ldg(bm + (k >> 5));
    atomicAdd(cnt + v.y + (uint32_t)__popc(v.x & ((1u << (k & 31)) - 1u)), 1u);
  }
}

// Weight of every cell: prod over its first N-1 coordinates of 1/p, times 1/s.
__global__ void k_cell_w(SampleModes sm, int64_t ncell, uint32_t ncell_inner, float inv_s, float* __restrict__ cell_w) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c32 = (uint32_t)c;
    uint32_t rem = c32 - (c32 / ncell_inner) * ncell_inner;
    float w = inv_s;
    for (int m = sm.N - 2; m >= 0; --m) {
      const uint32_t Im = (uint32_t)sm.I[m];
      const uint32_t q = rem / Im;
      w *= sm.invp[m][rem - q * Im];
      rem = q;
    }
    cell_w[c] = w;
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
  (void)m;
  if (s < 1 || s >= (int64_t(1) << 31)) return kr_fail(ctx, KR_EINVAL, "sketch: s=%lld outside [1, 2^31)", (long long)s);
  return KR_OK;
}

bool kr_group_by_rank(const kr_ctx* ctx, int64_t s, int64_t keyspace) {
  if (keyspace > (int64_t(1) << 32)) return false;
  if (ctx->grouping == 1) return false;
  if (ctx->grouping == 2 || ctx->grouping == 3) return true;
  return keyspace <= 64 * s;
}

// Grouping by rank with dense per-key counters (the default form of it): the key space's
// counters (4 bytes per key) must fit the budget.
static bool kr_group_dense(const kr_ctx* ctx, int64_t s, int64_t keyspace) {
  if (!kr_group_by_rank(ctx, s, keyspace) || ctx->grouping == 2) return false;
  return keyspace * (int64_t)sizeof(uint32_t) <= (int64_t(4) << 30);
}

// The context's dense per-key counters, all zero between sketch builds (the rank kernel
// resets every counter it reads); grown on demand, zeroed when (re)allocated or left dirty
// by an interrupted build.
static kr_status kr_dcnt_reserve(kr_ctx* ctx, int64_t keys) {
  const size_t bytes = (size_t)keys * sizeof(uint32_t);
  if (bytes > ctx->dcnt_size) {
    if (ctx->gm.on && ctx->gm.capturing)
      return kr_fail(ctx, KR_ENOTIMPL, "inside a capture: the key counters would have to grow (run the call once outside the capture first)");
    KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->dcnt) cudaFree(ctx->dcnt);
    ctx->dcnt = nullptr;
    ctx->dcnt_size = 0;
    cudaError_t e = cudaMalloc((void**)&ctx->dcnt, bytes);
    if (e != cudaSuccess) {
      ctx->dcnt = nullptr;
      cudaGetLastError();
      return kr_fail(ctx, KR_ENOMEM, "dense key counters: allocation of %zu bytes failed", bytes);
    }
    ctx->dcnt_size = bytes;
    ctx->dcnt_clean = false;
  }
  if (!ctx->dcnt_clean) {
    KR_CUDA(ctx, cudaMemsetAsync(ctx->dcnt, 0, ctx->dcnt_size, ctx->stream));
    ctx->dcnt_clean = true;
  }
  return KR_OK;
}

// Second phase of the sketch build, with scratch carved from `cv`: draw the row keys,
// group them (radix sort and runs of equal keys, or ranks in a bitmap of the key space),
// and write the merged entries of every cell.
kr_status kr_sketch_fill(kr_ctx* ctx, const Modes& m, const FactorTables& t, const float* b, uint64_t seed,
                         uint64_t call_id, int row, kr_sketch* sk, Carve& cv, bool defer_distinct) {
  const int N = m.N;
  const int64_t s = sk->s, ncell = sk->ncell;
  const uint32_t IT = (uint32_t)sk->IT;
  uint32_t* keys = cv.take<uint32_t>(s);
  uint32_t* alt = cv.take<uint32_t>(s);
  uint32_t* hp = cv.take<uint32_t>(s + 1);
  uint32_t* mcnt = cv.take<uint32_t>(rle_scratch_words(s));
  uint32_t* meta = cv.take<uint32_t>(4);
  unsigned long long* dsum = cv.take<unsigned long long>(1);
  uint16_t* gbuf = cv.take<uint16_t>((size_t)KR_MAX_MODES * GUIDE_MAX);
  uint16_t* prkbuf = cv.take<uint16_t>((size_t)KR_MAX_MODES * PRK_MAX);
  const int64_t keyspace = ncell * (int64_t)IT;
  const bool ranked = kr_group_by_rank(ctx, s, keyspace);
  const bool dense = kr_group_dense(ctx, s, keyspace);
  const int64_t nw = ranked ? (keyspace + 31) / 32 : 0;
  const int nbt = (int)((nw + BM_TILE - 1) / BM_TILE);
  uint2* bm = ranked ? cv.take<uint2>(nw) : nullptr;
  uint32_t* btc = ranked ? cv.take<uint32_t>(2 * (size_t)nbt) : nullptr;
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "sketch: workspace too small");
  SampleModes sm = make_sample_modes(m, t);
  DrawModes dm = {};
  dm.N = N;
  for (int n = 0; n < N; ++n) {
    int gb = 0;
    while ((1 << gb) < m.I[n]) ++gb;
    dm.I[n] = m.I[n];
    dm.M[n] = 1 << gb;
    dm.shift[n] = 53 - gb;
    dm.thr[n] = t.thr[n];
    dm.guide[n] = gbuf + (size_t)n * GUIDE_MAX;
    KR_LAUNCH(ctx, k_guide, grid_for(ctx, dm.M[n], 256), 256, 0, t.thr[n], m.I[n], dm.shift[n], dm.M[n],
              gbuf + (size_t)n * GUIDE_MAX);
  }
  KR_CUDA(ctx, cudaMemsetAsync(sk->cell_nd, 0, sizeof(uint32_t) * ncell, ctx->stream));
  KR_CUDA(ctx, cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), ctx->stream));
  if (ranked) KR_CUDA(ctx, cudaMemsetAsync(bm, 0, sizeof(uint2) * nw, ctx->stream));
  uint32_t* dcnt = nullptr;
  CountMap cmap = {};
  cmap.N = N;
  cmap.IT = IT;
  cmap.ncell_inner = (uint32_t)sk->ncell_inner;
  if (dense) {
    KR_TRY(kr_dcnt_reserve(ctx, keyspace));
    dcnt = ctx->dcnt;
    ctx->dcnt_clean = false;  // until the rank kernel below has been enqueued
    bool small = true;
    for (int n = 0; n < N; ++n) small = small && m.I[n] <= PRK_MAX;
    if (small) {  // counters addressed by probability ranks
      ProbRanks pr = {};
      for (int n = 0; n < N; ++n) {
        pr.I[n] = m.I[n];
        pr.prob[n] = t.prob[n];
        pr.out[n] = prkbuf + (size_t)n * PRK_MAX;
        dm.prk[n] = pr.out[n];
        cmap.I[n] = (uint32_t)m.I[n];
        cmap.prk[n] = pr.out[n];
      }
      int imax = 1;
      for (int n = 0; n < N; ++n) imax = m.I[n] > imax ? m.I[n] : imax;
      KR_LAUNCH(ctx, k_prob_rank, dim3(N, (imax + 255) / 256), 256, 0, pr);
    }
  }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32), cid = (uint32_t)call_id;
  {
    const int gs = grid_for(ctx, s, 256);
#define KR_DRAW_KEYS(NN)                                                                                         \
  case NN:                                                                                                       \
    KR_LAUNCH(ctx, k_draw_keys<NN>, gs, 256, 0, dm, sk->s_row, sk->nrow, k0, k1, (uint32_t)row, cid,             \
              (uint32_t)sk->ncell_inner, keys, bm, dcnt);                                                        \
    break;
    switch (N) {
      KR_DRAW_KEYS(1)
      KR_DRAW_KEYS(2)
      KR_DRAW_KEYS(3)
      KR_DRAW_KEYS(4)
      KR_DRAW_KEYS(5)
      KR_DRAW_KEYS(6)
      KR_DRAW_KEYS(7)
      KR_DRAW_KEYS(8)
      default:
        return kr_fail(ctx, KR_EINVAL, "sketch: N=%d", N);
    }
#undef KR_DRAW_KEYS
  }
  // runs: (key, multiplicity) in increasing key order, as run starts into the sorted keys
  // (hp) or as distinct keys (alt) with their counts (hp)
  const int ntile = (int)((s + RLE_TILE - 1) / RLE_TILE);
  const int nrt = (int)((s + RUN_TILE - 1) / RUN_TILE);  // run tiles (the run count is at most s)
  uint32_t* tcnt = mcnt;
  uint32_t* toff = tcnt + ntile;
  uint32_t* ecnt = toff + ntile;
  uint32_t* eoff = ecnt + nrt;
  uint32_t* runkeys = alt;
  if (ranked) {
    KR_LAUNCH(ctx, k_bm_tcount, nbt, RLE_THREADS, 0, bm, nw, btc);
    {
      Carve sc = cv;
      KR_TRY(kr_scan_u32(ctx, btc, btc + nbt, nbt, sc));
    }
    KR_LAUNCH(ctx, k_bm_rank, nbt, RLE_THREADS, 0, bm, nw, btc + nbt, nbt, alt, hp, meta, dcnt, cmap);
    if (dense)
      ctx->dcnt_clean = true;  // the rank kernel resets every counter the draws set
    else
      KR_LAUNCH(ctx, k_bm_count, grid_for(ctx, s, 256), 256, 0, keys, s, bm, hp);
    KR_LAUNCH(ctx, k_rle_ecount<true>, nrt, RLE_THREADS, 0, hp, meta, ecnt);
  } else {
    int nbits = 0;
    while (nbits < 32 && (uint64_t(1) << nbits) < (uint64_t)keyspace) ++nbits;
    {
      Carve sc = cv;
      KR_TRY(kr_radix_sort_u32(ctx, keys, alt, s, nbits, &runkeys, sc));
    }
    // run merge: tile head counts, run starts, long-run extras (small per-tile arrays
    // carved from the entry-count scratch)
    KR_LAUNCH(ctx, k_rle_tcount, ntile, RLE_THREADS, 0, runkeys, s, tcnt);
    {
      Carve sc = cv;
      KR_TRY(kr_scan_u32(ctx, tcnt, toff, ntile, sc));
    }
    KR_LAUNCH(ctx, k_rle_starts, ntile, RLE_THREADS, 0, runkeys, s, toff, ntile, hp, meta);
    KR_LAUNCH(ctx, k_rle_ecount<false>, nrt, RLE_THREADS, 0, hp, meta, ecnt);
  }
  {
    Carve sc = cv;
    KR_TRY(kr_scan_u32(ctx, ecnt, eoff, nrt, sc));
  }
  // b may still be arriving on the context's copy stream (host-buffer solves): the gather
  // is its first reader
  if (ctx->b_wait) KR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->b_wait, 0));
  if (ranked)
    KR_LAUNCH(ctx, k_rle_emit<true>, nrt, RLE_THREADS, 0, runkeys, hp, ecnt, eoff, meta, IT,
              (uint32_t)sk->ncell_inner, sk->xI, sk->xPafter, b, sk->ent, sk->bt, sk->cell_nd, dsum);
  else
    KR_LAUNCH(ctx, k_rle_emit<false>, nrt, RLE_THREADS, 0, runkeys, hp, ecnt, eoff, meta, IT,
              (uint32_t)sk->ncell_inner, sk->xI, sk->xPafter, b, sk->ent, sk->bt, sk->cell_nd, dsum);
  {
    Carve sc = cv;
    KR_TRY(kr_scan_u32(ctx, sk->cell_nd, sk->cell_start, ncell, sc));
  }
  KR_LAUNCH(ctx, k_cell_w, grid_for(ctx, ncell, 256), 256, 0, sm, ncell, (uint32_t)sk->ncell_inner,
            (float)(1.0 / (double)sk->s_row), sk->cell_w);
  if (sk->want_desc) {
    Carve sc = cv;
    KR_TRY(kr_balance_perm(ctx, sk->cell_nd, ncell, sk->perm, sc));
    KR_LAUNCH(ctx, k_build_desc, grid_for(ctx, ncell, 256), 256, 0, sk->perm, sk->cell_start, sk->cell_nd,
              sk->cell_w, ncell, sk->desc);
  }
  KR_CUDA(ctx, cudaMemcpyAsync(sk->invpT, t.invp[N - 1], sizeof(float) * IT, cudaMemcpyDeviceToDevice, ctx->stream));
  KR_TRY(kr_hbuf_reserve(ctx, 4096));
  if (ctx->gm.on) {  // a captured sweep or an asynchronous solve: the count stays on the device
    KR_CUDA(ctx, cudaMemcpyAsync(ctx->gm.distinct, dsum, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    sk->distinct = -1;
    return KR_OK;
  }
  if (defer_distinct) {  // read by the caller after its next synchronisation
    KR_CUDA(ctx, cudaMemcpyAsync((char*)ctx->hbuf + KR_HBUF_DISTINCT, dsum, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    sk->distinct = -1;
    return KR_OK;
  }
  KR_CUDA(ctx, cudaMemcpyAsync(ctx->hbuf, dsum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  sk->distinct = (int64_t)(*(unsigned long long*)ctx->hbuf);
  return KR_OK;
}

void kr_sketch_scratch_need(const kr_ctx* ctx, int64_t s, int64_t ncell, int64_t IT, Need& nd) {
  nd.add<uint32_t>(s);      // keys
  nd.add<uint32_t>(s);      // sort buffer / distinct keys
  nd.add<uint32_t>(s + 1);  // run starts / multiplicities
  nd.add<uint32_t>(rle_scratch_words(s));  // run merge: tile head counts and offsets, long-run extras
  nd.add<uint32_t>(4);
  nd.add<unsigned long long>(1);
  nd.add<uint16_t>((size_t)KR_MAX_MODES * GUIDE_MAX);
  nd.add<uint16_t>((size_t)KR_MAX_MODES * PRK_MAX);
  if (kr_group_by_rank(ctx, s, ncell * IT)) {
    const int64_t nw = (ncell * IT + 31) / 32;
    nd.add<uint2>(nw);                                       // key bitmap with word ranks
    nd.add<uint32_t>(2 * ((nw + BM_TILE - 1) / BM_TILE));  // its tile counts and offsets
  }
  Need a, c;
  if (kr_group_by_rank(ctx, s, ncell * IT))
    kr_scan_need(((ncell * IT + 31) / 32 + BM_TILE - 1) / BM_TILE, c);
  else
    kr_radix_need(s, a);
  kr_scan_need(s, c);
  kr_scan_need(ncell, c);
  kr_perm_need(ncell, c);
  nd.off += (a.off > c.off ? a.off : c.off) + 256;
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

// The last threshold is 2^53, above every U, whatever cdf[n - 1] holds: a table whose last
// entry is below 1 (or not a number) clamps to the last row, as the bounded binary search
// does, and the guided search never steps past the table.
__global__ void k_thr_from_cdf(const double* cdf, uint64_t* thr, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    thr[i] = i == n - 1 ? (uint64_t(1) << 53) : (uint64_t)ceil(cdf[i] * 9007199254740992.0);
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
  kr_sketch_scratch_need(ctx, s, ncell, m.I[m.N - 1], nd);
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
