// Device-wide exclusive scan of u32 counters and the work-balancing order of the
// sketch's cells (a stable bucket sort by distinct-row count, heaviest first).
#include "kr_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;  // 4096

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t* total) {
  // sh: SCAN_THREADS/32 words
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (SCAN_THREADS / 32) ? sh[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += t;
    }
    if (lane < (SCAN_THREADS / 32)) sh[lane] = wi - w;
    if (lane == (SCAN_THREADS / 32) - 1) sh[SCAN_THREADS / 32] = wi;
  }
  __syncthreads();
  uint32_t r = sh[warp] + incl - v;
  *total = sh[SCAN_THREADS / 32];
  __syncthreads();
  return r;
}

// Phase 1: per-tile sums.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t* __restrict__ in, int64_t n,
                                                              uint32_t* __restrict__ tile_sum) {
  __shared__ uint32_t sh[SCAN_THREADS / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint32_t total;
  block_excl_scan(s, sh, &total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// Phase 2: exclusive scan of the tile sums (one block, sequential chunks).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(uint32_t* __restrict__ tile_sum, int64_t ntile) {
  __shared__ uint32_t sh[SCAN_THREADS / 32 + 1];
  uint32_t carry = 0;
  for (int64_t b = 0; b < ntile; b += SCAN_THREADS) {
    int64_t i = b + threadIdx.x;
    uint32_t v = i < ntile ? tile_sum[i] : 0u;
    uint32_t total;
    uint32_t ex = block_excl_scan(v, sh, &total);
    if (i < ntile) tile_sum[i] = carry + ex;
    carry += total;
  }
}

// Phase 3: scan inside each tile (thread-contiguous runs), plus the tile offset (none when
// tile_off is null: a single tile is the whole scan).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const uint32_t* __restrict__ in, int64_t n,
                                                              const uint32_t* __restrict__ tile_off,
                                                              uint32_t* __restrict__ out) {
  __shared__ uint32_t sh[SCAN_THREADS / 32 + 1];
  // element j of the tile lives at buf[j + j/32] (padding keeps the thread-contiguous
  // reads below free of bank conflicts)
  __shared__ uint32_t buf[SCAN_TILE + SCAN_TILE / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#define PADJ(j) ((j) + ((j) >> 5))
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {  // coalesced load into shared memory
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    int j = k * SCAN_THREADS + threadIdx.x;
    buf[PADJ(j)] = i < n ? in[i] : 0u;
  }
  __syncthreads();
  uint32_t v[SCAN_PER_THREAD];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    v[k] = buf[PADJ(threadIdx.x * SCAN_PER_THREAD + k)];
    s += v[k];
  }
  uint32_t total;
  uint32_t run = (tile_off ? tile_off[blockIdx.x] : 0u) + block_excl_scan(s, sh, &total);
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    buf[PADJ(threadIdx.x * SCAN_PER_THREAD + k)] = run;
    run += v[k];
  }
  __syncthreads();
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) out[i] = buf[PADJ(k * SCAN_THREADS + threadIdx.x)];
  }
#undef PADJ
}

// ------------------------------------------------------------------ balance order

constexpr int NB = 32;            // buckets: 0 for empty cells, 1 + floor(log2(nd)) otherwise
constexpr int PERM_TILE = 2048;   // cells per block (256 threads x 8 chunks, in order)

__device__ __forceinline__ int bucket_of(uint32_t nd) { return nd == 0 ? 0 : min(NB - 1, 32 - __clz(nd)); }

// Per-block histogram of buckets, stored heaviest bucket first:
// tbl[(NB - 1 - b) * nblk + blk]. An exclusive scan of tbl then gives each (bucket,
// block) its first output position.
__global__ void __launch_bounds__(256) k_perm_count(const uint32_t* __restrict__ nd, int64_t ncell,
                                                     uint32_t* __restrict__ tbl, int nblk) {
  __shared__ uint32_t h[NB];
  if (threadIdx.x < NB) h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * PERM_TILE;
  for (int k = threadIdx.x; k < PERM_TILE; k += blockDim.x) {
    int64_t c = base + k;
    if (c < ncell) atomicAdd(&h[bucket_of(nd[c])], 1u);
  }
  __syncthreads();
  if (threadIdx.x < NB) tbl[(int64_t)(NB - 1 - threadIdx.x) * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: cells of one bucket keep their index order.
__global__ void __launch_bounds__(256) k_perm_scatter(const uint32_t* __restrict__ nd, int64_t ncell,
                                                       const uint32_t* __restrict__ tbl, int nblk,
                                                       uint32_t* __restrict__ perm) {
  __shared__ uint32_t base[NB];
  __shared__ uint32_t wcnt[8][NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < NB) base[threadIdx.x] = tbl[(int64_t)(NB - 1 - threadIdx.x) * nblk + blockIdx.x];
  const int64_t c0 = (int64_t)blockIdx.x * PERM_TILE;
  for (int chunk = 0; chunk < PERM_TILE; chunk += 256) {
    for (int k = threadIdx.x; k < 8 * NB; k += 256) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t c = c0 + chunk + threadIdx.x;
    const bool live = c < ncell;
    const int b = live ? bucket_of(nd[c]) : NB;  // NB: no bucket
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (live && rank == 0) wcnt[warp][b] = __popc(peers);
    __syncthreads();
    if (live) {
      uint32_t before = 0;
      for (int w = 0; w < warp; ++w) before += wcnt[w][b];
      perm[base[b] + before + rank] = (uint32_t)c;
    }
    __syncthreads();
    if (threadIdx.x < NB) {
      uint32_t tot = 0;
      for (int w = 0; w < 8; ++w) tot += wcnt[w][threadIdx.x];
      base[threadIdx.x] += tot;
    }
    __syncthreads();
  }
}

}  // namespace

void kr_scan_need(int64_t n, Need& nd) { nd.add<uint32_t>((n + SCAN_TILE - 1) / SCAN_TILE + 1); }

kr_status kr_scan_u32(kr_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, Carve& cv) {
  const int64_t ntile = (n + SCAN_TILE - 1) / SCAN_TILE;
  uint32_t* ts = cv.take<uint32_t>(ntile + 1);
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "scan: workspace too small");
  if (ntile == 0) return KR_OK;
  if (ntile == 1) {  // one block scans it all
    KR_LAUNCH(ctx, k_scan_apply, 1, SCAN_THREADS, 0, in, n, (const uint32_t*)nullptr, out);
    return KR_OK;
  }
  KR_LAUNCH(ctx, k_scan_tiles, (unsigned)ntile, SCAN_THREADS, 0, in, n, ts);
  KR_LAUNCH(ctx, k_scan_sums, 1, SCAN_THREADS, 0, ts, ntile);
  KR_LAUNCH(ctx, k_scan_apply, (unsigned)ntile, SCAN_THREADS, 0, in, n, ts, out);
  return KR_OK;
}

void kr_perm_need(int64_t ncell, Need& nd) {
  const int64_t t = (int64_t)NB * ((ncell + PERM_TILE - 1) / PERM_TILE);
  nd.add<uint32_t>(t);
  kr_scan_need(t, nd);
}

kr_status kr_balance_perm(kr_ctx* ctx, const uint32_t* nd, int64_t ncell, uint32_t* perm, Carve& cv) {
  const int nblk = (int)((ncell + PERM_TILE - 1) / PERM_TILE);
  uint32_t* tbl = cv.take<uint32_t>((size_t)NB * nblk);
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "balance order: workspace too small");
  KR_LAUNCH(ctx, k_perm_count, nblk, 256, 0, nd, ncell, tbl, nblk);
  KR_TRY(kr_scan_u32(ctx, tbl, tbl, (int64_t)NB * nblk, cv));
  KR_LAUNCH(ctx, k_perm_scatter, nblk, 256, 0, nd, ncell, tbl, nblk, perm);
  return KR_OK;
}
