// Stable LSD radix sort of 32-bit keys (9-bit digits), used to group the sampled rows
// of a sketch by (cell, last coordinate): after the sort, repeated rows are adjacent
// and cells appear in increasing order (the sets S_1, S_2, B_S of the proof of
// Thm 4.4 with T = the last mode).
//
// Each pass: per-tile digit histograms (digit-major table), an exclusive scan of the
// table, then a stable scatter. Inside a tile of 4096 keys every warp owns a contiguous
// 512-key chunk and ranks its keys round by round (lanes of equal digit found with nine
// ballots); the per-warp counts give every key its place in the tile, the tile is
// reordered in shared memory and written out digit run by digit run. Nine-bit digits sort
// the 27-bit row keys of a 512^3 problem in three passes.
#include "kr_internal.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_BITS = 9;
constexpr int RS_BUCKETS = 1 << RS_BITS;
constexpr int RS_DPT = RS_BUCKETS / RS_THREADS;  // digits per thread in the per-digit steps
static_assert(RS_DPT * RS_THREADS == RS_BUCKETS, "digits per thread");

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* __restrict__ in, int64_t n, int shift,
                                                           uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t h[RS_BUCKETS];
#pragma unroll
  for (int k = 0; k < RS_DPT; ++k) h[threadIdx.x + k * RS_THREADS] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t idx = base + (int64_t)i * RS_THREADS + threadIdx.x;
    if (idx < n) atomicAdd(&h[(__ldg(in + idx) >> shift) & (RS_BUCKETS - 1)], 1u);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RS_DPT; ++k) {
    const int d = threadIdx.x + k * RS_THREADS;
    hist[(int64_t)d * nblk + blockIdx.x] = h[d];
  }
}

// hist: exclusive scan of the digit-major table (first output position of every
// (digit, tile)).
__global__ void __launch_bounds__(RS_THREADS, 3) k_radix_scatter(const uint32_t* __restrict__ in,
                                                              uint32_t* __restrict__ out, int64_t n, int shift,
                                                              const uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t s_keys[RS_TILE];
  __shared__ uint32_t s_wcnt[RS_WARPS][RS_BUCKETS];
  __shared__ uint32_t s_loc[RS_BUCKETS];
  __shared__ uint32_t s_glob[RS_BUCKETS];
  __shared__ uint32_t s_wtot[RS_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const int64_t wbase = base + (int64_t)warp * (RS_ITEMS * 32);
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < RS_BUCKETS / 32; ++i) s_wcnt[warp][i * 32 + lane] = 0u;
#pragma unroll
  for (int k = 0; k < RS_DPT; ++k) {
    const int d = threadIdx.x + k * RS_THREADS;
    s_glob[d] = hist[(int64_t)d * nblk + blockIdx.x];
  }
  __syncwarp();
  uint32_t key[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    const bool valid = idx < n;
    key[r] = valid ? __ldg(in + idx) : 0u;
    const uint32_t d = (key[r] >> shift) & (RS_BUCKETS - 1);
    unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < RS_BITS; ++b) {
      const bool bit = (d >> b) & 1u;
      const unsigned bb = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bb : ~bb;
    }
    const uint32_t prev = s_wcnt[warp][d];
    rank[r] = prev + (uint32_t)__popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0u) s_wcnt[warp][d] = prev + (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // tile totals per digit (RS_DPT consecutive digits per thread), exclusive scan over
     // digits, then per-warp starts
    const int d0 = threadIdx.x * RS_DPT;
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < RS_DPT; ++k)
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) mine += s_wcnt[w][d0 + k];
    uint32_t inc = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += v;
    }
    if (lane == 31) s_wtot[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_wtot[w];
    uint32_t acc = before + inc - mine;
#pragma unroll
    for (int k = 0; k < RS_DPT; ++k) {
      const int d = d0 + k;
      s_loc[d] = acc;
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = acc;
        acc += c;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    if (idx < n) {
      const uint32_t d = (key[r] >> shift) & (RS_BUCKETS - 1);
      s_keys[s_wcnt[warp][d] + rank[r]] = key[r];
    }
  }
  __syncthreads();
  const int64_t cnt = (n - base) < RS_TILE ? (n - base) : RS_TILE;
  for (int j = threadIdx.x; j < cnt; j += RS_THREADS) {
    const uint32_t k = s_keys[j];
    const uint32_t d = (k >> shift) & (RS_BUCKETS - 1);
    out[s_glob[d] + (uint32_t)j - s_loc[d]] = k;
  }
}

}  // namespace

void kr_radix_need(int64_t n, Need& nd) {
  const int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
  nd.add<uint32_t>((size_t)RS_BUCKETS * nblk);
  kr_scan_need((int64_t)RS_BUCKETS * nblk, nd);
}

kr_status kr_radix_sort_u32(kr_ctx* ctx, uint32_t* keys, uint32_t* alt, int64_t n, int nbits, uint32_t** sorted,
                            Carve& cv) {
  *sorted = keys;
  if (n <= 1 || nbits <= 0) return KR_OK;
  if (n >= (int64_t(1) << 32) - RS_TILE) return kr_fail(ctx, KR_EINVAL, "radix sort: %lld keys", (long long)n);
  const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
  uint32_t* hist = cv.take<uint32_t>((size_t)RS_BUCKETS * nblk);
  if (cv.off > cv.cap) return kr_fail(ctx, KR_ENOMEM, "radix sort: workspace too small");
  uint32_t* src = keys;
  uint32_t* dst = alt;
  for (int shift = 0; shift < nbits; shift += RS_BITS) {
    KR_LAUNCH(ctx, k_radix_hist, nblk, RS_THREADS, 0, src, n, shift, hist, nblk);
    {
      Carve sc = cv;
      KR_TRY(kr_scan_u32(ctx, hist, hist, (int64_t)RS_BUCKETS * nblk, sc));
    }
    KR_LAUNCH(ctx, k_radix_scatter, nblk, RS_THREADS, 0, src, dst, n, shift, hist, nblk);
    uint32_t* t = src;
    src = dst;
    dst = t;
  }
  *sorted = src;
  return KR_OK;
}
