// Mode products with a contiguous contracted index on the 5th-generation tensor cores:
//   Y[m, j] = sum_k X[m, k] B[j, k]            (X: M x K row-major, B: J x K, Y: M x J)
// i.e. the n-mode product of KronMatMul (Lemma 4.3) along the last mode of a C-order
// tensor, where the contraction runs over contiguous memory: the first product of K^T b
// on a dense right-hand side, and the projections of exact TuckerALS (App. C).
//
// FP32 accuracy from the TF32 tensor path (3xTF32): every operand is split as x = hi + lo
// with hi = x with its low 13 mantissa bits cleared (exact in TF32) and lo = x - hi (exact
// in FP32, at most 13 significant bits), and X B^T ~ Xhi Bhi^T + Xhi Blo^T + Xlo Bhi^T with
// FP32 accumulation in tensor memory; the dropped Xlo Blo^T term is below 2^-20 of the
// product and the TF32 rounding of lo below 2^-21, so the result stays within a few FP32
// units of the exact sum.
//
// One persistent CTA per SM walks 128-row tiles of X. Warp roles:
//   warp 0     TMA producer: X tile (128 rows x 32 floats, 128-byte swizzle) and the
//              pre-split B planes of the same 32 columns, into a ring of stages
//   warps 2-5  split the landed X tile in place into hi and a lo plane (same layout)
//   warp 1     one thread issues tcgen05.mma (kind::tf32, M = 128, N = padded J, K = 8),
//              3 per K step, into one of two TMEM buffers (tiles in flight); within a tile
//              the 32-float K stages alternate over up to 4 accumulators, because the tensor
//              core's accumulation loses about one FP32 unit per step with a sign that does
//              not average out (measured: the error grew linearly with K), so shorter chains
//              added in FP32 by the epilogue keep the product's error a few FP32 units
//              at K = 1024; commits free the stage
//   warps 6-9  epilogue: tcgen05.ld of the finished accumulator (one row per thread),
//              stores to Y, then release the buffer to the next tile's MMAs
// Every mbarrier wait is bounded: a wait that runs out sets the CTA's abort flag and an
// error code in global memory (the host reports KR_ETIMEOUT); the other roles see the flag
// and leave, the producer waits (bounded) for its own copies in flight, the MMA thread for
// its own MMAs, and the allocating warp frees the tensor memory.
#include <cuda.h>

#include <mutex>

#include "kr_internal.cuh"

namespace {

constexpr int TC_BM = 128;      // rows of X per tile = TMEM lanes of the accumulator
constexpr int TC_BK = 32;       // floats of one stage row (one 128-byte swizzle row)
constexpr int TC_THREADS = 320;  // 10 warps
constexpr int TC_SPLIT_T = 128;  // splitter threads (warps 2-5)
constexpr int TC_EPI_T = 128;    // epilogue threads (warps 6-9)
constexpr long long TC_WAIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

struct TcShape {
  int bnp;        // J padded to a multiple of 32 (MMA N and accumulator columns)
  int stages;     // ring depth
  int nacc;       // accumulators per tile (K stages interleaved over them)
  uint32_t a_bytes, b_bytes, stage_bytes, tx_bytes;
  uint32_t bar_off;   // mbarriers after the stages
  uint32_t smem;      // dynamic shared memory (bytes), including 1 KB of alignment slack
  uint32_t tmem_cols; // power of two >= 2 * nacc * bnp
};

TcShape tc_shape(int J) {
  TcShape s;
  s.bnp = (J + 31) / 32 * 32;
  s.a_bytes = TC_BM * TC_BK * 4;                       // 16 KB
  s.b_bytes = (uint32_t)s.bnp * TC_BK * 4;             // bnp rows of 128 B
  s.stage_bytes = 2 * s.a_bytes + 2 * s.b_bytes;       // X hi, X lo, B hi, B lo
  s.tx_bytes = s.a_bytes + 2 * s.b_bytes;              // what TMA lands per stage
  const uint32_t budget = 200 * 1024;
  int st = (int)(budget / s.stage_bytes);
  s.stages = st > 6 ? 6 : st;
  s.bar_off = (uint32_t)s.stages * s.stage_bytes;
  // full, split, empty per stage; tfull, tempty per accumulator; drain; then tmem slot, abort
  const uint32_t bars = (uint32_t)(3 * s.stages + 5) * 8;
  uint32_t smem = 1024 + s.bar_off + bars + 16;
  // more than half of the SM's shared memory, so no second CTA of this kernel shares the
  // SM's tensor memory
  if (smem < 120 * 1024) smem = 120 * 1024;
  s.smem = smem;
  // K stages alternate over nacc accumulators per tile (two tiles in flight): the tensor
  // core's FP32 accumulation chains get nacc times shorter, and the epilogue adds them
  s.nacc = 512 / (2 * s.bnp);
  if (s.nacc > 4) s.nacc = 4;
  uint32_t c = 32;
  while (c < 2u * (uint32_t)(s.nacc * s.bnp)) c <<= 1;
  s.tmem_cols = c;
  return s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits until the phase with this parity has completed. Gives up (false) when the CTA's
// abort flag is set, or after TC_WAIT_CYCLES, in which case it sets the flag and the code.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err, int code,
                          bool heed_abort = true) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (heed_abort && *abort_flag) return false;
    if (clock64() - t0 > TC_WAIT_CYCLES) {
      *abort_flag = 1;
      atomicCAS(err, 0, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle layout that
// TMA writes for a box of 128-byte rows: 8-row groups 1024 bytes apart (stride byte
// offset), the leading byte offset unused, descriptor version 1 (bits 46-48), swizzle mode
// 2 (128 B) in bits 61-63. Start address in 16-byte units.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 32 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes, one lane per thread.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct TcArgs {
  float* Y;
  int64_t M, ldy;
  int K, J;
  int bnp, stages, nacc;
  uint32_t a_bytes, b_bytes, stage_bytes, tx_bytes, bar_off, tmem_cols;
  int* err;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mBh,
              const __grid_constant__ CUtensorMap mBl, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // stages start on a 1024-byte boundary (the period of the 128-byte swizzle)
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tc_smem_raw + (base - raw);
  const int S = a.stages;
  const uint32_t bars = base + a.bar_off;
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto split = [&](int s) { return bars + 8u * (uint32_t)(S + s); };
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(2 * S + s); };
  auto tfull = [&](int b) { return bars + 8u * (uint32_t)(3 * S + b); };
  auto tempty = [&](int b) { return bars + 8u * (uint32_t)(3 * S + 2 + b); };
  const uint32_t drain = bars + 8u * (uint32_t)(3 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + a.bar_off + 8u * (uint32_t)(3 * S + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto xhi = [&](int s) { return base + (uint32_t)s * a.stage_bytes; };
  auto xlo = [&](int s) { return xhi(s) + a.a_bytes; };
  auto bhi = [&](int s) { return xhi(s) + 2 * a.a_bytes; };
  auto blo = [&](int s) { return bhi(s) + a.b_bytes; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(split(s), TC_SPLIT_T);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), TC_EPI_T);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t ntiles = (a.M + TC_BM - 1) / TC_BM;
  const int nk = (a.K + TC_BK - 1) / TC_BK;

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0) {
      int64_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = (int)(it % S);
          const uint32_t r = (uint32_t)(it / S);
          if (!mbar_wait(empty(s), (r & 1u) ^ 1u, abort_flag, a.err, 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full(s), a.tx_bytes);
          tma_load_2d(xhi(s), &mX, kb * TC_BK, (int)(t * TC_BM), full(s));
          tma_load_2d(bhi(s), &mBh, kb * TC_BK, 0, full(s));
          tma_load_2d(blo(s), &mBl, kb * TC_BK, 0, full(s));
        }
      }
      // copies still in flight land before the CTA can leave: wait (bounded) for the last
      // round issued on every stage
      for (int s = 0; s < S; ++s) {
        if (it <= s) break;
        const int64_t last = it - 1 - ((it - 1 - s) % S);  // last index issued on stage s
        mbar_wait(full(s), (uint32_t)(last / S) & 1u, abort_flag, a.err, 2, false);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(TC_BM, a.bnp);
      int64_t it = 0, ti = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++ti) {
        const int b = (int)(ti & 1);
        const uint32_t u = (uint32_t)(ti >> 1);
        if (!mbar_wait(tempty(b), (u & 1u) ^ 1u, abort_flag, a.err, 3)) break;
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(b * a.nacc * a.bnp);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const uint32_t d = d0 + (uint32_t)((kb % a.nacc) * a.bnp);
          const int s = (int)(it % S);
          const uint32_t r = (uint32_t)(it / S);
          if (!mbar_wait(split(s), r & 1u, abort_flag, a.err, 4)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < TC_BK / 8; ++ks) {
            const uint32_t off = (uint32_t)ks * 32u;  // 8 TF32 = 32 bytes along the swizzled row
            const uint64_t dah = sdesc_sw128(xhi(s) + off), dal = sdesc_sw128(xlo(s) + off);
            const uint64_t dbh = sdesc_sw128(bhi(s) + off), dbl = sdesc_sw128(blo(s) + off);
            tc_mma_tf32(d, dal, dbh, idesc, (kb >= a.nacc || ks != 0) ? 1u : 0u);
            tc_mma_tf32(d, dah, dbl, idesc, 1u);
            tc_mma_tf32(d, dah, dbh, idesc, 1u);
          }
          tc_commit(empty(s));  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        tc_commit(tfull(b));
      }
      // every MMA issued has completed before the tensor memory is released
      tc_commit(drain);
      mbar_wait(drain, 0u, abort_flag, a.err, 5, false);
    }
  } else if (warp < 6) {
    // ---- split the landed X tile into hi (in place) and lo
    const int st = threadIdx.x - 64;
    int64_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = (int)(it % S);
        const uint32_t r = (uint32_t)(it / S);
        if (!mbar_wait(full(s), r & 1u, abort_flag, a.err, 6)) {
          ok = false;
          break;
        }
        float4* ph = reinterpret_cast<float4*>(gbase + (xhi(s) - base));
        float4* pl = reinterpret_cast<float4*>(gbase + (xlo(s) - base));
#pragma unroll 4
        for (int j = st; j < TC_BM * TC_BK / 4; j += TC_SPLIT_T) {
          const float4 x = ph[j];
          const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
          ph[j] = h;
          pl[j] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(split(s));
      }
    }
  } else {
    // ---- epilogue: accumulator rows to Y
    const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31 belong to this warp
    int64_t ti = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
      const int b = (int)(ti & 1);
      const uint32_t u = (uint32_t)(ti >> 1);
      if (!mbar_wait(tfull(b), u & 1u, abort_flag, a.err, 7)) break;
      tc_fence_after();
      const int64_t row = t * TC_BM + 32 * q + lane;
      float* yr = a.Y + row * a.ldy;
      const int nused = nk < a.nacc ? nk : a.nacc;
      for (int c0 = 0; c0 < a.bnp; c0 += 32) {
        float v[32];
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * a.nacc * a.bnp + c0);
        tc_ld32(tl, v);
        for (int u2 = 1; u2 < nused; ++u2) {
          float w[32];
          tc_ld32(tl + (uint32_t)(u2 * a.bnp), w);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] += w[i];
        }
        if (row < a.M) {
          const int nc = a.J - c0 < 32 ? a.J - c0 : 32;
          if (nc == 32 && ((reinterpret_cast<uintptr_t>(yr + c0) & 15) == 0)) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(yr + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < nc) yr[c0 + i] = v[i];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(tempty(b));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// B (J x K, or stored K x J when trans) split into TF32 hi and lo planes, J x K row-major.
__global__ void k_tc_split_b(const float* __restrict__ B, int J, int K, int trans, float* __restrict__ bh,
                             float* __restrict__ bl) {
  const int64_t n = (int64_t)J * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / K), k = (int)(e - (int64_t)j * K);
    const float x = trans ? B[(int64_t)k * J + j] : B[e];
    const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    bh[e] = h;
    bl[e] = x - h;
  }
}

}  // namespace

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, fetched once through the runtime (no link against libcuda).
EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// Row-major FP32 matrix (rows x cols) read in boxes of box_rows x 32 floats with the 128-byte
// swizzle; reads past the edges fill zeros.
bool map_fp32_sw128(CUtensorMap* m, const float* base, int64_t rows, int64_t cols, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)cols * 4};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dim, stride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool kr_tc_eligible(const kr_ctx* ctx, const float* X, int64_t M, int K, int J) {
  if (!ctx->tensor_cores || ctx->cc_major != 10) return false;
  if (M < TC_BM * 8 || M > (int64_t(1) << 31) - TC_BM || K < TC_BK || K % 4 != 0 || J < 1 || J > 256) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return false;
  return encoder() != nullptr;
}

kr_status kr_gemm_tc(kr_ctx* ctx, const float* X, int64_t M, int K, const float* B, int J, int trans, float* Y,
                     int64_t ldy) {
  if (!kr_tc_eligible(ctx, X, M, K, J) || ldy < J) return KR_ENOTIMPL;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  KR_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
  const size_t need = (size_t)2 * J * K * sizeof(float);
  if (need > ctx->tc_size) {
    if (cap != cudaStreamCaptureStatusNone) return KR_ENOTIMPL;  // no allocation inside a capture
    if (ctx->tc_buf) {
      KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      KR_CUDA(ctx, cudaFree(ctx->tc_buf));
      ctx->tc_buf = nullptr;
      ctx->tc_size = 0;
    }
    if (cudaMalloc(&ctx->tc_buf, need) != cudaSuccess) {
      cudaGetLastError();
      ctx->tc_buf = nullptr;
      return KR_ENOTIMPL;
    }
    ctx->tc_size = need;
  }
  if (!ctx->tc_err) {
    if (cap != cudaStreamCaptureStatusNone) return KR_ENOTIMPL;
    KR_CUDA(ctx, cudaMalloc(&ctx->tc_err, sizeof(int)));
    KR_CUDA(ctx, cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->stream));
  }
  float* bh = ctx->tc_buf;
  float* bl = bh + (size_t)J * K;
  const TcShape sh = tc_shape(J);
  if (sh.stages < 2 || sh.smem > ctx->smem_optin) return KR_ENOTIMPL;
  CUtensorMap mX, mBh, mBl;
  if (!map_fp32_sw128(&mX, X, M, K, TC_BM) || !map_fp32_sw128(&mBh, bh, J, K, sh.bnp) ||
      !map_fp32_sw128(&mBl, bl, J, K, sh.bnp))
    return KR_ENOTIMPL;
  {
    int blocks = (int)(((int64_t)J * K + 255) / 256);
    if (blocks > ctx->num_sms * 4) blocks = ctx->num_sms * 4;
    KR_LAUNCH(ctx, k_tc_split_b, blocks, 256, 0, B, J, K, trans, bh, bl);
  }
  if ((int)sh.smem > ctx->tc_attr) {  // once per context (not again inside a stream capture)
    KR_CUDA(ctx, cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin));
    ctx->tc_attr = (int)ctx->smem_optin;
  }
  TcArgs a;
  a.Y = Y;
  a.M = M;
  a.ldy = ldy;
  a.K = K;
  a.J = J;
  a.bnp = sh.bnp;
  a.stages = sh.stages;
  a.nacc = sh.nacc;
  a.a_bytes = sh.a_bytes;
  a.b_bytes = sh.b_bytes;
  a.stage_bytes = sh.stage_bytes;
  a.tx_bytes = sh.tx_bytes;
  a.bar_off = sh.bar_off;
  a.tmem_cols = sh.tmem_cols;
  a.err = ctx->tc_err;
  const int64_t ntiles = (M + TC_BM - 1) / TC_BM;
  const int grid = (int)(ntiles < ctx->num_sms ? ntiles : ctx->num_sms);
  KR_LAUNCH(ctx, k_gemm_tc, grid, TC_THREADS, sh.smem, mX, mBh, mBl, a);
  ctx->tc_launches++;
  return KR_OK;
}

kr_status kr_tc_check(kr_ctx* ctx) {
  if (!ctx->tc_err) return KR_OK;
  KR_TRY(kr_hbuf_reserve(ctx, 64));
  int* h = reinterpret_cast<int*>(ctx->hbuf);
  KR_CUDA(ctx, cudaMemcpyAsync(h, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (*h != 0) {
    const int code = *h;
    KR_CUDA(ctx, cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->stream));
    return kr_fail(ctx, KR_ETIMEOUT, "tensor-core mode product: a bounded wait ran out (role %d)", code);
  }
  return KR_OK;
}

extern "C" int64_t kr_tc_launch_count(const kr_ctx* ctx) { return ctx ? ctx->tc_launches : 0; }

extern "C" int64_t kr_graph_count(const kr_ctx* ctx) { return ctx ? ctx->graphs : 0; }
