// Context, errors, workspace and argument validation of libkron.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "kr_internal.cuh"

kr_status kr_fail(kr_ctx* ctx, kr_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

kr_status kr_fail_cuda(kr_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
  kr_status st = (e == cudaErrorMemoryAllocation) ? KR_ENOMEM : KR_ECUDA;
  return kr_fail(ctx, st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

static std::mutex g_smem_attr_mu;

kr_status kr_func_smem(kr_ctx* ctx, const void* func, size_t bytes) {
  std::lock_guard<std::mutex> lock(g_smem_attr_mu);
  cudaFuncAttributes fa;
  KR_CUDA(ctx, cudaFuncGetAttributes(&fa, func));
  if (bytes > (size_t)fa.maxDynamicSharedSizeBytes)
    KR_CUDA(ctx, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return KR_OK;
}

int64_t kr_sample_count(int64_t R, double eps, double c) {
  if (!(eps > 0.0 && eps < 1.0) || R < 1) return -1;
  if (!(c > 0.0)) c = 4.0;
  if (R <= 1) return 1;
  const double v = ceil(c * (double)R * log((double)R) / eps);
  return v < 1.0 ? 1 : (int64_t)v;
}

extern "C" int64_t kron_sample_count(int64_t R, double eps, double c) { return kr_sample_count(R, eps, c); }

extern "C" kr_status kr_create(kr_ctx** out, void* stream, size_t workspace_bytes) {
  if (!out) return KR_EINVAL;
  *out = nullptr;
  kr_ctx* ctx = new kr_ctx();
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  ctx->smem_optin = (size_t)optin;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_major, cudaDevAttrComputeCapabilityMajor, ctx->device);
  for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ctx->pev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete ctx;
    return e == cudaErrorMemoryAllocation ? KR_ENOMEM : KR_ECUDA;
  }
  ctx->stream = (cudaStream_t)stream;
  // an asynchronous solve's device state and the side stream of captured loop bodies, made
  // here so that a solve captured into the caller's graph allocates nothing
  if (cudaMalloc(&ctx->gm_async, KR_GM_ASYNC_BYTES) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    kr_destroy(ctx);
    return KR_ENOMEM;
  }
  if (workspace_bytes > 0 && kr_ws_reserve(ctx, workspace_bytes) != KR_OK) {
    kr_destroy(ctx);
    return KR_ENOMEM;
  }
  *out = ctx;
  return KR_OK;
}

extern "C" kr_status kr_set_option(kr_ctx* ctx, int32_t key, int64_t value) {
  if (!ctx) return KR_EINVAL;
  switch (key) {
    case KR_OPT_SLAB_PASS:
      if (value != 0 && value != 1) return kr_fail(ctx, KR_EINVAL, "kr_set_option: slab pass must be 0 or 1");
      ctx->slab_pass = (int)value;
      return KR_OK;
    case KR_OPT_SLAB_TILE_ENTRIES:
      if (value < 256 || value > (int64_t(1) << 22))
        return kr_fail(ctx, KR_EINVAL, "kr_set_option: tile entries %lld outside [256, 2^22]", (long long)value);
      ctx->slab_tile_entries = (uint32_t)value;
      return KR_OK;
    case KR_OPT_DEVICE_LOOP:
      if (value != 0 && value != 1) return kr_fail(ctx, KR_EINVAL, "kr_set_option: device loop must be 0 or 1");
      ctx->device_loop = (int)value;
      return KR_OK;
    case KR_OPT_BATCH_WORKERS:
      if (value < 1 || value > 32) return kr_fail(ctx, KR_EINVAL, "kr_set_option: batch workers must be in [1, 32]");
      ctx->batch_workers = (int)value;
      return KR_OK;
    case KR_OPT_GROUPING:
      if (value < 0 || value > 3) return kr_fail(ctx, KR_EINVAL, "kr_set_option: grouping must be 0, 1, 2 or 3");
      ctx->grouping = (int)value;
      return KR_OK;
    case KR_OPT_JL_K:
      if (value < 0 || value > 64) return kr_fail(ctx, KR_EINVAL, "kr_set_option: JL columns must be in [0, 64]");
      ctx->jl_k = (int)value;
      return KR_OK;
    case KR_OPT_JL_SEED:
      ctx->jl_seed = (uint64_t)value;
      return KR_OK;
    case KR_OPT_TENSOR_CORES:
      if (value != 0 && value != 1) return kr_fail(ctx, KR_EINVAL, "kr_set_option: tensor cores must be 0 or 1");
      ctx->tensor_cores = (int)value;
      return KR_OK;
    case KR_OPT_BATCH_MODE:
      if (value != 0 && value != 1) return kr_fail(ctx, KR_EINVAL, "kr_set_option: batch mode must be 0 or 1");
      ctx->batch_mode = (int)value;
      return KR_OK;
    case KR_OPT_AUTOTUNE:
      if (value != 0 && value != 1) return kr_fail(ctx, KR_EINVAL, "kr_set_option: autotune must be 0 or 1");
      ctx->autotune = (int)value;
      return KR_OK;
    case KR_OPT_HOST_GATHER:
      if (value != 0 && value != 1) return kr_fail(ctx, KR_EINVAL, "kr_set_option: host gather must be 0 or 1");
      ctx->host_gather = (int)value;
      return KR_OK;
    default:
      return kr_fail(ctx, KR_EINVAL, "kr_set_option: unknown key %d", key);
  }
}

extern "C" void kr_destroy(kr_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (kr_ctx* w : ctx->workers) kr_destroy(w);
  for (cudaStream_t s : ctx->worker_streams) cudaStreamDestroy(s);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  if (ctx->b_ready) cudaEventDestroy(ctx->b_ready);
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->io) cudaFree(ctx->io);
  if (ctx->split_buf) cudaFree(ctx->split_buf);
  if (ctx->dcnt) cudaFree(ctx->dcnt);
  if (ctx->tc_buf) cudaFree(ctx->tc_buf);
  if (ctx->loop_ev) cudaEventDestroy(ctx->loop_ev);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->gm_async) cudaFree(ctx->gm_async);
  for (cudaEvent_t e : ctx->tune_ev)
    if (e) cudaEventDestroy(e);
  kr_tune_free(ctx);
  if (ctx->tc_err) cudaFree(ctx->tc_err);
  if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
  for (int i = 0; i < 10; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (int i = 0; i < 2; ++i)
    if (ctx->pev[i]) cudaEventDestroy(ctx->pev[i]);
  delete ctx;
}

extern "C" kr_status kr_set_stream(kr_ctx* ctx, void* stream) {
  if (!ctx) return KR_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return KR_OK;
}

extern "C" const char* kr_last_error(const kr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int64_t kr_launch_count(const kr_ctx* ctx) { return ctx ? ctx->launches : 0; }

kr_status kr_io_reserve(kr_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->io_size) return KR_OK;
  if (ctx->gm.on && ctx->gm.capturing) return kr_fail(ctx, KR_ENOTIMPL, "inside a capture: the host-buffer staging would have to grow (run the call once outside the capture first)");
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->copy_stream) KR_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
  if (ctx->io) {
    cudaFree(ctx->io);
    ctx->io = nullptr;
    ctx->io_size = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->io, bytes);
  if (e != cudaSuccess) {
    ctx->io = nullptr;
    cudaGetLastError();
    return kr_fail(ctx, KR_ENOMEM, "host-buffer staging allocation of %zu bytes failed", bytes);
  }
  ctx->io_size = bytes;
  return KR_OK;
}

kr_status kr_ws_reserve(kr_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_size) return KR_OK;
  if (ctx->gm.on && ctx->gm.capturing) return kr_fail(ctx, KR_ENOTIMPL, "inside a capture: the workspace would have to grow (run the call once outside the capture first)");
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
  }
  size_t want = bytes + bytes / 8 + (1 << 20);
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    ctx->ws = nullptr;
    cudaGetLastError();
    return kr_fail(ctx, KR_ENOMEM, "workspace allocation of %zu bytes failed", want);
  }
  ctx->ws_size = want;
  return KR_OK;
}

kr_status kr_split_reserve(kr_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->split_size) return KR_OK;
  if (ctx->gm.on && ctx->gm.capturing) return kr_fail(ctx, KR_ENOTIMPL, "inside a capture: the split-K buffer would have to grow (run the call once outside the capture first)");
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->split_buf) cudaFree(ctx->split_buf);
  ctx->split_buf = nullptr;
  ctx->split_size = 0;
  cudaError_t e = cudaMalloc((void**)&ctx->split_buf, bytes);
  if (e != cudaSuccess) {
    ctx->split_buf = nullptr;
    cudaGetLastError();
    return kr_fail(ctx, KR_ENOMEM, "split-K buffer allocation of %zu bytes failed", bytes);
  }
  ctx->split_size = bytes;
  return KR_OK;
}

kr_status kr_hbuf_reserve(kr_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->hbuf_size) return KR_OK;
  if (ctx->gm.on && ctx->gm.capturing) return kr_fail(ctx, KR_ENOTIMPL, "inside a capture: the pinned read-back buffer would have to grow (run the call once outside the capture first)");
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
  ctx->hbuf = nullptr;
  ctx->hbuf_size = 0;
  KR_CUDA(ctx, cudaMallocHost((void**)&ctx->hbuf, bytes));
  ctx->hbuf_size = bytes;
  return KR_OK;
}

int64_t kr_prod_I(const Modes& m) {
  int64_t p = 1;
  for (int n = 0; n < m.N; ++n) p *= m.I[n];
  return p;
}

int64_t kr_prod_R(const Modes& m) {
  int64_t p = 1;
  for (int n = 0; n < m.N; ++n) p *= m.R[n];
  return p;
}

kr_status kr_check_factors(kr_ctx* ctx, const kr_factors* f, Modes* m) {
  if (!f) return kr_fail(ctx, KR_EINVAL, "factors: null descriptor");
  if (f->N < 1 || f->N > KR_MAX_MODES) return kr_fail(ctx, KR_EINVAL, "factors: N=%d outside [1,%d]", f->N, KR_MAX_MODES);
  m->N = f->N;
  int64_t prodI = 1;
  for (int n = 0; n < f->N; ++n) {
    if (f->I[n] < 1 || f->I[n] > 65535)
      return kr_fail(ctx, KR_EINVAL, "factors: I[%d]=%lld outside [1,65535]", n, (long long)f->I[n]);
    if (f->R[n] < 1 || f->R[n] > KR_MAX_RANK)
      return kr_fail(ctx, KR_EINVAL, "factors: R[%d]=%d outside [1,%d]", n, f->R[n], KR_MAX_RANK);
    if (f->R[n] > f->I[n])
      return kr_fail(ctx, KR_EINVAL, "factors: R[%d]=%d exceeds I[%d]=%lld", n, f->R[n], n, (long long)f->I[n]);
    if (!f->A[n]) return kr_fail(ctx, KR_EINVAL, "factors: A[%d] is null", n);
    m->I[n] = (int)f->I[n];
    m->R[n] = f->R[n];
    m->A[n] = f->A[n];
    prodI *= f->I[n];
  }
  if (prodI >= (int64_t(1) << 32)) return kr_fail(ctx, KR_EINVAL, "factors: prod(I) >= 2^32");
  return KR_OK;
}

// ------------------------------------------------------------------ timing instrumentation

cudaEvent_t kr_timing_event(kr_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int kr_kind_of(const char* k) {
  std::string s(k);
  if (s.find("k_resid") != std::string::npos) return KR_K_RESID;
  if (s.find("k_slab") != std::string::npos) return KR_K_SLAB;
  if (s.find("k_mode_product") != std::string::npos || s.find("k_gemm_tc") != std::string::npos ||
      s.find("k_tc_split") != std::string::npos)
    return KR_K_MODEPROD;
  if (s.find("k_sample") != std::string::npos || s.find("k_draw") != std::string::npos) return KR_K_SAMPLE;
  if (s.find("k_guide") != std::string::npos || s.find("k_prob_rank") != std::string::npos) return KR_K_TABLES;
  if (s.find("k_radix") != std::string::npos || s.find("k_bm_") != std::string::npos) return KR_K_SCATTER;
  if (s.find("k_rle") != std::string::npos || s.find("k_cell_w") != std::string::npos) return KR_K_DEDUP;
  if (s.find("k_gram") != std::string::npos || s.find("k_chol") != std::string::npos ||
      s.find("k_leverage") != std::string::npos || s.find("k_cdf") != std::string::npos ||
      s.find("k_jacobi") != std::string::npos)
    return KR_K_TABLES;
  return KR_K_VECTOR;
}

static void kr_timing_drain(kr_ctx* ctx) {
  for (auto& t : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      ctx->t_ms[t.kind] += ms;
      ctx->t_n[t.kind] += 1;
    }
    ctx->pool.push_back(t.a);
    ctx->pool.push_back(t.b);
  }
  ctx->pending.clear();
  cudaGetLastError();
}

extern "C" kr_status kr_timing_enable(kr_ctx* ctx, int32_t on) {
  if (!ctx) return KR_EINVAL;
  ctx->timing = on != 0;
  return KR_OK;
}

extern "C" kr_status kr_timing_read(kr_ctx* ctx, int32_t kind, double* total_ms, int64_t* launches) {
  if (!ctx || kind < 0 || kind >= KR_K_KINDS) return KR_EINVAL;
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  kr_timing_drain(ctx);
  if (total_ms) *total_ms = ctx->t_ms[kind];
  if (launches) *launches = ctx->t_n[kind];
  return KR_OK;
}

extern "C" kr_status kr_timing_reset(kr_ctx* ctx) {
  if (!ctx) return KR_EINVAL;
  KR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  kr_timing_drain(ctx);
  for (int k = 0; k < KR_K_KINDS; ++k) {
    ctx->t_ms[k] = 0.0;
    ctx->t_n[k] = 0;
  }
  return KR_OK;
}
