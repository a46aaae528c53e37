// Batching support: the rendezvous that runs a fused batch's Richardson loops (Alg. 2's
// "until convergence" loop, one per problem) as concurrent conditional-WHILE nodes of one
// CUDA graph, and the autotuner's table of slab-pass tile budgets per shape class.
#include <condition_variable>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "kr_internal.cuh"

struct kr_shared_loop {
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;         // problems that may still add a loop
  int added = 0;          // loops added to the current round's graph
  uint64_t gen = 0;       // rounds launched so far
  bool round_bad = false;  // a capture of this round failed: the round is not launched
  bool last_ok = true;    // the last round ran to completion
  cudaGraph_t graph = nullptr;
  cudaStream_t stream = nullptr;    // the batch's stream (the caller's context's)
  std::vector<cudaEvent_t> wait;    // members' work before this round

  // Launches the round (mutex held): the batch's stream waits for every member's earlier
  // work, runs the graph and is synchronised; members wake up with the outcome.
  void launch_locked() {
    bool ok = !round_bad && graph != nullptr;
    for (cudaEvent_t e : wait) ok = ok && cudaStreamWaitEvent(stream, e, 0) == cudaSuccess;
    cudaGraphExec_t exec = nullptr;
    ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    ok = ok && cudaGraphLaunch(exec, stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(stream) == cudaSuccess;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (!ok) cudaGetLastError();
    graph = nullptr;
    wait.clear();
    added = 0;
    round_bad = false;
    last_ok = ok;
    ++gen;
    cv.notify_all();
  }
};

kr_shared_loop* kr_shared_loop_new(cudaStream_t stream, int members) {
  kr_shared_loop* sl = new kr_shared_loop();
  sl->stream = stream;
  sl->active = members;
  return sl;
}

void kr_shared_loop_delete(kr_shared_loop* sl) { delete sl; }

bool kr_shared_loop_run(kr_shared_loop* sl, kr_ctx* ctx,
                        const std::function<kr_status(cudaGraphConditionalHandle, int)>& body, int64_t* per_step) {
  std::unique_lock<std::mutex> lk(sl->mu);
  *per_step = 0;
  bool ok = true;
  if (!ctx->loop_ev) ok = cudaEventCreateWithFlags(&ctx->loop_ev, cudaEventDisableTiming) == cudaSuccess;
  if (ok && !sl->graph) ok = cudaGraphCreate(&sl->graph, 0) == cudaSuccess;
  cudaGraphConditionalHandle hnd = 0;
  ok = ok && cudaGraphConditionalHandleCreate(&hnd, sl->graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  ok = ok && cudaGraphAddNode(&node, sl->graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
  // this problem's earlier work (setup, first step) precedes the round
  ok = ok && cudaEventRecord(ctx->loop_ev, ctx->stream) == cudaSuccess;
  if (ok) sl->wait.push_back(ctx->loop_ev);
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
  if (!ok) {
    cudaGetLastError();
    sl->round_bad = true;  // every member of this round continues with its host loop
  }
  ++sl->added;
  const uint64_t g = sl->gen;
  if (sl->added == sl->active) sl->launch_locked();
  else sl->cv.wait(lk, [&] { return sl->gen != g; });
  return sl->last_ok;
}

void kr_shared_loop_leave(kr_shared_loop* sl) {
  std::unique_lock<std::mutex> lk(sl->mu);
  --sl->active;
  if (sl->added > 0 && sl->added == sl->active) sl->launch_locked();
}

// ------------------------------------------------------------------ autotuner table

struct kr_tune_entry {
  int64_t key[6];
  uint32_t et;
  float ms[8];
  int nc;
};

struct kr_tune_table {
  std::mutex mu;
  std::vector<kr_tune_entry> e;
};

static kr_tune_table* tune_table(kr_ctx* ctx) {
  if (!ctx->tune) {
    ctx->tune = new kr_tune_table();
    ctx->tune_owned = true;
  }
  return ctx->tune;
}

uint32_t kr_tune_lookup(kr_ctx* ctx, const int64_t* key) {
  kr_tune_table* t = tune_table(ctx);
  if (!key) return 0;
  std::lock_guard<std::mutex> lk(t->mu);
  for (const kr_tune_entry& x : t->e) {
    bool eq = true;
    for (int i = 0; i < 6; ++i) eq = eq && x.key[i] == key[i];
    if (eq) return x.et;
  }
  return 0;
}

void kr_tune_record(kr_ctx* ctx, const int64_t* key, uint32_t et, const float* ms, int nc) {
  kr_tune_table* t = tune_table(ctx);
  std::lock_guard<std::mutex> lk(t->mu);
  for (const kr_tune_entry& x : t->e) {
    bool eq = true;
    for (int i = 0; i < 6; ++i) eq = eq && x.key[i] == key[i];
    if (eq) return;  // a concurrent problem of the same class measured first
  }
  kr_tune_entry x = {};
  for (int i = 0; i < 6; ++i) x.key[i] = key[i];
  x.et = et;
  x.nc = nc < 8 ? nc : 8;
  for (int i = 0; i < x.nc; ++i) x.ms[i] = ms[i];
  t->e.push_back(x);
}

void kr_tune_free(kr_ctx* ctx) {
  if (ctx->tune_owned) delete ctx->tune;
  ctx->tune = nullptr;
  ctx->tune_owned = false;
}

extern "C" int64_t kr_autotune_report(kr_ctx* ctx, char* buf, int64_t cap) {
  if (!ctx) return 0;
  std::string out;
  kr_tune_table* t = tune_table(ctx);
  {
    std::lock_guard<std::mutex> lk(t->mu);
    for (const kr_tune_entry& x : t->e) {
      char line[256];
      int n = snprintf(line, sizeof(line), "%lld %lld %lld %lld %lld %lld %u", (long long)x.key[0], (long long)x.key[1],
                       (long long)x.key[2], (long long)x.key[3], (long long)x.key[4], (long long)x.key[5], x.et);
      for (int i = 0; i < x.nc && n < (int)sizeof(line) - 16; ++i) n += snprintf(line + n, sizeof(line) - n, " %.4f", x.ms[i]);
      out += line;
      out += "\n";
    }
  }
  if (buf && cap > 0) {
    const int64_t k = (int64_t)out.size() < cap - 1 ? (int64_t)out.size() : cap - 1;
    for (int64_t i = 0; i < k; ++i) buf[i] = out[(size_t)i];
    buf[k] = 0;
  }
  return (int64_t)out.size();
}
