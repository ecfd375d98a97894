// Batches of independent problems (tf_batch_*): the block products of several operators
// forked over internal streams, optionally recorded once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/tf.h"
#include "tf_driver.h"

struct tf_batch {
  std::vector<tf_op*> ops;
  std::vector<tfk::OpInfo> info;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;  // one per internal stream
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;   // capture origin (not the caller's stream)
  // the recorded graph and what it was recorded for
  cudaGraphExec_t exec = nullptr;
  int64_t key_B = -1;
  std::vector<const void*> key_ptrs;
  std::vector<tfk::OpLaunchKey> key_ops;
  int seen = 0;  // identical calls in a row (1: eager warm-up done, 2+: graph)
};

namespace {

using tfk::api_fail;

#define TRY_CUDA(call, what)                                                   \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return api_fail(e_ == cudaErrorMemoryAllocation ? TF_ENOMEM : TF_ECUDA,  \
                      "%s: %s", what, cudaGetErrorString(e_));                 \
  } while (0)

void release(tf_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

// The forked launches: stream j serves operators j, j + S, ...; `main` is ordered after all.
tf_status issue(tf_batch* b, int64_t B, const void* const* X, void* const* D, const void* const* Y,
                void* const* XT, cudaStream_t main) {
  TRY_CUDA(cudaEventRecord(b->fork, main), "cudaEventRecord");
  for (auto s : b->streams) TRY_CUDA(cudaStreamWaitEvent(s, b->fork, 0), "cudaStreamWaitEvent");
  const size_t S = b->streams.size();
  for (size_t i = 0; i < b->ops.size(); ++i) {
    cudaStream_t s = b->streams[i % S];
    const tfk::OpInfo& in = b->info[i];
    if (X && X[i] && D && D[i]) {
      tf_status st = tf_matmat(b->ops[i], B, X[i], in.n, D[i], in.m, nullptr, nullptr, s);
      if (st != TF_OK) return st;
    }
    if (Y && Y[i] && XT && XT[i]) {
      tf_status st = tf_rmatmat(b->ops[i], B, Y[i], in.m, XT[i], in.n, nullptr, nullptr, s);
      if (st != TF_OK) return st;
    }
  }
  for (size_t j = 0; j < S; ++j) {
    TRY_CUDA(cudaEventRecord(b->joins[j], b->streams[j]), "cudaEventRecord");
    TRY_CUDA(cudaStreamWaitEvent(main, b->joins[j], 0), "cudaStreamWaitEvent");
  }
  return TF_OK;
}

}  // namespace

extern "C" {

tf_status tf_batch_create(tf_op* const* ops, int count, int streams, tf_batch** out) {
  if (!out) return api_fail(TF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ops || count < 1) return api_fail(TF_EINVAL, "need count >= 1 operators");
  if (streams < 1) return api_fail(TF_EINVAL, "streams must be >= 1");
  tf_batch* b = new tf_batch();
  for (int i = 0; i < count; ++i) {
    tfk::OpInfo in;
    tf_status st = ops[i] ? tfk::op_info(ops[i], &in) : api_fail(TF_EINVAL, "operator %d is NULL", i);
    if (st != TF_OK) { release(b); return st; }
    b->ops.push_back(ops[i]);
    b->info.push_back(in);
  }
  const int S = streams < count ? streams : count;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int j = 0; e == cudaSuccess && j < S; ++j) {
    cudaStream_t s;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->streams.push_back(s);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->joins.push_back(ev);
  }
  if (e != cudaSuccess) {
    release(b);
    return api_fail(TF_ECUDA, "tf_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return TF_OK;
}

tf_status tf_batch_destroy(tf_batch* batch) {
  if (batch) cudaDeviceSynchronize();
  release(batch);
  return TF_OK;
}

tf_status tf_batch_products(tf_batch* b, int64_t B, const void* const* X, void* const* D,
                            const void* const* Y, void* const* XT, int use_graph, tf_stream stream) {
  if (!b) return api_fail(TF_EINVAL, "batch is NULL");
  if (B < 0) return api_fail(TF_EINVAL, "B must be >= 0");
  if (B == 0) return TF_OK;
  cudaStream_t main = (cudaStream_t)stream;
  if (!use_graph) return issue(b, B, X, D, Y, XT, main);
  // what a recorded graph depends on
  const size_t n = b->ops.size();
  std::vector<const void*> ptrs(4 * n, nullptr);
  std::vector<tfk::OpLaunchKey> keys(n);
  for (size_t i = 0; i < n; ++i) {
    ptrs[4 * i] = X ? X[i] : nullptr;
    ptrs[4 * i + 1] = D ? D[i] : nullptr;
    ptrs[4 * i + 2] = Y ? Y[i] : nullptr;
    ptrs[4 * i + 3] = XT ? XT[i] : nullptr;
    keys[i] = tfk::op_launch_key(b->ops[i]);
  }
  const bool same = B == b->key_B && ptrs == b->key_ptrs && keys == b->key_ops;
  if (same && b->exec) {
    TRY_CUDA(cudaGraphLaunch(b->exec, main), "cudaGraphLaunch");
    return TF_OK;
  }
  if (!same || b->seen == 0) {
    // eager run: sizes every workspace and raises kernel attributes before any capture
    tf_status st = issue(b, B, X, D, Y, XT, main);
    if (st != TF_OK) return st;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    b->key_B = B;
    b->key_ptrs = ptrs;
    for (size_t i = 0; i < n; ++i) keys[i] = tfk::op_launch_key(b->ops[i]);  // after any growth
    b->key_ops = keys;
    b->seen = 1;
    return TF_OK;
  }
  // record the forked launches on the internal origin stream, then launch on `main`
  TRY_CUDA(cudaStreamSynchronize(main), "cudaStreamSynchronize");
  TRY_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  tf_status st = issue(b, B, X, D, Y, XT, b->origin);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->origin, &graph);
  if (st != TF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) return api_fail(TF_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { b->exec = nullptr; return api_fail(TF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); }
  b->seen = 2;
  TRY_CUDA(cudaGraphLaunch(b->exec, main), "cudaGraphLaunch");
  return TF_OK;
}

}  // extern "C"
