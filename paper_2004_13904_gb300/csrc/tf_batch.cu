// Batches of independent problems (tf_batch_*): the block products of several operators
// forked over internal streams, optionally recorded once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <vector>

#include <algorithm>
#include <cstring>

#include "../../include/tf.h"
#include "tf_driver.h"
#include "tf_internal.h"

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
  // persistent mode (tf_batch_persistent): per-problem workspaces of both directions,
  // the device-side work list and control words, and the recorded launch
  struct Persist {
    int64_t B = 0;                   // columns the workspaces hold
    std::vector<void*> ws;           // per problem: fw1, fw2, aw1, aw2 in one allocation
    void* dev = nullptr;             // segments | arguments | counters | work | status
    size_t dev_bytes = 0;
    std::vector<unsigned char> host; // the uploaded segments and arguments (kept alive)
    tfk::BatchCtl ctl{};
    size_t smem = 0;
    int tb = 0, tk = 0, grid = 0;
    size_t ctl_off = 0, ctl_bytes = 0;  // the zeroed region (counters, work, status)
    // key of the uploaded work list / recorded graph
    int64_t key_B = -1;
    std::vector<const void*> key_ptrs;
    std::vector<tfk::OpLaunchKey> key_ops;
    int key_tb = 0, key_tk = 0, key_claim = 0;
    unsigned long long key_budget = 0;
    const int* key_gate = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* status_host = nullptr;      // page-locked word the status is copied to
  } p;
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
  if (b->p.exec) cudaGraphExecDestroy(b->p.exec);
  for (void* w : b->p.ws) cudaFree(w);
  cudaFree(b->p.dev);
  if (b->p.status_host) cudaFreeHost(b->p.status_host);
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

// ---- persistent mode ---------------------------------------------------------------------

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Builds the work list of one launch: for each stage (rows, columns, rows), every
// problem's forward then transpose segment; a segment of stage s > 0 waits, per column,
// on its direction's stage s - 1.  Uploads segments and arguments, (re)allocates the
// per-problem workspaces, and fills b->p.ctl.
template <typename T>
tf_status persist_prepare(tf_batch* b, int64_t B, const void* const* X, void* const* D,
                          const void* const* Y, void* const* XT, int tb, int tk, int claim,
                          unsigned long long budget, const int* gate) {
  auto& P = b->p;
  const size_t n = b->ops.size();
  std::vector<tfk::OpGeneric> g(n);
  for (size_t i = 0; i < n; ++i) g[i] = tfk::op_generic(b->ops[i]);
  // workspaces: forward W1, W2 and transpose W1, W2 for B columns each
  if (P.B < B || P.ws.size() != n) {
    TRY_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    for (void* w : P.ws) cudaFree(w);
    P.ws.assign(n, nullptr);
    P.B = 0;
    for (size_t i = 0; i < n; ++i) {
      const size_t per = (size_t)(g[i].w1_per_col + g[i].w2_per_col) * g[i].csize;
      TRY_CUDA(cudaMalloc(&P.ws[i], 2 * per * (size_t)B), "cudaMalloc(batch workspace)");
    }
    P.B = B;
  }
  std::vector<tfk::BatchSeg> seg;
  std::vector<tfk::BatchArgs<T>> args;
  int counters = 0;
  long long item = 0;
  size_t smem = 0;
  std::vector<tfk::ProductStages<T>> st(n);
  std::vector<int> cbase(n * 6, -1);   // counter base per (problem, stage of 6)
  for (size_t i = 0; i < n; ++i) {
    const size_t w1 = (size_t)g[i].w1_per_col * g[i].csize * (size_t)P.B;
    const size_t w2 = (size_t)g[i].w2_per_col * g[i].csize * (size_t)P.B;
    unsigned char* base = (unsigned char*)P.ws[i];
    tfk::op_product_stages<T>(b->ops[i], X ? (const T*)X[i] : nullptr, D ? (T*)D[i] : nullptr,
                              Y ? (const T*)Y[i] : nullptr, XT ? (T*)XT[i] : nullptr, base,
                              base + w1, base + w1 + w2, base + 2 * w1 + w2, &st[i]);
    smem = std::max({smem, tfk::smem_rows(g[i].n1, g[i].tw1, tb, g[i].csize),
                     tfk::smem_cols(g[i].n2, g[i].tw2, tk, g[i].csize)});
  }
  auto add = [&](int kind, int tiles, int wait, int wait_target, const tfk::BatchArgs<T>& a) {
    tfk::BatchSeg sg;
    sg.first = item;
    sg.kind = kind;
    sg.tiles = tiles;
    sg.cols = (int)B;
    sg.args = (int)args.size();
    sg.wait = wait;
    sg.wait_target = wait_target;
    sg.count = counters;
    counters += (int)B;
    item += (long long)tiles * B;
    seg.push_back(sg);
    args.push_back(a);
    return sg.count;
  };
  auto rows_tiles = [&](int nrows) { return (int)(((nrows + 1) / 2 + tb - 1) / tb); };
  auto cols_tiles = [&](int nh) { return (int)((nh + tk - 1) / tk); };
  std::vector<int> tiles_of(n * 6, 0);
  for (int stage = 0; stage < 3; ++stage)
    for (size_t i = 0; i < n; ++i)
      for (int dir = 0; dir < 2; ++dir) {
        const bool on = dir == 0 ? (X && X[i] && D && D[i]) : (Y && Y[i] && XT && XT[i]);
        if (!on) continue;
        const int k = (int)i * 6 + dir * 3 + stage;
        tfk::BatchArgs<T> a;
        std::memset(&a, 0, sizeof a);
        int kind, tiles;
        if (dir == 0) {
          if (stage == 0) { a.r2c = st[i].f0; kind = 0; tiles = rows_tiles(g[i].rows_model); }
          else if (stage == 1) { a.fwd = st[i].f1; kind = 1; tiles = cols_tiles(g[i].nh); }
          else { a.c2r = st[i].f2; kind = 2; tiles = rows_tiles(g[i].rows_data); }
        } else {
          if (stage == 0) { a.r2c = st[i].a0; kind = 0; tiles = rows_tiles(g[i].rows_data); }
          else if (stage == 1) { a.adj = st[i].a1; kind = 3; tiles = cols_tiles(g[i].nh); }
          else { a.c2r = st[i].a2; kind = 2; tiles = rows_tiles(g[i].rows_model); }
        }
        tiles_of[k] = tiles;
        cbase[k] = add(kind, tiles, stage ? cbase[k - 1] : -1, stage ? tiles_of[k - 1] : 0, a);
      }
  if (seg.empty()) return TF_OK;
  // device layout: segments | arguments | counters | work word | status word
  const size_t seg_b = align256(seg.size() * sizeof(tfk::BatchSeg));
  const size_t arg_b = align256(args.size() * sizeof(tfk::BatchArgs<T>));
  const size_t ctr_b = align256((size_t)counters * sizeof(int));
  const size_t need = seg_b + arg_b + ctr_b + 256 + 256;
  if (P.dev_bytes < need) {
    TRY_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    cudaFree(P.dev);
    P.dev = nullptr;
    P.dev_bytes = 0;
    TRY_CUDA(cudaMalloc(&P.dev, need), "cudaMalloc(batch work list)");
    P.dev_bytes = need;
  }
  P.host.assign(seg_b + arg_b, 0);
  std::memcpy(P.host.data(), seg.data(), seg.size() * sizeof(tfk::BatchSeg));
  std::memcpy(P.host.data() + seg_b, args.data(), args.size() * sizeof(tfk::BatchArgs<T>));
  TRY_CUDA(cudaMemcpy(P.dev, P.host.data(), seg_b + arg_b, cudaMemcpyHostToDevice),
           "cudaMemcpy(batch work list)");
  unsigned char* d = (unsigned char*)P.dev;
  P.ctl.seg = (const tfk::BatchSeg*)d;
  P.ctl.args = d + seg_b;
  P.ctl.counters = (int*)(d + seg_b + arg_b);
  P.ctl.work = (unsigned long long*)(d + seg_b + arg_b + ctr_b);
  P.ctl.status = (int*)(d + seg_b + arg_b + ctr_b + 256);
  P.ctl.gate = gate;
  P.ctl.total = item;
  P.ctl.nseg = (int)seg.size();
  P.ctl.budget_ns = budget;
  P.ctl.claim = claim;
  P.ctl_off = seg_b + arg_b;
  P.ctl_bytes = ctr_b + 512;
  P.smem = smem;
  P.tb = tb;
  P.tk = tk;
  return TF_OK;
}

// One launch: zero the counters, work and status words, run the kernel.
template <typename T>
tf_status persist_issue(tf_batch* b, cudaStream_t s) {
  auto& P = b->p;
  if (P.ctl.total == 0) return TF_OK;
  TRY_CUDA(cudaMemsetAsync((unsigned char*)P.dev + P.ctl_off, 0, P.ctl_bytes, s), "cudaMemsetAsync");
  cudaError_t e = tfk::launch_batch<T>(P.ctl, P.tb, P.tk, P.smem, s, &P.grid);
  if (e == cudaErrorInvalidValue)
    return api_fail(TF_EINVAL, "tile pair %d x %d is not compiled for this dtype", P.tb, P.tk);
  TRY_CUDA(e, "persistent batch launch");
  return TF_OK;
}

template <typename T>
tf_status persist_run(tf_batch* b, int64_t B, const void* const* X, void* const* D,
                      const void* const* Y, void* const* XT, const tf_batch_opts* o,
                      cudaStream_t main) {
  auto& P = b->p;
  const bool f32 = std::is_same<T, float>::value;
  const int tb = o && o->rows_tile ? o->rows_tile : (f32 ? 8 : 4);
  const int tk = o && o->cols_tile ? o->cols_tile : (f32 ? 8 : 4);
  const int claim = o && o->claim > 0 ? o->claim : 2;
  const double wait_ms = o && o->wait_ms > 0 ? o->wait_ms : 2000.0;
  const unsigned long long budget = (unsigned long long)(wait_ms * 1e6);
  const int* gate = o ? o->gate : nullptr;
  const bool graph = o && o->use_graph;
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
  const bool same = B == P.key_B && ptrs == P.key_ptrs && keys == P.key_ops && tb == P.key_tb &&
                    tk == P.key_tk && claim == P.key_claim && budget == P.key_budget &&
                    gate == P.key_gate;
  if (!same) {
    if (P.exec) { cudaGraphExecDestroy(P.exec); P.exec = nullptr; }
    tf_status st = persist_prepare<T>(b, B, X, D, Y, XT, tb, tk, claim, budget, gate);
    if (st != TF_OK) { P.key_B = -1; return st; }
    P.key_B = B; P.key_ptrs = ptrs; P.key_ops = keys; P.key_tb = tb; P.key_tk = tk;
    P.key_claim = claim; P.key_budget = budget; P.key_gate = gate;
  }
  if (!P.status_host) TRY_CUDA(cudaMallocHost((void**)&P.status_host, sizeof(int)), "cudaMallocHost");
  if (graph && P.exec) {
    TRY_CUDA(cudaGraphLaunch(P.exec, main), "cudaGraphLaunch");
  } else if (graph && same) {
    // record the memset and the launch once (the work list is already on the device)
    TRY_CUDA(cudaStreamSynchronize(main), "cudaStreamSynchronize");
    TRY_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    tf_status st = persist_issue<T>(b, b->origin);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->origin, &gr);
    if (st != TF_OK) { if (gr) cudaGraphDestroy(gr); return st; }
    if (e != cudaSuccess) return api_fail(TF_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&P.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) { P.exec = nullptr; return api_fail(TF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); }
    TRY_CUDA(cudaGraphLaunch(P.exec, main), "cudaGraphLaunch");
  } else {
    tf_status st = persist_issue<T>(b, main);
    if (st != TF_OK) return st;
  }
  if (P.ctl.total == 0) return TF_OK;
  TRY_CUDA(cudaMemcpyAsync(P.status_host, P.ctl.status, sizeof(int), cudaMemcpyDeviceToHost, main),
           "cudaMemcpyAsync(status)");
  TRY_CUDA(cudaStreamSynchronize(main), "persistent batch");
  if (*P.status_host == TF_ETIMEOUT)
    return api_fail(TF_ETIMEOUT, "tf_batch_persistent: a device-side wait exceeded %.3f ms", wait_ms);
  if (*P.status_host != 0) return api_fail(TF_ECUDA, "tf_batch_persistent: status %d", *P.status_host);
  return TF_OK;
}

}  // namespace

extern "C" tf_status tf_batch_persistent(tf_batch* b, int64_t B, const void* const* X,
                                         void* const* D, const void* const* Y, void* const* XT,
                                         const tf_batch_opts* opts, tf_stream stream) {
  if (!b) return api_fail(TF_EINVAL, "batch is NULL");
  if (B < 0) return api_fail(TF_EINVAL, "B must be >= 0");
  if (B == 0) return TF_OK;
  if (B > (int64_t)1 << 24) return api_fail(TF_EINVAL, "B too large for the work list");
  if (opts && (opts->claim < 0 || opts->rows_tile < 0 || opts->cols_tile < 0))
    return api_fail(TF_EINVAL, "negative option");
  const tf_dtype dt = b->info[0].dtype;
  for (const auto& in : b->info)
    if (in.dtype != dt) return api_fail(TF_EINVAL, "persistent mode needs one dtype for all operators");
  cudaStream_t s = (cudaStream_t)stream;
  return dt == TF_F32 ? persist_run<float>(b, B, X, D, Y, XT, opts, s)
                      : persist_run<double>(b, B, X, D, Y, XT, opts, s);
}
