// C ABI of libtf.so: operator set-up (layer spectra), products, tuning and profiling.
// Declarations and argument contracts are in include/tf.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <cstdarg>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tf.h"
#include "tf_driver.h"
#include "tf_internal.h"

using tfk::CT;
using tfk::FftPlan;

namespace {

thread_local std::string g_err;

tf_status fail(tf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

tf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TF_ENOMEM : TF_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

constexpr int kMaxFft = 1024;
constexpr int kStages = 6;

// radices of one length-n transform; false if n has a prime factor above 7
bool factor(int n, std::vector<int>& rad) {
  rad.clear();
  int m = n;
  while (m % 8 == 0) { rad.push_back(8); m /= 8; }
  if (m % 4 == 0) { rad.push_back(4); m /= 4; }
  if (m % 2 == 0) { rad.push_back(2); m /= 2; }
  for (int p : {7, 5, 3})
    while (m % p == 0) { rad.push_back(p); m /= p; }
  return m == 1 && (int)rad.size() <= tfk::kMaxPass;
}

// Transform length >= nmin.  Lengths with a compile-time plan run about twice as fast
// per element as the generic engine, so the smallest of those is taken when one fits;
// otherwise the generic length of least cost ~ n * (passes + 1), since every pass moves
// all n values through shared memory once and the stage loads/stores once more.
// Length 1 would have no pass at all (the fused first/last steps run inside passes), so
// the shortest transform is 2.
int choose_length(int nmin, bool use_menu) {
  if (nmin < 2) nmin = 2;
  if (use_menu)
    for (int i = 0; i < tfk::ct_menu_count(); ++i)
      if (tfk::ct_menu_length(i) >= nmin) return tfk::ct_menu_length(i);
  int best = -1;
  double best_cost = 1e300;
  std::vector<int> rad;
  for (int n = nmin; n <= 2 * nmin + 16; ++n) {
    if (!factor(n, rad)) continue;
    const double cost = (double)n * (rad.size() + 1);
    if (cost < best_cost) { best_cost = cost; best = n; }
  }
  return best;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, double* x, double* w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    long double z = cosl(pi * (i + 0.75L) / (n + 0.5L));
    long double dp = 1;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1);
      const long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    long double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = (double)z;
    w[i] = (double)(2.0L / ((1 - z * z) * dp * dp));
  }
}

struct HostPlan {
  FftPlan plan;
  std::vector<double> tw;  // interleaved re, im
};

HostPlan make_plan_from(int n, const std::vector<int>& rad) {
  HostPlan h;
  std::memset(&h.plan, 0, sizeof h.plan);
  h.plan.n = n;
  h.plan.np = (int)rad.size();
  int ns = 1, off = 0;
  for (int p = 0; p < h.plan.np; ++p) {
    const int R = rad[p];
    h.plan.radix[p] = R;
    h.plan.ns[p] = ns;
    h.plan.tw_off[p] = off;
    const long double L = (long double)ns * R;
    for (int k = 0; k < ns; ++k)
      for (int r = 1; r < R; ++r) {
        // w^(r k) with w = exp(-2 pi i / (ns R)); r*k < ns*R, so no reduction is needed
        const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (r * k) / L;
        h.tw.push_back((double)cosl(ang));
        h.tw.push_back((double)sinl(ang));
      }
    off += ns * (R - 1);
    ns *= R;
  }
  h.plan.tw_count = off;
  return h;
}

HostPlan make_plan(int n) {
  std::vector<int> rad;
  factor(n, rad);
  return make_plan_from(n, rad);
}

// The compile-time menu's radix list for length n (false when n has no compiled plan).
bool ct_radices(int n, std::vector<int>& rad) {
  for (int i = 0; i < tfk::ct_menu_count(); ++i) {
    if (tfk::ct_menu_length(i) != n) continue;
    int r[tfk::kMaxPass];
    const int np = tfk::ct_menu_radices(i, r);
    rad.assign(r, r + np);
    return true;
  }
  return false;
}

}  // namespace

struct tf_op {
  // geometry
  int sx, sy, nz, nx, ny, pxl, pxr, pyl, pyr;
  double dx, dy, station_z;
  std::vector<double> z_edges;
  int kind;  // 0 gravity, 1 magnetic
  double inc, dec, field;
  tf_dtype dtype;
  int device;
  // transforms
  int n1, n2, nh;
  int hs;               // row stride of half-spectrum buffers: nh rounded up to 16
  HostPlan p1, p2;
  void* tw1 = nullptr;  // device twiddles in the op dtype (generic plans)
  void* tw2 = nullptr;
  HostPlan p1ct, p2ct;  // compile-time plans (their own radix lists)
  void* tw1ct = nullptr;
  void* tw2ct = nullptr;
  void* spec = nullptr; // [nz][n2][hs] complex of the op dtype
  // workspace
  void* w1 = nullptr;   // chunk * nz*ny*hs complex
  void* w2 = nullptr;   // chunk * sy*hs complex
  int64_t chunk = 0;       // columns the allocated workspace holds
  int64_t chunk_cap = 0;   // most columns per chunk (grown into on demand)
  int rows_tile = 8, cols_tile = 8;
  bool ct1 = false, ct2 = false;  // compile-time plans exist for n1 / n2
  int engine = 0;                 // 0: compile-time plans where available, 1: generic
  // host-buffer pipeline (tf_products_host): device staging slots and their streams/events
  static constexpr int kSlots = 3;
  void* stage[2][kSlots] = {};   // [direction][slot]: one chunk's input then output
  size_t stage_bytes = 0;        // bytes of each slot
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2][kSlots] = {}, ev_cmp[2][kSlots] = {}, ev_out[2][kSlots] = {};
  cudaEvent_t ev_fork = nullptr;
  // profiling
  bool prof = false;
  struct Rec { int stage; int64_t cols; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;

  size_t csize() const { return dtype == TF_F32 ? sizeof(float2) : sizeof(double2); }
  int64_t m() const { return (int64_t)sx * sy; }
  int64_t n() const { return (int64_t)nx * ny * nz; }
  int64_t w1_per_col() const { return (int64_t)nz * ny * hs; }
  int64_t w2_per_col() const { return (int64_t)sy * hs; }
};

namespace {

void free_op(tf_op* op) {
  if (!op) return;
  cudaFree(op->tw1);
  cudaFree(op->tw2);
  cudaFree(op->tw1ct);
  cudaFree(op->tw2ct);
  cudaFree(op->spec);
  cudaFree(op->w1);
  cudaFree(op->w2);
  for (int dir = 0; dir < 2; ++dir)
    for (int k = 0; k < tf_op::kSlots; ++k) {
      cudaFree(op->stage[dir][k]);
      if (op->ev_in[dir][k]) cudaEventDestroy(op->ev_in[dir][k]);
      if (op->ev_cmp[dir][k]) cudaEventDestroy(op->ev_cmp[dir][k]);
      if (op->ev_out[dir][k]) cudaEventDestroy(op->ev_out[dir][k]);
    }
  if (op->ev_fork) cudaEventDestroy(op->ev_fork);
  if (op->s_in) cudaStreamDestroy(op->s_in);
  if (op->s_out) cudaStreamDestroy(op->s_out);
  for (auto& r : op->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : op->pool) cudaEventDestroy(e);
  delete op;
}

// ---- scratch of the allocation-free forward product (tf_matvec_noalloc) ---------------
//
// A file-scope __device__ array: every device on which the library's module is loaded
// holds kNoallocScratchBytes of it until the process exits.  Host code cannot use the
// array's name as a device address; the address is looked up per device with
// cudaGetSymbolAddress.  That lookup loads this module under CUDA's lazy loading (an
// allocation), so it is made when an operator is created (tf_create_*), never by
// tf_matvec_noalloc itself.

constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch layout for one column: the row-transformed layers (W1) at 0 and the column-stage
// output (W2) at noalloc_w2_offset, each followed by the same guard tail of n2*hs values
// that the operator's own workspace buffers carry.
size_t noalloc_guard(const tf_op* op) { return (size_t)op->n2 * op->hs * op->csize(); }
size_t noalloc_w2_offset(const tf_op* op) {
  return round256((size_t)op->w1_per_col() * op->csize() + noalloc_guard(op));
}
size_t noalloc_need(const tf_op* op) {
  return noalloc_w2_offset(op) + (size_t)op->w2_per_col() * op->csize() + noalloc_guard(op);
}

// Address of the scratch array on device dev (looked up once, then cached).
cudaError_t noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// Everything tf_matvec_noalloc would otherwise do on its first call on the operator's
// device: look up the scratch address (which loads the module holding it) and load the
// generic forward kernels at the operator's tiles with their shared-memory limits raised.
// Runs at creation and whenever the tiles change; a no-op for operators too large for the
// scratch.  The operator's device must be current.
tf_status noalloc_prepare(const tf_op* op) {
  if (noalloc_need(op) > kNoallocScratchBytes) return TF_OK;
  void* p = nullptr;
  cudaError_t e = noalloc_scratch(op->device, &p);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
  e = op->dtype == TF_F32
          ? tfk::prepare_forward_generic<float>(op->n1, op->p1.plan.tw_count, op->n2,
                                                op->p2.plan.tw_count, op->rows_tile, op->cols_tile)
          : tfk::prepare_forward_generic<double>(op->n1, op->p1.plan.tw_count, op->n2,
                                                 op->p2.plan.tw_count, op->rows_tile, op->cols_tile);
  return e == cudaSuccess ? TF_OK : cuda_fail(e, "loading the generic product kernels");
}

tf_status upload_twiddles(const HostPlan& h, tf_dtype dt, void** dst) {
  const size_t count = h.tw.size() / 2;
  const size_t bytes = std::max<size_t>(1, count) * (dt == TF_F32 ? sizeof(float2) : sizeof(double2));
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(twiddles)");
  if (count == 0) return TF_OK;
  if (dt == TF_F64) {
    e = cudaMemcpy(*dst, h.tw.data(), count * sizeof(double2), cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f(h.tw.size());
    for (size_t i = 0; i < f.size(); ++i) f[i] = (float)h.tw[i];
    e = cudaMemcpy(*dst, f.data(), count * sizeof(float2), cudaMemcpyHostToDevice);
  }
  return e == cudaSuccess ? TF_OK : cuda_fail(e, "cudaMemcpy(twiddles)");
}

// Each workspace buffer carries a guard tail of one full transform column block
// (n2 * hs complex values) beyond the last column it serves, so that no read near the
// end of a column block can leave the allocation.
tf_status alloc_workspace(tf_op* op, int64_t chunk, cudaError_t* err = nullptr) {
  cudaFree(op->w1);
  cudaFree(op->w2);
  op->w1 = op->w2 = nullptr;
  op->chunk = 0;
  const size_t guard = (size_t)op->n2 * op->hs * op->csize();
  cudaError_t e = cudaMalloc(&op->w1, (size_t)chunk * op->w1_per_col() * op->csize() + guard);
  if (e == cudaSuccess) e = cudaMalloc(&op->w2, (size_t)chunk * op->w2_per_col() * op->csize() + guard);
  if (err) *err = e;
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
  // zero once: the row padding (values nh..hs-1) is never written by the row kernels
  e = cudaMemset(op->w1, 0, (size_t)chunk * op->w1_per_col() * op->csize() + guard);
  if (e == cudaSuccess) e = cudaMemset(op->w2, 0, (size_t)chunk * op->w2_per_col() * op->csize() + guard);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(workspace)");
  op->chunk = chunk;
  return TF_OK;
}

// Most columns per chunk: a workspace budget of 16 GiB, or an eighth of the device's free
// memory when that is less.  Larger chunks mean fewer launch tails: measured on the c4 block
// (2510 columns), 39.6 ms per G X + G^T Y step with 234-column chunks (2 GiB), 38.6 ms with
// 837 and 38.5 ms with 1255; on the c2 block one chunk of 1260 columns ran 20 % faster than
// L2-sized chunks of 48.
int64_t default_chunk_cap(const tf_op* op) {
  const double per = (double)(op->w1_per_col() + op->w2_per_col()) * op->csize();
  double budget = 16.0 * 1073741824.0;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (double)fr / 8 < budget)
    budget = std::max((double)fr / 8, 268435456.0);
  int64_t c = (int64_t)(budget / per);
  if (c < 1) c = 1;
  if (c > 4096) c = 4096;
  return c;
}

// Columns per chunk for a block of B columns with room for `chunk`: the fewest chunks, of
// equal size (no short last chunk, whose launches would fill a fraction of the GPU).
int64_t balanced_chunk(int64_t B, int64_t chunk) {
  if (B <= 0) return 0;
  if (chunk <= 0 || B <= chunk) return B;
  const int64_t n = (B + chunk - 1) / chunk;
  return (B + n - 1) / n;
}

// Grows the workspace (once, stream-ordered through cudaFree's implicit
// synchronisation) so that a block of B columns runs in as few chunks as the cap allows.
// When the device cannot hold that many columns (other operators, the caller's buffers),
// the product still runs in more, smaller chunks: the request halves until it fits, and
// the smaller size becomes the operator's cap.
tf_status ensure_workspace(tf_op* op, int64_t B) {
  int64_t want = balanced_chunk(B, op->chunk_cap);
  if (op->chunk >= want) return TF_OK;
  for (;;) {
    cudaError_t e = cudaSuccess;
    const tf_status st = alloc_workspace(op, want, &e);
    if (st == TF_OK || e != cudaErrorMemoryAllocation || want <= 1) return st;
    cudaGetLastError();   // the failed allocation's (non-sticky) error
    want = (want + 1) / 2;
    op->chunk_cap = want;
  }
}

tf_status create_common(const tf_grid* g, int kind, double inc, double dec, double field,
                        tf_dtype dt, tf_stream stream, tf_op** out) {
  if (!out) return fail(TF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!g) return fail(TF_EINVAL, "grid is NULL");
  if (dt != TF_F32 && dt != TF_F64) return fail(TF_EINVAL, "unknown dtype %d", (int)dt);
  if (g->sx < 1 || g->sy < 1 || g->nz < 1)
    return fail(TF_EINVAL, "sx, sy, nz must be >= 1 (got %d, %d, %d)", g->sx, g->sy, g->nz);
  if (g->pxl < 0 || g->pxr < 0 || g->pyl < 0 || g->pyr < 0)
    return fail(TF_EINVAL, "padding counts must be >= 0");
  if (!(g->dx > 0) || !(g->dy > 0)) return fail(TF_EINVAL, "dx, dy must be > 0");
  if (!g->z_edges) return fail(TF_EINVAL, "z_edges is NULL");
  for (int r = 0; r < g->nz; ++r)
    if (!(g->z_edges[r + 1] > g->z_edges[r]))
      return fail(TF_EINVAL, "z_edges must be strictly increasing (index %d)", r);
  if (!(g->z_edges[0] >= g->station_z))
    return fail(TF_EINVAL, "stations must lie at or above the top of the volume");
  if (kind == 1 && !(field > 0)) return fail(TF_EINVAL, "field strength must be > 0");

  tf_op* op = new tf_op();
  op->sx = g->sx; op->sy = g->sy; op->nz = g->nz;
  op->pxl = g->pxl; op->pxr = g->pxr; op->pyl = g->pyl; op->pyr = g->pyr;
  op->nx = g->sx + g->pxl + g->pxr;
  op->ny = g->sy + g->pyl + g->pyr;
  op->dx = g->dx; op->dy = g->dy; op->station_z = g->station_z;
  op->z_edges.assign(g->z_edges, g->z_edges + g->nz + 1);
  op->kind = kind; op->inc = inc; op->dec = dec; op->field = field;
  op->dtype = dt;
  cudaGetDevice(&op->device);

  const int n1min = op->sx + op->nx - 1, n2min = op->sy + op->ny - 1;
  op->n1 = choose_length(n1min, true);
  op->n2 = choose_length(n2min, true);
  if (op->n1 < 0 || op->n2 < 0 || op->n1 > kMaxFft || op->n2 > kMaxFft) {
    delete op;
    return fail(TF_EUNSUPPORTED, "embedding %d x %d exceeds the supported %d per axis", n1min,
                n2min, kMaxFft);
  }
  op->nh = op->n1 / 2 + 1;
  op->hs = (op->nh + 15) & ~15;
  op->p1 = make_plan(op->n1);
  op->p2 = make_plan(op->n2);
  {
    std::vector<int> rad;
    if ((op->ct1 = ct_radices(op->n1, rad))) op->p1ct = make_plan_from(op->n1, rad);
    if ((op->ct2 = ct_radices(op->n2, rad))) {
      int r[tfk::kMaxPass];  // single-precision column kernels have their own menu
      const int np = dt == TF_F32 ? tfk::ct_menu_cols_radices(op->n2, r) : 0;
      if (np > 0) rad.assign(r, r + np);
      op->p2ct = make_plan_from(op->n2, rad);
    }
  }
  op->rows_tile = dt == TF_F32 ? 8 : 4;
  op->cols_tile = dt == TF_F32 ? 8 : 4;

  cudaStream_t s = (cudaStream_t)stream;
  tf_status st = TF_OK;
  double* d_z = nullptr;
  double* d_tab = nullptr;
  double2* d_ht = nullptr;
  double2* d_spec64 = nullptr;
  void* tw1_64 = nullptr;
  void* tw2_64 = nullptr;
  cudaError_t e;
  const int64_t ntab = (int64_t)op->nz * n2min * n1min;
  const int64_t nht = (int64_t)op->nz * n2min * op->nh;
  const int64_t nspec = (int64_t)op->nz * op->n2 * op->hs;

#define TF_TRY(call, what)                       \
  do {                                           \
    e = (call);                                  \
    if (e != cudaSuccess) { st = cuda_fail(e, what); goto done; } \
  } while (0)

  if ((st = upload_twiddles(op->p1, dt, &op->tw1)) != TF_OK) goto done;
  if ((st = upload_twiddles(op->p2, dt, &op->tw2)) != TF_OK) goto done;
  if (op->ct1 && (st = upload_twiddles(op->p1ct, dt, &op->tw1ct)) != TF_OK) goto done;
  if (op->ct2 && (st = upload_twiddles(op->p2ct, dt, &op->tw2ct)) != TF_OK) goto done;
  if (dt == TF_F32) {
    if ((st = upload_twiddles(op->p1, TF_F64, &tw1_64)) != TF_OK) goto done;
    if ((st = upload_twiddles(op->p2, TF_F64, &tw2_64)) != TF_OK) goto done;
  } else {
    tw1_64 = op->tw1;
    tw2_64 = op->tw2;
  }
  TF_TRY(cudaMalloc(&d_z, sizeof(double) * (op->nz + 1)), "cudaMalloc(z_edges)");
  TF_TRY(cudaMemcpy(d_z, op->z_edges.data(), sizeof(double) * (op->nz + 1), cudaMemcpyHostToDevice),
         "cudaMemcpy(z_edges)");
  TF_TRY(cudaMalloc(&d_tab, sizeof(double) * ntab), "cudaMalloc(kernel table)");
  TF_TRY(cudaMalloc(&d_ht, sizeof(double2) * nht), "cudaMalloc(row spectra)");
  TF_TRY(cudaMalloc(&d_spec64, sizeof(double2) * nspec), "cudaMalloc(spectra)");
  TF_TRY(cudaMemsetAsync(d_spec64, 0, sizeof(double2) * nspec, s), "cudaMemsetAsync(spectra)");
  {
    tfk::TableArgs ta;
    ta.kind = kind; ta.n1min = n1min; ta.n2min = n2min; ta.nz = op->nz;
    ta.nx = op->nx; ta.ny = op->ny; ta.pxl = op->pxl; ta.pyl = op->pyl;
    ta.dx = op->dx; ta.dy = op->dy; ta.station_z = op->station_z; ta.z_edges = d_z;
    const double I = inc * 3.14159265358979323846 / 180.0, D = dec * 3.14159265358979323846 / 180.0;
    ta.fx = cos(I) * cos(D); ta.fy = cos(I) * sin(D); ta.fz = sin(I); ta.field = field;
    ta.out = d_tab;
    gauss_legendre(6, ta.g6x, ta.g6w);
    gauss_legendre(8, ta.g8x, ta.g8w);
    gauss_legendre(14, ta.g14x, ta.g14w);
    TF_TRY(tfk::launch_table(ta, s), "kernel table launch");

    tfk::RowsR2C<double> ra;
    ra.src = d_tab; ra.src_ld = 0; ra.row_len = n1min; ra.nrows = op->nz * n2min;
    ra.seq_off = 0; ra.scale = nullptr; ra.dst = d_ht; ra.dst_ld = 0; ra.nh = op->nh; ra.hs = op->nh;
    ra.plan = op->p1.plan; ra.tw = (const double2*)tw1_64;
    TF_TRY(tfk::launch_rows_r2c<double>(ra, 1, 4, s), "row FFT of kernel table");

    tfk::SpecArgs sa;
    sa.ht = d_ht; sa.n2min = n2min; sa.nh = op->nh; sa.nz = op->nz;
    sa.scale = 1.0 / ((double)op->n1 * op->n2);
    sa.spec = d_spec64; sa.hs = op->hs; sa.plan = op->p2.plan; sa.tw = (const double2*)tw2_64;
    TF_TRY(tfk::launch_spectrum(sa, 4, s), "column FFT of kernel table");
  }
  if (dt == TF_F64) {
    op->spec = d_spec64;
    d_spec64 = nullptr;
  } else {
    TF_TRY(cudaMalloc(&op->spec, sizeof(float2) * nspec), "cudaMalloc(spectra f32)");
    TF_TRY(tfk::launch_to_f32(d_spec64, (float2*)op->spec, nspec, s), "spectra rounding");
  }
  TF_TRY(cudaStreamSynchronize(s), "spectra set-up");
  op->chunk_cap = default_chunk_cap(op);
  if ((st = alloc_workspace(op, 1)) != TF_OK) goto done;
  if ((st = noalloc_prepare(op)) != TF_OK) goto done;

done:
#undef TF_TRY
  cudaFree(d_z);
  cudaFree(d_tab);
  cudaFree(d_ht);
  cudaFree(d_spec64);
  if (dt == TF_F32) { cudaFree(tw1_64); cudaFree(tw2_64); }
  if (st != TF_OK) { free_op(op); return st; }
  *out = op;
  return TF_OK;
}

cudaEvent_t take_event(tf_op* op) {
  if (!op->pool.empty()) { cudaEvent_t e = op->pool.back(); op->pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Runs one stage launch, bracketed by profiling events when enabled.
template <class F>
cudaError_t stage(tf_op* op, int id, int64_t cols, cudaStream_t s, F&& launch) {
  if (!op->prof) return launch();
  tf_op::Rec r{id, cols, take_event(op), take_event(op)};
  cudaEventRecord(r.a, s);
  cudaError_t e = launch();
  cudaEventRecord(r.b, s);
  op->recs.push_back(r);
  return e;
}

tf_status check_op(const tf_op* op) {
  if (!op) return fail(TF_EINVAL, "op is NULL");
  return TF_OK;
}

template <typename T>
tf_status forward_impl(tf_op* op, int64_t B, const T* X, int64_t ldx, T* D, int64_t ldd,
                       const T* cs, const T* rs, cudaStream_t s) {
  typedef typename CT<T>::C C;
  tf_status st = ensure_workspace(op, B);
  if (st != TF_OK) return st;
  C* w1 = (C*)op->w1;
  C* w2 = (C*)op->w2;
  const C* tw1 = (const C*)op->tw1;
  const C* tw2 = (const C*)op->tw2;
  const int64_t step = balanced_chunk(B, op->chunk);
  for (int64_t c0 = 0; c0 < B; c0 += step) {
    const int cb = (int)std::min<int64_t>(step, B - c0);
    tfk::RowsR2C<T> a;
    a.src = X + c0 * ldx; a.src_ld = ldx; a.row_len = op->nx; a.nrows = op->nz * op->ny;
    a.seq_off = 0; a.scale = cs; a.dst = w1; a.dst_ld = op->w1_per_col(); a.nh = op->nh; a.hs = op->hs;
    a.plan = op->p1.plan; a.tw = tw1;
    const bool c1 = op->engine == 0 && op->ct1, c2 = op->engine == 0 && op->ct2;
    cudaError_t e = stage(op, 0, cb, s, [&] {
      if (!c1) return tfk::launch_rows_r2c<T>(a, cb, op->rows_tile, s);
      tfk::RowsR2C<T> ac = a;
      ac.tw = (const C*)op->tw1ct;
      return tfk::ct_rows_r2c<T>(ac, cb, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "rows_r2c launch");
    tfk::ColsFwd<T> b;
    b.z = w1; b.z_ld = op->w1_per_col(); b.spec = (const C*)op->spec; b.s = w2;
    b.s_ld = op->w2_per_col(); b.nh = op->nh; b.hs = op->hs; b.ny = op->ny; b.sy = op->sy; b.nz = op->nz;
    b.plan = op->p2.plan; b.tw = tw2;
    e = stage(op, 1, cb, s, [&] {
      if (!c2) return tfk::launch_cols_fwd<T>(b, cb, op->cols_tile, s);
      tfk::ColsFwd<T> bc = b;
      bc.tw = (const C*)op->tw2ct;
      return tfk::ct_cols_fwd<T>(bc, cb, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "cols_fwd launch");
    tfk::RowsC2R<T> c;
    c.src = w2; c.src_ld = op->w2_per_col(); c.nh = op->nh; c.hs = op->hs; c.nrows = op->sy;
    c.dst = D + c0 * ldd; c.dst_ld = ldd; c.out_len = op->sx; c.seq_off = op->nx - 1;
    c.scale = rs; c.plan = op->p1.plan; c.tw = tw1;
    e = stage(op, 2, cb, s, [&] {
      if (!c1) return tfk::launch_rows_c2r<T>(c, cb, op->rows_tile, s);
      tfk::RowsC2R<T> cc = c;
      cc.tw = (const C*)op->tw1ct;
      return tfk::ct_rows_c2r<T>(cc, cb, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "rows_c2r launch");
  }
  return TF_OK;
}

template <typename T>
tf_status adjoint_impl(tf_op* op, int64_t B, const T* Y, int64_t ldy, T* X, int64_t ldx,
                       const T* cs, const T* rs, cudaStream_t s) {
  typedef typename CT<T>::C C;
  tf_status st = ensure_workspace(op, B);
  if (st != TF_OK) return st;
  C* w1 = (C*)op->w1;
  C* w2 = (C*)op->w2;
  const C* tw1 = (const C*)op->tw1;
  const C* tw2 = (const C*)op->tw2;
  const int64_t step = balanced_chunk(B, op->chunk);
  for (int64_t c0 = 0; c0 < B; c0 += step) {
    const int cb = (int)std::min<int64_t>(step, B - c0);
    tfk::RowsR2C<T> a;
    a.src = Y + c0 * ldy; a.src_ld = ldy; a.row_len = op->sx; a.nrows = op->sy;
    a.seq_off = op->nx - 1; a.scale = rs; a.dst = w2; a.dst_ld = op->w2_per_col();
    a.nh = op->nh; a.hs = op->hs; a.plan = op->p1.plan; a.tw = tw1;
    const bool c1 = op->engine == 0 && op->ct1, c2 = op->engine == 0 && op->ct2;
    cudaError_t e = stage(op, 3, cb, s, [&] {
      if (!c1) return tfk::launch_rows_r2c<T>(a, cb, op->rows_tile, s);
      tfk::RowsR2C<T> ac = a;
      ac.tw = (const C*)op->tw1ct;
      return tfk::ct_rows_r2c<T>(ac, cb, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "rows_r2c launch");
    tfk::ColsAdj<T> b;
    b.z = w2; b.z_ld = op->w2_per_col(); b.spec = (const C*)op->spec; b.u = w1;
    b.u_ld = op->w1_per_col(); b.nh = op->nh; b.hs = op->hs; b.ny = op->ny; b.sy = op->sy; b.nz = op->nz;
    b.plan = op->p2.plan; b.tw = tw2;
    e = stage(op, 4, cb, s, [&] {
      if (!c2) return tfk::launch_cols_adj<T>(b, cb, op->cols_tile, s);
      tfk::ColsAdj<T> bc = b;
      bc.tw = (const C*)op->tw2ct;
      return tfk::ct_cols_adj<T>(bc, cb, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "cols_adj launch");
    tfk::RowsC2R<T> c;
    c.src = w1; c.src_ld = op->w1_per_col(); c.nh = op->nh; c.hs = op->hs; c.nrows = op->nz * op->ny;
    c.dst = X + c0 * ldx; c.dst_ld = ldx; c.out_len = op->nx; c.seq_off = 0; c.scale = cs;
    c.plan = op->p1.plan; c.tw = tw1;
    e = stage(op, 5, cb, s, [&] {
      if (!c1) return tfk::launch_rows_c2r<T>(c, cb, op->rows_tile, s);
      tfk::RowsC2R<T> cc = c;
      cc.tw = (const C*)op->tw1ct;
      return tfk::ct_rows_c2r<T>(cc, cb, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "rows_c2r launch");
  }
  return TF_OK;
}

}  // namespace

extern "C" {

tf_status tf_create_gravity(const tf_grid* grid, tf_dtype dtype, tf_stream stream, tf_op** out) {
  return create_common(grid, 0, 90.0, 0.0, 1.0, dtype, stream, out);
}

tf_status tf_create_magnetic(const tf_grid* grid, double inc_deg, double dec_deg,
                             double field_nt, tf_dtype dtype, tf_stream stream, tf_op** out) {
  return create_common(grid, 1, inc_deg, dec_deg, field_nt, dtype, stream, out);
}

tf_status tf_destroy(tf_op* op) {
  if (!op) return TF_OK;
  // A fault of earlier work surfaces here; report it rather than let the next call on
  // this device be the first to see it.
  const cudaError_t e = cudaDeviceSynchronize();
  const unsigned pipe = e == cudaSuccess ? tfk::ct_pipe_status(true) : 0u;
  free_op(op);
  if (e != cudaSuccess) return cuda_fail(e, "work pending at tf_destroy");
  if (pipe) return fail(TF_ETIMEOUT, "a row kernel's bounded wait for its input copy ran out");
  return TF_OK;
}

tf_status tf_dims(const tf_op* op, int64_t* m, int64_t* n) {
  if (check_op(op)) return TF_EINVAL;
  if (m) *m = op->m();
  if (n) *n = op->n();
  return TF_OK;
}

tf_status tf_fft_dims(const tf_op* op, int* n1, int* n2) {
  if (check_op(op)) return TF_EINVAL;
  if (n1) *n1 = op->n1;
  if (n2) *n2 = op->n2;
  return TF_OK;
}

tf_status tf_matmat(tf_op* op, int64_t B, const void* X, int64_t ldx, void* D, int64_t ldd,
                    const void* colscale, const void* rowscale, tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  if (B < 0) return fail(TF_EINVAL, "B must be >= 0");
  if (B == 0) return TF_OK;
  if (!X || !D) return fail(TF_EINVAL, "X and D must be non-NULL");
  if (ldx < op->n() || ldd < op->m())
    return fail(TF_EINVAL, "ldx (%lld) must be >= n (%lld) and ldd (%lld) >= m (%lld)",
                (long long)ldx, (long long)op->n(), (long long)ldd, (long long)op->m());
  cudaStream_t s = (cudaStream_t)stream;
  if (op->dtype == TF_F32)
    return forward_impl<float>(op, B, (const float*)X, ldx, (float*)D, ldd,
                               (const float*)colscale, (const float*)rowscale, s);
  return forward_impl<double>(op, B, (const double*)X, ldx, (double*)D, ldd,
                              (const double*)colscale, (const double*)rowscale, s);
}

tf_status tf_rmatmat(tf_op* op, int64_t B, const void* Y, int64_t ldy, void* X, int64_t ldx,
                     const void* colscale, const void* rowscale, tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  if (B < 0) return fail(TF_EINVAL, "B must be >= 0");
  if (B == 0) return TF_OK;
  if (!X || !Y) return fail(TF_EINVAL, "Y and X must be non-NULL");
  if (ldy < op->m() || ldx < op->n())
    return fail(TF_EINVAL, "ldy (%lld) must be >= m (%lld) and ldx (%lld) >= n (%lld)",
                (long long)ldy, (long long)op->m(), (long long)ldx, (long long)op->n());
  cudaStream_t s = (cudaStream_t)stream;
  if (op->dtype == TF_F32)
    return adjoint_impl<float>(op, B, (const float*)Y, ldy, (float*)X, ldx,
                               (const float*)colscale, (const float*)rowscale, s);
  return adjoint_impl<double>(op, B, (const double*)Y, ldy, (double*)X, ldx,
                              (const double*)colscale, (const double*)rowscale, s);
}

tf_status tf_matvec(tf_op* op, const void* x, void* d, const void* colscale,
                    const void* rowscale, tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  return tf_matmat(op, 1, x, op->n(), d, op->m(), colscale, rowscale, stream);
}

tf_status tf_rmatvec(tf_op* op, const void* y, void* x, const void* colscale,
                     const void* rowscale, tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  return tf_rmatmat(op, 1, y, op->m(), x, op->n(), colscale, rowscale, stream);
}

}  // extern "C"

namespace {

// Streams, events and staging slots of the host-buffer pipeline, created on first use and
// grown when a call needs larger slots (growth frees and allocates, which waits for the
// device to be idle).
tf_status ensure_host_pipeline(tf_op* op, size_t slot_bytes) {
  cudaError_t e = cudaSuccess;
  if (!op->s_in) {
    if ((e = cudaStreamCreateWithFlags(&op->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&op->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&op->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "host pipeline streams");
    for (int dir = 0; dir < 2; ++dir)
      for (int k = 0; k < tf_op::kSlots; ++k)
        if ((e = cudaEventCreateWithFlags(&op->ev_in[dir][k], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&op->ev_cmp[dir][k], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&op->ev_out[dir][k], cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(e, "host pipeline events");
  }
  if (op->stage_bytes >= slot_bytes) return TF_OK;
  for (int dir = 0; dir < 2; ++dir)
    for (int k = 0; k < tf_op::kSlots; ++k) {
      cudaFree(op->stage[dir][k]);
      op->stage[dir][k] = nullptr;
    }
  op->stage_bytes = 0;
  for (int dir = 0; dir < 2; ++dir)
    for (int k = 0; k < tf_op::kSlots; ++k)
      if ((e = cudaMalloc(&op->stage[dir][k], slot_bytes)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(host pipeline staging)");
  op->stage_bytes = slot_bytes;
  return TF_OK;
}

// cb columns of `rows` values between a column-major block (leading dimension ld, in
// elements) and a packed one, as one copy when the columns are contiguous.
cudaError_t copy_cols(void* dst, int64_t dld, const void* src, int64_t sld, int64_t rows,
                      int64_t cb, size_t esz, cudaMemcpyKind kind, cudaStream_t s) {
  if (dld == rows && sld == rows)
    return cudaMemcpyAsync(dst, src, (size_t)(rows * cb) * esz, kind, s);
  return cudaMemcpy2DAsync(dst, (size_t)dld * esz, src, (size_t)sld * esz, (size_t)rows * esz,
                           (size_t)cb, kind, s);
}

}  // namespace

extern "C" {

tf_status tf_products_host(tf_op* op, int64_t B1, const void* X, int64_t ldx, void* D,
                           int64_t ldd, int64_t B2, const void* Y, int64_t ldy, void* XT,
                           int64_t ldxt, const void* colscale, const void* rowscale, int chunks,
                           tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  if (B1 < 0 || B2 < 0 || chunks < 1) return fail(TF_EINVAL, "need B1, B2 >= 0 and chunks >= 1");
  if ((B1 > 0 && (!X || !D || ldx < op->n() || ldd < op->m())) ||
      (B2 > 0 && (!Y || !XT || ldy < op->m() || ldxt < op->n())))
    return fail(TF_EINVAL, "null block or leading dimension below the block's rows");
  if (B1 == 0 && B2 == 0) return TF_OK;
  const size_t esz = op->dtype == TF_F32 ? sizeof(float) : sizeof(double);
  const int64_t cmax = (std::max(B1, B2) + chunks - 1) / chunks;   // columns per chunk
  const size_t slot = (size_t)cmax * (size_t)(op->n() + op->m()) * esz;
  tf_status st = ensure_host_pipeline(op, slot);
  if (st != TF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
#define TF_HP(call, what) \
  do { if ((e = (call)) != cudaSuccess) return cuda_fail(e, what); } while (0)
  // the copy streams start after everything already queued on the caller's stream
  TF_HP(cudaEventRecord(op->ev_fork, s), "cudaEventRecord");
  TF_HP(cudaStreamWaitEvent(op->s_in, op->ev_fork, 0), "cudaStreamWaitEvent");
  TF_HP(cudaStreamWaitEvent(op->s_out, op->ev_fork, 0), "cudaStreamWaitEvent");
  // Per chunk: G^T's columns first, then G's, so that the two large copies (X in, G^T Y
  // out) of neighbouring chunks overlap on the full-duplex host link.  Chunk c of a
  // direction uses slot c % kSlots once the copy out of the slot's previous chunk is done.
  int64_t chunk_no[2] = {0, 0};
  for (int c = 0; c < chunks; ++c) {
    for (int dir = 1; dir >= 0; --dir) {
      const int64_t Bd = dir ? B2 : B1;
      const int64_t c0 = Bd * c / chunks, c1 = Bd * (c + 1) / chunks, cb = c1 - c0;
      if (cb <= 0) continue;
      const int k = (int)(chunk_no[dir]++ % tf_op::kSlots);
      const int64_t rin = dir ? op->m() : op->n(), rout = dir ? op->n() : op->m();
      unsigned char* din = (unsigned char*)op->stage[dir][k];
      unsigned char* dout = din + (size_t)cb * rin * esz;
      const unsigned char* hin = (const unsigned char*)(dir ? Y : X) + (size_t)(c0 * (dir ? ldy : ldx)) * esz;
      unsigned char* hout = (unsigned char*)(dir ? XT : D) + (size_t)(c0 * (dir ? ldxt : ldd)) * esz;
      TF_HP(cudaStreamWaitEvent(op->s_in, op->ev_out[dir][k], 0), "cudaStreamWaitEvent");
      TF_HP(copy_cols(din, rin, hin, dir ? ldy : ldx, rin, cb, esz, cudaMemcpyHostToDevice, op->s_in),
            "host-to-device copy");
      TF_HP(cudaEventRecord(op->ev_in[dir][k], op->s_in), "cudaEventRecord");
      TF_HP(cudaStreamWaitEvent(s, op->ev_in[dir][k], 0), "cudaStreamWaitEvent");
      st = dir ? tf_rmatmat(op, cb, din, rin, dout, rout, colscale, rowscale, stream)
               : tf_matmat(op, cb, din, rin, dout, rout, colscale, rowscale, stream);
      if (st != TF_OK) return st;
      TF_HP(cudaEventRecord(op->ev_cmp[dir][k], s), "cudaEventRecord");
      TF_HP(cudaStreamWaitEvent(op->s_out, op->ev_cmp[dir][k], 0), "cudaStreamWaitEvent");
      TF_HP(copy_cols(hout, dir ? ldxt : ldd, dout, rout, rout, cb, esz, cudaMemcpyDeviceToHost,
                      op->s_out),
            "device-to-host copy");
      TF_HP(cudaEventRecord(op->ev_out[dir][k], op->s_out), "cudaEventRecord");
    }
  }
  // the caller's stream resumes once the last copy out is done
  TF_HP(cudaEventRecord(op->ev_fork, op->s_out), "cudaEventRecord");
  TF_HP(cudaStreamWaitEvent(s, op->ev_fork, 0), "cudaStreamWaitEvent");
#undef TF_HP
  return TF_OK;
}

tf_status tf_get_spectra(const tf_op* op, void* dst, int64_t bytes, tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  const int64_t need = (int64_t)op->nz * op->n2 * op->nh * (int64_t)op->csize();
  if (!dst || bytes != need)
    return fail(TF_EINVAL, "dst must hold exactly %lld bytes", (long long)need);
  // the operator keeps rows of nh values at stride hs; the copy packs them
  cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)op->nh * op->csize(), op->spec,
                                    (size_t)op->hs * op->csize(), (size_t)op->nh * op->csize(),
                                    (size_t)op->nz * op->n2, cudaMemcpyDefault, (cudaStream_t)stream);
  return e == cudaSuccess ? TF_OK : cuda_fail(e, "cudaMemcpyAsync(spectra)");
}

tf_status tf_set_tuning(tf_op* op, int rows_tile, int cols_tile, int64_t chunk_cols) {
  if (check_op(op)) return TF_EINVAL;
  auto ok_tile = [](int t) { return t == 0 || t == 4 || t == 8 || t == 16; };
  if (!ok_tile(rows_tile) || !ok_tile(cols_tile) || chunk_cols < 0)
    return fail(TF_EINVAL, "tiles must be 0, 4, 8 or 16 and chunk_cols >= 0");
  const int rt = rows_tile ? rows_tile : op->rows_tile;
  const int ct = cols_tile ? cols_tile : op->cols_tile;
  const size_t lim = 227 * 1024;
  if (tfk::smem_rows(op->n1, op->p1.plan.tw_count, rt, op->csize()) > lim ||
      tfk::smem_cols(op->n2, op->p2.plan.tw_count, ct, op->csize()) > lim)
    return fail(TF_EUNSUPPORTED, "tile needs more than 227 KB of shared memory");
  const bool retiled = rt != op->rows_tile || ct != op->cols_tile;
  op->rows_tile = rt;
  op->cols_tile = ct;
  if (retiled) {
    const tf_status pst = noalloc_prepare(op);
    if (pst != TF_OK) return pst;
  }
  if (chunk_cols) {
    op->chunk_cap = chunk_cols;
    if (chunk_cols != op->chunk) {
      cudaDeviceSynchronize();
      return alloc_workspace(op, chunk_cols);
    }
  }
  return TF_OK;
}

tf_status tf_set_radices(tf_op* op, int axis, const int* radices, int count) {
  if (check_op(op)) return TF_EINVAL;
  if (axis != 0 && axis != 1) return fail(TF_EINVAL, "axis must be 0 (x) or 1 (y)");
  if (!radices || count < 1 || count > tfk::kMaxPass)
    return fail(TF_EINVAL, "need 1 to %d radices", tfk::kMaxPass);
  const int n = axis == 0 ? op->n1 : op->n2;
  int prod = 1;
  std::vector<int> rad(radices, radices + count);
  for (int r : rad) {
    if (r != 2 && r != 3 && r != 4 && r != 5 && r != 7 && r != 8)
      return fail(TF_EINVAL, "radix %d is not one of 2, 3, 4, 5, 7, 8", r);
    prod *= r;
  }
  if (prod != n) return fail(TF_EINVAL, "radices multiply to %d, the transform length is %d", prod, n);
  HostPlan h = make_plan_from(n, rad);
  void* tw = nullptr;
  tf_status st = upload_twiddles(h, op->dtype, &tw);
  if (st != TF_OK) { cudaFree(tw); return st; }
  cudaDeviceSynchronize();   // no product of this operator may still use the old table
  void*& old = axis == 0 ? op->tw1 : op->tw2;
  cudaFree(old);
  old = tw;
  (axis == 0 ? op->p1 : op->p2) = h;
  return TF_OK;
}

tf_status tf_get_radices(const tf_op* op, int axis, int* radices, int* count) {
  if (check_op(op)) return TF_EINVAL;
  if ((axis != 0 && axis != 1) || !radices || !count)
    return fail(TF_EINVAL, "axis must be 0 or 1, radices and count non-NULL");
  const tfk::FftPlan& p = axis == 0 ? op->p1.plan : op->p2.plan;
  for (int i = 0; i < p.np; ++i) radices[i] = p.radix[i];
  *count = p.np;
  return TF_OK;
}

tf_status tf_set_engine(tf_op* op, int engine) {
  if (check_op(op)) return TF_EINVAL;
  if (engine != 0 && engine != 1) return fail(TF_EINVAL, "engine must be 0 or 1");
  op->engine = engine;
  return TF_OK;
}

tf_status tf_get_engine(const tf_op* op, int* engine, int* compiled_rows, int* compiled_cols) {
  if (check_op(op)) return TF_EINVAL;
  if (engine) *engine = op->engine;
  if (compiled_rows) *compiled_rows = op->engine == 0 && op->ct1;
  if (compiled_cols) *compiled_cols = op->engine == 0 && op->ct2;
  return TF_OK;
}

tf_status tf_get_tuning(const tf_op* op, int* rows_tile, int* cols_tile, int64_t* chunk_cols) {
  if (check_op(op)) return TF_EINVAL;
  if (rows_tile) *rows_tile = op->rows_tile;
  if (cols_tile) *cols_tile = op->cols_tile;
  if (chunk_cols) *chunk_cols = op->chunk;
  return TF_OK;
}

tf_status tf_profile_enable(tf_op* op, int enable) {
  if (check_op(op)) return TF_EINVAL;
  for (auto& r : op->recs) { cudaEventSynchronize(r.b); op->pool.push_back(r.a); op->pool.push_back(r.b); }
  op->recs.clear();
  op->prof = enable != 0;
  return TF_OK;
}

tf_status tf_profile_read(tf_op* op, double* ms, int64_t* launches, int64_t* columns) {
  if (check_op(op)) return TF_EINVAL;
  if (!ms || !launches || !columns) return fail(TF_EINVAL, "output arrays must be non-NULL");
  for (int i = 0; i < kStages; ++i) { ms[i] = 0; launches[i] = 0; columns[i] = 0; }
  for (auto& r : op->recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float t = 0;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms[r.stage] += t;
    launches[r.stage] += 1;
    columns[r.stage] += r.cols;
  }
  return TF_OK;
}

tf_status tf_debug_oob(int* checked, int* site, int64_t* offset, int64_t* extent) {
  tfk::OobRecord recs[5];
  bool ok = tfk::oob_read_generic(&recs[0], true);
  ok = tfk::oob_read_ct_f32(&recs[1], true) && ok;
  ok = tfk::oob_read_ct_f64(&recs[2], true) && ok;
  ok = tfk::oob_read_batch_f32(&recs[3], true) && ok;
  ok = tfk::oob_read_batch_f64(&recs[4], true) && ok;
  if (checked) *checked = ok ? 1 : 0;
  if (site) *site = 0;
  if (offset) *offset = 0;
  if (extent) *extent = 0;
  for (auto& r : recs)
    if (r.hit) {
      if (site) *site = r.site;
      if (offset) *offset = r.off;
      if (extent) *extent = r.ext;
      break;
    }
  return TF_OK;
}

tf_status tf_rows_dot(tf_dtype dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                      const void* x, double* y, tf_stream stream) {
  if (dtype != TF_F32 && dtype != TF_F64) return fail(TF_EINVAL, "unknown dtype %d", (int)dtype);
  if (k < 0 || len < 0 || (k > 1 && lda < len)) return fail(TF_EINVAL, "need k, len >= 0 and lda >= len");
  if (k > 0 && (!A || !x || !y)) return fail(TF_EINVAL, "A, x and y must be non-NULL");
  if (k > 2147483647LL) return fail(TF_EINVAL, "k too large");
  cudaError_t e = tfk::launch_rows_dot(dtype == TF_F32 ? 0 : 1, A, lda, k, len, x, y, (cudaStream_t)stream);
  return e == cudaSuccess ? TF_OK : cuda_fail(e, "rows_dot launch");
}

tf_status tf_rows_axpy(tf_dtype dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                       const double* c, void* x, tf_stream stream) {
  if (dtype != TF_F32 && dtype != TF_F64) return fail(TF_EINVAL, "unknown dtype %d", (int)dtype);
  if (k < 0 || len < 0 || (k > 1 && lda < len)) return fail(TF_EINVAL, "need k, len >= 0 and lda >= len");
  if (k > 0 && len > 0 && (!A || !c || !x)) return fail(TF_EINVAL, "A, c and x must be non-NULL");
  cudaError_t e = tfk::launch_rows_axpy(dtype == TF_F32 ? 0 : 1, A, lda, k, len, c, x, (cudaStream_t)stream);
  return e == cudaSuccess ? TF_OK : cuda_fail(e, "rows_axpy launch");
}

tf_status tf_peak_probe(tf_dtype dtype, double* tflops, tf_stream stream) {
  if (!tflops) return fail(TF_EINVAL, "tflops is NULL");
  if (dtype != TF_F32 && dtype != TF_F64) return fail(TF_EINVAL, "unknown dtype %d", (int)dtype);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  const int blocks = sms * 8;
  const int iters = dtype == TF_F32 ? 65536 : 4096;
  void* out = nullptr;
  e = cudaMalloc(&out, (size_t)blocks * 256 * 8);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(probe)");
  float ms = 0;
  e = tfk::launch_fma_probe(dtype == TF_F32 ? 0 : 1, out, blocks, iters, &ms, (cudaStream_t)stream);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "FMA probe");
  *tflops = 2.0 * 8.0 * iters * (double)blocks * 256 / (ms * 1e-3) / 1e12;
  return TF_OK;
}

const char* tf_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace tfk {

tf_status op_info(const tf_op* op, OpInfo* out) {
  if (check_op(op)) return TF_EINVAL;
  out->dtype = op->dtype;
  out->m = op->m();
  out->n = op->n();
  out->nx = op->nx;
  out->ny = op->ny;
  out->nz = op->nz;
  out->z_edges = op->z_edges;
  out->station_z = op->station_z;
  out->device = op->device;
  return TF_OK;
}

OpGeneric op_generic(const tf_op* op) {
  OpGeneric g;
  g.dtype = op->dtype;
  g.m = op->m();
  g.n = op->n();
  g.w1_per_col = op->w1_per_col();
  g.w2_per_col = op->w2_per_col();
  g.csize = op->csize();
  g.n1 = op->n1;
  g.n2 = op->n2;
  g.tw1 = op->p1.plan.tw_count;
  g.tw2 = op->p2.plan.tw_count;
  g.rows_model = op->nz * op->ny;
  g.rows_data = op->sy;
  g.nh = op->nh;
  return g;
}

template <typename T>
void op_product_stages(const tf_op* op, const T* X, T* D, const T* Y, T* XT, void* fw1, void* fw2,
                       void* aw1, void* aw2, ProductStages<T>* out) {
  typedef typename CT<T>::C C;
  const C* tw1 = (const C*)op->tw1;
  const C* tw2 = (const C*)op->tw2;
  ProductStages<T>& o = *out;
  o.f0.src = X; o.f0.src_ld = op->n(); o.f0.row_len = op->nx; o.f0.nrows = op->nz * op->ny;
  o.f0.seq_off = 0; o.f0.scale = nullptr; o.f0.dst = (C*)fw1; o.f0.dst_ld = op->w1_per_col();
  o.f0.nh = op->nh; o.f0.hs = op->hs; o.f0.plan = op->p1.plan; o.f0.tw = tw1;
  o.f1.z = (const C*)fw1; o.f1.z_ld = op->w1_per_col(); o.f1.spec = (const C*)op->spec;
  o.f1.s = (C*)fw2; o.f1.s_ld = op->w2_per_col(); o.f1.nh = op->nh; o.f1.hs = op->hs;
  o.f1.ny = op->ny; o.f1.sy = op->sy; o.f1.nz = op->nz; o.f1.plan = op->p2.plan; o.f1.tw = tw2;
  o.f2.src = (const C*)fw2; o.f2.src_ld = op->w2_per_col(); o.f2.nh = op->nh; o.f2.hs = op->hs;
  o.f2.nrows = op->sy; o.f2.dst = D; o.f2.dst_ld = op->m(); o.f2.out_len = op->sx;
  o.f2.seq_off = op->nx - 1; o.f2.scale = nullptr; o.f2.plan = op->p1.plan; o.f2.tw = tw1;
  o.a0.src = Y; o.a0.src_ld = op->m(); o.a0.row_len = op->sx; o.a0.nrows = op->sy;
  o.a0.seq_off = op->nx - 1; o.a0.scale = nullptr; o.a0.dst = (C*)aw2; o.a0.dst_ld = op->w2_per_col();
  o.a0.nh = op->nh; o.a0.hs = op->hs; o.a0.plan = op->p1.plan; o.a0.tw = tw1;
  o.a1.z = (const C*)aw2; o.a1.z_ld = op->w2_per_col(); o.a1.spec = (const C*)op->spec;
  o.a1.u = (C*)aw1; o.a1.u_ld = op->w1_per_col(); o.a1.nh = op->nh; o.a1.hs = op->hs;
  o.a1.ny = op->ny; o.a1.sy = op->sy; o.a1.nz = op->nz; o.a1.plan = op->p2.plan; o.a1.tw = tw2;
  o.a2.src = (const C*)aw1; o.a2.src_ld = op->w1_per_col(); o.a2.nh = op->nh; o.a2.hs = op->hs;
  o.a2.nrows = op->nz * op->ny; o.a2.dst = XT; o.a2.dst_ld = op->n(); o.a2.out_len = op->nx;
  o.a2.seq_off = 0; o.a2.scale = nullptr; o.a2.plan = op->p1.plan; o.a2.tw = tw1;
}
template void op_product_stages<float>(const tf_op*, const float*, float*, const float*, float*,
                                       void*, void*, void*, void*, ProductStages<float>*);
template void op_product_stages<double>(const tf_op*, const double*, double*, const double*,
                                        double*, void*, void*, void*, void*, ProductStages<double>*);

OpLaunchKey op_launch_key(const tf_op* op) {
  return OpLaunchKey{op->w1, op->chunk, op->engine, op->rows_tile, op->cols_tile, op->tw1, op->tw2};
}

tf_status api_fail(tf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

}  // namespace tfk

// ---- forward product without any allocation --------------------------------------------
//
// tf_matvec_noalloc runs the generic engine's three forward stages for one column with
// its scratch (the row-transformed layers and the column-stage output) in the library's
// fixed device array instead of the operator's workspace.  The generic kernels load the
// scratch only at positions the same call has written (masked loads of rows < ny,
// values < nh), so what an earlier call left there never reaches the result.

namespace {

template <typename T>
tf_status noalloc_forward(const tf_op* op, const T* x, T* d, const T* cs, const T* rs,
                          void* scratch, cudaStream_t s) {
  typedef typename CT<T>::C C;
  C* w1 = (C*)scratch;
  C* w2 = (C*)((unsigned char*)scratch + noalloc_w2_offset(op));
  const C* tw1 = (const C*)op->tw1;
  const C* tw2 = (const C*)op->tw2;
  tfk::RowsR2C<T> a;
  a.src = x; a.src_ld = op->n(); a.row_len = op->nx; a.nrows = op->nz * op->ny;
  a.seq_off = 0; a.scale = cs; a.dst = w1; a.dst_ld = op->w1_per_col(); a.nh = op->nh; a.hs = op->hs;
  a.plan = op->p1.plan; a.tw = tw1;
  cudaError_t e = tfk::launch_rows_r2c<T>(a, 1, op->rows_tile, s);
  if (e != cudaSuccess) return cuda_fail(e, "rows_r2c launch");
  tfk::ColsFwd<T> b;
  b.z = w1; b.z_ld = op->w1_per_col(); b.spec = (const C*)op->spec; b.s = w2;
  b.s_ld = op->w2_per_col(); b.nh = op->nh; b.hs = op->hs; b.ny = op->ny; b.sy = op->sy; b.nz = op->nz;
  b.plan = op->p2.plan; b.tw = tw2;
  e = tfk::launch_cols_fwd<T>(b, 1, op->cols_tile, s);
  if (e != cudaSuccess) return cuda_fail(e, "cols_fwd launch");
  tfk::RowsC2R<T> c;
  c.src = w2; c.src_ld = op->w2_per_col(); c.nh = op->nh; c.hs = op->hs; c.nrows = op->sy;
  c.dst = d; c.dst_ld = op->m(); c.out_len = op->sx; c.seq_off = op->nx - 1;
  c.scale = rs; c.plan = op->p1.plan; c.tw = tw1;
  e = tfk::launch_rows_c2r<T>(c, 1, op->rows_tile, s);
  if (e != cudaSuccess) return cuda_fail(e, "rows_c2r launch");
  return TF_OK;
}

}  // namespace

extern "C" tf_status tf_matvec_noalloc(const tf_op* op, const void* x, void* d,
                                       const void* colscale, const void* rowscale,
                                       tf_stream stream) {
  if (check_op(op)) return TF_EINVAL;
  if (!x || !d) return fail(TF_EINVAL, "x and d must be non-NULL");
  const size_t need = noalloc_need(op);
  if (need > kNoallocScratchBytes)
    return fail(TF_EINVAL,
                "tf_matvec_noalloc: this operator needs %zu bytes of scratch per column, more "
                "than the library's fixed %zu-byte buffer; use tf_matvec",
                need, kNoallocScratchBytes);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != op->device)
    return fail(TF_EINVAL, "current device %d is not the operator's device %d", dev, op->device);
  void* scratch = nullptr;
  e = noalloc_scratch(dev, &scratch);   // cached since the operator's creation
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
  cudaStream_t s = (cudaStream_t)stream;
  if (op->dtype == TF_F32)
    return noalloc_forward<float>(op, (const float*)x, (float*)d, (const float*)colscale,
                                  (const float*)rowscale, scratch, s);
  return noalloc_forward<double>(op, (const double*)x, (double*)d, (const double*)colscale,
                                 (const double*)rowscale, scratch, s);
}
