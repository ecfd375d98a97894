// Product kernels on the compile-time FFT engine (tf_fft_ct.cuh), for the transform
// lengths of TF_CT_MENU.  They compute exactly what the generic kernels of
// tf_kernels.cu compute (same stages, same data layout, same twiddle tables); only the
// index arithmetic is resolved at compile time.  Included by tf_ct_f32.cu / tf_ct_f64.cu.
#pragma once
#include <cuda.h>

#include <atomic>
#include <type_traits>

#include "tf_bulk.cuh"
#include "tf_check.cuh"
#include "tf_fft_ct.cuh"
#include "tf_internal.h"
#include "tf_tmem.cuh"

// Transform lengths with a compile-time plan, and their radix lists (the same order
// the host planner produces: eights first, then a four or two, then 7, 5, 3).
#define TF_CT_MENU(X)        \
  X(32, 8, 4)                \
  X(64, 8, 8)                \
  X(96, 8, 4, 3)             \
  X(128, 8, 8, 2)            \
  X(160, 8, 4, 5)            \
  X(192, 8, 8, 3)            \
  X(224, 8, 4, 7)            \
  X(256, 8, 8, 4)            \
  X(320, 8, 8, 5)            \
  X(448, 8, 8, 7)            \
  X(512, 8, 8, 8)

// The column kernels' menu in single precision: n = 224 as two passes (16, 14), which
// moves each value through shared memory one time fewer than (8, 4, 7); the double
// kernels keep TF_CT_MENU (measured 2 % slower with the two-pass plan).
#define TF_CT_MENU_COLS_F32(X)                                                              \
  X(32, 8, 4) X(64, 8, 8) X(96, 8, 4, 3) X(128, 8, 8, 2) X(160, 8, 4, 5) X(192, 8, 8, 3)    \
  X(224, 16, 14) X(256, 8, 8, 4) X(320, 8, 8, 5) X(448, 8, 8, 7) X(512, 8, 8, 8)

namespace tfk {
namespace ctk {

using ct::Vec;

__host__ __device__ constexpr int twpad(int c) { return (c + 1) & ~1; }

template <typename C> __device__ __forceinline__ C zero() { return mk<C>(0, 0); }

// Half-spectrum rows are stored with a row stride hs that is a multiple of 16 values,
// so the V values k1 .. k1+V-1 (k1 a multiple of V) of a row are one aligned vector.
// Values at k1 + q >= nh lie in the row's padding: stored freely, and loaded as zero
// with MASK.  Buffers whose padding is known to be zero (the layer spectra, and the
// workspace rows read by cols_fwd) skip the mask, whose select would otherwise make
// the load complete at the point of issue.
template <int V, bool MASK, typename C>
__device__ __forceinline__ void ld_row_vec(const C* p, int k1, int nh, bool ok, C* o) {
  if (ok) {
    Vec<V, C>::ld(p, o);
    if constexpr (MASK) {
#pragma unroll
      for (int q = 1; q < V; ++q)
        if (k1 + q >= nh) o[q] = zero<C>();
    }
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) o[q] = zero<C>();
  }
}

// Loads of the layer spectra, which every column of a block reads again, with an L2
// evict-last policy (pol) in single precision; the row-transformed tiles that stream
// through once are copied with evict-first.
#ifndef TF_L2_HINTS
#define TF_L2_HINTS 1
#endif
template <int V, typename C>
__device__ __forceinline__ void ld_spec_vec(const C* p, int k1, int nh, bool ok, C* o, uint64_t pol) {
  if constexpr (TF_L2_HINTS && V == 2 && std::is_same<C, float2>::value) {
    if (ok) {
      const float4 t = bulk::ld_hint(p, pol);
      o[0] = make_float2(t.x, t.y);
      o[1] = make_float2(t.z, t.w);
    } else {
      o[0] = o[1] = zero<C>();
    }
  } else {
    ld_row_vec<V, false>(p, k1, nh, ok, o);
  }
}
template <typename C> __device__ __forceinline__ uint64_t spec_policy() {
  if constexpr (TF_L2_HINTS && std::is_same<C, float2>::value) return bulk::policy_evict_last();
  else return 0;
}

// Register budgets of the column kernels, as a minimum number of resident CTAs per SM
// for __launch_bounds__ (measured with 1260-column blocks at transform lengths 64 to
// 512: the single-precision forward kernel is fastest near 128 registers a thread, the
// adjoint near 100, and near 85 at n >= 448; the double kernels are indifferent).  At
// c4 (2510-column blocks) the tighter budgets spill and lose: cols_fwd at 768 threads
// per SM 16.1 -> 18.6 ms per step, cols_adj at 1024 14.6 -> 17.3 ms.
template <typename T> constexpr int cols_min_blocks(int nt, int threads_per_sm) {
  return std::is_same<T, float>::value && threads_per_sm / nt > 1 ? threads_per_sm / nt : 1;
}
template <typename T> constexpr int kFwdThreadsPerSM = 512;
// two-pass plans (first radix 16, 64-thread CTAs): about 170 registers (measured against
// 320, 448 and 512 resident threads per SM)
constexpr int kWideThreadsPerSM = 384;
// the adjoint at n >= 448 (256 threads per CTA) measured fastest with a tighter budget
#ifndef TF_ADJ_TPSM
#define TF_ADJ_TPSM 768
#endif
template <typename T, int N> constexpr int kAdjThreadsPerSM = N >= 448 ? TF_ADJ_TPSM : 640;
// Buffer positions from per-task bases (Buf's STEP): c4 cols_fwd 14.99 -> 13.71 ms per
// 2510-column step.  The adjoint with single-buffer passes measured slower with them
// (14.56 -> 16.3 ms at its 80-register budget, 16.0 ms at 128 registers).
// With the data spectrum in TMEM and two-buffer passes, the adjoint's single-precision
// 256-thread plans take per-task bases after all (c4: cols_adj 12.57 -> 12.41 ms at 80
// registers).
#ifndef TF_ADJ_STEP
#define TF_ADJ_STEP 3
#endif
template <typename T, int NT> constexpr int kAdjStepOf = std::is_same<T, float>::value && NT == 256 ? TF_ADJ_STEP : 0;
// The row kernels keep per-element positions too (with bases: rows_r2c 7.96 -> 8.8 ms, and
// at a 48-register budget 8.9 ms; rows_c2r 8.41 -> 8.62 ms).
constexpr int kRowsStep = 0;

// Visits every (element index n < E, pair group q < TP) once.  When E fills at least 4/5
// of the CTA's threads, each thread takes whole element indices and loops over the pair
// groups (the swizzled row position and the element's own index arithmetic are shared by
// the TP accesses); otherwise a flat walk over all pairs keeps the threads busy.
template <int NT, int TP, class Body>
__device__ __forceinline__ void visit_pairs(int E, const Body& body) {
  const int full = (E + NT - 1) / NT * NT;
  if (5 * E >= 4 * full) {
    for (int n = threadIdx.x; n < E; n += NT)
#pragma unroll
      for (int q = 0; q < TP; ++q) body(n, q);
  } else {
    for (int u = threadIdx.x; u < TP * E; u += NT) {
      const int q = u / E;
      body(u - q * E, q);
    }
  }
}

// The row kernels stage and unpack two adjacent sequences (2q, 2q + 1) per thread and
// element: one 16-byte shared-memory access (the pair is adjacent in the swizzled
// buffer), and the four real rows 2 (pair0 + 2q) + 0..3 that feed them.  The loops
// over (element, pair group) go through visit_pairs.
// ZHI: the rows' data lies in [0, N/2) of the sequence, so staging fills only that half
// and the first pass takes the upper half as zero.
// Register budgets of the single-precision row kernels at n > 256 (256-thread CTAs), as
// resident threads per SM for __launch_bounds__: 1536 for rows_r2c (40 registers) and 1280
// for rows_c2r (48).  Measured on 2510-column c4 blocks against the compiler's default
// budget (55 registers, 1024 threads): rows_r2c 10.7 -> 7.9 ms and rows_c2r 10.9 -> 8.4 ms
// per step; the two kernels wait on memory, and more resident CTAs overlap those waits.
template <typename T> constexpr int rows_min_blocks(int nt, int threads_per_sm) {
  return std::is_same<T, float>::value && nt == 256 ? threads_per_sm / nt : 1;
}

template <typename T, class P, int TB, int V, int NT, bool ZHI>
__global__ void __launch_bounds__(NT, rows_min_blocks<T>(NT, 1536)) k_rows_r2c(const RowsR2C<T> a) {
  typedef typename CT<T>::C C;
  constexpr int N = P::n, NH = N / 2 + 1, TP = TB / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + twpad(N - 1);
  for (int i = threadIdx.x; i < N - 1; i += NT) tw[i] = a.tw[i];
  const int pair0 = blockIdx.x * TB;
  const T* src = a.src + (int64_t)blockIdx.y * a.src_ld;
  const int len = a.row_len, off = a.seq_off, nrows = a.nrows;
  const int src_ext = nrows * len;
  const T* scale = a.scale;
  constexpr int NS = ZHI && P::can_zero_hi ? N / 2 : N;   // staged rows of the buffer
  visit_pairs<NT, TP>(NS, [&](int n, int q) {
    const ct::RowAt<C, TB, P::first_r> ra(n);
    const int e = n - off;
    const int r0 = 2 * (pair0 + 2 * q);
    T x[4] = {T(0), T(0), T(0), T(0)};
    if (e >= 0 && e < len) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (r0 + i >= nrows) break;
        const int o = (r0 + i) * len + e;
        if (TF_IN(kSiteR2cSrc, o, src_ext)) x[i] = src[o];
        if (scale && TF_IN(kSiteR2cScale, o, src_ext)) x[i] *= scale[o];
      }
    }
    const C v[2] = {mk<C>(x[0], x[1]), mk<C>(x[2], x[3])};
    const int p = ra(2 * q);
    if (TF_IN(kSiteSmem + 3, p + 1, N * TB)) Vec<2, C>::st(buf + p, v);
  });
  __syncthreads();
  const ct::Buf<C, TB, V, P::first_r, kRowsStep> b{buf, N * TB};
  P::template run<TB, V, NT, false, ZHI, kRowsStep>(tw, buf, b, b);
  C* dst = a.dst + (int64_t)blockIdx.y * a.dst_ld;
  const int hs = a.hs, dst_ext = nrows * hs;
  visit_pairs<NT, TP>(NH, [&](int k, int q) {
    const int r0 = 2 * (pair0 + 2 * q);
    if (r0 >= nrows) return;
    const ct::RowAt<C, TB, P::first_r> rk(k), rc(k ? N - k : 0);
    C z[2], zc[2];
    const int pk = rk(2 * q), pc = rc(2 * q);
    if (TF_IN(kSiteSmem + 3, pk + 1, N * TB)) Vec<2, C>::ld(buf + pk, z);
    if (TF_IN(kSiteSmem + 3, pc + 1, N * TB)) Vec<2, C>::ld(buf + pc, zc);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ra = r0 + 2 * h, rb = ra + 1;
      if (ra >= nrows) break;
      zc[h].y = -zc[h].y;
      if (TF_IN(kSiteR2cDst, ra * hs + k, dst_ext))
        dst[ra * hs + k] = mk<C>(T(0.5) * (z[h].x + zc[h].x), T(0.5) * (z[h].y + zc[h].y));
      if (rb < nrows && TF_IN(kSiteR2cDst, rb * hs + k, dst_ext))
        dst[rb * hs + k] = mk<C>(T(0.5) * (z[h].y - zc[h].y), T(-0.5) * (z[h].x - zc[h].x));
    }
  });
}

template <typename T, class P, int TB, int V, int NT>
__global__ void __launch_bounds__(NT, rows_min_blocks<T>(NT, 1280)) k_rows_c2r(const RowsC2R<T> a) {
  typedef typename CT<T>::C C;
  constexpr int N = P::n, NH = N / 2 + 1, TP = TB / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + twpad(N - 1);
  for (int i = threadIdx.x; i < N - 1; i += NT) tw[i] = a.tw[i];
  const int pair0 = blockIdx.x * TB;
  const int nrows = a.nrows;
  const C* src = a.src + (int64_t)blockIdx.y * a.src_ld;
  const int hs = a.hs, src_ext = nrows * hs;
  visit_pairs<NT, TP>(NH, [&](int k, int q) {
    const bool self = (k == 0) || (2 * k == N);
    const int r0 = 2 * (pair0 + 2 * q);
    C x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[i] = zero<C>();
      if (r0 + i < nrows && TF_IN(kSiteC2rSrc, (r0 + i) * hs + k, src_ext)) x[i] = src[(r0 + i) * hs + k];
    }
    C lo[2], hi[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      C xa = x[2 * h], xb = x[2 * h + 1];
      if (self) { xa.y = T(0); xb.y = T(0); }
      lo[h] = mk<C>(xa.x - xb.y, xa.y + xb.x);
      hi[h] = mk<C>(xa.x + xb.y, xb.x - xa.y);
    }
    const int pk = ct::RowAt<C, TB, P::first_r>(k)(2 * q);
    if (TF_IN(kSiteSmem + 3, pk + 1, N * TB)) Vec<2, C>::st(buf + pk, lo);
    if (!self) {
      const int pc = ct::RowAt<C, TB, P::first_r>(N - k)(2 * q);
      if (TF_IN(kSiteSmem + 3, pc + 1, N * TB)) Vec<2, C>::st(buf + pc, hi);
    }
  });
  __syncthreads();
  const ct::Buf<C, TB, V, P::first_r, kRowsStep> b{buf, N * TB};
  P::template run<TB, V, NT, true, false, kRowsStep>(tw, buf, b, b);
  T* dst = a.dst + (int64_t)blockIdx.y * a.dst_ld;
  const int L = a.out_len, off = a.seq_off;
  const int dst_ext = nrows * L;
  const T* scale = a.scale;
  visit_pairs<NT, TP>(L, [&](int i, int q) {
    const int r0 = 2 * (pair0 + 2 * q);
    if (r0 >= nrows) return;
    C z[2];
    const int p = ct::RowAt<C, TB, P::first_r>(off + i)(2 * q);
    if (TF_IN(kSiteSmem + 3, p + 1, N * TB)) Vec<2, C>::ld(buf + p, z);
    const T y[4] = {z[0].x, z[0].y, z[1].x, z[1].y};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (r0 + j >= nrows) break;
      const int o = (r0 + j) * L + i;
      if (TF_IN(kSiteC2rDst, o, dst_ext))
        dst[o] = (scale && TF_IN(kSiteC2rScale, o, dst_ext)) ? y[j] * scale[o] : y[j];
    }
  });
}

// Persistent row kernels with bulk copies (single precision).  A tile is 2 TB consecutive
// real rows (TB two-row sequences, PipeTiles), so its input is one contiguous block and so
// is its output.  Each CTA walks the tiles of all columns (stride gridDim.x).  One thread
// moves a tile's input into shared memory with bulk copies, issued right after the previous
// tile's first FFT pass has read its input, so it lands while the CTA transforms; the first
// pass reads the copied rows directly, and the output goes to a shared-memory tile in the
// global layout that leaves with one bulk store, which completes while the CTA works on the
// next tile.  DRAM latency is hidden by the copies in flight instead of by resident warps,
// so the kernels run few CTAs per SM (PipeTiles::PER_SM) with the registers that allows.
// The output tile of rows_r2c includes each row's padding [nh, hs), zeroed once, so the
// workspace's padding stays zero.  Every wait on the input barrier is bounded: past
// kPipeWaitNs the CTA records TF_ETIMEOUT in the status word and returns.
constexpr unsigned long long kPipeWaitNs = 2000000000ull;
static __device__ unsigned int g_pipe_status;   // TF_ETIMEOUT after a wait ran out
constexpr int kPipeStatusTimeout = 6;   // TF_ETIMEOUT
struct RowsPipe {
  int tiles_per_col, ncols;
  unsigned int* status;
};
// Buffer positions of the passes from per-task bases (Buf's STEP) in rows_c2r_pipe
// (measured c4: 7.97 -> 7.71 ms per step) but not in rows_r2c_pipe (7.05 -> 7.09 ms).
#ifndef TF_R2C_PIPE_STEP
#define TF_R2C_PIPE_STEP 0
#endif
#ifndef TF_C2R_PIPE_STEP
#define TF_C2R_PIPE_STEP 3
#endif

template <typename T, class P, int TB, int V, int NT, bool ZHI>
__global__ void __launch_bounds__(NT, 512 / NT) k_rows_r2c_pipe(const RowsR2C<T> a, const RowsPipe pp) {
  typedef typename CT<T>::C C;
  constexpr int N = P::n, NH = N / 2 + 1, TP = TB / 2, RT = 2 * TB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const int len = a.row_len, hs = a.hs, nrows = a.nrows, off = a.seq_off, tpc = pp.tiles_per_col;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + twpad(N - 1);
  C* out = buf + N * TB;                          // [RT][hs], the global layout
  T* in = reinterpret_cast<T*>(out + RT * hs);    // [RT][len]
  const int64_t ntiles = (int64_t)tpc * pp.ncols;
  auto issue = [&](int64_t t) {
    const int col = (int)(t / tpc), tile = (int)(t - (int64_t)col * tpc);
    const int rows = min(RT, nrows - tile * RT);
    const uint32_t bytes = (uint32_t)(rows * len * sizeof(T));
    bulk::mbar_expect_tx(&bar, bytes);
    bulk::load(in, a.src + (int64_t)col * a.src_ld + (int64_t)tile * RT * len, bytes, &bar);
  };
  if (threadIdx.x == 0) {
    bulk::mbar_init(&bar, 1);
    bulk::fence_mbar_init();
  }
  for (int i = threadIdx.x; i < N - 1; i += NT) tw[i] = a.tw[i];
  for (int i = threadIdx.x; i < RT * (hs - NH); i += NT) out[(i / (hs - NH)) * hs + NH + i % (hs - NH)] = zero<C>();
  __syncthreads();
  if (threadIdx.x == 0 && (int64_t)blockIdx.x < ntiles) issue(blockIdx.x);
  uint32_t phase = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const bool ok = bulk::mbar_wait_bounded(&bar, phase, kPipeWaitNs);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(pp.status, (unsigned)kPipeStatusTimeout);
        bulk::wait_all();
      }
      return;
    }
    const int col = (int)(t / tpc), tile = (int)(t - (int64_t)col * tpc);
    const int rows = min(RT, nrows - tile * RT);
    const T* scale = a.scale ? a.scale + (int64_t)tile * RT * len : nullptr;
    // the first pass reads the rows where the copy left them: sequence b holds rows 2b
    // (real part) and 2b + 1 (imaginary part)
    auto ld_in = [=](int idx, int b0, C* o) {
      const int e = idx - off;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int ra = 2 * (b0 + q);
        T x0 = T(0), x1 = T(0);
        if (e >= 0 && e < len) {
          if (ra < rows) x0 = in[ra * len + e];
          if (ra + 1 < rows) x1 = in[(ra + 1) * len + e];
          if (scale) {
            x0 *= scale[ra * len + e];
            x1 *= ra + 1 < rows ? scale[(ra + 1) * len + e] : T(0);
          }
        }
        o[q] = mk<C>(x0, x1);
      }
    };
    // after the first pass: the next tile's input may overwrite `in`, and the previous
    // tile's output must have left `out` before the unpacking below
    auto hook = [&]() {
      if (threadIdx.x == 0) {
        if (t + gridDim.x < ntiles) {
          bulk::fence_proxy_async();
          issue(t + gridDim.x);
        }
        bulk::wait_read_all();
      }
    };
    const ct::Buf<C, TB, V, P::first_r, TF_R2C_PIPE_STEP> b{buf, N * TB};
    P::template run_h<TB, V, NT, false, ZHI, TF_R2C_PIPE_STEP>(tw, buf, ld_in, b, hook);
    visit_pairs<NT, TP>(NH, [&](int k, int q) {
      const int r0 = 4 * q;
      if (r0 >= rows) return;
      const ct::RowAt<C, TB, P::first_r> rk(k), rc(k ? N - k : 0);
      C z[2], zc[2];
      const int pk = rk(2 * q), pc = rc(2 * q);
      if (TF_IN(kSiteSmem + 3, pk + 1, N * TB)) Vec<2, C>::ld(buf + pk, z);
      if (TF_IN(kSiteSmem + 3, pc + 1, N * TB)) Vec<2, C>::ld(buf + pc, zc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ra = r0 + 2 * h, rb = ra + 1;
        if (ra >= rows) break;
        zc[h].y = -zc[h].y;
        out[ra * hs + k] = mk<C>(T(0.5) * (z[h].x + zc[h].x), T(0.5) * (z[h].y + zc[h].y));
        if (rb < rows) out[rb * hs + k] = mk<C>(T(0.5) * (z[h].y - zc[h].y), T(-0.5) * (z[h].x - zc[h].x));
      }
    });
    bulk::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk::store(a.dst + (int64_t)col * a.dst_ld + (int64_t)tile * RT * hs, out, (uint32_t)(rows * hs * sizeof(C)));
      bulk::commit();
    }
  }
  if (threadIdx.x == 0) bulk::wait_all();
}

// Rows of the c2r input tile (RT rows) sit at row * hs + (64 / RT) (row / 4) values: the
// first pass's loads of rows 0, 4, ... (one per sequence pair of a half-warp) then fall in
// different banks.
template <int RT> __host__ __device__ constexpr int c2r_in_row(int r, int hs) { return r * hs + (64 / RT) * (r >> 2); }

template <typename T, class P, int TB, int V, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_rows_c2r_pipe(const RowsC2R<T> a, const RowsPipe pp) {
  typedef typename CT<T>::C C;
  constexpr int N = P::n, RT = 2 * TB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const int hs = a.hs, nrows = a.nrows, L = a.out_len, off = a.seq_off, tpc = pp.tiles_per_col;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + twpad(N - 1);
  C* in = buf + N * TB;                                   // rows at c2r_in_row
  T* out = reinterpret_cast<T*>(in + c2r_in_row<RT>(RT, hs));  // [RT][L], the global layout
  const int64_t ntiles = (int64_t)tpc * pp.ncols;
  auto issue = [&](int64_t t) {
    const int col = (int)(t / tpc), tile = (int)(t - (int64_t)col * tpc);
    const int rows = min(RT, nrows - tile * RT);
    const C* src = a.src + (int64_t)col * a.src_ld + (int64_t)tile * RT * hs;
    bulk::mbar_expect_tx(&bar, (uint32_t)(rows * hs * sizeof(C)));
    for (int r = 0; r < rows; ++r)
      bulk::load(in + c2r_in_row<RT>(r, hs), src + (int64_t)r * hs, (uint32_t)(hs * sizeof(C)), &bar);
  };
  if (threadIdx.x == 0) {
    bulk::mbar_init(&bar, 1);
    bulk::fence_mbar_init();
  }
  for (int i = threadIdx.x; i < N - 1; i += NT) tw[i] = a.tw[i];
  __syncthreads();
  if (threadIdx.x == 0 && (int64_t)blockIdx.x < ntiles) issue(blockIdx.x);
  uint32_t phase = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const bool ok = bulk::mbar_wait_bounded(&bar, phase, kPipeWaitNs);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(pp.status, (unsigned)kPipeStatusTimeout);
        bulk::wait_all();
      }
      return;
    }
    const int col = (int)(t / tpc), tile = (int)(t - (int64_t)col * tpc);
    const int rows = min(RT, nrows - tile * RT);
    // first pass: element idx of sequence b = Xa[idx] + i Xb[idx], the Hermitian extensions
    // of the half spectra of rows 2b and 2b + 1 (X[N - k] = conj X[k]; the imaginary parts
    // at k = 0 and N/2 dropped)
    auto ld_in = [=](int idx, int b0, C* o) {
      const bool up = 2 * idx > N;
      const int k = up ? N - idx : idx;
      const bool self = (k == 0) || (2 * k == N);
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int ra = 2 * (b0 + q);
        C xa = ra < rows ? in[c2r_in_row<RT>(ra, hs) + k] : zero<C>();
        C xb = ra + 1 < rows ? in[c2r_in_row<RT>(ra + 1, hs) + k] : zero<C>();
        if (self) { xa.y = T(0); xb.y = T(0); }
        o[q] = up ? mk<C>(xa.x + xb.y, xb.x - xa.y) : mk<C>(xa.x - xb.y, xa.y + xb.x);
      }
    };
    const T* scale = a.scale ? a.scale + (int64_t)tile * RT * L : nullptr;
    // last pass: the window [off, off + L) of each sequence's real and imaginary parts
    // straight into the output tile
    auto st_out = [=](int idx, int b0, const C* v, int) {
      const int i = idx - off;
      if (i < 0 || i >= L) return;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int ra = 2 * (b0 + q);
        if (ra < rows) out[ra * L + i] = scale ? v[q].x * scale[ra * L + i] : v[q].x;
        if (ra + 1 < rows) out[(ra + 1) * L + i] = scale ? v[q].y * scale[(ra + 1) * L + i] : v[q].y;
      }
    };
    auto hook = [&]() {
      if (threadIdx.x == 0) {
        if (t + gridDim.x < ntiles) {
          bulk::fence_proxy_async();
          issue(t + gridDim.x);
        }
        bulk::wait_read_all();   // the previous tile's output has left `out`
      }
    };
    P::template run_h<TB, V, NT, true, false, TF_C2R_PIPE_STEP>(tw, buf, ld_in, st_out, hook);
    bulk::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk::store(a.dst + (int64_t)col * a.dst_ld + (int64_t)tile * RT * L, out, (uint32_t)(rows * L * sizeof(T)));
      bulk::commit();
    }
  }
  if (threadIdx.x == 0) bulk::wait_all();
}

// Spectrum values are staged in registers ahead of use in single precision only (the
// double kernels measured no gain from it).
template <typename T> constexpr bool kSpecPrefetch = std::is_same<T, float>::value;

// The forward column kernel keeps its layer accumulators in tensor memory (tf_tmem.cuh)
// in single precision with 256-thread CTAs, and then transforms MC = 2 model columns per
// CTA: each layer's spectrum values, loaded into registers once, multiply both columns'
// transforms, so the CTA reads them from L2 half as often.  TMEM: 128 columns per CTA, 64
// per half of the CTA's warps, 32 per model column, 4 per slot (two complex values), one
// slot per output of the thread's last-pass tasks.  Those tasks fill every thread, so each
// TMEM access is warp-uniform.  The launch asks for at least kTmemSmemFloor bytes of shared
// memory, which caps residency at 4 CTAs per SM (228 KB, 1 KB reserved per CTA), so 4 x 128
// TMEM columns fit the SM's 512 and no allocation waits.
// Measured (c4, 2510-column steps): the accumulator in TMEM instead of shared memory
// 16.08 -> 15.45 ms per step.  (The adjoint's data spectrum, read once per layer, measured
// slower from TMEM: 14.6 -> 15.1 ms at the adjoint's 80-register budget, which the TMEM
// loads push into spills.)
#ifndef TF_COLS_TMEM
#define TF_COLS_TMEM 1
#endif
#ifndef TF_FWD_MC
#define TF_FWD_MC 2
#endif
#ifndef TF_FWD_PP
#define TF_FWD_PP 1   // measured: c4 cols_fwd 13.72 -> 12.66 ms per step with the two buffers
#endif
// Values between consecutive model columns' layer tiles ([ny][TB] each) in cols_fwd's
// shared memory: the tile rounded up to 128 bytes, the alignment of a tensor copy's
// shared-memory destination.
template <typename C, int TB> __host__ __device__ constexpr int fwd_tile_stride(int ny) {
  return (int)(((size_t)ny * TB * sizeof(C) + 127) / 128 * 128 / sizeof(C));
}
template <typename T, class P, int TB, int V, int NT> struct FwdTmem {
  typedef ct::PassMap<P::last_r, P::last_ns, P::n, TB, V> LM;
  static constexpr int ITA = (LM::TOTAL + NT - 1) / NT;
  static constexpr int kColWords = 32;                       // TMEM columns per model column
  static constexpr bool on = TF_COLS_TMEM && std::is_same<T, float>::value && NT == 256 && V == 2 &&
                             LM::TOTAL % NT == 0 && ITA * P::last_r * 4 <= kColWords;
  static constexpr int MC = on ? TF_FWD_MC : 1;              // model columns per CTA
  static constexpr bool pp = on && TF_FWD_PP;                // passes alternate two buffers
  static constexpr int nbuf = on && !pp ? 1 : 2;             // shared-memory buffers of N x TB
  static constexpr int kCols = 2 * MC * kColWords;           // allocation (both halves)
};
constexpr size_t kTmemSmemFloor = 47104;   // > 228 KB / 5 - 1 KB: at most 4 resident CTAs
// Column stage of G x (ZHI: ny <= N/2, the layer rows fill the lower half).  In single
// precision each thread loads the spectrum values that its last forward pass multiplies
// at the start of every layer, into registers, so that their global-memory latency
// overlaps the layer's first passes.
template <typename T, class P, int TB, int V, int NT, bool ZHI, bool TILE>
__global__ void __launch_bounds__(NT, cols_min_blocks<T>(NT, P::first_r >= 16 ? kWideThreadsPerSM : kFwdThreadsPerSM<T>)) k_cols_fwd(const ColsFwd<T> a, const __grid_constant__ CUtensorMap zmap) {
  typedef typename CT<T>::C C;
  typedef FwdTmem<T, P, TB, V, NT> FT;
  constexpr int N = P::n;
  constexpr bool kPre = kSpecPrefetch<T>;
  constexpr int RL = P::last_r, NSL = P::last_ns;
  typedef ct::PassMap<RL, NSL, N, TB, V> LM;
  constexpr int ITL = kPre ? (LM::TOTAL + NT - 1) / NT : 0;
  // accumulator slots of the last pass (it * RL + rr) in TMEM, or [N][TB] in shared memory
  constexpr int ITA = FT::ITA;
  constexpr bool kTm = FT::on;
  static_assert(!kTm || (kPre && V == 2), "TMEM accumulators: register-staged spectrum, pairs");
  constexpr int MC = FT::MC;
  // with the accumulators in TMEM, the second buffer pairs with the first so that
  // consecutive passes alternate between them (Plan::run2: no barrier inside a pass)
  constexpr bool kPP = FT::pp;
  static_assert(!kPP || FT::nbuf == 2, "ping-pong needs the second buffer");
  // TILE: each layer's row-transformed tile of a model column ([ny][TB]) arrives in shared
  // memory by one tensor copy (zmap: the workspace as rows of 2 hs floats, box TB x ny),
  // issued right after the column's previous layer, and the first pass reads it there
  constexpr bool kTile = TILE && kTm;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t tm_base;
  __shared__ __align__(8) uint64_t zbar[MC];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + twpad(N - 1);
  C* acc = buf + N * TB;
  // [MC][ny][TB] with TILE, 128-byte aligned (the launch adds 128 bytes)
  C* ztile = reinterpret_cast<C*>((reinterpret_cast<uintptr_t>(acc + N * TB) + 127) & ~(uintptr_t)127);
  // a tensor copy writes shared memory at 128-byte boundaries: each column's tile starts on one
  const int zstride = fwd_tile_stride<C, TB>(a.ny);
  if constexpr (kTm)
    if (threadIdx.x < 32) tmem::alloc(&tm_base, FT::kCols);
  if constexpr (kTile)
    if (threadIdx.x == 0) {
#pragma unroll
      for (int c = 0; c < MC; ++c) bulk::mbar_init(&zbar[c], 1);
      bulk::fence_mbar_init();
    }
  for (int i = threadIdx.x; i < N - 1; i += NT) tw[i] = a.tw[i];
  if constexpr (kTm) tmem::fence_before_sync();
  __syncthreads();
  uint32_t tacc = 0;
  if constexpr (kTm) {
    tmem::fence_after_sync();
    tacc = tmem::lane_addr(tm_base, (threadIdx.x >> 7) * (FT::kCols / 2));
    // zero accumulators: every layer, the first included, is then one multiply-add
    const float z4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < MC; ++c)
#pragma unroll
      for (int sl = 0; sl < ITA * RL; ++sl) tmem::st4(tacc + c * FT::kColWords + sl * 4, z4);
    tmem::wait_st();
  }
  const int k0 = blockIdx.x * TB;
  const int nh = a.nh, hs = a.hs, ny = a.ny, sy = a.sy;
  const int col0 = blockIdx.y * MC;
  const int mc = MC > 1 && a.ncols - col0 < MC ? a.ncols - col0 : MC;   // the CTA's columns
  const int z_ext = a.nz * ny * hs, g_ext = a.nz * N * hs, s_ext = sy * hs;
  const C* spec = a.spec;
  const int zrows = (int)(a.z_ld / hs);   // workspace rows per model column
  const uint64_t spol = spec_policy<C>();
  const uint64_t zpol = TF_L2_HINTS && kTile ? bulk::policy_evict_first() : 0;
  auto issue = [&](int c, int r) {
    if (threadIdx.x == 0) {
      bulk::fence_proxy_async();
      bulk::mbar_expect_tx(&zbar[c], (uint32_t)(ny * TB * sizeof(C)));
      if constexpr (TF_L2_HINTS)
        bulk::load_tile_2d_hint(ztile + c * zstride, &zmap, 2 * k0, (col0 + c) * zrows + r * ny, &zbar[c], zpol);
      else
        bulk::load_tile_2d(ztile + c * zstride, &zmap, 2 * k0, (col0 + c) * zrows + r * ny, &zbar[c]);
    }
  };
  if constexpr (kTile)
    for (int c = 0; c < mc; ++c) issue(c, 0);
  C gpre[kPre ? ITL * RL : 1][V];
  for (int r = 0; r < a.nz; ++r) {
    const int zoff = r * ny * hs, goff = r * N * hs;
#pragma unroll
    for (int it = 0; it < ITL; ++it) {
      const int u = threadIdx.x + it * NT;
      int b0 = 0;
      const int base = LM::first_idx(u < LM::TOTAL ? u : 0, b0);
      const int k1 = k0 + b0;
#pragma unroll
      for (int rr = 0; rr < RL; ++rr) {
        const int e = goff + (base + rr * NSL) * hs + k1;
        ld_spec_vec<V>(spec + e, k1, nh, u < LM::TOTAL && k1 < nh && TF_IN(kSiteFwdSpec, e + V - 1, g_ext),
                       gpre[it * RL + rr], spol);
      }
    }
    const bool first_layer = (r == 0);
    for (int c = 0; c < MC; ++c) {
      if (c >= mc) break;
      const C* z = a.z + (int64_t)(col0 + c) * a.z_ld;
      const uint32_t tcol = tacc + c * FT::kColWords;
      // Row-transformed layers as aligned vectors without a padding mask: the workspace is
      // zeroed when allocated, the row kernels never write its padding, and the column
      // kernels write zeros there (their padded sequences have zero inputs).  A masked load
      // measured much slower here (the mask's select waits for the load).
      if constexpr (kTile) {
        const bool ok = bulk::mbar_wait_bounded(&zbar[c], r & 1, kPipeWaitNs);
        if (__syncthreads_or(!ok)) {   // a copy never completed: report, free TMEM, return
          tmem::fence_before_sync();
          __syncthreads();
          if (threadIdx.x < 32) {
            tmem::fence_after_sync();
            tmem::dealloc(tm_base, FT::kCols);
          }
          if (threadIdx.x == 0) atomicExch(&g_pipe_status, (unsigned)kPipeStatusTimeout);
          return;
        }
      }
      const C* zt = ztile + c * zstride;
      auto load = [=](int idx, int b0, C* o) {
        if constexpr (kTile) {
          if (idx < ny && TF_IN(kSiteSmem + 4, idx * TB + b0 + V - 1, ny * TB)) {
            Vec<V, C>::ld(zt + idx * TB + b0, o);
          } else {
#pragma unroll
            for (int q = 0; q < V; ++q) o[q] = zero<C>();
          }
        } else {
          const int k1 = k0 + b0;
          const int e = zoff + idx * hs + k1;
          ld_row_vec<V, false>(z + e, k1, nh, idx < ny && k1 < nh && TF_IN(kSiteFwdZ, e + V - 1, z_ext), o);
        }
      };
      auto mac = [&](int idx, int b0, const C* v, int slot) {
        if constexpr (kTm) {
          // acc += g v as four fused multiply-adds per complex value (accumulators zeroed)
          float f[4];
          tmem::ld4(tcol + slot * 4, f);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const C g = gpre[slot][q];
            f[2 * q] = fmaf(g.x, v[q].x, f[2 * q]);
            f[2 * q] = fmaf(-g.y, v[q].y, f[2 * q]);
            f[2 * q + 1] = fmaf(g.x, v[q].y, f[2 * q + 1]);
            f[2 * q + 1] = fmaf(g.y, v[q].x, f[2 * q + 1]);
          }
          tmem::st4(tcol + slot * 4, f);
        } else {
          C cur[V];
          const bool acc_ok = TF_IN(kSiteSmem + 2, idx * TB + b0 + V - 1, N * TB);
          if (!first_layer && acc_ok) Vec<V, C>::ld(acc + idx * TB + b0, cur);
          C gv[V];
          if constexpr (!kPre) {
            const int k1 = k0 + b0;
            const int e = goff + idx * hs + k1;
            ld_row_vec<V, false>(spec + e, k1, nh, k1 < nh && TF_IN(kSiteFwdSpec, e + V - 1, g_ext), gv);
          }
#pragma unroll
          for (int q = 0; q < V; ++q) {
            const C g = kPre ? gpre[slot][q] : gv[q];
            const C p = cmul(g, v[q]);
            cur[q] = first_layer ? p : cadd(cur[q], p);
          }
          if (acc_ok) Vec<V, C>::st(acc + idx * TB + b0, cur);
        }
      };
      if constexpr (kPP) P::template run2<TB, V, NT, false, ZHI, 3>(tw, buf, acc, load, mac);
      else P::template run<TB, V, NT, false, ZHI, 3>(tw, buf, load, mac);
      if constexpr (kTm) tmem::wait_st();
      if constexpr (kTile)
        if (r + 1 < a.nz) issue(c, r + 1);   // the passes ended at a barrier: the tile is free
    }
  }
  for (int c = 0; c < MC; ++c) {
    if (c >= mc) break;
    C* s = a.s + (int64_t)(col0 + c) * a.s_ld;
    auto lacc = [=](int idx, int b0, C* o) {
      if (TF_IN(kSiteSmem + 2, idx * TB + b0 + V - 1, N * TB)) Vec<V, C>::ld(acc + idx * TB + b0, o);
    };
    auto store = [=](int idx, int b0, const C* v, int) {
      const int j = idx - (ny - 1), k1 = k0 + b0;
      if (j < 0 || j >= sy || k1 >= nh) return;
      if (TF_IN(kSiteFwdS, j * hs + k1 + V - 1, s_ext)) Vec<V, C>::st(s + j * hs + k1, v);
    };
    if constexpr (kTm) {
      // the accumulator from TMEM into the working buffer, in the inverse's input order
      const uint32_t tcol = tacc + c * FT::kColWords;
#pragma unroll
      for (int it = 0; it < ITA; ++it) {
        int b0;
        const int base = LM::first_idx(threadIdx.x + it * NT, b0);
#pragma unroll
        for (int rr = 0; rr < RL; ++rr) {
          float f[4];
          tmem::ld4(tcol + (it * RL + rr) * 4, f);
          const C v[2] = {mk<C>(f[0], f[1]), mk<C>(f[2], f[3])};
          const int e = ct::at<C, TB, P::first_r>(base + rr * NSL, b0);
          if (TF_IN(kSiteSmem + 2, e + V - 1, N * TB)) Vec<V, C>::st((kPP ? acc : buf) + e, v);
        }
      }
      tmem::fence_before_sync();
      __syncthreads();
      if (c == mc - 1 && threadIdx.x < 32) {
        tmem::fence_after_sync();
        tmem::dealloc(tm_base, FT::kCols);
      }
      if constexpr (kPP) {
        const ct::Buf<C, TB, V, P::first_r, 3, 1> b{acc, N * TB};
        P::template run2<TB, V, NT, true, false, 3>(tw, buf, acc, b, store);
      } else {
        const ct::Buf<C, TB, V, P::first_r, 3> b{buf, N * TB};
        P::template run<TB, V, NT, true, false, 3>(tw, buf, b, store);
      }
    } else {
      P::template run<TB, V, NT, true, false, 3>(tw, buf, lacc, store);
    }
  }
}

// G^T y with the data spectrum in tensor memory (single precision, 256-thread CTAs): each
// thread keeps the inputs of its first inverse-pass task (8 slots of two complex values,
// 32 TMEM columns per half of the CTA's warps), which frees the second shared buffer for
// passes that alternate between two buffers (Plan::run2).
#ifndef TF_ADJ_TMPP
#define TF_ADJ_TMPP 1
#endif
template <typename T, class P, int TB, int V, int NT> struct AdjTmem {
  static constexpr int R0 = P::first_r, NB0 = P::n / R0, TOTAL0 = NB0 * (TB / V);
  static constexpr bool on = TF_ADJ_TMPP && TF_COLS_TMEM && std::is_same<T, float>::value && NT == 256 &&
                             V == 2 && TOTAL0 % 32 == 0 && TOTAL0 <= NT && R0 == 8;
  static constexpr int kCols = 64;
};

// First inverse pass of G^T y's layer with the data spectrum in TMEM: a task's 8 inputs
// (32 columns) in two 16-column loads, times conj(G_r) loaded from global memory first.
template <typename C, int V> struct AdjSpecTask {
  static constexpr bool kTaskLoad = true;
  uint32_t tspec;
  const C* spec;
  int goff, hs, k0, nh, g_ext;
  uint64_t pol;
  template <int R, int NB> __device__ __forceinline__ void task(int j, int b0, C (&v)[V][R]) const {
    static_assert(V == 2 && R == 8, "32 TMEM columns per task");
    const int k1 = k0 + b0;
    C gv[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = goff + (j + r * NB) * hs + k1;
      ld_spec_vec<V>(spec + e, k1, nh, k1 < nh && TF_IN(kSiteAdjSpec, e + V - 1, g_ext), gv[r], pol);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float f[16];
      tmem::ld16(tspec + 16 * h, f);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[0][4 * h + i] = cmulc(mk<C>(f[4 * i], f[4 * i + 1]), gv[4 * h + i][0]);
        v[1][4 * h + i] = cmulc(mk<C>(f[4 * i + 2], f[4 * i + 3]), gv[4 * h + i][1]);
      }
    }
  }
};

// Column stage of G^T y: forward transform of the data columns into shared memory, then
// per layer the product with conj(G_r) and the inverse transform.
template <typename T, class P, int TB, int V, int NT>
__global__ void __launch_bounds__(NT, cols_min_blocks<T>(NT, P::first_r >= 16 ? kWideThreadsPerSM : kAdjThreadsPerSM<T, P::n>)) k_cols_adj(const ColsAdj<T> a) {
  typedef typename CT<T>::C C;
  typedef AdjTmem<T, P, TB, V, NT> AT;
  constexpr int N = P::n;
  constexpr bool kTm = AT::on;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t tm_base;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + twpad(N - 1);
  C* acc = buf + N * TB;
  if constexpr (kTm)
    if (threadIdx.x < 32) tmem::alloc(&tm_base, AT::kCols);
  for (int i = threadIdx.x; i < N - 1; i += NT) tw[i] = a.tw[i];
  if constexpr (kTm) tmem::fence_before_sync();
  __syncthreads();
  uint32_t tspec = 0;
  if constexpr (kTm) {
    tmem::fence_after_sync();
    tspec = tmem::lane_addr(tm_base, (threadIdx.x >> 7) * (AT::kCols / 2));
  }
  const int k0 = blockIdx.x * TB;
  const int nh = a.nh, hs = a.hs, ny = a.ny, sy = a.sy;
  const C* z = a.z + (int64_t)blockIdx.y * a.z_ld;
  const int z_ext = sy * hs, g_ext = a.nz * N * hs, u_ext = a.nz * ny * hs;
  auto load = [=](int idx, int b0, C* o) {
    const int j = idx - (ny - 1), k1 = k0 + b0;
    ld_row_vec<V, true>(z + j * hs + k1, k1, nh,
                  j >= 0 && j < sy && k1 < nh && TF_IN(kSiteAdjZ, j * hs + k1 + V - 1, z_ext), o);
  };
  // the data spectrum in natural order: into acc, or with TMEM into the buffer that the
  // two-buffer transform's last pass does not read (pass K reads slot (K + 1) mod 2)
  C* const dsp = kTm && (P::npasses - 1) % 2 == 0 ? buf : acc;
  auto sacc = [=](int idx, int b0, const C* v, int) {
    if (TF_IN(kSiteSmem + 2, idx * TB + b0 + V - 1, N * TB)) Vec<V, C>::st(dsp + idx * TB + b0, v);
  };
  if constexpr (kTm) {
    P::template run2<TB, V, NT, false, false, kAdjStepOf<T, NT>>(tw, buf, acc, load, sacc);
    // slot r of a thread: input r of its first-pass task (element j + r NB0 of pair b0)
    if (threadIdx.x < AT::TOTAL0) {
      const int j = threadIdx.x / (TB / V), b0 = (threadIdx.x % (TB / V)) * V;
#pragma unroll
      for (int r = 0; r < AT::R0; ++r) {
        C v[2] = {zero<C>(), zero<C>()};
        const int e = (j + r * AT::NB0) * TB + b0;
        if (TF_IN(kSiteSmem + 2, e + V - 1, N * TB)) Vec<V, C>::ld(dsp + e, v);
        const float f[4] = {v[0].x, v[0].y, v[1].x, v[1].y};
        tmem::st4(tspec + r * 4, f);
      }
    }
    tmem::wait_st();
    __syncthreads();
  } else {
    P::template run<TB, V, NT, false, false, kAdjStepOf<T, NT>>(tw, buf, load, sacc);
  }
  C* u = a.u + (int64_t)blockIdx.y * a.u_ld;
  const C* spec = a.spec;
  const uint64_t spol = spec_policy<C>();
  for (int r = 0; r < a.nz; ++r) {
    const int goff = r * N * hs, uoff = r * ny * hs;
    auto prod = [=](int idx, int b0, C* o) {
      C cur[V], gv[V];
      if (TF_IN(kSiteSmem + 2, idx * TB + b0 + V - 1, N * TB)) Vec<V, C>::ld(acc + idx * TB + b0, cur);
      const int k1 = k0 + b0;
      const int e = goff + idx * hs + k1;
      ld_row_vec<V, false>(spec + e, k1, nh, k1 < nh && TF_IN(kSiteAdjSpec, e + V - 1, g_ext), gv);
#pragma unroll
      for (int q = 0; q < V; ++q) o[q] = cmulc(cur[q], gv[q]);
    };
    auto store = [=](int idx, int b0, const C* v, int) {
      const int k1 = k0 + b0;
      if (idx >= ny || k1 >= nh) return;
      const int e = uoff + idx * hs + k1;
      if (TF_IN(kSiteAdjU, e + V - 1, u_ext)) Vec<V, C>::st(u + e, v);
    };
    if constexpr (kTm) {
      const AdjSpecTask<C, V> pt{tspec, spec, goff, hs, k0, nh, g_ext, spol};
      P::template run2<TB, V, NT, true, false, kAdjStepOf<T, NT>>(tw, buf, acc, pt, store);
    } else {
      P::template run<TB, V, NT, true, false, kAdjStepOf<T, NT>>(tw, buf, prod, store);
    }
  }
  if constexpr (kTm) {
    tmem::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
      tmem::fence_after_sync();
      tmem::dealloc(tm_base, AT::kCols);
    }
  }
}

// Dynamic shared memory above 48 KB needs an opt-in; it is raised only when a launch needs
// more than any earlier launch of the same kernel on the current device (the attribute
// is per device), so steady-state launches (and launches under CUDA-graph capture) make
// no attribute call.
constexpr int kSmemDevices = 64;
template <auto Kernel> inline cudaError_t set_smem(size_t smem) {
  static std::atomic<size_t> granted[kSmemDevices];   // one per kernel and device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kSmemDevices)
    return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  size_t have = granted[dev].load(std::memory_order_relaxed);
  if (smem <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    while (have < smem && !granted[dev].compare_exchange_weak(have, smem)) {}
  return e;
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Tiles: sequences per CTA (TB), sequences per thread (V), threads (NT).
template <typename T, int N> struct Tiles;
// Threads per CTA grow with N so that every pass needs about one butterfly task per
// thread (no second, mostly idle iteration holding registers).
template <int N> struct Tiles<float, N> {
  static constexpr int TB = N <= 96 ? 16 : 8, V = 2;
  static constexpr int NT = N <= 64 ? 64 : (N <= 256 ? 128 : 256);
};
template <int N> struct Tiles<double, N> {
  static constexpr int TB = N <= 96 ? 8 : 4, V = 2, NT = 64;
};

template <auto K, class A>
cudaError_t launch_k(const A& a, dim3 grid, int nt, size_t sm, cudaStream_t s) {
  cudaError_t e = set_smem<K>(sm);
  if (e != cudaSuccess) return e;
  K<<<grid, nt, sm, s>>>(a);
  return cudaGetLastError();
}

// Column kernels' tiles: those of the length, except for plans starting with radix 16
// (two passes), which have half the butterfly tasks per pass: 8 sequences per CTA on 64
// threads (measured against 16 sequences on 128 threads: 2.52 vs 2.75 ms per c2 step).
template <typename T, class P, bool WIDE = (P::first_r >= 16)> struct ColTiles : Tiles<T, P::n> {};
template <typename T, class P> struct ColTiles<T, P, true> {
  static constexpr int TB = 8, V = 2, NT = 64;
};

// The persistent bulk-copy row kernels serve single-precision plans on 256-thread CTAs
// (n > 256) when every tile's input and output block starts on a 16-byte boundary and
// spans a multiple of 16 bytes; other launches take the per-tile kernels above.
#ifndef TF_ROWS_PIPE
#define TF_ROWS_PIPE 1
#endif
template <typename T, class P> constexpr bool kRowsPipe =
    TF_ROWS_PIPE && std::is_same<T, float>::value && Tiles<T, P::n>::NT == 256;

inline bool aligned16(const void* p, int64_t ld_bytes) {
  return ((uintptr_t)p & 15) == 0 && ld_bytes % 16 == 0;
}
// A block of `rows` rows of `row_bytes` each, for full tiles and the tail tile.
inline bool tiles_ok(int nrows, int rt, int64_t row_bytes) {
  const int tail = nrows % rt;
  return (rt * row_bytes) % 16 == 0 && (tail * row_bytes) % 16 == 0;
}
struct PipeDev {
  int sms = 0;
  unsigned int* status = nullptr;
};
inline cudaError_t pipe_dev(PipeDev* out) {
  static PipeDev per[kSmemDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kSmemDevices) return cudaErrorNotSupported;
  if (!per[dev].status) {
    PipeDev d;
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&d.status, g_pipe_status);
    if (e != cudaSuccess) return e;
    per[dev] = d;
  }
  *out = per[dev];
  return cudaSuccess;
}

// Tiles of the bulk-copy row kernels: TB sequences (2 TB rows) per CTA.
#ifndef TF_PIPE_TB
#define TF_PIPE_TB 4
#endif
struct PipeTiles {
  static constexpr int TB = TF_PIPE_TB, V = 2, NT = 32 * TB, PER_SM = 16 / TB;
};
template <typename T, class P>
cudaError_t rows_r2c_pipe(const RowsR2C<T>& a, int ncols, cudaStream_t s, bool* used) {
  typedef PipeTiles TL;
  constexpr int RT = 2 * TL::TB;
  typedef typename CT<T>::C C;
  *used = false;
  if (!aligned16(a.src, a.src_ld * (int64_t)sizeof(T)) || !aligned16(a.dst, a.dst_ld * (int64_t)sizeof(C)) ||
      !tiles_ok(a.nrows, RT, (int64_t)a.row_len * sizeof(T)))
    return cudaSuccess;
  PipeDev d;
  if (pipe_dev(&d) != cudaSuccess) return cudaSuccess;
  const size_t in_bytes = ((size_t)RT * a.row_len * sizeof(T) + 15) & ~(size_t)15;
  const size_t sm = (size_t)(twpad(P::n - 1) + P::n * TL::TB + RT * a.hs) * sizeof(C) + in_bytes;
  RowsPipe pp{(a.nrows + RT - 1) / RT, ncols, d.status};
  const int64_t ntiles = (int64_t)pp.tiles_per_col * ncols;
  const int grid = (int)std::min<int64_t>(ntiles, TL::PER_SM * (int64_t)d.sms);
  if (grid <= 0) return cudaSuccess;
  *used = true;
  const bool zhi = P::can_zero_hi && a.seq_off >= 0 && a.seq_off + a.row_len <= P::n / 2;
  cudaError_t e;
  if (zhi) {
    constexpr auto k = k_rows_r2c_pipe<T, P, TL::TB, TL::V, TL::NT, true>;
    e = set_smem<k>(sm);
    if (e == cudaSuccess) k<<<grid, TL::NT, sm, s>>>(a, pp);
  } else {
    constexpr auto k = k_rows_r2c_pipe<T, P, TL::TB, TL::V, TL::NT, false>;
    e = set_smem<k>(sm);
    if (e == cudaSuccess) k<<<grid, TL::NT, sm, s>>>(a, pp);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}
template <typename T, class P>
cudaError_t rows_c2r_pipe(const RowsC2R<T>& a, int ncols, cudaStream_t s, bool* used) {
  typedef PipeTiles TL;
  constexpr int RT = 2 * TL::TB;
  typedef typename CT<T>::C C;
  *used = false;
  if (!aligned16(a.src, a.src_ld * (int64_t)sizeof(C)) || !aligned16(a.dst, a.dst_ld * (int64_t)sizeof(T)) ||
      !tiles_ok(a.nrows, RT, (int64_t)a.out_len * sizeof(T)))
    return cudaSuccess;
  PipeDev d;
  if (pipe_dev(&d) != cudaSuccess) return cudaSuccess;
  const size_t sm = (size_t)(twpad(P::n - 1) + P::n * TL::TB + c2r_in_row<RT>(RT, a.hs)) * sizeof(C) +
                    (((size_t)RT * a.out_len * sizeof(T) + 15) & ~(size_t)15);
  RowsPipe pp{(a.nrows + RT - 1) / RT, ncols, d.status};
  const int64_t ntiles = (int64_t)pp.tiles_per_col * ncols;
  const int grid = (int)std::min<int64_t>(ntiles, TL::PER_SM * (int64_t)d.sms);
  if (grid <= 0) return cudaSuccess;
  *used = true;
  constexpr auto k = k_rows_c2r_pipe<T, P, TL::TB, TL::V, TL::NT>;
  cudaError_t e = set_smem<k>(sm);
  if (e == cudaSuccess) k<<<grid, TL::NT, sm, s>>>(a, pp);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, class P>
cudaError_t rows_r2c(const RowsR2C<T>& a, int ncols, cudaStream_t s) {
  typedef Tiles<T, P::n> TL;
  if constexpr (kRowsPipe<T, P>) {
    bool used = false;
    const cudaError_t e = rows_r2c_pipe<T, P>(a, ncols, s, &used);
    if (used || e != cudaSuccess) return e;
  }
  const size_t sm = (size_t)(twpad(P::n - 1) + P::n * TL::TB) * sizeof(typename CT<T>::C);
  const dim3 grid(cdiv((a.nrows + 1) / 2, TL::TB), ncols);
  if (P::can_zero_hi && a.seq_off >= 0 && a.seq_off + a.row_len <= P::n / 2)
    return launch_k<k_rows_r2c<T, P, TL::TB, TL::V, TL::NT, true>>(a, grid, TL::NT, sm, s);
  return launch_k<k_rows_r2c<T, P, TL::TB, TL::V, TL::NT, false>>(a, grid, TL::NT, sm, s);
}
template <typename T, class P>
cudaError_t rows_c2r(const RowsC2R<T>& a, int ncols, cudaStream_t s) {
  typedef Tiles<T, P::n> TL;
  if constexpr (kRowsPipe<T, P>) {
    bool used = false;
    const cudaError_t e = rows_c2r_pipe<T, P>(a, ncols, s, &used);
    if (used || e != cudaSuccess) return e;
  }
  constexpr auto k = k_rows_c2r<T, P, TL::TB, TL::V, TL::NT>;
  const size_t sm = (size_t)(twpad(P::n - 1) + P::n * TL::TB) * sizeof(typename CT<T>::C);
  cudaError_t e = set_smem<k>(sm);
  if (e != cudaSuccess) return e;
  k<<<dim3(cdiv((a.nrows + 1) / 2, TL::TB), ncols), TL::NT, sm, s>>>(a);
  return cudaGetLastError();
}
#ifndef TF_FWD_TILE
#define TF_FWD_TILE 1
#endif
template <auto K, class A>
cudaError_t launch_fwd(const A& a, const CUtensorMap& m, dim3 grid, int nt, size_t sm, cudaStream_t s) {
  cudaError_t e = set_smem<K>(sm);
  if (e != cudaSuccess) return e;
  K<<<grid, nt, sm, s>>>(a, m);
  return cudaGetLastError();
}
// A column-stage workspace of `ncols` columns (ld complex values each) as a 2-D tensor of
// single-precision values: rows of 2 hs floats (stride hs complex values), ld / hs rows per
// column; box 2 tb x ny.
// False when the driver entry point is missing or the layout does not fit a tensor map.
inline bool encode_rows_map(const void* base, int64_t ld, int hs, int ny, int ncols, int tb, CUtensorMap* m) {
  typedef CUresult (*Encode)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  static bool looked = false;
  if (!looked) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<Encode>(fn);
    looked = true;
  }
  if (!enc) return false;
  if (((uintptr_t)base & 15) != 0 || ld % hs != 0 || (hs * 8) % 16 != 0 || ny < 1 || ny > 256) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * hs, (cuuint64_t)(ld / hs) * (cuuint64_t)ncols};
  const cuuint64_t strides[1] = {(cuuint64_t)hs * 8};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * tb), (cuuint32_t)ny};
  const cuuint32_t estr[2] = {1, 1};
  if (dims[1] >= (1ull << 32)) return false;
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
constexpr size_t kFwdTileSmemMax = 228 * 1024 / 2 - 1024 - 256;   // two CTAs per SM
template <typename T, class P>
cudaError_t cols_fwd(const ColsFwd<T>& a, int ncols, cudaStream_t s) {
  typedef ColTiles<T, P> TL;
  typedef FwdTmem<T, P, TL::TB, TL::V, TL::NT> FT;
  const bool zhi = P::can_zero_hi && a.ny <= P::n / 2;
  size_t sm = (size_t)(twpad(P::n - 1) + FT::nbuf * P::n * TL::TB) * sizeof(typename CT<T>::C);
  if (FT::on && sm < kTmemSmemFloor) sm = kTmemSmemFloor;   // the residency cap of FwdTmem
  const dim3 grid(cdiv(a.nh, TL::TB), cdiv(ncols, FT::MC));
  ColsFwd<T> ac = a;
  ac.ncols = ncols;
  CUtensorMap zmap;
  memset(&zmap, 0, sizeof(zmap));
  if constexpr (FT::on && TF_FWD_TILE) {
    // tensor-copied layer tiles: a box of TB values by ny rows, and room for the tiles
    // within the two CTAs per SM that the register budget allows
    typedef typename CT<T>::C C;
    const size_t st = sm + 128 + (size_t)FT::MC * fwd_tile_stride<C, TL::TB>(a.ny) * sizeof(C);
    if (st <= kFwdTileSmemMax && encode_rows_map(a.z, a.z_ld, a.hs, a.ny, ncols, TL::TB, &zmap)) {
      if (zhi) return launch_fwd<k_cols_fwd<T, P, TL::TB, TL::V, TL::NT, true, true>>(ac, zmap, grid, TL::NT, st, s);
      return launch_fwd<k_cols_fwd<T, P, TL::TB, TL::V, TL::NT, false, true>>(ac, zmap, grid, TL::NT, st, s);
    }
  }
  if (zhi) return launch_fwd<k_cols_fwd<T, P, TL::TB, TL::V, TL::NT, true, false>>(ac, zmap, grid, TL::NT, sm, s);
  return launch_fwd<k_cols_fwd<T, P, TL::TB, TL::V, TL::NT, false, false>>(ac, zmap, grid, TL::NT, sm, s);
}
template <typename T, class P>
cudaError_t cols_adj(const ColsAdj<T>& a, int ncols, cudaStream_t s) {
  typedef ColTiles<T, P> TL;
  constexpr auto k = k_cols_adj<T, P, TL::TB, TL::V, TL::NT>;
  size_t sm = (size_t)(twpad(P::n - 1) + 2 * P::n * TL::TB) * sizeof(typename CT<T>::C);
  if (AdjTmem<T, P, TL::TB, TL::V, TL::NT>::on && sm < kTmemSmemFloor) sm = kTmemSmemFloor;
  cudaError_t e = set_smem<k>(sm);
  if (e != cudaSuccess) return e;
  k<<<dim3(cdiv(a.nh, TL::TB), ncols), TL::NT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ctk

#define TF_CT_CASE(FN, ...) \
  case TF_CT_FIRST(__VA_ARGS__): return ctk::FN<T, ct::Plan<__VA_ARGS__>>(a, ncols, s);
#define TF_CT_FIRST(x, ...) x

// Defines the dtype's four dispatchers: cudaErrorNotSupported for lengths off the menu.
#define TF_CT_DEFINE_DISPATCH(TYPE, COLS_MENU)                                             \
  template <>                                                                              \
  cudaError_t ct_rows_r2c<TYPE>(const RowsR2C<TYPE>& a, int ncols, cudaStream_t s) {       \
    typedef TYPE T;                                                                        \
    switch (a.plan.n) {                                                                    \
      TF_CT_MENU(TF_CT_R2C_CASE)                                                           \
      default: return cudaErrorNotSupported;                                               \
    }                                                                                      \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t ct_rows_c2r<TYPE>(const RowsC2R<TYPE>& a, int ncols, cudaStream_t s) {       \
    typedef TYPE T;                                                                        \
    switch (a.plan.n) {                                                                    \
      TF_CT_MENU(TF_CT_C2R_CASE)                                                           \
      default: return cudaErrorNotSupported;                                               \
    }                                                                                      \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t ct_cols_fwd<TYPE>(const ColsFwd<TYPE>& a, int ncols, cudaStream_t s) {       \
    typedef TYPE T;                                                                        \
    switch (a.plan.n) {                                                                    \
      COLS_MENU(TF_CT_FWD_CASE)                                                            \
      default: return cudaErrorNotSupported;                                               \
    }                                                                                      \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t ct_cols_adj<TYPE>(const ColsAdj<TYPE>& a, int ncols, cudaStream_t s) {       \
    typedef TYPE T;                                                                        \
    switch (a.plan.n) {                                                                    \
      COLS_MENU(TF_CT_ADJ_CASE)                                                            \
      default: return cudaErrorNotSupported;                                               \
    }                                                                                      \
  }

#define TF_CT_R2C_CASE(...) TF_CT_CASE(rows_r2c, __VA_ARGS__)
#define TF_CT_C2R_CASE(...) TF_CT_CASE(rows_c2r, __VA_ARGS__)
#define TF_CT_FWD_CASE(...) TF_CT_CASE(cols_fwd, __VA_ARGS__)
#define TF_CT_ADJ_CASE(...) TF_CT_CASE(cols_adj, __VA_ARGS__)

}  // namespace tfk
