// The generic FFT engine's product stages as device functions (tf_fft.cuh passes with
// runtime plans): each computes one tile (a group of sequences) of one column, so that the
// per-stage kernels (tf_kernels.cu) and the persistent batch kernel (tf_batch_kernels.cu)
// run the same code.  Stage contracts are those of RowsR2C / RowsC2R / ColsFwd / ColsAdj
// in tf_internal.h (App. A: 1-D FFTs of the rows, then of the columns, with the layer
// spectra's multiply-accumulate fused into the column transforms).
#pragma once
#include "tf_check.cuh"
#include "tf_internal.h"

namespace tfk {
namespace gen {

constexpr int kThreads = 256;
constexpr int kSmemDevices = 64;   // devices with a per-device shared-memory record

template <int V> struct Log2 { static constexpr int value = 1 + Log2<V / 2>::value; };
template <> struct Log2<1> { static constexpr int value = 0; };

__host__ __device__ inline int tw_pad(int count) { return (count + 1) & ~1; }

template <typename C> __device__ __forceinline__ C czero() { return mk<C>(0, 0); }

// Each stage is a device function over one tile (a group of sequences, `tile`) of one
// column (`col`); smem_raw is the CTA's dynamic shared memory (smem_rows / smem_cols bytes).
// The bodies end without a barrier: a caller that reuses the shared memory for another
// tile synchronises first.
template <typename T, int TB>
__device__ __forceinline__ void rows_r2c_body(const RowsR2C<T>& a, int tile, int col,
                                              unsigned char* smem_raw) {
  typedef typename CT<T>::C C;
  C* tw = reinterpret_cast<C*>(smem_raw);
  const int N = a.plan.n;
  constexpr int ld = TB + 1;
  C* bufA = tw + tw_pad(a.plan.tw_count);
  C* bufB = bufA + N * ld;
  for (int i = threadIdx.x; i < a.plan.tw_count; i += blockDim.x) tw[i] = a.tw[i];

  const int pair0 = tile * TB;
  const T* src = a.src + (int64_t)col * a.src_ld;
  // stage two real rows per complex sequence into bufB, rows of x contiguous in global
  for (int u = threadIdx.x; u < TB * N; u += blockDim.x) {
    const int pp = u / N, n = u - pp * N;
    const int ra = 2 * (pair0 + pp), rb = ra + 1;
    const int e = n - a.seq_off;
    const int64_t ext = (int64_t)a.nrows * a.row_len;
    T xa = T(0), xb = T(0);
    if (e >= 0 && e < a.row_len) {
      if (ra < a.nrows) {
        const int64_t o = (int64_t)ra * a.row_len + e;
        if (TF_IN(100 + kSiteR2cSrc, o, ext)) xa = src[o];
        if (a.scale && TF_IN(100 + kSiteR2cScale, o, ext)) xa *= a.scale[o];
      }
      if (rb < a.nrows) {
        const int64_t o = (int64_t)rb * a.row_len + e;
        if (TF_IN(100 + kSiteR2cSrc, o, ext)) xb = src[o];
        if (a.scale && TF_IN(100 + kSiteR2cScale, o, ext)) xb *= a.scale[o];
      }
    }
    bufB[n * ld + pp] = mk<C>(xa, xb);
  }
  __syncthreads();
  C* fin = ((a.plan.np - 1) & 1) ? bufB : bufA;
  fft_run<false>(a.plan, tw, bufA, bufB, ld, Log2<TB>::value, SmemLoad<C>{bufB, ld, N * ld},
                 SmemStore<C>{fin, ld, N * ld});
  // split the packed transform into the two rows' half spectra
  C* dst = a.dst + (int64_t)col * a.dst_ld;
  const int nh = a.nh;
  for (int u = threadIdx.x; u < TB * nh; u += blockDim.x) {
    const int pp = u / nh, k = u - pp * nh;
    const int ra = 2 * (pair0 + pp), rb = ra + 1;
    if (ra >= a.nrows) continue;
    const C z = fin[k * ld + pp];
    C zc = fin[(k ? N - k : 0) * ld + pp];
    zc.y = -zc.y;
    const int64_t ext = (int64_t)a.nrows * a.hs;
    if (TF_IN(100 + kSiteR2cDst, (int64_t)ra * a.hs + k, ext))
      dst[(int64_t)ra * a.hs + k] = mk<C>(T(0.5) * (z.x + zc.x), T(0.5) * (z.y + zc.y));
    if (rb < a.nrows && TF_IN(100 + kSiteR2cDst, (int64_t)rb * a.hs + k, ext))
      dst[(int64_t)rb * a.hs + k] = mk<C>(T(0.5) * (z.y - zc.y), T(-0.5) * (z.x - zc.x));
  }
}

template <typename T, int TB>
__device__ __forceinline__ void rows_c2r_body(const RowsC2R<T>& a, int tile, int col,
                                              unsigned char* smem_raw) {
  typedef typename CT<T>::C C;
  C* tw = reinterpret_cast<C*>(smem_raw);
  const int N = a.plan.n;
  constexpr int ld = TB + 1;
  C* bufA = tw + tw_pad(a.plan.tw_count);
  C* bufB = bufA + N * ld;
  for (int i = threadIdx.x; i < a.plan.tw_count; i += blockDim.x) tw[i] = a.tw[i];

  const int pair0 = tile * TB;
  const int nh = a.nh;
  const C* src = a.src + (int64_t)col * a.src_ld;
  // pack two Hermitian half spectra into one complex sequence: Z = Xa + i Xb
  for (int u = threadIdx.x; u < TB * nh; u += blockDim.x) {
    const int pp = u / nh, k = u - pp * nh;
    const int ra = 2 * (pair0 + pp), rb = ra + 1;
    const int64_t ext = (int64_t)a.nrows * a.hs;
    C xa = czero<C>(), xb = czero<C>();
    if (ra < a.nrows && TF_IN(100 + kSiteC2rSrc, (int64_t)ra * a.hs + k, ext)) xa = src[(int64_t)ra * a.hs + k];
    if (rb < a.nrows && TF_IN(100 + kSiteC2rSrc, (int64_t)rb * a.hs + k, ext)) xb = src[(int64_t)rb * a.hs + k];
    const bool self = (k == 0) || (2 * k == N);
    if (self) { xa.y = T(0); xb.y = T(0); }
    bufB[k * ld + pp] = mk<C>(xa.x - xb.y, xa.y + xb.x);
    if (!self) bufB[(N - k) * ld + pp] = mk<C>(xa.x + xb.y, xb.x - xa.y);
  }
  __syncthreads();
  C* fin = ((a.plan.np - 1) & 1) ? bufB : bufA;
  fft_run<true>(a.plan, tw, bufA, bufB, ld, Log2<TB>::value, SmemLoad<C>{bufB, ld, N * ld},
                SmemStore<C>{fin, ld, N * ld});
  T* dst = a.dst + (int64_t)col * a.dst_ld;
  const int L = a.out_len;
  for (int u = threadIdx.x; u < TB * L; u += blockDim.x) {
    const int pp = u / L, i = u - pp * L;
    const int ra = 2 * (pair0 + pp), rb = ra + 1;
    if (ra >= a.nrows) continue;
    const C z = fin[(a.seq_off + i) * ld + pp];
    const int64_t ext = (int64_t)a.nrows * L;
    const int64_t oa = (int64_t)ra * L + i;
    if (TF_IN(100 + kSiteC2rDst, oa, ext))
      dst[oa] = (a.scale && TF_IN(100 + kSiteC2rScale, oa, ext)) ? z.x * a.scale[oa] : z.x;
    if (rb < a.nrows) {
      const int64_t ob = (int64_t)rb * L + i;
      if (TF_IN(100 + kSiteC2rDst, ob, ext))
        dst[ob] = (a.scale && TF_IN(100 + kSiteC2rScale, ob, ext)) ? z.y * a.scale[ob] : z.y;
    }
  }
}

template <typename T, int TK>
__device__ __forceinline__ void cols_fwd_body(const ColsFwd<T>& a, int tile, int col,
                                              unsigned char* smem_raw) {
  typedef typename CT<T>::C C;
  C* tw = reinterpret_cast<C*>(smem_raw);
  const int N = a.plan.n;
  C* bufA = tw + tw_pad(a.plan.tw_count);
  C* bufB = bufA + N * TK;
  C* acc = bufB + N * TK;
  for (int i = threadIdx.x; i < a.plan.tw_count; i += blockDim.x) tw[i] = a.tw[i];
  __syncthreads();

  const int k0 = tile * TK;
  const int nh = a.nh, hs = a.hs, ny = a.ny, sy = a.sy;
  const C* z = a.z + (int64_t)col * a.z_ld;
  const int64_t z_ext = (int64_t)a.nz * ny * hs, g_ext = (int64_t)a.nz * N * hs;
  const C* spec = a.spec;
  for (int r = 0; r < a.nz; ++r) {
    const int64_t zoff = (int64_t)r * ny * hs, goff = (int64_t)r * N * hs;
    const bool first_layer = (r == 0);
    auto load = [=](int idx, int tk) -> C {
      const int k1 = k0 + tk;
      const int64_t e = zoff + (int64_t)idx * hs + k1;
      C v = czero<C>();
      if (idx < ny && k1 < nh && TF_IN(100 + kSiteFwdZ, e, z_ext)) v = z[e];
      return v;
    };
    auto mac = [=](int idx, int tk, C v) {
      const int k1 = k0 + tk;
      const int64_t e = goff + (int64_t)idx * hs + k1;
      C g = czero<C>();
      if (k1 < nh && TF_IN(100 + kSiteFwdSpec, e, g_ext)) g = spec[e];
      const C p = cmul(g, v);
      C* d = acc + idx * TK + tk;
      *d = first_layer ? p : cadd(*d, p);
    };
    fft_run<false>(a.plan, tw, bufA, bufB, TK, Log2<TK>::value, load, mac);
  }
  C* s = a.s + (int64_t)col * a.s_ld;
  const int64_t s_ext = (int64_t)sy * hs;
  auto store = [=](int idx, int tk, C v) {
    const int j = idx - (ny - 1), k1 = k0 + tk;
    if (j >= 0 && j < sy && k1 < nh && TF_IN(100 + kSiteFwdS, (int64_t)j * hs + k1, s_ext))
      s[(int64_t)j * hs + k1] = v;
  };
  fft_run<true>(a.plan, tw, bufA, bufB, TK, Log2<TK>::value, SmemLoad<C>{acc, TK, N * TK}, store);
}

template <typename T, int TK>
__device__ __forceinline__ void cols_adj_body(const ColsAdj<T>& a, int tile, int col,
                                              unsigned char* smem_raw) {
  typedef typename CT<T>::C C;
  C* tw = reinterpret_cast<C*>(smem_raw);
  const int N = a.plan.n;
  C* bufA = tw + tw_pad(a.plan.tw_count);
  C* bufB = bufA + N * TK;
  C* acc = bufB + N * TK;
  for (int i = threadIdx.x; i < a.plan.tw_count; i += blockDim.x) tw[i] = a.tw[i];
  __syncthreads();

  const int k0 = tile * TK;
  const int nh = a.nh, hs = a.hs, ny = a.ny, sy = a.sy;
  const C* z = a.z + (int64_t)col * a.z_ld;
  const int64_t z_ext = (int64_t)sy * hs, g_ext = (int64_t)a.nz * N * hs;
  const int64_t u_ext = (int64_t)a.nz * ny * hs;
  const C* spec = a.spec;
  auto load = [=](int idx, int tk) -> C {
    const int j = idx - (ny - 1), k1 = k0 + tk;
    C v = czero<C>();
    if (j >= 0 && j < sy && k1 < nh && TF_IN(100 + kSiteAdjZ, (int64_t)j * hs + k1, z_ext))
      v = z[(int64_t)j * hs + k1];
    return v;
  };
  fft_run<false>(a.plan, tw, bufA, bufB, TK, Log2<TK>::value, load, SmemStore<C>{acc, TK, N * TK});
  C* u = a.u + (int64_t)col * a.u_ld;
  for (int r = 0; r < a.nz; ++r) {
    const int64_t goff = (int64_t)r * N * hs, uoff = (int64_t)r * ny * hs;
    auto prod = [=](int idx, int tk) -> C {
      const int k1 = k0 + tk;
      const int64_t e = goff + (int64_t)idx * hs + k1;
      C v = czero<C>();
      if (k1 < nh && TF_IN(100 + kSiteAdjSpec, e, g_ext)) v = cmulc(acc[idx * TK + tk], spec[e]);
      return v;
    };
    auto store = [=](int idx, int tk, C v) {
      const int k1 = k0 + tk;
      const int64_t e = uoff + (int64_t)idx * hs + k1;
      if (idx < ny && k1 < nh && TF_IN(100 + kSiteAdjU, e, u_ext)) u[e] = v;
    };
    fft_run<true>(a.plan, tw, bufA, bufB, TK, Log2<TK>::value, prod, store);
  }
}

}  // namespace gen
}  // namespace tfk
