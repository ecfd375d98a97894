// CUDA kernels of the BTTB/BCCB products (App. A) and of the layer-spectra set-up.
//
// A forward product G x runs as three stages per chunk of columns:
//   rows_r2c  : x rows (scaled by colscale, zero-embedded) -> 1-D FFT along x (half spectra)
//   cols_fwd  : per k1 column: 1-D FFT along y of each layer, multiply by that layer's
//               spectrum and accumulate over layers, inverse FFT along y, keep sy rows
//   rows_c2r  : inverse FFT along x of the sy rows, keep the sx station window, scale
// The transpose product G^T y runs rows_r2c (data rows), cols_adj (one forward FFT,
// then per layer a conjugate-spectrum product and an inverse FFT), rows_c2r (model rows).
#include <math.h>

#include <algorithm>
#include <atomic>

#include "tf_check.cuh"
#include "tf_generic.cuh"
#include "tf_internal.h"

namespace tfk {

namespace {

using namespace gen;

template <typename T, int TB>
__global__ void __launch_bounds__(kThreads) k_rows_r2c(const RowsR2C<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_r2c_body<T, TB>(a, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename T, int TB>
__global__ void __launch_bounds__(kThreads) k_rows_c2r(const RowsC2R<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_c2r_body<T, TB>(a, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename T, int TK>
__global__ void __launch_bounds__(kThreads) k_cols_fwd(const ColsFwd<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cols_fwd_body<T, TK>(a, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename T, int TK>
__global__ void __launch_bounds__(kThreads) k_cols_adj(const ColsAdj<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cols_adj_body<T, TK>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// ---- layer spectra set-up (FP64) ------------------------------------------------------

// ln(a + r), r = sqrt(a^2 + rest2), without cancellation for a < 0
__device__ __forceinline__ double log_plus(double a, double rest2, double r) {
  return a >= 0.0 ? log(a + r) : log(rest2 / (r - a));
}

// Vertical attraction (m/s^2 per kg/m^3 / gamma) of the prism [x1,x2]x[y1,y2]x[z1,z2]
// relative to the station (z down): sum over corners of
// (-1)^(i+j+k) [x ln(y+R) + y ln(x+R) - z atan2(xy, zR)].
__device__ double prism_gz(double x1, double x2, double y1, double y2, double z1, double z2) {
  const double xs[2] = {x1, x2}, ys[2] = {y1, y2}, zs[2] = {z1, z2};
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double x = xs[i], y = ys[j], z = zs[k];
        const double x2_ = x * x, y2_ = y * y, z2_ = z * z;
        const double R = sqrt(x2_ + y2_ + z2_);
        const double f = x * log_plus(y, x2_ + z2_, R) + y * log_plus(x, y2_ + z2_, R) -
                         z * atan2(x * y, z * R);
        acc += ((i + j + k) & 1) ? -f : f;
      }
  return acc;
}

// Total-field anomaly factor f.T.f of the prism's second-derivative tensor of
// Int 1/R dV (Poisson's relation for a uniformly induced prism).
__device__ double prism_ftf(double x1, double x2, double y1, double y2, double z1, double z2,
                            double fx, double fy, double fz) {
  const double xs[2] = {x1, x2}, ys[2] = {y1, y2}, zs[2] = {z1, z2};
  double txx = 0, tyy = 0, tzz = 0, txy = 0, txz = 0, tyz = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double x = xs[i], y = ys[j], z = zs[k];
        const double x2_ = x * x, y2_ = y * y, z2_ = z * z;
        const double R = sqrt(x2_ + y2_ + z2_);
        // product of per-axis signs, +1 at the upper limit of each axis
        const double cu = ((i + j + k) & 1) ? 1.0 : -1.0;
        txx -= cu * atan(y * z / (x * R));
        tyy -= cu * atan(x * z / (y * R));
        tzz -= cu * atan2(x * y, z * R);
        txy += cu * log_plus(z, x2_ + y2_, R);
        txz += cu * log_plus(y, x2_ + z2_, R);
        tyz += cu * log_plus(x, y2_ + z2_, R);
      }
  return fx * fx * txx + fy * fy * tyy + fz * fz * tzz +
         2.0 * (fx * fy * txy + fx * fz * txz + fy * fz * tyz);
}

// Tensor Gauss-Legendre rule with n points per axis of the point-source kernel over a
// prism: kind 0 integrates z/R^3, kind 1 integrates (3 (f.R)^2 - R^2)/R^5.
__device__ double prism_quad(int kind, double x1, double x2, double y1, double y2, double z1,
                             double z2, int n, const double* t, const double* w, double fx,
                             double fy, double fz) {
  const double cx = 0.5 * (x1 + x2), hx = 0.5 * (x2 - x1);
  const double cy = 0.5 * (y1 + y2), hy = 0.5 * (y2 - y1);
  const double cz = 0.5 * (z1 + z2), hz = 0.5 * (z2 - z1);
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = cx + hx * t[i];
    for (int j = 0; j < n; ++j) {
      const double y = cy + hy * t[j];
      const double wij = w[i] * w[j];
      double row = 0.0;
      for (int k = 0; k < n; ++k) {
        const double z = cz + hz * t[k];
        const double r2 = x * x + y * y + z * z;
        const double rr = r2 * sqrt(r2);
        double f;
        if (kind == 0) {
          f = z / rr;
        } else {
          const double fr = fx * x + fy * y + fz * z;
          f = (3.0 * fr * fr - r2) / (r2 * rr);
        }
        row += w[k] * f;
      }
      acc += wij * row;
    }
  }
  return acc * hx * hy * hz;
}

// One table entry per thread.  The closed forms sum corner terms much larger than the
// result and lose ~(D/L)^3 ulps at distance D from a cell of longest side L, so cells
// with D >= 2 L are integrated by Gauss-Legendre quadrature instead (14 points per
// axis below 4 L, 8 below 8 L, 6 beyond), which keeps every entry near 1e-13 relative.
__global__ void k_table(const TableArgs a) {
  const int64_t total = (int64_t)a.nz * a.n2min * a.n1min;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e % a.n1min);
    const int t = (int)((e / a.n1min) % a.n2min);
    const int r = (int)(e / ((int64_t)a.n1min * a.n2min));
    // cell centre minus station for table entry (s, t)
    const double cx = -(double)(s - (a.nx - 1) + a.pxl) * a.dx;
    const double cy = -(double)(t - (a.ny - 1) + a.pyl) * a.dy;
    const double z1 = a.z_edges[r] - a.station_z, z2 = a.z_edges[r + 1] - a.station_z;
    const double x1 = cx - 0.5 * a.dx, x2 = cx + 0.5 * a.dx;
    const double y1 = cy - 0.5 * a.dy, y2 = cy + 0.5 * a.dy;
    const double cz = 0.5 * (z1 + z2);
    const double L = fmax(fmax(a.dx, a.dy), z2 - z1);
    const double D = sqrt(cx * cx + cy * cy + cz * cz);
    double v;
    if (D < 2.0 * L) {
      v = a.kind == 0 ? prism_gz(x1, x2, y1, y2, z1, z2)
                      : prism_ftf(x1, x2, y1, y2, z1, z2, a.fx, a.fy, a.fz);
    } else if (D < 4.0 * L) {
      v = prism_quad(a.kind, x1, x2, y1, y2, z1, z2, 14, a.g14x, a.g14w, a.fx, a.fy, a.fz);
    } else if (D < 8.0 * L) {
      v = prism_quad(a.kind, x1, x2, y1, y2, z1, z2, 8, a.g8x, a.g8w, a.fx, a.fy, a.fz);
    } else {
      v = prism_quad(a.kind, x1, x2, y1, y2, z1, z2, 6, a.g6x, a.g6w, a.fx, a.fy, a.fz);
    }
    // gravity: gamma [m^3/(kg s^2)] * 1000 [kg/m^3 per g/cc] * 1e5 [mGal per m/s^2];
    // magnetic: F / (4 pi) for unit SI susceptibility
    a.out[e] = a.kind == 0 ? 6.67430e-3 * v : a.field / (4.0 * 3.14159265358979323846) * v;
  }
}

template <int TK>
__global__ void __launch_bounds__(kThreads) k_spectrum(const SpecArgs a) {
  typedef double2 C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  const int N = a.plan.n;
  C* bufA = tw + tw_pad(a.plan.tw_count);
  C* bufB = bufA + N * TK;
  for (int i = threadIdx.x; i < a.plan.tw_count; i += blockDim.x) tw[i] = a.tw[i];
  __syncthreads();
  const int k0 = blockIdx.x * TK, r = blockIdx.y, nh = a.nh, n2min = a.n2min;
  const C* ht = a.ht + (int64_t)r * n2min * nh;
  C* out = a.spec + (int64_t)r * N * a.hs;
  const double sc = a.scale;
  auto load = [=](int idx, int tk) -> C {
    const int k1 = k0 + tk;
    return (idx < n2min && k1 < nh) ? ht[(int64_t)idx * nh + k1] : czero<C>();
  };
  auto store = [=](int idx, int tk, C v) {
    const int k1 = k0 + tk;
    if (k1 < nh) out[(int64_t)idx * a.hs + k1] = cscale(v, sc);
  };
  fft_run<false>(a.plan, tw, bufA, bufB, TK, Log2<TK>::value, load, store);
}

__global__ void k_to_f32(const double2* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

// Raises a kernel's dynamic shared-memory limit when a launch needs more than any
// earlier one did on the current device, so that steady-state launches (and launches
// under CUDA-graph capture) make no attribute call.  The attribute is per device, so the
// record is too.
template <auto Kernel>
cudaError_t prep(size_t smem) {
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

// Loads a kernel's code on the current device now (CUDA loads modules lazily, at a
// kernel's first launch, which allocates device memory) and raises its shared-memory
// limit for launches of `smem` bytes.
template <auto Kernel>
cudaError_t load_and_prep(size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, Kernel);
  return e == cudaSuccess ? prep<Kernel>(smem) : e;
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

size_t smem_rows(int n, int tw_count, int tb, size_t csize) {
  return ((size_t)tw_pad(tw_count) + 2 * (size_t)n * (tb + 1)) * csize;
}
size_t smem_cols(int n, int tw_count, int tk, size_t csize) {
  return ((size_t)tw_pad(tw_count) + 3 * (size_t)n * tk) * csize;
}

template <typename T, int TB>
static cudaError_t rows_r2c_tb(const RowsR2C<T>& a, int ncols, cudaStream_t s) {
  const size_t sm = smem_rows(a.plan.n, a.plan.tw_count, TB, sizeof(typename CT<T>::C));
  cudaError_t e = prep<k_rows_r2c<T, TB>>(sm);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div((a.nrows + 1) / 2, TB), ncols);
  k_rows_r2c<T, TB><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int TB>
static cudaError_t rows_c2r_tb(const RowsC2R<T>& a, int ncols, cudaStream_t s) {
  const size_t sm = smem_rows(a.plan.n, a.plan.tw_count, TB, sizeof(typename CT<T>::C));
  cudaError_t e = prep<k_rows_c2r<T, TB>>(sm);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div((a.nrows + 1) / 2, TB), ncols);
  k_rows_c2r<T, TB><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int TK>
static cudaError_t cols_fwd_tk(const ColsFwd<T>& a, int ncols, cudaStream_t s) {
  const size_t sm = smem_cols(a.plan.n, a.plan.tw_count, TK, sizeof(typename CT<T>::C));
  cudaError_t e = prep<k_cols_fwd<T, TK>>(sm);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(a.nh, TK), ncols);
  k_cols_fwd<T, TK><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int TK>
static cudaError_t cols_adj_tk(const ColsAdj<T>& a, int ncols, cudaStream_t s) {
  const size_t sm = smem_cols(a.plan.n, a.plan.tw_count, TK, sizeof(typename CT<T>::C));
  cudaError_t e = prep<k_cols_adj<T, TK>>(sm);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(a.nh, TK), ncols);
  k_cols_adj<T, TK><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_r2c(const RowsR2C<T>& a, int ncols, int tb, cudaStream_t s) {
  switch (tb) {
    case 4: return rows_r2c_tb<T, 4>(a, ncols, s);
    case 8: return rows_r2c_tb<T, 8>(a, ncols, s);
    case 16: return rows_r2c_tb<T, 16>(a, ncols, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t launch_rows_c2r(const RowsC2R<T>& a, int ncols, int tb, cudaStream_t s) {
  switch (tb) {
    case 4: return rows_c2r_tb<T, 4>(a, ncols, s);
    case 8: return rows_c2r_tb<T, 8>(a, ncols, s);
    case 16: return rows_c2r_tb<T, 16>(a, ncols, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t launch_cols_fwd(const ColsFwd<T>& a, int ncols, int tk, cudaStream_t s) {
  switch (tk) {
    case 4: return cols_fwd_tk<T, 4>(a, ncols, s);
    case 8: return cols_fwd_tk<T, 8>(a, ncols, s);
    case 16: return cols_fwd_tk<T, 16>(a, ncols, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t launch_cols_adj(const ColsAdj<T>& a, int ncols, int tk, cudaStream_t s) {
  switch (tk) {
    case 4: return cols_adj_tk<T, 4>(a, ncols, s);
    case 8: return cols_adj_tk<T, 8>(a, ncols, s);
    case 16: return cols_adj_tk<T, 16>(a, ncols, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int TB>
static cudaError_t prep_rows_tb(int n, int tw_count) {
  const size_t sm = smem_rows(n, tw_count, TB, sizeof(typename CT<T>::C));
  cudaError_t e = load_and_prep<k_rows_r2c<T, TB>>(sm);
  return e == cudaSuccess ? load_and_prep<k_rows_c2r<T, TB>>(sm) : e;
}
template <typename T, int TK>
static cudaError_t prep_cols_fwd_tk(int n, int tw_count) {
  return load_and_prep<k_cols_fwd<T, TK>>(smem_cols(n, tw_count, TK, sizeof(typename CT<T>::C)));
}

template <typename T>
cudaError_t prepare_forward_generic(int n1, int tw1, int n2, int tw2, int tb, int tk) {
  cudaError_t e;
  switch (tb) {
    case 4: e = prep_rows_tb<T, 4>(n1, tw1); break;
    case 8: e = prep_rows_tb<T, 8>(n1, tw1); break;
    case 16: e = prep_rows_tb<T, 16>(n1, tw1); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  switch (tk) {
    case 4: return prep_cols_fwd_tk<T, 4>(n2, tw2);
    case 8: return prep_cols_fwd_tk<T, 8>(n2, tw2);
    case 16: return prep_cols_fwd_tk<T, 16>(n2, tw2);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t prepare_forward_generic<float>(int, int, int, int, int, int);
template cudaError_t prepare_forward_generic<double>(int, int, int, int, int, int);

template cudaError_t launch_rows_r2c<float>(const RowsR2C<float>&, int, int, cudaStream_t);
template cudaError_t launch_rows_r2c<double>(const RowsR2C<double>&, int, int, cudaStream_t);
template cudaError_t launch_rows_c2r<float>(const RowsC2R<float>&, int, int, cudaStream_t);
template cudaError_t launch_rows_c2r<double>(const RowsC2R<double>&, int, int, cudaStream_t);
template cudaError_t launch_cols_fwd<float>(const ColsFwd<float>&, int, int, cudaStream_t);
template cudaError_t launch_cols_fwd<double>(const ColsFwd<double>&, int, int, cudaStream_t);
template cudaError_t launch_cols_adj<float>(const ColsAdj<float>&, int, int, cudaStream_t);
template cudaError_t launch_cols_adj<double>(const ColsAdj<double>&, int, int, cudaStream_t);

cudaError_t launch_table(const TableArgs& a, cudaStream_t s) {
  const int64_t total = (int64_t)a.nz * a.n2min * a.n1min;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_table<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_spectrum(const SpecArgs& a, int tk, cudaStream_t s) {
  (void)tk;
  constexpr int TK = 4;
  const size_t sm = ((size_t)tw_pad(a.plan.tw_count) + 2 * (size_t)a.plan.n * TK) * sizeof(double2);
  cudaError_t e = prep<k_spectrum<TK>>(sm);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(a.nh, TK), a.nz);
  k_spectrum<TK><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double2* src, float2* dst, int64_t count, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 8);
  k_to_f32<<<blocks, 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

// ---- re-orthogonalisation kernels ------------------------------------------------------

// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2 (about 44 bits).
// Knuth's TwoSum and the FMA-based TwoProd give exact error terms on the FP32 pipe,
// which on this GPU is far faster than its FP64 pipe.  The _rn intrinsics round each
// step on its own (the compiler never fuses them into FMAs), which the error terms need.
struct DF { float hi, lo; };
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {   // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  const float t = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, t);
}
__device__ __forceinline__ DF df_mul_ff(float a, float b) {   // exact product of floats
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ DF df_mul_df(DF c, float a) {      // (c.hi + c.lo) * a
  const DF p = df_mul_ff(c.hi, a);
  return df_fast_two_sum(p.hi, fmaf(c.lo, a, p.lo));
}

// y[j] = sum_i A[j*lda + i] * x[i] for j < k: one CTA per row, fixed reduction order
// (deterministic).  Accumulation in FP64 for double data, in double-float for float data.
__global__ void __launch_bounds__(256) k_rows_dot_d(const double* __restrict__ A, int64_t lda,
                                                    int64_t len, const double* __restrict__ x,
                                                    double* __restrict__ y) {
  const double* a = A + (int64_t)blockIdx.x * lda;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) acc = fma(a[i], x[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += part[w];
    y[blockIdx.x] = sum;
  }
}

__global__ void __launch_bounds__(256) k_rows_dot_f(const float* __restrict__ A, int64_t lda,
                                                    int64_t len, const float* __restrict__ x,
                                                    double* __restrict__ y) {
  const float* a = A + (int64_t)blockIdx.x * lda;
  DF acc = {0.f, 0.f};
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) acc = df_add(acc, df_mul_ff(a[i], x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF other = {__shfl_down_sync(0xffffffffu, acc.hi, o), __shfl_down_sync(0xffffffffu, acc.lo, o)};
    acc = df_add(acc, other);
  }
  __shared__ DF part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += (double)part[w].hi + (double)part[w].lo;
    y[blockIdx.x] = sum;
  }
}

// x[i] -= sum_j c[j] * A[j*lda + i] for j < k: FP64 accumulation for double data; for
// float data the coefficients are split into float pairs in shared memory and the sum is
// accumulated in double-float.
__global__ void __launch_bounds__(256) k_rows_axpy_d(const double* __restrict__ A, int64_t lda,
                                                     int64_t k, int64_t len,
                                                     const double* __restrict__ c,
                                                     double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t j = 0; j < k; ++j) acc = fma(c[j], A[j * lda + i], acc);
    x[i] -= acc;
  }
}

constexpr int kAxpyTile = 2048;

__global__ void __launch_bounds__(256) k_rows_axpy_f(const float* __restrict__ A, int64_t lda,
                                                     int64_t k, int64_t len,
                                                     const double* __restrict__ c,
                                                     float* __restrict__ x) {
  __shared__ DF cs[kAxpyTile];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  DF acc = {0.f, 0.f};
  for (int64_t j0 = 0; j0 < k; j0 += kAxpyTile) {
    const int nt = (int)((k - j0) < kAxpyTile ? (k - j0) : kAxpyTile);
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      const double v = c[j0 + t];
      const float hi = (float)v;
      cs[t] = {hi, (float)(v - (double)hi)};
    }
    __syncthreads();
    if (i < len) {
      const float* a = A + j0 * lda + i;
      int t = 0;
      for (; t + 4 <= nt; t += 4) {          // four independent loads in flight
        const float a0 = a[(int64_t)t * lda], a1 = a[(int64_t)(t + 1) * lda];
        const float a2 = a[(int64_t)(t + 2) * lda], a3 = a[(int64_t)(t + 3) * lda];
        acc = df_add(acc, df_mul_df(cs[t], a0));
        acc = df_add(acc, df_mul_df(cs[t + 1], a1));
        acc = df_add(acc, df_mul_df(cs[t + 2], a2));
        acc = df_add(acc, df_mul_df(cs[t + 3], a3));
      }
      for (; t < nt; ++t) acc = df_add(acc, df_mul_df(cs[t], a[(int64_t)t * lda]));
    }
  }
  if (i < len) {
    const DF r = df_add({x[i], 0.f}, {-acc.hi, -acc.lo});
    x[i] = r.hi + r.lo;
  }
}

cudaError_t launch_rows_dot(int dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                            const void* x, double* y, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  if (dtype == 0) k_rows_dot_f<<<(unsigned)k, 256, 0, s>>>((const float*)A, lda, len, (const float*)x, y);
  else k_rows_dot_d<<<(unsigned)k, 256, 0, s>>>((const double*)A, lda, len, (const double*)x, y);
  return cudaGetLastError();
}

cudaError_t launch_rows_axpy(int dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                             const double* c, void* x, cudaStream_t s) {
  if (k <= 0 || len <= 0) return cudaSuccess;
  if (dtype == 0) {
    // one element per thread so that every thread of a CTA meets the tile barriers
    const unsigned blocks = (unsigned)((len + 255) / 256);
    k_rows_axpy_f<<<blocks, 256, 0, s>>>((const float*)A, lda, k, len, c, (float*)x);
  } else {
    const unsigned blocks = (unsigned)std::min<int64_t>((len + 255) / 256, 152 * 16);
    k_rows_axpy_d<<<blocks, 256, 0, s>>>((const double*)A, lda, k, len, c, (double*)x);
  }
  return cudaGetLastError();
}

// ---- FMA throughput probe -------------------------------------------------------------

// Eight independent fused multiply-add chains per thread; the result is stored so that
// nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = T(threadIdx.x + k) * T(1e-6);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t fma_probe(void* out, int blocks, int iters, float* ms, cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<T><<<blocks, 256, 0, s>>>((T*)out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e0, s);
  k_fma_probe<T><<<blocks, 256, 0, s>>>((T*)out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t launch_fma_probe(int dtype, void* out, int blocks, int iters, float* ms, cudaStream_t s) {
  return dtype == 0 ? fma_probe<float>(out, blocks, iters, ms, s)
                    : fma_probe<double>(out, blocks, iters, ms, s);
}

TF_DEFINE_OOB_READER(oob_read_generic)

}  // namespace tfk
