// IRLS focusing inversion drivers tf_gkb / tf_rsvd (Sec. 2.3; Alg. 1 and Alg. 2; Sec. 3.1)
// on the library's products, and the host helpers of their projected solves.
//
// Every product with G~ = W_d G W^-1 (Sec. 2.5, Eq. (10)) is one tf_matvec / tf_rmatvec /
// tf_matmat / tf_rmatmat call with colscale = W^-1 and rowscale = W_d.  The GKB loop keeps
// its norms on the device (no host round trip per step); the re-orthogonalisation runs in
// the FP64 / double-float row kernels (tf_rows_dot, tf_rows_axpy).  The projected
// problems are small and solved on the host in FP64:
//  * GKB: the Golub-Kahan form of B (zero diagonal, off-diagonal gam_0, bet_0, gam_1, ...)
//    is tridiagonal; its positive eigenvalues are the s_i and its eigenvectors' first
//    components are the first row of U over sqrt(2), which is all that UPRE and Eq. (11)
//    use; the Tikhonov solution on all t_p terms is the least squares solution of
//    [B; alpha I] y = [||r~|| e_1; 0], computed with Givens rotations.
//  * RSVD: QR factors from cuSOLVER, B^T B with cuBLAS, its eigen-decomposition with
//    cuSOLVER, then the truncated Tikhonov filter on the t largest singular values.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <numeric>
#include <vector>

#include "../../include/tf.h"
#include "tf_driver.h"

namespace {

using tfk::api_fail;

// ------------------------------------------------------------------ host numerics

// Implicit QL with Wilkinson shifts on the symmetric tridiagonal (d, e), accumulating
// only the first row of the eigenvector matrix.  Returns false without convergence.
// An off-diagonal entry is negligible below eps times its diagonal neighbours, or below
// eps times the matrix norm (absolute accuracy eps ||T||, the accuracy the iteration has
// anyway; without it a zero eigenvalue between zero diagonal entries deflates only once
// its coupling underflows).
bool tridiag_ql_first(int n, double* d, double* e, double* first) {
  for (int i = 0; i < n; ++i) first[i] = i == 0 ? 1.0 : 0.0;
  if (n <= 1) return true;
  e[n - 1] = 0.0;
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    tnorm = std::max(tnorm, fabs(d[i]) + fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0));
  const double tiny = DBL_EPSILON * tnorm;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double scale = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= DBL_EPSILON * scale || fabs(e[m]) <= tiny) break;
      }
      if (m == l) break;
      if (iter >= 64) return false;
      // shift: the eigenvalue of the leading 2 x 2 block closer to d[l]
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // the rotation splits the matrix: restart from the top
          d[i + 1] -= p;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        const double zi = first[i], zi1 = first[i + 1];
        first[i + 1] = s * zi + c * zi1;
        first[i] = c * zi - s * zi1;
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return true;
}

// Givens QR of [B; alpha I] for the lower bidiagonal B (diag gam, subdiag bet), right
// hand side [b0 e_1; 0], and back substitution of the upper bidiagonal factor.
void damped_bidiag_solve(int tp, const double* gam, const double* bet, double alpha, double b0,
                         double* y) {
  std::vector<double> rd(tp), re(tp, 0.0), g(tp);
  double x = gam[0], f = b0;  // current diagonal entry and right-hand side of row j
  for (int j = 0; j < tp; ++j) {
    // rotate the damping row (alpha at column j) into row j
    double r = hypot(x, alpha);
    double c = r > 0 ? x / r : 1.0;
    x = r;
    f = c * f;
    // rotate row j + 1 (bet[j] at column j, gam[j+1] at column j+1) into row j
    r = hypot(x, bet[j]);
    c = r > 0 ? x / r : 1.0;
    const double s = r > 0 ? bet[j] / r : 0.0;
    rd[j] = r;
    g[j] = c * f;
    if (j + 1 < tp) {
      re[j] = s * gam[j + 1];
      x = c * gam[j + 1];
    }
    f = -s * f;
  }
  for (int j = tp - 1; j >= 0; --j) {
    const double num = g[j] - (j + 1 < tp ? re[j] * y[j + 1] : 0.0);
    y[j] = rd[j] != 0.0 ? num / rd[j] : 0.0;
  }
}

// UPRE for whitened noise on t terms, alpha-independent terms dropped; c2 = coef^2.
double upre(double alpha, const double* s, const double* c2, int t) {
  const double a2 = alpha * alpha;
  double fit = 0.0, tr = 0.0;
  for (int i = 0; i < t; ++i) {
    const double s2 = s[i] * s[i];
    const double phi = s2 / (s2 + a2);
    fit += (1.0 - phi) * (1.0 - phi) * c2[i];
    tr += phi;
  }
  return fit + 2.0 * tr - t;
}

// argmin UPRE: 200-point log grid on [max(s_t, 1e-14 s_1)/10, s_1], then 80 golden-section
// steps in log alpha between the best grid point's neighbours.
double choose_alpha(const double* s, const double* c2, int t) {
  const double gold = (sqrt(5.0) - 1.0) / 2.0;
  const double lo = log(std::max(s[t - 1], 1e-14 * s[0]) / 10.0), hi = log(s[0]);
  const int np = 200;
  const double step = (hi - lo) / (np - 1);
  std::vector<double> grid(np), val(np);
  int k = 0;
  for (int i = 0; i < np; ++i) {
    grid[i] = exp(i == np - 1 ? hi : i * step + lo);
    val[i] = upre(grid[i], s, c2, t);
    if (val[i] < val[k]) k = i;
  }
  double left = log(grid[std::max(k - 1, 0)]), right = log(grid[std::min(k + 1, np - 1)]);
  double x1 = right - gold * (right - left), x2 = left + gold * (right - left);
  double f1 = upre(exp(x1), s, c2, t), f2 = upre(exp(x2), s, c2, t);
  for (int it = 0; it < 80; ++it) {
    if (f1 <= f2) {
      right = x2; x2 = x1; f2 = f1;
      x1 = right - gold * (right - left);
      f1 = upre(exp(x1), s, c2, t);
    } else {
      left = x1; x1 = x2; f1 = f2;
      x2 = left + gold * (right - left);
      f2 = upre(exp(x2), s, c2, t);
    }
  }
  const double mid = exp(0.5 * (left + right));
  return upre(mid, s, c2, t) <= val[k] ? mid : grid[k];
}

// Eq. (11): (n/m)^3.5 s_1 / mean of the t retained singular values above 1e-14 s_1.
double alpha_start(int64_t n, int64_t m, const double* s, int t) {
  double sum = 0.0;
  int cnt = 0;
  for (int i = 0; i < t; ++i)
    if (s[i] > 1e-14 * s[0]) { sum += s[i]; ++cnt; }
  return pow((double)n / (double)m, 3.5) * s[0] / (sum / cnt);
}

// ------------------------------------------------------------------ device kernels

constexpr int kRedBlocks = 256, kRedThreads = 256;

__device__ __forceinline__ float to_t(double v, float) { return (float)v; }
__device__ __forceinline__ double to_t(double v, double) { return v; }

template <typename T> __global__ void k_fill(T* x, T v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}
// x -= (T)(*s) * y
template <typename T> __global__ void k_sub_scaled(T* x, const T* y, const double* s, int64_t n) {
  const T a = to_t(*s, T());
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= a * y[i];
}
// x /= (T)(*nrm)
template <typename T> __global__ void k_div(T* x, const double* nrm, int64_t n) {
  const T a = to_t(*nrm, T());
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] /= a;
}
// per-block partial sums of x^2 in FP64, fixed order (deterministic)
template <typename T> __global__ void __launch_bounds__(kRedThreads) k_sumsq_part(const T* x, int64_t n, double* part) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)kRedBlocks * kRedThreads) {
    const double v = (double)x[i];
    acc += v * v;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// out = sum of the partials (or its square root)
__global__ void __launch_bounds__(kRedThreads) k_sumsq_final(const double* part, double* out, int root) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = root ? sqrt(sh[0]) : sh[0];
}
// winv = 1 / (wz * wl), wl = 1 (first) or ((m1 - m2)^2 + eps2)^ex, in the data type
template <typename T>
__global__ void k_weights(T* winv, const T* wz, const T* m1, const T* m2, T eps2, T ex, int first, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T wl = T(1);
    if (!first) {
      const T dm = m1[i] - m2[i];
      wl = pow(dm * dm + eps2, ex);
    }
    winv[i] = T(1) / (wz[i] * wl);
  }
}
// out = wd * (a - b)
template <typename T> __global__ void k_wdiff(T* out, const T* wd, const T* a, const T* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = wd[i] * (a[i] - b[i]);
}
// wd = 1 / sigma
template <typename T> __global__ void k_recip(T* out, const T* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = T(1) / x[i];
}
// m_new = clamp(m1 + winv * z, lo, hi)
template <typename T>
__global__ void k_update(T* mnew, const T* m1, const T* winv, const T* z, T lo, T hi, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    mnew[i] = fmin(fmax(m1[i] + winv[i] * z[i], lo), hi);
}
template <typename T> __global__ void k_to_f64(double* out, const T* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)x[i];
}

inline unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// ------------------------------------------------------------------ driver plumbing

struct DevMem {
  std::vector<void*> ptrs;
  ~DevMem() { for (void* p : ptrs) cudaFree(p); }
  template <typename X> cudaError_t get(X** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(X));
    if (e == cudaSuccess) { ptrs.push_back(q); *p = (X*)q; }
    return e;
  }
};

#define TRY_CUDA(call, what)                                                   \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return api_fail(e_ == cudaErrorMemoryAllocation ? TF_ENOMEM : TF_ECUDA,  \
                      "%s: %s", what, cudaGetErrorString(e_));                 \
  } while (0)
#define TRY_TF(call)                  \
  do {                                \
    tf_status s_ = (call);            \
    if (s_ != TF_OK) return s_;       \
  } while (0)
#define TRY_LIB(call, what)                                                    \
  do {                                                                         \
    int e_ = (int)(call);                                                      \
    if (e_ != 0) return api_fail(TF_ECUDA, "%s failed (status %d)", what, e_);  \
  } while (0)

template <typename T> tf_dtype dtype_of();
template <> tf_dtype dtype_of<float>() { return TF_F32; }
template <> tf_dtype dtype_of<double>() { return TF_F64; }

// Shared state of one IRLS run: weights, iterates and the steps around the solver.
template <typename T> struct Irls {
  tf_op* op;
  const tf_irls_params* p;
  tfk::OpInfo info;
  cudaStream_t s;
  DevMem mem;
  T *wz, *wd, *winv, *m1, *m2, *mnew, *rt, *dv, *z;
  double *part, *scal;  // reduction partials; device scalars
  const T* dobs;

  tf_status init(tf_op* op_, const tf_irls_params* p_, const void* d_obs, const void* sigma,
                 cudaStream_t s_) {
    op = op_; p = p_; s = s_;
    dobs = (const T*)d_obs;
    const int64_t n = info.n, m = info.m;
    for (T** q : {&wz, &winv, &m1, &m2, &mnew, &z}) TRY_CUDA(mem.get(q, n), "cudaMalloc(driver)");
    for (T** q : {&wd, &rt, &dv}) TRY_CUDA(mem.get(q, m), "cudaMalloc(driver)");
    TRY_CUDA(mem.get(&part, kRedBlocks), "cudaMalloc(driver)");
    TRY_CUDA(mem.get(&scal, 4), "cudaMalloc(driver)");
    // W_z: (mean depth of layer r below the stations)^(-beta), rounded to T
    const int64_t layer = (int64_t)info.nx * info.ny;
    for (int r = 0; r < info.nz; ++r) {
      const double zbar = 0.5 * ((info.z_edges[r] - info.station_z) + (info.z_edges[r + 1] - info.station_z));
      const T v = (T)pow(zbar, -p->beta);
      k_fill<T><<<grid_for(layer), 256, 0, s>>>(wz + r * layer, v, layer);
    }
    k_recip<T><<<grid_for(m), 256, 0, s>>>(wd, (const T*)sigma, m);
    k_fill<T><<<grid_for(n), 256, 0, s>>>(m1, T(0), n);
    k_fill<T><<<grid_for(n), 256, 0, s>>>(m2, T(0), n);
    TRY_CUDA(cudaGetLastError(), "driver set-up kernels");
    return TF_OK;
  }
  // *out = ||x|| (or ||x||^2) on the device
  tf_status norm(const T* x, int64_t len, double* out, bool root = true) {
    k_sumsq_part<T><<<kRedBlocks, kRedThreads, 0, s>>>(x, len, part);
    k_sumsq_final<<<1, kRedThreads, 0, s>>>(part, out, root ? 1 : 0);
    TRY_CUDA(cudaGetLastError(), "norm kernels");
    return TF_OK;
  }
  // W^-1 for iteration k and r~ = W_d (d_obs - G m^(k-1))
  tf_status begin(int k) {
    const int64_t n = info.n, m = info.m;
    k_weights<T><<<grid_for(n), 256, 0, s>>>(winv, wz, m1, m2, (T)p->eps2, (T)((p->lam - 2.0) / 4.0),
                                             k == 1 ? 1 : 0, n);
    TRY_CUDA(cudaGetLastError(), "weights kernel");
    TRY_TF(tf_matvec(op, m1, dv, nullptr, nullptr, s));
    k_wdiff<T><<<grid_for(m), 256, 0, s>>>(rt, wd, dobs, dv, m);
    TRY_CUDA(cudaGetLastError(), "residual kernel");
    return TF_OK;
  }
  // m^(k) = clip(m^(k-1) + W^-1 z); chi^2 of m^(k); shift the iterates
  tf_status finish(double* chi2) {
    const int64_t n = info.n, m = info.m;
    k_update<T><<<grid_for(n), 256, 0, s>>>(mnew, m1, winv, z, (T)p->lower, (T)p->upper, n);
    TRY_CUDA(cudaGetLastError(), "update kernel");
    TRY_TF(tf_matvec(op, mnew, dv, nullptr, nullptr, s));
    k_wdiff<T><<<grid_for(m), 256, 0, s>>>(dv, wd, dv, dobs, m);
    TRY_TF(norm(dv, m, scal + 3, false));
    TRY_CUDA(cudaMemcpyAsync(chi2, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s), "chi2 copy");
    TRY_CUDA(cudaStreamSynchronize(s), "IRLS iteration");
    T* t = m2; m2 = m1; m1 = mnew; mnew = t;
    return TF_OK;
  }
};

tf_status check_params(const tf_irls_params* p, const tfk::OpInfo& info) {
  if (!p) return api_fail(TF_EINVAL, "params is NULL");
  if (p->tp < 1 || p->t < 1 || p->t > p->tp)
    return api_fail(TF_EINVAL, "need 1 <= t <= tp (got t=%d, tp=%d)", p->t, p->tp);
  if (p->kmax < 1) return api_fail(TF_EINVAL, "kmax must be >= 1");
  if (!(p->eps2 > 0)) return api_fail(TF_EINVAL, "eps2 must be > 0");
  if (!(p->lower <= p->upper)) return api_fail(TF_EINVAL, "need lower <= upper");
  if (p->reorth != 0 && p->reorth != 1) return api_fail(TF_EINVAL, "reorth must be 0 or 1");
  for (int r = 0; r < info.nz; ++r)
    if (!(0.5 * (info.z_edges[r] + info.z_edges[r + 1]) - info.station_z > 0))
      return api_fail(TF_EINVAL, "layer %d has no positive mean depth below the stations", r);
  return TF_OK;
}

void report_step(tf_irls_report* rep, int k, double alpha, double chi2, double sec) {
  if (!rep) return;
  rep->iterations = k;
  if (rep->alpha) rep->alpha[k - 1] = alpha;
  if (rep->chi2) rep->chi2[k - 1] = chi2;
  if (rep->seconds) rep->seconds[k - 1] = sec;
}

// x <- x minus its components along the first k rows of V (orthonormal, row stride ld)
template <typename T>
tf_status orthogonalise(const T* V, int64_t ld, int k, int64_t len, T* x, int method, double* coef,
                        cudaStream_t s) {
  if (k == 0) return TF_OK;
  const tf_dtype dt = dtype_of<T>();
  if (method == 1) {  // modified Gram-Schmidt, rows in order
    for (int j = 0; j < k; ++j) {
      TRY_TF(tf_rows_dot(dt, V + j * ld, ld, 1, len, x, coef, s));
      TRY_TF(tf_rows_axpy(dt, V + j * ld, ld, 1, len, coef, x, s));
    }
  } else {  // classical Gram-Schmidt applied twice
    for (int pass = 0; pass < 2; ++pass) {
      TRY_TF(tf_rows_dot(dt, V, ld, k, len, x, coef, s));
      TRY_TF(tf_rows_axpy(dt, V, ld, k, len, coef, x, s));
    }
  }
  return TF_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <typename T>
tf_status gkb_run(tf_op* op, const tf_irls_params* p, const void* d_obs, const void* sigma, void* m_out,
                  tf_irls_report* rep, cudaStream_t s) {
  Irls<T> st;
  TRY_TF(tfk::op_info(op, &st.info));
  TRY_TF(check_params(p, st.info));
  const int64_t n = st.info.n, m = st.info.m;
  const int tp = p->tp, t = p->t;
  TRY_TF(st.init(op, p, d_obs, sigma, s));
  T *A, *H;
  double *diag, *sub, *coef;
  TRY_CUDA(st.mem.get(&A, (size_t)tp * n), "cudaMalloc(GKB basis A)");
  TRY_CUDA(st.mem.get(&H, (size_t)(tp + 1) * m), "cudaMalloc(GKB basis H)");
  TRY_CUDA(st.mem.get(&diag, tp), "cudaMalloc(driver)");
  TRY_CUDA(st.mem.get(&sub, tp), "cudaMalloc(driver)");
  TRY_CUDA(st.mem.get(&coef, std::max(tp + 1, 1)), "cudaMalloc(driver)");
  double* rnorm = st.scal;
  std::vector<double> gam(tp), bet(tp), dd(2 * tp + 1), ee(2 * tp + 1), first(2 * tp + 1), y(tp);
  for (int k = 1; k <= p->kmax; ++k) {
    const double t0 = now_s();
    TRY_TF(st.begin(k));
    // Alg. 1: H e_1 = r~ / ||r~||; then a_i, h_{i+1} with B(i,i) = gamma_i, B(i+1,i) = beta_{i+1}
    TRY_TF(st.norm(st.rt, m, rnorm));
    TRY_CUDA(cudaMemcpyAsync(H, st.rt, m * sizeof(T), cudaMemcpyDeviceToDevice, s), "copy");
    k_div<T><<<grid_for(m), 256, 0, s>>>(H, rnorm, m);
    for (int i = 0; i < tp; ++i) {
      T* a = A + (int64_t)i * n;
      T* h = H + (int64_t)i * m;
      T* h1 = H + (int64_t)(i + 1) * m;
      TRY_TF(tf_rmatvec(op, h, a, st.winv, st.wd, s));
      if (i > 0) k_sub_scaled<T><<<grid_for(n), 256, 0, s>>>(a, A + (int64_t)(i - 1) * n, sub + i - 1, n);
      TRY_TF(orthogonalise(A, n, i, n, a, p->reorth, coef, s));
      TRY_TF(st.norm(a, n, diag + i));
      k_div<T><<<grid_for(n), 256, 0, s>>>(a, diag + i, n);
      TRY_TF(tf_matvec(op, a, h1, st.winv, st.wd, s));
      k_sub_scaled<T><<<grid_for(m), 256, 0, s>>>(h1, h, diag + i, m);
      TRY_TF(orthogonalise(H, m, i + 1, m, h1, p->reorth, coef, s));
      TRY_TF(st.norm(h1, m, sub + i));
      k_div<T><<<grid_for(m), 256, 0, s>>>(h1, sub + i, m);
      TRY_CUDA(cudaGetLastError(), "GKB step kernels");
    }
    double rn = 0;
    TRY_CUDA(cudaMemcpyAsync(gam.data(), diag, tp * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaMemcpyAsync(bet.data(), sub, tp * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaMemcpyAsync(&rn, rnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaStreamSynchronize(s), "GKB factorisation");
    // Golub-Kahan form of B: the (2 t_p + 1)-square symmetric tridiagonal matrix with zero
    // diagonal and off-diagonal gam_0, bet_0, gam_1, bet_1, ... (the matrix [0 B; B^T 0]
    // with rows and columns interleaved u_1, v_1, u_2, ...).  Its eigenvalues are +-s_i and
    // 0, and the eigenvector of +s_i is (u_i, v_i) / sqrt(2) interleaved, so its first
    // component is U(1, i) / sqrt(2).  Working on it instead of on B B^T keeps small s_i
    // to absolute accuracy eps s_1 rather than eps s_1^2 / s_i.
    const int ng = 2 * tp + 1;
    for (int i = 0; i < ng; ++i) {
      dd[i] = 0.0;
      ee[i] = i + 1 < ng ? ((i & 1) ? bet[i / 2] : gam[i / 2]) : 0.0;
    }
    if (!tridiag_ql_first(ng, dd.data(), ee.data(), first.data()))
      return api_fail(TF_ENOTCONV, "tf_gkb: tridiagonal eigenvalue iteration did not converge");
    std::vector<int> order(ng);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dd[a] > dd[b]; });
    std::vector<double> sv(tp), c2(tp);
    for (int i = 0; i < tp; ++i) {  // the t_p largest eigenvalues are s_1 >= ... >= s_tp
      sv[i] = std::max(dd[order[i]], 0.0);
      c2[i] = 2.0 * rn * rn * first[order[i]] * first[order[i]];
    }
    double alpha;
    if (p->alphas) alpha = p->alphas[k - 1];
    else if (k == 1) alpha = alpha_start(n, m, sv.data(), t);
    else alpha = choose_alpha(sv.data(), c2.data(), t);
    damped_bidiag_solve(tp, gam.data(), bet.data(), alpha, rn, y.data());
    // z = A y  (tf_rows_axpy subtracts: pass -y)
    for (double& v : y) v = -v;
    TRY_CUDA(cudaMemcpyAsync(coef, y.data(), tp * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    k_fill<T><<<grid_for(n), 256, 0, s>>>(st.z, T(0), n);
    TRY_TF(tf_rows_axpy(dtype_of<T>(), A, n, tp, n, coef, st.z, s));
    double chi2 = 0;
    TRY_TF(st.finish(&chi2));
    report_step(rep, k, alpha, chi2, now_s() - t0);
    if (p->chi2_stop && chi2 <= m + sqrt(2.0 * m)) break;
  }
  TRY_CUDA(cudaMemcpyAsync(m_out, st.m1, n * sizeof(T), cudaMemcpyDeviceToDevice, s), "copy");
  TRY_CUDA(cudaStreamSynchronize(s), "tf_gkb");
  return TF_OK;
}

// ---- cuSOLVER / cuBLAS pieces of the RSVD driver ----

struct Handles {
  cusolverDnHandle_t sol = nullptr;
  cublasHandle_t blas = nullptr;
  ~Handles() {
    if (sol) cusolverDnDestroy(sol);
    if (blas) cublasDestroy(blas);
  }
};

// Typed cuSOLVER / cuBLAS entry points of the QR pieces.
int geqrf_lwork(cusolverDnHandle_t h, int m, int n, float* A, int lda, int* lw) {
  return (int)cusolverDnSgeqrf_bufferSize(h, m, n, A, lda, lw);
}
int geqrf_lwork(cusolverDnHandle_t h, int m, int n, double* A, int lda, int* lw) {
  return (int)cusolverDnDgeqrf_bufferSize(h, m, n, A, lda, lw);
}
int orgqr_lwork(cusolverDnHandle_t h, int m, int n, float* A, int lda, const float* tau, int* lw) {
  return (int)cusolverDnSorgqr_bufferSize(h, m, n, n, A, lda, tau, lw);
}
int orgqr_lwork(cusolverDnHandle_t h, int m, int n, double* A, int lda, const double* tau, int* lw) {
  return (int)cusolverDnDorgqr_bufferSize(h, m, n, n, A, lda, tau, lw);
}
int geqrf(cusolverDnHandle_t h, int m, int n, float* A, int lda, float* tau, float* w, int lw, int* info) {
  return (int)cusolverDnSgeqrf(h, m, n, A, lda, tau, w, lw, info);
}
int geqrf(cusolverDnHandle_t h, int m, int n, double* A, int lda, double* tau, double* w, int lw, int* info) {
  return (int)cusolverDnDgeqrf(h, m, n, A, lda, tau, w, lw, info);
}
int orgqr(cusolverDnHandle_t h, int m, int n, float* A, int lda, const float* tau, float* w, int lw, int* info) {
  return (int)cusolverDnSorgqr(h, m, n, n, A, lda, tau, w, lw, info);
}
int orgqr(cusolverDnHandle_t h, int m, int n, double* A, int lda, const double* tau, double* w, int lw, int* info) {
  return (int)cusolverDnDorgqr(h, m, n, n, A, lda, tau, w, lw, info);
}
int gemm_nn(cublasHandle_t h, int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C,
            int ldc) {
  const float one = 1.0f, zero = 0.0f;
  return (int)cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, A, lda, B, ldb, &zero, C, ldc);
}
int gemm_nn(cublasHandle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
            double* C, int ldc) {
  const double one = 1.0, zero = 0.0;
  return (int)cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, A, lda, B, ldb, &zero, C, ldc);
}

// The k x k upper triangle of src (ld lds) into dst (ld ldd), zeros below the diagonal.
template <typename T>
__global__ void k_copy_upper(T* dst, int64_t ldd, const T* src, int64_t lds, int k) {
  const int64_t total = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k), c = (int)(e / k);
    dst[r + c * ldd] = r <= c ? src[r + c * lds] : T(0);
  }
}

// Blocks handed to one cuSOLVER / cuBLAS call stay below 2^30 elements (their 32-bit
// interfaces index matrices with int).  TF_QR_BLOCK_ELEMS lowers the bound (tests use it
// to take the tall-skinny path on small problems).
int64_t qr_max_elems() {
  const int64_t cap = (int64_t)1 << 30;
  const char* v = getenv("TF_QR_BLOCK_ELEMS");
  if (!v) return cap;
  const long long x = atoll(v);
  return x >= 1 && x < cap ? (int64_t)x : cap;
}

// Householder QR of the column-major len x k block Y (ld = len) in place, Q kept.
template <typename T>
tf_status qr_inplace(Handles& h, DevMem& mem, T* Y, int64_t len, int k) {
  if (len * k > ((int64_t)1 << 30)) return api_fail(TF_EUNSUPPORTED, "QR block of %lld x %d too large", (long long)len, k);
  int lw1 = 0, lw2 = 0;
  T *tau, *work;
  int* info;
  TRY_CUDA(mem.get(&tau, k), "cudaMalloc(QR)");
  TRY_CUDA(mem.get(&info, 1), "cudaMalloc(QR)");
  TRY_LIB(geqrf_lwork(h.sol, (int)len, k, Y, (int)len, &lw1), "geqrf buffer");
  TRY_LIB(orgqr_lwork(h.sol, (int)len, k, Y, (int)len, tau, &lw2), "orgqr buffer");
  TRY_CUDA(mem.get(&work, std::max(lw1, lw2)), "cudaMalloc(QR)");
  TRY_LIB(geqrf(h.sol, (int)len, k, Y, (int)len, tau, work, std::max(lw1, lw2), info), "geqrf");
  TRY_LIB(orgqr(h.sol, (int)len, k, Y, (int)len, tau, work, std::max(lw1, lw2), info), "orgqr");
  return TF_OK;
}

// Buffers of the tall QR, allocated on first use and kept for the driver's later steps.
template <typename T> struct QrWork {
  T *W = nullptr, *W2 = nullptr, *Rs = nullptr, *tau = nullptr, *work = nullptr;
  int* info = nullptr;
  int lwork = 0;
};

// Rows of Y (k x len, row-major = column-major len x k) replaced by an orthonormal basis
// of their span (economic QR of Y^T, Q kept).  Needs k <= len.  A block above
// qr_max_elems() elements is factored as a tall-skinny QR: its nb row blocks Y_i = Q_i R_i each, the stacked
// [R_1; ...; R_nb] = Q_s R once more, and Q = diag(Q_i) Q_s (orthonormal, the same span).
template <typename T>
tf_status qr_rows(Handles& h, DevMem& mem, QrWork<T>& qw, T* Y, int64_t len, int k, cudaStream_t s) {
  const int64_t cap = qr_max_elems();
  if (len * k <= cap) return qr_inplace(h, mem, Y, len, k);
  const int nb = (int)((len * k + cap - 1) / cap);
  const int64_t L = (len + nb - 1) / nb;
  if (L < k || (int64_t)nb * k * k > ((int64_t)1 << 30))
    return api_fail(TF_EUNSUPPORTED, "QR of %lld x %d: row blocks shorter than the width", (long long)len, k);
  if (!qw.W) {
    TRY_CUDA(mem.get(&qw.W, (size_t)(L * k)), "cudaMalloc(QR blocks)");
    TRY_CUDA(mem.get(&qw.W2, (size_t)(L * k)), "cudaMalloc(QR blocks)");
    TRY_CUDA(mem.get(&qw.Rs, (size_t)nb * k * k), "cudaMalloc(QR blocks)");
    TRY_CUDA(mem.get(&qw.tau, k), "cudaMalloc(QR)");
    TRY_CUDA(mem.get(&qw.info, 1), "cudaMalloc(QR)");
    int lw1 = 0, lw2 = 0;
    TRY_LIB(geqrf_lwork(h.sol, (int)L, k, qw.W, (int)L, &lw1), "geqrf buffer");
    TRY_LIB(orgqr_lwork(h.sol, (int)L, k, qw.W, (int)L, qw.tau, &lw2), "orgqr buffer");
    qw.lwork = std::max(lw1, lw2);
    TRY_CUDA(mem.get(&qw.work, qw.lwork), "cudaMalloc(QR)");
  }
  const size_t es = sizeof(T);
  const int64_t ldr = (int64_t)nb * k;
  for (int i = 0; i < nb; ++i) {
    const int64_t r0 = i * L, Li = std::min<int64_t>(L, len - r0);
    TRY_CUDA(cudaMemcpy2DAsync(qw.W, Li * es, Y + r0, len * es, Li * es, k, cudaMemcpyDeviceToDevice, s), "copy");
    TRY_LIB(geqrf(h.sol, (int)Li, k, qw.W, (int)Li, qw.tau, qw.work, qw.lwork, qw.info), "geqrf");
    k_copy_upper<T><<<grid_for((int64_t)k * k), 256, 0, s>>>(qw.Rs + (int64_t)i * k, ldr, qw.W, Li, k);
    TRY_CUDA(cudaGetLastError(), "R copy");
    TRY_LIB(orgqr(h.sol, (int)Li, k, qw.W, (int)Li, qw.tau, qw.work, qw.lwork, qw.info), "orgqr");
    TRY_CUDA(cudaMemcpy2DAsync(Y + r0, len * es, qw.W, Li * es, Li * es, k, cudaMemcpyDeviceToDevice, s), "copy");
  }
  TRY_TF(qr_inplace(h, mem, qw.Rs, ldr, k));
  for (int i = 0; i < nb; ++i) {
    const int64_t r0 = i * L, Li = std::min<int64_t>(L, len - r0);
    TRY_CUDA(cudaMemcpy2DAsync(qw.W, Li * es, Y + r0, len * es, Li * es, k, cudaMemcpyDeviceToDevice, s), "copy");
    TRY_LIB(gemm_nn(h.blas, (int)Li, k, k, qw.W, (int)Li, qw.Rs + (int64_t)i * k, (int)ldr, qw.W2, (int)Li),
            "gemm(Q_i Q_s)");
    TRY_CUDA(cudaMemcpy2DAsync(Y + r0, len * es, qw.W2, Li * es, Li * es, k, cudaMemcpyDeviceToDevice, s), "copy");
  }
  return TF_OK;
}

template <typename T>
tf_status rsvd_run(tf_op* op, const tf_irls_params* p, const void* d_obs, const void* sigma,
                   const void* omega, void* m_out, tf_irls_report* rep, cudaStream_t s) {
  Irls<T> st;
  TRY_TF(tfk::op_info(op, &st.info));
  TRY_TF(check_params(p, st.info));
  const int64_t n = st.info.n, m = st.info.m;
  const int tp = p->tp, t = p->t;
  if (tp > std::min(n, m)) return api_fail(TF_EINVAL, "tf_rsvd needs tp <= min(m, n)");
  if (!omega) return api_fail(TF_EINVAL, "omega is NULL");
  TRY_TF(st.init(op, p, d_obs, sigma, s));
  Handles h;
  TRY_LIB(cusolverDnCreate(&h.sol), "cusolverDnCreate");
  TRY_LIB(cusolverDnSetStream(h.sol, s), "cusolverDnSetStream");
  TRY_LIB(cublasCreate(&h.blas), "cublasCreate");
  TRY_LIB(cublasSetStream(h.blas, s), "cublasSetStream");
  T *Q, *Q1, *Bt;
  double *Bd, *M, *W, *rtd, *btr, *coef;
  int* info;
  TRY_CUDA(st.mem.get(&Q, (size_t)tp * n), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&Q1, (size_t)tp * m), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&Bt, (size_t)tp * m), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&Bd, (size_t)tp * m), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&M, (size_t)tp * tp), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&W, tp), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&rtd, m), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&btr, tp), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&coef, tp), "cudaMalloc(RSVD)");
  TRY_CUDA(st.mem.get(&info, 1), "cudaMalloc(RSVD)");
  int lw = 0;
  TRY_LIB(cusolverDnDsyevd_bufferSize(h.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, tp, M, tp, W, &lw),
          "syevd buffer");
  double* ework;
  TRY_CUDA(st.mem.get(&ework, lw), "cudaMalloc(RSVD)");
  std::vector<double> D(tp), V((size_t)tp * tp), bt(tp), w(tp);
  QrWork<T> qn, qm;
  for (int k = 1; k <= p->kmax; ++k) {
    const double t0 = now_s();
    TRY_TF(st.begin(k));
    // Alg. 2 with one power iteration; blocks are row-major (row j = column j)
    TRY_TF(tf_rmatmat(op, tp, omega, m, Q, n, st.winv, st.wd, s));   // Y = Omega G~
    TRY_TF(qr_rows(h, st.mem, qn, Q, n, tp, s));                      // [Q, ~] = qr(Y^T)
    TRY_TF(tf_matmat(op, tp, Q, n, Q1, m, st.winv, st.wd, s));        // Y = G~ Q
    TRY_TF(qr_rows(h, st.mem, qm, Q1, m, tp, s));                     // [Q1, ~] = qr(Y)
    TRY_TF(tf_rmatmat(op, tp, Q1, m, Q, n, st.winv, st.wd, s));       // Y = Q1^T G~
    TRY_TF(qr_rows(h, st.mem, qn, Q, n, tp, s));                      // [Q, ~] = qr(Y^T)
    TRY_TF(tf_matmat(op, tp, Q, n, Bt, m, st.winv, st.wd, s));        // B = G~ Q
    // B^T B and B^T r~ in FP64, eigen-decomposition of B^T B
    k_to_f64<T><<<grid_for((int64_t)tp * m), 256, 0, s>>>(Bd, Bt, (int64_t)tp * m);
    k_to_f64<T><<<grid_for(m), 256, 0, s>>>(rtd, st.rt, m);
    TRY_CUDA(cudaGetLastError(), "conversion kernels");
    const double one = 1.0, zero = 0.0;
    TRY_LIB(cublasDgemm(h.blas, CUBLAS_OP_T, CUBLAS_OP_N, tp, tp, (int)m, &one, Bd, (int)m, Bd, (int)m, &zero, M, tp),
            "cublasDgemm(B^T B)");
    TRY_LIB(cublasDgemv(h.blas, CUBLAS_OP_T, (int)m, tp, &one, Bd, (int)m, rtd, 1, &zero, btr, 1),
            "cublasDgemv(B^T r)");
    TRY_LIB(cusolverDnDsyevd(h.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, tp, M, tp, W, ework, lw, info),
            "cusolverDnDsyevd");
    int dinfo = 0;
    TRY_CUDA(cudaMemcpyAsync(D.data(), W, tp * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaMemcpyAsync(V.data(), M, (size_t)tp * tp * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaMemcpyAsync(bt.data(), btr, tp * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaMemcpyAsync(&dinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    TRY_CUDA(cudaStreamSynchronize(s), "RSVD factorisation");
    if (dinfo != 0) return api_fail(TF_ENOTCONV, "tf_rsvd: eigen-decomposition failed (info %d)", dinfo);
    // S = sqrt|D| in descending order (stable), the t largest kept
    std::vector<double> S(tp);
    for (int i = 0; i < tp; ++i) S[i] = sqrt(fabs(D[i]));
    std::vector<int> order(tp);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return S[a] > S[b]; });
    std::vector<double> St(t), cf(t), c2(t);
    for (int j = 0; j < t; ++j) {  // coef_j = (V_j / S_j)^T (B^T r~)
      const int c = order[j];
      St[j] = S[c];
      double acc = 0.0;
      for (int i = 0; i < tp; ++i) acc += V[(size_t)c * tp + i] * bt[i];
      cf[j] = acc / St[j];
      c2[j] = cf[j] * cf[j];
    }
    double alpha;
    if (p->alphas) alpha = p->alphas[k - 1];
    else if (k == 1) alpha = alpha_start(n, m, St.data(), t);
    else alpha = choose_alpha(St.data(), c2.data(), t);
    // w = V_t (coef * S / (S^2 + alpha^2)); z = Q^T w (tf_rows_axpy subtracts: pass -w)
    std::fill(w.begin(), w.end(), 0.0);
    for (int j = 0; j < t; ++j) {
      const int c = order[j];
      const double f = cf[j] * St[j] / (St[j] * St[j] + alpha * alpha);
      for (int i = 0; i < tp; ++i) w[i] += V[(size_t)c * tp + i] * f;
    }
    for (double& v : w) v = -v;
    TRY_CUDA(cudaMemcpyAsync(coef, w.data(), tp * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    k_fill<T><<<grid_for(n), 256, 0, s>>>(st.z, T(0), n);
    TRY_TF(tf_rows_axpy(dtype_of<T>(), Q, n, tp, n, coef, st.z, s));
    double chi2 = 0;
    TRY_TF(st.finish(&chi2));
    report_step(rep, k, alpha, chi2, now_s() - t0);
    if (p->chi2_stop && chi2 <= m + sqrt(2.0 * m)) break;
  }
  TRY_CUDA(cudaMemcpyAsync(m_out, st.m1, n * sizeof(T), cudaMemcpyDeviceToDevice, s), "copy");
  TRY_CUDA(cudaStreamSynchronize(s), "tf_rsvd");
  return TF_OK;
}

tf_status check_args(tf_op* op, const void* d_obs, const void* sigma, void* m_out, tfk::OpInfo* info) {
  if (!op) return api_fail(TF_EINVAL, "op is NULL");
  if (!d_obs || !sigma || !m_out) return api_fail(TF_EINVAL, "d_obs, sigma and m_out must be non-NULL");
  return tfk::op_info(op, info);
}

}  // namespace

extern "C" {

tf_status tf_gkb(tf_op* op, const tf_irls_params* params, const void* d_obs, const void* sigma,
                 void* m_out, tf_irls_report* report, tf_stream stream) {
  tfk::OpInfo info;
  TRY_TF(check_args(op, d_obs, sigma, m_out, &info));
  if (report) report->iterations = 0;
  cudaStream_t s = (cudaStream_t)stream;
  return info.dtype == TF_F32 ? gkb_run<float>(op, params, d_obs, sigma, m_out, report, s)
                              : gkb_run<double>(op, params, d_obs, sigma, m_out, report, s);
}

tf_status tf_rsvd(tf_op* op, const tf_irls_params* params, const void* d_obs, const void* sigma,
                  const void* omega, void* m_out, tf_irls_report* report, tf_stream stream) {
  tfk::OpInfo info;
  TRY_TF(check_args(op, d_obs, sigma, m_out, &info));
  if (report) report->iterations = 0;
  cudaStream_t s = (cudaStream_t)stream;
  return info.dtype == TF_F32 ? rsvd_run<float>(op, params, d_obs, sigma, omega, m_out, report, s)
                              : rsvd_run<double>(op, params, d_obs, sigma, omega, m_out, report, s);
}

tf_status tf_tridiag_eig_first(int n, double* d, double* e, double* first) {
  if (n < 0 || (n > 0 && (!d || !e || !first))) return api_fail(TF_EINVAL, "need n >= 0 and non-NULL arrays");
  if (!tridiag_ql_first(n, d, e, first))
    return api_fail(TF_ENOTCONV, "tridiagonal eigenvalue iteration did not converge");
  return TF_OK;
}

tf_status tf_damped_bidiag_solve(int tp, const double* gam, const double* bet, double alpha, double b0,
                                 double* y) {
  if (tp < 1 || !gam || !bet || !y) return api_fail(TF_EINVAL, "need tp >= 1 and non-NULL arrays");
  damped_bidiag_solve(tp, gam, bet, alpha, b0, y);
  return TF_OK;
}

}  // extern "C"
