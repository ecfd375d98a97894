// Mixed-radix Stockham FFT engine staged through shared memory (device code).
//
// The 2-D FFTs of App. A ("the 2DFFT of W is computed as 1DFFT((1DFFT(W))^T)^T") are
// evaluated here as batches of 1-D transforms: a CTA holds TB independent sequences of
// length N as a [N][ld] array (sequence index fastest), and every radix-R pass moves
// each element once through registers (load R values at stride N/R, twiddle, radix-R
// butterfly, store with Stockham's self-sorting index).  The first pass may read its
// input through a caller functor (global memory, zero padding, a spectral product) and
// the last pass may write through one (a layer accumulation, a windowed global store),
// so that those steps cost no extra shared-memory round trip.
//
// Forward transforms use exp(-2 pi i n k / N); inverse transforms use the conjugate and
// are unnormalised (the 1/(N1 N2) factor is folded into the stored layer spectra).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tf_check.cuh"

namespace tfk {

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 C; };
template <> struct CT<double> { typedef double2 C; };

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// cos / sin of 2 pi m / R for the odd radices (mathematical constants, 25 digits)
template <int R> __device__ __forceinline__ double cs_cos(int m);
template <int R> __device__ __forceinline__ double cs_sin(int m);
template <> __device__ __forceinline__ double cs_cos<3>(int m) { return -0.5; }
template <> __device__ __forceinline__ double cs_sin<3>(int m) { return m == 1 ? 0.8660254037844386467637232 : -0.8660254037844386467637232; }
template <> __device__ __forceinline__ double cs_cos<5>(int m) {
  return (m == 1 || m == 4) ? 0.3090169943749474241022934 : -0.8090169943749474241022934;
}
template <> __device__ __forceinline__ double cs_sin<5>(int m) {
  return m == 1 ? 0.9510565162951535721164393 : m == 2 ? 0.5877852522924731291687060
       : m == 3 ? -0.5877852522924731291687060 : -0.9510565162951535721164393;
}
template <> __device__ __forceinline__ double cs_cos<7>(int m) {
  return (m == 1 || m == 6) ? 0.6234898018587335305250049
       : (m == 2 || m == 5) ? -0.2225209339563144042889026 : -0.9009688679024191262361023;
}
template <> __device__ __forceinline__ double cs_sin<7>(int m) {
  return m == 1 ? 0.7818314824680298087084445 : m == 2 ? 0.9749279121818236070181317
       : m == 3 ? 0.4338837391175581204757683 : m == 4 ? -0.4338837391175581204757683
       : m == 5 ? -0.9749279121818236070181317 : -0.7818314824680298087084445;
}

// Odd-radix DFT from the symmetric/antisymmetric pairs a_n +- a_{R-n}.
template <int R, bool INV, typename C> __device__ __forceinline__ void dft_odd(C* v) {
  typedef decltype(C::x) T;
  constexpr int H = (R - 1) / 2;
  C s[H + 1], d[H + 1];
  C y0 = v[0];
#pragma unroll
  for (int n = 1; n <= H; ++n) {
    s[n] = cadd(v[n], v[R - n]);
    d[n] = csub(v[n], v[R - n]);
    y0 = cadd(y0, s[n]);
  }
  C out[R];
  out[0] = y0;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    C A = v[0], B = mk<C>(T(0), T(0));
#pragma unroll
    for (int n = 1; n <= H; ++n) {
      const T c = T(cs_cos<R>((n * k) % R));
      const T sn = T(cs_sin<R>((n * k) % R));
      A = mk<C>(A.x + c * s[n].x, A.y + c * s[n].y);
      B = mk<C>(B.x + sn * d[n].x, B.y + sn * d[n].y);
    }
    // forward: y_k = A - iB, y_{R-k} = A + iB ; inverse: signs swapped
    const C iB = mk<C>(-B.y, B.x);
    out[k] = INV ? cadd(A, iB) : csub(A, iB);
    out[R - k] = INV ? csub(A, iB) : cadd(A, iB);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <int R, bool INV, typename C> struct Dft;
template <bool INV, typename C> struct Dft<2, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};
template <bool INV, typename C> struct Dft<4, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    C s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13); v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13); v[3] = csub(d02, d13);
  }
};
template <bool INV, typename C> struct Dft<8, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    typedef decltype(C::x) T;
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV, C>::run(e);
    Dft<4, INV, C>::run(o);
    const T h = T(0.7071067811865475244008444);
    // w8^1 = h(1 -+ i), w8^2 = -+i, w8^3 = h(-1 -+ i)
    C o1 = INV ? mk<C>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
               : mk<C>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    C o2 = mul_mi<INV>(o[2]);
    C o3 = INV ? mk<C>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
               : mk<C>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
};
template <bool INV, typename C> struct Dft<3, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_odd<3, INV>(v); }
};
template <bool INV, typename C> struct Dft<5, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_odd<5, INV>(v); }
};
template <bool INV, typename C> struct Dft<7, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_odd<7, INV>(v); }
};

// cos and sin of 2 pi m / R as compile-time constants.  The fraction m / R is reduced,
// in integers, to an angle in [0, pi/4] by the symmetries of the circle, whose sine and
// cosine are then summed from their Taylor series (terms to x^27, below 1e-18 there).
namespace trig {
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k <= 13; ++k) { t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0)); s += t; }
  return s;
}
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k <= 13; ++k) { t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k)); s += t; }
  return s;
}
// (cos, sin)(2 pi num / den) for 0 <= num / den <= 1/8 is the Taylor pair; larger
// fractions fold onto it: f -> 1 - f (sin flips), f -> 1/2 - f (cos flips), f -> 1/4 - f
// (cos and sin swap).
constexpr double cos_frac(long long num, long long den, bool want_sin) {
  num %= den;
  if (num < 0) num += den;
  double sign = 1.0;
  if (2 * num > den) {            // f in (1/2, 1): cos(2 pi f) = cos(2 pi (1 - f))
    num = den - num;
    if (want_sin) sign = -sign;
  }
  if (4 * num > den) {            // f in (1/4, 1/2]: cos = -cos(2 pi (1/2 - f)), sin same
    num = den - 2 * num;
    den *= 2;
    if (!want_sin) sign = -sign;
  }
  if (8 * num > den) {            // f in (1/8, 1/4]: cos = sin(2 pi (1/4 - f)) and vice versa
    num = den - 4 * num;
    den *= 4;
    want_sin = !want_sin;
  }
  const double x = kTwoPi * (double)num / (double)den;
  return sign * (want_sin ? taylor_sin(x) : taylor_cos(x));
}
constexpr double cos2pi(int m, int R) { return cos_frac(m, R, false); }
constexpr double sin2pi(int m, int R) { return cos_frac(m, R, true); }
}  // namespace trig

// Radix R = P Q from length-P and length-Q transforms (Cooley-Tukey within a thread):
// X[k1 + P k2] = sum_n2 w_Q^(n2 k2) w_R^(n2 k1) sum_n1 w_P^(n1 k1) x[Q n1 + n2].
// Twiddles w_R^m = exp(-+ 2 pi i m / R) are compile-time constants; multiples of a
// quarter turn are applied as sign swaps.
template <int P, int Q, bool INV, typename C> struct DftPQ {
  static __device__ __forceinline__ void run(C* v) {
    typedef decltype(C::x) T;
    constexpr int R = P * Q;
    C y[Q][P];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) y[n2][n1] = v[Q * n1 + n2];
      Dft<P, INV, C>::run(y[n2]);
#pragma unroll
      for (int k1 = 1; k1 < P; ++k1) {
        const int m = (n2 * k1) % R;
        if (m == 0) continue;
        const C a = y[n2][k1];
        if (4 * m == R) {              // w = -+i
          y[n2][k1] = mul_mi<INV>(a);
        } else if (2 * m == R) {       // w = -1
          y[n2][k1] = mk<C>(-a.x, -a.y);
        } else if (4 * m == 3 * R) {   // w = +-i
          y[n2][k1] = mul_mi<!INV>(a);
        } else {
          const T c = T(trig::cos2pi(m, R)), s = T(trig::sin2pi(m, R));
          y[n2][k1] = cmul(a, mk<C>(c, INV ? s : -s));
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      C z[Q];
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) z[n2] = y[n2][k1];
      Dft<Q, INV, C>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = z[k2];
    }
  }
};
// Radix 16 as 4 x 4 (outputs k1 + 4 k2) and radix 14 as 2 x 7 (even and odd
// subsequences, outputs k and k + 7).
template <bool INV, typename C> struct Dft<16, INV, C> : DftPQ<4, 4, INV, C> {};
template <bool INV, typename C> struct Dft<14, INV, C> : DftPQ<7, 2, INV, C> {};

constexpr int kMaxPass = 16;

// A 1-D transform of length n as np radix passes.  Pass p has radix radix[p], stride
// ns[p] = product of the earlier radices, and its twiddles w^(r k), k < ns[p],
// 1 <= r < radix[p], stored at tw[tw_off[p] + k (radix[p]-1) + r - 1] with
// w = exp(-2 pi i / (ns[p] radix[p])).  The table holds n - 1 entries in total.
struct FftPlan {
  int n;
  int np;
  int tw_count;
  int radix[kMaxPass];
  int ns[kMaxPass];
  int tw_off[kMaxPass];
};

// One Stockham pass over TB = 2^tbs interleaved sequences.
template <int R, bool INV, typename C, class L, class S>
__device__ __forceinline__ void fft_pass(int nb, int Ns, int tbs, const C* __restrict__ tw,
                                         const L& load, const S& store) {
  const int tbm = (1 << tbs) - 1;
  const int total = nb << tbs;
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    const int j = u >> tbs, b = u & tbm;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = load(j + r * nb, b);
    if (Ns > 1) {
      const C* t = tw + k * (R - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = t[r - 1];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Dft<R, INV, C>::run(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) store(base + r * Ns, b, v[r]);
  }
}

template <bool INV, typename C, class L, class S>
__device__ __forceinline__ void fft_pass_any(int R, int nb, int Ns, int tbs, const C* tw,
                                             const L& load, const S& store) {
  switch (R) {
    case 2: fft_pass<2, INV>(nb, Ns, tbs, tw, load, store); break;
    case 3: fft_pass<3, INV>(nb, Ns, tbs, tw, load, store); break;
    case 4: fft_pass<4, INV>(nb, Ns, tbs, tw, load, store); break;
    case 5: fft_pass<5, INV>(nb, Ns, tbs, tw, load, store); break;
    case 7: fft_pass<7, INV>(nb, Ns, tbs, tw, load, store); break;
    default: fft_pass<8, INV>(nb, Ns, tbs, tw, load, store); break;
  }
}

template <typename C> struct SmemLoad {
  const C* p; int ld; int ext;
  __device__ __forceinline__ C operator()(int idx, int b) const {
    C v; v.x = 0; v.y = 0;
    if (TF_IN(kSiteSmem + 100, idx * ld + b, ext)) v = p[idx * ld + b];
    return v;
  }
};
template <typename C> struct SmemStore {
  C* p; int ld; int ext;
  __device__ __forceinline__ void operator()(int idx, int b, C v) const {
    if (TF_IN(kSiteSmem + 100, idx * ld + b, ext)) p[idx * ld + b] = v;
  }
};

// Full transform: pass 0 reads through `first`, the last pass writes through `last`,
// intermediate passes ping-pong between bufA (even passes write) and bufB (odd).
// Every pass ends with __syncthreads().  Callers synchronise before the first pass
// if `first` reads shared memory written earlier.
template <bool INV, typename C, class L0, class SL>
__device__ __forceinline__ void fft_run(const FftPlan& P, const C* tw, C* bufA, C* bufB, int ld,
                                        int tbs, const L0& first, const SL& last) {
  for (int p = 0; p < P.np; ++p) {
    const int R = P.radix[p];
    const int nb = P.n / R;
    const int Ns = P.ns[p];
    const C* twp = tw + P.tw_off[p];
    SmemLoad<C> sl{(p & 1) ? bufA : bufB, ld, P.n * ld};
    SmemStore<C> ss{(p & 1) ? bufB : bufA, ld, P.n * ld};
    const bool f = (p == 0), l = (p == P.np - 1);
    if (f && l) fft_pass_any<INV>(R, nb, Ns, tbs, twp, first, last);
    else if (f) fft_pass_any<INV>(R, nb, Ns, tbs, twp, first, ss);
    else if (l) fft_pass_any<INV>(R, nb, Ns, tbs, twp, sl, last);
    else fft_pass_any<INV>(R, nb, Ns, tbs, twp, sl, ss);
    __syncthreads();
  }
}

}  // namespace tfk
