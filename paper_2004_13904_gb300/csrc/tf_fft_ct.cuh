// Compile-time-sized Stockham FFT passes (device code) for the product kernels.
//
// Same transform as tf_fft.cuh (a batch of TB interleaved length-N sequences in a
// [N][TB] shared-memory array, radix-R passes with Stockham's self-sorting index), but
// N, the radix list, every stride and the thread count are template constants, so the
// index arithmetic folds to shifts and constant multiplies.  Each thread transforms V
// adjacent sequences at once: they share the twiddle factors and move through shared
// memory as one 8*V-byte access.  Passes are in place: a thread loads its inputs,
// computes, waits at a barrier, then stores, so one buffer serves all passes.
#pragma once
#include <type_traits>

#include "tf_check.cuh"
#include "tf_fft.cuh"

namespace tfk {
namespace ct {

// V consecutive complex values to / from shared memory
template <int V, typename C> struct Vec {
  static __device__ __forceinline__ void ld(const C* p, C* o) {
#pragma unroll
    for (int i = 0; i < V; ++i) o[i] = p[i];
  }
  static __device__ __forceinline__ void st(C* p, const C* v) {
#pragma unroll
    for (int i = 0; i < V; ++i) p[i] = v[i];
  }
};
template <> struct Vec<2, float2> {
  static __device__ __forceinline__ void ld(const float2* p, float2* o) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = make_float2(t.x, t.y);
    o[1] = make_float2(t.z, t.w);
  }
  static __device__ __forceinline__ void st(float2* p, const float2* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  }
};
template <> struct Vec<4, float2> {
  static __device__ __forceinline__ void ld(const float2* p, float2* o) {
    Vec<2, float2>::ld(p, o);
    Vec<2, float2>::ld(p + 2, o + 2);
  }
  static __device__ __forceinline__ void st(float2* p, const float2* v) {
    Vec<2, float2>::st(p, v);
    Vec<2, float2>::st(p + 2, v + 2);
  }
};

// Position of sequence b at element idx in the [N][TB] working buffer.  The sequence
// index is XOR-swizzled by an even function of the row, so that walking idx at fixed b
// (the staging and unpacking phases) spreads over the shared-memory banks instead of
// hitting one bank group, while pairs (2k, 2k+1) stay adjacent for 16-byte accesses.
template <typename C, int TB> __host__ __device__ constexpr int swz(int row) {
  constexpr int rows_per_line = (int)(128 / (TB * sizeof(C))) > 1 ? (int)(128 / (TB * sizeof(C))) : 1;
  return TB >= 4 ? ((row / rows_per_line) & (TB / 2 - 1)) << 1 : 0;
}
// Rows of 128/q bytes (q = 2 or 4) fill 1/q of the 32 banks, the part given by the row
// index mod q.  The first pass of a plan with first radix S stores rows idx, idx + S,
// idx + 2S, ... in the same quarter-warp phase; XOR-ing the low bits of the row with the
// block number (idx / S) mod q puts q consecutive blocks in different bank parts.  (A
// permutation of [0, N) for N divisible by q.)
template <typename C, int TB, int S = 8> __host__ __device__ constexpr int row_of(int idx) {
  constexpr int q = TB * (int)sizeof(C) == 64 ? 2 : TB * (int)sizeof(C) == 32 ? 4 : 1;
  return q > 1 ? idx ^ ((idx / S) & (q - 1)) : idx;
}
template <typename C, int TB, int S = 8> __host__ __device__ constexpr int at(int idx, int b) {
  const int row = row_of<C, TB, S>(idx);
  return row * TB + (b ^ swz<C, TB>(row));
}

// How the R positions idx = f + r st of one task (f its first index) move in the buffer,
// checked over every task of a pass at compile time: 1 when at(f + r st, b) = at(f, b) +
// r st TB for all r and b (the addresses are one base plus constant offsets), 2 when that
// holds separately for even r (base at(f)) and odd r (base at(f + st)), 0 otherwise.
// Loads of a pass have f = j, st = NB; its stores f = (j - j mod Ns) R + j mod Ns, st = Ns.
// (A third form for the first pass's stores, two bases plus a per-element XOR of the
// sequence index, measured no faster at n = 448 and slower for the radix-16 first pass.)
template <typename C, int TB, int S>
constexpr int step_mode(int NB, int R, int Ns, bool store) {
  const int st = store ? Ns : NB;
  bool one = true, two = true;
  for (int j = 0; j < NB && (one || two); ++j) {
    const int f = store ? (j - j % Ns) * R + j % Ns : j;
    for (int b = 0; b < TB; ++b)
      for (int r = 0; r < R; ++r) {
        const int e = at<C, TB, S>(f + r * st, b);
        if (e != at<C, TB, S>(f, b) + r * st * TB) one = false;
        if (e != at<C, TB, S>(f + (r & 1) * st, b) + (r - (r & 1)) * st * TB) two = false;
      }
  }
  return one ? 1 : two ? 2 : 0;
}
template <typename C, int TB, int S, int NB, int R, int Ns, bool STORE>
constexpr int kStepMode = step_mode<C, TB, S>(NB, R, Ns, STORE);


// at(idx, b) for a fixed idx and varying even b: the row's base and swizzle computed once.
template <typename C, int TB, int S = 8> struct RowAt {
  int base, sw;
  __device__ __forceinline__ explicit RowAt(int idx) {
    const int row = row_of<C, TB, S>(idx);
    base = row * TB;
    sw = swz<C, TB>(row);
  }
  __device__ __forceinline__ int operator()(int b) const { return base + (b ^ sw); }
};

// The working buffer: [N][TB] complex, sequence index fastest (swizzled).
// STEP (bit 0 loads, bit 1 stores): a pass whose loads / stores go through this buffer
// computes each task's positions from one or two bases (step_mode) instead of per element;
// kernels with a tight register budget keep the per-element form, which needs fewer live
// registers.
// SLOT names the buffer: a pass whose loads and stores go through Buf's of the same slot
// works in place (a barrier between its loads and its stores).
template <typename C, int TB, int V, int S = 8, int STEP = 0, int SLOT = 0> struct Buf {
  static constexpr bool kIsBuf = true;
  static constexpr int kStep = STEP, kSlot = SLOT;
  static constexpr int kTB = TB, kS = S;
  C* p;
  int ext;  // elements of the buffer (checked builds test every access against it)
  __device__ __forceinline__ void operator()(int idx, int b0, C* o) const {
    const int e = at<C, TB, S>(idx, b0);
    if (TF_IN(kSiteSmem, e + V - 1, ext) && TF_IN(kSiteSmem, e, ext)) Vec<V, C>::ld(p + e, o);
  }
  __device__ __forceinline__ void operator()(int idx, int b0, const C* v, int) const {
    const int e = at<C, TB, S>(idx, b0);
    if (TF_IN(kSiteSmem, e + V - 1, ext) && TF_IN(kSiteSmem, e, ext)) Vec<V, C>::st(p + e, v);
  }
};

template <class T, class = void> struct IsBuf : std::false_type {};
template <class T> struct IsBuf<T, std::void_t<decltype(T::kIsBuf)>> : std::true_type {};
// A loader that marks itself with kTaskLoad supplies a first pass's R inputs of one task
// at once: task<R, NB>(j, b0, v) fills v[q][r] with element j + r NB of sequence b0 + q.
template <class T, class = void> struct IsTaskLoad : std::false_type {};
template <class T> struct IsTaskLoad<T, std::void_t<decltype(T::kTaskLoad)>> : std::true_type {};
template <class L, class S, bool = IsBuf<L>::value && IsBuf<S>::value> struct SameBuf : std::false_type {};
template <class L, class S> struct SameBuf<L, S, true> : std::bool_constant<L::kSlot == S::kSlot> {};

// step_mode of a pass's buffer loads / stores (0 for other loaders and storers).
template <class L, typename C, int NB, int R, bool = IsBuf<L>::value> struct LoadMode {
  static constexpr int value = 0;
};
template <class L, typename C, int NB, int R> struct LoadMode<L, C, NB, R, true> {
  static constexpr int value = (L::kStep & 1) ? kStepMode<C, L::kTB, L::kS, NB, R, 1, false> : 0;
};
template <class S, typename C, int NB, int R, int Ns, bool = IsBuf<S>::value> struct StoreMode {
  static constexpr int value = 0;
};
template <class S, typename C, int NB, int R, int Ns> struct StoreMode<S, C, NB, R, Ns, true> {
  static constexpr int value = (S::kStep & 2) ? kStepMode<C, S::kTB, S::kS, NB, R, Ns, true> : 0;
};

// The task -> (output index, sequence) mapping of a pass, as the pass computes it: task
// u writes first_idx(u) + r * Ns, r < R, for sequences b0 .. b0 + V - 1.
template <int R, int Ns, int N, int TB, int V> struct PassMap {
  static constexpr int NB = N / R, G = TB / V, TOTAL = NB * G;
  __device__ __forceinline__ static int first_idx(int u, int& b0) {
    const int j = u / G;
    b0 = (u % G) * V;
    const int k = j % Ns;
    return (j - k) * R + k;
  }
};

// One radix-R pass with stride Ns over TB sequences, V per thread, NT threads.
// Loader: ld(idx, b0, C out[V]); storer: st(idx, b0, const C in[V], slot) where slot =
// it * R + r numbers the thread's outputs of the pass (a compile-time constant).
// Radix-R butterfly whose inputs r >= R/2 are zero (first pass of a zero-upper-half
// sequence): the same outputs as Dft<R> without the additions of those zeros.
template <int R, bool INV, typename C> struct DftZhi {
  static __device__ __forceinline__ void run(C* v) { Dft<R, INV, C>::run(v); }
};
template <bool INV, typename C> struct DftZhi<8, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    typedef decltype(C::x) T;
    // length-4 transforms of (v0, v2, 0, 0) and (v1, v3, 0, 0)
    const C m2 = mul_mi<INV>(v[2]), m3 = mul_mi<INV>(v[3]);
    const C e[4] = {cadd(v[0], v[2]), cadd(v[0], m2), csub(v[0], v[2]), csub(v[0], m2)};
    const C o[4] = {cadd(v[1], v[3]), cadd(v[1], m3), csub(v[1], v[3]), csub(v[1], m3)};
    const T h = T(0.7071067811865475244008444);
    const C o1 = INV ? mk<C>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                     : mk<C>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    const C o2 = mul_mi<INV>(o[2]);
    const C o3 = INV ? mk<C>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                     : mk<C>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
};

// ZHI (first pass only, R even): the inputs of the upper half, rows >= N/2 (the r >= R/2
// inputs of every task), are known zeros; they are neither loaded nor computed with.
template <int R, int Ns, int N, int TB, int V, int NT, bool INV, bool ZHI = false, typename C, class L, class S>
__device__ __forceinline__ void pass(const C* __restrict__ tw, const L& ld, const S& st) {
  static_assert(!ZHI || (Ns == 1 && R % 2 == 0), "zero upper half needs an even first radix");
  constexpr int NB = N / R;
  constexpr int G = TB / V;
  constexpr int TOTAL = NB * G;
  constexpr int ITER = (TOTAL + NT - 1) / NT;
  constexpr bool kInPlace = SameBuf<L, S>::value;
  C v[ITER][V][R];
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int u = threadIdx.x + it * NT;
    if (TOTAL % NT == 0 || u < TOTAL) {
      const int j = u / G, b0 = (u % G) * V;
      constexpr int LMODE = LoadMode<L, C, NB, R>::value;
      int e0 = 0, e1 = 0;
      if constexpr (LMODE > 0) {
        e0 = at<C, TB, L::kS>(j, b0);
        if constexpr (LMODE == 2) e1 = at<C, TB, L::kS>(j + NB, b0);
      }
      if constexpr (IsTaskLoad<L>::value) {
        static_assert(Ns == 1 && !ZHI, "task loaders feed first passes");
        ld.template task<R, NB>(j, b0, v[it]);
      } else
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C t[V];
        if (ZHI && r >= R / 2) {
#pragma unroll
          for (int q = 0; q < V; ++q) t[q] = mk<C>(0, 0);
        } else if constexpr (LMODE > 0) {
          const int e = (LMODE == 2 && (r & 1)) ? e1 + (r - 1) * NB * TB : e0 + r * NB * TB;
          if (TF_IN(kSiteSmem, e + V - 1, ld.ext) && TF_IN(kSiteSmem, e, ld.ext)) Vec<V, C>::ld(ld.p + e, t);
        } else {
          ld(j + r * NB, b0, t);
        }
#pragma unroll
        for (int q = 0; q < V; ++q) v[it][q][r] = t[q];
      }
      if (Ns > 1) {
        const int k = j % Ns;
        const C* w = tw + k * (R - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C f = mk<C>(1, 0);
          if (TF_IN(kSiteSmem + 1, (int)(w - tw) + r - 1, Ns * (R - 1))) f = w[r - 1];
          if (INV) f.y = -f.y;
#pragma unroll
          for (int q = 0; q < V; ++q) v[it][q][r] = cmul(v[it][q][r], f);
        }
      }
#pragma unroll
      for (int q = 0; q < V; ++q) {
        if constexpr (ZHI) DftZhi<R, INV, C>::run(v[it][q]);
        else Dft<R, INV, C>::run(v[it][q]);
      }
    }
  }
  if (kInPlace) __syncthreads();
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int u = threadIdx.x + it * NT;
    if (TOTAL % NT == 0 || u < TOTAL) {
      int b0;
      const int base = PassMap<R, Ns, N, TB, V>::first_idx(u, b0);
      constexpr int SMODE = StoreMode<S, C, NB, R, Ns>::value;
      int e0 = 0, e1 = 0;
      if constexpr (SMODE > 0) {
        e0 = at<C, TB, S::kS>(base, b0);
        if constexpr (SMODE == 2) e1 = at<C, TB, S::kS>(base + Ns, b0);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C t[V];
#pragma unroll
        for (int q = 0; q < V; ++q) t[q] = v[it][q][r];
        if constexpr (SMODE > 0) {
          const int e = (SMODE == 2 && (r & 1)) ? e1 + (r - 1) * Ns * TB : e0 + r * Ns * TB;
          if (TF_IN(kSiteSmem, e + V - 1, st.ext) && TF_IN(kSiteSmem, e, st.ext)) Vec<V, C>::st(st.p + e, t);
        } else {
          st(base + r * Ns, b0, t, it * R + r);
        }
      }
    }
  }
  __syncthreads();
}

// Passes of a radix list; pass 0 loads through `first`, the last pass stores through
// `last`, the others use the shared buffer.  Twiddle layout as in FftPlan.
template <int N, int Ns, int TwOff, int... Rs> struct Run;
// Pass K of a plan stores into buffer slot (PP ? K mod 2 : 0) and loads from the slot
// the previous pass stored into; with PP (two buffers, bufs[0] and bufs[1]) consecutive
// passes alternate slots and need no barrier between their loads and stores.
// A hook runs (in every thread) after the first pass's closing barrier, when the first
// loader's source is no longer read.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};
template <int N, int Ns, int TwOff, int R, int... Rest> struct Run<N, Ns, TwOff, R, Rest...> {
  template <int TB, int V, int NT, bool INV, bool FIRST, bool ZHI, int S, int STEP, bool PP, int K, typename C,
            class L0, class SL, class H>
  static __device__ __forceinline__ void go(const C* tw, C* const* bufs, const L0& first, const SL& last,
                                            const H& hook) {
    constexpr bool LAST = sizeof...(Rest) == 0;
    constexpr int SO = PP ? K % 2 : 0, SI = PP ? (K + 1) % 2 : 0;
    const Buf<C, TB, V, S, STEP, SO> bo{bufs[SO], N * TB};
    const Buf<C, TB, V, S, STEP, SI> bi{bufs[SI], N * TB};
    if constexpr (FIRST && LAST) pass<R, Ns, N, TB, V, NT, INV, ZHI>(tw + TwOff, first, last);
    else if constexpr (FIRST) pass<R, Ns, N, TB, V, NT, INV, ZHI>(tw + TwOff, first, bo);
    else if constexpr (LAST) pass<R, Ns, N, TB, V, NT, INV>(tw + TwOff, bi, last);
    else pass<R, Ns, N, TB, V, NT, INV>(tw + TwOff, bi, bo);
    if constexpr (FIRST) hook();
    if constexpr (!LAST)
      Run<N, Ns * R, TwOff + Ns * (R - 1), Rest...>::template go<TB, V, NT, INV, false, false, S, STEP, PP,
                                                                   K + 1>(tw, bufs, first, last, hook);
  }
};

template <int... Rs> struct LastOf;
template <int R> struct LastOf<R> { static constexpr int r = R, prod_before = 1; };
template <int R, int... Rest> struct LastOf<R, Rest...> {
  static constexpr int r = LastOf<Rest...>::r;
  static constexpr int prod_before = R * LastOf<Rest...>::prod_before;
};

template <int R, int... Rest> struct FirstOf { static constexpr int r = R; };

template <int N, int... Rs> struct Plan {
  static constexpr int n = N;
  static constexpr int npasses = (int)sizeof...(Rs);
  static constexpr int last_r = LastOf<Rs...>::r;          // radix of the last pass
  static constexpr int last_ns = LastOf<Rs...>::prod_before;  // its stride
  // The upper half of the input may be declared zero (run<..., ZHI = true>) when the
  // first radix is even.
  static constexpr int first_r = FirstOf<Rs...>::r;        // radix of the first pass
  static constexpr bool can_zero_hi = first_r % 2 == 0;
  template <int TB, int V, int NT, bool INV, bool ZHI = false, int STEP = 0, typename C, class L0, class SL>
  static __device__ __forceinline__ void run(const C* tw, C* buf, const L0& first, const SL& last) {
    C* const bufs[2] = {buf, buf};
    Run<N, 1, 0, Rs...>::template go<TB, V, NT, INV, true, ZHI && can_zero_hi, first_r, STEP, false, 0>(
        tw, bufs, first, last, NoHook{});
  }
  // run with a hook after the first pass
  template <int TB, int V, int NT, bool INV, bool ZHI = false, int STEP = 0, typename C, class L0, class SL, class H>
  static __device__ __forceinline__ void run_h(const C* tw, C* buf, const L0& first, const SL& last, const H& hook) {
    C* const bufs[2] = {buf, buf};
    Run<N, 1, 0, Rs...>::template go<TB, V, NT, INV, true, ZHI && can_zero_hi, first_r, STEP, false, 0>(
        tw, bufs, first, last, hook);
  }
  // The same with two buffers: pass K stores into slot K mod 2 (a first loader that is a
  // Buf of slot 1 reads bufs[1]).
  template <int TB, int V, int NT, bool INV, bool ZHI = false, int STEP = 0, typename C, class L0, class SL>
  static __device__ __forceinline__ void run2(const C* tw, C* buf0, C* buf1, const L0& first, const SL& last) {
    C* const bufs[2] = {buf0, buf1};
    Run<N, 1, 0, Rs...>::template go<TB, V, NT, INV, true, ZHI && can_zero_hi, first_r, STEP, true, 0>(
        tw, bufs, first, last, NoHook{});
  }
};

}  // namespace ct
}  // namespace tfk
