// Shared-memory Stockham FFT engine for the PM solver (sm_103a).
//
// One thread block transforms a batch of independent 1-D sequences of length N.  Each thread
// owns E elements (E/R butterflies of radix R per stage); T = N/E threads cooperate on one
// sequence.  The first stage reads its inputs straight from the caller (global memory or
// shared memory), the last stage writes straight to the caller; intermediate stages exchange
// through shared memory (Stockham autosort: output in natural order, no bit reversal).
//
// Conventions: forward = exp(-2 pi i n k / N), inverse = exp(+2 pi i n k / N), neither scaled.
// Twiddles come from a float2 table tw[m] = exp(-2 pi i m / NT) computed in float64 on the
// host; stage twiddles exp(-2 pi i m / N) are read at tw[m * TWS] with NT = N * TWS.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

namespace cola {

// Complex arithmetic with every rounding spelled out (__fadd_rn / __fmul_rn are never fused
// into an FMA by the compiler): a kernel body then rounds identically in every kernel it is
// inlined into, so the single-box and the ensemble kernels give bit-identical results.
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, __fmul_rn(-a.y, b.y)), fmaf(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s)); }
// multiply by -i (forward sign) or +i (inverse sign)
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Compile-time sine/cosine (Taylor series in double; arguments in [0, 2 pi)) for the constant
// twiddles inside the small in-register DFTs.
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double cx_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 40; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
constexpr double cx_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 40; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}

template <int R, int K, bool INV>
struct ConstTw {
  static constexpr float re = (float)cx_cos(2.0 * kPi * K / R);
  static constexpr float im = (INV ? 1.0f : -1.0f) * (float)cx_sin(2.0 * kPi * K / R);
};

// y <- x * exp(-+2 pi i K / R), with the trivial angles special-cased
template <int R, int K, bool INV>
__device__ __forceinline__ float2 mul_const_tw(float2 x) {
  if constexpr (K == 0) {
    return x;
  } else if constexpr (4 * K == R) {
    return c_rot<INV>(x);
  } else {
    return c_mul(x, make_float2(ConstTw<R, K, INV>::re, ConstTw<R, K, INV>::im));
  }
}

// ---- small in-register DFTs -------------------------------------------------------------
template <int R, bool INV>
struct DFT;

template <bool INV>
struct DFT<2, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
  }
};

template <bool INV>
struct DFT<3, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    // omega = exp(-+2 pi i / 3) = -1/2 + i s,  s = -+sqrt(3)/2
    constexpr float s = INV ? 0.866025403784438647f : -0.866025403784438647f;
    const float2 t1 = c_add(v[1], v[2]);
    const float2 t2 = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
    const float2 t3 = c_sub(v[1], v[2]);
    v[0] = c_add(v[0], t1);
    v[1] = make_float2(fmaf(-s, t3.y, t2.x), fmaf(s, t3.x, t2.y));
    v[2] = make_float2(fmaf(s, t3.y, t2.x), fmaf(-s, t3.x, t2.y));
  }
};

template <bool INV>
struct DFT<4, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 t0 = c_add(v[0], v[2]), t1 = c_sub(v[0], v[2]);
    const float2 t2 = c_add(v[1], v[3]), t3 = c_rot<INV>(c_sub(v[1], v[3]));
    v[0] = c_add(t0, t2);
    v[2] = c_sub(t0, t2);
    v[1] = c_add(t1, t3);
    v[3] = c_sub(t1, t3);
  }
};

// Even composite radices R = 2H (6, 8, 12, 16): one radix-2 decimation-in-time split.
template <int R, bool INV>
struct DFT {
  static_assert(R % 2 == 0 && R <= 16, "unsupported radix");
  static constexpr int H = R / 2;
  template <int... K>
  __device__ __forceinline__ static void combine(float2* v, const float2* e, const float2* o,
                                                 std::integer_sequence<int, K...>) {
    ((v[K] = c_add(e[K], mul_const_tw<R, K, INV>(o[K])), v[K + H] = c_sub(e[K], mul_const_tw<R, K, INV>(o[K]))), ...);
  }
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    DFT<H, INV>::run(e);
    DFT<H, INV>::run(o);
    combine(v, e, o, std::make_integer_sequence<int, H>{});
  }
};

// ---- size table: radix list (product N) and elements per thread E --------------------------
template <int... Rs>
struct Radices {};

template <int N>
struct FFTConf;
#define COLA_FFT_CONF(N_, E_, ...)            \
  template <>                                 \
  struct FFTConf<N_> {                        \
    static constexpr int N = N_;              \
    static constexpr int E = E_;              \
    static constexpr int T = N_ / E_;         \
    using radices = Radices<__VA_ARGS__>;     \
  };
COLA_FFT_CONF(16, 16, 16)
COLA_FFT_CONF(24, 24, 8, 3)
COLA_FFT_CONF(32, 8, 8, 4)
COLA_FFT_CONF(48, 12, 4, 4, 3)
COLA_FFT_CONF(64, 8, 8, 8)
COLA_FFT_CONF(96, 24, 8, 12)
COLA_FFT_CONF(128, 16, 16, 8)
COLA_FFT_CONF(192, 24, 8, 8, 3)
COLA_FFT_CONF(256, 16, 16, 16)
COLA_FFT_CONF(384, 24, 8, 8, 6)
COLA_FFT_CONF(512, 8, 8, 8, 8)
COLA_FFT_CONF(768, 24, 8, 8, 12)
COLA_FFT_CONF(1024, 16, 16, 16, 4)
COLA_FFT_CONF(1536, 24, 8, 8, 8, 3)
COLA_FFT_CONF(2048, 16, 16, 16, 8)
#undef COLA_FFT_CONF

// Radix variants: FFTConfV<N, 0> is FFTConf<N>; FFTConfV<N, 1> is a second factorisation with a
// different number of elements per thread (the ensemble autotuner times both).
template <int N, int V>
struct FFTConfV : FFTConf<N> {};
#define COLA_FFT_ALT(N_, E_, ...)             \
  template <>                                 \
  struct FFTConfV<N_, 1> {                    \
    static constexpr int N = N_;              \
    static constexpr int E = E_;              \
    static constexpr int T = N_ / E_;         \
    using radices = Radices<__VA_ARGS__>;     \
  };
COLA_FFT_ALT(32, 4, 4, 4, 2)
COLA_FFT_ALT(48, 24, 8, 6)
COLA_FFT_ALT(64, 16, 16, 4)
COLA_FFT_ALT(96, 12, 4, 4, 6)
COLA_FFT_ALT(128, 8, 8, 4, 4)
COLA_FFT_ALT(192, 12, 4, 4, 12)
COLA_FFT_ALT(256, 8, 8, 8, 4)
#undef COLA_FFT_ALT

template <class L>
struct FirstRadix;
template <int R0, int... Rs>
struct FirstRadix<Radices<R0, Rs...>> {
  static constexpr int value = R0;
};

// padded index of the row-layout exchange buffers: the first Stockham stage stores with stride
// R0 (its radix) between consecutive threads, so one pad slot per R0 entries (per 8 for R0 <= 8)
// puts those stores on distinct banks (row pitch xrow_ld, 8 mod 16, leaves room for either)
template <int R0>
__device__ __forceinline__ int xpad(int n) {
  constexpr int shift = R0 >= 16 ? 4 : 3;
  return n + (n >> shift);
}
template <class C>
__host__ __device__ constexpr int first_radix() {
  return FirstRadix<typename C::radices>::value;
}
template <int M>
__host__ __device__ constexpr int xrow_ld() {
  return ((M + 1 + ((M + 1) >> 3) + 1) + 15) / 16 * 16 + 8;
}

// ---- stage twiddle tables in shared memory ------------------------------------------------
// A stage of radix R after NS combined points multiplies input r of butterfly j (0 < r < R) by
// w^r, w = exp(-2 pi i (j mod NS) / (NS R)).  From the base table these are R - 1 scattered
// 8-byte loads per butterfly; a block may instead copy every stage's twiddles once into shared
// memory, butterfly by butterfly, and read them as 16-byte pairs.  Row pitch stw_pitch(R) float2
// (an even count, 2 mod 4): eight consecutive butterflies' pair loads fall on distinct banks.
// A tight table (TIGHT) gives radix-4 stages pitch 4 instead of 6: two-way bank conflicts on
// the pair loads, a third less shared memory for the largest stage of a 1024-point transform.
__host__ __device__ constexpr int stw_pitch(int R, bool tight = false) {
  const int pairs = R / 2;  // ceil((R - 1) / 2)
  return (tight && R == 4) ? 4 : 2 * pairs + ((pairs % 2 == 0) ? 2 : 0);
}
template <int... Rs>
__host__ __device__ constexpr int stw_offset_of(Radices<Rs...>, int ns_target, bool tight = false) {
  int ns = 1, off = 0;
  for (int r : {Rs...}) {
    if (ns == ns_target) return off;
    if (ns > 1) off += ns * stw_pitch(r, tight);
    ns *= r;
  }
  return off;
}
// float2 entries of the table of configuration C
template <class C, bool TIGHT = false>
__host__ __device__ constexpr int stw_size() {
  return stw_offset_of(typename C::radices{}, C::N, TIGHT);
}

// Fill the table of configuration C from the base table tw (stage twiddle m at tw[m * TWS]):
// threads tid = 0 .. nth - 1 of the block; the first use comes after the transform's first
// block barrier, so the fill needs no barrier of its own.
template <int N, int TWS, bool TIGHT, int... Rs>
__device__ __forceinline__ void stw_fill_stages(Radices<Rs...>, float2* dst, const float2* __restrict__ tw,
                                                int tid, int nth) {
  int ns = 1, off = 0;
  (
      [&] {
        constexpr int R = Rs;
        if (ns > 1) {
          const int p = stw_pitch(R, TIGHT), cnt = ns * (R - 1), step = N / (ns * R);
          for (int i = tid; i < cnt; i += nth) {
            const int j = i / (R - 1), r = i - j * (R - 1) + 1;
            dst[off + j * p + r - 1] = __ldg(tw + (int64_t)j * r * step * TWS);
          }
          off += ns * p;
        }
        ns *= R;
      }(),
      ...);
}
template <class C, int TWS, bool TIGHT = false>
__device__ __forceinline__ void stw_fill(float2* dst, const float2* __restrict__ tw, int tid, int nth) {
  stw_fill_stages<C::N, TWS, TIGHT>(typename C::radices{}, dst, tw, tid, nth);
}

// twiddle source reading the shared-memory table of configuration C (16-byte aligned)
template <class C, bool TIGHT = false>
struct SmemTw {
  const float2* base;
  template <int R, int NS, bool INV>
  __device__ __forceinline__ void apply(unsigned j, float2* x) const {
    constexpr int off = stw_offset_of(typename C::radices{}, NS, TIGHT), p = stw_pitch(R, TIGHT);
    const float4* q = reinterpret_cast<const float4*>(base + off + j * p);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const float4 w2 = q[k];
      const int r = 2 * k + 1;
      x[r] = c_mul(x[r], make_float2(w2.x, INV ? -w2.y : w2.y));
      if (r + 1 < R) x[r + 1] = c_mul(x[r + 1], make_float2(w2.z, INV ? -w2.w : w2.w));
    }
  }
};

// ---- Stockham stages --------------------------------------------------------------------
template <int N, int E, int TWS, bool INV>
struct Stockham {
  static constexpr int T = N / E;

  // Butterfly j = t + T q of a stage (0 <= t < T).  Two compile-time cases spare the per-element
  // division by NS: if NS divides T, j / NS = t / NS + q T / NS and j mod NS = t mod NS for every
  // q; if NS >= T E / R, every j is below NS (j / NS = 0, j mod NS = j).
  template <int R, int NS>
  __device__ __forceinline__ static unsigned j_mod(unsigned t, int q) {
    if constexpr (T % NS == 0) return t % NS;
    else if constexpr (NS >= T * (E / R)) return t + T * q;
    else return (t + T * q) % NS;
  }

  // twiddle and in-register DFT of every butterfly this thread owns (butterfly j = t + T q,
  // inputs v[q R + r] = x[j + r N/R]), for a stage of radix R after NS points were combined
  // (tw: the base table, or an SmemTw stage table)
  template <int R, int NS, class TW>
  __device__ __forceinline__ static void compute(float2 (&v)[E], int t, const TW& tw) {
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
      if constexpr (NS > 1) {
        const unsigned jj = j_mod<R, NS>((unsigned)t, q);
        if constexpr (!std::is_class<TW>::value) {
#pragma unroll
          for (int r = 1; r < R; ++r) {
            float2 w = __ldg(tw + jj * (r * (N / (NS * R)) * TWS));
            if (INV) w.y = -w.y;
            v[q * R + r] = c_mul(v[q * R + r], w);
          }
        } else {
          tw.template apply<R, NS, INV>(jj, &v[q * R]);
        }
      }
      DFT<R, INV>::run(&v[q * R]);
    }
  }

  // output position of element r of butterfly j = t + T q
  template <int R, int NS>
  __device__ __forceinline__ static int out_index(int t, int q, int r) {
    if constexpr (T % NS == 0) {
      const unsigned ut = (unsigned)t;
      return (int)((ut / NS) * (NS * R) + ut % NS) + q * (T * R) + r * NS;
    } else if constexpr (NS >= T * (E / R)) {
      return t + T * q + r * NS;
    } else {
      const int j = t + T * q;
      return (j / NS) * NS * R + (j % NS) + r * NS;
    }
  }

  // Run the stages NS.. of the radix list.  v holds the inputs of the first listed stage.
  // mem(n) -> float2& : exchange buffer slot for element n of this thread's sequence.
  // store(n, x)       : final output of element n.
  // before() / after(): called by every thread just before / after the first block barrier,
  // the one that separates the first stage's reads of its inputs from the first exchange
  // writes (a block that reads its inputs from a buffer may hand the buffer on after it).
  template <int NS, int R, int... Rest, class TW, class Mem, class Store, class Before, class After>
  __device__ __forceinline__ static void run(float2 (&v)[E], int t, const TW& tw, Mem& mem, Store& store,
                                             Before& before, After& after) {
    compute<R, NS>(v, t, tw);
    if constexpr (sizeof...(Rest) == 0) {
      static_assert(NS * R == N, "radix list does not multiply to N");
      if constexpr (NS == 1) before();
      __syncthreads();
      if constexpr (NS == 1) after();
#pragma unroll
      for (int q = 0; q < E / R; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) store(out_index<R, NS>(t, q, r), v[q * R + r]);
    } else {
      if constexpr (NS == 1) before();
      __syncthreads();
      if constexpr (NS == 1) after();
#pragma unroll
      for (int q = 0; q < E / R; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) mem(out_index<R, NS>(t, q, r)) = v[q * R + r];
      __syncthreads();
      constexpr int R2 = FirstRadix<Radices<Rest...>>::value;
#pragma unroll
      for (int q = 0; q < E / R2; ++q)
#pragma unroll
        for (int r = 0; r < R2; ++r) v[q * R2 + r] = mem(t + T * q + r * (N / R2));
      run<NS * R, Rest...>(v, t, tw, mem, store, before, after);
    }
  }

  template <int... Rs, class TW, class Mem, class Store, class Before, class After>
  __device__ __forceinline__ static void run_all(Radices<Rs...>, float2 (&v)[E], int t, const TW& tw, Mem& mem,
                                                 Store& store, Before& before, After& after) {
    run<1, Rs...>(v, t, tw, mem, store, before, after);
  }
};

// Convenience wrapper: load the first-stage inputs with load(n) and run the whole transform,
// with before() / after() around the first block barrier (see Stockham::run).
template <int N, int TWS, bool INV, class C = FFTConf<N>, class TW, class Load, class Mem, class Store,
          class Before, class After>
__device__ __forceinline__ void fft_1d_hooked(int t, const TW& tw, Load& load, Mem& mem, Store& store,
                                              Before& before, After& after) {
  static_assert(C::N == N, "configuration of another length");
  constexpr int E = C::E, T = C::T;
  constexpr int R0 = FirstRadix<typename C::radices>::value;
  float2 v[E];
#pragma unroll
  for (int q = 0; q < E / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) v[q * R0 + r] = load(t + T * q + r * (N / R0));
  Stockham<N, E, TWS, INV>::run_all(typename C::radices{}, v, t, tw, mem, store, before, after);
}

template <int N, int TWS, bool INV, class C = FFTConf<N>, class TW, class Load, class Mem, class Store>
__device__ __forceinline__ void fft_1d(int t, const TW& tw, Load& load, Mem& mem, Store& store) {
  auto none = [] {};
  fft_1d_hooked<N, TWS, INV, C>(t, tw, load, mem, store, none, none);
}

}  // namespace cola
