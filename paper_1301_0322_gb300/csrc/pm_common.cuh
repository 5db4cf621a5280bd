// Device helpers shared by the particle-mesh kernels: the fixed-point CIC coordinates.
#pragma once
#include "cola_internal.cuh"

namespace cola {

// Lattice index of particle p = (iz np + iy) np + ix.
__device__ __forceinline__ void lattice_index(const Geometry& g, int64_t p, int& ix, int& iy, int& iz) {
  if (g.np3 <= 0xFFFFFFFFLL) {
    // quotients by np as multiply-highs (set_np_divider): integer-pipe instructions only
    const unsigned pu = (unsigned)p, n = (unsigned)g.np;
    auto div_np = [&](unsigned v) -> unsigned {
      const unsigned t = __umulhi(g.np_mul, v);
      return (t + ((v - t) >> g.np_sh1)) >> g.np_sh2;
    };
    const unsigned r = div_np(pu);
    ix = (int)(pu - r * n);
    iz = (int)div_np(r);
    iy = (int)(r - (unsigned)iz * n);
  } else {
    const int64_t r = p / g.np;
    ix = (int)(p - r * g.np);
    iz = (int)(r / g.np);
    iy = (int)(r - (int64_t)iz * g.np);
  }
}

// Fixed-point coordinate of one axis (the library's CIC quantisation, shared bit for bit
// with the deposit test oracle):
//   f = (floor(i ng 2^F / np) + floor(fl32(s * fl32(ng/L)) * 2^F)) mod (ng 2^F)
// returns the cell (f >> F) and the upper-neighbour weight t = f mod 2^F.
__device__ __forceinline__ void fixed_axis(const Geometry& g, int i, float s, int& cell, int& t) {
  const float w = __fmul_rn(s, g.scale32);
  // 2^F from its bit pattern (no 64-bit integer conversion); exact power-of-two scaling
  const float ws = __fmul_rn(w, __int_as_float((127 + g.fbits) << 23));
  if (g.fast32 && fabsf(ws) < 4194304.0f) {
    // the same in 32 bits: the lattice offset is below ng 2^F <= 2^30 and |floor(ws)| < 2^22 <=
    // ng 2^F, so f lies in (-2^22, 2^30 + 2^22) and one wrap brings it into [0, ng 2^F).
    // floor(ws) without a conversion instruction: ws + 1.5 2^23 rounded down lies in
    // [2^23, 2^24), where floats are the integers and their bit patterns consecutive.
    const int period = g.ng << g.fbits;
    int f = ((i * g.ratio) << g.fbits) + (__float_as_int(__fadd_rd(ws, 12582912.0f)) - 0x4B400000);
    if (f < 0) f += period;
    else if (f >= period) f -= period;
    cell = f >> g.fbits;
    t = f & ((1 << g.fbits) - 1);
    return;
  }
  const int64_t one = 1LL << g.fbits;
  const int64_t period = (int64_t)g.ng << g.fbits;
  const int64_t q = g.ratio ? ((int64_t)i * g.ratio) << g.fbits : (((int64_t)i * g.ng) << g.fbits) / g.np;
  int64_t f;
  if (fabsf(ws) < 4194304.0f) {
    f = q + (int64_t)(__float_as_int(__fadd_rd(ws, 12582912.0f)) - 0x4B400000);
  } else {
    f = q + (int64_t)floorf(ws);
  }
  if (f < 0) f += period;
  if (f >= period) f -= period;
  if (f < 0 || f >= period) {  // displacement beyond one box length
    f %= period;
    if (f < 0) f += period;
  }
  cell = (int)(f >> g.fbits);
  t = (int)(f & (one - 1));
}

__device__ __forceinline__ int wrap_inc(int c, int n) { return c + 1 == n ? 0 : c + 1; }

// float32 nearest to v (ties to even), v < 2^62, as __ull2float_rn but with 32-bit integer and
// float32 instructions only (a 64-bit conversion runs on the narrow float64 pipe of sm_103a):
// with lz leading zeros in the high word, m = the 32 bits of v from its leading one down, its
// lowest bit ORed with every bit below them (sticky); m's rounding to 24 bits is v's rounding,
// and the scale 2^(32 - lz) is exact.
__device__ __forceinline__ float u64_to_f32_rn(unsigned long long v) {
  const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
  const unsigned lz = __clz(hi);                       // 32 if hi == 0
  unsigned m = __funnelshift_lc(lo, hi, lz);           // top 32 bits of v << lz (lo when lz = 32)
  m |= __funnelshift_lc(0u, lo, lz) != 0u ? 1u : 0u;   // bits of lo shifted out below m
  return __fmul_rn(__uint2float_rn(m), __int_as_float((int)(127 + 32 - lz) << 23));
}

// Exact 64-bit accumulation in shared memory held as two 32-bit words per cell, the low words
// in one array and the high words in another: the low word is added with carry detection (the
// atomic returns the previous value; the add wrapped iff the new value is below it) and the
// high word receives the upper half plus that carry.  lo[i] + 2^32 hi[i] is the 64-bit sum
// modulo 2^64, whatever the order of the adds.  Two 32-bit shared atomics run at about twice
// the rate of one 64-bit shared atomic on sm_103a.
__device__ __forceinline__ void acc_add64(unsigned* lo, unsigned* hi, int i, unsigned long long w) {
  const unsigned l = (unsigned)w, h = (unsigned)(w >> 32);
  const unsigned old = atomicAdd(lo + i, l);
  const unsigned up = h + ((old + l < old) ? 1u : 0u);
  if (up) atomicAdd(hi + i, up);
}
__device__ __forceinline__ unsigned long long acc_value(const unsigned* lo, const unsigned* hi, int i) {
  return ((unsigned long long)hi[i] << 32) | lo[i];
}

}  // namespace cola
