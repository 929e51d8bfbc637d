// ss_ff.cuh -- float-float ("double-float") arithmetic for the 2D blend.
//
// GB300 issues fp64 at a small fraction of its fp32 rate (measured: 0.5 T
// fp64 FMA/s against 36 T fp32 FMA/s), so an fp64 bilinear blend is bound by
// the fp64 pipe long before HBM.  A value is instead carried as an unevaluated
// sum hi + lo of two floats (about 48 significant bits, relative error near
// 2^-47 per operation), built from the error-free transformations of Knuth
// (two-sum), Dekker (fast two-sum) and the fma-based exact product.  Doubles
// are split into hi + lo with integer bit operations, so the hot loop issues
// no fp64 arithmetic except one final add per output value.
//
// The interpolation weights are formed exactly: for a target x in cell
// [X_c, X_c+1] whose binary exponents differ by at most kMaxCellOctaves,
// x - X_c is an integer multiple of 2^(e_c - 1075) computed exactly in 64-bit
// integers; it is then scaled by the per-cell factor g_c = 2^(e_c-1075) / gap_c.
#pragma once

#include "ss_common.cuh"

namespace ss {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// 1 - w for w in [0, 1]
__device__ __forceinline__ ff ff_one_minus(ff w) {
  const ff s = two_sum(1.0f, -w.hi);
  return fast_two_sum(s.hi, s.lo - w.lo);
}

constexpr int kMaxCellOctaves = 10;   // exact integer weights when a cell spans at most 2^10
constexpr int kFFMinExp = 1023 - 70;  // doubles split into float-float must lie in [2^-70, 2^101)
constexpr int kFFMaxExp = 1023 + 100;

// Float whose value is the power of two 2^k (k in the normal range).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// Split a finite double with biased exponent in [kFFMinExp, kFFMaxExp] (or
// zero) into hi + lo exactly up to 2^-48 relative.  Returns false (and
// leaves hi/lo zero) for anything else.
__device__ __forceinline__ bool d2ff(double d, ff& r) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(d));
  const int e = (int)((u >> 52) & 0x7FF);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  r.hi = 0.0f;
  r.lo = 0.0f;
  if ((u << 1) == 0) return true;                      // +-0
  if (e < kFFMinExp || e > kFFMaxExp) return false;
  const uint64_t M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // 53-bit significand
  // hi: top 24 bits, exponent e-1023; lo: the remaining 29 bits (rounded to 24)
  r.hi = __int_as_float((int)(sign | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)((M >> 29) & 0x7FFFFF)));
  const float rem = (float)(uint32_t)(M & 0x1FFFFFFFull) * pow2f(e - 1075);
  r.lo = sign ? -rem : rem;
  return true;
}

// Double nearest to hi + lo (the float-to-double widening is exact and done
// with integer operations; one fp64 add rounds the sum).
__device__ __forceinline__ double widen(float f) {
  const uint32_t b = (uint32_t)__float_as_int(f);
  const uint32_t ef = (b >> 23) & 0xFF;
  if (ef == 0) return 0.0;                              // zero (subnormal parts dropped: < 2^-126)
  const uint64_t hi = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(ef - 127 + 1023) << 52) |
                      ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)hi);
}

__device__ __forceinline__ double ff2d(ff a) { return widen(a.hi) + widen(a.lo); }

// Unsigned 64-bit integer D > 0 as float-float, exact up to 2^-47 relative.
__device__ __forceinline__ ff u64_to_ff(uint64_t D) {
  const int lz = __clzll((long long)D);
  const uint64_t N = D << lz;                           // leading one at bit 63
  ff r;
  r.hi = __int_as_float((int)(((uint32_t)(127 + 63 - lz) << 23) | (uint32_t)((N >> 40) & 0x7FFFFF)));
  r.lo = (float)(uint32_t)((N >> 16) & 0xFFFFFF) * pow2f(16 - lz);
  return r;
}

// Per-cell data staged in shared memory for the float-float path.
struct CellFF {
  uint64_t xbits;   // bit pattern of X[c] (positive normal)
  float ghi, glo;   // g_c = 2^(e_c - 1075) / (X[c+1] - X[c]) as float-float
};

// Both weights of target x (bit pattern u, positive normal, X[c] < x <= X[c+1])
// in cell c: w = (x - X[c]) / gap and wbar = (X[c+1] - x) / gap.  Each
// numerator is an exact integer (no cancellation), so wbar keeps full
// relative precision when w is close to 1 instead of being formed as 1 - w.
struct Weights {
  ff w, wbar;
};

__device__ __forceinline__ Weights cell_weights(uint64_t u, const CellFF& cell, uint64_t next_bits) {
  const int ex = (int)((u >> 52) & 0x7FF);
  const int ec = (int)((cell.xbits >> 52) & 0x7FF);
  const int en = (int)((next_bits >> 52) & 0x7FF);
  const uint64_t Mx = ((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (ex - ec);
  const uint64_t Mc = (cell.xbits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const uint64_t Mn = ((next_bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (en - ec);
  const uint64_t D = Mx - Mc;          // x - X[c]    in units of 2^(ec - 1075)
  const uint64_t Dn = Mn - Mx;         // X[c+1] - x  in the same units
  const ff g{cell.ghi, cell.glo};
  Weights r;
  r.w = D == 0 ? ff{0.0f, 0.0f} : ff_mul(u64_to_ff(D), g);
  r.wbar = Dn == 0 ? ff{0.0f, 0.0f} : ff_mul(u64_to_ff(Dn), g);
  return r;
}

__device__ __forceinline__ ff ff_clamp01(ff w) {
  if (w.hi < 0.0f) return {0.0f, 0.0f};
  if (w.hi > 1.0f || (w.hi == 1.0f && w.lo > 0.0f)) return {1.0f, 0.0f};
  return w;
}

}  // namespace ss
