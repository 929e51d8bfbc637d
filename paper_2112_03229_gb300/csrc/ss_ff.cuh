// ss_ff.cuh -- float-float ("double-float") arithmetic for the 2D blend.
//
// GB300 issues fp64 at a small fraction of its fp32 rate (measured: 0.5 T
// fp64 FMA/s against 36 T fp32 FMA/s), so an fp64 bilinear blend is bound by
// the fp64 pipe long before HBM.  A value is instead carried as an unevaluated
// sum hi + lo of two floats (about 48 significant bits, relative error near
// 2^-47 per operation), built from the error-free transformations of Knuth
// (two-sum), Dekker (fast two-sum) and the fma-based exact product.  Doubles
// are split into hi + lo with integer bit operations, so the hot loop issues
// no fp64 arithmetic except the final widening and add per output value.
//
// The interpolation weights are formed from exact integers: for a target x in
// cell [X_c, X_c+1] whose binary exponents differ by at most kMaxCellOctaves,
// x - X_c and X_c+1 - x are integer multiples of 2^(e_c - 1075) computed in
// 64-bit integers; the smaller of the two is scaled by the per-cell factor
// 1 / (X_c+1 - X_c) in the same units, and the other weight is 1 minus it.
// That one is at least 1/2, so both weights keep full relative precision.
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

constexpr int kMaxCellOctaves = 10;   // exact integer weights when a cell spans at most 2^10
constexpr int kFFMinExp = 1023 - 70;  // doubles split into float-float must lie in [2^-70, 2^101)
constexpr int kFFMaxExp = 1023 + 100;

// Product and sum of two float-float values, left unnormalised: the pair
// still sums exactly to the represented value, and the final widening to
// double adds hi and lo anyway, so no fast two-sum is spent on them.
__device__ __forceinline__ ff ff_mul_u(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return {p, e};
}

__device__ __forceinline__ ff ff_add_u(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return {s.hi, s.lo + (a.lo + b.lo)};
}

// Split a positive double with biased exponent in [kFFMinExp, kFFMaxExp] into
// hi (its top 24 significant bits, truncated) + lo (the other 29 bits rounded
// to 24), exact up to 2^-48 relative.  Integer bit operations and one int to
// float conversion.  Returns false for zero, negative or out-of-range values.
__device__ __forceinline__ bool d2ff(double d, ff& r) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(d));
  const uint32_t hw = (uint32_t)(u >> 32);
  const bool ok = (hw - ((uint32_t)kFFMinExp << 20)) < ((uint32_t)(kFFMaxExp + 1 - kFFMinExp) << 20);
  const uint32_t hb = (uint32_t)((u - (896ull << 52)) >> 29);        // float bits: exponent rebiased
  r.hi = __uint_as_float(hb);
  const float unit = __uint_as_float((hb & 0x7F800000u) - (52u << 23));  // 2^(e - 1075)
  r.lo = (float)((uint32_t)u & 0x1FFFFFFFu) * unit;
  return ok;
}

// Double nearest to hi + lo: both floats widen exactly (the hardware
// conversion, which measured faster than building the bit patterns with
// integer operations), and one fp64 add rounds the exact sum.
__device__ __forceinline__ double ff2d(ff a) { return (double)a.hi + (double)a.lo; }

// Per-cell data for the float-float weights, as computed.
struct CellW {
  uint64_t Mc;      // significand of X[c] (53 bits with the implicit one)
  uint64_t MnS;     // significand of X[c+1] shifted left by e(X[c+1]) - e(X[c])
  int ec;           // biased exponent of X[c]
  int pad;
  float ghi, glo;   // 2^48 / (MnS - Mc) as float-float
};

// Cell data as stored in memory, 24 bytes per cell in a 16-byte aligned
// region: an array of 16-byte records A[c] = {Mc | ec << 53, MnS} (the
// exponent sits above the 53-bit significand), then an array of 8-byte
// scales G[c] = {ghi, glo}.  Each array is read with one load per cell at its
// own stride, which spreads a warp's random reads over all shared-memory
// banks; 32-byte records read field by field put the same field of every
// cell on one quarter of the banks and conflicted about twice as often.
// The scale is only needed at the end of the weight computation, so it is
// read there and the record's registers are free by then.
constexpr int kCellBytes = 24;

struct CellTable {
  const ulonglong2* a;
  const float2* g;
#ifdef SS_CHECKED
  int n;                // cells (checked build)
#endif
};

__device__ __forceinline__ CellTable cell_table(const void* region, int ncell) {
  const ulonglong2* a = reinterpret_cast<const ulonglong2*>(region);
#ifdef SS_CHECKED
  return {a, reinterpret_cast<const float2*>(a + ncell), ncell};
#else
  return {a, reinterpret_cast<const float2*>(a + ncell)};
#endif
}

__device__ __forceinline__ void store_cell(void* region, int ncell, int c, const CellW& w) {
  ulonglong2* a = reinterpret_cast<ulonglong2*>(region);
  a[c] = make_ulonglong2(w.Mc | ((uint64_t)w.ec << 53), w.MnS);
  reinterpret_cast<float2*>(a + ncell)[c] = make_float2(w.ghi, w.glo);
}

// Cell data of [a, b]; false if the cell is outside the float-float preconditions.
__device__ __forceinline__ bool make_cell(double a, double b, CellW& c) {
  const uint64_t ua = static_cast<uint64_t>(__double_as_longlong(a));
  const uint64_t ub = static_cast<uint64_t>(__double_as_longlong(b));
  const int ea = (int)((ua >> 52) & 0x7FF), eb = (int)((ub >> 52) & 0x7FF);
  c = CellW{0, 0, ea, 0, 0.0f, 0.0f};
  if ((ua >> 63) != 0 || ea < kFFMinExp || eb > kFFMaxExp || eb - ea > kMaxCellOctaves || !(b > a)) return false;
  c.Mc = (ua & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  c.MnS = ((ub & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (eb - ea);
  const double g = 0x1.0p48 / (double)(c.MnS - c.Mc);
  c.ghi = __double2float_rn(g);
  c.glo = __double2float_rn(g - (double)c.ghi);
  return true;
}

// Integer 0 < v < 2^63 as a float pair scaled by 2^-48, from 32-bit
// operations only: v is normalised so that its leading one sits at bit 63
// (shift s = clz(v), taken on the nonzero word), and its top 48 bits are
// split into two 24-bit halves.  The high half becomes a float by placing
// its 24 bits under the exponent 2^(15-s) (no conversion); the low half is
// converted (exact: under 2^24) and scaled by 2^(-32-s).  The low half is
// below one unit of the high half's last place, so products with it stay
// accurate to 2^-47 whatever the magnitude of v.
__device__ __forceinline__ ff numerator(uint64_t v) {
  const uint32_t vh = (uint32_t)(v >> 32), vl = (uint32_t)v;
  const bool z = vh == 0;
  const uint32_t a = z ? vl : vh, b = z ? 0u : vl;      // the nonzero leading word and the one after it
  const int c = __clz((int)a);
  const uint32_t th = __funnelshift_l(b, a, c), tl = b << c;   // bits 63..32 and 31..0 of v << s
  const int s = c + (z ? 32 : 0);
  const float hi = __uint_as_float(((uint32_t)(141 - s) << 23) + (th >> 8));
  const float lo = (float)(__funnelshift_r(tl, th, 16) & 0xFFFFFFu) * __uint_as_float((uint32_t)(95 - s) << 23);
  return {hi, lo};
}

// Both weights of target x (bit pattern u, X[c] < x <= X[c+1]) in cell c:
// w = (x - X[c]) / gap and wbar = (X[c+1] - x) / gap, each numerator exact
// and normalised on its own (so a small wbar keeps its relative precision).
struct Weights {
  ff w, wbar;
};

// 1 - a for 0 <= a <= 1/2 (plus rounding): the result is at least 1/2, so
// the float-float difference keeps its relative precision.  1 >= |a.hi|, so
// the exact sum of the high parts needs only the ordered (fast) form.
__device__ __forceinline__ ff one_minus(ff a) {
  const ff s = fast_two_sum(1.0f, -a.hi);
  return fast_two_sum(s.hi, s.lo - a.lo);
}

// Only the smaller weight needs its exact numerator: it is at most 1/2, and
// the larger one, 1 minus it, is at least 1/2, where the float-float
// subtraction loses nothing relative to its size.  Both weights so keep
// their full relative precision (however small the smaller one is).
// ANY: the target may lie outside the cell (a caller that computes the
// weights of every target and then picks the end weights of clamped ones
// without a branch); the exponent difference is then taken modulo 64 so
// every step stays defined, and the result is meaningless but unused.
template <bool ANY = false>
__device__ __forceinline__ Weights cell_weights(uint64_t u, const CellTable& t, int c) {
#ifdef SS_CHECKED
  c = SS_IX(c, t.n);
#endif
  const ulonglong2 rec = t.a[c];
  const int ec = (int)(rec.x >> 53);
  const uint64_t Mc = rec.x & ((1ull << 53) - 1), MnS = rec.y;
  const int ex = (int)((u >> 52) & 0x7FF);
  const uint64_t MxS = ((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (ANY ? ((ex - ec) & 63) : (ex - ec));
  const uint64_t D = MxS - Mc, Dn = MnS - MxS;
  const bool low = D <= Dn;                      // the target sits in the lower half of the cell
  const uint64_t v = low ? D : Dn;
  const float2 gs = t.g[c];
  const ff g{gs.x, gs.y};
  const ff small = v == 0 ? ff{0.0f, 0.0f} : ff_mul_u(numerator(v), g);
  const ff large = one_minus(small);
  Weights r;
  r.w = low ? small : large;
  r.wbar = low ? large : small;
  return r;
}

}  // namespace ss
