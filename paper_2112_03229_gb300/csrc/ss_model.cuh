// ss_model.cuh -- position models that propose where a target falls in a
// table (the learned counterpart of the analytic hashes of Sec. 3.4-3.5).
//
// MLP: 2 -> 16 -> 1, ReLU hidden layer, fp32.  Inputs are read from the
// IEEE-754 bits of the target: x0 = (e - e_lo) * e_scale with e the unbiased
// base-2 exponent, x1 = f the mantissa fraction in [0, 1).  The output
// approximates idx / (n - 1).  Parameter layout (65 floats): W1[16][2],
// b1[16], w2[16], b2 -- the same order as the CPU oracle.
//
// Spline: piecewise linear in the order-preserving key between knots spaced
// 2^shift apart; the knot values are the counts of table keys below each
// knot, i.e. exactly the bucket directory.  The proposal interpolates
// between the two knots around the query key.
#pragma once

#include "ss_common.cuh"

namespace ss {

constexpr int kHidden = 16;
constexpr int kMlpParams = 4 * kHidden + 1;   // 65

struct MlpFeatScale {
  float e_lo, e_scale;
};

// Features from the bits of t.  f keeps the top 23 mantissa bits (exact in fp32).
__device__ __forceinline__ void mlp_features(double t, const MlpFeatScale& s, float& x0, float& x1) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(t));
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  x1 = __int_as_float(0x3F800000 | (int)((u >> 29) & 0x7FFFFF)) - 1.0f;
  x0 = ((float)e - s.e_lo) * s.e_scale;
}

__device__ __forceinline__ float mlp_forward(const float* __restrict__ p, float x0, float x1) {
  float y = p[4 * kHidden];
#pragma unroll
  for (int k = 0; k < kHidden; ++k) {
    const float h = fmaxf(fmaf(p[2 * k], x0, fmaf(p[2 * k + 1], x1, p[2 * kHidden + k])), 0.0f);
    y = fmaf(p[3 * kHidden + k], h, y);
  }
  return y;
}

// Adds the gradient of scale * (y - target)^2 with respect to the 65
// parameters into g (chain rule through the ReLU); returns the squared error.
__device__ __forceinline__ float mlp_backward_accum(const float* __restrict__ p, float x0, float x1, float target,
                                                    float scale, float* g) {
  float h[kHidden];
  float y = p[4 * kHidden];
#pragma unroll
  for (int k = 0; k < kHidden; ++k) {
    h[k] = fmaf(p[2 * k], x0, fmaf(p[2 * k + 1], x1, p[2 * kHidden + k]));
    y = fmaf(p[3 * kHidden + k], fmaxf(h[k], 0.0f), y);
  }
  const float r = y - target;
  const float dy = 2.0f * r * scale;
  g[4 * kHidden] += dy;
#pragma unroll
  for (int k = 0; k < kHidden; ++k) {
    const float hk = fmaxf(h[k], 0.0f);
    g[3 * kHidden + k] = fmaf(dy, hk, g[3 * kHidden + k]);
    const float dz = h[k] > 0.0f ? dy * p[3 * kHidden + k] : 0.0f;
    g[2 * k] = fmaf(dz, x0, g[2 * k]);
    g[2 * k + 1] = fmaf(dz, x1, g[2 * k + 1]);
    g[2 * kHidden + k] += dz;
  }
  return r * r;
}

// Adam (Kingma & Ba, 2015), one parameter.
__device__ __forceinline__ void adam_update(float& p, float g, float& m1, float& m2, float lr, float b1, float b2,
                                            float eps, float c1, float c2) {
  m1 = b1 * m1 + (1.0f - b1) * g;
  m2 = b2 * m2 + (1.0f - b2) * g * g;
  p -= lr * (m1 / c1) / (sqrtf(m2 / c2) + eps);
}

// Proposal of the MLP for target t: rint(y * (n-1)) clamped to [0, n-1].
__device__ __forceinline__ int mlp_propose(const float* __restrict__ p, const MlpFeatScale& s, int n, double t) {
  float x0, x1;
  mlp_features(t, s, x0, x1);
  const float y = mlp_forward(p, x0, x1);
  const float pos = rintf(y * (float)(n - 1));
  return (int)fminf(fmaxf(pos, 0.0f), (float)(n - 1));     // NaN -> 0 through fmaxf
}

// Position (in directory count units, fractional) proposed by the spline for
// query key q over directory dir[0..nb] (counts of keys below each knot
// (base + b) << shift): linear interpolation between the two knots around q.
template <class D>   // D: directory entry type
__device__ __forceinline__ float spline_position(const D* __restrict__ dir, int shift, uint64_t base, int nb,
                                                 uint64_t q) {
  if (shift >= 32) {
    // cuts no finer than 2^-20 of an octave (the usual case, uniform per
    // table): the bucket comes from the key's high word, and the fraction's
    // 24 bits are the key bits just below the cut (the same bits and the same
    // float arithmetic as the general form below)
    const uint32_t hb = (uint32_t)(q >> 32) >> (shift - 32);
    if (hb < (uint32_t)base) return 0.0f;
    const uint32_t d = hb - (uint32_t)base;
    if (d >= (uint32_t)nb) return (float)dir[nb];
    const int lo = (int)dir[d], hi = (int)dir[d + 1];
    const float frac = (float)((uint32_t)(q >> (shift - 24)) & 0xFFFFFFu) * __int_as_float((127 - 24) << 23);
    return (float)lo + frac * (float)(hi - lo);
  }
  const uint64_t hb = q >> shift;
  if (hb < base) return 0.0f;
  const uint64_t d = hb - base;
  if (d >= (uint64_t)nb) return (float)dir[nb];
  const int b = (int)d;
  const int lo = (int)dir[b], hi = (int)dir[b + 1];
  // fraction of the way through the bucket, from the key bits below the shift
  // (the top 24 of those bits fit a 32-bit integer: int-to-float stays on the 32-bit path)
  const uint64_t below = shift > 0 ? (q & ((1ull << shift) - 1)) : 0ull;
  const float frac = shift > 0 ? (float)(uint32_t)(below >> (shift > 24 ? shift - 24 : 0)) *
                                     __int_as_float((127 - min(shift, 24)) << 23)
                               : 0.0f;
  return (float)lo + frac * (float)(hi - lo);
}

// The MLP's proposals for W targets at once, hidden unit by hidden unit:
// each unit's four parameters are read once for all W targets, so only
// they, and not all 65, are live at a time.  Same arithmetic, in the same
// order, as mlp_propose for each target.
template <int W>
__device__ __forceinline__ void mlp_propose_w(const float* __restrict__ p, const MlpFeatScale& s, int n,
                                              const double (&t)[W], int (&prop)[W]) {
  float x0[W], x1[W], y[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    mlp_features(t[j], s, x0[j], x1[j]);
    y[j] = p[4 * kHidden];
  }
#pragma unroll 2
  for (int k = 0; k < kHidden; ++k) {
    const float w0 = p[2 * k], w1 = p[2 * k + 1], bk = p[2 * kHidden + k], vk = p[3 * kHidden + k];
#pragma unroll
    for (int j = 0; j < W; ++j) y[j] = fmaf(vk, fmaxf(fmaf(w0, x0[j], fmaf(w1, x1[j], bk)), 0.0f), y[j]);
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    const float pos = rintf(y[j] * (float)(n - 1));
    prop[j] = (int)fminf(fmaxf(pos, 0.0f), (float)(n - 1));
  }
}

// Logarithm hash of Sec. 3.4 as a position proposal (no training).  With the
// base b fitted so that the table's range spans n-1 steps (Eq. 1) and the
// offset of Eq. 2, hash(t) = floor(log_b t - log_b X[0]) is the count of
// entries below t for an exactly log-spaced table.  log2 t is taken from the
// bits of t: the unbiased exponent plus log2 of the significand's top 23
// bits (fp32).  a = 1 / log2 b, c = -log2(X[0]) / log2 b; a table without a
// positive range has a = c = 0 (every proposal is 0, the window covers the
// table).  Negative targets propose 0; NaN proposes 0 through fmaxf.
__device__ __forceinline__ float log2_of_bits(double t) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(t));
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  const float m = __int_as_float(0x3F800000 | (int)((u >> 29) & 0x7FFFFF));   // significand in [1, 2)
  return (float)e + __log2f(m);
}

__device__ __forceinline__ int loghash_propose(float a, float c, int nk, double t) {
  if (__double_as_longlong(t) < 0) return 0;
  const float p = floorf(fmaf(a, log2_of_bits(t), c));
  return (int)fminf(fmaxf(p, 0.0f), (float)nk);
}

}  // namespace ss
