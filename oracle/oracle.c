/*
 * oracle.c -- plain, slow CPU reference of the sorted-table search and of
 * the bilinear lookup that the search feeds.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library; each function states the passage of the paper it
 * follows ("Sec." = section of arXiv 2112.03229, "Listing"/"Eq." likewise).
 *
 * Every routine is written for obviousness, not speed: plain bisection on
 * IEEE doubles with the comparison operators of C, fp64 arithmetic with FMA
 * contraction disabled (-ffp-contract=off), one element at a time.
 *
 * Readings of the paper that these routines fix (all listed in the design
 * notes of the repository):
 *   R1  The answer for target t is  max(0, c - 1)  where c counts the table
 *       entries strictly below t (side 0, "largest element less than the
 *       target", Sec. 1) or at most t (side 1, "less than or equal", Sec. 3).
 *       This one formula yields both end clamps of Sec. 3: a target below
 *       X[0] gets 0, a target above X[n-1] gets n-1.
 *   R2  NaN targets compare false against every entry, so c = 0 and the
 *       index is 0; an interpolated value at a NaN target is NaN.
 *   R3  -0 and +0 compare equal (IEEE 754), so they give the same index.
 *   R4  The 2D lookup (Sec. 1, 2.2: EOSPAC bounds a density/temperature
 *       target in both grids and interpolates; no formula is printed) is
 *       bilinear in linear coordinates on cell c = min(i, n-2) of each axis,
 *       with weights clamped to [0,1] and the convex form
 *       (1-w)((1-u)F00 + u F01) + w((1-u)F10 + u F11).
 *   R6  Interpolation options (the paper is silent; EOSPAC-style table
 *       libraries offer both): extrap 1 drops the clamp of R4 (linear
 *       extrapolation from the edge cell); logspace 1 takes the weights in
 *       natural-log axis coordinates, w = (ln x - ln X[c]) / (ln X[c+1] -
 *       ln X[c]), with C's log (so x = 0 gives -inf and x < 0 NaN, which the
 *       clamp and R2 then treat like any other value).
 *   R5  The exponent hash of Sec. 3.5 is taken as the top bits of an
 *       order-preserving integer image of the double; with a shift of 52 on
 *       positive doubles it is exactly the IEEE-754 base-2 exponent.  The
 *       directory entry of bucket b is the number of entries whose bucket is
 *       below b (the count form; it replaces the minimum-index table of
 *       Eq. 3 and its empty-bin rule, which the printed listing garbles).
 *
 * Parity pins (tests/test_oracle_pins.py): brute-force linear counts on tiny
 * tables, the interval invariant, IEEE special values, an affine field that
 * bilinear interpolation reproduces exactly, the 34-octave / 3.2-entries-per-
 * bin example of Sec. 4.2, central finite differences for the model gradient.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Sec. 3, problem statement: number of entries X[j] that lie below t.       */
/* side 0: X[j] <  t   (Sec. 1 wording, the default)                         */
/* side 1: X[j] <= t   (Sec. 3 wording)                                      */
/* Plain bisection on the monotone predicate; X must be strictly increasing. */
/* ------------------------------------------------------------------------ */
static int64_t count_below(const double* X, int64_t n, double t, int side) {
  int64_t lo = 0, hi = n;            /* answer lies in [lo, hi] */
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int below = side ? (X[mid] <= t) : (X[mid] < t);
    if (below) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* Sec. 3: lower-bound index with both end clamps (reading R1). */
static int32_t lower_bound_index(const double* X, int64_t n, double t, int side) {
  int64_t c = count_below(X, n, t, side);
  return (int32_t)(c > 0 ? c - 1 : 0);
}

/* Sec. 3: the search over a whole target array, one target at a time. */
void oracle_search_1d(const double* X, int32_t n, const double* Y, int64_t m,
                      int32_t side, int32_t* lowbounds) {
  for (int64_t i = 0; i < m; ++i) lowbounds[i] = lower_bound_index(X, n, Y[i], side);
}

/* Same, for a list of (table, target) pairs given by index: used to check
 * sampled outputs of very large runs one by one. */
void oracle_search_1d_sampled(const double* X, int32_t n, const double* Y,
                              const int64_t* sample, int64_t ns, int32_t side,
                              int32_t* lowbounds) {
  for (int64_t k = 0; k < ns; ++k) lowbounds[k] = lower_bound_index(X, n, Y[sample[k]], side);
}

/* ------------------------------------------------------------------------ */
/* Sec. 1 and 2.2 (EOSPAC interpolation of a density x temperature table),   */
/* reading R4.  R[nr], T[nt] strictly increasing; F row-major [nr][nt];      */
/* Y2 holds m interleaved (rho, T) pairs; lowbounds2 receives m interleaved  */
/* (i_rho, i_T) pairs; values receives m doubles.                            */
/* ------------------------------------------------------------------------ */
static double clamp01(double w) {
  if (w < 0.0) return 0.0;
  if (w > 1.0) return 1.0;
  return w;                          /* NaN passes through (reading R2) */
}

/* Weight of coordinate x in cell [X[c], X[c+1]] (readings R4 and R6). */
static double axis_weight(const double* X, int32_t c, double x, int extrap, int logspace) {
  double w;
  if (logspace) w = (log(x) - log(X[c])) / (log(X[c + 1]) - log(X[c]));
  else w = (x - X[c]) / (X[c + 1] - X[c]);
  return extrap ? w : clamp01(w);
}

static void interp_one_opts(const double* R, int32_t nr, const double* T, int32_t nt,
                            const double* F, double rho, double tem, int extrap, int logspace,
                            int32_t* ir_out, int32_t* it_out, double* v_out) {
  int32_t ir = lower_bound_index(R, nr, rho, 0);
  int32_t it = lower_bound_index(T, nt, tem, 0);
  int32_t cr = ir < nr - 2 ? ir : nr - 2;
  int32_t ct = it < nt - 2 ? it : nt - 2;
  double wr = axis_weight(R, cr, rho, extrap, logspace);
  double wt = axis_weight(T, ct, tem, extrap, logspace);
  double f00 = F[(int64_t)cr * nt + ct];
  double f01 = F[(int64_t)cr * nt + ct + 1];
  double f10 = F[(int64_t)(cr + 1) * nt + ct];
  double f11 = F[(int64_t)(cr + 1) * nt + ct + 1];
  double lo_row = (1.0 - wt) * f00 + wt * f01;
  double hi_row = (1.0 - wt) * f10 + wt * f11;
  *ir_out = ir;
  *it_out = it;
  *v_out = (1.0 - wr) * lo_row + wr * hi_row;
}

static void interp_one(const double* R, int32_t nr, const double* T, int32_t nt,
                       const double* F, double rho, double tem,
                       int32_t* ir_out, int32_t* it_out, double* v_out) {
  interp_one_opts(R, nr, T, nt, F, rho, tem, 0, 0, ir_out, it_out, v_out);
}

/* The 2D lookup with the interpolation options of reading R6. */
void oracle_search_interp_2d_opts(const double* R, int32_t nr, const double* T, int32_t nt,
                                  const double* F, const double* Y2, int64_t m,
                                  int32_t extrap, int32_t logspace,
                                  int32_t* lowbounds2, double* values) {
  for (int64_t i = 0; i < m; ++i)
    interp_one_opts(R, nr, T, nt, F, Y2[2 * i], Y2[2 * i + 1], extrap, logspace,
                    &lowbounds2[2 * i], &lowbounds2[2 * i + 1], &values[i]);
}

void oracle_search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt,
                             const double* F, const double* Y2, int64_t m,
                             int32_t* lowbounds2, double* values) {
  for (int64_t i = 0; i < m; ++i)
    interp_one(R, nr, T, nt, F, Y2[2 * i], Y2[2 * i + 1],
               &lowbounds2[2 * i], &lowbounds2[2 * i + 1], &values[i]);
}

void oracle_search_interp_2d_sampled(const double* R, int32_t nr, const double* T, int32_t nt,
                                     const double* F, const double* Y2,
                                     const int64_t* sample, int64_t ns,
                                     int32_t* lowbounds2, double* values) {
  for (int64_t k = 0; k < ns; ++k) {
    int64_t i = sample[k];
    interp_one(R, nr, T, nt, F, Y2[2 * i], Y2[2 * i + 1],
               &lowbounds2[2 * k], &lowbounds2[2 * k + 1], &values[k]);
  }
}

/* ------------------------------------------------------------------------ */
/* Batched forms: many independent tables, each with its own targets.        */
/* CSR offsets: table k is X[X_off[k] .. X_off[k+1]), its targets are        */
/* Y[Y_off[k] .. Y_off[k+1]).  Each table is searched exactly as above.      */
/* ------------------------------------------------------------------------ */
void oracle_search_1d_batched(int32_t ntables, const int64_t* X_off, const double* X,
                              const int64_t* Y_off, const double* Y, int32_t side,
                              int32_t* lowbounds) {
  for (int32_t k = 0; k < ntables; ++k) {
    const double* Xk = X + X_off[k];
    int32_t nk = (int32_t)(X_off[k + 1] - X_off[k]);
    oracle_search_1d(Xk, nk, Y + Y_off[k], Y_off[k + 1] - Y_off[k], side, lowbounds + Y_off[k]);
  }
}

void oracle_search_interp_2d_batched_opts(int32_t ntables,
                                          const int64_t* R_off, const double* R,
                                          const int64_t* T_off, const double* T,
                                          const int64_t* F_off, const double* F,
                                          const int64_t* Y_off, const double* Y2,
                                          int32_t extrap, int32_t logspace,
                                          int32_t* lowbounds2, double* values) {
  for (int32_t k = 0; k < ntables; ++k) {
    int32_t nr = (int32_t)(R_off[k + 1] - R_off[k]);
    int32_t nt = (int32_t)(T_off[k + 1] - T_off[k]);
    int64_t y0 = Y_off[k];
    oracle_search_interp_2d_opts(R + R_off[k], nr, T + T_off[k], nt, F + F_off[k],
                                 Y2 + 2 * y0, Y_off[k + 1] - y0, extrap, logspace,
                                 lowbounds2 + 2 * y0, values + y0);
  }
}

void oracle_search_interp_2d_batched(int32_t ntables,
                                     const int64_t* R_off, const double* R,
                                     const int64_t* T_off, const double* T,
                                     const int64_t* F_off, const double* F,
                                     const int64_t* Y_off, const double* Y2,
                                     int32_t* lowbounds2, double* values) {
  oracle_search_interp_2d_batched_opts(ntables, R_off, R, T_off, T, F_off, F, Y_off, Y2, 0, 0,
                                       lowbounds2, values);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5, exponent hash search, reading R5.                               */
/* Order-preserving integer image of a double: negative values are mapped by */
/* two's-complement negation of their bit pattern, non-negative ones by      */
/* setting the top bit; -0 is first replaced by +0 so that equal doubles get */
/* equal images.  For non-NaN a, b:  a < b  <=>  image(a) < image(b).        */
/* ------------------------------------------------------------------------ */
uint64_t oracle_order_key(double x) {
  uint64_t u;
  if (x == 0.0) x = 0.0;             /* -0 -> +0 (reading R3) */
  memcpy(&u, &x, sizeof u);
  if (u >> 63) return (uint64_t)0 - u;
  return u | ((uint64_t)1 << 63);
}

/* Directory of the bucket function h(x) = image(x) >> shift over the buckets
 * from h(X[0]) to h(X[n-1]).  L[b] = number of entries whose bucket lies below
 * bucket h(X[0]) + b, for b = 0 .. B (so L[0] = 0 and L[B] = n).  Returns B,
 * or -1 if B + 1 exceeds cap (then L is left unspecified).  *base receives
 * h(X[0]). */
int64_t oracle_bucket_directory(const double* X, int32_t n, int32_t shift,
                                uint64_t* base, int32_t* L, int64_t cap) {
  uint64_t b0 = oracle_order_key(X[0]) >> shift;
  uint64_t b1 = oracle_order_key(X[n - 1]) >> shift;
  *base = b0;
  if (b1 - b0 + 1 >= (uint64_t)cap) return -1;   /* B + 1 entries must fit in cap */
  int64_t B = (int64_t)(b1 - b0) + 1;
  for (int64_t b = 0; b <= B; ++b) {
    int32_t c = 0;
    for (int32_t j = 0; j < n; ++j)  /* linear count, one bucket at a time */
      if ((oracle_order_key(X[j]) >> shift) < b0 + (uint64_t)b) ++c;
    L[b] = c;
  }
  return B;
}

/* The finest shift whose directory has at most cap_buckets buckets. */
int32_t oracle_bucket_shift(const double* X, int32_t n, int64_t cap_buckets) {
  uint64_t k0 = oracle_order_key(X[0]), k1 = oracle_order_key(X[n - 1]);
  for (int32_t s = 0; s < 64; ++s)   /* spans are unsigned: a table may cover most of the key range */
    if ((k1 >> s) - (k0 >> s) < (uint64_t)cap_buckets) return s;
  return 63;
}

/* ------------------------------------------------------------------------ */
/* Position models (not in the paper; they play the part of the analytic     */
/* hash of Sec. 3.4-3.5 as a learned map from target to table position).     */
/* ------------------------------------------------------------------------ */

/* Piecewise-linear spline over the order-preserving image: knot j sits at
 * kappa_j = image(X[0]) + j * delta, delta = ceil((image(X[n-1]) - image(X[0]) + 1) / K),
 * and its value is the count of entries whose image is below kappa_j.
 * counts must hold K + 1 values. */
void oracle_spline_knots(const double* X, int32_t n, int32_t K, uint64_t* delta_out,
                         int32_t* counts) {
  uint64_t k0 = oracle_order_key(X[0]), k1 = oracle_order_key(X[n - 1]);
  uint64_t span = k1 - k0 + 1;
  uint64_t delta = span / (uint64_t)K + (span % (uint64_t)K != 0);
  *delta_out = delta;
  for (int32_t j = 0; j <= K; ++j) {
    uint64_t kappa = k0 + (uint64_t)j * delta;
    int32_t c = 0;
    for (int32_t i = 0; i < n; ++i)
      if (oracle_order_key(X[i]) < kappa) ++c;
    counts[j] = c;
  }
}

/* Features of a target for the 2 -> 16 -> 1 MLP: the unbiased base-2
 * exponent e and the mantissa fraction f in [0,1) read from the IEEE-754
 * bits; the exponent is rescaled with the table's exponent range,
 * x0 = (e - e_lo) * e_scale, x1 = f. */
void oracle_mlp_features(double t, double e_lo, double e_scale, double* x0, double* x1) {
  uint64_t u;
  memcpy(&u, &t, sizeof u);
  double e = (double)((int64_t)((u >> 52) & 0x7FF) - 1023);
  double f = (double)(u & (((uint64_t)1 << 52) - 1)) / 4503599627370496.0; /* 2^52 */
  *x0 = (e - e_lo) * e_scale;
  *x1 = f;
}

/* Parameter layout (65 values): W1[16][2], b1[16], w2[16], b2. */
#define H 16
static double relu(double a) { return a > 0.0 ? a : 0.0; }

static double mlp_forward_one(const double* p, double x0, double x1, double* h) {
  const double* W1 = p;
  const double* b1 = p + 2 * H;
  const double* w2 = p + 3 * H;
  double b2 = p[4 * H];
  double y = b2;
  for (int k = 0; k < H; ++k) {
    h[k] = relu(W1[2 * k] * x0 + W1[2 * k + 1] * x1 + b1[k]);
    y += w2[k] * h[k];
  }
  return y;
}

/* Forward pass for B feature pairs (x interleaved). */
void oracle_mlp_forward(const double* params, const double* x, int64_t B, double* y) {
  double h[H];
  for (int64_t i = 0; i < B; ++i) y[i] = mlp_forward_one(params, x[2 * i], x[2 * i + 1], h);
}

/* Mean squared error over the batch and its gradient with respect to all 65
 * parameters (analytic backward pass, written out by the chain rule). */
double oracle_mlp_loss_grad(const double* params, const double* x, const double* target,
                            int64_t B, double* grad) {
  const double* w2 = params + 3 * H;
  double h[H];
  double loss = 0.0;
  for (int k = 0; k < 4 * H + 1; ++k) grad[k] = 0.0;
  for (int64_t i = 0; i < B; ++i) {
    double x0 = x[2 * i], x1 = x[2 * i + 1];
    double y = mlp_forward_one(params, x0, x1, h);
    double r = y - target[i];
    loss += r * r;
    double dy = 2.0 * r / (double)B;                 /* dL/dy */
    grad[4 * H] += dy;                               /* b2 */
    for (int k = 0; k < H; ++k) {
      grad[3 * H + k] += dy * h[k];                  /* w2[k] */
      if (h[k] > 0.0) {
        double dz = dy * w2[k];                      /* through ReLU */
        grad[2 * k] += dz * x0;                      /* W1[k][0] */
        grad[2 * k + 1] += dz * x1;                  /* W1[k][1] */
        grad[2 * H + k] += dz;                       /* b1[k] */
      }
    }
  }
  return loss / (double)B;
}

/* One Adam step (Kingma & Ba, 2015) on the 65 parameters; step counts from 1. */
void oracle_adam_step(double* params, const double* grad, double* mom1, double* mom2,
                      int64_t step, double lr, double beta1, double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, (double)step);
  double c2 = 1.0 - pow(beta2, (double)step);
  for (int k = 0; k < 4 * H + 1; ++k) {
    mom1[k] = beta1 * mom1[k] + (1.0 - beta1) * grad[k];
    mom2[k] = beta2 * mom2[k] + (1.0 - beta2) * grad[k] * grad[k];
    double mhat = mom1[k] / c1;
    double vhat = mom2[k] / c2;
    params[k] -= lr * mhat / (sqrt(vhat) + eps);
  }
}
#undef H
