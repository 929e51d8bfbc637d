// plan_2d.cu -- 2D plans: many density x temperature tables (Sec. 1, 2.2),
// each axis prepared like a 1D table (with its own learned proposal when a
// model is requested) plus per-cell float-float weight data, the value grids
// converted once to float-float, and a persistent kernel over a tile queue
// of (table, pair range) work items.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "plan.h"
#include "plan_host.h"

namespace ss {

int default_dir_cap(int n);

// Per-cell data of one axis blob and its float-float eligibility.
__global__ void __launch_bounds__(256) k_prep_cells(PrepArgs a) {
  const int k = blockIdx.x;
  if (k >= a.ntables) return;
  const double* X = a.X + a.X_off[k];
  const int n = (int)(a.X_off[k + 1] - a.X_off[k]);
  unsigned char* blob = a.blobs + a.blob_off[k];
  BlobHdr* h = reinterpret_cast<BlobHdr*>(blob);
  unsigned char* cells = blob + h->off_cells;
  bool ok = true;
  for (int c = threadIdx.x; c < n - 1; c += blockDim.x) {
    CellW w;
    ok &= make_cell(X[c], X[c + 1], w);
    store_cell(cells, n - 1, c, w);
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) h->ffok = ok ? 1 : 0;
}

// Value grids to per-cell corner records: cell (i, j) of a table holds
// F[i][j], F[i][j+1], F[i+1][j], F[i+1][j+1] as float-float in 32 bytes, so
// the four gathers of a lookup are two 16-byte loads from one 32-byte sector.
// Values the split does not cover (zero, negative, or outside
// [2^-70, 2^101)) get a NaN high part and set *bad, so the plan keeps the
// caller's fp64 grid for them.  One block per table.
__global__ void __launch_bounds__(256) k_grid_cells(const double* __restrict__ F, const int64_t* __restrict__ F_off,
                                                    const int64_t* __restrict__ R_off,
                                                    const int64_t* __restrict__ T_off,
                                                    const int64_t* __restrict__ cell_off, float4* __restrict__ cells,
                                                    unsigned* bad) {
  const int k = blockIdx.x;
  const int nr = (int)(R_off[k + 1] - R_off[k]), nt = (int)(T_off[k + 1] - T_off[k]);
  const double* f = F + F_off[k];
  float4* out = cells + 2 * cell_off[k];
  const int64_t ncell = (int64_t)(nr - 1) * (nt - 1);
  bool ok = true;
  auto split = [&ok](double v) {
    ff r;
    if (d2ff(v, r)) return r;
    ok = false;
    return ff{__int_as_float(0x7FC00000), 0.0f};
  };
  for (int64_t c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int64_t i = c / (nt - 1), j = c - i * (nt - 1);
    const double* q = f + i * nt + j;
    const ff a00 = split(q[0]), a01 = split(q[1]), a10 = split(q[nt]), a11 = split(q[nt + 1]);
    out[2 * c] = make_float4(a00.hi, a00.lo, a01.hi, a01.lo);
    out[2 * c + 1] = make_float4(a10.hi, a10.lo, a11.hi, a11.lo);
  }
  if (!ok) atomicOr(bad, 1u);
}

// Exact count for one axis with the axis' algorithm (LEARNED: the position
// models are compiled in; a plan without them runs a kernel built without).
template <bool LEARNED>
__device__ __forceinline__ int axis_count(const StagedView& v, double t, uint64_t q, int& fallbacks) {
  if (!LEARNED) return v.h.algo == BL_BINARY ? plain_binary(v, q) : plain_bucket(v, q);
  switch (v.h.algo) {
    case BL_BINARY: return plain_binary(v, q);
    case BL_SPLINE: return spline_count(v, q, fallbacks);
    case BL_MLP: return mlp_count(v, t, q, fallbacks);
    case BL_LOGHASH: return loghash_count(v, t, q, fallbacks);
    default: return plain_bucket(v, q);
  }
}

// Weights (w, 1 - w) of a coordinate on an axis (float-float; fp64 division
// when the axis is outside the float-float preconditions).
__device__ __forceinline__ double entry_value(const StagedView& v, int j) {
  const uint64_t k = j == 0 ? v.h.k0 : key_at(v, j - 1);
  const uint64_t u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : (0ull - k);
  return __longlong_as_double((long long)u);
}

__device__ __forceinline__ Weights axis_weights(const StagedView& v, int i, int c, uint64_t k, double x) {
  const BlobHdr& h = v.h;
  if (i >= h.n - 1) return {{1.0f, 0.0f}, {0.0f, 0.0f}};
  if (i == 0 && k <= h.k0) return {{0.0f, 0.0f}, {1.0f, 0.0f}};
  if (h.ffok) return cell_weights(static_cast<uint64_t>(__double_as_longlong(x)), v.cells, c);
  const double a = entry_value(v, c), b = entry_value(v, c + 1);
  double w = (x - a) / (b - a);
  w = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
  const double wb = 1.0 - w;
  Weights r;
  r.w.hi = __double2float_rn(w);
  r.w.lo = __double2float_rn(w - (double)r.w.hi);
  r.wbar.hi = __double2float_rn(wb);
  r.wbar.lo = __double2float_rn(wb - (double)r.wbar.hi);
  return r;
}

constexpr uint64_t kKeyNegInf = 0x0010000000000000ull;   // image of -inf; NaNs map below it

// One pair: the two axis counts (CR, CT: the searches the tile dispatched),
// four gathers from the grid, and the blend.
// fp64 weight of coordinate x in cell c for the interpolation options:
// linear or natural-log coordinates, clamped to [0, 1] unless extrapolating.
__device__ __forceinline__ double option_weight(const StagedView& v, int c, double x, int extrap, int logspace) {
  const double a = entry_value(v, c), b = entry_value(v, c + 1);
  const double w = logspace ? (log(x) - log(a)) / (log(b) - log(a)) : (x - a) / (b - a);
  return extrap ? w : (w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w));
}

template <class CR, class CT>
__device__ __forceinline__ void pair_2d(const StagedView& vr, const StagedView& vt, const float4* __restrict__ G,
                                        const double* __restrict__ G64, double rho, double tem, int& ir, int& it,
                                        double& v, int& nans, CR&& count_r, CT&& count_t, int extrap = 0,
                                        int logspace = 0) {
  const uint64_t kr = order_key(rho), kt = order_key(tem);
  const bool nan = (kr < kKeyNegInf) | (kt < kKeyNegInf);
  nans += (kr < kKeyNegInf) + (kt < kKeyNegInf);
  ir = count_r(rho, kr);
  it = count_t(tem, kt);
  const int nt = vt.h.n;
  const int cr = min(ir, vr.h.n - 2), ct = min(it, nt - 2);
  const int64_t cell = (int64_t)cr * (nt - 1) + ct;
  float q[8];
  ld_nc_v8_policy(reinterpret_cast<const float*>(G + 2 * cell), q, l2_policy_evict_last());   // 32-byte aligned
  const float2 g00 = make_float2(q[0], q[1]), g01 = make_float2(q[2], q[3]);
  const float2 g10 = make_float2(q[4], q[5]), g11 = make_float2(q[6], q[7]);
  if (logspace | extrap) {
    const bool outside = (ir >= vr.h.n - 1) | (ir == 0 && kr <= vr.h.k0) | (it >= nt - 1) | (it == 0 && kt <= vt.h.k0);
    if (logspace | outside) {
      const int64_t o = (int64_t)cr * nt + ct;
      const double w1 = option_weight(vr, cr, rho, extrap, logspace), w2 = option_weight(vt, ct, tem, extrap, logspace);
      const double lo = (1.0 - w2) * G64[o] + w2 * G64[o + 1];
      const double hi = (1.0 - w2) * G64[o + nt] + w2 * G64[o + nt + 1];
      v = (1.0 - w1) * lo + w1 * hi;
      return;
    }
  }
  const Weights wr = axis_weights(vr, ir, cr, kr, rho);
  const Weights wt = axis_weights(vt, it, ct, kt, tem);
  if (nan) {
    v = __longlong_as_double(0x7FF8000000000000ll);
  } else if (G64 == nullptr || !(isnan(g00.x) | isnan(g01.x) | isnan(g10.x) | isnan(g11.x))) {
    // (a plan keeps the fp64 grid only when some value is outside the float-float range)
    const ff lo = ff_add_u(ff_mul_u(wt.wbar, ff{g00.x, g00.y}), ff_mul_u(wt.w, ff{g01.x, g01.y}));
    const ff hi = ff_add_u(ff_mul_u(wt.wbar, ff{g10.x, g10.y}), ff_mul_u(wt.w, ff{g11.x, g11.y}));
    v = ff2d(ff_add_u(ff_mul_u(wr.wbar, lo), ff_mul_u(wr.w, hi)));
  } else {
    const int64_t o = (int64_t)cr * nt + ct;
    const double w1 = ff2d(wr.w), w1b = ff2d(wr.wbar), w2 = ff2d(wt.w), w2b = ff2d(wt.wbar);
    const double lo = w2b * G64[o] + w2 * G64[o + 1];
    const double hi = w2b * G64[o + nt] + w2 * G64[o + nt + 1];
    v = w1b * lo + w1 * hi;
  }
}

// Streams one tile's pairs: scalar head to an even pair, two pairs per
// thread with 128-bit loads and stores, scalar tail.
template <class CR, class CT>
__device__ __forceinline__ void stream_pairs(const BatchArgs2D& a, const StagedView& vr, const StagedView& vt,
                                             const float4* __restrict__ G, const double* __restrict__ G64,
                                             const Tile& tile, int& nans, int& fallbacks, CR&& count_r,
                                             CT&& count_t) {
  const int64_t b = tile.begin;
  const int cnt = tile.count;
  auto scalar = [&](int i) {
    int ir, it;
    double v;
    pair_2d(vr, vt, G, G64, a.Y2[2 * (b + i)], a.Y2[2 * (b + i) + 1], ir, it, v, nans, count_r, count_t, a.extrap,
            a.logspace);
    a.idx[2 * (b + i)] = ir;
    a.idx[2 * (b + i) + 1] = it;
    a.val[b + i] = v;
  };
  const int head = a.vec ? min(cnt, (int)(b & 1)) : cnt;
  const int np2 = (cnt - head) >> 1;
  for (int i = threadIdx.x; i < head; i += blockDim.x) scalar(i);
  const double2* Y = reinterpret_cast<const double2*>(a.Y2) + b + head;
  int4* I4 = reinterpret_cast<int4*>(a.idx + 2 * (b + head));
  double2* V2 = reinterpret_cast<double2*>(a.val + b + head);
  for (int g = threadIdx.x; g < np2; g += blockDim.x) {
    double2 p0, p1;
    if (a.vec == 2) {       // both pairs in one 256-bit load
      double y[4];
      ld_stream4(reinterpret_cast<const double*>(Y + 2 * g), y);
      p0 = make_double2(y[0], y[1]);
      p1 = make_double2(y[2], y[3]);
    } else {
      p0 = ld_stream(Y + 2 * g);
      p1 = ld_stream(Y + 2 * g + 1);
    }
    int i0, j0, i1, j1;
    double v0, v1;
    pair_2d(vr, vt, G, G64, p0.x, p0.y, i0, j0, v0, nans, count_r, count_t, a.extrap, a.logspace);
    pair_2d(vr, vt, G, G64, p1.x, p1.y, i1, j1, v1, nans, count_r, count_t, a.extrap, a.logspace);
    st_stream(I4 + g, make_int4(i0, j0, i1, j1));
    st_stream(V2 + g, make_double2(v0, v1));
  }
  for (int i = head + 2 * np2 + threadIdx.x; i < cnt; i += blockDim.x) scalar(i);
}

// Hunt order (SS_MODEL_HUNT, coherent sequences): a thread's first pair is
// searched with each axis' own search (the tile's fast path where it
// applies), its second pair hunts on each axis from the first pair's
// indices (hunt_from: probes in doubling steps, then bisects; exact for any
// guess).  Head and tail pairs take the axes' own searches.
template <class CR, class CT>
__device__ __forceinline__ void stream_pairs_hunt(const BatchArgs2D& a, const StagedView& vr, const StagedView& vt,
                                                  const float4* __restrict__ G, const double* __restrict__ G64,
                                                  const Tile& tile, int& nans, CR&& count_r, CT&& count_t) {
  const int64_t b = tile.begin;
  const int cnt = tile.count;
  auto scalar = [&](int i) {
    int ir, it;
    double v;
    pair_2d(vr, vt, G, G64, a.Y2[2 * (b + i)], a.Y2[2 * (b + i) + 1], ir, it, v, nans, count_r, count_t, a.extrap,
            a.logspace);
    a.idx[2 * (b + i)] = ir;
    a.idx[2 * (b + i) + 1] = it;
    a.val[b + i] = v;
  };
  const int head = a.vec ? min(cnt, (int)(b & 1)) : cnt;
  const int np2 = (cnt - head) >> 1;
  for (int i = threadIdx.x; i < head; i += blockDim.x) scalar(i);
  const double2* Y = reinterpret_cast<const double2*>(a.Y2) + b + head;
  int4* I4 = reinterpret_cast<int4*>(a.idx + 2 * (b + head));
  double2* V2 = reinterpret_cast<double2*>(a.val + b + head);
  for (int g = threadIdx.x; g < np2; g += blockDim.x) {
    double2 p0, p1;
    if (a.vec == 2) {
      double y[4];
      ld_stream4(reinterpret_cast<const double*>(Y + 2 * g), y);
      p0 = make_double2(y[0], y[1]);
      p1 = make_double2(y[2], y[3]);
    } else {
      p0 = ld_stream(Y + 2 * g);
      p1 = ld_stream(Y + 2 * g + 1);
    }
    int i0, j0, i1, j1;
    double v0, v1;
    pair_2d(vr, vt, G, G64, p0.x, p0.y, i0, j0, v0, nans, count_r, count_t, a.extrap, a.logspace);
    pair_2d(vr, vt, G, G64, p1.x, p1.y, i1, j1, v1, nans,
            [&](double, uint64_t q) { return hunt_count(vr, i0, q); },
            [&](double, uint64_t q) { return hunt_count(vt, j0, q); }, a.extrap, a.logspace);
    st_stream(I4 + g, make_int4(i0, j0, i1, j1));
    st_stream(V2 + g, make_double2(v0, v1));
  }
  for (int i = head + 2 * np2 + threadIdx.x; i < cnt; i += blockDim.x) scalar(i);
}

// Three blocks per SM (80 registers).  A plan without position models runs
// the kernel built without them (LEARNED false), which fits that budget
// without spilling.
template <bool HUNT, bool LEARNED>
__global__ void __launch_bounds__(kNumThreads, 3) k_batched_2d(BatchArgs2D a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ int s_tile;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  int cur = -1;
  StagedView vr{}, vt{};
  int t_off = 0;
  bool ok = true;
  int nans = 0, fallbacks = 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    if (tile.table != cur) {
      const unsigned char* br = a.blobs + a.blob_off[2 * tile.table];
      const unsigned char* bt = a.blobs + a.blob_off[2 * tile.table + 1];
      // the rho axis goes first, the T axis at the next 128-byte boundary
      const BlobHdr* hr = reinterpret_cast<const BlobHdr*>(br);
      int lo, hi;
      BlobHdr hcopy;
      const int4* g4 = reinterpret_cast<const int4*>(hr);
      int4* c4 = reinterpret_cast<int4*>(&hcopy);
#pragma unroll
      for (int i = 0; i < 8; ++i) c4[i] = __ldg(g4 + i);
      staged_range(hcopy, lo, hi);
      t_off = (((int)sizeof(BlobHdr) + hi - lo) + 127) & ~127;
      vr = stage_blob(br, smem, &bar, phase, ok);
      if (ok) vt = stage_blob(bt, smem + t_off, &bar, phase, ok);
      cur = tile.table;
      if (!ok) break;
    }
    const float4* G = a.cells + 2 * a.cell_off[tile.table];
    const double* G64 = a.grid64 != nullptr ? a.grid64 + a.grid_off[tile.table] : nullptr;
    // one uniform branch per tile: both axes plain bucket searches over whole
    // staged tables with at most two keys per bucket (the common case) take a
    // branch-free two-key scan; every other combination the generic dispatch
    auto generic = [&](const StagedView& v) {
      return [&v, &fallbacks](double t, uint64_t q) { return axis_count<LEARNED>(v, t, q, fallbacks); };
    };
    auto scan2 = [](const StagedView& v) {
      const uint64_t* keys = v.keys;
      const uint16_t* dir = v.dir;
      const int shift = v.h.shift, nb = v.h.nb;
      const uint64_t base = v.h.base;
      return [=](double, uint64_t q) { return search_bucket<2>(keys, dir, shift, base, nb, q); };
    };
    auto fast = [](const StagedView& v) {
      return v.h.algo == BL_BUCKET && v.h.stride == 1 && v.h.occ <= 2;
    };
    if (HUNT) {
      if (fast(vr) && fast(vt)) stream_pairs_hunt(a, vr, vt, G, G64, tile, nans, scan2(vr), scan2(vt));
      else stream_pairs_hunt(a, vr, vt, G, G64, tile, nans, generic(vr), generic(vt));
    } else if (fast(vr) && fast(vt)) {
      stream_pairs(a, vr, vt, G, G64, tile, nans, fallbacks, scan2(vr), scan2(vt));
    } else {
      // a plan's model is the same on both axes: one uniform branch per tile
      // picks its proposal, so the pairs run it as straight-line code
      bool done = false;
      if constexpr (LEARNED) {
        const int al = vr.h.algo;
        if (al == vt.h.algo && al == BL_SPLINE) {
          stream_pairs(a, vr, vt, G, G64, tile, nans, fallbacks,
                              [&](double, uint64_t q) { return spline_count(vr, q, fallbacks); },
                              [&](double, uint64_t q) { return spline_count(vt, q, fallbacks); });
          done = true;
        } else if (al == vt.h.algo && al == BL_LOGHASH) {
          stream_pairs(a, vr, vt, G, G64, tile, nans, fallbacks,
                              [&](double t, uint64_t q) { return loghash_count(vr, t, q, fallbacks); },
                              [&](double t, uint64_t q) { return loghash_count(vt, t, q, fallbacks); });
          done = true;
        } else if (al == vt.h.algo && al == BL_MLP) {
          stream_pairs(a, vr, vt, G, G64, tile, nans, fallbacks,
                              [&](double t, uint64_t q) { return mlp_count(vr, t, q, fallbacks); },
                              [&](double t, uint64_t q) { return mlp_count(vt, t, q, fallbacks); });
          done = true;
        }
      }
      if (!done) stream_pairs(a, vr, vt, G, G64, tile, nans, fallbacks, generic(vr), generic(vt));
    }
  }
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  fallbacks = __reduce_add_sync(0xFFFFFFFFu, fallbacks);
  if (a.stat != nullptr && (threadIdx.x & 31) == 0) {
    if (nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
    if (fallbacks) atomicAdd(&a.stat->fallbacks, (unsigned long long)fallbacks);
  }
  if (a.stat != nullptr && threadIdx.x == 0 && !ok) atomicOr(&a.stat->flags, SS_FLAG_STAGING_TIMEOUT);
  SS_BOUNDS_FOLD(a.stat);
}

// ---------------------------------------------------------------------------
// Lean kernel for the common case, launched when every axis of the plan is
// searched by the bucket directory over a whole staged table with at most
// two keys per bucket, every cell is in the float-float range and no
// interpolation option is set (checked on the device when a batch is bound,
// k_fast_2d_check): per axis it keeps only the handful of fields that case
// reads, as shared-memory offsets, so fewer registers stay live and more
// warps fit on an SM than in the general kernel.  Plans with a position
// model (spline, MLP, logarithm hash) run instances of it (MODEL) when,
// besides, every axis is that model's proposal with a window of at most
// kProbeWindow keys: the proposal is proved by the walk of the general
// kernel (same answers, same fallbacks), the fallback is the two-key bucket
// scan.  Hunt plans (Sec. 2.1) run the instance in which a thread's second
// pair of a step hunts from the first pair's answers, as in the general
// kernel.
// ---------------------------------------------------------------------------
enum FastModel { kFastPlain = 0, kFastSpline = 1, kFastLogHash = 2, kFastMlp = 3, kFastHunt = 4 };

struct FastAxis {
  int keys, dir, ca, cg;     // shared-memory byte offsets: keys, directory, cell records, cell scales
  int shift, nb, n;
  int E;                     // learned half-window (learned instances)
  float la, lc;              // logarithm-hash coefficients (that instance)
  int mlp;                   // shared-memory byte offset of the MLP parameters (that instance)
  MlpFeatScale sc;           // MLP feature scaling (that instance)
  uint64_t base, k0;
};

__device__ __forceinline__ FastAxis fast_axis(const StagedView& v, const unsigned char* smem) {
  FastAxis f;
  f.keys = (int)(reinterpret_cast<const unsigned char*>(v.keys) - smem);
  f.dir = (int)(reinterpret_cast<const unsigned char*>(v.dir) - smem);
  f.ca = (int)(reinterpret_cast<const unsigned char*>(v.cells.a) - smem);
  f.cg = (int)(reinterpret_cast<const unsigned char*>(v.cells.g) - smem);
  f.shift = v.h.shift;
  f.nb = v.h.nb;
  f.n = v.h.n;
  f.base = v.h.base;
  f.k0 = v.h.k0;
  f.E = v.h.E;
  f.la = f.lc = 0.0f;
  if (v.h.algo == BL_LOGHASH) {
    f.la = v.mlp[kMlpParams];
    f.lc = v.mlp[kMlpParams + 1];
  }
  f.mlp = (int)(reinterpret_cast<const unsigned char*>(v.mlp) - smem);
  f.sc = MlpFeatScale{v.h.e_lo, v.h.e_scale};
  return f;
}

// The MLP's proposal (mlp_propose, same arithmetic in the same order) with
// its parameters read four at a time.  The staged part of an MLP axis
// begins with its parameters, right after the 128-byte header, and each
// axis is staged at a 128-byte boundary of shared memory, so p is 16-byte
// aligned (the bounds-checked build takes mlp_propose for any p that is
// not, which nothing staged produces).
__device__ __forceinline__ int fast_mlp_propose(const float* __restrict__ p, const MlpFeatScale& s, int n,
                                                double t) {
#ifdef SS_CHECKED
  if ((reinterpret_cast<uintptr_t>(p) & 15) != 0) return mlp_propose(p, s, n, t);
#endif
  float x0, x1;
  mlp_features(t, s, x0, x1);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  float y = p[4 * kHidden];
#pragma unroll
  for (int k4 = 0; k4 < kHidden / 4; ++k4) {
    // units 4 k4 .. 4 k4 + 3: input weights (interleaved pairs), biases, output weights
    const float4 wa = p4[2 * k4], wb = p4[2 * k4 + 1];
    const float4 bk = p4[kHidden / 2 + k4], vk = p4[3 * kHidden / 4 + k4];
    y = fmaf(vk.x, fmaxf(fmaf(wa.x, x0, fmaf(wa.y, x1, bk.x)), 0.0f), y);
    y = fmaf(vk.y, fmaxf(fmaf(wa.z, x0, fmaf(wa.w, x1, bk.y)), 0.0f), y);
    y = fmaf(vk.z, fmaxf(fmaf(wb.x, x0, fmaf(wb.y, x1, bk.z)), 0.0f), y);
    y = fmaf(vk.w, fmaxf(fmaf(wb.z, x0, fmaf(wb.w, x1, bk.w)), 0.0f), y);
  }
  const float pos = rintf(y * (float)(n - 1));
  return (int)fminf(fmaxf(pos, 0.0f), (float)(n - 1));     // NaN -> 0 through fmaxf
}

// Count of keys below q on a fast axis: the bucket directory's two-key scan,
// or (learned instances) the model's proposal proved by a walk of at most E
// keys, with the scan as fallback, or (hunt instance, guess >= 0) a hunt
// from the guess with the scan beyond its probes.  n - 1 keys are searched.
template <int MODEL, int HI>
__device__ __forceinline__ int fast_count(const unsigned char* smem, const FastAxis& f, double t, uint64_t q,
                                          int& fallbacks, int guess) {
  const uint64_t* keys = reinterpret_cast<const uint64_t*>(smem + f.keys);
  const uint16_t* dir = reinterpret_cast<const uint16_t*>(smem + f.dir);
  if constexpr (MODEL == kFastHunt) {
    (void)t;
    (void)fallbacks;
    if (guess >= 0) {
      const int lim = f.n - 1 + kPad;
      return hunt_from([keys, lim](int i) { return keys[SS_IX(i, lim)]; }, f.n - 1, guess, q,
                       [&](uint64_t qq) { return search_bucket<2, HI>(keys, dir, f.shift, f.base, f.nb, qq); });
    }
  } else if constexpr (MODEL != kFastPlain) {
    (void)guess;
    const int nk = f.n - 1;
    int p;
    if constexpr (MODEL == kFastSpline) p = min((int)rintf(spline_position(dir, f.shift, f.base, f.nb, q)), nk);
    else if constexpr (MODEL == kFastLogHash) p = loghash_propose(f.la, f.lc, nk, t);
    else p = fast_mlp_propose(reinterpret_cast<const float*>(smem + f.mlp), f.sc, f.n, t);
    int c;
    if (walk_count(keys, nk + kPad, nk, f.E, p, q, c)) return c;
    ++fallbacks;
  } else {
    (void)t;
    (void)fallbacks;
    (void)guess;
  }
  return search_bucket<2, HI>(keys, dir, f.shift, f.base, f.nb, q);
}

// Weights of coordinate bits u (key k, index i, cell c) on a fast axis.
__device__ __forceinline__ Weights fast_weights(const unsigned char* smem, const FastAxis& f, int i, int c, uint64_t k,
                                                uint64_t u) {
  if (i >= f.n - 1) return {{1.0f, 0.0f}, {0.0f, 0.0f}};
  if (i == 0 && k <= f.k0) return {{0.0f, 0.0f}, {1.0f, 0.0f}};
#ifdef SS_CHECKED
  const CellTable t{reinterpret_cast<const ulonglong2*>(smem + f.ca), reinterpret_cast<const float2*>(smem + f.cg),
                    f.n - 1};
#else
  const CellTable t{reinterpret_cast<const ulonglong2*>(smem + f.ca), reinterpret_cast<const float2*>(smem + f.cg)};
#endif
  return cell_weights(u, t, c);
}

// gr, gt: the hunt instance's guesses (below zero: none)
template <int MODEL, int HI>   // HI 1: both bucket shifts are 32 or more; -1: decided per call
__device__ __forceinline__ void pair_fast(const unsigned char* smem, const FastAxis& fr, const FastAxis& ft,
                                          const float4* __restrict__ G, uint64_t keep, double rho, double tem,
                                          int& ir, int& it, double& v, int& nans, int& fallbacks, int gr = -1,
                                          int gt = -1) {
  const uint64_t ur = static_cast<uint64_t>(__double_as_longlong(rho));
  const uint64_t ut = static_cast<uint64_t>(__double_as_longlong(tem));
  const uint64_t kr = order_key(rho), kt = order_key(tem);
  const bool nan = (kr < kKeyNegInf) | (kt < kKeyNegInf);
  nans += (kr < kKeyNegInf) + (kt < kKeyNegInf);
  ir = fast_count<MODEL, HI>(smem, fr, rho, kr, fallbacks, gr);
  it = fast_count<MODEL, HI>(smem, ft, tem, kt, fallbacks, gt);
  const int cr = min(ir, fr.n - 2), ct = min(it, ft.n - 2);
  const int64_t cell = (int64_t)cr * (ft.n - 1) + ct;
  float q[8];
  ld_nc_v8_policy(reinterpret_cast<const float*>(G + 2 * cell), q, keep);
  const Weights wr = fast_weights(smem, fr, ir, cr, kr, ur);
  const Weights wt = fast_weights(smem, ft, it, ct, kt, ut);
  const ff lo = ff_add_u(ff_mul_u(wt.wbar, ff{q[0], q[1]}), ff_mul_u(wt.w, ff{q[2], q[3]}));
  const ff hi = ff_add_u(ff_mul_u(wt.wbar, ff{q[4], q[5]}), ff_mul_u(wt.w, ff{q[6], q[7]}));
  v = nan ? __longlong_as_double(0x7FF8000000000000ll) : ff2d(ff_add_u(ff_mul_u(wr.wbar, lo), ff_mul_u(wr.w, hi)));
}

// Four blocks of 256 threads per SM (at most 64 registers, no spills, in
// every instance; the general kernel's 80 registers allow three).  Two pairs per thread and step, as in
// the general kernel: one pair per step measured 6 % slower.  Corner
// gathers carry an evict-last L2 policy and the 256-bit target loads an
// evict-first one (1-2 % measured).
template <int MODEL>
__global__ void __launch_bounds__(kNumThreads, 4) k_batched_2d_fast(BatchArgs2D a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint64_t keep = l2_policy_evict_last(), pass = l2_policy_evict_first();
  __shared__ uint64_t bar;
  __shared__ int s_tile;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  int cur = -1;
  FastAxis fr{}, ft{};
  bool ok = true;
  int nans = 0, fallbacks = 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    if (tile.table != cur) {
      const unsigned char* br = a.blobs + a.blob_off[2 * tile.table];
      const unsigned char* bt = a.blobs + a.blob_off[2 * tile.table + 1];
      BlobHdr hcopy;
      const int4* g4 = reinterpret_cast<const int4*>(br);
      int4* c4 = reinterpret_cast<int4*>(&hcopy);
#pragma unroll
      for (int i = 0; i < 8; ++i) c4[i] = __ldg(g4 + i);
      int lo, hi;
      staged_range(hcopy, lo, hi);
      const int t_off = (((int)sizeof(BlobHdr) + hi - lo) + 127) & ~127;
      const StagedView vr = stage_blob(br, smem, &bar, phase, ok);
      if (!ok) break;
      const StagedView vt = stage_blob(bt, smem + t_off, &bar, phase, ok);
      if (!ok) break;
      fr = fast_axis(vr, smem);
      ft = fast_axis(vt, smem);
      cur = tile.table;
    }
    const float4* G = a.cells + 2 * a.cell_off[tile.table];
    const int64_t b = tile.begin;
    const int cnt = tile.count;
    auto scalar = [&](int i) {
      int ir, it;
      double v;
      pair_fast<MODEL, -1>(smem, fr, ft, G, keep, a.Y2[2 * (b + i)], a.Y2[2 * (b + i) + 1], ir, it, v, nans,
                           fallbacks);
      a.idx[2 * (b + i)] = ir;
      a.idx[2 * (b + i) + 1] = it;
      a.val[b + i] = v;
    };
    if (!a.vec) {            // arrays off 16-byte alignment: scalar accesses
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) scalar(i);
      continue;
    }
    const int head = min(cnt, (int)(b & 1));
    const int np2 = (cnt - head) >> 1;
    for (int i = threadIdx.x; i < head; i += blockDim.x) scalar(i);
    const double2* Y = reinterpret_cast<const double2*>(a.Y2) + b + head;
    int4* I4 = reinterpret_cast<int4*>(a.idx + 2 * (b + head));
    double2* V2 = reinterpret_cast<double2*>(a.val + b + head);
    // the bucket index from the keys' high words when both shifts allow
    // (straight-line pairs; 2 % measured), else decided per call
    auto pairs = [&](auto hi) {
      constexpr int HI = decltype(hi)::value;
      for (int g = threadIdx.x; g < np2; g += blockDim.x) {
        double2 p0, p1;
        if (a.vec == 2) {
          double y[4];
          ld_stream4_policy(reinterpret_cast<const double*>(Y + 2 * g), y, pass);
          p0 = make_double2(y[0], y[1]);
          p1 = make_double2(y[2], y[3]);
        } else {
          p0 = ld_stream(Y + 2 * g);
          p1 = ld_stream(Y + 2 * g + 1);
        }
        int i0, j0, i1, j1;
        double v0, v1;
        pair_fast<MODEL, HI>(smem, fr, ft, G, keep, p0.x, p0.y, i0, j0, v0, nans, fallbacks);
        pair_fast<MODEL, HI>(smem, fr, ft, G, keep, p1.x, p1.y, i1, j1, v1, nans, fallbacks, i0, j0);
        st_stream(I4 + g, make_int4(i0, j0, i1, j1));
        st_stream(V2 + g, make_double2(v0, v1));
      }
    };
    if (fr.shift >= 32 && ft.shift >= 32) pairs(std::integral_constant<int, 1>{});
    else pairs(std::integral_constant<int, -1>{});
    for (int i = head + 2 * np2 + threadIdx.x; i < cnt; i += blockDim.x) scalar(i);
  }
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  if (a.stat != nullptr && (threadIdx.x & 31) == 0 && nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
  if constexpr (MODEL != kFastPlain) {
    fallbacks = __reduce_add_sync(0xFFFFFFFFu, fallbacks);
    if (a.stat != nullptr && (threadIdx.x & 31) == 0 && fallbacks)
      atomicAdd(&a.stat->fallbacks, (unsigned long long)fallbacks);
  }
  if (a.stat != nullptr && threadIdx.x == 0 && !ok) atomicOr(&a.stat->flags, SS_FLAG_STAGING_TIMEOUT);
  SS_BOUNDS_FOLD(a.stat);
}

// Eligibility of a plan for the lean kernel: *not_fast stays 0 when every
// axis is searched with algorithm `algo` over a whole staged table with at
// most two keys per bucket and float-float cell data, and, for a position
// model (spline, MLP, logarithm hash), with a window of at most kProbeWindow
// keys.
__global__ void k_fast_2d_check(const unsigned char* __restrict__ blobs, const int64_t* __restrict__ blob_off,
                                int naxes, int algo, unsigned* not_fast) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < naxes; j += gridDim.x * blockDim.x) {
    const BlobHdr* h = reinterpret_cast<const BlobHdr*>(blobs + blob_off[j]);
    if (!(h->algo == algo && h->stride == 1 && h->occ <= 2 && h->ffok == 1 && h->off_cells >= 0 &&
          (algo == BL_BUCKET || h->E <= kProbeWindow)))
      atomicOr(not_fast, 1u);
  }
}

const void* batched_2d_fast_kernel(int algo, bool hunt) {
  if (hunt) return reinterpret_cast<const void*>(&k_batched_2d_fast<kFastHunt>);
  if (algo == BL_SPLINE) return reinterpret_cast<const void*>(&k_batched_2d_fast<kFastSpline>);
  if (algo == BL_LOGHASH) return reinterpret_cast<const void*>(&k_batched_2d_fast<kFastLogHash>);
  if (algo == BL_MLP) return reinterpret_cast<const void*>(&k_batched_2d_fast<kFastMlp>);
  return reinterpret_cast<const void*>(&k_batched_2d_fast<kFastPlain>);
}

// Kernel entry of the batched 2D lookup (template stubs stay local to this unit).
const void* batched_2d_kernel(bool hunt, bool learned) {
  if (learned)
    return hunt ? reinterpret_cast<const void*>(&k_batched_2d<true, true>) : reinterpret_cast<const void*>(&k_batched_2d<false, true>);
  return hunt ? reinterpret_cast<const void*>(&k_batched_2d<true, false>) : reinterpret_cast<const void*>(&k_batched_2d<false, false>);
}

void plan_cell_offsets(PlanBase* p) {
  p->cell_off.assign(p->ntables + 1, 0);
  for (int k = 0; k < p->ntables; ++k)
    p->cell_off[k + 1] = p->cell_off[k] + (int64_t)(p->sizes[k] - 1) * (p->sizes_t[k] - 1);
}

ss_status plan_build_2d(ss_plan* p, const double* R, const double* T, const double* F, cudaStream_t stream) {
  const int nt = p->ntables;
  const ss_plan_opts& o = p->opts;
  p->dir_cap.resize(2 * nt);
  p->algo.assign(2 * nt, initial_algo(o));
  p->blob_off.resize(2 * nt);
  int64_t off = 0;
  for (int k = 0; k < nt; ++k) {
    for (int ax = 0; ax < 2; ++ax) {
      const int n = ax == 0 ? p->sizes[k] : p->sizes_t[k];
      const int j = 2 * k + ax;
      p->dir_cap[j] = o.dir_cap > 0 ? o.dir_cap : default_dir_cap(n);
      p->blob_off[j] = off;
      off += (blob_geom_dev(n, p->dir_cap[j], true).bytes + 255) & ~(int64_t)255;
    }
  }
  p->blob_bytes = off;
  for (int b = 0; b < kNumBuckets; ++b) {
    p->bucket_algo[b] = initial_algo(o);
    p->bucket_tile[b] = o.tile > 0 ? o.tile : kDefaultTile / 2;
    p->bucket_tables[b] = 0;
  }
  for (int k = 0; k < nt; ++k) p->bucket_tables[size_bucket(std::max(p->sizes[k], p->sizes_t[k]))]++;
  const int64_t gcount = p->grid_off[nt];
  plan_cell_offsets(p);
  const int64_t ncells = p->cell_off[nt];
  std::vector<int64_t> offR(nt), offT(nt), axR(nt + 1), axT(nt + 1);
  for (int k = 0; k < nt; ++k) { offR[k] = p->blob_off[2 * k]; offT[k] = p->blob_off[2 * k + 1]; }
  for (int k = 0; k <= nt; ++k) { axR[k] = p->X_off[k]; axT[k] = p->X_off[nt + 1 + k]; }
  std::vector<int> capR(nt), capT(nt), algR(nt), algT(nt);
  for (int k = 0; k < nt; ++k) {
    capR[k] = p->dir_cap[2 * k]; capT[k] = p->dir_cap[2 * k + 1];
    algR[k] = p->algo[2 * k]; algT[k] = p->algo[2 * k + 1];
  }
  std::vector<void*> temps;
  auto dev_copy = [&](const void* src, size_t bytes) -> void* {
    void* d = nullptr;
    if (cudaMalloc(&d, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    temps.push_back(d);
    if (cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return d;
  };
  auto cleanup = [&]() { for (void* d : temps) cudaFree(d); };
  if (cudaMalloc(&p->d_blobs, p->blob_bytes) != cudaSuccess ||
      cudaMalloc(&p->d_grid, std::max<int64_t>(ncells, 1) * 4 * sizeof(float2)) != cudaSuccess) {
    return fail(SS_ENOMEM, "plan: device allocation failed");
  }
  p->device_bytes = p->blob_bytes + ncells * 4 * (int64_t)sizeof(float2);
  ss_status st = [&]() -> ss_status {
    SS_CHECK_CUDA(cudaMalloc(&p->d_blob_off, 2 * nt * sizeof(int64_t)));
    SS_CHECK_CUDA(cudaMemcpy(p->d_blob_off, p->blob_off.data(), 2 * nt * sizeof(int64_t), cudaMemcpyHostToDevice));
    SS_CHECK_CUDA(cudaMalloc(&p->d_grid_off, (nt + 1) * sizeof(int64_t)));
    SS_CHECK_CUDA(cudaMemcpy(p->d_grid_off, p->grid_off.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    SS_CHECK_CUDA(cudaMalloc(&p->d_cell_off, (nt + 1) * sizeof(int64_t)));
    SS_CHECK_CUDA(cudaMemcpy(p->d_cell_off, p->cell_off.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    auto* dR = (int64_t*)dev_copy(offR.data(), nt * 8);
    auto* dT = (int64_t*)dev_copy(offT.data(), nt * 8);
    auto* dAR = (int64_t*)dev_copy(axR.data(), (nt + 1) * 8);
    auto* dAT = (int64_t*)dev_copy(axT.data(), (nt + 1) * 8);
    auto* dCR = (int*)dev_copy(capR.data(), nt * 4);
    auto* dCT = (int*)dev_copy(capT.data(), nt * 4);
    auto* dGR = (int*)dev_copy(algR.data(), nt * 4);
    auto* dGT = (int*)dev_copy(algT.data(), nt * 4);
    unsigned zero[2] = {0, 0};
    auto* dBad = (unsigned*)dev_copy(zero, 8);
    if (!dR || !dT || !dAR || !dAT || !dCR || !dCT || !dGR || !dGT || !dBad) return fail(SS_ENOMEM, "plan: device allocation failed");
    PrepArgs pr{nt, dAR, R, p->d_blobs, dR, dCR, dGR, 1, dBad};
    PrepArgs pt{nt, dAT, T, p->d_blobs, dT, dCT, dGT, 1, dBad};
    k_prep_1d<<<nt, 256, 0, stream>>>(pr);
    k_prep_1d<<<nt, 256, 0, stream>>>(pt);
    k_prep_cells<<<nt, 256, 0, stream>>>(pr);
    k_prep_cells<<<nt, 256, 0, stream>>>(pt);
    SS_CHECK_CUDA(cudaGetLastError());
    k_grid_cells<<<nt, 256, 0, stream>>>(F, p->d_grid_off, dAR, dAT, p->d_cell_off,
                                          reinterpret_cast<float4*>(p->d_grid), dBad + 1);
    SS_CHECK_CUDA(cudaGetLastError());
    if (o.model == SS_MODEL_MLP && o.mlp_epochs > 0) {
      TrainArgs ta{2 * nt, p->d_blobs, p->d_blob_off, o.mlp_epochs,
                   o.mlp_lr > 0 ? o.mlp_lr : 2e-3f, o.seed};
      k_train_mlp<<<2 * nt, 256, 0, stream>>>(ta);
      SS_CHECK_CUDA(cudaGetLastError());
    }
    if (o.model != SS_MODEL_NONE) {
      WindowArgs wa{2 * nt, p->d_blobs, p->d_blob_off, o.seed ^ 0xA5A5A5A5ull};
      k_window<<<2 * nt, 256, 0, stream>>>(wa);
      SS_CHECK_CUDA(cudaGetLastError());
    }
    SS_CHECK_CUDA(cudaStreamSynchronize(stream));
    unsigned bad[2];
    SS_CHECK_CUDA(cudaMemcpy(bad, dBad, 8, cudaMemcpyDeviceToHost));
    if (bad[0]) return fail(SS_ENOTSORTED, "ss_plan_create_2d: an axis is not strictly increasing (or holds NaN)");
    if (bad[1] || o.extrap || o.logspace) {
      // some values need the fp64 blend (values outside the float-float
      // range, or the interpolation options): keep a copy of the caller's grids
      SS_CHECK_CUDA(cudaMalloc(&p->d_grid64, gcount * sizeof(double)));
      SS_CHECK_CUDA(cudaMemcpy(p->d_grid64, F, gcount * sizeof(double), cudaMemcpyDeviceToDevice));
      p->device_bytes += gcount * (int64_t)sizeof(double);
    }
    return SS_OK;
  }();
  cleanup();
  if (st != SS_OK) return st;
  if (o.autotune) {
    if ((st = plan_tune(p, stream)) != SS_OK) return st;
  }
  return plan_window_stats(p);
}

}  // namespace ss

using namespace ss;

extern "C" ss_status ss_plan_create_2d(ss_plan** out, int32_t ntables, const int64_t* R_off, const double* R,
                                       const int64_t* T_off, const double* T, const int64_t* F_off, const double* F,
                                       const ss_plan_opts* opts_in, cudaStream_t stream) {
  if (out == nullptr || R_off == nullptr || T_off == nullptr || F_off == nullptr || R == nullptr || T == nullptr ||
      F == nullptr)
    return fail(SS_EINVAL, "ss_plan_create_2d: null pointer");
  *out = nullptr;
  if (ntables < 1) return fail(SS_EINVAL, "ss_plan_create_2d: ntables must be >= 1");
  if (!aligned(R, 8) || !aligned(T, 8) || !aligned(F, 8)) return fail(SS_EINVAL, "ss_plan_create_2d: misaligned pointer");
  ss_plan_opts o;
  ss_plan_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (ss_status st = check_plan_opts(o, 2)) return st;
  auto* p = new ss_plan();
  p->kind = 2;
  p->ntables = ntables;
  p->opts = o;
  p->sizes.resize(ntables);
  p->sizes_t.resize(ntables);
  p->X_off.resize(2 * (ntables + 1));
  p->grid_off.assign(F_off, F_off + ntables + 1);
  for (int k = 0; k <= ntables; ++k) {
    p->X_off[k] = R_off[k];
    p->X_off[ntables + 1 + k] = T_off[k];
  }
  for (int k = 0; k < ntables; ++k) {
    const int64_t nr = R_off[k + 1] - R_off[k], ntt = T_off[k + 1] - T_off[k];
    if (nr < 2 || ntt < 2 || nr > (1 << 20) || ntt > (1 << 20) || F_off[k + 1] - F_off[k] != nr * ntt || F_off[k] < 0) {
      delete p;
      return fail(SS_EINVAL, "ss_plan_create_2d: each table needs axes of >= 2 entries and nr*nt values");
    }
    p->sizes[k] = (int)nr;
    p->sizes_t[k] = (int)ntt;
  }
  ss_status st = plan_build_2d(p, R, T, F, stream);
  if (st != SS_OK) {
    delete p;
    return st;
  }
  *out = p;
  return SS_OK;
}

extern "C" ss_status ss_plan_bind_2d(ss_plan* p, const int64_t* Y_off, const double* Y2, int32_t* lowbounds2,
                                     double* values, ss_devstat* stat, cudaStream_t stream) {
  if (p == nullptr || Y_off == nullptr) return fail(SS_EINVAL, "ss_plan_bind_2d: null pointer");
  if (p->kind != 2) return fail(SS_EINVAL, "ss_plan_bind_2d: not a 2D plan");
  if (Y_off[p->ntables] > 0 && (Y2 == nullptr || lowbounds2 == nullptr || values == nullptr))
    return fail(SS_EINVAL, "ss_plan_bind_2d: null pointer");
  if (!aligned(Y2, 8) || !aligned(lowbounds2, 4) || !aligned(values, 8))
    return fail(SS_EINVAL, "ss_plan_bind_2d: misaligned pointer");
  for (int k = 0; k < p->ntables; ++k)
    if (Y_off[k + 1] < Y_off[k] || Y_off[k] < 0) return fail(SS_EINVAL, "ss_plan_bind_2d: offsets must be non-decreasing");
  return plan_bind(p, std::vector<int64_t>(Y_off, Y_off + p->ntables + 1), Y2, lowbounds2, values, stat, stream);
}
