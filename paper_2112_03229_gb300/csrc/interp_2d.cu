// interp_2d.cu -- one-shot fused 2D lookup (Sec. 1 and 2.2: EOSPAC bounds
// each (density, temperature) target in both grids of a SESAME table and
// interpolates).  Per pair: two exact searches (the 1D routines of
// ss_table.cuh on two staged axes), cell selection c = min(i, n-2), clamped
// weights, four gathers from the row-major value grid and the convex
// bilinear blend.
//
// Two arithmetic paths, chosen once per launch from the staged axes:
//  * float-float (default): exact integer weight numerators and a
//    float-float blend on the fp32 pipe (ss_ff.cuh); needs positive axes
//    with entries in [2^-70, 2^101) and cells spanning at most 2^10.
//    A pair whose four grid values are not positive and in that range is
//    finished in fp64.
//  * fp64: weights (x - X[c]) * (1 / gap) and the blend in double.
// Both agree with an fp64 evaluation of the formula to well within 1e-12
// relative for positive grids.
//
// Interpolation options: linear extrapolation (no weight clamp) sends the
// pairs outside either axis to the fp64 path with unclamped weights; log
// coordinates (weights (ln x - ln X[c]) / (ln X[c+1] - ln X[c]), per-entry
// logarithms staged with the axis) run every pair on the fp64 path.
//
// The value grid stays in global memory (L2-resident for the sizes of
// interest); axes, bucket directories and per-cell data live in shared memory.
#include <algorithm>

#include "ss_ff.cuh"
#include "ss_table.cuh"

namespace ss {

constexpr int kMaxAxis2D = SS_MAX_AXIS_2D;   // largest axis staged whole with its per-cell data

struct Axis2D {                    // shared-memory offsets of one axis
  Layout1D lay;
  int cells;                       // cell table of n-1 cells (CellTable layout): exact weight numerators' data and scale
  int rg;                          // double[n-1]: 1 / (X[c+1] - X[c]) for the fp64 path (X[c] read from global);
                                   // in log coordinates 1 / (ln X[c+1] - ln X[c])
  int lx;                          // double[n]: ln X[j] (log coordinates only, else -1)
  int aux;                         // AxisAux
};

struct AxisAux {
  uint64_t k0;                     // key of X[0]
  int ffok;                        // 1 if the float-float path applies to this axis
};

struct Args2D {
  const double* R;
  int nr;
  const double* T;
  int nt;
  const double* F;
  const double* Y2;
  int64_t m;
  int32_t* idx;
  double* val;
  int64_t head;     // pairs [0, head) scalar
  int64_t np2;      // pairs in the vector body, in units of 2 pairs
  int algo;         // SS_ALGO_BUCKET or SS_ALGO_BINARY
  int force_fp64;   // 1: skip the float-float path
  int extrap;       // 1: linear extrapolation (weights not clamped)
  int logspace;     // 1: weights in natural-log axis coordinates (fp64 path)
  int grid_smem;    // offset of the float-float grid in shared memory (-1: grid stays in global memory)
  Axis2D ar, at;
  ss_devstat* stat;
};

// Per-cell data and the float-float eligibility of one axis.
static __device__ void stage_cells(const double* __restrict__ X, int n, const Axis2D& ax, unsigned char* smem) {
  double* rg = reinterpret_cast<double*>(smem + ax.rg);
  double* lx = ax.lx >= 0 ? reinterpret_cast<double*>(smem + ax.lx) : nullptr;
  AxisAux& aux = *reinterpret_cast<AxisAux*>(smem + ax.aux);
  bool ok = true;
  for (int c = threadIdx.x; c < n - 1; c += blockDim.x) {
    const double a = __ldg(X + c), b = __ldg(X + c + 1);
    if (lx != nullptr) {
      const double la = log(a), lb = log(b);
      lx[c] = la;
      if (c == n - 2) lx[n - 1] = lb;
      rg[c] = 1.0 / (lb - la);
    } else {
      rg[c] = 1.0 / (b - a);
    }
    CellW w;
    ok &= make_cell(a, b, w);
    store_cell(smem + ax.cells, n - 1, c, w);
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) {
    aux.k0 = order_key(__ldg(X));
    aux.ffok = ok ? 1 : 0;
  }
}

// Clamp to [0, 1]; NaN passes through.
__device__ __forceinline__ double clamp01(double w) { return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w); }

struct AxisView {
  const uint64_t* keys;
  const uint64_t* eyt;
  const int* dir;
  CellTable cells;
  const double* x;           // the axis in global memory
  const double* rg;
  const double* lx;          // ln X[j] (log coordinates), else nullptr
  int extrap;                // 1: weights not clamped
  int shift, nb, T, D, n;
  uint64_t base, k0;
};

__device__ __forceinline__ AxisView view_of(const Axis2D& ax, const unsigned char* smem) {
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + ax.lay.hdr);
  const AxisAux& aux = *reinterpret_cast<const AxisAux*>(smem + ax.aux);
  AxisView v;
  v.keys = ax.lay.keys >= 0 ? reinterpret_cast<const uint64_t*>(smem + ax.lay.keys) : nullptr;
  v.eyt = ax.lay.eyt >= 0 ? reinterpret_cast<const uint64_t*>(smem + ax.lay.eyt) : nullptr;
  v.dir = ax.lay.dir >= 0 ? reinterpret_cast<const int*>(smem + ax.lay.dir) : nullptr;
  v.cells = cell_table(smem + ax.cells, h.n - 1);
  v.rg = reinterpret_cast<const double*>(smem + ax.rg);
  v.lx = ax.lx >= 0 ? reinterpret_cast<const double*>(smem + ax.lx) : nullptr;
  v.extrap = 0;
  v.shift = h.shift;
  v.nb = h.nb;
  v.T = h.occ > 0 ? 32 - __clz(h.occ) : 0;
  v.D = h.D;
  v.n = h.n;
  v.base = h.base;
  v.k0 = aux.k0;
  return v;
}

template <int MODE>
__device__ __forceinline__ int axis_search(const AxisView& a, uint64_t k) {
  if (MODE == 0) return search_bucket<1>(a.keys, a.dir, a.shift, a.base, a.nb, k);
  if (MODE == 1) return search_bucket_bisect(a.keys, a.dir, a.shift, a.base, a.nb, a.T, k);
  if (MODE == 3) return search_bucket<2>(a.keys, a.dir, a.shift, a.base, a.nb, k);
  return search_eyt_rt(a.eyt, a.D, k);
}

// Float-float weights (w, 1 - w) of a target with key k and bits u whose lower-bound index is i.
__device__ __forceinline__ Weights axis_weights_ff(const AxisView& a, int i, int c, uint64_t k, uint64_t u) {
  if (i >= a.n - 1) return {{1.0f, 0.0f}, {0.0f, 0.0f}};          // above the last entry
  if (i == 0 && k <= a.k0) return {{0.0f, 0.0f}, {1.0f, 0.0f}};   // at or below the first entry
  return cell_weights(u, a.cells, c);
}

// fp64 weight of coordinate x in cell c: linear or log coordinates, clamped
// to [0, 1] unless the axis extrapolates.
__device__ __forceinline__ double weight64(const AxisView& a, int c, double x) {
  const double w = a.lx != nullptr ? (log(x) - a.lx[c]) * a.rg[c] : (x - __ldg(a.x + c)) * a.rg[c];
  return a.extrap ? w : clamp01(w);
}

// Convex blend in fp64 (fallback path of a pair).
__device__ __forceinline__ double blend64(double wr, double wt, double f00, double f01, double f10, double f11) {
  const double lo = (1.0 - wt) * f00 + wt * f01;
  const double hi = (1.0 - wt) * f10 + wt * f11;
  return (1.0 - wr) * lo + wr * hi;
}

// Same with both weights of each axis given.
__device__ __forceinline__ double blend64w(double wr, double wrb, double wt, double wtb, double f00, double f01,
                                          double f10, double f11) {
  return wrb * (wtb * f00 + wt * f01) + wr * (wtb * f10 + wt * f11);
}

// One pair: indices and value.  MODE 0: both axes bucket with occupancy <= 1;
// 3: occupancy <= 2 (a branch-free two-key scan); 1: bucket with bounded
// bisection; 2: breadth-first binary.  FF: arithmetic
// path.  SG: the value grid is staged in shared memory as float-float (a NaN
// high part marks a value the split does not cover; that pair is finished in
// fp64 from the caller's grid).
template <int MODE, bool FF, bool SG>
__device__ __forceinline__ void lookup_pair(const AxisView& vr, const AxisView& vt, const double* __restrict__ F,
                                            const float2* __restrict__ Gs, int nt, double rho, double tem, int& ir,
                                            int& it, double& v, int& nans, bool gall) {
  const uint64_t ur = static_cast<uint64_t>(__double_as_longlong(rho));
  const uint64_t ut = static_cast<uint64_t>(__double_as_longlong(tem));
  const uint64_t kr = order_key(rho), kt = order_key(tem);
  const bool nan = (kr < 0x0010000000000000ull) | (kt < 0x0010000000000000ull);
  nans += (kr < 0x0010000000000000ull) + (kt < 0x0010000000000000ull);
  ir = axis_search<MODE>(vr, kr);
  it = axis_search<MODE>(vt, kt);
  const int cr = min(ir, vr.n - 2), ct = min(it, nt - 2);
  const int64_t o = (int64_t)cr * nt + ct;
  if (!FF) {
    const double* f = F + o;
    const double f00 = __ldg(f), f01 = __ldg(f + 1), f10 = __ldg(f + nt), f11 = __ldg(f + nt + 1);
    v = blend64(weight64(vr, cr, rho), weight64(vt, ct, tem), f00, f01, f10, f11);
    return;
  }
  if (vr.extrap) {
    // linear extrapolation: a pair outside either axis takes the fp64 path with unclamped weights
    const bool outside = (ir >= vr.n - 1) | (ir == 0 && kr <= vr.k0) | (it >= vt.n - 1) | (it == 0 && kt <= vt.k0);
    if (outside) {
      const double* f = F + o;
      v = blend64(weight64(vr, cr, rho), weight64(vt, ct, tem), __ldg(f), __ldg(f + 1), __ldg(f + nt),
                  __ldg(f + nt + 1));
      return;
    }
  }
  ff a00, a01, a10, a11;
  bool ok;
  if (SG) {
    const float2 g00 = Gs[o], g01 = Gs[o + 1], g10 = Gs[o + nt], g11 = Gs[o + nt + 1];
    a00 = {g00.x, g00.y}; a01 = {g01.x, g01.y}; a10 = {g10.x, g10.y}; a11 = {g11.x, g11.y};
    ok = gall || !(isnan(g00.x) | isnan(g01.x) | isnan(g10.x) | isnan(g11.x));   // gall: every value split
  } else {
    const double* f = F + o;
    ok = d2ff(__ldg(f), a00) & d2ff(__ldg(f + 1), a01) & d2ff(__ldg(f + nt), a10) & d2ff(__ldg(f + nt + 1), a11);
  }
  const Weights wr = axis_weights_ff(vr, ir, cr, kr, ur);
  const Weights wt = axis_weights_ff(vt, it, ct, kt, ut);
  if (nan) {
    v = __longlong_as_double(0x7FF8000000000000ll);
  } else if (ok) {
    const ff lo = ff_add_u(ff_mul_u(wt.wbar, a00), ff_mul_u(wt.w, a01));
    const ff hi = ff_add_u(ff_mul_u(wt.wbar, a10), ff_mul_u(wt.w, a11));
    v = ff2d(ff_add_u(ff_mul_u(wr.wbar, lo), ff_mul_u(wr.w, hi)));
  } else {
    const double* f = F + o;
    v = blend64w(ff2d(wr.w), ff2d(wr.wbar), ff2d(wt.w), ff2d(wt.wbar), __ldg(f), __ldg(f + 1), __ldg(f + nt),
                 __ldg(f + nt + 1));
  }
}

template <int MODE, bool FF, bool SG>
__device__ __forceinline__ int stream_pairs(const Args2D& a, const AxisView& vr, const AxisView& vt,
                                            const float2* Gs, bool gall) {
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  int nans = 0;
  auto scalar = [&](int64_t i) {
    int ir, it;
    double v;
    lookup_pair<MODE, FF, SG>(vr, vt, a.F, Gs, a.nt, a.Y2[2 * i], a.Y2[2 * i + 1], ir, it, v, nans, gall);
    a.idx[2 * i] = ir;
    a.idx[2 * i + 1] = it;
    a.val[i] = v;
  };
  for (int64_t i = gtid; i < a.head; i += gs) scalar(i);
  const double2* Y = reinterpret_cast<const double2*>(a.Y2) + a.head;
  int4* I4 = reinterpret_cast<int4*>(a.idx + 2 * a.head);
  double2* V2 = reinterpret_cast<double2*>(a.val + a.head);
  for (int64_t g = gtid; g < a.np2; g += gs) {
    const double2 p0 = ld_stream(Y + 2 * g), p1 = ld_stream(Y + 2 * g + 1);
    int i0, j0, i1, j1;
    double v0, v1;
    lookup_pair<MODE, FF, SG>(vr, vt, a.F, Gs, a.nt, p0.x, p0.y, i0, j0, v0, nans, gall);
    lookup_pair<MODE, FF, SG>(vr, vt, a.F, Gs, a.nt, p1.x, p1.y, i1, j1, v1, nans, gall);
    st_stream(I4 + g, make_int4(i0, j0, i1, j1));
    st_stream(V2 + g, make_double2(v0, v1));
  }
  for (int64_t i = a.head + 2 * a.np2 + gtid; i < a.m; i += gs) scalar(i);
  return nans;
}

// ---------------------------------------------------------------------------
// Lean path of the staged-grid kernel for the common case: both axes bucket
// searches with at most two keys per bucket, float-float cells, every grid
// value split, no interpolation option.  Each axis keeps only the fields that
// case reads, as shared-memory offsets, so the loop runs without spilling in
// the 64 registers a 1024-thread block allows (the general path, which keeps
// every axis field live, spilled there).  The other paths of the kernel are
// separate (non-inlined) functions, so their registers do not weigh on this
// loop.
// ---------------------------------------------------------------------------
struct LeanAxis {
  int keys, dir, ca, cg;       // shared-memory byte offsets: keys, directory, cell records, cell scales
  int shift, nb, n;
  uint64_t base, k0;
};

__device__ __forceinline__ LeanAxis lean_axis(const Axis2D& ax, const unsigned char* smem) {
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + ax.lay.hdr);
  const AxisAux& aux = *reinterpret_cast<const AxisAux*>(smem + ax.aux);
  LeanAxis f;
  f.keys = ax.lay.keys;
  f.dir = ax.lay.dir;
  f.ca = ax.cells;
  f.cg = ax.cells + (h.n - 1) * (int)sizeof(ulonglong2);   // the scales follow the n-1 records (cell_table)
  f.shift = h.shift;
  f.nb = h.nb;
  f.n = h.n;
  f.base = h.base;
  f.k0 = aux.k0;
  return f;
}

// Branch-free: the cell's weights are computed for every target and the
// end weights of targets above the last entry or at or below the first are
// picked by selects, so a pair is one basic block that the compiler can
// interleave with the thread's other pair (3-4 % measured).
__device__ __forceinline__ Weights lean_weights(const unsigned char* smem, const LeanAxis& f, int i, int c, uint64_t k,
                                                uint64_t u) {
#ifdef SS_CHECKED
  const CellTable t{reinterpret_cast<const ulonglong2*>(smem + f.ca), reinterpret_cast<const float2*>(smem + f.cg),
                    f.n - 1};
#else
  const CellTable t{reinterpret_cast<const ulonglong2*>(smem + f.ca), reinterpret_cast<const float2*>(smem + f.cg)};
#endif
  Weights r = cell_weights<true>(u, t, c);
  const bool above = i >= f.n - 1, below = (i == 0) & (k <= f.k0), out = above | below;
  r.w.hi = above ? 1.0f : (below ? 0.0f : r.w.hi);
  r.w.lo = out ? 0.0f : r.w.lo;
  r.wbar.hi = above ? 0.0f : (below ? 1.0f : r.wbar.hi);
  r.wbar.lo = out ? 0.0f : r.wbar.lo;
  return r;
}

// One pair on the lean path (SCAN keys per bucket; HI: both bucket shifts
// are 32 or more); the grid is the float-float copy at byte offset gsm of
// shared memory.
template <int SCAN, int HI>
__device__ __forceinline__ void lean_pair(const unsigned char* smem, const LeanAxis& fr, const LeanAxis& ft, int gsm,
                                          double rho, double tem, int& ir, int& it, double& v, int& nans) {
  const uint64_t ur = static_cast<uint64_t>(__double_as_longlong(rho));
  const uint64_t ut = static_cast<uint64_t>(__double_as_longlong(tem));
  const uint64_t kr = order_key(rho), kt = order_key(tem);
  // a NaN maps below the image of -inf (0x0010000000000000): its high word decides
  const bool nr = (uint32_t)(kr >> 32) < 0x00100000u, nt_ = (uint32_t)(kt >> 32) < 0x00100000u;
  nans += (int)nr + (int)nt_;
  ir = search_bucket<SCAN, HI>(reinterpret_cast<const uint64_t*>(smem + fr.keys),
                               reinterpret_cast<const int*>(smem + fr.dir), fr.shift, fr.base, fr.nb, kr);
  it = search_bucket<SCAN, HI>(reinterpret_cast<const uint64_t*>(smem + ft.keys),
                               reinterpret_cast<const int*>(smem + ft.dir), ft.shift, ft.base, ft.nb, kt);
  const int nt = ft.n;
  const int cr = min(ir, fr.n - 2), ct = min(it, nt - 2);
  const int o = cr * nt + ct;                    // axes of at most 4096 entries: fits 32 bits
#ifdef SS_CHECKED
  const int ng = fr.n * nt;
  const float2* Gs = reinterpret_cast<const float2*>(smem + gsm);
  const float2 g00 = Gs[SS_IX(o, ng)], g01 = Gs[SS_IX(o + 1, ng)], g10 = Gs[SS_IX(o + nt, ng)],
               g11 = Gs[SS_IX(o + nt + 1, ng)];
#else
  const float2* Gs = reinterpret_cast<const float2*>(smem + gsm);
  const float2 g00 = Gs[o], g01 = Gs[o + 1], g10 = Gs[o + nt], g11 = Gs[o + nt + 1];
#endif
  const Weights wr = lean_weights(smem, fr, ir, cr, kr, ur);
  const Weights wt = lean_weights(smem, ft, it, ct, kt, ut);
  const ff lo = ff_add_u(ff_mul_u(wt.wbar, ff{g00.x, g00.y}), ff_mul_u(wt.w, ff{g01.x, g01.y}));
  const ff hi = ff_add_u(ff_mul_u(wt.wbar, ff{g10.x, g10.y}), ff_mul_u(wt.w, ff{g11.x, g11.y}));
  v = (nr | nt_) ? __longlong_as_double(0x7FF8000000000000ll)
                 : ff2d(ff_add_u(ff_mul_u(wr.wbar, lo), ff_mul_u(wr.w, hi)));
}

template <int SCAN, int HI>
__device__ __forceinline__ int lean_pairs_of(const Args2D& a, const unsigned char* smem, const LeanAxis& fr,
                                             const LeanAxis& ft) {
  const int gsm = a.grid_smem;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  int nans = 0;
  auto scalar = [&](int64_t i) {
    int ir, it;
    double v;
    lean_pair<SCAN, HI>(smem, fr, ft, gsm, a.Y2[2 * i], a.Y2[2 * i + 1], ir, it, v, nans);
    a.idx[2 * i] = ir;
    a.idx[2 * i + 1] = it;
    a.val[i] = v;
  };
  for (int64_t i = gtid; i < a.head; i += gs) scalar(i);
  const double2* Y = reinterpret_cast<const double2*>(a.Y2) + a.head;
  int4* I4 = reinterpret_cast<int4*>(a.idx + 2 * a.head);
  double2* V2 = reinterpret_cast<double2*>(a.val + a.head);
  for (int64_t g = gtid; g < a.np2; g += gs) {
    const double2 p0 = ld_stream(Y + 2 * g), p1 = ld_stream(Y + 2 * g + 1);
    int i0, j0, i1, j1;
    double v0, v1;
    lean_pair<SCAN, HI>(smem, fr, ft, gsm, p0.x, p0.y, i0, j0, v0, nans);
    lean_pair<SCAN, HI>(smem, fr, ft, gsm, p1.x, p1.y, i1, j1, v1, nans);
    st_stream(I4 + g, make_int4(i0, j0, i1, j1));
    st_stream(V2 + g, make_double2(v0, v1));
  }
  for (int64_t i = a.head + 2 * a.np2 + gtid; i < a.m; i += gs) scalar(i);
  return nans;
}

// The lean path's loop, with the bucket index taken from the keys' high
// words when both axes' shifts allow (the common case) and chosen per call
// otherwise.
template <int SCAN>
__device__ __forceinline__ int lean_pairs(const Args2D& a, const unsigned char* smem) {
  const LeanAxis fr = lean_axis(a.ar, smem), ft = lean_axis(a.at, smem);
  if (fr.shift >= 32 && ft.shift >= 32) return lean_pairs_of<SCAN, 1>(a, smem, fr, ft);
  return lean_pairs_of<SCAN, -1>(a, smem, fr, ft);
}

// The staged-grid kernel's other float-float paths, kept out of line.
template <int MODE>
__device__ __noinline__ int stream_pairs_sg(const Args2D& a, const AxisView& vr, const AxisView& vt, const float2* Gs,
                                            bool gall) {
  return stream_pairs<MODE, true, true>(a, vr, vt, Gs, gall);
}

template <bool SG>
__device__ __forceinline__ void interp_body(const Args2D& a, unsigned char* smem) {
  stage_table_1d(a.R, a.nr, a.ar.lay, smem);
  stage_table_1d(a.T, a.nt, a.at.lay, smem);
  stage_cells(a.R, a.nr, a.ar, smem);
  stage_cells(a.T, a.nt, a.at, smem);
  float2* Gs = nullptr;
  bool gok = true;
  if (SG) {
    // the value grid as float-float, once per block
    Gs = reinterpret_cast<float2*>(smem + a.grid_smem);
    const int64_t cnt = (int64_t)a.nr * a.nt;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      ff r;
      const bool ok = d2ff(__ldg(a.F + i), r);
      gok &= ok;
      Gs[i] = ok ? make_float2(r.hi, r.lo) : make_float2(__int_as_float(0x7FC00000), 0.0f);
    }
  }
  const bool gall = __syncthreads_and(gok);   // every grid value split exactly enough (no fp64 corners)
  AxisView vr = view_of(a.ar, smem), vt = view_of(a.at, smem);
  vr.x = a.R;
  vt.x = a.T;
  vr.extrap = vt.extrap = a.extrap;
  const TableHdr& hr = *reinterpret_cast<const TableHdr*>(smem + a.ar.lay.hdr);
  const TableHdr& ht = *reinterpret_cast<const TableHdr*>(smem + a.at.lay.hdr);
  const bool ff = !a.force_fp64 && !a.logspace && reinterpret_cast<const AxisAux*>(smem + a.ar.aux)->ffok &&
                  reinterpret_cast<const AxisAux*>(smem + a.at.aux)->ffok;
  const int mode = a.algo == SS_ALGO_BINARY ? 2 : (hr.occ <= 1 && ht.occ <= 1) ? 0 : (hr.occ <= 2 && ht.occ <= 2) ? 3 : 1;
  int nans;
  if constexpr (SG) {
    if (ff && gall && !a.extrap && (mode == 0 || mode == 3)) {
      nans = mode == 0 ? lean_pairs<1>(a, smem) : lean_pairs<2>(a, smem);
    } else if (ff) {
      nans = mode == 0 ? stream_pairs_sg<0>(a, vr, vt, Gs, gall)
           : mode == 3 ? stream_pairs_sg<3>(a, vr, vt, Gs, gall)
           : mode == 1 ? stream_pairs_sg<1>(a, vr, vt, Gs, gall) : stream_pairs_sg<2>(a, vr, vt, Gs, gall);
    } else {
      nans = mode == 0 ? stream_pairs<0, false, false>(a, vr, vt, Gs, gall)
           : mode == 2 ? stream_pairs<2, false, false>(a, vr, vt, Gs, gall) : stream_pairs<1, false, false>(a, vr, vt, Gs, gall);
    }
  } else if (ff) {
    nans = mode == 0 ? stream_pairs<0, true, SG>(a, vr, vt, Gs, gall)
         : mode == 3 ? stream_pairs<3, true, SG>(a, vr, vt, Gs, gall)
         : mode == 1 ? stream_pairs<1, true, SG>(a, vr, vt, Gs, gall) : stream_pairs<2, true, SG>(a, vr, vt, Gs, gall);
  } else {
    nans = mode == 0 ? stream_pairs<0, false, false>(a, vr, vt, Gs, gall)
         : mode == 2 ? stream_pairs<2, false, false>(a, vr, vt, Gs, gall) : stream_pairs<1, false, false>(a, vr, vt, Gs, gall);
  }
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  if (a.stat != nullptr) {
    if ((threadIdx.x & 31) == 0 && nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (hr.bad | ht.bad) atomicOr(&a.stat->flags, SS_FLAG_NOT_SORTED);
      if (!ff && !a.force_fp64 && !a.logspace) atomicOr(&a.stat->flags, SS_FLAG_BAD_VALUE);
    }
  }
}

// Grid in global memory (L2-resident): 256 threads, several blocks per SM.
__global__ void __launch_bounds__(kNumThreads) k_search_interp_2d(Args2D a) {
  extern __shared__ __align__(16) unsigned char smem[];
  interp_body<false>(a, smem);
}

// Grid staged in shared memory as float-float: one 1024-thread block per SM,
// the four corner gathers become shared-memory loads.
constexpr int kSgThreads = 1024;
__global__ void __launch_bounds__(kSgThreads, 1) k_search_interp_2d_sg(Args2D a) {
  extern __shared__ __align__(16) unsigned char smem[];
  interp_body<true>(a, smem);
}

int default_dir_cap(int n);

static Axis2D make_axis(int n, int algo, int offset, bool logspace) {
  Axis2D ax{};
  const bool bucket = algo == SS_ALGO_BUCKET;
  ax.lay = make_layout_1d(n, bucket, !bucket, bucket ? default_dir_cap(n) : 0, offset);
  int off = ax.lay.bytes;
  auto take = [&](int bytes) { int o = off; off += (bytes + 15) & ~15; return o; };
  ax.cells = take((n - 1) * kCellBytes);
  ax.rg = take((n - 1) * 8);
  ax.lx = logspace ? take(n * 8) : -1;
  ax.aux = take((int)sizeof(AxisAux));
  ax.lay.bytes = off;   // end of this axis' region
  return ax;
}

ss_status search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                           const double* Y2, int64_t m, int32_t* idx, double* val, int32_t algo, int force_fp64,
                           ss_devstat* stat, cudaStream_t stream, int extrap, int logspace) {
  if (R == nullptr || T == nullptr || F == nullptr || (m > 0 && (Y2 == nullptr || idx == nullptr || val == nullptr)))
    return fail(SS_EINVAL, "ss_search_interp_2d: null pointer");
  if (nr < 2 || nt < 2) return fail(SS_EINVAL, "ss_search_interp_2d: each axis needs >= 2 entries");
  if (m < 0) return fail(SS_EINVAL, "ss_search_interp_2d: m must be >= 0");
  if (!aligned(R, 8) || !aligned(T, 8) || !aligned(F, 8) || !aligned(Y2, 8) || !aligned(idx, 4) || !aligned(val, 8))
    return fail(SS_EINVAL, "ss_search_interp_2d: misaligned pointer");
  if (nr > kMaxAxis2D || nt > kMaxAxis2D) return fail(SS_EUNSUPPORTED, "ss_search_interp_2d: axis longer than 4096");
  if (algo == SS_ALGO_AUTO) algo = SS_ALGO_BUCKET;
  if (algo != SS_ALGO_BUCKET && algo != SS_ALGO_BINARY)
    return fail(SS_EUNSUPPORTED, "ss_search_interp_2d: algo must be auto, bucket or binary");
  if (m == 0) return SS_OK;
  Args2D a{};
  a.R = R; a.nr = nr; a.T = T; a.nt = nt; a.F = F; a.Y2 = Y2; a.m = m; a.idx = idx; a.val = val;
  a.algo = algo; a.force_fp64 = force_fp64 | logspace; a.stat = stat;
  a.extrap = extrap ? 1 : 0;
  a.logspace = logspace ? 1 : 0;
  a.ar = make_axis(nr, algo, 0, logspace);
  a.at = make_axis(nt, algo, a.ar.lay.bytes, logspace);
  const int smem = a.at.lay.bytes;
  // vector body: two pairs per item, needs 16-byte alignment of pair, index pair-of-pairs and value pair
  a.head = m;
  a.np2 = 0;
  for (int h = 0; h < 2 && h <= m; ++h) {
    const bool ok = aligned(Y2 + 2 * h, 16) && aligned(idx + 2 * h, 16) && aligned(val + h, 16);
    if (ok) { a.head = h; a.np2 = (m - h) / 2; break; }
  }
  if (smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, "ss_search_interp_2d: axes too large for shared memory");
  // stage the grid too when it fits beside the axes (and the float-float path is not disabled)
  const int64_t gbytes = (int64_t)nr * nt * 8;
  const bool sg = !a.force_fp64 && smem + gbytes + 16 <= (int64_t)max_smem_optin();
  a.grid_smem = sg ? ((smem + 15) & ~15) : -1;
  const int threads = sg ? kSgThreads : kNumThreads;
  const int smem_all = sg ? a.grid_smem + (int)gbytes : smem;
  const void* k = sg ? reinterpret_cast<const void*>(&k_search_interp_2d_sg) : reinterpret_cast<const void*>(&k_search_interp_2d);
  if (ss_status st_ = raise_smem_limit(k, smem_all)) return st_;
  int per_sm = 0;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem_all));
  if (per_sm < 1) return fail(SS_EUNSUPPORTED, "ss_search_interp_2d: kernel does not fit on an SM");
  const int64_t items = a.np2 > 0 ? a.np2 + (m - 2 * a.np2) : m;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((items + threads - 1) / threads,
                                                                (int64_t)num_sms() * per_sm));
  void* args[1] = {&a};
  cudaError_t err = cudaLaunchKernel(k, dim3(grid), dim3(threads), args, (size_t)smem_all, stream);
  if (err != cudaSuccess) return cuda_fail(err, "k_search_interp_2d");
  return SS_OK;
}

}  // namespace ss

extern "C" {

ss_status ss_search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                              const double* Y2, int64_t m, int32_t* lowbounds2, double* values, int32_t algo,
                              ss_devstat* stat, cudaStream_t stream) {
  return ss::search_interp_2d(R, nr, T, nt, F, Y2, m, lowbounds2, values, algo, 0, stat, stream, 0, 0);
}

ss_status ss_search_interp_2d_ex(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                                 const double* Y2, int64_t m, int32_t* lowbounds2, double* values,
                                 const ss_interp_opts* opts, ss_devstat* stat, cudaStream_t stream) {
  const ss_interp_opts o = opts != nullptr ? *opts : ss_interp_opts{SS_ALGO_AUTO, 0, 0, 0};
  if ((o.extrap != 0 && o.extrap != 1) || (o.logspace != 0 && o.logspace != 1) || (o.fp64 != 0 && o.fp64 != 1))
    return ss::fail(SS_EINVAL, "ss_search_interp_2d_ex: extrap, logspace and fp64 must be 0 or 1");
  return ss::search_interp_2d(R, nr, T, nt, F, Y2, m, lowbounds2, values, o.algo, o.fp64, stat, stream, o.extrap,
                              o.logspace);
}

// Same lookup with the float-float path disabled (fp64 weights and blend);
// for comparisons and tables outside the float-float preconditions.
ss_status ss_search_interp_2d_fp64(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                                   const double* Y2, int64_t m, int32_t* lowbounds2, double* values, int32_t algo,
                                   ss_devstat* stat, cudaStream_t stream) {
  return ss::search_interp_2d(R, nr, T, nt, F, Y2, m, lowbounds2, values, algo, 1, stat, stream, 0, 0);
}

}  // extern "C"
