// interp_2d.cu -- one-shot fused 2D lookup (Sec. 1 and 2.2: EOSPAC bounds
// each (density, temperature) target in both grids of a SESAME table and
// interpolates).  Per pair: two exact searches (the 1D routines of
// ss_table.cuh on two staged axes), cell selection c = min(i, n-2), clamped
// weights from per-cell reciprocal gaps staged once per block, four gathers
// from the row-major value grid and the convex bilinear blend.
//
// The value grid stays in global memory (L2-resident for the sizes of interest);
// axes, bucket directories and per-cell origins / reciprocal gaps live in
// shared memory.
#include <algorithm>

#include "ss_table.cuh"

namespace ss {

constexpr int kMaxAxis2D = 4096;   // largest axis staged whole with its per-cell data

struct Axis2D {                    // shared-memory offsets of one axis
  Layout1D lay;
  int cx;                          // double[n-1]: left end X[c] of cell c
  int cg;                          // double[n-1]: 1 / (X[c+1] - X[c])
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
  Axis2D ar, at;
  ss_devstat* stat;
};

static __device__ void stage_cells(const double* __restrict__ X, int n, const Axis2D& ax, unsigned char* smem) {
  double* cx = reinterpret_cast<double*>(smem + ax.cx);
  double* cg = reinterpret_cast<double*>(smem + ax.cg);
  for (int c = threadIdx.x; c < n - 1; c += blockDim.x) {
    const double a = __ldg(X + c), b = __ldg(X + c + 1);
    cx[c] = a;
    cg[c] = 1.0 / (b - a);
  }
}

// Clamp to [0, 1]; NaN passes through.
__device__ __forceinline__ double clamp01(double w) { return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w); }

struct AxisView {
  const uint64_t* keys;
  const uint64_t* eyt;
  const int* dir;
  const double* cx;
  const double* cg;
  int shift, nb, T, D, n;
  uint64_t base;
};

__device__ __forceinline__ AxisView view_of(const Axis2D& ax, const unsigned char* smem) {
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + ax.lay.hdr);
  AxisView v;
  v.keys = ax.lay.keys >= 0 ? reinterpret_cast<const uint64_t*>(smem + ax.lay.keys) : nullptr;
  v.eyt = ax.lay.eyt >= 0 ? reinterpret_cast<const uint64_t*>(smem + ax.lay.eyt) : nullptr;
  v.dir = ax.lay.dir >= 0 ? reinterpret_cast<const int*>(smem + ax.lay.dir) : nullptr;
  v.cx = reinterpret_cast<const double*>(smem + ax.cx);
  v.cg = reinterpret_cast<const double*>(smem + ax.cg);
  v.shift = h.shift;
  v.nb = h.nb;
  v.T = h.occ > 0 ? 32 - __clz(h.occ) : 0;
  v.D = h.D;
  v.n = h.n;
  v.base = h.base;
  return v;
}

// One pair: indices and value.  MODE 0: both axes bucket with occupancy <= 1;
// 1: bucket with bounded bisection; 2: breadth-first binary.
template <int MODE>
__device__ __forceinline__ void lookup_pair(const AxisView& vr, const AxisView& vt, const double* __restrict__ F,
                                            int nt, double rho, double tem, int& ir, int& it, double& v, int& nans) {
  const uint64_t kr = order_key(rho), kt = order_key(tem);
  nans += (kr < 0x0010000000000000ull) + (kt < 0x0010000000000000ull);
  if (MODE == 0) {
    ir = search_bucket<1>(vr.keys, vr.dir, vr.shift, vr.base, vr.nb, kr);
    it = search_bucket<1>(vt.keys, vt.dir, vt.shift, vt.base, vt.nb, kt);
  } else if (MODE == 1) {
    ir = search_bucket_bisect(vr.keys, vr.dir, vr.shift, vr.base, vr.nb, vr.T, kr);
    it = search_bucket_bisect(vt.keys, vt.dir, vt.shift, vt.base, vt.nb, vt.T, kt);
  } else {
    ir = search_eyt_rt(vr.eyt, vr.D, kr);
    it = search_eyt_rt(vt.eyt, vt.D, kt);
  }
  const int cr = min(ir, vr.n - 2), ct = min(it, nt - 2);
  const double wr = clamp01((rho - vr.cx[cr]) * vr.cg[cr]);
  const double wt = clamp01((tem - vt.cx[ct]) * vt.cg[ct]);
  const double* f = F + (int64_t)cr * nt + ct;
  const double f00 = __ldg(f), f01 = __ldg(f + 1), f10 = __ldg(f + nt), f11 = __ldg(f + nt + 1);
  const double lo = (1.0 - wt) * f00 + wt * f01;
  const double hi = (1.0 - wt) * f10 + wt * f11;
  v = (1.0 - wr) * lo + wr * hi;
}

template <int MODE>
__device__ __forceinline__ int stream_pairs(const Args2D& a, const AxisView& vr, const AxisView& vt) {
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  int nans = 0;
  auto scalar = [&](int64_t i) {
    int ir, it;
    double v;
    lookup_pair<MODE>(vr, vt, a.F, a.nt, a.Y2[2 * i], a.Y2[2 * i + 1], ir, it, v, nans);
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
    lookup_pair<MODE>(vr, vt, a.F, a.nt, p0.x, p0.y, i0, j0, v0, nans);
    lookup_pair<MODE>(vr, vt, a.F, a.nt, p1.x, p1.y, i1, j1, v1, nans);
    st_stream(I4 + g, make_int4(i0, j0, i1, j1));
    st_stream(V2 + g, make_double2(v0, v1));
  }
  for (int64_t i = a.head + 2 * a.np2 + gtid; i < a.m; i += gs) scalar(i);
  return nans;
}

__global__ void __launch_bounds__(kNumThreads) k_search_interp_2d(Args2D a) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table_1d(a.R, a.nr, a.ar.lay, smem);
  stage_table_1d(a.T, a.nt, a.at.lay, smem);
  stage_cells(a.R, a.nr, a.ar, smem);
  stage_cells(a.T, a.nt, a.at, smem);
  __syncthreads();
  const AxisView vr = view_of(a.ar, smem), vt = view_of(a.at, smem);
  const TableHdr& hr = *reinterpret_cast<const TableHdr*>(smem + a.ar.lay.hdr);
  const TableHdr& ht = *reinterpret_cast<const TableHdr*>(smem + a.at.lay.hdr);
  int nans;
  if (a.algo == SS_ALGO_BINARY) nans = stream_pairs<2>(a, vr, vt);
  else if (hr.occ <= 1 && ht.occ <= 1) nans = stream_pairs<0>(a, vr, vt);
  else nans = stream_pairs<1>(a, vr, vt);
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  if (a.stat != nullptr) {
    if ((threadIdx.x & 31) == 0 && nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (hr.bad | ht.bad)) atomicOr(&a.stat->flags, SS_FLAG_NOT_SORTED);
  }
}

int default_dir_cap(int n);

static Axis2D make_axis(int n, int algo, int offset) {
  Axis2D ax{};
  const bool bucket = algo == SS_ALGO_BUCKET;
  ax.lay = make_layout_1d(n, bucket, !bucket, bucket ? default_dir_cap(n) : 0, offset);
  int off = ax.lay.bytes;
  ax.cx = off;
  off += ((n - 1) * 8 + 15) & ~15;
  ax.cg = off;
  off += ((n - 1) * 8 + 15) & ~15;
  ax.lay.bytes = off;   // end of this axis' region
  return ax;
}

ss_status search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                           const double* Y2, int64_t m, int32_t* idx, double* val, int32_t algo, ss_devstat* stat,
                           cudaStream_t stream) {
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
  a.algo = algo; a.stat = stat;
  a.ar = make_axis(nr, algo, 0);
  a.at = make_axis(nt, algo, a.ar.lay.bytes);
  const int smem = a.at.lay.bytes;
  // vector body: two pairs per item, needs 16-byte alignment of pair, index pair-of-pairs and value pair
  a.head = m;
  a.np2 = 0;
  for (int h = 0; h < 2 && h <= m; ++h) {
    const bool ok = aligned(Y2 + 2 * h, 16) && aligned(idx + 2 * h, 16) && aligned(val + h, 16);
    if (ok) { a.head = h; a.np2 = (m - h) / 2; break; }
  }
  if (smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, "ss_search_interp_2d: axes too large for shared memory");
  const void* k = reinterpret_cast<const void*>(&k_search_interp_2d);
  SS_CHECK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kNumThreads, smem));
  if (per_sm < 1) return fail(SS_EUNSUPPORTED, "ss_search_interp_2d: kernel does not fit on an SM");
  const int64_t items = a.np2 > 0 ? a.np2 + (m - 2 * a.np2) : m;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((items + kNumThreads - 1) / kNumThreads,
                                                                (int64_t)num_sms() * per_sm));
  void* args[1] = {&a};
  cudaError_t err = cudaLaunchKernel(k, dim3(grid), dim3(kNumThreads), args, (size_t)smem, stream);
  if (err != cudaSuccess) return cuda_fail(err, "k_search_interp_2d");
  return SS_OK;
}

}  // namespace ss

extern "C" ss_status ss_search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                                         const double* Y2, int64_t m, int32_t* lowbounds2, double* values,
                                         int32_t algo, ss_devstat* stat, cudaStream_t stream) {
  return ss::search_interp_2d(R, nr, T, nt, F, Y2, m, lowbounds2, values, algo, stat, stream);
}
