// search_1d.cu -- one-shot 1D search (Sec. 3): every thread block stages the
// table in shared memory once, then streams targets through 128-bit loads and
// stores in a grid-stride loop.  Variants (identical results):
//   binary  : branchless search over the breadth-first key layout (Sec. 3.2)
//   bucket  : bucket directory on the key's top bits + bounded scan (Sec. 3.5)
//   ballot  : warp-cooperative (G+1)-ary search with __ballot_sync/__popc
//   branchy : textbook bisection with data-dependent branches (Sec. 5.4)
// Tables with more than kMaxSmemKeys searched entries use a sampled top
// level in shared memory and finish the search in global memory (Sec. 3.3).
#include <algorithm>

#include "ss_table.cuh"

namespace ss {

struct Args1D {
  const double* X;
  int n;
  const double* Y;
  int64_t m;
  int32_t* out;
  int64_t head;       // targets [0, head) take the scalar path (alignment prologue)
  int64_t nq;         // quads in the vector body that follows
  int w256;           // 1: Y + head is 32-byte aligned, quads load as one 256-bit access
  uint64_t le;        // 1 for side "<=", else 0 (added to the query key)
  Layout1D lay;
  ss_devstat* stat;
};

constexpr uint64_t kKeyNegInf = 0x0010000000000000ull;   // image of -inf; NaNs map below it

__device__ __forceinline__ int nan_flag(uint64_t key) { return key < kKeyNegInf ? 1 : 0; }

// Grid-stride streaming of targets through `idx_of(key)`; two quads in flight
// per thread in the 128-bit body.
template <class F>
__device__ __forceinline__ int stream_targets(const Args1D& a, F&& idx_of) {
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  int nans = 0;
  for (int64_t i = gtid; i < a.head; i += gs) {
    const uint64_t k = order_key(a.Y[i]);
    nans += nan_flag(k);
    a.out[i] = idx_of(k + a.le);
  }
  const double2* Y2 = reinterpret_cast<const double2*>(a.Y + a.head);
  int4* O4 = reinterpret_cast<int4*>(a.out + a.head);
  int64_t g = gtid;
  for (; g + gs < a.nq; g += 2 * gs) {
    double y[8];
    if (a.w256) {
      ld_stream4(reinterpret_cast<const double*>(Y2 + 2 * g), *reinterpret_cast<double(*)[4]>(y));
      ld_stream4(reinterpret_cast<const double*>(Y2 + 2 * (g + gs)), *reinterpret_cast<double(*)[4]>(y + 4));
    } else {
      const double2 p0 = ld_stream(Y2 + 2 * g), p1 = ld_stream(Y2 + 2 * g + 1);
      const double2 p2 = ld_stream(Y2 + 2 * (g + gs)), p3 = ld_stream(Y2 + 2 * (g + gs) + 1);
      y[0] = p0.x; y[1] = p0.y; y[2] = p1.x; y[3] = p1.y;
      y[4] = p2.x; y[5] = p2.y; y[6] = p3.x; y[7] = p3.y;
    }
    uint64_t k[8] = {order_key(y[0]), order_key(y[1]), order_key(y[2]), order_key(y[3]),
                     order_key(y[4]), order_key(y[5]), order_key(y[6]), order_key(y[7])};
    int r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      nans += nan_flag(k[j]);
      r[j] = idx_of(k[j] + a.le);
    }
    st_stream(O4 + g, make_int4(r[0], r[1], r[2], r[3]));
    st_stream(O4 + g + gs, make_int4(r[4], r[5], r[6], r[7]));
  }
  if (g < a.nq) {
    const double2 p0 = ld_stream(Y2 + 2 * g), p1 = ld_stream(Y2 + 2 * g + 1);
    uint64_t k[4] = {order_key(p0.x), order_key(p0.y), order_key(p1.x), order_key(p1.y)};
    int r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      nans += nan_flag(k[j]);
      r[j] = idx_of(k[j] + a.le);
    }
    st_stream(O4 + g, make_int4(r[0], r[1], r[2], r[3]));
  }
  for (int64_t i = a.head + 4 * a.nq + gtid; i < a.m; i += gs) {
    const uint64_t k = order_key(a.Y[i]);
    nans += nan_flag(k);
    a.out[i] = idx_of(k + a.le);
  }
  return nans;
}

__device__ __forceinline__ void finish_block(const Args1D& a, const TableHdr& h, int nans) {
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  if (a.stat != nullptr) {
    if ((threadIdx.x & 31) == 0 && nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
    if (blockIdx.x == 0 && threadIdx.x == 0 && h.bad) atomicOr(&a.stat->flags, SS_FLAG_NOT_SORTED);
  }
}

// Final index from the count of staged keys below q (two-level tables finish in global memory).
__device__ __forceinline__ int finish_count(const Args1D& a, const TableHdr& h, int c, uint64_t q) {
  return h.stride == 1 ? c : search_leaf_global(a.X, h.nk, h.stride, c, q);
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

template <int D, bool TWO_LEVEL>
__global__ void __launch_bounds__(kNumThreads) k_search_1d_binary(Args1D a) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table_1d(a.X, a.n, a.lay, smem);
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + a.lay.hdr);
  const uint64_t* eyt = reinterpret_cast<const uint64_t*>(smem + a.lay.eyt);
  const int nans = stream_targets(a, [&](uint64_t q) {
    const int c = search_eyt<D>(eyt, q);
    return TWO_LEVEL ? finish_count(a, h, c, q) : c;
  });
  finish_block(a, h, nans);
}

__global__ void __launch_bounds__(kNumThreads) k_search_1d_bucket(Args1D a) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table_1d(a.X, a.n, a.lay, smem);
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + a.lay.hdr);
  const uint64_t* keys = reinterpret_cast<const uint64_t*>(smem + a.lay.keys);
  const int* dir = reinterpret_cast<const int*>(smem + a.lay.dir);
  const int shift = h.shift, nb = h.nb, occ = h.occ;
  const uint64_t base = h.base;
  int nans;
  // occupancy is the same for every block: a uniform branch picks the loop
  // (tables staged whole, the common case, also skip the two-level finish)
  if (occ <= 1 && h.stride == 1) {
    nans = stream_targets(a, [&](uint64_t q) { return search_bucket<1>(keys, dir, shift, base, nb, q); });
  } else if (occ <= 1) {
    nans = stream_targets(a, [&](uint64_t q) { return finish_count(a, h, search_bucket<1>(keys, dir, shift, base, nb, q), q); });
  } else if (occ == 2) {
    nans = stream_targets(a, [&](uint64_t q) { return finish_count(a, h, search_bucket<2>(keys, dir, shift, base, nb, q), q); });
  } else if (occ <= 4) {
    nans = stream_targets(a, [&](uint64_t q) { return finish_count(a, h, search_bucket<4>(keys, dir, shift, base, nb, q), q); });
  } else {
    const int T = 32 - __clz(occ);
    nans = stream_targets(a, [&](uint64_t q) {
      return finish_count(a, h, search_bucket_bisect(keys, dir, shift, base, nb, T, q), q);
    });
  }
  finish_block(a, h, nans);
}

__global__ void __launch_bounds__(kNumThreads) k_search_1d_branchy(Args1D a) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table_1d(a.X, a.n, a.lay, smem);
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + a.lay.hdr);
  const uint64_t* keys = reinterpret_cast<const uint64_t*>(smem + a.lay.keys);
  const int ns = h.ns;
  const int nans = stream_targets(a, [&](uint64_t q) { return finish_count(a, h, search_branchy(keys, ns, q), q); });
  finish_block(a, h, nans);
}

// Warp-cooperative variant: loops are warp-uniform so every __ballot_sync
// sees all 32 lanes.  Each lane loads a quad of targets; the G-lane groups
// then resolve the 4*G targets of their lanes one after another.
template <int G>
__global__ void __launch_bounds__(kNumThreads) k_search_1d_ballot(Args1D a, int S0) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table_1d(a.X, a.n, a.lay, smem);
  const TableHdr& h = *reinterpret_cast<const TableHdr*>(smem + a.lay.hdr);
  const uint64_t* keys = reinterpret_cast<const uint64_t*>(smem + a.lay.keys);
  const int ns = h.ns;
  const int lane = threadIdx.x & 31;
  const int gbase = lane & ~(G - 1);
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int nans = 0;
  auto resolve = [&](uint64_t (&q)[4], int (&r)[4], int slots) {
    for (int src = 0; src < G; ++src) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (s >= slots) break;
        const uint64_t qq = __shfl_sync(0xFFFFFFFFu, q[s], gbase + src);
        const int c = finish_count(a, h, search_ballot<G>(keys, ns, S0, qq), qq);
        if ((lane & (G - 1)) == src) r[s] = c;
      }
    }
  };
  // scalar ranges: [0, head) and [head + 4 nq, m), one target per lane
  auto scalar_range = [&](int64_t begin, int64_t end) {
    for (int64_t w = begin + wid * 32; w < end; w += nw * 32) {
      const int64_t i = w + lane;
      const bool ok = i < end;
      uint64_t q[4] = {0, 0, 0, 0};
      int r[4] = {0, 0, 0, 0};
      if (ok) {
        const uint64_t k = order_key(a.Y[i]);
        nans += nan_flag(k);
        q[0] = k + a.le;
      }
      resolve(q, r, 1);
      if (ok) a.out[i] = r[0];
    }
  };
  scalar_range(0, a.head);
  const double2* Y2 = reinterpret_cast<const double2*>(a.Y + a.head);
  int4* O4 = reinterpret_cast<int4*>(a.out + a.head);
  for (int64_t w = wid * 32; w < a.nq; w += nw * 32) {
    const int64_t g = w + lane;
    const bool ok = g < a.nq;
    uint64_t q[4] = {0, 0, 0, 0};
    int r[4] = {0, 0, 0, 0};
    if (ok) {
      const double2 p0 = ld_stream(Y2 + 2 * g), p1 = ld_stream(Y2 + 2 * g + 1);
      const double t[4] = {p0.x, p0.y, p1.x, p1.y};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint64_t k = order_key(t[s]);
        nans += nan_flag(k);
        q[s] = k + a.le;
      }
    }
    resolve(q, r, 4);
    if (ok) st_stream(O4 + g, make_int4(r[0], r[1], r[2], r[3]));
  }
  scalar_range(a.head + 4 * a.nq, a.m);
  finish_block(a, h, nans);
}

// ---------------------------------------------------------------------------
// Host launch
// ---------------------------------------------------------------------------

// Split [0, m) into a scalar prologue, a vector body of quads and a tail.
// The body needs Y+head 16-byte aligned (32-byte for 256-bit loads) and
// out+head 16-byte aligned.
static void split_vector(const void* Y, const void* out, int64_t m, int64_t& head, int64_t& nq, int& w256) {
  head = m;
  nq = 0;
  w256 = 0;
  for (int h = 0; h < 4 && h <= m; ++h) {
    const uintptr_t y = reinterpret_cast<uintptr_t>(Y) + 8u * h;
    const uintptr_t o = reinterpret_cast<uintptr_t>(out) + 4u * h;
    if ((y & 31) == 0 && (o & 15) == 0) {
      head = h;
      nq = (m - h) / 4;
      w256 = 1;
      return;
    }
  }
  for (int h = 0; h < 4 && h <= m; ++h) {
    const uintptr_t y = reinterpret_cast<uintptr_t>(Y) + 8u * h;
    const uintptr_t o = reinterpret_cast<uintptr_t>(out) + 4u * h;
    if ((y & 15) == 0 && (o & 15) == 0) {
      head = h;
      nq = (m - h) / 4;
      return;
    }
  }
}

// Launch `kernel` (a __global__ function taking Args1D and, for the ballot
// variant, an int) with a grid of at most (#SMs x resident blocks per SM).
static ss_status launch(const void* kernel, const Layout1D& lay, int64_t work_items, cudaStream_t stream,
                        const char* name, Args1D a, const int* extra = nullptr) {
  const int smem = lay.bytes;
  if (smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, std::string(name) + ": table too large for shared memory");
  if (ss_status st_ = raise_smem_limit(kernel, smem)) return st_;
  int per_sm = 0;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kNumThreads, smem));
  if (per_sm < 1) return fail(SS_EUNSUPPORTED, std::string(name) + ": kernel does not fit on an SM");
  const int64_t want = (work_items + kNumThreads - 1) / kNumThreads;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
  int ex = extra ? *extra : 0;
  void* args[2] = {&a, &ex};
  cudaError_t err = cudaLaunchKernel(kernel, dim3(grid), dim3(kNumThreads), args, (size_t)smem, stream);
  if (err != cudaSuccess) return cuda_fail(err, name);
  return SS_OK;
}

template <bool TWO>
static const void* binary_kernel(int D) {
  switch (D) {
#define SS_CASE(d) case d: return reinterpret_cast<const void*>(&k_search_1d_binary<d, TWO>);
    SS_CASE(1) SS_CASE(2) SS_CASE(3) SS_CASE(4) SS_CASE(5) SS_CASE(6) SS_CASE(7)
    SS_CASE(8) SS_CASE(9) SS_CASE(10) SS_CASE(11) SS_CASE(12) SS_CASE(13) SS_CASE(14)
#undef SS_CASE
    default: return nullptr;
  }
}

// Bucket budget: about four buckets per entry keeps the occupancy of a
// log-spaced table at one or two; sampled (two-level) tables take the largest
// directory so that it also serves as a fine spline.
int default_dir_cap(int n) { return n - 1 > kMaxSmemKeys ? 8192 : std::min(4096, std::max(64, 4 * n)); }

ss_status search_1d(const double* X, int32_t n, const double* Y, int64_t m, int32_t* out, int32_t side,
                    int32_t algo, ss_devstat* stat, cudaStream_t stream, int dir_cap_override, int ballot_g) {
  if (X == nullptr || (m > 0 && (Y == nullptr || out == nullptr)))
    return fail(SS_EINVAL, "ss_search_1d: null pointer");
  if (n < 2) return fail(SS_EINVAL, "ss_search_1d: n must be >= 2");
  if (m < 0) return fail(SS_EINVAL, "ss_search_1d: m must be >= 0");
  if (side != SS_SIDE_LT && side != SS_SIDE_LE) return fail(SS_EINVAL, "ss_search_1d: bad side");
  if (!aligned(X, 8) || !aligned(Y, 8) || !aligned(out, 4)) return fail(SS_EINVAL, "ss_search_1d: misaligned pointer");
  if (algo < SS_ALGO_AUTO || algo > SS_ALGO_BRANCHY) return fail(SS_EINVAL, "ss_search_1d: bad algo");
  if (m == 0) return SS_OK;
  Args1D a{};
  a.X = X; a.n = n; a.Y = Y; a.m = m; a.out = out; a.le = side == SS_SIDE_LE ? 1 : 0; a.stat = stat;
  split_vector(Y, out, m, a.head, a.nq, a.w256);
  const int64_t items = a.nq > 0 ? a.head + a.nq + (m - a.head - 4 * a.nq) : m;
  const bool fits = (n - 1) <= kMaxSmemKeys;
  if (algo == SS_ALGO_AUTO) algo = fits ? SS_ALGO_BUCKET : SS_ALGO_BINARY;
  switch (algo) {
    case SS_ALGO_BINARY: {
      a.lay = make_layout_1d(n, false, true, 0);
      const void* k = a.lay.stride > 1 ? binary_kernel<true>(a.lay.D) : binary_kernel<false>(a.lay.D);
      if (k == nullptr) return fail(SS_EUNSUPPORTED, "ss_search_1d: table depth out of range");
      return launch(k, a.lay, items, stream, "k_search_1d_binary", a);
    }
    case SS_ALGO_BUCKET: {
      a.lay = make_layout_1d(n, true, false, dir_cap_override > 0 ? dir_cap_override : default_dir_cap(n));
      return launch(reinterpret_cast<const void*>(&k_search_1d_bucket), a.lay, items, stream, "k_search_1d_bucket", a);
    }
    case SS_ALGO_BRANCHY: {
      a.lay = make_layout_1d(n, true, false, 0);
      return launch(reinterpret_cast<const void*>(&k_search_1d_branchy), a.lay, items, stream, "k_search_1d_branchy", a);
    }
    case SS_ALGO_BALLOT: {
      a.lay = make_layout_1d(n, true, false, 0);
      const int G = ballot_g > 0 ? ballot_g : 32;
      int S0 = 1;
      while ((int64_t)S0 * (G + 1) < (int64_t)a.lay.ns + 1) S0 *= (G + 1);
      if (G != 8 && G != 16 && G != 32) return fail(SS_EINVAL, "ballot group must be 8, 16 or 32");
      const void* k = G == 8 ? reinterpret_cast<const void*>(&k_search_1d_ballot<8>)
                    : G == 16 ? reinterpret_cast<const void*>(&k_search_1d_ballot<16>)
                              : reinterpret_cast<const void*>(&k_search_1d_ballot<32>);
      return launch(k, a.lay, items, stream, "k_search_1d_ballot", a, &S0);
    }
    default:
      return fail(SS_EINVAL, "ss_search_1d: bad algo");
  }
}

}  // namespace ss

extern "C" {

ss_status ss_search_1d(const double* X, int32_t n, const double* Y, int64_t m, int32_t* lowbounds, int32_t side,
                       int32_t algo, ss_devstat* stat, cudaStream_t stream) {
  return ss::search_1d(X, n, Y, m, lowbounds, side, algo, stat, stream, 0, 0);
}

// Tuning entry point (bucket budget, ballot group width); not part of the
// stable interface but exported for the autotuner and the benchmarks.
ss_status ss_search_1d_tuned(const double* X, int32_t n, const double* Y, int64_t m, int32_t* lowbounds,
                             int32_t side, int32_t algo, int32_t dir_cap, int32_t ballot_g, ss_devstat* stat,
                             cudaStream_t stream) {
  if (dir_cap < 0 || dir_cap > SS_MAX_DIR_CAP) return ss::fail(SS_EINVAL, "ss_search_1d_tuned: dir_cap out of range");
  return ss::search_1d(X, n, Y, m, lowbounds, side, algo, stat, stream, dir_cap, ballot_g);
}

}  // extern "C"
