// ss_table.cuh -- staging of one sorted table into shared memory and the
// in-block search routines that run on the staged copy.
//
// The searched set is the n-1 entries X[1..n-1]: counting how many of them lie
// below the target gives max(0, #{X[j] < t} - 1) directly, i.e. the index of
// Sec. 3 with both end clamps, and needs only ceil(log2 n) comparisons.
// Side "<=" is served by the same count with query key(t)+1.
//
// Layouts staged per thread block (all in dynamic shared memory):
//   keys[nk + kPad]  sorted images of X[1..n-1], then kPad copies of kKeyMax
//   eyt[P]           the same keys in breadth-first (Eytzinger) order, P a
//                    power of two >= n, slot 0 unused, missing nodes kKeyMax
//   dir[nb + 1]      bucket directory: dir[b] = #{keys whose bucket < base+b},
//                    bucket(key) = key >> shift  (Sec. 3.5 with shift 52 is
//                    the IEEE exponent hash; finer shifts add mantissa bits)
//
// For tables too large for shared memory the staged keys are a sample of
// every `stride`-th entry (a skip list in the sense of Sec. 3.3) and the last
// log2(stride) bisection steps read X from global memory.
#pragma once

#include "ss_common.cuh"

namespace ss {

constexpr int kPad = 64;               // sentinel keys after the sorted array
constexpr int kMaxSmemKeys = 8192 - kPad;   // largest nk staged whole

struct TableHdr {                      // in shared memory, written by staging
  int n, nk;                           // table length, searched keys (n-1)
  int P, D;                            // Eytzinger size (power of two) and depth
  int shift, nb, occ;                  // bucket shift, bucket count, max bucket occupancy
  int stride;                          // sample stride (1 = whole table staged)
  int ns;                              // number of staged (sampled) keys
  unsigned bad;                        // table not strictly increasing / NaN
  uint64_t base;                       // bucket of keys[0]
};

struct Layout1D {                      // byte offsets into dynamic shared memory
  int hdr, keys, eyt, dir, bytes;
  int dir_cap;                         // bucket budget (0: no directory)
  int stride;                          // >1: two-level (sampled) staging
  int P, D;                            // Eytzinger geometry of the staged keys
  int ns;                              // staged key count
};

__host__ __device__ inline int ceil_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
__host__ __device__ inline int ilog2(int p) {  // p a power of two
  int d = 0;
  while ((1 << d) < p) ++d;
  return d;
}

// Host: shared-memory plan for a table of n entries.
// want_eyt / want_keys / dir_cap select what is staged.
inline Layout1D make_layout_1d(int n, bool want_keys, bool want_eyt, int dir_cap, int offset = 0) {
  Layout1D L{};
  const int nk = n - 1;
  L.stride = 1;
  while ((nk + L.stride - 1) / L.stride > kMaxSmemKeys) L.stride <<= 1;
  L.ns = (nk + L.stride - 1) / L.stride;
  L.P = ceil_pow2(L.ns + 1);
  L.D = ilog2(L.P);
  L.dir_cap = dir_cap;
  int off = offset;
  auto take = [&](int bytes) { int o = off; off += (bytes + 15) & ~15; return o; };
  L.hdr = take(sizeof(TableHdr));
  L.keys = want_keys ? take((L.ns + kPad) * 8) : -1;
  L.eyt = want_eyt ? take(L.P * 8) : -1;
  L.dir = dir_cap > 0 ? take((dir_cap + 1) * 4) : -1;
  L.bytes = off;
  return L;
}

// In-order rank of breadth-first node i (1-based) in a complete tree of depth D.
__device__ __forceinline__ int eyt_rank(int i, int D) {
  const int l = 31 - __clz(i);
  const int p = i - (1 << l);
  return ((2 * p + 1) << (D - 1 - l)) - 1;
}

// Count of staged keys below q by branchless bisection (fixed trip count).
__device__ __forceinline__ int lower_count(const uint64_t* keys, int nk, uint64_t q) {
  int lo = 0, len = nk;
  while (len > 0) {
    const int half = len >> 1;
    if (keys[lo + half] < q) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Staging.  Every thread of the block must call it; it ends with a barrier.
// X is read through the read-only path; the check of strict increase covers
// X[0] too (a NaN fails every comparison).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stage_table_1d(const double* __restrict__ X, int n, const Layout1D& lay,
                               unsigned char* smem) {
  TableHdr& h = *reinterpret_cast<TableHdr*>(smem + lay.hdr);
  uint64_t* keys = lay.keys >= 0 ? reinterpret_cast<uint64_t*>(smem + lay.keys) : nullptr;
  uint64_t* eyt = lay.eyt >= 0 ? reinterpret_cast<uint64_t*>(smem + lay.eyt) : nullptr;
  int* dir = lay.dir >= 0 ? reinterpret_cast<int*>(smem + lay.dir) : nullptr;
  const int nk = n - 1, tid = threadIdx.x, nt = blockDim.x;
  const int stride = lay.stride, ns = lay.ns;
  if (tid == 0) {
    h.n = n; h.nk = nk; h.P = lay.P; h.D = lay.D; h.stride = stride; h.ns = ns;
    h.bad = 0u; h.shift = 0; h.nb = 0; h.occ = 0; h.base = 0;
  }
  __syncthreads();
  // sortedness check over the whole table (strided over threads)
  bool bad = false;
  for (int j = tid; j < nk; j += nt) {
    const double a = __ldg(X + j), b = __ldg(X + j + 1);
    bad |= !(b > a);
  }
  if (__syncthreads_or(bad) && tid == 0) h.bad = 1u;
  // staged keys: the (sampled) images of X[1..n-1]; sample s covers entry s*stride+1 .. +stride
  // and holds the LAST key of its block so that counting samples below q counts whole blocks.
  auto staged_key = [&](int s) -> uint64_t {
    const int j = min((s + 1) * stride, nk);   // 1-based entry index of the block's last key
    return order_key(__ldg(X + j));
  };
  if (keys != nullptr) {
    for (int s = tid; s < ns + kPad; s += nt) keys[s] = s < ns ? staged_key(s) : kKeyMax;
  }
  if (eyt != nullptr) {
    for (int i = tid; i < lay.P; i += nt) {
      if (i == 0) { eyt[0] = kKeyMax; continue; }
      const int r = eyt_rank(i, lay.D);
      eyt[i] = r < ns ? staged_key(r) : kKeyMax;
    }
  }
  __syncthreads();
  if (dir != nullptr) {
    if (tid == 0) {
      const uint64_t k0 = keys[0], k1 = keys[ns - 1];
      // smallest shift s with (k1 >> s) - (k0 >> s) < dir_cap.  That
      // difference never grows with s, and exceeds span / 2^s - 1, so every
      // s below bitlen(span) - bitlen(dir_cap + 1) still leaves it at least
      // dir_cap: the scan starts there (a step or two instead of up to 63).
      // The span is unsigned: a table may cover more than half of the key range.
      const uint64_t span = k1 - k0;
      const int bl = 64 - __clzll((long long)span), bc = 32 - __clz(lay.dir_cap + 1);
      int s = max(0, bl - bc - 1);
      while (s < 63 && ((k1 >> s) - (k0 >> s)) >= (uint64_t)lay.dir_cap) ++s;
      h.shift = s;
      h.base = k0 >> s;
      h.nb = (int)min((k1 >> s) - (k0 >> s) + 1, (uint64_t)lay.dir_cap);
    }
    __syncthreads();
    const int s = h.shift, nb = h.nb;
    const uint64_t base = h.base;
    for (int b = tid; b <= nb; b += nt)
      dir[b] = b == nb ? ns : lower_count(keys, ns, (base + (uint64_t)b) << s);
    __syncthreads();
    int occ = 0;
    for (int b = tid; b < nb; b += nt) occ = max(occ, dir[b + 1] - dir[b]);
    occ = __reduce_max_sync(0xFFFFFFFFu, occ);
    if ((tid & 31) == 0) atomicMax(&h.occ, occ);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Search routines on a staged table.  Each returns the count of staged keys
// below q; for stride 1 that is the final index.
// ---------------------------------------------------------------------------

// Branchless binary search over the breadth-first layout (Sec. 3.2, with the
// bound selection turned into an index update i = 2i + [eyt[i] < q]).
template <int D>
__device__ __forceinline__ int search_eyt(const uint64_t* __restrict__ eyt, uint64_t q) {
  int i = 1;
#pragma unroll
  for (int l = 0; l < D; ++l) i = 2 * i + (eyt[i] < q ? 1 : 0);
  return i - (1 << D);
}

__device__ __forceinline__ int search_eyt_rt(const uint64_t* __restrict__ eyt, int D, uint64_t q) {
  int i = 1;
  for (int l = 0; l < D; ++l) i = 2 * i + (eyt[i] < q ? 1 : 0);
  return i - (1 << D);
}

// Bucket of query key q, clamped to [0, nb-1].  Shifts of 32 or more (the
// common case: buckets no finer than 2^-20 of an octave) need only the key's
// high word.  HI fixes that case at compile time, so a caller that has
// checked the shift once per table runs the search as straight-line code.
template <bool HI>
__device__ __forceinline__ int bucket_index_t(uint64_t q, int shift, uint64_t base, int nb) {
  if (HI) {
    const uint32_t hb = (uint32_t)(q >> 32) >> (shift - 32);
    const uint32_t d = hb - (uint32_t)base;                 // base < 2^32 here
    return hb < (uint32_t)base ? 0 : (int)min(d, (uint32_t)(nb - 1));
  }
  const uint64_t hb = q >> shift;
  return hb < base ? 0 : (int)min(hb - base, (uint64_t)(nb - 1));
}

// The same with the case taken per call (the branch is uniform across a block).
__device__ __forceinline__ int bucket_index(uint64_t q, int shift, uint64_t base, int nb) {
  return shift >= 32 ? bucket_index_t<true>(q, shift, base, nb) : bucket_index_t<false>(q, shift, base, nb);
}

// Bucket directory + fixed-length scan (occupancy <= SCAN, Sec. 3.5's
// linear search inside a bin).  Keys past the bucket are larger than q (they
// sit in later buckets) or are sentinels, so scanning them adds nothing.
// D: directory entry type (int in one-shot calls, uint16_t in plans); HI:
// 1 when the shift is known to be 32 or more, 0 when it is known not to be,
// -1 to decide per call.
template <int SCAN, int HI = -1, class D>
__device__ __forceinline__ int search_bucket(const uint64_t* __restrict__ keys, const D* __restrict__ dir,
                                             int shift, uint64_t base, int nb, uint64_t q) {
  const int b = HI < 0 ? bucket_index(q, shift, base, nb) : bucket_index_t<(HI > 0)>(q, shift, base, nb);
  const int lo = dir[b];
  int c = lo;
#pragma unroll
  for (int j = 0; j < SCAN; ++j) c += keys[lo + j] < q ? 1 : 0;
  return c;
}

// Bucket directory + bounded bisection inside the bucket (T = bit length of
// the largest occupancy).
template <class D>
__device__ __forceinline__ int search_bucket_bisect(const uint64_t* __restrict__ keys, const D* __restrict__ dir,
                                                    int shift, uint64_t base, int nb, int T, uint64_t q) {
  const int b = bucket_index(q, shift, base, nb);
  int lo = dir[b], len = dir[b + 1] - lo;
  for (int it = 0; it < T; ++it) {
    const int half = len >> 1;
    const bool go = len > 0 && keys[lo + half] < q;
    lo = go ? lo + half + 1 : lo;
    len = go ? len - half - 1 : half;
  }
  return lo;
}

// Textbook bisection with data-dependent branches and trip count (the
// "branching" variant of the Sec. 5.4 comparison).
__device__ __forceinline__ int search_branchy(const uint64_t* __restrict__ keys, int nk, uint64_t q) {
  int lo = 0, hi = nk;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < q) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Warp-cooperative (G+1)-ary search: G lanes each compare q against one
// pivot, __ballot_sync collects the outcomes and __popc counts the pivots
// below q.  Every lane of the G-lane group must call it with the group's q
// (the caller broadcasts q).  S0 = (G+1)^(levels-1).
template <int G>
__device__ __forceinline__ int search_ballot(const uint64_t* __restrict__ keys, int nk, int S0, uint64_t q) {
  const int lane = threadIdx.x & 31;
  const int g = lane & (G - 1);
  const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  int lo = 0;
  for (int S = S0; S >= 1; S /= (G + 1)) {
    const int idx = lo + (g + 1) * S - 1;
    const uint64_t piv = keys[min(idx, nk)];                 // keys[nk] is a sentinel
    const unsigned vote = __ballot_sync(0xFFFFFFFFu, piv < q) & gmask;
    lo += __popc(vote) * S;
  }
  return lo;
}

// Last log2(stride) steps of the two-level search: count the entries
// X[1 + c*stride .. ] of block c that lie below q, reading X from global.
__device__ __forceinline__ int search_leaf_global(const double* __restrict__ X, int nk, int stride, int c,
                                                  uint64_t q) {
  // all keys of blocks 0..c-1 lie below q; when every sample does (c = ns)
  // the count is nk even if the last block is short
  int lo = min(c * stride, nk);
  int len = min(stride, nk - lo);
  while (len > 0) {
    const int half = len >> 1;
    const uint64_t k = order_key(__ldg(X + 1 + lo + half));
    if (k < q) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

}  // namespace ss
