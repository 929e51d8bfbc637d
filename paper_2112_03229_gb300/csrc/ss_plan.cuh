// ss_plan.cuh -- prepared tables ("blobs") kept in device memory by a plan,
// staged into shared memory with one TMA bulk copy per table, and the
// searches that run on a staged blob (plain, bucket, ballot, and the two
// learned proposals with their exact fix-up).
//
// Set-up happens once per loaded table, as Sec. 5.3 prescribes for EOSPAC
// (tables are loaded once at program start), so the per-call work is only
// the stream of targets.
//
// Blob layout (all offsets from the blob start, 16-byte aligned):
//   [BlobHdr 128 B][mlp 65 floats, padded to 272 B][dir (cap+1) uint16]
//   [keys (ns + kPad) uint64][eyt P uint64]           <- staged part
//   [full keys nk + kPad uint64][fine dir]             <- global only (stride > 1)
//   [wide section]                                    <- tables of 8129 .. ~76K keys
// keys hold the images of X[1..n-1] (sampled every `stride` entries for big
// tables, see ss_table.cuh); full keys hold all of them.
//
// Wide section (a table too large for shared memory as 8-byte keys, but not
// as 16-bit offsets): the keys form leaves of 16; per leaf, its last key (the
// sample), a shift, and the first 15 keys as offsets from the previous
// leaf's last key, shifted right until they fit 15 bits (stored in 16, with
// bit 15 set so that the packed comparison needs no mask of its own); the
// 16th slot holds the shift (the 16th key is the sample itself).  A target's
// leaf comes from a bucket directory over the samples; inside the leaf a
// packed comparison of the offsets, two per 32-bit word, decides every key
// except those whose offset equals the target's, which are compared in full
// from global memory (rare: the truncation would have to land on the same
// step).  Everything else is one shared-memory stage of about 2.5 bytes per
// key.
#pragma once

#include "ss_ff.cuh"
#include "ss_model.cuh"
#include "ss_table.cuh"

namespace ss {

enum BlobAlgo : int { BL_BUCKET = 0, BL_BINARY = 1, BL_BALLOT8 = 2, BL_BALLOT16 = 3, BL_BALLOT32 = 4,
                      BL_SPLINE = 5, BL_MLP = 6, BL_LOGHASH = 7, BL_WIDE = 8, BL_NUM = 9 };

struct __align__(16) BlobHdr {
  int n, nk, ns, stride;     // table length, searched keys, staged keys, sample stride
  int algo;                  // BlobAlgo in use (written by plan creation / the autotuner)
  int D;                     // Eytzinger depth of the staged keys
  int shift, nb, occ;        // bucket directory (also the spline knots)
  int E;                     // learned half-window (count units); proposals are checked exactly
  int S0;                    // top-level stride of the ballot search
  int dir_cap;
  int off_mlp, off_dir, off_keys, off_eyt;   // staged sections
  int staged_end;            // end of the staged part
  int gshift;                // fine directory over all keys (sampled tables): bucket shift
  int64_t off_full;          // full keys (global)
  uint64_t base;             // bucket of keys[0]
  uint64_t k0;               // key of X[0]
  float e_lo, e_scale;       // MLP feature scaling
  float loss;                // final training loss of the MLP (diagnostic)
  int gnb;                   // fine directory: bucket count (0: none)
  // 2D axes only: per-cell float-float data follows the staged part
  int off_cells;             // cell table of n-1 cells (staged with the axis, 16-byte aligned), -1 for 1D
  int ffok;                  // cells usable by the float-float path
  uint64_t gbase;            // fine directory: bucket of the first key
};
static_assert(sizeof(BlobHdr) == 128, "blob header must stay 128 bytes");

constexpr int kMlpBytes = 272;

struct BlobGeom {
  int ns, stride, P, D;
  int off_mlp, off_dir, off_keys, off_eyt, off_cells, staged_end;
  int64_t off_full, off_wide, bytes;   // off_wide: -1 without a wide section
};

// Bucket budget of the fine directory of a sampled table (all keys, global memory).
__host__ __device__ inline int fine_dir_cap(int nk) { return nk < (1 << 16) ? 4 * nk : (1 << 18); }

// Wide section geometry (offsets from the section start, 16-byte aligned).
constexpr int kLeaf = 16;                         // keys per leaf
constexpr int kWideSmemBudget = 224 * 1024;       // header + section, staged whole

struct WideHdr {                                  // first 48 bytes of the section
  uint64_t base;                                  // bucket of samples[0]
  int shift, nb, occ;                             // bucket directory over the samples
  int L;                                          // leaves (= samples)
  int dcap;
  int off_dir, off_samples, off_shift, off_leaf;
  int pad;
};
static_assert(sizeof(WideHdr) == 48, "wide header size");

struct WideGeom {
  int L, dcap, off_dir, off_samples, off_shift, off_leaf, bytes;
};

// Bytes of a wide section besides its directory: header, samples (with
// sentinels), shifts (a copy of each leaf's slot 15, which the search reads;
// the copy is checked when a plan file is read) and leaves.
__host__ __device__ inline int wide_rest_bytes(int L) {
  return (int)sizeof(WideHdr) + ((((L + kPad) * 8) + 15) & ~15) + ((L + 15) & ~15) + L * kLeaf * 2;
}

// The sample directory holds 16-bit counts (at most L samples) and takes
// the shared memory the rest of the section leaves within the budget, up to
// six buckets per sample: on clustered tables a finer directory leaves
// fewer samples per bucket to search.
__host__ __device__ inline WideGeom wide_geom(int nk) {
  WideGeom w{};
  w.L = (nk + kLeaf - 1) / kLeaf;
  const int room = (kWideSmemBudget - (int)sizeof(BlobHdr) - wide_rest_bytes(w.L) - 16) / 2 - 1;
  w.dcap = room < 64 ? 64 : (room > 6 * w.L ? 6 * w.L : room);
  int off = (int)sizeof(WideHdr);
  w.off_dir = off;     off += (((w.dcap + 1) * 2) + 15) & ~15;
  w.off_samples = off; off += (((w.L + kPad) * 8) + 15) & ~15;
  w.off_shift = off;   off += (w.L + 15) & ~15;
  w.off_leaf = off;    off += w.L * kLeaf * 2;
  w.bytes = off;
  return w;
}

// A table gets a wide section when its keys exceed shared memory as 8-byte
// keys and the section fits the budget with a directory of at least two
// buckets per sample (at most 8192) in 32-bit entries.
__host__ __device__ inline bool wide_eligible(int nk) {
  if (nk <= kMaxSmemKeys) return false;
  const int L = (nk + kLeaf - 1) / kLeaf;
  const int dmin = L * 2 > 8192 ? 8192 : L * 2;
  return (int64_t)sizeof(BlobHdr) + wide_rest_bytes(L) + ((((dmin + 1) * 4) + 15) & ~15) <= kWideSmemBudget;
}

// Blob offset of the wide section: after the global-only keys and fine directory.
__host__ __device__ inline int64_t wide_offset(int64_t off_full, int nk) {
  return (off_full + (int64_t)(nk + kPad) * 8 + (int64_t)(fine_dir_cap(nk) + 1) * 4 + 15) & ~(int64_t)15;
}

// Byte range of the staged part that an algorithm needs: [lo, hi) besides the header.
__host__ __device__ inline void staged_range(const BlobHdr& h, int& lo, int& hi) {
  if (h.algo == BL_WIDE) {
    lo = (int)wide_offset(h.off_full, h.nk);
    hi = lo + wide_geom(h.nk).bytes;
    return;
  }
  switch (h.algo) {
    case BL_BINARY: lo = h.off_eyt; hi = h.off_eyt + (1 << h.D) * 8; break;
    case BL_BALLOT8: case BL_BALLOT16: case BL_BALLOT32: lo = h.off_keys; hi = h.off_keys + (h.ns + kPad) * 8; break;
    default: lo = h.off_mlp; hi = h.off_keys + (h.ns + kPad) * 8; break;   // bucket, spline, mlp, loghash
  }
  if (h.off_cells >= 0) {
    // 2D axes keep their cells right after, and always their keys: the
    // weights and the hunt read entries of the axis whatever its search
    hi = h.staged_end;
    lo = lo < h.off_keys ? lo : h.off_keys;
  }
  lo &= ~15;
  hi = (hi + 15) & ~15;
}

// ---------------------------------------------------------------------------
// TMA bulk copy global -> shared, completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier; gives up after a bounded number of
// polls and returns false (the caller records an error instead of hanging).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// View of a staged blob in shared memory.
struct StagedView {
  BlobHdr h;                 // header fields, held in registers
  const float* mlp;
  const uint16_t* dir;       // bucket directory: counts of staged keys (at most 8128) in 16 bits
  const uint64_t* keys;
  const uint64_t* eyt;
  CellTable cells;           // 2D axes: per-cell weight data
  const uint64_t* full;      // global full keys (stride > 1)
  const int* gdir;           // global fine directory over all keys (stride > 1)
};

// Stage blob `src` (global) into smem at `dst`: header, then the range the
// algorithm needs placed right after it.  Must be called by all threads;
// thread 0 issues the copies.  Returns the view (pointers into dst) and
// sets ok=false if the wait timed out.
__device__ __forceinline__ StagedView stage_blob(const unsigned char* __restrict__ src, unsigned char* dst,
                                                 uint64_t* bar, uint32_t& phase, bool& ok) {
  const BlobHdr* gh = reinterpret_cast<const BlobHdr*>(src);
  BlobHdr hdr;
  // every thread reads the header through the read-only path (it is tiny and cached)
  const int4* gh4 = reinterpret_cast<const int4*>(gh);
  int4* hp = reinterpret_cast<int4*>(&hdr);
#pragma unroll
  for (int i = 0; i < 8; ++i) hp[i] = __ldg(gh4 + i);
  int lo, hi;
  staged_range(hdr, lo, hi);
#ifdef SS_CHECKED
  // the staged bytes must fit the block's dynamic shared memory from dst on,
  // and every array the table's search reads must lie inside the staged range
  bool fits;
  {
    extern __shared__ unsigned char ss_dynamic_smem[];
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    fits = dst >= ss_dynamic_smem && dst + sizeof(BlobHdr) + (hi - lo) <= ss_dynamic_smem + dyn && hi >= lo;
    auto inside = [&](int off, int64_t bytes) { return off >= lo && (int64_t)off + bytes <= (int64_t)hi; };
    const int a = hdr.algo;
    const bool keys = a == BL_BUCKET || a == BL_SPLINE || a == BL_MLP || a == BL_LOGHASH ||
                      (a >= BL_BALLOT8 && a <= BL_BALLOT32) || hdr.off_cells >= 0;
    const bool dir = a == BL_BUCKET || a == BL_SPLINE || a == BL_MLP || a == BL_LOGHASH;
    bool ok_arrays = true;
    if (keys) ok_arrays &= inside(hdr.off_keys, (int64_t)(hdr.ns + kPad) * 8);
    if (dir) ok_arrays &= inside(hdr.off_dir, (int64_t)(hdr.nb + 1) * 2) && hdr.nb <= hdr.dir_cap;
    if (a == BL_MLP || a == BL_LOGHASH) ok_arrays &= inside(hdr.off_mlp, kMlpBytes);
    if (a == BL_BINARY) ok_arrays &= inside(hdr.off_eyt, (int64_t)8 << hdr.D);
    if (hdr.off_cells >= 0) ok_arrays &= inside(hdr.off_cells, (int64_t)(hdr.n - 1) * kCellBytes);
    if (threadIdx.x == 0) SS_CHECK(!fits || !ok_arrays);
  }
#endif
  __syncthreads();          // previous users of dst are done
  if (threadIdx.x == 0) {
    fence_proxy_async();
    const uint32_t bytes = (uint32_t)(sizeof(BlobHdr) + (hi - lo));
#ifdef SS_CHECKED
    if (!fits) {
      mbar_arrive(bar);     // nothing copied: the phase completes, the block gives up below
    } else
#endif
    {
      mbar_expect_tx(bar, bytes);
      tma_load_1d(dst, src, (uint32_t)sizeof(BlobHdr), bar);
      if (hi > lo) tma_load_1d(dst + sizeof(BlobHdr), src + lo, (uint32_t)(hi - lo), bar);
    }
  }
  ok &= mbar_wait(bar, phase);
#ifdef SS_CHECKED
  ok &= fits;
#endif
  ok = __syncthreads_and(ok);          // uniform outcome for the whole block
  phase ^= 1u;
  const int shift_off = (int)sizeof(BlobHdr) - lo;     // smem position of blob offset o is o + shift_off
  StagedView v;
  v.h = hdr;
  v.mlp = reinterpret_cast<const float*>(dst + hdr.off_mlp + shift_off);
  v.dir = reinterpret_cast<const uint16_t*>(dst + hdr.off_dir + shift_off);
  v.keys = reinterpret_cast<const uint64_t*>(dst + hdr.off_keys + shift_off);
  v.eyt = reinterpret_cast<const uint64_t*>(dst + hdr.off_eyt + shift_off);
  v.cells = hdr.off_cells >= 0 ? cell_table(dst + hdr.off_cells + shift_off, hdr.n - 1) : CellTable{nullptr, nullptr};
  v.full = hdr.off_full >= 0 ? reinterpret_cast<const uint64_t*>(src + hdr.off_full) : nullptr;
  v.gdir = hdr.gnb > 0 ? reinterpret_cast<const int*>(src + hdr.off_full + (int64_t)(hdr.nk + kPad) * 8) : nullptr;
  return v;
}

// Staged wide section (shared memory, right after the staged header).
struct WideView {
  WideHdr w;                    // directory parameters, in registers
  const uint16_t* dir;          // bucket directory over the samples (16-bit counts)
  const uint64_t* samples;      // last key of each leaf, then kPad sentinels
  const uint16_t* leaf;         // offsets 0..7 of every leaf (16 bytes each), then offsets 8..15 of every leaf
  const uint64_t* full;         // all keys, global memory (ties)
  uint64_t k0;                  // key of X[0]: the base of leaf 0
  int nk;
};

__device__ __forceinline__ WideView wide_view(const unsigned char* sec, const StagedView& v) {
  WideView wv;
  wv.w = *reinterpret_cast<const WideHdr*>(sec);
  wv.dir = reinterpret_cast<const uint16_t*>(sec + wv.w.off_dir);
  wv.samples = reinterpret_cast<const uint64_t*>(sec + wv.w.off_samples);
  wv.leaf = reinterpret_cast<const uint16_t*>(sec + wv.w.off_leaf);
  wv.full = v.full;
  wv.k0 = v.h.k0;
  wv.nk = v.h.nk;
  return wv;
}

// Number of the sixteen slots of a leaf (a, b: eight 32-bit words, two
// 16-bit slots each) that are at least t (t <= 0x8000).  Slots 0..14 hold
// the leaf's 15-bit key offsets with bit 15 set: (0x8000 | x) - t keeps bit
// 15 set exactly when x >= t and never borrows into the other half of the
// word.  Slot 15 holds the leaf's shift instead (its key is the leaf's
// sample, at least the target by the choice of the leaf) and always counts.
// The flags of four words are gathered at distinct bit positions (shifts
// 0..3) for one popc; slot 15's lands on bit 28.
__device__ __forceinline__ int count_ge15(const uint4& a, const uint4& b, uint32_t t) {
  const uint32_t t2 = t | (t << 16);
  const uint32_t m = 0x80008000u;
  const uint32_t pa = ((a.x - t2) & m) | (((a.y - t2) & m) >> 1) | (((a.z - t2) & m) >> 2) | (((a.w - t2) & m) >> 3);
  const uint32_t pb = ((b.x - t2) & m) | (((b.y - t2) & m) >> 1) | (((b.z - t2) & m) >> 2) | (((b.w - t2) & m) >> 3);
  return __popc(pa) + __popc(pb | (1u << 28));
}

// Count of keys below q on a wide section: the leaf from the sample
// directory (SCAN 1 or 2: at most that many samples per bucket, compared
// with independent reads; 0: bisection inside the bucket); in the leaf, the
// 16 offsets (15 bits each) are compared with the target's, two per 32-bit
// word: offsets below it belong to smaller keys, above it to larger ones;
// the keys whose offset equals the target's are compared in full.
template <int SCAN>
__device__ __forceinline__ int wide_count(const WideView& wv, uint64_t q) {
  const int nsamp = wv.w.L + kPad, ndir = wv.w.dcap + 1;   // array sizes (checked build)
  (void)nsamp;
  (void)ndir;
  const int bk = bucket_index(q, wv.w.shift, wv.w.base, wv.w.nb);
  const int lo = wv.dir[SS_IX(bk, ndir)];
  int s = lo;
  uint64_t base;                                 // last key of the previous leaf
  if (SCAN >= 1) {
    // samples past the bucket are larger than q, or sentinels; the leaf's base
    // is one of the samples just compared unless no sample is below q
    const uint64_t k0 = wv.samples[SS_IX(lo, nsamp)], k1 = SCAN >= 2 ? wv.samples[SS_IX(lo + 1, nsamp)] : 0;
    s += (k0 < q ? 1 : 0) + (SCAN >= 2 && k1 < q ? 1 : 0);
    if (s >= wv.w.L) return wv.nk;
    base = s == lo ? (lo > 0 ? wv.samples[SS_IX(lo - 1, nsamp)] : wv.k0) : (s == lo + 1 ? k0 : k1);
  } else {
    int len = wv.dir[SS_IX(bk + 1, ndir)] - s;
    const int T = 32 - __clz(wv.w.occ);
    for (int it = 0; it < T; ++it) {
      const int half = len >> 1;
      const bool go = len > 0 && wv.samples[SS_IX(s + half, nsamp)] < q;
      s = go ? s + half + 1 : s;
      len = go ? len - half - 1 : half;
    }
    if (s >= wv.w.L) return wv.nk;
    base = s > 0 ? wv.samples[SS_IX(s - 1, nsamp)] : wv.k0;
  }
  if (q <= base) return kLeaf * s;               // only below X[0] (leaf 0)
  // the two halves of a leaf sit in two arrays of 16-byte entries: read at a
  // 16-byte stride, a warp's random leaves spread over all shared-memory banks
  // (one 32-byte leaf read as two 16-byte halves used half of them); the
  // leaf's shift is its last slot
  const uint4* l4 = reinterpret_cast<const uint4*>(wv.leaf);
  const uint4 a = l4[SS_IX(s, wv.w.L)], b = l4[SS_IX(wv.w.L + s, 2 * wv.w.L)];
  const uint32_t tq = (uint32_t)((q - base) >> (b.w >> 16));   // < 2^15: q <= samples[s]
  int c = kLeaf - count_ge15(a, b, tq);                          // offsets below the target's
  // a leaf's offsets never decrease, so offsets equal to the target's (whose
  // keys are compared in full) start at position c; offset c, picked from the
  // words already in registers, rules them out, and only a tie pays for the
  // second packed count
  const int wi = c >> 1;
  const uint32_t wc = wi < 4 ? (wi < 2 ? (wi == 0 ? a.x : a.y) : (wi == 2 ? a.z : a.w))
                             : (wi < 6 ? (wi == 4 ? b.x : b.y) : (wi == 6 ? b.z : b.w));
  if (c < kLeaf && ((c & 1) ? (wc >> 16) : (wc & 0xFFFFu)) == (tq | 0x8000u)) {
    const int le = kLeaf - count_ge15(a, b, tq + 1);             // offsets at most the target's
    for (; c < le; ++c) {
      const int j = kLeaf * s + c;
      if (j >= wv.nk || __ldg(wv.full + SS_IX(j, wv.nk + kPad)) >= q) break;
    }
  }
  return kLeaf * s + c;
}

// Count over the full searched set after the staged count c (two-level tables).
__device__ __forceinline__ int finish_full(const StagedView& v, int c, uint64_t q) {
  const BlobHdr& h = v.h;
  if (h.stride == 1) return c;
  int lo = min(c * h.stride, h.nk);
  int len = min(h.stride, h.nk - lo);
  while (len > 0) {
    const int half = len >> 1;
    if (__ldg(v.full + SS_IX(lo + half, h.nk + kPad)) < q) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

// Key i (0-based among X[1..n-1]) of the table, from shared memory when the
// whole table is staged, else from the global full keys.
__device__ __forceinline__ uint64_t key_at(const StagedView& v, int i) {
  return v.h.stride == 1 ? v.keys[SS_IX(i, v.h.ns + kPad)] : __ldg(v.full + SS_IX(i, v.h.nk + kPad));
}

// Plain count of keys below q with the bucket directory (any occupancy).
__device__ __forceinline__ int plain_bucket(const StagedView& v, uint64_t q) {
  const BlobHdr& h = v.h;
  const int T = h.occ > 0 ? 32 - __clz(h.occ) : 0;
  const int c = h.occ <= 1 ? search_bucket<1>(v.keys, v.dir, h.shift, h.base, h.nb, q)
                           : search_bucket_bisect(v.keys, v.dir, h.shift, h.base, h.nb, T, q);
  return finish_full(v, c, q);
}

__device__ __forceinline__ int plain_binary(const StagedView& v, uint64_t q) {
  return finish_full(v, search_eyt_rt(v.eyt, v.h.D, q), q);
}

// Learned search in a window: proposal p (count units), exact check that the
// answer lies in [p-E, p+E], then the count inside the window; plain bucket
// search if the check fails.  Windows of at most 6 keys are scanned with
// independent loads (one memory round trip), wider ones bisected.  KEYS reads
// the keys from shared memory (whole table staged) or global memory (sampled
// table).  Staged tables with small windows walk from the proposal instead
// (learned_count).
template <class KEYS>
__device__ __forceinline__ int window_count(KEYS key, int nk, int E, int p, uint64_t q, bool& ok) {
  const int lo = max(p - E, 0), hi = min(p + E, nk);
  // both key arrays end in sentinels above every key, so key(hi) exists for
  // hi == nk and the check needs no branch
  const uint64_t kb = key(lo > 0 ? lo - 1 : 0), ke = key(hi);
  ok = ((lo == 0) | (kb < q)) & (ke >= q);
  if (E <= 3) {
    // 2E keys from lo (the window's length at most): those from hi on are at
    // least key(hi), so when the check holds they add nothing (and the answer
    // is discarded when it fails); the branch on E is uniform per table
    int c = lo;
    if (E <= 1) {
      c += (key(lo) < q ? 1 : 0) + (key(lo + 1) < q ? 1 : 0);
    } else if (E == 2) {
#pragma unroll
      for (int j = 0; j < 4; ++j) c += key(lo + j) < q ? 1 : 0;
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) c += key(lo + j) < q ? 1 : 0;
    }
    return c;
  }
  int c = lo, len = hi - lo;
  while (len > 0) {
    const int half = len >> 1;
    if (key(c + half) < q) { c += half + 1; len -= half + 1; } else { len = half; }
  }
  return c;
}

// Largest learned half-window that a staged table walks from the proposal
// (wider windows are checked and bisected by window_count).
constexpr int kProbeWindow = 4;

// Walk from proposal p on staged keys (nk searched keys, keys[nk] a
// sentinel, E <= kProbeWindow): the proposal's two neighbouring keys decide
// it in one shared-memory round trip (the answer is p when key(p-1) < q <=
// key(p)); otherwise they show the direction, and the answer is walked to,
// each step proved by the keys on both sides of it, for at most E keys.
// Returns false when the answer lies farther (the caller searches plainly).
// On staged tables this reads two keys where the window check and scan read
// 2E + 2.
__device__ __forceinline__ bool walk_count(const uint64_t* __restrict__ keys, int lim, int nk, int E, int p,
                                           uint64_t q, int& c) {
  (void)lim;
  const int pp = min(max(p, 0), nk);
  const uint64_t kb = keys[SS_IX(max(pp - 1, 0), lim)], ke = keys[SS_IX(pp, lim)];
  const bool below = (pp > 0) & (kb >= q), above = ke < q;
  c = pp;
  if (!(below | above)) return true;
  if (above) {                               // key(pp) < q: the answer is above pp
    for (int j = pp + 1, st = 0; st < E && j <= nk; ++st, ++j)
      if (q <= keys[SS_IX(j, lim)]) { c = j; return true; }
  } else {                                   // key(pp-1) >= q: the answer is below pp
    for (int j = pp - 1, st = 0; st < E; ++st, --j)
      if (j == 0 || keys[SS_IX(j - 1, lim)] < q) { c = j; return true; }
  }
  return false;
}

__device__ __forceinline__ int learned_count(const StagedView& v, int p, uint64_t q, int& fallbacks) {
  const BlobHdr& h = v.h;
  bool ok;
  int c;
  if (h.stride == 1) {
    const uint64_t* keys = v.keys;
    const int lim = h.ns + kPad;
    if (h.E <= kProbeWindow) {   // uniform per table
      if (walk_count(keys, lim, h.nk, h.E, p, q, c)) return c;
      ++fallbacks;
      return plain_bucket(v, q);
    }
    c = window_count([keys, lim](int i) { return keys[SS_IX(i, lim)]; }, h.nk, h.E, p, q, ok);
  } else {
    const uint64_t* full = v.full;
    const int lim = h.nk + kPad;
    c = window_count([full, lim](int i) { return __ldg(full + SS_IX(i, lim)); }, h.nk, h.E, p, q, ok);
  }
  if (!ok) {
    ++fallbacks;
    return plain_bucket(v, q);
  }
  return c;
}

// Hunt and locate (Sec. 2.1; coherent targets, Sec. 5.5): the count of keys
// below q starting from a guess p in [0, nk], the answer of a nearby target.
// The keys around the guess are read together, so an answer of p or p + 1
// costs one memory round trip; otherwise the bracket grows away from the
// guess in doubling steps (2, 4, ... up to 2^kHuntProbes keys) until a key on
// the far side of q is found, and a bisection inside the last step finishes.
// A target further away than the probes reach is searched with the table's
// own search (`plain`), which costs O(1) round trips with the bucket
// directory: on the GPU that bound beats an unbounded probe (measured).
// Exact for any guess; every loop is bounded.  key(nk) must be a sentinel
// above every query.
constexpr int kHuntProbes = 4;

template <class KEYS, class PLAIN>
__device__ __forceinline__ int hunt_from(KEYS key, int nk, int p, uint64_t q, PLAIN&& plain) {
  p = min(max(p, 0), nk);
  const uint64_t km1 = p > 0 ? key(p - 1) : 0, k0 = key(p), kp1 = key(min(p + 1, nk));
  int lo, hi;                                      // the answer lies in [lo, hi]
  if (q <= k0) {
    if (p == 0 || km1 < q) return p;
    hi = p - 1;                                    // below the guess: probe downwards
    lo = -1;
    int s = 2;
    for (int it = 0; it < kHuntProbes; ++it, s <<= 1) {
      const int j = hi - s;
      if (j < 0) { lo = 0; break; }
      if (key(j) < q) { lo = j + 1; break; }
      hi = j;
    }
    if (lo < 0) return plain(q);
  } else {
    if (q <= kp1) return p + 1;                    // k0 < q: p < nk, so p + 1 <= nk
    lo = p + 2;                                    // above: probe upwards
    hi = -1;
    int s = 2;
    for (int it = 0; it < kHuntProbes; ++it, s <<= 1) {
      const int j = min(lo + s - 1, nk);
      if (key(j) >= q) { hi = j; break; }        // key(nk), a sentinel, always ends the probe
      lo = j + 1;
    }
    if (hi < 0) return plain(q);
  }
  int len = hi - lo;                               // keys [lo, hi) still to count
  for (int it = 0; it < kHuntProbes + 1 && len > 0; ++it) {
    const int half = len >> 1;
    if (key(lo + half) < q) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

// Hunt on a staged table (keys in shared memory) or a two-level table (all
// keys in global memory).  A guess below zero means "none": the table's own
// search runs.
__device__ __forceinline__ int hunt_count(const StagedView& v, int p, uint64_t q) {
  const BlobHdr& h = v.h;
  auto plain = [&v](uint64_t qq) { return v.h.algo == BL_BINARY ? plain_binary(v, qq) : plain_bucket(v, qq); };
  if (p < 0) return plain(q);
  if (h.stride == 1) {
    const uint64_t* keys = v.keys;
    const int lim = h.ns + kPad;
    return hunt_from([keys, lim](int i) { return keys[SS_IX(i, lim)]; }, h.nk, p, q, plain);
  }
  const uint64_t* full = v.full;
  const int lim = h.nk + kPad;
  return hunt_from([full, lim](int i) { return __ldg(full + SS_IX(i, lim)); }, h.nk, p, q, plain);
}

// Spline proposal in count units of the whole table.  A sampled (two-level)
// table uses its fine directory over all keys, kept in global memory (two
// L2 loads), so the proposal is as sharp as for a staged table.
__device__ __forceinline__ int spline_proposal(const StagedView& v, uint64_t q) {
  const BlobHdr& h = v.h;
  if (h.stride > 1 && h.gnb > 0) return min((int)rintf(spline_position(v.gdir, h.gshift, h.gbase, h.gnb, q)), h.nk);
  const float pos = spline_position(v.dir, h.shift, h.base, h.nb, q);
  return min((int)rintf(pos * (float)h.stride), h.nk);
}

__device__ __forceinline__ int spline_count(const StagedView& v, uint64_t q, int& fallbacks) {
  return learned_count(v, spline_proposal(v, q), q, fallbacks);
}

// Logarithm-hash proposal: its two coefficients sit after the MLP parameters.
__device__ __forceinline__ int loghash_count(const StagedView& v, double t, uint64_t q, int& fallbacks) {
  return learned_count(v, loghash_propose(v.mlp[kMlpParams], v.mlp[kMlpParams + 1], v.h.nk, t), q, fallbacks);
}

__device__ __forceinline__ int mlp_count(const StagedView& v, double t, uint64_t q, int& fallbacks) {
  const BlobHdr& h = v.h;
  const MlpFeatScale sc{h.e_lo, h.e_scale};
  return learned_count(v, mlp_propose(v.mlp, sc, h.n, t), q, fallbacks);
}

}  // namespace ss
