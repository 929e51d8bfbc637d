// plan_1d.cu -- device side of 1D plans: table preparation (keys, bucket
// directory / spline knots, breadth-first layout, MLP initialisation),
// on-GPU training of the MLP position model, the learned half-window, and the
// persistent batched search kernel that walks a tile queue.
#include "learned.cuh"
#include "plan.h"

namespace ss {

// ---------------------------------------------------------------------------
// Counter-based generator (SplitMix64, Steele, Lea & Flood 2014) for the
// training targets of the position model.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Inverse of order_key for keys of non-NaN doubles.
__device__ __forceinline__ double key_to_double(uint64_t k) {
  const uint64_t u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : (0ull - k);
  return __longlong_as_double((long long)u);
}

// ---------------------------------------------------------------------------
// Preparation: one block per table.  Writes the blob of table k.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prep_1d(PrepArgs a) {
  const int k = blockIdx.x;
  if (k >= a.ntables) return;
  const double* X = a.X + a.X_off[k];
  const int n = (int)(a.X_off[k + 1] - a.X_off[k]);
  unsigned char* blob = a.blobs + a.blob_off[k];
  const BlobGeom g = blob_geom_dev(n, a.dir_cap[k], a.cells);
  BlobHdr* h = reinterpret_cast<BlobHdr*>(blob);
  uint64_t* keys = reinterpret_cast<uint64_t*>(blob + g.off_keys);
  uint64_t* eyt = reinterpret_cast<uint64_t*>(blob + g.off_eyt);
  uint16_t* dir = reinterpret_cast<uint16_t*>(blob + g.off_dir);
  float* mlp = reinterpret_cast<float*>(blob + g.off_mlp);
  uint64_t* full = g.off_full >= 0 ? reinterpret_cast<uint64_t*>(blob + g.off_full) : nullptr;
  const int nk = n - 1, tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_bad, s_occ, s_shift, s_nb;
  __shared__ uint64_t s_base;
  if (tid == 0) { s_bad = 0; s_occ = 0; }
  __syncthreads();
  bool bad = false;
  for (int j = tid; j < nk; j += nt) bad |= !(X[j + 1] > X[j]);
  if (bad) atomicOr(&s_bad, 1);
  // keys: staged sample (last key of each stride block) and, for big tables, all keys
  for (int s = tid; s < g.ns + kPad; s += nt)
    keys[s] = s < g.ns ? order_key(X[min((s + 1) * g.stride, nk)]) : kKeyMax;
  if (full != nullptr)
    for (int j = tid; j < nk + kPad; j += nt) full[j] = j < nk ? order_key(X[j + 1]) : kKeyMax;
  for (int i = tid; i < g.P; i += nt) {
    if (i == 0) { eyt[0] = kKeyMax; continue; }
    const int r = eyt_rank(i, g.D);
    eyt[i] = r < g.ns ? order_key(X[min((r + 1) * g.stride, nk)]) : kKeyMax;
  }
  __syncthreads();
  if (tid == 0) {
    const uint64_t k0 = keys[0], k1 = keys[g.ns - 1];
    int s = 0;
    while (s < 63 && ((k1 >> s) - (k0 >> s)) >= (uint64_t)a.dir_cap[k]) ++s;
    s_shift = s;
    s_base = k0 >> s;
    s_nb = (int)min((k1 >> s) - (k0 >> s) + 1, (uint64_t)a.dir_cap[k]);
  }
  __syncthreads();
  const int shift = s_shift, nb = s_nb;
  const uint64_t base = s_base;
  for (int b = tid; b <= nb; b += nt)
    dir[b] = (uint16_t)(b == nb ? g.ns : lower_count(keys, g.ns, (base + (uint64_t)b) << shift));
  __syncthreads();
  int occ = 0;
  for (int b = tid; b < nb; b += nt) occ = max(occ, dir[b + 1] - dir[b]);
  occ = __reduce_max_sync(0xFFFFFFFFu, occ);
  if ((tid & 31) == 0) atomicMax(&s_occ, occ);
  // fine directory over all keys for sampled tables (global memory)
  __shared__ int s_gshift, s_gnb;
  __shared__ uint64_t s_gbase;
  if (full != nullptr) {
    int* gdir = reinterpret_cast<int*>(blob + g.off_full + (int64_t)(nk + kPad) * 8);
    const int cap = fine_dir_cap(nk);
    __syncthreads();
    if (tid == 0) {
      const uint64_t k0 = full[0], k1 = full[nk - 1];
      int s2 = 0;
      while (s2 < 63 && ((k1 >> s2) - (k0 >> s2)) >= (uint64_t)cap) ++s2;
      s_gshift = s2;
      s_gbase = k0 >> s2;
      s_gnb = (int)min((k1 >> s2) - (k0 >> s2) + 1, (uint64_t)cap);
    }
    __syncthreads();
    for (int b = tid; b <= s_gnb; b += nt)
      gdir[b] = b == s_gnb ? nk : lower_count(full, nk, (s_gbase + (uint64_t)b) << s_gshift);
  } else if (tid == 0) {
    s_gshift = 0;
    s_gnb = 0;
    s_gbase = 0;
  }
  // MLP feature scaling and initial parameters: hinge units spread evenly over
  // the normalised log2 coordinate z = x0 + e_scale * x1 of the table's range
  const uint64_t u0 = static_cast<uint64_t>(__double_as_longlong(X[0]));
  const uint64_t u1 = static_cast<uint64_t>(__double_as_longlong(X[nk]));
  const float e_lo = (float)((int)((u0 >> 52) & 0x7FF) - 1023);
  const float e_hi = (float)((int)((u1 >> 52) & 0x7FF) - 1023);
  const float e_scale = 1.0f / fmaxf(e_hi - e_lo + 1.0f, 1.0f);
  if (tid < kHidden) {
    mlp[2 * tid] = 1.0f;
    mlp[2 * tid + 1] = e_scale;
    mlp[2 * kHidden + tid] = -((float)tid + 0.5f) / (float)kHidden;
    mlp[3 * kHidden + tid] = 0.0f;
  }
  if (tid == kHidden) {
    mlp[4 * kHidden] = 0.5f;
    for (int i = kMlpParams; i < kMlpBytes / 4; ++i) mlp[i] = 0.0f;
    // logarithm-hash coefficients (Eqs. 1-2: n-1 steps of base b between the end points)
    const double x0 = X[0], x1 = X[nk];
    if (x0 > 0.0 && isfinite(x1)) {
      const double steps_per_log2 = (double)nk / (log2(x1) - log2(x0));
      mlp[kMlpParams] = (float)steps_per_log2;
      mlp[kMlpParams + 1] = (float)(-log2(x0) * steps_per_log2);
    }
  }
  __syncthreads();
  // wide section (tables too large for shared memory as 8-byte keys): leaf
  // samples, per-leaf shifts and 16-bit offsets, directory over the samples
  if (g.off_wide >= 0) {
    const WideGeom wg = wide_geom(nk);
    unsigned char* sec = blob + g.off_wide;
    uint16_t* wdir = reinterpret_cast<uint16_t*>(sec + wg.off_dir);
    uint64_t* ws = reinterpret_cast<uint64_t*>(sec + wg.off_samples);
    uint8_t* wsh = sec + wg.off_shift;
    uint16_t* wl = reinterpret_cast<uint16_t*>(sec + wg.off_leaf);
    __shared__ int s_wshift, s_wnb, s_wocc;
    __shared__ uint64_t s_wbase;
    for (int s = tid; s < wg.L + kPad; s += nt) ws[s] = s < wg.L ? full[min((s + 1) * kLeaf, nk) - 1] : kKeyMax;
    __syncthreads();
    const uint64_t kx0 = order_key(X[0]);
    for (int s = tid; s < wg.L; s += nt) {
      const uint64_t b = s > 0 ? ws[s - 1] : kx0;
      const uint64_t d = ws[s] - b;                          // > 0 for a strictly increasing table
      const int sh = max(0, 64 - __clzll((long long)d) - 15);   // offsets fit 15 bits
      wsh[s] = (uint8_t)sh;
      // leaf s: offsets 0..7 at wl[8s..], offsets 8..15 in a second array after all leaves
      for (int j = 0; j < kLeaf; ++j) {
        const int i = s * kLeaf + j;
        const int at = j < kLeaf / 2 ? s * (kLeaf / 2) + j : (wg.L + s) * (kLeaf / 2) + (j - kLeaf / 2);
        // slot 15 holds the shift: its key is the leaf's sample, which the
        // search never counts (the chosen leaf's sample is at least the target)
        wl[at] = j == kLeaf - 1 ? (uint16_t)sh
                 : i < nk       ? (uint16_t)(0x8000u | (uint32_t)((full[i] - b) >> sh))
                                : (uint16_t)0xFFFF;
      }
    }
    if (tid == 0) {
      const uint64_t a0 = ws[0], a1 = ws[wg.L - 1];
      int sft = 0;
      while (sft < 63 && ((a1 >> sft) - (a0 >> sft)) >= (uint64_t)wg.dcap) ++sft;
      s_wshift = sft;
      s_wbase = a0 >> sft;
      s_wnb = (int)min((a1 >> sft) - (a0 >> sft) + 1, (uint64_t)wg.dcap);
      s_wocc = 0;
    }
    __syncthreads();
    for (int b = tid; b <= s_wnb; b += nt)
      wdir[b] = (uint16_t)(b == s_wnb ? wg.L : lower_count(ws, wg.L, (s_wbase + (uint64_t)b) << s_wshift));
    __syncthreads();
    int oc = 0;
    for (int b = tid; b < s_wnb; b += nt) oc = max(oc, wdir[b + 1] - wdir[b]);
    oc = __reduce_max_sync(0xFFFFFFFFu, oc);
    if ((tid & 31) == 0) atomicMax(&s_wocc, oc);
    __syncthreads();
    if (tid == 0) {
      WideHdr wh{};
      wh.base = s_wbase;
      wh.shift = s_wshift; wh.nb = s_wnb; wh.occ = s_wocc;
      wh.L = wg.L; wh.dcap = wg.dcap;
      wh.off_dir = wg.off_dir; wh.off_samples = wg.off_samples; wh.off_shift = wg.off_shift; wh.off_leaf = wg.off_leaf;
      *reinterpret_cast<WideHdr*>(sec) = wh;
    }
  }
  if (tid == 0) {
    BlobHdr hh{};
    hh.n = n; hh.nk = nk; hh.ns = g.ns; hh.stride = g.stride;
    hh.algo = a.algo[k];
    hh.D = g.D;
    hh.shift = shift; hh.nb = nb; hh.occ = s_occ;
    hh.E = s_occ * g.stride;                   // spline window: the bucket occupancy bounds its error
    int S0 = 1;
    const int G = hh.algo == BL_BALLOT8 ? 8 : hh.algo == BL_BALLOT16 ? 16 : 32;
    while ((int64_t)S0 * (G + 1) < (int64_t)g.ns + 1) S0 *= (G + 1);
    hh.S0 = S0;
    hh.dir_cap = a.dir_cap[k];
    hh.off_mlp = g.off_mlp; hh.off_dir = g.off_dir; hh.off_keys = g.off_keys; hh.off_eyt = g.off_eyt;
    hh.staged_end = g.staged_end;
    hh.off_full = g.off_full;
    hh.base = base;
    hh.k0 = order_key(X[0]);
    hh.e_lo = e_lo; hh.e_scale = e_scale;
    hh.loss = 0.0f;
    hh.off_cells = g.off_cells;
    hh.ffok = 0;
    hh.gshift = s_gshift;
    hh.gnb = s_gnb;
    hh.gbase = s_gbase;
    *h = hh;
    if (s_bad) atomicOr(a.bad_flag, 1u);
  }
}

// ---------------------------------------------------------------------------
// MLP training: one block per table, full-batch Adam over a training set of
// table keys (every entry, or an evenly strided subset) and targets drawn
// uniformly in key space over the table range with SplitMix64.  Labels are
// exact counts of keys below each sample, normalised by n-1.
// ---------------------------------------------------------------------------
constexpr int kTrainThreads = 256;
constexpr int kTrainSamples = 2048;

__device__ __forceinline__ int count_keys_below(const StagedView& v, uint64_t q) { return plain_bucket(v, q); }

__global__ void __launch_bounds__(kTrainThreads) k_train_mlp(TrainArgs a) {
  const int k = blockIdx.x;
  if (k >= a.ntables) return;
  unsigned char* blob = a.blobs + a.blob_off[k];
  BlobHdr* gh = reinterpret_cast<BlobHdr*>(blob);
  const BlobHdr h = *gh;
  __shared__ float xs[kTrainSamples][2];
  __shared__ float ys[kTrainSamples];
  __shared__ float p[kMlpParams];
  __shared__ float red[kTrainThreads / 32][kMlpParams + 1];
  float* gp = reinterpret_cast<float*>(blob + h.off_mlp);
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) p[i] = gp[i];
  // global view of the blob for labelling (no staging needed: reads hit L2)
  StagedView v;
  v.h = h;
  v.dir = reinterpret_cast<const uint16_t*>(blob + h.off_dir);
  v.keys = reinterpret_cast<const uint64_t*>(blob + h.off_keys);
  v.full = h.off_full >= 0 ? reinterpret_cast<const uint64_t*>(blob + h.off_full) : nullptr;
  v.gdir = h.gnb > 0 ? reinterpret_cast<const int*>(blob + h.off_full + (int64_t)(h.nk + kPad) * 8) : nullptr;
  const MlpFeatScale sc{h.e_lo, h.e_scale};
  const uint64_t k0 = h.k0, k1 = h.stride == 1 ? v.keys[h.nk - 1] : v.full[h.nk - 1];
  const int nkeys = min(h.n, kTrainSamples / 2);
  const float inv = 1.0f / (float)max(h.nk, 1);
  for (int i = threadIdx.x; i < kTrainSamples; i += blockDim.x) {
    uint64_t q;
    if (i < nkeys) {
      // table entry j (evenly strided), nudged to just above the entry so its count includes it
      const int j = (int)(((int64_t)i * (h.n - 1)) / max(nkeys - 1, 1));
      q = (j == 0 ? k0 : (h.stride == 1 ? v.keys[j - 1] : v.full[j - 1])) + 1;
    } else {
      const uint64_t r = splitmix64(a.seed ^ ((uint64_t)k << 32) ^ (uint64_t)i);
      q = k0 + (uint64_t)((double)(r >> 11) * 0x1.0p-53 * (double)(k1 - k0));
    }
    const double t = key_to_double(q);
    float x0, x1;
    mlp_features(t, sc, x0, x1);
    xs[i][0] = x0;
    xs[i][1] = x1;
    ys[i] = (float)count_keys_below(v, q) * inv;
  }
  __syncthreads();
  // Initialisation from the data: hinge k sits at the normalised log2
  // coordinate z of the table entry at quantile k/16, and the output weights
  // make the network the piecewise-linear interpolant of the 17 quantile
  // points (slope changes at the hinges).  Adam then minimises the MSE.
  if (threadIdx.x == 0) {
    float zk[kHidden + 1], yk[kHidden + 1];
    for (int q = 0; q <= kHidden; ++q) {
      const int i = (int)(((int64_t)q * (nkeys - 1)) / kHidden);
      zk[q] = xs[i][0] + h.e_scale * xs[i][1];
      yk[q] = ys[i];
    }
    float prev = 0.0f;
    for (int q = 0; q < kHidden; ++q) {
      const float dz = zk[q + 1] - zk[q];
      const float slope = dz > 0.0f ? (yk[q + 1] - yk[q]) / dz : 0.0f;
      p[2 * q] = 1.0f;
      p[2 * q + 1] = h.e_scale;
      p[2 * kHidden + q] = -zk[q];
      p[3 * kHidden + q] = slope - prev;
      prev = slope;
    }
    p[4 * kHidden] = yk[0];
  }
  __syncthreads();
  float m1 = 0.0f, m2 = 0.0f;     // Adam moments of parameter threadIdx.x
  const float lr = a.lr, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float scale = 1.0f / (float)kTrainSamples;
  float loss = 0.0f;
  for (int step = 1; step <= a.epochs; ++step) {
    float g[kMlpParams];
#pragma unroll
    for (int i = 0; i < kMlpParams; ++i) g[i] = 0.0f;
    float l = 0.0f;
    for (int i = threadIdx.x; i < kTrainSamples; i += blockDim.x) l += mlp_backward_accum(p, xs[i][0], xs[i][1], ys[i], scale, g);
    block_reduce_params(g, l, red);
    loss = red[0][kMlpParams] * scale;
    if (threadIdx.x < kMlpParams) {
      const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
      // cosine decay of the learning rate to 5% over the run
      const float lr_t = lr * (0.05f + 0.475f * (1.0f + cospif((float)(step - 1) / (float)a.epochs)));
      float pv = p[threadIdx.x];
      adam_update(pv, red[0][threadIdx.x], m1, m2, lr_t, b1, b2, eps, c1, c2);
      p[threadIdx.x] = pv;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) gp[i] = p[i];
  if (threadIdx.x == 0) gh->loss = a.epochs > 0 ? loss : 0.0f;
}

// ---------------------------------------------------------------------------
// Learned half-window: the largest |proposal - exact count| over probes
// (every key, one unit above it, and key-space samples), plus one.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_window(WindowArgs a) {
  const int k = blockIdx.x;
  if (k >= a.ntables) return;
  unsigned char* blob = a.blobs + a.blob_off[k];
  BlobHdr* gh = reinterpret_cast<BlobHdr*>(blob);
  const BlobHdr h = *gh;
  if (h.algo != BL_SPLINE && h.algo != BL_MLP && h.algo != BL_LOGHASH) return;
  StagedView v;
  v.h = h;
  v.mlp = reinterpret_cast<const float*>(blob + h.off_mlp);
  v.dir = reinterpret_cast<const uint16_t*>(blob + h.off_dir);
  v.keys = reinterpret_cast<const uint64_t*>(blob + h.off_keys);
  v.full = h.off_full >= 0 ? reinterpret_cast<const uint64_t*>(blob + h.off_full) : nullptr;
  v.gdir = h.gnb > 0 ? reinterpret_cast<const int*>(blob + h.off_full + (int64_t)(h.nk + kPad) * 8) : nullptr;
  const MlpFeatScale sc{h.e_lo, h.e_scale};
  __shared__ int s_err;
  if (threadIdx.x == 0) s_err = 0;
  __syncthreads();
  const uint64_t k0 = h.k0, k1 = key_at(v, h.nk - 1);
  int err = 0;
  const int nprobe = 2 * h.nk + 4096;
  for (int i = threadIdx.x; i < nprobe; i += blockDim.x) {
    uint64_t q;
    if (i < 2 * h.nk) q = key_at(v, i >> 1) + (uint64_t)(i & 1);
    else q = k0 + (uint64_t)((double)(splitmix64(a.seed ^ ((uint64_t)k << 40) ^ (uint64_t)i) >> 11) * 0x1.0p-53 *
                             (double)(k1 - k0));
    const int c = plain_bucket(v, q);
    const int prop = h.algo == BL_SPLINE    ? spline_proposal(v, q)
                     : h.algo == BL_LOGHASH ? loghash_propose(v.mlp[kMlpParams], v.mlp[kMlpParams + 1], h.nk,
                                                              key_to_double(q))
                                            : mlp_propose(v.mlp, sc, h.n, key_to_double(q));
    err = max(err, abs(prop - c));
  }
  err = __reduce_max_sync(0xFFFFFFFFu, err);
  if ((threadIdx.x & 31) == 0) atomicMax(&s_err, err);
  __syncthreads();
  if (threadIdx.x == 0) gh->E = s_err + 1;
}

// ---------------------------------------------------------------------------
// Persistent batched search.  Each block takes tiles from a global counter
// (one atomicAdd per tile), stages the tile's table with a TMA bulk copy when
// it differs from the one already in shared memory, and streams the tile's
// targets.  Targets of a tile are contiguous in Y / out.
// ---------------------------------------------------------------------------
// Algorithm families compiled into one instance of the batched kernel: the
// plain searches only, plus the spline and the logarithm hash, plus the MLP.  A plan launches the
// smallest family that covers its tables, which keeps registers (and so
// resident warps) at the level the plain searches need.
enum : int { FAM_PLAIN = 0, FAM_SPLINE = 1, FAM_MLP = 2, FAM_HUNT = 3 };

constexpr uint64_t kKeyNegInf = 0x0010000000000000ull;   // image of -inf; NaNs map below it

// Streams one tile's targets through count(y, q): a scalar head up to a
// 4-target boundary, then quads two at a time (both loads issue before any
// search, and the eight searches are independent code, so their
// shared-memory round trips overlap), one last quad, and a scalar tail.
// vec: 0 scalar only, 1 quads as two 128-bit loads, 2 quads as one 256-bit
// load (Y 32-byte aligned).
template <class F>
__device__ __forceinline__ void stream_tile(const double* __restrict__ Y, int32_t* __restrict__ out, int64_t b,
                                            int cnt, int vec, uint64_t le, int& nans, F&& count) {
  const int bs = blockDim.x;
  const int head = vec ? min(cnt, (int)((-b) & 3)) : cnt;
  const int nq = (cnt - head) >> 2;
  for (int i = threadIdx.x; i < head; i += bs) {
    const double y = Y[b + i];
    const uint64_t k = order_key(y);
    nans += k < kKeyNegInf;
    out[b + i] = count(y, k + le);
  }
  const double2* Y2 = reinterpret_cast<const double2*>(Y + b + head);
  int4* O4 = reinterpret_cast<int4*>(out + b + head);
  int g = threadIdx.x;
  for (; g + bs < nq; g += 2 * bs) {
    double y[8];
    if (vec == 2) {
      double* lo = y;
      double* hi = y + 4;
      ld_stream4(reinterpret_cast<const double*>(Y2 + 2 * g), *reinterpret_cast<double(*)[4]>(lo));
      ld_stream4(reinterpret_cast<const double*>(Y2 + 2 * (g + bs)), *reinterpret_cast<double(*)[4]>(hi));
    } else {
      const double2 p0 = ld_stream(Y2 + 2 * g), p1 = ld_stream(Y2 + 2 * g + 1);
      const double2 p2 = ld_stream(Y2 + 2 * (g + bs)), p3 = ld_stream(Y2 + 2 * (g + bs) + 1);
      y[0] = p0.x; y[1] = p0.y; y[2] = p1.x; y[3] = p1.y;
      y[4] = p2.x; y[5] = p2.y; y[6] = p3.x; y[7] = p3.y;
    }
    int r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t k = order_key(y[j]);
      nans += k < kKeyNegInf;
      r[j] = count(y[j], k + le);
    }
    st_stream(O4 + g, make_int4(r[0], r[1], r[2], r[3]));
    st_stream(O4 + g + bs, make_int4(r[4], r[5], r[6], r[7]));
  }
  if (g < nq) {
    const double2 p0 = ld_stream(Y2 + 2 * g), p1 = ld_stream(Y2 + 2 * g + 1);
    const double y[4] = {p0.x, p0.y, p1.x, p1.y};
    int r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t k = order_key(y[j]);
      nans += k < kKeyNegInf;
      r[j] = count(y[j], k + le);
    }
    st_stream(O4 + g, make_int4(r[0], r[1], r[2], r[3]));
  }
  for (int i = head + 4 * nq + threadIdx.x; i < cnt; i += bs) {
    const double y = Y[b + i];
    const uint64_t k = order_key(y);
    nans += k < kKeyNegInf;
    out[b + i] = count(y, k + le);
  }
}

// stream_tile for the MLP proposal: the eight proposals of a thread's two
// quads are evaluated together (mlp_propose_w), then each is checked.
__device__ __forceinline__ void stream_tile_mlp(const StagedView& v, const double* __restrict__ Y,
                                                int32_t* __restrict__ out, int64_t b, int cnt, int vec, uint64_t le,
                                                int& nans, int& fallbacks) {
  const int bs = blockDim.x;
  const BlobHdr& h = v.h;
  const MlpFeatScale sc{h.e_lo, h.e_scale};
  auto one = [&](int64_t i) {
    const double y = Y[i];
    const uint64_t k = order_key(y);
    nans += k < kKeyNegInf;
    out[i] = mlp_count(v, y, k + le, fallbacks);
  };
  const int head = vec ? min(cnt, (int)((-b) & 3)) : cnt;
  const int nq = (cnt - head) >> 2;
  for (int i = threadIdx.x; i < head; i += bs) one(b + i);
  const double2* Y2 = reinterpret_cast<const double2*>(Y + b + head);
  int4* O4 = reinterpret_cast<int4*>(out + b + head);
  int g = threadIdx.x;
  for (; g + bs < nq; g += 2 * bs) {
    double y[8];
    if (vec == 2) {
      ld_stream4(reinterpret_cast<const double*>(Y2 + 2 * g), *reinterpret_cast<double(*)[4]>(y));
      ld_stream4(reinterpret_cast<const double*>(Y2 + 2 * (g + bs)), *reinterpret_cast<double(*)[4]>(y + 4));
    } else {
      const double2 p0 = ld_stream(Y2 + 2 * g), p1 = ld_stream(Y2 + 2 * g + 1);
      const double2 p2 = ld_stream(Y2 + 2 * (g + bs)), p3 = ld_stream(Y2 + 2 * (g + bs) + 1);
      y[0] = p0.x; y[1] = p0.y; y[2] = p1.x; y[3] = p1.y;
      y[4] = p2.x; y[5] = p2.y; y[6] = p3.x; y[7] = p3.y;
    }
    int prop[8], r[8];
    mlp_propose_w<8>(v.mlp, sc, h.n, y, prop);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t k = order_key(y[j]);
      nans += k < kKeyNegInf;
      r[j] = learned_count(v, prop[j], k + le, fallbacks);
    }
    st_stream(O4 + g, make_int4(r[0], r[1], r[2], r[3]));
    st_stream(O4 + g + bs, make_int4(r[4], r[5], r[6], r[7]));
  }
  for (; g < nq; g += bs)
    for (int j = 0; j < 4; ++j) one(b + head + 4 * (int64_t)g + j);
  for (int i = head + 4 * nq + threadIdx.x; i < cnt; i += bs) one(b + i);
}

// Hunt order (SS_MODEL_HUNT, coherent targets): a lane takes eight
// consecutive targets per step (two 256-bit loads; a warp covers 256
// consecutive targets): the first is searched with the table's own search,
// each of the other seven hunts from the first one's answer (hunt_from;
// independent of each other, so their shared-memory round trips overlap).
// Head and tail targets take the table's own search.  Every answer is exact
// whatever the guess.  (A chain in which each target hunts from the one
// before it measured slower: its dependent round trips serialise.)
__device__ __forceinline__ void stream_tile_hunt(const StagedView& v, const double* __restrict__ Y,
                                                 int32_t* __restrict__ out, int64_t b, int cnt, int vec,
                                                 uint64_t le, int& nans) {
  const int bs = blockDim.x;
  auto one = [&](int64_t i) {
    const double y = Y[i];
    const uint64_t k = order_key(y);
    nans += k < kKeyNegInf;
    out[i] = hunt_count(v, -1, k + le);
  };
  const int head = vec ? min(cnt, (int)((-b) & 3)) : cnt;
  const int np = (cnt - head) >> 3;                    // runs of eight targets (two quads)
  for (int i = threadIdx.x; i < head; i += bs) one(b + i);
  const double2* Y2 = reinterpret_cast<const double2*>(Y + b + head);
  int4* O4 = reinterpret_cast<int4*>(out + b + head);
  for (int g = threadIdx.x; g < np; g += bs) {
    double y[8];
    if (vec == 2) {
      ld_stream4(reinterpret_cast<const double*>(Y2 + 4 * g), *reinterpret_cast<double(*)[4]>(y));
      ld_stream4(reinterpret_cast<const double*>(Y2 + 4 * g + 2), *reinterpret_cast<double(*)[4]>(y + 4));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double2 p = ld_stream(Y2 + 4 * g + j);
        y[2 * j] = p.x;
        y[2 * j + 1] = p.y;
      }
    }
    int r[8];
    uint64_t q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t k = order_key(y[j]);
      nans += k < kKeyNegInf;
      q[j] = k + le;
    }
    r[0] = hunt_count(v, -1, q[0]);
#pragma unroll
    for (int j = 1; j < 8; ++j) r[j] = hunt_count(v, r[0], q[j]);
    st_stream(O4 + 2 * g, make_int4(r[0], r[1], r[2], r[3]));
    st_stream(O4 + 2 * g + 1, make_int4(r[4], r[5], r[6], r[7]));
  }
  for (int i = head + 8 * np + threadIdx.x; i < cnt; i += bs) one(b + i);
}

template <int G>
__device__ __forceinline__ void ballot_tile(const StagedView& v, const double* __restrict__ Y, int32_t* __restrict__ out,
                                            int64_t b, int cnt, uint64_t le, int& nans) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gbase = lane & ~(G - 1);
  const BlobHdr& h = v.h;
  for (int base = w * 32; base < cnt; base += nw * 32) {
    const int i = base + lane;
    const bool ok = i < cnt;
    uint64_t q = 0;
    if (ok) {
      const uint64_t k = order_key(Y[b + i]);
      nans += k < kKeyNegInf;
      q = k + le;
    }
    int r = 0;
    for (int src = 0; src < G; ++src) {
      const uint64_t qq = __shfl_sync(0xFFFFFFFFu, q, gbase + src);
      const int c = finish_full(v, search_ballot<G>(v.keys, h.ns, h.S0, qq), qq);
      if ((lane & (G - 1)) == src) r = c;
    }
    if (ok) out[b + i] = r;
  }
}

// Launched with 256 threads, or with 512 when a staged table leaves room for
// fewer than four 256-thread blocks on an SM (the bound keeps 64 registers
// per thread either way, so an SM holds 1024 threads in both shapes).
constexpr int kPlanMaxThreads = 512;
int batched_1d_max_threads() { return kPlanMaxThreads; }

template <bool LE, int FAM>
__global__ void __launch_bounds__(kPlanMaxThreads, 2) k_batched_1d(BatchArgs1D a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ int s_tile;
  __shared__ int s_err;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_err = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  int cur_table = -1;
  StagedView v{};
  bool ok = true;
  int nans = 0, fallbacks = 0;
  const uint64_t le = LE ? 1 : 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();                      // everyone has read s_tile before it is rewritten
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    if (tile.table != cur_table) {
      v = stage_blob(a.blobs + a.blob_off[tile.table], smem, &bar, phase, ok);
      cur_table = tile.table;
      if (!ok) break;
    }
    const BlobHdr& h = v.h;
    const int algo = h.algo;
    const int64_t b = tile.begin;
    const int cnt = tile.count;
    if (algo >= BL_BALLOT8 && algo <= BL_BALLOT32) {
      if (algo == BL_BALLOT8) ballot_tile<8>(v, a.Y, a.out, b, cnt, le, nans);
      else if (algo == BL_BALLOT16) ballot_tile<16>(v, a.Y, a.out, b, cnt, le, nans);
      else ballot_tile<32>(v, a.Y, a.out, b, cnt, le, nans);
      continue;
    }
    // one uniform branch per tile picks the search; inside the tile the
    // searches are branch-free straight-line code where the table allows it
    const int vec = a.vec;
    if constexpr (FAM == FAM_HUNT) {
      // the hunt reads the staged keys: only a table staged for the bucket
      // search carries them (plan creation gives hunt plans no other; a
      // table staged otherwise, e.g. from an edited plan file, is searched
      // plainly)
      if (algo == BL_BUCKET) stream_tile_hunt(v, a.Y, a.out, b, cnt, vec, le, nans);
      else if (algo == BL_BINARY)
        stream_tile(a.Y, a.out, b, cnt, vec, le, nans, [&](double, uint64_t q) { return plain_binary(v, q); });
      else if (algo == BL_BALLOT8) ballot_tile<8>(v, a.Y, a.out, b, cnt, le, nans);
      else if (algo == BL_BALLOT16) ballot_tile<16>(v, a.Y, a.out, b, cnt, le, nans);
      else if (algo == BL_BALLOT32) ballot_tile<32>(v, a.Y, a.out, b, cnt, le, nans);
      else stream_tile(a.Y, a.out, b, cnt, vec, le, nans, [&](double, uint64_t q) { return plain_bucket(v, q); });
      continue;
    }
    if (FAM >= FAM_MLP && algo == BL_MLP) {
      // staged tables: the eight proposals of a thread together; sampled
      // tables (wide windows searched in global memory) one by one
      if (h.stride == 1) stream_tile_mlp(v, a.Y, a.out, b, cnt, vec, le, nans, fallbacks);
      else stream_tile(a.Y, a.out, b, cnt, vec, le, nans, [&](double y, uint64_t q) { return mlp_count(v, y, q, fallbacks); });
    } else if (FAM >= FAM_SPLINE && algo == BL_SPLINE) {
      stream_tile(a.Y, a.out, b, cnt, vec, le, nans, [&](double, uint64_t q) { return spline_count(v, q, fallbacks); });
    } else if (FAM >= FAM_SPLINE && algo == BL_LOGHASH) {
      const float la = v.mlp[kMlpParams], lc = v.mlp[kMlpParams + 1];
      const int nk = h.nk;
      stream_tile(a.Y, a.out, b, cnt, vec, le, nans,
                  [&](double y, uint64_t q) { return learned_count(v, loghash_propose(la, lc, nk, y), q, fallbacks); });
    } else if (algo == BL_BINARY) {
      stream_tile(a.Y, a.out, b, cnt, vec, le, nans, [&](double, uint64_t q) { return plain_binary(v, q); });
    } else if (h.stride == 1 && h.occ <= 2) {
      const uint64_t* keys = v.keys;
      const uint16_t* dir = v.dir;
      const int shift = h.shift, nb = h.nb;
      const uint64_t base = h.base;
      if (h.occ <= 1)
        stream_tile(a.Y, a.out, b, cnt, vec, le, nans,
                    [&](double, uint64_t q) { return search_bucket<1>(keys, dir, shift, base, nb, q); });
      else
        stream_tile(a.Y, a.out, b, cnt, vec, le, nans,
                    [&](double, uint64_t q) { return search_bucket<2>(keys, dir, shift, base, nb, q); });
    } else {
      stream_tile(a.Y, a.out, b, cnt, vec, le, nans, [&](double, uint64_t q) { return plain_bucket(v, q); });
    }
  }
  if (!ok && threadIdx.x == 0) s_err = 1;
  __syncthreads();
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  fallbacks = __reduce_add_sync(0xFFFFFFFFu, fallbacks);
  if (a.stat != nullptr && (threadIdx.x & 31) == 0) {
    if (nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
    if (fallbacks) atomicAdd(&a.stat->fallbacks, (unsigned long long)fallbacks);
  }
  if (a.stat != nullptr && threadIdx.x == 0 && s_err) atomicOr(&a.stat->flags, SS_FLAG_STAGING_TIMEOUT);
  SS_BOUNDS_FOLD(a.stat);
}

// Persistent batched search over tables with a wide section: one block of
// 1024 threads per SM holds a whole wide section (up to 224 KB) in shared
// memory; otherwise the same tile loop as k_batched_1d.
template <bool LE>
__global__ void __launch_bounds__(kWideThreads, 1) k_batched_1d_wide(BatchArgs1D a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ int s_tile;
  __shared__ int s_err;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_err = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  int cur_table = -1;
  StagedView v{};
  bool ok = true;
  int nans = 0;
  const uint64_t le = LE ? 1 : 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    if (tile.table != cur_table) {
      v = stage_blob(a.blobs + a.blob_off[tile.table], smem, &bar, phase, ok);
      cur_table = tile.table;
      if (!ok) break;
    }
    const WideView wv = wide_view(smem + sizeof(BlobHdr), v);
    if (wv.w.occ <= 1)
      stream_tile(a.Y, a.out, tile.begin, tile.count, a.vec, le, nans,
                  [&](double, uint64_t q) { return wide_count<1>(wv, q); });
    else if (wv.w.occ <= 2)
      stream_tile(a.Y, a.out, tile.begin, tile.count, a.vec, le, nans,
                  [&](double, uint64_t q) { return wide_count<2>(wv, q); });
    else
      stream_tile(a.Y, a.out, tile.begin, tile.count, a.vec, le, nans,
                  [&](double, uint64_t q) { return wide_count<0>(wv, q); });
  }
  if (!ok && threadIdx.x == 0) s_err = 1;
  __syncthreads();
  nans = __reduce_add_sync(0xFFFFFFFFu, nans);
  if (a.stat != nullptr && (threadIdx.x & 31) == 0 && nans) atomicAdd(&a.stat->nan_targets, (unsigned long long)nans);
  if (a.stat != nullptr && threadIdx.x == 0 && s_err) atomicOr(&a.stat->flags, SS_FLAG_STAGING_TIMEOUT);
  SS_BOUNDS_FOLD(a.stat);
}

const void* batched_1d_wide_kernel(bool le) {
  return le ? reinterpret_cast<const void*>(&k_batched_1d_wide<true>)
            : reinterpret_cast<const void*>(&k_batched_1d_wide<false>);
}

// Kernel entry of the batched search (template stubs stay local to this unit).
const void* batched_1d_kernel(bool le, int family) {
  if (family == FAM_HUNT)
    return le ? reinterpret_cast<const void*>(&k_batched_1d<true, FAM_HUNT>) : reinterpret_cast<const void*>(&k_batched_1d<false, FAM_HUNT>);
  if (family >= FAM_MLP)
    return le ? reinterpret_cast<const void*>(&k_batched_1d<true, FAM_MLP>) : reinterpret_cast<const void*>(&k_batched_1d<false, FAM_MLP>);
  if (family == FAM_SPLINE)
    return le ? reinterpret_cast<const void*>(&k_batched_1d<true, FAM_SPLINE>)
              : reinterpret_cast<const void*>(&k_batched_1d<false, FAM_SPLINE>);
  return le ? reinterpret_cast<const void*>(&k_batched_1d<true, FAM_PLAIN>) : reinterpret_cast<const void*>(&k_batched_1d<false, FAM_PLAIN>);
}

}  // namespace ss
