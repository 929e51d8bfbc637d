// plan.cu -- host side of plans: set-up once per set of tables (Sec. 5.3:
// EOSPAC loads its tables once, so search set-up is paid once), binding of a
// target batch to a tile queue captured in a CUDA graph, the autotuner, and
// plan save/load.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "plan.h"
#include "plan_host.h"

namespace ss {

int default_dir_cap(int n);

int size_bucket(int n) {
  int l = 0;
  while ((1 << (l + 1)) <= n) ++l;           // floor(log2 n)
  return std::min(kNumBuckets - 1, std::max(0, (l - 2) / 2));
}

const char* algo_name(int a) {
  static const char* names[BL_NUM] = {"bucket", "binary", "ballot8", "ballot16", "ballot32", "spline", "mlp",
                                              "loghash", "wide"};
  return a >= 0 && a < BL_NUM ? names[a] : "?";
}

int algo_from_name(const std::string& s) {
  for (int a = 0; a < BL_NUM; ++a)
    if (s == algo_name(a)) return a;
  return -1;
}

// Shared-memory bytes a table needs when staged for `algo`.
int staged_bytes(int n, int dir_cap, bool cells, int algo) {
  const BlobGeom g = blob_geom_dev(n, dir_cap, cells);
  BlobHdr h{};
  h.n = n; h.nk = n - 1; h.ns = g.ns; h.D = g.D; h.algo = algo;
  h.off_mlp = g.off_mlp; h.off_dir = g.off_dir; h.off_keys = g.off_keys; h.off_eyt = g.off_eyt;
  h.off_cells = g.off_cells; h.staged_end = g.staged_end;
  int lo, hi;
  staged_range(h, lo, hi);
  return (int)sizeof(BlobHdr) + (hi - lo);
}

void free_dev(void* p) {
  if (p != nullptr) cudaFree(p);
}

PlanBase::~PlanBase() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  free_dev(d_blobs);
  free_dev(d_blob_off);
  free_dev(d_tiles);
  free_dev(d_counter);
  free_dev(d_grid);
  free_dev(d_grid64);
  free_dev(d_grid_off);
  free_dev(d_cell_off);
  if (cap_stream) cudaStreamDestroy(cap_stream);
}

// Upload a host vector into a fresh device allocation.
template <class T>
static ss_status upload(const std::vector<T>& v, T** d) {
  *d = nullptr;
  if (v.empty()) return SS_OK;
  if (cudaMalloc(reinterpret_cast<void**>(d), v.size() * sizeof(T)) != cudaSuccess)
    return fail(SS_ENOMEM, "plan: device allocation failed");
  SS_CHECK_CUDA(cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SS_OK;
}

// Tiles of a target batch: each table's targets split into runs of the
// table's bucket tile size; the queue lists large tables first so that the
// last tiles taken are small (shorter tail).
std::vector<Tile> make_tiles(const std::vector<int64_t>& Y_off, const std::vector<int>& bucket_of,
                             const int* bucket_tile, int64_t& total) {
  std::vector<Tile> tiles;
  const int nt = (int)Y_off.size() - 1;
  std::vector<int> order(nt);
  for (int k = 0; k < nt; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (Y_off[a + 1] - Y_off[a]) > (Y_off[b + 1] - Y_off[b]);
  });
  total = 0;
  for (int k : order) {
    const int64_t cnt = Y_off[k + 1] - Y_off[k];
    const int ts = std::max(64, bucket_tile[bucket_of[k]]);
    for (int64_t s = 0; s < cnt; s += ts) tiles.push_back(Tile{k, (int)std::min<int64_t>(ts, cnt - s), Y_off[k] + s});
    total += cnt;
  }
  return tiles;
}

// Automatic tile size: about six tiles per resident block for balance, and
// at least 16x the staged table bytes in target traffic so that staging a
// table costs under ~6% of streaming its tile; scaled by the tuned multiple.
int auto_tile(int64_t total, int blocks, int staged_bytes, float mult) {
  int64_t t = total / std::max<int64_t>(1, (int64_t)blocks * 6);
  // at least 8192 targets per tile, so that a tile's queue step and staging
  // stay small against its stream; a small batch (under about 5M targets)
  // takes smaller tiles so that every block still gets one
  t = std::max<int64_t>(t, std::min<int64_t>(8192, std::max<int64_t>(1024, total / std::max(1, blocks))));
  t = std::max<int64_t>(t, (int64_t)staged_bytes * 16 / 12);
  t = std::min<int64_t>(t, 1 << 20);
  t = (int64_t)((double)t * mult);
  t = std::max<int64_t>(1024, std::min<int64_t>(t, 1 << 22));
  return (int)(t & ~(int64_t)255);
}

}  // namespace ss

using namespace ss;

// ---------------------------------------------------------------------------
// Options
// ---------------------------------------------------------------------------
extern "C" void ss_plan_opts_default(ss_plan_opts* o) {
  if (o == nullptr) return;
  std::memset(o, 0, sizeof(*o));
  o->side = SS_SIDE_LT;
  o->algo = SS_ALGO_AUTO;
  o->model = SS_MODEL_NONE;
  o->autotune = 0;
  o->tile = 0;
  o->mlp_epochs = 400;
  o->mlp_lr = 2e-3f;
  o->dir_cap = 0;
  o->seed = 0x5EEDull;
  o->tune_cache = nullptr;
}

// Options of a 1D (kind 1) or 2D (kind 2) plan: at creation and again when a
// plan is read from a file.
ss_status ss::check_plan_opts(const ss_plan_opts& o, int kind) {
  if (o.tile < 0 || o.mlp_epochs < 0 || o.dir_cap < 0) return fail(SS_EINVAL, "plan: negative option");
  if (o.dir_cap > SS_MAX_DIR_CAP) return fail(SS_EINVAL, "plan: dir_cap above SS_MAX_DIR_CAP");
  if (!(o.mlp_lr >= 0.0f && o.mlp_lr < 1e30f)) return fail(SS_EINVAL, "plan: mlp_lr must be finite and >= 0");
  if (kind == 1) {
    if (o.side != SS_SIDE_LT && o.side != SS_SIDE_LE) return fail(SS_EINVAL, "plan: bad side");
    if (o.model < SS_MODEL_NONE || o.model > SS_MODEL_AUTO) return fail(SS_EINVAL, "plan: bad model");
    // the hunt reads the staged keys, which a 1D table staged for the
    // breadth-first binary search or the ballot search does not carry
    if (o.model == SS_MODEL_HUNT && o.algo != SS_ALGO_AUTO && o.algo != SS_ALGO_BUCKET)
      return fail(SS_EINVAL, "plan: a 1D hunt plan starts its runs with the bucket search (algo auto or bucket)");
    if (o.algo < SS_ALGO_AUTO || o.algo > SS_ALGO_BALLOT)
      return fail(SS_EINVAL, "plan: algo must be auto, binary, bucket or ballot");
    return SS_OK;
  }
  if (o.side != SS_SIDE_LT) return fail(SS_EINVAL, "ss_plan_create_2d: the 2D lookup uses side SS_SIDE_LT");
  if (o.model == SS_MODEL_AUTO) return fail(SS_EINVAL, "ss_plan_create_2d: SS_MODEL_AUTO is for 1D plans");
  if ((o.extrap != 0 && o.extrap != 1) || (o.logspace != 0 && o.logspace != 1))
    return fail(SS_EINVAL, "ss_plan_create_2d: extrap and logspace must be 0 or 1");
  if (o.model < SS_MODEL_NONE || o.model > SS_MODEL_HUNT || o.algo == SS_ALGO_BALLOT || o.algo == SS_ALGO_BRANCHY ||
      o.algo < 0 || o.algo > SS_ALGO_BALLOT)
    return fail(SS_EINVAL, "ss_plan_create_2d: algo must be auto, binary or bucket");
  return SS_OK;
}

// Default per-table algorithm before tuning.
int ss::initial_algo(const ss_plan_opts& o) {
  if (o.model == SS_MODEL_SPLINE) return BL_SPLINE;
  if (o.model == SS_MODEL_MLP) return BL_MLP;
  if (o.model == SS_MODEL_LOGHASH) return BL_LOGHASH;
  if (o.algo == SS_ALGO_BINARY) return BL_BINARY;
  if (o.algo == SS_ALGO_BALLOT) return BL_BALLOT32;
  return BL_BUCKET;
}

// ---------------------------------------------------------------------------
// 1D plans
// ---------------------------------------------------------------------------
extern "C" ss_status ss_plan_create_1d(ss_plan** out, int32_t ntables, const int64_t* X_off, const double* X,
                                       const ss_plan_opts* opts_in, cudaStream_t stream) {
  if (out == nullptr || X_off == nullptr || X == nullptr) return fail(SS_EINVAL, "ss_plan_create_1d: null pointer");
  *out = nullptr;
  if (ntables < 1) return fail(SS_EINVAL, "ss_plan_create_1d: ntables must be >= 1");
  if (!aligned(X, 8)) return fail(SS_EINVAL, "ss_plan_create_1d: misaligned table pointer");
  ss_plan_opts o;
  ss_plan_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (ss_status st = check_plan_opts(o, 1)) return st;
  auto* p = new ss_plan();
  p->kind = 1;
  p->ntables = ntables;
  p->opts = o;
  p->sizes.resize(ntables);
  p->X_off.assign(X_off, X_off + ntables + 1);
  for (int k = 0; k < ntables; ++k) {
    const int64_t n = X_off[k + 1] - X_off[k];
    if (n < 2 || n > (1 << 30) || X_off[k] < 0) {
      delete p;
      return fail(SS_EINVAL, "ss_plan_create_1d: every table needs 2 <= n entries and non-negative offsets");
    }
    p->sizes[k] = (int)n;
  }
  ss_status st = plan_build_1d(p, X, stream);
  if (st != SS_OK) {
    delete p;
    return st;
  }
  *out = p;
  return SS_OK;
}

extern "C" ss_status ss_plan_bind_1d(ss_plan* p, const int64_t* Y_off, const double* Y, int32_t* lowbounds,
                                     ss_devstat* stat, cudaStream_t stream) {
  if (p == nullptr || Y_off == nullptr) return fail(SS_EINVAL, "ss_plan_bind_1d: null pointer");
  if (p->kind != 1) return fail(SS_EINVAL, "ss_plan_bind_1d: not a 1D plan");
  if (Y_off[p->ntables] > 0 && (Y == nullptr || lowbounds == nullptr)) return fail(SS_EINVAL, "ss_plan_bind_1d: null pointer");
  if (!aligned(Y, 8) || !aligned(lowbounds, 4)) return fail(SS_EINVAL, "ss_plan_bind_1d: misaligned pointer");
  for (int k = 0; k < p->ntables; ++k)
    if (Y_off[k + 1] < Y_off[k] || Y_off[k] < 0) return fail(SS_EINVAL, "ss_plan_bind_1d: offsets must be non-decreasing");
  return plan_bind(p, std::vector<int64_t>(Y_off, Y_off + p->ntables + 1), Y, lowbounds, nullptr, stat, stream);
}

extern "C" ss_status ss_plan_execute(ss_plan* p, cudaStream_t stream) {
  if (p == nullptr) return fail(SS_EINVAL, "ss_plan_execute: null plan");
  if (!p->bound) return fail(SS_EINVAL, "ss_plan_execute: bind targets first");
  if (p->ntiles == 0) return SS_OK;
  SS_CHECK_CUDA(cudaGraphLaunch(p->exec, stream));
  return SS_OK;
}

extern "C" ss_status ss_plan_info_get(const ss_plan* p, ss_plan_info* out) {
  if (p == nullptr || out == nullptr) return fail(SS_EINVAL, "ss_plan_info_get: null pointer");
  std::memset(out, 0, sizeof(*out));
  out->kind = p->kind;
  out->ntables = p->ntables;
  out->device_bytes = p->device_bytes;
  out->max_window = p->max_window;
  out->mean_window = p->mean_window;
  out->train_loss = p->train_loss;
  out->nbuckets = kNumBuckets;
  for (int b = 0; b < kNumBuckets; ++b) {
    out->bucket_algo[b] = p->bucket_algo[b];
    out->bucket_tile[b] = p->bucket_tile[b];
    out->bucket_tables[b] = p->bucket_tables[b];
  }
  out->ntiles = p->ntiles;
  out->tuned = p->tuned;
  out->kernels = p->kernels;
  out->block_threads = p->threads;
  out->smem_bytes = p->smem_bytes;
  out->max_occupancy = p->max_occupancy;
  out->lean_kernel = p->lean != 0 ? 1 : 0;
  return SS_OK;
}

extern "C" void ss_plan_destroy(ss_plan* p) { delete p; }
