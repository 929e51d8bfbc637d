// static_batched.cu -- a batched 1D search that allocates no device memory.
//
// Some callers are not allowed to call cudaMalloc: code that runs under a
// fixed device-memory budget handed out by a host framework (where an extra
// allocation would fail or fragment the framework's pool), latency-critical
// loops that cannot afford cudaMalloc's implicit device synchronisation, and
// plug-ins that must leave device memory management entirely to their host.
// For them this entry point keeps all of its working memory -- the prepared
// tables, the tile list and the tile counter -- in one fixed-size array that
// is part of the library image, instead of the allocations a plan makes.  The
// caller still provides the tables, targets and outputs.
//
// Costs of that choice: every GPU that loads the library holds the array
// (kStaticScratchBytes) until the process exits; the array is shared by all
// calls, so calls are ordered on the GPU -- each call's work waits for the
// previous call's (one event per device, recorded after every call), which
// keeps calls from different streams or host threads from overwriting each
// other's tables, at the price of running them one after another; and a
// batch whose prepared tables and tiles do not fit is rejected.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"
#include "plan_host.h"

namespace ss {

int default_dir_cap(int n);

constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB per GPU
constexpr int kStaticDirCap = 2048;                        // bucket budget per table here

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Per device: the array's device address (looked up once: the array's name
// is only a host-side handle), the event recorded after the last call's work,
// and a lock held while a call queues its work, so that the wait on the
// previous call and the record of this one come in the order of the calls.
struct StaticDevice {
  std::mutex mu;
  unsigned char* addr = nullptr;
  cudaEvent_t done = nullptr;
  bool used = false;
};

static ss_status static_device(StaticDevice** out) {
  static StaticDevice devs[64];
  int dev = 0;
  SS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SS_EUNSUPPORTED, "ss_search_1d_batched_static: device ordinal out of range");
  StaticDevice& d = devs[dev];
  std::lock_guard<std::mutex> lock(d.mu);
  if (d.addr == nullptr) {
    void* p = nullptr;
    SS_CHECK_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    d.addr = static_cast<unsigned char*>(p);
  }
  if (d.done == nullptr) SS_CHECK_CUDA(cudaEventCreateWithFlags(&d.done, cudaEventDisableTiming));
  *out = &d;
  return SS_OK;
}

// Byte offsets inside the array: tile counter, table-check flag, table
// offsets, blob offsets, directory budgets, algorithms, tiles, then the
// prepared tables.
struct StaticLayout {
  int64_t counter, flag, xoff, boff, caps, algo, tiles, blobs, end;
};

static StaticLayout static_layout(int ntables, size_t ntiles, int64_t blob_bytes) {
  auto up = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  StaticLayout l;
  l.counter = 0;
  l.flag = 256;
  l.xoff = 512;
  l.boff = l.xoff + up((int64_t)(ntables + 1) * 8);
  l.caps = l.boff + up((int64_t)ntables * 8);
  l.algo = l.caps + up((int64_t)ntables * 4);
  l.tiles = l.algo + up((int64_t)ntables * 4);
  l.blobs = l.tiles + up((int64_t)ntiles * (int64_t)sizeof(Tile));
  l.end = l.blobs + blob_bytes;
  return l;
}

// The work of one call, queued on `stream`: metadata into the array,
// preparation of the tables there, and the persistent search over the tiles.
static ss_status queue_static(const StaticLayout& l, unsigned char* base, int32_t ntables, const int64_t* X_off,
                              const double* X, const double* Y, int32_t* lowbounds, int32_t side, ss_devstat* stat,
                              const std::vector<int64_t>& blob_off, const std::vector<int>& caps,
                              const std::vector<int>& algo, const std::vector<Tile>& tiles, int smem,
                              cudaStream_t stream) {
  // the copies read pageable host memory, which the runtime stages before
  // returning, so the host vectors may go out of scope
  SS_CHECK_CUDA(cudaMemsetAsync(base + l.counter, 0, 512, stream));   // tile counter and table-check flag
  SS_CHECK_CUDA(cudaMemcpyAsync(base + l.xoff, X_off, (ntables + 1) * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + l.boff, blob_off.data(), ntables * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + l.caps, caps.data(), ntables * 4, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + l.algo, algo.data(), ntables * 4, cudaMemcpyHostToDevice, stream));
  if (!tiles.empty())
    SS_CHECK_CUDA(cudaMemcpyAsync(base + l.tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, stream));
  // prepare the tables into the array; an unsorted table sets SS_FLAG_NOT_SORTED
  unsigned* flag = stat != nullptr ? &stat->flags : reinterpret_cast<unsigned*>(base + l.flag);
  PrepArgs pa{ntables, reinterpret_cast<const int64_t*>(base + l.xoff), X, base + l.blobs,
              reinterpret_cast<const int64_t*>(base + l.boff), reinterpret_cast<const int*>(base + l.caps),
              reinterpret_cast<const int*>(base + l.algo), 0, flag};
  k_prep_1d<<<ntables, 256, 0, stream>>>(pa);
  SS_CHECK_CUDA(cudaGetLastError());
  if (tiles.empty()) return SS_OK;
  const void* kern = batched_1d_kernel(side == SS_SIDE_LE, 0);
  if (ss_status st_ = raise_smem_limit(kern, smem)) return st_;
  int per_sm = 0;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNumThreads, smem));
  if (per_sm < 1) return fail(SS_EUNSUPPORTED, "ss_search_1d_batched_static: kernel does not fit on an SM");
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, (int64_t)tiles.size()));
  BatchArgs1D a{base + l.blobs, reinterpret_cast<const int64_t*>(base + l.boff),
                reinterpret_cast<const Tile*>(base + l.tiles), (int)tiles.size(),
                reinterpret_cast<int*>(base + l.counter), Y, lowbounds,
                (aligned(Y, 16) && aligned(lowbounds, 16)) ? 1 : 0, stat};
  void* args[1] = {&a};
  SS_CHECK_CUDA(cudaLaunchKernel(kern, dim3(grid), dim3(kNumThreads), args, (size_t)smem, stream));
  return SS_OK;
}

}  // namespace ss

using namespace ss;

extern "C" ss_status ss_search_1d_batched_static(int32_t ntables, const int64_t* X_off, const double* X,
                                                 const int64_t* Y_off, const double* Y, int32_t* lowbounds,
                                                 int32_t side, ss_devstat* stat, cudaStream_t stream) {
  const char* me = "ss_search_1d_batched_static";
  if (X_off == nullptr || Y_off == nullptr || X == nullptr) return fail(SS_EINVAL, std::string(me) + ": null pointer");
  if (ntables < 1) return fail(SS_EINVAL, std::string(me) + ": ntables must be >= 1");
  if (side != SS_SIDE_LT && side != SS_SIDE_LE) return fail(SS_EINVAL, std::string(me) + ": bad side");
  if (Y_off[ntables] > 0 && (Y == nullptr || lowbounds == nullptr)) return fail(SS_EINVAL, std::string(me) + ": null pointer");
  if (!aligned(X, 8) || !aligned(Y, 8) || !aligned(lowbounds, 4)) return fail(SS_EINVAL, std::string(me) + ": misaligned pointer");
  // host-side layout of the array
  std::vector<int> caps(ntables), algo(ntables, BL_BUCKET), bucket_of(ntables, 0);
  std::vector<int64_t> blob_off(ntables);
  int64_t blobs = 0;
  int smem = 0;
  for (int k = 0; k < ntables; ++k) {
    const std::string tab = std::string(me) + ": table " + std::to_string(k);
    if (X_off[k] < 0) return fail(SS_EINVAL, tab + ": negative table offset X_off[k] = " + std::to_string(X_off[k]));
    const int64_t n = X_off[k + 1] - X_off[k];
    if (n < 0)
      return fail(SS_EINVAL, tab + ": table offsets decrease (X_off[k+1] - X_off[k] = " + std::to_string(n) + ")");
    if (n < 2) return fail(SS_EINVAL, tab + " has " + std::to_string(n) + " entries; every table needs >= 2");
    if (n > (1 << 30)) return fail(SS_EINVAL, tab + " has " + std::to_string(n) + " entries, more than 2^30");
    if (Y_off[k] < 0) return fail(SS_EINVAL, tab + ": negative target offset Y_off[k] = " + std::to_string(Y_off[k]));
    if (Y_off[k + 1] < Y_off[k])
      return fail(SS_EINVAL, tab + ": target offsets decrease (Y_off[k+1] - Y_off[k] = " +
                                 std::to_string(Y_off[k + 1] - Y_off[k]) + ")");
    caps[k] = std::min(default_dir_cap((int)n), kStaticDirCap);
    blob_off[k] = blobs;
    blobs += (blob_geom_dev((int)n, caps[k], false).bytes + 255) & ~(int64_t)255;
    smem = std::max(smem, staged_bytes((int)n, caps[k], false, BL_BUCKET));
  }
  int tile_size[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) tile_size[b] = kDefaultTile;
  int64_t total = 0;
  const std::vector<Tile> tiles = make_tiles(std::vector<int64_t>(Y_off, Y_off + ntables + 1), bucket_of, tile_size, total);
  const StaticLayout l = static_layout(ntables, tiles.size(), blobs);
  if (l.end > (int64_t)kStaticScratchBytes)
    return fail(SS_EINVAL, std::string(me) + ": the batch needs " + std::to_string(l.end) +
                               " bytes of working memory, more than the fixed " +
                               std::to_string(kStaticScratchBytes) + " bytes of this entry point");
  if (tiles.size() > (size_t)0x7FFFFFFF) return fail(SS_EUNSUPPORTED, std::string(me) + ": too many tiles");
  smem = (smem + 127) & ~127;
  if (smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, std::string(me) + ": a table is too large for shared memory");
  // the metadata goes to the array by copies from pageable host memory, which
  // a stream being captured into a graph cannot take: such a call is refused
  // before anything is queued (the checks above are host-only), so the caller's capture stays valid
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SS_CHECK_CUDA(cudaStreamIsCapturing(stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(SS_EUNSUPPORTED, std::string(me) + ": the stream is capturing; this entry point copies its "
                                               "metadata from pageable host memory and cannot be captured");
  StaticDevice* d = nullptr;
  if (ss_status st = static_device(&d)) return st;
  std::lock_guard<std::mutex> lock(d->mu);
  // order this call after the previous one on the GPU; the event is
  // recorded after whatever this call queued, on its error paths too
  if (d->used) SS_CHECK_CUDA(cudaStreamWaitEvent(stream, d->done, 0));
  const ss_status st = queue_static(l, d->addr, ntables, X_off, X, Y, lowbounds, side, stat, blob_off, caps, algo,
                                    tiles, smem, stream);
  const cudaError_t e = cudaEventRecord(d->done, stream);
  if (e != cudaSuccess) return st != SS_OK ? st : cuda_fail(e, "cudaEventRecord");
  d->used = true;
  return st;
}
