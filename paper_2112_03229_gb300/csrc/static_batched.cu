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
// calls, so two calls whose work overlaps on the GPU (different streams, or
// different host threads) overwrite each other's tables -- serialise them;
// and a batch whose prepared tables and tiles do not fit is rejected.
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

// Device address of the array for the current device, looked up once per
// device (the array's name is only a host-side handle, not a device address).
static ss_status static_scratch(unsigned char** out) {
  static std::mutex mu;
  static void* addr[256] = {nullptr};
  int dev = 0;
  SS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(SS_EUNSUPPORTED, "ss_search_1d_batched_static: device ordinal out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    SS_CHECK_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(addr[dev]);
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
  // host-side layout of the scratch array
  std::vector<int> sizes(ntables), caps(ntables), algo(ntables, BL_BUCKET), bucket_of(ntables);
  std::vector<int64_t> blob_off(ntables);
  int64_t blobs = 0;
  int smem = 0;
  for (int k = 0; k < ntables; ++k) {
    const int64_t n = X_off[k + 1] - X_off[k];
    if (n < 2 || n > (1 << 30) || X_off[k] < 0) return fail(SS_EINVAL, std::string(me) + ": every table needs >= 2 entries");
    if (Y_off[k + 1] < Y_off[k] || Y_off[k] < 0) return fail(SS_EINVAL, std::string(me) + ": target offsets must be non-decreasing");
    sizes[k] = (int)n;
    caps[k] = std::min(default_dir_cap((int)n), kStaticDirCap);
    bucket_of[k] = 0;
    blob_off[k] = blobs;
    blobs += (blob_geom_dev((int)n, caps[k], false).bytes + 255) & ~(int64_t)255;
    smem = std::max(smem, staged_bytes((int)n, caps[k], false, BL_BUCKET));
  }
  int tile_size[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) tile_size[b] = kDefaultTile;
  int64_t total = 0;
  const std::vector<Tile> tiles = make_tiles(std::vector<int64_t>(Y_off, Y_off + ntables + 1), bucket_of, tile_size, total);
  auto up = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  const int64_t o_counter = 0;
  const int64_t o_flag = 256;
  const int64_t o_xoff = 512;
  const int64_t o_boff = o_xoff + up((ntables + 1) * 8);
  const int64_t o_caps = o_boff + up(ntables * 8);
  const int64_t o_algo = o_caps + up(ntables * 4);
  const int64_t o_tiles = o_algo + up(ntables * 4);
  const int64_t o_blobs = o_tiles + up((int64_t)tiles.size() * (int64_t)sizeof(Tile));
  const int64_t need = o_blobs + blobs;
  if (need > (int64_t)kStaticScratchBytes)
    return fail(SS_EINVAL, std::string(me) + ": the batch needs " + std::to_string(need) +
                               " bytes of working memory, more than the fixed " +
                               std::to_string(kStaticScratchBytes) + " bytes of this entry point");
  if (tiles.size() > (size_t)0x7FFFFFFF) return fail(SS_EUNSUPPORTED, std::string(me) + ": too many tiles");
  smem = (smem + 127) & ~127;
  if (smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, std::string(me) + ": a table is too large for shared memory");
  unsigned char* base = nullptr;
  if (ss_status st = static_scratch(&base)) return st;
  // metadata in; the copies read pageable host memory, which the runtime
  // stages before returning, so the host vectors may go out of scope
  SS_CHECK_CUDA(cudaMemsetAsync(base + o_counter, 0, 512, stream));   // tile counter and table-check flag
  SS_CHECK_CUDA(cudaMemcpyAsync(base + o_xoff, X_off, (ntables + 1) * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + o_boff, blob_off.data(), ntables * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + o_caps, caps.data(), ntables * 4, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + o_algo, algo.data(), ntables * 4, cudaMemcpyHostToDevice, stream));
  if (!tiles.empty())
    SS_CHECK_CUDA(cudaMemcpyAsync(base + o_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, stream));
  // prepare the tables into the array; an unsorted table sets SS_FLAG_NOT_SORTED
  unsigned* flag = stat != nullptr ? &stat->flags : reinterpret_cast<unsigned*>(base + o_flag);
  PrepArgs pa{ntables, reinterpret_cast<const int64_t*>(base + o_xoff), X, base + o_blobs,
              reinterpret_cast<const int64_t*>(base + o_boff), reinterpret_cast<const int*>(base + o_caps),
              reinterpret_cast<const int*>(base + o_algo), 0, flag};
  k_prep_1d<<<ntables, 256, 0, stream>>>(pa);
  SS_CHECK_CUDA(cudaGetLastError());
  if (tiles.empty()) return SS_OK;
  const void* kern = batched_1d_kernel(side == SS_SIDE_LE, 0);
  SS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNumThreads, smem));
  if (per_sm < 1) return fail(SS_EUNSUPPORTED, std::string(me) + ": kernel does not fit on an SM");
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, (int64_t)tiles.size()));
  BatchArgs1D a{base + o_blobs, reinterpret_cast<const int64_t*>(base + o_boff),
                reinterpret_cast<const Tile*>(base + o_tiles), (int)tiles.size(),
                reinterpret_cast<int*>(base + o_counter), Y, lowbounds,
                (aligned(Y, 16) && aligned(lowbounds, 16)) ? 1 : 0, stat};
  void* args[1] = {&a};
  SS_CHECK_CUDA(cudaLaunchKernel(kern, dim3(grid), dim3(kNumThreads), args, (size_t)smem, stream));
  return SS_OK;
}
