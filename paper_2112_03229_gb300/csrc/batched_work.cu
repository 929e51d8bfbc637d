// batched_work.cu -- a batched 1D search whose working memory (prepared
// tables, tile list, tile counter) lives in one device buffer the caller of
// these helpers provides: the fixed array of the no-allocation entry point,
// or a stream-ordered allocation of the one-shot batched search.  The host
// computes the layout and the tiles from the offsets alone (no table is read
// on the host), so everything after the argument checks is queued on the
// stream: metadata copies, table preparation, the persistent search.
#include <algorithm>
#include <string>
#include <vector>

#include "plan.h"
#include "plan_host.h"

namespace ss {

int default_dir_cap(int n);

ss_status batch_work_1d(const char* me, int32_t ntables, const int64_t* X_off, const int64_t* Y_off,
                        int dir_cap_max, BatchWork1D& w) {
  w.caps.assign(ntables, 0);
  w.algo.assign(ntables, BL_BUCKET);
  w.blob_off.assign(ntables, 0);
  std::vector<int> bucket_of(ntables, 0);
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
    w.caps[k] = std::min(default_dir_cap((int)n), dir_cap_max);
    w.blob_off[k] = blobs;
    blobs += (blob_geom_dev((int)n, w.caps[k], false).bytes + 255) & ~(int64_t)255;
    smem = std::max(smem, staged_bytes((int)n, w.caps[k], false, BL_BUCKET));
  }
  int tile_size[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) tile_size[b] = kDefaultTile;
  int64_t total = 0;
  w.tiles = make_tiles(std::vector<int64_t>(Y_off, Y_off + ntables + 1), bucket_of, tile_size, total);
  if (w.tiles.size() > (size_t)0x7FFFFFFF) return fail(SS_EUNSUPPORTED, std::string(me) + ": too many tiles");
  auto up = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  w.counter = 0;
  w.flag = 256;
  w.xoff = 512;
  w.boff = w.xoff + up((int64_t)(ntables + 1) * 8);
  w.caps_off = w.boff + up((int64_t)ntables * 8);
  w.algo_off = w.caps_off + up((int64_t)ntables * 4);
  w.tiles_off = w.algo_off + up((int64_t)ntables * 4);
  w.blobs_off = w.tiles_off + up((int64_t)w.tiles.size() * (int64_t)sizeof(Tile));
  w.end = w.blobs_off + blobs;
  w.smem = (smem + 127) & ~127;
  if (w.smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, std::string(me) + ": a table is too large for shared memory");
  return SS_OK;
}

ss_status queue_work_1d(const BatchWork1D& w, unsigned char* base, int32_t ntables, const int64_t* X_off,
                        const double* X, const double* Y, int32_t* lowbounds, int32_t side, ss_devstat* stat,
                        cudaStream_t stream) {
  // the copies read pageable host memory, which the runtime stages before
  // returning, so the host vectors may go out of scope
  SS_CHECK_CUDA(cudaMemsetAsync(base + w.counter, 0, 512, stream));   // tile counter and table-check flag
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.xoff, X_off, (ntables + 1) * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.boff, w.blob_off.data(), ntables * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.caps_off, w.caps.data(), ntables * 4, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.algo_off, w.algo.data(), ntables * 4, cudaMemcpyHostToDevice, stream));
  if (!w.tiles.empty())
    SS_CHECK_CUDA(cudaMemcpyAsync(base + w.tiles_off, w.tiles.data(), w.tiles.size() * sizeof(Tile),
                                  cudaMemcpyHostToDevice, stream));
  // prepare the tables into the buffer; an unsorted table sets SS_FLAG_NOT_SORTED
  unsigned* flag = stat != nullptr ? &stat->flags : reinterpret_cast<unsigned*>(base + w.flag);
  PrepArgs pa{ntables, reinterpret_cast<const int64_t*>(base + w.xoff), X, base + w.blobs_off,
              reinterpret_cast<const int64_t*>(base + w.boff), reinterpret_cast<const int*>(base + w.caps_off),
              reinterpret_cast<const int*>(base + w.algo_off), 0, flag};
  k_prep_1d<<<ntables, 256, 0, stream>>>(pa);
  SS_CHECK_CUDA(cudaGetLastError());
  if (w.tiles.empty()) return SS_OK;
  const void* kern = batched_1d_kernel(side == SS_SIDE_LE, 0);
  if (ss_status st_ = raise_smem_limit(kern, w.smem)) return st_;
  int per_sm = 0;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNumThreads, w.smem));
  if (per_sm < 1) return fail(SS_EUNSUPPORTED, "batched search: kernel does not fit on an SM");
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, (int64_t)w.tiles.size()));
  BatchArgs1D a{base + w.blobs_off, reinterpret_cast<const int64_t*>(base + w.boff),
                reinterpret_cast<const Tile*>(base + w.tiles_off), (int)w.tiles.size(),
                reinterpret_cast<int*>(base + w.counter), Y, lowbounds,
                (aligned(Y, 16) && aligned(lowbounds, 16)) ? 1 : 0, stat};
  void* args[1] = {&a};
  SS_CHECK_CUDA(cudaLaunchKernel(kern, dim3(grid), dim3(kNumThreads), args, (size_t)w.smem, stream));
  return SS_OK;
}

}  // namespace ss
