// batched_work_2d.cu -- the batched 2D lookup (Sec. 1 and 2.2: EOSPAC bounds
// density/temperature pairs in many SESAME tables and interpolates) as one
// call queued on the caller's stream.
//
// The host lays the batch out from the offsets alone (no table is read on
// the host): prepared axes (bucket directories of the default budget),
// per-table corner records and the tile list share one buffer from the
// stream-ordered allocator.  On the stream follow: the metadata copies, the
// preparation of every axis and its cell data, the corner records, the
// eligibility check of the lean kernel, a one-thread kernel that hands the
// tile queue to the lean or to the general persistent kernel, both
// persistent launches (the one without tiles returns at its first queue
// step), and the release of the buffer.  Nothing waits on the host.
//
// The general kernel receives the caller's fp64 grids for the pairs whose
// corner values are outside the float-float range, so the one launch
// covers every table.
#include <algorithm>
#include <string>
#include <vector>

#include "plan.h"
#include "plan_host.h"

namespace ss {

int default_dir_cap(int n);

// Hands every tile to the lean kernel (counter 0) when no axis or grid
// value needs the general one, else to the general kernel (counter 1): the
// other kernel's counter starts at the tile count, so its blocks find the
// queue empty.
__global__ void k_pick_2d(const unsigned* gate, int* counters, int ntiles) {
  const bool lean = *gate == 0;
  counters[0] = lean ? 0 : ntiles;
  counters[1] = lean ? ntiles : 0;
}

ss_status batch_work_2d(const char* me, int32_t ntables, const int64_t* R_off, const int64_t* T_off,
                        const int64_t* F_off, const int64_t* Y_off, BatchWork2D& w) {
  const int nt = ntables;
  w.caps_r.assign(nt, 0);
  w.caps_t.assign(nt, 0);
  w.algo.assign(nt, BL_BUCKET);
  w.blob_off.assign(2 * nt, 0);
  w.off_r.assign(nt, 0);
  w.off_t.assign(nt, 0);
  w.cell_off.assign(nt + 1, 0);
  std::vector<int> bucket_of(nt, 0);
  int64_t blobs = 0;
  int smem = 0;
  for (int k = 0; k < nt; ++k) {
    const std::string tab = std::string(me) + ": table " + std::to_string(k);
    for (const int64_t* o : {R_off, T_off, F_off, Y_off})
      if (o[k] < 0) return fail(SS_EINVAL, tab + ": negative offset " + std::to_string(o[k]));
    const int64_t nr = R_off[k + 1] - R_off[k], ntt = T_off[k + 1] - T_off[k];
    if (nr < 2 || ntt < 2)
      return fail(SS_EINVAL, tab + " has axes of " + std::to_string(nr) + " and " + std::to_string(ntt) +
                                 " entries; each axis needs >= 2");
    if (nr > SS_MAX_AXIS_2D || ntt > SS_MAX_AXIS_2D)
      return fail(SS_EUNSUPPORTED, tab + ": an axis is longer than " + std::to_string(SS_MAX_AXIS_2D) + " entries");
    if (F_off[k + 1] - F_off[k] != nr * ntt)
      return fail(SS_EINVAL, tab + ": F_off[k+1] - F_off[k] = " + std::to_string(F_off[k + 1] - F_off[k]) +
                                 ", the grid needs nr * nt = " + std::to_string(nr * ntt) + " values");
    if (Y_off[k + 1] < Y_off[k])
      return fail(SS_EINVAL, tab + ": target offsets decrease (Y_off[k+1] - Y_off[k] = " +
                                 std::to_string(Y_off[k + 1] - Y_off[k]) + ")");
    w.caps_r[k] = default_dir_cap((int)nr);
    w.caps_t[k] = default_dir_cap((int)ntt);
    w.off_r[k] = w.blob_off[2 * k] = blobs;
    blobs += (blob_geom_dev((int)nr, w.caps_r[k], true).bytes + 255) & ~(int64_t)255;
    w.off_t[k] = w.blob_off[2 * k + 1] = blobs;
    blobs += (blob_geom_dev((int)ntt, w.caps_t[k], true).bytes + 255) & ~(int64_t)255;
    const int a = (staged_bytes((int)nr, w.caps_r[k], true, BL_BUCKET) + 127) & ~127;
    smem = std::max(smem, a + staged_bytes((int)ntt, w.caps_t[k], true, BL_BUCKET));
    w.cell_off[k + 1] = w.cell_off[k] + (nr - 1) * (ntt - 1);
    bucket_of[k] = size_bucket((int)std::max(nr, ntt));
  }
  w.smem = (smem + 127) & ~127;
  if (w.smem > max_smem_optin()) return fail(SS_EUNSUPPORTED, std::string(me) + ": axes too large for shared memory");
  // tiles as a plan without tuning takes them, capped for the corner records in flight
  int per_sm = 0;
  if (ss_status st_ = raise_smem_limit(batched_2d_fast_kernel(BL_BUCKET), w.smem)) return st_;
  SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_2d_fast_kernel(BL_BUCKET), kNumThreads, w.smem));
  const int resident = std::max(1, num_sms() * per_sm);
  const int64_t total = Y_off[nt] - Y_off[0];
  int dev = 0, l2 = 0;
  SS_CHECK_CUDA(cudaGetDevice(&dev));
  SS_CHECK_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
  int tile = auto_tile(total, resident, w.smem, 1.0f);
  if (const int c = tile_cap_2d((double)total, 32.0 * (double)w.cell_off[nt], resident, l2)) tile = std::min(tile, c);
  int tile_size[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) tile_size[b] = tile;
  int64_t counted = 0;
  w.tiles = make_tiles(std::vector<int64_t>(Y_off, Y_off + nt + 1), bucket_of, tile_size, counted);
  if (w.tiles.size() > (size_t)0x7FFFFFFF) return fail(SS_EUNSUPPORTED, std::string(me) + ": too many tiles");
  auto up = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  w.counters = 0;
  w.gate = 256;
  w.flag = 384;
  w.xr = 512;
  w.xt = w.xr + up((int64_t)(nt + 1) * 8);
  w.fo = w.xt + up((int64_t)(nt + 1) * 8);
  w.bo = w.fo + up((int64_t)(nt + 1) * 8);
  w.ro = w.bo + up((int64_t)2 * nt * 8);
  w.to = w.ro + up((int64_t)nt * 8);
  w.cr = w.to + up((int64_t)nt * 8);
  w.ct = w.cr + up((int64_t)nt * 4);
  w.al = w.ct + up((int64_t)nt * 4);
  w.co = w.al + up((int64_t)nt * 4);
  w.tiles_off = w.co + up((int64_t)(nt + 1) * 8);
  w.blobs_off = w.tiles_off + up((int64_t)w.tiles.size() * (int64_t)sizeof(Tile));
  w.cells_off = w.blobs_off + up(blobs);
  w.end = w.cells_off + std::max<int64_t>(w.cell_off[nt], 1) * 32;
  return SS_OK;
}

ss_status queue_work_2d(const BatchWork2D& w, unsigned char* base, int32_t ntables, const int64_t* R_off,
                        const double* R, const int64_t* T_off, const double* T, const int64_t* F_off, const double* F,
                        const double* Y2, int32_t* lowbounds2, double* values, ss_devstat* stat, cudaStream_t stream) {
  const int nt = ntables;
  // counters, gate and flag are cleared; the copies read pageable host
  // memory, which the runtime stages before returning
  SS_CHECK_CUDA(cudaMemsetAsync(base, 0, 512, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.xr, R_off, (nt + 1) * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.xt, T_off, (nt + 1) * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.fo, F_off, (nt + 1) * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.bo, w.blob_off.data(), 2 * nt * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.ro, w.off_r.data(), nt * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.to, w.off_t.data(), nt * 8, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.cr, w.caps_r.data(), nt * 4, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.ct, w.caps_t.data(), nt * 4, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.al, w.algo.data(), nt * 4, cudaMemcpyHostToDevice, stream));
  SS_CHECK_CUDA(cudaMemcpyAsync(base + w.co, w.cell_off.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, stream));
  if (!w.tiles.empty())
    SS_CHECK_CUDA(cudaMemcpyAsync(base + w.tiles_off, w.tiles.data(), w.tiles.size() * sizeof(Tile),
                                  cudaMemcpyHostToDevice, stream));
  auto* gate = reinterpret_cast<unsigned*>(base + w.gate);
  // an axis that is not strictly increasing sets SS_FLAG_NOT_SORTED
  unsigned* flag = stat != nullptr ? &stat->flags : reinterpret_cast<unsigned*>(base + w.flag);
  unsigned char* blobs = base + w.blobs_off;
  const auto* blob_off = reinterpret_cast<const int64_t*>(base + w.bo);
  const auto* al = reinterpret_cast<const int*>(base + w.al);
  PrepArgs pr{nt, reinterpret_cast<const int64_t*>(base + w.xr), R, blobs, reinterpret_cast<const int64_t*>(base + w.ro),
              reinterpret_cast<const int*>(base + w.cr), al, 1, flag};
  PrepArgs pt{nt, reinterpret_cast<const int64_t*>(base + w.xt), T, blobs, reinterpret_cast<const int64_t*>(base + w.to),
              reinterpret_cast<const int*>(base + w.ct), al, 1, flag};
  k_prep_1d<<<nt, 256, 0, stream>>>(pr);
  k_prep_1d<<<nt, 256, 0, stream>>>(pt);
  k_prep_cells<<<nt, 256, 0, stream>>>(pr);
  k_prep_cells<<<nt, 256, 0, stream>>>(pt);
  SS_CHECK_CUDA(cudaGetLastError());
  auto* cells = reinterpret_cast<float4*>(base + w.cells_off);
  // a value outside the float-float range, or an axis off the common path,
  // sends the batch to the general kernel
  k_grid_cells<<<nt, 256, 0, stream>>>(F, reinterpret_cast<const int64_t*>(base + w.fo),
                                       reinterpret_cast<const int64_t*>(base + w.xr),
                                       reinterpret_cast<const int64_t*>(base + w.xt),
                                       reinterpret_cast<const int64_t*>(base + w.co), cells, gate);
  k_fast_2d_check<<<std::max(1, std::min(1024, (2 * nt + 255) / 256)), 256, 0, stream>>>(blobs, blob_off, 2 * nt,
                                                                                      BL_BUCKET, gate);
  SS_CHECK_CUDA(cudaGetLastError());
  if (w.tiles.empty()) return SS_OK;
  const int ntiles = (int)w.tiles.size();
  auto* counters = reinterpret_cast<int*>(base + w.counters);
  k_pick_2d<<<1, 1, 0, stream>>>(gate, counters, ntiles);
  SS_CHECK_CUDA(cudaGetLastError());
  const int vec = (aligned(Y2, 16) && aligned(lowbounds2, 16) && aligned(values, 16)) ? (aligned(Y2, 32) ? 2 : 1) : 0;
  const void* kerns[2] = {batched_2d_fast_kernel(BL_BUCKET), batched_2d_kernel(false, false)};
  for (int j = 0; j < 2; ++j) {
    if (ss_status st_ = raise_smem_limit(kerns[j], w.smem)) return st_;
    int per_sm = 0;
    SS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kerns[j], kNumThreads, w.smem));
    if (per_sm < 1) return fail(SS_EUNSUPPORTED, "batched 2D lookup: kernel does not fit on an SM");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, ntiles));
    BatchArgs2D a{blobs, blob_off, cells, F, reinterpret_cast<const int64_t*>(base + w.fo),
                  reinterpret_cast<const int64_t*>(base + w.co), 0, 0,
                  reinterpret_cast<const Tile*>(base + w.tiles_off), ntiles, counters + j, Y2, lowbounds2, values,
                  vec, stat};
    void* args[1] = {&a};
    SS_CHECK_CUDA(cudaLaunchKernel(kerns[j], dim3(grid), dim3(kNumThreads), args, (size_t)w.smem, stream));
  }
  return SS_OK;
}

}  // namespace ss
