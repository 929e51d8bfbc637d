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
  BatchWork1D w;
  if (ss_status st = batch_work_1d(me, ntables, X_off, Y_off, kStaticDirCap, w)) return st;
  if (w.end > (int64_t)kStaticScratchBytes)
    return fail(SS_EINVAL, std::string(me) + ": the batch needs " + std::to_string(w.end) +
                               " bytes of working memory, more than the fixed " +
                               std::to_string(kStaticScratchBytes) + " bytes of this entry point");
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
  const ss_status st = queue_work_1d(w, d->addr, ntables, X_off, X, Y, lowbounds, side, stat, stream);
  const cudaError_t e = cudaEventRecord(d->done, stream);
  if (e != cudaSuccess) return st != SS_OK ? st : cuda_fail(e, "cudaEventRecord");
  d->used = true;
  return st;
}
