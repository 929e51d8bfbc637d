// host_api.cu -- the one-shot searches over host-resident arrays.
//
// EOSPAC's callers hand over host arrays of targets (Sec. 1, 2.2).  Two ways
// through the GPU:
//  * page-locked target and result buffers are mapped into the device's
//    address space, so the search kernels stream them directly over the
//    host link: reads of targets and writes of results are in flight
//    together and no staging copy is made (the tables, a few KB, are copied
//    to the device first);
//  * pageable buffers move in chunks, with the host-to-device copy of chunk
//    c+1, the search of chunk c and the device-to-host copy of chunk c-1
//    running at the same time on two streams.
// The device buffers (tables, and the chunks of the pageable path) are
// allocated on first use and kept per device (grown on demand); calls on one
// device are serialised.
#include <algorithm>
#include <mutex>

#include "ss_common.cuh"

namespace ss {

ss_status search_1d(const double* X, int32_t n, const double* Y, int64_t m, int32_t* out, int32_t side,
                    int32_t algo, ss_devstat* stat, cudaStream_t stream, int dir_cap_override, int ballot_g);
ss_status search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt, const double* F,
                           const double* Y2, int64_t m, int32_t* idx, double* val, int32_t algo, int force_fp64,
                           ss_devstat* stat, cudaStream_t stream, int extrap, int logspace);

namespace {

struct Workspace {
  unsigned char* buf = nullptr;   // [table area][2 x chunk area]
  size_t bytes = 0;
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaEvent_t ready = nullptr;
};

std::mutex g_mu;
Workspace g_ws[64];

constexpr int64_t kChunk1D = int64_t(1) << 24;    // targets per chunk (128 MB in, 64 MB out)
constexpr int64_t kChunk2D = int64_t(1) << 23;    // pairs per chunk (128 MB in, 64 + 64 MB out)

ss_status workspace(size_t bytes, Workspace** out) {
  int dev = 0;
  SS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SS_EUNSUPPORTED, "host search: device ordinal out of range");
  Workspace& w = g_ws[dev];
  if (w.st[0] == nullptr) {
    SS_CHECK_CUDA(cudaStreamCreateWithFlags(&w.st[0], cudaStreamNonBlocking));
    SS_CHECK_CUDA(cudaStreamCreateWithFlags(&w.st[1], cudaStreamNonBlocking));
    SS_CHECK_CUDA(cudaEventCreateWithFlags(&w.ready, cudaEventDisableTiming));
  }
  if (w.bytes < bytes) {
    if (w.buf) cudaFree(w.buf);
    w.buf = nullptr;
    w.bytes = 0;
    if (cudaMalloc(&w.buf, bytes) != cudaSuccess) return fail(SS_ENOMEM, "host search: staging allocation failed");
    w.bytes = bytes;
  }
  *out = &w;
  return SS_OK;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of page-locked, mapped host memory [p, p + bytes), or
// nullptr if either end is not such memory (pageable, device, unregistered)
// or the two ends do not map to one contiguous device range (two separate
// page-locked allocations that happen to sit side by side in host memory).
template <class T>
T* mapped(T* p, size_t bytes) {
  if (p == nullptr || bytes == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  const unsigned char* last = reinterpret_cast<const unsigned char*>(p) + bytes - 1;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();   // clear the query's error state
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
  if (static_cast<const unsigned char*>(b.devicePointer) != static_cast<const unsigned char*>(a.devicePointer) + bytes - 1)
    return nullptr;
  return static_cast<T*>(a.devicePointer);
}

// Waits for everything queued on the workspace's two streams, so that no copy
// into the caller's buffers is still in flight when a call returns, an error
// part way through the chunks included.  The first failure is returned.
ss_status drain(Workspace* w, ss_status st) {
  const cudaError_t e0 = cudaStreamSynchronize(w->st[0]);
  const cudaError_t e1 = cudaStreamSynchronize(w->st[1]);
  if (st != SS_OK) return st;
  if (e0 != cudaSuccess) return cuda_fail(e0, "cudaStreamSynchronize");
  if (e1 != cudaSuccess) return cuda_fail(e1, "cudaStreamSynchronize");
  return SS_OK;
}

}  // namespace
}  // namespace ss

using namespace ss;

extern "C" ss_status ss_search_1d_host(const double* X, int32_t n, const double* Y, int64_t m, int32_t* lowbounds,
                                       int32_t side, int32_t algo) {
  if (X == nullptr || (m > 0 && (Y == nullptr || lowbounds == nullptr))) return fail(SS_EINVAL, "ss_search_1d_host: null pointer");
  if (n < 2 || m < 0) return fail(SS_EINVAL, "ss_search_1d_host: need n >= 2 and m >= 0");
  if (m == 0) return SS_OK;
  std::lock_guard<std::mutex> lock(g_mu);
  const size_t tab = up256((size_t)n * 8);
  const size_t cin = up256((size_t)kChunk1D * 8), cout = up256((size_t)kChunk1D * 4);
  const double* mY = mapped(Y, (size_t)m * 8);
  int32_t* mO = mapped(lowbounds, (size_t)m * 4);
  const bool direct = mY != nullptr && mO != nullptr;
  Workspace* w = nullptr;
  if (ss_status st = workspace(direct ? tab : tab + 2 * (cin + cout), &w)) return st;
  double* dX = reinterpret_cast<double*>(w->buf);
  auto queue = [&]() -> ss_status {
    SS_CHECK_CUDA(cudaMemcpyAsync(dX, X, (size_t)n * 8, cudaMemcpyHostToDevice, w->st[0]));
    // page-locked buffers: one launch streams them over the link
    if (direct) return search_1d(dX, n, mY, m, mO, side, algo, nullptr, w->st[0], 0, 0);
    SS_CHECK_CUDA(cudaEventRecord(w->ready, w->st[0]));
    SS_CHECK_CUDA(cudaStreamWaitEvent(w->st[1], w->ready, 0));
    for (int64_t off = 0, c = 0; off < m; off += kChunk1D, ++c) {
      const int64_t cnt = std::min(kChunk1D, m - off);
      cudaStream_t s = w->st[c & 1];
      double* dY = reinterpret_cast<double*>(w->buf + tab + (c & 1) * (cin + cout));
      int32_t* dO = reinterpret_cast<int32_t*>(w->buf + tab + (c & 1) * (cin + cout) + cin);
      SS_CHECK_CUDA(cudaMemcpyAsync(dY, Y + off, (size_t)cnt * 8, cudaMemcpyHostToDevice, s));
      if (ss_status st = search_1d(dX, n, dY, cnt, dO, side, algo, nullptr, s, 0, 0)) return st;
      SS_CHECK_CUDA(cudaMemcpyAsync(lowbounds + off, dO, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s));
    }
    return SS_OK;
  };
  return drain(w, queue());
}

extern "C" ss_status ss_search_interp_2d_host(const double* R, int32_t nr, const double* T, int32_t nt,
                                              const double* F, const double* Y2, int64_t m, int32_t* lowbounds2,
                                              double* values, int32_t algo) {
  if (R == nullptr || T == nullptr || F == nullptr || (m > 0 && (Y2 == nullptr || lowbounds2 == nullptr || values == nullptr)))
    return fail(SS_EINVAL, "ss_search_interp_2d_host: null pointer");
  if (nr < 2 || nt < 2 || m < 0) return fail(SS_EINVAL, "ss_search_interp_2d_host: need axes >= 2 and m >= 0");
  if (nr > SS_MAX_AXIS_2D || nt > SS_MAX_AXIS_2D)
    return fail(SS_EUNSUPPORTED, "ss_search_interp_2d_host: axis longer than SS_MAX_AXIS_2D");
  if (m == 0) return SS_OK;
  std::lock_guard<std::mutex> lock(g_mu);
  const size_t tr = up256((size_t)nr * 8), tt = up256((size_t)nt * 8), tf = up256((size_t)nr * nt * 8);
  const size_t cin = up256((size_t)kChunk2D * 16), cidx = up256((size_t)kChunk2D * 8), cval = up256((size_t)kChunk2D * 8);
  const size_t chunk = cin + cidx + cval;
  const double* mY = mapped(Y2, (size_t)m * 16);
  int32_t* mI = mapped(lowbounds2, (size_t)m * 8);
  double* mV = mapped(values, (size_t)m * 8);
  const bool direct = mY != nullptr && mI != nullptr && mV != nullptr;
  Workspace* w = nullptr;
  if (ss_status st = workspace(direct ? tr + tt + tf : tr + tt + tf + 2 * chunk, &w)) return st;
  double* dR = reinterpret_cast<double*>(w->buf);
  double* dT = reinterpret_cast<double*>(w->buf + tr);
  double* dF = reinterpret_cast<double*>(w->buf + tr + tt);
  auto queue = [&]() -> ss_status {
    SS_CHECK_CUDA(cudaMemcpyAsync(dR, R, (size_t)nr * 8, cudaMemcpyHostToDevice, w->st[0]));
    SS_CHECK_CUDA(cudaMemcpyAsync(dT, T, (size_t)nt * 8, cudaMemcpyHostToDevice, w->st[0]));
    SS_CHECK_CUDA(cudaMemcpyAsync(dF, F, (size_t)nr * nt * 8, cudaMemcpyHostToDevice, w->st[0]));
    if (direct) return search_interp_2d(dR, nr, dT, nt, dF, mY, m, mI, mV, algo, 0, nullptr, w->st[0], 0, 0);
    SS_CHECK_CUDA(cudaEventRecord(w->ready, w->st[0]));
    SS_CHECK_CUDA(cudaStreamWaitEvent(w->st[1], w->ready, 0));
    unsigned char* base = w->buf + tr + tt + tf;
    for (int64_t off = 0, c = 0; off < m; off += kChunk2D, ++c) {
      const int64_t cnt = std::min(kChunk2D, m - off);
      cudaStream_t s = w->st[c & 1];
      unsigned char* b = base + (c & 1) * chunk;
      double* dY = reinterpret_cast<double*>(b);
      int32_t* dI = reinterpret_cast<int32_t*>(b + cin);
      double* dV = reinterpret_cast<double*>(b + cin + cidx);
      SS_CHECK_CUDA(cudaMemcpyAsync(dY, Y2 + 2 * off, (size_t)cnt * 16, cudaMemcpyHostToDevice, s));
      if (ss_status st = search_interp_2d(dR, nr, dT, nt, dF, dY, cnt, dI, dV, algo, 0, nullptr, s, 0, 0)) return st;
      SS_CHECK_CUDA(cudaMemcpyAsync(lowbounds2 + 2 * off, dI, (size_t)cnt * 8, cudaMemcpyDeviceToHost, s));
      SS_CHECK_CUDA(cudaMemcpyAsync(values + off, dV, (size_t)cnt * 8, cudaMemcpyDeviceToHost, s));
    }
    return SS_OK;
  };
  return drain(w, queue());
}
