// capi.cu -- host-side plumbing of the C ABI: per-thread error messages,
// device properties, the polling status read-back.
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "ss_common.cuh"

namespace ss {

static thread_local std::string g_last_error;

ss_status fail(ss_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

ss_status cuda_fail(cudaError_t err, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  return SS_ECUDA;
}

int num_sms() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v > 0 ? v : 48 * 1024;
}

// The dynamic shared-memory limit of a kernel is a process-wide attribute.
// Lowering it while another host thread holds a launch (or a captured graph)
// sized for a larger limit would make that launch fail, so the limit is only
// ever raised: per device and kernel, the largest size asked for so far.
ss_status raise_smem_limit(const void* kernel, int smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> set;
  int dev = 0;
  SS_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int& cur = set[std::make_pair(dev, kernel)];
  if (smem > cur) {
    SS_CHECK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cur = smem;
  }
  return SS_OK;
}

#ifdef SS_CHECKED
static std::vector<ss_status (*)(unsigned long long*, bool)>& bounds_counters() {
  static std::vector<ss_status (*)(unsigned long long*, bool)> v;
  return v;
}

void register_bounds_counter(ss_status (*read)(unsigned long long*, bool)) { bounds_counters().push_back(read); }

// One check of an index past the end of a 3-entry array: counted, never read.
__global__ void k_checked_selftest(int i) { (void)SS_IX(i, 3); }
#endif

}  // namespace ss

extern "C" {

ss_status ss_checked_hits(uint64_t* hits, int32_t reset) {
#ifdef SS_CHECKED
  if (hits == nullptr) return ss::fail(SS_EINVAL, "ss_checked_hits: null pointer");
  SS_CHECK_CUDA(cudaDeviceSynchronize());
  uint64_t sum = 0;
  for (auto read : ss::bounds_counters()) {
    unsigned long long v = 0;
    if (ss_status st = read(&v, reset != 0)) return st;
    sum += v;
  }
  *hits = sum;
  return SS_OK;
#else
  (void)hits;
  (void)reset;
  return ss::fail(SS_EUNSUPPORTED, "ss_checked_hits: the library was built without -DSS_CHECKED");
#endif
}

ss_status ss_checked_selftest(void) {
#ifdef SS_CHECKED
  ss::k_checked_selftest<<<1, 1>>>(5);
  SS_CHECK_CUDA(cudaGetLastError());
  SS_CHECK_CUDA(cudaDeviceSynchronize());
  return SS_OK;
#else
  return ss::fail(SS_EUNSUPPORTED, "ss_checked_selftest: the library was built without -DSS_CHECKED");
#endif
}

const char* ss_last_error(void) { return ss::g_last_error.c_str(); }

int32_t ss_version(void) { return 1 * 10000 + 0 * 100 + 0; }

ss_status ss_sync_status(cudaStream_t stream, const ss_devstat* stat, ss_devstat* out, int32_t timeout_ms) {
  if (stat == nullptr || out == nullptr || timeout_ms < 0) return ss::fail(SS_EINVAL, "ss_sync_status: null pointer or negative timeout");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    cudaError_t q = cudaStreamQuery(stream);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return ss::cuda_fail(q, "cudaStreamQuery");
    if (std::chrono::steady_clock::now() >= deadline) return ss::fail(SS_ETIMEOUT, "ss_sync_status: stream still busy at the deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  SS_CHECK_CUDA(cudaMemcpy(out, stat, sizeof(ss_devstat), cudaMemcpyDeviceToHost));
  return SS_OK;
}

}  // extern "C"
