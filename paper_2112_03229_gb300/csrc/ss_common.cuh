// ss_common.cuh -- device helpers shared by every kernel of the library:
// the order-preserving integer image of a float64, streaming 128- and
// 256-bit loads and stores, and host-side error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/simdsearch.h"

namespace ss {

constexpr uint64_t kKeyMax = ~0ull;                    // sentinel above every real key
constexpr uint64_t kKeyPosInf = 0xFFF0000000000000ull;  // image of +inf
constexpr int kNumThreads = 256;                       // threads per block of the streaming kernels

// ---------------------------------------------------------------------------
// Order-preserving image of a double (Sec. 3.5 reads the exponent bits of the
// IEEE-754 pattern; this extends that to a total order over all non-NaN
// doubles).  Non-negative values: set the sign bit.  Negative values: two's
// complement of the pattern, which also sends -0 onto +0.  For non-NaN a, b:
// a < b  <=>  key(a) < key(b), and key(-0) == key(+0).
// A NaN target is mapped to 0, below every table key, so that its count of
// smaller entries is 0 (index 0).  Negative NaNs already land below key(-inf);
// positive NaNs land above key(+inf) and are moved down explicitly.
// All integer work: no fp64 instruction is issued.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t order_key(double x) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(x));
  const uint64_t neg = static_cast<uint64_t>(static_cast<int64_t>(u) >> 63);  // all ones if negative
  uint64_t k = (u ^ (neg | 0x8000000000000000ull)) - neg;                      // ~u + 1 or u | 2^63
  return k > kKeyPosInf ? 0ull : k;
}

// Streaming (evict-first) 128-bit global accesses for data touched once.
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(int4* p, int4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double2* p, double2 v) { __stcs(p, v); }

// Streaming 256-bit load of four doubles (p must be 32-byte aligned).
__device__ __forceinline__ void ld_stream4(const double* p, double (&r)[4]) {
  asm("ld.global.cs.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3]) : "l"(p));
}

// One 256-bit read-only load of 32 bytes (p must be 32-byte aligned): a
// gathered record costs one L1 request instead of two 128-bit ones.
__device__ __forceinline__ void ld_nc_v8(const float* p, float (&r)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
      : "l"(p));
}

// L2 eviction priorities (createpolicy descriptors) for the 2D plans: the
// corner records a batch gathers are reused by every pair that falls in their
// cell, while the targets stream past once, so the gathers are marked
// evict-last and the target loads evict-first, and the stream of targets does
// not push the records of the tables in flight out of L2.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// ld_nc_v8 with an L2 policy.
__device__ __forceinline__ void ld_nc_v8_policy(const float* p, float (&r)[8], uint64_t pol) {
  asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
      : "l"(p), "l"(pol));
}

// 256-bit load of four doubles read once (no L1 allocation) with an L2 policy.
__device__ __forceinline__ void ld_stream4_policy(const double* p, double (&r)[4], uint64_t pol) {
  asm("ld.global.L1::no_allocate.L2::cache_hint.v4.f64 {%0, %1, %2, %3}, [%4], %5;"
      : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3])
      : "l"(p), "l"(pol));
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
ss_status fail(ss_status code, const std::string& msg);
ss_status cuda_fail(cudaError_t err, const char* what);
int num_sms();
int max_smem_optin();
ss_status raise_smem_limit(const void* kernel, int smem);   // raise-only, thread-safe

#define SS_CHECK_CUDA(call)                                   \
  do {                                                        \
    cudaError_t err_ = (call);                                \
    if (err_ != cudaSuccess) return ::ss::cuda_fail(err_, #call); \
  } while (0)

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// ---------------------------------------------------------------------------
// Bounds-checked build (-DSS_CHECKED).  SS_IX(i, n) is index i of an array
// of n entries: in the ordinary build it is i itself; in the checked build
// an index outside [0, n) is counted (per translation unit, in device
// memory) and replaced by 0, so the read that follows stays inside the
// array instead of faulting.  SS_BOUNDS_FOLD(stat) at the end of a kernel
// sets SS_FLAG_BOUNDS in the caller's status record when the count of this
// unit is not zero.  ss_checked_hits (C ABI) adds up the counts of every
// unit: each unit registers a reader of its own counter at load time.
// ---------------------------------------------------------------------------
#ifdef SS_CHECKED
static __device__ unsigned long long g_ss_bounds_hits;

__device__ __forceinline__ int ss_checked_index(int i, int n) {
  if ((unsigned)i < (unsigned)n) return i;
  atomicAdd(&g_ss_bounds_hits, 1ull);
  return 0;
}

__device__ __forceinline__ void ss_checked_flag(bool bad) {
  if (bad) atomicAdd(&g_ss_bounds_hits, 1ull);
}

void register_bounds_counter(ss_status (*read)(unsigned long long*, bool));

static ss_status read_bounds_counter(unsigned long long* v, bool reset) {
  SS_CHECK_CUDA(cudaMemcpyFromSymbol(v, g_ss_bounds_hits, sizeof(*v)));
  if (reset) {
    const unsigned long long zero = 0;
    SS_CHECK_CUDA(cudaMemcpyToSymbol(g_ss_bounds_hits, &zero, sizeof(zero)));
  }
  return SS_OK;
}

namespace {
struct BoundsCounterRegistration {
  BoundsCounterRegistration() { register_bounds_counter(&read_bounds_counter); }
};
static BoundsCounterRegistration g_bounds_registration;
}  // namespace

#define SS_IX(i, n) ::ss::ss_checked_index((i), (n))
#define SS_CHECK(bad) ::ss::ss_checked_flag(bad)
#define SS_BOUNDS_FOLD(stat)                                                              \
  do {                                                                                    \
    if ((stat) != nullptr && threadIdx.x == 0 && ::ss::g_ss_bounds_hits != 0)            \
      atomicOr(&(stat)->flags, SS_FLAG_BOUNDS);                                           \
  } while (0)
#else
#define SS_IX(i, n) (i)
#define SS_CHECK(bad) ((void)0)
#define SS_BOUNDS_FOLD(stat) ((void)0)
#endif

}  // namespace ss
