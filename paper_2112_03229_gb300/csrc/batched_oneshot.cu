// batched_oneshot.cu -- the batched searches (Sec. 1 and 2.2 applied to many
// tables at once) as single calls.
//
// 1D: asynchronous on the caller's stream.  The host lays the batch out from
// the offsets alone; a stream-ordered allocation holds the prepared tables
// and tiles; the preparation, the persistent bucket search and the release
// of that memory are queued behind each other, and the call returns without
// waiting.  A table that is not strictly increasing is flagged in the
// caller's status record (SS_FLAG_NOT_SORTED) by the preparation on the GPU.
//
// 2D: a plan without a model is prepared, bound to the caller's batch,
// executed once and released; the call waits for the launch before
// releasing the plan's memory, so it is synchronous.
//
// Callers that search the same tables again keep a plan instead and pay the
// preparation once (Sec. 5.3).
#include <string>

#include "plan.h"
#include "plan_host.h"

namespace {

ss_plan_opts oneshot_opts(int32_t side) {
  ss_plan_opts o;
  ss_plan_opts_default(&o);
  o.side = side;
  o.model = SS_MODEL_NONE;
  o.autotune = 0;
  return o;
}

// Bind, execute, wait, release; the first failure's status is returned.
template <class Bind>
ss_status run_and_release(ss_plan* p, Bind&& bind, cudaStream_t stream) {
  ss_status st = bind(p);
  if (st == SS_OK) st = ss_plan_execute(p, stream);
  if (st == SS_OK) {
    const cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = ss::cuda_fail(e, "cudaStreamSynchronize");
  }
  ss_plan_destroy(p);
  return st;
}

}  // namespace

extern "C" ss_status ss_search_1d_batched(int32_t ntables, const int64_t* X_off, const double* X,
                                          const int64_t* Y_off, const double* Y, int32_t* lowbounds, int32_t side,
                                          ss_devstat* stat, cudaStream_t stream) {
  using namespace ss;
  const char* me = "ss_search_1d_batched";
  if (X_off == nullptr || Y_off == nullptr || X == nullptr) return fail(SS_EINVAL, std::string(me) + ": null pointer");
  if (ntables < 1) return fail(SS_EINVAL, std::string(me) + ": ntables must be >= 1");
  if (side != SS_SIDE_LT && side != SS_SIDE_LE) return fail(SS_EINVAL, std::string(me) + ": bad side");
  if (Y_off[ntables] > 0 && (Y == nullptr || lowbounds == nullptr)) return fail(SS_EINVAL, std::string(me) + ": null pointer");
  if (!aligned(X, 8) || !aligned(Y, 8) || !aligned(lowbounds, 4)) return fail(SS_EINVAL, std::string(me) + ": misaligned pointer");
  BatchWork1D w;
  if (ss_status st = batch_work_1d(me, ntables, X_off, Y_off, SS_MAX_DIR_CAP, w)) return st;
  // the metadata is copied from pageable host memory, which a stream being
  // captured into a graph cannot take: refused before anything is queued
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SS_CHECK_CUDA(cudaStreamIsCapturing(stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(SS_EUNSUPPORTED, std::string(me) + ": the stream is capturing; keep a plan to replay in a graph");
  unsigned char* base = nullptr;
  SS_CHECK_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&base), (size_t)w.end, stream));
  const ss_status st = queue_work_1d(w, base, ntables, X_off, X, Y, lowbounds, side, stat, stream);
  const cudaError_t e = cudaFreeAsync(base, stream);        // after the queued work, on every path
  if (st != SS_OK) return st;
  return e == cudaSuccess ? SS_OK : cuda_fail(e, "cudaFreeAsync");
}

extern "C" ss_status ss_search_interp_2d_batched(int32_t ntables, const int64_t* R_off, const double* R,
                                                 const int64_t* T_off, const double* T, const int64_t* F_off,
                                                 const double* F, const int64_t* Y_off, const double* Y2,
                                                 int32_t* lowbounds2, double* values, ss_devstat* stat,
                                                 cudaStream_t stream) {
  if (Y_off == nullptr) return ss::fail(SS_EINVAL, "ss_search_interp_2d_batched: null pointer");
  const ss_plan_opts o = oneshot_opts(SS_SIDE_LT);
  ss_plan* p = nullptr;
  if (ss_status st = ss_plan_create_2d(&p, ntables, R_off, R, T_off, T, F_off, F, &o, stream)) return st;
  return run_and_release(
      p, [&](ss_plan* q) { return ss_plan_bind_2d(q, Y_off, Y2, lowbounds2, values, stat, stream); }, stream);
}
