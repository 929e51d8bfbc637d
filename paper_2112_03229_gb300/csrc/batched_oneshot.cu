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
// 2D: the same, with both axes of every table prepared, the corner records
// built and the lean or the general persistent kernel picked on the GPU
// (batched_work_2d.cu).
//
// Callers that search the same tables again keep a plan instead and pay the
// preparation once (Sec. 5.3).
#include <string>

#include "plan.h"
#include "plan_host.h"

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
  using namespace ss;
  const char* me = "ss_search_interp_2d_batched";
  if (R_off == nullptr || T_off == nullptr || F_off == nullptr || Y_off == nullptr || R == nullptr || T == nullptr ||
      F == nullptr)
    return fail(SS_EINVAL, std::string(me) + ": null pointer");
  if (ntables < 1) return fail(SS_EINVAL, std::string(me) + ": ntables must be >= 1");
  if (Y_off[ntables] > 0 && (Y2 == nullptr || lowbounds2 == nullptr || values == nullptr))
    return fail(SS_EINVAL, std::string(me) + ": null pointer");
  if (!aligned(R, 8) || !aligned(T, 8) || !aligned(F, 8) || !aligned(Y2, 8) || !aligned(lowbounds2, 4) ||
      !aligned(values, 8))
    return fail(SS_EINVAL, std::string(me) + ": misaligned pointer");
  BatchWork2D w;
  if (ss_status st = batch_work_2d(me, ntables, R_off, T_off, F_off, Y_off, w)) return st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SS_CHECK_CUDA(cudaStreamIsCapturing(stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(SS_EUNSUPPORTED, std::string(me) + ": the stream is capturing; keep a plan to replay in a graph");
  unsigned char* base = nullptr;
  SS_CHECK_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&base), (size_t)w.end, stream));
  const ss_status st = queue_work_2d(w, base, ntables, R_off, R, T_off, T, F_off, F, Y2, lowbounds2, values, stat,
                                     stream);
  const cudaError_t e = cudaFreeAsync(base, stream);        // after the queued work, on every path
  if (st != SS_OK) return st;
  return e == cudaSuccess ? SS_OK : cuda_fail(e, "cudaFreeAsync");
}
