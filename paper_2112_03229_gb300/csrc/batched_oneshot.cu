// batched_oneshot.cu -- the batched searches (Sec. 1 and 2.2 applied to many
// tables at once) as single calls: a plan without a model is prepared, bound
// to the caller's batch, executed once and released.  The call waits for the
// launch before releasing the plan's memory, so it is synchronous; callers
// that search the same tables again keep a plan instead and pay the
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
  if (Y_off == nullptr) return ss::fail(SS_EINVAL, "ss_search_1d_batched: null pointer");
  const ss_plan_opts o = oneshot_opts(side);
  ss_plan* p = nullptr;
  if (ss_status st = ss_plan_create_1d(&p, ntables, X_off, X, &o, stream)) return st;
  return run_and_release(
      p, [&](ss_plan* q) { return ss_plan_bind_1d(q, Y_off, Y, lowbounds, stat, stream); }, stream);
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
