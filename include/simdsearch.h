/*
 * simdsearch.h -- C ABI of the GB300 (sm_103a) sorted-table search library.
 *
 * The operation (arXiv 2112.03229, Sec. 3): for a strictly increasing float64
 * table X[0..n-1] and targets Y[0..m-1], return for every target the index of
 * the largest entry of X below the target, with the two end clamps of Sec. 3
 * (a target below X[0] gives 0, a target above X[n-1] gives n-1).  Written as
 * a count:
 *
 *     lowbounds[i] = max(0, #{ j : X[j] < Y[i] } - 1)      side SS_SIDE_LT
 *     lowbounds[i] = max(0, #{ j : X[j] <= Y[i] } - 1)     side SS_SIDE_LE
 *
 * SS_SIDE_LT ("largest element less than the target", Sec. 1) is the default;
 * SS_SIDE_LE is the "less than or equal" wording of Sec. 3.  Comparisons are
 * exact IEEE-754 float64 comparisons: -0 == +0, a NaN target compares false
 * against every entry (index 0), -inf gives 0, +inf gives n-1.
 *
 * The 2D lookup (Sec. 1 and 2.2: EOSPAC bounds a density/temperature target
 * in both grids of a SESAME table and interpolates; the paper prints no
 * formula) is, per (rho, T) pair:
 *     i = lowbound(R, rho), j = lowbound(T, T)              (the index outputs)
 *     c = min(i, nr-2), d = min(j, nt-2)
 *     w = clamp((rho - R[c]) / (R[c+1] - R[c]), 0, 1),  u likewise on T
 *     v = (1-w)((1-u) F[c][d] + u F[c][d+1]) + w((1-u) F[c+1][d] + u F[c+1][d+1])
 * with F row-major [nr][nt].  Values agree with an fp64 evaluation of this
 * formula to 1e-12 relative; indices are exact.
 *
 * Conventions for every entry point:
 *  - Pointers marked (device) are device memory of the current CUDA device;
 *    (host) marks host memory.  The caller owns every buffer it passes.
 *  - All calls are asynchronous on `stream`; the returned status covers
 *    argument checks and launch errors only.  Data-dependent conditions (a
 *    table that is not strictly increasing, NaN targets, learned proposals
 *    that failed their check) are recorded in an optional caller-owned device
 *    record `ss_devstat` (pass NULL to skip); zero it before the call.
 *  - Element pointers must be naturally aligned (8 bytes for double, 4 for
 *    int32).  16-byte alignment of the target and output arrays selects the
 *    128-bit load/store path; other alignments are handled, more slowly.
 *  - n >= 2 (each 2D axis >= 2), m >= 0; m == 0 launches nothing.
 *  - Results for a table that is not strictly increasing are unspecified
 *    (the table check sets SS_FLAG_NOT_SORTED) but every index stays in
 *    [0, n-1] and nothing outside the buffers is touched.
 *  - On an error the message of the failing call is kept per host thread and
 *    returned by ss_last_error().
 */
#ifndef SIMDSEARCH_H
#define SIMDSEARCH_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ss_status {
  SS_OK = 0,
  SS_EINVAL = 1,        /* bad argument (null pointer, size, alignment, option) */
  SS_ENOTSORTED = 2,    /* table not strictly increasing or holds NaN (plan creation) */
  SS_ENOMEM = 3,        /* device or host allocation failed */
  SS_ECUDA = 4,         /* a CUDA call failed; ss_last_error() names it */
  SS_ETIMEOUT = 5,      /* ss_sync_status() deadline passed before the stream finished */
  SS_EUNSUPPORTED = 6   /* the option is valid but not available for this size */
} ss_status;

typedef enum ss_side { SS_SIDE_LT = 0, SS_SIDE_LE = 1 } ss_side;

/* Search algorithm inside a thread block (all give identical indices). */
typedef enum ss_algo {
  SS_ALGO_AUTO = 0,     /* library choice (bucket directory for small tables) */
  SS_ALGO_BINARY = 1,   /* branchless binary search, breadth-first (Eytzinger) key layout (Sec. 3.2) */
  SS_ALGO_BUCKET = 2,   /* exponent-bit bucket directory + bounded scan (Sec. 3.5) */
  SS_ALGO_BALLOT = 3,   /* warp-cooperative 33-ary search: one key per lane, __ballot_sync/__popc */
  SS_ALGO_BRANCHY = 4   /* textbook bisection with data-dependent branches (Sec. 5.4 comparison) */
} ss_algo;

/* Device-side status record; caller-owned device memory, zeroed by the caller. */
typedef struct ss_devstat {
  unsigned long long nan_targets;   /* targets (or pair coordinates) that were NaN */
  unsigned long long fallbacks;     /* learned proposals rejected by the interval check */
  unsigned int flags;               /* SS_FLAG_* bits */
  unsigned int max_window;          /* largest learned fix-up window used */
} ss_devstat;

#define SS_FLAG_NOT_SORTED 0x1u     /* a table was not strictly increasing (or held NaN) */
#define SS_FLAG_BAD_VALUE 0x2u      /* a 2D value-path precondition failed; fp64 path used */

/* ---------------------------------------------------------------------- */
/* One-shot calls: no set-up kept between calls ("zero set-up cost",       */
/* Sec. 5.3).  Each thread block stages the table in shared memory once.    */
/* ---------------------------------------------------------------------- */

/* Sec. 3: lowbounds[i] for m targets over one table.
 * X (device) [n] float64, strictly increasing; Y (device) [m] float64;
 * lowbounds (device) [m] int32 output.  algo: ss_algo.  side: ss_side. */
ss_status ss_search_1d(const double* X, int32_t n, const double* Y, int64_t m,
                       int32_t* lowbounds, int32_t side, int32_t algo,
                       ss_devstat* stat, cudaStream_t stream);

/* Sec. 1 / 2.2 (EOSPAC 2D lookup): search both axes and interpolate.
 * R (device) [nr], T (device) [nt] strictly increasing float64 axes;
 * F (device) [nr*nt] float64 row-major values; Y2 (device) [2m] interleaved
 * (rho, T) pairs; lowbounds2 (device) [2m] int32 output, interleaved
 * (i_rho, i_T); values (device) [m] float64 output.  algo applies to both
 * axis searches. */
ss_status ss_search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt,
                              const double* F, const double* Y2, int64_t m,
                              int32_t* lowbounds2, double* values, int32_t algo,
                              ss_devstat* stat, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Status and diagnostics                                                  */
/* ---------------------------------------------------------------------- */

/* Wait up to timeout_ms for `stream` to drain (polling, never blocking
 * forever), then copy *stat (device) into *out (host).  SS_ETIMEOUT if the
 * stream is still busy at the deadline; *out is then left untouched. */
ss_status ss_sync_status(cudaStream_t stream, const ss_devstat* stat, ss_devstat* out,
                         int32_t timeout_ms);

/* Message of the last failing call on this host thread ("" if none). */
const char* ss_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t ss_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SIMDSEARCH_H */
