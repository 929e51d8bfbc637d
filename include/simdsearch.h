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
 *    vector load/store path (32-byte aligned targets load as 256-bit
 *    accesses); other alignments are handled, more slowly.
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

/* Largest bucket-directory budget a caller may ask for (ss_plan_opts.dir_cap). */
#define SS_MAX_DIR_CAP 65536

/* Longest axis of the one-shot 2D lookups, which stage both axes with their
 * per-cell data in shared memory (plans take axes of up to 2^20 entries). */
#define SS_MAX_AXIS_2D 4096

#define SS_FLAG_NOT_SORTED 0x1u     /* a table was not strictly increasing (or held NaN) */
#define SS_FLAG_BAD_VALUE 0x2u      /* a 2D value-path precondition failed; fp64 path used */
#define SS_FLAG_STAGING_TIMEOUT 0x4u /* a shared-memory staging copy did not complete in time; outputs incomplete */
#define SS_FLAG_BOUNDS 0x8u          /* bounds-checked build only: an index outside its array was caught (the
                                        read was skipped); see ss_checked_hits */

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
 * axis searches.  Each axis holds 2 .. SS_MAX_AXIS_2D entries
 * (SS_EUNSUPPORTED above). */
ss_status ss_search_interp_2d(const double* R, int32_t nr, const double* T, int32_t nt,
                              const double* F, const double* Y2, int64_t m,
                              int32_t* lowbounds2, double* values, int32_t algo,
                              ss_devstat* stat, cudaStream_t stream);

/* Interpolation options of the 2D lookup.  The paper prints no
 * interpolation formula (Sec. 1, 2.2); the default is bilinear in linear
 * axis coordinates with weights clamped to [0, 1] (constant extrapolation
 * beyond the grid).  extrap = 1 drops the clamp: targets outside an axis are
 * extrapolated linearly from its edge cell.  logspace = 1 takes each weight
 * in natural-log axis coordinates, w = (ln x - ln X[c]) / (ln X[c+1] -
 * ln X[c]) (a coordinate <= 0 gives a weight of -inf or NaN, which the clamp
 * and the NaN rule then handle).  Pairs that need either option are
 * evaluated in fp64; logspace = 1 evaluates every pair in fp64. */
typedef struct ss_interp_opts {
  int32_t algo;       /* ss_algo of both axis searches (AUTO, BUCKET or BINARY) */
  int32_t extrap;     /* 0: clamp the weights (default); 1: linear extrapolation */
  int32_t logspace;   /* 0: linear axis coordinates (default); 1: natural-log coordinates */
  int32_t fp64;       /* 1: fp64 weights and blend for every pair */
} ss_interp_opts;

/* ss_search_interp_2d with interpolation options (NULL opts: the defaults). */
ss_status ss_search_interp_2d_ex(const double* R, int32_t nr, const double* T, int32_t nt,
                                 const double* F, const double* Y2, int64_t m,
                                 int32_t* lowbounds2, double* values, const ss_interp_opts* opts,
                                 ss_devstat* stat, cudaStream_t stream);

/* Host-array forms of the two calls above, for callers whose targets live
 * in host memory (EOSPAC's callers pass host arrays, Sec. 1 and 2.2).  Every
 * pointer is host memory.  When the target and result buffers are
 * page-locked (cudaHostAlloc / cudaHostRegister) the search kernels read and
 * write them directly over the host link, reads and writes in flight
 * together, with no staging copy; pageable buffers are moved in chunks,
 * overlapping host-to-device copies, the search and device-to-host copies
 * on two streams.  Synchronous: the results are in host memory when the call
 * returns.  Device memory (the tables, and the chunks of the pageable path)
 * is allocated on first use per device and kept; calls on one device are
 * serialised. */
ss_status ss_search_1d_host(const double* X, int32_t n, const double* Y, int64_t m, int32_t* lowbounds,
                            int32_t side, int32_t algo);
ss_status ss_search_interp_2d_host(const double* R, int32_t nr, const double* T, int32_t nt,
                                   const double* F, const double* Y2, int64_t m, int32_t* lowbounds2,
                                   double* values, int32_t algo);

/* ---------------------------------------------------------------------- */
/* Plans: set-up once per set of loaded tables, then many searches.        */
/* EOSPAC loads its tables once at program start, so search set-up is paid  */
/* once (Sec. 5.3).  A plan prepares every table on the GPU (order-         */
/* preserving keys, bucket directory, breadth-first layout, optional        */
/* learned position model trained by the library's own kernels), chooses    */
/* per table-size bucket the in-block algorithm and tile size (autotuner),  */
/* and runs a whole batch of tables -- each with its own targets -- in one  */
/* persistent kernel launch that walks a tile queue, captured in a CUDA     */
/* graph.  The plan owns all device memory it allocates.                    */
/* ---------------------------------------------------------------------- */
typedef struct ss_plan ss_plan;

/* Learned position model used as the proposal of every table of a plan.
 * The model only proposes: each index is proved exactly against the table
 * (the answer must lie in a window [p-E, p+E] whose ends are compared with
 * the target, or, on a table staged whole with E <= 4, the keys on both
 * sides of the answer are read while walking at most E keys from p) and a
 * failed proof falls back to the plain search, so results are identical
 * with or without a model. */
typedef enum ss_model {
  SS_MODEL_NONE = 0,    /* plain search only */
  SS_MODEL_SPLINE = 1,  /* piecewise-linear map of the target's key, knots = bucket directory */
  SS_MODEL_MLP = 2,     /* 2-16-1 fp32 MLP on the target's exponent and mantissa, trained on the GPU */
  SS_MODEL_LOGHASH = 3, /* no training: the logarithm hash of Sec. 3.4 (Eqs. 1-2), base fitted to the end points */
  SS_MODEL_HUNT = 4,    /* hunt and locate (Sec. 2.1) for coherent sequences (Sec. 5.5), 1D and 2D plans: the
                           first of a thread's consecutive targets (2D: pairs) takes the table's own search, the
                           others start from its answer, probe away in doubling steps and bisect the last step;
                           exact for any order.  1D hunt plans use the bucket search (algo auto or bucket) */
  SS_MODEL_AUTO = 5     /* 1D plans: with autotune, the tuner picks per table-size bucket the fastest of the plain
                           searches and the untrained proposals (spline, logarithm hash), timed on the bucket's
                           own tables; every index stays exact whatever it picks.  Without autotune: as NONE */
} ss_model;

typedef struct ss_plan_opts {
  int32_t side;             /* ss_side */
  int32_t algo;             /* plain algorithm without a model: AUTO (tuner or bucket), BINARY, BUCKET, BALLOT */
  int32_t model;            /* ss_model */
  int32_t autotune;         /* 1: time the candidates of each table-size bucket and keep the fastest */
  int32_t tile;             /* targets per tile; 0: library default or tuned */
  int32_t mlp_epochs;       /* full-batch Adam steps of the MLP (default 400; 0 keeps the untrained initialisation) */
  float mlp_lr;             /* peak Adam learning rate, cosine-decayed (default 2e-3) */
  int32_t dir_cap;          /* bucket-directory budget per table.  0: fitted to each table's keys at plan creation
                               (4 n clamped to [64, 4096], refined where a bucket would hold two or more keys,
                               see ss_plan_info.max_occupancy; 8192 above 8128 entries); 1 .. SS_MAX_DIR_CAP: that
                               budget for every table (SS_EINVAL above it; SS_EUNSUPPORTED at bind when the
                               directory does not fit shared memory) */
  uint64_t seed;            /* seed of the counter-based sampler of training and probe targets */
  const char* tune_cache;   /* JSON file the autotuner reads and writes (NULL: none) */
  int32_t extrap;           /* 2D plans: interpolation options as in ss_interp_opts */
  int32_t logspace;
} ss_plan_opts;

typedef struct ss_plan_info {
  int32_t kind;             /* 1: 1D tables, 2: 2D tables */
  int32_t ntables;
  int64_t device_bytes;     /* device memory held by the plan */
  int32_t max_window;       /* largest learned half-window E over tables (0 without a model) */
  float mean_window;
  float train_loss;         /* mean final training loss of the MLP (MLP model only) */
  int32_t nbuckets;         /* table-size buckets [2,16) [16,64) [64,256) ... */
  int32_t bucket_algo[8];   /* chosen algorithm per bucket: 0 bucket, 1 binary, 2-4 ballot 8/16/32, 5 spline, 6 mlp, 7 loghash, 8 wide */
  int32_t bucket_tile[8];   /* chosen targets per tile per bucket */
  int32_t bucket_tables[8]; /* tables per bucket */
  int64_t ntiles;           /* tiles of the bound batch */
  int32_t tuned;            /* 1 if the autotuner (or its cache) set the choices */
  int32_t kernels;          /* kernels one ss_plan_execute launches for the bound batch (0, 1 or 2) */
  int32_t block_threads;    /* threads per block of the bound batched kernel (256, or 512 for large staged tables) */
  int32_t smem_bytes;       /* dynamic shared memory per block of that kernel */
  int32_t max_occupancy;    /* most keys in one directory bucket over the tables staged whole */
  int32_t lean_kernel;      /* 2D: 1 if the bound batch runs the lean kernel (every axis searched over a whole
                               staged axis with at most two keys per directory bucket, float-float cells, no
                               interpolation option; no position model, the hunt, or the spline, MLP or
                               logarithm-hash model with every learned half-window at most 4 keys) */
} ss_plan_info;

/* Fill *opts with the defaults. */
void ss_plan_opts_default(ss_plan_opts* opts);

/* Prepare ntables 1D tables.  X_off (host) [ntables+1] offsets into X
 * (device), table k = X[X_off[k] .. X_off[k+1]), each strictly increasing with
 * at least 2 entries.  Synchronises `stream`; SS_ENOTSORTED if a table is not
 * strictly increasing.  X is no longer needed once this returns. */
ss_status ss_plan_create_1d(ss_plan** plan, int32_t ntables, const int64_t* X_off, const double* X,
                            const ss_plan_opts* opts, cudaStream_t stream);

/* Prepare ntables 2D tables (Sec. 1 / 2.2 lookup): axes R, T and row-major
 * value grids F, each given by host offsets into device arrays (R_off, T_off,
 * F_off have ntables+1 entries; F_off[k+1]-F_off[k] = nr_k * nt_k). */
ss_status ss_plan_create_2d(ss_plan** plan, int32_t ntables, const int64_t* R_off, const double* R,
                            const int64_t* T_off, const double* T, const int64_t* F_off, const double* F,
                            const ss_plan_opts* opts, cudaStream_t stream);

/* Bind a batch: table k's targets are Y[Y_off[k] .. Y_off[k+1]) (Y_off host,
 * non-decreasing; empty tables allowed) and its results go to the same
 * positions of lowbounds.  Builds the tile queue and captures the launch in a
 * CUDA graph; buffers must stay valid while the plan executes.  Y and
 * lowbounds (and the 2D buffers below) are device memory or page-locked host
 * memory; the latter is streamed over the host link by the kernel itself. */
ss_status ss_plan_bind_1d(ss_plan* plan, const int64_t* Y_off, const double* Y, int32_t* lowbounds,
                          ss_devstat* stat, cudaStream_t stream);

/* 2D batch: pairs of table k are Y2[2 Y_off[k] .. 2 Y_off[k+1]) (interleaved
 * rho, T); lowbounds2 interleaved index pairs; values one double per pair. */
ss_status ss_plan_bind_2d(ss_plan* plan, const int64_t* Y_off, const double* Y2, int32_t* lowbounds2,
                          double* values, ss_devstat* stat, cudaStream_t stream);

/* Run the bound batch: one graph launch (a counter reset and the persistent kernel). */
ss_status ss_plan_execute(ss_plan* plan, cudaStream_t stream);

ss_status ss_plan_info_get(const ss_plan* plan, ss_plan_info* info);

/* Write the prepared tables, models and tuning choices to a file, and read
 * them back (the loaded plan gives identical results; bind it again).  The
 * file records the layout version of the prepared tables; ss_plan_load
 * returns SS_EINVAL for a file of another version (prepare the plan again)
 * and for a file whose layout is inconsistent: before any kernel sees a
 * loaded plan, its options, offsets and every prepared table's header,
 * bucket directories, occupancies and strides are checked on the host
 * against the sizes and budgets it records, so that no search reads outside
 * the plan.  Model weights and learned windows are not checked beyond their
 * sign: a wrong one costs fallbacks to the plain search, not exactness. */
ss_status ss_plan_save(const ss_plan* plan, const char* path);
ss_status ss_plan_load(ss_plan** plan, const char* path, cudaStream_t stream);

void ss_plan_destroy(ss_plan* plan);

/* One-shot batched forms: the search of Sec. 1 (and the 2D lookup of
 * Sec. 2.2) over many tables in one call, with the same results as a plan
 * without a model.  Table k is X[X_off[k] .. X_off[k+1]) with targets
 * Y[Y_off[k] .. Y_off[k+1]); X_off and Y_off are host arrays of ntables+1
 * entries (Y_off non-decreasing, empty tables allowed), X, Y and lowbounds
 * device arrays; table k's answers go to the same positions of lowbounds.
 * The 1D call is asynchronous on `stream`: it lays the batch out on the
 * host from the offsets, takes its working memory (prepared tables, tiles)
 * from the stream-ordered allocator, and queues the preparation, one
 * persistent launch of the bucket search and the release of that memory;
 * X, Y and lowbounds must stay valid until the stream reaches that point.
 * A table that is not strictly increasing sets SS_FLAG_NOT_SORTED in *stat
 * (its indices are then unspecified but in [0, n-1]; the other tables' are
 * exact).  Bad offsets are refused with SS_EINVAL naming the table; a
 * stream being captured is refused with SS_EUNSUPPORTED (the metadata is
 * copied from pageable host memory).  Callers that search the same tables
 * again should keep a plan: its preparation is paid once. */
ss_status ss_search_1d_batched(int32_t ntables, const int64_t* X_off, const double* X,
                               const int64_t* Y_off, const double* Y, int32_t* lowbounds,
                               int32_t side, ss_devstat* stat, cudaStream_t stream);

/* 2D: table k has axes R[R_off[k] ..], T[T_off[k] ..] (each of 2 ..
 * SS_MAX_AXIS_2D entries) and the row-major nr_k x nt_k grid
 * F[F_off[k] ..]; its pairs are Y2[2 Y_off[k] .. 2 Y_off[k+1]) interleaved
 * (rho, T); lowbounds2 receives interleaved index pairs and values one
 * double per pair.  Offsets are host arrays, the rest device arrays.
 * Asynchronous on `stream` like the 1D call: the host lays the batch out
 * from the offsets, the working memory (prepared axes, corner records,
 * tiles) comes from the stream-ordered allocator, and the preparation, the
 * choice between the lean and the general persistent kernel (made on the
 * GPU: values outside the float-float range or crowded buckets take the
 * general one), the lookup and the release of that memory are queued;
 * R, T, F, Y2, lowbounds2 and values must stay valid until the stream
 * reaches that point.  An axis that is not strictly increasing sets
 * SS_FLAG_NOT_SORTED in *stat (the other tables' results are exact).  Bad
 * offsets are refused with SS_EINVAL naming the table, a stream being
 * captured with SS_EUNSUPPORTED.  The 2D lookup uses side SS_SIDE_LT (the
 * cell of a target equal to an axis entry is the one above it either way,
 * and so is the interpolated value). */
ss_status ss_search_interp_2d_batched(int32_t ntables, const int64_t* R_off, const double* R,
                                      const int64_t* T_off, const double* T, const int64_t* F_off,
                                      const double* F, const int64_t* Y_off, const double* Y2,
                                      int32_t* lowbounds2, double* values, ss_devstat* stat,
                                      cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Batched search without device allocation                                */
/* ---------------------------------------------------------------------- */

/* The paper has no counterpart of this entry point; it exists for callers
 * that may not allocate device memory themselves or through this library:
 * code that works inside a fixed device-memory budget owned by a host
 * framework, loops that cannot take cudaMalloc's implicit synchronisation,
 * plug-ins that leave all device memory management to their host.
 *
 * Same result as a plan without a model (bucket search) over ntables tables:
 * table k is X[X_off[k] .. X_off[k+1]) and its targets Y[Y_off[k] ..
 * Y_off[k+1]) (X_off, Y_off host arrays of ntables+1 entries; X, Y,
 * lowbounds device), answers at the same positions of lowbounds.  It calls
 * no cudaMalloc/cudaFree: prepared tables, tile list and tile counter live in
 * one 8 MiB array inside the library that every GPU loading the library
 * holds until the process exits.  A batch whose working set exceeds 8 MiB is
 * rejected with SS_EINVAL (about 250 tables of 2000 entries fit).  Every
 * call reuses that array and clears what must start at zero, so calls are
 * ordered on the GPU: each call's work waits for the previous call's (on
 * any stream, from any host thread), and calls from different streams run
 * one after another.  The metadata of a call is copied from pageable host
 * memory, so a call on a stream that is being captured is refused with
 * SS_EUNSUPPORTED before anything is queued (the capture stays valid).  The
 * first call on each device looks up the array's device address and creates
 * its event.  Bad offsets (negative, decreasing, a table of fewer than 2 or
 * more than 2^30 entries) are refused with SS_EINVAL naming the table.  A
 * table that is not strictly increasing sets SS_FLAG_NOT_SORTED in *stat;
 * its indices are then unspecified but stay in [0, n-1], and the other
 * tables' indices are unaffected. */
ss_status ss_search_1d_batched_static(int32_t ntables, const int64_t* X_off, const double* X,
                                      const int64_t* Y_off, const double* Y, int32_t* lowbounds,
                                      int32_t side, ss_devstat* stat, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Status and diagnostics                                                  */
/* ---------------------------------------------------------------------- */

/* Wait up to timeout_ms for `stream` to drain (polling, never blocking
 * forever), then copy *stat (device) into *out (host).  SS_ETIMEOUT if the
 * stream is still busy at the deadline; *out is then left untouched. */
ss_status ss_sync_status(cudaStream_t stream, const ss_devstat* stat, ss_devstat* out,
                         int32_t timeout_ms);

/* Bounds-checked build (the library compiled with -DSS_CHECKED; the paper
 * has no counterpart: a debugging aid).  In that build the staging of a
 * table, the wide-section search, the learned windows, the hunt and the
 * searches in global memory check every index against its array; an index
 * outside is not used (the read is skipped), the kernel sets SS_FLAG_BOUNDS
 * in the caller's status record, and the count of such indices is kept on
 * each device.  ss_checked_hits waits for the device, adds the counts of
 * every part of the library into *hits and, if reset is nonzero, clears
 * them.  ss_checked_selftest launches one check of an index that is out of
 * range (no memory is read) so that a test can see the count move.  Both
 * return SS_EUNSUPPORTED in the ordinary build. */
ss_status ss_checked_hits(uint64_t* hits, int32_t reset);
ss_status ss_checked_selftest(void);

/* Message of the last failing call on this host thread ("" if none). */
const char* ss_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t ss_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SIMDSEARCH_H */
