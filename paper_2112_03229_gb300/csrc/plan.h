// plan.h -- structures shared by the plan's host code and its kernels.
#pragma once

#include "ss_plan.cuh"

namespace ss {

__host__ __device__ inline BlobGeom blob_geom_dev(int n, int dir_cap, bool cells) {
  BlobGeom g{};
  const int nk = n - 1;
  g.stride = 1;
  while ((nk + g.stride - 1) / g.stride > kMaxSmemKeys) g.stride <<= 1;
  g.ns = (nk + g.stride - 1) / g.stride;
  g.P = ceil_pow2(g.ns + 1);
  g.D = ilog2(g.P);
  int off = (int)sizeof(BlobHdr);
  g.off_mlp = off;  off += kMlpBytes;
  g.off_dir = off;  off += (((dir_cap + 1) * 2) + 15) & ~15;   // 16-bit counts (staged keys <= 8128)
  g.off_keys = off; off += (g.ns + kPad) * 8;
  g.off_eyt = off;  off += g.P * 8;
  g.off_cells = -1;
  if (cells) { off = (off + 15) & ~15; g.off_cells = off; off += (((n - 1) * kCellBytes) + 15) & ~15; }   // 16-byte aligned cell table
  g.staged_end = off;
  g.off_full = g.stride > 1 ? off : -1;
  g.bytes = g.stride > 1 ? wide_offset(off, nk) : ((off + 15) & ~15);
  g.off_wide = -1;
  if (!cells && g.stride > 1 && wide_eligible(nk)) {   // 1D tables only
    g.off_wide = g.bytes;
    g.bytes += wide_geom(nk).bytes;
  }
  return g;
}

struct Tile {            // a contiguous run of targets of one table
  int table;
  int count;
  int64_t begin;         // index of the first target (pair for 2D) in Y / out
};

struct PrepArgs {
  int ntables;
  const int64_t* X_off;  // device
  const double* X;
  unsigned char* blobs;
  const int64_t* blob_off;
  const int* dir_cap;
  const int* algo;
  int cells;
  unsigned* bad_flag;
};

struct TrainArgs {
  int ntables;
  unsigned char* blobs;
  const int64_t* blob_off;
  int epochs;
  float lr;
  uint64_t seed;
};

struct WindowArgs {
  int ntables;
  unsigned char* blobs;
  const int64_t* blob_off;
  uint64_t seed;
};

struct BatchArgs1D {
  const unsigned char* blobs;
  const int64_t* blob_off;
  const Tile* tiles;
  int ntiles;
  int* counter;
  const double* Y;
  int32_t* out;
  int vec;               // 1: Y and out 16-byte aligned (128-bit loads); 2: Y also 32-byte aligned (256-bit)
  ss_devstat* stat;
};

struct BatchArgs2D {
  const unsigned char* blobs;
  const int64_t* blob_off;      // [2*ntables]: rho axis, T axis
  const float4* cells;          // per cell of every table: two float4 = four float-float corners
  const double* grid64;         // the caller's fp64 values, row-major (fallback)
  const int64_t* grid_off;      // [ntables] value offsets of grid64
  const int64_t* cell_off;      // [ntables] cell offsets of cells (in cells)
  int extrap;                   // 1: linear extrapolation (pairs outside an axis in fp64, unclamped)
  int logspace;                 // 1: weights in natural-log coordinates (every pair in fp64)
  const Tile* tiles;
  int ntiles;
  int* counter;
  const double* Y2;
  int32_t* idx;
  double* val;
  int vec;
  ss_devstat* stat;
};

__global__ void k_prep_1d(PrepArgs a);
__global__ void k_train_mlp(TrainArgs a);
__global__ void k_window(WindowArgs a);
const void* batched_1d_kernel(bool le, int family);   // family: 0 plain, 1 +spline/loghash, 2 +mlp, 3 hunt
const void* batched_2d_fast_kernel(int algo, bool hunt = false);   // the lean 2D kernel for axes searched by
                                                       // algo (bucket, spline, mlp or loghash; see k_fast_2d_check),
                                                       // or its hunt instance (bucket axes)
__global__ void k_fast_2d_check(const unsigned char* __restrict__ blobs, const int64_t* __restrict__ blob_off,
                                int naxes, int algo, unsigned* not_fast);
const void* batched_1d_wide_kernel(bool le);          // tables searched through their wide section
constexpr int kWideThreads = 1024;
const void* batched_2d_kernel(bool hunt, bool learned);   // hunt: second pair of a thread starts from the first; learned: position models compiled in
__global__ void k_grid_to_ff(const double* F, float2* G, int64_t count, unsigned* bad);
__global__ void k_prep_cells(PrepArgs a);

}  // namespace ss
