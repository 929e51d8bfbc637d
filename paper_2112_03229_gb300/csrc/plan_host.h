// plan_host.h -- the host-side plan object and the helpers shared by the
// plan translation units.
#pragma once

#include <string>
#include <vector>

#include "plan.h"

namespace ss {

constexpr int kNumBuckets = 8;       // table-size buckets: [2,16) [16,64) [64,256) ... [65536, inf)
constexpr int kDefaultTile = 16384;  // targets per tile before tuning

int size_bucket(int n);
const char* algo_name(int a);
int algo_from_name(const std::string& s);
int staged_bytes(int n, int dir_cap, bool cells, int algo);
int initial_algo(const ss_plan_opts& o);
ss_status check_plan_opts(const ss_plan_opts& o, int kind);   // kind 1: 1D plan, 2: 2D plan
std::vector<Tile> make_tiles(const std::vector<int64_t>& Y_off, const std::vector<int>& bucket_of,
                             const int* bucket_tile, int64_t& total);
int auto_tile(int64_t total, int blocks, int staged_bytes, float mult);
void free_dev(void* p);

struct PlanBase {
  virtual ~PlanBase();
  int kind = 0;                       // 1: 1D tables, 2: 2D tables
  int ntables = 0;
  ss_plan_opts opts{};
  std::vector<int> sizes;             // 1D: n per table; 2D: nr per table
  std::vector<int> sizes_t;           // 2D: nt per table
  std::vector<int64_t> X_off;
  std::vector<int> dir_cap;           // per blob
  std::vector<int> algo;              // per blob (BlobAlgo)
  std::vector<int64_t> blob_off;      // per blob
  int64_t blob_bytes = 0;
  unsigned char* d_blobs = nullptr;
  int64_t* d_blob_off = nullptr;
  // 2D value grids: per cell its four corners as float-float (CellCorners,
  // cell offsets cell_off), and the caller's fp64 grids, row-major (grid_off),
  // kept only when some value needs the fp64 blend
  float2* d_grid = nullptr;
  double* d_grid64 = nullptr;
  int64_t* d_grid_off = nullptr;
  int64_t* d_cell_off = nullptr;
  std::vector<int64_t> grid_off;
  std::vector<int64_t> cell_off;
  // autotuner choices per table-size bucket
  int bucket_algo[kNumBuckets] = {0};
  int bucket_tile[kNumBuckets] = {0};      // targets per tile used by the bound batch
  float bucket_mult[kNumBuckets] = {1, 1, 1, 1, 1, 1, 1, 1};   // tuned multiple of the automatic tile
  int bucket_tables[kNumBuckets] = {0};
  int tuned = 0;
  // bound batch
  bool bound = false;
  Tile* d_tiles = nullptr;
  int64_t ntiles = 0;
  int* d_counter = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  int grid_blocks = 0;
  int kernels = 0;                    // kernels in the bound graph
  int smem_bytes = 0;
  int threads = 0;                    // threads per block of the bound batched kernel
  int lean = 0;                       // 2D: the bound batch runs the lean kernel (every axis on the common path)
  // diagnostics
  int64_t device_bytes = 0;
  int max_window = 0;
  float mean_window = 0.0f;
  float train_loss = 0.0f;
  int max_occupancy = 0;              // most keys in one bucket over the tables staged whole
};

// A batched 1D search in one caller-provided device buffer (batched_work.cu):
// per table its directory budget, algorithm (the bucket search) and blob
// offset, the tiles, and the byte offsets of each part inside the buffer.
struct BatchWork1D {
  std::vector<int> caps, algo;
  std::vector<int64_t> blob_off;
  std::vector<Tile> tiles;
  int smem = 0;
  int64_t counter = 0, flag = 0, xoff = 0, boff = 0, caps_off = 0, algo_off = 0, tiles_off = 0, blobs_off = 0, end = 0;
};
// Host checks of the offsets (each bad one refused with a message naming the
// table) and the layout; nothing is queued.
ss_status batch_work_1d(const char* me, int32_t ntables, const int64_t* X_off, const int64_t* Y_off,
                        int dir_cap_max, BatchWork1D& w);
// Metadata copies, table preparation and the persistent search, queued on stream.
ss_status queue_work_1d(const BatchWork1D& w, unsigned char* base, int32_t ntables, const int64_t* X_off,
                        const double* X, const double* Y, int32_t* lowbounds, int32_t side, ss_devstat* stat,
                        cudaStream_t stream);

// The batched 2D lookup in one call, laid out and queued like the 1D one;
// both persistent kernels are queued and the GPU picks the one that applies.
struct BatchWork2D {
  std::vector<int> caps_r, caps_t, algo;
  std::vector<int64_t> blob_off, off_r, off_t, cell_off;
  std::vector<Tile> tiles;
  int smem = 0;
  int64_t counters = 0, gate = 0, flag = 0, xr = 0, xt = 0, fo = 0, bo = 0, ro = 0, to = 0, cr = 0, ct = 0,
          al = 0, co = 0, tiles_off = 0, blobs_off = 0, cells_off = 0, end = 0;
};
ss_status batch_work_2d(const char* me, int32_t ntables, const int64_t* R_off, const int64_t* T_off,
                        const int64_t* F_off, const int64_t* Y_off, BatchWork2D& w);
ss_status queue_work_2d(const BatchWork2D& w, unsigned char* base, int32_t ntables, const int64_t* R_off,
                        const double* R, const int64_t* T_off, const double* T, const int64_t* F_off, const double* F,
                        const double* Y2, int32_t* lowbounds2, double* values, ss_devstat* stat, cudaStream_t stream);
// Tile cap of a 2D batch so that the corner records in flight fit a sixth
// of L2 (0: the batch's records fit there, no cap).
int tile_cap_2d(double pairs, double rec, int resident, int l2);
__global__ void k_grid_cells(const double* __restrict__ F, const int64_t* __restrict__ F_off,
                             const int64_t* __restrict__ R_off, const int64_t* __restrict__ T_off,
                             const int64_t* __restrict__ cell_off, float4* __restrict__ cells, unsigned* bad);

ss_status plan_build_1d(ss_plan* p, const double* X, cudaStream_t stream);
ss_status plan_build_2d(ss_plan* p, const double* R, const double* T, const double* F, cudaStream_t stream);
ss_status plan_bind(ss_plan* p, const std::vector<int64_t>& Y_off, const double* Y, int32_t* out, double* val,
                    ss_devstat* stat, cudaStream_t stream);
ss_status plan_set_algos(ss_plan* p, cudaStream_t stream);
ss_status plan_tune(ss_plan* p, cudaStream_t stream);
ss_status plan_window_stats(ss_plan* p);
void plan_cell_offsets(PlanBase* p);   // cell_off from the axis sizes (2D)

}  // namespace ss

struct ss_plan : public ss::PlanBase {};
