// learned.cuh -- shared pieces of the model kernels: a deterministic block
// reduction of the 65 gradient entries (plus one extra value).
#pragma once

#include "ss_model.cuh"

namespace ss {

// Sums g[0..64] and `extra` over all threads of the block into red[0][0..65]
// (fixed order: warp shuffle tree, then warps in index order).  red must hold
// blockDim.x/32 rows.  Ends with a barrier.
__device__ __forceinline__ void block_reduce_params(float (&g)[kMlpParams], float extra,
                                                    float (*red)[kMlpParams + 1]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k <= kMlpParams; ++k) {
    float v = k < kMlpParams ? g[k] : extra;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if (lane == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x <= kMlpParams) {
    float s = 0.0f;
    for (int i = 0; i < nw; ++i) s += red[i][threadIdx.x];
    red[0][threadIdx.x] = s;
  }
  __syncthreads();
}

}  // namespace ss
