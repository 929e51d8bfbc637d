// learned.cu -- training and inference kernels of the MLP position model,
// exposed for gradient checks (forward, loss+gradient, Adam step), and the
// per-table trainer used by plan creation.
//
// The paper's position maps are analytic (the logarithm hash of Sec. 3.4
// and the exponent hash of Sec. 3.5); the MLP is a learned replacement whose
// output is only a proposal: every index it proposes is verified exactly
// and a failed check falls back to the plain search.
#include <algorithm>

#include "learned.cuh"

namespace ss {

// ---------------------------------------------------------------------------
// Single-block kernels used by the C ABI check entry points.  One block keeps
// the reduction order fixed, so results are deterministic.
// ---------------------------------------------------------------------------
constexpr int kCheckThreads = 512;

__global__ void __launch_bounds__(kCheckThreads) k_mlp_loss_grad(const float* __restrict__ params,
                                                                  const float* __restrict__ x,
                                                                  const float* __restrict__ y, int64_t B,
                                                                  float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float p[kMlpParams];
  __shared__ float red[kCheckThreads / 32][kMlpParams + 1];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  float g[kMlpParams];
#pragma unroll
  for (int k = 0; k < kMlpParams; ++k) g[k] = 0.0f;
  float l = 0.0f;
  const float scale = 1.0f / (float)B;
  for (int64_t i = threadIdx.x; i < B; i += blockDim.x) l += mlp_backward_accum(p, x[2 * i], x[2 * i + 1], y[i], scale, g);
  block_reduce_params(g, l, red);
  if (threadIdx.x < kMlpParams) grad[threadIdx.x] = red[0][threadIdx.x];
  if (threadIdx.x == 0) *loss = red[0][kMlpParams] * scale;
}

__global__ void k_mlp_forward(const float* __restrict__ params, const float* __restrict__ x, int64_t B,
                              float* __restrict__ y) {
  __shared__ float p[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = mlp_forward(p, x[2 * i], x[2 * i + 1]);
}

__global__ void k_adam_step(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, int step, float lr, float b1, float b2, float eps) {
  const int k = threadIdx.x;
  if (k >= kMlpParams) return;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  float p = params[k], a = m1[k], v = m2[k];
  adam_update(p, grad[k], a, v, lr, b1, b2, eps, c1, c2);
  params[k] = p;
  m1[k] = a;
  m2[k] = v;
}

}  // namespace ss

extern "C" {

ss_status ss_mlp_loss_grad(const float* params, const float* x, const float* y, int64_t B, float* grad, float* loss,
                           cudaStream_t stream) {
  if (params == nullptr || grad == nullptr || loss == nullptr || (B > 0 && (x == nullptr || y == nullptr)))
    return ss::fail(SS_EINVAL, "ss_mlp_loss_grad: null pointer");
  if (B <= 0) return ss::fail(SS_EINVAL, "ss_mlp_loss_grad: batch must be > 0");
  ss::k_mlp_loss_grad<<<1, ss::kCheckThreads, 0, stream>>>(params, x, y, B, grad, loss);
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? SS_OK : ss::cuda_fail(err, "k_mlp_loss_grad");
}

ss_status ss_mlp_forward(const float* params, const float* x, int64_t B, float* y, cudaStream_t stream) {
  if (params == nullptr || (B > 0 && (x == nullptr || y == nullptr))) return ss::fail(SS_EINVAL, "ss_mlp_forward: null pointer");
  if (B < 0) return ss::fail(SS_EINVAL, "ss_mlp_forward: batch must be >= 0");
  if (B == 0) return SS_OK;
  const int grid = (int)std::min<int64_t>((B + 255) / 256, (int64_t)ss::num_sms() * 8);
  ss::k_mlp_forward<<<grid, 256, 0, stream>>>(params, x, B, y);
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? SS_OK : ss::cuda_fail(err, "k_mlp_forward");
}

ss_status ss_mlp_adam_step(float* params, const float* grad, float* m1, float* m2, int32_t step, float lr, float beta1,
                           float beta2, float eps, cudaStream_t stream) {
  if (params == nullptr || grad == nullptr || m1 == nullptr || m2 == nullptr)
    return ss::fail(SS_EINVAL, "ss_mlp_adam_step: null pointer");
  if (step < 1) return ss::fail(SS_EINVAL, "ss_mlp_adam_step: step counts from 1");
  ss::k_adam_step<<<1, 96, 0, stream>>>(params, grad, m1, m2, step, lr, beta1, beta2, eps);
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? SS_OK : ss::cuda_fail(err, "k_adam_step");
}

}  // extern "C"
