// The conventional least-squares misfit the paper sets the EMD against (Sec. 2.1,
// f_L2 = 1/2 integral (Pcal - Pobs)^2 dx dt) and its adjoint source (Sec. 2.3,
// d f_L2 / d Pcal = Pcal - Pobs), discretised with the cell area: one streaming pass that
// writes area * (Pcal - Pobs) (and its negative) and sums (Pcal - Pobs)^2 in FP64.
#pragma once

#include "emd_kernels.cuh"

namespace emd {

__global__ void __launch_bounds__(kThreads)
    k_lsd(const float *__restrict__ p_obs, const float *__restrict__ p_pred, size_t n, float area,
          float *__restrict__ grad_pred, float *__restrict__ grad_obs, double *acc) {
  double s = 0.0;
  for (size_t i = static_cast<size_t>(blockIdx.x) * kThreads + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * kThreads) {
    const float d = p_pred[i] - p_obs[i];
    s += static_cast<double>(d) * static_cast<double>(d);
    if (grad_pred) grad_pred[i] = area * d;
    if (grad_obs) grad_obs[i] = -area * d;
  }
  __shared__ double red[kThreads / 32];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    atomicAdd(acc, t);
  }
}

}  // namespace emd
