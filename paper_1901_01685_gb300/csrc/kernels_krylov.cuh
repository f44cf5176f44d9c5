// Vector kernels of BiCGSTAB preconditioned by the p-multigrid V-cycle (Sec. 5,
// "p-Multigrid as a preconditioner").  FP64; the updates round every operation
// separately (no fused multiply-add) so that each follows the order of the
// algorithm's steps; dot products use the fixed-partition, fixed-tree
// reduction of the norm kernels (deterministic).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace pmgk {

// partial[b] = sum over block b's fixed chunk of x_i y_i
__global__ void __launch_bounds__(kNormThreads) k_dot_partial(int n, const double* __restrict__ x,
                                                             const double* __restrict__ y,
                                                             double* __restrict__ partial) {
  __shared__ double sh[kNormThreads];
  const long long chunk = (n + (long long)gridDim.x - 1) / gridDim.x;
  const long long beg = blockIdx.x * chunk;
  const long long end = beg + chunk < n ? beg + chunk : n;
  double s = 0.0;
  for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) s += x[i] * y[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// *out = sum of the partials (one block, fixed order)
__global__ void __launch_bounds__(kNormThreads) k_sum_partials(int nparts, const double* __restrict__ partial,
                                                              double* out) {
  __shared__ double sh[kNormThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// p = r + beta (p - omega v)
__global__ void k_bicg_direction(int n, double beta, double omega, const double* __restrict__ r,
                                 const double* __restrict__ v, double* __restrict__ p) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = __dadd_rn(r[i], __dmul_rn(beta, __dsub_rn(p[i], __dmul_rn(omega, v[i]))));
}

// out = x - a y
__global__ void k_sub_scaled(int n, const double* __restrict__ x, double a, const double* __restrict__ y,
                             double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __dsub_rn(x[i], __dmul_rn(a, y[i]));
}

// u = (u + alpha ph) + omega sh   (omega = 0 and sh = null for the half-step exit)
__global__ void k_bicg_solution(int n, double alpha, const double* __restrict__ ph, double omega,
                                const double* __restrict__ sh, double* __restrict__ u) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double t = __dadd_rn(u[i], __dmul_rn(alpha, ph[i]));
    u[i] = sh ? __dadd_rn(t, __dmul_rn(omega, sh[i])) : t;
  }
}

}  // namespace pmgk
