// Multi-vector kernels of the Krylov methods on FP64 L-vectors (projection
// onto previous solutions, flexible GMRES): dots of one vector against many
// in the unique-dof inner product, linear combinations of many vectors.
#pragma once
#include "sem_internal.cuh"
#include "reduce.cuh"

namespace sem {
namespace {

constexpr int kDotChunk = 8;          // vectors per dot pass

// out[i0 + i] = <V[i0 + i], b> = sum_L V b / mult, i < cnt (fixed-order reduction)
template <int NV>
__global__ void __launch_bounds__(kRedThreads)
k_mdot(int64_t n, const double* const* __restrict__ V, int i0, int cnt,
       const double* __restrict__ b, const float* __restrict__ imult, double* __restrict__ out,
       double* __restrict__ partials, unsigned* __restrict__ counter) {
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  const double* v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = i < cnt ? V[i0 + i] : nullptr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double bq = b[q] * (double)imult[q];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < cnt) acc[i] = fma(v[i][q], bq, acc[i]);
  }
  double tot[NV];
  if (grid_sum<NV>(acc, partials, counter, tot) && threadIdx.x == 0)
    for (int i = 0; i < cnt; ++i) out[i0 + i] = tot[i];
}

// out = base + s sum_{i < cnt} coef[i] V[i]  (base may be NULL or equal out)
__global__ void __launch_bounds__(256)
k_mcomb(int64_t n, const double* const* __restrict__ V, int cnt, const double* __restrict__ coef,
        double s, const double* base, double* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < cnt; ++i) acc = fma(coef[i], V[i][q], acc);
    out[q] = (base ? base[q] : 0.0) + s * acc;
  }
}

// out = a + b, or out = a - b + c
__global__ void k_lin3(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, double sb, double* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = a[q] + sb * b[q] + (c ? c[q] : 0.0);
}

__global__ void k_scale2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                         double s, double* __restrict__ oa, double* __restrict__ ob) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    oa[q] = s * a[q];
    ob[q] = s * b[q];
  }
}

inline int lin_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sem_num_sms()));
}

}  // namespace
}  // namespace sem
