// Deterministic grid reductions: warp shuffles, then one partial per block,
// then the last block to finish (ticket on a self-resetting counter) sums the
// partials in a fixed order.  Results are bitwise reproducible run to run.
#pragma once
#include "sem_internal.cuh"

namespace sem {

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
}

// Block-reduce v (valid in thread 0 afterwards).  blockDim.x must be a multiple of 32.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  warp_sum<NV>(v);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = lane < nw ? sh[q][lane] : 0.0;
    warp_sum<NV>(v);
  }
}

// Write this block's partials; the last block returns true with the grid
// totals in tot (thread 0).  partials holds NV * gridDim.x doubles.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* counter,
                                         double (&tot)[NV]) {
  __shared__ bool am_last;
  block_sum<NV>(v);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[q * nb + blockIdx.x] = v[q];
    __threadfence();
    unsigned int t = atomicInc(counter, (unsigned)nb - 1u);
    am_last = (t == (unsigned)nb - 1u);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double a[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) a[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < NV; ++q) a[q] += __ldcg(partials + q * nb + b);
  block_sum<NV>(a);
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = a[q];
  return true;
}

}  // namespace sem
