// reduce.cuh -- deterministic grid reductions of the vector kernels.
//
// Every reduction runs on a fixed grid (vec_grid of the vector length): each
// CTA reduces its threads' values in a fixed order and writes one partial per
// sum; the last CTA to finish (ticket counter) adds the partials in CTA order.
// The same input therefore gives the same bits on every run.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace sem {

// Reduce NS per-thread values over the grid; the last CTA writes out[s].
template <int NS>
__device__ void grid_reduce(double (&v)[NS], double *__restrict__ partials,
                            unsigned int *__restrict__ counter, double *const *out) {
  __shared__ double sh[NS][kVecThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int q = 0; q < kVecThreads / 32; ++q) x += sh[s][q];
      partials[(size_t)blockIdx.x * NS + s] = x;
    }
    __threadfence();
    unsigned int ticket = atomicAdd(counter, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      x += __ldcg(&partials[(size_t)b * NS + s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int q = 0; q < kVecThreads / 32; ++q) x += sh[s][q];
      *out[s] = x;
    }
    *counter = 0u;
  }
}

template <int NS>
struct OutPtrs {
  double *p[NS];
};

}  // namespace sem
