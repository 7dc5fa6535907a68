// Deterministic FP64 block reductions with a last-block finish.
//
// Every reducing kernel is launched with a grid size that depends only on the
// problem size.  Each block reduces its fixed share in a fixed order, writes
// NV partial sums to ``partials[block]``, and the block that finishes last
// (found with one atomic counter, no waiting) sums the partials in index
// order and runs an epilogue on the totals.  The result is therefore the
// same bit for bit from run to run.  The counter is reset by the last block,
// so one scratch area serves every reduction issued on one stream in order.
#pragma once

#include "hdcr_internal.cuh"

namespace hdcr {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1184;  // 8 per SM on a 148..152-SM part; partial buffers sized for this
constexpr int RED_MAX_NV = 4;

struct RedScratch {
  double* partials;       // RED_MAX_BLOCKS * RED_MAX_NV doubles
  unsigned int* counter;  // one unsigned, zero between kernels
};

// grid size for a reduction over n items, independent of the device
inline int red_blocks(long long n) { return num_blocks(n, RED_THREADS * 4, RED_MAX_BLOCKS); }

template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
  __shared__ double sh[NV][RED_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i][warp] = v[i];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = lane < nw ? sh[i][lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    }
  }
  __syncthreads();
}

// Reduce v over the grid.  Returns true in thread 0 of the last block, with
// the grid totals in ``tot``; that thread then runs the caller's epilogue.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], RedScratch rs, double (&tot)[NV]) {
  __shared__ bool is_last;
  block_reduce<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) rs.partials[blockIdx.x * NV + i] = v[i];
    __threadfence();
    const unsigned int t = atomicAdd(rs.counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double w[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) w[i] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) w[i] += __ldcg(rs.partials + b * NV + i);
  block_reduce<NV>(w);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = w[i];
    *rs.counter = 0u;
    return true;
  }
  return false;
}

// Scratch for host-side users of reductions: partial sums, the counter and a
// few device scalars, allocated together.
struct RedBuffers {
  RedScratch rs;
  double* scal;  // device scalars
  int nscal;
  void* base;
};
int red_buffers_alloc(RedBuffers* rb, int nscal);
void red_buffers_free(RedBuffers* rb);

}  // namespace hdcr
