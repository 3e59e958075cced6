// Deterministic block and grid reductions.
//
// A reducing kernel gives every thread W values.  Each CTA sums them with a
// fixed shuffle tree and writes W partials; the last CTA to finish (ticket
// counter) adds all partials in CTA-index order with the same fixed tree and
// calls the finaliser with the W totals.  The result is bitwise reproducible
// run to run for a given launch shape.
#pragma once
#include "msmg_internal.cuh"

namespace msmg {

// Sum of W values over the CTA; the totals are valid in thread 0.
template <int W>
__device__ __forceinline__ void block_sum(double (&v)[W], double* sh /* W * 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    double t = warp_sum(v[w]);
    if (lane == 0) sh[w * 32 + warp] = t;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double t = lane < nwarp ? sh[w * 32 + lane] : 0.0;
      v[w] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Grid-wide deterministic reduction over the nblk CTAs that share ``red``
// (CTA index blk among them); ``fin(totals)`` runs once, in thread 0 of the
// last of them.  Every one of those CTAs must call this exactly once.
template <int W, typename Fin>
__device__ __forceinline__ void grid_reduce_b(double (&v)[W], const RedSlot& red, unsigned blk, unsigned nblk,
                                              Fin fin) {
  __shared__ double sh[W * 32];
  __shared__ int am_last;
  block_sum<W>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) red.partials[(size_t)blk * W + w] = v[w];
    __threadfence();
    unsigned t = atomicAdd(red.counter, 1u);
    am_last = (t == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double acc[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w] = 0.0;
  // (unrolled so that the loads are in flight together; the order of the sums
  // is unchanged)
#pragma unroll 8
  for (unsigned i = threadIdx.x; i < nblk; i += blockDim.x) {
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] += __ldcg(&red.partials[(size_t)i * W + w]);
  }
  block_sum<W>(acc, sh);
  if (threadIdx.x == 0) {
    fin(acc);
    *red.counter = 0u;
    __threadfence();
  }
}

// The same over the whole grid of a launch.
template <int W, typename Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[W], const RedSlot& red, Fin fin) {
  grid_reduce_b<W>(v, red, blockIdx.x, gridDim.x, fin);
}

// Batched form: right-hand side bi.r reduces over its own CTAs into its slice.
template <int W, typename Fin>
__device__ __forceinline__ void grid_reduce_r(double (&v)[W], const RedSlot& red, const BatchIdx& bi, Fin fin) {
  grid_reduce_b<W>(v, red_for(red, bi.r), bi.blk, bi.nblk, fin);
}

}  // namespace msmg
