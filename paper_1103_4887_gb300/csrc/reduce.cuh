// Single-pass deterministic FP64 sums over a grid of kBlock-thread CTAs, for
// the whole-path kernels (action, gradient, HMC energies): each CTA writes
// its fixed-order sums of K values, and the last CTA to arrive (ticket) adds
// the CTA sums -- every thread a fixed stride of CTAs, then a fixed tree -- so
// the result depends only on the grid, not on arrival order.
#pragma once

#include "internal.h"

namespace pimc {

// Fixed-order tree sum over a warp (lane 0 holds the result).
template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ double warp_sum_fp64(double v) { return warp_sum<double>(v); }

// v: this thread's K partial sums.  out[k] (written by thread 0 of the last
// CTA) receives the grid totals; *last tells the caller which CTA that is.
// Uses c.red[cta * kRedStride + k] (K <= kRedStride) and c.ticket.
template <int K>
__device__ void grid_sums_last_block(const Ctx& c, double (&v)[K], double* out, double (*wsum)[kBlock / 32],
                                     int* last)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double w = warp_sum_fp64(v[k]);
        if (lane == 0) wsum[k][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int j = 0; j < kBlock / 32; ++j) t += wsum[k][j];
            c.red[(int64_t)blockIdx.x * kRedStride + k] = t;
        }
        __threadfence();
        *last = (atomicAdd(c.ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (*last) {
        __threadfence();
        double t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += kBlock) {
#pragma unroll
            for (int k = 0; k < K; ++k) t[k] += __ldcg(&c.red[(int64_t)i * kRedStride + k]);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double w = warp_sum_fp64(t[k]);
            if (lane == 0) wsum[k][wid] = w;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 0; k < K; ++k) {
                double s = 0.0;
                for (int j = 0; j < kBlock / 32; ++j) s += wsum[k][j];
                out[k] = s;
            }
            *c.ticket = 0u;
        }
    }
}

}  // namespace pimc
