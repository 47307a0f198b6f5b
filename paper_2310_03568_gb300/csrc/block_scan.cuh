// Block-wide scans in thread order (forward) and reverse thread order, for an
// associative, not necessarily commutative, operator.
#pragma once

#include "common.cuh"

namespace adc {

// Exclusive scan over the block's threads in increasing thread order.
// Returns x_0 . ... . x_{tid-1}; *total receives the whole block's value.
// `tmp` is shared scratch of THREADS/32 states.  Contains __syncthreads().
template <class Op, int THREADS, typename S>
__device__ __forceinline__ S block_exclusive_fwd(const Op &op, const S &v, S *tmp, S *total) {
    constexpr int NW = THREADS / kWarp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S inc = warp_inclusive_scan(op, v);
    __syncthreads();
    if (lane == kWarp - 1) tmp[warp] = inc;
    __syncthreads();
    S wpre = op.identity();
    for (int w = 0; w < warp; ++w) wpre = op.combine(wpre, tmp[w]);
    S all = wpre;
    for (int w = warp; w < NW; ++w) all = op.combine(all, tmp[w]);
    if (total) *total = all;
    S ex = shfl_up(inc, 1);
    if (lane == 0) ex = op.identity();
    return op.combine(wpre, ex);
}

// Exclusive scan in decreasing thread order: returns x_{tid+1} . ... . x_{THREADS-1}.
template <class Op, int THREADS, typename S>
__device__ __forceinline__ S block_exclusive_rev(const Op &op, const S &v, S *tmp) {
    constexpr int NW = THREADS / kWarp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S inc = v;  // lane l: x_l . x_{l+1} . ... . x_31
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const S dn = shfl_down(inc, o);
        if (lane + o < kWarp) inc = op.combine(inc, dn);
    }
    __syncthreads();
    if (lane == 0) tmp[warp] = inc;
    __syncthreads();
    S wsuf = op.identity();
    for (int w = NW - 1; w > warp; --w) wsuf = op.combine(tmp[w], wsuf);
    S ex = shfl_down(inc, 1);
    if (lane == kWarp - 1) ex = op.identity();
    return op.combine(ex, wsuf);
}

}  // namespace adc
