// reduce.cuh -- deterministic FP64 block reductions (warp shuffles in a
// fixed tree; no floating-point atomics) of the Nusselt kernels.  The
// residual's double-float reductions are in residual.cuh.
#pragma once

namespace lbm {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of N values per thread (fixed order).  Every thread of the
// block (THREADS of them, 1-D or 2-D, a multiple of 32) must call it; the
// thread with linear index 0 receives the totals.
template <int N, int THREADS>
__device__ __forceinline__ void block_sum(double (&v)[N])
{
    __shared__ double sh[THREADS / 32][N];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double w = (lane < THREADS / 32) ? sh[lane][k] : 0.0;
            v[k] = warp_sum(w);
        }
    }
    __syncthreads();
}

}  // namespace lbm
