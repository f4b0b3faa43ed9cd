// reduce.cuh -- deterministic block reductions (warp shuffles in a fixed
// tree; no floating-point atomics), shared by the residual and Nusselt
// kernels.
#pragma once

namespace lbm {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
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

// Block-wide sums of N FP32 values per thread: a fixed FP32 shuffle tree
// within each warp (32 values), then FP64 across the block's warps.  FP64 is
// a narrow pipe on GB300 (about 1/64 of the FP32 rate), so FP64 arithmetic
// per cell would bound a kernel that is otherwise a pass over memory; here it
// costs a few operations per warp.  Every thread of the block (THREADS of
// them, a multiple of 32) must call it; thread 0 receives the totals in out.
template <int N, int THREADS>
__device__ __forceinline__ void block_sum_f32(const float (&v)[N], double (&out)[N])
{
    __shared__ double sh[THREADS / 32][N];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    float w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[warp][k] = static_cast<double>(w[k]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = 0.0;
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = warp_sum((lane < THREADS / 32) ? sh[lane][k] : 0.0);
    }
    __syncthreads();
}

}  // namespace lbm
