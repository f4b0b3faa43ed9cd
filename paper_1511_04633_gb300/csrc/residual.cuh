// residual.cuh -- the convergence residual (reading A11 of the paper's
// unstated convergence rule) taken inside a step kernel: each cell compares
// its fields theta, u with the snapshot of the previous residual point,
// refreshes the snapshot, and the block sums the four squared norms
//   |theta - theta_prev|^2, |theta|^2, |u - u_prev|^2, |u|^2
// into one partial per block; residual_finish (aux.cu) adds the partials in
// block order and forms r.
//
// Precision.  A cell's four terms are FP32, formed from the FP32 fields (a
// difference and a square, or three squares added with fused multiply-adds:
// a relative error of at most a few units of 2^-24 per term).  From there
// on every sum is kept in double-float form, an unevaluated pair hi + lo of
// floats added with Knuth's error-free TwoSum (s + e = a + b exactly) and a
// renormalisation (Dekker, Numer. Math. 18, 1971).  That keeps about 48
// significand bits: for the non-negative terms here each addition loses at
// most a few units of 2^-48, so the sums carry the terms' own FP32 error and
// nothing more.  The alternative, FP64 additions from the cell upwards, runs
// on GB300's FP64 pipe at about 1/64 of the FP32 rate; double-float costs a
// few FP32 instructions per cell.  Only the final totals are FP64.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// A double-float number hi + lo with |lo| <= ulp(hi) / 2.
struct DF {
    float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum; no ordering of |a|, |b| needed).
__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    const float e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return {s, e};
}

// Sum of two double-float numbers, renormalised (|e| <= |s| after TwoSum,
// so the closing step is Dekker's FastTwoSum).
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s.hi, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}

__device__ __forceinline__ DF df_shfl_down(DF v, int o)
{
    return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

// Where a step kernel takes a residual point: the snapshot of the previous
// point (4 planes of `cells` floats: theta, u_x, u_y, u_z), refreshed with
// the current fields, and one partial per block (8 floats: hi and lo of the
// four sums) at partials + 8 * (linear block index).  *points (device) is
// the number of points taken since the last reset (0, 1 or 2, kept by the
// finishing kernel); at 0 there is no previous point and the differences
// are taken as zero.  Reading it on the device lets a captured graph serve
// every interval.
struct ResidualArgs {
    float *snap;
    float *partials;
    const double *points;
    unsigned cells;
};

// Index of this block in the (x fastest) grid.
__device__ __forceinline__ unsigned block_linear()
{
    return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
}

// The four FP32 terms of one cell, given its snapshot values prev.
__device__ __forceinline__ void residual_cell_terms(int have_prev, float th, float ux, float uy, float uz,
                                                    const float prev[4], float t[4])
{
    const float now[4] = {th, ux, uy, uz};
    float dv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) dv[k] = have_prev ? __fsub_rn(now[k], prev[k]) : 0.0f;
    t[0] = __fmul_rn(dv[0], dv[0]);
    t[1] = __fmul_rn(th, th);
    t[2] = __fmaf_rn(dv[1], dv[1], __fmaf_rn(dv[2], dv[2], __fmul_rn(dv[3], dv[3])));
    t[3] = __fmaf_rn(ux, ux, __fmaf_rn(uy, uy, __fmul_rn(uz, uz)));
}

// One cell per thread at cell index c.  The kernels load the snapshot with
// their populations (residual_cell_load, so the two round trips to memory
// overlap) and use it after their stores (residual_cell): the four terms go
// into acc and the snapshot takes the current fields.
__device__ __forceinline__ void residual_cell_load(const ResidualArgs &R, unsigned c, float prev[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) prev[k] = R.snap[k * R.cells + c];
}

__device__ __forceinline__ void residual_cell(const ResidualArgs &R, unsigned c, const float prev[4], float th,
                                              float ux, float uy, float uz, DF acc[4])
{
    float t[4];
    residual_cell_terms(*R.points > 0.0, th, ux, uy, uz, prev, t);
    const float now[4] = {th, ux, uy, uz};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        R.snap[k * R.cells + c] = now[k];
        acc[k] = DF{t[k], 0.0f};
    }
}

// Two cells per thread, c and c + 1 (c even: the snapshot planes hold float2
// pairs there), with the fields of lane x (cell c) and lane y (cell c + 1);
// loaded and used as for one cell.
__device__ __forceinline__ void residual_pair_load(const ResidualArgs &R, unsigned c, float2 prev[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) prev[k] = *reinterpret_cast<const float2 *>(R.snap + k * R.cells + c);
}

__device__ __forceinline__ void residual_pair(const ResidualArgs &R, unsigned c, const float2 prev[4], float2 th,
                                              float2 ux, float2 uy, float2 uz, DF acc[4])
{
    const float p0[4] = {prev[0].x, prev[1].x, prev[2].x, prev[3].x};
    const float p1[4] = {prev[0].y, prev[1].y, prev[2].y, prev[3].y};
    float t0[4], t1[4];
    const int have_prev = *R.points > 0.0;
    residual_cell_terms(have_prev, th.x, ux.x, uy.x, uz.x, p0, t0);
    residual_cell_terms(have_prev, th.y, ux.y, uy.y, uz.y, p1, t1);
    const float2 now[4] = {th, ux, uy, uz};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        *reinterpret_cast<float2 *>(R.snap + k * R.cells + c) = now[k];
        acc[k] = df_two_sum(t0[k], t1[k]);
    }
}

// Block sum of the four per-thread sums in a fixed order (a shuffle tree in
// each warp, then the warps in order by warp 0) and the store of the
// block's partial.  Every thread of the block must call it, once; the block
// holds a whole number of warps (at most 32).
__device__ __forceinline__ void residual_block_store(DF acc[4], float *partials)
{
    __shared__ DF sh[32][4];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int nwarps = static_cast<int>(blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] = df_add(acc[k], df_shfl_down(acc[k], o));
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[warp][k] = acc[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            DF w = lane < nwarps ? sh[lane][k] : DF{0.0f, 0.0f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = df_add(w, df_shfl_down(w, o));
            if (lane == 0) {
                float *p = partials + 8 * static_cast<size_t>(block_linear());
                p[2 * k] = w.hi;
                p[2 * k + 1] = w.lo;
            }
        }
    }
}

}  // namespace lbm
