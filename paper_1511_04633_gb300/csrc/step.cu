// step.cu -- the fused double-MRT time step (arXiv:1511.04633, Eqs. (14),
// (19), (29)): for every cell, pull the 19 + 7 populations from the
// neighbours (wall rules inline), collide both lattices in moment space, add
// the buoyancy force and store the result in the other buffer (A-B scheme).
//
// Layout: 26 planes [q][z][y][x] of float32, x fastest, planes G.plane
// elements apart.  One thread per cell, x along threadIdx.x, so every load of
// a warp is one contiguous 128-byte run (shifted by one element for the
// +-x links) and every store a full aligned run.
#include "internal.h"

namespace lbm {

template <int WALL>
__global__ void __launch_bounds__(256) step_kernel(const float *__restrict__ src,
                                                   float *__restrict__ dst, const Geometry G,
                                                   const CollideParams C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= G.nx || y >= G.ny) return;
    float d[19], g[7];
    pull_f<WALL>(src, G, x, y, z, d);
    pull_g<WALL>(src, G, x, y, z, g);
    collide_cell(C, d, g);
    const int self = (z * G.ny + y) * G.nx + x;
    const long long P = G.plane;
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        dst[i * P + self] = d[i];
    });
    static_for<0, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        dst[(19 + i) * P + self] = g[i];
    });
}

cudaError_t launch_step(int wall, const float *src, float *dst, const Geometry &G,
                        const CollideParams &C, BlockShape b, cudaStream_t s)
{
    dim3 block(b.bx, b.by, 1);
    dim3 grid((G.nx + b.bx - 1) / b.bx, (G.ny + b.by - 1) / b.by, G.nz);
    switch (wall) {
    case 0: step_kernel<0><<<grid, block, 0, s>>>(src, dst, G, C); break;
    case 1: step_kernel<1><<<grid, block, 0, s>>>(src, dst, G, C); break;
    case 2: step_kernel<2><<<grid, block, 0, s>>>(src, dst, G, C); break;
    case 3: step_kernel<3><<<grid, block, 0, s>>>(src, dst, G, C); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm
