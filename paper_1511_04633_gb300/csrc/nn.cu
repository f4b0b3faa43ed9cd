// nn.cu -- kernels of the warm-start surrogate: a 3-D convolutional U-Net
// that maps a cavity's parameters (Ra, wall type) to an approximate steady
// state (u, v, w, theta).  Forward and backward passes, the loss and the
// Adam update are all here; surrogate.cu strings them together.
//
// Layout: activations channels-last [n][z][y][x][c] (c fastest), weights of a
// k^3 convolution [tap][cout][cin] (cin fastest), taps ordered
// (dz, dy, dx) with dx fastest, each in -(k/2)..(k/2); zero padding.  The
// storage type of activations and weights is float or bfloat16 (T); every
// sum accumulates in FP32; gradients are FP32.  Every reduction runs in a
// fixed order (per-block partials, then an ordered finishing pass), so the
// training is bitwise repeatable.
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "internal.h"
#include "nn.h"
#include "umma.cuh"

namespace lbm {
namespace nn {

namespace {

template <typename T>
__device__ __forceinline__ float ldf(const T *p);
template <>
__device__ __forceinline__ float ldf<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <typename T>
__device__ __forceinline__ void stf(T *p, float v);
template <>
__device__ __forceinline__ void stf<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

constexpr float kSlope = 0.1f;  // leaky ReLU

// ---------------------------------------------------------------- convolution

// Direct convolution, one block per (sample, z, 8 x 8 tile of (y, x), group
// of 32 output channels).  The input tile with its halo and the weights of
// the group are staged in shared memory 8 input channels at a time; each of
// the 256 threads owns 2 voxels x 4 output channels (64 x 32 / 256).
constexpr int kTile = 8;
constexpr int kCoTile = 32;
constexpr int kCiChunk = 8;

template <typename TI, typename TW, typename TO, int K>
__global__ void __launch_bounds__(256) conv3d_kernel(const TI *__restrict__ x, const TW *__restrict__ w,
                                                     const float *__restrict__ bias,
                                                     TO *__restrict__ y, int n, int cin, int cout,
                                                     int act)
{
    constexpr int R = K / 2;
    constexpr int H = kTile + 2 * R;  // halo tile edge
    __shared__ float xs[K][H][H][kCiChunk];
    // weights padded to 9 per output channel: the 8 channel groups of a warp
    // then hit 8 different banks
    __shared__ float ws[K * K * K][kCoTile][kCiChunk + 1];
    const int tiles = n / kTile;
    int bid = blockIdx.x;
    const int tx0 = (bid % tiles) * kTile;
    bid /= tiles;
    const int ty0 = (bid % tiles) * kTile;
    bid /= tiles;
    const int z = bid % n;
    const int b = bid / n;
    const int co0 = blockIdx.y * kCoTile;
    const int t = threadIdx.x;
    // thread -> 2 voxels (vx, vx + 32 in the flattened 8 x 8 tile) x 4 channels
    const int cg = t & 7;          // channel group: channels co0 + cg*4 .. +3
    const int v0 = t >> 3;         // 0..31
    float acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const long long plane = static_cast<long long>(n) * n;
    const TI *xb = x + static_cast<long long>(b) * n * plane * cin;
    for (int ci0 = 0; ci0 < cin; ci0 += kCiChunk) {
        // stage the input halo tile for channels ci0 .. ci0 + 7
        for (int e = t; e < K * H * H * kCiChunk; e += 256) {
            const int c = e % kCiChunk;
            int r = e / kCiChunk;
            const int hx = r % H;
            r /= H;
            const int hy = r % H;
            const int hz = r / H;
            const int gz = z + hz - R, gy = ty0 + hy - R, gx = tx0 + hx - R;
            float v = 0.f;
            if (gz >= 0 && gz < n && gy >= 0 && gy < n && gx >= 0 && gx < n && ci0 + c < cin)
                v = ldf(xb + ((static_cast<long long>(gz) * n + gy) * n + gx) * cin + ci0 + c);
            xs[hz][hy][hx][c] = v;
        }
        for (int e = t; e < K * K * K * kCoTile * kCiChunk; e += 256) {
            const int c = e % kCiChunk;
            int r = e / kCiChunk;
            const int co = r % kCoTile;
            const int tap = r / kCoTile;
            float v = 0.f;
            if (co0 + co < cout && ci0 + c < cin)
                v = ldf(w + (static_cast<long long>(tap) * cout + co0 + co) * cin + ci0 + c);
            ws[tap][co][c] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int tap = 0; tap < K * K * K; ++tap) {
            const int dz = tap / (K * K), dy = (tap / K) % K, dx = tap % K;
#pragma unroll
            for (int c = 0; c < kCiChunk; ++c) {
                float xv[2], wv[4];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int v = v0 + 32 * i;
                    xv[i] = xs[dz][(v >> 3) + dy][(v & 7) + dx][c];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = ws[tap][cg * 4 + j][c];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], wv[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int v = v0 + 32 * i;
        const int gy = ty0 + (v >> 3), gx = tx0 + (v & 7);
        TO *yo = y + (((static_cast<long long>(b) * n + z) * n + gy) * n + gx) * cout;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int co = co0 + cg * 4 + j;
            if (co >= cout) continue;
            float r = acc[i][j] + (bias ? bias[co] : 0.f);
            if (act) r = r > 0.f ? r : kSlope * r;
            stf(yo + co, r);
        }
    }
}

// Tensor-core convolution for bfloat16 inputs and weights (implicit GEMM
// with mma.sync m16n8k16, FP32 accumulation).  One block of 4 warps per
// (sample, z, 8 x 8 tile of (y, x), 32 output channels): GEMM rows are the
// 64 voxels of the tile, columns the 32 channels, and the reduction runs
// over taps x input channels in chunks of 16.  The input halo tile and the
// weights of one z-plane of taps are staged in shared memory with 24-element
// strides per voxel / channel, which keeps the fragment loads free of bank
// conflicts (8 rows x 12 words cover the 32 banks).  Warp w owns tile rows
// 16w..16w+15 (two y-rows of 8 voxels) and all 4 column tiles.
constexpr int kMmaStride = 24;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                               unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int K, typename TO>
__global__ void __launch_bounds__(128) conv3d_mma_kernel(const __nv_bfloat16 *__restrict__ x,
                                                         const __nv_bfloat16 *__restrict__ w,
                                                         const float *__restrict__ bias,
                                                         TO *__restrict__ y, int n, int cin, int cout,
                                                         int act)
{
    constexpr int R = K / 2;
    constexpr int H = kTile + 2 * R;
    __shared__ __align__(16) __nv_bfloat16 xs[K][H][H][kMmaStride];
    __shared__ __align__(16) __nv_bfloat16 ws[K * K][kCoTile][kMmaStride];
    const int tiles = n / kTile;
    int bid = blockIdx.x;
    const int tx0 = (bid % tiles) * kTile;
    bid /= tiles;
    const int ty0 = (bid % tiles) * kTile;
    bid /= tiles;
    const int z = bid % n;
    const int b = bid / n;
    const int co0 = blockIdx.y * kCoTile;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = lane >> 2, tig = lane & 3;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    const long long plane = static_cast<long long>(n) * n;
    const __nv_bfloat16 *xb = x + static_cast<long long>(b) * n * plane * cin;
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (int ci0 = 0; ci0 < cin; ci0 += 16) {
        // input halo tile: 16-byte granules of 8 channels
        for (int e = t; e < K * H * H * 2; e += 128) {
            const int half = e & 1;
            int r = e >> 1;
            const int hx = r % H;
            r /= H;
            const int hy = r % H;
            const int hz = r / H;
            const int gz = z + hz - R, gy = ty0 + hy - R, gx = tx0 + hx - R;
            const int c = ci0 + 8 * half;
            uint4 v = zero4;
            if (gz >= 0 && gz < n && gy >= 0 && gy < n && gx >= 0 && gx < n && c < cin)
                v = *reinterpret_cast<const uint4 *>(xb + ((static_cast<long long>(gz) * n + gy) * n + gx) * cin + c);
            *reinterpret_cast<uint4 *>(&xs[hz][hy][hx][8 * half]) = v;
        }
        for (int tz = 0; tz < K; ++tz) {
            __syncthreads();  // previous plane's weights fully consumed
            for (int e = t; e < K * K * kCoTile * 2; e += 128) {
                const int half = e & 1;
                int r = e >> 1;
                const int co = r % kCoTile;
                const int tp = r / kCoTile;
                const int c = ci0 + 8 * half;
                uint4 v = zero4;
                if (co0 + co < cout && c < cin)
                    v = *reinterpret_cast<const uint4 *>(
                        w + (static_cast<long long>(tz * K * K + tp) * cout + co0 + co) * cin + c);
                *reinterpret_cast<uint4 *>(&ws[tp][co][8 * half]) = v;
            }
            __syncthreads();
#pragma unroll
            for (int tp = 0; tp < K * K; ++tp) {
                const int ty = tp / K, tx = tp % K;
                // A: rows g (voxel (2 warp, g)) and g + 8 (voxel (2 warp + 1, g))
                const __nv_bfloat16 *r0 = &xs[tz][2 * warp + ty][g + tx][0];
                const __nv_bfloat16 *r1 = &xs[tz][2 * warp + 1 + ty][g + tx][0];
                unsigned a[4];
                a[0] = *reinterpret_cast<const unsigned *>(r0 + 2 * tig);
                a[1] = *reinterpret_cast<const unsigned *>(r1 + 2 * tig);
                a[2] = *reinterpret_cast<const unsigned *>(r0 + 2 * tig + 8);
                a[3] = *reinterpret_cast<const unsigned *>(r1 + 2 * tig + 8);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const __nv_bfloat16 *wc = &ws[tp][8 * j + g][0];
                    const unsigned b0 = *reinterpret_cast<const unsigned *>(wc + 2 * tig);
                    const unsigned b1 = *reinterpret_cast<const unsigned *>(wc + 2 * tig + 8);
                    mma_bf16_16816(acc[j], a, b0, b1);
                }
            }
        }
        __syncthreads();  // xs consumed before the next chunk overwrites it
    }
    // epilogue: c0, c1 -> row g; c2, c3 -> row g + 8; columns 2 tig, 2 tig + 1
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int gy = ty0 + 2 * warp + half, gx = tx0 + g;
        TO *yo = y + (((static_cast<long long>(b) * n + z) * n + gy) * n + gx) * cout;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int co = co0 + 8 * j + 2 * tig + q;
                if (co >= cout) continue;
                float r = acc[j][2 * half + q] + (bias ? bias[co] : 0.f);
                if (act) r = r > 0.f ? r : kSlope * r;
                stf(yo + co, r);
            }
        }
    }
}

// Tensor-core weight gradient for bfloat16 inputs and output gradients:
// dw[tap][co][ci] = sum over voxels v of dy[v][co] x[v + tap][ci] is a GEMM
// with M = output channels, N = input channels and K = voxels.  One block of
// 4 warps per (tap, group of 64 output channels, group of 32 input channels,
// chunk of voxels); each stage stages 64 voxels of dy and of the shifted x
// transposed ([channel][voxel], 72-element rows: conflict-free fragment
// loads), then every warp runs 4 k-steps x 4 mma for its 16 output channels.
// Partial sums per chunk go to partials[chunk][tap][co][ci].
constexpr int kWgVox = 64;
constexpr int kWgRow = kWgVox + 8;

template <int K>
__global__ void __launch_bounds__(128) wgrad_mma_kernel(const __nv_bfloat16 *__restrict__ x,
                                                        const __nv_bfloat16 *__restrict__ dy,
                                                        float *__restrict__ partials, int batch, int n,
                                                        int cin, int cout, int chunk, int co_groups)
{
    constexpr int R = K / 2;
    constexpr int TAPS = K * K * K;
    __shared__ __align__(16) __nv_bfloat16 sa[64][kWgRow];  // dy^T: [co][voxel]
    __shared__ __align__(16) __nv_bfloat16 sb[32][kWgRow];  // x_tap^T: [ci][voxel]
    int bid = blockIdx.x;
    const int tap = bid % TAPS;
    bid /= TAPS;
    const int cog = bid % co_groups;
    const int cig = bid / co_groups;
    const int co0 = cog * 64, ci0 = cig * 32;
    const int dz = tap / (K * K) - R, dyo = (tap / K) % K - R, dx = tap % K - R;
    const long long total = static_cast<long long>(batch) * n * n * n;
    const long long v_begin = static_cast<long long>(blockIdx.y) * chunk;
    const long long v_end = v_begin + chunk < total ? v_begin + chunk : total;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = lane >> 2, tig = lane & 3;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (long long vb = v_begin; vb < v_end; vb += kWgVox) {
        // dy granules: 64 voxels x 8 granules of 8 output channels
        for (int e = t; e < kWgVox * 8; e += 128) {
            const int vi = e >> 3, gr = e & 7;
            const int co = co0 + 8 * gr;
            uint4 v = zero4;
            if (vb + vi < v_end && co < cout)
                v = *reinterpret_cast<const uint4 *>(dy + (vb + vi) * cout + co);
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q) sa[8 * gr + q][vi] = h[q];
        }
        // x granules at the voxel shifted by the tap: 64 voxels x 4 granules
        for (int e = t; e < kWgVox * 4; e += 128) {
            const int vi = e >> 2, gr = e & 3;
            const int ci = ci0 + 8 * gr;
            uint4 v = zero4;
            if (vb + vi < v_end && ci < cin) {
                long long r = vb + vi;
                const int gx = static_cast<int>(r % n);
                r /= n;
                const int gy = static_cast<int>(r % n);
                r /= n;
                const int gz = static_cast<int>(r % n);
                const long long bb = r / n;
                const int sz = gz + dz, sy = gy + dyo, sx = gx + dx;
                if (sz >= 0 && sz < n && sy >= 0 && sy < n && sx >= 0 && sx < n)
                    v = *reinterpret_cast<const uint4 *>(x + (((bb * n + sz) * n + sy) * n + sx) * cin + ci);
            }
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q) sb[8 * gr + q][vi] = h[q];
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kWgVox / 16; ++ks) {
            const __nv_bfloat16 *r0 = &sa[16 * warp + g][16 * ks];
            const __nv_bfloat16 *r1 = &sa[16 * warp + g + 8][16 * ks];
            unsigned a[4];
            a[0] = *reinterpret_cast<const unsigned *>(r0 + 2 * tig);
            a[1] = *reinterpret_cast<const unsigned *>(r1 + 2 * tig);
            a[2] = *reinterpret_cast<const unsigned *>(r0 + 2 * tig + 8);
            a[3] = *reinterpret_cast<const unsigned *>(r1 + 2 * tig + 8);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const __nv_bfloat16 *bc = &sb[8 * j + g][16 * ks];
                const unsigned b0 = *reinterpret_cast<const unsigned *>(bc + 2 * tig);
                const unsigned b1 = *reinterpret_cast<const unsigned *>(bc + 2 * tig + 8);
                mma_bf16_16816(acc[j], a, b0, b1);
            }
        }
        __syncthreads();
    }
    float *out = partials + (static_cast<long long>(blockIdx.y) * TAPS + tap) * cout * cin;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int co = co0 + 16 * warp + g + (q >> 1) * 8;
            const int ci = ci0 + 8 * j + 2 * tig + (q & 1);
            if (co < cout && ci < cin) out[static_cast<long long>(co) * cin + ci] = acc[j][q];
        }
}

// Tensor-core weight gradient of a 3^3 convolution, all 27 taps per block:
// dw[tap][co][ci] = sum over voxels v of dy[v][co] x[v + tap][ci].  A block
// owns 16 output x 16 input channels and a run of 8 x 8 x 4 voxel tiles of
// one sample.  Per tile it stages dy (256 voxels) and the x halo (10 x 10 x 6
// voxels) once, unmodified (channels-last rows padded to 24 elements, which
// keeps the 8 rows of every ldmatrix conflict-free), and every tap reads the
// shifted x rows straight from the halo: ldmatrix takes one row address per
// thread, so the shift costs nothing.  The transposed 8 x 8 loads
// (ldmatrix .trans) turn the channels-last rows into the A = dy^T (co x
// voxels) and B = x_tap (voxels x ci) fragments of mma.m16n8k16.  Warp w
// accumulates taps w, w + 8, w + 16 (and w + 24 < 27) for both 8-channel
// halves of ci: 6 or 8 accumulator tiles.  The block's sums over its tiles go
// to partials[chunk][tap][co][ci], summed in chunk order afterwards.
constexpr int kWtX = 8, kWtY = 8, kWtZ = 4;                  // voxel tile
constexpr int kWtHX = kWtX + 2, kWtHY = kWtY + 2, kWtHZ = kWtZ + 2;
constexpr int kWtVox = kWtX * kWtY * kWtZ;                   // 256
constexpr int kWtHalo = kWtHX * kWtHY * kWtHZ;               // 600
constexpr int kWtRow = 24;                                   // bf16 per staged row

__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], const void *p)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__global__ void __launch_bounds__(256) wgrad_taps_kernel(const __nv_bfloat16 *__restrict__ x,
                                                         const __nv_bfloat16 *__restrict__ dy,
                                                         float *__restrict__ partials, int n,
                                                         int cin, int cout, int tiles_per_sample,
                                                         int total_tiles, int tiles_per_block)
{
    __shared__ __align__(16) __nv_bfloat16 xs[kWtHalo][kWtRow];
    __shared__ __align__(16) __nv_bfloat16 gs[kWtVox][kWtRow];
    const int ci_tiles = cin > 8 ? cin / 16 : 1;
    const int co0 = (blockIdx.x / ci_tiles) * 16, ci0 = (blockIdx.x % ci_tiles) * 16;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int ntap = warp + 24 < 27 ? 4 : 3;
    float acc[4][2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const int tx_n = n / kWtX, ty_n = n / kWtY;
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    // ldmatrix row of this thread: matrix j = lane / 8, row r = lane % 8
    const int mj = lane >> 3, mr = lane & 7;
    const int t_begin = blockIdx.y * tiles_per_block;
    const int t_end = min(t_begin + tiles_per_block, total_tiles);
    for (int tile = t_begin; tile < t_end; ++tile) {
        const int b = tile / tiles_per_sample;
        int r = tile % tiles_per_sample;
        const int x0 = (r % tx_n) * kWtX;
        r /= tx_n;
        const int y0 = (r % ty_n) * kWtY;
        const int z0 = (r / ty_n) * kWtZ;
        const long long sample = static_cast<long long>(b) * n * n * n;
        // x halo: 600 voxels x 2 granules of 8 channels (zero outside the
        // grid and beyond cin)
        for (int e = t; e < kWtHalo * 2; e += 256) {
            const int half = e & 1, h = e >> 1;
            const int hx = h % kWtHX, hy = (h / kWtHX) % kWtHY, hz = h / (kWtHX * kWtHY);
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
            const int c = ci0 + 8 * half;
            uint4 v = zero4;
            if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n && c < cin)
                v = *reinterpret_cast<const uint4 *>(
                    x + (sample + (static_cast<long long>(gz) * n + gy) * n + gx) * cin + c);
            *reinterpret_cast<uint4 *>(&xs[h][8 * half]) = v;
        }
        // dy tile: 256 voxels x 2 granules
        for (int e = t; e < kWtVox * 2; e += 256) {
            const int half = e & 1, vi = e >> 1;
            const int vx = vi % kWtX, vy = (vi / kWtX) % kWtY, vz = vi / (kWtX * kWtY);
            const uint4 v = *reinterpret_cast<const uint4 *>(
                dy + (sample + (static_cast<long long>(z0 + vz) * n + y0 + vy) * n + x0 + vx) * cout +
                co0 + 8 * half);
            *reinterpret_cast<uint4 *>(&gs[vi][8 * half]) = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int ks = 0; ks < kWtVox / 16; ++ks) {
            // k-step ks: voxels 16 ks .. 16 ks + 15 = two x-rows (z, y), (z, y + 1)
            const int vz = ks / (kWtY / 2), vy = 2 * (ks % (kWtY / 2));
            unsigned a[4];
            // A = dy^T: matrices (v 0-7, co 0-7), (v 0-7, co 8-15), (v 8-15, co 0-7), (v 8-15, co 8-15)
            ldsm_x4_trans(a, &gs[16 * ks + 8 * (mj >> 1) + mr][8 * (mj & 1)]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i < ntap) {
                    const int tap = warp + 8 * i;
                    const int dz = tap / 9, dyy = (tap / 3) % 3, dx = tap % 3;
                    // B rows: voxel row (mj & 1) of the k-step, x = mr, shifted by the tap;
                    // matrices (v 0-7, ci 0-7), (v 8-15, ci 0-7), (v 0-7, ci 8-15), (v 8-15, ci 8-15)
                    const int h = ((vz + dz) * kWtHY + vy + (mj & 1) + dyy) * kWtHX + mr + dx;
                    unsigned bb[4];
                    ldsm_x4_trans(bb, &xs[h][8 * (mj >> 1)]);
                    mma_bf16_16816(acc[i][0], a, bb[0], bb[1]);
                    mma_bf16_16816(acc[i][1], a, bb[2], bb[3]);
                }
            }
        }
        __syncthreads();
    }
    // acc[i][j]: rows co0 + g (+8), columns ci0 + 8 j + 2 tig (+1)
    const int g = lane >> 2, tig = lane & 3;
    float *out = partials + static_cast<long long>(blockIdx.y) * 27 * cout * cin;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i >= ntap) continue;
        const int tap = warp + 8 * i;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int co = co0 + g + 8 * (q >> 1);
                const int ci = ci0 + 8 * j + 2 * tig + (q & 1);
                if (ci < cin)
                    out[(static_cast<long long>(tap) * cout + co) * cin + ci] = acc[i][j][q];
            }
    }
}

// Weight gradient of a 1^3 convolution with few channels (the output head):
// dw[co][ci] = sum over voxels of dy[v][co] x[v][ci] on CUDA cores.  Each
// thread sums a strided set of voxels into CO x CI registers; the block
// reduces its threads in a fixed tree and writes partials[block][co][ci].
template <typename TI, int CO, int CI>
__global__ void __launch_bounds__(256) wgrad_small_kernel(const TI *__restrict__ x,
                                                          const float *__restrict__ dy,
                                                          float *__restrict__ partials, long long voxels,
                                                          int cin, int cout, long long chunk)
{
    float acc[CO][CI];
#pragma unroll
    for (int o = 0; o < CO; ++o)
#pragma unroll
        for (int i = 0; i < CI; ++i) acc[o][i] = 0.f;
    const long long v0 = blockIdx.x * chunk;
    const long long v1 = v0 + chunk < voxels ? v0 + chunk : voxels;
    for (long long v = v0 + threadIdx.x; v < v1; v += 256) {
        float xv[CI], gv[CO];
#pragma unroll
        for (int i = 0; i < CI; ++i) xv[i] = i < cin ? ldf(x + v * cin + i) : 0.f;
#pragma unroll
        for (int o = 0; o < CO; ++o) gv[o] = o < cout ? dy[v * cout + o] : 0.f;
#pragma unroll
        for (int o = 0; o < CO; ++o)
#pragma unroll
            for (int i = 0; i < CI; ++i) acc[o][i] = fmaf(gv[o], xv[i], acc[o][i]);
    }
    // fixed-order reduction: warp shuffle tree, then the 8 warps in order
    __shared__ float red[8][CO * CI];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 0; o < CO; ++o)
#pragma unroll
        for (int i = 0; i < CI; ++i) {
            float v = acc[o][i];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0) red[warp][o * CI + i] = v;
        }
    __syncthreads();
    for (int k = threadIdx.x; k < CO * CI; k += 256) {
        const int o = k / CI, i = k % CI;
        if (o >= cout || i >= cin) continue;
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += red[w][k];
        partials[(static_cast<long long>(blockIdx.x) * cout + o) * cin + i] = v;
    }
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

template <typename T>
__device__ __forceinline__ void st2(T *p, float a, float b);
template <>
__device__ __forceinline__ void st2<float>(float *p, float a, float b)
{
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16 *p, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

// Eight consecutive channels in one or two 16-byte stores (p 16-byte aligned).
template <typename T>
__device__ __forceinline__ void st8(T *p, const float *v);
template <>
__device__ __forceinline__ void st8<float>(float *p, const float *v)
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void st8<__nv_bfloat16>(__nv_bfloat16 *p, const float *v)
{
    uint4 u;
    __nv_bfloat162 h[4];
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    memcpy(&u, h, sizeof u);
    *reinterpret_cast<uint4 *>(p) = u;
}

// Tensor-core 3^3 convolution (implicit GEMM, mma.m16n8k16, FP32
// accumulation) over 8 x 8 x 4 voxel tiles: a block owns one tile of one
// sample and 8 NT output channels.  For every 16 input channels it stages
// the x halo (10 x 10 x 6 voxels) and the weights of all 27 taps for its
// channels (rows padded to 24 elements: conflict-free ldmatrix), then runs
// the 27 taps as shifted GEMMs: ldmatrix takes one row address per thread,
// so tap (dz, dy, dx) just reads the halo rows shifted by it.  Warp w owns
// voxel rows 32 w .. 32 w + 31 (two m16 tiles) and all NT n8 tiles.
// Dynamic shared memory: (600 + 27 * 8 NT) rows of 24 bfloat16.
template <int NT, typename TO>
__global__ void __launch_bounds__(256) conv3d_tc_kernel(const __nv_bfloat16 *__restrict__ x,
                                                        const __nv_bfloat16 *__restrict__ w,
                                                        const float *__restrict__ bias,
                                                        TO *__restrict__ y, int n, int cin, int cout,
                                                        int act)
{
    constexpr int CO = 8 * NT;
    extern __shared__ __align__(16) unsigned char conv_smem[];
    __nv_bfloat16(*xs)[kWtRow] = reinterpret_cast<__nv_bfloat16(*)[kWtRow]>(conv_smem);
    __nv_bfloat16(*ws)[kWtRow] = xs + kWtHalo;  // [tap * CO + co]
    const int tx_n = n / kWtX, ty_n = n / kWtY, tz_n = n / kWtZ;
    int r = blockIdx.x;
    const int x0 = (r % tx_n) * kWtX;
    r /= tx_n;
    const int y0 = (r % ty_n) * kWtY;
    r /= ty_n;
    const int z0 = (r % tz_n) * kWtZ;
    const int b = r / tz_n;
    const int co0 = blockIdx.y * CO;
    const long long sample = static_cast<long long>(b) * n * n * n;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int mj = lane >> 3, mr = lane & 7;
    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (int ci0 = 0; ci0 < cin; ci0 += 16) {
        for (int e = t; e < kWtHalo * 2; e += 256) {
            const int half = e & 1, h = e >> 1;
            const int hx = h % kWtHX, hy = (h / kWtHX) % kWtHY, hz = h / (kWtHX * kWtHY);
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
            const int c = ci0 + 8 * half;
            uint4 v = zero4;
            if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n && c < cin)
                v = *reinterpret_cast<const uint4 *>(
                    x + (sample + (static_cast<long long>(gz) * n + gy) * n + gx) * cin + c);
            *reinterpret_cast<uint4 *>(&xs[h][8 * half]) = v;
        }
        for (int e = t; e < 27 * CO * 2; e += 256) {
            const int half = e & 1, row = e >> 1;
            const int co = row % CO, tap = row / CO;
            const int c = ci0 + 8 * half;
            uint4 v = zero4;
            if (co0 + co < cout && c < cin)
                v = *reinterpret_cast<const uint4 *>(w + (static_cast<long long>(tap) * cout + co0 + co) * cin + c);
            *reinterpret_cast<uint4 *>(&ws[row][8 * half]) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9, dyy = (tap / 3) % 3, dx = tap % 3;
            unsigned a[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                // m16 tile 2 warp + i: voxel x-rows (vz, vy) and (vz, vy + 1)
                const int mt = 2 * warp + i;
                const int vz = mt / (kWtY / 2), vy = 2 * (mt % (kWtY / 2));
                const int h = ((vz + dz) * kWtHY + vy + (mj & 1) + dyy) * kWtHX + mr + dx;
                ldsm_x4(a[i], &xs[h][8 * (mj >> 1)]);
            }
#pragma unroll
            for (int j = 0; j < NT; j += 2) {
                // n8 tiles j, j + 1: matrices (co j, ci 0-7), (co j, ci 8-15), (co j+1, ...)
                unsigned bb[4];
                ldsm_x4(bb, &ws[tap * CO + 8 * (j + (mj >> 1)) + mr][8 * (mj & 1)]);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    mma_bf16_16816(acc[i][j], a[i], bb[0], bb[1]);
                    mma_bf16_16816(acc[i][j + 1], a[i], bb[2], bb[3]);
                }
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int mt = 2 * warp + i;
        const int vz = mt / (kWtY / 2), vy = 2 * (mt % (kWtY / 2));
#pragma unroll
        for (int hrow = 0; hrow < 2; ++hrow) {
            const long long vox = sample + (static_cast<long long>(z0 + vz) * n + y0 + vy + hrow) * n + x0 + g;
            TO *yo = y + vox * cout;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int co = co0 + 8 * j + 2 * tig;
                if (co >= cout) continue;
                float v0 = acc[i][j][2 * hrow] + (bias ? bias[co] : 0.f);
                float v1 = acc[i][j][2 * hrow + 1] + (bias ? bias[co + 1] : 0.f);
                if (act) {
                    v0 = v0 > 0.f ? v0 : kSlope * v0;
                    v1 = v1 > 0.f ? v1 : kSlope * v1;
                }
                st2(yo + co, v0, v1);
            }
        }
    }
}

// A 1^3 convolution with few channels (the output head and its input
// gradient) on CUDA cores: one voxel per thread, the weights and bias in
// shared memory, y[v][co] = act(sum_ci x[v][ci] w[co][ci] + b[co]).
template <typename TI, typename TW, typename TO, int CI, int CO>
__global__ void __launch_bounds__(256) conv1x1_small_kernel(const TI *__restrict__ x, const TW *__restrict__ w,
                                                            const float *__restrict__ bias, TO *__restrict__ y,
                                                            long long voxels, int cin, int cout, int act)
{
    __shared__ float ws[CO][CI];
    __shared__ float bs[CO];
    for (int e = threadIdx.x; e < CO * CI; e += blockDim.x) {
        const int o = e / CI, i = e % CI;
        ws[o][i] = (o < cout && i < cin) ? ldf(w + o * cin + i) : 0.f;
    }
    for (int o = threadIdx.x; o < CO; o += blockDim.x) bs[o] = (bias && o < cout) ? bias[o] : 0.f;
    __syncthreads();
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < voxels;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        float xv[CI];
#pragma unroll
        for (int i = 0; i < CI; ++i) xv[i] = i < cin ? ldf(x + v * cin + i) : 0.f;
#pragma unroll
        for (int o = 0; o < CO; ++o) {
            if (o >= cout) break;
            float r = bs[o];
#pragma unroll
            for (int i = 0; i < CI; ++i) r = fmaf(xv[i], ws[o][i], r);
            if (act) r = r > 0.f ? r : kSlope * r;
            stf(y + v * cout + o, r);
        }
    }
}

// 3^3 convolution on the 5th-generation tensor cores (tcgen05.mma with the
// accumulator in tensor memory).  A CTA of 4 warps owns a tile of 8 x 16
// voxels of one z-plane (M = 128 GEMM rows) and CO output channels (N).  Per
// 16 input channels it stages the x halo (10 x 18 x 3 voxels) and the
// weights of all 27 taps in the canonical K-major core-matrix layout (8 rows
// x 16 bytes per core matrix):
//   halo   [kg 2][z 3][y 18][x 10] x 16 B: the 8 rows of a core matrix are 8
//          consecutive x voxels, so tap (dz, dy, dx) is the same descriptor
//          shifted by ((dz * 18 + dy) * 10 + dx) * 16 bytes; SBO (next 8 rows
//          = next y row) = 160 B, LBO (next 8 channels) = 540 * 16 B;
//   weights [tap 27][kg 2][co CO] x 16 B: SBO (next 8 channels out) = 128 B,
//          LBO (next 8 channels in) = CO * 16 B.
// One thread issues the 27 MMAs (K = 16 each) and commits them to an
// mbarrier; everyone waits (bounded) before the buffers are restaged.  The
// epilogue reads each thread's accumulator row (TMEM lane = voxel) with
// tcgen05.ld and writes bias + activation.  A wait that runs out sets *err.
constexpr int kUmX = 8, kUmY = 16;
constexpr int kUmHX = kUmX + 2, kUmHY = kUmY + 2, kUmHZ = 3;
constexpr int kUmHalo = kUmHX * kUmHY * kUmHZ;                // 540 voxels
constexpr unsigned kUmHaloOff = 128;                         // after the barrier and TMEM slot
constexpr unsigned kUmHaloBytes = 2u * kUmHalo * 16u;        // 17280
template <int CO>
constexpr unsigned um_smem_bytes()
{
    return kUmHaloOff + kUmHaloBytes + 27u * 2u * CO * 16u;
}
constexpr unsigned kUmWaitPolls = 1u << 22;  // ~0.3 s of polling before giving up
// TMEM columns a CTA allocates (the accumulator needs CO, at least 32);
// DMRT_UMMA_TMEM_COLS raises it (a power of two up to 512).
#ifndef DMRT_UMMA_CTAS_PER_SM
#define DMRT_UMMA_CTAS_PER_SM 4
#endif
#ifndef DMRT_UMMA_TMEM_COLS
#define DMRT_UMMA_TMEM_COLS 0
#endif

// Streaming multiprocessors of the current device (152 on GB300), asked once
// per device.
int sm_count()
{
    static std::atomic<int> cached[64];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    if (dev >= 0 && dev < 64 && (sms = cached[dev].load(std::memory_order_relaxed)) > 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 152;
    }
    if (dev >= 0 && dev < 64) cached[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

// The z run of the streaming convolutions: each CTA walks zrun planes of an
// 8 x 16 column, xy columns in all, `slots` CTAs resident at once.  A run
// costs about zrun + 3 planes (the CTA's weights, two halo planes, the
// pipeline fill), and CTAs beyond the resident ones wait for whole runs, so
// the run minimises waves x (zrun + 3), longer runs among equals.  At 64^3
// x 4 samples this takes 512 CTAs of 16 planes in one wave; the earlier rule
// (about 4 CTAs per SM) gave 640 CTAs of 13 planes, 32 of them in a second
// wave, and the layer took almost two runs' time.
int conv_zrun(long long xy, int n, int slots)
{
    int best = n, best_cost = 0x7fffffff;
    for (int zs = 1; zs <= std::max(1, n / 2); ++zs) {
        const int zrun = (n + zs - 1) / zs;
        const long long ctas = xy * ((n + zrun - 1) / zrun);
        const long long waves = (ctas + slots - 1) / slots;
        const long long cost = waves * (zrun + 3);
        if (cost < best_cost || (cost == best_cost && zrun > best)) best = zrun, best_cost = static_cast<int>(cost);
    }
    return best;
}

template <int CO, typename TO>
__global__ void __launch_bounds__(128, 1) conv3d_umma_kernel(const __nv_bfloat16 *__restrict__ x,
                                                             const __nv_bfloat16 *__restrict__ w,
                                                             const float *__restrict__ bias,
                                                             TO *__restrict__ y, int n, int cin, int cout,
                                                             int act, int *err)
{
    extern __shared__ __align__(1024) unsigned char um_smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(um_smem);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(um_smem + 8);
    unsigned char *halo = um_smem + kUmHaloOff;
    unsigned char *wsm = halo + kUmHaloBytes;
    constexpr uint32_t kCols = DMRT_UMMA_TMEM_COLS > (CO < 32 ? 32 : CO) ? DMRT_UMMA_TMEM_COLS : (CO < 32 ? 32 : CO);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int tx_n = n / kUmX, ty_n = n / kUmY;
    int r = blockIdx.x;
    const int x0 = (r % tx_n) * kUmX;
    r /= tx_n;
    const int y0 = (r % ty_n) * kUmY;
    r /= ty_n;
    const int z = r % n;
    const int b = r / n;
    const int co0 = blockIdx.y * CO;
    const long long sample = static_cast<long long>(b) * n * n * n;
    if (t == 0) umma::mbar_init(bar, 1);
    if (warp == 0) umma::tmem_alloc(tslot, kCols);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(128, CO);
    const uint32_t halo_s = umma::smem_u32(halo), w_s = umma::smem_u32(wsm);
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    bool ok = true;
    uint32_t phase = 0;
    for (int ci0 = 0; ci0 < cin && ok; ci0 += 16) {
        for (int e = t; e < kUmHalo * 2; e += 128) {
            const int kg = e / kUmHalo, h = e % kUmHalo;
            const int hx = h % kUmHX, hy = (h / kUmHX) % kUmHY, hz = h / (kUmHX * kUmHY);
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z + hz - 1;
            const int c = ci0 + 8 * kg;
            uint4 v = zero4;
            if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n && c < cin)
                v = *reinterpret_cast<const uint4 *>(
                    x + (sample + (static_cast<long long>(gz) * n + gy) * n + gx) * cin + c);
            *reinterpret_cast<uint4 *>(halo + (kg * kUmHalo + h) * 16) = v;
        }
        for (int e = t; e < 27 * 2 * CO; e += 128) {
            const int co = e % CO, kg = (e / CO) % 2, tap = e / (2 * CO);
            const int c = ci0 + 8 * kg;
            uint4 v = zero4;
            if (co0 + co < cout && c < cin)
                v = *reinterpret_cast<const uint4 *>(w + (static_cast<long long>(tap) * cout + co0 + co) * cin + c);
            *reinterpret_cast<uint4 *>(wsm + ((tap * 2 + kg) * CO + co) * 16) = v;
        }
        umma::fence_proxy_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            umma::fence_after_sync();
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                const uint64_t ad = umma::smem_desc(halo_s + ((dz * kUmHY + dy) * kUmHX + dx) * 16,
                                                    kUmHalo * 16, kUmHX * 16);
                const uint64_t bd = umma::smem_desc(w_s + tap * 2 * CO * 16, CO * 16, 128);
                umma::mma_bf16(tmem, ad, bd, idesc, (ci0 > 0 || tap > 0) ? 1u : 0u);
            }
            umma::commit(bar);
        }
        // the MMAs read the staged tiles: wait for them before restaging
        if (!umma::mbar_wait(bar, phase, kUmWaitPolls)) ok = false;
        phase ^= 1u;
        umma::fence_after_sync();
        __syncthreads();
    }
    if (ok) {
        const int m = 32 * warp + lane;  // TMEM lane = GEMM row = voxel (x fastest)
        const long long vox = sample + (static_cast<long long>(z) * n + y0 + m / kUmX) * n + x0 + m % kUmX;
        TO *yo = y + vox * cout + co0;
#pragma unroll
        for (int c16 = 0; c16 < CO; c16 += 16) {
            float v[16];
            umma::ld_32x32b_x16(tmem + (static_cast<uint32_t>(32 * warp) << 16) + c16, v);
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const int co = co0 + c16 + j;
                float a = v[j] + (bias ? bias[co] : 0.f), bb = v[j + 1] + (bias ? bias[co + 1] : 0.f);
                if (act) {
                    a = a > 0.f ? a : kSlope * a;
                    bb = bb > 0.f ? bb : kSlope * bb;
                }
                st2(yo + c16 + j, a, bb);
            }
        }
    } else if (t == 0) {
        atomicExch(err, 1);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, kCols);
}

// 3^3 convolution on the tcgen05 tensor cores for few channels (cin <= 32,
// cout <= 32), streamed along z with its halo planes brought in by TMA and
// its roles split among warps.  A CTA owns an 8 x 16 tile (M = 128 GEMM
// rows, one per voxel) over a run of z-planes and keeps the weights of all
// taps resident in the layout of conv3d_umma_kernel ([tap][kg][co] x 16 B);
// tap (dz, dy, dx) of plane z is the halo descriptor of plane z - 1 + dz
// shifted by (dy * 10 + dx) * 16 bytes.
//  - the halo planes (10 x 18 voxels, 8 channels per k-group) arrive by
//    tiled TMA copies of the channels-last activations, viewed as the 5-D
//    tensor (c, x, y, z, sample): one box of 8 x 10 x 18 x 1 x 1 per k-group,
//    zero-filled outside the grid, into a ring of kUtRing plane slots with
//    one mbarrier each;
//  - warp 4 is the producer: one lane issues the copies and the 27 MMAs of a
//    plane into one of kUtAcc TMEM accumulators, and refills a ring slot as
//    soon as the MMAs that read it have completed;
//  - warps 0-3 are the epilogue (TMEM lanes 32 w .. 32 w + 31, one voxel
//    each): they wait for a plane's MMAs, read its accumulator, hand it back
//    on an mbarrier and write bias + activation.
// No thread waits at a block barrier inside the loop: the tensor cores, the
// copies and the epilogue run concurrently.  What bounds the narrow layers
// then is the tensor core's operand traffic: each of the 27 MMAs of a plane
// reads its 128 x 16 A tile (4 KB) from shared memory for only 16 or 32
// output channels.  Each k-group of a plane starts on a 128-byte boundary
// (2944 bytes apart), which the MMA descriptors take as the leading byte
// offset.  Every wait is bounded; one that runs out sets *err and ends its
// warp's loop, and the CTA waits (bounded) for its copies in flight before it
// releases its TMEM and exits.
constexpr int kUtRing = 6;
constexpr int kUtAcc = 4;  // TMEM accumulators
constexpr int kUtThreads = 160;
constexpr unsigned kUtKgBytes = (kUmHX * kUmHY * 16u + 127u) / 128u * 128u;  // 2944
constexpr unsigned kUtHead = 256;  // mbarriers and the TMEM slot
template <int KG>
constexpr unsigned ut_plane_bytes()
{
    return static_cast<unsigned>(KG) * kUtKgBytes;
}
template <int CO, int KG>
constexpr unsigned ut_smem_bytes()
{
    return 128u + kUtHead + kUtRing * ut_plane_bytes<KG>() + 27u * KG * CO * 16u;  // + alignment slack
}

template <int CO, int KG, typename TO>
__global__ void __launch_bounds__(kUtThreads, 4) conv3d_umma_tma_kernel(const __grid_constant__ CUtensorMap xmap,
                                                                     const __nv_bfloat16 *__restrict__ w,
                                                                     const float *__restrict__ bias,
                                                                     TO *__restrict__ y, int n, int cin, int cout,
                                                                     int act, int zrun, int *err)
{
    extern __shared__ __align__(1024) unsigned char ut_smem_raw[];
    // TMA destinations start on 128-byte boundaries whatever the base alignment
    unsigned char *ut_smem = ut_smem_raw + ((128u - (umma::smem_u32(ut_smem_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(ut_smem);  // [kUtRing]: a slot holds its plane
    uint64_t *acc_full = full + kUtRing;                      // [kUtAcc]: a plane's MMAs are done
    uint64_t *acc_empty = acc_full + kUtAcc;                  // [kUtAcc]: its accumulator was read
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acc_empty + kUtAcc);
    unsigned char *ring = ut_smem + kUtHead;
    constexpr unsigned kPlane = ut_plane_bytes<KG>();
    unsigned char *wsm = ring + kUtRing * kPlane;
    constexpr int kRow = kUmHX * kUmHY;  // 180 voxels of a halo plane
    constexpr uint32_t kPlaneTx = static_cast<uint32_t>(KG) * kRow * 16u;
    constexpr uint32_t kCols = kUtAcc * CO < 32 ? 32 : kUtAcc * CO;
    static_assert(kUtHead >= 8 * (kUtRing + 2 * kUtAcc) + 4, "mbarriers and TMEM slot");
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int tx_n = n / kUmX, ty_n = n / kUmY, zs_n = (n + zrun - 1) / zrun;
    int r = blockIdx.x;
    const int x0 = (r % tx_n) * kUmX;
    r /= tx_n;
    const int y0 = (r % ty_n) * kUmY;
    r /= ty_n;
    const int z_begin = (r % zs_n) * zrun;
    const int b = r / zs_n;
    const int z_end = min(z_begin + zrun, n);
    const long long sample = static_cast<long long>(b) * n * n * n;
    const int p0 = z_begin - 1;  // the first halo plane; the last one is z_end
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    if (t == 0) {
        for (int k = 0; k < kUtRing; ++k) umma::mbar_init(&full[k], 1);
        for (int k = 0; k < kUtAcc; ++k) {
            umma::mbar_init(&acc_full[k], 1);
            umma::mbar_init(&acc_empty[k], 4);  // one arrival per epilogue warp
        }
    }
    if (warp == 0) umma::tmem_alloc(tslot, kCols);
    // weights of all taps: [tap][kg][co] x 16 B
    for (int e = t; e < 27 * KG * CO; e += kUtThreads) {
        const int co = e % CO, kg = (e / CO) % KG, tap = e / (KG * CO);
        const int c = 8 * kg;
        uint4 v = zero4;
        if (co < cout && c < cin)
            v = *reinterpret_cast<const uint4 *>(w + (static_cast<long long>(tap) * cout + co) * cin + c);
        *reinterpret_cast<uint4 *>(wsm + ((tap * KG + kg) * CO + co) * 16) = v;
    }
    umma::fence_proxy_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool ok = true;
    if (warp == 4) {
        // ---- producer: copies and MMAs (one lane)
        if (lane == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(128, CO);
            const uint64_t a_base = umma::smem_desc(umma::smem_u32(ring), kUtKgBytes, kUmHX * 16);
            const uint64_t b_base = umma::smem_desc(umma::smem_u32(wsm), CO * 16, 128);
            // plane p (p0 <= p <= z_end) is load number (p - p0) / kUtRing of slot (p - p0) % kUtRing
            auto issue = [&](int p) {
                const int k = p - p0, slot = k % kUtRing;
                umma::mbar_arrive_expect_tx(&full[slot], kPlaneTx);
#pragma unroll
                for (int kg = 0; kg < KG; ++kg)
                    umma::tma_load_5d(&xmap, ring + slot * kPlane + kg * kUtKgBytes, &full[slot], 8 * kg, x0 - 1,
                                      y0 - 1, p, b);
            };
            auto wait_plane = [&](int p) {
                const int k = p - p0;
                return umma::mbar_wait(&full[k % kUtRing], static_cast<uint32_t>(k / kUtRing) & 1u, kUmWaitPolls);
            };
            int issued = p0 - 1;  // the last plane whose copies went out
            while (issued < z_end && issued + 1 - p0 < kUtRing) issue(++issued);
            for (int z = z_begin; z < z_end && ok; ++z) {
                const int j = z - z_begin, buf = j % kUtAcc;
                // the accumulator's previous plane has been read out
                if (j >= kUtAcc)
                    ok = umma::mbar_wait(&acc_empty[buf], static_cast<uint32_t>(j / kUtAcc - 1) & 1u, kUmWaitPolls);
                ok = ok && wait_plane(z - 1) && wait_plane(z) && wait_plane(z + 1);
                if (!ok) break;
                umma::fence_after_sync();
                // descriptors: the base ones plus each operand's offset / 16 in
                // the start-address field (shared addresses stay below 2^18)
                uint64_t a_plane[3];
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
                    a_plane[dz] = a_base + static_cast<uint64_t>((((z - 1 + dz - p0) % kUtRing) * kPlane) >> 4);
                const uint32_t dacc = tmem + buf * CO;
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
#pragma unroll
                    for (int kc = 0; kc < KG / 2; ++kc) {
                        const uint64_t ad =
                            a_plane[dz] + static_cast<uint64_t>(((dy * kUmHX + dx) * 16 + 2 * kc * kUtKgBytes) >> 4);
                        const uint64_t bd = b_base + static_cast<uint64_t>(((tap * KG + 2 * kc) * CO * 16) >> 4);
                        umma::mma_bf16(dacc, ad, bd, idesc, (tap > 0 || kc > 0) ? 1u : 0u);
                    }
                }
                umma::commit(&acc_full[buf]);
                // plane z - 1's MMAs were the last to read the slot of plane z - 2
                if (j >= 1 && issued < z_end) {
                    const int jp = j - 1;
                    ok = umma::mbar_wait(&acc_full[jp % kUtAcc], static_cast<uint32_t>(jp / kUtAcc) & 1u,
                                         kUmWaitPolls);
                    if (ok) issue(++issued);
                }
            }
            if (!ok) {
                atomicExch(err, 1);
                // copies still in flight land before the CTA's shared memory is released
                for (int p = max(p0, issued - kUtRing + 1); p <= issued; ++p) (void)wait_plane(p);
            }
        }
    } else {
        // ---- epilogue: warp w holds TMEM lanes 32 w .. 32 w + 31 (voxel m, x fastest)
        const int m = 32 * warp + lane;
        float bv[CO];  // the biases, read once
#pragma unroll
        for (int co = 0; co < CO; ++co) bv[co] = bias ? bias[co] : 0.f;
        for (int z = z_begin; z < z_end && ok; ++z) {
            const int j = z - z_begin, buf = j % kUtAcc;
            ok = umma::mbar_wait(&acc_full[buf], static_cast<uint32_t>(j / kUtAcc) & 1u, kUmWaitPolls);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            umma::fence_after_sync();
            float v[CO];
#pragma unroll
            for (int c16 = 0; c16 < CO; c16 += 16) {
                float part[16];
                umma::ld_32x32b_x16(tmem + (static_cast<uint32_t>(32 * warp) << 16) + buf * CO + c16, part);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[c16 + i] = part[i];
            }
            // the accumulator may take the next plane's MMAs
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(&acc_empty[buf]))
                                        : "memory");
            const long long vox = sample + (static_cast<long long>(z) * n + y0 + m / kUmX) * n + x0 + m % kUmX;
            TO *yo = y + vox * cout;
#pragma unroll
            for (int co = 0; co < CO; ++co) {
                const float a = v[co] + bv[co];
                v[co] = act && a <= 0.f ? kSlope * a : a;
            }
#pragma unroll
            for (int co = 0; co < CO; co += 8) st8(yo + co, v + co);
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, kCols);
}

// out = bfloat16(in)
__global__ void narrow_kernel(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, long long len)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// Weight gradient of a k^3 convolution: dw[tap][co][ci] = sum over samples
// and voxels of dy[v][co] * x[v + tap][ci].  One block per (tap, chunk of
// voxels); thread t owns input channel ci = t % cin and the output channels
// t / cin + j * (256 / cin), and sums its chunk in order (cin must divide
// 256; cin, cout <= 128).  partials[chunk][tap][co][ci] are summed in order
// afterwards.
template <typename TI, int K>
__global__ void __launch_bounds__(256) conv3d_wgrad_kernel(const TI *__restrict__ x,
                                                           const float *__restrict__ dy,
                                                           float *__restrict__ partials, int batch,
                                                           int n, int cin, int cout, int chunk)
{
    constexpr int R = K / 2;
    constexpr int VB = 32;  // voxels staged per round
    __shared__ float xs[VB][128];
    __shared__ float gs[VB][128];
    const int tap = blockIdx.x;
    const int dz = tap / (K * K) - R, dyo = (tap / K) % K - R, dx = tap % K - R;
    const long long total = static_cast<long long>(batch) * n * n * n;
    const long long v_begin = static_cast<long long>(blockIdx.y) * chunk;
    const long long v_end = v_begin + chunk < total ? v_begin + chunk : total;
    const int ci = threadIdx.x % cin;
    const int co0 = threadIdx.x / cin;
    const int step = 256 / cin;
    const int nco = (cout - co0 + step - 1) / step;  // output channels of this thread (<= 64)
    float acc[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) acc[k] = 0.f;
    for (long long vb = v_begin; vb < v_end; vb += VB) {
        const int nv = static_cast<int>(v_end - vb < VB ? v_end - vb : VB);
        for (int e = threadIdx.x; e < VB * cin; e += 256) {
            const int c = e % cin, vi = e / cin;
            float val = 0.f;
            if (vi < nv) {
                long long v = vb + vi;
                const int gx = static_cast<int>(v % n);
                v /= n;
                const int gy = static_cast<int>(v % n);
                v /= n;
                const int gz = static_cast<int>(v % n);
                const long long bb = v / n;
                const int sz = gz + dz, sy = gy + dyo, sx = gx + dx;
                if (sz >= 0 && sz < n && sy >= 0 && sy < n && sx >= 0 && sx < n)
                    val = ldf(x + (((bb * n + sz) * n + sy) * n + sx) * cin + c);
            }
            xs[vi][c] = val;
        }
        for (int e = threadIdx.x; e < VB * cout; e += 256) {
            const int c = e % cout, vi = e / cout;
            gs[vi][c] = vi < nv ? dy[(vb + vi) * cout + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 1
        for (int vi = 0; vi < nv; ++vi) {
            const float xv = xs[vi][ci];
#pragma unroll
            for (int k = 0; k < 64; ++k)
                if (k < nco) acc[k] = fmaf(gs[vi][co0 + k * step], xv, acc[k]);
        }
        __syncthreads();
    }
    float *out = partials + (static_cast<long long>(blockIdx.y) * gridDim.x + tap) * cout * cin;
#pragma unroll
    for (int k = 0; k < 64; ++k)
        if (k < nco) out[(co0 + k * step) * cin + ci] = acc[k];
}

// out[i] = sum over chunks of partials[chunk][i], in a fixed order: a block
// covers E consecutive elements (E = 32, or the power of two >= len when len
// is smaller) with 256 / E lanes of chunks; lane l adds chunks l, l + L, ...
// into four interleaved sums (chunk c goes to sum (c / L) % 4), and the lanes
// are then added in order.  Threads with consecutive elements read
// consecutive floats of one chunk.
__global__ void __launch_bounds__(256) sum_chunks_kernel(const float *__restrict__ partials,
                                                         float *__restrict__ out, long long len,
                                                         int chunks, int E)
{
    __shared__ float red[256];
    const int L = 256 / E;
    const int e = threadIdx.x % E, lane = threadIdx.x / E;
    const long long i = static_cast<long long>(blockIdx.x) * E + e;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (i < len) {
        int c = lane;
        for (; c + 3 * L < chunks; c += 4 * L) {
            s0 += partials[static_cast<long long>(c) * len + i];
            s1 += partials[static_cast<long long>(c + L) * len + i];
            s2 += partials[static_cast<long long>(c + 2 * L) * len + i];
            s3 += partials[static_cast<long long>(c + 3 * L) * len + i];
        }
        for (; c < chunks; c += L) s0 += partials[static_cast<long long>(c) * len + i];
    }
    red[threadIdx.x] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (lane == 0 && i < len) {
        float tot = 0.f;
        for (int l = 0; l < L; ++l) tot += red[l * E + e];
        out[i] = tot;
    }
}

// Bias gradient partials: per block of voxels, the sum of dy over them.
// Thread t adds channel t % cout of voxels lane, lane + lanes, ... (lane =
// t / cout, lanes = 256 / cout; four interleaved sums), so a warp reads
// consecutive floats; the lanes are then summed in order.
__global__ void __launch_bounds__(256) bias_grad_kernel(const float *__restrict__ dy,
                                                        float *__restrict__ partials, long long voxels,
                                                        int cout, long long chunk)
{
    __shared__ float red[256];
    const int lanes = 256 / cout;
    const int c = threadIdx.x % cout, lane = threadIdx.x / cout;
    const long long v0 = static_cast<long long>(blockIdx.x) * chunk;
    const long long v1 = v0 + chunk < voxels ? v0 + chunk : voxels;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (lane < lanes) {
        long long v = v0 + lane;
        for (; v + 3 * lanes < v1; v += 4 * lanes) {
            s0 += dy[v * cout + c];
            s1 += dy[(v + lanes) * cout + c];
            s2 += dy[(v + 2 * lanes) * cout + c];
            s3 += dy[(v + 3 * lanes) * cout + c];
        }
        for (; v < v1; v += lanes) s0 += dy[v * cout + c];
    }
    red[threadIdx.x] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (threadIdx.x < cout) {
        float tot = 0.f;
        for (int l = 0; l < lanes; ++l) tot += red[l * cout + threadIdx.x];
        partials[static_cast<long long>(blockIdx.x) * cout + threadIdx.x] = tot;
    }
}

// dy_pre = dy * slope where the (leaky ReLU) output was negative.
template <typename T>
__global__ void act_backward_kernel(const T *__restrict__ yout, float *__restrict__ dy, long long len)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        if (!(ldf(yout + i) > 0.f)) dy[i] *= kSlope;
}

// The leaky-ReLU backward (when act) fused with the bfloat16 copy of the
// resulting gradient: dy[i] *= slope where the output was not positive, then
// dyn[i] = bfloat16(dy[i]).  Four elements per thread (len % 4 == 0).
template <typename T>
__global__ void act_backward_narrow_kernel(const T *__restrict__ yout, float *__restrict__ dy,
                                           __nv_bfloat16 *__restrict__ dyn, long long len4, int act)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len4;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float4 g = reinterpret_cast<float4 *>(dy)[i];
        if (act) {
            const long long e = 4 * i;
            if (!(ldf(yout + e) > 0.f)) g.x *= kSlope;
            if (!(ldf(yout + e + 1) > 0.f)) g.y *= kSlope;
            if (!(ldf(yout + e + 2) > 0.f)) g.z *= kSlope;
            if (!(ldf(yout + e + 3) > 0.f)) g.w *= kSlope;
            reinterpret_cast<float4 *>(dy)[i] = g;
        }
        __nv_bfloat162 lo = __floats2bfloat162_rn(g.x, g.y), hi = __floats2bfloat162_rn(g.z, g.w);
        uint2 pk;
        pk.x = *reinterpret_cast<unsigned *>(&lo);
        pk.y = *reinterpret_cast<unsigned *>(&hi);
        reinterpret_cast<uint2 *>(dyn)[i] = pk;
    }
}

// act_backward_narrow_kernel that also sums the bias gradient: with a grid
// of a fixed number of blocks the grid stride is a multiple of the cout / 4
// channel groups, so every thread sees the same four channels and sums them;
// each block adds its threads per channel group in thread order and writes
// partials[block][cout].
template <typename T>
__global__ void __launch_bounds__(256) act_backward_narrow_bias_kernel(const T *__restrict__ yout,
                                                                       float *__restrict__ dy,
                                                                       __nv_bfloat16 *__restrict__ dyn,
                                                                       long long len4, int act, int c4,
                                                                       float *__restrict__ partials)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len4;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float4 g = reinterpret_cast<float4 *>(dy)[i];
        if (act) {
            const long long e = 4 * i;
            if (!(ldf(yout + e) > 0.f)) g.x *= kSlope;
            if (!(ldf(yout + e + 1) > 0.f)) g.y *= kSlope;
            if (!(ldf(yout + e + 2) > 0.f)) g.z *= kSlope;
            if (!(ldf(yout + e + 3) > 0.f)) g.w *= kSlope;
            reinterpret_cast<float4 *>(dy)[i] = g;
        }
        __nv_bfloat162 lo = __floats2bfloat162_rn(g.x, g.y), hi = __floats2bfloat162_rn(g.z, g.w);
        uint2 pk;
        pk.x = *reinterpret_cast<unsigned *>(&lo);
        pk.y = *reinterpret_cast<unsigned *>(&hi);
        reinterpret_cast<uint2 *>(dyn)[i] = pk;
        acc.x += g.x;
        acc.y += g.y;
        acc.z += g.z;
        acc.w += g.w;
    }
    __shared__ float4 red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (static_cast<int>(threadIdx.x) < c4) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = threadIdx.x; k < 256; k += c4) {
            t.x += red[k].x;
            t.y += red[k].y;
            t.z += red[k].z;
            t.w += red[k].w;
        }
        float *o = partials + static_cast<long long>(blockIdx.x) * 4 * c4 + 4 * threadIdx.x;
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    }
}

// wt[tap][ci][co] = w[K^3 - 1 - tap][co][ci] (weights of the transposed
// convolution, in the storage type).
template <typename TW>
__global__ void flip_transpose_kernel(const TW *__restrict__ w, TW *__restrict__ wt, int taps,
                                      int cout, int cin)
{
    const long long len = static_cast<long long>(taps) * cout * cin;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int co = static_cast<int>(i % cout);
        long long r = i / cout;
        const int ci = static_cast<int>(r % cin);
        const int tap = static_cast<int>(r / cin);
        wt[i] = w[(static_cast<long long>(taps - 1 - tap) * cout + co) * cin + ci];
    }
}

// ---------------------------------------------------------------- pooling, upsampling, skips

// Four consecutive channels as one access (c % 4 == 0).
struct F4 {
    float v[4];
};
template <typename T>
__device__ __forceinline__ F4 ld4(const T *p);
template <>
__device__ __forceinline__ F4 ld4<float>(const float *p)
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    return F4{{q.x, q.y, q.z, q.w}};
}
template <>
__device__ __forceinline__ F4 ld4<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const uint2 q = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.y));
    return F4{{a.x, a.y, b.x, b.y}};
}
template <typename T>
__device__ __forceinline__ void st4(T *p, const F4 &f);
template <>
__device__ __forceinline__ void st4<float>(float *p, const F4 &f)
{
    *reinterpret_cast<float4 *>(p) = make_float4(f.v[0], f.v[1], f.v[2], f.v[3]);
}
template <>
__device__ __forceinline__ void st4<__nv_bfloat16>(__nv_bfloat16 *p, const F4 &f)
{
    __nv_bfloat162 a = __floats2bfloat162_rn(f.v[0], f.v[1]), b = __floats2bfloat162_rn(f.v[2], f.v[3]);
    uint2 q;
    q.x = *reinterpret_cast<unsigned *>(&a);
    q.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = q;
}

// Element i of a [batch][n][n][n][c] tensor handled as (voxel, group of 4
// channels): i = voxel * c4 + q.  Voxel coordinates from the flat index.
__device__ __forceinline__ void voxel_xyz(long long v, int n, int &x, int &y, int &z, long long &b)
{
    x = static_cast<int>(v % n);
    v /= n;
    y = static_cast<int>(v % n);
    v /= n;
    z = static_cast<int>(v % n);
    b = v / n;
}

// 2 x 2 x 2 average pooling, n -> n / 2 (channels in groups of 4)
template <typename T>
__global__ void avgpool2_kernel(const T *__restrict__ x, T *__restrict__ y, int batch, int n, int c)
{
    const int m = n / 2, c4 = c / 4;
    const long long len = static_cast<long long>(batch) * m * m * m * c4;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(i % c4);
        int ox, oy, oz;
        long long b;
        voxel_xyz(i / c4, m, ox, oy, oz, b);
        F4 s{{0.f, 0.f, 0.f, 0.f}};
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * oz + (k >> 2), yy = 2 * oy + ((k >> 1) & 1), xx = 2 * ox + (k & 1);
            const F4 a = ld4(x + (((b * n + zz) * n + yy) * n + xx) * c + 4 * q);
#pragma unroll
            for (int j = 0; j < 4; ++j) s.v[j] += a.v[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) s.v[j] *= 0.125f;
        st4(y + 4 * i, s);
    }
}

// gradient of avgpool2: dx = dy / 8 broadcast (FP32)
__global__ void avgpool2_backward_kernel(const float *__restrict__ dy, float *__restrict__ dx,
                                         int batch, int n, int c)
{
    const int m = n / 2, c4 = c / 4;
    const long long len = static_cast<long long>(batch) * n * n * n * c4;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(i % c4);
        int xx, yy, zz;
        long long b;
        voxel_xyz(i / c4, n, xx, yy, zz, b);
        F4 a = ld4(dy + (((b * m + zz / 2) * m + yy / 2) * m + xx / 2) * c + 4 * q);
#pragma unroll
        for (int j = 0; j < 4; ++j) a.v[j] *= 0.125f;
        st4(dx + 4 * i, a);
    }
}

// nearest upsampling x2 (n -> 2n), plus an optional skip added: y = up(x) + s
template <typename T>
__global__ void up2_add_kernel(const T *__restrict__ x, const T *__restrict__ skip, T *__restrict__ y,
                               int batch, int n, int c)
{
    const int m = 2 * n, c4 = c / 4;
    const long long len = static_cast<long long>(batch) * m * m * m * c4;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(i % c4);
        int xx, yy, zz;
        long long b;
        voxel_xyz(i / c4, m, xx, yy, zz, b);
        F4 v = ld4(x + (((b * n + zz / 2) * n + yy / 2) * n + xx / 2) * c + 4 * q);
        if (skip) {
            const F4 sk = ld4(skip + 4 * i);
#pragma unroll
            for (int j = 0; j < 4; ++j) v.v[j] += sk.v[j];
        }
        st4(y + 4 * i, v);
    }
}

// gradient of nearest upsampling: dx = sum of the 8 children of dy (FP32)
__global__ void up2_backward_kernel(const float *__restrict__ dy, float *__restrict__ dx, int batch,
                                    int n, int c)
{
    const int m = 2 * n, c4 = c / 4;
    const long long len = static_cast<long long>(batch) * n * n * n * c4;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(i % c4);
        int ox, oy, oz;
        long long b;
        voxel_xyz(i / c4, n, ox, oy, oz, b);
        F4 s{{0.f, 0.f, 0.f, 0.f}};
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * oz + (k >> 2), yy = 2 * oy + ((k >> 1) & 1), xx = 2 * ox + (k & 1);
            const F4 a = ld4(dy + (((b * m + zz) * m + yy) * m + xx) * c + 4 * q);
#pragma unroll
            for (int j = 0; j < 4; ++j) s.v[j] += a.v[j];
        }
        st4(dx + 4 * i, s);
    }
}

// a += b, four floats per thread (len % 4 == 0)
__global__ void add_inplace_kernel(float *__restrict__ a, const float *__restrict__ b, long long len4)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len4;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float4 x = reinterpret_cast<float4 *>(a)[i];
        const float4 y = reinterpret_cast<const float4 *>(b)[i];
        x.x += y.x;
        x.y += y.y;
        x.z += y.z;
        x.w += y.w;
        reinterpret_cast<float4 *>(a)[i] = x;
    }
}

// ---------------------------------------------------------------- loss, optimiser, features

// Mean squared error: per-block partial sums of (y - t)^2 and dy = 2 (y - t) / len.
template <typename T>
__global__ void __launch_bounds__(256) mse_kernel(const T *__restrict__ yp, const float *__restrict__ tgt,
                                                  float *__restrict__ dy, double *__restrict__ partials,
                                                  long long len)
{
    __shared__ double sh[256];
    double s = 0.0;
    const float scale = 2.0f / static_cast<float>(len);
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < len; i += static_cast<long long>(gridDim.x) * 256) {
        const float d = ldf(yp + i) - tgt[i];
        s += static_cast<double>(d) * d;
        if (dy) dy[i] = scale * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void sum_doubles_kernel(const double *__restrict__ partials, int n, double scale,
                                   double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partials[i];
    *out = s * scale;
}

// Adam (Kingma & Ba 2015) on FP32 master weights; the storage copy is
// refreshed from the master.  bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
template <typename TW>
__global__ void adam_kernel(float *__restrict__ master, TW *__restrict__ wstore,
                            const float *__restrict__ grad, float *__restrict__ m1,
                            float *__restrict__ m2, long long len, float lr, float beta1,
                            float beta2, float eps, float bc1, float bc2)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float g = grad[i];
        const float a = beta1 * m1[i] + (1.f - beta1) * g;
        const float b = beta2 * m2[i] + (1.f - beta2) * g * g;
        m1[i] = a;
        m2[i] = b;
        const float mh = a / bc1, vh = b / bc2;
        const float wv = master[i] - lr * mh / (sqrtf(vh) + eps);
        master[i] = wv;
        stf(wstore + i, wv);
    }
}

template <typename TW>
__global__ void copy_to_store_kernel(const float *__restrict__ master, TW *__restrict__ wstore,
                                     long long len)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        stf(wstore + i, master[i]);
}

// Input features of one sample, channels-last [z][y][x][kFeatures]:
//  0: (log10 Ra - 4.5) / 1.5   1..3: one-hot wall type   4..6: x, y, z in [-1, 1]
//  7: the conduction profile 1/2 - Y (Y = (y + 1/2)/n)
template <typename T>
__global__ void features_kernel(const double *__restrict__ ra, const int *__restrict__ wall,
                                T *__restrict__ out, int batch, int n)
{
    // the per-sample feature (log10 Ra - 4.5) / 1.5, once per block (FP64 is slow)
    extern __shared__ float feat_ra[];
    for (int b = threadIdx.x; b < batch; b += blockDim.x)
        feat_ra[b] = static_cast<float>((log10(ra[b]) - 4.5) / 1.5);
    __syncthreads();
    const long long vox = static_cast<long long>(n) * n * n;
    const long long len = batch * vox;
    const float h = 1.0f / n;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int b = static_cast<int>(i / vox);
        int r = static_cast<int>(i - b * vox);
        const int xx = r % n;
        r /= n;
        const int yy = r % n;
        const int zz = r / n;
        const int wl = wall[b];
        const F4 lo{{feat_ra[b], wl == 1 ? 1.f : 0.f, wl == 2 ? 1.f : 0.f, wl == 3 ? 1.f : 0.f}};
        const F4 hi{{2.f * (xx + 0.5f) * h - 1.f, 2.f * (yy + 0.5f) * h - 1.f, 2.f * (zz + 0.5f) * h - 1.f,
                     0.5f - (yy + 0.5f) * h}};
        st4(out + i * kFeatures, lo);
        st4(out + i * kFeatures + 4, hi);
    }
}

// Trilinear resampling of one channels-last sample [m^3][c] (cell-centred
// grids on the same unit cube) to planar fields: channel k (< 5) becomes
// plane[k] of out ([*][N^3], float), as scale[k] * value + offset[k].
struct ResampleMap {
    int plane[5];
    float scale[5], offset[5];
};

template <typename T>
__global__ void resample_kernel(const T *__restrict__ in, int m, int c, float *__restrict__ out, int N,
                                const ResampleMap map)
{
    const long long vox = static_cast<long long>(N) * N * N;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < vox;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int xx = static_cast<int>(i % N);
        const int yy = static_cast<int>((i / N) % N);
        const int zz = static_cast<int>(i / (static_cast<long long>(N) * N));
        // position in input cell units, clamped to the range of cell centres
        auto coord = [&](int k, int &i0, float &f) {
            float p = (k + 0.5f) * m / N - 0.5f;
            p = fminf(fmaxf(p, 0.f), static_cast<float>(m - 1));
            i0 = static_cast<int>(floorf(p));
            if (i0 > m - 2) i0 = m - 2 > 0 ? m - 2 : 0;
            f = p - i0;
            if (m == 1) f = 0.f;
        };
        int x0, y0, z0;
        float fx, fy, fz;
        coord(xx, x0, fx);
        coord(yy, y0, fy);
        coord(zz, z0, fz);
        const int x1 = m > 1 ? x0 + 1 : x0, y1 = m > 1 ? y0 + 1 : y0, z1 = m > 1 ? z0 + 1 : z0;
        for (int k = 0; k < c && k < 5; ++k) {
            auto at = [&](int z, int y, int x) {
                return ldf(in + ((static_cast<long long>(z) * m + y) * m + x) * c + k);
            };
            const float c00 = at(z0, y0, x0) * (1 - fx) + at(z0, y0, x1) * fx;
            const float c01 = at(z0, y1, x0) * (1 - fx) + at(z0, y1, x1) * fx;
            const float c10 = at(z1, y0, x0) * (1 - fx) + at(z1, y0, x1) * fx;
            const float c11 = at(z1, y1, x0) * (1 - fx) + at(z1, y1, x1) * fx;
            const float c0 = c00 * (1 - fy) + c01 * fy, c1 = c10 * (1 - fy) + c11 * fy;
            out[map.plane[k] * vox + i] = fmaf(map.scale[k], c0 * (1 - fz) + c1 * fz, map.offset[k]);
        }
    }
}

template <typename T>
__global__ void widen_kernel(const T *__restrict__ in, float *__restrict__ out, long long len)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        out[i] = ldf(in + i);
}

__global__ void fill_kernel(float *__restrict__ p, float v, long long len)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        p[i] = v;
}

// Training target of one sample from planar fields, channels-last:
// out[v] = ((u_x, u_y, u_z) / u_c, theta, (rho - 1) / (3 u_c^2)).
__global__ void target_kernel(const float *__restrict__ u, const float *__restrict__ theta,
                              const float *__restrict__ rho, long long vox, float inv_uc,
                              float *__restrict__ out)
{
    const float inv_r = inv_uc * inv_uc / 3.0f;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < vox;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        out[5 * i + 0] = u[i] * inv_uc;
        out[5 * i + 1] = u[vox + i] * inv_uc;
        out[5 * i + 2] = u[2 * vox + i] * inv_uc;
        out[5 * i + 3] = theta[i];
        out[5 * i + 4] = rho ? (rho[i] - 1.0f) * inv_r : 0.0f;
    }
}

// Device word counting tcgen05 waits that ran out (see conv3d_umma_kernel).
__device__ int g_umma_err;

int *umma_error_word()
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_umma_err) != cudaSuccess) return nullptr;
    return static_cast<int *>(p);
}

// The tcgen05 convolution is used unless DMRT_NN_NO_TCGEN05 is set in the
// environment (read once).
bool umma_enabled()
{
    static const bool on = std::getenv("DMRT_NN_NO_TCGEN05") == nullptr;
    return on;
}

// Dynamic shared memory of conv3d_umma_kernel<CO>.  DMRT_UMMA_SMEM (bytes)
// overrides it with a larger allocation.
#ifndef DMRT_UMMA_SMEM
#define DMRT_UMMA_SMEM 0
#endif
template <int CO>
unsigned umma_smem()
{
    const unsigned need = um_smem_bytes<CO>();
    return DMRT_UMMA_SMEM > need ? DMRT_UMMA_SMEM : need;
}

// Elements per block of sum_chunks_kernel and its grid: one thread per
// element when there are few chunks, else 32 elements (fewer when len is
// smaller) with the remaining threads as lanes over the chunks.
int sum_width(long long len, int chunks)
{
    if (chunks <= 16) return 256;
    int e = 1;
    while (e < 32 && e < len) e *= 2;
    return e;
}
unsigned sum_blocks(long long len, int chunks)
{
    const int e = sum_width(len, chunks);
    return static_cast<unsigned>((len + e - 1) / e);
}

unsigned flat_blocks(long long len)
{
    long long b = (len + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return static_cast<unsigned>(b);
}

// Tensor map of a channels-last bf16 activation tensor [batch][n][n][n][cin]
// as the 5-D (c, x, y, z, sample) tensor conv3d_umma_tma_kernel loads its
// halo planes from: boxes of 8 channels x 10 x 18 x 1 x 1, zeros outside.
// False if the driver's encoder is missing or rejects the shape.
bool encode_act_map(const void *x, int batch, int n, int cin, CUtensorMap *map)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t N = static_cast<cuuint64_t>(n), C = static_cast<cuuint64_t>(cin);
    const cuuint64_t dims[5] = {C, N, N, N, static_cast<cuuint64_t>(batch)};
    const cuuint64_t strides[4] = {C * 2, N * C * 2, N * N * C * 2, N * N * N * C * 2};
    const cuuint32_t box[5] = {8, static_cast<cuuint32_t>(kUmHX), static_cast<cuuint32_t>(kUmHY), 1, 1};
    const cuuint32_t unit[5] = {1, 1, 1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(x), dims, strides, box, unit,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// ---------------------------------------------------------------- launchers

int tensor_core_errors(bool reset)
{
    int *p = umma_error_word();
    if (!p) return -1;
    int v = 0;
    if (cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (reset && cudaMemset(p, 0, sizeof v) != cudaSuccess) return -1;
    return v;
}

template <typename TI, typename TW, typename TO>
cudaError_t conv3d(const TI *x, const TW *w, const float *bias, TO *y, int batch, int n, int cin,
                   int cout, int k, int act, cudaStream_t s)
{
    if (n % kTile != 0 || (k != 1 && k != 3)) return cudaErrorInvalidValue;
    if (k == 1 && cin <= 16 && cout <= 16 && (cin < 8 || cout < 8)) {
        const long long voxels = static_cast<long long>(batch) * n * n * n;
        conv1x1_small_kernel<TI, TW, TO, 16, 16><<<flat_blocks(voxels), 256, 0, s>>>(x, w, bias, y, voxels, cin,
                                                                                  cout, act);
        return cudaGetLastError();
    }
    const int tiles = n / kTile;
    dim3 grid(static_cast<unsigned>(tiles) * tiles * n * batch, (cout + kCoTile - 1) / kCoTile);
    if constexpr (std::is_same_v<TI, __nv_bfloat16> && std::is_same_v<TW, __nv_bfloat16>) {
        // tensor cores: channels are read in 16-byte granules of 8, so the
        // channel count and both base pointers must keep 16-byte alignment
        const bool aligned =
            ((reinterpret_cast<unsigned long long>(x) | reinterpret_cast<unsigned long long>(w)) & 15ull) == 0;
        if (k == 3 && aligned && (cin == 8 || cin == 16 || cin == 32) && (cout == 16 || cout == 32) &&
            n % kUmY == 0 && umma_enabled()) {
            // stream along z: each CTA walks a run of zrun planes of one 8 x 16
            // column, the run chosen for the kernel's resident CTAs (conv_zrun)
            const long long xy = static_cast<long long>(batch) * (n / kUmX) * (n / kUmY);
            int *err = umma_error_word();
            if (!err) return cudaErrorInvalidValue;
            cudaError_t e = cudaSuccess;
            CUtensorMap xmap;
            if (encode_act_map(x, batch, n, cin, &xmap)) {
                // halo planes by TMA
                auto go_tma = [&](auto kernel, unsigned smem) {
                    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                    if (e != cudaSuccess) return;
                    // resident CTAs per SM of this variant: its shared memory
                    // (plus the 1 KB the runtime reserves per CTA) against the
                    // SM's 228 KB, at most DMRT_UMMA_CTAS_PER_SM (the launch
                    // bounds' minimum)
                    const int per_sm = std::max(
                        1, std::min(DMRT_UMMA_CTAS_PER_SM, static_cast<int>((228u * 1024u) / (smem + 1024u))));
                    const int zrun = conv_zrun(xy, n, per_sm * sm_count());
                    const unsigned grid = static_cast<unsigned>(xy * ((n + zrun - 1) / zrun));
                    kernel<<<grid, kUtThreads, smem, s>>>(xmap, w, bias, y, n, cin, cout, act, zrun, err);
                };
                if (cout == 16 && cin <= 16) go_tma(conv3d_umma_tma_kernel<16, 2, TO>, ut_smem_bytes<16, 2>());
                else if (cout == 16) go_tma(conv3d_umma_tma_kernel<16, 4, TO>, ut_smem_bytes<16, 4>());
                else if (cin <= 16) go_tma(conv3d_umma_tma_kernel<32, 2, TO>, ut_smem_bytes<32, 2>());
                else go_tma(conv3d_umma_tma_kernel<32, 4, TO>, ut_smem_bytes<32, 4>());
                if (e != cudaSuccess) return e;
                return cudaGetLastError();
            }
            // the driver's encoder rejected the shape: the plane-at-a-time kernel below
        }
        if (k == 3 && aligned && (cin == 8 || cin % 16 == 0) && cout % 16 == 0 && n % kUmY == 0 &&
            umma_enabled()) {
            const unsigned tiles = static_cast<unsigned>(batch) * (n / kUmX) * (n / kUmY) * n;
            int *err = umma_error_word();
            if (!err) return cudaErrorInvalidValue;
            cudaError_t e;
            if (cout % 64 == 0) {
                const unsigned smem = umma_smem<64>();
                e = cudaFuncSetAttribute(conv3d_umma_kernel<64, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                if (e != cudaSuccess) return e;
                conv3d_umma_kernel<64, TO><<<dim3(tiles, cout / 64), 128, smem, s>>>(x, w, bias, y, n, cin, cout, act,
                                                                                   err);
            } else if (cout % 32 == 0) {
                const unsigned smem = umma_smem<32>();
                e = cudaFuncSetAttribute(conv3d_umma_kernel<32, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                if (e != cudaSuccess) return e;
                conv3d_umma_kernel<32, TO><<<dim3(tiles, cout / 32), 128, smem, s>>>(x, w, bias, y, n, cin, cout, act,
                                                                                   err);
            } else {
                const unsigned smem = umma_smem<16>();
                e = cudaFuncSetAttribute(conv3d_umma_kernel<16, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                if (e != cudaSuccess) return e;
                conv3d_umma_kernel<16, TO><<<dim3(tiles, cout / 16), 128, smem, s>>>(x, w, bias, y, n, cin, cout, act,
                                                                                   err);
            }
            return cudaGetLastError();
        }
        if (k == 3 && aligned && (cin == 8 || cin % 16 == 0) && cout % 16 == 0 && n % kWtX == 0 &&
            n % kWtZ == 0) {
            const unsigned vtiles = static_cast<unsigned>(batch) * (n / kWtX) * (n / kWtY) * (n / kWtZ);
            // the dynamic shared memory exceeds the 48 KB default: opt in (per
            // call, so every device the kernel runs on gets the attribute)
            cudaError_t e;
            // 32 output channels per block, unless that leaves most SMs idle
            // (the 8^3 level: 32 blocks of 32 channels at batch 4): 16 per
            // block doubles the blocks; every output accumulates the same
            // MMAs in the same order either way, so the results are the same
            if (cout % 32 == 0 && vtiles * static_cast<unsigned>(cout / 32) >= 2u * sm_count()) {
                const int smem = (kWtHalo + 27 * 32) * kWtRow * 2;
                e = cudaFuncSetAttribute(conv3d_tc_kernel<4, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                if (e != cudaSuccess) return e;
                conv3d_tc_kernel<4, TO><<<dim3(vtiles, cout / 32), 256, smem, s>>>(x, w, bias, y, n, cin, cout, act);
            } else {
                const int smem = (kWtHalo + 27 * 16) * kWtRow * 2;
                e = cudaFuncSetAttribute(conv3d_tc_kernel<2, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                if (e != cudaSuccess) return e;
                conv3d_tc_kernel<2, TO><<<dim3(vtiles, cout / 16), 256, smem, s>>>(x, w, bias, y, n, cin, cout, act);
            }
            return cudaGetLastError();
        }
        if (cin % 8 == 0 && aligned) {
            if (k == 3)
                conv3d_mma_kernel<3, TO><<<grid, 128, 0, s>>>(x, w, bias, y, n, cin, cout, act);
            else
                conv3d_mma_kernel<1, TO><<<grid, 128, 0, s>>>(x, w, bias, y, n, cin, cout, act);
            return cudaGetLastError();
        }
    }
    if (k == 3)
        conv3d_kernel<TI, TW, TO, 3><<<grid, 256, 0, s>>>(x, w, bias, y, n, cin, cout, act);
    else
        conv3d_kernel<TI, TW, TO, 1><<<grid, 256, 0, s>>>(x, w, bias, y, n, cin, cout, act);
    return cudaGetLastError();
}

cudaError_t conv3d_wgrad_bf16(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *dw, float *scratch,
                              size_t scratch_floats, int batch, int n, int cin, int cout, int k,
                              cudaStream_t s)
{
    const bool aligned =
        ((reinterpret_cast<unsigned long long>(x) | reinterpret_cast<unsigned long long>(dy)) & 15ull) == 0;
    if (cin % 8 != 0 || cout % 8 != 0 || !aligned || (k != 1 && k != 3)) return cudaErrorInvalidValue;
    if (k == 3 && cout % 16 == 0 && (cin == 8 || cin % 16 == 0) && n % kWtX == 0 && n % kWtZ == 0) {
        const int ci_tiles = cin > 8 ? cin / 16 : 1;
        const long long blocks_per_chunk = static_cast<long long>(cout / 16) * ci_tiles;
        const long long pairs = static_cast<long long>(cin) * cout;
        const int tiles_per_sample = (n / kWtX) * (n / kWtY) * (n / kWtZ);
        const long long total_tiles = static_cast<long long>(batch) * tiles_per_sample;
        // one wave of 3 resident blocks per SM: fewer chunks keep the final
        // sum over chunks short
        long long chunks = (152 * 3 + blocks_per_chunk - 1) / blocks_per_chunk;
        if (chunks > total_tiles) chunks = total_tiles;
        while (chunks > 1 && static_cast<size_t>(chunks * 27 * pairs) > scratch_floats) chunks /= 2;
        if (static_cast<size_t>(chunks * 27 * pairs) > scratch_floats) return cudaErrorInvalidValue;
        const long long per = (total_tiles + chunks - 1) / chunks;
        chunks = (total_tiles + per - 1) / per;
        dim3 grid(static_cast<unsigned>(blocks_per_chunk), static_cast<unsigned>(chunks));
        wgrad_taps_kernel<<<grid, 256, 0, s>>>(x, dy, scratch, n, cin, cout, tiles_per_sample,
                                               static_cast<int>(total_tiles), static_cast<int>(per));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const long long len = 27 * pairs;
        sum_chunks_kernel<<<sum_blocks(len, static_cast<int>(chunks)), 256, 0, s>>>(
        scratch, dw, len, static_cast<int>(chunks), sum_width(len, static_cast<int>(chunks)));
        return cudaGetLastError();
    }
    const long long total = static_cast<long long>(batch) * n * n * n;
    const int taps = k * k * k;
    const int cogs = (cout + 63) / 64, cigs = (cin + 31) / 32;
    const long long pairs = static_cast<long long>(cin) * cout;
    const long long blocks_per_chunk = static_cast<long long>(taps) * cogs * cigs;
    long long chunks = (152 * 16 + blocks_per_chunk - 1) / blocks_per_chunk;
    const long long max_chunks = (total + kWgVox - 1) / kWgVox;
    if (chunks > max_chunks) chunks = max_chunks;
    while (chunks > 1 && static_cast<size_t>(chunks * taps * pairs) > scratch_floats) chunks /= 2;
    if (static_cast<size_t>(chunks * taps * pairs) > scratch_floats) return cudaErrorInvalidValue;
    // chunks of whole stages
    long long chunk = (total + chunks - 1) / chunks;
    chunk = (chunk + kWgVox - 1) / kWgVox * kWgVox;
    chunks = (total + chunk - 1) / chunk;
    dim3 grid(static_cast<unsigned>(blocks_per_chunk), static_cast<unsigned>(chunks));
    if (k == 3)
        wgrad_mma_kernel<3><<<grid, 128, 0, s>>>(x, dy, scratch, batch, n, cin, cout, static_cast<int>(chunk), cogs);
    else
        wgrad_mma_kernel<1><<<grid, 128, 0, s>>>(x, dy, scratch, batch, n, cin, cout, static_cast<int>(chunk), cogs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long len = taps * pairs;
    sum_chunks_kernel<<<sum_blocks(len, static_cast<int>(chunks)), 256, 0, s>>>(
        scratch, dw, len, static_cast<int>(chunks), sum_width(len, static_cast<int>(chunks)));
    return cudaGetLastError();
}

template <typename TI>
cudaError_t conv3d_wgrad(const TI *x, const float *dy, float *dw, float *scratch,
                         size_t scratch_floats, int batch, int n, int cin, int cout, int k,
                         cudaStream_t s)
{
    const long long total = static_cast<long long>(batch) * n * n * n;
    if (k == 1 && cout <= 8 && cin <= 16) {
        long long blocks = 152 * 4;
        if (blocks > total) blocks = total;
        const long long pairs = static_cast<long long>(cin) * cout;
        while (blocks > 1 && static_cast<size_t>(blocks * pairs) > scratch_floats) blocks /= 2;
        const long long chunk = (total + blocks - 1) / blocks;
        blocks = (total + chunk - 1) / chunk;
        if (cout <= 5)
            wgrad_small_kernel<TI, 5, 16><<<static_cast<unsigned>(blocks), 256, 0, s>>>(x, dy, scratch, total, cin,
                                                                                        cout, chunk);
        else
            wgrad_small_kernel<TI, 8, 16><<<static_cast<unsigned>(blocks), 256, 0, s>>>(x, dy, scratch, total, cin,
                                                                                        cout, chunk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        sum_chunks_kernel<<<sum_blocks(pairs, static_cast<int>(blocks)), 256, 0, s>>>(
        scratch, dw, pairs, static_cast<int>(blocks), sum_width(pairs, static_cast<int>(blocks)));
        return cudaGetLastError();
    }
    if (cin > 128 || cout > 128 || 256 % cin != 0) return cudaErrorInvalidValue;
    const int taps = k * k * k;
    const long long pairs = static_cast<long long>(cin) * cout;
    // chunks of voxels: enough blocks to fill the GPU, bounded by the scratch
    long long chunks = (152 * 8 + taps - 1) / taps;
    if (chunks > total) chunks = total;
    while (chunks > 1 && static_cast<size_t>(chunks * taps * pairs) > scratch_floats) chunks /= 2;
    if (static_cast<size_t>(chunks * taps * pairs) > scratch_floats) return cudaErrorInvalidValue;
    const int chunk = static_cast<int>((total + chunks - 1) / chunks);
    chunks = (total + chunk - 1) / chunk;
    dim3 grid(taps, static_cast<unsigned>(chunks));
    if (k == 3)
        conv3d_wgrad_kernel<TI, 3><<<grid, 256, 0, s>>>(x, dy, scratch, batch, n, cin, cout, chunk);
    else
        conv3d_wgrad_kernel<TI, 1><<<grid, 256, 0, s>>>(x, dy, scratch, batch, n, cin, cout, chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long len = taps * pairs;
    sum_chunks_kernel<<<sum_blocks(len, static_cast<int>(chunks)), 256, 0, s>>>(
        scratch, dw, len, static_cast<int>(chunks), sum_width(len, static_cast<int>(chunks)));
    return cudaGetLastError();
}

cudaError_t bias_grad(const float *dy, float *db, float *scratch, size_t scratch_floats,
                      long long voxels, int cout, cudaStream_t s)
{
    if (cout < 1 || cout > 256) return cudaErrorInvalidValue;
    long long blocks = 152 * 2;
    if (blocks > voxels) blocks = voxels;
    while (blocks > 1 && static_cast<size_t>(blocks * cout) > scratch_floats) blocks /= 2;
    const long long chunk = (voxels + blocks - 1) / blocks;
    blocks = (voxels + chunk - 1) / chunk;
    bias_grad_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(dy, scratch, voxels, cout, chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_chunks_kernel<<<sum_blocks(cout, static_cast<int>(blocks)), 256, 0, s>>>(
        scratch, db, cout, static_cast<int>(blocks), sum_width(cout, static_cast<int>(blocks)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t act_backward_narrow(const T *yout, float *dy, __nv_bfloat16 *dyn, long long len, int act,
                                cudaStream_t s)
{
    const bool aligned =
        ((reinterpret_cast<unsigned long long>(dy) & 15ull) | (reinterpret_cast<unsigned long long>(dyn) & 7ull)) == 0;
    if (len % 4 != 0 || !aligned) return cudaErrorInvalidValue;
    act_backward_narrow_kernel<T><<<flat_blocks(len / 4), 256, 0, s>>>(yout, dy, dyn, len / 4, act);
    return cudaGetLastError();
}

template <typename T>
cudaError_t act_backward_narrow_bias(const T *yout, float *dy, __nv_bfloat16 *dyn, long long voxels, int cout,
                                     int act, float *db, float *scratch, size_t scratch_floats, cudaStream_t s)
{
    constexpr int kBlocks = 152 * 4;
    const bool aligned =
        ((reinterpret_cast<unsigned long long>(dy) & 15ull) | (reinterpret_cast<unsigned long long>(dyn) & 7ull)) == 0;
    if (cout % 4 != 0 || 256 % (cout / 4) != 0 || !aligned || static_cast<size_t>(kBlocks) * cout > scratch_floats)
        return cudaErrorInvalidValue;
    const long long len4 = voxels * cout / 4;
    act_backward_narrow_bias_kernel<T><<<kBlocks, 256, 0, s>>>(yout, dy, dyn, len4, act, cout / 4, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_chunks_kernel<<<sum_blocks(cout, kBlocks), 256, 0, s>>>(scratch, db, cout, kBlocks, sum_width(cout, kBlocks));
    return cudaGetLastError();
}

template <typename T>
cudaError_t act_backward(const T *yout, float *dy, long long len, cudaStream_t s)
{
    act_backward_kernel<T><<<flat_blocks(len), 256, 0, s>>>(yout, dy, len);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t flip_transpose(const TW *w, TW *wt, int k, int cout, int cin, cudaStream_t s)
{
    const int taps = k * k * k;
    flip_transpose_kernel<TW><<<flat_blocks(static_cast<long long>(taps) * cout * cin), 256, 0, s>>>(
        w, wt, taps, cout, cin);
    return cudaGetLastError();
}

template <typename T>
cudaError_t avgpool2(const T *x, T *y, int batch, int n, int c, cudaStream_t s)
{
    if (c % 4 != 0) return cudaErrorInvalidValue;
    const long long len = static_cast<long long>(batch) * (n / 2) * (n / 2) * (n / 2) * (c / 4);
    avgpool2_kernel<T><<<flat_blocks(len), 256, 0, s>>>(x, y, batch, n, c);
    return cudaGetLastError();
}

cudaError_t avgpool2_backward(const float *dy, float *dx, int batch, int n, int c, cudaStream_t s)
{
    if (c % 4 != 0) return cudaErrorInvalidValue;
    const long long len = static_cast<long long>(batch) * n * n * n * (c / 4);
    avgpool2_backward_kernel<<<flat_blocks(len), 256, 0, s>>>(dy, dx, batch, n, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t up2_add(const T *x, const T *skip, T *y, int batch, int n, int c, cudaStream_t s)
{
    if (c % 4 != 0) return cudaErrorInvalidValue;
    const long long len = static_cast<long long>(batch) * 8LL * n * n * n * (c / 4);
    up2_add_kernel<T><<<flat_blocks(len), 256, 0, s>>>(x, skip, y, batch, n, c);
    return cudaGetLastError();
}

cudaError_t up2_backward(const float *dy, float *dx, int batch, int n, int c, cudaStream_t s)
{
    if (c % 4 != 0) return cudaErrorInvalidValue;
    const long long len = static_cast<long long>(batch) * n * n * n * (c / 4);
    up2_backward_kernel<<<flat_blocks(len), 256, 0, s>>>(dy, dx, batch, n, c);
    return cudaGetLastError();
}

cudaError_t add_inplace(float *a, const float *b, long long len, cudaStream_t s)
{
    if (len % 4 != 0) return cudaErrorInvalidValue;
    add_inplace_kernel<<<flat_blocks(len / 4), 256, 0, s>>>(a, b, len / 4);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mse(const T *yp, const float *tgt, float *dy, double *partials, double *loss,
                long long len, cudaStream_t s)
{
    const unsigned blocks = 256;
    mse_kernel<T><<<blocks, 256, 0, s>>>(yp, tgt, dy, partials, len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_doubles_kernel<<<1, 32, 0, s>>>(partials, blocks, 1.0 / static_cast<double>(len), loss);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t adam(float *master, TW *wstore, const float *grad, float *m1, float *m2, long long len,
                 float lr, float beta1, float beta2, float eps, int t, cudaStream_t s)
{
    const float bc1 = 1.f - powf(beta1, static_cast<float>(t));
    const float bc2 = 1.f - powf(beta2, static_cast<float>(t));
    adam_kernel<TW><<<flat_blocks(len), 256, 0, s>>>(master, wstore, grad, m1, m2, len, lr, beta1,
                                                     beta2, eps, bc1, bc2);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t copy_to_store(const float *master, TW *wstore, long long len, cudaStream_t s)
{
    copy_to_store_kernel<TW><<<flat_blocks(len), 256, 0, s>>>(master, wstore, len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t features(const double *ra, const int *wall, T *out, int batch, int n, cudaStream_t s)
{
    const size_t smem = static_cast<size_t>(batch) * sizeof(float);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    features_kernel<T><<<flat_blocks(static_cast<long long>(batch) * n * n * n), 256, smem, s>>>(
        ra, wall, out, batch, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t resample(const T *in, int m, int c, float *out, int N, const int plane[5],
                     const float scale[5], const float offset[5], cudaStream_t s)
{
    ResampleMap map;
    for (int k = 0; k < 5; ++k) {
        map.plane[k] = plane[k];
        map.scale[k] = scale[k];
        map.offset[k] = offset[k];
    }
    resample_kernel<T><<<flat_blocks(static_cast<long long>(N) * N * N), 256, 0, s>>>(in, m, c, out, N, map);
    return cudaGetLastError();
}

template <typename T>
cudaError_t widen(const T *in, float *out, long long len, cudaStream_t s)
{
    widen_kernel<T><<<flat_blocks(len), 256, 0, s>>>(in, out, len);
    return cudaGetLastError();
}

cudaError_t narrow(const float *in, __nv_bfloat16 *out, long long len, cudaStream_t s)
{
    narrow_kernel<<<flat_blocks(len), 256, 0, s>>>(in, out, len);
    return cudaGetLastError();
}

cudaError_t fill(float *p, float v, long long len, cudaStream_t s)
{
    fill_kernel<<<flat_blocks(len), 256, 0, s>>>(p, v, len);
    return cudaGetLastError();
}

cudaError_t target_from_fields(const float *u, const float *theta, const float *rho, long long vox,
                               float inv_uc, float *out, cudaStream_t s)
{
    target_kernel<<<flat_blocks(vox), 256, 0, s>>>(u, theta, rho, vox, inv_uc, out);
    return cudaGetLastError();
}

// explicit instantiations for float and bfloat16 storage
#define DMRT_NN_INST(T)                                                                        \
    template cudaError_t conv3d<T, T, T>(const T *, const T *, const float *, T *, int, int, int, \
                                         int, int, int, cudaStream_t);                          \
    template cudaError_t conv3d_wgrad<T>(const T *, const float *, float *, float *, size_t, int, \
                                         int, int, int, int, cudaStream_t);                     \
    template cudaError_t act_backward<T>(const T *, float *, long long, cudaStream_t);          \
    template cudaError_t act_backward_narrow<T>(const T *, float *, __nv_bfloat16 *, long long, int, \
                                                cudaStream_t);                                  \
    template cudaError_t act_backward_narrow_bias<T>(const T *, float *, __nv_bfloat16 *, long long, int, int, \
                                                     float *, float *, size_t, cudaStream_t);   \
    template cudaError_t flip_transpose<T>(const T *, T *, int, int, int, cudaStream_t);        \
    template cudaError_t avgpool2<T>(const T *, T *, int, int, int, cudaStream_t);              \
    template cudaError_t up2_add<T>(const T *, const T *, T *, int, int, int, cudaStream_t);    \
    template cudaError_t mse<T>(const T *, const float *, float *, double *, double *,          \
                                long long, cudaStream_t);                                       \
    template cudaError_t adam<T>(float *, T *, const float *, float *, float *, long long,      \
                                 float, float, float, float, int, cudaStream_t);                \
    template cudaError_t copy_to_store<T>(const float *, T *, long long, cudaStream_t);         \
    template cudaError_t features<T>(const double *, const int *, T *, int, int, cudaStream_t); \
    template cudaError_t resample<T>(const T *, int, int, float *, int, const int *, const float *, \
                                     const float *, cudaStream_t);                                 \
    template cudaError_t widen<T>(const T *, float *, long long, cudaStream_t);

DMRT_NN_INST(float)
DMRT_NN_INST(__nv_bfloat16)
#undef DMRT_NN_INST
// input gradients of bf16 layers on tensor cores: bf16 gradients, FP32 out
template cudaError_t conv3d<__nv_bfloat16, __nv_bfloat16, float>(const __nv_bfloat16 *,
                                                                const __nv_bfloat16 *, const float *,
                                                                float *, int, int, int, int, int, int,
                                                                cudaStream_t);
// input gradients of bf16 layers: FP32 gradients through bf16 weights
template cudaError_t conv3d<float, __nv_bfloat16, float>(const float *, const __nv_bfloat16 *,
                                                        const float *, float *, int, int, int, int,
                                                        int, int, cudaStream_t);

}  // namespace nn
}  // namespace lbm
