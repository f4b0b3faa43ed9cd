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
#include <cuda_bf16.h>

#include <type_traits>

#include "internal.h"
#include "nn.h"

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

// out[i] = sum over chunks (in order) of partials[chunk][i]
__global__ void sum_chunks_kernel(const float *__restrict__ partials, float *__restrict__ out,
                                  long long len, int chunks)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < chunks; ++c) s += partials[c * len + i];
        out[i] = s;
    }
}

// Bias gradient partials: per block of voxels, the sum of dy over them.
__global__ void bias_grad_kernel(const float *__restrict__ dy, float *__restrict__ partials,
                                 long long voxels, int cout, int chunk)
{
    const long long v0 = static_cast<long long>(blockIdx.x) * chunk;
    const long long v1 = v0 + chunk < voxels ? v0 + chunk : voxels;
    for (int c = threadIdx.x; c < cout; c += blockDim.x) {
        float s = 0.f;
        for (long long v = v0; v < v1; ++v) s += dy[v * cout + c];
        partials[static_cast<long long>(blockIdx.x) * cout + c] = s;
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

template <typename T>
__global__ void avgpool2_kernel(const T *__restrict__ x, T *__restrict__ y, int batch, int n, int c)
{
    const int m = n / 2;
    const long long len = static_cast<long long>(batch) * m * m * m * c;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ch = static_cast<int>(i % c);
        long long r = i / c;
        const int ox = static_cast<int>(r % m);
        r /= m;
        const int oy = static_cast<int>(r % m);
        r /= m;
        const int oz = static_cast<int>(r % m);
        const long long b = r / m;
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * oz + (k >> 2), yy = 2 * oy + ((k >> 1) & 1), xx = 2 * ox + (k & 1);
            s += ldf(x + (((b * n + zz) * n + yy) * n + xx) * c + ch);
        }
        stf(y + i, 0.125f * s);
    }
}

// gradient of avgpool2: dx = dy / 8 broadcast (FP32)
__global__ void avgpool2_backward_kernel(const float *__restrict__ dy, float *__restrict__ dx,
                                         int batch, int n, int c)
{
    const int m = n / 2;
    const long long len = static_cast<long long>(batch) * n * n * n * c;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ch = static_cast<int>(i % c);
        long long r = i / c;
        const int xx = static_cast<int>(r % n);
        r /= n;
        const int yy = static_cast<int>(r % n);
        r /= n;
        const int zz = static_cast<int>(r % n);
        const long long b = r / n;
        dx[i] = 0.125f * dy[(((b * m + zz / 2) * m + yy / 2) * m + xx / 2) * c + ch];
    }
}

// nearest upsampling x2 (n -> 2n), plus an optional skip added: y = up(x) + s
template <typename T>
__global__ void up2_add_kernel(const T *__restrict__ x, const T *__restrict__ skip, T *__restrict__ y,
                               int batch, int n, int c)
{
    const int m = 2 * n;
    const long long len = static_cast<long long>(batch) * m * m * m * c;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ch = static_cast<int>(i % c);
        long long r = i / c;
        const int xx = static_cast<int>(r % m);
        r /= m;
        const int yy = static_cast<int>(r % m);
        r /= m;
        const int zz = static_cast<int>(r % m);
        const long long b = r / m;
        float v = ldf(x + (((b * n + zz / 2) * n + yy / 2) * n + xx / 2) * c + ch);
        if (skip) v += ldf(skip + i);
        stf(y + i, v);
    }
}

// gradient of nearest upsampling: dx = sum of the 8 children of dy (FP32)
__global__ void up2_backward_kernel(const float *__restrict__ dy, float *__restrict__ dx, int batch,
                                    int n, int c)
{
    const int m = 2 * n;
    const long long len = static_cast<long long>(batch) * n * n * n * c;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ch = static_cast<int>(i % c);
        long long r = i / c;
        const int ox = static_cast<int>(r % n);
        r /= n;
        const int oy = static_cast<int>(r % n);
        r /= n;
        const int oz = static_cast<int>(r % n);
        const long long b = r / n;
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * oz + (k >> 2), yy = 2 * oy + ((k >> 1) & 1), xx = 2 * ox + (k & 1);
            s += dy[(((b * m + zz) * m + yy) * m + xx) * c + ch];
        }
        dx[i] = s;
    }
}

__global__ void add_inplace_kernel(float *__restrict__ a, const float *__restrict__ b, long long len)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        a[i] += b[i];
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
    const long long vox = static_cast<long long>(n) * n * n;
    const long long len = batch * vox;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long b = i / vox;
        long long r = i % vox;
        const int xx = static_cast<int>(r % n);
        r /= n;
        const int yy = static_cast<int>(r % n);
        const int zz = static_cast<int>(r / n);
        T *o = out + i * kFeatures;
        const float h = 1.0f / n;
        stf(o + 0, static_cast<float>((log10(ra[b]) - 4.5) / 1.5));
        stf(o + 1, wall[b] == 1 ? 1.f : 0.f);
        stf(o + 2, wall[b] == 2 ? 1.f : 0.f);
        stf(o + 3, wall[b] == 3 ? 1.f : 0.f);
        stf(o + 4, 2.f * (xx + 0.5f) * h - 1.f);
        stf(o + 5, 2.f * (yy + 0.5f) * h - 1.f);
        stf(o + 6, 2.f * (zz + 0.5f) * h - 1.f);
        stf(o + 7, 0.5f - (yy + 0.5f) * h);
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

unsigned flat_blocks(long long len)
{
    long long b = (len + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return static_cast<unsigned>(b);
}

}  // namespace

// ---------------------------------------------------------------- launchers

template <typename TI, typename TW, typename TO>
cudaError_t conv3d(const TI *x, const TW *w, const float *bias, TO *y, int batch, int n, int cin,
                   int cout, int k, int act, cudaStream_t s)
{
    if (n % kTile != 0 || (k != 1 && k != 3)) return cudaErrorInvalidValue;
    const int tiles = n / kTile;
    dim3 grid(static_cast<unsigned>(tiles) * tiles * n * batch, (cout + kCoTile - 1) / kCoTile);
    if constexpr (std::is_same_v<TI, __nv_bfloat16> && std::is_same_v<TW, __nv_bfloat16>) {
        // tensor cores: channels are read in 16-byte granules of 8, so the
        // channel count and both base pointers must keep 16-byte alignment
        const bool aligned =
            ((reinterpret_cast<unsigned long long>(x) | reinterpret_cast<unsigned long long>(w)) & 15ull) == 0;
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
    sum_chunks_kernel<<<flat_blocks(len), 256, 0, s>>>(scratch, dw, len, static_cast<int>(chunks));
    return cudaGetLastError();
}

template <typename TI>
cudaError_t conv3d_wgrad(const TI *x, const float *dy, float *dw, float *scratch,
                         size_t scratch_floats, int batch, int n, int cin, int cout, int k,
                         cudaStream_t s)
{
    if (cin > 128 || cout > 128 || 256 % cin != 0) return cudaErrorInvalidValue;
    const long long total = static_cast<long long>(batch) * n * n * n;
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
    sum_chunks_kernel<<<flat_blocks(len), 256, 0, s>>>(scratch, dw, len, static_cast<int>(chunks));
    return cudaGetLastError();
}

cudaError_t bias_grad(const float *dy, float *db, float *scratch, size_t scratch_floats,
                      long long voxels, int cout, cudaStream_t s)
{
    long long blocks = 152 * 4;
    if (blocks > voxels) blocks = voxels;
    while (blocks > 1 && static_cast<size_t>(blocks * cout) > scratch_floats) blocks /= 2;
    const int chunk = static_cast<int>((voxels + blocks - 1) / blocks);
    blocks = (voxels + chunk - 1) / chunk;
    bias_grad_kernel<<<static_cast<unsigned>(blocks), 128, 0, s>>>(dy, scratch, voxels, cout, chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_chunks_kernel<<<flat_blocks(cout), 256, 0, s>>>(scratch, db, cout, static_cast<int>(blocks));
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
    const long long len = static_cast<long long>(batch) * (n / 2) * (n / 2) * (n / 2) * c;
    avgpool2_kernel<T><<<flat_blocks(len), 256, 0, s>>>(x, y, batch, n, c);
    return cudaGetLastError();
}

cudaError_t avgpool2_backward(const float *dy, float *dx, int batch, int n, int c, cudaStream_t s)
{
    const long long len = static_cast<long long>(batch) * n * n * n * c;
    avgpool2_backward_kernel<<<flat_blocks(len), 256, 0, s>>>(dy, dx, batch, n, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t up2_add(const T *x, const T *skip, T *y, int batch, int n, int c, cudaStream_t s)
{
    const long long len = static_cast<long long>(batch) * 8LL * n * n * n * c;
    up2_add_kernel<T><<<flat_blocks(len), 256, 0, s>>>(x, skip, y, batch, n, c);
    return cudaGetLastError();
}

cudaError_t up2_backward(const float *dy, float *dx, int batch, int n, int c, cudaStream_t s)
{
    const long long len = static_cast<long long>(batch) * n * n * n * c;
    up2_backward_kernel<<<flat_blocks(len), 256, 0, s>>>(dy, dx, batch, n, c);
    return cudaGetLastError();
}

cudaError_t add_inplace(float *a, const float *b, long long len, cudaStream_t s)
{
    add_inplace_kernel<<<flat_blocks(len), 256, 0, s>>>(a, b, len);
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
    features_kernel<T><<<flat_blocks(static_cast<long long>(batch) * n * n * n), 256, 0, s>>>(
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
