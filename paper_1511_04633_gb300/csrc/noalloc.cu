// noalloc.cu -- dmrt_nusselt_noalloc: the Nusselt-number reduction of a
// caller's temperature field, with no device allocation at any point.
//
// Some callers may not allocate device memory once they are running: a host
// application whose own memory pool already owns the device memory, or a
// time-critical loop where a cudaMalloc / cudaFree would stall the device.
// This entry point serves them.  Its scratch (one partial per z row plus the
// three results) lives in a file-scope __device__ array of fixed size that the
// CUDA driver places when the library's module is loaded; every GPU that
// loads the library keeps that array until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host the name
// is only a stand-in, not a device address.  Every call, with the caller's
// device current, looks up the real address with cudaGetSymbolAddress (which
// allocates nothing); nothing is cached, so the call stays correct after the
// caller resets the device or tears down its context.
#include "dmrt.h"

namespace {

// Largest nz (number of z rows of the wall) one call accepts.
constexpr int kNoAllocMaxRows = 8192;
constexpr int kNoAllocThreads = 256;

// [0, 3*kNoAllocMaxRows): per-row (sum, centre-column sum, max) of local Nu;
// [3*kNoAllocMaxRows, +3): Nu_3D, Nu_2D, Nu_max of the last call.
static __device__ __align__(256) double g_nu_scratch[3 * kNoAllocMaxRows + 4];

__device__ __forceinline__ double nu_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double nu_warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Fixed-order block reduction of (sum, centre sum, max); thread 0 gets them.
__device__ void nu_block_reduce(double &s, double &mid, double &mx)
{
    __shared__ double sh[kNoAllocThreads / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s = nu_warp_sum(s);
    mid = nu_warp_sum(mid);
    mx = nu_warp_max(mx);
    if (lane == 0) {
        sh[warp][0] = s;
        sh[warp][1] = mid;
        sh[warp][2] = mx;
    }
    __syncthreads();
    if (warp == 0) {
        const bool live = lane < kNoAllocThreads / 32;
        s = nu_warp_sum(live ? sh[lane][0] : 0.0);
        mid = nu_warp_sum(live ? sh[lane][1] : 0.0);
        mx = nu_warp_max(live ? sh[lane][2] : -INFINITY);
    }
    __syncthreads();
}

// One block per z row: local Nu on the wall from theta 1/2 and 3/2 cells
// off it (same discretisation as dmrt_nusselt); every row slot is written.
__global__ void __launch_bounds__(kNoAllocThreads) nu_rows_noalloc(const float *__restrict__ theta,
                                                                   int nx, int ny, int wall,
                                                                   double *scratch)
{
    const int z = blockIdx.x;
    const int y1 = wall == 0 ? 0 : ny - 1;
    const int y2 = wall == 0 ? 1 : ny - 2;
    const double th_w = wall == 0 ? 0.5 : -0.5;
    const double H = static_cast<double>(ny);
    const int c_lo = (nx % 2 == 0) ? nx / 2 - 1 : (nx - 1) / 2;
    const int c_hi = (nx % 2 == 0) ? nx / 2 : (nx - 1) / 2;
    double s = 0.0, mid = 0.0, mx = -INFINITY;
    for (int x = threadIdx.x; x < nx; x += kNoAllocThreads) {
        const double t1 = theta[(static_cast<long long>(z) * ny + y1) * nx + x];
        const double t2 = theta[(static_cast<long long>(z) * ny + y2) * nx + x];
        const double dth_ds = (-8.0 * th_w + 9.0 * t1 - t2) / 3.0;
        const double nu = wall == 0 ? -H * dth_ds : H * dth_ds;
        s += nu;
        if (x == c_lo || x == c_hi) mid += nu;
        mx = fmax(mx, nu);
    }
    nu_block_reduce(s, mid, mx);
    if (threadIdx.x == 0) {
        scratch[3 * z + 0] = s;
        scratch[3 * z + 1] = mid;
        scratch[3 * z + 2] = mx;
    }
}

// Sums the nz row partials in a fixed order into the three result slots.
__global__ void __launch_bounds__(kNoAllocThreads) nu_finish_noalloc(int nx, int nz,
                                                                     double *scratch)
{
    double s = 0.0, mid = 0.0, mx = -INFINITY;
    for (int z = threadIdx.x; z < nz; z += kNoAllocThreads) {
        s += scratch[3 * z + 0];
        mid += scratch[3 * z + 1];
        mx = fmax(mx, scratch[3 * z + 2]);
    }
    nu_block_reduce(s, mid, mx);
    if (threadIdx.x == 0) {
        double *out = scratch + 3 * kNoAllocMaxRows;
        const int ncol = (nx % 2 == 0) ? 2 : 1;
        out[0] = s / (static_cast<double>(nx) * nz);
        out[1] = mid / (static_cast<double>(nz) * ncol);
        out[2] = mx;
    }
}

// Device address of the scratch array on the current device.
cudaError_t scratch_address(double **out)
{
    double *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_nu_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" dmrt_status dmrt_nusselt_noalloc(const float *theta, int nx, int ny, int nz, int wall,
                                            void *stream, double out[3])
{
    if (!theta || !out || nx < 1 || ny < 2 || nz < 1 || (wall != 0 && wall != 1))
        return DMRT_ERR_ARG;
    if (nz > kNoAllocMaxRows) return DMRT_ERR_ARG;
    if (static_cast<long long>(nx) * ny * nz >= (1LL << 31)) return DMRT_ERR_ARG;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return DMRT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    nu_rows_noalloc<<<nz, kNoAllocThreads, 0, s>>>(theta, nx, ny, wall, scratch);
    if (cudaGetLastError() != cudaSuccess) return DMRT_ERR_CUDA;
    nu_finish_noalloc<<<1, kNoAllocThreads, 0, s>>>(nx, nz, scratch);
    if (cudaGetLastError() != cudaSuccess) return DMRT_ERR_CUDA;
    if (cudaMemcpyAsync(out, scratch + 3 * kNoAllocMaxRows, 3 * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DMRT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DMRT_ERR_CUDA;
    return DMRT_OK;
}
