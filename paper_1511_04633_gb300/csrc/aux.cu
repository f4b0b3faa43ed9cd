// aux.cu -- the non-step kernels: fields of the pulled populations
// (Eqs. (20), (30)), the convergence residual, the Nusselt numbers
// (Eqs. (39)-(41)) and population / field import-export.
//
// Reductions are deterministic: each block reduces its cells in a fixed
// warp-shuffle tree into an FP64 partial, and one finishing block sums the
// partials in index order.  No floating-point atomics are used.
#include <cmath>

#include "internal.h"
#include "reduce.cuh"

namespace lbm {

namespace {

constexpr int kRedThreads = 256;  // threads of the per-cell reduction blocks
constexpr int kFinThreads = 512;  // threads of the finishing blocks

// ---------------------------------------------------------------- fields

template <int WALL, typename T>
__global__ void fields_kernel(const T *__restrict__ src, const Geometry G, float *rho, float *u,
                              float *theta)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= G.nx || y >= G.ny) return;
    float d[19], g[7];
    pull_f<WALL, T>(src, G, x, y, z, d);
    pull_g<WALL, T>(src, G, x, y, z, g);
    const Macro m = macro_of(d, g);
    const float r = 1.0f + m.drho;
    const long long c = (static_cast<long long>(z) * G.ny + y) * G.nx + x;
    const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
    if (rho) rho[c] = r;
    if (u) {
        u[c] = m.jx / r;
        u[cells + c] = m.jy / r;
        u[2 * cells + c] = m.jz / r;
    }
    if (theta) theta[c] = m.T;
}

// ---------------------------------------------------------------- residual

// Per block: sums of |dtheta|^2, |theta|^2, |du|^2, |u|^2 against the
// snapshot, which is then overwritten with the current fields.  Each cell's
// terms are FP32 (the difference of two floats, then fused squares), summed
// in FP32 over a warp's 32 cells and in FP64 from there on.
template <int WALL, typename T>
__global__ void __launch_bounds__(kRedThreads) residual_kernel(
    const T *__restrict__ src, const Geometry G, float *__restrict__ snap, int have_prev,
    double *__restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (x < G.nx && y < G.ny) {
        const long long c = (static_cast<long long>(z) * G.ny + y) * G.nx + x;
        const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
        // the snapshot is read before any of it is written back (and before
        // the pull), so its four loads overlap the population loads instead
        // of following one another behind possibly aliasing stores
        float prev[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) prev[k] = snap[k * cells + c];
        float d[19], g[7];
        pull_f<WALL, T>(src, G, x, y, z, d);
        pull_g<WALL, T>(src, G, x, y, z, g);
        const Macro m = macro_of(d, g);
        const float r = 1.0f + m.drho;
        const float now[4] = {m.T, m.jx / r, m.jy / r, m.jz / r};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dk = have_prev ? now[k] - prev[k] : 0.0f;
            const int slot = (k == 0) ? 0 : 2;
            v[slot] = __fmaf_rn(dk, dk, v[slot]);
            v[slot + 1] = __fmaf_rn(now[k], now[k], v[slot + 1]);
            snap[k * cells + c] = now[k];
        }
    }
    double s[4];
    block_sum_f32<4, kRedThreads>(v, s);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long b = (static_cast<long long>(blockIdx.z) * gridDim.y + blockIdx.y) *
                                gridDim.x + blockIdx.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) partials[b * 4 + k] = s[k];
    }
}

__device__ double rel_change(double num2, double den2)
{
    if (den2 == 0.0) return num2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(num2) / sqrt(den2);
}

__global__ void __launch_bounds__(kFinThreads) residual_finish(const double *__restrict__ partials,
                                                                 long long nparts, int have_prev,
                                                                 int K, double *result)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long p = threadIdx.x; p < nparts; p += kFinThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += partials[p * 4 + k];
    block_sum<4, kFinThreads>(v);
    if (threadIdx.x == 0) {
        bool finite = true;
        for (int k = 0; k < 4; ++k) {
            result[k] = v[k];
            finite = finite && isfinite(v[k]);
        }
        double r = have_prev ? fmax(rel_change(v[0], v[1]), rel_change(v[2], v[3])) / K : INFINITY;
        result[4] = finite ? r : NAN;
        result[5] = finite ? 0.0 : 1.0;
    }
}

// ---------------------------------------------------------------- Nusselt

// One block per z row: the local Nu of every wall cell of that row, from the
// pulled temperatures 1/2 and 3/2 cells off the wall (Eq. (39)).
template <int WALL, typename T>
__global__ void __launch_bounds__(kRedThreads) nusselt_kernel(const T *__restrict__ src,
                                                               const Geometry G, int wall,
                                                               float *local,
                                                               double *__restrict__ partials)
{
    const int z = blockIdx.x;
    const int y1 = wall == 0 ? 0 : G.ny - 1;
    const int y2 = wall == 0 ? 1 : G.ny - 2;
    const double th_w = wall == 0 ? 0.5 : -0.5;
    const double H = static_cast<double>(G.ny);
    const int c_lo = (G.nx % 2 == 0) ? G.nx / 2 - 1 : (G.nx - 1) / 2;
    const int c_hi = (G.nx % 2 == 0) ? G.nx / 2 : (G.nx - 1) / 2;
    double v[2] = {0.0, 0.0};
    double mx = -INFINITY;
    for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
        float g[7];
        pull_g<WALL, T>(src, G, x, y1, z, g);
        float t1 = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) t1 += g[i];
        pull_g<WALL, T>(src, G, x, y2, z, g);
        float t2 = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) t2 += g[i];
        const double dth_ds = (-8.0 * th_w + 9.0 * t1 - static_cast<double>(t2)) / 3.0;
        const double nu = wall == 0 ? -H * dth_ds : H * dth_ds;
        if (local) local[static_cast<long long>(z) * G.nx + x] = static_cast<float>(nu);
        v[0] += nu;
        if (x == c_lo || x == c_hi) v[1] += nu;
        mx = fmax(mx, nu);
    }
    __shared__ double shm[kRedThreads / 32];
    mx = warp_max(mx);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) shm[warp] = mx;
    block_sum<2, kRedThreads>(v);
    if (threadIdx.x == 0) {
        double m = shm[0];
        for (int w = 1; w < kRedThreads / 32; ++w) m = fmax(m, shm[w]);
        partials[z * 3 + 0] = v[0];
        partials[z * 3 + 1] = v[1];
        partials[z * 3 + 2] = m;
    }
}

// Sums the per-row partials in a fixed order: each thread takes rows
// t, t + 256, ...; then one fixed shuffle tree.
__global__ void __launch_bounds__(kRedThreads) nusselt_finish(const double *__restrict__ partials,
                                                               const Geometry G, double *out3)
{
    double v[2] = {0.0, 0.0};
    double mx = -INFINITY;
    for (int z = threadIdx.x; z < G.nz; z += kRedThreads) {
        v[0] += partials[z * 3 + 0];
        v[1] += partials[z * 3 + 1];
        mx = fmax(mx, partials[z * 3 + 2]);
    }
    __shared__ double shm[kRedThreads / 32];
    mx = warp_max(mx);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) shm[warp] = mx;
    block_sum<2, kRedThreads>(v);
    if (threadIdx.x == 0) {
        double m = shm[0];
        for (int w = 1; w < kRedThreads / 32; ++w) m = fmax(m, shm[w]);
        const int ncol = (G.nx % 2 == 0) ? 2 : 1;
        out3[0] = v[0] / (static_cast<double>(G.nx) * G.nz);
        out3[1] = v[1] / (static_cast<double>(G.nz) * ncol);
        out3[2] = m;
    }
}

// Link-flux Nusselt number of one z row: the heat carried across the wall
// links in one step by the stored populations of the first fluid layer,
// q = 2 w_T theta_w - 2 g*_(-y) (hot wall) or 2 g*_(+y) - 2 w_T theta_w
// (cold wall), Nu = H q / alpha.  Same per-row partials as nusselt_kernel.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) nusselt_flux_kernel(const T *__restrict__ src,
                                                                    const Geometry G, int wall,
                                                                    double inv_alpha, float *local,
                                                                    double *__restrict__ partials)
{
    const int z = blockIdx.x;
    const int y = wall == 0 ? 0 : G.ny - 1;
    const int plane = wall == 0 ? 19 + 4 : 19 + 3;  // D3Q7 -y / +y
    const double th_w = wall == 0 ? 0.5 : -0.5;
    const double H = static_cast<double>(G.ny);
    const int c_lo = (G.nx % 2 == 0) ? G.nx / 2 - 1 : (G.nx - 1) / 2;
    const int c_hi = (G.nx % 2 == 0) ? G.nx / 2 : (G.nx - 1) / 2;
    double v[2] = {0.0, 0.0};
    double mx = -INFINITY;
    for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
        const long long c = (static_cast<long long>(z) * G.ny + y) * G.nx + x;
        const double gl = Store<T>::ld(src + state_index(G, false, plane, c, x, y, z));
        const double q = wall == 0 ? 0.25 * th_w - 2.0 * gl : 2.0 * gl - 0.25 * th_w;
        const double nu = H * q * inv_alpha;
        if (local) local[static_cast<long long>(z) * G.nx + x] = static_cast<float>(nu);
        v[0] += nu;
        if (x == c_lo || x == c_hi) v[1] += nu;
        mx = fmax(mx, nu);
    }
    __shared__ double shm[kRedThreads / 32];
    mx = warp_max(mx);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) shm[warp] = mx;
    block_sum<2, kRedThreads>(v);
    if (threadIdx.x == 0) {
        double m = shm[0];
        for (int w = 1; w < kRedThreads / 32; ++w) m = fmax(m, shm[w]);
        partials[z * 3 + 0] = v[0];
        partials[z * 3 + 1] = v[1];
        partials[z * 3 + 2] = m;
    }
}

// ---------------------------------------------------------------- import / export

// Coordinates of the flat cell index c.
__device__ __forceinline__ void cell_xyz(const Geometry &G, long long c, int &x, int &y, int &z)
{
    x = static_cast<int>(c % G.nx);
    const long long r = c / G.nx;
    y = static_cast<int>(r % G.ny);
    z = static_cast<int>(r / G.ny);
}

// The state slots are addressed through state_index, so import and export
// see the same dense [q][cells] arrays whatever the buffer's layout.
template <typename T>
__global__ void set_populations_kernel(const float *__restrict__ f, const float *__restrict__ g,
                                       T *__restrict__ dst, const Geometry G, bool periodic)
{
    const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c < cells;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x = 0, y = 0, z = 0;  // only the streamed layout needs the coordinates
        if (G.layout == kLayoutStreamed) cell_xyz(G, c, x, y, z);
        static_for<0, 19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            Store<T>::st(dst + state_index(G, periodic, i, c, x, y, z), f[i * cells + c] - q19_w(i));
        });
        for (int i = 0; i < 7; ++i)
            Store<T>::st(dst + state_index(G, periodic, 19 + i, c, x, y, z), g[i * cells + c]);
    }
}

template <typename T>
__global__ void get_populations_kernel(const T *__restrict__ src, float *f, float *g,
                                       const Geometry G, bool periodic)
{
    const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c < cells;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x = 0, y = 0, z = 0;  // only the streamed layout needs the coordinates
        if (G.layout == kLayoutStreamed) cell_xyz(G, c, x, y, z);
        if (f)
            static_for<0, 19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                f[i * cells + c] = Store<T>::ld(src + state_index(G, periodic, i, c, x, y, z)) + q19_w(i);
            });
        if (g)
            for (int i = 0; i < 7; ++i)
                g[i * cells + c] = Store<T>::ld(src + state_index(G, periodic, 19 + i, c, x, y, z));
    }
}

// Equilibrium of given fields: d_i = f_eq,i(rho, u) - w_i (Eq. (17)) and
// g_i = w_T,i theta (1 + 4 e_i.u), the velocity form of n_eq (Eq. (33)).
template <typename T>
__global__ void init_fields_kernel(const float *__restrict__ rho, const float *__restrict__ u,
                                   const float *__restrict__ theta, T *__restrict__ dst,
                                   const Geometry G, bool periodic)
{
    const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c < cells;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x = 0, y = 0, z = 0;  // only the streamed layout needs the coordinates
        if (G.layout == kLayoutStreamed) cell_xyz(G, c, x, y, z);
        const float r = rho[c];
        const float dr = r - 1.0f;
        const float vx = u[c], vy = u[cells + c], vz = u[2 * cells + c];
        const float th = theta[c];
        const float vv = vx * vx + vy * vy + vz * vz;
        static_for<0, 19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr float ex = q19_ex(i), ey = q19_ey(i), ez = q19_ez(i);
            const float ev = ex * vx + ey * vy + ez * vz;
            Store<T>::st(dst + state_index(G, periodic, i, c, x, y, z),
                         q19_w(i) * (dr + r * (3.0f * ev + 4.5f * ev * ev - 1.5f * vv)));
        });
        static_for<0, 7>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr float ex = q7_ex(i), ey = q7_ey(i), ez = q7_ez(i);
            Store<T>::st(dst + state_index(G, periodic, 19 + i, c, x, y, z),
                         q7_w(i) * th * (1.0f + 4.0f * (ex * vx + ey * vy + ez * vz)));
        });
    }
}

// The storage rounding of the step kernel applied to a flat array.
template <typename T, bool SR>
__global__ void round_kernel(const float *in, float *out, long long n, unsigned seed)
{
    const unsigned hs = pcg_hash(seed);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        T v;
        if constexpr (SR) StoreSR<T>::st(&v, in[i], pcg_hash(static_cast<unsigned>(i) ^ hs));
        else Store<T>::st(&v, in[i]);
        out[i] = Store<T>::ld(&v);
    }
}

dim3 cell_grid(const Geometry &G, dim3 block)
{
    return dim3((G.nx + block.x - 1) / block.x, (G.ny + block.y - 1) / block.y, G.nz);
}

dim3 flat_grid(const Geometry &G)
{
    const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
    long long blocks = (cells + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    return dim3(static_cast<unsigned>(blocks));
}

const dim3 kRedBlock(32, kRedThreads / 32, 1);

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_fields(int wall, int storage, const void *src, const Geometry &G, float *rho,
                          float *u, float *theta, cudaStream_t s)
{
    const dim3 block(32, 4, 1);
    const dim3 grid = cell_grid(G, block);
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        fields_kernel<decltype(W)::value, T>
            <<<grid, block, 0, s>>>(static_cast<const T *>(src), G, rho, u, theta);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t residual_partials(const Geometry &G)
{
    dim3 grid = cell_grid(G, kRedBlock);
    return static_cast<size_t>(grid.x) * grid.y * grid.z;
}

cudaError_t launch_residual(int wall, int storage, const void *src, const Geometry &G,
                            float *snap, int have_prev, int K, double *partials, double *result,
                            cudaStream_t s)
{
    const dim3 grid = cell_grid(G, kRedBlock);
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        residual_kernel<decltype(W)::value, T>
            <<<grid, kRedBlock, 0, s>>>(static_cast<const T *>(src), G, snap, have_prev, partials);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long nparts = static_cast<long long>(grid.x) * grid.y * grid.z;
    residual_finish<<<1, kFinThreads, 0, s>>>(partials, nparts, have_prev, K, result);
    return cudaGetLastError();
}

cudaError_t launch_nusselt(int wall_type, int storage, const void *src, const Geometry &G,
                           int wall, float *local, double *partials, double *out3,
                           cudaStream_t s)
{
    cudaError_t e = dispatch(wall_type, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        nusselt_kernel<decltype(W)::value, T>
            <<<G.nz, kRedThreads, 0, s>>>(static_cast<const T *>(src), G, wall, local, partials);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nusselt_finish<<<1, kRedThreads, 0, s>>>(partials, G, out3);
    return cudaGetLastError();
}

cudaError_t launch_nusselt_flux(int storage, const void *src, const Geometry &G, int wall, double alpha,
                                float *local, double *partials, double *out3, cudaStream_t s)
{
    cudaError_t e = dispatch(1, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        nusselt_flux_kernel<T><<<G.nz, kRedThreads, 0, s>>>(static_cast<const T *>(src), G, wall, 1.0 / alpha,
                                                            local, partials);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nusselt_finish<<<1, kRedThreads, 0, s>>>(partials, G, out3);
    return cudaGetLastError();
}

cudaError_t launch_set_populations(int storage, const float *f, const float *g, void *dst,
                                   const Geometry &G, bool periodic, cudaStream_t s)
{
    cudaError_t e = dispatch(0, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        set_populations_kernel<T><<<flat_grid(G), 256, 0, s>>>(f, g, static_cast<T *>(dst), G, periodic);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_get_populations(int storage, const void *src, float *f, float *g,
                                   const Geometry &G, bool periodic, cudaStream_t s)
{
    cudaError_t e = dispatch(0, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        get_populations_kernel<T><<<flat_grid(G), 256, 0, s>>>(static_cast<const T *>(src), f, g, G, periodic);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_round(int storage, bool stochastic, const float *in, float *out, long long n,
                         unsigned seed, cudaStream_t s)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    cudaError_t e = dispatch(0, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        if constexpr (!std::is_same_v<T, float>) {
            if (stochastic) {
                round_kernel<T, true><<<static_cast<unsigned>(blocks), 256, 0, s>>>(in, out, n, seed);
                return cudaSuccess;
            }
        }
        round_kernel<T, false><<<static_cast<unsigned>(blocks), 256, 0, s>>>(in, out, n, seed);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_init_fields(int storage, const float *rho, const float *u, const float *theta,
                               void *dst, const Geometry &G, bool periodic, cudaStream_t s)
{
    cudaError_t e = dispatch(0, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        init_fields_kernel<T><<<flat_grid(G), 256, 0, s>>>(rho, u, theta, static_cast<T *>(dst), G, periodic);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lbm
