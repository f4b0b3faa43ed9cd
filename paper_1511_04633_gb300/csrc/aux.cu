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
#include "residual.cuh"
#include "step_body.cuh"

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
    // the moments as the step kernels form them (step_body.cuh), so a
    // residual point taken inside a step sees exactly these values
    const Conserved<float> m = conserved<float>(d, g);
    const long long c = (static_cast<long long>(z) * G.ny + y) * G.nx + x;
    const long long cells = static_cast<long long>(G.nx) * G.ny * G.nz;
    if (rho) rho[c] = m.rho;
    if (u) {
        u[c] = m.vx;
        u[cells + c] = m.vy;
        u[2 * cells + c] = m.vz;
    }
    if (theta) theta[c] = m.Tu;
}

// ---------------------------------------------------------------- residual

__device__ double rel_change(double num2, double den2)
{
    if (den2 == 0.0) return num2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(num2) / sqrt(den2);
}

// Block sum (fixed order) of four double-float values per thread; warp 0
// ends with the totals, lane 0 holding them.
template <int THREADS>
__device__ __forceinline__ void df_block_sum(DF v[4])
{
    __shared__ DF sh[THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] = df_add(v[k], df_shfl_down(v[k], o));
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = lane < THREADS / 32 ? sh[lane][k] : DF{0.0f, 0.0f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] = df_add(v[k], df_shfl_down(v[k], o));
        }
    }
}

constexpr int kGatherThreads = 256;
constexpr int kGatherPer = 8;  // partials per thread of a gathering block

// Finishes a residual point: adds the step kernel's `nparts` block partials
// (residual.cuh: hi, lo of the four sums per block) in double-float
// arithmetic and forms r (reading A11).  Each block adds 2048 consecutive
// partials (thread t takes t, t + 256, ...; then a fixed tree) into
// stage[block]; the block that finishes last (a ticket counter) adds the
// stage entries in index order, so the result does not depend on which
// block that is.  The totals become FP64 (hi + lo).  result[6] counts the
// points since the last reset (capped at 2); *ticket is left at 0.
__global__ void __launch_bounds__(kGatherThreads)
    residual_finish(const float *__restrict__ partials, long long nparts, float *stage, unsigned *ticket,
                    int K, double *result)
{
    DF v[4] = {};
    const long long base = static_cast<long long>(blockIdx.x) * (kGatherThreads * kGatherPer);
#pragma unroll
    for (int i = 0; i < kGatherPer; ++i) {
        const long long p = base + i * kGatherThreads + threadIdx.x;
        if (p < nparts) {
            const float4 a = *reinterpret_cast<const float4 *>(partials + p * 8);
            const float4 b = *reinterpret_cast<const float4 *>(partials + p * 8 + 4);
            v[0] = df_add(v[0], DF{a.x, a.y});
            v[1] = df_add(v[1], DF{a.z, a.w});
            v[2] = df_add(v[2], DF{b.x, b.y});
            v[3] = df_add(v[3], DF{b.z, b.w});
        }
    }
    df_block_sum<kGatherThreads>(v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        float *q = stage + 8 * static_cast<size_t>(blockIdx.x);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            q[2 * k] = v[k].hi;
            q[2 * k + 1] = v[k].lo;
        }
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    DF w[4] = {};
    for (unsigned p = threadIdx.x; p < gridDim.x; p += kGatherThreads) {
        const volatile float *q = stage + 8 * static_cast<size_t>(p);
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = df_add(w[k], DF{q[2 * k], q[2 * k + 1]});
    }
    df_block_sum<kGatherThreads>(w);
    if (threadIdx.x == 0) {
        const double points = result[6];
        double tot[4];
        bool finite = true;
        for (int k = 0; k < 4; ++k) {
            tot[k] = static_cast<double>(w[k].hi) + static_cast<double>(w[k].lo);
            result[k] = tot[k];
            finite = finite && isfinite(tot[k]);
        }
        const double r =
            points > 0.0 ? fmax(rel_change(tot[0], tot[1]), rel_change(tot[2], tot[3])) / K : INFINITY;
        result[4] = finite ? r : NAN;
        result[5] = finite ? 0.0 : 1.0;
        result[6] = fmin(points + 1.0, 2.0);
        *ticket = 0u;
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

size_t residual_stage_floats(long long nparts)
{
    const long long blocks = (nparts + kGatherThreads * kGatherPer - 1) / (kGatherThreads * kGatherPer);
    return static_cast<size_t>(blocks < 1 ? 1 : blocks) * 8;
}

cudaError_t launch_residual_finish(const float *partials, long long nparts, float *stage, unsigned *ticket,
                                  int K, double *result, cudaStream_t s)
{
    long long blocks = (nparts + kGatherThreads * kGatherPer - 1) / (kGatherThreads * kGatherPer);
    if (blocks < 1) blocks = 1;
    residual_finish<<<static_cast<unsigned>(blocks), kGatherThreads, 0, s>>>(partials, nparts, stage, ticket, K,
                                                                              result);
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
