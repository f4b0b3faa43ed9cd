// lattice.cuh -- device-side lattice and per-cell arithmetic of the fused
// double-MRT step (arXiv:1511.04633, Sec. 3).
//
// Everything here is resolved at compile time: the velocity sets, weights and
// the moment bases are constexpr functions, and every loop over populations or
// moments is a static_for, so the 19x19 and 7x7 transforms become straight-line
// FP32 adds with the zero entries removed.
//
// Storage convention of the GPU path: the D3Q19 populations are kept as
// deviations d_i = f_i - w_i from the rest equilibrium (rho = 1, V = 0), the
// D3Q7 populations g_i as they are (the rest temperature is theta = 0).  The
// moments of w are (1, -11, 3, 0, ..., 0), exactly the equilibrium moments at
// rest, so working on deviations changes no arithmetic of the collision; it
// only keeps FP32 rounding relative to the small deviations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

namespace lbm {

// ---------------------------------------------------------------- storage formats

// Population storage in HBM.  Every format holds the deviations f_i - w_i and
// the energy populations g_i; the collision always runs in FP32.
//  float         : as is (104 bytes per cell and buffer).
//  __nv_bfloat16 : rounded to nearest (52 bytes per cell and buffer).
//  __half        : stored times 2^10, rounded to nearest.  The deviations and
//                  g_i stay below ~0.2 in magnitude, so the scale keeps values
//                  down to ~6e-8 out of the FP16 subnormal range while the
//                  largest stay far below the FP16 maximum.  The scale is a
//                  power of two, so it adds no rounding of its own.  (The
//                  paired step kernels keep it through the collision instead
//                  of applying it at every load and store: pair_body.cuh.)
template <typename T>
struct Store;

template <>
struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};

template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

template <>
struct Store<__half> {
    static constexpr float kScale = 1024.0f;
    static __device__ __forceinline__ float ld(const __half *p)
    {
        return __half2float(*p) * (1.0f / kScale);
    }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v * kScale); }
};

// Storage code of the C ABI (0 = F32, 1 = BF16, 2 = F16) -> element size.
inline int storage_bytes(int storage) { return storage == 0 ? 4 : 2; }

// ---------------------------------------------------------------- stochastic rounding

// A 16-bit store rounds away every per-step change smaller than half an ulp,
// so a slowly evolving population stops evolving (the solution stagnates).
// Stochastic rounding keeps the expected stored value equal to the FP32 value:
// it rounds up with probability (v - lower) / ulp.  The random bits come from
// the PCG hash (one step of the 32-bit LCG with multiplier 747796405 and
// increment 2891336453, then the RXS-M-XS output permutation; O'Neill 2014, in
// the single-call form of Jarzynski and Olano, JCGT 9(3), 2020) of the cell
// index and the step number, spread over the 26 planes of a cell by a Weyl
// sequence with the golden-ratio increment.
__host__ __device__ __forceinline__ unsigned pcg_hash(unsigned v)
{
    const unsigned state = v * 747796405u + 2891336453u;
    const unsigned word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

constexpr unsigned kWeyl = 0x9E3779B9u;  // 2^32 / golden ratio

// The rounding itself is the hardware's stochastic-rounding conversion
// (cvt.rs, PTX ISA 8.7, sm_100a and later), which adds the random bits below
// the kept mantissa bits and truncates; one instruction per value.  Measured
// on GB300 it made the FP16 step 23 % and the BF16 step 5 % faster than the
// same rounding done with integer instructions.  Only the converted value of
// the pair's low half is kept.
template <typename T>
struct StoreSR;

template <>
struct StoreSR<__nv_bfloat16> {
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, unsigned r)
    {
        unsigned pair;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(pair) : "f"(0.0f), "f"(v), "r"(r));
        *reinterpret_cast<unsigned short *>(p) = static_cast<unsigned short>(pair);
    }
};

// half: the value times the 2^10 storage scale (exact), rounded likewise.
template <>
struct StoreSR<__half> {
    static __device__ __forceinline__ void st(__half *p, float v, unsigned r)
    {
        unsigned pair;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;"
            : "=r"(pair)
            : "f"(0.0f), "f"(v * Store<__half>::kScale), "r"(r));
        *reinterpret_cast<unsigned short *>(p) = static_cast<unsigned short>(pair);
    }
};

// ---------------------------------------------------------------- compile-time loops

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------- D3Q19 (Eqs. (12), (18))

__host__ __device__ constexpr int q19_ex(int i)
{
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int q19_ey(int i)
{
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int q19_ez(int i)
{
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int q19_e2(int i)
{
    return q19_ex(i) * q19_ex(i) + q19_ey(i) * q19_ey(i) + q19_ez(i) * q19_ez(i);
}
// weight w_i = 1/3 (rest), 1/18 (faces), 1/36 (edges)
__host__ __device__ constexpr float q19_w(int i)
{
    return q19_e2(i) == 0 ? 1.0f / 3.0f : (q19_e2(i) == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr int q19_opp(int i)
{
    int r = 0;
    for (int k = 0; k < 19; ++k)
        if (q19_ex(k) == -q19_ex(i) && q19_ey(k) == -q19_ey(i) && q19_ez(k) == -q19_ez(i)) r = k;
    return r;
}

// D3Q19 moment basis (Eq. (21), with row 14 = e_x e_y), written as the
// polynomials that define the moments of Eq. (22).
__host__ __device__ constexpr int m19(int k, int i)
{
    const int x = q19_ex(i), y = q19_ey(i), z = q19_ez(i);
    const int e2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1;                                   // rho
    case 1: return 19 * e2 - 30;                        // e
    case 2: return (21 * e2 * e2 - 53 * e2 + 24) / 2;   // epsilon
    case 3: return x;                                   // j_x
    case 4: return (5 * e2 - 9) * x;                    // q_x
    case 5: return y;                                   // j_y
    case 6: return (5 * e2 - 9) * y;                    // q_y
    case 7: return z;                                   // j_z
    case 8: return (5 * e2 - 9) * z;                    // q_z
    case 9: return 3 * x * x - e2;                      // 3 p_xx
    case 10: return (3 * e2 - 5) * (3 * x * x - e2);    // 3 pi_xx
    case 11: return y * y - z * z;                      // p_ww
    case 12: return (3 * e2 - 5) * (y * y - z * z);     // pi_ww
    case 13: return x * y;                              // p_xy
    case 14: return y * z;                              // p_yz
    case 15: return x * z;                              // p_xz
    case 16: return (y * y - z * z) * x;                // m_x
    case 17: return (z * z - x * x) * y;                // m_y
    default: return (x * x - y * y) * z;                // m_z
    }
}
__host__ __device__ constexpr int m19_norm2(int k)
{
    int s = 0;
    for (int i = 0; i < 19; ++i) s += m19(k, i) * m19(k, i);
    return s;
}

// ---------------------------------------------------------------- D3Q7 (Eqs. (28), (31), (32))

__host__ __device__ constexpr int q7_ex(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
__host__ __device__ constexpr int q7_ey(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
__host__ __device__ constexpr int q7_ez(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
__host__ __device__ constexpr int q7_opp(int i) { return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1); }
__host__ __device__ constexpr float q7_w(int i) { return i == 0 ? 0.25f : 0.125f; }

__host__ __device__ constexpr int m7(int k, int i)
{
    const int x = q7_ex(i), y = q7_ey(i), z = q7_ez(i);
    const int e2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return 6 - 7 * e2;
    case 5: return 3 * x * x - e2;
    default: return y * y - z * z;
    }
}
__host__ __device__ constexpr int m7_norm2(int k)
{
    int s = 0;
    for (int i = 0; i < 7; ++i) s += m7(k, i) * m7(k, i);
    return s;
}

// ---------------------------------------------------------------- per-step parameters

// Relaxation rates divided by the squared norm of their basis vector, so the
// back-transform M^-1 = M^T diag(1/|M_k|^2) needs no further scaling.
struct CollideParams {
    float rs[19];     // s_k / |M_k|^2 (Eq. (26)); entries 0,3,5,7 unused
    float ws[19];     // (1 - s_k) / |M_k|^2; entries 0,3,5,7 unused
    float rq[7];      // q_k / |N_k|^2 (Eqs. (35),(36)); entry 0 unused
    float gbeta;      // g beta dT (lattice units)
    float theta_ref;  // reference temperature of Eq. (16)
    // anisotropic diffusion (Eqs. (35)-(37) with off-diagonal tau_bar): the
    // 3x3 block of Q acting on the flux moments, divided by |N_k|^2 = 2;
    // used instead of rq[1..3] when aniso != 0
    float qa[9];
    int aniso;
};

// Relaxation rates of Eq. (26): s_k of the D3Q19 moments, except the five
// set by the viscosity (viscous_moment(k): s_nu = 1/(3 nu + 1/2)); the
// energy rates q_k of Eqs. (35),(36) are 1 except q_1..3 = 1/tau_a.
__host__ __device__ constexpr bool viscous_moment(int k)
{
    return k == 9 || k == 11 || k == 13 || k == 14 || k == 15;
}
__host__ __device__ constexpr double mrt_rate(int k)
{
    return k == 1 ? 1.19
         : (k == 2 || k == 10 || k == 12) ? 1.4
         : (k == 4 || k == 6 || k == 8) ? 1.2
         : (k >= 16) ? 1.98
         : 1.0;  // conserved moments 0, 3, 5, 7 (unused)
}

// The collision parameters of a cavity with viscosity nu, diffusivity alpha
// and buoyancy g beta dT (isotropic diffusion; aniso and qa are left alone).
inline void fill_collide_params(CollideParams &C, double nu, double alpha, double gbeta)
{
    const double s_nu = 1.0 / (3.0 * nu + 0.5);  // Eq. (26)
    for (int k = 0; k < 19; ++k) {
        const double s = viscous_moment(k) ? s_nu : mrt_rate(k);
        C.rs[k] = static_cast<float>(s / m19_norm2(k));
        C.ws[k] = static_cast<float>((1.0 - s) / m19_norm2(k));
    }
    const double tau_a = 0.5 + 4.0 * alpha;  // Eq. (36), eps = 1/4, dt = dx = 1
    for (int k = 0; k < 7; ++k) {
        const double q = (k >= 1 && k <= 3) ? 1.0 / tau_a : 1.0;
        C.rq[k] = static_cast<float>(q / m7_norm2(k));
    }
    C.gbeta = static_cast<float>(gbeta);
    C.theta_ref = 0.0f;  // T_l = (T_h + T_c)/2
}

// Where the stored state sits in a population buffer.  The state S is the
// set of post-collision populations of the last step, S_i(x) for every cell x
// and direction i (planes 0..18 D3Q19, 19..25 D3Q7).
//  kLayoutAB      : two-buffer (A-B) scheme, S_i(x) in plane i at cell x.
//  kLayoutSwapped : in-place scheme after an even number of steps, S_i(x) in
//                   plane opp(i) at cell x.
//  kLayoutStreamed: in-place scheme after an odd number of steps, S_i(x) in
//                   plane i at cell x + e_i (already streamed), or in plane
//                   opp(i) at cell x when x + e_i lies outside a walled box.
constexpr int kLayoutAB = 0, kLayoutSwapped = 1, kLayoutStreamed = 2;

struct Geometry {
    int nx, ny, nz;
    int layout;       // kLayout* of the buffer the aux kernels read or write
    long long plane;  // elements between consecutive population planes
    float inv_ny;     // 1/ny for the linear wall profile
};

// Launch-parameter tables of the step kernel for walled boxes: the source of
// plane q for a cell with flat index c is c + nb[q] (the neighbour at
// c - e_q), or c + bb[q] when that link leaves the box (the opposite plane
// of the cell itself).  32-bit indices: 26 * plane < 2^32.
struct StepGeometry {
    int nx, ny, nz;
    unsigned plane;
    int nb[26];
    int bb[26];
    float inv_ny;
};

// Tables of the in-place step's first phase (the kernel that reads the
// swapped layout and writes the streamed one): loads use load.nb / load.bb
// like StepGeometry; the value leaving cell c along q goes to c + sn[q], or
// to c + sb[q] when that link leaves the box.
struct InplaceGeometry {
    StepGeometry load;
    int sn[26];
    int sb[26];
};

// ---------------------------------------------------------------- pull with walls

// theta on a linear wall (Types 2 and 3, Eqs. (7), (10)) at the height of row
// y: 1/2 - (y + 1/2)/ny, with one rounding in a fixed form, so every kernel
// that applies the wall rule gets the same value.
__device__ __forceinline__ float theta_linear(int y, float inv_ny)
{
    return __fmaf_rn(-(static_cast<float>(y) + 0.5f), inv_ny, 0.5f);
}

// Wall rule of a D3Q7 link that leaves the box through a face on `axis`
// (0 = x, 1 = y, 2 = z): true for a Dirichlet wall (anti-bounce-back).
template <int WALL>
__device__ constexpr bool dirichlet_axis(int axis)
{
    return axis == 1 || (WALL == 2) || (WALL == 3 && axis == 0);
}

// Pull the 19 D3Q19 deviations that arrive at cell (x,y,z) from the stored
// post-collision state `src` (planes 0..18).  A link that leaves the box is
// replaced by half-way bounce-back from the resting wall: f_i(x) = f*_opp(x).
template <int WALL, typename T>
__device__ __forceinline__ void pull_f(const T *__restrict__ src, const Geometry &G,
                                       int x, int y, int z, float d[19])
{
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long P = G.plane;
    const int self = (z * ny + y) * nx + x;
    const bool xlo = (x == 0), xhi = (x == nx - 1);
    const bool ylo = (y == 0), yhi = (y == ny - 1);
    const bool zlo = (z == 0), zhi = (z == nz - 1);
    // plane and cell of S_i(x - e_i) (the population arriving at x) and of
    // S_opp(x) (its bounce-back source) in the buffer's layout
    const int L = G.layout;
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q19_ex(i), ey = q19_ey(i), ez = q19_ez(i);
        constexpr int opp = q19_opp(i);
        if constexpr (i == 0) {
            d[0] = Store<T>::ld(src + self);
        } else if constexpr (WALL == 0) {
            int sx = x - ex, sy = y - ey, sz = z - ez;
            sx = sx < 0 ? nx - 1 : (sx >= nx ? 0 : sx);
            sy = sy < 0 ? ny - 1 : (sy >= ny ? 0 : sy);
            sz = sz < 0 ? nz - 1 : (sz >= nz ? 0 : sz);
            const int c = (L == kLayoutStreamed) ? self : (sz * ny + sy) * nx + sx;
            const int p_in = (L == kLayoutSwapped) ? opp : i;
            d[i] = Store<T>::ld(src + p_in * P + c);
        } else {
            bool out = false;
            if constexpr (ex == 1) out = out || xlo;
            if constexpr (ex == -1) out = out || xhi;
            if constexpr (ey == 1) out = out || ylo;
            if constexpr (ey == -1) out = out || yhi;
            if constexpr (ez == 1) out = out || zlo;
            if constexpr (ez == -1) out = out || zhi;
            const int off = ex + ey * nx + ez * nx * ny;
            const int c_in = (L == kLayoutStreamed) ? self : self - off;
            const int p_in = (L == kLayoutSwapped) ? opp : i;
            const int p_out = (L == kLayoutAB) ? opp : i;
            const long long a = out ? (p_out * P + self) : (p_in * P + c_in);
            d[i] = Store<T>::ld(src + a);
        }
    });
}

// Pull the 7 D3Q7 populations arriving at (x,y,z) from planes 19..25 of
// `src`.  A link that leaves the box takes the thermal wall rule: on a
// Dirichlet wall anti-bounce-back g_i(x) = -g*_opp(x) + 2 w_T,i theta_w, on
// an adiabatic wall bounce-back g_i(x) = g*_opp(x).  theta_w is +1/2 on the
// hot wall y = 0, -1/2 on the cold wall y = H and 1/2 - (y + 1/2)/ny on the
// linear x / z walls of Types 2 and 3 (Eqs. (6),(7),(9),(10)).
template <int WALL, typename T>
__device__ __forceinline__ void pull_g(const T *__restrict__ src, const Geometry &G,
                                       int x, int y, int z, float g[7])
{
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long P = G.plane;
    const int self = (z * ny + y) * nx + x;
    const T *gs = src + 19 * P;
    const float th_lin = theta_linear(y, G.inv_ny);
    const int L = G.layout;
    static_for<0, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q7_ex(i), ey = q7_ey(i), ez = q7_ez(i);
        constexpr int opp = q7_opp(i);
        if constexpr (i == 0) {
            g[0] = Store<T>::ld(gs + self);
        } else if constexpr (WALL == 0) {
            int sx = x - ex, sy = y - ey, sz = z - ez;
            sx = sx < 0 ? nx - 1 : (sx >= nx ? 0 : sx);
            sy = sy < 0 ? ny - 1 : (sy >= ny ? 0 : sy);
            sz = sz < 0 ? nz - 1 : (sz >= nz ? 0 : sz);
            const int c = (L == kLayoutStreamed) ? self : (sz * ny + sy) * nx + sx;
            const int p_in = (L == kLayoutSwapped) ? opp : i;
            g[i] = Store<T>::ld(gs + p_in * P + c);
        } else {
            constexpr int axis = ex != 0 ? 0 : (ey != 0 ? 1 : 2);
            bool out;
            if constexpr (ex == 1) out = (x == 0);
            else if constexpr (ex == -1) out = (x == nx - 1);
            else if constexpr (ey == 1) out = (y == 0);
            else if constexpr (ey == -1) out = (y == ny - 1);
            else if constexpr (ez == 1) out = (z == 0);
            else out = (z == nz - 1);
            const int off = ex + ey * nx + ez * nx * ny;
            const int c_in = (L == kLayoutStreamed) ? self : self - off;
            const int p_in = (L == kLayoutSwapped) ? opp : i;
            const int p_out = (L == kLayoutAB) ? opp : i;
            const long long a = out ? (p_out * P + self) : (p_in * P + c_in);
            float v = Store<T>::ld(gs + a);
            if constexpr (dirichlet_axis<WALL>(axis)) {
                float tw;
                if constexpr (axis == 1) tw = (ey == 1) ? 0.5f : -0.5f;
                else tw = th_lin;
                v = out ? (0.25f * tw - v) : v;  // 2 w_T,i = 1/4
            }
            g[i] = v;
        }
    });
}

// Element index of S_q(x) (plane q = 0..25: D3Q19 direction q, or D3Q7
// direction q - 19) of cell c = (z ny + y) nx + x in the buffer's layout.
// `periodic`: the box wraps around (no walls).
__device__ __forceinline__ long long state_index(const Geometry &G, bool periodic, int q, long long c,
                                                 int x, int y, int z)
{
    int ex, ey, ez, opp;
    if (q < 19) {
        ex = q19_ex(q);
        ey = q19_ey(q);
        ez = q19_ez(q);
        opp = q19_opp(q);
    } else {
        ex = q7_ex(q - 19);
        ey = q7_ey(q - 19);
        ez = q7_ez(q - 19);
        opp = 19 + q7_opp(q - 19);
    }
    if (G.layout == kLayoutAB) return q * G.plane + c;
    if (G.layout == kLayoutSwapped) return opp * G.plane + c;
    int tx = x + ex, ty = y + ey, tz = z + ez;
    const bool inside = tx >= 0 && tx < G.nx && ty >= 0 && ty < G.ny && tz >= 0 && tz < G.nz;
    if (!inside && !periodic) return opp * G.plane + c;
    tx = tx < 0 ? G.nx - 1 : (tx >= G.nx ? 0 : tx);
    ty = ty < 0 ? G.ny - 1 : (ty >= G.ny ? 0 : ty);
    tz = tz < 0 ? G.nz - 1 : (tz >= G.nz ? 0 : tz);
    return q * G.plane + (static_cast<long long>(tz) * G.ny + ty) * G.nx + tx;
}

// ---------------------------------------------------------------- moments

// ---------------------------------------------------------------- host dispatch

// Calls f(std::integral_constant<int, WALL>{}, (T *)nullptr) for the runtime
// wall type (0..3) and storage code (0 = float, 1 = bf16, 2 = f16); the null
// pointer only carries the storage type.
template <typename T, typename F>
inline cudaError_t dispatch_wall(int wall, F &&f)
{
    T *tp = nullptr;
    switch (wall) {
    case 0: return f(std::integral_constant<int, 0>{}, tp);
    case 1: return f(std::integral_constant<int, 1>{}, tp);
    case 2: return f(std::integral_constant<int, 2>{}, tp);
    case 3: return f(std::integral_constant<int, 3>{}, tp);
    default: return cudaErrorInvalidValue;
    }
}

template <typename F>
inline cudaError_t dispatch(int wall, int storage, F &&f)
{
    switch (storage) {
    case 0: return dispatch_wall<float>(wall, f);
    case 1: return dispatch_wall<__nv_bfloat16>(wall, f);
    case 2: return dispatch_wall<__half>(wall, f);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
