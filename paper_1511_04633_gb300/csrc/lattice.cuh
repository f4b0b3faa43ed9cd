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

#include <cstdint>
#include <type_traits>

namespace lbm {

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
    float rq[7];      // q_k / |N_k|^2 (Eqs. (35),(36)); entry 0 unused
    float gbeta;      // g beta dT (lattice units)
    float theta_ref;  // reference temperature of Eq. (16)
};

struct Geometry {
    int nx, ny, nz;
    int pad;
    long long plane;  // elements between consecutive population planes
    float inv_ny;     // 1/ny for the linear wall profile
};

// ---------------------------------------------------------------- pull with walls

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
template <int WALL>
__device__ __forceinline__ void pull_f(const float *__restrict__ src, const Geometry &G,
                                       int x, int y, int z, float d[19])
{
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long P = G.plane;
    const int self = (z * ny + y) * nx + x;
    const bool xlo = (x == 0), xhi = (x == nx - 1);
    const bool ylo = (y == 0), yhi = (y == ny - 1);
    const bool zlo = (z == 0), zhi = (z == nz - 1);
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q19_ex(i), ey = q19_ey(i), ez = q19_ez(i);
        constexpr int opp = q19_opp(i);
        if constexpr (i == 0) {
            d[0] = src[self];
        } else if constexpr (WALL == 0) {
            int sx = x - ex, sy = y - ey, sz = z - ez;
            sx = sx < 0 ? nx - 1 : (sx >= nx ? 0 : sx);
            sy = sy < 0 ? ny - 1 : (sy >= ny ? 0 : sy);
            sz = sz < 0 ? nz - 1 : (sz >= nz ? 0 : sz);
            d[i] = src[i * P + (sz * ny + sy) * nx + sx];
        } else {
            bool out = false;
            if constexpr (ex == 1) out = out || xlo;
            if constexpr (ex == -1) out = out || xhi;
            if constexpr (ey == 1) out = out || ylo;
            if constexpr (ey == -1) out = out || yhi;
            if constexpr (ez == 1) out = out || zlo;
            if constexpr (ez == -1) out = out || zhi;
            const int off = ex + ey * nx + ez * nx * ny;
            const long long a = out ? (opp * P + self) : (i * P + (self - off));
            d[i] = src[a];
        }
    });
}

// Pull the 7 D3Q7 populations arriving at (x,y,z) from planes 19..25 of
// `src`.  A link that leaves the box takes the thermal wall rule: on a
// Dirichlet wall anti-bounce-back g_i(x) = -g*_opp(x) + 2 w_T,i theta_w, on
// an adiabatic wall bounce-back g_i(x) = g*_opp(x).  theta_w is +1/2 on the
// hot wall y = 0, -1/2 on the cold wall y = H and 1/2 - (y + 1/2)/ny on the
// linear x / z walls of Types 2 and 3 (Eqs. (6),(7),(9),(10)).
template <int WALL>
__device__ __forceinline__ void pull_g(const float *__restrict__ src, const Geometry &G,
                                       int x, int y, int z, float g[7])
{
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long P = G.plane;
    const int self = (z * ny + y) * nx + x;
    const float *gs = src + 19 * P;
    const float th_lin = 0.5f - (static_cast<float>(y) + 0.5f) * G.inv_ny;
    static_for<0, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q7_ex(i), ey = q7_ey(i), ez = q7_ez(i);
        constexpr int opp = q7_opp(i);
        if constexpr (i == 0) {
            g[0] = gs[self];
        } else if constexpr (WALL == 0) {
            int sx = x - ex, sy = y - ey, sz = z - ez;
            sx = sx < 0 ? nx - 1 : (sx >= nx ? 0 : sx);
            sy = sy < 0 ? ny - 1 : (sy >= ny ? 0 : sy);
            sz = sz < 0 ? nz - 1 : (sz >= nz ? 0 : sz);
            g[i] = gs[i * P + (sz * ny + sy) * nx + sx];
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
            const long long a = out ? (opp * P + self) : (i * P + (self - off));
            float v = gs[a];
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

// ---------------------------------------------------------------- collision

// Macroscopic moments of pulled populations (Eqs. (20), (30)).
struct Macro {
    float drho, jx, jy, jz, T;
};

__device__ __forceinline__ Macro macro_of(const float d[19], const float g[7])
{
    Macro m{0.f, 0.f, 0.f, 0.f, 0.f};
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        m.drho += d[i];
        if constexpr (q19_ex(i) == 1) m.jx += d[i];
        if constexpr (q19_ex(i) == -1) m.jx -= d[i];
        if constexpr (q19_ey(i) == 1) m.jy += d[i];
        if constexpr (q19_ey(i) == -1) m.jy -= d[i];
        if constexpr (q19_ez(i) == 1) m.jz += d[i];
        if constexpr (q19_ez(i) == -1) m.jz -= d[i];
    });
    static_for<0, 7>([&](auto I) { m.T += g[decltype(I)::value]; });
    return m;
}

// m_k = sum_i M_ki d_i for one moment k (zero coefficients dropped).
template <int K>
__device__ __forceinline__ float moment19(const float d[19])
{
    float acc = 0.f;
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int c = m19(K, i);
        if constexpr (c == 1) acc += d[i];
        else if constexpr (c == -1) acc -= d[i];
        else if constexpr (c != 0) acc = fmaf(static_cast<float>(c), d[i], acc);
    });
    return acc;
}

template <int K>
__device__ __forceinline__ float moment7(const float g[7])
{
    float acc = 0.f;
    static_for<0, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int c = m7(K, i);
        if constexpr (c == 1) acc += g[i];
        else if constexpr (c == -1) acc -= g[i];
        else if constexpr (c != 0) acc = fmaf(static_cast<float>(c), g[i], acc);
    });
    return acc;
}

// In-place collision of one cell: MRT relaxation of both lattices
// (Eqs. (19), (24), (29), (33)) and the buoyancy force (Eqs. (15)-(17)).
// d holds f - w, g the energy populations; on return both are post-collision.
__device__ __forceinline__ void collide_cell(const CollideParams &C, float d[19], float g[7])
{
    const Macro mc = macro_of(d, g);
    const float rho = 1.0f + mc.drho;
    const float jx = mc.jx, jy = mc.jy, jz = mc.jz;
    const float jxx = jx * jx, jyy = jy * jy, jzz = jz * jz;
    const float jj = jxx + jyy + jzz;

    // non-equilibrium part of each relaxed moment, scaled by s_k/|M_k|^2.
    // Equilibria of Eq. (24) with rho0 = 1, minus the rest moments.
    float a[19];
    a[1] = C.rs[1] * (moment19<1>(d) - (-11.0f * mc.drho + 19.0f * jj));
    a[2] = C.rs[2] * (moment19<2>(d) - (3.0f * mc.drho - 5.5f * jj));
    a[4] = C.rs[4] * (moment19<4>(d) + (2.0f / 3.0f) * jx);
    a[6] = C.rs[6] * (moment19<6>(d) + (2.0f / 3.0f) * jy);
    a[8] = C.rs[8] * (moment19<8>(d) + (2.0f / 3.0f) * jz);
    const float pxx = 2.0f * jxx - (jyy + jzz);
    const float pww = jyy - jzz;
    a[9] = C.rs[9] * (moment19<9>(d) - pxx);
    a[10] = C.rs[10] * (moment19<10>(d) + 0.5f * pxx);
    a[11] = C.rs[11] * (moment19<11>(d) - pww);
    a[12] = C.rs[12] * (moment19<12>(d) + 0.5f * pww);
    a[13] = C.rs[13] * (moment19<13>(d) - jx * jy);
    a[14] = C.rs[14] * (moment19<14>(d) - jy * jz);
    a[15] = C.rs[15] * (moment19<15>(d) - jx * jz);
    a[16] = C.rs[16] * moment19<16>(d);
    a[17] = C.rs[17] * moment19<17>(d);
    a[18] = C.rs[18] * moment19<18>(d);

    // buoyancy G = (0, 0, g beta (theta - theta_ref)) (Eq. (16), gravity -z)
    const float inv_rho = 1.0f / rho;
    const float vx = jx * inv_rho, vy = jy * inv_rho, vz = jz * inv_rho;
    const float vv = vx * vx + vy * vy + vz * vz;
    const float Gz3 = 3.0f * C.gbeta * (mc.T - C.theta_ref);  // G_z / c_s^2

    // back-transform of the collision increment plus the force
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        float dc = 0.f;
        static_for<1, 19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if constexpr (k != 3 && k != 5 && k != 7) {
                constexpr int c = m19(k, i);
                if constexpr (c == 1) dc += a[k];
                else if constexpr (c == -1) dc -= a[k];
                else if constexpr (c != 0) dc = fmaf(static_cast<float>(c), a[k], dc);
            }
        });
        constexpr float ex = q19_ex(i), ey = q19_ey(i), ez = q19_ez(i);
        const float ev = ex * vx + ey * vy + ez * vz;
        const float feq = rho * q19_w(i) * (1.0f + 3.0f * ev + 4.5f * ev * ev - 1.5f * vv);
        const float F = Gz3 * (ez - vz) * feq;  // Eq. (15)
        d[i] = d[i] - dc + F;
    });

    // energy: n - n_eq with n_eq = (T, V T, 3/4 T, 0, 0) (Eqs. (33),(34))
    float b[7];
    b[1] = C.rq[1] * (moment7<1>(g) - vx * mc.T);
    b[2] = C.rq[2] * (moment7<2>(g) - vy * mc.T);
    b[3] = C.rq[3] * (moment7<3>(g) - vz * mc.T);
    b[4] = C.rq[4] * (moment7<4>(g) - 0.75f * mc.T);
    b[5] = C.rq[5] * moment7<5>(g);
    b[6] = C.rq[6] * moment7<6>(g);
    static_for<0, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        float dc = 0.f;
        static_for<1, 7>([&](auto K) {
            constexpr int k = decltype(K)::value;
            constexpr int c = m7(k, i);
            if constexpr (c == 1) dc += b[k];
            else if constexpr (c == -1) dc -= b[k];
            else if constexpr (c != 0) dc = fmaf(static_cast<float>(c), b[k], dc);
        });
        g[i] -= dc;
    });
}

}  // namespace lbm
