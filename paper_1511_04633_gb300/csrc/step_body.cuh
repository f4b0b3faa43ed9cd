// step_body.cuh -- the per-cell body of the fused double-MRT step
// (arXiv:1511.04633, Eqs. (14), (19), (29)), shared by the single-cavity
// kernel (step.cu) and the ensemble kernel (ensemble.cu).
//
// The arithmetic is arranged to need few instructions:
//  - the D3Q19 transforms work on sums and differences of opposite-velocity
//    pairs: even moments need only the sums, odd moments only the
//    differences, and the back-transform of a pair shares one even and one
//    odd partial sum;
//  - the buoyancy force of Eq. (15) is added in moment space: M F has a short
//    closed form for each moment (derived below), which joins the relaxation
//    increment before the single back-transform;
//  - neighbour and bounce-back offsets of all 26 planes are 32-bit cell-index
//    offsets, from launch-parameter tables or computed from the strides.
#pragma once

#include "internal.h"

namespace lbm {

// Collision of one cell in place: d holds f - w, g the energy populations
// (pulled); on return both hold the post-collision values of Eqs. (14), (29).
__device__ __forceinline__ void collide_pairs(const CollideParams &C, float d[19], float g[7])
{
    // ---- opposite-velocity pairs (i, opp(i)): sums s and differences a
    const float s1 = d[1] + d[2], a1 = d[1] - d[2];          // (+-1, 0, 0)
    const float s3 = d[3] + d[4], a3 = d[3] - d[4];          // (0, +-1, 0)
    const float s5 = d[5] + d[6], a5 = d[5] - d[6];          // (0, 0, +-1)
    const float s7 = d[7] + d[10], a7 = d[7] - d[10];        // +-(1, 1, 0)
    const float s8 = d[8] + d[9], a8 = d[8] - d[9];          // +-(-1, 1, 0)
    const float s11 = d[11] + d[14], a11 = d[11] - d[14];    // +-(1, 0, 1)
    const float s12 = d[12] + d[13], a12 = d[12] - d[13];    // +-(-1, 0, 1)
    const float s15 = d[15] + d[18], a15 = d[15] - d[18];    // +-(0, 1, 1)
    const float s16 = d[16] + d[17], a16 = d[16] - d[17];    // +-(0, -1, 1)

    // ---- conserved moments (Eqs. (20), (30))
    const float SF = s1 + s3 + s5;                 // faces
    const float A = s7 + s8, B = s11 + s12, Cyz = s15 + s16;  // xy, xz, yz edges
    const float SE = A + B + Cyz;                  // edges
    const float drho = d[0] + SF + SE;
    const float X1 = a7 - a8, X2 = a11 - a12;
    const float Y1 = a7 + a8, Y2 = a15 - a16;
    const float Z1 = a11 + a12, Z2 = a15 + a16;
    const float Ex = X1 + X2, Ey = Y1 + Y2, Ez = Z1 + Z2;
    const float jx = a1 + Ex, jy = a3 + Ey, jz = a5 + Ez;

    const float tsx = g[1] + g[2], tax = g[1] - g[2];
    const float tsy = g[3] + g[4], tay = g[3] - g[4];
    const float tsz = g[5] + g[6], taz = g[5] - g[6];
    const float tsm = tsx + tsy + tsz;
    const float T = g[0] + tsm;

    const float rho = 1.0f + drho;
    const float ir = 1.0f / rho;
    const float vx = jx * ir, vy = jy * ir, vz = jz * ir;
    const float jxx = jx * jx, jyy = jy * jy, jzz = jz * jz;
    const float jj = jxx + jyy + jzz;

    // ---- non-equilibrium parts m_k - m_k^eq (Eq. (24), rho0 = 1; the rest
    // moments of w cancel between m and m^eq)
    const float n1 = (-30.0f * d[0] - 11.0f * SF + 8.0f * SE) - (-11.0f * drho + 19.0f * jj);
    const float n2 = (12.0f * d[0] - 4.0f * SF + SE) - (3.0f * drho - 5.5f * jj);
    const float n4 = (-4.0f * a1 + Ex) + (2.0f / 3.0f) * jx;
    const float n6 = (-4.0f * a3 + Ey) + (2.0f / 3.0f) * jy;
    const float n8 = (-4.0f * a5 + Ez) + (2.0f / 3.0f) * jz;
    const float s35 = s3 + s5, AB = A + B;
    const float pxx = 2.0f * jxx - (jyy + jzz);
    const float n9 = (2.0f * s1 - s35 + AB - 2.0f * Cyz) - pxx;
    const float n10 = (-4.0f * s1 + 2.0f * s35 + AB - 2.0f * Cyz) + 0.5f * pxx;
    const float d35 = s3 - s5, dAB = A - B;
    const float pww = jyy - jzz;
    const float n11 = (d35 + dAB) - pww;
    const float n12 = (-2.0f * d35 + dAB) + 0.5f * pww;
    const float n13 = (s7 - s8) - jx * jy;
    const float n14 = (s15 - s16) - jy * jz;
    const float n15 = (s11 - s12) - jx * jz;
    const float n16 = X1 - X2, n17 = Y2 - Y1, n18 = Z1 - Z2;

    // ---- buoyancy in moment space.  With G = (0, 0, G_z) (Eq. (16)) and
    // F_i = G_z (e_iz - V_z) f_eq,i / c_s^2 (Eqs. (15), (17)), the moments
    // F^_k = sum_i M_ki F_i are, with g = G_z rho and gv = g V_z:
    //   F^_1 = gv (38 - 57 V^2)          F^_2 = gv (33/2 V^2 - 11)
    //   F^_4 = 5 gv V_x                  F^_6 = 5 gv V_y
    //   F^_7 = g                         F^_8 = g (5/2 (V_x^2 + V_y^2) - 2/3)
    //   F^_9 = -gv (6 V_x^2 - 3 V_y^2 - 3 V_z^2 + 2)      F^_10 = -F^_9 / 2
    //   F^_11 = -gv (3 V_y^2 - 3 V_z^2 + 2)               F^_12 = -F^_11 / 2
    //   F^_13 = -3 gv V_x V_y   F^_14 = g V_y (1 - 3 V_z^2)   F^_15 = g V_x (1 - 3 V_z^2)
    //   F^_16 = -3 gv V_x       F^_17 = 3 gv V_y              F^_18 = 3/2 g (V_x^2 - V_y^2)
    // and F^_0 = F^_3 = F^_5 = 0 (the D3Q19 moments of f_eq up to fourth
    // order are the isotropic ones, which makes these sums exact).
    const float gr = C.gbeta * (T - C.theta_ref) * rho;
    const float gv = gr * vz;
    const float vxx = vx * vx, vyy = vy * vy, vzz = vz * vz;
    const float vv = vxx + vyy + vzz;
    const float F1 = gv * (38.0f - 57.0f * vv);
    const float F2 = gv * (16.5f * vv - 11.0f);
    const float F4 = 5.0f * gv * vx;
    const float F6 = 5.0f * gv * vy;
    const float F7 = gr;
    const float F8 = gr * (2.5f * (vxx + vyy) - 2.0f / 3.0f);
    const float F9 = -gv * (6.0f * vxx - 3.0f * (vyy + vzz) + 2.0f);
    const float F11 = -gv * (3.0f * (vyy - vzz) + 2.0f);
    const float F13 = -3.0f * gv * vx * vy;
    const float t1z = 1.0f - 3.0f * vzz;
    const float F14 = gr * vy * t1z;
    const float F15 = gr * vx * t1z;
    const float F16 = -3.0f * gv * vx;
    const float F17 = 3.0f * gv * vy;
    const float F18 = 1.5f * gr * (vxx - vyy);

    // ---- b_k = (s_k (m_k - m_k^eq) - F^_k) / |M_k|^2  (rates come divided)
    const float b1 = fmaf(C.rs[1], n1, F1 * (-1.0f / 2394.0f));
    const float b2 = fmaf(C.rs[2], n2, F2 * (-1.0f / 252.0f));
    const float b4 = fmaf(C.rs[4], n4, F4 * (-1.0f / 40.0f));
    const float b6 = fmaf(C.rs[6], n6, F6 * (-1.0f / 40.0f));
    const float b7 = F7 * (-1.0f / 10.0f);
    const float b8 = fmaf(C.rs[8], n8, F8 * (-1.0f / 40.0f));
    const float b9 = fmaf(C.rs[9], n9, F9 * (-1.0f / 36.0f));
    const float b10 = fmaf(C.rs[10], n10, F9 * (1.0f / 144.0f));
    const float b11 = fmaf(C.rs[11], n11, F11 * (-1.0f / 12.0f));
    const float b12 = fmaf(C.rs[12], n12, F11 * (1.0f / 48.0f));
    const float b13 = fmaf(C.rs[13], n13, F13 * -0.25f);
    const float b14 = fmaf(C.rs[14], n14, F14 * -0.25f);
    const float b15 = fmaf(C.rs[15], n15, F15 * -0.25f);
    const float b16 = fmaf(C.rs[16], n16, F16 * -0.125f);
    const float b17 = fmaf(C.rs[17], n17, F17 * -0.125f);
    const float b18 = fmaf(C.rs[18], n18, F18 * -0.125f);

    // ---- back-transform f* = f - M^T b, one even (E) and one odd (O) partial
    // sum per pair: f*_i = f_i - (E + O), f*_opp = f_opp - (E - O)
    d[0] -= -30.0f * b1 + 12.0f * b2;
    const float F0 = -11.0f * b1 - 4.0f * b2;  // every face
    const float G0 = 8.0f * b1 + b2;           // every edge
    const float Pf = 2.0f * b10 - b9, Qf = b11 - 2.0f * b12;
    const float Efx = F0 + 2.0f * b9 - 4.0f * b10;
    const float Efy = F0 + Pf + Qf, Efz = F0 + Pf - Qf;
    const float Ofx = -4.0f * b4, Ofy = -4.0f * b6, Ofz = b7 - 4.0f * b8;
    d[1] -= Efx + Ofx;
    d[2] -= Efx - Ofx;
    d[3] -= Efy + Ofy;
    d[4] -= Efy - Ofy;
    d[5] -= Efz + Ofz;
    d[6] -= Efz - Ofz;

    const float H = b9 + b10, K = b11 + b12;
    const float Exy = G0 + H + K, Exz = G0 + H - K, Eyz = G0 - 2.0f * H;
    const float b78 = b7 + b8;
    const float E7 = Exy + b13, O7 = (b4 + b6) + (b16 - b17);        // (1,1,0)
    const float E8 = Exy - b13, O8 = (b6 - b4) - (b16 + b17);        // (-1,1,0)
    const float E11 = Exz + b15, O11 = (b78 + b4) + (b18 - b16);     // (1,0,1)
    const float E12 = Exz - b15, O12 = (b78 - b4) + (b16 + b18);     // (-1,0,1)
    const float E15 = Eyz + b14, O15 = (b78 + b6) + (b17 - b18);     // (0,1,1)
    const float E16 = Eyz - b14, O16 = (b78 - b6) - (b17 + b18);     // (0,-1,1)
    d[7] -= E7 + O7;
    d[10] -= E7 - O7;
    d[8] -= E8 + O8;
    d[9] -= E8 - O8;
    d[11] -= E11 + O11;
    d[14] -= E11 - O11;
    d[12] -= E12 + O12;
    d[13] -= E12 - O12;
    d[15] -= E15 + O15;
    d[18] -= E15 - O15;
    d[16] -= E16 + O16;
    d[17] -= E16 - O16;

    // ---- energy: n - n^eq with n^eq = (T, V T, 3/4 T, 0, 0) (Eqs. (33),(34))
    const float e1 = tax - vx * T, e2 = tay - vy * T, e3 = taz - vz * T;
    float c1, c2, c3;
    if (C.aniso) {  // uniform: the full flux block of Q (Eq. (35))
        c1 = fmaf(C.qa[0], e1, fmaf(C.qa[1], e2, C.qa[2] * e3));
        c2 = fmaf(C.qa[3], e1, fmaf(C.qa[4], e2, C.qa[5] * e3));
        c3 = fmaf(C.qa[6], e1, fmaf(C.qa[7], e2, C.qa[8] * e3));
    } else {
        c1 = C.rq[1] * e1;
        c2 = C.rq[2] * e2;
        c3 = C.rq[3] * e3;
    }
    const float c4 = C.rq[4] * (6.0f * g[0] - tsm - 0.75f * T);
    const float c5 = C.rq[5] * (2.0f * tsx - (tsy + tsz));
    const float c6 = C.rq[6] * (tsy - tsz);
    g[0] -= 6.0f * c4;
    const float Etx = 2.0f * c5 - c4;
    const float Ety = c6 - c4 - c5, Etz = -c4 - c5 - c6;
    g[1] -= Etx + c1;
    g[2] -= Etx - c1;
    g[3] -= Ety + c2;
    g[4] -= Ety - c2;
    g[5] -= Etz + c3;
    g[6] -= Etz - c3;
}

// Neighbour / bounce-back offsets of the 26 planes: from the launch-parameter
// tables of one cavity.
struct TableOffsets {
    const StepGeometry &S;
    template <int Q>
    __device__ __forceinline__ unsigned nb() const { return static_cast<unsigned>(S.nb[Q]); }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const { return static_cast<unsigned>(S.bb[Q]); }
};

// The same offsets computed from the plane stride and the row / slab sizes
// (used where many cavities share one launch).
struct ComputedOffsets {
    unsigned plane, nx, nxy;
    template <int Q>
    __device__ __forceinline__ unsigned nb() const
    {
        // the neighbour offset e.(1, nx, nx*ny) is signed; the sum is taken
        // modulo 2^32 and is non-negative, since plane exceeds any offset
        if constexpr (Q < 19) {
            constexpr int ex = q19_ex(Q), ey = q19_ey(Q), ez = q19_ez(Q);
            const int off = ex + ey * static_cast<int>(nx) + ez * static_cast<int>(nxy);
            return Q * plane - static_cast<unsigned>(off);
        } else {
            constexpr int ex = q7_ex(Q - 19), ey = q7_ey(Q - 19), ez = q7_ez(Q - 19);
            const int off = ex + ey * static_cast<int>(nx) + ez * static_cast<int>(nxy);
            return Q * plane - static_cast<unsigned>(off);
        }
    }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const
    {
        if constexpr (Q < 19) return q19_opp(Q) * plane;
        else return (19 + q7_opp(Q - 19)) * plane;
    }
};

// WALL value of pull_offsets for a wall type known only at run time (Types
// 1-3); the x / z thermal walls are then Dirichlet where dir_x / dir_z say.
constexpr int kRuntimeWall = -1;

// Pull of walled boxes (Types 1-3): plane q of the neighbour at self + nb<q>,
// or the bounce-back source at self + bb<q> when the link leaves the box
// (Sec. 3.1 and 3.2 wall rules).
template <int WALL, typename T, typename Off>
__device__ __forceinline__ void pull_offsets(const T *__restrict__ src, const Off &O, int nx, int ny,
                                             int nz, float inv_ny, unsigned self, int x, int y,
                                             int z, float d[19], float g[7], bool dir_x = false,
                                             bool dir_z = false)
{
    const bool xlo = (x == 0), xhi = (x == nx - 1);
    const bool ylo = (y == 0), yhi = (y == ny - 1);
    const bool zlo = (z == 0), zhi = (z == nz - 1);
    d[0] = Store<T>::ld(src + self);
    static_for<1, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q19_ex(i), ey = q19_ey(i), ez = q19_ez(i);
        bool out = false;
        if constexpr (ex == 1) out = out || xlo;
        if constexpr (ex == -1) out = out || xhi;
        if constexpr (ey == 1) out = out || ylo;
        if constexpr (ey == -1) out = out || yhi;
        if constexpr (ez == 1) out = out || zlo;
        if constexpr (ez == -1) out = out || zhi;
        d[i] = Store<T>::ld(src + (self + (out ? O.template bb<i>() : O.template nb<i>())));
    });
    g[0] = Store<T>::ld(src + (self + O.template nb<19>()));
    const float th_lin = 0.5f - (static_cast<float>(y) + 0.5f) * inv_ny;
    static_for<1, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q7_ex(i), ey = q7_ey(i);
        constexpr int axis = ex != 0 ? 0 : (ey != 0 ? 1 : 2);
        bool out;
        if constexpr (i == 1) out = xlo;
        else if constexpr (i == 2) out = xhi;
        else if constexpr (i == 3) out = ylo;
        else if constexpr (i == 4) out = yhi;
        else if constexpr (i == 5) out = zlo;
        else out = zhi;
        float v = Store<T>::ld(src + (self + (out ? O.template bb<19 + i>() : O.template nb<19 + i>())));
        if constexpr (WALL == kRuntimeWall) {
            const bool dir = axis == 1 || (axis == 0 ? dir_x : dir_z);
            float tw;
            if constexpr (axis == 1) tw = (ey == 1) ? 0.5f : -0.5f;
            else tw = th_lin;
            v = (out && dir) ? fmaf(0.25f, tw, -v) : v;  // anti-bounce-back, 2 w_T,i = 1/4
        } else if constexpr (dirichlet_axis<WALL>(axis)) {
            float tw;
            if constexpr (axis == 1) tw = (ey == 1) ? 0.5f : -0.5f;
            else tw = th_lin;
            v = out ? fmaf(0.25f, tw, -v) : v;  // anti-bounce-back, 2 w_T,i = 1/4
        }
        g[i] = v;
    });
}

// ---------------------------------------------------------------- in-place streaming

// Direction q of the 26 planes (0..18 D3Q19, 19..25 D3Q7): velocity and the
// plane of the opposite direction.
template <int Q>
__device__ constexpr int plane_ex() { return Q < 19 ? q19_ex(Q) : q7_ex(Q - 19); }
template <int Q>
__device__ constexpr int plane_ey() { return Q < 19 ? q19_ey(Q) : q7_ey(Q - 19); }
template <int Q>
__device__ constexpr int plane_ez() { return Q < 19 ? q19_ez(Q) : q7_ez(Q - 19); }
template <int Q>
__device__ constexpr int plane_opp() { return Q < 19 ? q19_opp(Q) : 19 + q7_opp(Q - 19); }

// The box faces a cell touches, one bit each: x = 0, x = nx-1, y = 0,
// y = ny-1, z = 0, z = nz-1.
__device__ __forceinline__ unsigned face_bits(int x, int y, int z, int nx, int ny, int nz)
{
    return (x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u) | (y == 0 ? 4u : 0u) |
           (y == ny - 1 ? 8u : 0u) | (z == 0 ? 16u : 0u) | (z == nz - 1 ? 32u : 0u);
}

// Faces (face_bits) that x + e_Q crosses when x touches them.
template <int Q>
__device__ constexpr unsigned leaving_faces()
{
    constexpr int ex = plane_ex<Q>(), ey = plane_ey<Q>(), ez = plane_ez<Q>();
    return (ex == 1 ? 2u : (ex == -1 ? 1u : 0u)) | (ey == 1 ? 8u : (ey == -1 ? 4u : 0u)) |
           (ez == 1 ? 32u : (ez == -1 ? 16u : 0u));
}

// Phase-1 loads of the in-place scheme: population q of a cell arrives in its
// own slot of plane q.
struct LocalOffsets {
    unsigned plane;
    template <int Q>
    __device__ __forceinline__ unsigned nb() const { return Q * plane; }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const { return Q * plane; }
};

// Phase-0 offsets of the in-place scheme computed from the strides: S_q(x -
// e_q) sits in plane opp(q) at x - e_q (nb), the bounce-back source S_opp(x)
// in plane q at x (bb); the value leaving x along q goes to plane q at x +
// e_q (sn), or to plane opp(q) at x when that link leaves the box (sb).
struct SwappedOffsets {
    unsigned plane, nx, nxy;
    template <int Q>
    __device__ __forceinline__ int off() const
    {
        return plane_ex<Q>() + plane_ey<Q>() * static_cast<int>(nx) +
               plane_ez<Q>() * static_cast<int>(nxy);
    }
    template <int Q>
    __device__ __forceinline__ unsigned nb() const
    {
        return plane_opp<Q>() * plane - static_cast<unsigned>(off<Q>());
    }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const { return Q * plane; }
    template <int Q>
    __device__ __forceinline__ unsigned sn() const { return Q * plane + static_cast<unsigned>(off<Q>()); }
    template <int Q>
    __device__ __forceinline__ unsigned sb() const { return plane_opp<Q>() * plane; }
};

// Store the 26 post-collision values of one cell at A + addr(q), rounding
// stochastically with bits keyed by the direction q as store_cell does.
template <typename T, bool SR, typename Addr>
__device__ __forceinline__ void store_cell_to(T *A, const float d[19], const float g[7],
                                              unsigned base, Addr &&addr)
{
    static_for<0, 26>([&](auto I) {
        constexpr int q = decltype(I)::value;
        float v;
        if constexpr (q < 19) v = d[q];
        else v = g[q - 19];
        T *p = A + addr(I);
        if constexpr (SR) StoreSR<T>::st(p, v, base + q * kWeyl);
        else Store<T>::st(p, v);
    });
}

// Store the 26 post-collision values of one cell; SR selects stochastic
// rounding with the random word `base` (one Weyl step per plane).
template <typename T, bool SR>
__device__ __forceinline__ void store_cell(T *__restrict__ dst, unsigned self, unsigned plane,
                                           const float d[19], const float g[7], unsigned base)
{
    if constexpr (SR) {
        static_for<0, 19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            StoreSR<T>::st(dst + (self + i * plane), d[i], base + i * kWeyl);
        });
        static_for<0, 7>([&](auto I) {
            constexpr int i = decltype(I)::value;
            StoreSR<T>::st(dst + (self + (19 + i) * plane), g[i], base + (19 + i) * kWeyl);
        });
    } else {
        static_for<0, 19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            Store<T>::st(dst + (self + i * plane), d[i]);
        });
        static_for<0, 7>([&](auto I) {
            constexpr int i = decltype(I)::value;
            Store<T>::st(dst + (self + (19 + i) * plane), g[i]);
        });
    }
}

}  // namespace lbm
