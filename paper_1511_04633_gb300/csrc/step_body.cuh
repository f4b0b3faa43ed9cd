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
#include "vec2.cuh"

namespace lbm {

// The pulled populations' pair sums and differences and their conserved
// moments (Eqs. (20), (30)), in the order in which the collision forms them:
// rho = 1 + drho, j, T, and V = j / rho as j times the reciprocal of rho.
// The fields the library reports (fields, residual) are these values, so a
// residual point taken inside a step kernel and one taken from a pull of the
// stored state agree bitwise cell by cell.  With kShift > 0 the sums carry
// the storage scale S = 2^kShift; Tu, rho and V are unscaled and ir
// is 1/rho divided by S (see collide_from below).
template <typename V>
struct Conserved {
    V s1, a1, s3, a3, s5, a5, s7, a7, s8, a8, s11, a11, s12, a12, s15, a15, s16, a16;
    V SF, A, B, Cyz, SE, drho, X1, X2, Y1, Y2, Z1, Z2, Ex, Ey, Ez, jx, jy, jz;
    V tsx, tax, tsy, tay, tsz, taz, tsm, T, Tu, rho, ir, vx, vy, vz;
};

template <typename V, int kShift = 0>
__device__ __forceinline__ Conserved<V> conserved(const V d[19], const V g[7])
{
    constexpr bool kScaled = kShift != 0;
    constexpr float kS = static_cast<float>(1u << kShift), kU = 1.0f / kS;

    // ---- opposite-velocity pairs (i, opp(i)): sums s and differences a
    const V s1 = d[1] + d[2], a1 = d[1] - d[2];          // (+-1, 0, 0)
    const V s3 = d[3] + d[4], a3 = d[3] - d[4];          // (0, +-1, 0)
    const V s5 = d[5] + d[6], a5 = d[5] - d[6];          // (0, 0, +-1)
    const V s7 = d[7] + d[10], a7 = d[7] - d[10];        // +-(1, 1, 0)
    const V s8 = d[8] + d[9], a8 = d[8] - d[9];          // +-(-1, 1, 0)
    const V s11 = d[11] + d[14], a11 = d[11] - d[14];    // +-(1, 0, 1)
    const V s12 = d[12] + d[13], a12 = d[12] - d[13];    // +-(-1, 0, 1)
    const V s15 = d[15] + d[18], a15 = d[15] - d[18];    // +-(0, 1, 1)
    const V s16 = d[16] + d[17], a16 = d[16] - d[17];    // +-(0, -1, 1)

    // ---- conserved moments (Eqs. (20), (30))
    const V SF = (s1 + s3) + s5;                 // faces
    const V A = s7 + s8, B = s11 + s12, Cyz = s15 + s16;  // xy, xz, yz edges
    const V SE = (A + B) + Cyz;                  // edges
    const V drho = (d[0] + SF) + SE;
    const V X1 = a7 - a8, X2 = a11 - a12;
    const V Y1 = a7 + a8, Y2 = a15 - a16;
    const V Z1 = a11 + a12, Z2 = a15 + a16;
    const V Ex = X1 + X2, Ey = Y1 + Y2, Ez = Z1 + Z2;
    const V jx = a1 + Ex, jy = a3 + Ey, jz = a5 + Ez;

    const V tsx = g[1] + g[2], tax = g[1] - g[2];
    const V tsy = g[3] + g[4], tay = g[3] - g[4];
    const V tsz = g[5] + g[6], taz = g[5] - g[6];
    const V tsm = (tsx + tsy) + tsz;
    const V T = g[0] + tsm;

    // rho and T unscaled, 1/rho divided by S (the same values at kShift = 0)
    V Tu = T, rho, ir;
    if constexpr (kScaled) {
        Tu = T * V(kU);
        rho = fma(drho, V(kU), V(1.0f));
        ir = recip(rho) * V(kU);
    } else {
        rho = drho + V(1.0f);
        ir = recip(rho);
    }
    const V vx = jx * ir, vy = jy * ir, vz = jz * ir;
    return Conserved<V>{s1, a1, s3, a3, s5, a5, s7, a7, s8, a8, s11, a11, s12, a12, s15, a15, s16, a16,
                        SF, A, B, Cyz, SE, drho, X1, X2, Y1, Y2, Z1, Z2, Ex, Ey, Ez, jx, jy, jz,
                        tsx, tax, tsy, tay, tsz, taz, tsm, T, Tu, rho, ir, vx, vy, vz};
}

// Where collide_from puts each post-collision value: put_f<i>(v) for the 19
// flow populations, put_g<i>(v) for the 7 energy populations, each as soon as
// it is final (the energy populations first), so a sink that stores them
// lets their registers go at once.  InPlace writes them back over the pulled
// values.
template <typename V>
struct InPlace {
    V *d, *g;
    template <int I>
    __device__ __forceinline__ void put_f(V v) const { d[I] = v; }
    template <int I>
    __device__ __forceinline__ void put_g(V v) const { g[I] = v; }
};

// Collision of one cell (V = float) or of two cells at once (V = F2), in
// place: d holds f - w, g the energy populations (pulled); on return both
// hold the post-collision values of Eqs. (14), (29).  Both forms give the same
// bits given one rule that the code below keeps: no product is added or
// subtracted as a separate operation.  ptxas fuses a packed multiply into a
// following packed add or subtract (an FMA, one rounding fewer) even with
// explicit rounding modes, and the compiler may do the same to float code;
// so every such pair is written as fma(), and a product that is subtracted
// enters as the product of a negated factor.
//
// kShift > 0: d and g hold the populations times S = 2^kShift (the FP16
// storage scale, so the kernels load and store the stored numbers as they
// are), and the results are scaled alike.  The collision is linear in the
// populations except through rho, V and T, which are unscaled (rho, T) or
// divided by S through 1/rho (V), and through the products of two j
// components, which carry S^2 and lose one S through their constant factor
// or one multiply; the force terms take S in their constant factors.
// Multiplying by a power of two commutes with rounding, so every value is
// exactly S times its value at kShift = 0.
//
// C: a CollideParams, or any type with the same members (rs[k], ws[k],
// rq[k], qa[k], gbeta, theta_ref, aniso), e.g. one that supplies the rates
// that do not vary between cavities as constants.
template <typename V, int kShift, typename Sink, typename Params = CollideParams>
__device__ __forceinline__ void collide_from(const Params &C, const V d[19], const V g[7], const Conserved<V> &m0,
                                             Sink out)
{
    constexpr bool kScaled = kShift != 0;
    constexpr float kS = static_cast<float>(1u << kShift), kU = 1.0f / kS;
    const V s1 = m0.s1, a1 = m0.a1, s3 = m0.s3, a3 = m0.a3, s5 = m0.s5, a5 = m0.a5;
    const V s7 = m0.s7, a7 = m0.a7, s8 = m0.s8, a8 = m0.a8, s11 = m0.s11, a11 = m0.a11;
    const V s12 = m0.s12, a12 = m0.a12, s15 = m0.s15, a15 = m0.a15, s16 = m0.s16, a16 = m0.a16;
    const V SF = m0.SF, A = m0.A, B = m0.B, Cyz = m0.Cyz, SE = m0.SE, drho = m0.drho;
    const V X1 = m0.X1, X2 = m0.X2, Y1 = m0.Y1, Y2 = m0.Y2, Z1 = m0.Z1, Z2 = m0.Z2;
    const V Ex = m0.Ex, Ey = m0.Ey, Ez = m0.Ez, jx = m0.jx, jy = m0.jy, jz = m0.jz;
    const V tsx = m0.tsx, tax = m0.tax, tsy = m0.tsy, tay = m0.tay, tsz = m0.tsz, taz = m0.taz;
    const V tsm = m0.tsm, T = m0.T, Tu = m0.Tu, rho = m0.rho, ir = m0.ir, vx = m0.vx;
    const V vy = m0.vy, vz = m0.vz;
    const V njz = jz * V(-1.0f);
    const V jj = fma(jx, jx, fma(jy, jy, jz * jz));  // S^2 |j|^2
    const V pww = fma(jy, jy, njz * jz);             // S^2 (jy^2 - jz^2)
    // S times a product of two j components (identity at kShift = 0)
    auto unS = [&](V p) {
        if constexpr (kScaled) return p * V(kU);
        else return p;
    };

    // ---- energy: n - n^eq with n^eq = (T, V T, 3/4 T, 0, 0) (Eqs. (33),(34)).
    // The flux parts e = (ta - V T) relax with Q's flux block; with
    // T = g0 + tsm the even parts are t4 = q4 (21/4 g0 - 7/4 tsm),
    // t5 = q5 (3 tsx - tsm), t6 = q6 (tsy - tsz) (rates divided by the norms),
    // and the back-transform subtracts, per pair, an even part (2 t5 - t4 for
    // x, t6 - t4 - t5 for y, -(t4 + t5 + t6) for z) and +-the relaxed flux.
    const V nT = T * V(-1.0f);
    const V e1 = fma(vx, nT, tax), e2 = fma(vy, nT, tay), e3 = fma(vz, nT, taz);
    const V u4 = fma(V(5.25f), g[0], V(-1.75f) * tsm);
    const V u5 = fma(V(3.0f), tsx, tsm * V(-1.0f));
    const V u6 = tsy - tsz;
    const V t4 = V(C.rq[4]) * u4, nt4 = V(-C.rq[4]) * u4;
    out.template put_g<0>(fma(V(-6.0f), t4, g[0]));
    const V Etx = fma(V(2.0f * C.rq[5]), u5, nt4);     // 2 t5 - t4
    const V t45 = fma(V(C.rq[5]), u5, t4);             // t4 + t5
    const V nt45 = fma(V(-C.rq[5]), u5, nt4);          // -(t4 + t5)
    const V Ety = fma(V(C.rq[6]), u6, nt45);           // t6 - t4 - t5
    const V P = fma(V(C.rq[6]), u6, t45);              // t4 + t5 + t6
    if (C.aniso) {  // uniform: the full flux block of Q (Eq. (35))
        const V t1 = fma(V(C.qa[0]), e1, fma(V(C.qa[1]), e2, V(C.qa[2]) * e3));
        const V t2 = fma(V(C.qa[3]), e1, fma(V(C.qa[4]), e2, V(C.qa[5]) * e3));
        const V t3 = fma(V(C.qa[6]), e1, fma(V(C.qa[7]), e2, V(C.qa[8]) * e3));
        out.template put_g<1>((g[1] - Etx) - t1);
        out.template put_g<2>((g[2] - Etx) + t1);
        out.template put_g<3>((g[3] - Ety) - t2);
        out.template put_g<4>((g[4] - Ety) + t2);
        out.template put_g<5>((g[5] + P) - t3);
        out.template put_g<6>((g[6] + P) + t3);
    } else {
        out.template put_g<1>(fma(V(-C.rq[1]), e1, g[1] - Etx));
        out.template put_g<2>(fma(V(C.rq[1]), e1, g[2] - Etx));
        out.template put_g<3>(fma(V(-C.rq[2]), e2, g[3] - Ety));
        out.template put_g<4>(fma(V(C.rq[2]), e2, g[4] - Ety));
        out.template put_g<5>(fma(V(-C.rq[3]), e3, g[5] + P));
        out.template put_g<6>(fma(V(C.rq[3]), e3, g[6] + P));
    }

    // ---- moments m_k of the deviations (Eqs. (21), (22)): the moments of w
    // are the rest equilibrium moments and cancel against those of m^eq.
    //   m1 = -30 d0 - 11 SF + 8 SE     m2 = 12 d0 - 4 SF + SE
    //   m4 = -4 a1 + Ex (m6, m8 alike) m9 = 3 (s1 - Cyz) + SE - SF
    //   m10 = -6 s1 - 3 Cyz + 2 SF + SE
    //   m11 = (s3 - s5) + (A - B)      m12 = -2 (s3 - s5) + (A - B)
    //   m13 = s7 - s8, m14 = s15 - s16, m15 = s11 - s12
    //   m16 = X1 - X2, m17 = Y2 - Y1, m18 = Z1 - Z2
    // and their equilibria (Eq. (24), rho0 = 1), with j^2 = jj:
    //   m1eq = -11 drho + 19 jj   m2eq = 3 drho - 11/2 jj   m4eq = -2/3 jx
    //   m9eq = 3 jx^2 - jj        m10eq = -m9eq / 2
    //   m11eq = jy^2 - jz^2       m12eq = -m11eq / 2
    //   m13eq = jx jy, m14eq = jy jz, m15eq = jx jz, m16-18eq = 0
    const V d35 = s3 - s5, dAB = A - B;
    const V m1 = fma(V(-30.0f), d[0], fma(V(-11.0f), SF, V(8.0f) * SE));
    const V m2 = fma(V(12.0f), d[0], fma(V(-4.0f), SF, SE));
    const V m4 = fma(V(-4.0f), a1, Ex), m6 = fma(V(-4.0f), a3, Ey), m8 = fma(V(-4.0f), a5, Ez);
    const V m9 = fma(V(3.0f), s1 - Cyz, SE - SF);
    const V m10 = fma(V(-6.0f), s1, fma(V(-3.0f), Cyz, fma(V(2.0f), SF, SE)));
    const V m11 = d35 + dAB, m12 = fma(V(-2.0f), d35, dAB);
    const V m13 = s7 - s8, m14 = s15 - s16, m15 = s11 - s12;
    const V m16 = X1 - X2, m17 = Y2 - Y1, m18 = Z1 - Z2;
    const V meq9 = fma(V(3.0f) * jx, jx, jj * V(-1.0f));  // S^2 m9eq

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
    // order are the isotropic ones, which makes these sums exact).  Below,
    // h_k = F^_k / |M_k|^2 with |M_k|^2 = 2394, 252, 40, 40, 10, 40, 36, 72,
    // 12, 24, 4, 4, 4, 8, 8, 8 (k = 1, 2, 4, 6, 7, 8, 9, ..., 18), constants
    // folded in.
    const V gbt = V(C.gbeta) * (Tu - V(C.theta_ref));
    const V gr = gbt * rho;
    const V gv = gr * vz;
    const V vxy = fma(vx, vx, vy * vy);                  // V_x^2 + V_y^2
    const V vv = fma(vz, vz, vxy);                       // V^2
    const V dxy = fma(vx, vx, (vy * V(-1.0f)) * vy);     // V_x^2 - V_y^2
    const V dyz = fma(vy, vy, (vz * V(-1.0f)) * vz);     // V_y^2 - V_z^2
    const V gvx = gv * vx, gvy = gv * vy;
    const V h9 = gv * fma(V(-0.25f * kS), vx * vx,
                          fma(V((1.0f / 12.0f) * kS), vv, V((-1.0f / 18.0f) * kS)));
    const V h11 = gv * fma(V(-0.25f * kS), dyz, V((-1.0f / 6.0f) * kS));
    const V grz = gr * fma(V(-0.75f * kS), vz * vz, V(0.25f * kS));

    // ---- post-collision moments over their norms, c_k = m*_k / |M_k|^2 with
    // m*_k = m_k - s_k (m_k - m_k^eq) + F^_k (Eqs. (19), (24), (26)):
    // c_k = w_k m_k + r_k m_k^eq + h_k, w_k = (1 - s_k)/|M_k|^2, r_k = s_k/|M_k|^2.
    // The conserved moments keep m*_0 = drho, m*_3,5 = j_x,y, m*_7 = j_z + g.
    const V c1 = fma(m1, V(C.ws[1]), fma(V(C.rs[1]), fma(V(-11.0f), drho, V(19.0f * kU) * jj),
                                       gv * fma(V((-57.0f / 2394.0f) * kS), vv,
                                                V((38.0f / 2394.0f) * kS))));
    const V c2 = fma(m2, V(C.ws[2]), fma(V(C.rs[2]), fma(V(3.0f), drho, V(-5.5f * kU) * jj),
                                       gv * fma(V((16.5f / 252.0f) * kS), vv,
                                                V((-11.0f / 252.0f) * kS))));
    const V c4 = fma(m4, V(C.ws[4]), fma(V(C.rs[4]), jx * V(-2.0f / 3.0f), gvx * V(0.125f * kS)));
    const V c6 = fma(m6, V(C.ws[6]), fma(V(C.rs[6]), jy * V(-2.0f / 3.0f), gvy * V(0.125f * kS)));
    const V c8 = fma(m8, V(C.ws[8]), fma(V(C.rs[8]), jz * V(-2.0f / 3.0f),
                                       gr * fma(V(0.0625f * kS), vxy, V((-1.0f / 60.0f) * kS))));
    const V c9 = fma(m9, V(C.ws[9]), fma(V(C.rs[9]), unS(meq9), h9));
    const V c10 = fma(m10, V(C.ws[10]), fma(V(C.rs[10]), meq9 * V(-0.5f * kU), h9 * V(-0.25f)));
    const V c11 = fma(m11, V(C.ws[11]), fma(V(C.rs[11]), unS(pww), h11));
    const V c12 = fma(m12, V(C.ws[12]), fma(V(C.rs[12]), pww * V(-0.5f * kU), h11 * V(-0.25f)));
    const V c13 = fma(m13, V(C.ws[13]), fma(V(C.rs[13]), unS(jx * jy), (gvx * vy) * V(-0.75f * kS)));
    const V c14 = fma(m14, V(C.ws[14]), fma(V(C.rs[14]), unS(jy * jz), grz * vy));
    const V c15 = fma(m15, V(C.ws[15]), fma(V(C.rs[15]), unS(jx * jz), grz * vx));
    const V c16 = fma(m16, V(C.ws[16]), gvx * V(-0.375f * kS));
    const V c17 = fma(m17, V(C.ws[17]), gvy * V(0.375f * kS));
    const V c18 = fma(m18, V(C.ws[18]), (gr * V(0.1875f * kS)) * dxy);

    // ---- back-transform f* = M^T c (M^-1 = M^T diag(1/|M_k|^2)), one even (E)
    // and one odd (O) partial sum per pair: f*_i = E + O, f*_opp = E - O.
    // c0 = drho/19, c3 = jx/10, c5 = jy/10, c7 = (jz + g)/10 enter through fma.
    out.template put_f<0>(fma(V(-30.0f), c1, fma(V(12.0f), c2, drho * V(1.0f / 19.0f))));
    const V Fc = fma(V(-11.0f), c1, fma(V(-4.0f), c2, drho * V(1.0f / 19.0f)));  // every face
    const V Gc = fma(V(8.0f), c1, fma(drho, V(1.0f / 19.0f), c2));                // every edge
    const V Efx = fma(V(2.0f), c9, fma(V(-4.0f), c10, Fc));
    const V FP = fma(V(2.0f), c10, Fc - c9);
    const V Q = fma(V(-2.0f), c12, c11);
    const V Efy = FP + Q, Efz = FP - Q;
    V gbts = gbt;  // S g_beta (T - T_ref)
    if constexpr (kScaled) gbts = gbt * V(kS);
    const V jzg = fma(gbts, rho, jz);  // j_z + g
    const V Ofx = fma(V(-4.0f), c4, jx * V(0.1f));
    const V Ofy = fma(V(-4.0f), c6, jy * V(0.1f));
    const V Ofz = fma(V(-4.0f), c8, jzg * V(0.1f));
    out.template put_f<1>(Efx + Ofx);
    out.template put_f<2>(Efx - Ofx);
    out.template put_f<3>(Efy + Ofy);
    out.template put_f<4>(Efy - Ofy);
    out.template put_f<5>(Efz + Ofz);
    out.template put_f<6>(Efz - Ofz);

    const V H = c9 + c10, K = c11 + c12;
    const V GH = Gc + H;
    const V Exy = GH + K, Exz = GH - K, Eyz = fma(V(-2.0f), H, Gc);
    const V cx = fma(jx, V(0.1f), c4), cy = fma(jy, V(0.1f), c6), cz = fma(jzg, V(0.1f), c8);
    const V E7 = Exy + c13, O7 = (cx + cy) + (c16 - c17);        // (1,1,0)
    const V E8 = Exy - c13, O8 = (cy - cx) - (c16 + c17);        // (-1,1,0)
    const V E11 = Exz + c15, O11 = (cx + cz) + (c18 - c16);      // (1,0,1)
    const V E12 = Exz - c15, O12 = (cz - cx) + (c16 + c18);      // (-1,0,1)
    const V E15 = Eyz + c14, O15 = (cy + cz) + (c17 - c18);      // (0,1,1)
    const V E16 = Eyz - c14, O16 = (cz - cy) - (c17 + c18);      // (0,-1,1)
    out.template put_f<7>(E7 + O7);
    out.template put_f<10>(E7 - O7);
    out.template put_f<8>(E8 + O8);
    out.template put_f<9>(E8 - O8);
    out.template put_f<11>(E11 + O11);
    out.template put_f<14>(E11 - O11);
    out.template put_f<12>(E12 + O12);
    out.template put_f<13>(E12 - O12);
    out.template put_f<15>(E15 + O15);
    out.template put_f<18>(E15 - O15);
    out.template put_f<16>(E16 + O16);
    out.template put_f<17>(E16 - O16);

}

// Collision of the pulled populations d, g, the results written back over
// them (see collide_from).
template <typename V, int kShift = 0, typename Params = CollideParams>
__device__ __forceinline__ void collide(const Params &C, V d[19], V g[7])
{
    collide_from<V, kShift>(C, d, g, conserved<V, kShift>(d, g), InPlace<V>{d, g});
}

// One cell per thread: the float form of collide().
template <typename Params = CollideParams>
__device__ __forceinline__ void collide_cell(const Params &C, float d[19], float g[7])
{
    collide<float, 0>(C, d, g);
}

// Neighbour / bounce-back offsets of the 26 planes: from the launch-parameter
// tables of one cavity.
struct TableOffsets {
    const StepGeometry &S;
    static constexpr bool kLocal = false;
    template <int Q>
    __device__ __forceinline__ unsigned nb() const { return static_cast<unsigned>(S.nb[Q]); }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const { return static_cast<unsigned>(S.bb[Q]); }
};

// The same offsets computed from the plane stride and the row / slab sizes
// (used where many cavities share one launch).
struct ComputedOffsets {
    unsigned plane, nx, nxy;
    static constexpr bool kLocal = false;
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
    const float th_lin = theta_linear(y, inv_ny);
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
    static constexpr bool kLocal = true;  // every plane from the cell's own slot
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
    static constexpr bool kLocal = false;
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
