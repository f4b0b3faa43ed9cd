// pair_body.cuh -- the parts of the two-cells-per-thread kernels shared by
// the single-cavity kernels (step_pair.cu) and the ensemble kernels
// (ensemble.cu): two-element loads and stores of the storage formats, the
// stochastic-rounding bits of a pair, and the pull of a pair with the wall
// rules of Sec. 3 (arXiv:1511.04633).  A pair is the cells x0 and x0 + 1
// (x0 even) of one row; lane x of an F2 is cell x0.
#pragma once

#include "step_body.cuh"

namespace lbm {

// Two-element loads and stores of the storage formats: lane x is the cell at
// the lower address.  A 16-bit pair is packed into one 32-bit word (lane x in
// the low half), rounded to nearest (pack) or stochastically (pack_sr: bits
// 15..0 of r round lane x, bits 31..16 lane y; FP16 uses bits 12..0 and
// 28..16 of them).  Loads and stores move the stored numbers as they are:
// 2^kShift times the populations (FP16: the 2^10 storage scale), the units
// in which the paired kernels collide (collide<F2, kShift>).
template <typename T>
struct Pair;

template <>
struct Pair<float> {
    static constexpr int kShift = 0;
    static __device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ float ld1(const float *p) { return *p; }
    static __device__ __forceinline__ float2 gld2(const float *p) { return ld2(p); }
    static __device__ __forceinline__ float gld1(const float *p) { return ld1(p); }
    static __device__ __forceinline__ void st2(float *p, F2 v, unsigned) { *reinterpret_cast<float2 *>(p) = v.v; }
    static __device__ __forceinline__ void st_split(float *p0, float *p1, F2 v, unsigned)
    {
        *p0 = v.v.x;
        *p1 = v.v.y;
    }
};

template <typename T, typename Derived>
struct Pair16 {
    // global loads of a pair / one value with the L2 prefetch hint (below)
    static __device__ __forceinline__ unsigned gword(const T *p)
    {
        unsigned w;
        asm volatile("ld.global.L2::256B.b32 %0, [%1];" : "=r"(w) : "l"(p));
        return w;
    }
    static __device__ __forceinline__ unsigned short ghalf(const T *p)
    {
        unsigned short h;
        asm volatile("ld.global.L2::256B.b16 %0, [%1];" : "=h"(h) : "l"(p));
        return h;
    }
    template <bool SR>
    static __device__ __forceinline__ unsigned pack(F2 v, unsigned r)
    {
        if constexpr (SR) return Derived::pack_sr(v, r);
        else return Derived::pack_rn(v);
    }
    template <bool SR>
    static __device__ __forceinline__ void st2(T *p, F2 v, unsigned r)
    {
        *reinterpret_cast<unsigned *>(p) = pack<SR>(v, r);
    }
    template <bool SR>
    static __device__ __forceinline__ void st_split(T *p0, T *p1, F2 v, unsigned r)
    {
        const unsigned w = pack<SR>(v, r);
        *reinterpret_cast<unsigned short *>(p0) = static_cast<unsigned short>(w);
        *reinterpret_cast<unsigned short *>(p1) = static_cast<unsigned short>(w >> 16);
    }
};

// The pull's 16-bit loads from global memory (gld2 / gld1; ld2 / ld1 also
// read shared memory, in the TMA-staged kernel) ask L2 for the 256-byte block
// around each access (ld.global.L2::256B): the next warps' and rows' bytes
// are then on their way
// without registers held for them.  Measured on GB300 at 256^3 (Type 3): BF16
// 297.0 -> 293.8-295.3 us per step, FP16 306.7 -> 302.8 us; FP32 loads
// gained nothing and stay plain.  The asm declares no memory effect; no
// store of a step can move above these loads all the same, since every
// stored value depends on the moments of all 26 loaded ones (which matters
// for the in-place kernels, which write the slots they read).
template <>
struct Pair<__nv_bfloat16> : Pair16<__nv_bfloat16, Pair<__nv_bfloat16>> {
    static constexpr int kShift = 0;
    static __device__ __forceinline__ float2 unpack(unsigned w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p)
    {
        return unpack(*reinterpret_cast<const unsigned *>(p));
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float2 gld2(const __nv_bfloat16 *p) { return unpack(Pair16::gword(p)); }
    static __device__ __forceinline__ float gld1(const __nv_bfloat16 *p)
    {
        return __uint_as_float(static_cast<unsigned>(Pair16::ghalf(p)) << 16);
    }
    static __device__ __forceinline__ unsigned pack_rn(F2 v)
    {
        unsigned w;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(v.v.y), "f"(v.v.x));
        return w;
    }
    static __device__ __forceinline__ unsigned pack_sr(F2 v, unsigned r)
    {
        unsigned w;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        return w;
    }
};

// half: the stored numbers are 2^10 times the populations (Store<__half>);
// the paired kernels keep that scale through the collision, so no load or
// store multiplies by it.
template <>
struct Pair<__half> : Pair16<__half, Pair<__half>> {
    static constexpr int kShift = 10;
    static_assert(Store<__half>::kScale == static_cast<float>(1 << kShift), "FP16 storage scale");
    static __device__ __forceinline__ float2 ld2(const __half *p)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ float ld1(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ float2 gld2(const __half *p)
    {
        const unsigned w = Pair16::gword(p);
        __half2 h;
        memcpy(&h, &w, sizeof h);
        return __half22float2(h);
    }
    static __device__ __forceinline__ float gld1(const __half *p) { return __half2float(__ushort_as_half(Pair16::ghalf(p))); }
    static __device__ __forceinline__ unsigned pack_rn(F2 v)
    {
        unsigned w;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(v.v.y), "f"(v.v.x));
        return w;
    }
    static __device__ __forceinline__ unsigned pack_sr(F2 v, unsigned r)
    {
        unsigned w;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        return w;
    }
};

// Collision of a pair in the units of the stored numbers of format T.
template <typename T>
__device__ __forceinline__ void collide_stored(const CollideParams &C, F2 d[19], F2 g[7])
{
    collide<F2, Pair<T>::kShift>(C, d, g);
}

// Coefficient of T_w in the anti-bounce-back rule g = 2 w_T T_w - g* (2 w_T =
// 1/4, Sec. 3.2), in the units of the stored numbers of format T.
template <typename T>
__device__ __forceinline__ constexpr float wall_coef()
{
    return 0.25f * static_cast<float>(1 << Pair<T>::kShift);
}

// Store helpers that hide the float / 16-bit difference in the kernels.
template <typename T, bool SR>
__device__ __forceinline__ void store2(T *p, F2 v, unsigned r)
{
    if constexpr (std::is_same_v<T, float>) Pair<float>::st2(p, v, r);
    else Pair<T>::template st2<SR>(p, v, r);
}
template <typename T, bool SR>
__device__ __forceinline__ void store_split(T *p0, T *p1, F2 v, unsigned r)
{
    if constexpr (std::is_same_v<T, float>) Pair<float>::st_split(p0, p1, v, r);
    else Pair<T>::template st_split<SR>(p0, p1, v, r);
}

// Random word of plane q for both cells of a pair: r01 holds the low 16 bits
// of the two cells' base words (cell 0 in bits 15..0); the one-cell kernels
// round plane q of a cell with base + q * kWeyl, whose low 16 bits are the
// low 16 bits of the base plus those of q * kWeyl, modulo 2^16.
template <int Q>
__device__ __forceinline__ unsigned plane_bits(unsigned r01)
{
    constexpr unsigned kw = (static_cast<unsigned>(Q) * kWeyl) & 0xffffu;
    unsigned r;
    asm("add.u16x2 %0, %1, %2;" : "=r"(r) : "r"(r01), "r"(kw | (kw << 16)));
    return r;
}

// r01 of the pair whose first cell is `self`, with salt = pcg_hash(step)
// (the one-cell kernels' word of a cell is pcg_hash(cell ^ salt)).
__device__ __forceinline__ unsigned pair_bits_salted(unsigned self, unsigned salt)
{
    return __byte_perm(pcg_hash(self ^ salt), pcg_hash((self + 1u) ^ salt), 0x5410);
}

// r01 of the pair whose first cell is `self`, at step number `step`.
__device__ __forceinline__ unsigned pair_bits(unsigned self, unsigned step)
{
    return pair_bits_salted(self, pcg_hash(step));
}

// Faces the pair touches: cell 0 can sit on x = 0, cell 1 on x = nx - 1.
struct PairFaces {
    bool xlo, xhi, ylo, yhi, zlo, zhi;
};

// Pull of a pair (the wall rules of Sec. 3.1 and 3.2, as pull_offsets does
// for one cell): plane q of each cell from Bp + nb<q> (+1 for cell 1), or the
// bounce-back source at Bp + bb<q> where the link leaves the box.
// Offsets come from TableOffsets / ComputedOffsets / SwappedOffsets (lanes
// differ where a link leaves through an x face) or LocalOffsets (kLocal: the
// cells' own slots, the same offset for both lanes in every plane).  WALL =
// kRuntimeWall takes the x / z thermal rule from dir_x / dir_z.
template <int WALL, typename T, typename Off>
__device__ __forceinline__ void pull_pair(const T *Bp, const Off &O, const PairFaces &P, float th_lin,
                                          F2 d[19], F2 g[7], bool dir_x = false, bool dir_z = false)
{
    static_for<0, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q19_ex(i), ey = q19_ey(i), ez = q19_ez(i);
        bool oyz = false;
        if constexpr (ey == 1) oyz = oyz || P.ylo;
        if constexpr (ey == -1) oyz = oyz || P.yhi;
        if constexpr (ez == 1) oyz = oyz || P.zlo;
        if constexpr (ez == -1) oyz = oyz || P.zhi;
        const unsigned nb = O.template nb<i>(), bb = O.template bb<i>();
        if constexpr (ex == 0 || Off::kLocal) {
            d[i] = F2(Pair<T>::gld2(Bp + (oyz ? bb : nb)));
        } else {
            const bool o0 = oyz || (ex == 1 && P.xlo);
            const bool o1 = oyz || (ex == -1 && P.xhi);
            d[i] = F2(Pair<T>::gld1(Bp + (o0 ? bb : nb)), Pair<T>::gld1((Bp + (o1 ? bb : nb)) + 1));
        }
    });
    static_for<0, 7>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = q7_ex(i), ey = q7_ey(i);
        constexpr int axis = ex != 0 ? 0 : (ey != 0 ? 1 : 2);
        const unsigned nb = O.template nb<19 + i>(), bb = O.template bb<19 + i>();
        float v0, v1;
        bool o0, o1;
        if constexpr (axis == 0 && i != 0) {
            o0 = (i == 1) && P.xlo;
            o1 = (i == 2) && P.xhi;
            if constexpr (Off::kLocal) {
                const float2 v = Pair<T>::gld2(Bp + nb);
                v0 = v.x;
                v1 = v.y;
            } else {
                v0 = Pair<T>::gld1(Bp + (o0 ? bb : nb));
                v1 = Pair<T>::gld1((Bp + (o1 ? bb : nb)) + 1);
            }
        } else {
            bool o = false;
            if constexpr (i == 3) o = P.ylo;
            else if constexpr (i == 4) o = P.yhi;
            else if constexpr (i == 5) o = P.zlo;
            else if constexpr (i == 6) o = P.zhi;
            const float2 v = Pair<T>::gld2(Bp + (o ? bb : nb));
            v0 = v.x;
            v1 = v.y;
            o0 = o1 = o;
        }
        if constexpr (i != 0 && WALL == kRuntimeWall) {
            const bool dir = axis == 1 || (axis == 0 ? dir_x : dir_z);
            float tw;
            if constexpr (axis == 1) tw = (ey == 1) ? 0.5f : -0.5f;
            else tw = th_lin;
            v0 = (o0 && dir) ? fmaf(wall_coef<T>(), tw, -v0) : v0;  // anti-bounce-back
            v1 = (o1 && dir) ? fmaf(wall_coef<T>(), tw, -v1) : v1;
        } else if constexpr (i != 0 && dirichlet_axis<WALL>(axis)) {
            float tw;
            if constexpr (axis == 1) tw = (ey == 1) ? 0.5f : -0.5f;
            else tw = th_lin;
            v0 = o0 ? fmaf(wall_coef<T>(), tw, -v0) : v0;  // anti-bounce-back
            v1 = o1 ? fmaf(wall_coef<T>(), tw, -v1) : v1;
        }
        g[i] = F2(v0, v1);
    });
}

// The plane stride, hidden from the compiler: store addresses computed from
// it are recomputed after the collision instead of being kept live from the
// loads (which address the same planes), which would cost ~26 registers.
__device__ __forceinline__ unsigned opaque(unsigned v)
{
    unsigned r;
    asm volatile("mov.b32 %0, %1;" : "=r"(r) : "r"(v));
    return r;
}

// A collision sink (collide_from) that hands each post-collision value of
// plane q (0..18 flow, 19..25 energy) to store(std::integral_constant<int,
// q>, value) as soon as it is final.
template <typename F>
struct PlaneSink {
    F store;
    template <int I>
    __device__ __forceinline__ void put_f(F2 v) const { store(std::integral_constant<int, I>{}, v); }
    template <int I>
    __device__ __forceinline__ void put_g(F2 v) const { store(std::integral_constant<int, 19 + I>{}, v); }
};

template <typename F>
__device__ __forceinline__ PlaneSink<F> plane_sink(F f)
{
    return PlaneSink<F>{f};
}

// Value of plane q (0..25) of a collided pair.
template <int Q>
__device__ __forceinline__ F2 plane_value(const F2 d[19], const F2 g[7])
{
    if constexpr (Q < 19) return d[Q];
    else return g[Q - 19];
}

}  // namespace lbm
