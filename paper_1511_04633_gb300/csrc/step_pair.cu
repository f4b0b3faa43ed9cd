// step_pair.cu -- the fused double-MRT time step (arXiv:1511.04633, Eqs. (14),
// (19), (29)) of one walled cavity with TWO cells per thread: the cells x0 and
// x0 + 1 (x0 even) of one row.  It does the work of step_kernel (step.cu) and
// stores bitwise the same values, with fewer instructions per cell:
//  - the collision runs on both cells at once in Blackwell's packed f32x2
//    arithmetic (collide<F2>, step_body.cuh), half the instructions of two
//    one-cell collisions;
//  - the 14 planes whose links have no x component (e_x = 0) arrive as one
//    aligned 2-element load per pair; the 12 with e_x = +-1 are shifted by one
//    cell and load each cell's value on its own;
//  - every plane is stored with one 2-element store, and a 16-bit pair is
//    rounded by one stochastic-rounding conversion: the hardware takes the
//    low half's random bits from bits 15..0 of its operand and the high
//    half's from bits 31..16, so the operand carries the same bits that the
//    one-cell kernel gives each cell (pcg_hash of the cell and the step, one
//    Weyl step per plane, of which the conversion uses the low 16 bits).
// The same pairing serves both phases of in-place streaming
// (step_inplace_pair_kernel, the counterpart of step_inplace.cu).  The
// kernels need an even row length nx (rows then start on even elements, and
// the planes are padded to 64 elements), which the launchers check.
#include "step_body.cuh"

namespace lbm {

namespace {

// Two-element loads and stores of the storage formats: lane x is the cell at
// the lower address.  A 16-bit pair is packed into one 32-bit word (lane x in
// the low half), rounded to nearest (pack) or stochastically (pack_sr: bits
// 15..0 of r round lane x, bits 31..16 lane y; FP16 uses bits 12..0 and
// 28..16 of them).
template <typename T>
struct Pair;

template <>
struct Pair<float> {
    static __device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ float ld1(const float *p) { return *p; }
    static __device__ __forceinline__ void st2(float *p, F2 v, unsigned) { *reinterpret_cast<float2 *>(p) = v.v; }
    static __device__ __forceinline__ void st_split(float *p0, float *p1, F2 v, unsigned)
    {
        *p0 = v.v.x;
        *p1 = v.v.y;
    }
};

template <typename T, typename Derived>
struct Pair16 {
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

template <>
struct Pair<__nv_bfloat16> : Pair16<__nv_bfloat16, Pair<__nv_bfloat16>> {
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p)
    {
        const unsigned w = *reinterpret_cast<const unsigned *>(p);
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
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

// half: stored times 2^10 like Store<__half>; the scale is exact both ways
template <>
struct Pair<__half> : Pair16<__half, Pair<__half>> {
    static __device__ __forceinline__ float2 ld2(const __half *p)
    {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p));
        return (F2(f) * F2(1.0f / Store<__half>::kScale)).v;
    }
    static __device__ __forceinline__ float ld1(const __half *p) { return Store<__half>::ld(p); }
    static __device__ __forceinline__ unsigned pack_rn(F2 v)
    {
        const F2 s = v * F2(Store<__half>::kScale);
        unsigned w;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(s.v.y), "f"(s.v.x));
        return w;
    }
    static __device__ __forceinline__ unsigned pack_sr(F2 v, unsigned r)
    {
        const F2 s = v * F2(Store<__half>::kScale);
        unsigned w;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(s.v.y), "f"(s.v.x), "r"(r));
        return w;
    }
};

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

// r01 of the pair whose first cell is `self`, at step number `step`.
__device__ __forceinline__ unsigned pair_bits(unsigned self, unsigned step)
{
    const unsigned hs = pcg_hash(step);
    return __byte_perm(pcg_hash(self ^ hs), pcg_hash((self + 1u) ^ hs), 0x5410);
}

// Plane offsets of a pair: from a StepGeometry table (two-buffer step and
// in-place phase 0; lanes differ where a link leaves through an x face), or
// the cells' own slots (in-place phase 1, kLocal: the same offset for both
// lanes in every plane).
struct PairTable {
    const StepGeometry &S;
    static constexpr bool kLocal = false;
    template <int Q>
    __device__ __forceinline__ unsigned nb() const { return static_cast<unsigned>(S.nb[Q]); }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const { return static_cast<unsigned>(S.bb[Q]); }
};
struct PairLocal {
    unsigned plane;
    static constexpr bool kLocal = true;
    template <int Q>
    __device__ __forceinline__ unsigned nb() const { return Q * plane; }
    template <int Q>
    __device__ __forceinline__ unsigned bb() const { return Q * plane; }
};

// Faces the pair touches: cell 0 can sit on x = 0, cell 1 on x = nx - 1.
struct PairFaces {
    bool xlo, xhi, ylo, yhi, zlo, zhi;
};

// Pull of a pair (the wall rules of Sec. 3.1 and 3.2, as pull_offsets does
// for one cell): plane q of each cell from Bp + nb<q> (+1 for cell 1), or the
// bounce-back source at Bp + bb<q> where the link leaves the box.
template <int WALL, typename T, typename Off>
__device__ __forceinline__ void pull_pair(const T *Bp, const Off &O, const PairFaces &P, float th_lin,
                                          F2 d[19], F2 g[7])
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
            d[i] = F2(Pair<T>::ld2(Bp + (oyz ? bb : nb)));
        } else {
            const bool o0 = oyz || (ex == 1 && P.xlo);
            const bool o1 = oyz || (ex == -1 && P.xhi);
            d[i] = F2(Pair<T>::ld1(Bp + (o0 ? bb : nb)), Pair<T>::ld1((Bp + (o1 ? bb : nb)) + 1));
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
                const float2 v = Pair<T>::ld2(Bp + nb);
                v0 = v.x;
                v1 = v.y;
            } else {
                v0 = Pair<T>::ld1(Bp + (o0 ? bb : nb));
                v1 = Pair<T>::ld1((Bp + (o1 ? bb : nb)) + 1);
            }
        } else {
            bool o = false;
            if constexpr (i == 3) o = P.ylo;
            else if constexpr (i == 4) o = P.yhi;
            else if constexpr (i == 5) o = P.zlo;
            else if constexpr (i == 6) o = P.zhi;
            const float2 v = Pair<T>::ld2(Bp + (o ? bb : nb));
            v0 = v.x;
            v1 = v.y;
            o0 = o1 = o;
        }
        if constexpr (i != 0 && dirichlet_axis<WALL>(axis)) {
            float tw;
            if constexpr (axis == 1) tw = (ey == 1) ? 0.5f : -0.5f;
            else tw = th_lin;
            v0 = o0 ? fmaf(0.25f, tw, -v0) : v0;  // anti-bounce-back, 2 w_T,i = 1/4
            v1 = o1 ? fmaf(0.25f, tw, -v1) : v1;
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

// Value of plane q (0..25) of a collided pair.
template <int Q>
__device__ __forceinline__ F2 plane_value(const F2 d[19], const F2 g[7])
{
    if constexpr (Q < 19) return d[Q];
    else return g[Q - 19];
}

// Registers: 128-thread blocks, DMRT_PAIR_MIN_BLOCKS resident per SM (4 caps
// the kernel at 128 registers: 512 threads, 1024 cells in flight per SM, as
// many as the one-cell kernel at 64 registers).
#ifndef DMRT_PAIR_MIN_BLOCKS
#define DMRT_PAIR_MIN_BLOCKS 4
#endif

// Thread -> pair: x0 = 2 (block x * block width + thread x) must be < nx.
struct PairCoords {
    int x0, y, z;
    unsigned self;
    PairFaces faces;
    float th_lin;
    bool valid;
};

__device__ __forceinline__ PairCoords pair_coords(const StepGeometry &S)
{
    PairCoords c;
    c.x0 = 2 * static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z;
    c.valid = c.x0 < S.nx && c.y < S.ny;
    c.self = (static_cast<unsigned>(c.z) * S.ny + c.y) * S.nx + c.x0;
    c.faces = {c.x0 == 0, c.x0 + 2 == S.nx, c.y == 0, c.y == S.ny - 1, c.z == 0, c.z == S.nz - 1};
    c.th_lin = theta_linear(c.y, S.inv_ny);
    return c;
}

template <int WALL, typename T, bool SR>
__global__ void __launch_bounds__(128, DMRT_PAIR_MIN_BLOCKS)
    step_pair_kernel(const T *__restrict__ src, T *__restrict__ dst, const StepGeometry S,
                     const CollideParams C)
{
    // programmatic dependent launch, as in the one-cell kernel
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const PairCoords c = pair_coords(S);
    if (!c.valid) return;
    F2 d[19], g[7];
    pull_pair<WALL, T>(src + c.self, PairTable{S}, c.faces, c.th_lin, d, g);
    collide(C, d, g);
    // every plane of the pair: one 2-element store at the cells' own slots
    unsigned r01 = 0;
    if constexpr (SR) {
        const size_t counter_at = static_cast<size_t>(kPlanes) * S.plane;
        const unsigned step = *reinterpret_cast<const unsigned *>(src + counter_at);
        if (c.self == 0) *reinterpret_cast<unsigned *>(dst + counter_at) = step + 1u;
        r01 = pair_bits(c.self, step);
    }
    T *Dp = dst + c.self;
    const unsigned plane = opaque(S.plane);
    static_for<0, 26>([&](auto I) {
        constexpr int q = decltype(I)::value;
        store2<T, SR>(Dp + q * plane, plane_value<q>(d, g), SR ? plane_bits<q>(r01) : 0u);
    });
}

// In-place streaming with two cells per thread: the two phases of
// step_inplace_kernel (step_inplace.cu), bitwise the same values.  Phase 1
// reads and writes the cells' own slots, so every plane moves as an aligned
// pair; phase 0 pulls like the two-buffer step and writes S*_q to x + e_q,
// an aligned pair for the planes with e_x = 0 and one element per cell for
// the others (or, where the link leaves the box, plane opp(q) at the cell).
template <int WALL, typename T, bool SR, int PHASE>
__global__ void __launch_bounds__(128, DMRT_PAIR_MIN_BLOCKS)
    step_inplace_pair_kernel(T *__restrict__ A, const InplaceGeometry SI, const CollideParams C)
{
    const StepGeometry &S = SI.load;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const PairCoords c = pair_coords(S);
    if (!c.valid) return;
    F2 d[19], g[7];
    if constexpr (PHASE == 0) pull_pair<WALL, T>(A + c.self, PairTable{S}, c.faces, c.th_lin, d, g);
    else pull_pair<WALL, T>(A + c.self, PairLocal{S.plane}, c.faces, c.th_lin, d, g);
    collide(C, d, g);
    unsigned r01 = 0;
    if constexpr (SR) {
        unsigned *ctr = reinterpret_cast<unsigned *>(A + static_cast<size_t>(kPlanes) * S.plane);
        const unsigned step = ctr[PHASE];
        if (c.self == 0) ctr[PHASE ^ 1] = step + 1u;
        r01 = pair_bits(c.self, step);
    }
    T *Dp = A + c.self;
    const PairFaces &P = c.faces;
    const unsigned plane = opaque(S.plane);
    static_for<0, 26>([&](auto I) {
        constexpr int q = decltype(I)::value;
        const F2 v = plane_value<q>(d, g);
        const unsigned r = SR ? plane_bits<q>(r01) : 0u;
        if constexpr (PHASE == 1) {
            store2<T, SR>(Dp + plane_opp<q>() * plane, v, r);
        } else {
            constexpr int ex = plane_ex<q>(), ey = plane_ey<q>(), ez = plane_ez<q>();
            bool lyz = false;  // the link leaves through a y or z face
            if constexpr (ey == 1) lyz = lyz || P.yhi;
            if constexpr (ey == -1) lyz = lyz || P.ylo;
            if constexpr (ez == 1) lyz = lyz || P.zhi;
            if constexpr (ez == -1) lyz = lyz || P.zlo;
            const unsigned sn = static_cast<unsigned>(SI.sn[q]), sb = static_cast<unsigned>(SI.sb[q]);
            if constexpr (ex == 0) {
                store2<T, SR>(Dp + (lyz ? sb : sn), v, r);
            } else {
                const bool l0 = lyz || (ex == -1 && P.xlo);
                const bool l1 = lyz || (ex == 1 && P.xhi);
                store_split<T, SR>(Dp + (l0 ? sb : sn), (Dp + (l1 ? sb : sn)) + 1, v, r);
            }
        }
    });
}

}  // namespace

bool step_pair_supported(int wall, const Geometry &G)
{
    return wall >= 1 && wall <= 3 && G.nx % 2 == 0 && G.plane % 2 == 0;
}

namespace {

// Launch shape of the paired kernels: one row of up to 128 cells per block
// row, 128 threads per block.
cudaLaunchConfig_t pair_config(const Geometry &G, cudaStream_t s, cudaLaunchAttribute *attr, bool pdl)
{
    const int pairs = G.nx / 2;
    const int bx = pairs >= 64 ? 64 : (pairs >= 32 ? 32 : 16);
    const int by = 128 / bx;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((pairs + bx - 1) / bx, (G.ny + by - 1) / by, G.nz);
    cfg.blockDim = dim3(bx, by, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cfg;
}

}  // namespace

cudaError_t launch_step_pair(int wall, int storage, bool stochastic, const void *src, void *dst,
                             const StepGeometry &S, const Geometry &G, const CollideParams &C,
                             cudaStream_t s, bool pdl)
{
    if (!step_pair_supported(wall, G)) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(G, s, attr, pdl);
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        if constexpr (WL == 0) {
            return cudaErrorInvalidValue;
        } else {
            const T *a = static_cast<const T *>(src);
            T *b = static_cast<T *>(dst);
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic) return cudaLaunchKernelEx(&cfg, step_pair_kernel<WL, T, true>, a, b, S, C);
            }
            return cudaLaunchKernelEx(&cfg, step_pair_kernel<WL, T, false>, a, b, S, C);
        }
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_step_inplace_pair(int wall, int storage, bool stochastic, void *buf, int phase,
                                     const InplaceGeometry &SI, const Geometry &G,
                                     const CollideParams &C, cudaStream_t s, bool pdl)
{
    if (!step_pair_supported(wall, G) || (phase != 0 && phase != 1)) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(G, s, attr, pdl);
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        if constexpr (WL == 0) {
            return cudaErrorInvalidValue;
        } else {
            T *A = static_cast<T *>(buf);
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic)
                    return phase == 0
                               ? cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, true, 0>, A, SI, C)
                               : cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, true, 1>, A, SI, C);
            }
            return phase == 0 ? cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, false, 0>, A, SI, C)
                              : cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, false, 1>, A, SI, C);
        }
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lbm
