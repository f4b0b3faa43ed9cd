// step_inplace.cu -- the fused double-MRT time step (arXiv:1511.04633,
// Eqs. (14), (19), (29)) on ONE population buffer: in-place streaming halves
// the population memory of a cavity (26 values per cell instead of 52).
//
// Two kernels alternate (the AA access pattern of Bailey et al., "Accelerating
// lattice Boltzmann fluid flow simulations using graphics processors", ICPP
// 2009).  With S_i(x) the post-collision population of the previous step:
//  - phase 0 starts from the swapped layout (S_i(x) in plane opp(i) at x).
//    The cell pulls f_i(x) = S_i(x - e_i) from plane opp(i) at x - e_i, or,
//    across a wall, the bounce-back source S_opp(x) from plane i at x; it
//    collides and writes its S*_i(x) to plane i at x + e_i, or to plane
//    opp(i) at x when x + e_i lies outside the box (the streamed layout).
//  - phase 1 starts from the streamed layout, where every arriving
//    population already sits in the cell's own slot of plane i; it collides
//    and writes S*_i(x) to plane opp(i) at x, which is the swapped layout
//    again.
// In both phases each cell reads exactly the 26 slots it then writes, and no
// two cells share a slot, so the update is race-free in place.  The wall
// rules of Sec. 3 are applied where a population is read, as in the
// two-buffer kernel, and the stochastic-rounding bits are keyed by the
// producing cell and direction: the stored values are bitwise those of the
// two-buffer scheme, only their addresses differ.
#include "residual.cuh"
#include "step_body.cuh"

namespace lbm {

namespace {

// Minimum resident 256-thread blocks per SM of each FP32 phase (4 caps a
// kernel at 64 registers, 3 at 80; the kernels launch 128-thread blocks, so
// the bound below asks for twice as many of those).  The phase-0 kernel needs its store offsets
// beside the collision's values and spills ~50 bytes at 64 registers;
// measured on GB300 (128^3, FP32), 80 registers for both phases give
// 67.7 us per step against 75.2 us at 64.
#ifndef DMRT_INPLACE_MIN_BLOCKS0
#define DMRT_INPLACE_MIN_BLOCKS0 3
#endif
#ifndef DMRT_INPLACE_MIN_BLOCKS1
#define DMRT_INPLACE_MIN_BLOCKS1 3
#endif
// DMRT_INPLACE_BLOCK128 = N: compile both phases for the 128-thread blocks
// the cavities use, with N resident per SM (e.g. 7 gives 72 registers).
#ifndef DMRT_INPLACE_BLOCK128
#define DMRT_INPLACE_BLOCK128 0
#endif
#if DMRT_INPLACE_BLOCK128
#define DMRT_INPLACE_BOUNDS(PHASE, T) __launch_bounds__(128, DMRT_INPLACE_BLOCK128)
#else
// the 16-bit phases run at 72 registers (7 blocks of 128 threads), measured
// 3 % faster than at 80; the FP32 phases at 80 (measured 3 % faster than 72)
#define DMRT_INPLACE_BOUNDS(PHASE, T) \
    __launch_bounds__(128, std::is_same_v<T, float> ? 2 * (PHASE == 0 ? DMRT_INPLACE_MIN_BLOCKS0 : DMRT_INPLACE_MIN_BLOCKS1) : 7)
#endif

// Cell index of (x + dx, y + dy, z + dz) in a periodic box.
__device__ __forceinline__ unsigned wrapped_cell(const StepGeometry &S, int x, int y, int z)
{
    x = x < 0 ? S.nx - 1 : (x >= S.nx ? 0 : x);
    y = y < 0 ? S.ny - 1 : (y >= S.ny ? 0 : y);
    z = z < 0 ? S.nz - 1 : (z >= S.nz ? 0 : z);
    return (static_cast<unsigned>(z) * S.ny + y) * S.nx + x;
}

// Periodic boxes: the pull of either phase.
template <typename T, int PHASE>
__device__ __forceinline__ void load_periodic(const T *A, const StepGeometry &S, int x, int y, int z,
                                              unsigned self, float d[19], float g[7])
{
    static_for<0, 26>([&](auto I) {
        constexpr int q = decltype(I)::value;
        constexpr int ex = q < 19 ? q19_ex(q) : q7_ex(q - 19);
        constexpr int ey = q < 19 ? q19_ey(q) : q7_ey(q - 19);
        constexpr int ez = q < 19 ? q19_ez(q) : q7_ez(q - 19);
        constexpr int opp = q < 19 ? q19_opp(q) : 19 + q7_opp(q - 19);
        unsigned a;
        if constexpr (PHASE == 0) a = opp * S.plane + wrapped_cell(S, x - ex, y - ey, z - ez);
        else a = q * S.plane + self;
        const float v = Store<T>::ld(A + a);
        if constexpr (q < 19) d[q] = v;
        else g[q - 19] = v;
    });
}

// RES: this step also takes a residual point of the state it pulls.
template <int WALL, typename T, bool SR, int PHASE, bool RES>
__global__ void DMRT_INPLACE_BOUNDS(PHASE, T)
    step_inplace_kernel(T *__restrict__ A, const InplaceGeometry SI, const CollideParams C,
                        const ResidualArgs R)
{
    const StepGeometry &S = SI.load;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    // programmatic dependent launch, as in the two-buffer kernel
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    DF acc[4] = {};
    if (x < S.nx && y < S.ny) {
        const unsigned self = (static_cast<unsigned>(z) * S.ny + y) * S.nx + x;
        float d[19], g[7];
        float prev[4];
        if constexpr (RES) residual_cell_load(R, self, prev);
        if constexpr (WALL == 0) {
            load_periodic<T, PHASE>(A, S, x, y, z, self, d, g);
        } else if constexpr (PHASE == 0) {
            pull_offsets<WALL, T>(A, TableOffsets{S}, S.nx, S.ny, S.nz, S.inv_ny, self, x, y, z, d, g);
        } else {
            pull_offsets<WALL, T>(A, LocalOffsets{S.plane}, S.nx, S.ny, S.nz, S.inv_ny, self, x, y, z,
                                  d, g);
        }
        const Conserved<float> m0 = conserved<float>(d, g);
        // the fields a residual point compares, used after the stores
        const float th = m0.Tu, ux = m0.vx, uy = m0.vy, uz = m0.vz;
        collide_from<float, 0>(C, d, g, m0, InPlace<float>{d, g});
        unsigned base = 0;
        if constexpr (SR) {
            unsigned *ctr = reinterpret_cast<unsigned *>(A + static_cast<size_t>(kPlanes) * S.plane);
            const unsigned step = ctr[PHASE];
            if (self == 0) ctr[PHASE ^ 1] = step + 1u;
            base = pcg_hash(self ^ pcg_hash(step));
        }
        if constexpr (PHASE == 1) {
            store_cell_to<T, SR>(A, d, g, base, [&](auto I) -> unsigned {
                constexpr int q = decltype(I)::value;
                constexpr int opp = q < 19 ? q19_opp(q) : 19 + q7_opp(q - 19);
                return self + opp * S.plane;
            });
        } else if constexpr (WALL == 0) {
            store_cell_to<T, SR>(A, d, g, base, [&](auto I) -> unsigned {
                constexpr int q = decltype(I)::value;
                constexpr int ex = q < 19 ? q19_ex(q) : q7_ex(q - 19);
                constexpr int ey = q < 19 ? q19_ey(q) : q7_ey(q - 19);
                constexpr int ez = q < 19 ? q19_ez(q) : q7_ez(q - 19);
                return q * S.plane + wrapped_cell(S, x + ex, y + ey, z + ez);
            });
        } else {
            const unsigned edge = face_bits(x, y, z, S.nx, S.ny, S.nz);
            store_cell_to<T, SR>(A, d, g, base, [&](auto I) -> unsigned {
                constexpr int q = decltype(I)::value;
                constexpr unsigned faces = leaving_faces<q>();
                if constexpr (faces == 0) return self + static_cast<unsigned>(SI.sn[q]);
                else return self + static_cast<unsigned>((edge & faces) ? SI.sb[q] : SI.sn[q]);
            });
        }
        if constexpr (RES) residual_cell(R, self, prev, th, ux, uy, uz, acc);
    }
    if constexpr (RES) residual_block_store(acc, R.partials);
}

}  // namespace

void fill_inplace_geometry(const Geometry &G, InplaceGeometry &SI)
{
    StepGeometry &S = SI.load;
    S.nx = G.nx;
    S.ny = G.ny;
    S.nz = G.nz;
    S.plane = static_cast<unsigned>(G.plane);
    S.inv_ny = G.inv_ny;
    const long long sy = G.nx, sz = static_cast<long long>(G.nx) * G.ny;
    for (int q = 0; q < kPlanes; ++q) {
        const int ex = q < 19 ? q19_ex(q) : q7_ex(q - 19);
        const int ey = q < 19 ? q19_ey(q) : q7_ey(q - 19);
        const int ez = q < 19 ? q19_ez(q) : q7_ez(q - 19);
        const int opp = q < 19 ? q19_opp(q) : 19 + q7_opp(q - 19);
        const long long off = ex + ey * sy + ez * sz;
        // offsets are taken modulo 2^32 by the kernel (32-bit cell indices)
        S.nb[q] = static_cast<int>(static_cast<unsigned>(opp * G.plane - off));
        S.bb[q] = static_cast<int>(static_cast<unsigned>(q * G.plane));
        SI.sn[q] = static_cast<int>(static_cast<unsigned>(q * G.plane + off));
        SI.sb[q] = static_cast<int>(static_cast<unsigned>(opp * G.plane));
    }
}

cudaError_t launch_step_inplace(int wall, int storage, bool stochastic, void *buf, int phase,
                                const InplaceGeometry &SI, const Geometry &G,
                                const CollideParams &C, BlockShape b, cudaStream_t s, bool pdl,
                                const ResidualArgs *res)
{
    if (phase != 0 && phase != 1) return cudaErrorInvalidValue;
    // the residual's block reduction works on whole warps
    if (res && (b.bx * b.by) % 32 != 0) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((G.nx + b.bx - 1) / b.bx, (G.ny + b.by - 1) / b.by, G.nz);
    cfg.blockDim = dim3(b.bx, b.by, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const ResidualArgs R = res ? *res : ResidualArgs{};
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        T *A = static_cast<T *>(buf);
        auto go = [&](auto sr) {
            constexpr bool SRv = decltype(sr)::value;
            if (res)
                return phase == 0 ? cudaLaunchKernelEx(&cfg, step_inplace_kernel<WL, T, SRv, 0, true>, A, SI, C, R)
                                  : cudaLaunchKernelEx(&cfg, step_inplace_kernel<WL, T, SRv, 1, true>, A, SI, C, R);
            return phase == 0 ? cudaLaunchKernelEx(&cfg, step_inplace_kernel<WL, T, SRv, 0, false>, A, SI, C, R)
                              : cudaLaunchKernelEx(&cfg, step_inplace_kernel<WL, T, SRv, 1, false>, A, SI, C, R);
        };
        if constexpr (!std::is_same_v<T, float>) {
            if (stochastic) return go(std::true_type{});
        }
        return go(std::false_type{});
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lbm
