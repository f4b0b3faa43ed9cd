// step.cu -- the fused double-MRT time step (arXiv:1511.04633, Eqs. (14),
// (19), (29)) of one cavity: for every cell, pull the 19 + 7 populations from
// the neighbours (wall rules inline), collide both lattices in moment space,
// add the buoyancy force and store the result in the other buffer (A-B
// scheme).  The per-cell arithmetic is in step_body.cuh.
//
// Layout: 26 planes [q][z][y][x], x fastest, planes `plane` elements apart.
// One thread per cell, x along threadIdx.x, so every load of a warp is one
// contiguous run (shifted by one element for the +-x links) and every store
// a full aligned run.  The neighbour and bounce-back offsets of all 26 planes
// come precomputed in the launch parameters.
#include "residual.cuh"
#include "step_body.cuh"

namespace lbm {

namespace {

// Minimum resident 256-thread blocks per SM requested from the register
// allocator: 4 caps the kernel at 64 registers, i.e. 1024 resident threads
// per SM.  Measured on GB300 at 128^3 it beats the unconstrained 80-register
// build (68.9 vs 73.1 us per step): more loads in flight outweigh the
// register pressure, and nothing spills.
#ifndef DMRT_STEP_MIN_BLOCKS
#define DMRT_STEP_MIN_BLOCKS 4
#endif

// SR = true: 16-bit stores round stochastically.  The step number that seeds
// the random bits lives in a word after the populations of each buffer
// (`counter_at` elements in): every step reads it from its source buffer and
// one thread writes it, plus one, to the destination, so a replayed graph
// still draws fresh bits each step and runs stay bitwise reproducible.
// RES: this step also takes a residual point of the state it pulls (the
// fields of the pulled populations against the snapshot, residual.cuh).
template <int WALL, typename T, bool SR, bool RES>
__global__ void __launch_bounds__(256, DMRT_STEP_MIN_BLOCKS)
    step_kernel(const T *__restrict__ src, T *__restrict__ dst, const StepGeometry S,
                const Geometry G, const CollideParams C, const ResidualArgs R)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    // Programmatic dependent launch: this grid may be scheduled while the
    // previous step still drains; wait for it to complete (and its writes to
    // be visible) before reading, and let the next step's blocks be scheduled
    // as soon as every block of this one has started.  Both are no-ops for a
    // plain launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    DF acc[4] = {};
    if (x < S.nx && y < S.ny) {
        const unsigned self = (static_cast<unsigned>(z) * S.ny + y) * S.nx + x;
        float d[19], g[7];
        float prev[4];
        if constexpr (RES) residual_cell_load(R, self, prev);
        if constexpr (WALL == 0) {
            pull_f<0, T>(src, G, x, y, z, d);
            pull_g<0, T>(src, G, x, y, z, g);
        } else {
            pull_offsets<WALL, T>(src, TableOffsets{S}, S.nx, S.ny, S.nz, S.inv_ny, self, x, y, z, d,
                                  g);
        }
        const Conserved<float> m0 = conserved<float>(d, g);
        // the fields a residual point compares, used after the stores
        const float th = m0.Tu, ux = m0.vx, uy = m0.vy, uz = m0.vz;
        collide_from<float, 0>(C, d, g, m0, InPlace<float>{d, g});
        unsigned base = 0;
        if constexpr (SR) {
            const size_t counter_at = static_cast<size_t>(kPlanes) * S.plane;
            const unsigned step = *reinterpret_cast<const unsigned *>(src + counter_at);
            if (self == 0) *reinterpret_cast<unsigned *>(dst + counter_at) = step + 1u;
            base = pcg_hash(self ^ pcg_hash(step));
        }
        store_cell<T, SR>(dst, self, S.plane, d, g, base);
        if constexpr (RES) residual_cell(R, self, prev, th, ux, uy, uz, acc);
    }
    if constexpr (RES) residual_block_store(acc, R.partials);
}

}  // namespace

void fill_step_geometry(const Geometry &G, StepGeometry &S)
{
    S.nx = G.nx;
    S.ny = G.ny;
    S.nz = G.nz;
    S.plane = static_cast<unsigned>(G.plane);
    S.inv_ny = G.inv_ny;
    const long long sy = G.nx, sz = static_cast<long long>(G.nx) * G.ny;
    for (int i = 0; i < 19; ++i) {
        const long long off = q19_ex(i) + q19_ey(i) * sy + q19_ez(i) * sz;
        S.nb[i] = static_cast<int>(i * G.plane - off);
        S.bb[i] = static_cast<int>(q19_opp(i) * G.plane);
    }
    for (int i = 0; i < 7; ++i) {
        const long long off = q7_ex(i) + q7_ey(i) * sy + q7_ez(i) * sz;
        S.nb[19 + i] = static_cast<int>((19 + i) * G.plane - off);
        S.bb[19 + i] = static_cast<int>((19 + q7_opp(i)) * G.plane);
    }
}

cudaError_t launch_step(int wall, int storage, bool stochastic, const void *src, void *dst,
                        const StepGeometry &S, const Geometry &G, const CollideParams &C,
                        BlockShape b, cudaStream_t s, bool pdl, const ResidualArgs *res)
{
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
        const T *a = static_cast<const T *>(src);
        T *d = static_cast<T *>(dst);
        auto go = [&](auto sr) {
            constexpr bool SRv = decltype(sr)::value;
            if (res) return cudaLaunchKernelEx(&cfg, step_kernel<WL, T, SRv, true>, a, d, S, G, C, R);
            return cudaLaunchKernelEx(&cfg, step_kernel<WL, T, SRv, false>, a, d, S, G, C, R);
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
