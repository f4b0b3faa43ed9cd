// step_pair.cu -- the fused double-MRT time step (arXiv:1511.04633, Eqs. (14),
// (19), (29)) of one walled cavity with TWO cells per thread: the cells x0 and
// x0 + 1 (x0 even) of one row.  It does the work of step_kernel (step.cu) and
// stores bitwise the same values, with fewer instructions per cell:
//  - the collision runs on both cells at once in Blackwell's packed f32x2
//    arithmetic (collide<F2>, step_body.cuh), half the instructions of two
//    one-cell collisions; FP16 pairs collide in the stored units, 2^10 times
//    the populations (collide<F2, 10>), so no load or store multiplies;
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
#include <cuda.h>
#include <cudaTypedefs.h>

#include "pair_body.cuh"
#include "residual.cuh"
#include "umma.cuh"

namespace lbm {

namespace {

// Block shape: 128 threads, 5 blocks resident per SM (the register cap is
// 65536 / (128 x 5) = 102, rounded down to 96; the kernels need 108
// registers unconstrained).  Measured on GB300 at 256^3 Type 3, what counts
// is warps in flight, more than a small spill: BF16 takes 296 us (two
// buffers) and 306 us (in place) with 5 blocks (96 registers, 20 warps, 24-56
// bytes spilled), 328 us with 18 warps at 108 registers and 331 us with 24
// warps at 80.  FP16, which collides in the stored units, takes 333 us with 5
// blocks against 341 us with 4 (Type 1: 328 against 352 us; host-timed runs
// of 200 steps).  DMRT_PAIR_MIN_BLOCKS overrides the count for experiments.
constexpr int kPairThreads = 128;
#ifdef DMRT_PAIR_MIN_BLOCKS
constexpr int kPairBlocks = DMRT_PAIR_MIN_BLOCKS;
#else
constexpr int kPairBlocks = 5;
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

// The fields of a pulled pair that a residual point compares (unscaled):
// theta, u_x, u_y, u_z, kept from the moments until the stores are done.
// The snapshot is loaded with the populations and compared after the
// stores: measured on GB300 (128^3 FP32), a residual step then costs 27 us
// more than a plain one, against 44 us with the snapshot only prefetched to
// L2 early and 177 us with its loads after the stores.
struct PairFields {
    F2 th, ux, uy, uz;
};

// Blocks per SM of the kernels that take a residual point: 4 (128
// registers), so that the snapshot and the kept fields do not spill; the
// other steps keep kPairBlocks.
constexpr int kPairBlocksRes = 4;

// RES: this step also takes a residual point of the state it pulls (the
// fields of the pulled populations against the snapshot, residual.cuh).
template <int WALL, typename T, bool SR, bool RES>
__global__ void __launch_bounds__(kPairThreads, RES ? kPairBlocksRes : kPairBlocks)
    step_pair_kernel(const T *__restrict__ src, T *__restrict__ dst, const StepGeometry S,
                     const CollideParams C, const ResidualArgs R)
{
    // programmatic dependent launch, as in the one-cell kernel
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const PairCoords c = pair_coords(S);
    DF acc[4] = {};
    if (c.valid) {
        F2 d[19], g[7];
        float2 prev[4];
        if constexpr (RES) residual_pair_load(R, c.self, prev);
        pull_pair<WALL, T>(src + c.self, TableOffsets{S}, c.faces, c.th_lin, d, g);
        const Conserved<F2> m0 = conserved<F2, Pair<T>::kShift>(d, g);
        const PairFields fl{m0.Tu, m0.vx, m0.vy, m0.vz};
        unsigned r01 = 0;
        if constexpr (SR) {
            const size_t counter_at = static_cast<size_t>(kPlanes) * S.plane;
            const unsigned step = *reinterpret_cast<const unsigned *>(src + counter_at);
            if (c.self == 0) *reinterpret_cast<unsigned *>(dst + counter_at) = step + 1u;
            r01 = pair_bits(c.self, step);
        }
        // every plane of the pair: one 2-element store at the cells' own
        // slots, as soon as the collision has its value
        T *Dp = dst + c.self;
        const unsigned plane = opaque(S.plane);
        collide_from<F2, Pair<T>::kShift>(C, d, g, m0, plane_sink([&](auto I, F2 v) {
            constexpr int q = decltype(I)::value;
            store2<T, SR>(Dp + q * plane, v, SR ? plane_bits<q>(r01) : 0u);
        }));
        if constexpr (RES) residual_pair(R, c.self, prev, fl.th.v, fl.ux.v, fl.uy.v, fl.uz.v, acc);
    }
    if constexpr (RES) residual_block_store(acc, R.partials);
}

// In-place streaming with two cells per thread: the two phases of
// step_inplace_kernel (step_inplace.cu), bitwise the same values.  Phase 1
// reads and writes the cells' own slots, so every plane moves as an aligned
// pair; phase 0 pulls like the two-buffer step and writes S*_q to x + e_q,
// an aligned pair for the planes with e_x = 0 and one element per cell for
// the others (or, where the link leaves the box, plane opp(q) at the cell).
template <int WALL, typename T, bool SR, int PHASE, bool RES>
__global__ void __launch_bounds__(kPairThreads, RES ? kPairBlocksRes : kPairBlocks)
    step_inplace_pair_kernel(T *__restrict__ A, const InplaceGeometry SI, const CollideParams C,
                             const ResidualArgs R)
{
    const StepGeometry &S = SI.load;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const PairCoords c = pair_coords(S);
    DF acc[4] = {};
    if (c.valid) {
        F2 d[19], g[7];
        float2 prev[4];
        if constexpr (RES) residual_pair_load(R, c.self, prev);
        if constexpr (PHASE == 0) pull_pair<WALL, T>(A + c.self, TableOffsets{S}, c.faces, c.th_lin, d, g);
        else pull_pair<WALL, T>(A + c.self, LocalOffsets{S.plane}, c.faces, c.th_lin, d, g);
        const Conserved<F2> m0 = conserved<F2, Pair<T>::kShift>(d, g);
        const PairFields fl{m0.Tu, m0.vx, m0.vy, m0.vz};
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
        collide_from<F2, Pair<T>::kShift>(C, d, g, m0, plane_sink([&](auto I, F2 v) {
            constexpr int q = decltype(I)::value;
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
        }));
        if constexpr (RES) residual_pair(R, c.self, prev, fl.th.v, fl.ux.v, fl.uy.v, fl.uz.v, acc);
    }
    if constexpr (RES) residual_block_store(acc, R.partials);
}


// ---------------------------------------------------------------- TMA-staged pairs
//
// The paired kernel above holds its loaded values in registers, and at 124
// registers only 16 warps per SM fit: too few bytes in flight to keep HBM
// busy.  step_pair_tma_kernel moves the loads into the asynchronous copy
// engine: a block of 64 x 8 threads owns 8 rows of 128 cells and marches
// along z.  For each z, one thread issues 26 TMA copies (one 144 x 8 box per
// plane: the eight source rows y - e_y at slab z - e_z, from 8 elements left
// of the block's first cell to 8 right of its last) into a ring of three
// shared-memory stages (60 KB each), two slabs ahead, completing on one
// mbarrier per stage.  Boxes of 2.3 KB keep the number of TMA operations per
// cell low; with 2-row boxes of 576 B the kernel ran 25 % slower than with
// direct loads.
// Threads then read their values from shared memory, shifted by -e_x.  Boxes
// that fall outside the box's rows or slabs are filled with zeros by the TMA
// unit; those links leave the box, and their bounce-back sources (the
// cell's own slot of the opposite plane) are needed instead.  For the x faces,
// which every row meets, blocks at x = 0 and x = nx - 1 stage them too: one
// 8 x 2 box of each opposite plane at the face, with the same mbarrier.  The
// rarer y and z faces take direct loads issued before the wait.  Every wait is
// bounded: one that runs out sets *err, the block stops, waits (bounded) for
// its copies in flight and returns.

constexpr int kTmaPairs = 64;                   // pairs per block row (128 cells)
constexpr int kTmaRows = 8;                     // rows per block (and per box)
constexpr int kTmaBoxW = 2 * kTmaPairs + 16;    // box width in elements (16-byte multiple)
constexpr int kTmaPlaneBytes = kTmaBoxW * kTmaRows * 2;  // one plane's box: 2304 B, a multiple of 128
constexpr int kTmaEdgeW = 8;                    // edge box width in elements (16 bytes)
constexpr int kTmaEdgeLinks = 6;                // links with e_x = +1 (or -1): 5 D3Q19, 1 D3Q7
constexpr int kTmaEdgeSlot = 128;               // one edge box (8 x 8 x 2 B)
constexpr int kTmaEdgeTx = kTmaEdgeLinks * kTmaEdgeW * kTmaRows * 2;  // bytes of one side's boxes
constexpr int kTmaStageBytes = kPlanes * kTmaPlaneBytes + 2 * kTmaEdgeLinks * kTmaEdgeSlot;
constexpr int kTmaStages = 3;
constexpr uint32_t kTmaStageTx = kPlanes * kTmaBoxW * kTmaRows * 2;  // bytes a stage receives
constexpr int kTmaSmemBytes = kTmaStages * kTmaStageBytes + kTmaStages * 8 + 128;  // + alignment slack
constexpr uint32_t kTmaWaitPolls = 1u << 20;    // with a 64 ns sleep each: well over 60 ms

__host__ __device__ constexpr int plane_ex_of(int p) { return p < 19 ? q19_ex(p) : q7_ex(p - 19); }

// Slot of link q among the links with its sign of e_x, in plane order (0..5).
template <int Q>
__device__ constexpr int edge_slot()
{
    int k = 0;
    for (int p = 0; p < Q; ++p)
        if (plane_ex_of(p) == plane_ex_of(Q)) ++k;
    return k;
}

// One TMA tile copy of a 4-D box at (x, y, z, plane) into shared memory.
__device__ __forceinline__ void tma_box(const CUtensorMap *map, unsigned char *dst, uint32_t bar, int x, int y,
                                        int z, int q)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(umma::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(q), "r"(bar)
        : "memory");
}

// Issue the boxes of slab z into one stage (one thread): the 26 plane boxes
// and, for a block at the x = 0 (left) or x = nx - 1 (right) face, the edge
// boxes of the opposite planes of the links leaving through it.
__device__ __forceinline__ void tma_issue_slab(const CUtensorMap *map, const CUtensorMap *edge,
                                               unsigned char *stage, uint64_t *bar, int xs, int y0, int z,
                                               bool left, bool right, int nx)
{
    const uint32_t b = umma::smem_u32(bar);
    const uint32_t tx = kTmaStageTx + (left ? kTmaEdgeTx : 0) + (right ? kTmaEdgeTx : 0);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(tx) : "memory");
    static_for<0, kPlanes>([&](auto I) {
        constexpr int q = decltype(I)::value;
        tma_box(map, stage + q * kTmaPlaneBytes, b, xs - 8, y0 - plane_ey<q>(), z - plane_ez<q>(), q);
    });
    unsigned char *eb = stage + kPlanes * kTmaPlaneBytes;
    static_for<0, kPlanes>([&](auto I) {
        constexpr int q = decltype(I)::value;
        if constexpr (plane_ex<q>() == 1) {
            if (left) tma_box(edge, eb + edge_slot<q>() * kTmaEdgeSlot, b, 0, y0, z, plane_opp<q>());
        } else if constexpr (plane_ex<q>() == -1) {
            if (right)
                tma_box(edge, eb + (kTmaEdgeLinks + edge_slot<q>()) * kTmaEdgeSlot, b, nx - kTmaEdgeW, y0, z,
                        plane_opp<q>());
        }
    });
}

static_assert(kTmaPlaneBytes % 128 == 0 && kTmaEdgeW * kTmaRows * 2 <= kTmaEdgeSlot, "stage layout");

// 512 threads (64 pairs x 8 rows) at up to 128 registers: one block per SM.
template <int WALL, typename T, bool SR>
__global__ void __launch_bounds__(kTmaPairs * kTmaRows, 1)
    step_pair_tma_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap edge,
                         const T *__restrict__ src, T *__restrict__ dst, const StepGeometry S,
                         const CollideParams C, int zper, unsigned *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // stage boxes start on 128-byte boundaries whatever the base alignment
    unsigned char *smem = smem_raw + ((128u - (umma::smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kTmaStages * kTmaStageBytes);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int xs = blockIdx.x * (2 * kTmaPairs);
    const int x0 = xs + 2 * tx;
    const int y0 = blockIdx.y * kTmaRows, y = y0 + ty;
    const int zb = blockIdx.z * zper;
    const int ze = min(zb + zper, S.nz);
    const bool valid = x0 < S.nx && y < S.ny;
    const bool leader = tx == 0 && ty == 0;
    const bool left = xs == 0, right = xs + 2 * kTmaPairs >= S.nx;  // the block meets x = 0 / x = nx - 1
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    if (leader) {
        for (int k = 0; k < kTmaStages; ++k) umma::mbar_init(&bar[k], 1);
        for (int k = 0; k < kTmaStages - 1 && zb + k < ze; ++k)
            tma_issue_slab(&map, &edge, smem + k * kTmaStageBytes, &bar[k], xs, y0, zb + k, left, right, S.nx);
    }
    __syncthreads();

    unsigned step = 0;
    if constexpr (SR) step = *reinterpret_cast<const unsigned *>(src + static_cast<size_t>(kPlanes) * S.plane);
    const bool xlo = x0 == 0, xhi = x0 + 2 == S.nx, ylo = y == 0, yhi = y == S.ny - 1;
    const float th_lin = theta_linear(y, S.inv_ny);
    const int k0 = 2 * tx + 8;  // cell 0's element in a staged row
    bool ok = true;
    int j = 0;
    for (int z = zb; z < ze; ++z, ++j) {
        const int s = j % kTmaStages;
        const bool zlo = z == 0, zhi = z == S.nz - 1;
        const unsigned self = (static_cast<unsigned>(z) * S.ny + y) * S.nx + x0;
        const T *Bp = src + self;
        // ---- bounce-back sources of links that leave through a y or z face:
        // direct loads, issued before the wait so that they overlap it (the x
        // faces' sources arrive in the edge boxes)
        float v0[kPlanes], v1[kPlanes];
        bool o0[kPlanes], o1[kPlanes];
        static_for<0, kPlanes>([&](auto I) {
            constexpr int q = decltype(I)::value;
            constexpr int ex = plane_ex<q>(), ey = plane_ey<q>(), ez = plane_ez<q>();
            bool oyz = false;
            if constexpr (ey == 1) oyz = oyz || ylo;
            if constexpr (ey == -1) oyz = oyz || yhi;
            if constexpr (ez == 1) oyz = oyz || zlo;
            if constexpr (ez == -1) oyz = oyz || zhi;
            const bool xo0 = ex == 1 && xlo, xo1 = ex == -1 && xhi;
            o0[q] = valid && (oyz || xo0);
            o1[q] = valid && (oyz || xo1);
            const unsigned bb = static_cast<unsigned>(S.bb[q]);
            v0[q] = o0[q] && !xo0 ? Pair<T>::ld1(Bp + bb) : 0.0f;
            v1[q] = o1[q] && !xo1 ? Pair<T>::ld1((Bp + bb) + 1) : 0.0f;
        });
        ok = umma::mbar_wait(&bar[s], (j / kTmaStages) & 1, kTmaWaitPolls);
        if (!__syncthreads_and(ok)) break;
        // every thread is past its reads of the stage last used at z - 1: refill it
        if (leader && z + kTmaStages - 1 < ze)
            tma_issue_slab(&map, &edge, smem + ((j + kTmaStages - 1) % kTmaStages) * kTmaStageBytes,
                           &bar[(j + kTmaStages - 1) % kTmaStages], xs, y0, z + kTmaStages - 1, left, right,
                           S.nx);
        if (valid) {
            // ---- values from the staged rows, shifted by -e_x
            const unsigned char *st = smem + s * kTmaStageBytes + ty * (kTmaBoxW * 2);
            const unsigned char *eb = smem + s * kTmaStageBytes + kPlanes * kTmaPlaneBytes + ty * (kTmaEdgeW * 2);
            F2 d[19], g[7];
            static_for<0, kPlanes>([&](auto I) {
                constexpr int q = decltype(I)::value;
                constexpr int ex = plane_ex<q>();
                const T *row = reinterpret_cast<const T *>(st + q * kTmaPlaneBytes);
                float a = v0[q], b = v1[q];
                if constexpr (ex == 0) {
                    if (!o0[q]) {
                        const float2 w = Pair<T>::ld2(row + k0);
                        a = w.x;
                        b = w.y;
                    }
                } else {
                    if (!o0[q]) a = Pair<T>::ld1(row + k0 - ex);
                    if (!o1[q]) b = Pair<T>::ld1(row + k0 + 1 - ex);
                    // x faces: the opposite plane's own slot from the edge box
                    if constexpr (ex == 1) {
                        if (xlo) a = Pair<T>::ld1(reinterpret_cast<const T *>(eb + edge_slot<q>() * kTmaEdgeSlot));
                    } else {
                        if (xhi)
                            b = Pair<T>::ld1(reinterpret_cast<const T *>(
                                                 eb + (kTmaEdgeLinks + edge_slot<q>()) * kTmaEdgeSlot) +
                                             (kTmaEdgeW - 1));
                    }
                }
                if constexpr (q >= 20 && dirichlet_axis<WALL>(plane_ex<q>() != 0 ? 0 : (plane_ey<q>() != 0 ? 1 : 2))) {
                    constexpr int axis = plane_ex<q>() != 0 ? 0 : (plane_ey<q>() != 0 ? 1 : 2);
                    float tw;
                    if constexpr (axis == 1) tw = (plane_ey<q>() == 1) ? 0.5f : -0.5f;
                    else tw = th_lin;
                    a = o0[q] ? fmaf(wall_coef<T>(), tw, -a) : a;  // anti-bounce-back
                    b = o1[q] ? fmaf(wall_coef<T>(), tw, -b) : b;
                }
                if constexpr (q < 19) d[q] = F2(a, b);
                else g[q - 19] = F2(a, b);
            });
            collide_stored<T>(C, d, g);
            unsigned r01 = 0;
            if constexpr (SR) {
                if (self == 0) *reinterpret_cast<unsigned *>(dst + static_cast<size_t>(kPlanes) * S.plane) = step + 1u;
                r01 = pair_bits(self, step);
            }
            T *Dp = dst + self;
            const unsigned plane = opaque(S.plane);
            static_for<0, 26>([&](auto I) {
                constexpr int q = decltype(I)::value;
                store2<T, SR>(Dp + q * plane, plane_value<q>(d, g), SR ? plane_bits<q>(r01) : 0u);
            });
        }
    }
    if (!ok) {
        // a stage never completed: report it, then give the copies already
        // issued (slabs j .. j + kTmaStages - 2) a bounded time to land
        if (leader) {
            atomicOr(err, 1u);
            for (int k = 0; k < kTmaStages - 1 && zb + j + k < ze; ++k)
                umma::mbar_wait(&bar[(j + k) % kTmaStages], ((j + k) / kTmaStages) & 1, kTmaWaitPolls);
        }
        __syncthreads();
    }
}

}  // namespace

bool step_pair_supported(int wall, const Geometry &G)
{
    return wall >= 1 && wall <= 3 && G.nx % 2 == 0 && G.plane % 2 == 0;
}

namespace {

// Launch shape of the paired kernels: one row of up to 128 cells per block
// row, kPairThreads threads per block.
cudaLaunchConfig_t pair_config(const Geometry &G, cudaStream_t s, cudaLaunchAttribute *attr, bool pdl)
{
    const int threads = kPairThreads;
    const int pairs = G.nx / 2;
    // the tile width (in pairs) that launches the fewest idle threads along a
    // row, the widest of equals: 48 pairs take 3 tiles of 16, not 2 of 32
    int bx = 16, slots = (pairs + 15) / 16 * 16;
    for (int cand : {32, 64}) {
        const int c = (pairs + cand - 1) / cand * cand;
        if (c <= slots) bx = cand, slots = c;
    }
    const int by = threads / bx > 0 ? threads / bx : 1;
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

size_t pair_blocks(const Geometry &G)
{
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pair_config(G, nullptr, attr, false);
    return static_cast<size_t>(cfg.gridDim.x) * cfg.gridDim.y * cfg.gridDim.z;
}

cudaError_t launch_step_pair(int wall, int storage, bool stochastic, const void *src, void *dst,
                             const StepGeometry &S, const Geometry &G, const CollideParams &C,
                             cudaStream_t s, bool pdl, const ResidualArgs *res)
{
    if (!step_pair_supported(wall, G)) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(G, s, attr, pdl);
    const ResidualArgs R = res ? *res : ResidualArgs{};
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        if constexpr (WL == 0) {
            return cudaErrorInvalidValue;
        } else {
            const T *a = static_cast<const T *>(src);
            T *b = static_cast<T *>(dst);
            auto go = [&](auto sr) {
                constexpr bool SRv = decltype(sr)::value;
                if (res) return cudaLaunchKernelEx(&cfg, step_pair_kernel<WL, T, SRv, true>, a, b, S, C, R);
                return cudaLaunchKernelEx(&cfg, step_pair_kernel<WL, T, SRv, false>, a, b, S, C, R);
            };
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic) return go(std::true_type{});
            }
            return go(std::false_type{});
        }
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

bool step_pair_tma_supported(int wall, int storage, const Geometry &G)
{
    return step_pair_supported(wall, G) && storage != 0 && G.nx % 8 == 0;
}

cudaError_t encode_pair_tma_map(const void *buf, const Geometry &G, void *map, int box_width)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    // the buffer as [26 planes][nz][ny][nx] 16-bit elements; strides in bytes
    const cuuint64_t dims[4] = {static_cast<cuuint64_t>(G.nx), static_cast<cuuint64_t>(G.ny),
                                static_cast<cuuint64_t>(G.nz), static_cast<cuuint64_t>(kPlanes)};
    const cuuint64_t strides[3] = {static_cast<cuuint64_t>(G.nx) * 2, static_cast<cuuint64_t>(G.nx) * G.ny * 2,
                                   static_cast<cuuint64_t>(G.plane) * 2};
    const cuuint32_t box[4] = {static_cast<cuuint32_t>(box_width), kTmaRows, 1, 1};
    const cuuint32_t unit[4] = {1, 1, 1, 1};
    const CUresult r = encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_UINT16, 4,
                              const_cast<void *>(buf), dims, strides, box, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t prepare_step_pair_tma(int wall, int storage)
{
    return dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        if constexpr (WL == 0 || std::is_same_v<T, float>) {
            return cudaErrorInvalidValue;
        } else {
            cudaError_t e = cudaFuncSetAttribute(step_pair_tma_kernel<WL, T, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmemBytes);
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(step_pair_tma_kernel<WL, T, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmemBytes);
        }
    });
}

cudaError_t encode_pair_tma_maps(const void *buf, const Geometry &G, void *maps)
{
    cudaError_t e = encode_pair_tma_map(buf, G, maps, kTmaBoxW);
    if (e != cudaSuccess) return e;
    return encode_pair_tma_map(buf, G, static_cast<unsigned char *>(maps) + sizeof(CUtensorMap), kTmaEdgeW);
}

cudaError_t launch_step_pair_tma(int wall, int storage, bool stochastic, const void *map, const void *src,
                                 void *dst, const StepGeometry &S, const Geometry &G, const CollideParams &C,
                                 unsigned *err, cudaStream_t s, bool pdl)
{
    if (!step_pair_tma_supported(wall, storage, G)) return cudaErrorInvalidValue;
    const int xblocks = (G.nx / 2 + kTmaPairs - 1) / kTmaPairs;
    const int yblocks = (G.ny + kTmaRows - 1) / kTmaRows;
    // z chunks: about eight waves of one resident block on each of 152 SMs
    const int cols = xblocks * yblocks;
    int zchunks = (8 * 152 + cols / 2) / cols;
    zchunks = zchunks < 1 ? 1 : (zchunks > G.nz ? G.nz : zchunks);
    const int zper = (G.nz + zchunks - 1) / zchunks;
    zchunks = (G.nz + zper - 1) / zper;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(xblocks, yblocks, zchunks);
    cfg.blockDim = dim3(kTmaPairs, kTmaRows, 1);
    cfg.dynamicSmemBytes = kTmaSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const CUtensorMap &m = static_cast<const CUtensorMap *>(map)[0];
    const CUtensorMap &me = static_cast<const CUtensorMap *>(map)[1];
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        if constexpr (WL == 0 || std::is_same_v<T, float>) {
            return cudaErrorInvalidValue;
        } else {
            const T *a = static_cast<const T *>(src);
            T *b = static_cast<T *>(dst);
            if (stochastic)
                return cudaLaunchKernelEx(&cfg, step_pair_tma_kernel<WL, T, true>, m, me, a, b, S, C, zper, err);
            return cudaLaunchKernelEx(&cfg, step_pair_tma_kernel<WL, T, false>, m, me, a, b, S, C, zper, err);
        }
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_step_inplace_pair(int wall, int storage, bool stochastic, void *buf, int phase,
                                     const InplaceGeometry &SI, const Geometry &G,
                                     const CollideParams &C, cudaStream_t s, bool pdl,
                                     const ResidualArgs *res)
{
    if (!step_pair_supported(wall, G) || (phase != 0 && phase != 1)) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(G, s, attr, pdl);
    const ResidualArgs R = res ? *res : ResidualArgs{};
    cudaError_t e = dispatch(wall, storage, [&](auto W, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int WL = decltype(W)::value;
        if constexpr (WL == 0) {
            return cudaErrorInvalidValue;
        } else {
            T *A = static_cast<T *>(buf);
            auto go = [&](auto sr) {
                constexpr bool SRv = decltype(sr)::value;
                if (res)
                    return phase == 0
                               ? cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, SRv, 0, true>, A, SI, C, R)
                               : cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, SRv, 1, true>, A, SI, C, R);
                return phase == 0
                           ? cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, SRv, 0, false>, A, SI, C, R)
                           : cudaLaunchKernelEx(&cfg, step_inplace_pair_kernel<WL, T, SRv, 1, false>, A, SI, C, R);
            };
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic) return go(std::true_type{});
            }
            return go(std::false_type{});
        }
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lbm
