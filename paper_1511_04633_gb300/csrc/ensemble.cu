// ensemble.cu -- many independent cavities advanced together, a few kernel
// launches per time step for the whole ensemble, and a residual interval of
// K steps replayed as one captured CUDA graph.
//
// Each cavity keeps its own 26-plane population slab inside two shared
// ping-pong buffers (A-B scheme, as for a single cavity), or inside one
// buffer updated in place by two alternating kernels (the in-place scheme of
// step_inplace.cu, half the population memory).  Two step paths:
//  - shape groups (two cells per thread, few distinct shapes): one launch
//    per shape (and per 64 members), the shape's offset tables in the launch
//    parameters as for a single cavity, the grid a single cavity's with its
//    z extent repeated per member; in a captured interval each group runs as
//    its own chain on a side stream;
//  - tables (otherwise): one launch per 64 members of any shapes, their
//    sizes, strides and rates in the launch parameters, a block map in device
//    memory giving each block its tile.
// The residual and Nusselt kernels read the descriptors from device memory.
// The per-cell arithmetic is the single-cavity body (step_body.cuh), and
// stochastic rounding draws the same bits from the cell index and step
// number, so a member evolves bitwise like a single handle of the same
// cavity.  When every member has an even row length the kernels take two
// cells per thread (pair_body.cuh), as a single cavity does.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "dmrt.h"
#include "reduce.cuh"
#include "pair_body.cuh"

namespace lbm {

struct __align__(8) CavityDesc {
    int nx, ny, nz, wall;
    unsigned plane, nxy;
    float inv_ny;
    int bx, by;              // step tile shape, bx * by = threads per block (bx a power of two)
    int tiles_x, tiles_y;    // step tiles along x and y
    long long offset;        // element offset of the cavity's slab in each buffer
    long long snap_offset;   // float offset of its 4 snapshot planes
    long long red_start;     // first residual block (32 x 8 tiles)
    int red_tiles_x, red_tiles_y;
    CollideParams C;
};

// The step tile of one thread block: its cavity and the tile's coordinates,
// laid out on the host so that a block finds its cells without division.
struct __align__(16) BlockTile {
    int member, tx, ty, z;
};

// The collision parameters that differ between members.  The others (the
// rates of Eq. (26) not set by the viscosity, q_0 and q_4..6, theta_ref = 0,
// isotropic diffusion) are the same for every cavity and come from a
// constant table (kFixedRates); fill_collide_params computes both.
struct MemberRates {
    float rs9, rs11, rs13;  // s_nu / |M_k|^2 for k = 9, 11 and 13..15 (equal norms)
    float ws9, ws11, ws13;  // (1 - s_nu) / |M_k|^2, likewise
    float rq1;              // q_k / |N_k|^2, k = 1, 2, 3 (Eq. (36); equal rates and norms)
    float gbeta;
    // always 0 (isotropic diffusion), but read at run time: the collision's
    // branch on it splits the energy part for the scheduler, and with a
    // constant 0 the in-place kernels spilled about 100 bytes
    int aniso;
};
static_assert(m19_norm2(13) == m19_norm2(14) && m19_norm2(13) == m19_norm2(15),
              "one rate entry serves moments 13, 14 and 15");
static_assert(m7_norm2(1) == m7_norm2(2) && m7_norm2(1) == m7_norm2(3), "one entry serves q_1..3");

struct FixedRates {
    float rs[19], ws[19], rq[7];
};
__host__ __device__ constexpr FixedRates fixed_rates()
{
    FixedRates r{};
    for (int k = 0; k < 19; ++k) {
        r.rs[k] = static_cast<float>(mrt_rate(k) / m19_norm2(k));
        r.ws[k] = static_cast<float>((1.0 - mrt_rate(k)) / m19_norm2(k));
    }
    for (int k = 0; k < 7; ++k) r.rq[k] = static_cast<float>(1.0 / m7_norm2(k));
    return r;
}
// in the constant bank at fixed addresses, so that the collision reads them
// as instruction operands (the entries of the member-dependent rates unused)
__constant__ FixedRates kFixedRates = fixed_rates();

// The parameter set collide_from reads, for one member: the member's rates
// from the launch's parameters, the rest from kFixedRates.
struct MemberCollide {
    struct Rs {
        float r9, r11, r13;
        __device__ __forceinline__ float operator[](int k) const
        {
            return k == 9 ? r9 : k == 11 ? r11 : viscous_moment(k) ? r13 : kFixedRates.rs[k];
        }
    };
    struct Ws {
        float r9, r11, r13;
        __device__ __forceinline__ float operator[](int k) const
        {
            return k == 9 ? r9 : k == 11 ? r11 : viscous_moment(k) ? r13 : kFixedRates.ws[k];
        }
    };
    struct Rq {
        float r1;
        __device__ __forceinline__ float operator[](int k) const
        {
            return (k >= 1 && k <= 3) ? r1 : kFixedRates.rq[k];
        }
    };
    struct Qa {
        __device__ __forceinline__ float operator[](int) const { return 0.0f; }
    };
    Rs rs;
    Ws ws;
    Rq rq;
    Qa qa;
    float gbeta;
    static constexpr float theta_ref = 0.0f;
    int aniso;
    __device__ __forceinline__ explicit MemberCollide(const MemberRates &r)
        : rs{r.rs9, r.rs11, r.rs13}, ws{r.ws9, r.ws11, r.ws13}, rq{r.rq1}, qa{}, gbeta(r.gbeta), aniso(r.aniso)
    {
    }
};

// What a step kernel needs of one member.  A launch carries the members it
// covers by value in its parameters (StepTable, at most kStepTableMembers):
// the block's member then follows from the block index alone, so every field
// is the same for the whole block and lives in the constant bank; the
// kernels read them as operands there instead of holding them in registers
// or re-reading them from shared memory.
struct MemberStep {
    int nx, ny, nz, wall;
    unsigned plane, nxy;
    float inv_ny;
    int bx_log2, by;         // step tile shape (see CavityDesc; bx = 2^bx_log2)
    long long offset;        // element offset of the member's slab in each buffer
    MemberRates r;
};

constexpr int kStepTableMembers = 64;

struct StepTable {
    int count;                                // members of this launch
    int first_block[kStepTableMembers + 1];   // their first blocks in the launch's grid, then its size
    MemberStep m[kStepTableMembers];
};
static_assert(sizeof(StepTable) <= 32000, "a launch's parameters hold at most 32764 bytes");

namespace {

constexpr int kEnsRedThreads = 256;
constexpr int kMinBlocksEns = 4;
// Minimum resident 256-thread blocks per SM of the in-place phases (4 caps a
// kernel at 64 registers, 3 at 80).  Measured on GB300 (64 members, FP32):
// 64 registers everywhere gave 805 us per step, 80 registers 842 us.
#ifndef DMRT_ENS_INPLACE_MIN_BLOCKS0
#define DMRT_ENS_INPLACE_MIN_BLOCKS0 4
#endif
#ifndef DMRT_ENS_INPLACE_MIN_BLOCKS1
#define DMRT_ENS_INPLACE_MIN_BLOCKS1 4
#endif
// DMRT_ENS_INPLACE_BLOCK128 = N: the in-place phases are compiled for blocks
// of 128 threads with N resident per SM (e.g. 7 gives 72 registers), and
// autotuning tries only 128-thread blocks for in-place ensembles.
#ifndef DMRT_ENS_INPLACE_BLOCK128
#define DMRT_ENS_INPLACE_BLOCK128 7  // 72 registers, no spills; measured 1 % faster than 64
#endif
#if DMRT_ENS_INPLACE_BLOCK128
#define DMRT_ENS_INPLACE_BOUNDS(PHASE) __launch_bounds__(128, DMRT_ENS_INPLACE_BLOCK128)
#else
#define DMRT_ENS_INPLACE_BOUNDS(PHASE) \
    __launch_bounds__(256, PHASE == 0 ? DMRT_ENS_INPLACE_MIN_BLOCKS0 : DMRT_ENS_INPLACE_MIN_BLOCKS1)
#endif

// ---------------------------------------------------------------- step

// The member of this block in a launch's table: the last whose first block
// is not above the block index (a search over block-uniform values).
__device__ __forceinline__ const MemberStep &member_of_block(const StepTable &P)
{
    const int b = static_cast<int>(blockIdx.x);
    int lo = 0, hi = P.count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P.first_block[mid] <= b) lo = mid;
        else hi = mid;
    }
    return P.m[lo];
}

// The thread's cell (x, or the pair index along x) in the block's tile of
// member D: false if it lies outside the member.
__device__ __forceinline__ void tile_position(const MemberStep &D, const BlockTile *__restrict__ blockmap, int &x,
                                              int &y, int &z)
{
    const BlockTile t = blockmap[blockIdx.x];
    const int tid = static_cast<int>(threadIdx.x);
    x = (t.tx << D.bx_log2) + (tid & ((1 << D.bx_log2) - 1));
    y = t.ty * D.by + (tid >> D.bx_log2);
    z = t.z;
}

// One cell of a walled cavity (Types 1-3; the wall type is a per-cavity
// runtime value, which only changes the thermal rule on the x and z walls).
template <typename T, bool SR>
__device__ __forceinline__ void ensemble_cell(const T *__restrict__ src, T *__restrict__ dst,
                                              const MemberStep &D, int x, int y, int z,
                                              unsigned salt)
{
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const unsigned plane = D.plane;
    const unsigned self = (static_cast<unsigned>(z) * ny + y) * nx + x;
    float d[19], g[7];
    const bool dir_x = D.wall != 1;  // Types 2 and 3: linear x walls
    const bool dir_z = D.wall == 2;  // Type 2: linear z walls
    pull_offsets<kRuntimeWall, T>(src, ComputedOffsets{plane, static_cast<unsigned>(nx), D.nxy}, nx,
                                  ny, nz, D.inv_ny, self, x, y, z, d, g, dir_x, dir_z);
    collide_cell(MemberCollide(D.r), d, g);
    // the store offsets from a stride the compiler cannot see through
    // (see ensemble_inplace_kernel); the same random word as a single
    // cavity (step.cu) at the same step
    store_cell<T, SR>(dst, self, opaque(D.plane), d, g, SR ? pcg_hash(self ^ salt) : 0u);
}

template <typename T, bool SR>
__global__ void __launch_bounds__(256, kMinBlocksEns)
    ensemble_step_kernel(const T *__restrict__ srcb, T *__restrict__ dstb, const BlockTile *__restrict__ blockmap,
                         long long counter_at, const __grid_constant__ StepTable P)
{
    // programmatic dependent launch (see step.cu)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    unsigned salt = 0;
    if constexpr (SR) {
        const unsigned step = *reinterpret_cast<const unsigned *>(srcb + counter_at);
        if (blockIdx.x == 0 && threadIdx.x == 0)
            *reinterpret_cast<unsigned *>(dstb + counter_at) = step + 1u;
        salt = pcg_hash(step);
    }
    const MemberStep &D = member_of_block(P);
    int x, y, z;
    tile_position(D, blockmap, x, y, z);
    if (x >= D.nx || y >= D.ny) return;
    ensemble_cell<T, SR>(srcb + D.offset, dstb + D.offset, D, x, y, z, salt);
}

// In-place scheme (see step_inplace.cu): phase 0 pulls from the neighbours'
// swapped slots and pushes to theirs, phase 1 works on the cell's own slots.
// The buffer's tail holds two step counters: phase p reads word p and writes
// word p ^ 1.
template <typename T, bool SR, int PHASE>
__global__ void DMRT_ENS_INPLACE_BOUNDS(PHASE)
    ensemble_inplace_kernel(T *__restrict__ buf, const BlockTile *__restrict__ blockmap, long long counter_at,
                            const __grid_constant__ StepTable P)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    unsigned salt = 0;
    if constexpr (SR) {
        unsigned *ctr = reinterpret_cast<unsigned *>(buf + counter_at);
        const unsigned step = ctr[PHASE];
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[PHASE ^ 1] = step + 1u;
        salt = pcg_hash(step);
    }
    const MemberStep &D = member_of_block(P);
    int x, y, z;
    tile_position(D, blockmap, x, y, z);
    if (x >= D.nx || y >= D.ny) return;
    T *A = buf + D.offset;
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const unsigned plane = D.plane;
    const unsigned self = (static_cast<unsigned>(z) * ny + y) * nx + x;
    const bool dir_x = D.wall != 1, dir_z = D.wall == 2;
    const SwappedOffsets O{plane, static_cast<unsigned>(nx), D.nxy};
    float d[19], g[7];
    if constexpr (PHASE == 0)
        pull_offsets<kRuntimeWall, T>(A, O, nx, ny, nz, D.inv_ny, self, x, y, z, d, g, dir_x, dir_z);
    else
        pull_offsets<kRuntimeWall, T>(A, LocalOffsets{plane}, nx, ny, nz, D.inv_ny, self, x, y, z, d,
                                      g, dir_x, dir_z);
    collide_cell(MemberCollide(D.r), d, g);
    const unsigned base = SR ? pcg_hash(self ^ salt) : 0u;
    // The store offsets equal the load offsets (each cell writes the slots it
    // read); left to itself the compiler keeps all 26 of them live through the
    // collision and spills.  A stride it cannot see through (opaque) makes it
    // recompute them at the stores instead.
    const unsigned splane = opaque(D.plane);
    if constexpr (PHASE == 1) {
        store_cell_to<T, SR>(A, d, g, base, [&](auto I) -> unsigned {
            return self + plane_opp<decltype(I)::value>() * splane;
        });
    } else {
        const SwappedOffsets SO{splane, static_cast<unsigned>(D.nx), D.nxy};
        const unsigned edge = face_bits(x, y, z, D.nx, D.ny, D.nz);
        store_cell_to<T, SR>(A, d, g, base, [&](auto I) -> unsigned {
            constexpr int q = decltype(I)::value;
            constexpr unsigned faces = leaving_faces<q>();
            if constexpr (faces == 0) return self + SO.template sn<q>();
            else return self + ((edge & faces) ? SO.template sb<q>() : SO.template sn<q>());
        });
    }
}

// ---------------------------------------------------------------- two cells per thread

// 128-thread blocks, 5 resident per SM (96 registers), as the single-cavity
// paired kernels of BF16 storage.
constexpr int kEnsPairBlocks = 5;

// The pair of the thread (tiles of pairs): the cells x0, x0 + 1 with x0 =
// 2 (tile x * bx + thread x); false if it lies outside the member.
__device__ __forceinline__ bool locate_pair(const MemberStep &D, const BlockTile *__restrict__ blockmap, int &x0,
                                            int &y, int &z)
{
    int xp;
    tile_position(D, blockmap, xp, y, z);
    x0 = 2 * xp;
    return x0 < D.nx && y < D.ny;
}

__device__ __forceinline__ PairFaces pair_faces(const MemberStep &D, int x0, int y, int z)
{
    return PairFaces{x0 == 0, x0 + 2 == D.nx, y == 0, y == D.ny - 1, z == 0, z == D.nz - 1};
}

// One pair of a member: pull (the wall type, which only sets the thermal
// rule of the x and z walls, is a runtime value: taken at compile time per
// block, the three bodies spilled 300-400 bytes), collide, and store each
// plane as soon as the collision has its value.
template <typename T, bool SR>
__device__ __forceinline__ void ensemble_pair_body(const T *__restrict__ src, T *__restrict__ dst,
                                                   const MemberStep &D, int x0, int y, int z, unsigned salt)
{
    const unsigned self = (static_cast<unsigned>(z) * D.ny + y) * D.nx + x0;
    F2 d[19], g[7];
    pull_pair<kRuntimeWall, T>(src + self, ComputedOffsets{D.plane, static_cast<unsigned>(D.nx), D.nxy},
                               pair_faces(D, x0, y, z), theta_linear(y, D.inv_ny), d, g, D.wall != 1,
                               D.wall == 2);
    const unsigned r01 = SR ? pair_bits_salted(self, salt) : 0u;
    T *Dp = dst + self;
    const unsigned plane = opaque(D.plane);  // (see ensemble_inplace_pair_body)
    collide_from<F2, Pair<T>::kShift>(MemberCollide(D.r), d, g, conserved<F2, Pair<T>::kShift>(d, g),
                                      plane_sink([&](auto I, F2 v) {
                                          constexpr int q = decltype(I)::value;
                                          store2<T, SR>(Dp + q * plane, v, SR ? plane_bits<q>(r01) : 0u);
                                      }));
}

template <typename T, bool SR>
__global__ void __launch_bounds__(128, kEnsPairBlocks)
    ensemble_pair_kernel(const T *__restrict__ srcb, T *__restrict__ dstb, const BlockTile *__restrict__ blockmap,
                         long long counter_at, const __grid_constant__ StepTable P)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    unsigned salt = 0;
    if constexpr (SR) {
        const unsigned step = *reinterpret_cast<const unsigned *>(srcb + counter_at);
        if (blockIdx.x == 0 && threadIdx.x == 0)
            *reinterpret_cast<unsigned *>(dstb + counter_at) = step + 1u;
        salt = pcg_hash(step);
    }
    const MemberStep &D = member_of_block(P);
    int x0, y, z;
    if (!locate_pair(D, blockmap, x0, y, z)) return;
    ensemble_pair_body<T, SR>(srcb + D.offset, dstb + D.offset, D, x0, y, z, salt);
}

// In-place scheme with two cells per thread (see step_inplace_pair_kernel).
template <typename T, bool SR, int PHASE>
__device__ __forceinline__ void ensemble_inplace_pair_body(T *__restrict__ A, const MemberStep &D, int x0, int y,
                                                           int z, unsigned salt)
{
    const unsigned self = (static_cast<unsigned>(z) * D.ny + y) * D.nx + x0;
    const PairFaces P = pair_faces(D, x0, y, z);
    F2 d[19], g[7];
    if constexpr (PHASE == 0)
        pull_pair<kRuntimeWall, T>(A + self, SwappedOffsets{D.plane, static_cast<unsigned>(D.nx), D.nxy}, P,
                                   theta_linear(y, D.inv_ny), d, g, D.wall != 1, D.wall == 2);
    else
        pull_pair<kRuntimeWall, T>(A + self, LocalOffsets{D.plane}, P, theta_linear(y, D.inv_ny), d, g,
                                   D.wall != 1, D.wall == 2);
    const unsigned r01 = SR ? pair_bits_salted(self, salt) : 0u;
    // store addresses from a stride the compiler cannot see through, so that
    // it recomputes them instead of keeping the load addresses live
    T *Dp = A + self;
    const SwappedOffsets SO{opaque(D.plane), static_cast<unsigned>(D.nx), D.nxy};
    collide_from<F2, Pair<T>::kShift>(MemberCollide(D.r), d, g, conserved<F2, Pair<T>::kShift>(d, g), plane_sink([&](auto I, F2 v) {
        constexpr int q = decltype(I)::value;
        const unsigned r = SR ? plane_bits<q>(r01) : 0u;
        if constexpr (PHASE == 1) {
            store2<T, SR>(Dp + plane_opp<q>() * SO.plane, v, r);
        } else {
            constexpr int ex = plane_ex<q>(), ey = plane_ey<q>(), ez = plane_ez<q>();
            bool lyz = false;  // the link leaves through a y or z face
            if constexpr (ey == 1) lyz = lyz || P.yhi;
            if constexpr (ey == -1) lyz = lyz || P.ylo;
            if constexpr (ez == 1) lyz = lyz || P.zhi;
            if constexpr (ez == -1) lyz = lyz || P.zlo;
            const unsigned sn = SO.template sn<q>(), sb = SO.template sb<q>();
            if constexpr (ex == 0) {
                store2<T, SR>(Dp + (lyz ? sb : sn), v, r);
            } else {
                const bool l0 = lyz || (ex == -1 && P.xlo);
                const bool l1 = lyz || (ex == 1 && P.xhi);
                store_split<T, SR>(Dp + (l0 ? sb : sn), (Dp + (l1 ? sb : sn)) + 1, v, r);
            }
        }
    }));
}

template <typename T, bool SR, int PHASE>
__global__ void __launch_bounds__(128, kEnsPairBlocks)
    ensemble_inplace_pair_kernel(T *__restrict__ buf, const BlockTile *__restrict__ blockmap, long long counter_at,
                                 const __grid_constant__ StepTable P)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    unsigned salt = 0;
    if constexpr (SR) {
        unsigned *ctr = reinterpret_cast<unsigned *>(buf + counter_at);
        const unsigned step = ctr[PHASE];
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[PHASE ^ 1] = step + 1u;
        salt = pcg_hash(step);
    }
    const MemberStep &D = member_of_block(P);
    int x0, y, z;
    if (!locate_pair(D, blockmap, x0, y, z)) return;
    ensemble_inplace_pair_body<T, SR, PHASE>(buf + D.offset, D, x0, y, z, salt);
}

// ---------------------------------------------------------------- shape groups

// The members of one shape (nx, ny, nz) stepped together, two cells per
// thread: the shape's offset tables are launch parameters, as a single
// cavity's are (StepGeometry / InplaceGeometry, read as instruction
// operands), and the grid is that of a single cavity with its z extent
// repeated once per member, so a block finds its member as blockIdx.z / nz.
// The member's slab, wall type and rates come from the launch's table.
struct GroupMember {
    long long offset;  // element offset of the member's slab in each buffer
    MemberRates r;
    int wall;
};

constexpr int kGroupMembers = 64;

struct GroupTable {
    int count;
    GroupMember m[kGroupMembers];
};
static_assert(sizeof(GroupTable) + sizeof(InplaceGeometry) + 64 <= 32000, "launch parameters");

// Step counters of a group launch (stochastic rounding): the kernel draws
// its bits from the step number *read and writes that number plus one to
// *write (and to *tail if not null).  Run one after another, the launches
// use the buffer's own counters; run as concurrent chains (one per launch
// of a step, within a captured interval), each chain keeps its own pair and
// also keeps the buffer's counter current.
struct GroupCounters {
    const unsigned *read;
    unsigned *write;
    unsigned *tail;
};

__device__ __forceinline__ unsigned group_step(const GroupCounters &K)
{
    const unsigned step = *K.read;
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) {
        *K.write = step + 1u;
        if (K.tail) *K.tail = step + 1u;
    }
    return step;
}

// Copy a buffer's step counter into word `from` of each chain's pair (the
// start of a concurrently captured interval).
__global__ void ensemble_counter_sync(const unsigned *__restrict__ tail, unsigned *__restrict__ pairs, int n, int from)
{
    if (threadIdx.x < static_cast<unsigned>(n)) pairs[2 * threadIdx.x + from] = *tail;
}

// The block's member, z slab and pair (x0 even); false outside the shape.
__device__ __forceinline__ bool group_pair(const StepGeometry &S, unsigned &m, int &x0, int &y, int &z)
{
    m = blockIdx.z / static_cast<unsigned>(S.nz);
    z = static_cast<int>(blockIdx.z - m * static_cast<unsigned>(S.nz));
    x0 = 2 * static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    y = static_cast<int>(blockIdx.y * blockDim.y + threadIdx.y);
    return x0 < S.nx && y < S.ny;
}

// srcb is not declared read-only (const __restrict__): through the
// read-only load path this kernel ran 4 % slower (16 members of 96^3, BF16:
// 286 against 275 us per step), while the single-cavity kernel's speed did
// not depend on it.
template <typename T, bool SR>
__global__ void __launch_bounds__(128, kEnsPairBlocks)
    ensemble_group_pair_kernel(const T *srcb, T *dstb, const StepGeometry S, const GroupCounters K,
                               const __grid_constant__ GroupTable P)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    unsigned salt = 0;
    if constexpr (SR) salt = pcg_hash(group_step(K));
    unsigned m;
    int x0, y, z;
    if (!group_pair(S, m, x0, y, z)) return;
    const GroupMember &M = P.m[m];
    const unsigned self = (static_cast<unsigned>(z) * S.ny + y) * S.nx + x0;
    const PairFaces faces{x0 == 0, x0 + 2 == S.nx, y == 0, y == S.ny - 1, z == 0, z == S.nz - 1};
    F2 d[19], g[7];
    pull_pair<kRuntimeWall, T>(srcb + M.offset + self, TableOffsets{S}, faces, theta_linear(y, S.inv_ny), d, g,
                               M.wall != 1, M.wall == 2);
    const unsigned r01 = SR ? pair_bits_salted(self, salt) : 0u;
    T *Dp = dstb + M.offset + self;
    const unsigned plane = opaque(S.plane);  // (see ensemble_inplace_pair_body)
    collide_from<F2, Pair<T>::kShift>(MemberCollide(M.r), d, g, conserved<F2, Pair<T>::kShift>(d, g),
                                      plane_sink([&](auto I, F2 v) {
                                          constexpr int q = decltype(I)::value;
                                          store2<T, SR>(Dp + q * plane, v, SR ? plane_bits<q>(r01) : 0u);
                                      }));
}

// In-place scheme (step_inplace_pair_kernel's two phases) for a shape group.
template <typename T, bool SR, int PHASE>
__global__ void __launch_bounds__(128, kEnsPairBlocks)
    ensemble_group_inplace_pair_kernel(T *__restrict__ buf, const InplaceGeometry SI, const GroupCounters K,
                                       const __grid_constant__ GroupTable P)
{
    const StepGeometry &S = SI.load;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    unsigned salt = 0;
    if constexpr (SR) salt = pcg_hash(group_step(K));
    unsigned m;
    int x0, y, z;
    if (!group_pair(S, m, x0, y, z)) return;
    const GroupMember &M = P.m[m];
    T *A = buf + M.offset;
    const unsigned self = (static_cast<unsigned>(z) * S.ny + y) * S.nx + x0;
    const PairFaces P2{x0 == 0, x0 + 2 == S.nx, y == 0, y == S.ny - 1, z == 0, z == S.nz - 1};
    F2 d[19], g[7];
    if constexpr (PHASE == 0)
        pull_pair<kRuntimeWall, T>(A + self, TableOffsets{S}, P2, theta_linear(y, S.inv_ny), d, g, M.wall != 1,
                                   M.wall == 2);
    else
        pull_pair<kRuntimeWall, T>(A + self, LocalOffsets{S.plane}, P2, theta_linear(y, S.inv_ny), d, g,
                                   M.wall != 1, M.wall == 2);
    const unsigned r01 = SR ? pair_bits_salted(self, salt) : 0u;
    T *Dp = A + self;
    const unsigned plane = opaque(S.plane);
    collide_from<F2, Pair<T>::kShift>(MemberCollide(M.r), d, g, conserved<F2, Pair<T>::kShift>(d, g),
                                      plane_sink([&](auto I, F2 v) {
        constexpr int q = decltype(I)::value;
        const unsigned r = SR ? plane_bits<q>(r01) : 0u;
        if constexpr (PHASE == 1) {
            store2<T, SR>(Dp + plane_opp<q>() * plane, v, r);
        } else {
            constexpr int ex = plane_ex<q>(), ey = plane_ey<q>(), ez = plane_ez<q>();
            bool lyz = false;  // the link leaves through a y or z face
            if constexpr (ey == 1) lyz = lyz || P2.yhi;
            if constexpr (ey == -1) lyz = lyz || P2.ylo;
            if constexpr (ez == 1) lyz = lyz || P2.zhi;
            if constexpr (ez == -1) lyz = lyz || P2.zlo;
            const unsigned sn = static_cast<unsigned>(SI.sn[q]), sb = static_cast<unsigned>(SI.sb[q]);
            if constexpr (ex == 0) {
                store2<T, SR>(Dp + (lyz ? sb : sn), v, r);
            } else {
                const bool l0 = lyz || (ex == -1 && P2.xlo);
                const bool l1 = lyz || (ex == 1 && P2.xhi);
                store_split<T, SR>(Dp + (l0 ? sb : sn), (Dp + (l1 ? sb : sn)) + 1, v, r);
            }
        }
    }));
}

// ---------------------------------------------------------------- residual

__device__ __forceinline__ Geometry geometry_of(const CavityDesc &D, int layout)
{
    Geometry G;
    G.nx = D.nx;
    G.ny = D.ny;
    G.nz = D.nz;
    G.layout = layout;
    G.plane = D.plane;
    G.inv_ny = D.inv_ny;
    return G;
}

template <int WALL, typename T>
__device__ __forceinline__ Conserved<float> pulled_moments(const T *src, const Geometry &G, int x, int y, int z)
{
    float d[19], g[7];
    pull_f<WALL, T>(src, G, x, y, z, d);
    pull_g<WALL, T>(src, G, x, y, z, g);
    return conserved<float>(d, g);
}

// Per residual block (32 x 8 cells of one cavity): a residual point of the
// current state (reading A11) against the cavity's snapshot, which is then
// refreshed.  The fields are the moments as the step kernels form them and
// the sums are those of a single cavity's step kernel (residual.cuh): FP32
// terms per cell, double-float sums, one partial per block.
template <typename T>
__global__ void __launch_bounds__(kEnsRedThreads)
    ensemble_residual_kernel(const T *__restrict__ srcb, const CavityDesc *__restrict__ descs,
                             const int *__restrict__ redmap, int layout, float *__restrict__ snapb,
                             const double *__restrict__ points, float *__restrict__ partials)
{
    const int c = redmap[blockIdx.x];
    const CavityDesc &D = descs[c];
    const long long b = static_cast<long long>(blockIdx.x) - D.red_start;
    const int x = static_cast<int>(b % D.red_tiles_x) * 32 + threadIdx.x;
    const long long r = b / D.red_tiles_x;
    const int y = static_cast<int>(r % D.red_tiles_y) * 8 + threadIdx.y;
    const int z = static_cast<int>(r / D.red_tiles_y);
    DF acc[4] = {};
    if (x < D.nx && y < D.ny) {
        const unsigned cells = static_cast<unsigned>(D.nx) * D.ny * D.nz;
        const unsigned cell = (static_cast<unsigned>(z) * D.ny + y) * D.nx + x;
        const ResidualArgs R{snapb + D.snap_offset, partials, points, cells};
        float prev[4];
        residual_cell_load(R, cell, prev);  // with the populations' loads
        const Geometry G = geometry_of(D, layout);
        const T *src = srcb + D.offset;
        Conserved<float> m;
        switch (D.wall) {
        case 0: m = pulled_moments<0, T>(src, G, x, y, z); break;
        case 1: m = pulled_moments<1, T>(src, G, x, y, z); break;
        case 2: m = pulled_moments<2, T>(src, G, x, y, z); break;
        default: m = pulled_moments<3, T>(src, G, x, y, z); break;
        }
        residual_cell(R, cell, prev, m.Tu, m.vx, m.vy, m.vz, acc);
    }
    residual_block_store(acc, partials);
}

__device__ double ens_rel_change(double num2, double den2)
{
    if (den2 == 0.0) return num2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(num2) / sqrt(den2);
}

// One block per member: its residual blocks' partials summed in index
// order in double-float arithmetic (as residual_finish does for a single
// cavity), the totals in FP64, r of reading A11.  *points counts the
// residual points since the last reset (capped at 2); the block that
// finishes last (a ticket counter, left at 0) raises it, after every block
// has read it.
constexpr int kEnsFinThreads = 256;

__global__ void __launch_bounds__(kEnsFinThreads)
    ensemble_residual_finish(const CavityDesc *__restrict__ descs, const float *__restrict__ partials, int K,
                             double *result, double *points, unsigned *ticket)
{
    const int c = blockIdx.x;
    const bool have_prev = *points > 0.0;
    const CavityDesc &D = descs[c];
    const long long nb = static_cast<long long>(D.red_tiles_x) * D.red_tiles_y * D.nz;
    DF v[4] = {};
    for (long long p = threadIdx.x; p < nb; p += kEnsFinThreads) {
        const float4 a = *reinterpret_cast<const float4 *>(partials + (D.red_start + p) * 8);
        const float4 b = *reinterpret_cast<const float4 *>(partials + (D.red_start + p) * 8 + 4);
        v[0] = df_add(v[0], DF{a.x, a.y});
        v[1] = df_add(v[1], DF{a.z, a.w});
        v[2] = df_add(v[2], DF{b.x, b.y});
        v[3] = df_add(v[3], DF{b.z, b.w});
    }
    __shared__ DF sh[kEnsFinThreads / 32][4];
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
    if (warp != 0) return;
    double tot[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        DF w = lane < kEnsFinThreads / 32 ? sh[lane][k] : DF{0.0f, 0.0f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = df_add(w, df_shfl_down(w, o));
        tot[k] = static_cast<double>(w.hi) + static_cast<double>(w.lo);
    }
    if (lane == 0) {
        bool finite = true;
        for (int k = 0; k < 4; ++k) finite = finite && isfinite(tot[k]);
        const double rr =
            have_prev ? fmax(ens_rel_change(tot[0], tot[1]), ens_rel_change(tot[2], tot[3])) / K : INFINITY;
        result[c * 2 + 0] = finite ? rr : NAN;
        result[c * 2 + 1] = finite ? 0.0 : 1.0;
        __threadfence();
        if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
            *points = fmin(*points + 1.0, 2.0);
            *ticket = 0u;
        }
    }
}

// ---------------------------------------------------------------- Nusselt

template <int WALL, typename T>
__device__ __forceinline__ float pulled_T(const T *src, const Geometry &G, int x, int y, int z)
{
    float g[7];
    pull_g<WALL, T>(src, G, x, y, z, g);
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 7; ++i) t += g[i];
    return t;
}

// Block (z, cavity): local Nu of one row of the wall (as nusselt_kernel).
template <typename T>
__global__ void __launch_bounds__(kEnsRedThreads)
    ensemble_nusselt_kernel(const T *__restrict__ srcb, const CavityDesc *__restrict__ descs,
                            int layout, int wall, int max_nz, double *__restrict__ partials)
{
    const int c = blockIdx.y, z = blockIdx.x;
    const CavityDesc &D = descs[c];
    if (z >= D.nz) return;  // uniform per block
    const Geometry G = geometry_of(D, layout);
    const T *src = srcb + D.offset;
    const int y1 = wall == 0 ? 0 : D.ny - 1;
    const int y2 = wall == 0 ? 1 : D.ny - 2;
    const double th_w = wall == 0 ? 0.5 : -0.5;
    const double H = static_cast<double>(D.ny);
    const int c_lo = (D.nx % 2 == 0) ? D.nx / 2 - 1 : (D.nx - 1) / 2;
    const int c_hi = (D.nx % 2 == 0) ? D.nx / 2 : (D.nx - 1) / 2;
    double v[2] = {0.0, 0.0};
    double mx = -INFINITY;
    for (int x = threadIdx.x; x < D.nx; x += kEnsRedThreads) {
        float t1, t2;
        switch (D.wall) {
        case 0: t1 = pulled_T<0, T>(src, G, x, y1, z); t2 = pulled_T<0, T>(src, G, x, y2, z); break;
        case 1: t1 = pulled_T<1, T>(src, G, x, y1, z); t2 = pulled_T<1, T>(src, G, x, y2, z); break;
        case 2: t1 = pulled_T<2, T>(src, G, x, y1, z); t2 = pulled_T<2, T>(src, G, x, y2, z); break;
        default: t1 = pulled_T<3, T>(src, G, x, y1, z); t2 = pulled_T<3, T>(src, G, x, y2, z); break;
        }
        const double dth_ds = (-8.0 * th_w + 9.0 * t1 - static_cast<double>(t2)) / 3.0;
        const double nu = wall == 0 ? -H * dth_ds : H * dth_ds;
        v[0] += nu;
        if (x == c_lo || x == c_hi) v[1] += nu;
        mx = fmax(mx, nu);
    }
    __shared__ double shm[kEnsRedThreads / 32];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
    block_sum<2, kEnsRedThreads>(v);
    if (threadIdx.x == 0) {
        double m = shm[0];
        for (int w = 1; w < kEnsRedThreads / 32; ++w) m = fmax(m, shm[w]);
        double *p = partials + (static_cast<long long>(c) * max_nz + z) * 3;
        p[0] = v[0];
        p[1] = v[1];
        p[2] = m;
    }
}

__global__ void __launch_bounds__(kEnsRedThreads)
    ensemble_nusselt_finish(const CavityDesc *__restrict__ descs, const double *__restrict__ partials,
                            int max_nz, double *out)
{
    const int c = blockIdx.x;
    const CavityDesc &D = descs[c];
    double v[2] = {0.0, 0.0};
    double mx = -INFINITY;
    for (int z = threadIdx.x; z < D.nz; z += kEnsRedThreads) {
        const double *p = partials + (static_cast<long long>(c) * max_nz + z) * 3;
        v[0] += p[0];
        v[1] += p[1];
        mx = fmax(mx, p[2]);
    }
    __shared__ double shm[kEnsRedThreads / 32];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
    block_sum<2, kEnsRedThreads>(v);
    if (threadIdx.x == 0) {
        double m = shm[0];
        for (int w = 1; w < kEnsRedThreads / 32; ++w) m = fmax(m, shm[w]);
        const int ncol = (D.nx % 2 == 0) ? 2 : 1;
        out[c * 3 + 0] = v[0] / (static_cast<double>(D.nx) * D.nz);
        out[c * 3 + 1] = v[1] / (static_cast<double>(D.nz) * ncol);
        out[c * 3 + 2] = m;
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_ensemble_step(int storage, bool stochastic, const void *src, void *dst, const StepTable &P,
                                 const BlockTile *blockmap, long long blocks, int threads, long long counter_at,
                                 cudaStream_t s, bool pdl, bool pairs)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = dispatch(1, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        const T *a = static_cast<const T *>(src);
        T *b = static_cast<T *>(dst);
        if (pairs) {
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic)
                    return cudaLaunchKernelEx(&cfg, ensemble_pair_kernel<T, true>, a, b, blockmap, counter_at, P);
            }
            return cudaLaunchKernelEx(&cfg, ensemble_pair_kernel<T, false>, a, b, blockmap, counter_at, P);
        }
        if constexpr (!std::is_same_v<T, float>) {
            if (stochastic)
                return cudaLaunchKernelEx(&cfg, ensemble_step_kernel<T, true>, a, b, blockmap, counter_at, P);
        }
        return cudaLaunchKernelEx(&cfg, ensemble_step_kernel<T, false>, a, b, blockmap, counter_at, P);
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_ensemble_inplace(int storage, bool stochastic, void *buf, int phase, const StepTable &P,
                                    const BlockTile *blockmap, long long blocks, int threads, long long counter_at,
                                    cudaStream_t s, bool pdl, bool pairs)
{
    if (phase != 0 && phase != 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = dispatch(1, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        T *A = static_cast<T *>(buf);
        auto go = [&](auto kernel) { return cudaLaunchKernelEx(&cfg, kernel, A, blockmap, counter_at, P); };
        if (pairs) {
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic)
                    return phase == 0 ? go(ensemble_inplace_pair_kernel<T, true, 0>)
                                      : go(ensemble_inplace_pair_kernel<T, true, 1>);
            }
            return phase == 0 ? go(ensemble_inplace_pair_kernel<T, false, 0>)
                              : go(ensemble_inplace_pair_kernel<T, false, 1>);
        }
        if constexpr (!std::is_same_v<T, float>) {
            if (stochastic)
                return phase == 0 ? go(ensemble_inplace_kernel<T, true, 0>) : go(ensemble_inplace_kernel<T, true, 1>);
        }
        return phase == 0 ? go(ensemble_inplace_kernel<T, false, 0>) : go(ensemble_inplace_kernel<T, false, 1>);
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// One shape group's chunk: grid (tiles along x, tiles along y, nz * members)
// of bx x (128 / bx) threads; phase < 0: two-buffer step from src to dst,
// else the in-place phase on src.
cudaError_t launch_ensemble_group(int storage, bool stochastic, const void *src, void *dst, int phase,
                                  const InplaceGeometry &SI, const GroupTable &P, int bx, const GroupCounters &K,
                                  cudaStream_t s, bool pdl)
{
    const StepGeometry &S = SI.load;
    const int by = 128 / bx;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>((S.nx / 2 + bx - 1) / bx), static_cast<unsigned>((S.ny + by - 1) / by),
                       static_cast<unsigned>(S.nz) * static_cast<unsigned>(P.count));
    cfg.blockDim = dim3(bx, by, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = dispatch(1, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        if (phase < 0) {
            const T *a = static_cast<const T *>(src);
            T *b = static_cast<T *>(dst);
            if constexpr (!std::is_same_v<T, float>) {
                if (stochastic)
                    return cudaLaunchKernelEx(&cfg, ensemble_group_pair_kernel<T, true>, a, b, S, K, P);
            }
            return cudaLaunchKernelEx(&cfg, ensemble_group_pair_kernel<T, false>, a, b, S, K, P);
        }
        T *A = static_cast<T *>(const_cast<void *>(src));
        auto go = [&](auto kernel) { return cudaLaunchKernelEx(&cfg, kernel, A, SI, K, P); };
        if constexpr (!std::is_same_v<T, float>) {
            if (stochastic)
                return phase == 0 ? go(ensemble_group_inplace_pair_kernel<T, true, 0>)
                                  : go(ensemble_group_inplace_pair_kernel<T, true, 1>);
        }
        return phase == 0 ? go(ensemble_group_inplace_pair_kernel<T, false, 0>)
                          : go(ensemble_group_inplace_pair_kernel<T, false, 1>);
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_counter_sync(const unsigned *tail, unsigned *pairs, int n, int from, cudaStream_t s)
{
    ensemble_counter_sync<<<1, 32, 0, s>>>(tail, pairs, n, from);
    return cudaGetLastError();
}

// points: the count of residual points (device), followed by the finishing
// kernel's ticket word.
cudaError_t launch_ensemble_residual(int storage, const void *src, int layout, const CavityDesc *descs,
                                     const int *redmap, long long red_blocks, int count,
                                     float *snap, int K, float *partials, double *result, double *points,
                                     cudaStream_t s)
{
    cudaError_t e = dispatch(1, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        ensemble_residual_kernel<T><<<static_cast<unsigned>(red_blocks), dim3(32, 8), 0, s>>>(
            static_cast<const T *>(src), descs, redmap, layout, snap, points, partials);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ensemble_residual_finish<<<count, kEnsFinThreads, 0, s>>>(descs, partials, K, result, points,
                                                              reinterpret_cast<unsigned *>(points + 1));
    return cudaGetLastError();
}

cudaError_t launch_ensemble_nusselt(int storage, const void *src, int layout, const CavityDesc *descs,
                                    int count, int max_nz, int wall, double *partials,
                                    double *out, cudaStream_t s)
{
    cudaError_t e = dispatch(1, storage, [&](auto, auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        ensemble_nusselt_kernel<T><<<dim3(max_nz, count), kEnsRedThreads, 0, s>>>(
            static_cast<const T *>(src), descs, layout, wall, max_nz, partials);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ensemble_nusselt_finish<<<count, kEnsRedThreads, 0, s>>>(descs, partials, max_nz, out);
    return cudaGetLastError();
}

}  // namespace lbm

// ====================================================================== host

struct dmrt_ensemble {
    int device = 0;
    int count = 0;
    int storage = DMRT_STORE_F32;
    bool stochastic = false;
    int K = 100;
    std::vector<dmrt_cavity_desc> in;
    std::vector<double> nu, alpha, gbeta;
    std::vector<lbm::CavityDesc> desc;
    lbm::CavityDesc *d_desc = nullptr;
    lbm::BlockTile *d_blockmap = nullptr;
    long long step_blocks = 0;
    size_t blockmap_cap = 0;
    // The step launches of one cell per thread: the members of each, by
    // value (its parameters), and its range of the block map.
    std::vector<lbm::StepTable> tables;
    std::vector<long long> table_first, table_blocks;
    // Two cells per thread: the members grouped by shape, one launch per
    // chunk of a group (geometry of the shape, tile width, member table).
    struct GroupChunk {
        int group;
        lbm::GroupTable table;
    };
    std::vector<lbm::InplaceGeometry> group_geom;
    std::vector<int> group_bx;
    std::vector<GroupChunk> chunks;
    bool grouped = false;  // steps by shape groups (else by the tables)
    // Captured intervals of shape groups run one chain of launches per
    // chunk, concurrently (side streams, fork / join events), each with its
    // own pair of step counters.
    static constexpr int kMaxChains = 8;
    cudaStream_t side[kMaxChains] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kMaxChains] = {};
    unsigned *chain_ctr = nullptr;  // 2 words per chain
    int graph_extra = 0;            // kernels a captured interval adds (counter sync)
    int *d_redmap = nullptr;
    long long red_blocks = 0;
    int threads = 128;
    int max_nz = 0;
    long long total_elems = 0;  // population elements per buffer (all cavities)
    long long total_cells = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    bool inplace = false;  // one buffer, in-place streaming (buf[0])
    bool pairs = false;    // two cells per thread (every member has an even nx)
    int parity = 0;        // in-place: layout of the state (steps mod 2)
    long long device_bytes = 0;
    float *snap = nullptr;
    double *partials = nullptr;
    size_t npartials = 0;
    double *dres = nullptr;  // 2 doubles per member
    double *dnu = nullptr;   // 3 doubles per member
    float *staging = nullptr;
    size_t staging_floats = 0;
    cudaStream_t own = nullptr, stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool use_graphs = true;
    bool use_pdl = true;
    long steps = 0;
    int snaps = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<long> ev_counts;
    long step_launches = 0, total_launches = 0, timed_steps = 0;
    double step_ms = 0.0;
    std::string err;
};

namespace {

constexpr long kEnsMaxGraphSteps = 1000;
// Most launches per step for which shape groups replace the tables.
constexpr size_t kMaxGroupLaunches = dmrt_ensemble::kMaxChains;

dmrt_status efail(dmrt_ensemble_t *e, dmrt_status st, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

dmrt_status efail(dmrt_ensemble_t *e, dmrt_status st, const char *fmt, ...)
{
    if (e) {
        char b[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b, sizeof b, fmt, ap);
        va_end(ap);
        e->err = b;
    }
    return st;
}

dmrt_status ecuda(dmrt_ensemble_t *e, cudaError_t c, const char *what)
{
    return efail(e, c == cudaErrorMemoryAllocation ? DMRT_ERR_OOM : DMRT_ERR_CUDA, "%s: %s (%s)",
                 what, cudaGetErrorName(c), cudaGetErrorString(c));
}

#define ECK(e, call, what)                                   \
    do {                                                     \
        cudaError_t c_ = (call);                             \
        if (c_ != cudaSuccess) return ecuda(e, c_, what);    \
    } while (0)

struct EDeviceGuard {
    int prev = -1;
    explicit EDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~EDeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void fill_rates_desc(lbm::CavityDesc &D, double nu, double alpha, double gbeta)
{
    lbm::fill_collide_params(D.C, nu, alpha, gbeta);
}

// Default tile width in threads: the widest of 128 / 64 / 32 not wider than
// the cavity (rounded up to 32), limited by the block size.  With two cells
// per thread a row holds nx / 2 threads, and tiles of 16 are allowed too.
int default_bx(int nx, int threads, bool pairs)
{
    if (pairs) {
        // as a single cavity's paired kernel: the tile width that launches the
        // fewest idle threads along a row, the widest of equals
        const int units = nx / 2;
        int bx = 16, slots = (units + 15) / 16 * 16;
        for (int cand : {32, 64}) {
            const int c = (units + cand - 1) / cand * cand;
            if (c <= slots && cand <= threads) bx = cand, slots = c;
        }
        return bx;
    }
    const int units = nx;
    const int q = pairs ? 16 : 32;
    const int w = (units + q - 1) / q * q;
    int bx = q;
    for (int cand : {32, 64, 128})
        if (cand > bx && cand <= w && cand <= threads) bx = cand;
    return bx;
}

// Lay out step tiles (and block starts) for the members in `which` with the
// current bx of each; returns the block map (x tiles fastest, then y, then z).
std::vector<lbm::BlockTile> layout_step(dmrt_ensemble_t *e, const std::vector<int> &which)
{
    std::vector<lbm::BlockTile> map;
    for (int c : which) {
        lbm::CavityDesc &D = e->desc[c];
        D.by = e->threads / D.bx;
        const int units = e->pairs ? D.nx / 2 : D.nx;  // threads along a row
        D.tiles_x = (units + D.bx - 1) / D.bx;
        D.tiles_y = (D.ny + D.by - 1) / D.by;
        for (int z = 0; z < D.nz; ++z)
            for (int ty = 0; ty < D.tiles_y; ++ty)
                for (int tx = 0; tx < D.tiles_x; ++tx) map.push_back(lbm::BlockTile{c, tx, ty, z});
    }
    return map;
}

void drop_graphs(dmrt_ensemble_t *e)
{
    for (auto &g : e->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

lbm::MemberRates member_rates(const lbm::CavityDesc &D)
{
    lbm::MemberRates r;
    std::memset(&r, 0, sizeof r);
    r.rs9 = D.C.rs[9];
    r.rs11 = D.C.rs[11];
    r.rs13 = D.C.rs[13];
    r.ws9 = D.C.ws[9];
    r.ws11 = D.C.ws[11];
    r.ws13 = D.C.ws[13];
    r.rq1 = D.C.rq[1];
    r.gbeta = D.C.gbeta;
    r.aniso = D.C.aniso;
    return r;
}

lbm::MemberStep member_step(const lbm::CavityDesc &D)
{
    lbm::MemberStep M;
    std::memset(&M, 0, sizeof M);
    M.nx = D.nx;
    M.ny = D.ny;
    M.nz = D.nz;
    M.wall = D.wall;
    M.plane = D.plane;
    M.nxy = D.nxy;
    M.inv_ny = D.inv_ny;
    M.bx_log2 = 0;
    while ((2 << M.bx_log2) <= D.bx) ++M.bx_log2;  // bx is a power of two
    M.by = D.by;
    M.offset = D.offset;
    M.r = member_rates(D);
    return M;
}

// The step kernels take every rate but the member's from kFixedRates; a
// member whose parameters differ from those (which fill_collide_params rules
// out) is refused rather than stepped with other rates.
bool rates_match_the_fixed_table(const lbm::CollideParams &C)
{
    constexpr lbm::FixedRates F = lbm::fixed_rates();
    for (int k = 0; k < 19; ++k) {
        const int own = k == 9 ? 9 : k == 11 ? 11 : lbm::viscous_moment(k) ? 13 : -1;
        const float rs = own >= 0 ? C.rs[own] : F.rs[k];
        const float ws = own >= 0 ? C.ws[own] : F.ws[k];
        if (rs != C.rs[k] || ws != C.ws[k]) return false;
    }
    for (int k = 0; k < 7; ++k)
        if (((k >= 1 && k <= 3) ? C.rq[1] : F.rq[k]) != C.rq[k]) return false;
    return C.theta_ref == 0.0f && C.aniso == 0;
}

// Split a block map (each member's blocks contiguous) into step launches of
// at most kStepTableMembers members each.
void build_step_tables(dmrt_ensemble_t *e, const std::vector<lbm::BlockTile> &map)
{
    e->tables.clear();
    e->table_first.clear();
    e->table_blocks.clear();
    size_t b = 0;
    while (b < map.size()) {
        e->tables.emplace_back();
        lbm::StepTable &T = e->tables.back();
        std::memset(&T, 0, sizeof T);
        const size_t first = b;
        int count = 0;
        while (b < map.size() && count < lbm::kStepTableMembers) {
            const int c = map[b].member;
            T.first_block[count] = static_cast<int>(b - first);
            T.m[count] = member_step(e->desc[c]);
            ++count;
            while (b < map.size() && map[b].member == c) ++b;
        }
        T.count = count;
        T.first_block[count] = static_cast<int>(b - first);
        e->table_first.push_back(static_cast<long long>(first));
        e->table_blocks.push_back(static_cast<long long>(b - first));
    }
}

// Group the members of a block map (two cells per thread) by shape, in order
// of first appearance, and split each group into launches of at most
// kGroupMembers members (and at most 65535 z blocks).
void build_groups(dmrt_ensemble_t *e, const std::vector<lbm::BlockTile> &map)
{
    e->group_geom.clear();
    e->group_bx.clear();
    e->chunks.clear();
    std::vector<std::vector<int>> lists;
    std::map<std::vector<int>, int> index;
    for (size_t b = 0; b < map.size(); ++b) {
        const int c = map[b].member;
        if (b > 0 && map[b - 1].member == c) continue;
        const lbm::CavityDesc &D = e->desc[c];
        const std::vector<int> key{D.nx, D.ny, D.nz};
        auto it = index.find(key);
        if (it == index.end()) {
            it = index.emplace(key, static_cast<int>(lists.size())).first;
            lists.emplace_back();
        }
        lists[it->second].push_back(c);
    }
    for (size_t g = 0; g < lists.size(); ++g) {
        const lbm::CavityDesc &D = e->desc[lists[g].front()];
        lbm::Geometry G{};
        G.nx = D.nx;
        G.ny = D.ny;
        G.nz = D.nz;
        G.plane = D.plane;
        G.inv_ny = D.inv_ny;
        lbm::InplaceGeometry SI{};
        if (e->inplace) lbm::fill_inplace_geometry(G, SI);
        else lbm::fill_step_geometry(G, SI.load);
        e->group_geom.push_back(SI);
        e->group_bx.push_back(D.bx);
        const size_t per = static_cast<size_t>(std::min(lbm::kGroupMembers, 65535 / D.nz));
        for (size_t i = 0; i < lists[g].size(); i += per) {
            e->chunks.emplace_back();
            auto &ch = e->chunks.back();
            ch.group = static_cast<int>(g);
            std::memset(&ch.table, 0, sizeof ch.table);
            const size_t n = std::min(per, lists[g].size() - i);
            ch.table.count = static_cast<int>(n);
            for (size_t k = 0; k < n; ++k) {
                const lbm::CavityDesc &M = e->desc[lists[g][i + k]];
                ch.table.m[k].offset = M.offset;
                ch.table.m[k].r = member_rates(M);
                ch.table.m[k].wall = M.wall;
            }
        }
    }
}

dmrt_status upload_layout(dmrt_ensemble_t *e, const std::vector<lbm::BlockTile> &map)
{
    // captured graphs hold the previous launches' tables
    drop_graphs(e);
    build_step_tables(e, map);
    // Shape groups where they take few launches: each launch has a ramp and
    // a drain, so an ensemble of many distinct shapes keeps the tables (one
    // launch per 64 members, whatever their shapes).
    e->grouped = false;
    if (e->pairs) {
        build_groups(e, map);
        e->grouped = e->chunks.size() <= kMaxGroupLaunches;
    }
    if (map.size() > e->blockmap_cap) {
        if (e->d_blockmap) cudaFree(e->d_blockmap);
        e->d_blockmap = nullptr;
        e->blockmap_cap = 0;
        ECK(e, cudaMalloc(&e->d_blockmap, map.size() * sizeof(lbm::BlockTile)), "cudaMalloc(blockmap)");
        e->blockmap_cap = map.size();
    }
    ECK(e, cudaMemcpyAsync(e->d_blockmap, map.data(), map.size() * sizeof(lbm::BlockTile),
                           cudaMemcpyHostToDevice, e->stream),
        "copy blockmap");
    ECK(e, cudaMemcpyAsync(e->d_desc, e->desc.data(), e->desc.size() * sizeof(lbm::CavityDesc),
                           cudaMemcpyHostToDevice, e->stream),
        "copy descriptors");
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    e->step_blocks = static_cast<long long>(map.size());
    return DMRT_OK;
}


// The alternating state of the ensemble: the current buffer (A-B) or the
// layout parity (in-place).
int &phase(dmrt_ensemble_t *e) { return e->inplace ? e->parity : e->cur; }

int state_layout(const dmrt_ensemble_t *e)
{
    return !e->inplace ? lbm::kLayoutAB : (e->parity ? lbm::kLayoutStreamed : lbm::kLayoutSwapped);
}

// A residual point of every member's state `from` (the buffer, or the
// in-place layout) and its finishing kernel.
cudaError_t launch_residual_point(dmrt_ensemble_t *e, int from)
{
    const int layout = !e->inplace ? lbm::kLayoutAB : (from ? lbm::kLayoutStreamed : lbm::kLayoutSwapped);
    return lbm::launch_ensemble_residual(e->storage, e->buf[e->inplace ? 0 : from], layout, e->d_desc,
                                         e->d_redmap, e->red_blocks, e->count, e->snap, e->K,
                                         reinterpret_cast<float *>(e->partials), e->dres, e->dres + 5 * e->count,
                                         e->stream);
}

// The step counter that a step from state `b` reads (A-B: the tail of
// buf[b]; in place: word b of the buffer's tail).
unsigned *step_counter(dmrt_ensemble_t *e, int b)
{
    char *base = static_cast<char *>(e->buf[e->inplace ? 0 : b]) +
                 static_cast<size_t>(e->total_elems) * lbm::storage_bytes(e->storage);
    return reinterpret_cast<unsigned *>(base) + (e->inplace ? b : 0);
}

// Chunk i of the shape groups, one step from state `from` on stream s; in a
// chain (concurrent capture) with the chain's own counters.
cudaError_t launch_group_chunk(dmrt_ensemble_t *e, size_t i, int from, cudaStream_t s, bool chain)
{
    const auto &ch = e->chunks[i];
    lbm::GroupCounters K;
    if (chain) {
        K.read = e->chain_ctr + 2 * i + from;
        K.write = e->chain_ctr + 2 * i + (from ^ 1);
        K.tail = step_counter(e, from ^ 1);
    } else {
        K.read = step_counter(e, from);
        K.write = step_counter(e, from ^ 1);
        K.tail = nullptr;
    }
    return lbm::launch_ensemble_group(e->storage, e->stochastic, e->buf[e->inplace ? 0 : from],
                                      e->inplace ? nullptr : e->buf[from ^ 1], e->inplace ? from : -1,
                                      e->group_geom[ch.group], ch.table, e->group_bx[ch.group], K, s, e->use_pdl);
}

// One step of every member from state `from`; with `res` a residual point of
// that state is taken first (the points are the states that the last step
// of every K-step interval starts from, as in a single cavity).
cudaError_t launch_one_step(dmrt_ensemble_t *e, int from, bool res = false)
{
    if (res) {
        const cudaError_t c = launch_residual_point(e, from);
        if (c != cudaSuccess) return c;
    }
    if (e->grouped) {
        for (size_t i = 0; i < e->chunks.size(); ++i) {
            const cudaError_t c = launch_group_chunk(e, i, from, e->stream, false);
            if (c != cudaSuccess) return c;
        }
        return cudaSuccess;
    }
    for (size_t i = 0; i < e->tables.size(); ++i) {
        const lbm::BlockTile *map = e->d_blockmap + e->table_first[i];
        const cudaError_t c =
            e->inplace ? lbm::launch_ensemble_inplace(e->storage, e->stochastic, e->buf[0], from, e->tables[i], map,
                                                      e->table_blocks[i], e->threads, e->total_elems, e->stream,
                                                      e->use_pdl, e->pairs)
                       : lbm::launch_ensemble_step(e->storage, e->stochastic, e->buf[from], e->buf[from ^ 1],
                                                   e->tables[i], map, e->table_blocks[i], e->threads,
                                                   e->total_elems, e->stream, e->use_pdl, e->pairs);
        if (c != cudaSuccess) return c;
    }
    return cudaSuccess;
}

// Side streams, events and chain counters for concurrent chains.
bool ensure_chains(dmrt_ensemble_t *e)
{
    if (!e->chain_ctr) {
        if (cudaMalloc(&e->chain_ctr, 2 * dmrt_ensemble::kMaxChains * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            e->chain_ctr = nullptr;
            return false;
        }
        e->device_bytes += 2 * dmrt_ensemble::kMaxChains * sizeof(unsigned);
    }
    if (!e->fork_ev && cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming) != cudaSuccess) return false;
    for (int i = 0; i < dmrt_ensemble::kMaxChains; ++i) {
        if (!e->side[i] && cudaStreamCreateWithFlags(&e->side[i], cudaStreamNonBlocking) != cudaSuccess) return false;
        if (!e->join_ev[i] && cudaEventCreateWithFlags(&e->join_ev[i], cudaEventDisableTiming) != cudaSuccess)
            return false;
    }
    return true;
}

// A whole interval as concurrent chains: the chunks of the shape groups are
// independent within a step, so chunk i of step s only waits for chunk i of
// step s - 1 (its own stream); the chains meet before the residual point
// (taken before the last step, on the main stream) and at the end.  A chain
// draws the same step numbers as the one-after-another launches.
bool capture_chains(dmrt_ensemble_t *e, int start)
{
    const int n = static_cast<int>(e->chunks.size());
    int cur = start;
    auto fork = [&]() {
        if (cudaEventRecord(e->fork_ev, e->stream) != cudaSuccess) return false;
        for (int i = 0; i < n; ++i)
            if (cudaStreamWaitEvent(e->side[i], e->fork_ev, 0) != cudaSuccess) return false;
        return true;
    };
    auto join = [&]() {
        for (int i = 0; i < n; ++i) {
            if (cudaEventRecord(e->join_ev[i], e->side[i]) != cudaSuccess) return false;
            if (cudaStreamWaitEvent(e->stream, e->join_ev[i], 0) != cudaSuccess) return false;
        }
        return true;
    };
    e->graph_extra = 0;
    if (e->stochastic) {
        if (lbm::launch_counter_sync(step_counter(e, cur), e->chain_ctr, n, cur, e->stream) != cudaSuccess)
            return false;
        e->graph_extra = 1;
    }
    if (!fork()) return false;
    for (long s = 0; s < e->K; ++s) {
        if (s == e->K - 1) {
            if (!join() || launch_residual_point(e, cur) != cudaSuccess || !fork()) return false;
        }
        for (int i = 0; i < n; ++i)
            if (launch_group_chunk(e, static_cast<size_t>(i), cur, e->side[i], true) != cudaSuccess) return false;
        cur ^= 1;
    }
    return join();
}

bool capture_interval(dmrt_ensemble_t *e, int start)
{
    if (e->stream == nullptr) return false;
    const bool chains = e->grouped && e->chunks.size() > 1 && ensure_chains(e);
    if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int cur = start;
    bool ok = true;
    if (chains) {
        ok = capture_chains(e, start);
    } else {
        e->graph_extra = 0;
        for (long s = 0; s < e->K && ok; ++s) {
            ok = launch_one_step(e, cur, s == e->K - 1) == cudaSuccess;
            cur ^= 1;
        }
    }
    cudaGraph_t graph = nullptr;
    ok = (cudaStreamEndCapture(e->stream, &graph) == cudaSuccess) && ok && graph;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        return false;
    }
    e->graph[start] = exec;
    return true;
}

dmrt_status run_steps(dmrt_ensemble_t *e, long n)
{
    long done = 0;
    while (done < n) {
        const long chunk = std::min(n - done, e->K - (e->steps % e->K));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (e->timing) {
            ECK(e, cudaEventCreate(&e0), "cudaEventCreate");
            ECK(e, cudaEventCreate(&e1), "cudaEventCreate");
            ECK(e, cudaEventRecord(e0, e->stream), "cudaEventRecord");
        }
        bool graphed = false;
        int &ph = phase(e);
        if (chunk == e->K && e->K <= kEnsMaxGraphSteps && e->use_graphs) {
            if (!e->graph[ph] && !capture_interval(e, ph)) e->use_graphs = false;
            if (e->graph[ph]) {
                ECK(e, cudaGraphLaunch(e->graph[ph], e->stream), "cudaGraphLaunch");
                if (e->K & 1) ph ^= 1;
                graphed = true;
            }
        }
        bool took = graphed;  // a whole interval ends with a residual point
        for (long s = 0; s < chunk && !graphed; ++s) {
            const bool res = (e->steps + s + 1) % e->K == 0;
            ECK(e, launch_one_step(e, ph, res), "ensemble step");
            took = took || res;
            ph ^= 1;
        }
        e->steps += chunk;
        const long per_step = static_cast<long>(e->grouped ? e->chunks.size() : e->tables.size());  // launches
        e->step_launches += chunk * per_step;
        e->total_launches += chunk * per_step + (took ? 2 : 0) + (graphed ? e->graph_extra : 0);
        if (took && e->snaps < 2) e->snaps++;
        if (e->timing) {
            ECK(e, cudaEventRecord(e1, e->stream), "cudaEventRecord");
            e->ev_pending.emplace_back(e0, e1);
            e->ev_counts.push_back(chunk);
        }
        done += chunk;
    }
    return DMRT_OK;
}

dmrt_status ensure_staging(dmrt_ensemble_t *e, size_t floats)
{
    if (e->staging_floats >= floats) return DMRT_OK;
    if (e->staging) cudaFree(e->staging);
    e->device_bytes -= static_cast<long long>(e->staging_floats * sizeof(float));
    e->staging = nullptr;
    e->staging_floats = 0;
    ECK(e, cudaMalloc(&e->staging, floats * sizeof(float)), "cudaMalloc(staging)");
    e->staging_floats = floats;
    e->device_bytes += static_cast<long long>(floats * sizeof(float));
    return DMRT_OK;
}

lbm::Geometry member_geometry(const dmrt_ensemble_t *e, const lbm::CavityDesc &D)
{
    lbm::Geometry G{};
    G.layout = state_layout(e);
    G.nx = D.nx;
    G.ny = D.ny;
    G.nz = D.nz;
    G.plane = D.plane;
    G.inv_ny = D.inv_ny;
    return G;
}

void *member_ptr(dmrt_ensemble_t *e, int member, int which)
{
    return static_cast<char *>(e->buf[which]) +
           static_cast<size_t>(e->desc[member].offset) * lbm::storage_bytes(e->storage);
}

}  // namespace

extern "C" {

dmrt_status dmrt_ensemble_create(dmrt_ensemble_t **out, int count, const dmrt_cavity_desc *cav,
                                 const dmrt_opts *opts)
{
    if (!out) return DMRT_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !cav) return DMRT_ERR_ARG;
    int storage = DMRT_STORE_F32, K = 100, rounding = DMRT_ROUND_AUTO, streaming = DMRT_STREAM_AB;
    int cpt = 0;
    if (opts) {
        storage = opts->storage;
        rounding = opts->rounding;
        streaming = opts->streaming;
        cpt = opts->cells_per_thread;
        if (opts->residual_interval > 0) K = opts->residual_interval;
        if (opts->residual_interval < 0) return DMRT_ERR_ARG;
        if (cpt < 0 || cpt > 2) return DMRT_ERR_ARG;
        if (opts->pair_loads < 0 || opts->pair_loads > 1) return DMRT_ERR_ARG;
    }
    // two cells per thread where every member's rows have an even length
    bool even = true;
    for (int c = 0; c < count && cav; ++c) even = even && cav[c].grid[0] % 2 == 0;
    if (cpt == 2 && !even) return DMRT_ERR_ARG;
    if (streaming != DMRT_STREAM_AB && streaming != DMRT_STREAM_INPLACE) return DMRT_ERR_ARG;
    if (storage < DMRT_STORE_F32 || storage > DMRT_STORE_F16) return DMRT_ERR_ARG;
    if (rounding < DMRT_ROUND_AUTO || rounding > DMRT_ROUND_STOCHASTIC) return DMRT_ERR_ARG;

    dmrt_ensemble_t *e = new (std::nothrow) dmrt_ensemble();
    if (!e) return DMRT_ERR_OOM;
    auto bail = [&](dmrt_status st) {
        dmrt_ensemble_destroy(e);
        return st;
    };
    if (cudaGetDevice(&e->device) != cudaSuccess) return bail(DMRT_ERR_CUDA);
    e->count = count;
    e->storage = storage;
    e->stochastic = storage != DMRT_STORE_F32 && rounding != DMRT_ROUND_NEAREST;
    e->inplace = streaming == DMRT_STREAM_INPLACE;
    e->pairs = cpt == 2 || (cpt == 0 && even);
    e->K = K;
    e->in.assign(cav, cav + count);
    e->desc.resize(count);
    long long offset = 0, snap_off = 0, red_start = 0;
    std::vector<int> redmap;
    for (int c = 0; c < count; ++c) {
        const dmrt_cavity_desc &d = cav[c];
        const int nx = d.grid[0], ny = d.grid[1], nz = d.grid[2];
        const int minext = 2;
        if (d.wall_type < 1 || d.wall_type > 3 || nx < minext || ny < 2 || nz < minext ||
            nx > 65535 || ny > 65535 || nz > 65535 || !(d.Ra > 0.0) || !(d.Pr > 0.0) ||
            !(d.Ma > 0.0) || !(d.Ma < 0.3) || !std::isfinite(d.Ra) || !std::isfinite(d.Pr))
            return bail(DMRT_ERR_ARG);
        const long long cells = static_cast<long long>(nx) * ny * nz;
        const long long plane = (cells + 63) / 64 * 64;
        if (plane * lbm::kPlanes >= (1LL << 32)) return bail(DMRT_ERR_ARG);
        // Eq. (38), H = ny, dT = 1 (as dmrt_create)
        const double H = ny, uc = d.Ma / std::sqrt(3.0);
        const double gb = uc * uc / H, nu = uc * H * std::sqrt(d.Pr / d.Ra), al = nu / d.Pr;
        e->nu.push_back(nu);
        e->alpha.push_back(al);
        e->gbeta.push_back(gb);
        lbm::CavityDesc &D = e->desc[c];
        D = lbm::CavityDesc{};
        D.nx = nx;
        D.ny = ny;
        D.nz = nz;
        D.wall = d.wall_type;
        D.plane = static_cast<unsigned>(plane);
        D.nxy = static_cast<unsigned>(nx) * ny;
        D.inv_ny = 1.0f / static_cast<float>(ny);
        D.bx = default_bx(nx, e->threads, e->pairs);
        D.offset = offset;
        D.snap_offset = snap_off;
        D.red_tiles_x = (nx + 31) / 32;
        D.red_tiles_y = (ny + 7) / 8;
        D.red_start = red_start;
        const long long nred = static_cast<long long>(D.red_tiles_x) * D.red_tiles_y * nz;
        redmap.insert(redmap.end(), static_cast<size_t>(nred), c);
        red_start += nred;
        fill_rates_desc(D, nu, al, gb);
        if (!rates_match_the_fixed_table(D.C)) return bail(DMRT_ERR_ARG);
        offset += plane * lbm::kPlanes;
        snap_off += 4 * cells;
        e->total_cells += cells;
        e->max_nz = std::max(e->max_nz, nz);
    }
    e->total_elems = offset;
    e->red_blocks = red_start;
    std::vector<int> all(count);
    for (int c = 0; c < count; ++c) all[c] = c;
    const std::vector<lbm::BlockTile> map = layout_step(e, all);

    cudaError_t c;
    const size_t buf_bytes = static_cast<size_t>(offset) * lbm::storage_bytes(storage) + 256;
    const int nbuf = e->inplace ? 1 : 2;
    for (int b = 0; b < nbuf; ++b) {
        c = cudaMalloc(&e->buf[b], buf_bytes);
        if (c != cudaSuccess) return bail(c == cudaErrorMemoryAllocation ? DMRT_ERR_OOM : DMRT_ERR_CUDA);
        e->device_bytes += static_cast<long long>(buf_bytes);
    }
    if (cudaMalloc(&e->snap, static_cast<size_t>(snap_off) * sizeof(float)) != cudaSuccess)
        return bail(DMRT_ERR_OOM);
    e->device_bytes += snap_off * static_cast<long long>(sizeof(float));
    e->npartials = std::max<size_t>(static_cast<size_t>(red_start) * 4,
                                    static_cast<size_t>(count) * e->max_nz * 3);
    if (cudaMalloc(&e->partials, e->npartials * sizeof(double)) != cudaSuccess) return bail(DMRT_ERR_OOM);
    // 2 residual and 3 Nusselt doubles per member, then the count of residual
    // points and the residual finishing kernel's ticket word
    if (cudaMalloc(&e->dres, (static_cast<size_t>(count) * 5 + 2) * sizeof(double)) != cudaSuccess)
        return bail(DMRT_ERR_OOM);
    if (cudaMemset(e->dres, 0, (static_cast<size_t>(count) * 5 + 2) * sizeof(double)) != cudaSuccess)
        return bail(DMRT_ERR_CUDA);
    e->dnu = e->dres + 2 * count;
    if (cudaMalloc(&e->d_desc, static_cast<size_t>(count) * sizeof(lbm::CavityDesc)) != cudaSuccess)
        return bail(DMRT_ERR_OOM);
    if (cudaMalloc(&e->d_redmap, redmap.size() * sizeof(int)) != cudaSuccess) return bail(DMRT_ERR_OOM);
    e->device_bytes += static_cast<long long>(e->npartials * sizeof(double) + (count * 5 + 2) * sizeof(double) +
                                              count * sizeof(lbm::CavityDesc) + redmap.size() * sizeof(int));
    if (cudaStreamCreateWithFlags(&e->own, cudaStreamNonBlocking) != cudaSuccess)
        return bail(DMRT_ERR_CUDA);
    e->stream = e->own;
    if (cudaMemcpyAsync(e->d_redmap, redmap.data(), redmap.size() * sizeof(int),
                        cudaMemcpyHostToDevice, e->stream) != cudaSuccess)
        return bail(DMRT_ERR_CUDA);
    if (upload_layout(e, map) != DMRT_OK) return bail(DMRT_ERR_CUDA);
    for (int b = 0; b < nbuf; ++b)
        if (cudaMemsetAsync(e->buf[b], 0, buf_bytes, e->stream) != cudaSuccess) return bail(DMRT_ERR_CUDA);
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return bail(DMRT_ERR_CUDA);
    *out = e;
    return DMRT_OK;
}

void dmrt_ensemble_destroy(dmrt_ensemble_t *e)
{
    if (!e) return;
    EDeviceGuard dg(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    for (auto &p : e->ev_pending) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    drop_graphs(e);
    for (int b = 0; b < 2; ++b)
        if (e->buf[b]) cudaFree(e->buf[b]);
    if (e->snap) cudaFree(e->snap);
    if (e->partials) cudaFree(e->partials);
    if (e->dres) cudaFree(e->dres);
    if (e->d_desc) cudaFree(e->d_desc);
    if (e->d_blockmap) cudaFree(e->d_blockmap);
    if (e->d_redmap) cudaFree(e->d_redmap);
    if (e->staging) cudaFree(e->staging);
    if (e->own) cudaStreamDestroy(e->own);
    for (int i = 0; i < dmrt_ensemble::kMaxChains; ++i) {
        if (e->side[i]) cudaStreamDestroy(e->side[i]);
        if (e->join_ev[i]) cudaEventDestroy(e->join_ev[i]);
    }
    if (e->fork_ev) cudaEventDestroy(e->fork_ev);
    if (e->chain_ctr) cudaFree(e->chain_ctr);
    delete e;
}

dmrt_status dmrt_ensemble_set_stream(dmrt_ensemble_t *e, void *stream)
{
    if (!e) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    e->stream = stream ? static_cast<cudaStream_t>(stream) : e->own;
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_sync(dmrt_ensemble_t *e)
{
    if (!e) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_set_timing(dmrt_ensemble_t *e, int enabled)
{
    if (!e) return DMRT_ERR_ARG;
    e->timing = enabled != 0;
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_get_stats(dmrt_ensemble_t *e, dmrt_stats *out, int reset)
{
    if (!e || !out) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    for (size_t k = 0; k < e->ev_pending.size(); ++k) {
        auto &p = e->ev_pending[k];
        ECK(e, cudaEventSynchronize(p.second), "cudaEventSynchronize");
        float ms = 0.f;
        ECK(e, cudaEventElapsedTime(&ms, p.first, p.second), "cudaEventElapsedTime");
        e->step_ms += ms;
        e->timed_steps += e->ev_counts[k];
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    e->ev_pending.clear();
    e->ev_counts.clear();
    out->step_launches = e->step_launches;
    out->total_launches = e->total_launches;
    out->step_ms = e->step_ms;
    out->timed_steps = e->timed_steps;
    out->bytes_per_cell = 2.0 * lbm::kPlanes * lbm::storage_bytes(e->storage);
    if (reset) {
        e->step_launches = e->total_launches = e->timed_steps = 0;
        e->step_ms = 0.0;
    }
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_autotune(dmrt_ensemble_t *e, int trials, char *report, int report_len)
{
    if (!e || trials < 1) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    drop_graphs(e);
    // In-place ensembles are timed on a scratch copy of their buffer (each
    // launch rewrites its input); two-buffer ones on the live buffers, where
    // every launch recomputes the same next state from buf[cur].
    void *live = e->buf[0];
    void *scratch = nullptr;
    if (e->inplace) {
        const size_t bytes = static_cast<size_t>(e->total_elems) * lbm::storage_bytes(e->storage) + 256;
        cudaError_t c = cudaMalloc(&scratch, bytes);
        if (c != cudaSuccess) {
            cudaGetLastError();
            return efail(e, DMRT_ERR_OOM, "autotune of an in-place ensemble needs a scratch copy "
                                          "of %zu bytes", bytes);
        }
        c = cudaMemcpyAsync(scratch, live, bytes, cudaMemcpyDeviceToDevice, e->stream);
        if (c != cudaSuccess) {
            cudaFree(scratch);
            return ecuda(e, c, "copy to scratch");
        }
        e->buf[0] = scratch;
    }
    struct Restore {
        dmrt_ensemble_t *e;
        void *live, *scratch;
        ~Restore()
        {
            if (!scratch) return;
            cudaStreamSynchronize(e->stream);
            e->buf[0] = live;
            cudaFree(scratch);
        }
    } restore{e, live, scratch};
    cudaEvent_t t0, t1;
    ECK(e, cudaEventCreate(&t0), "cudaEventCreate");
    ECK(e, cudaEventCreate(&t1), "cudaEventCreate");
    int ph = phase(e);
    auto one = [&]() {
        const cudaError_t c = launch_one_step(e, ph);
        if (e->inplace) ph ^= 1;  // the scratch state advances
        return c;
    };
    // time `trials` launches of the current layout of `which`
    auto time_layout = [&](const std::vector<int> &which, float *ms) -> dmrt_status {
        dmrt_status st = upload_layout(e, layout_step(e, which));
        if (st != DMRT_OK) return st;
        ECK(e, one(), "autotune warm-up");
        ECK(e, cudaEventRecord(t0, e->stream), "cudaEventRecord");
        for (int t = 0; t < trials; ++t) ECK(e, one(), "autotune launch");
        ECK(e, cudaEventRecord(t1, e->stream), "cudaEventRecord");
        ECK(e, cudaEventSynchronize(t1), "cudaEventSynchronize");
        ECK(e, cudaEventElapsedTime(ms, t0, t1), "cudaEventElapsedTime");
        *ms /= trials;
        return DMRT_OK;
    };
    std::map<int, std::vector<int>> groups;  // nx -> members
    for (int c = 0; c < e->count; ++c) groups[e->desc[c].nx].push_back(c);
    std::vector<int> all(e->count);
    for (int c = 0; c < e->count; ++c) all[c] = c;
    int best_threads = e->threads;
    float best_total = INFINITY;
    std::vector<int> best_bx(e->count);
    std::string rep, cand_rep;
    for (int threads : {128, 256}) {
        if (DMRT_ENS_INPLACE_BLOCK128 && e->inplace && threads != 128) continue;
        if (e->pairs && threads != 128) continue;  // the paired kernels are built for 128
        e->threads = threads;
        for (auto &g : groups) {
            int best = -1;
            float best_ms = INFINITY;
            const int units = e->pairs ? g.first / 2 : g.first;  // threads along a row
            for (int bx : {16, 32, 64, 128}) {
                if (bx == 16 && !e->pairs) continue;
                if (bx > threads || bx > (units + 15) / 16 * 16 + 32) continue;
                for (int c : g.second) e->desc[c].bx = bx;
                float ms = 0.f;
                dmrt_status st = time_layout(g.second, &ms);
                if (st != DMRT_OK) return st;
                char c_line[64];
                snprintf(c_line, sizeof c_line, " nx%d/t%d/bx%d:%.1fus", g.first, threads, bx, ms * 1e3f);
                cand_rep += c_line;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = bx;
                }
            }
            for (int c : g.second) e->desc[c].bx = best;
        }
        float total = 0.f;
        dmrt_status st = time_layout(all, &total);
        if (st != DMRT_OK) return st;
        char line[160];
        snprintf(line, sizeof line, "threads=%d:%.1fus[", threads, total * 1e3f);
        rep += line;
        for (auto &g : groups) {
            snprintf(line, sizeof line, " nx%d:bx%d", g.first, e->desc[g.second[0]].bx);
            rep += line;
        }
        rep += " ] ";
        if (total < best_total) {
            best_total = total;
            best_threads = threads;
            for (int c = 0; c < e->count; ++c) best_bx[c] = e->desc[c].bx;
        }
    }
    e->threads = best_threads;
    for (int c = 0; c < e->count; ++c) e->desc[c].bx = best_bx[c];
    dmrt_status st = upload_layout(e, layout_step(e, all));
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != DMRT_OK) return st;
    char line[64];
    snprintf(line, sizeof line, "chosen threads=%d;", best_threads);
    rep += line + cand_rep;
    if (report && report_len > 0) snprintf(report, static_cast<size_t>(report_len), "%s", rep.c_str());
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_step(dmrt_ensemble_t *e, long n)
{
    if (!e) return DMRT_ERR_ARG;
    if (n < 0) return efail(e, DMRT_ERR_ARG, "dmrt_ensemble_step: n = %ld < 0", n);
    EDeviceGuard dg(e->device);
    return run_steps(e, n);
}

dmrt_status dmrt_ensemble_residual(dmrt_ensemble_t *e, double *r)
{
    if (!e || !r) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    if (e->snaps < 2) {
        for (int c = 0; c < e->count; ++c) r[c] = INFINITY;
        return DMRT_OK;
    }
    std::vector<double> res(static_cast<size_t>(e->count) * 2);
    ECK(e, cudaMemcpyAsync(res.data(), e->dres, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           e->stream),
        "copy residuals");
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    dmrt_status st = DMRT_OK;
    for (int c = 0; c < e->count; ++c) {
        r[c] = res[2 * c];
        if (res[2 * c + 1] != 0.0 && st == DMRT_OK)
            st = efail(e, DMRT_ERR_DIVERGED, "member %d holds non-finite fields at step %ld", c,
                       e->steps);
    }
    return st;
}

dmrt_status dmrt_ensemble_run_to_steady(dmrt_ensemble_t *e, double tol, long max_steps,
                                        long *steps_taken, int *converged)
{
    if (!e || !(tol > 0.0) || max_steps < 0) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    std::vector<double> r(static_cast<size_t>(e->count), INFINITY);
    long taken = 0;
    int conv = 0;
    dmrt_status st = DMRT_OK;
    while (true) {
        if (e->snaps >= 2) {
            st = dmrt_ensemble_residual(e, r.data());
            conv = 0;
            for (double v : r) conv += (v < tol);
            if (st != DMRT_OK || conv == e->count) break;
        }
        if (taken >= max_steps) {
            st = efail(e, DMRT_ERR_TIMEOUT, "%d of %d members below %g after %ld steps", conv,
                       e->count, tol, taken);
            break;
        }
        long chunk = e->K - (e->steps % e->K);
        if (chunk > max_steps - taken) chunk = max_steps - taken;
        st = run_steps(e, chunk);
        if (st != DMRT_OK) break;
        taken += chunk;
    }
    if (steps_taken) *steps_taken = taken;
    if (converged) *converged = conv;
    return st;
}

dmrt_status dmrt_ensemble_nusselt(dmrt_ensemble_t *e, int wall, double *out)
{
    if (!e || !out || (wall != 0 && wall != 1)) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    ECK(e,
        lbm::launch_ensemble_nusselt(e->storage, e->buf[e->cur], state_layout(e), e->d_desc, e->count, e->max_nz,
                                     wall, e->partials, e->dnu, e->stream),
        "ensemble nusselt");
    e->total_launches += 2;
    ECK(e, cudaMemcpyAsync(out, e->dnu, static_cast<size_t>(e->count) * 3 * sizeof(double),
                           cudaMemcpyDeviceToHost, e->stream),
        "copy nusselt");
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_fields(dmrt_ensemble_t *e, int member, float *rho, float *u,
                                 float *theta, int on_device)
{
    if (!e || member < 0 || member >= e->count) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    const lbm::CavityDesc &D = e->desc[member];
    const lbm::Geometry G = member_geometry(e, D);
    const size_t cells = static_cast<size_t>(D.nx) * D.ny * D.nz;
    float *dr = rho, *du = u, *dt = theta;
    if (!on_device) {
        dmrt_status st = ensure_staging(e, 5 * cells);
        if (st != DMRT_OK) return st;
        dr = rho ? e->staging : nullptr;
        du = u ? e->staging + cells : nullptr;
        dt = theta ? e->staging + 4 * cells : nullptr;
    }
    ECK(e, lbm::launch_fields(D.wall, e->storage, member_ptr(e, member, e->cur), G, dr, du, dt, e->stream),
        "fields kernel");
    e->total_launches++;
    if (!on_device) {
        if (rho) ECK(e, cudaMemcpyAsync(rho, dr, cells * 4, cudaMemcpyDeviceToHost, e->stream), "copy rho");
        if (u) ECK(e, cudaMemcpyAsync(u, du, 3 * cells * 4, cudaMemcpyDeviceToHost, e->stream), "copy u");
        if (theta)
            ECK(e, cudaMemcpyAsync(theta, dt, cells * 4, cudaMemcpyDeviceToHost, e->stream), "copy theta");
    }
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_init_fields(dmrt_ensemble_t *e, int member, const float *rho,
                                      const float *u, const float *theta, int on_device)
{
    if (!e || member < 0 || member >= e->count || !rho || !u || !theta) return DMRT_ERR_ARG;
    EDeviceGuard dg(e->device);
    const lbm::CavityDesc &D = e->desc[member];
    const lbm::Geometry G = member_geometry(e, D);
    const size_t cells = static_cast<size_t>(D.nx) * D.ny * D.nz;
    const float *dr = rho, *du = u, *dt = theta;
    if (!on_device) {
        dmrt_status st = ensure_staging(e, 5 * cells);
        if (st != DMRT_OK) return st;
        ECK(e, cudaMemcpyAsync(e->staging, rho, cells * 4, cudaMemcpyHostToDevice, e->stream), "copy rho");
        ECK(e, cudaMemcpyAsync(e->staging + cells, u, 3 * cells * 4, cudaMemcpyHostToDevice, e->stream),
            "copy u");
        ECK(e, cudaMemcpyAsync(e->staging + 4 * cells, theta, cells * 4, cudaMemcpyHostToDevice, e->stream),
            "copy theta");
        dr = e->staging;
        du = e->staging + cells;
        dt = e->staging + 4 * cells;
    }
    ECK(e, lbm::launch_init_fields(e->storage, dr, du, dt, member_ptr(e, member, e->cur), G, false, e->stream),
        "init kernel");
    e->total_launches++;
    e->snaps = 0;
    ECK(e, cudaMemsetAsync(e->dres + 5 * e->count, 0, sizeof(double), e->stream), "reset residual points");
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_get_populations(dmrt_ensemble_t *e, int member, float *f, float *g,
                                          int on_device)
{
    if (!e || member < 0 || member >= e->count) return DMRT_ERR_ARG;
    if (!f && !g) return DMRT_OK;
    EDeviceGuard dg(e->device);
    const lbm::CavityDesc &D = e->desc[member];
    const lbm::Geometry G = member_geometry(e, D);
    const size_t cells = static_cast<size_t>(D.nx) * D.ny * D.nz;
    float *df = f, *dgp = g;
    if (!on_device) {
        dmrt_status st = ensure_staging(e, 26 * cells);
        if (st != DMRT_OK) return st;
        df = f ? e->staging : nullptr;
        dgp = g ? e->staging + 19 * cells : nullptr;
    }
    ECK(e, lbm::launch_get_populations(e->storage, member_ptr(e, member, e->cur), df, dgp, G, false, e->stream),
        "get kernel");
    e->total_launches++;
    if (!on_device) {
        if (f) ECK(e, cudaMemcpyAsync(f, df, 19 * cells * 4, cudaMemcpyDeviceToHost, e->stream), "copy f");
        if (g) ECK(e, cudaMemcpyAsync(g, dgp, 7 * cells * 4, cudaMemcpyDeviceToHost, e->stream), "copy g");
    }
    ECK(e, cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_ensemble_member_params(const dmrt_ensemble_t *e, int member, dmrt_params *out)
{
    if (!e || !out || member < 0 || member >= e->count) return DMRT_ERR_ARG;
    const lbm::CavityDesc &D = e->desc[member];
    out->nx = D.nx;
    out->ny = D.ny;
    out->nz = D.nz;
    out->wall_type = D.wall;
    out->storage = e->storage;
    out->residual_interval = e->K;
    out->rounding = e->stochastic ? DMRT_ROUND_STOCHASTIC : DMRT_ROUND_NEAREST;
    out->nu = e->nu[member];
    out->alpha = e->alpha[member];
    out->gbeta = e->gbeta[member];
    out->tau_nu = 3.0 * e->nu[member] + 0.5;
    out->tau_alpha = 0.5 + 4.0 * e->alpha[member];
    out->steps = e->steps;
    out->streaming = e->inplace ? DMRT_STREAM_INPLACE : DMRT_STREAM_AB;
    out->cells_per_thread = e->pairs ? 2 : 1;
    out->pair_loads = e->pairs && !e->inplace ? 1 : 0;
    out->device_bytes = e->device_bytes;
    return DMRT_OK;
}

const char *dmrt_ensemble_last_error(const dmrt_ensemble_t *e)
{
    if (!e) return "null ensemble";
    return e->err.c_str();
}

}  // extern "C"
