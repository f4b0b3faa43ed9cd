// internal.h -- launchers shared by the library's translation units (not part
// of the public ABI; the public calls are declared in include/dmrt.h).
#pragma once

#include <cuda_runtime.h>

#include "lattice.cuh"
#include "residual.cuh"

namespace lbm {

// Storage codes follow dmrt_storage: 0 = float, 1 = bf16, 2 = f16.

// Planes in one population buffer: 19 D3Q19 deviations, then 7 D3Q7.
constexpr int kPlanes = 26;

// Default thread-block shape of the per-cell kernels (x fastest).
struct BlockShape {
    int bx, by;
};

// Offset tables of the step kernel for a geometry (see StepGeometry).
void fill_step_geometry(const Geometry &G, StepGeometry &S);

// One fused time step: pull from `src`, collide, force, store into `dst`.
// stochastic: 16-bit stores round stochastically (ignored for FP32).
// pdl: launch with programmatic stream serialisation (the kernel waits for
// the previous grid itself).  Each buffer holds kPlanes * plane elements and
// then one 32-bit step counter (used by stochastic rounding).  res: when not
// null, the step also takes a residual point of the state it pulls (one
// partial per block of the launch's grid; residual.cuh), to be finished by
// launch_residual_finish.
cudaError_t launch_step(int wall, int storage, bool stochastic, const void *src, void *dst,
                        const StepGeometry &S, const Geometry &G, const CollideParams &C,
                        BlockShape b, cudaStream_t s, bool pdl, const ResidualArgs *res = nullptr);

// The same step with two neighbouring cells of a row per thread (x0 even):
// bitwise the values of launch_step, in packed FP32x2 arithmetic.  Needs a
// walled box (wall 1..3) and an even nx (step_pair_supported); the launcher
// picks its own block shape.
bool step_pair_supported(int wall, const Geometry &G);
cudaError_t launch_step_pair(int wall, int storage, bool stochastic, const void *src, void *dst,
                             const StepGeometry &S, const Geometry &G, const CollideParams &C,
                             cudaStream_t s, bool pdl, const ResidualArgs *res = nullptr);
// Blocks of the paired kernels' grid (the residual partials they write).
size_t pair_blocks(const Geometry &G);

// In-place streaming (one buffer).  The state alternates between two
// layouts (see kLayoutSwapped / kLayoutStreamed): phase 0 reads the swapped
// layout and leaves the streamed one, phase 1 the reverse.  Both phases do
// the arithmetic of launch_step on the same populations, so the state after
// any number of steps holds the same values as the two-buffer scheme's.  The
// buffer's tail holds two 32-bit step counters: phase p reads word p and
// writes word p ^ 1.
void fill_inplace_geometry(const Geometry &G, InplaceGeometry &SI);
cudaError_t launch_step_inplace(int wall, int storage, bool stochastic, void *buf, int phase,
                                const InplaceGeometry &SI, const Geometry &G,
                                const CollideParams &C, BlockShape b, cudaStream_t s, bool pdl,
                                const ResidualArgs *res = nullptr);
// The two-buffer paired step with its loads staged by TMA into shared memory
// (16-bit storage, walled box, nx a multiple of 8): bitwise the values of
// launch_step_pair.  `map` holds the two tensor maps of `src` (the row boxes
// and the x-face edge boxes; two CUtensorMap, 128 bytes each, 64-byte
// aligned) made by encode_pair_tma_maps; a copy wait that runs out sets *err
// (device memory) and the kernel returns early.
bool step_pair_tma_supported(int wall, int storage, const Geometry &G);
cudaError_t encode_pair_tma_maps(const void *buf, const Geometry &G, void *maps);
// Once per device and kernel variant, outside stream capture: allow the
// staged kernel its shared memory (about 49 KB per block).
cudaError_t prepare_step_pair_tma(int wall, int storage);
cudaError_t launch_step_pair_tma(int wall, int storage, bool stochastic, const void *map, const void *src,
                                 void *dst, const StepGeometry &S, const Geometry &G, const CollideParams &C,
                                 unsigned *err, cudaStream_t s, bool pdl);

// Both in-place phases with two cells per thread (same conditions as
// launch_step_pair); bitwise the values of launch_step_inplace.
cudaError_t launch_step_inplace_pair(int wall, int storage, bool stochastic, void *buf, int phase,
                                     const InplaceGeometry &SI, const Geometry &G,
                                     const CollideParams &C, cudaStream_t s, bool pdl,
                                     const ResidualArgs *res = nullptr);

// Fields of the pulled populations (any output may be null).
cudaError_t launch_fields(int wall, int storage, const void *src, const Geometry &G, float *rho,
                          float *u, float *theta, cudaStream_t s);

// The end of a residual point taken by a step kernel: adds its `nparts`
// block partials (8 floats each) and writes `result` (8 doubles): [0..3] =
// sums |dtheta|^2, |theta|^2, |du|^2, |u|^2; [4] = r; [5] = nonfinite;
// [6] = points taken since the last reset (read, then raised, capped at 2;
// the step kernels read it through ResidualArgs::points).  `stage` needs
// residual_stage_floats(nparts) floats; *ticket (device) must be 0 and is
// left at 0.
size_t residual_stage_floats(long long nparts);
cudaError_t launch_residual_finish(const float *partials, long long nparts, float *stage, unsigned *ticket,
                                  int K, double *result, cudaStream_t s);

// Nusselt numbers of wall 0 (hot) / 1 (cold): `partials` needs 3 * nz doubles,
// `out3` 3 doubles; `local` (nullable) receives the [z][x] map.
cudaError_t launch_nusselt(int wall_type, int storage, const void *src, const Geometry &G,
                           int wall, float *local, double *partials, double *out3,
                           cudaStream_t s);

// Link-flux Nusselt numbers of wall 0 / 1 from the stored populations.
cudaError_t launch_nusselt_flux(int storage, const void *src, const Geometry &G, int wall, double alpha,
                                float *local, double *partials, double *out3, cudaStream_t s);

// Population and field import / export (dense [q][cells] arrays) in the
// layout G.layout; `periodic`: the box has no walls.
cudaError_t launch_set_populations(int storage, const float *f, const float *g, void *dst,
                                   const Geometry &G, bool periodic, cudaStream_t s);
cudaError_t launch_get_populations(int storage, const void *src, float *f, float *g,
                                   const Geometry &G, bool periodic, cudaStream_t s);
cudaError_t launch_init_fields(int storage, const float *rho, const float *u, const float *theta,
                               void *dst, const Geometry &G, bool periodic, cudaStream_t s);

// Round a flat float array to the storage format and back (the step
// kernel's store rounding; stochastic bits from pcg_hash(i ^ pcg_hash(seed))).
cudaError_t launch_round(int storage, bool stochastic, const float *in, float *out, long long n,
                         unsigned seed, cudaStream_t s);

}  // namespace lbm
