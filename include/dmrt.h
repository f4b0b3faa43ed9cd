/*
 * dmrt.h -- C ABI of the GB300 double-MRT thermal lattice Boltzmann library.
 *
 * Method: "LBM Simulation of 3-D Natural Convection with Double MRT Model"
 * (arXiv:1511.04633).  Flow: D3Q19 MRT (Sec. 3.1, Eqs. (11)-(26)); energy:
 * D3Q7 MRT (Sec. 3.2, Eqs. (27)-(37)); coupling: Boussinesq buoyancy force
 * (Eqs. (15)-(17)); problem: a box of nx*ny*nz cells with the hot wall at
 * y = 0 and the cold wall at y = H = ny (Sec. 2, Eqs. (6)-(10)); lattice
 * units and Nusselt numbers: Sec. 4, Eqs. (38)-(41).
 *
 * Conventions shared by every call:
 *  - Temperatures are theta = (T - T_c)/(T_h - T_c) - 1/2, so the hot wall is
 *    +1/2 and the cold wall -1/2.  Velocities are lattice units (c = 1).
 *  - Field arrays are float32 in [z][y][x] order, x fastest; the velocity is
 *    three such planes [3][z][y][x] (u_x, u_y, u_z).  Population arrays are
 *    [q][z][y][x] with q in the velocity order of Eq. (12) (D3Q19) or
 *    Eq. (28) (D3Q7).
 *  - `on_device` = 1: the pointer is CUDA device memory (e.g. a torch
 *    tensor's data_ptr) on the handle's device; 0: host memory.  The caller
 *    owns every array it passes; the library copies and never keeps it.
 *  - Every call returns a dmrt_status; none throws or aborts.  After an error
 *    dmrt_last_error() describes it.  Work is queued on the handle's stream;
 *    calls that return data to the host synchronise that stream.
 *  - The handle owns all device memory it allocates; dmrt_destroy frees it.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef DMRT_H
#define DMRT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrt dmrt_t;

typedef enum {
    DMRT_OK = 0,
    DMRT_ERR_ARG = 1,      /* invalid argument; nothing was changed */
    DMRT_ERR_CUDA = 2,     /* a CUDA call failed; see dmrt_last_error */
    DMRT_ERR_OOM = 3,      /* device allocation failed */
    DMRT_ERR_DIVERGED = 4, /* a NaN/Inf was found in the fields */
    DMRT_ERR_TIMEOUT = 5,  /* a step budget ran out before convergence */
} dmrt_status;

/* Wall types (Sec. 2).  All walls are no-slip (Eq. (8)); y = 0 is hot and
 * y = H cold (Eqs. (6),(7)).
 *  TYPE1: the x and z walls adiabatic.
 *  TYPE2: the x and z walls carry the linear profile of Eq. (9).
 *  TYPE3: the x walls linear, the z walls adiabatic (Eq. (10)).
 *  PERIODIC: no walls at all (a test configuration for conservation laws). */
typedef enum {
    DMRT_WALL_PERIODIC = 0,
    DMRT_WALL_TYPE1 = 1,
    DMRT_WALL_TYPE2 = 2,
    DMRT_WALL_TYPE3 = 3,
} dmrt_wall;

/* Population storage format in HBM.  Every format stores the deviations
 * f_i - w_i from the rest equilibrium (rho = 1, u = 0) and the g_i; the
 * collision always runs in FP32.
 *  F32 : float32, 208 bytes moved per cell update.
 *  BF16: bfloat16 rounded to nearest, 104 bytes per cell update.
 *  F16 : IEEE half of the values times 2^10, rounded to nearest, 104 bytes. */
typedef enum {
    DMRT_STORE_F32 = 0,
    DMRT_STORE_BF16 = 1,
    DMRT_STORE_F16 = 2,
} dmrt_storage;

/* Rounding of the 16-bit stores (no effect on F32).  A 16-bit store drops
 * any per-step change below half an ulp, so with round-to-nearest a slowly
 * evolving solution stagnates; stochastic rounding keeps the expected stored
 * value equal to the FP32 value (random bits: a PCG hash of the cell index and
 * the step number).  AUTO = STOCHASTIC for BF16 and F16. */
typedef enum {
    DMRT_ROUND_AUTO = 0,
    DMRT_ROUND_NEAREST = 1,
    DMRT_ROUND_STOCHASTIC = 2,
} dmrt_rounding;

/* How the populations stream (the method is the same; only the memory
 * scheme differs).
 *  AB     : two population buffers; each step pulls from one and writes the
 *           other (2 x 26 values per cell held on the device).
 *  INPLACE: one buffer updated in place by two alternating kernels (the AA
 *           access pattern): half the population memory, the same HBM
 *           traffic per step, and bitwise the same results as AB in every
 *           call of this API (single cavities and ensembles). */
typedef enum {
    DMRT_STREAM_AB = 0,
    DMRT_STREAM_INPLACE = 1,
} dmrt_streaming;

/* Optional creation settings; pass NULL for the defaults (zero-initialised
 * fields select the defaults). */
typedef struct dmrt_opts {
    int storage;           /* dmrt_storage; default DMRT_STORE_F32 */
    int residual_interval; /* K of the convergence residual; 0 = 100 */
    int rounding;          /* dmrt_rounding; default DMRT_ROUND_AUTO */
    int streaming;         /* dmrt_streaming; default DMRT_STREAM_AB */
    int cells_per_thread;  /* cells one thread of the step kernel updates:
                            * 0 = auto, 1, or 2 (two neighbouring cells of a
                            * row, collided together in packed FP32x2
                            * arithmetic; needs a walled box and an even nx,
                            * else DMRT_ERR_ARG).  Either streaming scheme.
                            * The stored values are bitwise the same either
                            * way.  Auto takes 2 where allowed; for an
                            * ensemble, where every member's nx is even. */
    int pair_loads;        /* how the two-cell kernel of two-buffer 16-bit
                            * storage loads: 0 = auto (direct), 1 = direct
                            * loads, 2 = staged: TMA copies of each plane's
                            * source rows into shared memory, two slabs ahead
                            * (nx a multiple of 8, else DMRT_ERR_ARG).  Same
                            * values either way. */
} dmrt_opts;

/* Derived lattice parameters of a handle (read-only view). */
typedef struct dmrt_params {
    int nx, ny, nz, wall_type, storage, residual_interval, rounding;
    double nu, alpha, gbeta;   /* lattice viscosity, diffusivity, g*beta*dT */
    double tau_nu, tau_alpha;  /* 3 nu + 1/2 (Eq. (26)); 1/2 + 4 alpha (Eq. (36)) */
    long steps;                /* time steps taken since creation / last reset */
    int streaming;             /* dmrt_streaming */
    long long device_bytes;    /* device memory the handle holds now */
    int cells_per_thread;      /* 1 or 2: the step kernel in use */
    int pair_loads;            /* 1 = direct, 2 = staged (0 for one cell) */
} dmrt_params;

/* Counters for profiling and for the benchmark's launch count. */
typedef struct dmrt_stats {
    long step_launches;    /* fused step kernels launched */
    long total_launches;   /* every kernel this handle launched */
    double step_ms;        /* summed CUDA-event time of timed step-kernel runs */
    long timed_steps;      /* step kernels inside those timed runs */
    double bytes_per_cell; /* algorithmic HBM bytes per cell update */
} dmrt_stats;

/* Create a cavity of grid[0]*grid[1]*grid[2] = nx*ny*nz cells from the
 * physical numbers of Sec. 4: Rayleigh Ra > 0, Prandtl Pr > 0 and Mach
 * 0 < Ma < 0.3.  Lattice parameters follow Eq. (38) with H = ny, dT = 1:
 * u_c = Ma/sqrt(3), nu = u_c H sqrt(Pr/Ra), alpha = nu/Pr, g*beta = u_c^2/H.
 * The fluid starts at rest: rho = 1, u = 0, theta = 0 (populations at the
 * equilibrium of Eq. (17), energy populations zero).  Runs on the current
 * CUDA device.  Every grid dimension must be >= 2 (>= 1 for PERIODIC) and
 * at most 65535, and nx*ny*nz <= 165,191,040 (the 26 population planes are
 * addressed with 32-bit indices; e.g. up to 548^3).  On error *out is NULL. */
dmrt_status dmrt_create(dmrt_t **out, const int grid[3], double Ra, double Pr, double Ma,
                        int wall_type);

/* dmrt_create with settings (opts may be NULL). */
dmrt_status dmrt_create_ex(dmrt_t **out, const int grid[3], double Ra, double Pr, double Ma,
                           int wall_type, const dmrt_opts *opts);

/* Create from lattice parameters directly: viscosity nu > 0, diffusivity
 * alpha > 0 and buoyancy g*beta*dT (any finite value; 0 decouples the flow
 * from the temperature).  Same start state as dmrt_create. */
dmrt_status dmrt_create_lattice(dmrt_t **out, const int grid[3], double nu, double alpha,
                                double gbeta, int wall_type, const dmrt_opts *opts);

/* Free every resource of the handle (NULL is a no-op).  Synchronises. */
void dmrt_destroy(dmrt_t *h);

/* Use this CUDA stream (a cudaStream_t; NULL = the handle's own stream) for
 * all later work.  The caller keeps the stream alive while it is set. */
dmrt_status dmrt_set_stream(dmrt_t *h, void *stream);

/* Advance n >= 0 time steps (Eqs. (14), (19), (29)): each step is one fused
 * kernel that, for every cell, pulls the D3Q19 and D3Q7 populations from its
 * neighbours (bounce-back / anti-bounce-back at walls), collides them in
 * moment space, adds the buoyancy force and stores them.  The last step of
 * every K-step interval (K = residual_interval; the steps from the states
 * K - 1, 2K - 1, ... counted from creation) also takes a residual point: it
 * compares the fields of the state it pulls with the snapshot of the
 * previous point and reduces the sums of dmrt_residual, in the same pass
 * (a small kernel then adds the block sums).  Asynchronous: returns once the
 * work is queued. */
dmrt_status dmrt_step(dmrt_t *h, long n);

/* Wait for the handle's queued work; reports deferred CUDA errors. */
dmrt_status dmrt_sync(dmrt_t *h);

/* Fields at the current step: the moments of the pulled (pre-collision)
 * populations, Eqs. (20),(30): rho, u = j/rho ([3][z][y][x]) and theta.
 * Any pointer may be NULL to skip that field.  Synchronises. */
dmrt_status dmrt_fields(dmrt_t *h, float *rho, float *u, float *theta, int on_device);

/* Nusselt numbers on wall 0 (hot, y = 0) or 1 (cold, y = H), Eqs. (39)-(41):
 * out[0] = Nu_3D (mean over the wall), out[1] = Nu_2D (mean over z at
 * X = 1/2: the two centre x columns for even nx, the centre one for odd nx),
 * out[2] = Nu_max.  The local Nu uses the second-order one-sided difference
 * (-8 theta_w + 9 theta_1 - theta_2)/3 with cells 1/2 and 3/2 from the wall;
 * sums are accumulated in FP64 in a fixed order.  `out` is host memory.
 * Requires ny >= 2.  Synchronises. */
dmrt_status dmrt_nusselt(dmrt_t *h, int wall, double out[3]);

/* Conservative cross-check of dmrt_nusselt (same three outputs): the heat
 * carried across the wall links in the coming step by the stored
 * populations of the first fluid layer, q = 2 w_T theta_w - 2 g*_(-y) on the
 * hot wall and 2 g*_(+y) - 2 w_T theta_w on the cold wall (anti-bounce-back
 * returns -g* + 2 w_T theta_w), Nu = H q / alpha.  Exact for the conduction
 * state; equal on both walls at a steady state.  Walled cavities only. */
dmrt_status dmrt_nusselt_flux(dmrt_t *h, int wall, double out[3]);

/* The local Nusselt number of wall 0 or 1 as a float32 [z][x] map. */
dmrt_status dmrt_nusselt_local(dmrt_t *h, int wall, float *local, int on_device);

/* Nusselt numbers of a caller's temperature field without allocating any
 * device memory.  The paper has no counterpart: this serves callers that may
 * not allocate device memory once running (a host application whose memory
 * pool owns the device memory, or a time-critical loop where cudaMalloc /
 * cudaFree would stall the device).
 *
 * theta: device pointer, float32 [z][y][x] (nx*ny*nz), e.g. filled by
 * dmrt_fields(..., on_device = 1).  wall 0 = hot wall y = 0, 1 = cold wall
 * y = H.  The result out[3] (host memory) is (Nu_3D, Nu_2D, Nu_max), with the
 * discretisation of dmrt_nusselt.  stream: a cudaStream_t (NULL = the legacy
 * default stream); the call synchronises it.
 *
 * Scratch: a fixed array of 3 * 8192 + 4 doubles (about 192 KB) in the
 * library's own device memory, placed when the library is loaded on a GPU and
 * held by every GPU that loads it until the process exits.  nz may be at most
 * 8192; larger nz, nx*ny*nz >= 2^31, ny < 2, a NULL pointer or a wall other
 * than 0 / 1 return DMRT_ERR_ARG before any GPU work.  The call never calls
 * cudaMalloc or cudaFree.  theta must live on the current device: every
 * call, with that device current, looks up the array's device address there
 * (cudaGetSymbolAddress, which allocates nothing).  The call ends by
 * synchronising the stream and copying the result to host memory, so it
 * must not be called on a stream that is being captured into a CUDA graph.
 * Every call shares the one array: each call writes every slot it reads, so
 * nothing carries over, but calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * DMRT_ERR_CUDA if a CUDA call fails. */
dmrt_status dmrt_nusselt_noalloc(const float *theta, int nx, int ny, int nz, int wall,
                                 void *stream, double out[3]);

/* The convergence residual (the paper states no convergence rule; this is
 * the library's reading of it) from the last two residual points, the
 * states n and n - K pulled by the last steps of two consecutive intervals
 * (see dmrt_step): r = max(|theta^n - theta^{n-K}|_2 / |theta^n|_2,
 * |u^n - u^{n-K}|_2 / |u^n|_2) / K.  Each cell's four terms are FP32 (from
 * the FP32 fields, exactly those dmrt_fields reports for that state); they
 * are summed in double-float arithmetic (about 48 significand bits) and r is
 * formed in FP64, so r carries the rounding of the cells' FP32 terms only (a
 * few units of 2^-24, relative).  +inf until two points exist; the points
 * restart after dmrt_set_populations, dmrt_init_fields or a warm start.
 * Returns DMRT_ERR_DIVERGED if the fields hold a NaN or Inf.  Synchronises. */
dmrt_status dmrt_residual(dmrt_t *h, double *r);

/* Step until the residual falls below tol or max_steps more steps are taken
 * (then DMRT_ERR_TIMEOUT).  *steps_taken and *r (either may be NULL) receive
 * the steps run by this call and the last residual. */
dmrt_status dmrt_run_to_steady(dmrt_t *h, double tol, long max_steps, long *steps_taken,
                               double *r);

/* Replace the stored (post-collision) populations: f is [19][z][y][x], g is
 * [7][z][y][x], float32.  Resets the residual history. */
dmrt_status dmrt_set_populations(dmrt_t *h, const float *f, const float *g, int on_device);

/* Copy out the stored populations in the layout of dmrt_set_populations.
 * Either pointer may be NULL.  Synchronises. */
dmrt_status dmrt_get_populations(dmrt_t *h, float *f, float *g, int on_device);

/* Set the state to the equilibrium of given fields: f = f_eq(rho, u) of
 * Eq. (17), g = w_T theta (1 + 4 e.u), the D3Q7 equilibrium of Eq. (33).
 * Resets the residual history (used for warm starts). */
dmrt_status dmrt_init_fields(dmrt_t *h, const float *rho, const float *u, const float *theta,
                             int on_device);

/* Checkpoint / resume.  A checkpoint is a self-describing host byte blob:
 * the handle's grid, wall type, storage, streaming scheme, lattice
 * parameters and step count, its stored populations (with the
 * stochastic-rounding step counters, in the buffer's own layout) and its
 * residual history.  Loading it into a handle created with the same grid,
 * wall type, storage, streaming scheme, residual interval and lattice
 * parameters restores the state exactly: the continued run is bitwise identical to an uninterrupted
 * one.  dmrt_checkpoint_size gives the blob size; save writes it to `dst`
 * (host, `size` bytes at least); load reads it (DMRT_ERR_ARG if the blob does
 * not match the handle).  Both synchronise. */
long long dmrt_checkpoint_size(const dmrt_t *h);
dmrt_status dmrt_checkpoint_save(dmrt_t *h, void *dst, long long size);
dmrt_status dmrt_checkpoint_load(dmrt_t *h, const void *src, long long size);

/* Anisotropic diffusion (Eqs. (35)-(37)): replace the isotropic thermal
 * relaxation by the full tensor D (row-major 3x3, lattice units, symmetric
 * positive definite): tau_bar_ij = delta_ij / 2 + 4 D_ij, and the flux
 * moments relax with the inverse of that block.  dmrt_nusselt_flux then uses
 * D_yy.  DMRT_ERR_ARG if D is not symmetric positive definite. */
dmrt_status dmrt_set_diffusion(dmrt_t *h, const double D[9]);

/* Read the derived lattice parameters. */
dmrt_status dmrt_get_params(const dmrt_t *h, dmrt_params *out);

/* Enable (1) or disable (0) CUDA-event timing of the step kernels. */
dmrt_status dmrt_set_timing(dmrt_t *h, int enabled);

/* Read the launch counters and the event timing (synchronises when timing
 * is on).  reset = 1 zeroes them afterwards. */
dmrt_status dmrt_get_stats(dmrt_t *h, dmrt_stats *out, int reset);

/* ------------------------------------------------------------------------
 * Ensembles: many independent cavities advanced together.  Every time step
 * is a few kernel launches: one per cavity shape when the rows are even and
 * the shapes few (the shape's offset tables and its cavities' rates in the
 * launch parameters), else one per 64 cavities (their sizes and rates in the
 * launch parameters, a block map in device memory giving each thread block
 * its cavity's tile); a whole residual interval of K steps
 * replays one captured CUDA graph.  Cavities may differ in size, Ra, Pr, Ma
 * and wall type; they share the storage format and K.  Members are numbered
 * 0..count-1 in the order given.  The method per cavity is exactly that of a
 * single handle (same kernels' arithmetic, bitwise identical results).
 * ---------------------------------------------------------------------- */
typedef struct dmrt_ensemble dmrt_ensemble_t;

/* One member: grid, physical numbers (as dmrt_create) and wall type. */
typedef struct dmrt_cavity_desc {
    int grid[3];
    double Ra, Pr, Ma;
    int wall_type;
} dmrt_cavity_desc;

/* Create an ensemble of `count` >= 1 cavities (each validated as by
 * dmrt_create, walled types 1-3 only; the first invalid one fails the call
 * with DMRT_ERR_ARG).  All
 * start from rest.  opts as for dmrt_create_ex (NULL = defaults).  The total
 * population storage must fit the 32-bit cell indexing of each member and the
 * device memory. */
dmrt_status dmrt_ensemble_create(dmrt_ensemble_t **out, int count, const dmrt_cavity_desc *cavities,
                                 const dmrt_opts *opts);

void dmrt_ensemble_destroy(dmrt_ensemble_t *e);

/* As dmrt_set_stream / dmrt_sync / dmrt_set_timing / dmrt_get_stats. */
dmrt_status dmrt_ensemble_set_stream(dmrt_ensemble_t *e, void *stream);
dmrt_status dmrt_ensemble_sync(dmrt_ensemble_t *e);
dmrt_status dmrt_ensemble_set_timing(dmrt_ensemble_t *e, int enabled);
dmrt_status dmrt_ensemble_get_stats(dmrt_ensemble_t *e, dmrt_stats *out, int reset);

/* Pick the thread-block size (128 or 256 threads; 128 only in place or with two cells
 * per thread) and, per distinct cavity width, the tile width along x in
 * threads (32, 64 or 128, and 16 with two cells per thread, where a thread
 * covers two cells of the row) by timing `trials` launches of each candidate
 * on the live buffers (in place: on a scratch copy; the state is not
 * advanced).  `report` (may be NULL) receives a one-line summary: the
 * choices and the total per thread-block size, "chosen threads=T;", then
 * every candidate's time as " nxW/tT/bxB:Mus".  Without a call the defaults
 * are 128 threads and, with one cell per thread, the widest tile not wider
 * than the row's threads (rounded up to 32); with two cells per thread, the
 * tile of 16, 32 or 64 pairs that leaves the fewest idle threads along a row
 * (the widest of equals), as for a single cavity. */
dmrt_status dmrt_ensemble_autotune(dmrt_ensemble_t *e, int trials, char *report, int report_len);

/* Advance every member n >= 0 steps (residual points as in dmrt_step, per
 * member: taken by a reduction kernel just before the last step of every
 * K-step interval, with the sums of a single cavity). */
dmrt_status dmrt_ensemble_step(dmrt_ensemble_t *e, long n);

/* Per-member residuals r[count] (as dmrt_residual; +inf before two residual
 * points).  DMRT_ERR_DIVERGED if any member holds a NaN/Inf; the r of that
 * member is NaN.  Synchronises. */
dmrt_status dmrt_ensemble_residual(dmrt_ensemble_t *e, double *r);

/* Step until every member's residual is below tol or max_steps more steps
 * are taken (DMRT_ERR_TIMEOUT).  Members that diverge end the run with
 * DMRT_ERR_DIVERGED.  *steps_taken and *converged (either may be NULL)
 * receive the steps run and how many members are below tol. */
dmrt_status dmrt_ensemble_run_to_steady(dmrt_ensemble_t *e, double tol, long max_steps,
                                        long *steps_taken, int *converged);

/* Nusselt numbers of wall 0 or 1 for every member: out[3*i + 0..2] =
 * (Nu_3D, Nu_2D, Nu_max) of member i (as dmrt_nusselt).  Synchronises. */
dmrt_status dmrt_ensemble_nusselt(dmrt_ensemble_t *e, int wall, double *out);

/* Per-member access, with the layouts of the single-handle calls. */
dmrt_status dmrt_ensemble_fields(dmrt_ensemble_t *e, int member, float *rho, float *u,
                                 float *theta, int on_device);
dmrt_status dmrt_ensemble_init_fields(dmrt_ensemble_t *e, int member, const float *rho,
                                      const float *u, const float *theta, int on_device);
dmrt_status dmrt_ensemble_get_populations(dmrt_ensemble_t *e, int member, float *f, float *g,
                                          int on_device);
dmrt_status dmrt_ensemble_member_params(const dmrt_ensemble_t *e, int member, dmrt_params *out);

/* Text of the last error on this ensemble ("" if none). */
const char *dmrt_ensemble_last_error(const dmrt_ensemble_t *e);

/* ------------------------------------------------------------------------
 * Warm-start surrogate: a 3-D convolutional U-Net mapping a cavity's
 * parameters (Ra, wall type) to an approximate steady state on an n^3 grid:
 * 5 channels (u_x, u_y, u_z)/u_c, theta and (rho - 1)/(3 u_c^2) (the density
 * carries the hydrostatic balance of the buoyancy, so a warm start with it
 * releases no pressure transient), trained on the GPU by this library's own forward
 * and backward kernels (FP32 accumulation; weights and activations in FP32 or
 * BF16).  Its prediction only initialises a cavity (dmrt_warm_start); the
 * lattice Boltzmann solve then runs to its own convergence criterion.
 * The paper has no such component: it serves the time-to-steady-state goal.
 *
 * Network with depth D and channels c_0..c_D (8 input features per voxel:
 * (log10 Ra - 4.5)/1.5, one-hot wall type, x, y, z in [-1, 1], 1/2 - Y):
 *   a_0 = act(conv3(x; 8 -> c_0)), s_0 = act(conv3(a_0; c_0 -> c_0));
 *   a_l = act(conv3(avgpool2(s_{l-1}); c_{l-1} -> c_l)), s_l = act(conv3(a_l))
 *   for l = 1..D; h_D = s_D; for l = D-1..0: d_l = act(conv3(h_{l+1};
 *   c_{l+1} -> c_l)), m_l = up2(d_l) + s_l, h_l = act(conv3(m_l; c_l -> c_l));
 *   out = conv1(h_0; c_0 -> 5).  act: leaky ReLU, slope 0.1.  Loss: mean
 *   squared error.  Optimiser: Adam (0.9, 0.999, 1e-8) on FP32 master weights.
 * Tensors are channels-last [batch][z][y][x][channel]; parameters are one
 * flat FP32 vector, layer by layer in the order above (each conv's weights
 * [tap][cout][cin], taps (dz, dy, dx) with dx fastest, then its biases).
 * ---------------------------------------------------------------------- */
typedef struct dmrt_surrogate dmrt_surrogate_t;

typedef struct dmrt_surrogate_cfg {
    int grid;        /* n: edge of the cubic grid; n / 2^depth a multiple of 8 */
    int depth;       /* pooling levels D, 1..3 */
    int channels[4]; /* c_0..c_D, each 4, 8, 16, 32, 64 or 128 */
    int storage;     /* DMRT_STORE_F32 or DMRT_STORE_BF16 */
    int max_batch;   /* largest batch of one call */
    unsigned seed;   /* initial weights: He-uniform from a PCG hash of the seed
                        (the 1x1 output head and all biases start at zero) */
} dmrt_surrogate_cfg;

dmrt_status dmrt_surrogate_create(dmrt_surrogate_t **out, const dmrt_surrogate_cfg *cfg);
void dmrt_surrogate_destroy(dmrt_surrogate_t *s);
dmrt_status dmrt_surrogate_set_stream(dmrt_surrogate_t *s, void *stream);

/* Number of parameters (-1 for NULL); get / set the FP32 master parameters
 * (host arrays of that length; set also resets the Adam state). */
long long dmrt_surrogate_param_count(const dmrt_surrogate_t *s);
dmrt_status dmrt_surrogate_get_params(dmrt_surrogate_t *s, float *params, long long count);
dmrt_status dmrt_surrogate_set_params(dmrt_surrogate_t *s, const float *params, long long count);

/* Prediction for `batch` samples (host arrays Ra[batch] > 0, wall[batch] in
 * 1..3): out[batch][n^3][5] FP32 (host or device per on_device). */
dmrt_status dmrt_surrogate_predict(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                   float *out, int on_device);

/* One Adam step on a batch; target is a DEVICE array [batch][n^3][5] FP32;
 * *loss (may be NULL) receives the batch loss before the step. */
dmrt_status dmrt_surrogate_train_step(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                      const float *target, float lr, double *loss);

/* Loss and its gradient with respect to every parameter (host grad[count]),
 * without updating; and the loss alone. */
dmrt_status dmrt_surrogate_gradients(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                     const float *target, float *grad, double *loss);
dmrt_status dmrt_surrogate_loss(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                const float *target, double *loss);

/* Training target of one sample from the planar device fields of
 * dmrt_fields (u [3][n^3], theta [n^3], rho [n^3] or NULL for rho = 1):
 * target[n^3][5] (device), velocities divided by uc, density as
 * (rho - 1)/(3 uc^2).  Queued on `stream` (NULL = legacy default stream). */
dmrt_status dmrt_surrogate_target_from_fields(const float *u, const float *theta, const float *rho, int n,
                                              double uc, float *target, void *stream);

/* Initialise a cubic cavity from the surrogate's prediction for (Ra, wall):
 * the n^3 prediction is resampled trilinearly to the cavity's grid, the
 * velocity scaled by the cavity's u_c = sqrt(g beta H) and the density by
 * 3 u_c^2, and the cavity set to the equilibrium of (rho, u, theta) as by
 * dmrt_init_fields.  Allocates a
 * temporary device buffer of 5 floats per cavity cell. */
dmrt_status dmrt_warm_start(dmrt_t *h, dmrt_surrogate_t *s, double Ra, int wall);

const char *dmrt_surrogate_last_error(const dmrt_surrogate_t *s);

/* One convolution layer of the surrogate on device arrays (for testing and
 * reuse): y = act(conv_k(x, w) + bias) with the layouts above; storage
 * DMRT_STORE_BF16 reads x and w as bfloat16 (tensor cores when cin is a
 * multiple of 8 and both pointers are 16-byte aligned) and writes y as
 * bfloat16 (out_f32 = 0) or float (out_f32 = 1); DMRT_STORE_F32 is all float.
 * k in {1, 3}; n a multiple of 8; act 0 = none, 1 = leaky ReLU (0.1); bias
 * (float, may be NULL).  Queued on `stream`; synchronises it. */
dmrt_status dmrt_nn_conv3d(const void *x, const void *w, const float *bias, void *y, int batch, int n,
                           int cin, int cout, int k, int act, int storage, int out_f32, void *stream);

/* Diagnostic of the tensor-core convolutions: the number of launches whose
 * bounded wait for the tensor cores ran out (their output was not written;
 * it stays 0 in a healthy run).  reset != 0 clears the count.  -1 on a CUDA
 * error.  Synchronises the device. */
int dmrt_nn_tensor_core_errors(int reset);

/* Round n float32 values to a population storage format and back, exactly
 * as the step kernel stores populations: in and out are device arrays of n
 * floats (may alias); storage is a dmrt_storage, rounding a dmrt_rounding
 * (AUTO = stochastic for 16-bit).  Stochastic rounding draws its bits from
 * the PCG hash of (i XOR hash(seed)) for element i, so a call is
 * deterministic.  F16 values are stored times 2^10, as in the cavity
 * buffers.  Queued on `stream` (NULL = the legacy default stream); does not
 * synchronise.  DMRT_ERR_ARG for a bad storage, rounding or n < 0. */
dmrt_status dmrt_round_to_storage(int storage, int rounding, const float *in, float *out, long long n,
                                  unsigned seed, void *stream);

/* Text of the last error on this handle ("" if none; static if h is NULL). */
const char *dmrt_last_error(const dmrt_t *h);

/* Name of a status code. */
const char *dmrt_status_string(int status);

/* Library version string. */
const char *dmrt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DMRT_H */
