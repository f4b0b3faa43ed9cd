// api.cu -- host implementation of the C ABI declared in include/dmrt.h.
//
// The handle owns its population buffers (two for the A-B ping-pong scheme,
// one for in-place streaming; 26 planes each), the residual snapshot and the
// reduction scratch.  Every entry point validates
// its arguments, queues work on the handle's stream and converts CUDA errors
// into a dmrt_status plus a message; nothing throws across the ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dmrt.h"
#include "internal.h"

using lbm::CollideParams;
using lbm::Geometry;

struct dmrt {
    int device = 0;
    int wall = 1;
    int storage = DMRT_STORE_F32;
    bool stochastic = false;  // 16-bit stores round stochastically
    int K = 100;
    double nu = 0, alpha = 0, gbeta = 0;
    Geometry G{};
    lbm::StepGeometry S{};
    CollideParams C{};
    lbm::BlockShape block{32, 4};
    int cells_per_thread = 1;  // 2: the paired step kernels (walled box, even nx)
    int pair_loads = 0;        // paired two-buffer step: 1 direct loads, 2 TMA-staged
    alignas(64) unsigned char tma_map[2][256] = {};  // tensor maps of buf[0], buf[1] (rows, x edges)
    unsigned *derr = nullptr;  // device word: a staged kernel's copy wait ran out

    void *buf[2] = {nullptr, nullptr};   // ping-pong population buffers (storage type)
    int cur = 0;                          // buffer holding the current state
    bool inplace = false;                 // one buffer, in-place streaming (buf[0])
    int parity = 0;                       // in-place: layout of the state (steps mod 2)
    lbm::InplaceGeometry SI{};
    long long device_bytes = 0;           // device memory held by the handle
    float *snap = nullptr;                // residual snapshot: theta, u (4 planes)
    double *partials = nullptr;           // reduction scratch (Nu rows; residual block partials)
    size_t npartials = 0;
    long long res_blocks = 0;             // blocks of a residual step's grid (its partials)
    double *dres = nullptr;               // residual result (8 doubles; [6] = points taken,
                                          // [7] the finishing kernel's ticket word)
    double *dnu = nullptr;                // Nusselt result (3 doubles)
    float *staging = nullptr;             // device staging for host transfers
    size_t staging_floats = 0;

    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;

    long steps = 0;
    int snaps = 0;  // residual points taken since the last reset (capped at 2)

    // CUDA graphs of one full residual interval (K steps), one per starting
    // buffer (A-B) or layout (in-place); captured on first use, replayed
    // afterwards.
    bool use_graphs = true;
    bool use_pdl = true;
    cudaGraphExec_t interval_graph[2] = {nullptr, nullptr};

    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<long> ev_counts;
    long step_launches = 0, total_launches = 0, timed_steps = 0;
    double step_ms = 0.0;

    std::string err;
};

namespace {

// Longest residual interval that is replayed as one captured graph.
constexpr long kMaxGraphSteps = 1000;

const char *kStatusNames[] = {"DMRT_OK", "DMRT_ERR_ARG", "DMRT_ERR_CUDA", "DMRT_ERR_OOM",
                              "DMRT_ERR_DIVERGED", "DMRT_ERR_TIMEOUT"};

dmrt_status fail(dmrt_t *h, dmrt_status st, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

dmrt_status fail(dmrt_t *h, dmrt_status st, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

dmrt_status cuda_fail(dmrt_t *h, cudaError_t e, const char *what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? DMRT_ERR_OOM : DMRT_ERR_CUDA, "%s: %s (%s)",
                what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(h, call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

// Keeps the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

long long cell_count(const Geometry &G)
{
    return static_cast<long long>(G.nx) * G.ny * G.nz;
}

// Geometry of the current state, with the layout the aux kernels must read.
Geometry state_geometry(const dmrt_t *h)
{
    Geometry G = h->G;
    G.layout = !h->inplace ? lbm::kLayoutAB
                           : (h->parity ? lbm::kLayoutStreamed : lbm::kLayoutSwapped);
    return G;
}

// Which of the two alternating states the handle is in: the current buffer
// (A-B) or the layout parity (in-place).  Toggles with every step.
int &phase(dmrt_t *h) { return h->inplace ? h->parity : h->cur; }

// One fused step from state `ph`; with `res` the step also takes the
// residual point of the state it pulls, and the finishing kernel follows.
// The staged (TMA) handles take that step with the direct-load paired
// kernel, which stores bitwise the same populations.
cudaError_t launch_one_step(dmrt_t *h, int ph, bool res)
{
    const lbm::ResidualArgs R{h->snap, reinterpret_cast<float *>(h->partials), h->dres + 6,
                              static_cast<unsigned>(cell_count(h->G))};
    const lbm::ResidualArgs *rp = res ? &R : nullptr;
    cudaError_t e;
    if (h->inplace && h->cells_per_thread == 2)
        e = lbm::launch_step_inplace_pair(h->wall, h->storage, h->stochastic, h->buf[0], ph, h->SI, h->G, h->C,
                                          h->stream, h->use_pdl, rp);
    else if (h->inplace)
        e = lbm::launch_step_inplace(h->wall, h->storage, h->stochastic, h->buf[0], ph, h->SI, h->G, h->C,
                                     h->block, h->stream, h->use_pdl, rp);
    else if (h->pair_loads == 2 && !res)
        e = lbm::launch_step_pair_tma(h->wall, h->storage, h->stochastic, h->tma_map[ph], h->buf[ph],
                                      h->buf[ph ^ 1], h->S, h->G, h->C, h->derr, h->stream, h->use_pdl);
    else if (h->cells_per_thread == 2)
        e = lbm::launch_step_pair(h->wall, h->storage, h->stochastic, h->buf[ph], h->buf[ph ^ 1], h->S, h->G,
                                  h->C, h->stream, h->use_pdl, rp);
    else
        e = lbm::launch_step(h->wall, h->storage, h->stochastic, h->buf[ph], h->buf[ph ^ 1], h->S, h->G, h->C,
                             h->block, h->stream, h->use_pdl, rp);
    if (e != cudaSuccess || !res) return e;
    return lbm::launch_residual_finish(R.partials, h->res_blocks, R.partials + 8 * h->res_blocks,
                                       reinterpret_cast<unsigned *>(h->dres + 7), h->K, h->dres, h->stream);
}

// Does the step from the current step count take a residual point?  The
// points are the states pulled by the last step of every K-step interval.
bool residual_step(const dmrt_t *h, long steps_done) { return (steps_done + 1) % h->K == 0; }

// Forget the residual history (a new state was written).
dmrt_status reset_residual(dmrt_t *h)
{
    h->snaps = 0;
    CK(h, cudaMemsetAsync(h->dres + 6, 0, sizeof(double), h->stream), "reset residual points");
    return DMRT_OK;
}

bool periodic(const dmrt_t *h) { return h->wall == DMRT_WALL_PERIODIC; }

// A staged step kernel whose copy wait ran out has set *derr and left its
// cells unwritten: report it once (after a synchronisation) and clear it.
dmrt_status check_stage_errors(dmrt_t *h)
{
    if (h->pair_loads != 2) return DMRT_OK;
    unsigned v = 0;
    CK(h, cudaMemcpyAsync(&v, h->derr, sizeof v, cudaMemcpyDeviceToHost, h->stream), "copy stage error word");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (v == 0) return DMRT_OK;
    CK(h, cudaMemsetAsync(h->derr, 0, sizeof v, h->stream), "clear stage error word");
    return fail(h, DMRT_ERR_TIMEOUT, "a staged step kernel's copy wait ran out; the state is invalid");
}

// Relaxation rates of Eq. (26) (flow) and Eqs. (35),(36) (energy), folded with
// the squared norms of the moment basis.
void fill_rates(dmrt_t *h) { lbm::fill_collide_params(h->C, h->nu, h->alpha, h->gbeta); }

dmrt_status ensure_staging(dmrt_t *h, size_t floats)
{
    if (h->staging_floats >= floats) return DMRT_OK;
    if (h->staging) cudaFree(h->staging);
    h->device_bytes -= static_cast<long long>(h->staging_floats * sizeof(float));
    h->staging = nullptr;
    h->staging_floats = 0;
    CK(h, cudaMalloc(&h->staging, floats * sizeof(float)), "cudaMalloc(staging)");
    h->staging_floats = floats;
    h->device_bytes += static_cast<long long>(floats * sizeof(float));
    return DMRT_OK;
}

cudaEvent_t take_event(dmrt_t *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

dmrt_status collect_timing(dmrt_t *h)
{
    for (size_t k = 0; k < h->ev_pending.size(); ++k) {
        auto &p = h->ev_pending[k];
        CK(h, cudaEventSynchronize(p.second), "cudaEventSynchronize");
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, p.first, p.second), "cudaEventElapsedTime");
        h->step_ms += ms;
        h->timed_steps += h->ev_counts[k];
        h->ev_pool.push_back(p.first);
        h->ev_pool.push_back(p.second);
    }
    h->ev_pending.clear();
    h->ev_counts.clear();
    return DMRT_OK;
}

// Capture K consecutive step launches starting from state `start` into an
// executable graph.  Returns false (and leaves graphs off) if the stream
// cannot be captured, e.g. the legacy default stream.
bool capture_interval(dmrt_t *h, int start)
{
    if (h->stream == nullptr) return false;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int ph = start;
    bool ok = true;
    for (long s = 0; s < h->K && ok; ++s) {
        ok = launch_one_step(h, ph, s == h->K - 1) == cudaSuccess;
        ph ^= 1;
    }
    cudaGraph_t graph = nullptr;
    ok = (cudaStreamEndCapture(h->stream, &graph) == cudaSuccess) && ok && graph;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        return false;
    }
    h->interval_graph[start] = exec;
    return true;
}

// Launch n fused steps; the last step of every K-step interval also takes
// a residual point.  A whole interval of K steps replays a captured graph.
dmrt_status run_steps(dmrt_t *h, long n)
{
    long done = 0;
    while (done < n) {
        long until_res = h->K - (h->steps % h->K);
        long chunk = std::min(n - done, until_res);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing) {
            e0 = take_event(h);
            e1 = take_event(h);
            if (!e0 || !e1) return fail(h, DMRT_ERR_CUDA, "cudaEventCreate failed");
            CK(h, cudaEventRecord(e0, h->stream), "cudaEventRecord");
        }
        bool graphed = false;
        int &ph = phase(h);
        if (chunk == h->K && h->K <= kMaxGraphSteps && h->use_graphs) {
            if (!h->interval_graph[ph] && !capture_interval(h, ph)) h->use_graphs = false;
            if (h->interval_graph[ph]) {
                CK(h, cudaGraphLaunch(h->interval_graph[ph], h->stream), "cudaGraphLaunch");
                if (h->K & 1) ph ^= 1;
                h->steps += chunk;
                h->step_launches += chunk;
                h->total_launches += chunk + 1;  // and the residual's finishing kernel
                if (h->snaps < 2) h->snaps++;
                graphed = true;
            }
        }
        for (long s = 0; s < chunk && !graphed; ++s) {
            const bool res = residual_step(h, h->steps);
            CK(h, launch_one_step(h, ph, res), "step kernel");
            ph ^= 1;
            h->steps++;
            h->step_launches++;
            h->total_launches += res ? 2 : 1;
            if (res && h->snaps < 2) h->snaps++;
        }
        if (h->timing) {
            CK(h, cudaEventRecord(e1, h->stream), "cudaEventRecord");
            h->ev_pending.emplace_back(e0, e1);
            h->ev_counts.push_back(chunk);
        }
        done += chunk;
    }
    return DMRT_OK;
}

// In-place handles: before a whole new state is written, return to the
// swapped layout, carrying the step counter over to the word the next
// phase-0 step reads.
dmrt_status reset_layout(dmrt_t *h)
{
    if (!h->inplace || h->parity == 0) return DMRT_OK;
    unsigned *ctr = reinterpret_cast<unsigned *>(
        static_cast<char *>(h->buf[0]) +
        static_cast<size_t>(h->G.plane) * lbm::kPlanes * lbm::storage_bytes(h->storage));
    CK(h, cudaMemcpyAsync(ctr, ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream),
       "copy step counter");
    h->parity = 0;
    return DMRT_OK;
}

dmrt_status create_common(dmrt_t **out, const int grid[3], double nu, double alpha, double gbeta,
                          int wall_type, const dmrt_opts *opts)
{
    if (!out) return DMRT_ERR_ARG;
    *out = nullptr;
    if (!grid) return DMRT_ERR_ARG;
    if (wall_type < 0 || wall_type > 3) return DMRT_ERR_ARG;
    const int minext = wall_type == DMRT_WALL_PERIODIC ? 1 : 2;
    for (int a = 0; a < 3; ++a)
        if (grid[a] < minext || grid[a] > 65535) return DMRT_ERR_ARG;
    const long long cells = static_cast<long long>(grid[0]) * grid[1] * grid[2];
    // the step kernel addresses all 26 planes with 32-bit indices
    if ((cells + 63) / 64 * 64 * lbm::kPlanes >= (1LL << 32)) return DMRT_ERR_ARG;
    if (!(nu > 0.0) || !(alpha > 0.0) || !std::isfinite(nu) || !std::isfinite(alpha) ||
        !std::isfinite(gbeta))
        return DMRT_ERR_ARG;
    int storage = DMRT_STORE_F32, K = 100, rounding = DMRT_ROUND_AUTO, streaming = DMRT_STREAM_AB;
    int cpt = 0, ploads = 0;
    if (opts) {
        storage = opts->storage;
        rounding = opts->rounding;
        streaming = opts->streaming;
        cpt = opts->cells_per_thread;
        ploads = opts->pair_loads;
        if (opts->residual_interval > 0) K = opts->residual_interval;
        if (opts->residual_interval < 0) return DMRT_ERR_ARG;
    }
    if (cpt < 0 || cpt > 2 || ploads < 0 || ploads > 2) return DMRT_ERR_ARG;
    if (rounding < DMRT_ROUND_AUTO || rounding > DMRT_ROUND_STOCHASTIC) return DMRT_ERR_ARG;
    if (streaming != DMRT_STREAM_AB && streaming != DMRT_STREAM_INPLACE) return DMRT_ERR_ARG;
    if (storage != DMRT_STORE_F32 && storage != DMRT_STORE_BF16 && storage != DMRT_STORE_F16)
        return DMRT_ERR_ARG;

    dmrt_t *h = new (std::nothrow) dmrt();
    if (!h) return DMRT_ERR_OOM;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return DMRT_ERR_CUDA;
    }
    h->wall = wall_type;
    h->storage = storage;
    h->stochastic = storage != DMRT_STORE_F32 && rounding != DMRT_ROUND_NEAREST;
    h->inplace = streaming == DMRT_STREAM_INPLACE;
    h->K = K;
    h->nu = nu;
    h->alpha = alpha;
    h->gbeta = gbeta;
    h->G.nx = grid[0];
    h->G.ny = grid[1];
    h->G.nz = grid[2];
    h->G.layout = lbm::kLayoutAB;
    // pad each plane to a whole number of 128-byte lines (and 256-byte
    // alignment of every plane start)
    h->G.plane = (cells + 63) / 64 * 64;
    h->G.inv_ny = 1.0f / static_cast<float>(grid[1]);
    lbm::fill_step_geometry(h->G, h->S);
    lbm::fill_inplace_geometry(h->G, h->SI);
    fill_rates(h);
    // two cells per thread: the paired kernels serve walled boxes with even
    // nx, and auto takes them there (measured faster for every storage
    // format; the one-cell 16-bit kernels are bound by instruction issue)
    const bool pair_ok = lbm::step_pair_supported(wall_type, h->G);
    if (cpt == 2 && !pair_ok) {
        delete h;
        return DMRT_ERR_ARG;
    }
    h->cells_per_thread = (cpt == 2 || (cpt == 0 && pair_ok)) ? 2 : 1;
    // loads of the paired two-buffer kernel: TMA-staged where the tensor map
    // allows it (16-bit storage, nx a multiple of 8)
    const bool tma_ok = h->cells_per_thread == 2 && !h->inplace &&
                        lbm::step_pair_tma_supported(wall_type, storage, h->G);
    if (ploads == 2 && !tma_ok) {
        delete h;
        return DMRT_ERR_ARG;
    }
    h->pair_loads = h->cells_per_thread != 2 || h->inplace ? 0 : (tma_ok && ploads == 2 ? 2 : 1);
#ifdef DMRT_BLOCK_X
    h->block = {DMRT_BLOCK_X, DMRT_BLOCK_Y};
#else
    if (grid[0] >= 128) h->block = {128, 1};
    else if (grid[0] >= 64) h->block = {64, 2};
    else h->block = {32, 4};
#endif

    auto bail = [&](dmrt_status st) {
        dmrt_destroy(h);
        return st;
    };
    cudaError_t e;
    // populations, then a 256-byte tail holding the step counter(s)
    const size_t buf_bytes =
        static_cast<size_t>(h->G.plane) * lbm::kPlanes * lbm::storage_bytes(h->storage) + 256;
    const int nbuf = h->inplace ? 1 : 2;
    for (int b = 0; b < nbuf; ++b) {
        e = cudaMalloc(&h->buf[b], buf_bytes);
        if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? DMRT_ERR_OOM : DMRT_ERR_CUDA);
        h->device_bytes += static_cast<long long>(buf_bytes);
    }
    e = cudaMalloc(&h->snap, static_cast<size_t>(cells) * 4 * sizeof(float));
    if (e != cudaSuccess) return bail(DMRT_ERR_OOM);
    h->device_bytes += cells * 4 * static_cast<long long>(sizeof(float));
    // residual partials: 8 floats (4 doubles' room) per block of the grid of
    // the kernel that takes the residual points
    if (h->cells_per_thread == 2)
        h->res_blocks = static_cast<long long>(lbm::pair_blocks(h->G));
    else
        h->res_blocks = static_cast<long long>((grid[0] + h->block.bx - 1) / h->block.bx) *
                        ((grid[1] + h->block.by - 1) / h->block.by) * grid[2];
    // and the finishing kernel's stage after them
    h->npartials = static_cast<size_t>(h->res_blocks) * 4 + lbm::residual_stage_floats(h->res_blocks) / 2;
    if (h->npartials < 3 * static_cast<size_t>(grid[2])) h->npartials = 3 * grid[2];
    e = cudaMalloc(&h->partials, h->npartials * sizeof(double));
    if (e != cudaSuccess) return bail(DMRT_ERR_OOM);
    h->device_bytes += static_cast<long long>(h->npartials * sizeof(double));
    e = cudaMalloc(&h->dres, 16 * sizeof(double));
    if (e != cudaSuccess) return bail(DMRT_ERR_OOM);
    h->device_bytes += 16 * static_cast<long long>(sizeof(double));
    h->dnu = h->dres + 8;
    h->derr = reinterpret_cast<unsigned *>(h->dres + 12);  // doubles 12..15: error words
    if (cudaMemset(h->dres, 0, 16 * sizeof(double)) != cudaSuccess) return bail(DMRT_ERR_CUDA);
    if (h->pair_loads == 2) {
        e = lbm::prepare_step_pair_tma(wall_type, storage);
        if (e != cudaSuccess) return bail(DMRT_ERR_CUDA);
        for (int b = 0; b < 2; ++b) {
            e = lbm::encode_pair_tma_maps(h->buf[b], h->G, h->tma_map[b]);
            if (e != cudaSuccess) {
                if (ploads == 2) return bail(DMRT_ERR_CUDA);
                h->pair_loads = 1;  // auto: the direct-load kernel does the same work
                break;
            }
        }
    }
    e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(DMRT_ERR_CUDA);
    h->stream = h->own;
#ifdef DMRT_NO_GRAPHS
    h->use_graphs = false;
#endif
#ifdef DMRT_NO_PDL
    h->use_pdl = false;
#endif
    // start from rest: f = w (zero deviations), g = 0 (theta = 0); the zero
    // state and counters are the same in every layout
    for (int b = 0; b < nbuf; ++b) {
        e = cudaMemsetAsync(h->buf[b], 0, buf_bytes, h->stream);
        if (e != cudaSuccess) return bail(DMRT_ERR_CUDA);
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(DMRT_ERR_CUDA);
    *out = h;
    return DMRT_OK;
}

}  // namespace

extern "C" {

dmrt_status dmrt_create(dmrt_t **out, const int grid[3], double Ra, double Pr, double Ma,
                        int wall_type)
{
    return dmrt_create_ex(out, grid, Ra, Pr, Ma, wall_type, nullptr);
}

dmrt_status dmrt_create_ex(dmrt_t **out, const int grid[3], double Ra, double Pr, double Ma,
                           int wall_type, const dmrt_opts *opts)
{
    if (out) *out = nullptr;
    if (!grid || !(Ra > 0.0) || !(Pr > 0.0) || !(Ma > 0.0) || !(Ma < 0.3) || !std::isfinite(Ra) ||
        !std::isfinite(Pr))
        return DMRT_ERR_ARG;
    if (grid[1] < 2) return DMRT_ERR_ARG;
    // Eq. (38) with H = ny, dT = 1, c = 1: Ma = u_c / c_s, u_c^2 = g beta dT H,
    // Ra = g beta dT H^3 Pr / nu^2, Pr = nu / alpha.
    const double H = static_cast<double>(grid[1]);
    const double uc = Ma / std::sqrt(3.0);
    const double gbeta = uc * uc / H;
    const double nu = uc * H * std::sqrt(Pr / Ra);
    const double alpha = nu / Pr;
    return create_common(out, grid, nu, alpha, gbeta, wall_type, opts);
}

dmrt_status dmrt_create_lattice(dmrt_t **out, const int grid[3], double nu, double alpha,
                                double gbeta, int wall_type, const dmrt_opts *opts)
{
    return create_common(out, grid, nu, alpha, gbeta, wall_type, opts);
}

void dmrt_destroy(dmrt_t *h)
{
    if (!h) return;
    DeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto &p : h->ev_pending) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (auto &g : h->interval_graph)
        if (g) cudaGraphExecDestroy(g);
    for (int b = 0; b < 2; ++b)
        if (h->buf[b]) cudaFree(h->buf[b]);
    if (h->snap) cudaFree(h->snap);
    if (h->partials) cudaFree(h->partials);
    if (h->dres) cudaFree(h->dres);
    if (h->staging) cudaFree(h->staging);
    if (h->own) cudaStreamDestroy(h->own);
    delete h;
}

dmrt_status dmrt_set_stream(dmrt_t *h, void *stream)
{
    if (!h) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    // order the new stream after everything queued so far
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own;
    return DMRT_OK;
}

dmrt_status dmrt_step(dmrt_t *h, long n)
{
    if (!h) return DMRT_ERR_ARG;
    if (n < 0) return fail(h, DMRT_ERR_ARG, "dmrt_step: n = %ld < 0", n);
    DeviceGuard dg(h->device);
    return run_steps(h, n);
}

dmrt_status dmrt_sync(dmrt_t *h)
{
    if (!h) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return check_stage_errors(h);
}

dmrt_status dmrt_fields(dmrt_t *h, float *rho, float *u, float *theta, int on_device)
{
    if (!h) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    const size_t cells = static_cast<size_t>(cell_count(h->G));
    float *drho = rho, *du = u, *dth = theta;
    if (!on_device) {
        dmrt_status st = ensure_staging(h, 5 * cells);
        if (st != DMRT_OK) return st;
        drho = rho ? h->staging : nullptr;
        du = u ? h->staging + cells : nullptr;
        dth = theta ? h->staging + 4 * cells : nullptr;
    }
    CK(h, lbm::launch_fields(h->wall, h->storage, h->buf[h->cur], state_geometry(h), drho, du, dth, h->stream),
       "fields kernel");
    h->total_launches++;
    if (!on_device) {
        if (rho)
            CK(h, cudaMemcpyAsync(rho, drho, cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
               "copy rho");
        if (u)
            CK(h, cudaMemcpyAsync(u, du, 3 * cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
               "copy u");
        if (theta)
            CK(h, cudaMemcpyAsync(theta, dth, cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
               "copy theta");
    }
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_nusselt(dmrt_t *h, int wall, double out[3])
{
    if (!h || !out) return DMRT_ERR_ARG;
    if (wall != 0 && wall != 1) return fail(h, DMRT_ERR_ARG, "dmrt_nusselt: wall must be 0 or 1");
    if (h->G.ny < 2) return fail(h, DMRT_ERR_ARG, "dmrt_nusselt: needs ny >= 2");
    DeviceGuard dg(h->device);
    CK(h,
       lbm::launch_nusselt(h->wall, h->storage, h->buf[h->cur], state_geometry(h), wall, nullptr, h->partials,
                           h->dnu, h->stream),
       "nusselt kernel");
    h->total_launches += 2;
    CK(h, cudaMemcpyAsync(out, h->dnu, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
       "copy nusselt");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_nusselt_flux(dmrt_t *h, int wall, double out[3])
{
    if (!h || !out) return DMRT_ERR_ARG;
    if (wall != 0 && wall != 1) return fail(h, DMRT_ERR_ARG, "dmrt_nusselt_flux: wall must be 0 or 1");
    if (h->wall == DMRT_WALL_PERIODIC) return fail(h, DMRT_ERR_ARG, "dmrt_nusselt_flux: needs walls");
    DeviceGuard dg(h->device);
    CK(h,
       lbm::launch_nusselt_flux(h->storage, h->buf[h->cur], state_geometry(h), wall, h->alpha, nullptr, h->partials, h->dnu,
                                h->stream),
       "nusselt flux kernel");
    h->total_launches += 2;
    CK(h, cudaMemcpyAsync(out, h->dnu, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy nusselt");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_nusselt_local(dmrt_t *h, int wall, float *local, int on_device)
{
    if (!h || !local) return DMRT_ERR_ARG;
    if (wall != 0 && wall != 1) return fail(h, DMRT_ERR_ARG, "dmrt_nusselt_local: wall must be 0 or 1");
    if (h->G.ny < 2) return fail(h, DMRT_ERR_ARG, "dmrt_nusselt_local: needs ny >= 2");
    DeviceGuard dg(h->device);
    const size_t n = static_cast<size_t>(h->G.nx) * h->G.nz;
    float *dst = local;
    if (!on_device) {
        dmrt_status st = ensure_staging(h, n);
        if (st != DMRT_OK) return st;
        dst = h->staging;
    }
    CK(h,
       lbm::launch_nusselt(h->wall, h->storage, h->buf[h->cur], state_geometry(h), wall, dst, h->partials,
                           h->dnu, h->stream),
       "nusselt kernel");
    h->total_launches += 2;
    if (!on_device)
        CK(h, cudaMemcpyAsync(local, dst, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
           "copy local nusselt");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_residual(dmrt_t *h, double *r)
{
    if (!h || !r) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    if (h->snaps < 2) {
        *r = INFINITY;
        return DMRT_OK;
    }
    double res[8];
    CK(h, cudaMemcpyAsync(res, h->dres, sizeof res, cudaMemcpyDeviceToHost, h->stream),
       "copy residual");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    *r = res[4];
    const dmrt_status se = check_stage_errors(h);
    if (se != DMRT_OK) return se;
    if (res[5] != 0.0 || !std::isfinite(res[4]))
        return fail(h, DMRT_ERR_DIVERGED, "non-finite fields at step %ld", h->steps);
    return DMRT_OK;
}

dmrt_status dmrt_run_to_steady(dmrt_t *h, double tol, long max_steps, long *steps_taken,
                               double *r)
{
    if (!h || !(tol > 0.0) || max_steps < 0) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    long taken = 0;
    double res = INFINITY;
    dmrt_status st = DMRT_OK;
    while (true) {
        if (h->snaps >= 2) {
            st = dmrt_residual(h, &res);
            if (st != DMRT_OK) break;
            if (res < tol) break;
        }
        if (taken >= max_steps) {
            st = fail(h, DMRT_ERR_TIMEOUT, "no convergence to %g within %ld steps (r = %g)", tol,
                      max_steps, res);
            break;
        }
        long chunk = h->K - (h->steps % h->K);
        if (chunk > max_steps - taken) chunk = max_steps - taken;
        st = run_steps(h, chunk);
        if (st != DMRT_OK) break;
        taken += chunk;
    }
    if (steps_taken) *steps_taken = taken;
    if (r) *r = res;
    return st;
}

dmrt_status dmrt_set_populations(dmrt_t *h, const float *f, const float *g, int on_device)
{
    if (!h || !f || !g) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    const size_t cells = static_cast<size_t>(cell_count(h->G));
    const float *df = f, *dg_ = g;
    if (!on_device) {
        dmrt_status st = ensure_staging(h, 26 * cells);
        if (st != DMRT_OK) return st;
        CK(h, cudaMemcpyAsync(h->staging, f, 19 * cells * sizeof(float), cudaMemcpyHostToDevice, h->stream),
           "copy f");
        CK(h, cudaMemcpyAsync(h->staging + 19 * cells, g, 7 * cells * sizeof(float),
                              cudaMemcpyHostToDevice, h->stream),
           "copy g");
        df = h->staging;
        dg_ = h->staging + 19 * cells;
    }
    {
        dmrt_status st = reset_layout(h);
        if (st != DMRT_OK) return st;
    }
    CK(h, lbm::launch_set_populations(h->storage, df, dg_, h->buf[h->cur], state_geometry(h), periodic(h),
                                      h->stream),
       "set kernel");
    h->total_launches++;
    {
        dmrt_status st = reset_residual(h);
        if (st != DMRT_OK) return st;
    }
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_get_populations(dmrt_t *h, float *f, float *g, int on_device)
{
    if (!h) return DMRT_ERR_ARG;
    if (!f && !g) return DMRT_OK;
    DeviceGuard dg(h->device);
    const size_t cells = static_cast<size_t>(cell_count(h->G));
    float *df = f, *dg_ = g;
    if (!on_device) {
        dmrt_status st = ensure_staging(h, 26 * cells);
        if (st != DMRT_OK) return st;
        df = f ? h->staging : nullptr;
        dg_ = g ? h->staging + 19 * cells : nullptr;
    }
    CK(h, lbm::launch_get_populations(h->storage, h->buf[h->cur], df, dg_, state_geometry(h), periodic(h),
                                      h->stream),
       "get kernel");
    h->total_launches++;
    if (!on_device) {
        if (f)
            CK(h, cudaMemcpyAsync(f, df, 19 * cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
               "copy f");
        if (g)
            CK(h, cudaMemcpyAsync(g, dg_, 7 * cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
               "copy g");
    }
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_init_fields(dmrt_t *h, const float *rho, const float *u, const float *theta,
                             int on_device)
{
    if (!h || !rho || !u || !theta) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    const size_t cells = static_cast<size_t>(cell_count(h->G));
    const float *dr = rho, *du = u, *dt = theta;
    if (!on_device) {
        dmrt_status st = ensure_staging(h, 5 * cells);
        if (st != DMRT_OK) return st;
        CK(h, cudaMemcpyAsync(h->staging, rho, cells * sizeof(float), cudaMemcpyHostToDevice, h->stream),
           "copy rho");
        CK(h, cudaMemcpyAsync(h->staging + cells, u, 3 * cells * sizeof(float), cudaMemcpyHostToDevice,
                              h->stream),
           "copy u");
        CK(h, cudaMemcpyAsync(h->staging + 4 * cells, theta, cells * sizeof(float),
                              cudaMemcpyHostToDevice, h->stream),
           "copy theta");
        dr = h->staging;
        du = h->staging + cells;
        dt = h->staging + 4 * cells;
    }
    {
        dmrt_status st = reset_layout(h);
        if (st != DMRT_OK) return st;
    }
    CK(h, lbm::launch_init_fields(h->storage, dr, du, dt, h->buf[h->cur], state_geometry(h), periodic(h),
                                  h->stream),
       "init kernel");
    h->total_launches++;
    {
        dmrt_status st = reset_residual(h);
        if (st != DMRT_OK) return st;
    }
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

namespace {

struct CheckpointHeader {
    char magic[8];
    int version, nx, ny, nz, wall, storage, stochastic, K, snaps;
    int streaming, parity;  // in-place streaming and the layout of the saved buffer
    double nu, alpha, gbeta;
    long long steps, pop_bytes, snap_bytes;
};

constexpr char kMagic[8] = {'D', 'M', 'R', 'T', 'C', 'K', 'P', '1'};
constexpr int kCheckpointVersion = 2;

long long pop_bytes(const dmrt_t *h)
{
    return static_cast<long long>(h->G.plane) * lbm::kPlanes * lbm::storage_bytes(h->storage) + 256;
}

long long snap_bytes(const dmrt_t *h) { return cell_count(h->G) * 4 * static_cast<long long>(sizeof(float)); }

}  // namespace

long long dmrt_checkpoint_size(const dmrt_t *h)
{
    if (!h) return -1;
    return static_cast<long long>(sizeof(CheckpointHeader)) + pop_bytes(h) + snap_bytes(h) + 8 * sizeof(double);
}

dmrt_status dmrt_checkpoint_save(dmrt_t *h, void *dst, long long size)
{
    if (!h || !dst || size < dmrt_checkpoint_size(h)) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    CheckpointHeader hd{};
    memcpy(hd.magic, kMagic, 8);
    hd.version = kCheckpointVersion;
    hd.streaming = h->inplace ? DMRT_STREAM_INPLACE : DMRT_STREAM_AB;
    hd.parity = h->parity;
    hd.nx = h->G.nx;
    hd.ny = h->G.ny;
    hd.nz = h->G.nz;
    hd.wall = h->wall;
    hd.storage = h->storage;
    hd.stochastic = h->stochastic ? 1 : 0;
    hd.K = h->K;
    hd.snaps = h->snaps;
    hd.nu = h->nu;
    hd.alpha = h->alpha;
    hd.gbeta = h->gbeta;
    hd.steps = h->steps;
    hd.pop_bytes = pop_bytes(h);
    hd.snap_bytes = snap_bytes(h);
    char *p = static_cast<char *>(dst);
    memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    CK(h, cudaMemcpyAsync(p, h->buf[h->cur], hd.pop_bytes, cudaMemcpyDeviceToHost, h->stream), "copy populations");
    p += hd.pop_bytes;
    CK(h, cudaMemcpyAsync(p, h->snap, hd.snap_bytes, cudaMemcpyDeviceToHost, h->stream), "copy snapshot");
    p += hd.snap_bytes;
    CK(h, cudaMemcpyAsync(p, h->dres, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy residual");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_checkpoint_load(dmrt_t *h, const void *src, long long size)
{
    if (!h || !src || size < static_cast<long long>(sizeof(CheckpointHeader))) return DMRT_ERR_ARG;
    CheckpointHeader hd;
    memcpy(&hd, src, sizeof hd);
    if (memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kCheckpointVersion)
        return fail(h, DMRT_ERR_ARG, "not a dmrt checkpoint");
    if (hd.nx != h->G.nx || hd.ny != h->G.ny || hd.nz != h->G.nz || hd.wall != h->wall ||
        hd.storage != h->storage || hd.stochastic != (h->stochastic ? 1 : 0) || hd.K != h->K ||
        hd.streaming != (h->inplace ? DMRT_STREAM_INPLACE : DMRT_STREAM_AB) || hd.parity < 0 || hd.parity > 1 ||
        hd.nu != h->nu || hd.alpha != h->alpha || hd.gbeta != h->gbeta || hd.pop_bytes != pop_bytes(h) ||
        hd.snap_bytes != snap_bytes(h) || size < dmrt_checkpoint_size(h))
        return fail(h, DMRT_ERR_ARG,
                    "checkpoint of a different cavity (grid, walls, storage, streaming or parameters)");
    DeviceGuard dg(h->device);
    const char *p = static_cast<const char *>(src) + sizeof hd;
    CK(h, cudaMemcpyAsync(h->buf[h->cur], p, hd.pop_bytes, cudaMemcpyHostToDevice, h->stream), "copy populations");
    p += hd.pop_bytes;
    CK(h, cudaMemcpyAsync(h->snap, p, hd.snap_bytes, cudaMemcpyHostToDevice, h->stream), "copy snapshot");
    p += hd.snap_bytes;
    CK(h, cudaMemcpyAsync(h->dres, p, 8 * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy residual");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    h->steps = hd.steps;
    h->snaps = hd.snaps;
    h->parity = hd.parity;
    return DMRT_OK;
}

dmrt_status dmrt_get_params(const dmrt_t *h, dmrt_params *out)
{
    if (!h || !out) return DMRT_ERR_ARG;
    out->nx = h->G.nx;
    out->ny = h->G.ny;
    out->nz = h->G.nz;
    out->wall_type = h->wall;
    out->storage = h->storage;
    out->rounding = h->storage == DMRT_STORE_F32 ? DMRT_ROUND_NEAREST
                    : (h->stochastic ? DMRT_ROUND_STOCHASTIC : DMRT_ROUND_NEAREST);
    out->residual_interval = h->K;
    out->nu = h->nu;
    out->alpha = h->alpha;
    out->gbeta = h->gbeta;
    out->tau_nu = 3.0 * h->nu + 0.5;
    out->tau_alpha = 0.5 + 4.0 * h->alpha;
    out->steps = h->steps;
    out->streaming = h->inplace ? DMRT_STREAM_INPLACE : DMRT_STREAM_AB;
    out->device_bytes = h->device_bytes;
    out->cells_per_thread = h->cells_per_thread;
    out->pair_loads = h->pair_loads;
    return DMRT_OK;
}

dmrt_status dmrt_set_diffusion(dmrt_t *h, const double D[9])
{
    if (!h || !D) return DMRT_ERR_ARG;
    // symmetric positive definite (leading minors), finite
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(D[k])) return fail(h, DMRT_ERR_ARG, "dmrt_set_diffusion: non-finite entry");
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (D[3 * i + j] != D[3 * j + i]) return fail(h, DMRT_ERR_ARG, "dmrt_set_diffusion: D not symmetric");
    const double m1 = D[0], m2 = D[0] * D[4] - D[1] * D[3];
    const double m3 = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                      D[2] * (D[3] * D[7] - D[4] * D[6]);
    if (!(m1 > 0.0 && m2 > 0.0 && m3 > 0.0))
        return fail(h, DMRT_ERR_ARG, "dmrt_set_diffusion: D not positive definite");
    // Eq. (36): tau_bar = I/2 + D / eps, eps = 1/4; the flux block of Q is its inverse
    double t[9];
    for (int k = 0; k < 9; ++k) t[k] = 4.0 * D[k] + ((k % 4 == 0) ? 0.5 : 0.0);
    const double det = t[0] * (t[4] * t[8] - t[5] * t[7]) - t[1] * (t[3] * t[8] - t[5] * t[6]) +
                       t[2] * (t[3] * t[7] - t[4] * t[6]);
    const double inv[9] = {(t[4] * t[8] - t[5] * t[7]) / det, (t[2] * t[7] - t[1] * t[8]) / det,
                           (t[1] * t[5] - t[2] * t[4]) / det, (t[5] * t[6] - t[3] * t[8]) / det,
                           (t[0] * t[8] - t[2] * t[6]) / det, (t[2] * t[3] - t[0] * t[5]) / det,
                           (t[3] * t[7] - t[4] * t[6]) / det, (t[1] * t[6] - t[0] * t[7]) / det,
                           (t[0] * t[4] - t[1] * t[3]) / det};
    for (int k = 0; k < 9; ++k) h->C.qa[k] = static_cast<float>(inv[k] / 2.0);  // |N_1|^2 = 2
    h->C.aniso = 1;
    h->alpha = D[4];  // the wall-normal diffusivity, used by dmrt_nusselt_flux
    // captured graphs hold the old parameters
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (auto &gx : h->interval_graph)
        if (gx) {
            cudaGraphExecDestroy(gx);
            gx = nullptr;
        }
    return DMRT_OK;
}

dmrt_status dmrt_set_timing(dmrt_t *h, int enabled)
{
    if (!h) return DMRT_ERR_ARG;
    h->timing = enabled != 0;
    return DMRT_OK;
}

dmrt_status dmrt_get_stats(dmrt_t *h, dmrt_stats *out, int reset)
{
    if (!h || !out) return DMRT_ERR_ARG;
    DeviceGuard dg(h->device);
    dmrt_status st = collect_timing(h);
    if (st != DMRT_OK) return st;
    out->step_launches = h->step_launches;
    out->total_launches = h->total_launches;
    out->step_ms = h->step_ms;
    out->timed_steps = h->timed_steps;
    out->bytes_per_cell = 2.0 * lbm::kPlanes * lbm::storage_bytes(h->storage);
    if (reset) {
        h->step_launches = h->total_launches = h->timed_steps = 0;
        h->step_ms = 0.0;
    }
    return DMRT_OK;
}

dmrt_status dmrt_round_to_storage(int storage, int rounding, const float *in, float *out, long long n,
                                  unsigned seed, void *stream)
{
    if (storage != DMRT_STORE_F32 && storage != DMRT_STORE_BF16 && storage != DMRT_STORE_F16)
        return DMRT_ERR_ARG;
    if (rounding < DMRT_ROUND_AUTO || rounding > DMRT_ROUND_STOCHASTIC || n < 0) return DMRT_ERR_ARG;
    if (n == 0) return DMRT_OK;
    if (!in || !out) return DMRT_ERR_ARG;
    const bool stochastic = storage != DMRT_STORE_F32 && rounding != DMRT_ROUND_NEAREST;
    if (lbm::launch_round(storage, stochastic, in, out, n, seed, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return DMRT_ERR_CUDA;
    return DMRT_OK;
}

const char *dmrt_last_error(const dmrt_t *h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}

const char *dmrt_status_string(int status)
{
    if (status < 0 || status > DMRT_ERR_TIMEOUT) return "DMRT_UNKNOWN";
    return kStatusNames[status];
}

const char *dmrt_version(void) { return "dmrt-gb300 0.1 (sm_103a)"; }

}  // extern "C"
