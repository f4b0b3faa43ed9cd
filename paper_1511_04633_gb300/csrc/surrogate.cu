// surrogate.cu -- the warm-start surrogate: a 3-D convolutional U-Net,
// trained on the GPU by the kernels of nn.cu, whose prediction of a steady
// state initialises a cavity (the LBM then runs to its own convergence).
//
// Network (depth D, channels c_0..c_D, F = 8 input features):
//   a_0 = act(conv3(x; F -> c_0))          s_0 = act(conv3(a_0; c_0 -> c_0))
//   for l = 1..D:  p = avgpool2(s_{l-1})
//                  a_l = act(conv3(p; c_{l-1} -> c_l))  s_l = act(conv3(a_l; c_l -> c_l))
//   h_D = s_D
//   for l = D-1..0: d_l = act(conv3(h_{l+1}; c_{l+1} -> c_l))   (at level l+1)
//                   m_l = up2(d_l) + s_l                          (skip connection)
//                   h_l = act(conv3(m_l; c_l -> c_l))
//   out = conv1(h_0; c_0 -> 5)   ((u, v, w)/u_c, theta, (rho - 1)/(3 u_c^2))
// act = leaky ReLU (slope 0.1); loss = mean squared error; Adam on FP32
// master weights.  The backward pass is written out by hand below.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "dmrt.h"
#include "internal.h"
#include "nn.h"

namespace {

constexpr int kOut = 5;  // (u_x, u_y, u_z)/u_c, theta, (rho - 1)/(3 u_c^2)

struct Layer {
    int cin, cout, k, act;
    long long w_off, b_off;  // offsets in the flat parameter vector
    int level;               // resolution level it runs at
};

}  // namespace

struct dmrt_surrogate {
    int device = 0;
    int n = 64, depth = 3, storage = DMRT_STORE_BF16, max_batch = 1;
    int ch[4] = {16, 32, 64, 128};
    unsigned seed = 1;
    std::vector<Layer> layers;
    long long nparams = 0;
    float *master = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    void *wstore = nullptr;  // weights in the storage type
    void *wt = nullptr;      // transposed weights scratch (largest layer)
    // activations (storage type), per sample batch
    void *x0 = nullptr;
    std::vector<void *> a, s, dd, m, h, pin;  // by level (pin: pooled encoder inputs)
    void *out = nullptr;
    // FP32 gradient buffers (three of the largest activation size) and skip grads
    float *g0 = nullptr, *g1 = nullptr, *g2 = nullptr;
    __nv_bfloat16 *gnarrow = nullptr;  // bf16 copy of an output gradient
    std::vector<float *> gs;  // d loss / d s_l
    float *target = nullptr;
    float *scratch = nullptr;
    size_t scratch_floats = 0;
    float *bscratch = nullptr;  // partial sums of the bias gradients
    size_t bscratch_floats = 0;
    double *dpart = nullptr, *dloss = nullptr;
    double *dra = nullptr;
    int *dwall = nullptr;
    int step = 0;
    cudaStream_t stream = nullptr, own = nullptr;
    std::string err;
};

namespace {

dmrt_status sfail(dmrt_surrogate_t *s, dmrt_status st, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

dmrt_status sfail(dmrt_surrogate_t *s, dmrt_status st, const char *fmt, ...)
{
    if (s) {
        char b[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b, sizeof b, fmt, ap);
        va_end(ap);
        s->err = b;
    }
    return st;
}

#define SCK(s, call, what)                                                                    \
    do {                                                                                      \
        cudaError_t c_ = (call);                                                              \
        if (c_ != cudaSuccess)                                                                \
            return sfail(s, c_ == cudaErrorMemoryAllocation ? DMRT_ERR_OOM : DMRT_ERR_CUDA, \
                         "%s: %s", what, cudaGetErrorString(c_));                           \
    } while (0)

struct SGuard {
    int prev = -1;
    explicit SGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~SGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

inline int edge(const dmrt_surrogate_t *s, int level) { return s->n >> level; }
inline long long voxels(const dmrt_surrogate_t *s, int level)
{
    const long long e = edge(s, level);
    return e * e * e;
}
inline size_t esize(const dmrt_surrogate_t *s) { return s->storage == DMRT_STORE_F32 ? 4 : 2; }

// Layer table in execution order: encoder (a_0, s_0, ..., a_D, s_D), decoder
// (d_{D-1}, h_{D-1}, ..., d_0, h_0), head.
void build_layers(dmrt_surrogate_t *s)
{
    long long off = 0;
    auto add = [&](int cin, int cout, int k, int act, int level) {
        Layer L{cin, cout, k, act, off, 0, level};
        off += static_cast<long long>(k) * k * k * cout * cin;
        L.b_off = off;
        off += cout;
        s->layers.push_back(L);
    };
    add(lbm::nn::kFeatures, s->ch[0], 3, 1, 0);
    add(s->ch[0], s->ch[0], 3, 1, 0);
    for (int l = 1; l <= s->depth; ++l) {
        add(s->ch[l - 1], s->ch[l], 3, 1, l);
        add(s->ch[l], s->ch[l], 3, 1, l);
    }
    for (int l = s->depth - 1; l >= 0; --l) {
        add(s->ch[l + 1], s->ch[l], 3, 1, l + 1);
        add(s->ch[l], s->ch[l], 3, 1, l);
    }
    add(s->ch[0], kOut, 1, 0, 0);
    s->nparams = off;
}

const Layer &enc_a(const dmrt_surrogate_t *s, int l) { return s->layers[2 * l]; }
const Layer &enc_s(const dmrt_surrogate_t *s, int l) { return s->layers[2 * l + 1]; }
const Layer &dec_d(const dmrt_surrogate_t *s, int l)
{
    return s->layers[2 * (s->depth + 1) + 2 * (s->depth - 1 - l)];
}
const Layer &dec_h(const dmrt_surrogate_t *s, int l)
{
    return s->layers[2 * (s->depth + 1) + 2 * (s->depth - 1 - l) + 1];
}
const Layer &head(const dmrt_surrogate_t *s) { return s->layers.back(); }

// Deterministic He-uniform initial weights (biases zero) from the PCG hash;
// the 1x1 output head starts at zero, so training starts from a constant
// output (without normalisation layers, the deep network's random initial
// output is large and destabilises the first Adam steps).
void init_params(dmrt_surrogate_t *s, std::vector<float> &p)
{
    p.assign(static_cast<size_t>(s->nparams), 0.f);
    for (const Layer &L : s->layers) {
        if (&L == &s->layers.back()) break;
        const long long nw = static_cast<long long>(L.k) * L.k * L.k * L.cout * L.cin;
        const double a = std::sqrt(6.0 / (static_cast<double>(L.k) * L.k * L.k * L.cin));
        for (long long i = 0; i < nw; ++i) {
            const unsigned r = lbm::pcg_hash(static_cast<unsigned>(L.w_off + i) ^ lbm::pcg_hash(s->seed));
            const double u = (r >> 8) * (1.0 / 16777216.0);
            p[static_cast<size_t>(L.w_off + i)] = static_cast<float>((2.0 * u - 1.0) * a);
        }
    }
}

// ---------------------------------------------------------------- forward / backward

template <typename T>
const T *W(const dmrt_surrogate_t *s, const Layer &L)
{
    return static_cast<const T *>(s->wstore) + L.w_off;
}
inline const float *B(const dmrt_surrogate_t *s, const Layer &L) { return s->master + L.b_off; }

template <typename T>
dmrt_status conv_fwd(dmrt_surrogate_t *s, const Layer &L, const void *in, void *out, int batch)
{
    SCK(s,
        (lbm::nn::conv3d<T, T, T>(static_cast<const T *>(in), W<T>(s, L), B(s, L), static_cast<T *>(out),
                                  batch, edge(s, L.level), L.cin, L.cout, L.k, L.act, s->stream)),
        "conv3d");
    return DMRT_OK;
}

template <typename T>
dmrt_status forward(dmrt_surrogate_t *s, int batch)
{
    dmrt_status st;
    const int D = s->depth;
    if ((st = conv_fwd<T>(s, enc_a(s, 0), s->x0, s->a[0], batch))) return st;
    if ((st = conv_fwd<T>(s, enc_s(s, 0), s->a[0], s->s[0], batch))) return st;
    for (int l = 1; l <= D; ++l) {
        SCK(s,
            lbm::nn::avgpool2<T>(static_cast<const T *>(s->s[l - 1]), static_cast<T *>(s->pin[l]), batch,
                                 edge(s, l - 1), s->ch[l - 1], s->stream),
            "avgpool2");
        if ((st = conv_fwd<T>(s, enc_a(s, l), s->pin[l], s->a[l], batch))) return st;
        if ((st = conv_fwd<T>(s, enc_s(s, l), s->a[l], s->s[l], batch))) return st;
    }
    for (int l = D - 1; l >= 0; --l) {
        const void *below = (l + 1 == D) ? s->s[D] : s->h[l + 1];
        if ((st = conv_fwd<T>(s, dec_d(s, l), below, s->dd[l], batch))) return st;
        SCK(s,
            lbm::nn::up2_add<T>(static_cast<const T *>(s->dd[l]), static_cast<const T *>(s->s[l]),
                                static_cast<T *>(s->m[l]), batch, edge(s, l + 1), s->ch[l], s->stream),
            "up2_add");
        if ((st = conv_fwd<T>(s, dec_h(s, l), s->m[l], s->h[l], batch))) return st;
    }
    return conv_fwd<T>(s, head(s), s->h[0], s->out, batch);
}

// Backward through one convolution whose output gradient is gin (FP32,
// overwritten): activation derivative, weight and bias gradients, and (if
// gout is not null) the input gradient into gout.
template <typename T>
dmrt_status conv_bwd(dmrt_surrogate_t *s, const Layer &L, const void *in, const void *outv,
                     float *gin, float *gout, int batch)
{
    const int e = edge(s, L.level);
    const long long vox = static_cast<long long>(batch) * e * e * e;
    bool wgrad_done = false;
    bool act_done = false;
    bool bias_done = false;
    if constexpr (std::is_same_v<T, __nv_bfloat16>) {
        // bf16 storage: the output gradient in bf16 feeds the tensor cores
        // (the activation backward, the narrowing and the bias gradient in
        // one pass when the channel count allows; otherwise separately)
        if (lbm::nn::act_backward_narrow_bias<T>(static_cast<const T *>(outv), gin, s->gnarrow, vox, L.cout, L.act,
                                                 s->grad + L.b_off, s->bscratch, s->bscratch_floats,
                                                 s->stream) == cudaSuccess) {
            act_done = true;
            bias_done = true;
        } else if ((vox * L.cout) % 4 == 0 &&
                   lbm::nn::act_backward_narrow<T>(static_cast<const T *>(outv), gin, s->gnarrow, vox * L.cout,
                                                   L.act, s->stream) == cudaSuccess) {
            cudaGetLastError();
            act_done = true;
        } else {
            cudaGetLastError();
            if (L.act)
                SCK(s, lbm::nn::act_backward<T>(static_cast<const T *>(outv), gin, vox * L.cout, s->stream),
                    "act_backward");
            act_done = true;
            SCK(s, lbm::nn::narrow(gin, s->gnarrow, vox * L.cout, s->stream), "narrow");
        }
        if (L.cin % 8 == 0 && L.cout % 8 == 0) {
            SCK(s,
                lbm::nn::conv3d_wgrad_bf16(static_cast<const __nv_bfloat16 *>(in), s->gnarrow, s->grad + L.w_off,
                                           s->scratch, s->scratch_floats, batch, e, L.cin, L.cout, L.k, s->stream),
                "conv3d_wgrad (tensor cores)");
            wgrad_done = true;
        }
    }
    if (L.act && !act_done)
        SCK(s, lbm::nn::act_backward<T>(static_cast<const T *>(outv), gin, vox * L.cout, s->stream),
            "act_backward");
    if (!wgrad_done)
        SCK(s,
            lbm::nn::conv3d_wgrad<T>(static_cast<const T *>(in), gin, s->grad + L.w_off, s->scratch,
                                     s->scratch_floats, batch, e, L.cin, L.cout, L.k, s->stream),
            "conv3d_wgrad");
    if (!bias_done)
        SCK(s, lbm::nn::bias_grad(gin, s->grad + L.b_off, s->scratch, s->scratch_floats, vox, L.cout, s->stream),
            "bias_grad");
    if (gout) {
        SCK(s, lbm::nn::flip_transpose<T>(W<T>(s, L), static_cast<T *>(s->wt), L.k, L.cout, L.cin, s->stream),
            "flip_transpose");
        if constexpr (std::is_same_v<T, __nv_bfloat16>) {
            SCK(s,
                (lbm::nn::conv3d<__nv_bfloat16, __nv_bfloat16, float>(
                    s->gnarrow, static_cast<const __nv_bfloat16 *>(s->wt), nullptr, gout, batch, e, L.cout,
                    L.cin, L.k, 0, s->stream)),
                "conv3d (input gradient)");
        } else {
            SCK(s,
                (lbm::nn::conv3d<float, T, float>(gin, static_cast<const T *>(s->wt), nullptr, gout, batch, e,
                                                  L.cout, L.cin, L.k, 0, s->stream)),
                "conv3d (input gradient)");
        }
    }
    return DMRT_OK;
}

// Loss and gradients for a batch whose features are in x0 and targets in
// s->target; leaves d loss / d params in s->grad and the loss in s->dloss.
template <typename T>
dmrt_status forward_backward(dmrt_surrogate_t *s, int batch)
{
    dmrt_status st;
    if ((st = forward<T>(s, batch))) return st;
    const int D = s->depth;
    const long long fine = static_cast<long long>(batch) * voxels(s, 0);
    // dout in g0
    SCK(s, lbm::nn::mse<T>(static_cast<const T *>(s->out), s->target, s->g0, s->dpart, s->dloss, fine * kOut,
                           s->stream),
        "mse");
    // head: d h_0 into g1
    if ((st = conv_bwd<T>(s, head(s), s->h[0], s->out, s->g0, s->g1, batch))) return st;
    float *gh = s->g1;  // d loss / d h_l (current level)
    float *free_a = s->g0, *free_b = s->g2;
    for (int l = 0; l < D; ++l) {
        // h_l = act(conv3(m_l)): gradient of m_l into free_a
        if ((st = conv_bwd<T>(s, dec_h(s, l), s->m[l], s->h[l], gh, free_a, batch))) return st;
        // m_l = up2(d_l) + s_l: skip gradient, and d d_l (at level l+1) into free_b
        const long long ns = static_cast<long long>(batch) * voxels(s, l) * s->ch[l];
        SCK(s, cudaMemcpyAsync(s->gs[l], free_a, ns * sizeof(float), cudaMemcpyDeviceToDevice, s->stream),
            "copy skip gradient");
        SCK(s, lbm::nn::up2_backward(free_a, free_b, batch, edge(s, l + 1), s->ch[l], s->stream), "up2_backward");
        // d_l = act(conv3(h_{l+1})): gradient of h_{l+1} into free_a
        const void *below = (l + 1 == D) ? s->s[D] : s->h[l + 1];
        if ((st = conv_bwd<T>(s, dec_d(s, l), below, s->dd[l], free_b, free_a, batch))) return st;
        float *t = gh;
        gh = free_a;
        free_a = t;
    }
    // gh = d loss / d s_D (from the decoder)
    {
        const long long n = static_cast<long long>(batch) * voxels(s, D) * s->ch[D];
        SCK(s, cudaMemcpyAsync(s->gs[D], gh, n * sizeof(float), cudaMemcpyDeviceToDevice, s->stream),
            "copy bottleneck gradient");
    }
    for (int l = D; l >= 0; --l) {
        // s_l = act(conv3(a_l)): gradient of a_l into free_a
        if ((st = conv_bwd<T>(s, enc_s(s, l), s->a[l], s->s[l], s->gs[l], free_a, batch))) return st;
        // a_l = act(conv3(p_l)): gradient of p_l (l >= 1) into free_b
        const void *in = (l == 0) ? s->x0 : s->pin[l];
        if ((st = conv_bwd<T>(s, enc_a(s, l), in, s->a[l], free_a, l == 0 ? nullptr : free_b, batch)))
            return st;
        if (l >= 1) {
            // p_l = avgpool2(s_{l-1}): add the pooled gradient to d s_{l-1}
            SCK(s, lbm::nn::avgpool2_backward(free_b, free_a, batch, edge(s, l - 1), s->ch[l - 1], s->stream),
                "avgpool2_backward");
            const long long n = static_cast<long long>(batch) * voxels(s, l - 1) * s->ch[l - 1];
            SCK(s, lbm::nn::add_inplace(s->gs[l - 1], free_a, n, s->stream), "add skip");
        }
    }
    return DMRT_OK;
}

template <typename T>
dmrt_status make_features(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall)
{
    SCK(s, cudaMemcpyAsync(s->dra, ra, batch * sizeof(double), cudaMemcpyHostToDevice, s->stream), "copy Ra");
    SCK(s, cudaMemcpyAsync(s->dwall, wall, batch * sizeof(int), cudaMemcpyHostToDevice, s->stream), "copy wall");
    SCK(s, lbm::nn::features<T>(s->dra, s->dwall, static_cast<T *>(s->x0), batch, s->n, s->stream), "features");
    return DMRT_OK;
}

dmrt_status check_batch(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall)
{
    if (batch < 1 || batch > s->max_batch || !ra || !wall)
        return sfail(s, DMRT_ERR_ARG, "batch must be 1..%d with Ra and wall arrays", s->max_batch);
    for (int b = 0; b < batch; ++b)
        if (!(ra[b] > 0.0) || wall[b] < 1 || wall[b] > 3)
            return sfail(s, DMRT_ERR_ARG, "sample %d: Ra > 0 and wall type 1..3 required", b);
    return DMRT_OK;
}

template <typename F>
dmrt_status by_storage(dmrt_surrogate_t *s, F &&f)
{
    if (s->storage == DMRT_STORE_F32) return f(static_cast<float *>(nullptr));
    return f(static_cast<__nv_bfloat16 *>(nullptr));
}

}  // namespace

extern "C" {

dmrt_status dmrt_surrogate_create(dmrt_surrogate_t **out, const dmrt_surrogate_cfg *cfg)
{
    if (!out || !cfg) return DMRT_ERR_ARG;
    *out = nullptr;
    if (cfg->depth < 1 || cfg->depth > 3 || cfg->grid < 8 || cfg->max_batch < 1) return DMRT_ERR_ARG;
    if ((cfg->grid >> cfg->depth) % 8 != 0 || (cfg->grid >> cfg->depth) < 8) return DMRT_ERR_ARG;
    if (cfg->storage != DMRT_STORE_F32 && cfg->storage != DMRT_STORE_BF16) return DMRT_ERR_ARG;
    for (int l = 0; l <= cfg->depth; ++l) {
        const int c = cfg->channels[l];
        if (c < 4 || c > 128 || 256 % c != 0) return DMRT_ERR_ARG;  // 4, 8, 16, 32, 64 or 128
    }
    dmrt_surrogate_t *s = new (std::nothrow) dmrt_surrogate();
    if (!s) return DMRT_ERR_OOM;
    auto bail = [&](dmrt_status st) {
        dmrt_surrogate_destroy(s);
        return st;
    };
    if (cudaGetDevice(&s->device) != cudaSuccess) return bail(DMRT_ERR_CUDA);
    s->n = cfg->grid;
    s->depth = cfg->depth;
    s->storage = cfg->storage;
    s->max_batch = cfg->max_batch;
    s->seed = cfg->seed;
    for (int l = 0; l <= cfg->depth; ++l) s->ch[l] = cfg->channels[l];
    build_layers(s);
    const int Bm = s->max_batch;
    const size_t es = esize(s);
    auto dalloc = [&](void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    const size_t P = static_cast<size_t>(s->nparams);
    bool ok = dalloc(reinterpret_cast<void **>(&s->master), P * 4) &&
              dalloc(reinterpret_cast<void **>(&s->grad), P * 4) &&
              dalloc(reinterpret_cast<void **>(&s->m1), P * 4) && dalloc(reinterpret_cast<void **>(&s->m2), P * 4) &&
              dalloc(&s->wstore, P * es);
    long long wt_max = 0;
    for (const Layer &L : s->layers)
        wt_max = std::max(wt_max, static_cast<long long>(L.k) * L.k * L.k * L.cin * L.cout);
    ok = ok && dalloc(&s->wt, static_cast<size_t>(wt_max) * es);
    ok = ok && dalloc(&s->x0, static_cast<size_t>(Bm) * voxels(s, 0) * lbm::nn::kFeatures * es);
    s->a.assign(s->depth + 1, nullptr);
    s->s.assign(s->depth + 1, nullptr);
    s->m.assign(s->depth + 1, nullptr);
    s->h.assign(s->depth + 1, nullptr);
    s->dd.assign(s->depth + 1, nullptr);
    s->gs.assign(s->depth + 1, nullptr);
    s->pin.assign(s->depth + 1, nullptr);
    for (int l = 0; l <= s->depth && ok; ++l) {
        const size_t nb = static_cast<size_t>(Bm) * voxels(s, l) * s->ch[l];
        ok = dalloc(&s->a[l], nb * es) && dalloc(&s->s[l], nb * es) && dalloc(&s->h[l], nb * es) &&
             dalloc(reinterpret_cast<void **>(&s->gs[l]), nb * 4);
        ok = ok && dalloc(&s->m[l], nb * es);  // skip sums of the decoder
        if (l > 0)                              // pooled inputs of the encoder
            ok = ok && dalloc(&s->pin[l], static_cast<size_t>(Bm) * voxels(s, l) * s->ch[l - 1] * es);
        if (l < s->depth)
            ok = ok && dalloc(&s->dd[l], static_cast<size_t>(Bm) * voxels(s, l + 1) * s->ch[l] * es);
    }
    long long gmax = 0;
    for (int l = 0; l <= s->depth; ++l)
        gmax = std::max(gmax, static_cast<long long>(Bm) * voxels(s, l) * std::max(s->ch[l], l > 0 ? s->ch[l - 1] : lbm::nn::kFeatures));
    gmax = std::max(gmax, static_cast<long long>(Bm) * voxels(s, 0) * kOut);
    ok = ok && dalloc(&s->out, static_cast<size_t>(Bm) * voxels(s, 0) * kOut * es) &&
         dalloc(reinterpret_cast<void **>(&s->g0), gmax * 4) && dalloc(reinterpret_cast<void **>(&s->g1), gmax * 4) &&
         dalloc(reinterpret_cast<void **>(&s->g2), gmax * 4) &&
         dalloc(reinterpret_cast<void **>(&s->gnarrow), gmax * 2) &&
         dalloc(reinterpret_cast<void **>(&s->target), static_cast<size_t>(Bm) * voxels(s, 0) * kOut * 4);
    s->scratch_floats = std::max<size_t>(static_cast<size_t>(27) * 128 * 128 * 64, 4u << 20);
    s->bscratch_floats = static_cast<size_t>(152) * 4 * 128;
    ok = ok && dalloc(reinterpret_cast<void **>(&s->scratch), s->scratch_floats * 4) &&
         dalloc(reinterpret_cast<void **>(&s->bscratch), s->bscratch_floats * 4) &&
         dalloc(reinterpret_cast<void **>(&s->dpart), 512 * sizeof(double)) &&
         dalloc(reinterpret_cast<void **>(&s->dloss), sizeof(double)) &&
         dalloc(reinterpret_cast<void **>(&s->dra), Bm * sizeof(double)) &&
         dalloc(reinterpret_cast<void **>(&s->dwall), Bm * sizeof(int));
    if (!ok) return bail(DMRT_ERR_OOM);
    if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess) return bail(DMRT_ERR_CUDA);
    s->stream = s->own;
    std::vector<float> p;
    init_params(s, p);
    if (dmrt_surrogate_set_params(s, p.data(), s->nparams) != DMRT_OK) return bail(DMRT_ERR_CUDA);
    *out = s;
    return DMRT_OK;
}

void dmrt_surrogate_destroy(dmrt_surrogate_t *s)
{
    if (!s) return;
    SGuard g(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    void *ptrs[] = {s->master, s->grad, s->m1, s->m2, s->wstore, s->wt, s->x0, s->out, s->g0, s->g1,
                    s->g2, s->gnarrow, s->target, s->scratch, s->bscratch, s->dpart, s->dloss, s->dra, s->dwall};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto *v : {&s->a, &s->s, &s->m, &s->h, &s->dd, &s->pin})
        for (void *p : *v)
            if (p) cudaFree(p);
    for (float *p : s->gs)
        if (p) cudaFree(p);
    if (s->own) cudaStreamDestroy(s->own);
    delete s;
}

long long dmrt_surrogate_param_count(const dmrt_surrogate_t *s) { return s ? s->nparams : -1; }

dmrt_status dmrt_surrogate_set_stream(dmrt_surrogate_t *s, void *stream)
{
    if (!s) return DMRT_ERR_ARG;
    SGuard g(s->device);
    SCK(s, cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    s->stream = stream ? static_cast<cudaStream_t>(stream) : s->own;
    return DMRT_OK;
}

dmrt_status dmrt_surrogate_set_params(dmrt_surrogate_t *s, const float *params, long long count)
{
    if (!s || !params || count != s->nparams) return DMRT_ERR_ARG;
    SGuard g(s->device);
    const size_t P = static_cast<size_t>(s->nparams);
    SCK(s, cudaMemcpyAsync(s->master, params, P * 4, cudaMemcpyHostToDevice, s->stream), "copy params");
    SCK(s, cudaMemsetAsync(s->m1, 0, P * 4, s->stream), "reset Adam");
    SCK(s, cudaMemsetAsync(s->m2, 0, P * 4, s->stream), "reset Adam");
    s->step = 0;
    dmrt_status st = by_storage(s, [&](auto *tp) -> dmrt_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        SCK(s, lbm::nn::copy_to_store<T>(s->master, static_cast<T *>(s->wstore), s->nparams, s->stream),
            "copy to storage");
        return DMRT_OK;
    });
    if (st != DMRT_OK) return st;
    SCK(s, cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_surrogate_get_params(dmrt_surrogate_t *s, float *params, long long count)
{
    if (!s || !params || count != s->nparams) return DMRT_ERR_ARG;
    SGuard g(s->device);
    SCK(s, cudaMemcpyAsync(params, s->master, static_cast<size_t>(count) * 4, cudaMemcpyDeviceToHost, s->stream),
        "copy params");
    SCK(s, cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

dmrt_status dmrt_surrogate_predict(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                   float *out, int on_device)
{
    if (!s || !out) return DMRT_ERR_ARG;
    dmrt_status st = check_batch(s, batch, ra, wall);
    if (st != DMRT_OK) return st;
    SGuard g(s->device);
    const long long len = static_cast<long long>(batch) * voxels(s, 0) * kOut;
    st = by_storage(s, [&](auto *tp) -> dmrt_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        dmrt_status r = make_features<T>(s, batch, ra, wall);
        if (r != DMRT_OK) return r;
        r = forward<T>(s, batch);
        if (r != DMRT_OK) return r;
        SCK(s, lbm::nn::widen<T>(static_cast<const T *>(s->out), s->g0, len, s->stream), "widen");
        return DMRT_OK;
    });
    if (st != DMRT_OK) return st;
    SCK(s, cudaMemcpyAsync(out, s->g0, len * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s->stream),
        "copy prediction");
    SCK(s, cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return DMRT_OK;
}

// Shared part of train_step / gradients / loss: features, targets, and the
// forward (+ backward) pass.
static dmrt_status run_batch(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                             const float *target, bool backward)
{
    dmrt_status st = check_batch(s, batch, ra, wall);
    if (st != DMRT_OK) return st;
    if (!target) return DMRT_ERR_ARG;
    const long long len = static_cast<long long>(batch) * voxels(s, 0) * kOut;
    SCK(s, cudaMemcpyAsync(s->target, target, len * 4, cudaMemcpyDeviceToDevice, s->stream), "copy target");
    return by_storage(s, [&](auto *tp) -> dmrt_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        dmrt_status r = make_features<T>(s, batch, ra, wall);
        if (r != DMRT_OK) return r;
        if (backward) return forward_backward<T>(s, batch);
        r = forward<T>(s, batch);
        if (r != DMRT_OK) return r;
        SCK(s, lbm::nn::mse<T>(static_cast<const T *>(s->out), s->target, nullptr, s->dpart, s->dloss, len,
                               s->stream),
            "mse");
        return DMRT_OK;
    });
}

static dmrt_status read_loss(dmrt_surrogate_t *s, double *loss)
{
    double l = 0.0;
    SCK(s, cudaMemcpyAsync(&l, s->dloss, sizeof l, cudaMemcpyDeviceToHost, s->stream), "copy loss");
    SCK(s, cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    if (loss) *loss = l;
    return DMRT_OK;
}

dmrt_status dmrt_surrogate_train_step(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                      const float *target, float lr, double *loss)
{
    if (!s || !(lr > 0.f)) return DMRT_ERR_ARG;
    SGuard g(s->device);
    dmrt_status st = run_batch(s, batch, ra, wall, target, true);
    if (st != DMRT_OK) return st;
    s->step++;
    st = by_storage(s, [&](auto *tp) -> dmrt_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        SCK(s, lbm::nn::adam<T>(s->master, static_cast<T *>(s->wstore), s->grad, s->m1, s->m2, s->nparams, lr,
                                0.9f, 0.999f, 1e-8f, s->step, s->stream),
            "adam");
        return DMRT_OK;
    });
    if (st != DMRT_OK) return st;
    return loss ? read_loss(s, loss) : DMRT_OK;
}

dmrt_status dmrt_surrogate_gradients(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                     const float *target, float *grad, double *loss)
{
    if (!s || !grad) return DMRT_ERR_ARG;
    SGuard g(s->device);
    dmrt_status st = run_batch(s, batch, ra, wall, target, true);
    if (st != DMRT_OK) return st;
    SCK(s, cudaMemcpyAsync(grad, s->grad, static_cast<size_t>(s->nparams) * 4, cudaMemcpyDeviceToHost, s->stream),
        "copy gradients");
    return read_loss(s, loss);
}

dmrt_status dmrt_surrogate_loss(dmrt_surrogate_t *s, int batch, const double *ra, const int *wall,
                                const float *target, double *loss)
{
    if (!s || !loss) return DMRT_ERR_ARG;
    SGuard g(s->device);
    dmrt_status st = run_batch(s, batch, ra, wall, target, false);
    if (st != DMRT_OK) return st;
    return read_loss(s, loss);
}

dmrt_status dmrt_surrogate_target_from_fields(const float *u, const float *theta, const float *rho, int n,
                                              double uc, float *target, void *stream)
{
    if (!u || !theta || !target || n < 1 || !(uc > 0.0)) return DMRT_ERR_ARG;
    const long long vox = static_cast<long long>(n) * n * n;
    if (lbm::nn::target_from_fields(u, theta, rho, vox, static_cast<float>(1.0 / uc), target,
                                    static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return DMRT_ERR_CUDA;
    return DMRT_OK;
}

dmrt_status dmrt_warm_start(dmrt_t *h, dmrt_surrogate_t *s, double Ra, int wall)
{
    if (!h || !s) return DMRT_ERR_ARG;
    dmrt_params p;
    dmrt_status st = dmrt_get_params(h, &p);
    if (st != DMRT_OK) return st;
    if (p.nx != p.ny || p.ny != p.nz)
        return sfail(s, DMRT_ERR_ARG, "warm start needs a cubic cavity (got %dx%dx%d)", p.nx, p.ny, p.nz);
    SGuard g(s->device);
    // the prediction at the network grid, FP32 channels-last, in g1
    const long long len = voxels(s, 0) * kOut;
    st = by_storage(s, [&](auto *tp) -> dmrt_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        dmrt_status r = make_features<T>(s, 1, &Ra, &wall);
        if (r != DMRT_OK) return r;
        r = check_batch(s, 1, &Ra, &wall);
        if (r != DMRT_OK) return r;
        r = forward<T>(s, 1);
        if (r != DMRT_OK) return r;
        SCK(s, lbm::nn::widen<T>(static_cast<const T *>(s->out), s->g1, len, s->stream), "widen");
        return DMRT_OK;
    });
    if (st != DMRT_OK) return st;
    // trilinear resampling to the cavity grid; u scaled back by u_c
    const int N = p.nx;
    const long long vox = static_cast<long long>(N) * N * N;
    float *fields = nullptr;  // planar rho, u_x, u_y, u_z, theta
    SCK(s, cudaMalloc(&fields, static_cast<size_t>(vox) * 5 * 4), "cudaMalloc(warm start)");
    const float uc = static_cast<float>(std::sqrt(p.gbeta * p.ny));
    const int plane[5] = {1, 2, 3, 4, 0};
    const float scale[5] = {uc, uc, uc, 1.f, 3.f * uc * uc};
    const float offset[5] = {0.f, 0.f, 0.f, 0.f, 1.f};
    cudaError_t e = lbm::nn::resample<float>(s->g1, s->n, kOut, fields, N, plane, scale, offset, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaFree(fields);
        return sfail(s, DMRT_ERR_CUDA, "warm start: %s", cudaGetErrorString(e));
    }
    st = dmrt_init_fields(h, fields, fields + vox, fields + 4 * vox, 1);
    if (st == DMRT_OK) st = dmrt_sync(h);
    cudaFree(fields);
    return st;
}

const char *dmrt_surrogate_last_error(const dmrt_surrogate_t *s)
{
    if (!s) return "null surrogate";
    return s->err.c_str();
}

int dmrt_nn_tensor_core_errors(int reset) { return lbm::nn::tensor_core_errors(reset != 0); }

dmrt_status dmrt_nn_conv3d(const void *x, const void *w, const float *bias, void *y, int batch, int n,
                           int cin, int cout, int k, int act, int storage, int out_f32, void *stream)
{
    if (!x || !w || !y || batch < 1 || n < 8 || n % 8 != 0 || cin < 1 || cout < 1 || (k != 1 && k != 3))
        return DMRT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (storage == DMRT_STORE_BF16) {
        const auto *xb = static_cast<const __nv_bfloat16 *>(x);
        const auto *wb = static_cast<const __nv_bfloat16 *>(w);
        if (out_f32)
            e = lbm::nn::conv3d<__nv_bfloat16, __nv_bfloat16, float>(xb, wb, bias, static_cast<float *>(y), batch,
                                                                     n, cin, cout, k, act, st);
        else
            e = lbm::nn::conv3d<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16>(
                xb, wb, bias, static_cast<__nv_bfloat16 *>(y), batch, n, cin, cout, k, act, st);
    } else if (storage == DMRT_STORE_F32) {
        e = lbm::nn::conv3d<float, float, float>(static_cast<const float *>(x), static_cast<const float *>(w),
                                                 bias, static_cast<float *>(y), batch, n, cin, cout, k, act, st);
    } else {
        return DMRT_ERR_ARG;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? DMRT_OK : DMRT_ERR_CUDA;
}

}  // extern "C"
