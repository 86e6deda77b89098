// api_learned.cu -- C ABI of the learned far-field correction: the MLP
// object (weights, normalisation, AdamW state), training samples drawn from
// a context (walk features at a coarse theta + direct-sum labels), training,
// and forces / steps that use the coarse walk plus the correction, judged
// every call by a sampled direct sum with a fine-theta fallback.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

using namespace bonsai;

struct bonsai_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *P = nullptr, *norm = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    uint32_t *idx = nullptr;
    long long idx_cap = 0;
    int step = 0;
    bool fitted = false;
    std::string err;
};

namespace bonsai {

__global__ void k_judge_targets(uint32_t *targets, int ntar, long long n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ntar) targets[k] = (uint32_t)(((long long)k * n) / ntar);
}

// Stratified judge sample: every (n / ntar)-th body in key order.
cudaError_t launch_judge_targets(Ctx &c) {
    const int ntar = (int)(c.n < JUDGE_MAX ? c.n : JUDGE_MAX);
    if (c.judge_n == ntar) return cudaSuccess;
    k_judge_targets<<<(ntar + 255) / 256, 256, 0, c.stream>>>(c.judge_targets, ntar, c.n);
    c.judge_n = ntar;
    return cudaGetLastError();
}

// Decides whether this learned evaluation is judged: every k-th one counted
// from the last bonsai_set_learned / bonsai_set_judge_interval (k = 0: never,
// and then never a fallback).
__global__ void k_judge_gate(DevState *st, int every) {
    if (threadIdx.x != 0) return;
    const unsigned t = st->judge_tick;
    st->judge_on = (every > 0 && t % (unsigned)every == 0u) ? 1u : 0u;
    if (every <= 0) st->fallback = 0u;
    st->judge_tick = t + 1u;
}

__global__ void k_gated_walk_reset(DevState *st) {
    if (threadIdx.x == 0 && st->fallback) { st->walk_next = 0; st->walk_next2 = 0; }
}

cudaError_t launch_gated_walk_reset(Ctx &c) {
    k_gated_walk_reset<<<1, 32, 0, c.stream>>>(c.st);
    return cudaGetLastError();
}

// Coarse walk with features -> MLP correction -> judge (direct sum at the
// stratified sample, p99 vs budget; on the evaluations the interval selects)
// -> fine-theta walk, which runs only while the last judgement asked for the
// fallback.  No host synchronisation.
cudaError_t pipeline_learned_forces(Ctx &c, float eps) {
    cudaError_t e;
    const unsigned *gate = &c.st->judge_on;
    k_judge_gate<<<1, 32, 0, c.stream>>>(c.st, c.judge_every);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_open_radius(c, c.theta_coarse)) != cudaSuccess) return e;
    if ((e = launch_walk(c, eps, true)) != cudaSuccess) return e;
    if ((e = launch_mlp_infer(c, c.mlp_P, c.mlp_norm)) != cudaSuccess) return e;
    if ((e = launch_judge_targets(c)) != cudaSuccess) return e;
    if ((e = launch_direct(c, c.judge_targets, c.judge_n, eps, c.judge_partial, JUDGE_SPLIT, c.judge_direct,
                           gate)) != cudaSuccess)
        return e;
    if ((e = launch_judge(c, c.judge_targets, c.judge_n, c.judge_direct, c.p99_budget, gate)) != cudaSuccess)
        return e;
    if ((e = launch_gated_walk_reset(c)) != cudaSuccess) return e;
    if ((e = launch_open_radius(c, c.theta_fine, &c.st->fallback)) != cudaSuccess) return e;
    return launch_walk(c, eps, false, &c.st->fallback);
}

}  // namespace bonsai

namespace {

int mfail(bonsai_mlp *m, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    cudaGetLastError();
    std::string s = what;
    if (e != cudaSuccess) { s += ": "; s += cudaGetErrorString(e); }
    if (m) m->err = s;
    return code;
}

int cfail(bonsai_ctx *ctx, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    cudaGetLastError();
    std::string s = what;
    if (e != cudaSuccess) { s += ": "; s += cudaGetErrorString(e); }
    if (ctx) ctx->c.err = s;
    return code;
}

#define MCK(call)                                                                 \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) return mfail(m, BONSAI_ERR_CUDA, #call, _e);        \
    } while (0)
#define CCK(call)                                                                 \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) return cfail(ctx, BONSAI_ERR_CUDA, #call, _e);      \
    } while (0)

// xorshift64* and a Box-Muller normal for the weight initialisation and the
// epoch shuffles (host side, seeded).
struct Rng {
    unsigned long long s;
    explicit Rng(unsigned long long seed) : s(seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull) {
        if (!s) s = 1;
    }
    unsigned long long next() {
        s ^= s >> 12; s ^= s << 25; s ^= s >> 27;
        return s * 0x2545F4914F6CDD1Dull;
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    double normal() {
        double u1 = uniform(), u2 = uniform();
        if (u1 < 1e-300) u1 = 1e-300;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

int ensure_idx(bonsai_mlp *m, long long n) {
    if (n <= m->idx_cap) return BONSAI_OK;
    if (m->idx) cudaFree(m->idx);
    m->idx = nullptr;
    MCK(cudaMalloc(&m->idx, sizeof(uint32_t) * (size_t)n));
    m->idx_cap = n;
    return BONSAI_OK;
}

// Copies host rows to a temporary device buffer when needed.
struct DevView {
    const float *p = nullptr;
    float *owned = nullptr;
    ~DevView() { if (owned) cudaFree(owned); }
};

cudaError_t to_device(DevView &d, const float *src, size_t count, int on_device, cudaStream_t s) {
    if (on_device) { d.p = src; return cudaSuccess; }
    cudaError_t e = cudaMalloc(&d.owned, count * sizeof(float));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d.owned, src, count * sizeof(float), cudaMemcpyHostToDevice, s);
    d.p = d.owned;
    return e;
}

}  // namespace

extern "C" {

int bonsai_mlp_create(bonsai_mlp **out, unsigned long long seed) {
    if (!out) return BONSAI_ERR_INVALID_ARG;
    *out = nullptr;
    bonsai_mlp *m = new (std::nothrow) bonsai_mlp();
    if (!m) return BONSAI_ERR_OOM;
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaStreamCreate(&m->stream);
    float *buf = nullptr;
    const size_t total = 4 * (size_t)MLP_NPARAM + MLP_NNORM + 1;
    if (e == cudaSuccess) e = cudaMalloc(&buf, total * sizeof(float));
    if (e != cudaSuccess) {
        if (m->stream) cudaStreamDestroy(m->stream);
        delete m;
        cudaGetLastError();
        return BONSAI_ERR_CUDA;
    }
    m->P = buf; m->grad = buf + MLP_NPARAM; m->m = buf + 2 * MLP_NPARAM; m->v = buf + 3 * MLP_NPARAM;
    m->norm = buf + 4 * MLP_NPARAM; m->loss = m->norm + MLP_NNORM;
    // He-normal weights (std sqrt(2 / fan_in)), zero biases, identity
    // normalisation.
    std::vector<float> h(total, 0.f);
    Rng r(seed);
    const int fan[3] = {MLP_IN, MLP_H, MLP_H}, rows[3] = {MLP_H, MLP_H, MLP_OUT};
    int off = 0;
    for (int l = 0; l < 3; l++) {
        const double sd = std::sqrt(2.0 / fan[l]);
        for (int i = 0; i < rows[l] * fan[l]; i++) h[off + i] = (float)(sd * r.normal());
        off += rows[l] * fan[l] + rows[l];
    }
    for (int k = 0; k < MLP_IN; k++) h[4 * MLP_NPARAM + MLP_IN + k] = 1.f;
    h[4 * MLP_NPARAM + 2 * MLP_IN] = 1.f;
    e = cudaMemcpy(buf, h.data(), total * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { bonsai_mlp_destroy(m); cudaGetLastError(); return BONSAI_ERR_CUDA; }
    *out = m;
    return BONSAI_OK;
}

void bonsai_mlp_destroy(bonsai_mlp *m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->P) cudaFree(m->P);
    if (m->idx) cudaFree(m->idx);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

const char *bonsai_mlp_last_error(const bonsai_mlp *m) { return m ? m->err.c_str() : ""; }

int bonsai_mlp_set_params(bonsai_mlp *m, const float *params, const float *norm) {
    if (!m) return BONSAI_ERR_INVALID_ARG;
    if (params) MCK(cudaMemcpy(m->P, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    if (norm) { MCK(cudaMemcpy(m->norm, norm, MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice)); m->fitted = true; }
    return BONSAI_OK;
}

int bonsai_mlp_get_params(bonsai_mlp *m, float *params, float *norm) {
    if (!m) return BONSAI_ERR_INVALID_ARG;
    MCK(cudaStreamSynchronize(m->stream));
    if (params) MCK(cudaMemcpy(params, m->P, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (norm) MCK(cudaMemcpy(norm, m->norm, MLP_NNORM * sizeof(float), cudaMemcpyDeviceToHost));
    return BONSAI_OK;
}

int bonsai_mlp_fit_norm(bonsai_mlp *m, const float *X, const float *Y, long long n, int on_device) {
    if (!m || !X || !Y || n < 1 || n > (1ll << 30)) return BONSAI_ERR_INVALID_ARG;
    DevView dx, dy;
    MCK(to_device(dx, X, (size_t)n * MLP_IN, on_device, m->stream));
    MCK(to_device(dy, Y, (size_t)n * MLP_OUT, on_device, m->stream));
    MCK(launch_feature_stats(m->stream, dx.p, dy.p, (int)n, m->norm));
    MCK(cudaStreamSynchronize(m->stream));
    m->fitted = true;
    return BONSAI_OK;
}

int bonsai_mlp_predict(bonsai_mlp *m, const float *X, float *Y, long long n, int on_device) {
    if (!m || !X || !Y || n < 1 || n > (1ll << 30)) return BONSAI_ERR_INVALID_ARG;
    DevView dx;
    MCK(to_device(dx, X, (size_t)n * MLP_IN, on_device, m->stream));
    float *dy = Y, *owned = nullptr;
    if (!on_device) { MCK(cudaMalloc(&owned, (size_t)n * MLP_OUT * sizeof(float))); dy = owned; }
    cudaError_t e = launch_mlp_rows(m->stream, m->P, m->norm, dx.p, dy, (int)n);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(Y, dy, (size_t)n * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (owned) cudaFree(owned);
    if (e != cudaSuccess) return mfail(m, BONSAI_ERR_CUDA, "bonsai_mlp_predict", e);
    return BONSAI_OK;
}

int bonsai_mlp_grad(bonsai_mlp *m, const float *X, const float *Y, long long n, int on_device, float *grad,
                    float *loss) {
    if (!m || !X || !Y || n < 1 || n > (1ll << 24)) return BONSAI_ERR_INVALID_ARG;
    DevView dx, dy;
    MCK(to_device(dx, X, (size_t)n * MLP_IN, on_device, m->stream));
    MCK(to_device(dy, Y, (size_t)n * MLP_OUT, on_device, m->stream));
    int r = ensure_idx(m, n);
    if (r) return r;
    std::vector<uint32_t> id((size_t)n);
    for (long long i = 0; i < n; i++) id[(size_t)i] = (uint32_t)i;
    MCK(cudaMemcpyAsync(m->idx, id.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice, m->stream));
    MCK(cudaMemsetAsync(m->grad, 0, MLP_NPARAM * sizeof(float), m->stream));
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
    MCK(launch_mlp_grad(m->stream, m->P, m->norm, dx.p, dy.p, m->idx, (int)n, m->grad, m->loss));
    if (grad) MCK(cudaMemcpyAsync(grad, m->grad, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (loss) MCK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return BONSAI_OK;
}

int bonsai_mlp_train(bonsai_mlp *m, const float *X, const float *Y, long long n, int on_device, int epochs,
                     int batch, float lr, float wd, unsigned long long seed, float *loss_per_epoch) {
    if (!m || !X || !Y || n < 1 || n > (1ll << 30) || epochs < 1 || batch < 1 || !(lr > 0.f))
        return BONSAI_ERR_INVALID_ARG;
    DevView dx, dy;
    MCK(to_device(dx, X, (size_t)n * MLP_IN, on_device, m->stream));
    MCK(to_device(dy, Y, (size_t)n * MLP_OUT, on_device, m->stream));
    if (!m->fitted) {
        MCK(launch_feature_stats(m->stream, dx.p, dy.p, (int)n, m->norm));
        m->fitted = true;
    }
    int r = ensure_idx(m, n);
    if (r) return r;
    Rng rng(seed);
    std::vector<uint32_t> perm((size_t)n);
    for (long long i = 0; i < n; i++) perm[(size_t)i] = (uint32_t)i;
    const long long nb = (n + batch - 1) / batch;
    for (int ep = 0; ep < epochs; ep++) {
        for (long long i = n - 1; i > 0; i--) {               // Fisher-Yates
            const long long j = (long long)(rng.next() % (unsigned long long)(i + 1));
            std::swap(perm[(size_t)i], perm[(size_t)j]);
        }
        MCK(cudaMemcpyAsync(m->idx, perm.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice, m->stream));
        MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
        for (long long b = 0; b < nb; b++) {
            const int bsz = (int)std::min<long long>(batch, n - b * batch);
            MCK(cudaMemsetAsync(m->grad, 0, MLP_NPARAM * sizeof(float), m->stream));
            MCK(launch_mlp_grad(m->stream, m->P, m->norm, dx.p, dy.p, m->idx + b * batch, bsz, m->grad, m->loss));
            MCK(launch_adamw(m->stream, m->P, m->grad, m->m, m->v, lr, wd, ++m->step));
        }
        if (loss_per_epoch) {
            float l = 0.f;
            MCK(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
            MCK(cudaStreamSynchronize(m->stream));
            loss_per_epoch[ep] = l / (float)nb;
        }
        // the host permutation buffer is reused next epoch: wait for the copy
        MCK(cudaStreamSynchronize(m->stream));
    }
    return BONSAI_OK;
}

int bonsai_learn_samples(bonsai_ctx *ctx, float theta, float eps, int ntar, unsigned long long seed, float *X,
                         float *Y, uint32_t *ids, int on_device) {
    if (!ctx || !X || !Y || ntar < 1 || ntar > JUDGE_MAX) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.moments_ready)
        return cfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_learn_samples: call bonsai_build and bonsai_multipoles first");
    if (ntar > c.n) ntar = (int)c.n;
    // ntar distinct sorted positions (partial Fisher-Yates on the host).
    std::vector<uint32_t> pool((size_t)c.n);
    for (long long i = 0; i < c.n; i++) pool[(size_t)i] = (uint32_t)i;
    Rng rng(seed);
    for (int k = 0; k < ntar; k++) {
        const long long j = k + (long long)(rng.next() % (unsigned long long)(c.n - k));
        std::swap(pool[(size_t)k], pool[(size_t)j]);
    }
    uint32_t *tg = c.judge_targets;   // borrowed: the judge sample is rebuilt on its next use
    c.judge_n = 0;
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    c.graph_n = -1;
    CCK(cudaMemcpyAsync(tg, pool.data(), sizeof(uint32_t) * ntar, cudaMemcpyHostToDevice, c.stream));
    CCK(launch_reset(c));
    CCK(launch_open_radius(c, theta));
    CCK(launch_walk(c, eps, true));
    CCK(launch_direct(c, tg, ntar, eps, c.judge_partial, JUDGE_SPLIT, c.judge_direct));
    float *dX = X, *dY = Y, *owned = nullptr;
    uint32_t *dI = ids;
    if (!on_device) {
        CCK(cudaMalloc(&owned, (size_t)ntar * (MLP_IN + MLP_OUT + 1) * sizeof(float)));
        dX = owned; dY = owned + (size_t)ntar * MLP_IN;
        dI = ids ? (uint32_t *)(owned + (size_t)ntar * (MLP_IN + MLP_OUT)) : nullptr;
    }
    cudaError_t e = launch_gather_features(c, tg, ntar, dX, dI);
    if (e == cudaSuccess) e = launch_labels(c, tg, ntar, c.judge_direct, dY);
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(X, dX, (size_t)ntar * MLP_IN * sizeof(float), cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Y, dY, (size_t)ntar * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess && ids)
            e = cudaMemcpyAsync(ids, dI, (size_t)ntar * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (owned) cudaFree(owned);
    if (e != cudaSuccess) return cfail(ctx, BONSAI_ERR_CUDA, "bonsai_learn_samples", e);
    c.have_acc = true;
    c.theta = theta;
    c.eps = eps;
    return BONSAI_OK;
}

int bonsai_judge(bonsai_ctx *ctx, float eps, float *p99) {
    if (!ctx || !p99) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_acc) return cfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_judge: no forces yet");
    CCK(launch_judge_targets(c));
    CCK(launch_direct(c, c.judge_targets, c.judge_n, eps, c.judge_partial, JUDGE_SPLIT, c.judge_direct));
    CCK(launch_judge(c, c.judge_targets, c.judge_n, c.judge_direct, 1e30f));
    CCK(cudaMemcpyAsync(p99, &c.st->judge_p99, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
    CCK(cudaStreamSynchronize(c.stream));
    return BONSAI_OK;
}

int bonsai_set_learned(bonsai_ctx *ctx, const bonsai_mlp *m, float theta_coarse, float theta_fine,
                       float p99_budget) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (m && (!(theta_coarse > 0.f && theta_coarse <= 1.15f) || !(theta_fine > 0.f && theta_fine <= 1.15f) ||
              !(p99_budget >= 0.f)))
        return cfail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_set_learned: need thetas in (0, 1.15] and budget >= 0");
    c.mlp_P = m ? m->P : nullptr;
    c.mlp_norm = m ? m->norm : nullptr;
    c.theta_coarse = theta_coarse;
    c.theta_fine = theta_fine;
    c.p99_budget = p99_budget;
    CCK(cudaMemsetAsync(&c.st->fallback, 0, 3 * sizeof(unsigned), c.stream));   // fallback, tick, on
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    c.graph_n = -1;
    return BONSAI_OK;
}

int bonsai_set_judge_interval(bonsai_ctx *ctx, int every) {
    if (!ctx || every < 0) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    c.judge_every = every;
    CCK(cudaMemsetAsync(&c.st->fallback, 0, 3 * sizeof(unsigned), c.stream));
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    c.graph_n = -1;
    return BONSAI_OK;
}

int bonsai_forces_learned(bonsai_ctx *ctx, float eps, float *acc, float *pot, int on_device) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.mlp_P) return cfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_forces_learned: call bonsai_set_learned first");
    if (!c.moments_ready)
        return cfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_forces_learned: call bonsai_build and bonsai_multipoles first");
    if (!(eps > 0.f)) return cfail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_forces_learned: eps > 0");
    CCK(launch_reset(c));
    CCK(pipeline_learned_forces(c, eps));
    c.have_acc = true;
    c.eps = eps;
    if (acc || pot) {
        if (on_device) {
            CCK(launch_scatter_forces(c, acc, pot));
        } else {
            float *sa = c.stage, *sp = c.stage + 3 * c.n;
            CCK(launch_scatter_forces(c, acc ? sa : nullptr, pot ? sp : nullptr));
            if (acc) CCK(cudaMemcpyAsync(acc, sa, 12 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
            if (pot) CCK(cudaMemcpyAsync(pot, sp, 4 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
            CCK(cudaStreamSynchronize(c.stream));
        }
    }
    return BONSAI_OK;
}

int bonsai_get_judge(bonsai_ctx *ctx, float *p99, int *fell_back) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    float v = 0.f;
    unsigned f = 0;
    CCK(cudaMemcpyAsync(&v, &c.st->judge_p99, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
    CCK(cudaMemcpyAsync(&f, &c.st->fallback, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    CCK(cudaStreamSynchronize(c.stream));
    if (p99) *p99 = v;
    if (fell_back) *fell_back = (int)f;
    return BONSAI_OK;
}

}  // extern "C"
