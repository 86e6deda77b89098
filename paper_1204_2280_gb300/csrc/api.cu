// api.cu -- the C ABI of libbonsai (declared in include/bonsai.h).
//
// All device memory of a context comes from one cudaMalloc arena sized for
// the body count; every stage is a kernel launch ordered on the context's
// stream; bonsai_step contains no host synchronisation and is replayed from a
// CUDA graph.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

using namespace bonsai;

static thread_local std::string g_create_err;

namespace bonsai {
// Errors of calls without a context (bonsai_create, bonsai_sort_keys_static).
void set_global_error(const char *msg) { g_create_err = msg; }
}  // namespace bonsai

static int fail(bonsai_ctx *ctx, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    cudaGetLastError();   // a failed runtime call must not leak into the next launch check
    std::string s = what;
    if (e != cudaSuccess) {
        s += ": ";
        s += cudaGetErrorString(e);
    }
    if (ctx) ctx->c.err = s; else g_create_err = s;
    return code;
}

#define CK(call)                                                               \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return fail(ctx, BONSAI_ERR_CUDA, #call, _e);   \
    } while (0)

namespace {

struct Arena {
    size_t off = 0;
    template <class T> void take(T *&p, size_t count, std::vector<std::pair<void **, size_t>> &plan) {
        off = (off + 255) & ~size_t(255);
        plan.push_back({(void **)&p, off});
        off += count * sizeof(T);
    }
};

void drop_graph(CallGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = CallGraph{};
}

void free_bodies(Ctx &c) {
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    drop_graph(c.build_graph); drop_graph(c.mom_graph); drop_graph(c.forces_graph);
    if (c.pos4) cudaFree(c.pos4);
    c.pos4 = nullptr;
    c.ncap = 0;
}

cudaError_t alloc_bodies(Ctx &c, long long n) {
    free_bodies(c);
    const long long ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    const long long nbb = (n + BUILD_BODIES - 1) / BUILD_BODIES;
    // Cells: at most n leaves and n/(nleaf+1) internal cells per level.
    const long long ccap = n + (long long)MAX_LEVEL * (n / (c.nleaf + 1)) + 64;
    std::vector<std::pair<void **, size_t>> plan;
    Arena a;
    a.take(c.pos4, n, plan); a.take(c.vel4, n, plan); a.take(c.acc4, n, plan);
    a.take(c.pos4_alt, n, plan); a.take(c.vel4_alt, n, plan);
    a.take(c.id, n, plan); a.take(c.id_alt, n, plan); a.take(c.sysid, n, plan);
    a.take(c.keys, n, plan); a.take(c.keys_alt, n, plan);
    a.take(c.vals, n, plan); a.take(c.vals_alt, n, plan);
    a.take(c.tile_status, (size_t)(SORT_PASSES + 1) * ntiles * SORT_RADIX, plan);
    a.take(c.blockcount, (size_t)BUILD_ROWS * nbb, plan);
    a.take(c.build_entries, (size_t)nbb * BUILD_BODIES, plan);
    a.take(c.cell_body, ccap, plan); a.take(c.cell_link, ccap, plan);
    a.take(c.cell_level, ccap, plan); a.take(c.cell_parent, ccap, plan);
    a.take(c.cell_done, ccap, plan); a.take(c.cell_cb, ccap, plan); a.take(c.cell_start, ccap, plan);
    a.take(c.mono, ccap, plan); a.take(c.quadA, ccap, plan); a.take(c.quadB, ccap, plan);
    a.take(c.test, ccap, plan); a.take(c.delta, ccap, plan); a.take(c.cext, ccap, plan);
    a.take(c.shadow, 10 * (size_t)(ccap < 585 * MAX_SYSTEMS ? ccap : 585 * MAX_SYSTEMS), plan);   // FP64 root terms of the level-1 cells
    a.take(c.groups, n, plan); a.take(c.groups_raw, n, plan);
    a.take(c.group_lvl, n, plan); a.take(c.group_flag, n, plan); a.take(c.group_bcount, (n + PACK_THREADS - 1) / PACK_THREADS, plan);
    a.take(c.counts, n, plan); a.take(c.feat, FEAT_STRIDE * (size_t)n, plan);
    const long long stage_floats = 7 * n > STAGE_MIN_FLOATS ? 7 * n : STAGE_MIN_FLOATS;
    a.take(c.stage, (size_t)stage_floats, plan);
    a.take(c.judge_targets, JUDGE_MAX, plan); a.take(c.judge_direct, JUDGE_MAX, plan);
    a.take(c.judge_partial, (size_t)JUDGE_SPLIT * JUDGE_MAX, plan);
    char *base = nullptr;
    if (c.arena_limit > 0 && (long long)a.off > c.arena_limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&base, a.off);
    if (e != cudaSuccess) return e;
    for (auto &p : plan) *p.first = base + p.second;
    c.ncap = n;
    c.arena_gen++;
    c.stage_floats = stage_floats;
    c.ntiles = (int)ntiles;
    c.nbblocks = (int)nbb;
    c.ccap = ccap;
    c.judge_n = 0;
    return cudaMemsetAsync(base, 0, a.off, c.stream);
}

// The cell count of the current tree, read back (synchronises the stream):
// it sizes the multipole launch (any count stays correct; the launch loops).
cudaError_t refresh_cells_hint(Ctx &c) {
    unsigned nc = 0;
    cudaError_t e = cudaMemcpyAsync(&nc, &c.st->ncells, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) c.cells_hint = nc;
    return e;
}

// keys -> sort -> reorder -> build; the domain accumulators must hold the
// bounding box of the pre-sort positions.
// The launches of body() on the context's stream: direct the first time a
// key is seen, captured into a graph the second time, replayed from then on
// while the key holds (the first run also sets up what the launches cache:
// function attributes, occupancy).  A capture that fails falls back to
// direct launches for that key; while the stream is being captured by the
// caller, the launches go into the caller's graph.
template <class F>
cudaError_t run_cached(Ctx &c, CallGraph &g, const long long *key, int nkey, F body) {
    if (!c.use_graph) return body();
    // inside a capture of the caller's own: the launches join that graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ec = cudaStreamIsCapturing(c.stream, &cs);
    if (ec != cudaSuccess) return ec;
    if (cs != cudaStreamCaptureStatusNone) return body();
    bool same = g.nkey == nkey;
    for (int i = 0; same && i < nkey; i++) same = g.key[i] == key[i];
    if (same && g.exec) return cudaGraphLaunch(g.exec, c.stream);
    if (same && !g.failed) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = body();
            e = cudaStreamEndCapture(c.stream, &graph);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) return cudaGraphLaunch(g.exec, c.stream);
        cudaGetLastError();
        g.exec = nullptr;
        g.failed = true;
        return body();
    }
    drop_graph(g);
    for (int i = 0; i < nkey; i++) g.key[i] = key[i];
    g.nkey = nkey;
    return body();
}

long long fbits(float x) {
    unsigned u;
    std::memcpy(&u, &x, sizeof u);
    return (long long)u;
}

cudaError_t pipeline_tree(Ctx &c) {
    cudaError_t e;
    if ((e = launch_keys(c)) != cudaSuccess) return e;
    if ((e = launch_sort(c)) != cudaSuccess) return e;
    if ((e = launch_reorder(c)) != cudaSuccess) return e;
    return launch_build(c);
}

cudaError_t pipeline_forces(Ctx &c, float theta, float eps) {
    cudaError_t e;
    if ((e = launch_open_radius(c, theta)) != cudaSuccess) return e;
    return launch_walk(c, eps);
}

// One kick-drift-kick step; events between the stages give per-stage times.
// During stream capture the events become event-record nodes of the graph
// (cudaEventRecordExternal), so replays are timed too.
cudaError_t pipeline_step(Ctx &c, float dt) {
    cudaError_t e;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(c.stream, &cs)) != cudaSuccess) return e;
    const unsigned evf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
#define STAGE(i, call)                                                                                     \
    if (c.stage_timing && (e = cudaEventRecordWithFlags(c.ev[i], c.stream, evf)) != cudaSuccess) return e; \
    if ((e = (call)) != cudaSuccess) return e;
    STAGE(0, launch_reset(c));
    if ((e = launch_kick_drift_bbox(c, dt)) != cudaSuccess) return e;
    STAGE(1, launch_keys(c));
    STAGE(2, launch_sort(c));
    STAGE(3, launch_reorder(c));
    STAGE(4, launch_build(c));
    // Plain steps: the multipole pass also writes the MAC records for the
    // step's theta (the learned path sets its own opening angles).
    const bool plain = c.mlp_P == nullptr;
    STAGE(5, launch_multipoles(c, plain ? c.theta : 0.f));
    STAGE(6, plain ? launch_walk(c, c.eps) : pipeline_learned_forces(c, c.eps));
    STAGE(7, launch_kick(c, dt));
#undef STAGE
    return c.stage_timing ? cudaEventRecordWithFlags(c.ev[8], c.stream, evf) : cudaSuccess;
}

}  // namespace

extern "C" {

const char *bonsai_version(void) { return "bonsai-gb300 0.1 (sm_103a)"; }

const char *bonsai_last_error(const bonsai_ctx *ctx) {
    return ctx ? ctx->c.err.c_str() : g_create_err.c_str();
}

int bonsai_create(bonsai_ctx **out, const bonsai_config *cfg, void *cuda_stream) {
    bonsai_ctx *ctx = nullptr;
    if (!out) return fail(nullptr, BONSAI_ERR_INVALID_ARG, "bonsai_create: out is NULL");
    *out = nullptr;
    ctx = new (std::nothrow) bonsai_ctx();
    if (!ctx) return fail(nullptr, BONSAI_ERR_OOM, "bonsai_create: host allocation failed");
    Ctx &c = ctx->c;
    if (cfg) {
        if (cfg->nleaf) c.nleaf = cfg->nleaf;
        if (cfg->ncrit) c.ncrit = cfg->ncrit;
        if (cfg->list_capacity) c.list_capacity = cfg->list_capacity;
        if (cfg->walk_warps) c.walk_warps = cfg->walk_warps;
        if (cfg->max_spin) c.max_spin = cfg->max_spin;
        if (cfg->use_graph < 0) c.use_graph = 0;
        c.group_pack = cfg->group_pack;
        c.arena_limit = cfg->arena_limit_mib > 0 ? (long long)cfg->arena_limit_mib << 20 : cfg->arena_limit_mib;
    }
    if (c.nleaf < 1 || c.nleaf > 64 || c.ncrit < 1 || c.ncrit > 64 || c.list_capacity < 64 ||
        c.list_capacity > 8192 || c.max_spin < 1 || c.walk_warps < 1 || c.walk_warps > 8 ||
        c.group_pack < 0 || c.group_pack > 1 || c.arena_limit < 0) {
        int r = fail(nullptr, BONSAI_ERR_INVALID_ARG,
                     "bonsai_create: need 1<=nleaf<=64, 1<=ncrit<=64, 64<=list_capacity<=8192, "
                     "1<=walk_warps<=8, group_pack 0 or 1, arena_limit_mib >= 0");
        delete ctx;
        return r;
    }
    c.list_capacity = (c.list_capacity + 31) & ~31;   // keeps per-warp shared rings 16-byte aligned
    cudaError_t e = cudaGetDevice(&c.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
    if (e == cudaSuccess) {
        if (cuda_stream) c.stream = (cudaStream_t)cuda_stream;
        else { e = cudaStreamCreate(&c.stream); c.own_stream = true; }   // blocking: ordered with the legacy stream
    }
    if (e == cudaSuccess) e = cudaMalloc(&c.st, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(&c.st_host, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemsetAsync(c.st, 0, sizeof(DevState), c.stream);
    for (int i = 0; i <= Ctx::NSTAGE && e == cudaSuccess; i++) e = cudaEventCreate(&c.ev[i]);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int r = fail(nullptr, BONSAI_ERR_CUDA, "bonsai_create", e);
        bonsai_destroy(ctx);
        return r;
    }
    *out = ctx;
    return BONSAI_OK;
}

void bonsai_destroy(bonsai_ctx *ctx) {
    if (!ctx) return;
    Ctx &c = ctx->c;
    if (c.stream) cudaStreamSynchronize(c.stream);
    free_bodies(c);
    if (c.st) cudaFree(c.st);
    if (c.st_host) cudaFreeHost(c.st_host);
    for (int i = 0; i <= Ctx::NSTAGE; i++)
        if (c.ev[i]) cudaEventDestroy(c.ev[i]);
    if (c.side) { cudaStreamSynchronize(c.side); cudaStreamDestroy(c.side); }
    if (c.ev_fork) cudaEventDestroy(c.ev_fork);
    if (c.ev_join) cudaEventDestroy(c.ev_join);
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
    delete ctx;
}

int bonsai_set_bodies(bonsai_ctx *ctx, const float *pos, const float *mass, const float *vel,
                      long long n, int on_device) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!pos || !mass || n < 1 || n > (1ll << 26))
        return fail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_set_bodies: need pos, mass and 1 <= n <= 2^26");
    if (n > c.ncap) {
        const cudaError_t e = alloc_bodies(c, n);
        if (e != cudaSuccess) {
            // the old arena is gone: the context holds no bodies now
            c.n = 0;
            c.have_bodies = c.built = c.moments_ready = c.have_acc = c.tree_fresh = c.timed_step = false;
            c.graph_n = -1;
            return fail(ctx, e == cudaErrorMemoryAllocation ? BONSAI_ERR_OOM : BONSAI_ERR_CUDA,
                        "bonsai_set_bodies: device arena", e);
        }
    }
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    c.graph_n = -1;
    if (n != c.n) c.cells_hint = 0;
    c.n = n;
    const float *p = pos, *m = mass, *v = vel;
    // Page-locked host buffers (cudaHostAlloc / cudaHostRegister) are read by
    // the pack kernel directly over the host link, through the device
    // address the runtime reports for them: no staging copies.  Any other
    // host buffer is copied to the staging area first.
    auto mapped = [](const float *q, const float *&d) {
        d = q;
        if (!q) return true;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess) { cudaGetLastError(); return false; }
        if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
        d = static_cast<const float *>(at.devicePointer);
        return true;
    };
    const float *dp, *dm, *dv;
    if (!on_device && mapped(pos, dp) && mapped(mass, dm) && mapped(vel, dv)) {
        p = dp; m = dm; v = dv;
    } else if (!on_device) {
        float *s = c.stage;
        CK(cudaMemcpyAsync(s, pos, 12 * (size_t)n, cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(s + 3 * n, mass, 4 * (size_t)n, cudaMemcpyHostToDevice, c.stream));
        if (vel) CK(cudaMemcpyAsync(s + 4 * n, vel, 12 * (size_t)n, cudaMemcpyHostToDevice, c.stream));
        p = s; m = s + 3 * n; v = vel ? s + 4 * n : nullptr;
    }
    CK(launch_pack(c, p, m, v));
    // One system holding every body until bonsai_set_systems says otherwise.
    c.nsys = 1;
    unsigned off1[2] = {0u, (unsigned)n};
    CK(cudaMemcpyAsync(c.st->sys_off, off1, sizeof(off1), cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemsetAsync(c.sysid, 0, (size_t)n, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    // The state now lives in the pre-sort (*_alt) arrays; nothing derived
    // from earlier bodies stays valid.
    c.have_bodies = true;
    c.built = c.moments_ready = c.have_acc = false;
    c.err.clear();
    return BONSAI_OK;
}

int bonsai_set_systems(bonsai_ctx *ctx, const long long *offsets, int nsys) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_bodies) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_set_systems: no bodies");
    if (!offsets || nsys < 1 || nsys > MAX_SYSTEMS)
        return fail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_set_systems: need offsets and 1 <= nsys <= 256");
    std::vector<unsigned> off(nsys + 1);
    if (offsets[0] != 0 || offsets[nsys] != c.n)
        return fail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_set_systems: offsets must run from 0 to n");
    for (int s = 0; s <= nsys; s++) {
        if (s > 0 && offsets[s] <= offsets[s - 1])
            return fail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_set_systems: every system needs at least one body");
        off[s] = (unsigned)offsets[s];
    }
    if (c.built || c.have_acc)
        return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_set_systems: call it right after bonsai_set_bodies");
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    c.graph_n = -1;
    c.nsys = nsys;
    CK(cudaMemcpyAsync(c.st->sys_off, off.data(), sizeof(unsigned) * (nsys + 1), cudaMemcpyHostToDevice,
                       c.stream));
    CK(launch_fill_sysid(c));
    CK(cudaStreamSynchronize(c.stream));
    c.built = c.moments_ready = c.have_acc = false;
    return BONSAI_OK;
}

int bonsai_build(bonsai_ctx *ctx) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_bodies) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_build: no bodies");
    const bool again = c.built;
    const long long key[] = {c.n, c.arena_gen, c.nsys, c.nleaf, c.ncrit, c.group_pack, c.max_spin, again};
    CK(run_cached(c, c.build_graph, key, (int)(sizeof key / sizeof key[0]), [&]() -> cudaError_t {
        cudaError_t e;
        if (again) {
            // rebuild from the current (sorted) state: copy it to the pre-sort arrays
            if ((e = cudaMemcpyAsync(c.pos4_alt, c.pos4, 16 * (size_t)c.n, cudaMemcpyDeviceToDevice, c.stream)))
                return e;
            if ((e = cudaMemcpyAsync(c.vel4_alt, c.vel4, 16 * (size_t)c.n, cudaMemcpyDeviceToDevice, c.stream)))
                return e;
            if ((e = cudaMemcpyAsync(c.id_alt, c.id, 4 * (size_t)c.n, cudaMemcpyDeviceToDevice, c.stream)))
                return e;
        }
        if ((e = launch_reset(c)) != cudaSuccess) return e;
        if ((e = launch_bbox(c)) != cudaSuccess) return e;
        return pipeline_tree(c);
    }));
    c.built = c.tree_fresh = true;
    c.moments_ready = c.have_acc = false;
    return BONSAI_OK;
}

int bonsai_multipoles(bonsai_ctx *ctx) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.built) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_multipoles: call bonsai_build first");
    // The launch is sized from the last known cell count (a tree of the same
    // bodies changes little); only a context without one reads it back.
    if (c.cells_hint == 0) CK(refresh_cells_hint(c));
    const long long key[] = {c.n, c.arena_gen, c.nsys, c.cells_hint};
    CK(run_cached(c, c.mom_graph, key, (int)(sizeof key / sizeof key[0]), [&]() { return launch_multipoles(c); }));
    c.moments_ready = true;
    return BONSAI_OK;
}

static int check_theta_eps(bonsai_ctx *ctx, float theta, float eps) {
    if (!(theta > 0.f && theta <= 1.15f) || !(eps > 0.f) || !(eps < 1e30f))
        return fail(ctx, BONSAI_ERR_INVALID_ARG, "need 0 < theta <= 1.15 and eps > 0");
    return BONSAI_OK;
}

int bonsai_set_params(bonsai_ctx *ctx, float theta, float eps) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    int r = check_theta_eps(ctx, theta, eps);
    if (r) return r;
    ctx->c.theta = theta;
    ctx->c.eps = eps;
    return BONSAI_OK;
}

int bonsai_forces(bonsai_ctx *ctx, float theta, float eps, float *acc, float *pot, int on_device) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    int r = check_theta_eps(ctx, theta, eps);
    if (r) return r;
    if (!c.moments_ready)
        return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_forces: call bonsai_build and bonsai_multipoles first");
    c.theta = theta;
    c.eps = eps;
    const long long key[] = {c.n, c.arena_gen, c.nsys, c.ncrit, c.group_pack, c.walk_warps, c.list_capacity,
                             c.max_spin, fbits(theta), fbits(eps), c.block_kmax};
    CK(run_cached(c, c.forces_graph, key, (int)(sizeof key / sizeof key[0]), [&]() -> cudaError_t {
        const cudaError_t e = launch_reset(c);
        return e != cudaSuccess ? e : pipeline_forces(c, theta, eps);
    }));
    c.have_acc = true;
    if (acc || pot) {
        if (on_device) {
            CK(launch_scatter_forces(c, acc, pot));
        } else {
            float *sa = c.stage, *sp = c.stage + 3 * c.n;
            CK(launch_scatter_forces(c, acc ? sa : nullptr, pot ? sp : nullptr));
            if (acc) CK(cudaMemcpyAsync(acc, sa, 12 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
            if (pot) CK(cudaMemcpyAsync(pot, sp, 4 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
            CK(cudaStreamSynchronize(c.stream));
        }
    }
    return BONSAI_OK;
}

int bonsai_step(bonsai_ctx *ctx, float dt) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_bodies) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_step: no bodies");
    if (!(dt == dt) || dt > 1e30f || dt < -1e30f) return fail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_step: bad dt");
    if (!c.have_acc) {
        int r;
        if (!c.built && (r = bonsai_build(ctx))) return r;
        if (!c.moments_ready && (r = bonsai_multipoles(ctx))) return r;
        if ((r = bonsai_forces(ctx, c.theta, c.eps, nullptr, nullptr, 1))) return r;
    }
    // The first step with a given (dt, theta, eps, N) runs eagerly; the second
    // captures the step into a CUDA graph, later ones replay it.
    const bool same = c.graph_dt == dt && c.graph_theta == c.theta && c.graph_eps == c.eps &&
                      c.graph_n == c.n && c.graph_timing == c.stage_timing;
    if (c.use_graph && same && c.step_graph) {
        CK(cudaGraphLaunch(c.step_graph, c.stream));
    } else if (c.use_graph && same) {
        // the captured launches are sized from the tree of the eager step before
        CK(refresh_cells_hint(c));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = pipeline_step(c, dt);
            e = cudaStreamEndCapture(c.stream, &g);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c.step_graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c.step_graph = nullptr;
            c.use_graph = 0;           // fall back to direct launches
            CK(pipeline_step(c, dt));
        } else {
            CK(cudaGraphLaunch(c.step_graph, c.stream));
        }
    } else {
        if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
        CK(pipeline_step(c, dt));
        c.graph_dt = dt; c.graph_theta = c.theta; c.graph_eps = c.eps; c.graph_n = c.n;
        c.graph_timing = c.stage_timing;
    }
    c.built = c.moments_ready = c.have_acc = c.tree_fresh = true;
    c.timed_step = c.stage_timing;
    return BONSAI_OK;
}

int bonsai_set_stage_timing(bonsai_ctx *ctx, int on) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    ctx->c.stage_timing = on != 0;
    return BONSAI_OK;
}

int bonsai_get_stage_times(bonsai_ctx *ctx, float *ms, int n) {
    if (!ctx || !ms || n < 0) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.timed_step)
        return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_stage_times: the last step recorded no stage times");
    CK(cudaStreamSynchronize(c.stream));
    int k = n < Ctx::NSTAGE ? n : Ctx::NSTAGE;
    for (int i = 0; i < k; i++) CK(cudaEventElapsedTime(&ms[i], c.ev[i], c.ev[i + 1]));
    return k;
}

int bonsai_autotune(bonsai_ctx *ctx, float theta, float eps, int *best_ncrit, int *best_warps,
                    float *best_ms) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    int r = check_theta_eps(ctx, theta, eps);
    if (r) return r;
    if (!c.have_bodies) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_autotune: no bodies");
    static const int ncrits[] = {16, 32, 48, 64};
    static const int warps[] = {2, 4, 8};
    static const int caps[] = {128, 256, 512};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bn = c.ncrit, bw = c.walk_warps, bp = c.group_pack, bc = c.list_capacity;
    cudaError_t e = cudaSuccess;
    for (int cand = 0; cand < 8; cand++) {
        const int nc = ncrits[cand & 3], pk = cand >> 2;
        c.ncrit = nc;
        c.group_pack = pk;
        if ((r = bonsai_build(ctx)) || (r = bonsai_multipoles(ctx))) break;
        for (int wc = 0; wc < 9; wc++) {
            const int w = warps[wc / 3];
            c.walk_warps = w;
            c.list_capacity = caps[wc % 3];
            // one untimed walk, then the mean of two timed ones
            if ((e = launch_reset(c)) != cudaSuccess || (e = pipeline_forces(c, theta, eps)) != cudaSuccess) break;
            if ((e = cudaEventRecord(e0, c.stream)) != cudaSuccess) break;
            for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
                e = launch_reset(c);
                if (e == cudaSuccess) e = pipeline_forces(c, theta, eps);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            unsigned status = 0;
            if ((e = cudaMemcpy(&status, &c.st->status, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
                break;
            if (status) {                     // e.g. stack overflow: not a valid choice
                if ((e = cudaMemset(&c.st->status, 0, sizeof(unsigned))) != cudaSuccess) break;
                continue;
            }
            if (ms / 2 < best) { best = ms / 2; bn = nc; bw = w; bp = pk; bc = c.list_capacity; }
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    if (e != cudaSuccess) return fail(ctx, BONSAI_ERR_CUDA, "bonsai_autotune", e);
    c.ncrit = bn;
    c.walk_warps = bw;
    c.group_pack = bp;
    c.list_capacity = bc;
    if (c.step_graph) { cudaGraphExecDestroy(c.step_graph); c.step_graph = nullptr; }
    c.graph_n = -1;
    if ((r = bonsai_build(ctx)) || (r = bonsai_multipoles(ctx)) ||
        (r = bonsai_forces(ctx, theta, eps, nullptr, nullptr, 1)))
        return r;
    if (best_ncrit) *best_ncrit = bn;
    if (best_warps) *best_warps = bw;
    if (best_ms) *best_ms = best;
    return BONSAI_OK;
}

int bonsai_get_config(const bonsai_ctx *ctx, bonsai_config *out) {
    if (!ctx || !out) return BONSAI_ERR_INVALID_ARG;
    const Ctx &c = ctx->c;
    std::memset(out, 0, sizeof(*out));
    out->nleaf = c.nleaf;
    out->ncrit = c.ncrit;
    out->walk_warps = c.walk_warps;
    out->list_capacity = c.list_capacity;
    out->use_graph = c.use_graph ? 1 : -1;
    out->group_pack = c.group_pack;
    out->arena_limit_mib = (int)(c.arena_limit >> 20);
    out->max_spin = c.max_spin;
    return BONSAI_OK;
}

int bonsai_get_bodies(bonsai_ctx *ctx, float *pos, float *vel, int on_device) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_bodies) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_bodies: no bodies");
    const float4 *P = c.built ? c.pos4 : c.pos4_alt;
    const float4 *V = c.built ? c.vel4 : c.vel4_alt;
    const uint32_t *I = c.built ? c.id : c.id_alt;
    Ctx tmp = c;   // view with the arrays that hold the state
    tmp.pos4 = (float4 *)P; tmp.vel4 = (float4 *)V; tmp.id = (uint32_t *)I;
    if (on_device) {
        CK(launch_scatter_bodies(tmp, pos, vel));
    } else {
        float *sp = c.stage, *sv = c.stage + 3 * c.n;
        CK(launch_scatter_bodies(tmp, pos ? sp : nullptr, vel ? sv : nullptr));
        if (pos) CK(cudaMemcpyAsync(pos, sp, 12 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
        if (vel) CK(cudaMemcpyAsync(vel, sv, 12 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    tmp.step_graph = nullptr;   // the copy must not own the graph
    return BONSAI_OK;
}

int bonsai_diagnostics(bonsai_ctx *ctx, double out[8]) {
    if (!ctx || !out) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_acc) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_diagnostics: no forces yet");
    CK(cudaMemsetAsync(&c.st->diag[0], 0, 8 * sizeof(double), c.stream));
    CK(launch_diag(c));
    CK(cudaMemcpyAsync(out, &c.st->diag[0], 8 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    out[2] = out[0] + out[1];
    return BONSAI_OK;
}

int bonsai_sync(bonsai_ctx *ctx) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    CK(cudaStreamSynchronize(c.stream));
    unsigned s = 0;
    CK(cudaMemcpy(&s, &c.st->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    CK(cudaMemset(&c.st->status, 0, sizeof(unsigned)));
    if (s & ST_TIMEOUT) return fail(ctx, BONSAI_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (s & ST_CAPACITY) return fail(ctx, BONSAI_ERR_CAPACITY, "walk stack or cell capacity exceeded");
    if (s & ST_NAN) return fail(ctx, BONSAI_ERR_NAN, "non-finite body positions");
    return BONSAI_OK;
}

static int read_state(bonsai_ctx *ctx) {
    Ctx &c = ctx->c;
    CK(cudaMemcpyAsync(c.st_host, c.st, sizeof(DevState), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (c.built) c.cells_hint = c.st_host->ncells;
    return BONSAI_OK;
}

int bonsai_get_sizes(bonsai_ctx *ctx, long long *n, long long *ncells, long long *ngroups) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    int r = read_state(ctx);
    if (r) return r;
    if (n) *n = ctx->c.n;
    if (ncells) *ncells = ctx->c.built ? ctx->c.st_host->ncells : 0;
    if (ngroups) *ngroups = ctx->c.built ? ctx->c.st_host->ngroups : 0;
    return BONSAI_OK;
}

int bonsai_get_domain(bonsai_ctx *ctx, float mn[3], float side[1]) {
    return bonsai_get_domains(ctx, mn, side);
}

int bonsai_get_domains(bonsai_ctx *ctx, float *mn, float *side) {
    if (!ctx || !mn || !side) return BONSAI_ERR_INVALID_ARG;
    if (!ctx->c.built) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_domains: not built");
    int r = read_state(ctx);
    if (r) return r;
    for (int s = 0; s < ctx->c.nsys; s++) {
        for (int d = 0; d < 3; d++) mn[3 * s + d] = ctx->c.st_host->mn[3 * s + d];
        side[s] = ctx->c.st_host->side[s];
    }
    return BONSAI_OK;
}

int bonsai_get_keys(bonsai_ctx *ctx, uint64_t *keys, uint32_t *perm) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.built) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_keys: not built");
    if (keys) CK(cudaMemcpyAsync(keys, c.keys, 8 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
    if (perm) CK(cudaMemcpyAsync(perm, c.id, 4 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return BONSAI_OK;
}

// The introspection getters stream the cells through the context's staging
// area (7 floats per body, at least STAGE_MIN_FLOATS) in chunks of at least
// 409 cells: no allocation per call.
int bonsai_get_tree(bonsai_ctx *ctx, int32_t *bb, int32_t *bc, int32_t *cb, int32_t *nc, int32_t *lv) {
    if (!ctx || !bb || !bc || !cb || !nc || !lv) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.built) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_tree: not built");
    int r = read_state(ctx);
    if (r) return r;
    const unsigned ncells = c.st_host->ncells;
    CK(launch_internal_counts(c));
    const unsigned chunk = (unsigned)(c.stage_floats / 5);       // 5 int32 per cell
    int32_t *tmp = reinterpret_cast<int32_t *>(c.stage);
    int32_t *dst[5] = {bb, bc, cb, nc, lv};
    for (unsigned c0 = 0; c0 < ncells; c0 += chunk) {
        const unsigned cnt = ncells - c0 < chunk ? ncells - c0 : chunk;
        CK(launch_tree_export(c, c0, cnt, tmp, tmp + cnt, tmp + 2 * (size_t)cnt, tmp + 3 * (size_t)cnt,
                              tmp + 4 * (size_t)cnt));
        for (int k = 0; k < 5; k++)
            CK(cudaMemcpyAsync(dst[k] + c0, tmp + (size_t)k * cnt, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               c.stream));
        CK(cudaStreamSynchronize(c.stream));   // the next chunk reuses the staging area
    }
    return BONSAI_OK;
}

int bonsai_get_groups(bonsai_ctx *ctx, int32_t *begin, int32_t *count) {
    if (!ctx || !begin || !count) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.built) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_groups: not built");
    int r = read_state(ctx);
    if (r) return r;
    size_t ng = c.st_host->ngroups;
    std::vector<uint2> h(ng);
    CK(cudaMemcpy(h.data(), c.groups, ng * sizeof(uint2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < ng; i++) { begin[i] = (int32_t)h[i].x; count[i] = (int32_t)h[i].y; }
    return BONSAI_OK;
}

int bonsai_get_moments(bonsai_ctx *ctx, float *mono, float *quad) {
    if (!ctx || !mono || !quad) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.moments_ready) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_moments: no moments");
    int r = read_state(ctx);
    if (r) return r;
    const unsigned ncells = c.st_host->ncells;
    const unsigned chunk = (unsigned)(c.stage_floats / 10);      // 10 floats per cell
    float *tmp = c.stage;
    for (unsigned c0 = 0; c0 < ncells; c0 += chunk) {
        const unsigned cnt = ncells - c0 < chunk ? ncells - c0 : chunk;
        CK(launch_moments_export(c, c0, cnt, tmp, tmp + 4 * (size_t)cnt));
        CK(cudaMemcpyAsync(mono + 4 * (size_t)c0, tmp, 4 * (size_t)cnt * sizeof(float), cudaMemcpyDeviceToHost,
                           c.stream));
        CK(cudaMemcpyAsync(quad + 6 * (size_t)c0, tmp + 4 * (size_t)cnt, 6 * (size_t)cnt * sizeof(float),
                           cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    return BONSAI_OK;
}

int bonsai_get_counts(bonsai_ctx *ctx, uint32_t *n_pc, uint32_t *n_pp, unsigned long long tot[2]) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_acc) return fail(ctx, BONSAI_ERR_NOT_READY, "bonsai_get_counts: no walk yet");
    if (n_pc || n_pp) {
        uint32_t *sa = (uint32_t *)c.stage, *sb = (uint32_t *)c.stage + c.n;
        CK(launch_scatter_counts(c, n_pc ? sa : nullptr, n_pp ? sb : nullptr));
        if (n_pc) CK(cudaMemcpyAsync(n_pc, sa, 4 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
        if (n_pp) CK(cudaMemcpyAsync(n_pp, sb, 4 * (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
    }
    int r = read_state(ctx);
    if (r) return r;
    if (tot) { tot[0] = c.st_host->inter[0]; tot[1] = c.st_host->inter[1]; }
    return BONSAI_OK;
}

int bonsai_debug_hold_sort_tile(bonsai_ctx *ctx, int tile) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (tile < -1) return fail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_debug_hold_sort_tile: need tile >= -1");
    const unsigned v = (unsigned)(tile + 1);
    CK(cudaMemcpyAsync(&c.st->hold_tile, &v, sizeof(unsigned), cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return BONSAI_OK;
}

int bonsai_bench_fma(int blocks, int threads, long long iters, float *ms, double *flop) {
    if (blocks < 1 || blocks > 65535 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !ms ||
        !flop)
        return fail(nullptr, BONSAI_ERR_INVALID_ARG,
                    "bonsai_bench_fma: need 1 <= blocks <= 65535, threads a multiple of 32 in [32, 1024], iters >= 1");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = launch_fma_peak(blocks, threads, 1, sink);       // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = launch_fma_peak(blocks, threads, iters, sink);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(nullptr, BONSAI_ERR_CUDA, "bonsai_bench_fma", e);
    *flop = (double)blocks * threads * (double)iters * 8.0 * 2.0 * 2.0;
    return BONSAI_OK;
}

}  // extern "C"
