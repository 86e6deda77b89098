// api_block.cu -- block (hierarchical) time steps (paper Sect. 1 and 3).
//
// With the whole tree-code on the GPU the paper points out that a block
// time-step scheme only walks the N_active bodies whose step ends (the walk
// time falls by N / N_active) and that between rebuilds only the multipole
// moments need recomputing; the full tree is rebuilt when the walk slows
// down.  The scheme itself is ours (the paper names it, not its rules):
//  * body i steps with dt_max / 2^k_i, k_i the smallest level in [0, kmax]
//    with dt_max / 2^k <= eta sqrt(eps / |a_i|), decided in float32 as
//    16^k >= c |a|^2, c = dt_max^4 / (eta^4 eps^2);
//  * a cycle of dt_max is 2^kmax substeps of dt_min = dt_max / 2^kmax with
//    every body synchronised at both ends: opening half kicks for all at the
//    start; per substep a drift of every body and, where some body's step
//    ends, a rebuild (every `rebuild_every` substeps; one scheduled for a
//    substep where no step ends is taken at the next one where some step
//    does) or a refit (moments of the existing cells at the current
//    positions; opening radii from each cell's build-time cube enlarged to
//    hold its bodies, so a cell holding a walked body is never accepted by
//    that body's group), a walk of the bodies whose step ends, and their
//    closing half kick, new level (never coarser than the substep allows)
//    and opening half kick; the last substep only closes.
// A body's level lives in vel4.w, which the rebuild's reorder carries along.
// The substeps without a step end only drift: every kick also takes the
// minimum over all bodies of the substep at which each one's step ends
// next, and the host reads that one word to schedule the next substep that
// needs tree work and a walk (one synchronisation per walked substep).
#include <cmath>
#include <string>

#include "common.cuh"

using namespace bonsai;

namespace bonsai {

// Level of a body from its acceleration: smallest k in [0, kmax] with
// 16^k >= r, r = c |a|^2 (|a|^2 summed x, y, z with separate roundings).
__device__ __forceinline__ int block_level(const float4 a, float c, int kmax) {
    const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y)), __fmul_rn(a.z, a.z));
    const float r = __fmul_rn(c, a2);
    int k = 0;
    float t = 1.f;
    while (k < kmax && t < r) { t *= 16.f; k++; }
    return k;
}

// Half kick of a body on level k: (2^(kmax-k) dt_min) / 2, exact in float32.
__device__ __forceinline__ float block_half(int k, int kmax, float dtm) {
    return __fmul_rn(__fmul_rn((float)(1u << (kmax - k)), dtm), 0.5f);
}

// Substep at which the step of a body on level k ends next after substep s
// (s on the level's grid for a body that just kicked; the next grid point
// otherwise).
__device__ __forceinline__ unsigned block_next_end(int k, unsigned s, int kmax) {
    return ((s >> (kmax - k)) + 1u) << (kmax - k);
}

// The minimum of e over the block's threads into st->blk_next and (cnt !=
// nullptr) the sum of cnt into st->cyc_active: warp reductions, then one
// shared-memory atomic per warp and one global atomic per block (every
// thread of the block calls, outside divergent code).
__device__ __forceinline__ void block_totals(unsigned e, const unsigned *cnt, DevState *st) {
    __shared__ unsigned s_min, s_cnt;
    if (threadIdx.x == 0) { s_min = 0xffffffffu; s_cnt = 0u; }
    __syncthreads();
    e = __reduce_min_sync(0xffffffffu, e);
    const unsigned c = cnt ? __reduce_add_sync(0xffffffffu, *cnt) : 0u;
    if ((threadIdx.x & 31) == 0) {
        if (e != 0xffffffffu) atomicMin_block(&s_min, e);
        if (c) atomicAdd_block(&s_cnt, c);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_min != 0xffffffffu) atomicMin(&st->blk_next, s_min);
        if (s_cnt) atomicAdd(&st->cyc_active, (unsigned long long)s_cnt);
    }
}

// Cycle start: every body takes its level and the opening half kick.
__global__ void k_block_open(float4 *vel, const float4 *__restrict__ acc, int n, float c, int kmax, float dtm,
                             DevState *st) {
    unsigned nx = 0xffffffffu;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = acc[i];
        float4 v = vel[i];
        const int k = block_level(a, c, kmax);
        const float h = block_half(k, kmax, dtm);
        v.x = fmaf(a.x, h, v.x); v.y = fmaf(a.y, h, v.y); v.z = fmaf(a.z, h, v.z);
        v.w = (float)k;
        vel[i] = v;
        nx = min(nx, block_next_end(k, 0u, kmax));
    }
    block_totals(nx, nullptr, st);
}

// Substep s: the bodies whose step ends take the closing half kick and,
// unless the cycle ends, a new level (no coarser than kmax - trailing zeros
// of s, so that the next step ends on the level's grid) and its opening
// half kick.  Counts the ended steps of the cycle and takes the next
// substep at which a step ends.
__global__ void k_block_kick(float4 *vel, const float4 *__restrict__ acc, int n, unsigned s, int kmax, float c,
                             float dtm, int last, DevState *st) {
    unsigned cnt = 0, nx = 0xffffffffu;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 v = vel[i];
        if (!block_active(v.w, s, kmax)) {
            nx = min(nx, block_next_end((int)v.w, s, kmax));
            continue;
        }
        cnt++;
        const float4 a = acc[i];
        const float h = block_half((int)v.w, kmax, dtm);
        v.x = fmaf(a.x, h, v.x); v.y = fmaf(a.y, h, v.y); v.z = fmaf(a.z, h, v.z);
        if (!last) {
            const int k = max(block_level(a, c, kmax), kmax - (__ffs((int)s) - 1));
            const float h2 = block_half(k, kmax, dtm);
            v.x = fmaf(a.x, h2, v.x); v.y = fmaf(a.y, h2, v.y); v.z = fmaf(a.z, h2, v.z);
            v.w = (float)k;
            nx = min(nx, block_next_end(k, s, kmax));
        }
        vel[i] = v;
    }
    block_totals(nx, &cnt, st);
}

// `times` drifts of every body by dt in place (substeps that only drift,
// then a refit substep's own: the order stays), each rounded as one.
__global__ void k_block_drift(float4 *pos, const float4 *__restrict__ vel, int n, float dt, unsigned times) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 x = pos[i];
        const float4 u = vel[i];
        for (unsigned t = 0; t < times; t++) {
            x.x = fmaf(u.x, dt, x.x); x.y = fmaf(u.y, dt, x.y); x.z = fmaf(u.z, dt, x.z);
        }
        pos[i] = x;
    }
}

// The walk's interaction totals of a substep added to the cycle's; the
// next-step-end minimum starts over for the kick that follows.
__global__ void k_block_accum(DevState *st, int first) {
    if (threadIdx.x != 0) return;
    if (first) { st->cyc_active = 0ull; st->cyc_inter[0] = 0ull; st->cyc_inter[1] = 0ull; }
    else { st->cyc_inter[0] += st->inter[0]; st->cyc_inter[1] += st->inter[1]; }
    st->blk_next = 0xffffffffu;
}

// Levels in caller order (a query: nothing changes).
__global__ void k_block_levels(const float4 *__restrict__ acc, const uint32_t *__restrict__ id, int n, float c,
                               int kmax, int32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[id[i]] = block_level(acc[i], c, kmax);
}

// c = dt_max^4 / (eta^4 eps^2) in double from the float parameters, rounded
// to float once.
static float block_constant(float dt_max, float eta, float eps) {
    const double d = dt_max, e = eta, s = eps;
    const double d2 = d * d, e2 = e * e;
    return (float)((d2 * d2) / ((e2 * e2) * (s * s)));
}

// The next substep at which some body's step ends, as the last kick left it
// (one word read back; the host waits for the stream).  A value out of
// (s, nsub] cannot come from a kick; it falls back to the next substep.
static cudaError_t block_next(Ctx &c, unsigned s, unsigned nsub, unsigned &nx) {
    cudaError_t e = cudaMemcpyAsync(&c.st_host->blk_next, &c.st->blk_next, sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    nx = c.st_host->blk_next;
    if (nx <= s || nx > nsub) nx = s + 1u;
    return e;
}

static cudaError_t block_cycle(Ctx &c, float dt_max, int kmax, float eta, int rebuild) {
    const int n = (int)c.n;
    const int grid = (int)std::min<long long>((c.n + 255) / 256, (long long)c.num_sms * 8);
    const float dtm = ldexpf(dt_max, -kmax);
    const float cc = block_constant(dt_max, eta, c.eps);
    const unsigned nsub = 1u << kmax;
    cudaError_t e;
    c.blk_walked = c.blk_rebuilt = 0;
    k_block_accum<<<1, 32, 0, c.stream>>>(c.st, 1);
    k_block_open<<<grid, 256, 0, c.stream>>>(c.vel4, c.acc4, n, cc, kmax, dtm, c.st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bool due = false, rebuilt = false;
    for (unsigned s = 0; s < nsub;) {
        unsigned nx;
        if ((e = block_next(c, s, nsub, nx)) != cudaSuccess) return e;
        // substeps s+1 .. nx-1 only drift; a rebuild scheduled on any of
        // them (or on nx) is due at nx
        for (unsigned t = s + 1u; t <= nx; t++) due |= (t - 1u) % (unsigned)rebuild == 0u;
        const unsigned quiet = nx - s - 1u;
        if ((e = launch_reset(c)) != cudaSuccess) return e;
        rebuilt = due;
        if (due) {
            if (quiet) k_block_drift<<<grid, 256, 0, c.stream>>>(c.pos4, c.vel4, n, dtm, quiet);
            if ((e = launch_drift_bbox(c, dtm)) != cudaSuccess) return e;
            if ((e = launch_keys(c)) != cudaSuccess) return e;
            if ((e = launch_sort(c)) != cudaSuccess) return e;
            if ((e = launch_reorder(c)) != cudaSuccess) return e;
            if ((e = launch_build(c)) != cudaSuccess) return e;
            if ((e = launch_multipoles(c)) != cudaSuccess) return e;
            due = false;
            c.blk_rebuilt++;
        } else {
            k_block_drift<<<grid, 256, 0, c.stream>>>(c.pos4, c.vel4, n, dtm, quiet + 1u);
            if ((e = launch_multipoles_refit(c)) != cudaSuccess) return e;
        }
        if ((e = launch_open_radius(c, c.theta)) != cudaSuccess) return e;
        c.block_kmax = kmax;
        c.block_s = nx;
        e = launch_walk(c, c.eps);
        c.block_kmax = -1;
        if (e != cudaSuccess) return e;
        c.blk_walked++;
        k_block_accum<<<1, 32, 0, c.stream>>>(c.st, 0);
        k_block_kick<<<grid, 256, 0, c.stream>>>(c.vel4, c.acc4, n, nx, kmax, cc, dtm, nx == nsub ? 1 : 0, c.st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        s = nx;
    }
    c.tree_fresh = rebuilt;    // the last substep rebuilt
    return cudaSuccess;
}

}  // namespace bonsai

static int bfail(bonsai_ctx *ctx, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    cudaGetLastError();
    std::string s = what;
    if (e != cudaSuccess) { s += ": "; s += cudaGetErrorString(e); }
    if (ctx) ctx->c.err = s;
    return code;
}

extern "C" {

int bonsai_block_cycle(bonsai_ctx *ctx, float dt_max, int max_level, float eta, int rebuild_every) {
    if (!ctx) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_bodies) return bfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_block_cycle: no bodies");
    if (c.nsys != 1) return bfail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_block_cycle: one system only");
    if (!(dt_max > 0.f) || !(dt_max < 1e30f) || max_level < 0 || max_level > 20 || !(eta > 0.f) ||
        !(eta < 1e30f) || rebuild_every < 1)
        return bfail(ctx, BONSAI_ERR_INVALID_ARG,
                     "bonsai_block_cycle: need dt_max > 0, 0 <= max_level <= 20, eta > 0, rebuild_every >= 1");
    if (!c.have_acc) {
        int r;
        if (!c.built && (r = bonsai_build(ctx))) return r;
        if (!c.moments_ready && (r = bonsai_multipoles(ctx))) return r;
        if ((r = bonsai_forces(ctx, c.theta, c.eps, nullptr, nullptr, 1))) return r;
    }
    cudaError_t e = block_cycle(c, dt_max, max_level, eta, rebuild_every);
    if (e != cudaSuccess) return bfail(ctx, BONSAI_ERR_CUDA, "bonsai_block_cycle", e);
    c.built = c.moments_ready = c.have_acc = true;
    return BONSAI_OK;
}

int bonsai_block_substeps(bonsai_ctx *ctx, int32_t out[2]) {
    if (!ctx || !out) return BONSAI_ERR_INVALID_ARG;
    out[0] = ctx->c.blk_walked;
    out[1] = ctx->c.blk_rebuilt;
    return BONSAI_OK;
}

int bonsai_block_levels(bonsai_ctx *ctx, float dt_max, int max_level, float eta, int32_t *levels) {
    if (!ctx || !levels) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.have_acc) return bfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_block_levels: no forces yet");
    if (!(dt_max > 0.f) || max_level < 0 || max_level > 20 || !(eta > 0.f))
        return bfail(ctx, BONSAI_ERR_INVALID_ARG, "bonsai_block_levels: need dt_max > 0, 0 <= max_level <= 20, eta > 0");
    int32_t *tmp = reinterpret_cast<int32_t *>(c.stage);
    const int n = (int)c.n;
    k_block_levels<<<(n + 255) / 256, 256, 0, c.stream>>>(c.acc4, c.id, n, block_constant(dt_max, eta, c.eps),
                                                           max_level, tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(levels, tmp, 4 * (size_t)n, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return bfail(ctx, BONSAI_ERR_CUDA, "bonsai_block_levels", e);
    return BONSAI_OK;
}

int bonsai_block_stats(bonsai_ctx *ctx, long long out[3]) {
    if (!ctx || !out) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    cudaError_t e = cudaMemcpyAsync(c.st_host, c.st, sizeof(DevState), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return bfail(ctx, BONSAI_ERR_CUDA, "bonsai_block_stats", e);
    out[0] = (long long)c.st_host->cyc_active;
    out[1] = (long long)c.st_host->cyc_inter[0];
    out[2] = (long long)c.st_host->cyc_inter[1];
    return BONSAI_OK;
}

}  // extern "C"
