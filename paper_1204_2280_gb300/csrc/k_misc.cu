// k_misc.cu -- second leapfrog kick, caller-order outputs, FP64 diagnostics
// and introspection exports.
#include "common.cuh"

namespace bonsai {

// Second half of the kick-drift-kick step: v += a dt/2 (sorted order).
#ifndef KK_ITEMS
#define KK_ITEMS 2                    // bodies per thread of the kick, loads first (1 or 4: 0.012 ms at 2^20, 2: 0.010)
#endif
__global__ void k_kick(float4 *vel, const float4 *__restrict__ acc, int n, float h) {
    const int i0 = blockIdx.x * blockDim.x * KK_ITEMS + threadIdx.x;
    float4 vv[KK_ITEMS], aa[KK_ITEMS];
#pragma unroll
    for (int k = 0; k < KK_ITEMS; k++) {
        const int i = i0 + k * (int)blockDim.x;
        if (i < n) { vv[k] = vel[i]; aa[k] = acc[i]; }
    }
#pragma unroll
    for (int k = 0; k < KK_ITEMS; k++) {
        const int i = i0 + k * (int)blockDim.x;
        if (i < n) {
            float4 v = vv[k];
            const float4 a = aa[k];
            v.x = fmaf(a.x, h, v.x); v.y = fmaf(a.y, h, v.y); v.z = fmaf(a.z, h, v.z);
            vel[i] = v;
        }
    }
}

cudaError_t launch_kick(Ctx &c, float dt) {
    int n = (int)c.n;
    k_kick<<<(n + 256 * KK_ITEMS - 1) / (256 * KK_ITEMS), 256, 0, c.stream>>>(c.vel4, c.acc4, n, 0.5f * dt);
    return cudaGetLastError();
}

// Sorted -> caller order through the stored caller index.
__global__ void k_scatter_forces(const float4 *__restrict__ acc, const uint32_t *__restrict__ id,
                                 int n, float *a, float *p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = acc[i];
    uint32_t j = id[i];
    if (a) { a[3 * (size_t)j] = v.x; a[3 * (size_t)j + 1] = v.y; a[3 * (size_t)j + 2] = v.z; }
    if (p) p[j] = v.w;
}

cudaError_t launch_scatter_forces(Ctx &c, float *acc, float *pot) {
    int n = (int)c.n;
    k_scatter_forces<<<(n + 255) / 256, 256, 0, c.stream>>>(c.acc4, c.id, n, acc, pot);
    return cudaGetLastError();
}

__global__ void k_scatter_bodies(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                 const uint32_t *__restrict__ id, int n, float *x, float *v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    size_t j = id[i];
    if (x) { float4 q = pos[i]; x[3 * j] = q.x; x[3 * j + 1] = q.y; x[3 * j + 2] = q.z; }
    if (v) { float4 q = vel[i]; v[3 * j] = q.x; v[3 * j + 1] = q.y; v[3 * j + 2] = q.z; }
}

cudaError_t launch_scatter_bodies(Ctx &c, float *pos, float *vel) {
    int n = (int)c.n;
    k_scatter_bodies<<<(n + 255) / 256, 256, 0, c.stream>>>(c.pos4, c.vel4, c.id, n, pos, vel);
    return cudaGetLastError();
}

__global__ void k_scatter_counts(const uint2 *__restrict__ cnt, const uint32_t *__restrict__ id,
                                 int n, uint32_t *a, uint32_t *b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint2 v = cnt[i];
    uint32_t j = id[i];
    if (a) a[j] = v.x;
    if (b) b[j] = v.y;
}

cudaError_t launch_scatter_counts(Ctx &c, uint32_t *npc, uint32_t *npp) {
    int n = (int)c.n;
    k_scatter_counts<<<(n + 255) / 256, 256, 0, c.stream>>>(c.counts, c.id, n, npc, npp);
    return cudaGetLastError();
}

// FP64 diagnostics: K, W, E(filled on host), Px, Py, Pz, Mtot, Lz.
__global__ void __launch_bounds__(256)
k_diag(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
       const float4 *__restrict__ acc, int n, DevState *st) {
    __shared__ double red[8][8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < n) {
        float4 x = pos[i], u = vel[i];
        double m = x.w, vx = u.x, vy = u.y, vz = u.z;
        v[0] = 0.5 * m * (vx * vx + vy * vy + vz * vz);
        v[1] = 0.5 * m * (double)acc[i].w;
        v[3] = m * vx; v[4] = m * vy; v[5] = m * vz; v[6] = m;
        v[7] = m * ((double)x.x * vy - (double)x.y * vx);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][w] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0;
        for (int j = 0; j < 8; j++) s += red[threadIdx.x][j];
        if (threadIdx.x != 2) atomicAdd(&st->diag[threadIdx.x], s);
    }
}

cudaError_t launch_diag(Ctx &c) {
    int n = (int)c.n;
    k_diag<<<(n + 255) / 256, 256, 0, c.stream>>>(c.pos4, c.vel4, c.acc4, n, c.st);
    return cudaGetLastError();
}

// Introspection exports of cells [c0, c0 + cnt) into compact buffers (the
// getters stream them through the context's staging area in chunks).
__global__ void k_tree_export(const uint2 *__restrict__ body, const uint2 *__restrict__ link,
                              const uint8_t *__restrict__ level, unsigned c0, unsigned cnt,
                              int32_t *bb, int32_t *bc, int32_t *cb, int32_t *nc, int32_t *lv) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const unsigned c = c0 + i;
    uint2 b = body[c], l = link[c];
    bool leaf = (l.y & LEAF_BIT) != 0u;
    bb[i] = (int32_t)b.x; bc[i] = (int32_t)b.y;
    cb[i] = leaf ? 0 : (int32_t)l.x;
    nc[i] = leaf ? 0 : (int32_t)l.y;
    lv[i] = level[c];
}

cudaError_t launch_tree_export(Ctx &c, unsigned c0, unsigned cnt, int32_t *bb, int32_t *bc, int32_t *cb,
                               int32_t *nc, int32_t *lv) {
    if (cnt == 0) return cudaSuccess;
    k_tree_export<<<(cnt + 255) / 256, 256, 0, c.stream>>>(c.cell_body, c.cell_link, c.cell_level, c0, cnt, bb, bc,
                                                            cb, nc, lv);
    return cudaGetLastError();
}

__global__ void k_moments_export(const float4 *__restrict__ mono, const float4 *__restrict__ qa,
                                 const float2 *__restrict__ qb, unsigned c0, unsigned cnt, float *m, float *q) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const unsigned c = c0 + i;
    float4 a = mono[c], b = qa[c];
    float2 d = qb[c];
    m[4 * (size_t)i] = a.x; m[4 * (size_t)i + 1] = a.y; m[4 * (size_t)i + 2] = a.z; m[4 * (size_t)i + 3] = a.w;
    float *o = q + 6 * (size_t)i;
    o[0] = -b.x; o[1] = -b.y; o[2] = -b.z; o[3] = -b.w; o[4] = -d.x; o[5] = -d.y;   // stored as -Q
}

cudaError_t launch_moments_export(Ctx &c, unsigned c0, unsigned cnt, float *mono, float *quad) {
    if (cnt == 0) return cudaSuccess;
    k_moments_export<<<(cnt + 255) / 256, 256, 0, c.stream>>>(c.mono, c.quadA, c.quadB, c0, cnt, mono, quad);
    return cudaGetLastError();
}

// FP32 peak microbenchmark: eight independent chains of packed FP32x2 fused
// multiply-adds per thread (x <- x * a + b keeps every value bounded for
// |a| < 1).  The result feeds one conditional store so the chains stay live.
__global__ void k_fma_peak(long long iters, float2 a, float2 b, float *sink) {
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = make_float2(threadIdx.x * 1e-3f + k, blockIdx.x * 1e-3f - k);
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = __ffma2_rn(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k].x + x[k].y;
    if (s == 1234.5f) sink[0] = s;
}

cudaError_t launch_fma_peak(int blocks, int threads, long long iters, float *sink) {
    k_fma_peak<<<blocks, threads>>>(iters, make_float2(0.999f, 0.998f), make_float2(1e-3f, 2e-3f), sink);
    return cudaGetLastError();
}

}  // namespace bonsai
