// k_keys.cu -- body packing, leapfrog drift, domain cube and Morton keys.
//
// Paper Sect. 2, "Sorting of the particles along a Space Filling Curve
// (Morton)": every body gets a 63-bit Z-order key from its position quantised
// on a 2^21 grid per axis over the domain cube.  The cube corner is the
// per-axis minimum and its side S the smallest power of two strictly greater
// than the largest extent, so that every quantisation below is exact:
//   q_d = floor((x_d - mn_d) * 2^21 / S)
// is computed as (int)(__fsub_rd(x_d, mn_d) * (2^21 / S)): the round-down
// subtraction never exceeds the exact difference and floor(v 2^21/S)*S/2^21
// is itself a float <= v, so both floors agree; the multiply by a power of
// two is exact.
#include "common.cuh"

namespace bonsai {

// ---------------------------------------------------------------------------
__global__ void k_reset(DevState *st, int what, int nsys) {
    int t = threadIdx.x;
    if (what & 1) {                        // build inputs
        for (int i = t; i < 3 * nsys; i += blockDim.x) {
            int sys = i / 3, d = i % 3;
            st->dom[6 * sys + d] = 0x7fffffff;
            st->dom[6 * sys + 3 + d] = (int)0x80000000;
        }
        for (int i = t; i < (SORT_PASSES + 1) * SORT_RADIX; i += blockDim.x) st->hist[i] = 0;
        if (t < SORT_PASSES + 1) st->sort_tile[t] = 0;
    }
    if (what & 2) {                        // walk inputs
        if (t == 0) { st->walk_next = 0; st->walk_next2 = 0; st->inter[0] = 0; st->inter[1] = 0; }
    }
    if (what & 4) {
        if (t < 8) st->diag[t] = 0.0;
    }
}

cudaError_t launch_reset(Ctx &c) {
    k_reset<<<1, 256, 0, c.stream>>>(c.st, 7, c.nsys);
    return cudaGetLastError();
}

// System id of every body position from the segment offsets.
__global__ void k_fill_sysid(const DevState *__restrict__ st, int nsys, int n, uint8_t *sysid) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsys - 1;               // last system with sys_off <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (st->sys_off[mid] <= (unsigned)i) lo = mid; else hi = mid - 1;
    }
    sysid[i] = (uint8_t)lo;
}

cudaError_t launch_fill_sysid(Ctx &c) {
    int n = (int)c.n;
    k_fill_sysid<<<(n + 255) / 256, 256, 0, c.stream>>>(c.st, c.nsys, n, c.sysid);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Caller arrays (pos N x 3, mass N, vel N x 3 or null) -> pos4_alt, vel4_alt,
// id_alt = caller index.  Flags non-finite input.
__global__ void k_pack(const float *__restrict__ pos, const float *__restrict__ mass,
                       const float *__restrict__ vel, int n, float4 *pos4,
                       float4 *vel4, uint32_t *id, DevState *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], m = mass[i];
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (vel) { vx = vel[3 * i]; vy = vel[3 * i + 1]; vz = vel[3 * i + 2]; }
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(m))) atomicOr(&st->status, ST_NAN);
    pos4[i] = make_float4(x, y, z, m);
    vel4[i] = make_float4(vx, vy, vz, 0.f);
    id[i] = (uint32_t)i;
}

cudaError_t launch_pack(Ctx &c, const float *pos, const float *mass, const float *vel) {
    int n = (int)c.n;
    k_pack<<<(n + 255) / 256, 256, 0, c.stream>>>(pos, mass, vel, n, c.pos4_alt, c.vel4_alt,
                                                  c.id_alt, c.st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-system min/max of the positions.  Systems are contiguous runs of body
// positions, so a block almost always lies inside one system: then a block
// reduction and six atomics; warps that straddle a boundary fall back to
// warp reductions per uniform warp or per-lane atomics.
__device__ __forceinline__ void dom_atomics(DevState *st, int sys, const float (&v)[6]) {
    for (int d = 0; d < 3; d++) {
        atomicMin(&st->dom[6 * sys + d], f2ord(v[d]));
        atomicMax(&st->dom[6 * sys + 3 + d], f2ord(v[3 + d]));
    }
}

__device__ __forceinline__ void bbox_accumulate(float x, float y, float z, bool valid, int sys,
                                                DevState *st) {
    __shared__ float red[6][32];
    __shared__ int s_sys[2];
    if (threadIdx.x == 0) { s_sys[0] = 1 << 30; s_sys[1] = -1; }
    __syncthreads();
    if (valid) { atomicMin(&s_sys[0], sys); atomicMax(&s_sys[1], sys); }
    __syncthreads();
    const bool uniform_block = s_sys[0] == s_sys[1];
    float v[6] = {x, y, z, x, y, z};
    if (!valid) { v[0] = v[1] = v[2] = INFINITY; v[3] = v[4] = v[5] = -INFINITY; }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (!uniform_block) {
        if (s_sys[1] < 0) return;            // no valid body in the block
        const int s0 = __shfl_sync(0xffffffffu, valid ? sys : -1, 0);
        const bool wu = __all_sync(0xffffffffu, !valid || sys == s0) && s0 >= 0;
        if (!wu) {
            if (valid) dom_atomics(st, sys, v);
            return;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int d = 0; d < 3; d++) {
                v[d] = fminf(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
                v[3 + d] = fmaxf(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
            }
        if (l == 0) dom_atomics(st, s0, v);
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            v[d] = fminf(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
            v[3 + d] = fmaxf(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
        }
    }
    if (l == 0)
        for (int d = 0; d < 6; d++) red[d][w] = v[d];
    __syncthreads();
    if (w == 0) {
        float r[6];
        for (int d = 0; d < 6; d++) {
            r[d] = l < nw ? red[d][l] : (d < 3 ? INFINITY : -INFINITY);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float q = __shfl_xor_sync(0xffffffffu, r[d], o);
                r[d] = d < 3 ? fminf(r[d], q) : fmaxf(r[d], q);
            }
        }
        if (l == 0) dom_atomics(st, s_sys[0], r);
    }
}

__global__ void k_bbox(const float4 *__restrict__ p, const uint8_t *__restrict__ sysid, int n,
                       DevState *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float4 q = i < n ? p[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    bbox_accumulate(q.x, q.y, q.z, i < n, i < n ? sysid[i] : 0, st);
}

cudaError_t launch_bbox(Ctx &c) {
    int n = (int)c.n;
    k_bbox<<<(n + 255) / 256, 256, 0, c.stream>>>(c.pos4_alt, c.sysid, n, c.st);
    return cudaGetLastError();
}

// First half of the kick-drift-kick leapfrog fused with the domain reduction:
// v' = v + a dt/2, x' = x + v' dt (written to the pre-sort arrays).
__global__ void k_kick_drift_bbox(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                  const float4 *__restrict__ acc, const uint32_t *__restrict__ id,
                                  const uint8_t *__restrict__ sysid, int n, float dt, float4 *pos_o,
                                  float4 *vel_o, uint32_t *id_o, DevState *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
        float4 v = vel[i], a = acc[i];
        x = pos[i];
        float h = 0.5f * dt;
        v.x = fmaf(a.x, h, v.x); v.y = fmaf(a.y, h, v.y); v.z = fmaf(a.z, h, v.z);
        x.x = fmaf(v.x, dt, x.x); x.y = fmaf(v.y, dt, x.y); x.z = fmaf(v.z, dt, x.z);
        if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z))) atomicOr(&st->status, ST_NAN);
        pos_o[i] = x; vel_o[i] = v; id_o[i] = id[i];
    }
    bbox_accumulate(x.x, x.y, x.z, i < n, i < n ? sysid[i] : 0, st);
}

// One system: grid-stride loop, running min/max per thread, one block
// reduction and six atomics per block (no per-body system bookkeeping).
__device__ __forceinline__ void block_bbox_atomics(float (&v)[6], DevState *st) {
    __shared__ float red[6][8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int d = 0; d < 3; d++) {
            v[d] = fminf(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
            v[3 + d] = fmaxf(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
        }
    if (l == 0)
#pragma unroll
        for (int d = 0; d < 6; d++) red[d][w] = v[d];
    __syncthreads();
    if (w == 0) {
        float r[6];
#pragma unroll
        for (int d = 0; d < 6; d++) {
            r[d] = l < 8 ? red[d][l] : (d < 3 ? INFINITY : -INFINITY);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                const float q = __shfl_xor_sync(0xffffffffu, r[d], o);
                r[d] = d < 3 ? fminf(r[d], q) : fmaxf(r[d], q);
            }
        }
        if (l == 0) dom_atomics(st, 0, r);
    }
}

#ifndef KD_ITEMS
#define KD_ITEMS 4                    // bodies per thread and pass of the fused kick-drift-bbox (1: 6% slower)
#endif
__global__ void __launch_bounds__(256)
k_kick_drift_bbox1(const float4 *__restrict__ pos, const float4 *__restrict__ vel, const float4 *__restrict__ acc,
                   const uint32_t *__restrict__ id, int n, float dt, float4 *pos_o, float4 *vel_o, uint32_t *id_o,
                   DevState *st) {
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    const float h = 0.5f * dt;
    // KD_ITEMS bodies per thread and pass, all loads issued first
    constexpr int KD = KD_ITEMS;
    for (int i0 = blockIdx.x * blockDim.x * KD + threadIdx.x; i0 < n; i0 += gridDim.x * blockDim.x * KD) {
        float4 uu[KD], xx[KD], aa[KD];
        uint32_t dd[KD];
#pragma unroll
        for (int k = 0; k < KD; k++) {
            const int i = i0 + k * (int)blockDim.x;
            if (i < n) {
                uu[k] = vel[i]; xx[k] = pos[i]; dd[k] = id[i];
                aa[k] = acc ? acc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < KD; k++) {
            const int i = i0 + k * (int)blockDim.x;
            if (i >= n) break;
            float4 u = uu[k], x = xx[k];
            if (acc) {                     // acc NULL: drift only
                const float4 a = aa[k];
                u.x = fmaf(a.x, h, u.x); u.y = fmaf(a.y, h, u.y); u.z = fmaf(a.z, h, u.z);
            }
            x.x = fmaf(u.x, dt, x.x); x.y = fmaf(u.y, dt, x.y); x.z = fmaf(u.z, dt, x.z);
            bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z));
            pos_o[i] = x; vel_o[i] = u; id_o[i] = dd[k];
            v[0] = fminf(v[0], x.x); v[1] = fminf(v[1], x.y); v[2] = fminf(v[2], x.z);
            v[3] = fmaxf(v[3], x.x); v[4] = fmaxf(v[4], x.y); v[5] = fmaxf(v[5], x.z);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->status, ST_NAN);
    block_bbox_atomics(v, st);
}

// Drift of every body by dt into the pre-sort arrays, with the domain box
// (one system): the input of a rebuild during block time steps.
cudaError_t launch_drift_bbox(Ctx &c, float dt) {
    const int n = (int)c.n;
    const int grid = min((n + 256 * KD_ITEMS - 1) / (256 * KD_ITEMS), c.num_sms * 8);
    k_kick_drift_bbox1<<<grid, 256, 0, c.stream>>>(c.pos4, c.vel4, nullptr, c.id, n, dt, c.pos4_alt, c.vel4_alt,
                                                    c.id_alt, c.st);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift_bbox(Ctx &c, float dt) {
    int n = (int)c.n;
    if (c.nsys == 1) {
        const int grid = min((n + 256 * KD_ITEMS - 1) / (256 * KD_ITEMS), c.num_sms * 8);
        k_kick_drift_bbox1<<<grid, 256, 0, c.stream>>>(c.pos4, c.vel4, c.acc4, c.id, n, dt, c.pos4_alt,
                                                        c.vel4_alt, c.id_alt, c.st);
        return cudaGetLastError();
    }
    k_kick_drift_bbox<<<(n + 255) / 256, 256, 0, c.stream>>>(c.pos4, c.vel4, c.acc4, c.id, c.sysid, n,
                                                             dt, c.pos4_alt, c.vel4_alt, c.id_alt, c.st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Smallest power of two strictly greater than the exact difference hi - lo.
__device__ float pow2_above_diff(float hi, float lo) {
    float e_rd = __fsub_rd(hi, lo), e_ru = __fsub_ru(hi, lo);
    if (!(e_ru > 0.f)) return 0.f;
    int ex;
    float m = frexpf(e_ru, &ex);           // e_ru = m 2^ex, m in [0.5, 1)
    if (e_rd == e_ru) return ldexpf(1.f, ex);          // exact: 2^(floor(log2 e) + 1)
    return (m == 0.5f) ? e_ru : ldexpf(1.f, ex);       // inexact: smallest pow2 >= e_ru
}

// Spread the low 21 bits of v to every third bit (bit b -> bit 3b).
__device__ __forceinline__ unsigned long long spread3(unsigned v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Domain of every system from its bounding box, and the histogram of the
// extra radix pass on the system id (the system sizes).
__global__ void k_domains(DevState *st, int nsys) {
    for (int sys = threadIdx.x; sys < MAX_SYSTEMS; sys += blockDim.x) {
        if (sys < nsys) {
            float S = 0x1p-64f;
            for (int d = 0; d < 3; d++) {
                float lo = ord2f(st->dom[6 * sys + d]), hi = ord2f(st->dom[6 * sys + 3 + d]);
                st->mn[3 * sys + d] = lo;
                S = fmaxf(S, pow2_above_diff(hi, lo));
            }
            int ex;
            frexpf(S, &ex);                // S = 2^(ex-1)
            st->side[sys] = S;
            st->scale[sys] = ldexpf(1.f, KEY_BITS_PER_AXIS - (ex - 1));
            st->hist[SORT_PASSES * SORT_RADIX + sys] = st->sys_off[sys + 1] - st->sys_off[sys];
        } else {
            st->hist[SORT_PASSES * SORT_RADIX + sys] = 0u;
        }
    }
}

cudaError_t launch_domains(Ctx &c) {
    k_domains<<<1, 256, 0, c.stream>>>(c.st, c.nsys);
    return cudaGetLastError();
}

constexpr int KEYS_THREADS = 256;
constexpr int KEYS_ITEMS = 8;
#ifndef KEYS_BLOCKS_PER_SM
#define KEYS_BLOCKS_PER_SM 16         // key blocks per SM, each flushing its 8 x 256 digit counts once
#endif                                // (a block per 2048 bodies: 0.132 ms at 2^24; 16 per SM: 0.097 ms)

// Keys of all bodies (each quantised in its own system's cube) plus the 8
// digit histograms of the radix sort; also clears the pass-0 tile status of
// the sort.
__global__ void __launch_bounds__(KEYS_THREADS)
k_keys(const float4 *__restrict__ p, const uint8_t *__restrict__ sysid, int n, int nsys,
       DevState *st, unsigned long long *keys, unsigned *status0, int nstatus) {
    __shared__ unsigned h[SORT_PASSES * SORT_RADIX];
    __shared__ float4 s_dom[MAX_SYSTEMS];   // mn xyz, scale
    for (int i = threadIdx.x; i < SORT_PASSES * SORT_RADIX; i += blockDim.x) h[i] = 0;
    for (int i = threadIdx.x; i < nsys; i += blockDim.x)
        s_dom[i] = make_float4(st->mn[3 * i], st->mn[3 * i + 1], st->mn[3 * i + 2], st->scale[i]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nstatus; i += gridDim.x * blockDim.x)
        status0[i] = 0;
    __syncthreads();
    const unsigned qmax = (1u << KEY_BITS_PER_AXIS) - 1u;
    // chunks of KEYS_THREADS * KEYS_ITEMS bodies, grid-stride: a block sums
    // its chunks in shared memory and adds each digit count to the global
    // histograms once
    for (int base = blockIdx.x * KEYS_THREADS * KEYS_ITEMS + threadIdx.x; base - (int)threadIdx.x < n;
         base += gridDim.x * KEYS_THREADS * KEYS_ITEMS) {
    // all of the chunk's loads first (KEYS_ITEMS in flight per thread), then
    // the keys and the shared-memory histogram atomics
    float4 qs[KEYS_ITEMS];
    uint8_t ss[KEYS_ITEMS];
#pragma unroll
    for (int k = 0; k < KEYS_ITEMS; k++) {
        const int i = base + k * KEYS_THREADS;
        qs[k] = i < n ? p[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        ss[k] = i < n ? sysid[i] : (uint8_t)0;
    }
#pragma unroll
    for (int k = 0; k < KEYS_ITEMS; k++) {
        int i = base + k * KEYS_THREADS;
        if (i < n) {
            const float4 q = qs[k];
            const float4 dm = s_dom[ss[k]];
            unsigned qx = min((unsigned)(__fsub_rd(q.x, dm.x) * dm.w), qmax);
            unsigned qy = min((unsigned)(__fsub_rd(q.y, dm.y) * dm.w), qmax);
            unsigned qz = min((unsigned)(__fsub_rd(q.z, dm.z) * dm.w), qmax);
            unsigned long long key = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
            keys[i] = key;
            // one shared-memory atomic per digit (counting the digits a warp
            // shares with one atomic per warp measured slower: 23.7 against
            // 18.2 us at 2^20)
#pragma unroll
            for (int d = 0; d < SORT_PASSES; d++)
                atomicAdd(&h[d * SORT_RADIX + (unsigned)((key >> (SORT_BITS * d)) & (SORT_RADIX - 1))], 1u);
        }
    }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SORT_PASSES * SORT_RADIX; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

cudaError_t launch_keys(Ctx &c) {
    int n = (int)c.n;
    int per = KEYS_THREADS * KEYS_ITEMS;
    cudaError_t e = launch_domains(c);
    if (e != cudaSuccess) return e;
    // The sort ping-pongs between c.keys and c.keys_alt and must end in
    // c.keys: with an odd number of passes (one more on the system id for an
    // ensemble) it starts from the alternate buffer.
    const int npass = SORT_PASSES + (c.nsys > 1 ? 1 : 0);
    unsigned long long *out = (npass & 1) ? c.keys_alt : c.keys;
    const int grid = min((n + per - 1) / per, c.num_sms * KEYS_BLOCKS_PER_SM);
    k_keys<<<grid, KEYS_THREADS, 0, c.stream>>>(c.pos4_alt, c.sysid, n, c.nsys, c.st, out, c.tile_status,
                                                c.ntiles * SORT_RADIX);
    return cudaGetLastError();
}

}  // namespace bonsai
