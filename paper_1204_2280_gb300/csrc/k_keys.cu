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
__global__ void k_reset(DevState *st, int what) {
    int t = threadIdx.x;
    if (what & 1) {                        // build inputs
        if (t < 3) { st->dom[t] = 0x7fffffff; st->dom[3 + t] = (int)0x80000000; }
        for (int i = t; i < SORT_PASSES * 256; i += blockDim.x) st->hist[i] = 0;
        if (t < SORT_PASSES) st->sort_tile[t] = 0;
    }
    if (what & 2) {                        // walk inputs
        if (t == 0) { st->walk_next = 0; st->walk_next2 = 0; st->inter[0] = 0; st->inter[1] = 0; }
    }
    if (what & 4) {
        if (t < 8) st->diag[t] = 0.0;
    }
}

cudaError_t launch_reset(Ctx &c) {
    k_reset<<<1, 256, 0, c.stream>>>(c.st, 7);
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
// Block min/max of three floats -> one atomic per component per block.
__device__ __forceinline__ void bbox_accumulate(float x, float y, float z, bool valid,
                                                DevState *st) {
    __shared__ float red[6][32];
    float v[6] = {x, y, z, x, y, z};
    if (!valid) { v[0] = v[1] = v[2] = INFINITY; v[3] = v[4] = v[5] = -INFINITY; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            v[d] = fminf(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
            v[3 + d] = fmaxf(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
        }
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
        for (int d = 0; d < 6; d++) red[d][w] = v[d];
    __syncthreads();
    if (w == 0) {
        for (int d = 0; d < 6; d++) {
            float r = l < nw ? red[d][l] : (d < 3 ? INFINITY : -INFINITY);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float s = __shfl_xor_sync(0xffffffffu, r, o);
                r = d < 3 ? fminf(r, s) : fmaxf(r, s);
            }
            if (l == 0) {
                if (d < 3) atomicMin(&st->dom[d], f2ord(r));
                else atomicMax(&st->dom[d], f2ord(r));
            }
        }
    }
}

__global__ void k_bbox(const float4 *__restrict__ p, int n, DevState *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float4 q = i < n ? p[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    bbox_accumulate(q.x, q.y, q.z, i < n, st);
}

cudaError_t launch_bbox(Ctx &c) {
    int n = (int)c.n;
    k_bbox<<<(n + 255) / 256, 256, 0, c.stream>>>(c.pos4_alt, n, c.st);
    return cudaGetLastError();
}

// First half of the kick-drift-kick leapfrog fused with the domain reduction:
// v' = v + a dt/2, x' = x + v' dt (written to the pre-sort arrays).
__global__ void k_kick_drift_bbox(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                  const float4 *__restrict__ acc, const uint32_t *__restrict__ id,
                                  int n, float dt, float4 *pos_o, float4 *vel_o, uint32_t *id_o,
                                  DevState *st) {
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
    bbox_accumulate(x.x, x.y, x.z, i < n, st);
}

cudaError_t launch_kick_drift_bbox(Ctx &c, float dt) {
    int n = (int)c.n;
    k_kick_drift_bbox<<<(n + 255) / 256, 256, 0, c.stream>>>(c.pos4, c.vel4, c.acc4, c.id, n, dt,
                                                             c.pos4_alt, c.vel4_alt, c.id_alt, c.st);
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

constexpr int KEYS_THREADS = 256;
constexpr int KEYS_ITEMS = 8;

// Keys of all bodies plus the 8 digit histograms of the radix sort; also
// clears the pass-0 tile status of the sort.
__global__ void __launch_bounds__(KEYS_THREADS)
k_keys(const float4 *__restrict__ p, int n, DevState *st, unsigned long long *keys,
       unsigned *status0, int nstatus) {
    __shared__ unsigned h[SORT_PASSES * 256];
    __shared__ float s_mn[3], s_scale;
    for (int i = threadIdx.x; i < SORT_PASSES * 256; i += blockDim.x) h[i] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nstatus; i += gridDim.x * blockDim.x)
        status0[i] = 0;
    if (threadIdx.x == 0) {
        float S = 0x1p-64f;
        for (int d = 0; d < 3; d++) {
            float lo = ord2f(st->dom[d]), hi = ord2f(st->dom[3 + d]);
            s_mn[d] = lo;
            S = fmaxf(S, pow2_above_diff(hi, lo));
        }
        int ex;
        frexpf(S, &ex);                    // S = 2^(ex-1)
        s_scale = ldexpf(1.f, KEY_BITS_PER_AXIS - (ex - 1));
        if (blockIdx.x == 0) {
            st->mn[0] = s_mn[0]; st->mn[1] = s_mn[1]; st->mn[2] = s_mn[2];
            st->side = S;
        }
    }
    __syncthreads();
    const float mx = s_mn[0], my = s_mn[1], mz = s_mn[2], sc = s_scale;
    const unsigned qmax = (1u << KEY_BITS_PER_AXIS) - 1u;
    int base = blockIdx.x * KEYS_THREADS * KEYS_ITEMS + threadIdx.x;
#pragma unroll
    for (int k = 0; k < KEYS_ITEMS; k++) {
        int i = base + k * KEYS_THREADS;
        if (i < n) {
            float4 q = p[i];
            unsigned qx = min((unsigned)(__fsub_rd(q.x, mx) * sc), qmax);
            unsigned qy = min((unsigned)(__fsub_rd(q.y, my) * sc), qmax);
            unsigned qz = min((unsigned)(__fsub_rd(q.z, mz) * sc), qmax);
            unsigned long long key = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
            keys[i] = key;
#pragma unroll
            for (int d = 0; d < SORT_PASSES; d++)
                atomicAdd(&h[d * 256 + (unsigned)((key >> (8 * d)) & 0xffu)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SORT_PASSES * 256; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

cudaError_t launch_keys(Ctx &c) {
    int n = (int)c.n;
    int per = KEYS_THREADS * KEYS_ITEMS;
    k_keys<<<(n + per - 1) / per, KEYS_THREADS, 0, c.stream>>>(c.pos4_alt, n, c.st, c.keys,
                                                              c.tile_status, c.ntiles * 256);
    return cudaGetLastError();
}

}  // namespace bonsai
