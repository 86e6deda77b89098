// k_judge.cu -- direct summation on a sample of bodies: the labels of the
// learned correction and the per-step judge of its error (paper Sect. 1: the
// O(N^2) method is the exact reference the tree approximates).
//
// For T target bodies (sorted positions) the softened acceleration and
// potential from all N bodies: sources are streamed through shared memory in
// tiles, each tile summed in FP32 and added with Kahan compensation; the
// source range is split over blocks and the partial sums are added in FP32
// with Kahan compensation too (FP64 on the GPU is kept to the root
// multipoles and the energy diagnostics).
// Tiles run on packed FP32x2 arithmetic, two targets per thread.
// The judge then ranks the relative errors of the current accelerations at
// the targets and compares their 99th percentile with a budget.
#include "common.cuh"

namespace bonsai {

#ifndef DS_PAIRS
#define DS_PAIRS 1                     // packed target pairs per thread (2: 3% slower at 2^22 with
#endif                                 // twice the source splits, 21% slower with as many)
constexpr int DS_THREADS = 128;        // threads per block, 2 DS_PAIRS targets each
constexpr int DS_TILE = 256;           // sources per shared tile

__device__ __forceinline__ void kadd(float &s, float &c, float v) {
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Partial sums of split blockIdx.y over sources [chunk*y, chunk*(y+1)).
// Each thread owns 2 DS_PAIRS targets, k + i DS_THREADS (i < 2 DS_PAIRS),
// as DS_PAIRS packed FP32x2 operands; the tile holds every source twice per
// component ((x, x, y, y), (z, z, m, m)), so two broadcast loads feed
// 13 DS_PAIRS packed operations.  Per target the arithmetic and its order
// are those of one scalar loop over the sources.  A non-null gate that
// reads 0 skips the work (all kernels of this file).
__global__ void __launch_bounds__(DS_THREADS)
k_direct_partial(const float4 *__restrict__ pos4, int n, const uint32_t *__restrict__ targets, int ntar,
                 float eps2, int chunk, float4 *partial, const unsigned *__restrict__ gate) {
    if (gate && *gate == 0u) return;
    constexpr int P = DS_PAIRS, TT = 2 * DS_PAIRS;
    __shared__ float4 tile[2 * DS_TILE];
    int kk[TT];
    bool live[TT];
    float2 nx[P], ny[P], nz[P];
#pragma unroll
    for (int i = 0; i < TT; i++) {
        kk[i] = blockIdx.x * TT * DS_THREADS + i * DS_THREADS + threadIdx.x;
        live[i] = kk[i] < ntar;
    }
#pragma unroll
    for (int q = 0; q < P; q++) {
        const float4 m0 = live[2 * q] ? pos4[targets[kk[2 * q]]] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 m1 = live[2 * q + 1] ? pos4[targets[kk[2 * q + 1]]] : make_float4(0.f, 0.f, 0.f, 0.f);
        nx[q] = make_float2(-m0.x, -m1.x); ny[q] = make_float2(-m0.y, -m1.y); nz[q] = make_float2(-m0.z, -m1.z);
    }
    const float2 e2 = make_float2(eps2, eps2);
    float ax[TT], ay[TT], az[TT], ph[TT], cx[TT], cy[TT], cz[TT], cp[TT];
#pragma unroll
    for (int i = 0; i < TT; i++) ax[i] = ay[i] = az[i] = ph[i] = cx[i] = cy[i] = cz[i] = cp[i] = 0.f;
    const int s0 = blockIdx.y * chunk, s1 = min(n, s0 + chunk);
    for (int b = s0; b < s1; b += DS_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < DS_TILE; i += DS_THREADS) {
            const float4 v = b + i < s1 ? pos4[b + i] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
            tile[2 * i] = make_float4(v.x, v.x, v.y, v.y);
            tile[2 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
        }
        __syncthreads();
        float2 px[P], py[P], pz[P], pq[P];                              // pq: +sum m/r
#pragma unroll
        for (int q = 0; q < P; q++) px[q] = py[q] = pz[q] = pq[q] = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int j = 0; j < DS_TILE; j++) {
            const float4 u = tile[2 * j], w = tile[2 * j + 1];
#pragma unroll
            for (int q = 0; q < P; q++) {
                const float2 dx = __fadd2_rn(make_float2(u.x, u.y), nx[q]);
                const float2 dy = __fadd2_rn(make_float2(u.z, u.w), ny[q]);
                const float2 dz = __fadd2_rn(make_float2(w.x, w.y), nz[q]);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e2)));
                const float2 rinv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                const float2 mr = __fmul2_rn(make_float2(w.z, w.w), rinv);
                const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, rinv), rinv);
                pq[q] = __fadd2_rn(pq[q], mr);
                px[q] = __ffma2_rn(mr3, dx, px[q]);
                py[q] = __ffma2_rn(mr3, dy, py[q]);
                pz[q] = __ffma2_rn(mr3, dz, pz[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < P; q++) {
            kadd(ax[2 * q], cx[2 * q], px[q].x); kadd(ay[2 * q], cy[2 * q], py[q].x);
            kadd(az[2 * q], cz[2 * q], pz[q].x); kadd(ph[2 * q], cp[2 * q], -pq[q].x);
            kadd(ax[2 * q + 1], cx[2 * q + 1], px[q].y); kadd(ay[2 * q + 1], cy[2 * q + 1], py[q].y);
            kadd(az[2 * q + 1], cz[2 * q + 1], pz[q].y); kadd(ph[2 * q + 1], cp[2 * q + 1], -pq[q].y);
        }
    }
#pragma unroll
    for (int i = 0; i < TT; i++)
        if (live[i])
            partial[(size_t)blockIdx.y * ntar + kk[i]] =
                make_float4(ax[i] - cx[i], ay[i] - cy[i], az[i] - cz[i], ph[i] - cp[i]);
}

// Sum the splits in order with Kahan compensation (FP32) and remove the
// target's own -m/eps term from the potential.
__global__ void k_direct_reduce(const float4 *__restrict__ pos4, const uint32_t *__restrict__ targets,
                                int ntar, int nsplit, float eps2, const float4 *__restrict__ partial,
                                float4 *out, const unsigned *__restrict__ gate) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ntar || (gate && *gate == 0u)) return;
    float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
    for (int y = 0; y < nsplit; y++) {
        const float4 p = partial[(size_t)y * ntar + k];
        kadd(ax, cx, p.x); kadd(ay, cy, p.y); kadd(az, cz, p.z); kadd(ph, cp, p.w);
    }
    kadd(ph, cp, pos4[targets[k]].w * rsqrtf(eps2));
    out[k] = make_float4(ax - cx, ay - cy, az - cz, ph - cp);
}

cudaError_t launch_direct(Ctx &c, const uint32_t *targets, int ntar, float eps, float4 *partial,
                          int nsplit, float4 *out, const unsigned *gate) {
    const int n = (int)c.n;
    const int chunk = ((n + nsplit - 1) / nsplit + DS_TILE - 1) / DS_TILE * DS_TILE;
    dim3 grid((ntar + 2 * DS_PAIRS * DS_THREADS - 1) / (2 * DS_PAIRS * DS_THREADS), nsplit);
    k_direct_partial<<<grid, DS_THREADS, 0, c.stream>>>(c.pos4, n, targets, ntar, eps * eps, chunk, partial, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_direct_reduce<<<(ntar + 255) / 256, 256, 0, c.stream>>>(c.pos4, targets, ntar, nsplit, eps * eps,
                                                              partial, out, gate);
    return cudaGetLastError();
}

// Judge: relative errors |a - a_direct| / |a_direct| at the targets, their
// 99th percentile (linear interpolation between order statistics, as numpy's
// default), and the fallback flag p99 > budget.  One block of 1024 threads,
// bitonic sort of up to 4096 values in shared memory.  Skipped by the gate,
// it leaves the last judgement (p99 and flag) in place.
__global__ void __launch_bounds__(1024)
k_judge_p99(const float4 *__restrict__ acc4, const uint32_t *__restrict__ targets, int ntar,
            const float4 *__restrict__ direct, float budget, DevState *st, const unsigned *__restrict__ gate) {
    if (gate && *gate == 0u) return;
    __shared__ float v[JUDGE_MAX];
    for (int i = threadIdx.x; i < JUDGE_MAX; i += blockDim.x) {
        float e = INFINITY;
        if (i < ntar) {
            const float4 a = acc4[targets[i]], d = direct[i];
            const float ex = a.x - d.x, ey = a.y - d.y, ez = a.z - d.z;
            const float dn = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            e = dn > 0.f ? sqrtf(ex * ex + ey * ey + ez * ez) / dn : 0.f;
        }
        v[i] = e;
    }
    __syncthreads();
    for (int k = 2; k <= JUDGE_MAX; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < JUDGE_MAX; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const float a = v[i], b = v[l];
                    if ((a > b) == up) { v[i] = b; v[l] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        const float pos = 0.99f * (float)(ntar - 1);
        const int i0 = (int)pos;
        const int i1 = min(i0 + 1, ntar - 1);
        const float p99 = v[i0] + (pos - (float)i0) * (v[i1] - v[i0]);
        st->judge_p99 = p99;
        st->fallback = p99 > budget ? 1u : 0u;
    }
}

cudaError_t launch_judge(Ctx &c, const uint32_t *targets, int ntar, const float4 *direct, float budget,
                         const unsigned *gate) {
    k_judge_p99<<<1, 1024, 0, c.stream>>>(c.acc4, targets, ntar, direct, budget, c.st, gate);
    return cudaGetLastError();
}

}  // namespace bonsai
