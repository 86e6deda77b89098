// mlp.cu -- the learned far-field correction: a per-body MLP 12 -> 64 -> 64
// -> 3 (ReLU) that predicts, from features the walk already produces, the
// residual between the coarse-theta tree acceleration and the direct sum:
//   y = (a_direct - a_tree) / |a_tree| / ysig,   a_corrected = a_tree + ysig y |a_tree|.
//
// Arithmetic (the same in training and inference): inputs normalised in FP32
// ((x - mu) / sigma), then inputs, weights and hidden activations rounded to
// BF16, products accumulated in FP32, biases FP32.  Inference runs on the
// tensor cores (mma.sync m16n8k16, BF16 x BF16 -> FP32; the accumulator
// layout of one layer is the A-fragment layout of the next, so activations
// never leave registers).  Training: one thread per sample for forward and
// backward in FP32 on the same BF16-rounded values, warp-reduced gradients,
// AdamW on FP32 master weights.
//
// The correction is rotation-equivariant: the 12 inputs are invariants of
// the body (log|a_tree|, log(-phi_tree), log(1 + accepted cells) in the level
// bins 0-3, 4-6, 7-9, 10-21, log(1 + body-body interactions), log of the
// group density n_G / (e_G^3 + eps^3), log((d_G + eps)/eps), the offset o of
// the body from its group box's centre as |o| / (d_G / 2) and the cosine
// between o and a_tree, log n_G), and the 3 outputs are the coefficients of
// the residual along a body-local frame: e0 = a_tree/|a_tree|, e1 = the unit
// part of o orthogonal to e0 (the coordinate axis least aligned with e0 when
// o is parallel to e0 or zero), e2 = e0 x e1.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace bonsai {

// Parameter block layout (FP32 master copy, row-major W[out][in]).
constexpr int OFF_W1 = 0;                       // 64 x 12
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_IN;  // 64
constexpr int OFF_W2 = OFF_B1 + MLP_H;           // 64 x 64
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;   // 64
constexpr int OFF_W3 = OFF_B2 + MLP_H;           // 3 x 64
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_H; // 3
static_assert(OFF_B3 + MLP_OUT == MLP_NPARAM, "parameter count");

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

struct Frame {
    float3 e0, e1, e2;
    float an;
};

// The 12 raw (unnormalised) inputs of a body and its local frame, from its
// tree acceleration/potential and its walk features f (FEAT_STRIDE floats).
__device__ __forceinline__ void body_inputs(const float4 a, const float *__restrict__ f, float (&x)[MLP_IN],
                                            Frame &F) {
    const float an = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
    F.an = an;
    float3 e0 = an > 0.f ? make_float3(a.x / an, a.y / an, a.z / an) : make_float3(1.f, 0.f, 0.f);
    const float ox = f[7], oy = f[8], oz = f[9];
    const float on = sqrtf(ox * ox + oy * oy + oz * oz);
    const float od = ox * e0.x + oy * e0.y + oz * e0.z;
    float px = ox - od * e0.x, py = oy - od * e0.y, pz = oz - od * e0.z;
    float pn = sqrtf(px * px + py * py + pz * pz);
    if (!(pn > 1e-6f * on && pn > 0.f)) {      // o zero or along e0: least-aligned axis
        const float ax = fabsf(e0.x), ay = fabsf(e0.y), az = fabsf(e0.z);
        const float ux = (ax <= ay && ax <= az) ? 1.f : 0.f;
        const float uy = (ux == 0.f && ay <= az) ? 1.f : 0.f;
        const float uz = (ux == 0.f && uy == 0.f) ? 1.f : 0.f;
        const float ud = ux * e0.x + uy * e0.y + uz * e0.z;
        px = ux - ud * e0.x; py = uy - ud * e0.y; pz = uz - ud * e0.z;
        pn = sqrtf(px * px + py * py + pz * pz);
    }
    const float3 e1 = make_float3(px / pn, py / pn, pz / pn);
    F.e0 = e0;
    F.e1 = e1;
    F.e2 = make_float3(e0.y * e1.z - e0.z * e1.y, e0.z * e1.x - e0.x * e1.z, e0.x * e1.y - e0.y * e1.x);
    const float diag = f[11];
    x[0] = logf(fmaxf(an, 1e-30f));
    x[1] = logf(fmaxf(-a.w, 1e-30f));
#pragma unroll
    for (int k = 0; k < 7; k++) x[2 + k] = f[k];
    x[9] = diag > 0.f ? on / (0.5f * diag) : 0.f;
    x[10] = on > 0.f ? od / on : 0.f;
    x[11] = f[10];
}

// The 12 inputs of a body, normalised (FP32, before BF16 rounding).
__device__ __forceinline__ void body_features(const float4 a, const float *__restrict__ wf,
                                              const float *__restrict__ norm, float (&x)[MLP_IN], Frame &F) {
    body_inputs(a, wf, x, F);
#pragma unroll
    for (int k = 0; k < MLP_IN; k++) x[k] = (x[k] - norm[k]) / norm[MLP_IN + k];
}

// ---------------------------------------------------------------------------
// Inference on tensor cores.  One warp per 16 bodies.
// ---------------------------------------------------------------------------
constexpr int INF_WARPS = 4;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights as BF16 pairs in shared memory: W1 64 x 16 (inputs padded to 16),
// W2 64 x 64, W3 8 x 64 (outputs padded to 8); row n holds W[n][k..].
struct InfShared {
    uint32_t w1[MLP_H * 8];
    uint32_t w2[MLP_H * 32];
    uint32_t w3[8 * 32];
    float b1[MLP_H], b2[MLP_H], b3[8];
    float norm[2 * MLP_IN], ysig;
    float xs[INF_WARPS][16][17];
    float ys[INF_WARPS][16][4];
    float fr[INF_WARPS][16][10];     // frame e0 e1 e2 and |a| of each row
};

__device__ void stage_weights(InfShared &S, const float *__restrict__ P, const float *__restrict__ norm) {
    const int tid = threadIdx.x;
    for (int i = tid; i < MLP_H * 8; i += blockDim.x) {
        const int r = i / 8, c = 2 * (i % 8);
        const float a = c < MLP_IN ? P[OFF_W1 + r * MLP_IN + c] : 0.f;
        const float b = c + 1 < MLP_IN ? P[OFF_W1 + r * MLP_IN + c + 1] : 0.f;
        S.w1[i] = pack_bf16(a, b);
    }
    for (int i = tid; i < MLP_H * 32; i += blockDim.x) {
        const int r = i / 32, c = 2 * (i % 32);
        S.w2[i] = pack_bf16(P[OFF_W2 + r * MLP_H + c], P[OFF_W2 + r * MLP_H + c + 1]);
    }
    for (int i = tid; i < 8 * 32; i += blockDim.x) {
        const int r = i / 32, c = 2 * (i % 32);
        S.w3[i] = r < MLP_OUT ? pack_bf16(P[OFF_W3 + r * MLP_H + c], P[OFF_W3 + r * MLP_H + c + 1]) : 0u;
    }
    for (int i = tid; i < MLP_H; i += blockDim.x) { S.b1[i] = P[OFF_B1 + i]; S.b2[i] = P[OFF_B2 + i]; }
    if (tid < 8) S.b3[tid] = tid < MLP_OUT ? P[OFF_B3 + tid] : 0.f;
    if (tid < 2 * MLP_IN) S.norm[tid] = norm[tid];
    if (tid == 0) S.ysig = norm[2 * MLP_IN];
}

__device__ __forceinline__ void relu_pack(const float (&h)[8][4], uint32_t (&a2)[4][4]) {
#pragma unroll
    for (int kc = 0; kc < 4; kc++) {
        a2[kc][0] = pack_bf16(fmaxf(h[2 * kc][0], 0.f), fmaxf(h[2 * kc][1], 0.f));
        a2[kc][1] = pack_bf16(fmaxf(h[2 * kc][2], 0.f), fmaxf(h[2 * kc][3], 0.f));
        a2[kc][2] = pack_bf16(fmaxf(h[2 * kc + 1][0], 0.f), fmaxf(h[2 * kc + 1][1], 0.f));
        a2[kc][3] = pack_bf16(fmaxf(h[2 * kc + 1][2], 0.f), fmaxf(h[2 * kc + 1][3], 0.f));
    }
}

// Forward of 16 rows (normalised inputs xs[16][<=16]) on the tensor cores;
// the raw outputs land in ys[16][0..2].  Whole warp.
__device__ void mma_forward16(const InfShared &S, const float (*xs)[17], float (*ys)[4], int lane) {
    const int g = lane >> 2, t = lane & 3;
    uint32_t a[4] = {pack_bf16(xs[g][2 * t], xs[g][2 * t + 1]), pack_bf16(xs[g + 8][2 * t], xs[g + 8][2 * t + 1]),
                     pack_bf16(xs[g][2 * t + 8], xs[g][2 * t + 9]),
                     pack_bf16(xs[g + 8][2 * t + 8], xs[g + 8][2 * t + 9])};
    float h[8][4];
#pragma unroll
    for (int j = 0; j < 8; j++) {                 // layer 1: 8 n-tiles of 8 hidden units
        const int col = 8 * j + 2 * t, row = 8 * j + g;
        h[j][0] = S.b1[col]; h[j][1] = S.b1[col + 1]; h[j][2] = S.b1[col]; h[j][3] = S.b1[col + 1];
        mma_bf16(h[j], a, S.w1[row * 8 + t], S.w1[row * 8 + t + 4]);
    }
    uint32_t a2[4][4];
    relu_pack(h, a2);                             // accumulator layout == next A layout
#pragma unroll
    for (int j = 0; j < 8; j++) {                 // layer 2
        const int col = 8 * j + 2 * t, row = 8 * j + g;
        h[j][0] = S.b2[col]; h[j][1] = S.b2[col + 1]; h[j][2] = S.b2[col]; h[j][3] = S.b2[col + 1];
#pragma unroll
        for (int kc = 0; kc < 4; kc++)
            mma_bf16(h[j], a2[kc], S.w2[row * 32 + 8 * kc + t], S.w2[row * 32 + 8 * kc + t + 4]);
    }
    relu_pack(h, a2);
    float y[4] = {S.b3[2 * t], S.b3[2 * t + 1], S.b3[2 * t], S.b3[2 * t + 1]};
#pragma unroll
    for (int kc = 0; kc < 4; kc++)                // layer 3 (outputs padded to 8)
        mma_bf16(y, a2[kc], S.w3[g * 32 + 8 * kc + t], S.w3[g * 32 + 8 * kc + t + 4]);
    if (t < 2) {
        ys[g][2 * t] = y[0]; ys[g][2 * t + 1] = y[1];
        ys[g + 8][2 * t] = y[2]; ys[g + 8][2 * t + 1] = y[3];
    }
}

// Corrects the tree accelerations in place: a += ysig |a| (y0 e0 + y1 e1 + y2 e2).
__global__ void __launch_bounds__(INF_WARPS * 32)
k_mlp_infer(const float *__restrict__ P, const float *__restrict__ norm, float4 *acc4,
            const float *__restrict__ feat, int n, const DevState *__restrict__ st) {
    __shared__ InfShared S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (st->status & ST_TIMEOUT) return;
    stage_weights(S, P, norm);
    __syncthreads();
    const int nwarps_total = gridDim.x * INF_WARPS;
    for (int base = (blockIdx.x * INF_WARPS + warp) * 16; base < n; base += nwarps_total * 16) {
        if (lane < 16) {
            const int i = base + lane;
            float x[MLP_IN];
            Frame F{};
            if (i < n) {
                body_features(acc4[i], feat + FEAT_STRIDE * (size_t)i, S.norm, x, F);
            } else {
#pragma unroll
                for (int k = 0; k < MLP_IN; k++) x[k] = 0.f;
            }
            float *fr = S.fr[warp][lane];
            fr[0] = F.e0.x; fr[1] = F.e0.y; fr[2] = F.e0.z; fr[3] = F.e1.x; fr[4] = F.e1.y;
            fr[5] = F.e1.z; fr[6] = F.e2.x; fr[7] = F.e2.y; fr[8] = F.e2.z; fr[9] = F.an;
#pragma unroll
            for (int k = 0; k < MLP_IN; k++) S.xs[warp][lane][k] = x[k];
#pragma unroll
            for (int k = MLP_IN; k < 16; k++) S.xs[warp][lane][k] = 0.f;
        }
        __syncwarp();
        mma_forward16(S, S.xs[warp], S.ys[warp], lane);
        __syncwarp();
        if (lane < 16 && base + lane < n) {
            const int i = base + lane;
            float4 av = acc4[i];
            const float *fr = S.fr[warp][lane];
            const float s = fr[9] * S.ysig;
            const float c0 = S.ys[warp][lane][0] * s, c1 = S.ys[warp][lane][1] * s, c2 = S.ys[warp][lane][2] * s;
            av.x += c0 * fr[0] + c1 * fr[3] + c2 * fr[6];
            av.y += c0 * fr[1] + c1 * fr[4] + c2 * fr[7];
            av.z += c0 * fr[2] + c1 * fr[5] + c2 * fr[8];
            acc4[i] = av;
        }
        __syncwarp();
    }
}

// Raw network outputs for feature rows X (n x 12, not normalised) -> Y (n x 3).
__global__ void __launch_bounds__(INF_WARPS * 32)
k_mlp_rows(const float *__restrict__ P, const float *__restrict__ norm, const float *__restrict__ X,
           float *Y, int n) {
    __shared__ InfShared S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    stage_weights(S, P, norm);
    __syncthreads();
    const int nwarps_total = gridDim.x * INF_WARPS;
    for (int base = (blockIdx.x * INF_WARPS + warp) * 16; base < n; base += nwarps_total * 16) {
        if (lane < 16) {
            const int i = base + lane;
#pragma unroll
            for (int k = 0; k < 16; k++)
                S.xs[warp][lane][k] = (k < MLP_IN && i < n)
                                          ? (X[(size_t)i * MLP_IN + k] - S.norm[k]) / S.norm[MLP_IN + k]
                                          : 0.f;
        }
        __syncwarp();
        mma_forward16(S, S.xs[warp], S.ys[warp], lane);
        __syncwarp();
        if (lane < 16 && base + lane < n)
            for (int o = 0; o < MLP_OUT; o++) Y[(size_t)(base + lane) * MLP_OUT + o] = S.ys[warp][lane][o];
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Training: forward + backward, one thread per sample.
// ---------------------------------------------------------------------------
constexpr int TR_THREADS = 256;

struct TrShared {
    float w[MLP_NPARAM];      // BF16-rounded weights (biases exact)
    float g[MLP_NPARAM];      // block gradient sums
    float loss;
};

// X: n x 12 raw features, Y: n x 3 targets (divided by ysig here), idx:
// the samples of this batch.  grad += d(loss)/dP with loss = mean over the
// batch and the 3 outputs of the squared error.
__global__ void __launch_bounds__(TR_THREADS)
k_mlp_grad(const float *__restrict__ P, const float *__restrict__ norm, const float *__restrict__ X,
           const float *__restrict__ Y, const uint32_t *__restrict__ idx, int bsz, float *grad,
           float *loss) {
    extern __shared__ float smem_f[];
    TrShared &S = *reinterpret_cast<TrShared *>(smem_f);
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < MLP_NPARAM; i += blockDim.x) {
        const bool bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) || i >= OFF_B3;
        S.w[i] = bias ? P[i] : bf16r(P[i]);
        S.g[i] = 0.f;
    }
    if (tid == 0) S.loss = 0.f;
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + tid;
    const bool live = k < bsz;
    const uint32_t sidx = live ? idx[k] : 0u;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; i++)
        x[i] = live ? bf16r((X[(size_t)sidx * MLP_IN + i] - norm[i]) / norm[MLP_IN + i]) : 0.f;
    float h1[MLP_H], h2[MLP_H];
    for (int j = 0; j < MLP_H; j++) {
        float s = S.w[OFF_B1 + j];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) s = fmaf(S.w[OFF_W1 + j * MLP_IN + i], x[i], s);
        h1[j] = bf16r(fmaxf(s, 0.f));
    }
    for (int j = 0; j < MLP_H; j++) {
        float s = S.w[OFF_B2 + j];
        for (int i = 0; i < MLP_H; i++) s = fmaf(S.w[OFF_W2 + j * MLP_H + i], h1[i], s);
        h2[j] = bf16r(fmaxf(s, 0.f));
    }
    float dy[MLP_OUT];
    float l = 0.f;
    const float sc = 2.f / (3.f * (float)bsz);
#pragma unroll
    for (int o = 0; o < MLP_OUT; o++) {
        float s = S.w[OFF_B3 + o];
        for (int i = 0; i < MLP_H; i++) s = fmaf(S.w[OFF_W3 + o * MLP_H + i], h2[i], s);
        const float r = live ? s - Y[(size_t)sidx * MLP_OUT + o] / norm[2 * MLP_IN] : 0.f;
        l += r * r;
        dy[o] = sc * r;
    }
    // Backward: dh2 = W3^T dy (ReLU gate), dh1 = W2^T dh2 (ReLU gate).
    float dh2[MLP_H];
    for (int i = 0; i < MLP_H; i++) {
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < MLP_OUT; o++) s = fmaf(S.w[OFF_W3 + o * MLP_H + i], dy[o], s);
        dh2[i] = h2[i] > 0.f ? s : 0.f;
    }
    float dh1[MLP_H];
    for (int i = 0; i < MLP_H; i++) {
        float s = 0.f;
        for (int j = 0; j < MLP_H; j++) s = fmaf(S.w[OFF_W2 + j * MLP_H + i], dh2[j], s);
        dh1[i] = h1[i] > 0.f ? s : 0.f;
    }
    // Warp-reduced parameter gradients, then shared, then global.
    auto put = [&](int p, float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&S.g[p], v);
    };
    for (int o = 0; o < MLP_OUT; o++) {
        put(OFF_B3 + o, dy[o]);
        for (int i = 0; i < MLP_H; i++) put(OFF_W3 + o * MLP_H + i, dy[o] * h2[i]);
    }
    for (int j = 0; j < MLP_H; j++) {
        put(OFF_B2 + j, dh2[j]);
        for (int i = 0; i < MLP_H; i++) put(OFF_W2 + j * MLP_H + i, dh2[j] * h1[i]);
    }
    for (int j = 0; j < MLP_H; j++) {
        put(OFF_B1 + j, dh1[j]);
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) put(OFF_W1 + j * MLP_IN + i, dh1[j] * x[i]);
    }
    {
        float v = l;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&S.loss, v);
    }
    __syncthreads();
    for (int i = tid; i < MLP_NPARAM; i += blockDim.x) atomicAdd(&grad[i], S.g[i]);
    if (tid == 0) atomicAdd(loss, S.loss / (3.f * (float)bsz));
}

// AdamW (decoupled weight decay on the weight matrices, not the biases).
__global__ void k_adamw(float *P, const float *__restrict__ grad, float *m, float *v, float lr, float b1,
                        float b2, float eps, float wd, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const bool bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) || i >= OFF_B3;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float w = P[i];
    w -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + (bias ? 0.f : wd * w));
    P[i] = w;
}

cudaError_t launch_mlp_infer(Ctx &c, const float *P, const float *norm) {
    const int n = (int)c.n;
    int blocks = (n + INF_WARPS * 16 - 1) / (INF_WARPS * 16);
    const int cap = c.num_sms * 8;
    if (blocks > cap) blocks = cap;
    k_mlp_infer<<<blocks, INF_WARPS * 32, 0, c.stream>>>(P, norm, c.acc4, c.feat, n, c.st);
    return cudaGetLastError();
}

cudaError_t launch_mlp_rows(cudaStream_t s, const float *P, const float *norm, const float *X, float *Y, int n) {
    int blocks = (n + INF_WARPS * 16 - 1) / (INF_WARPS * 16);
    if (blocks > 1216) blocks = 1216;
    k_mlp_rows<<<blocks, INF_WARPS * 32, 0, s>>>(P, norm, X, Y, n);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(cudaStream_t s, const float *P, const float *norm, const float *X, const float *Y,
                            const uint32_t *idx, int bsz, float *grad, float *loss) {
    static size_t attr_done[MAX_DEVICES] = {};
    const size_t smem = sizeof(TrShared);
    cudaError_t e = allow_dyn_smem((const void *)k_mlp_grad, smem, attr_done);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<(bsz + TR_THREADS - 1) / TR_THREADS, TR_THREADS, smem, s>>>(P, norm, X, Y, idx, bsz, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adamw(cudaStream_t s, float *P, const float *grad, float *m, float *v, float lr, float wd,
                         int step) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_adamw<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, grad, m, v, lr, b1, b2, 1e-8f, wd, bc1, bc2);
    return cudaGetLastError();
}

// Per-body features in caller-independent form for training sets:
// X[k] (12 raw inputs) of the sampled sorted positions.
__global__ void k_gather_features(const float4 *__restrict__ acc4, const float *__restrict__ feat,
                                  const uint32_t *__restrict__ targets, int ntar, float *X,
                                  const uint32_t *__restrict__ id, uint32_t *ids) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ntar) return;
    const uint32_t i = targets[k];
    if (ids) ids[k] = id[i];
    float x[MLP_IN];
    Frame F;
    body_inputs(acc4[i], feat + FEAT_STRIDE * (size_t)i, x, F);
    for (int j = 0; j < MLP_IN; j++) X[(size_t)k * MLP_IN + j] = x[j];
}

cudaError_t launch_gather_features(Ctx &c, const uint32_t *targets, int ntar, float *X, uint32_t *ids) {
    k_gather_features<<<(ntar + 255) / 256, 256, 0, c.stream>>>(c.acc4, c.feat, targets, ntar, X, c.id, ids);
    return cudaGetLastError();
}

// Training targets: the relative residual r = (a_direct - a_tree) / |a_tree|
// at target k in the body's local frame, Y[k] = (r.e0, r.e1, r.e2).
__global__ void k_labels(const float4 *__restrict__ acc4, const float *__restrict__ feat,
                         const uint32_t *__restrict__ targets, int ntar, const float4 *__restrict__ direct,
                         float *Y) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ntar) return;
    const uint32_t i = targets[k];
    const float4 a = acc4[i], d = direct[k];
    float x[MLP_IN];
    Frame F;
    body_inputs(a, feat + FEAT_STRIDE * (size_t)i, x, F);
    const float inv = F.an > 0.f ? 1.f / F.an : 0.f;
    const float rx = (d.x - a.x) * inv, ry = (d.y - a.y) * inv, rz = (d.z - a.z) * inv;
    Y[3 * (size_t)k] = rx * F.e0.x + ry * F.e0.y + rz * F.e0.z;
    Y[3 * (size_t)k + 1] = rx * F.e1.x + ry * F.e1.y + rz * F.e1.z;
    Y[3 * (size_t)k + 2] = rx * F.e2.x + ry * F.e2.y + rz * F.e2.z;
}

cudaError_t launch_labels(Ctx &c, const uint32_t *targets, int ntar, const float4 *direct, float *Y) {
    k_labels<<<(ntar + 255) / 256, 256, 0, c.stream>>>(c.acc4, c.feat, targets, ntar, direct, Y);
    return cudaGetLastError();
}

// Input normalisation of a training set: per-feature mean and standard
// deviation (FP64 sums), and the RMS of the targets.  One block.
__global__ void __launch_bounds__(1024) k_feature_stats(const float *__restrict__ X, const float *__restrict__ Y,
                                                        int n, float *norm) {
    __shared__ double red[32][2 * MLP_IN + 1];
    double s[MLP_IN], q[MLP_IN], yy = 0.0;
    for (int k = 0; k < MLP_IN; k++) { s[k] = 0.0; q[k] = 0.0; }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        for (int k = 0; k < MLP_IN; k++) {
            const double v = X[(size_t)i * MLP_IN + k];
            s[k] += v; q[k] += v * v;
        }
        for (int o = 0; o < MLP_OUT; o++) { const double v = Y[(size_t)i * MLP_OUT + o]; yy += v * v; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < MLP_IN; k++) {
        for (int o = 16; o > 0; o >>= 1) {
            s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
            q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
        }
    }
    for (int o = 16; o > 0; o >>= 1) yy += __shfl_xor_sync(0xffffffffu, yy, o);
    if (lane == 0) {
        for (int k = 0; k < MLP_IN; k++) { red[w][k] = s[k]; red[w][MLP_IN + k] = q[k]; }
        red[w][2 * MLP_IN] = yy;
    }
    __syncthreads();
    if (threadIdx.x < 2 * MLP_IN + 1) {
        double t = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); j++) t += red[j][threadIdx.x];
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x < MLP_IN) {
        const int k = threadIdx.x;
        const double mu = red[0][k] / n, var = red[0][MLP_IN + k] / n - mu * mu;
        norm[k] = (float)mu;
        norm[MLP_IN + k] = (float)fmax(sqrt(fmax(var, 0.0)), 1e-6);
    }
    if (threadIdx.x == 0) norm[2 * MLP_IN] = (float)fmax(sqrt(red[0][2 * MLP_IN] / (3.0 * n)), 1e-12);
}

cudaError_t launch_feature_stats(cudaStream_t s, const float *X, const float *Y, int n, float *norm) {
    k_feature_stats<<<1, 1024, 0, s>>>(X, Y, n, norm);
    return cudaGetLastError();
}

}  // namespace bonsai
