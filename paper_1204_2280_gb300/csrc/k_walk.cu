// k_walk.cu -- the group-wise Barnes-Hut tree-traverse (paper Sect. 2,
// "tree-traverse"; MAC after Barnes 1994 combined with the vector-machine
// group walk of Barnes 1990).  This is the dominant kernel (>80% of a step).
//
// One warp owns one group (<= 64 bodies that share an interaction list).  A
// persistent grid pulls groups from one atomic queue in key order -- for an
// ensemble, the groups of all systems, each walked from its own root.  Per warp:
//  * a stack of child ranges (first child, count <= 8) in shared memory; each
//    round pops up to 32 cells, one per lane, and tests them against the
//    group's bounding box: a cell is opened when the squared distance from its
//    com to the box is below r_open^2 (r_open = l/theta + delta);
//  * accepted cells are staged (com, M, Q) into a 64-slot ring in shared
//    memory; the bodies of opened leaves into a second ring; opened internal
//    cells push their child range;
//  * whenever a ring holds 32 sources the warp evaluates that tile: every
//    lane streams the sources from shared memory (broadcast reads) two at a
//    time through the packed FP32x2 instructions (add/mul/fma .f32x2, one
//    issue slot for two operations).  Groups of <= 32 bodies: a group of n
//    bodies uses s = max(2, next_pow2(n)) body slots and the 32/s lanes
//    sharing a body split the tile's 16 source pairs (summed at the end), so
//    small groups still keep all lanes busy.  Groups of 17..24 bodies (at
//    most 32 per group) run in a second instantiation with three bodies per
//    lane in 8 body slots and four phases, 24 body places where one body per
//    lane would leave 8..15 of 32 lanes empty; groups of 33..64 bodies (larger
//    ncrit) in one with two bodies per lane.  The bodies of a lane share
//    every source read;
//  * each tile is summed in plain FP32 and added to the body's accumulators
//    with Kahan compensation (one compensated add per tile and component).
// Body-cell (monopole + traceless quadrupole, softened):
//   d = com - x, r^2 = |d|^2 + eps^2, q = d.Q.d
//   phi -= M/r + q/(2 r^5),  a += ((M/r + 5q/(2 r^5)) / r^2) d - Q d / r^5
// Body-body: a += m d / r^3, phi -= m / r.  The body's own term has d = 0
// (zero force); its potential -m/eps is removed after the walk.
#include "common.cuh"

namespace bonsai {

constexpr int RING = 64;          // sources per ring
constexpr int RPAIR = RING / 2;   // source pairs per ring
#ifndef WALK_UNROLL
#define WALK_UNROLL 8             // unroll depth of the tile loops (4: 1% slower, 16: 9% slower)
#endif
constexpr int kWalkUnroll = WALK_UNROLL;

// Rings in source-pair layout: pair k holds sources 2k (low half) and 2k+1
// (high half) of two components per float4, so one 16-byte shared load
// yields two packed (even, odd) operand pairs for the FP32x2 instructions.
// Quadrupoles arrive negated from the cell arrays, which turns every
// subtraction of the body-cell formula into an addition.
struct WarpRings {
    float4 c0[RPAIR];   // x x' y y'
    float4 c1[RPAIR];   // z z' M M'
    float4 c2[RPAIR];   // -Qxx -Qxx' -Qyy -Qyy'
    float4 c3[RPAIR];   // -Qzz -Qzz' -Qxy -Qxy'
    float4 c4[RPAIR];   // -Qxz -Qxz' -Qyz -Qyz'
    float4 b0[RPAIR];   // body sources: x x' y y'
    float4 b1[RPAIR];   //               z z' m m'
    uint2 leaf[32];     // opened leaves of a round: first body, offset in the round's body list
};

// Staging into pair layout: component array i of a ring or tile starts at
// base + i * STRIDE float4s; source s goes to pair s/2, half s%2.
// qa, qb: -Q as stored in the cell arrays.
template <int STRIDE>
__device__ __forceinline__ void put_cell_at(float4 *base, int s, const float4 mo, const float4 qa, const float2 qb) {
    float *f = reinterpret_cast<float *>(base + (s >> 1)) + (s & 1);
    constexpr int C = 4 * STRIDE;               // floats between component arrays
    f[0] = mo.x; f[2] = mo.y; f[C] = mo.z; f[C + 2] = mo.w;
    f[2 * C] = qa.x; f[2 * C + 2] = qa.y; f[3 * C] = qa.z; f[3 * C + 2] = qa.w;
    f[4 * C] = qb.x; f[4 * C + 2] = qb.y;
}

template <int STRIDE>
__device__ __forceinline__ void put_body_at(float4 *base, int s, const float4 p) {
    float *f = reinterpret_cast<float *>(base + (s >> 1)) + (s & 1);
    constexpr int C = 4 * STRIDE;
    f[0] = p.x; f[2] = p.y; f[C] = p.z; f[C + 2] = p.w;
}

__device__ __forceinline__ void put_cell(WarpRings &R, int s, const float4 mo, const float4 qa, const float2 qb) {
    put_cell_at<RPAIR>(R.c0, s, mo, qa, qb);
}

__device__ __forceinline__ void put_body(WarpRings &R, int s, const float4 p) { put_body_at<RPAIR>(R.b0, s, p); }

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

struct Acc {
    float ax, ay, az, ph;    // running sums
    float cx, cy, cz, cp;    // Kahan compensations
};

// Per-tile partial sums of one body: (even sources, odd sources) pairs; the
// potential is summed with the opposite sign (mr + q/(2 r^5) > 0 terms).
struct Part2 {
    float2 x, y, z, p;
};

// The body as packed operands: negated coordinates in both halves.
struct Me2 {
    float2 nx, ny, nz;
};

__device__ __forceinline__ Me2 me2_of(const float4 me) {
    return Me2{make_float2(-me.x, -me.x), make_float2(-me.y, -me.y), make_float2(-me.z, -me.z)};
}

// Two body-cell interactions (sources 2k, 2k+1) of one body:
//   d = com - x, r^2 = |d|^2 + eps^2, q = d.Q.d,
//   phi -= M/r + q/(2 r^5),  a += ((M/r + 5q/(2 r^5)) / r^2) d - Q d / r^5,
// with -Q staged, so q and Q d arrive negated (33 FP32 operations each).
__device__ __forceinline__ void pc_two(const float4 v0, const float4 v1, const float4 v2, const float4 v3,
                                       const float4 v4, const Me2 &m, const float2 eps2, Part2 &P) {
    const float2 dx = __fadd2_rn(make_float2(v0.x, v0.y), m.nx);
    const float2 dy = __fadd2_rn(make_float2(v0.z, v0.w), m.ny);
    const float2 dz = __fadd2_rn(make_float2(v1.x, v1.y), m.nz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, eps2)));
    const float2 rinv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
    const float2 rinv2 = __fmul2_rn(rinv, rinv);
    const float2 mr = __fmul2_rn(make_float2(v1.z, v1.w), rinv);
    const float2 nqxx = make_float2(v2.x, v2.y), nqyy = make_float2(v2.z, v2.w);
    const float2 nqzz = make_float2(v3.x, v3.y), nqxy = make_float2(v3.z, v3.w);
    const float2 nqxz = make_float2(v4.x, v4.y), nqyz = make_float2(v4.z, v4.w);
    const float2 qx = __ffma2_rn(nqxy, dy, __ffma2_rn(nqxz, dz, __fmul2_rn(nqxx, dx)));   // -(Q d)
    const float2 qy = __ffma2_rn(nqxy, dx, __ffma2_rn(nqyz, dz, __fmul2_rn(nqyy, dy)));
    const float2 qz = __ffma2_rn(nqxz, dx, __ffma2_rn(nqyz, dy, __fmul2_rn(nqzz, dz)));
    const float2 q = __ffma2_rn(dz, qz, __ffma2_rn(dy, qy, __fmul2_rn(dx, qx)));          // -q
    const float2 rinv5 = __fmul2_rn(__fmul2_rn(rinv2, rinv2), rinv);
    const float2 qr5 = __fmul2_rn(q, rinv5);                                               // -q / r^5
    P.p = __fadd2_rn(P.p, __ffma2_rn(make_float2(-0.5f, -0.5f), qr5, mr));
    const float2 sc = __fmul2_rn(__ffma2_rn(make_float2(-2.5f, -2.5f), qr5, mr), rinv2);   // (M/r + 5q/(2r^5)) / r^2
    P.x = __ffma2_rn(rinv5, qx, __ffma2_rn(sc, dx, P.x));
    P.y = __ffma2_rn(rinv5, qy, __ffma2_rn(sc, dy, P.y));
    P.z = __ffma2_rn(rinv5, qz, __ffma2_rn(sc, dz, P.z));
}

// Two body-body interactions: a += m d / r^3, phi -= m / r.
__device__ __forceinline__ void pp_two(const float4 v0, const float4 v1, const Me2 &m, const float2 eps2,
                                       Part2 &P) {
    const float2 dx = __fadd2_rn(make_float2(v0.x, v0.y), m.nx);
    const float2 dy = __fadd2_rn(make_float2(v0.z, v0.w), m.ny);
    const float2 dz = __fadd2_rn(make_float2(v1.x, v1.y), m.nz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, eps2)));
    const float2 rinv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
    const float2 mr = __fmul2_rn(make_float2(v1.z, v1.w), rinv);
    const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, rinv), rinv);
    P.p = __fadd2_rn(P.p, mr);
    P.x = __ffma2_rn(mr3, dx, P.x);
    P.y = __ffma2_rn(mr3, dy, P.y);
    P.z = __ffma2_rn(mr3, dz, P.z);
}

// Adds a tile's partial sums to the compensated accumulators (one Kahan add
// per component).
template <int BPL>
__device__ __forceinline__ void commit(const Part2 (&P)[BPL], Acc (&A)[BPL]) {
#pragma unroll
    for (int b = 0; b < BPL; b++) {
        kahan_add(A[b].ax, A[b].cx, __fadd_rn(P[b].x.x, P[b].x.y));
        kahan_add(A[b].ay, A[b].cy, __fadd_rn(P[b].y.x, P[b].y.y));
        kahan_add(A[b].az, A[b].cz, __fadd_rn(P[b].z.x, P[b].z.y));
        kahan_add(A[b].ph, A[b].cp, -__fadd_rn(P[b].p.x, P[b].p.y));
    }
}

// Tile evaluation.  NPH lanes share one body and split the tile's 16 source
// pairs (lane phase p takes pairs p, p+NPH, ...): the trip count 16/NPH and
// the stride are compile-time constants, so the shared-memory reads use
// immediate offsets and there is no per-interaction loop bookkeeping.  Each
// lane holds BPL bodies that reuse every source read.  Partial tiles are
// padded with massless sources far away, which add exactly zero.
template <int NPH, int BPL, int STRIDE>
__device__ __forceinline__ void eval_pc(const float4 *__restrict__ base, int phase, const float4 (&me)[BPL],
                                        const float2 eps2, Acc (&A)[BPL]) {
    constexpr int T = 16 / NPH;
    const int k0 = phase;
    Me2 m[BPL];
    Part2 P[BPL];
#pragma unroll
    for (int b = 0; b < BPL; b++) {
        m[b] = me2_of(me[b]);
        P[b] = Part2{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
#pragma unroll kWalkUnroll
    for (int j = 0; j < T; j++) {
        const int k = k0 + j * NPH;
        const float4 v0 = base[k], v1 = base[STRIDE + k], v2 = base[2 * STRIDE + k],
                     v3 = base[3 * STRIDE + k], v4 = base[4 * STRIDE + k];
#pragma unroll
        for (int b = 0; b < BPL; b++) pc_two(v0, v1, v2, v3, v4, m[b], eps2, P[b]);
    }
    commit<BPL>(P, A);
}
template <int NPH, int BPL, int STRIDE>
__device__ __forceinline__ void eval_pp(const float4 *__restrict__ base, int phase, const float4 (&me)[BPL],
                                        const float2 eps2, Acc (&A)[BPL]) {
    constexpr int T = 16 / NPH;
    const int k0 = phase;
    Me2 m[BPL];
    Part2 P[BPL];
#pragma unroll
    for (int b = 0; b < BPL; b++) {
        m[b] = me2_of(me[b]);
        P[b] = Part2{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
#pragma unroll kWalkUnroll
    for (int j = 0; j < T; j++) {
        const int k = k0 + j * NPH;
        const float4 v0 = base[k], v1 = base[STRIDE + k];
#pragma unroll
        for (int b = 0; b < BPL; b++) pp_two(v0, v1, m[b], eps2, P[b]);
    }
    commit<BPL>(P, A);
}

// Which instantiation walks a group of ng bodies: one body per lane below
// WALK_BPL2_FROM bodies (17..33), two from there on.  33 is the measured
// best: two bodies per lane from 17 or 25 bodies on (16 body slots, two
// phases: as many body places as one body per lane) run the 2^20 walk 3%
// slower (128 registers, 16 warps per SM).
#ifndef WALK_BPL2_FROM
#define WALK_BPL2_FROM 33
#endif
static_assert(WALK_BPL2_FROM >= 17 && WALK_BPL2_FROM <= 33, "two bodies per lane need >= 16 body slots");
// With `three` (walks without learned features, groups of at most 32
// bodies), groups of 17..24 bodies (active bodies, in a block substep) go to
// a third instantiation with three bodies per lane in 8 body slots (four
// phases): 24 body places instead of the 32 lanes of one body per lane,
// where 8..15 of them would hold no body.
#ifndef WALK_BPL3
#define WALK_BPL3 1
#endif
__host__ __device__ constexpr int walk_bpl(int ng, bool three) {
    return three && ng > 16 && ng <= 24 ? 3 : ng < WALK_BPL2_FROM ? 1 : 2;
}

// log2 of the body slots of a group: one body per lane, next power of two
// (>= 2: at most 16 phases share the 16 source pairs); two bodies per lane,
// 16 slots (two phases) up to 32 bodies, 32 slots beyond; three bodies per
// lane, 8 slots (four phases).
template <int BPL>
__device__ __forceinline__ int walk_lg(int ng) {
    if (BPL == 3) return 3;
    if (BPL == 2) return ng <= 32 ? 4 : 5;
    return ng <= 2 ? 1 : 32 - __clz(ng - 1);
}

// Warp-uniform dispatch on log2(body slots).
template <int BPL, int STRIDE>
__device__ __forceinline__ void tile_pc(int lg, const float4 *__restrict__ base, int phase, const float4 (&me)[BPL],
                                        const float2 eps2, Acc (&A)[BPL]) {
    if constexpr (BPL == 3) {
        eval_pc<4, 3, STRIDE>(base, phase, me, eps2, A);
    } else if constexpr (BPL == 2) {
        if (lg == 4) eval_pc<2, 2, STRIDE>(base, phase, me, eps2, A);
        else eval_pc<1, 2, STRIDE>(base, phase, me, eps2, A);
    } else {
        switch (lg) {
            case 1: eval_pc<16, 1, STRIDE>(base, phase, me, eps2, A); break;
            case 2: eval_pc<8, 1, STRIDE>(base, phase, me, eps2, A); break;
            case 3: eval_pc<4, 1, STRIDE>(base, phase, me, eps2, A); break;
            case 4: eval_pc<2, 1, STRIDE>(base, phase, me, eps2, A); break;
            default: eval_pc<1, 1, STRIDE>(base, phase, me, eps2, A); break;
        }
    }
}
template <int BPL, int STRIDE>
__device__ __forceinline__ void tile_pp(int lg, const float4 *__restrict__ base, int phase, const float4 (&me)[BPL],
                                        const float2 eps2, Acc (&A)[BPL]) {
    if constexpr (BPL == 3) {
        eval_pp<4, 3, STRIDE>(base, phase, me, eps2, A);
    } else if constexpr (BPL == 2) {
        if (lg == 4) eval_pp<2, 2, STRIDE>(base, phase, me, eps2, A);
        else eval_pp<1, 2, STRIDE>(base, phase, me, eps2, A);
    } else {
        switch (lg) {
            case 1: eval_pp<16, 1, STRIDE>(base, phase, me, eps2, A); break;
            case 2: eval_pp<8, 1, STRIDE>(base, phase, me, eps2, A); break;
            case 3: eval_pp<4, 1, STRIDE>(base, phase, me, eps2, A); break;
            case 4: eval_pp<2, 1, STRIDE>(base, phase, me, eps2, A); break;
            default: eval_pp<1, 1, STRIDE>(base, phase, me, eps2, A); break;
        }
    }
}

__device__ __forceinline__ unsigned lanemask_lt_w() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Level bins of accepted cells for the learned correction's features.
__device__ __forceinline__ int level_bin(int lvl) { return lvl <= 3 ? 0 : lvl <= 6 ? 1 : lvl <= 9 ? 2 : 3; }

// Pops up to 32 cells (whole child ranges from the top of the stack), one
// per lane: warp scan of the entries' child counts; the entry of each output
// lane from one reduction of the entries' start offsets (bit excl of every
// taken entry; all distinct, < 32).  Warp-uniform; requires sp > 0.
__device__ __forceinline__ void walk_pop(const unsigned *stk, int &sp, int lane, unsigned &cell, bool &has) {
    const int avail = min(sp, 32);
    const unsigned ent = lane < avail ? stk[sp - 1 - lane] : 0u;
    const int cnt = lane < avail ? (int)(ent & 7u) + 1 : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned take = __ballot_sync(0xffffffffu, lane < avail && incl <= 32);
    const int m = __popc(take);
    const int T = __shfl_sync(0xffffffffu, incl, m - 1);
    const int excl = incl - cnt;
    sp -= m;
    const unsigned starts = __reduce_or_sync(0xffffffffu, ((take >> lane) & 1u) ? (1u << excl) : 0u);
    const int e = __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
    const unsigned ent_e = __shfl_sync(0xffffffffu, ent, e);
    const int excl_e = __shfl_sync(0xffffffffu, excl, e);
    has = lane < T;
    cell = (ent_e >> 3) + (unsigned)(lane - excl_e);
}

// BPL: bodies per lane (walk_bpl picks the groups of each).  FEAT
// also writes per body (12 floats) the walk quantities the learned far-field
// correction uses: log(1 + accepted cells) in four level bins, log(1 +
// body-body interactions), log(n_G / (extent^3 + eps^3)), log((diagonal +
// eps)/eps), the body's offset from the centre of its group's box (3),
// log(n_G) and the box diagonal.
#ifndef WALK_MIN_BLOCKS1
#define WALK_MIN_BLOCKS1 0          // 0: the compiler picks the register budget
#endif
#ifndef WALK_MIN_BLOCKS2
#define WALK_MIN_BLOCKS2 0
#endif
#ifndef WALK_SPEC_LOADS
#define WALK_SPEC_LOADS 1           // 1: load a tested cell's moments with its MAC record
#endif
#ifndef WALK_SMALL_LAST
#define WALK_SMALL_LAST 16          // > 0: groups of at most this many bodies in a second pass
#endif
#ifndef WALK_MAXNREG1
#define WALK_MAXNREG1 0             // > 0: register cap of the one-body-per-lane walk
#endif
#if WALK_MAXNREG1 > 0
#define WALK_ATTRS __launch_bounds__(256) __maxnreg__(BPL == 1 ? WALK_MAXNREG1 : BPL == 2 ? 255 : 128)
#else
#define WALK_ATTRS __launch_bounds__(256, BPL == 1 ? WALK_MIN_BLOCKS1 : BPL == 2 ? WALK_MIN_BLOCKS2 : 2)
#endif
template <int BPL, bool FEAT, bool BLOCK>
__global__ void WALK_ATTRS
k_walk(const DevState *__restrict__ stc, DevState *st, const uint2 *__restrict__ groups,
       const float4 *__restrict__ pos4, const float4 *__restrict__ test,
       const uint2 *__restrict__ link, const float4 *__restrict__ mono,
       const float4 *__restrict__ quadA, const float2 *__restrict__ quadB,
       const uint8_t *__restrict__ sysid, float eps, int stack_cap, unsigned max_rounds,
       float4 *acc4, uint2 *counts, const uint8_t *__restrict__ cell_level, float *feat,
       const unsigned *__restrict__ gate, const float4 *__restrict__ actv, unsigned act_s, int act_kmax,
       bool three) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t warp_bytes = sizeof(WarpRings) + (size_t)stack_cap * sizeof(unsigned);
    char *wbase = (char *)smem4 + warp * warp_bytes;
    WarpRings &R = *reinterpret_cast<WarpRings *>(wbase);
    unsigned *stk = reinterpret_cast<unsigned *>(wbase + sizeof(WarpRings));
    // Nothing to do after a timed-out sort, or when a gate flag (the learned
    // path's fallback decision) is clear.
    const unsigned ngroups =
        ((stc->status & ST_TIMEOUT) || (gate && *gate == 0u) || stc->ncells == 0u) ? 0u : stc->ngroups;
    const float eps2 = eps * eps;
    const float2 eps2x2 = make_float2(eps2, eps2);
    const unsigned lt = lanemask_lt_w();
    unsigned *queue = BPL == 1 ? &st->walk_next : &st->walk_next2;

    while (true) {
        unsigned g = 0;
        if (lane == 0) g = atomicAdd(queue, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
#if WALK_SMALL_LAST
        // two passes over the groups: larger ones first, then those of at
        // most WALK_SMALL_LAST bodies (a shorter tail at the end of the walk)
        const bool second = g >= ngroups;
        if (second) g -= ngroups;
#endif
        if (g >= ngroups) break;
        const uint2 gr = groups[g];
        const int gb = (int)gr.x, ng = (int)gr.y;
        // groups this instantiation can never take (by size; without block
        // time steps every body takes part, so the size decides)
        if (!BLOCK && walk_bpl(ng, three) != BPL) continue;
        if (BLOCK && ((BPL == 2 && walk_bpl(ng, three) != 2) || (BPL == 3 && ng <= 16))) continue;
#if WALK_SMALL_LAST
        if (second != (ng <= WALK_SMALL_LAST)) continue;
#endif
        // Body slots and source phases.
        // Block time steps, groups of <= 32 bodies: the active bodies are
        // compacted into the first body slots (in body order), and the
        // instantiation and slot count follow the active count (all active:
        // the plain layout, so the same sums as a plain walk).
        int nslot = ng;
        bool act = false;
        unsigned am = 0u;
        if (BLOCK && ng <= 32) {
            act = lane < ng && block_active(actv[gb + lane].w, act_s, act_kmax);
            am = __ballot_sync(0xffffffffu, act);
            nslot = __popc(am);
            if (nslot == 0) continue;
        }
        if (BLOCK && walk_bpl(nslot, three) != BPL) continue;   // another instantiation's group
        if (BLOCK && BPL != 2) {
            if (act) R.leaf[__popc(am & lt)].x = (unsigned)lane;
            __syncwarp();
        }
        const int lg = walk_lg<BPL>(nslot);
        const int slots = 1 << lg;
        const int bslot = lane & (slots - 1), phase = lane >> lg;
        bool live[BPL];
        int bi[BPL];
        float4 me[BPL];
        float bx0 = INFINITY, by0 = INFINITY, bz0 = INFINITY;
        float bx1 = -INFINITY, by1 = -INFINITY, bz1 = -INFINITY;
#pragma unroll
        for (int b = 0; b < BPL; b++) {
            const int slot = bslot + slots * b;
            live[b] = slot < nslot;
            int body = slot;
            if (BLOCK && BPL != 2) {
                if (live[b]) body = (int)R.leaf[slot].x;
            } else if (BLOCK && live[b]) {
                // only the bodies whose step ends at this substep
                live[b] = block_active(actv[gb + slot].w, act_s, act_kmax);
            }
            bi[b] = gb + (live[b] ? body : 0);
            me[b] = pos4[bi[b]];
            if (live[b]) {
                bx0 = fminf(bx0, me[b].x); by0 = fminf(by0, me[b].y); bz0 = fminf(bz0, me[b].z);
                bx1 = fmaxf(bx1, me[b].x); by1 = fmaxf(by1, me[b].y); bz1 = fmaxf(bz1, me[b].z);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
            by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
            bz0 = fminf(bz0, __shfl_xor_sync(0xffffffffu, bz0, o));
            bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
            by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
            bz1 = fmaxf(bz1, __shfl_xor_sync(0xffffffffu, bz1, o));
        }
        // Live body slots (bit = slot); a group without one is skipped.
        unsigned nlive = (unsigned)ng;
        if (BLOCK) {                               // a group without a live body is skipped
            nlive = 0u;
#pragma unroll
            for (int b = 0; b < BPL; b++) nlive += (unsigned)__popc(__ballot_sync(0xffffffffu, phase == 0 && live[b]));
            if (nlive == 0u) continue;
        }
        Acc A[BPL];
#pragma unroll
        for (int b = 0; b < BPL; b++) A[b] = Acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int sp = 1;
        // Root of the group's system: the level-0 cells are the system roots in
        // system order, so system s's root is cell s (range of one cell).
        if (lane == 0) stk[0] = (unsigned)sysid[gb] << 3;
        int pc_head = 0, pc_n = 0, pp_head = 0, pp_n = 0;
        unsigned npc = 0, npp = 0;
        unsigned nbin[4] = {0u, 0u, 0u, 0u};
        bool overflow = false, timeout = false;
        unsigned rounds = 0;
        __syncwarp();

        while (sp > 0) {
            if (++rounds > max_rounds) { timeout = true; break; }   // bounded traversal
            unsigned cell;
            bool has;
            walk_pop(stk, sp, lane, cell, has);

            bool open = false, acc = false, isleaf = false;
            uint2 lk = make_uint2(0u, 0u);
#if WALK_SPEC_LOADS
            float4 cmo = make_float4(0.f, 0.f, 0.f, 0.f), cqa = cmo;
            float2 cqb = make_float2(0.f, 0.f);
#endif
            if (has) {
                const float4 tc = __ldg(test + cell);
                lk = __ldg(link + cell);
#if WALK_SPEC_LOADS
                // the moments, in case the cell is accepted: one round trip per round
                cmo = __ldg(mono + cell); cqa = __ldg(quadA + cell); cqb = __ldg(quadB + cell);
#endif
                const float dx = fmaxf(fmaxf(bx0 - tc.x, tc.x - bx1), 0.f);
                const float dy = fmaxf(fmaxf(by0 - tc.y, tc.y - by1), 0.f);
                const float dz = fmaxf(fmaxf(bz0 - tc.z, tc.z - bz1), 0.f);
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                open = d2 < tc.w * tc.w;
                acc = !open;
                isleaf = (lk.y & LEAF_BIT) != 0u;
            }
            // Accepted cells -> body-cell ring.
            const unsigned am = __ballot_sync(0xffffffffu, acc);
            if (acc) {
                const int s = (pc_head + pc_n + __popc(am & lt)) & (RING - 1);
#if WALK_SPEC_LOADS
                put_cell(R, s, cmo, cqa, cqb);
#else
                put_cell(R, s, __ldg(mono + cell), __ldg(quadA + cell), __ldg(quadB + cell));
#endif
            }
            pc_n += __popc(am);
            npc += __popc(am);
            if (FEAT) {
                const int bin = acc ? level_bin(__ldg(cell_level + cell)) : -1;
#pragma unroll
                for (int k = 0; k < 4; k++) nbin[k] += __popc(__ballot_sync(0xffffffffu, bin == k));
            }
            // Opened internal cells -> push child ranges.
            const unsigned im = __ballot_sync(0xffffffffu, open && !isleaf);
            const int np = __popc(im);
            if (sp + np > stack_cap) {
                overflow = true;
            } else {
                if (open && !isleaf) {
                    stk[sp + __popc(im & lt)] = (lk.x << 3) | ((lk.y - 1u) & 7u);
                }
                sp += np;
            }
            // Opened leaves -> body-body ring: the bodies of all of the round's
            // opened leaves in lane order, 32 per pass, one load per lane.
            const bool ol = open && isleaf;
            const unsigned lm = __ballot_sync(0xffffffffu, ol);
            if (lm) {
                const unsigned lc = ol ? (lk.y & ~LEAF_BIT) : 0u;
                unsigned lincl = lc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, lincl, o);
                    if (lane >= o) lincl += y;
                }
                const unsigned total = __shfl_sync(0xffffffffu, lincl, 31);
                const unsigned lex = lincl - lc;
                if (ol) R.leaf[__popc(lm & lt)] = make_uint2(lk.x, lex);
                npp += total;
                __syncwarp();
                const unsigned upto = 0xffffffffu >> (31 - lane);
                for (unsigned base = 0; base < total; base += 32u) {
                    // leaf k of body base+lane: leaves starting before base plus
                    // those starting in [base, base+lane]
                    const unsigned starts =
                        __reduce_or_sync(0xffffffffu, ol && lex >= base && lex < base + 32u ? 1u << (lex - base) : 0u);
                    const int before = __popc(__ballot_sync(0xffffffffu, ol && lex < base));
                    const uint2 li = R.leaf[before + __popc(starts & upto) - 1];
                    const int nb = (int)min(32u, total - base);
                    if (lane < nb)
                        put_body(R, (pp_head + pp_n + lane) & (RING - 1), __ldg(pos4 + li.x + (base + lane - li.y)));
                    pp_n += nb;
                    if (pp_n >= 32) {
                        __syncwarp();
                        tile_pp<BPL, RPAIR>(lg, R.b0 + (pp_head >> 1), phase, me, eps2x2, A);
                        __syncwarp();
                        pp_head = (pp_head + 32) & (RING - 1);
                        pp_n -= 32;
                    }
                }
            }
            __syncwarp();
            if (pc_n >= 32) {
                tile_pc<BPL, RPAIR>(lg, R.c0 + (pc_head >> 1), phase, me, eps2x2, A);
                pc_head = (pc_head + 32) & (RING - 1);
                pc_n -= 32;
            }
            __syncwarp();
        }
        // Remaining partial tiles (head is 0 or 32, n < 32): pad to 32 with
        // massless sources far away, then evaluate as full tiles.
        const float FAR = 1e18f;
        if (pc_n > 0) {
            const int s = pc_head + pc_n + lane;
            if (lane < 32 - pc_n)
                put_cell(R, s, make_float4(FAR, FAR, FAR, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), make_float2(0.f, 0.f));
            __syncwarp();
            tile_pc<BPL, RPAIR>(lg, R.c0 + (pc_head >> 1), phase, me, eps2x2, A);
        }
        if (pp_n > 0) {
            if (lane < 32 - pp_n) put_body(R, pp_head + pp_n + lane, make_float4(FAR, FAR, FAR, 0.f));
            __syncwarp();
            tile_pp<BPL, RPAIR>(lg, R.b0 + (pp_head >> 1), phase, me, eps2x2, A);
        }
#pragma unroll
        for (int b = 0; b < BPL; b++) {
            float ax = A[b].ax - A[b].cx, ay = A[b].ay - A[b].cy, az = A[b].az - A[b].cz,
                  ph = A[b].ph - A[b].cp;
            for (int o = slots; o < 32; o <<= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
                az += __shfl_xor_sync(0xffffffffu, az, o);
                ph += __shfl_xor_sync(0xffffffffu, ph, o);
            }
            if (live[b] && phase == 0) {
                ph += me[b].w * rsqrtf(eps2);    // remove the self term -m/eps
                acc4[bi[b]] = make_float4(ax, ay, az, ph);
                counts[bi[b]] = make_uint2(npc, npp - 1u);
                if (FEAT) {
                    const float ex = bx1 - bx0, ey = by1 - by0, ez = bz1 - bz0;
                    const float ext = fmaxf(ex, fmaxf(ey, ez));
                    const float diag = sqrtf(ex * ex + ey * ey + ez * ez);
                    const float e3 = eps * eps * eps;
                    float *f = feat + FEAT_STRIDE * (size_t)bi[b];
                    f[0] = log1pf((float)nbin[0]); f[1] = log1pf((float)nbin[1]);
                    f[2] = log1pf((float)nbin[2]); f[3] = log1pf((float)nbin[3]);
                    f[4] = log1pf((float)(npp - 1u));
                    f[5] = logf((float)ng / (ext * ext * ext + e3));
                    f[6] = logf((diag + eps) / eps);
                    f[7] = me[b].x - 0.5f * (bx0 + bx1);
                    f[8] = me[b].y - 0.5f * (by0 + by1);
                    f[9] = me[b].z - 0.5f * (bz0 + bz1);
                    f[10] = logf((float)ng);
                    f[11] = diag;
                }
            }
        }
        if (lane == 0) {
            atomicAdd(&st->inter[0], (unsigned long long)npc * (unsigned long long)nlive);
            atomicAdd(&st->inter[1], (unsigned long long)(npp - 1u) * (unsigned long long)nlive);
            if (overflow) atomicOr(&st->status, ST_CAPACITY);
            if (timeout) atomicOr(&st->status, ST_TIMEOUT);
        }
        __syncwarp();
    }
}

size_t walk_smem_bytes(int warps, int stack_cap) {
    return (size_t)warps * (sizeof(WarpRings) + (size_t)stack_cap * sizeof(unsigned));
}

// Function attribute and occupancy are set up once per shape, before any
// stream capture of a step (the first step always runs eagerly).
template <int BPL, bool FEAT, bool BLOCK>
static cudaError_t launch_walk_t(Ctx &c, float eps, const unsigned *gate, bool three, cudaStream_t stream) {
    const unsigned polls = (unsigned)(c.max_spin < 0xffffffffll ? c.max_spin : 0xffffffffll);
    const int warps = c.walk_warps;
    const size_t smem = walk_smem_bytes(warps, c.list_capacity);
    // per device: the attribute applies to one device, and the occupancy is
    // that device's
    static size_t attr_done[MAX_DEVICES] = {}, occ_smem[MAX_DEVICES] = {};
    static int occ_warps[MAX_DEVICES] = {}, occ_per_sm[MAX_DEVICES] = {};
    cudaError_t ea = allow_dyn_smem((const void *)k_walk<BPL, FEAT, BLOCK>, smem, attr_done);
    if (ea != cudaSuccess) return ea;
    const int dv = c.device;
    if (dv < 0 || dv >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (occ_warps[dv] != warps || occ_smem[dv] != smem) {
        int per = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk<BPL, FEAT, BLOCK>, warps * 32, smem);
        if (e != cudaSuccess) return e;
        occ_warps[dv] = warps; occ_smem[dv] = smem; occ_per_sm[dv] = per < 1 ? 1 : per;
    }
    k_walk<BPL, FEAT, BLOCK><<<c.num_sms * occ_per_sm[dv], warps * 32, smem, stream>>>(
        c.st, c.st, c.groups, c.pos4, c.test, c.cell_link, c.mono, c.quadA, c.quadB, c.sysid, eps,
        c.list_capacity, polls, c.acc4, c.counts, c.cell_level, c.feat, gate,
        BLOCK ? c.vel4 : nullptr, c.block_s, c.block_kmax, three);
    return cudaGetLastError();
}

// One persistent launch per instantiation that can receive groups (group
// sizes are at most ncrit; oversize leaves are cut into chunks of ncrit).
// With both, the two-body launch runs on a side stream forked from and
// joined back into the context's stream (event edges inside a captured
// step), so the tail of each launch overlaps the other's work.
cudaError_t launch_walk(Ctx &c, float eps, bool features, const unsigned *gate) {
    // Second instantiation beside one body per lane: two bodies per lane for
    // groups of more than 32 bodies, or, in walks without learned features
    // and with groups of at most 32 bodies, three per lane for groups of
    // 17..24 (bodies that take part: the active ones of a block substep).
    const bool three = WALK_BPL3 && !features && c.ncrit > 16 && c.ncrit < WALK_BPL2_FROM;
    // instantiations: plain, with learned features, or block time steps
    auto one = [&](int bpl, cudaStream_t st) -> cudaError_t {
        if (c.block_kmax >= 0) {
            if (bpl == 3) return launch_walk_t<3, false, true>(c, eps, gate, true, st);
            return bpl == 2 ? launch_walk_t<2, false, true>(c, eps, gate, false, st)
                            : launch_walk_t<1, false, true>(c, eps, gate, three, st);
        }
        if (features)
            return bpl == 2 ? launch_walk_t<2, true, false>(c, eps, gate, false, st)
                            : launch_walk_t<1, true, false>(c, eps, gate, false, st);
        if (bpl == 3) return launch_walk_t<3, false, false>(c, eps, gate, true, st);
        return bpl == 2 ? launch_walk_t<2, false, false>(c, eps, gate, false, st)
                        : launch_walk_t<1, false, false>(c, eps, gate, three, st);
    };
    const int second = c.ncrit >= WALK_BPL2_FROM ? 2 : three ? 3 : 0;
    if (second == 0) return one(1, c.stream);
    cudaError_t e = cudaEventRecord(c.ev_fork, c.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.side, c.ev_fork, 0);
    // One body per lane first: each persistent launch fills the registers,
    // so the second starts as the first one's warps leave, and the first
    // one's tail (its last groups, ~0.1 ms each) overlaps the second's work.
    if (e == cudaSuccess) e = one(1, c.stream);
    if (e == cudaSuccess) e = one(second, c.side);
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_join, c.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.stream, c.ev_join, 0);
    return e;
}

}  // namespace bonsai

// ---------------------------------------------------------------------------
// Neighbour search and SPH density on the same tree (paper Sect. 3: the
// tree also serves neighbour search and smoothed particle hydrodynamics).
// The group walk with another opening rule and kernel: a cell is searched
// iff its cube (build-time centre, half side ext) comes within h_max of the
// group's box, h_max the largest smoothing length of the group; searched
// leaves feed their bodies through a ring of 64 in shared memory; each body
// i counts the sources j with r^2 < h_i^2 (r^2 = fma(dz, dz, fma(dy, dy,
// dx dx)), dx = x_j - x_i rounded: the decision the oracle takes) and sums
// m_j W(r, h_i), W the cubic spline of compact support h.  Up to 64 bodies
// per group: two body slots per lane.
namespace bonsai {

constexpr int SPH_RING = 64;

struct SphWarp {
    float4 src[SPH_RING];
};

// 8 / pi: the cubic spline's normalisation in three dimensions.
constexpr float SPH_NORM = 2.546479089470325f;

// One ring of sources: plain float32 sums per body, then one compensated
// (Kahan) add into the body's density.
__device__ __forceinline__ void sph_tile(const float4 *__restrict__ src, int nsrc, const float4 (&me)[2],
                                         const float (&h2)[2], const float (&ih)[2], const bool (&live)[2],
                                         float (&rho)[2], float (&comp)[2], unsigned (&cnt)[2]) {
    float part[2] = {0.f, 0.f};
    for (int k = 0; k < nsrc; k++) {
        const float4 s = src[k];
#pragma unroll
        for (int b = 0; b < 2; b++) {
            if (!live[b]) continue;
            const float dx = __fsub_rn(s.x, me[b].x), dy = __fsub_rn(s.y, me[b].y), dz = __fsub_rn(s.z, me[b].z);
            const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            if (r2 < h2[b]) {
                const float q = sqrtf(r2) * ih[b];
                const float t = fmaxf(1.f - q, 0.f);
                const float w = q <= 0.5f ? fmaf(6.f * q * q, q - 1.f, 1.f) : 2.f * t * t * t;
                part[b] = fmaf(s.w, w, part[b]);
                cnt[b]++;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < 2; b++) kahan_add(rho[b], comp[b], part[b]);
}

__global__ void __launch_bounds__(128)
k_sph_walk(const DevState *__restrict__ stc, DevState *st, const uint2 *__restrict__ groups,
           const float4 *__restrict__ pos4, const float *__restrict__ hs, const float4 *__restrict__ cext,
           const uint2 *__restrict__ link, const uint8_t *__restrict__ sysid, int stack_cap, unsigned max_rounds,
           float *rho_s, int32_t *cnt_s) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t warp_bytes = sizeof(SphWarp) + (size_t)stack_cap * sizeof(unsigned);
    char *wbase = (char *)smem4 + warp * warp_bytes;
    SphWarp &R = *reinterpret_cast<SphWarp *>(wbase);
    unsigned *stk = reinterpret_cast<unsigned *>(wbase + sizeof(SphWarp));
    const unsigned ngroups = (stc->status & ST_TIMEOUT) ? 0u : stc->ngroups;
    const unsigned lt = lanemask_lt_w();
    while (true) {
        unsigned g = 0;
        if (lane == 0) g = atomicAdd(&st->walk_next, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        const uint2 gr = groups[g];
        const int gb = (int)gr.x, ng = (int)gr.y;
        bool live[2];
        float4 me[2];
        float h2[2], ih[2], rho[2] = {0.f, 0.f}, comp[2] = {0.f, 0.f};
        unsigned cnt[2] = {0u, 0u};
        float bx0 = INFINITY, by0 = INFINITY, bz0 = INFINITY, bx1 = -INFINITY, by1 = -INFINITY, bz1 = -INFINITY;
        float hmax = 0.f;
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int slot = lane + 32 * b;
            live[b] = slot < ng;
            const int i = gb + (live[b] ? slot : 0);
            me[b] = pos4[i];
            const float h = hs[i];
            h2[b] = __fmul_rn(h, h);
            ih[b] = 1.f / h;
            if (live[b]) {
                bx0 = fminf(bx0, me[b].x); by0 = fminf(by0, me[b].y); bz0 = fminf(bz0, me[b].z);
                bx1 = fmaxf(bx1, me[b].x); by1 = fmaxf(by1, me[b].y); bz1 = fmaxf(bz1, me[b].z);
                hmax = fmaxf(hmax, h);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
            by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
            bz0 = fminf(bz0, __shfl_xor_sync(0xffffffffu, bz0, o));
            bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
            by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
            bz1 = fmaxf(bz1, __shfl_xor_sync(0xffffffffu, bz1, o));
            hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
        }
        // search radius with a relative slack: rounding may only open more
        const float reach2 = hmax * hmax * 1.0001f;
        int sp = 1, nsrc = 0;
        if (lane == 0) stk[0] = (unsigned)sysid[gb] << 3;   // the root of the group's system
        bool overflow = false, timeout = false;
        unsigned rounds = 0;
        __syncwarp();
        while (sp > 0) {
            if (++rounds > max_rounds) { timeout = true; break; }
            unsigned cell;
            bool has;
            walk_pop(stk, sp, lane, cell, has);
            bool open = false, isleaf = false;
            uint2 lk = make_uint2(0u, 0u);
            if (has) {
                const float4 ce = __ldg(cext + cell);
                lk = __ldg(link + cell);
                const float dx = fmaxf(fmaxf(bx0 - (ce.x + ce.w), (ce.x - ce.w) - bx1), 0.f);
                const float dy = fmaxf(fmaxf(by0 - (ce.y + ce.w), (ce.y - ce.w) - by1), 0.f);
                const float dz = fmaxf(fmaxf(bz0 - (ce.z + ce.w), (ce.z - ce.w) - bz1), 0.f);
                open = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) <= reach2;
                isleaf = (lk.y & LEAF_BIT) != 0u;
            }
            const unsigned im = __ballot_sync(0xffffffffu, open && !isleaf);
            const int np = __popc(im);
            if (sp + np > stack_cap) {
                overflow = true;
            } else {
                if (open && !isleaf) stk[sp + __popc(im & lt)] = (lk.x << 3) | ((lk.y - 1u) & 7u);
                sp += np;
            }
            // searched leaves, one at a time: their bodies into the ring
            unsigned lm = __ballot_sync(0xffffffffu, open && isleaf);
            while (lm) {
                const int src_lane = __ffs(lm) - 1;
                lm &= lm - 1;
                const unsigned first = __shfl_sync(0xffffffffu, lk.x, src_lane);
                const int n_l = (int)(__shfl_sync(0xffffffffu, lk.y, src_lane) & ~LEAF_BIT);
                for (int off = 0; off < n_l; off += 32) {
                    // a body farther than h_max from the group's box is no
                    // body's neighbour: only the others enter the ring
                    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool keep = false;
                    if (off + lane < n_l) {
                        p = __ldg(pos4 + first + off + lane);
                        const float ex = fmaxf(fmaxf(bx0 - p.x, p.x - bx1), 0.f);
                        const float ey = fmaxf(fmaxf(by0 - p.y, p.y - by1), 0.f);
                        const float ez = fmaxf(fmaxf(bz0 - p.z, p.z - bz1), 0.f);
                        keep = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= reach2;
                    }
                    const unsigned km = __ballot_sync(0xffffffffu, keep);
                    const int take = __popc(km);
                    if (nsrc + take > SPH_RING) {           // ring full: evaluate it
                        __syncwarp();
                        sph_tile(R.src, nsrc, me, h2, ih, live, rho, comp, cnt);
                        __syncwarp();
                        nsrc = 0;
                    }
                    if (keep) R.src[nsrc + __popc(km & lt)] = p;
                    nsrc += take;
                }
            }
            __syncwarp();
        }
        if (nsrc > 0) sph_tile(R.src, nsrc, me, h2, ih, live, rho, comp, cnt);
#pragma unroll
        for (int b = 0; b < 2; b++) {
            if (live[b]) {
                rho_s[gb + lane + 32 * b] = (rho[b] - comp[b]) * (SPH_NORM * ih[b] * ih[b] * ih[b]);
                cnt_s[gb + lane + 32 * b] = (int32_t)cnt[b];
            }
        }
        if (lane == 0) {
            if (overflow) atomicOr(&st->status, ST_CAPACITY);
            if (timeout) atomicOr(&st->status, ST_TIMEOUT);
        }
        __syncwarp();
    }
}

cudaError_t launch_sph_walk(Ctx &c, const float *hs, const float4 *cext, float *rho_s, int32_t *cnt_s) {
    const unsigned polls = (unsigned)(c.max_spin < 0xffffffffll ? c.max_spin : 0xffffffffll);
    const int warps = 4;
    const size_t smem = (size_t)warps * (sizeof(SphWarp) + (size_t)c.list_capacity * sizeof(unsigned));
    static size_t attr_done[MAX_DEVICES] = {}, occ_smem[MAX_DEVICES] = {};
    static int per_sm[MAX_DEVICES] = {};
    cudaError_t ea = allow_dyn_smem((const void *)k_sph_walk, smem, attr_done);
    if (ea != cudaSuccess) return ea;
    const int dv = c.device;
    if (dv < 0 || dv >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (occ_smem[dv] != smem) {
        int per = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sph_walk, warps * 32, smem);
        if (e != cudaSuccess) return e;
        occ_smem[dv] = smem; per_sm[dv] = per < 1 ? 1 : per;
    }
    k_sph_walk<<<c.num_sms * per_sm[dv], warps * 32, smem, c.stream>>>(c.st, c.st, c.groups, c.pos4, hs, cext,
                                                                    c.cell_link, c.sysid, c.list_capacity, polls,
                                                                    rho_s, cnt_s);
    return cudaGetLastError();
}

}  // namespace bonsai
