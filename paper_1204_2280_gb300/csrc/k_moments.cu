// k_moments.cu -- multipole moments of every cell (paper Sect. 2,
// "computation of the multipole moments") and the opening radius of the MAC.
//
// Per cell: mass M, centre of mass com and traceless quadrupole
//   Q_ij = sum m (3 y_i y_j - |y|^2 delta_ij),  y = x - com.
// Leaves are summed from their bodies in cell-relative coordinates (offsets
// from the first body, then from the com).  Parents combine their children
// by the parallel-axis theorem,
//   Q_p = sum_k [ Q_k + M_k (3 d_k d_k^T - |d_k|^2 I) ],  d_k = com_k - com_p,
// in a second launch: each thread finishing a cell counts down its parent's
// arrival word and the last internal child to arrive combines the parent
// (no waiting).
// The root of each system (level 0) combines in FP64: FP64 arithmetic runs
// at a small fraction of the FP32 rate here, so the thread finishing each
// level-1 cell writes that cell's FP64 terms about the root cube's centre O
// (the ones the root needs, computed on up to eight lanes of different warps
// at once), and the root sums them and shifts to its own com:
//   with e = com_k - O:  M = sum m_k,  com = O + (sum m_k e) / M,
//   Q = sum [Q_k + m_k (3 e e^T - |e|^2 I)] - M (3 s s^T - |s|^2 I),  s = com - O.
#include "common.cuh"

namespace bonsai {

__device__ __forceinline__ unsigned compact3(unsigned long long x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x00000000001fffffull;
    return (unsigned)x;
}

// Geometric centre and side of a cell at `level` of system `sys` whose
// first body has key k.
__device__ __forceinline__ float cell_cube(unsigned long long k, int level, int sys, const DevState *st, float3 &c) {
    unsigned long long pre = key_prefix(k, level);
    float l = ldexpf(st->side[sys], -level);
    const float *mn = st->mn + 3 * sys;
    c.x = fmaf((float)compact3(pre) + 0.5f, l, mn[0]);
    c.y = fmaf((float)compact3(pre >> 1) + 0.5f, l, mn[1]);
    c.z = fmaf((float)compact3(pre >> 2) + 0.5f, l, mn[2]);
    return l;
}

__device__ __forceinline__ float com_offset(float3 com, float3 c) {
    float dx = com.x - c.x, dy = com.y - c.y, dz = com.z - c.z;
    return sqrtf(dx * dx + dy * dy + dz * dz);
}

// (|com - geometric centre|, side) of a cell at `level` of system `sys`
// whose first body has key k.
__device__ float2 cell_delta(unsigned long long k, int level, int sys, float3 com, const DevState *st) {
    float3 c;
    const float l = cell_cube(k, level, sys, st, c);
    return make_float2(com_offset(com, c), l);
}

__device__ __forceinline__ float dist_inf(float3 a, float3 b) {
    return fmaxf(fabsf(a.x - b.x), fmaxf(fabsf(a.y - b.y), fabsf(a.z - b.z)));
}

struct Mom32 { float M, x, y, z, q[6]; };

#ifndef MOM_MINB
#define MOM_MINB 4            // resident 256-thread blocks per SM the launch bounds ask for (5 spills)
#endif
#ifndef MOM_CTHREADS
#define MOM_CTHREADS 128      // combine pass: threads per block
#endif
#ifndef MOM_MINB2
#define MOM_MINB2 6           // combine pass: resident blocks per SM the launch bounds ask for
#endif
#ifndef MOM_CPASYNC
#define MOM_CPASYNC 1         // combine: children's data through asynchronous copies to shared memory
#endif                        // (0: register loads in two round trips, 5-11% slower at 2^20..2^22)
#ifndef MOM_CBLOCKS
#define MOM_CBLOCKS 6         // combine pass: blocks per SM of its persistent grid (32 KB of staging each)
#endif
#ifndef MOM_LB
#define MOM_LB 8              // leaf bodies loaded per round trip (4: 3% slower at 2^22, 16 spills)
#endif

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// The quadrupole arrays hold -Q (negation is exact): the walk consumes it in
// that form, parents and the export negate it back.
__device__ __forceinline__ void store32(int c, const Mom32 &m, float4 *mono, float4 *qa, float2 *qb) {
    mono[c] = make_float4(m.x, m.y, m.z, m.M);
    qa[c] = make_float4(-m.q[0], -m.q[1], -m.q[2], -m.q[3]);
    qb[c] = make_float2(-m.q[4], -m.q[5]);
}

// delta[c] = (|com - centre|, side) and, when the step folds the opening
// radius in (test != nullptr), the walk's MAC record of the cell,
// test[c] = (com, side / theta + |com - centre|).
__device__ __forceinline__ void put_delta(unsigned c, const Mom32 &m, float2 dl, float2 *delta, float4 *test,
                                          float inv_theta) {
    delta[c] = dl;
    if (test) test[c] = make_float4(m.x, m.y, m.z, fmaf(dl.y, inv_theta, dl.x));
}

// FP64 terms of level-1 cell c for its root: with O the root cube's centre
// (from a key inside the cell) and e = com - O, (m, m e, Q + m (3 e e^T -
// |e|^2 I)); published by the arrival atomic on the root that follows.
__device__ __forceinline__ void root_terms(unsigned c, const Mom32 &m, unsigned long long kb, int sysb,
                                           const DevState *stc, double *shadow) {
    float3 o;
    cell_cube(kb, 0, sysb, stc, o);
    const double M = m.M, ex = (double)m.x - o.x, ey = (double)m.y - o.y, ez = (double)m.z - o.z;
    const double e2 = ex * ex + ey * ey + ez * ez;
    double *t = shadow + 10 * (size_t)c;
    t[0] = M; t[1] = M * ex; t[2] = M * ey; t[3] = M * ez;
    t[4] = m.q[0] + M * (3 * ex * ex - e2);
    t[5] = m.q[1] + M * (3 * ey * ey - e2);
    t[6] = m.q[2] + M * (3 * ez * ez - e2);
    t[7] = m.q[3] + M * (3 * ex * ey);
    t[8] = m.q[4] + M * (3 * ex * ez);
    t[9] = m.q[5] + M * (3 * ey * ez);
}

// REFIT (block time steps, between rebuilds): the bodies may have left the
// cells they were sorted into.  Each cell also gets ext = half side of a cube
// about its build-time centre that holds its bodies (at least l/2; a leaf
// from its bodies, a parent as max(l/2, max_k |centre_k - centre|_inf +
// ext_k)), stored with the centre in cext, and delta holds (|com - centre|,
// 2 ext): the opening radius 2 ext / theta + delta then keeps every cell that
// holds a body of a group opened for it (theta < 2 / sqrt(3)).
//
// Two launches.  The leaf pass sums every leaf from its bodies (no atomics,
// no fences), gives every internal cell its arrival word (the number of its
// internal children) and lists the internal cells without any.  The combine
// pass starts at the listed cells (all children leaves, complete since the
// leaf pass) and climbs: a finished cell decrements its parent's word and
// the child that brings it to zero combines the parent.

// 16-byte asynchronous copy global -> shared through L2 (zero fill when
// !valid: nothing is read).
__device__ __forceinline__ void cp_async16(float4 *sdst, const float4 *gsrc, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gsrc), "r"(valid ? 16 : 0)
                 : "memory");
}

struct MomArrays {
    const DevState *__restrict__ stc;
    const uint2 *__restrict__ cell_body;
    const uint2 *__restrict__ cell_link;
    const uint8_t *__restrict__ cell_level;
    const uint32_t *__restrict__ cell_parent;
    uint32_t *cell_done;
    const float4 *__restrict__ pos4;
    const unsigned long long *__restrict__ sk;
    const uint8_t *__restrict__ sysid;
    float4 *mono, *qa;
    float2 *qb, *delta;
    double *shadow;
    float4 *cext, *test;
    float inv_theta;
    bool multi;                       // several systems (else every body is in system 0)
    uint32_t *starts;                 // internal cells whose children are all leaves
    unsigned *nstart;                 // their number
};

// Leaf c (level lev, bodies link.x ..) from its bodies in one pass: mass,
// first and second moments of the offsets u = x - x0 from the first body;
// then with c = s/M the central moments C = S - s c^T and Q = 3C - tr(C) I.
// The offsets are at most the cell size, so nothing cancels beyond FP32
// rounding.  A level-1 leaf also writes its FP64 root terms.
template <bool REFIT>
__device__ __forceinline__ void leaf_finish(unsigned c, int lev, unsigned long long kb, int sysb, float4 x0, float M,
                                            float sx, float sy, float sz, float sxx, float syy, float szz, float sxy,
                                            float sxz, float syz, float3 ctr, float ext, const MomArrays &a);

template <bool REFIT>
__device__ __forceinline__ void leaf_cell(unsigned c, uint2 link, int lev, const MomArrays &a) {
    const unsigned b = link.x, cnt = link.y & ~LEAF_BIT;
    // The first body's key and system with its position (one round trip;
    // loaded after the sums they cost 2% at 2^22 bodies).
    const unsigned long long kb = a.sk[b];
    const int sysb = a.multi ? a.sysid[b] : 0;
    const float4 x0 = a.pos4[b];
    float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
    float3 ctr = make_float3(0.f, 0.f, 0.f);
    float ext = 0.f;
    if (REFIT) ext = 0.5f * cell_cube(kb, lev, sysb, a.stc, ctr);
    // The bodies' loads are issued LB at a time (one round trip per LB
    // bodies instead of one per body); the sums still run in body order.
    constexpr unsigned LB = MOM_LB;
    for (unsigned j0 = b; j0 < b + cnt; j0 += LB) {
        float4 pb[LB];
#pragma unroll
        for (unsigned u = 0; u < LB; u++) pb[u] = j0 + u < b + cnt ? a.pos4[j0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (unsigned u = 0; u < LB; u++) {
            if (j0 + u >= b + cnt) break;
            const float4 p = pb[u];
            if (REFIT) ext = fmaxf(ext, dist_inf(make_float3(p.x, p.y, p.z), ctr));
            const float ux = p.x - x0.x, uy = p.y - x0.y, uz = p.z - x0.z;
            const float wx = p.w * ux, wy = p.w * uy, wz = p.w * uz;
            M += p.w;
            sx += wx; sy += wy; sz += wz;
            sxx = fmaf(wx, ux, sxx); syy = fmaf(wy, uy, syy); szz = fmaf(wz, uz, szz);
            sxy = fmaf(wx, uy, sxy); sxz = fmaf(wx, uz, sxz); syz = fmaf(wy, uz, syz);
        }
    }
    leaf_finish<REFIT>(c, lev, kb, sysb, x0, M, sx, sy, sz, sxx, syy, szz, sxy, sxz, syz, ctr, ext, a);
}

// A leaf's moments from its sums about the first body x0 (mass, first and
// second moments of the offsets), and its stores.
template <bool REFIT>
__device__ __forceinline__ void leaf_finish(unsigned c, int lev, unsigned long long kb, int sysb, float4 x0, float M,
                                            float sx, float sy, float sz, float sxx, float syy, float szz, float sxy,
                                            float sxz, float syz, float3 ctr, float ext, const MomArrays &a) {
    Mom32 m;
    m.M = M;
    const float inv = M > 0.f ? 1.f / M : 0.f;
    const float cx = sx * inv, cy = sy * inv, cz = sz * inv;
    m.x = x0.x + cx; m.y = x0.y + cy; m.z = x0.z + cz;
    const float Cxx = fmaf(-sx, cx, sxx), Cyy = fmaf(-sy, cy, syy), Czz = fmaf(-sz, cz, szz);
    const float tr = Cxx + Cyy + Czz;
    m.q[0] = 3.f * Cxx - tr; m.q[1] = 3.f * Cyy - tr; m.q[2] = 3.f * Czz - tr;
    m.q[3] = 3.f * fmaf(-sx, cy, sxy); m.q[4] = 3.f * fmaf(-sx, cz, sxz); m.q[5] = 3.f * fmaf(-sy, cz, syz);
    store32(c, m, a.mono, a.qa, a.qb);
    if (REFIT) {
        put_delta(c, m, make_float2(com_offset(make_float3(m.x, m.y, m.z), ctr), 2.f * ext), a.delta, a.test,
                  a.inv_theta);
        a.cext[c] = make_float4(ctr.x, ctr.y, ctr.z, ext);
    } else {
        put_delta(c, m, cell_delta(kb, lev, sysb, make_float3(m.x, m.y, m.z), a.stc), a.delta, a.test, a.inv_theta);
    }
    if (lev == 1) root_terms(c, m, kb, sysb, a.stc, a.shadow);
}

// Internal cell c (level lv, children plk.x .. plk.x + plk.y - 1, all
// complete) from its children; kb, sysb: the key and system of a body inside
// it (its key prefix gives the cell's centre).  A root combines the FP64
// terms of its level-1 cells; a level-1 cell writes its own.
template <bool REFIT>
__device__ __forceinline__ void combine_cell(unsigned c, int lv, uint2 plk, unsigned long long kb, int sysb,
                                             const MomArrays &a, float4 *stage = nullptr) {
    const unsigned cb = plk.x, nch = plk.y;
    Mom32 m;
    if (lv == 0) {
        float3 o;
        cell_cube(kb, 0, sysb, a.stc, o);
        double t[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (unsigned k = 0; k < nch; k++) {
            const double *sk2 = a.shadow + 10 * (size_t)(cb + k);
#pragma unroll
            for (int i = 0; i < 10; i++) t[i] += __ldcg(sk2 + i);
        }
        const double inv2 = t[0] > 0 ? 1.0 / t[0] : 0.0;
        const double sx = t[1] * inv2, sy = t[2] * inv2, sz = t[3] * inv2;   // com - O
        const double s2 = sx * sx + sy * sy + sz * sz;
        m.M = (float)t[0];
        m.x = (float)(o.x + sx); m.y = (float)(o.y + sy); m.z = (float)(o.z + sz);
        m.q[0] = (float)(t[4] - t[0] * (3 * sx * sx - s2));
        m.q[1] = (float)(t[5] - t[0] * (3 * sy * sy - s2));
        m.q[2] = (float)(t[6] - t[0] * (3 * sz * sz - s2));
        m.q[3] = (float)(t[7] - t[0] * (3 * sx * sy));
        m.q[4] = (float)(t[8] - t[0] * (3 * sx * sz));
        m.q[5] = (float)(t[9] - t[0] * (3 * sy * sz));
    } else {
        // Children's moments loaded together (at most 8, unrolled): one
        // round trip to L2 per level instead of one per child.  By the
        // parallel-axis theorem,
        //   Q_p = sum_k [ Q_k + M_k (3 d_k d_k^T - |d_k|^2 I) ],  d_k = com_k - com_p.
        float4 mo[8];
#if MOM_CPASYNC
        // masses and centres and the quadrupoles' first four components
        // land in shared memory by asynchronous copies (no registers held),
        // the last two in registers: one round trip for all of it
        float2 qq2[8];
        if (stage) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const unsigned kk = k < (int)nch ? (unsigned)k : 0u;   // an address inside the arrays
                cp_async16(stage + k * MOM_CTHREADS, a.mono + cb + kk, k < (int)nch);
                cp_async16(stage + (8 + k) * MOM_CTHREADS, a.qa + cb + kk, k < (int)nch);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
#pragma unroll
        for (int k = 0; k < 8; k++) qq2[k] = k < (int)nch ? __ldcg(a.qb + cb + k) : make_float2(0.f, 0.f);
        if (stage) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
            for (int k = 0; k < 8; k++) mo[k] = stage[k * MOM_CTHREADS];
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) mo[k] = k < (int)nch ? __ldcg(a.mono + cb + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#else
#pragma unroll
        for (int k = 0; k < 8; k++) mo[k] = k < (int)nch ? __ldcg(a.mono + cb + k) : make_float4(0.f, 0.f, 0.f, 0.f);
#endif
        const float c0x = mo[0].x, c0y = mo[0].y, c0z = mo[0].z;
        float fM = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (k < (int)nch) {
                fM += mo[k].w;
                ax = fmaf(mo[k].w, mo[k].x - c0x, ax);
                ay = fmaf(mo[k].w, mo[k].y - c0y, ay);
                az = fmaf(mo[k].w, mo[k].z - c0z, az);
            }
        }
        const float inv2 = fM > 0.f ? 1.f / fM : 0.f;
        m.M = fM; m.x = c0x + ax * inv2; m.y = c0y + ay * inv2; m.z = c0z + az * inv2;
        for (int i = 0; i < 6; i++) m.q[i] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (k < (int)nch) {
#if MOM_CPASYNC
                const float4 q4 = stage ? stage[(8 + k) * MOM_CTHREADS] : __ldcg(a.qa + cb + k);
                const float2 q2 = qq2[k];
#else
                const float4 q4 = __ldcg(a.qa + cb + k);
                const float2 q2 = __ldcg(a.qb + cb + k);
#endif
                const float dx = mo[k].x - m.x, dy = mo[k].y - m.y, dz = mo[k].z - m.z;
                const float d2 = dx * dx + dy * dy + dz * dz;
                m.q[0] += -q4.x + mo[k].w * (3.f * dx * dx - d2);
                m.q[1] += -q4.y + mo[k].w * (3.f * dy * dy - d2);
                m.q[2] += -q4.z + mo[k].w * (3.f * dz * dz - d2);
                m.q[3] += -q4.w + mo[k].w * (3.f * dx * dy);
                m.q[4] += -q2.x + mo[k].w * (3.f * dx * dz);
                m.q[5] += -q2.y + mo[k].w * (3.f * dy * dz);
            }
        }
    }
    store32(c, m, a.mono, a.qa, a.qb);
    if (REFIT) {
        float3 pc;
        float e = 0.5f * cell_cube(kb, lv, sysb, a.stc, pc);
        for (unsigned k = 0; k < nch; k++) {
            const float4 ce = __ldcg(a.cext + cb + k);
            e = fmaxf(e, dist_inf(make_float3(ce.x, ce.y, ce.z), pc) + ce.w);
        }
        put_delta(c, m, make_float2(com_offset(make_float3(m.x, m.y, m.z), pc), 2.f * e), a.delta, a.test,
                  a.inv_theta);
        a.cext[c] = make_float4(pc.x, pc.y, pc.z, e);
    } else {
        put_delta(c, m, cell_delta(kb, lv, sysb, make_float3(m.x, m.y, m.z), a.stc), a.delta, a.test, a.inv_theta);
    }
    if (lv == 1) root_terms(c, m, kb, sysb, a.stc, a.shadow);
}

// Leaf pass: one thread per cell, from the end of the breadth-first
// numbering.  A leaf sums its bodies; an internal cell writes its arrival
// word, the number of its internal children (contiguous links), and one
// without any is appended to the start list (one atomic per warp, lanes in
// cell order, so the list runs roughly deepest first).
template <bool REFIT>
__global__ void __launch_bounds__(256, MOM_MINB)
k_mom_leaves(MomArrays a) {
    const unsigned nc = a.stc->ncells;
    if (a.stc->status & ST_TIMEOUT) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    // every lane of a warp runs the same iterations (the ballot below)
    for (unsigned i0 = blockIdx.x * blockDim.x; i0 < nc; i0 += gridDim.x * blockDim.x) {
        const unsigned i = i0 + threadIdx.x;
        const unsigned c = nc - 1u - i;
        bool start = false;
        if (i < nc) {
            const uint2 link = a.cell_link[c];
            const int lev = a.cell_level[c];
            if (link.y & LEAF_BIT) {
                leaf_cell<REFIT>(c, link, lev, a);
            } else {
                uint2 ch[8];
#pragma unroll
                for (int k = 0; k < 8; k++)
                    ch[k] = k < (int)link.y ? a.cell_link[link.x + k] : make_uint2(0u, LEAF_BIT);
                unsigned ni = 0;
#pragma unroll
                for (int k = 0; k < 8; k++) ni += (ch[k].y & LEAF_BIT) ? 0u : 1u;
                a.cell_done[c] = ni;
                start = ni == 0u;
            }
        }
        const unsigned sm = __ballot_sync(0xffffffffu, start);
        if (sm) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(a.nstart, (unsigned)__popc(sm));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (start) a.starts[base + __popc(sm & lt)] = c;
        }
    }
}


// Combine pass (persistent grid over the start list): a listed cell combines
// its children (all leaves), then climbs while it is the last internal child
// of its parent to arrive.  Arrival: release (this cell's moments are visible
// to whoever reads the word after the decrement) and acquire (the last child
// sees every sibling's moments: each sibling's decrement heads a release
// sequence that this read-modify-write extends).  Only the list's cells
// start, so a block is not held by climbs for cells that have nothing to do.
template <bool REFIT>
__global__ void __launch_bounds__(MOM_CTHREADS, MOM_MINB2)
k_mom_combine(MomArrays a) {
    if (a.stc->status & ST_TIMEOUT) return;
#if MOM_CPASYNC
    __shared__ float4 s_stage[16 * MOM_CTHREADS];     // per thread: 8 children x (mono, qa)
    float4 *stage = s_stage + threadIdx.x;
#else
    float4 *stage = nullptr;
#endif
    const unsigned ns = __ldcg(a.nstart);
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
        unsigned c = __ldcg(a.starts + j);
        uint2 plk = a.cell_link[c];
        int lv = a.cell_level[c];
        unsigned p = lv != 0 ? a.cell_parent[c] : 0u;
        // a body inside the cell: its key prefix gives the centre of the
        // cell and of every ancestor
        const unsigned b = a.cell_body[c].x;
        const unsigned long long kb = a.sk[b];
        const int sysb = a.multi ? a.sysid[b] : 0;
        combine_cell<REFIT>(c, lv, plk, kb, sysb, a, stage);
        while (lv != 0) {
            // the parent's link and level and the next parent are loaded with
            // the arrival atomic (the tree is read-only here)
            const uint2 pl = a.cell_link[p];
            const int plv = a.cell_level[p];
            const unsigned gp = plv != 0 ? a.cell_parent[p] : 0u;
            if (atom_add_acq_rel_gpu(&a.cell_done[p], 0xffffffffu) != 1u) break;   // decrement
            c = p; plk = pl; lv = plv; p = gp;
            combine_cell<REFIT>(c, lv, plk, kb, sysb, a, stage);
        }
    }
}

// Launch size: one thread per cell of the last known cell count (plus an
// eighth), or of a typical count for the leaf size when none is known; a
// grid-stride loop covers a tree that grew beyond it.
static unsigned multipole_blocks(const Ctx &c) {
    long long cells = c.cells_hint > 0 ? c.cells_hint + c.cells_hint / 8 + 1024 : 8 * c.n / c.nleaf + 1024;
    if (cells > c.ccap) cells = c.ccap;
    return (unsigned)((cells + 255) / 256);
}

static MomArrays mom_arrays(Ctx &c, float theta, bool refit) {
    return MomArrays{c.st, c.cell_body, c.cell_link, c.cell_level, c.cell_parent, c.cell_done, c.pos4, c.keys,
                     c.sysid, c.mono, c.quadA, c.quadB, c.delta, c.shadow, refit ? c.cext : nullptr,
                     theta > 0.f ? c.test : nullptr, theta > 0.f ? 1.0f / theta : 0.f, c.nsys > 1,
                     c.cell_start, &c.st->mom_starts};
}

// Both passes: the start list is emptied first (a memset node in a graph).
template <bool REFIT>
static cudaError_t launch_mom(Ctx &c, const MomArrays &a) {
    cudaError_t e = cudaMemsetAsync(a.nstart, 0, sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    k_mom_leaves<REFIT><<<multipole_blocks(c), 256, 0, c.stream>>>(a);
    k_mom_combine<REFIT><<<c.num_sms * MOM_CBLOCKS, MOM_CTHREADS, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// theta > 0: also the walk's MAC records for that opening angle (what
// launch_open_radius writes), so that a step needs no separate pass.
cudaError_t launch_multipoles(Ctx &c, float theta) {
    return launch_mom<false>(c, mom_arrays(c, theta, false));
}

// Moments of the existing cells at the bodies' current positions (block time
// steps between rebuilds), with each cell's cube enlarged to hold its bodies.
cudaError_t launch_multipoles_refit(Ctx &c) {
    return launch_mom<true>(c, mom_arrays(c, 0.f, true));
}

// cext[c] = (geometric centre, l / 2) of every cell from its first body's
// key: the cubes the neighbour search tests (the bodies lie in them right
// after a build).
__global__ void k_cell_cubes(const DevState *__restrict__ st, const uint2 *__restrict__ cell_body,
                             const uint8_t *__restrict__ cell_level, const unsigned long long *__restrict__ sk,
                             const uint8_t *__restrict__ sysid, float4 *cext) {
    const unsigned nc = st->ncells;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const unsigned b = cell_body[c].x;
        float3 ctr;
        const float l = cell_cube(sk[b], cell_level[c], sysid[b], st, ctr);
        cext[c] = make_float4(ctr.x, ctr.y, ctr.z, 0.5f * l);
    }
}

cudaError_t launch_cell_cubes(Ctx &c) {
    const unsigned grid = (unsigned)min((c.ccap + 255) / 256, (long long)c.num_sms * 8);
    k_cell_cubes<<<grid, 256, 0, c.stream>>>(c.st, c.cell_body, c.cell_level, c.keys, c.sysid, c.cext);
    return cudaGetLastError();
}

// test[c] = (com, l/theta + delta), l = S / 2^level: the opening radius of
// the Barnes (1994) criterion as read here.
__global__ void k_open_radius(const DevState *__restrict__ st, const float4 *__restrict__ mono,
                              const float2 *__restrict__ delta, float inv_theta, float4 *test,
                              const unsigned *__restrict__ gate) {
    if (gate && *gate == 0u) return;
    const unsigned nc = st->ncells;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const float4 m = mono[c];
        const float2 dl = delta[c];
        test[c] = make_float4(m.x, m.y, m.z, fmaf(dl.y, inv_theta, dl.x));
    }
}

cudaError_t launch_open_radius(Ctx &c, float theta, const unsigned *gate) {
    const unsigned grid = (unsigned)min((c.ccap + 255) / 256, (long long)c.num_sms * 8);
    k_open_radius<<<grid, 256, 0, c.stream>>>(c.st, c.mono, c.delta, 1.0f / theta, c.test, gate);
    return cudaGetLastError();
}

}  // namespace bonsai
