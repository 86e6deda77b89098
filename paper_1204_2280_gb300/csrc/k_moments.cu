// k_moments.cu -- multipole moments of every cell (paper Sect. 2,
// "computation of the multipole moments") and the opening radius of the MAC.
//
// Per cell: mass M, centre of mass com and traceless quadrupole
//   Q_ij = sum m (3 y_i y_j - |y|^2 delta_ij),  y = x - com.
// Leaves are summed from their bodies in cell-relative coordinates (offsets
// from the first body, then from the com).  Parents combine their children
// by the parallel-axis theorem,
//   Q_p = sum_k [ Q_k + M_k (3 d_k d_k^T - |d_k|^2 I) ],  d_k = com_k - com_p,
// in one launch: each thread finishing a cell bumps its parent's arrival
// counter and the last child to arrive combines the parent (no waiting).
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

// Sums over the MG lanes of a cell's lane group (xor butterfly: every lane
// ends with the same value, the adds being commutative).
constexpr int MG = 8;   // lanes per cell: a leaf's bodies, a parent's (<= 8) children
__device__ __forceinline__ float group_sum(float v, unsigned gm) {
#pragma unroll
    for (int o = MG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o);
    return v;
}
__device__ __forceinline__ float group_max(float v, unsigned gm) {
#pragma unroll
    for (int o = MG / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(gm, v, o));
    return v;
}

// REFIT (block time steps, between rebuilds): the bodies may have left the
// cells they were sorted into.  Each cell also gets ext = half side of a cube
// about its build-time centre that holds its bodies (at least l/2; a leaf
// from its bodies, a parent as max(l/2, max_k |centre_k - centre|_inf +
// ext_k)), stored with the centre in cext, and delta holds (|com - centre|,
// 2 ext): the opening radius 2 ext / theta + delta then keeps every cell that
// holds a body of a group opened for it (theta < 2 / sqrt(3)).
//
// One cell per group of MG lanes (sl = lane within the group, gm = the
// group's lane mask): a leaf's bodies are spread over the lanes and its sums
// reduced by shuffles; each parent's children (at most eight) are loaded and
// combined one per lane.  The group's first lane stores and takes the
// arrival atomics.
template <bool REFIT>
__device__ __forceinline__ void multipole_cell(unsigned c, int sl, unsigned gm, const DevState *__restrict__ stc,
                                               const uint2 *__restrict__ cell_link,
                                               const uint8_t *__restrict__ cell_level,
                                               const uint32_t *__restrict__ cell_parent, uint32_t *cell_done,
                                               const float4 *__restrict__ pos4, const unsigned long long *__restrict__ sk,
                                               const uint8_t *__restrict__ sysid, float4 *mono, float4 *qa, float2 *qb,
                                               float2 *delta, double *shadow, float4 *cext,
                                               float4 *test, float inv_theta) {
    uint2 link = cell_link[c];
    if (!(link.y & LEAF_BIT)) return;
    const int leader = (threadIdx.x & 31) & ~(MG - 1);

    // Leaf from its bodies in one pass: mass, first and second moments of
    // the offsets u = x - x0 from the first body; then with c = s/M the
    // central moments C = S - s c^T and Q = 3C - tr(C) I.  The offsets are
    // at most the cell size, so nothing cancels beyond FP32 rounding.
    const unsigned b = link.x, cnt = link.y & ~LEAF_BIT;
    int lev = cell_level[c];                         // level and parent, for the climb
    unsigned p = lev != 0 ? cell_parent[c] : 0u;
    const float4 x0 = pos4[b];
    float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
    float3 ctr = make_float3(0.f, 0.f, 0.f);
    float ext = 0.f;
    if (REFIT) ext = 0.5f * cell_cube(sk[b], lev, sysid[b], stc, ctr);
    for (unsigned j = b + sl; j < b + cnt; j += MG) {
        const float4 q = pos4[j];
        if (REFIT) ext = fmaxf(ext, dist_inf(make_float3(q.x, q.y, q.z), ctr));
        const float ux = q.x - x0.x, uy = q.y - x0.y, uz = q.z - x0.z;
        const float wx = q.w * ux, wy = q.w * uy, wz = q.w * uz;
        M += q.w;
        sx += wx; sy += wy; sz += wz;
        sxx = fmaf(wx, ux, sxx); syy = fmaf(wy, uy, syy); szz = fmaf(wz, uz, szz);
        sxy = fmaf(wx, uy, sxy); sxz = fmaf(wx, uz, sxz); syz = fmaf(wy, uz, syz);
    }
    M = group_sum(M, gm);
    sx = group_sum(sx, gm); sy = group_sum(sy, gm); sz = group_sum(sz, gm);
    sxx = group_sum(sxx, gm); syy = group_sum(syy, gm); szz = group_sum(szz, gm);
    sxy = group_sum(sxy, gm); sxz = group_sum(sxz, gm); syz = group_sum(syz, gm);
    if (REFIT) ext = group_max(ext, gm);
    Mom32 m;
    m.M = M;
    const float inv = M > 0.f ? 1.f / M : 0.f;
    const float cx = sx * inv, cy = sy * inv, cz = sz * inv;
    m.x = x0.x + cx; m.y = x0.y + cy; m.z = x0.z + cz;
    const float Cxx = fmaf(-sx, cx, sxx), Cyy = fmaf(-sy, cy, syy), Czz = fmaf(-sz, cz, szz);
    const float tr = Cxx + Cyy + Czz;
    m.q[0] = 3.f * Cxx - tr; m.q[1] = 3.f * Cyy - tr; m.q[2] = 3.f * Czz - tr;
    m.q[3] = 3.f * fmaf(-sx, cy, sxy); m.q[4] = 3.f * fmaf(-sx, cz, sxz); m.q[5] = 3.f * fmaf(-sy, cz, syz);
    // The first body's key shares the key prefix of the leaf and of every
    // ancestor: it gives every geometric centre on the way up.
    const unsigned long long kb = sk[b];
    const int sysb = sysid[b];
    if (sl == 0) {
        store32(c, m, mono, qa, qb);
        if (REFIT) {
            put_delta(c, m, make_float2(com_offset(make_float3(m.x, m.y, m.z), ctr), 2.f * ext), delta, test,
                      inv_theta);
            cext[c] = make_float4(ctr.x, ctr.y, ctr.z, ext);
        } else {
            put_delta(c, m, cell_delta(kb, lev, sysb, make_float3(m.x, m.y, m.z), stc), delta, test, inv_theta);
        }
    }

    // Up the tree while this group holds the last child to finish (roots are
    // the level-0 cells, one per system).  The tree is read-only here: the
    // parent's link and level and the next parent are loaded with the
    // arrival atomic, so only the children's moments wait for its acquire.
    while (lev != 0) {
        const uint2 plk = cell_link[p];          // (first child, child count) of the parent
        const int lv = cell_level[p];
        const unsigned gp = lv != 0 ? cell_parent[p] : 0u;
        if (lev == 1 && sl == 0) root_terms(c, m, kb, sysb, stc, shadow);
        // Release: this cell's moments (stored by the group's first lane)
        // are visible to whoever reads the counter after this add; acquire:
        // the last child to arrive sees every sibling's moments (each
        // sibling's add heads a release sequence that this read-modify-write
        // extends), and the warp barrier passes that view to the group.
        unsigned old = 0u;
        if (sl == 0) old = atom_add_acq_rel_gpu(&cell_done[p], 1u);
        old = __shfl_sync(gm, old, leader);
        if (old != plk.y - 1u) return;
        __syncwarp(gm);
        c = p;
        p = gp;
        const unsigned cb = plk.x, nch = plk.y;
        lev = lv;
        if (lv == 0) {
            if (sl != 0) return;
            float3 o;
            cell_cube(kb, 0, sysb, stc, o);
            double t[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (unsigned k = 0; k < nch; k++) {
                const double *sk2 = shadow + 10 * (size_t)(cb + k);
#pragma unroll
                for (int i = 0; i < 10; i++) t[i] += __ldcg(sk2 + i);
            }
            const double inv2 = t[0] > 0 ? 1.0 / t[0] : 0.0;
            const double sx2 = t[1] * inv2, sy2 = t[2] * inv2, sz2 = t[3] * inv2;   // com - O
            const double s2 = sx2 * sx2 + sy2 * sy2 + sz2 * sz2;
            m.M = (float)t[0];
            m.x = (float)(o.x + sx2); m.y = (float)(o.y + sy2); m.z = (float)(o.z + sz2);
            m.q[0] = (float)(t[4] - t[0] * (3 * sx2 * sx2 - s2));
            m.q[1] = (float)(t[5] - t[0] * (3 * sy2 * sy2 - s2));
            m.q[2] = (float)(t[6] - t[0] * (3 * sz2 * sz2 - s2));
            m.q[3] = (float)(t[7] - t[0] * (3 * sx2 * sy2));
            m.q[4] = (float)(t[8] - t[0] * (3 * sx2 * sz2));
            m.q[5] = (float)(t[9] - t[0] * (3 * sy2 * sz2));
        } else {
            // Child sl of the parent on lane sl: mass and com first (about
            // the first child's com), then the parallel-axis terms.
            const bool mine = (unsigned)sl < nch;
            const float4 mo = mine ? __ldcg(mono + cb + sl) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 a = mine ? __ldcg(qa + cb + sl) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float2 q2 = mine ? __ldcg(qb + cb + sl) : make_float2(0.f, 0.f);
            const float c0x = __shfl_sync(gm, mo.x, leader), c0y = __shfl_sync(gm, mo.y, leader),
                        c0z = __shfl_sync(gm, mo.z, leader);
            const float fM = group_sum(mo.w, gm);
            const float ax = group_sum(mo.w * (mo.x - c0x), gm), ay = group_sum(mo.w * (mo.y - c0y), gm),
                        az = group_sum(mo.w * (mo.z - c0z), gm);
            const float inv2 = fM > 0.f ? 1.f / fM : 0.f;
            m.M = fM; m.x = c0x + ax * inv2; m.y = c0y + ay * inv2; m.z = c0z + az * inv2;
            const float dx = mo.x - m.x, dy = mo.y - m.y, dz = mo.z - m.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            const float w = mo.w;     // 0 on lanes without a child: their terms vanish
            m.q[0] = group_sum(-a.x + w * (3.f * dx * dx - d2), gm);
            m.q[1] = group_sum(-a.y + w * (3.f * dy * dy - d2), gm);
            m.q[2] = group_sum(-a.z + w * (3.f * dz * dz - d2), gm);
            m.q[3] = group_sum(-a.w + w * (3.f * dx * dy), gm);
            m.q[4] = group_sum(-q2.x + w * (3.f * dx * dz), gm);
            m.q[5] = group_sum(-q2.y + w * (3.f * dy * dz), gm);
        }
        float3 pc = make_float3(0.f, 0.f, 0.f);
        float e = 0.f;
        if (REFIT) {
            e = 0.5f * cell_cube(kb, lv, sysb, stc, pc);
            if (lv == 0) {
                for (unsigned k = 0; k < nch; k++) {
                    const float4 ce = __ldcg(cext + cb + k);
                    e = fmaxf(e, dist_inf(make_float3(ce.x, ce.y, ce.z), pc) + ce.w);
                }
            } else {
                const float4 ce = (unsigned)sl < nch ? __ldcg(cext + cb + sl) : make_float4(pc.x, pc.y, pc.z, 0.f);
                e = group_max(fmaxf(e, dist_inf(make_float3(ce.x, ce.y, ce.z), pc) + ce.w), gm);
            }
        }
        if (sl == 0) {
            store32(c, m, mono, qa, qb);
            if (REFIT) {
                put_delta(c, m, make_float2(com_offset(make_float3(m.x, m.y, m.z), pc), 2.f * e), delta, test,
                          inv_theta);
                cext[c] = make_float4(pc.x, pc.y, pc.z, e);
            } else {
                put_delta(c, m, cell_delta(kb, lv, sysb, make_float3(m.x, m.y, m.z), stc), delta, test, inv_theta);
            }
        }
    }
}

// Groups of MG lanes take the cells from the end of the breadth-first
// numbering (the deepest leaves, whose climbs to the root are the longest,
// have the largest numbers, so those climbs start in the first wave); a
// grid-stride loop covers any cell count, and the launch is sized from the
// last known count so that nearly every group takes a single cell.
template <bool REFIT>
__global__ void __launch_bounds__(256, 4)
k_multipoles(const DevState *__restrict__ stc, const uint2 *__restrict__ cell_link,
             const uint8_t *__restrict__ cell_level, const uint32_t *__restrict__ cell_parent, uint32_t *cell_done,
             const float4 *__restrict__ pos4, const unsigned long long *__restrict__ sk,
             const uint8_t *__restrict__ sysid, float4 *mono, float4 *qa, float2 *qb, float2 *delta,
             double *shadow, float4 *cext, float4 *test, float inv_theta) {
    const unsigned nc = stc->ncells;
    if (stc->status & ST_TIMEOUT) return;
    const int lane = threadIdx.x & 31, sl = lane & (MG - 1);
    const unsigned gm = ((1u << MG) - 1u) << (lane & ~(MG - 1));
    const unsigned ngroups = gridDim.x * (blockDim.x / MG);
    for (unsigned i = (blockIdx.x * blockDim.x + threadIdx.x) / MG; i < nc; i += ngroups)
        multipole_cell<REFIT>(nc - 1u - i, sl, gm, stc, cell_link, cell_level, cell_parent, cell_done, pos4, sk,
                              sysid, mono, qa, qb, delta, shadow, cext, test, inv_theta);
}

// Launch size: one lane group per cell of the last known cell count (plus an
// eighth), or of a typical count for the leaf size when none is known.
static unsigned multipole_blocks(const Ctx &c) {
    long long cells = c.cells_hint > 0 ? c.cells_hint + c.cells_hint / 8 + 1024 : 8 * c.n / c.nleaf + 1024;
    if (cells > c.ccap) cells = c.ccap;
    return (unsigned)((cells * MG + 255) / 256);
}

// theta > 0: also the walk's MAC records for that opening angle (what
// launch_open_radius writes), so that a step needs no separate pass.
cudaError_t launch_multipoles(Ctx &c, float theta) {
    k_multipoles<false><<<multipole_blocks(c), 256, 0, c.stream>>>(
        c.st, c.cell_link, c.cell_level, c.cell_parent, c.cell_done, c.pos4, c.keys, c.sysid, c.mono, c.quadA,
        c.quadB, c.delta, c.shadow, nullptr, theta > 0.f ? c.test : nullptr, theta > 0.f ? 1.0f / theta : 0.f);
    return cudaGetLastError();
}

// Moments of the existing cells at the bodies' current positions (block time
// steps between rebuilds), with each cell's cube enlarged to hold its bodies.
cudaError_t launch_multipoles_refit(Ctx &c) {
    k_multipoles<true><<<multipole_blocks(c), 256, 0, c.stream>>>(
        c.st, c.cell_link, c.cell_level, c.cell_parent, c.cell_done, c.pos4, c.keys, c.sysid, c.mono, c.quadA,
        c.quadB, c.delta, c.shadow, c.cext, nullptr, 0.f);
    return cudaGetLastError();
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
