// k_tree.cu -- body reorder ("moving") and octree construction from sorted
// keys ("tree-construction"), paper Sect. 2.
//
// The tree is the level-by-level octree of the sorted keys: the root holds
// all bodies; a cell with more than nleaf bodies below the deepest level
// splits into its non-empty octants; cells are numbered breadth first, in key
// order within a level, so children are contiguous.
//
// Instead of 22 dependent level launches, the build uses the fact that the
// cells are runs of equal key prefixes: with cpl(a,b) the number of leading
// levels two keys share,
//   l0(t) = cpl(k[t-1], k[t]) + 1          first level at which body t starts a run
//   D(t)  = cpl(k[t], k[t+nleaf])          the run from t at level l has > nleaf
//                                          bodies iff l <= D(t)
// A cell (level l, first body t) exists iff the run at level l-1 containing t
// has more than nleaf bodies.  For l > l0(t) that run also starts at t; for
// l = l0(t) its length is read from per-level bit masks of run starts over a
// 64-body halo (a longer run is split in any case).  So body t starts exactly
// the cells of levels lo..hi with lo = l0(t) (if that parent run is split)
// and hi = max(lo, min(D(t)+1, 21)); the one at hi is a leaf.  Groups (cells
// with <= ncrit bodies whose parent has more) follow the same way with ncrit
// in place of nleaf.  Four launches: count per block and level, scan per
// level, write cells, link children and internal body counts.
#include "common.cuh"

namespace bonsai {

__global__ void k_reorder(const uint32_t *__restrict__ perm, const float4 *__restrict__ pin,
                          const float4 *__restrict__ vin, const uint32_t *__restrict__ idin, int n,
                          float4 *pout, float4 *vout, uint32_t *idout) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t s = perm[i];
    pout[i] = pin[s];
    vout[i] = vin[s];
    idout[i] = idin[s];
}

cudaError_t launch_reorder(Ctx &c) {
    int n = (int)c.n;
    k_reorder<<<(n + 255) / 256, 256, 0, c.stream>>>(c.vals, c.pos4_alt, c.vel4_alt, c.id_alt, n,
                                                     c.pos4, c.vel4, c.id);
    return cudaGetLastError();
}

// First index > t whose level-`level` key prefix differs from k[t], or n
// (the end of t's system): galloping then bisection.
__device__ int run_end(const unsigned long long *__restrict__ sk, int n, int t, int level) {
    if (level == 0) return n;
    int sh = 3 * (MAX_LEVEL - level);
    unsigned long long pre = sk[t] >> sh;
    int lo = t, hi = n, step = 1;
    while (true) {
        long long probe = (long long)t + step;
        if (probe >= n) { hi = n; break; }
        if ((sk[probe] >> sh) != pre) { hi = (int)probe; break; }
        lo = (int)probe;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int mid = lo + ((hi - lo) >> 1);
        if ((sk[mid] >> sh) == pre) lo = mid; else hi = mid;
    }
    return hi;
}

__device__ __forceinline__ unsigned digit_at(unsigned long long k, int level) {
    return (unsigned)(k >> (3 * (MAX_LEVEL - level))) & 7u;
}

struct BodyCells {
    bool has;
    int lo, hi, ngrp, lg;   // lg: group level (>hi: oversize leaf cut in chunks)
};

// Shared memory of a build block.  The block's bodies are [base, base+B);
// a halo of BW = 64 bodies on each side gives the extended range
// [base-BW, base+B+BW) of BCH chunks of 32 positions, plus one key below it.
//   M[l * BCH + c], bit i: position 32c + i of the extended range is the
//   first body of a level-l key-prefix run (l0 <= l; every position outside
//   [1, n) and every first body of a system counts as one).
// Any run that matters here (<= 64 bodies around a body of the block) is
// then answered by bit operations on at most five mask words per query.
constexpr int BW = 64;
constexpr int BCH = (BUILD_THREADS + 2 * BW) / 32;

struct BuildShared {
    unsigned long long *k;   // keys of [base-BW-1, base+B+BW)
    uint8_t *sy;             // system ids, same range
    unsigned *M;             // run-start masks, (MAX_LEVEL + 1) x BCH
    int base;
    __device__ unsigned long long key(int j) const { return k[j - base + BW + 1]; }
    __device__ uint8_t sys(int j) const { return sy[j - base + BW + 1]; }
    __device__ int cpl(int a, int b) const { return body_cpl(key(a), key(b), sys(a), sys(b)); }

    // First body s <= t and end e > t of the level-l run holding body t of
    // the block, as extended-range positions; -4096 / 1 << 20 when farther
    // than the two neighbouring chunks (then the run exceeds 64 bodies).
    __device__ void run_of(int t, int l, int &s, int &e) const {
        const int q = t - base + BW, c = q >> 5, i = q & 31;
        const unsigned *Ml = M + l * BCH;
        const unsigned a0 = Ml[c] & (0xffffffffu >> (31 - i));
        const unsigned a1 = Ml[c - 1], a2 = Ml[c - 2];
        s = a0 ? (c << 5) + 31 - __clz(a0)
               : a1 ? ((c - 1) << 5) + 31 - __clz(a1) : a2 ? ((c - 2) << 5) + 31 - __clz(a2) : -4096;
        const unsigned b0 = i == 31 ? 0u : (Ml[c] & (0xffffffffu << (i + 1)));
        const unsigned b1 = Ml[c + 1], b2 = Ml[c + 2];
        e = b0 ? (c << 5) + __ffs(b0) - 1
               : b1 ? ((c + 1) << 5) + __ffs(b1) - 1 : b2 ? ((c + 2) << 5) + __ffs(b2) - 1 : 1 << 20;
    }
    // Whether the level-l run holding t has more than w (<= 64) bodies.
    __device__ bool run_longer(int t, int l, int w) const {
        int s, e;
        run_of(t, l, s, e);
        return e - s > w;
    }
    // End (exclusive) of the level-l run starting at t: from the masks when
    // within the halo, else by the global search.
    __device__ int run_end_at(const unsigned long long *__restrict__ sk, int send, int t, int l) const {
        if (l == 0) return send;
        int s, e;
        run_of(t, l, s, e);
        return e < (1 << 20) ? min(send, base - BW + e) : run_end(sk, send, t, l);
    }
};

// Keys and system ids of the extended range, then the run-start masks: one
// chunk per warp and pass, 22 ballots, lane l keeps level l's mask.
__device__ BuildShared load_build_shared(void *smem, const unsigned long long *__restrict__ sk,
                                         const uint8_t *__restrict__ sysid, int n, int base) {
    BuildShared b;
    b.base = base;
    constexpr int NK = BUILD_THREADS + 2 * BW + 1;
    b.k = (unsigned long long *)smem;
    b.M = (unsigned *)(b.k + NK);
    b.sy = (uint8_t *)(b.M + (MAX_LEVEL + 1) * BCH);
    for (int i = threadIdx.x; i < NK; i += blockDim.x) {
        const int j = base - BW - 1 + i;
        const bool in = j >= 0 && j < n;
        b.k[i] = in ? sk[j] : 0ull;
        b.sy[i] = in ? sysid[j] : 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int c = threadIdx.x >> 5; c < BCH; c += BUILD_THREADS / 32) {
        const int j = base - BW + (c << 5) + lane;
        const int l0 = (j > 0 && j < n) ? b.cpl(j - 1, j) + 1 : 0;
        unsigned mine = 0u;
#pragma unroll
        for (int l = 0; l <= MAX_LEVEL; l++) {
            const unsigned m = __ballot_sync(0xffffffffu, l0 <= l);
            if (lane == l) mine = m;
        }
        if (lane <= MAX_LEVEL) b.M[lane * BCH + c] = mine;
    }
    __syncthreads();
    return b;
}

size_t build_smem_bytes(int, int) {
    return (size_t)(BUILD_THREADS + 2 * BW + 1) * 9 + (size_t)(MAX_LEVEL + 1) * BCH * 4;
}

// Which cells body t starts (levels lo..hi) and how many groups; send is the
// end of t's system.
__device__ BodyCells analyse_body(const BuildShared &b, int t, int n, int nleaf, int ncrit,
                                  const unsigned long long *__restrict__ sk, int send) {
    BodyCells r{false, 0, -1, 0, 0};
    if (t >= n) return r;
    const int l0 = t == 0 ? 0 : b.cpl(t - 1, t) + 1;
    if (l0 > MAX_LEVEL) return r;
    if (l0 > 0 && !b.run_longer(t, l0 - 1, nleaf)) return r;     // parent not split
    r.has = true;
    r.lo = l0;
    const int D = t + nleaf < n ? b.cpl(t, t + nleaf) : -1;
    r.hi = max(l0, min(D + 1, MAX_LEVEL));
    const int DG = t + ncrit < n ? b.cpl(t, t + ncrit) : -1;
    const int lg = max(l0, DG + 1);
    r.lg = lg;
    if (lg <= r.hi) {
        const bool starts = (lg > l0) || l0 == 0 || b.run_longer(t, l0 - 1, ncrit);
        r.ngrp = starts ? 1 : 0;
    } else {
        const int cnt = b.run_end_at(sk, send, t, r.hi) - t;
        r.ngrp = (cnt + ncrit - 1) / ncrit;
    }
    return r;
}

__device__ __forceinline__ int system_end(const DevState *__restrict__ st, const uint8_t *__restrict__ sysid,
                                          int t, int n) {
    return t < n ? (int)st->sys_off[sysid[t] + 1] : n;
}

__device__ __forceinline__ bool has_level(const BodyCells &bc, int r) {
    return bc.has && bc.lo <= r && r <= bc.hi;
}

// The levels on which any body of the warp starts a cell: [rlo, rhi]
// (empty, rlo > rhi, when none does).  Warp-uniform.
__device__ __forceinline__ void warp_level_range(const BodyCells &bc, int &rlo, int &rhi) {
    rlo = (int)__reduce_min_sync(0xffffffffu, bc.has ? (unsigned)bc.lo : (unsigned)(MAX_LEVEL + 1));
    rhi = (int)__reduce_max_sync(0xffffffffu, bc.has ? (unsigned)bc.hi : 0u);
    if (rlo > MAX_LEVEL) rhi = -1;
}

// Pass 1: per block, the number of cells of each level and of groups.
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_count(const unsigned long long *__restrict__ sk, const uint8_t *__restrict__ sysid, int n,
              int nleaf, int ncrit, unsigned *blockcount, int nblocks, const DevState *__restrict__ st) {
    extern __shared__ unsigned long long smem_u64[];
    __shared__ unsigned s_wc[NROWS][32];
    if (st->status & ST_TIMEOUT) return;        // keys not sorted: skip the build
    const int base = blockIdx.x * BUILD_THREADS, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    BuildShared b = load_build_shared(smem_u64, sk, sysid, n, base);
    const int t = base + tid;
    BodyCells bc = analyse_body(b, t, n, nleaf, ncrit, sk, system_end(st, sysid, t, n));
    int rlo, rhi;
    warp_level_range(bc, rlo, rhi);
    if (lane <= MAX_LEVEL && (lane < rlo || lane > rhi)) s_wc[lane][warp] = 0u;
    for (int r = rlo; r <= rhi; r++) {
        const unsigned m = __ballot_sync(0xffffffffu, has_level(bc, r));
        if (lane == 0) s_wc[r][warp] = __popc(m);
    }
    int g = bc.ngrp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (lane == 0) s_wc[GROUP_ROW][warp] = (unsigned)g;
    __syncthreads();
    if (tid < NROWS) {
        unsigned s = 0;
#pragma unroll 8
        for (int w = 0; w < BUILD_THREADS / 32; w++) s += s_wc[tid][w];
        blockcount[(size_t)tid * nblocks + blockIdx.x] = s;
    }
}

// Pass 2: exclusive scan of each row over blocks (one block per row).
__global__ void __launch_bounds__(1024)
k_build_scan(unsigned *blockcount, int nblocks, DevState *st) {
    __shared__ unsigned s_w[32];
    __shared__ unsigned s_carry;
    unsigned *row = blockcount + (size_t)blockIdx.x * nblocks;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += 1024) {
        int i = b0 + tid;
        unsigned v = i < nblocks ? row[i] : 0u, x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned w = s_w[lane], wx = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, wx, o);
                if (lane >= o) wx += y;
            }
            s_w[lane] = wx - w;
        }
        __syncthreads();
        unsigned carry = s_carry;
        if (i < nblocks) row[i] = carry + s_w[warp] + x - v;
        __syncthreads();
        if (tid == 1023) s_carry = carry + s_w[warp] + x;
        __syncthreads();
    }
    if (tid == 0) st->row_total[blockIdx.x] = s_carry;
}

// Pass 3: number every cell and write its first body, level and link.  For
// each cell (level r, first body t) it also records cb = the number of
// level-(r+1) cells that start before t, offset to level r+1's first index:
// for an internal cell that is its first child, and the children of a cell
// are the level-(r+1) cells between its cb and the next cell's cb.  Leaves
// get their body count here (a short search); internal cells in pass 4.
#ifndef BUILD_WRITE_MIN_BLOCKS
#define BUILD_WRITE_MIN_BLOCKS 2        // two 1024-thread blocks per SM (32 registers)
#endif
__global__ void __launch_bounds__(BUILD_THREADS, BUILD_WRITE_MIN_BLOCKS)
k_build_write(const unsigned long long *__restrict__ sk, const uint8_t *__restrict__ sysid, int n,
              int nleaf, int ncrit, const unsigned *__restrict__ blockcount, int nblocks, long long ccap,
              DevState *st,
              uint2 *cell_body, uint2 *cell_link, uint8_t *cell_level, uint32_t *cell_parent,
              uint32_t *cell_done, uint32_t *cell_cb, uint2 *groups, uint8_t *group_lvl) {
    extern __shared__ unsigned long long smem_u64[];
    __shared__ unsigned s_wc[NROWS][32];
    __shared__ unsigned s_base[NROWS];
    __shared__ int s_ok;
    const int base = blockIdx.x * BUILD_THREADS, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (st->status & ST_TIMEOUT) return;        // keys not sorted: skip the build
    if (warp == 0) {                             // level offsets: one lane per row
        const bool lvl = lane <= MAX_LEVEL;
        const unsigned tot = lane < NROWS ? st->row_total[lane] : 0u;
        const unsigned bcnt = lane < NROWS ? blockcount[(size_t)lane * nblocks + blockIdx.x] : 0u;
        unsigned x = lvl ? tot : 0u;             // inclusive scan of the level totals
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const unsigned run = __shfl_sync(0xffffffffu, x, MAX_LEVEL);   // all cells
        const unsigned excl = x - (lvl ? tot : 0u);
        if (lvl) s_base[lane] = excl + bcnt;
        if (lane == GROUP_ROW) s_base[GROUP_ROW] = bcnt;
        if (lvl && blockIdx.x == 0) st->level_start[lane] = excl;
        if (lane == 0) {
            s_ok = (long long)run <= ccap;
            if (blockIdx.x == 0) {
                st->level_start[MAX_LEVEL + 1] = run;
                st->ncells = run;
                st->ngroups = st->row_total[GROUP_ROW];
                if (!s_ok) atomicOr(&st->status, ST_CAPACITY);
            }
        }
    }
    __syncthreads();
    if (!s_ok) return;
    BuildShared b = load_build_shared(smem_u64, sk, sysid, n, base);
    const int t = base + tid;
    const int send = system_end(st, sysid, t, n);
    BodyCells bc = analyse_body(b, t, n, nleaf, ncrit, sk, send);
    const unsigned lt = (1u << lane) - 1u;
    int rlo, rhi;
    warp_level_range(bc, rlo, rhi);

    if (lane <= MAX_LEVEL && (lane < rlo || lane > rhi)) s_wc[lane][warp] = 0u;
    for (int r = rlo; r <= rhi; r++) {
        const unsigned m = __ballot_sync(0xffffffffu, has_level(bc, r));
        if (lane == 0) s_wc[r][warp] = __popc(m);
    }
    int gx = bc.ngrp;                            // inclusive warp scan of group counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, gx, o);
        if (lane >= o) gx += y;
    }
    if (lane == 31) s_wc[GROUP_ROW][warp] = (unsigned)gx;
    gx -= bc.ngrp;
    __syncthreads();
    constexpr int NW = BUILD_THREADS / 32;
    for (int row = warp; row < NROWS; row += NW) {   // exclusive prefix across warps per row
        unsigned v = lane < NW ? s_wc[row][lane] : 0u, x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncwarp();
        if (lane < NW) s_wc[row][lane] = x - v;
    }
    __syncthreads();

    unsigned bcur = rlo <= rhi ? __ballot_sync(0xffffffffu, has_level(bc, rlo)) : 0u;
    for (int r = rlo; r <= rhi; r++) {
        const unsigned bnext = r < MAX_LEVEL ? __ballot_sync(0xffffffffu, has_level(bc, r + 1)) : 0u;
        if (has_level(bc, r)) {
            const unsigned c = s_base[r] + s_wc[r][warp] + __popc(bcur & lt);
            const unsigned cb = r < MAX_LEVEL ? s_base[r + 1] + s_wc[r + 1][warp] + __popc(bnext & lt) : 0u;
            cell_cb[c] = cb;
            cell_level[c] = (uint8_t)r;
            cell_done[c] = 0u;
            if (r == 0) cell_parent[c] = 0xffffffffu;
            if (r == bc.hi) {
                int cnt = b.run_end_at(sk, send, t, r) - t;
                cell_body[c] = make_uint2((unsigned)t, (unsigned)cnt);
                cell_link[c] = make_uint2((unsigned)t, (unsigned)cnt | LEAF_BIT);
            } else {
                cell_body[c] = make_uint2((unsigned)t, 0u);
                cell_link[c] = make_uint2(cb, 0u);
            }
        }
        bcur = bnext;
    }
    // Groups in key order.
    if (bc.ngrp > 0) {
        unsigned g = s_base[GROUP_ROW] + s_wc[GROUP_ROW][warp] + (unsigned)gx;
        if (bc.lg <= bc.hi) {
            int e = b.run_end_at(sk, send, t, bc.lg);
            groups[g] = make_uint2((unsigned)t, (unsigned)(e - t));
            if (group_lvl) group_lvl[g] = (uint8_t)bc.lg;
        } else {
            int e = b.run_end_at(sk, send, t, bc.hi);
            for (int k = 0; k < bc.ngrp; k++) {
                int b0 = t + k * ncrit;
                groups[g + k] = make_uint2((unsigned)b0, (unsigned)min(ncrit, e - b0));
                if (group_lvl) group_lvl[g + k] = 0xffu;
            }
        }
    }
}

// Child count, children's parent and body count of internal cell c.
__device__ __forceinline__ void link_cell(unsigned c, const DevState *__restrict__ st,
                                               const uint32_t *__restrict__ cell_cb,
                                               const uint8_t *__restrict__ cell_level, uint2 *cell_link,
                                               uint2 *cell_body, uint32_t *cell_parent) {
    if (cell_link[c].y & LEAF_BIT) return;
    auto nchild_of = [&](unsigned d, int l) {
        unsigned next = (d + 1 < st->level_start[l + 1]) ? cell_cb[d + 1] : st->level_start[l + 2];
        return next - cell_cb[d];
    };
    const int l = cell_level[c];
    const unsigned cb = cell_cb[c];
    const unsigned nch = nchild_of(c, l);
    cell_link[c] = make_uint2(cb, nch);
    for (unsigned k = 0; k < nch; k++) cell_parent[cb + k] = c;
    unsigned d = cb + nch - 1;                   // last child, then its last child, ...
    int ld = l + 1;
    uint2 lk = cell_link[d];
    for (int it = 0; it < MAX_LEVEL && !(lk.y & LEAF_BIT); it++) {   // at most 21 levels
        d = cell_cb[d] + nchild_of(d, ld) - 1;
        ld++;
        lk = cell_link[d];
    }
    const unsigned t = cell_body[c].x;
    cell_body[c].y = lk.x + (lk.y & ~LEAF_BIT) - t;
}

// Pass 4 (grid-stride over the cells, internal cells only): child count from the cb of the next
// cell of the same level, parent pointers of the children, and the body
// count from the descent along last children to a leaf.
__global__ void k_build_link(const DevState *__restrict__ st, const uint32_t *__restrict__ cell_cb,
                             const uint8_t *__restrict__ cell_level, uint2 *cell_link,
                             uint2 *cell_body, uint32_t *cell_parent) {
    if (st->status & ST_TIMEOUT) return;
    const unsigned ncells = st->ncells;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x)
        link_cell(c, st, cell_cb, cell_level, cell_link, cell_body, cell_parent);
}

// ---- Sibling packing of the walk groups (group_pack = 1) -------------------
// The unpacked groups (above, in key order) are taken in order; a group that
// is a sibling of the previous one (both cells of one parent) joins the
// packed group the previous one belongs to while the sum stays <= ncrit
// bodies.  Siblings are consecutive in the list (a larger child in between
// puts its own descendants' groups there), and a cell has at most 8 children,
// so every decision looks at most 7 groups back.  Two launches: start flags
// with a count per block, then the block prefix and the packed groups.
// Whether unpacked group g (> 0) is a sibling of group g - 1: two cells of
// the same level l >= 1 (neither the root group nor a run of an oversize
// leaf, level 0xff) with the same level-(l-1) key prefix in the same system.
__device__ __forceinline__ bool group_sibling(unsigned g, const uint2 *__restrict__ graw,
                                              const uint8_t *__restrict__ glvl,
                                              const unsigned long long *__restrict__ sk,
                                              const uint8_t *__restrict__ sysid) {
    if (g == 0) return false;
    const int l = glvl[g];
    if (l == 0 || l > MAX_LEVEL || glvl[g - 1] != l) return false;
    const unsigned a = graw[g - 1].x, b = graw[g].x;
    return sysid[a] == sysid[b] && key_prefix(sk[a], l - 1) == key_prefix(sk[b], l - 1);
}

__device__ __forceinline__ unsigned block_sum_1024(unsigned v, unsigned *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    unsigned t = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0u;
    t = __reduce_add_sync(0xffffffffu, t);
    __syncthreads();
    return t;
}

// Pass 1 (grid-stride over chunks of PACK_THREADS unpacked groups):
// flag[g] = 1 iff group g starts a packed group (greedy from the first group
// of its sibling run); bcount[chunk] = flags set in the chunk.
__global__ void __launch_bounds__(PACK_THREADS)
k_group_mark(const DevState *__restrict__ st, const uint2 *__restrict__ graw, const uint8_t *__restrict__ glvl,
             const unsigned long long *__restrict__ sk, const uint8_t *__restrict__ sysid, int ncrit,
             uint8_t *gflag, unsigned *bcount) {
    if (st->status & ST_TIMEOUT) return;
    const unsigned ng = st->row_total[GROUP_ROW];
    const unsigned nchunk = (ng + PACK_THREADS - 1) / PACK_THREADS;
    for (unsigned ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const unsigned g = ch * PACK_THREADS + threadIdx.x;
        bool start = false;
        if (g < ng) {
            unsigned s = g;
            for (int k = 0; k < 8 && group_sibling(s, graw, glvl, sk, sysid); k++) s--;
            unsigned acc = graw[s].y;
            start = true;
            for (unsigned j = s + 1; j <= g; j++) {
                const unsigned cj = graw[j].y;
                start = acc + cj > (unsigned)ncrit;
                acc = start ? cj : acc + cj;
            }
            gflag[g] = start ? 1u : 0u;
        }
        const int cnt = __syncthreads_count(start);
        if (threadIdx.x == 0) bcount[ch] = (unsigned)cnt;
    }
}

// Pass 2 (same chunks): packed group index = flags set before g (chunks
// before this one, then a block scan); a start writes (first body, bodies up
// to the next start).  Block 0 also stores the packed group count.
__global__ void __launch_bounds__(PACK_THREADS)
k_group_pack(DevState *st, const uint2 *__restrict__ graw, const uint8_t *__restrict__ gflag,
             const unsigned *__restrict__ bcount, uint2 *groups) {
    __shared__ unsigned s_w[32];
    if (st->status & ST_TIMEOUT) return;
    const unsigned ng = st->row_total[GROUP_ROW];
    const unsigned nchunk = (ng + PACK_THREADS - 1) / PACK_THREADS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0) {
        unsigned v = 0;
        for (unsigned i = threadIdx.x; i < nchunk; i += PACK_THREADS) v += bcount[i];
        const unsigned tot = block_sum_1024(v, s_w);
        if (threadIdx.x == 0) st->ngroups = tot;
    }
    for (unsigned ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        unsigned v = 0;
        for (unsigned i = threadIdx.x; i < ch; i += PACK_THREADS) v += bcount[i];
        const unsigned base = block_sum_1024(v, s_w);
        const unsigned g = ch * PACK_THREADS + threadIdx.x;
        const unsigned f = g < ng ? gflag[g] : 0u;
        const unsigned m = __ballot_sync(0xffffffffu, f != 0u);
        if (lane == 0) s_w[warp] = __popc(m);
        __syncthreads();
        if (warp == 0) {                          // exclusive scan of the warp counts
            const unsigned w = s_w[lane];
            unsigned x = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x - w;
        }
        __syncthreads();
        if (f) {
            const unsigned idx = base + s_w[warp] + __popc(m & ((1u << lane) - 1u));
            unsigned cnt = graw[g].y, j = g + 1;
            for (int k = 0; k < 8 && j < ng && gflag[j] == 0u; k++, j++) cnt += graw[j].y;
            groups[idx] = make_uint2(graw[g].x, cnt);
        }
        __syncthreads();                          // s_w is reused by the next chunk
    }
}

cudaError_t launch_build(Ctx &c) {
    int n = (int)c.n;
    size_t smem = build_smem_bytes(c.nleaf, c.ncrit);
    k_build_count<<<c.nbblocks, BUILD_THREADS, smem, c.stream>>>(c.keys, c.sysid, n, c.nleaf, c.ncrit,
                                                                 c.blockcount, c.nbblocks, c.st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_build_scan<<<NROWS, 1024, 0, c.stream>>>(c.blockcount, c.nbblocks, c.st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool pack = c.group_pack != 0;
    k_build_write<<<c.nbblocks, BUILD_THREADS, smem, c.stream>>>(
        c.keys, c.sysid, n, c.nleaf, c.ncrit, c.blockcount, c.nbblocks, c.ccap, c.st, c.cell_body,
        c.cell_link, c.cell_level, c.cell_parent, c.cell_done, c.cell_cb, pack ? c.groups_raw : c.groups,
        pack ? c.group_lvl : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (pack) {
        // at most n unpacked groups: chunks of PACK_THREADS, two blocks per SM
        const unsigned pb = (unsigned)min((long long)(n + PACK_THREADS - 1) / PACK_THREADS, 2ll * c.num_sms);
        k_group_mark<<<pb, PACK_THREADS, 0, c.stream>>>(c.st, c.groups_raw, c.group_lvl, c.keys, c.sysid,
                                                         c.ncrit, c.group_flag, c.group_bcount);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_group_pack<<<pb, PACK_THREADS, 0, c.stream>>>(c.st, c.groups_raw, c.group_flag, c.group_bcount,
                                                         c.groups);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const unsigned grid = (unsigned)min((c.ccap + 255) / 256, (long long)c.num_sms * 8);
    k_build_link<<<grid, 256, 0, c.stream>>>(c.st, c.cell_cb, c.cell_level, c.cell_link, c.cell_body,
                                             c.cell_parent);
    return cudaGetLastError();
}

}  // namespace bonsai
