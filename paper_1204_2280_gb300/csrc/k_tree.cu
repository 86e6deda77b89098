// k_tree.cu -- body reorder ("moving") and octree construction from sorted
// keys ("tree-construction"), paper Sect. 2.
//
// The tree is the level-by-level octree of the sorted keys: the root holds
// all bodies; a cell with more than nleaf bodies below the deepest level
// splits into its non-empty octants; cells are numbered breadth first, in key
// order within a level, so children are contiguous.
//
// Instead of 22 dependent level launches, the build uses the fact that the
// cells are runs of equal key prefixes: every cell is identified by its level
// and its first body, and whether body t starts a cell on a level follows
// from a few common-prefix lengths of keys near t (pass 1 below).  Four
// launches: (1) per body, the levels on which it starts cells and its group,
// compacted per block into a list of the bodies that start any (about one per
// leaf), with counts per block and level; (2) scan of those counts over the
// blocks; (3) per listed body, the index, first body, level and link of each
// of its cells and its groups; (4) child counts and parents.  Internal
// cells' body counts, which no stage of a step reads, are derived on demand
// for the tree getter (k_internal_counts).
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
// (the end of t's system): galloping then bisection.  Only runs of identical
// keys at the deepest level can be longer than the build's 64-body halo.
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

__device__ __forceinline__ int system_end(const DevState *__restrict__ st, const uint8_t *__restrict__ sysid,
                                          int t, int n) {
    return t < n ? (int)st->sys_off[sysid[t] + 1] : n;
}

// ---- Pass 1: which cells and groups every body starts ----------------------
// For body t (within its system) let
//   l0(t) = cpl(k[t-1], k[t]) + 1   the first level at which t starts a key-prefix run
//                                   (0 for the first body of a system)
//   D(t)  = cpl(k[t], k[t+nleaf])   the run at level l from t has more than
//                                   nleaf bodies iff l <= D(t)   (-1: no such body)
//   DG(t) = cpl(k[t], k[t+ncrit])   the same for ncrit.
// The level-L run holding t has more than w bodies iff some window of w+1
// consecutive bodies containing t lies inside it, i.e. iff
//   max over i in [t-w, t] of cpl(k[i], k[i+w]) >= L.
// So t starts a cell on level l0 (the parent run, level l0-1, is split) iff
// l0 = 0 or that window maximum of D reaches l0 - 1; it then starts the cells
// of levels lo = l0 .. hi = max(l0, min(D(t) + 1, 21)), the one at hi a leaf.
// Its group (the cells with <= ncrit bodies whose parent has more) sits on
// level lg = max(l0, DG(t) + 1) if lg <= hi and t starts it (lg > l0, l0 = 0,
// or the window maximum of DG reaches l0 - 1); if lg > hi the leaf has more
// than ncrit bodies (identical keys at level 21, or ncrit < nleaf) and is cut
// into runs of ncrit.  Both window maxima come from a sparse table of
// pairwise maxima (log2(w+1) + 1 levels) in shared memory.
//
// The bodies that start cells (about one per leaf) are compacted, in key
// order, into the block's entry list: first body, leaf count (up to the next
// entry, which is the first body after the leaf), group body count and the
// levels.  Per block: cells per level (a difference array over lo..hi),
// groups, and entries.
constexpr int BH = 64;                              // halo: max(nleaf, ncrit)
constexpr int BB = BUILD_BODIES;                    // bodies per block (BUILD_BPT per thread)
constexpr int BTAB = BB + BH;                       // table positions [base - BH, base + BB)
constexpr int BKEYS = BB + 2 * BH + 1;              // keys of [base - BH - 1, base + BB + BH)

struct MarkShared {
    unsigned long long k[BKEYS];
    unsigned tab[2][BTAB];         // (D + 1) | (DG + 1) << 16, then maxima over 2^q positions
    unsigned e_t[BB];              // the block's entries: first body
    unsigned e_d[BB];              //   lo | hi << 8 | lg << 16 | kind << 24
    int cnt[MAX_LEVEL + 2];        // difference array of cells per level
    unsigned wcnt[BUILD_BPT][BUILD_THREADS / 32];
    unsigned ngrp, ne;
    uint8_t sy[BKEYS];
};

size_t build_mark_smem_bytes() { return sizeof(MarkShared); }

// End of the level-L run from body t (L >= 1), i.e. the first body after t
// whose key differs from k[t] above level L: a binary search over the
// block's keys and halo (the prefix shared with k[t] only shrinks along the
// sorted keys; positions past n or in another system share nothing), then
// the global search when the run reaches past the halo (identical keys at
// the deepest level).
__device__ __forceinline__ int run_end_local(const MarkShared &S, int k0, int base, int t, int L, int n,
                                             const unsigned long long *__restrict__ sk, int send) {
    const int last = base + BB + BH - 1;                     // last key in shared memory
    const unsigned long long kt = S.k[t - k0];
    const uint8_t st = S.sy[t - k0];
    auto inside = [&](int j) { return j < n && S.sy[j - k0] == st && key_cpl(kt, S.k[j - k0]) >= L; };
    if (last > t && inside(last)) return run_end(sk, send, t, L);
    int lo = t, hi = last;                                    // inside(lo), !inside(hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (inside(mid)) lo = mid; else hi = mid;
    }
    return hi;
}

// Maximum of the packed (16-bit) fields over table positions [it - w, it]
// from maxima over 2^q positions (w + 1 >= 2^q): overlapping lookups.
__device__ __forceinline__ unsigned window_max(const unsigned *T, int it, int w, int q) {
    const int h = 1 << q;
    unsigned m = T[it - h + 1];
    for (int a = it - w; a < it - h + 1; a += h) m = __vmaxu2(m, T[a]);
    return m;
}

__global__ void __launch_bounds__(BUILD_THREADS)
k_build_mark(const unsigned long long *__restrict__ sk, const uint8_t *__restrict__ sysid, int n, int nleaf,
             int ncrit, unsigned *blockcount, int nblocks, uint4 *entries, const DevState *__restrict__ st,
             bool multi) {
    extern __shared__ unsigned long long mark_smem[];
    MarkShared &S = *reinterpret_cast<MarkShared *>(mark_smem);
    if (st->status & ST_TIMEOUT) return;        // keys not sorted: skip the build
    const int base = blockIdx.x * BB, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = base - BH - 1;
    for (int i = tid; i < BKEYS; i += BUILD_THREADS) {
        const int j = k0 + i;
        const bool in = j >= 0 && j < n;
        S.k[i] = in ? sk[j] : 0ull;
        S.sy[i] = in ? sysid[j] : 0;
    }
    if (tid <= MAX_LEVEL + 1) S.cnt[tid] = 0;
    if (tid == 0) S.ngrp = 0u;
    __syncthreads();
    // with one system every body shares it: no system-id compare
    auto cpl = [&](int a, int b) {
        return multi ? body_cpl(S.k[a - k0], S.k[b - k0], S.sy[a - k0], S.sy[b - k0])
                     : key_cpl(S.k[a - k0], S.k[b - k0]);
    };
    for (int i = tid; i < BTAB; i += BUILD_THREADS) {
        const int j = base - BH + i;             // table position
        int d = -1, dg = -1;
        if (j >= 0 && j < n) {
            if (j + nleaf < n) d = cpl(j, j + nleaf);
            if (j + ncrit < n) dg = cpl(j, j + ncrit);
        }
        S.tab[0][i] = (unsigned)(d + 1) | ((unsigned)(dg + 1) << 16);
    }
    __syncthreads();

    // This thread's bodies t[h] = base + tid + h * BUILD_THREADS (h <
    // BUILD_BPT): own l0, D, DG, then the window maxima from maxima over 2^qb
    // positions, qb = floor(log2(min(nleaf, ncrit) + 1)) capped at 16 positions.
    int t[BUILD_BPT], l0[BUILD_BPT];
    unsigned own[BUILD_BPT];
#pragma unroll
    for (int h = 0; h < BUILD_BPT; h++) {
        t[h] = base + tid + h * BUILD_THREADS;
        own[h] = S.tab[0][t[h] - base + BH];
        l0[h] = (t[h] <= 0 || t[h] >= n) ? 0 : cpl(t[h] - 1, t[h]) + 1;
    }
    const int qb = min(4, 31 - __clz(min(nleaf, ncrit) + 1));
    int cur = 0;
    for (int q = 0; q < qb; q++) {               // uniform over the block
        const int hq = 1 << q;
        const unsigned *T = S.tab[cur];
        unsigned *U = S.tab[cur ^ 1];
        for (int i = tid; i + 2 * hq <= BTAB; i += BUILD_THREADS) U[i] = __vmaxu2(T[i], T[i + hq]);
        __syncthreads();
        cur ^= 1;
    }
    bool has[BUILD_BPT];
    unsigned desc[BUILD_BPT];
#pragma unroll
    for (int h = 0; h < BUILD_BPT; h++) {
        const int it = t[h] - base + BH;
        const int winD = (int)(window_max(S.tab[cur], it, nleaf, qb) & 0xffffu);   // 1 + max D
        has[h] = t[h] < n && l0[h] <= MAX_LEVEL && (l0[h] == 0 || winD >= l0[h]);
        desc[h] = 0u;
        if (has[h]) {
            const int D = (int)(own[h] & 0xffffu) - 1, DG = (int)(own[h] >> 16) - 1;
            const int hi = max(l0[h], min(D + 1, MAX_LEVEL));
            const int lg = max(l0[h], DG + 1);
            int kind = 2;
            if (lg <= hi) {
                const int winG = (int)(window_max(S.tab[cur], it, ncrit, qb) >> 16);   // 1 + max DG
                kind = (lg > l0[h] || l0[h] == 0 || winG >= l0[h]) ? 1 : 0;
            }
            desc[h] = (unsigned)l0[h] | ((unsigned)hi << 8) | ((unsigned)min(lg, 255) << 16) | ((unsigned)kind << 24);
        }
    }
    // compaction of the block's entries, in key order (slice h of the block's
    // bodies before slice h + 1)
    unsigned m[BUILD_BPT];
#pragma unroll
    for (int h = 0; h < BUILD_BPT; h++) {
        m[h] = __ballot_sync(0xffffffffu, has[h]);
        if (lane == 0) S.wcnt[h][warp] = __popc(m[h]);
    }
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = BUILD_THREADS / 32;
        unsigned carry = 0u;
#pragma unroll
        for (int h = 0; h < BUILD_BPT; h++) {
            const unsigned v = lane < NW ? S.wcnt[h][lane] : 0u;
            unsigned x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < NW) S.wcnt[h][lane] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) S.ne = carry;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < BUILD_BPT; h++) {
        if (has[h]) {
            const unsigned slot = S.wcnt[h][warp] + __popc(m[h] & ((1u << lane) - 1u));
            S.e_t[slot] = (unsigned)t[h];
            S.e_d[slot] = desc[h];
        }
    }
    __syncthreads();
    const unsigned ne = S.ne;
    for (unsigned e = (unsigned)tid; e < ne; e += BUILD_THREADS) {
        // A leaf ends where the next entry starts (the first body after a
        // leaf starts a cell); a group at level lg < hi ends at the first
        // later entry that starts on a level <= lg.  Only at the end of the
        // block's entries does a run end come from the keys.
        const unsigned et = S.e_t[e], ed = S.e_d[e];
        const int elo = (int)(ed & 0xffu), ehi = (int)((ed >> 8) & 0xffu), elg = (int)((ed >> 16) & 0xffu);
        const int kind = (int)(ed >> 24);
        const int send = system_end(st, sysid, (int)et, n);
        const int lend = e + 1 < ne ? (int)S.e_t[e + 1] : run_end_local(S, k0, base, (int)et, ehi, n, sk, send);
        const unsigned lcnt = (unsigned)lend - et;
        unsigned gcnt = 0u, ngrp = 0u;
        if (kind == 1) {
            if (elg == ehi) {
                gcnt = lcnt;
            } else {
                unsigned j = e + 1;
                while (j < ne && (S.e_d[j] & 0xffu) > (unsigned)elg) j++;
                const int gend = j < ne ? (int)S.e_t[j] : run_end_local(S, k0, base, (int)et, elg, n, sk, send);
                gcnt = (unsigned)gend - et;
            }
            ngrp = 1u;
        } else if (kind == 2) {
            gcnt = lcnt;
            ngrp = (lcnt + (unsigned)ncrit - 1u) / (unsigned)ncrit;
        }
        entries[(size_t)blockIdx.x * BB + e] = make_uint4(et, lcnt, gcnt, ed);
        atomicAdd(&S.cnt[elo], 1);
        atomicSub(&S.cnt[ehi + 1], 1);
        if (ngrp) atomicAdd(&S.ngrp, ngrp);
    }
    __syncthreads();
    if (warp == 0) {                             // cells per level: prefix of the difference array
        int x = lane <= MAX_LEVEL ? S.cnt[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane <= MAX_LEVEL) blockcount[(size_t)lane * nblocks + blockIdx.x] = (unsigned)x;
        if (lane == 0) {
            blockcount[(size_t)GROUP_ROW * nblocks + blockIdx.x] = S.ngrp;
            blockcount[(size_t)ENTRY_ROW * nblocks + blockIdx.x] = ne;
        }
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

// Pass 3 (over the entries of each body block): number every cell and write
// its first body, level and link.  The cell of level r started by entry t
// has index level_start[r] + (cells of level r started before t); it also
// records cb = the number of level-(r+1) cells that start before t, offset to
// level r+1's first index: for an internal cell that is its first child, and
// the children of a cell are the level-(r+1) cells between its cb and the
// next cell's cb.  Leaves get their body count here.
constexpr int WRITE_THREADS = 512;

__global__ void __launch_bounds__(WRITE_THREADS)
k_build_write(const uint4 *__restrict__ entries, int ncrit, const unsigned *__restrict__ blockcount, int nblocks,
              long long ccap, DevState *st, uint2 *cell_body, uint2 *cell_link, uint8_t *cell_level,
              uint32_t *cell_parent, uint32_t *cell_cb, uint2 *groups, uint8_t *group_lvl) {
    constexpr int NW = WRITE_THREADS / 32;
    __shared__ unsigned s_wc[NROWS][NW];
    __shared__ unsigned s_base[NROWS];
    __shared__ unsigned s_tot[NROWS];
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
                // over capacity (cannot happen for the arena's bound, kept as
                // a guard): no cells and no groups, so that every later
                // stage does nothing, and the error is reported
                st->ncells = s_ok ? run : 0u;
                st->ngroups = s_ok ? st->row_total[GROUP_ROW] : 0u;
                if (!s_ok) atomicOr(&st->status, ST_CAPACITY);
            }
        }
    }
    __syncthreads();
    if (!s_ok) return;
    const unsigned ne = blockcount[(size_t)ENTRY_ROW * nblocks + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    for (unsigned r0 = 0; r0 < ne; r0 += WRITE_THREADS) {   // rounds of entries (uniform)
        const unsigned i = r0 + (unsigned)tid;
        const bool valid = i < ne;
        const uint4 e = valid ? entries[(size_t)blockIdx.x * BB + i] : make_uint4(0u, 0u, 0u, 0u);
        const int lo = valid ? (int)(e.w & 0xffu) : MAX_LEVEL + 1;
        const int hi = valid ? (int)((e.w >> 8) & 0xffu) : -1;
        const int lg = (int)((e.w >> 16) & 0xffu), kind = (int)(e.w >> 24);
        const unsigned t = e.x;
        const unsigned ngrp = kind == 1 ? 1u : kind == 2 ? (e.z + (unsigned)ncrit - 1u) / (unsigned)ncrit : 0u;
        const int rlo = (int)__reduce_min_sync(0xffffffffu, (unsigned)lo);
        const int rhi = (int)__reduce_max_sync(0xffffffffu, (unsigned)(hi + 1)) - 1;   // -1: no entry
        if (lane <= MAX_LEVEL && (lane < rlo || lane > rhi)) s_wc[lane][warp] = 0u;
        for (int r = rlo; r <= rhi; r++) {
            const unsigned mm = __ballot_sync(0xffffffffu, lo <= r && r <= hi);
            if (lane == 0) s_wc[r][warp] = __popc(mm);
        }
        unsigned gx = ngrp;                      // inclusive warp scan of group counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, gx, o);
            if (lane >= o) gx += y;
        }
        if (lane == 31) s_wc[GROUP_ROW][warp] = gx;
        gx -= ngrp;
        __syncthreads();
        for (int row = warp; row < NROWS; row += NW) {   // exclusive prefix across warps per row
            const unsigned v = lane < NW ? s_wc[row][lane] : 0u;
            unsigned x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < NW) s_wc[row][lane] = x - v;
            if (lane == NW - 1) s_tot[row] = x;
        }
        __syncthreads();
        unsigned bcur = rlo <= rhi ? __ballot_sync(0xffffffffu, lo <= rlo && rlo <= hi) : 0u;
        for (int r = rlo; r <= rhi; r++) {
            const unsigned bnext = r < MAX_LEVEL ? __ballot_sync(0xffffffffu, lo <= r + 1 && r + 1 <= hi) : 0u;
            if (lo <= r && r <= hi) {
                const unsigned c = s_base[r] + s_wc[r][warp] + __popc(bcur & lt);
                const unsigned cb = r < MAX_LEVEL ? s_base[r + 1] + s_wc[r + 1][warp] + __popc(bnext & lt) : 0u;
                cell_cb[c] = cb;
                cell_level[c] = (uint8_t)r;
                if (r == 0) cell_parent[c] = 0xffffffffu;
                if (r == hi) {
                    cell_body[c] = make_uint2(t, e.y);
                    cell_link[c] = make_uint2(t, e.y | LEAF_BIT);
                } else {
                    cell_body[c] = make_uint2(t, 0u);
                    cell_link[c] = make_uint2(cb, 0u);
                }
            }
            bcur = bnext;
        }
        if (ngrp) {                              // groups in key order
            const unsigned g = s_base[GROUP_ROW] + s_wc[GROUP_ROW][warp] + gx;
            if (kind == 1) {
                groups[g] = make_uint2(t, e.z);
                if (group_lvl) group_lvl[g] = (uint8_t)lg;
            } else {
                for (unsigned k = 0; k < ngrp; k++) {
                    const unsigned b0 = t + k * (unsigned)ncrit;
                    groups[g + k] = make_uint2(b0, min((unsigned)ncrit, e.z - k * (unsigned)ncrit));
                    if (group_lvl) group_lvl[g + k] = 0xffu;
                }
            }
        }
        __syncthreads();                         // s_wc is rebuilt by the next round
        if (tid < NROWS) s_base[tid] += s_tot[tid];
        __syncthreads();
    }
}

// Child count and the children's parent of internal cell c: the children
// are the level-(l+1) cells from cb(c) up to the cb of the next cell of level
// l (or the end of level l+1).
__device__ __forceinline__ unsigned child_count(unsigned d, int l, const DevState *__restrict__ st,
                                                const uint32_t *__restrict__ cell_cb) {
    const unsigned next = (d + 1 < st->level_start[l + 1]) ? cell_cb[d + 1] : st->level_start[l + 2];
    return next - cell_cb[d];
}

// Pass 4 (grid-stride over the cells, internal cells only): child count
// and parent pointers of the children.
__global__ void k_build_link(const DevState *__restrict__ st, const uint32_t *__restrict__ cell_cb,
                             const uint8_t *__restrict__ cell_level, uint2 *cell_link, uint32_t *cell_parent) {
    if (st->status & ST_TIMEOUT) return;
    const unsigned ncells = st->ncells;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        if (cell_link[c].y & LEAF_BIT) continue;
        const unsigned cb = cell_cb[c], nch = child_count(c, cell_level[c], st, cell_cb);
        cell_link[c] = make_uint2(cb, nch);
        for (unsigned k = 0; k < nch; k++) cell_parent[cb + k] = c;
    }
}

// Body counts of the internal cells, which no stage of a step reads (the
// walk and the multipoles take leaves' body ranges and internal cells' child
// ranges from the links): filled on demand for the tree getter.  A cell ends
// where its last descendant leaf ends: descend along last children (at most
// 21 levels).
__global__ void k_internal_counts(const DevState *__restrict__ st, const uint2 *__restrict__ cell_link,
                                  uint2 *cell_body) {
    const unsigned ncells = st->ncells;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        uint2 lk = cell_link[c];
        if (lk.y & LEAF_BIT) continue;
        unsigned d = lk.x + lk.y - 1;            // last child, then its last child, ...
        lk = cell_link[d];
        for (int it = 0; it < MAX_LEVEL && !(lk.y & LEAF_BIT); it++) {
            d = lk.x + lk.y - 1;
            lk = cell_link[d];
        }
        cell_body[c].y = lk.x + (lk.y & ~LEAF_BIT) - cell_body[c].x;
    }
}

cudaError_t launch_internal_counts(Ctx &c) {
    const unsigned grid = (unsigned)min((c.ccap + 255) / 256, (long long)c.num_sms * 8);
    k_internal_counts<<<grid, 256, 0, c.stream>>>(c.st, c.cell_link, c.cell_body);
    return cudaGetLastError();
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
    // The chunk's groups and the 8 before it in shared memory, each with
    // whether it is a sibling of the one before: every thread's look-back
    // and greedy pass then run on shared memory (one round of global loads
    // per chunk instead of one per step back).
    constexpr int HALO = 8;
    __shared__ unsigned s_cnt[PACK_THREADS + HALO];
    __shared__ uint8_t s_sib[PACK_THREADS + HALO];
    if ((st->status & ST_TIMEOUT) || st->ncells == 0u) return;   // keys unsorted, or no tree
    const unsigned ng = st->row_total[GROUP_ROW];
    const unsigned nchunk = (ng + PACK_THREADS - 1) / PACK_THREADS;
    for (unsigned ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const long long g0 = (long long)ch * PACK_THREADS - HALO;
        for (int i = threadIdx.x; i < PACK_THREADS + HALO; i += PACK_THREADS) {
            const long long gg = g0 + i;
            const bool valid = gg >= 0 && gg < (long long)ng;
            s_cnt[i] = valid ? graw[gg].y : 0u;
            s_sib[i] = valid && group_sibling((unsigned)gg, graw, glvl, sk, sysid) ? 1u : 0u;
        }
        __syncthreads();
        const unsigned g = ch * PACK_THREADS + threadIdx.x;
        bool start = false;
        if (g < ng) {
            int s = (int)threadIdx.x + HALO;
            for (int k = 0; k < 8 && s_sib[s]; k++) s--;
            unsigned acc = s_cnt[s];
            start = true;
            for (int j = s + 1; j <= (int)threadIdx.x + HALO; j++) {
                const unsigned cj = s_cnt[j];
                start = acc + cj > (unsigned)ncrit;
                acc = start ? cj : acc + cj;
            }
            gflag[g] = start ? 1u : 0u;
        }
        const int cnt = __syncthreads_count(start);   // also: the shared arrays are free again
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
    if ((st->status & ST_TIMEOUT) || st->ncells == 0u) return;   // keys unsorted, or no tree
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
    static size_t attr_done[MAX_DEVICES] = {};
    cudaError_t e = allow_dyn_smem((const void *)k_build_mark, sizeof(MarkShared), attr_done);
    if (e != cudaSuccess) return e;
    k_build_mark<<<c.nbblocks, BUILD_THREADS, sizeof(MarkShared), c.stream>>>(
        c.keys, c.sysid, n, c.nleaf, c.ncrit, c.blockcount, c.nbblocks, c.build_entries, c.st, c.nsys > 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_build_scan<<<NROWS, 1024, 0, c.stream>>>(c.blockcount, c.nbblocks, c.st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool pack = c.group_pack != 0;
    k_build_write<<<c.nbblocks, WRITE_THREADS, 0, c.stream>>>(
        c.build_entries, c.ncrit, c.blockcount, c.nbblocks, c.ccap, c.st, c.cell_body, c.cell_link, c.cell_level,
        c.cell_parent, c.cell_cb, pack ? c.groups_raw : c.groups, pack ? c.group_lvl : nullptr);
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
    k_build_link<<<grid, 256, 0, c.stream>>>(c.st, c.cell_cb, c.cell_level, c.cell_link, c.cell_parent);
    return cudaGetLastError();
}

}  // namespace bonsai
