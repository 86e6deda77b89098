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
// l = l0(t) it does iff some window [j, j+nleaf] around t stays inside it:
//   E(t) = max_{t-nleaf <= j <= t} D(j) >= l0(t) - 1.
// So body t starts exactly the cells of levels lo..hi with lo = l0(t) (if
// E(t)) and hi = max(lo, min(D(t)+1, 21)); the one at hi is a leaf.  Groups
// (cells with <= ncrit bodies whose parent has more) follow the same way with
// ncrit in place of nleaf.  Three launches: count per block and level, scan
// per level, write cells.
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

// Shared memory of a build block: keys [base-W, base+B+W) and, for
// j in [base-W, base+B), D(j) = cpl(k[j], k[j+nleaf]) and DG(j) with ncrit
// (-1 where j+w is past the end).
struct BuildShared {
    unsigned long long *k;
    int *D, *DG, *TD, *TG;   // TD/TG: maxima of D/DG over [j, j + HD/HG)
    uint8_t *sy;
    int W, base, nleaf, ncrit, HD, HG;
    __device__ unsigned long long key(int j) const { return k[j - base + W]; }
    __device__ uint8_t sys(int j) const { return sy[j - base + W]; }
    __device__ int cpl(int a, int b) const { return body_cpl(key(a), key(b), sys(a), sys(b)); }
    __device__ int d(int j) const { return D[j - base + W]; }
    __device__ int dg(int j) const { return DG[j - base + W]; }
    // max D(j) over j in [t - nleaf, t] and max DG(j) over [t - ncrit, t]
    // (two overlapping power-of-two windows each)
    __device__ int dmax(int t) const { return max(TD[t - nleaf - base + W], TD[t - HD + 1 - base + W]); }
    __device__ int dgmax(int t) const { return max(TG[t - ncrit - base + W], TG[t - HG + 1 - base + W]); }
};

__device__ __forceinline__ int pow2_floor(int x) { return 1 << (31 - __clz(x)); }

// Keys and system ids of [base-W, base+B+W); D and DG of [base-W, base+B).
// Bodies of different systems share no level (cpl -1), so each system gets
// its own root on level 0.
__device__ BuildShared load_build_shared(void *smem, const unsigned long long *__restrict__ sk,
                                         const uint8_t *__restrict__ sysid, int n, int base,
                                         int nleaf, int ncrit) {
    BuildShared b;
    b.W = max(nleaf, ncrit);
    b.base = base;
    b.nleaf = nleaf;
    b.ncrit = ncrit;
    b.HD = pow2_floor(nleaf + 1);
    b.HG = pow2_floor(ncrit + 1);
    const int m = BUILD_THREADS + b.W;
    b.k = (unsigned long long *)smem;
    b.D = (int *)(b.k + BUILD_THREADS + 2 * b.W);
    b.DG = b.D + m;
    b.TD = b.DG + m;
    b.TG = b.TD + m;
    b.sy = (uint8_t *)(b.TG + m);
    for (int i = threadIdx.x; i < BUILD_THREADS + 2 * b.W; i += blockDim.x) {
        int j = base - b.W + i;
        const bool in = j >= 0 && j < n;
        b.k[i] = in ? sk[j] : 0ull;
        b.sy[i] = in ? sysid[j] : 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int j = base - b.W + i;
        b.D[i] = b.TD[i] = (j >= 0 && j + nleaf < n) ? b.cpl(j, j + nleaf) : -1;
        b.DG[i] = b.TG[i] = (j >= 0 && j + ncrit < n) ? b.cpl(j, j + ncrit) : -1;
    }
    __syncthreads();
    // Doubling: after the step with width h, T[i] = max over [i, i + 2h).
    // Entries whose window runs past the array keep a truncated maximum;
    // dmax/dgmax never read them.
    for (int h = 1; 2 * h <= b.HG; h <<= 1) {
        int nd[2], ng[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int i = threadIdx.x + r * BUILD_THREADS;
            nd[r] = ng[r] = 0;
            if (i < m) {
                nd[r] = (2 * h <= b.HD && i + h < m) ? max(b.TD[i], b.TD[i + h]) : b.TD[i];
                ng[r] = i + h < m ? max(b.TG[i], b.TG[i + h]) : b.TG[i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int i = threadIdx.x + r * BUILD_THREADS;
            if (i < m) { b.TD[i] = nd[r]; b.TG[i] = ng[r]; }
        }
        __syncthreads();
    }
    for (int h = b.HG; 2 * h <= b.HD; h <<= 1) {      // nleaf > ncrit: finish TD
        int nd[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int i = threadIdx.x + r * BUILD_THREADS;
            nd[r] = (i < m && i + h < m) ? max(b.TD[i], b.TD[i + h]) : (i < m ? b.TD[i] : 0);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int i = threadIdx.x + r * BUILD_THREADS;
            if (i < m) b.TD[i] = nd[r];
        }
        __syncthreads();
    }
    return b;
}

// run_end for a body t of the block, from the keys held in shared memory
// (indices below lim = min(send, base + BUILD_THREADS + W)); falls back to
// the global search only when the run reaches the end of that window.
// Leaf and group runs (<= nleaf, <= ncrit bodies) always end inside it.
__device__ int run_end_win(const BuildShared &b, const unsigned long long *__restrict__ sk, int send, int t,
                           int level) {
    if (level == 0) return send;
    const int sh = 3 * (MAX_LEVEL - level);
    const unsigned long long pre = b.key(t) >> sh;
    const int lim = min(send, b.base + BUILD_THREADS + b.W);
    const int last = lim - 1;
    if ((b.key(last) >> sh) == pre) return lim == send ? send : run_end(sk, send, last, level);
    int lo = t, hi = last, step = 1;          // key(lo) in the run, key(hi) not
    while (t + step < hi) {
        if ((b.key(t + step) >> sh) != pre) { hi = t + step; break; }
        lo = t + step;
        step <<= 1;
    }
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if ((b.key(mid) >> sh) == pre) lo = mid; else hi = mid;
    }
    return hi;
}

size_t build_smem_bytes(int nleaf, int ncrit) {
    int W = nleaf > ncrit ? nleaf : ncrit;
    return (size_t)(BUILD_THREADS + 2 * W) * 8 + 4 * (size_t)(BUILD_THREADS + W) * 4 +
           (size_t)(BUILD_THREADS + 2 * W);
}

// Which cells body t starts (levels lo..hi) and how many groups; send is the
// end of t's system.
__device__ BodyCells analyse_body(const BuildShared &b, int t, int n, int nleaf, int ncrit,
                                  const unsigned long long *__restrict__ sk, int send) {
    BodyCells r{false, 0, -1, 0, 0};
    if (t >= n) return r;
    int l0 = (t == 0) ? 0 : b.cpl(t - 1, t) + 1;
    if (l0 > MAX_LEVEL) return r;
    if (l0 > 0 && b.dmax(t) < l0 - 1) return r;
    r.has = true;
    r.lo = l0;
    r.hi = max(l0, min(b.d(t) + 1, MAX_LEVEL));
    int lg = max(l0, b.dg(t) + 1);
    r.lg = lg;
    if (lg <= r.hi) {
        const bool starts = (lg > l0) || l0 == 0 || b.dgmax(t) >= l0 - 1;
        r.ngrp = starts ? 1 : 0;
    } else {
        int cnt = run_end_win(b, sk, send, t, r.hi) - t;
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
    BuildShared b = load_build_shared(smem_u64, sk, sysid, n, base, nleaf, ncrit);
    const int t = base + tid;
    BodyCells bc = analyse_body(b, t, n, nleaf, ncrit, sk, system_end(st, sysid, t, n));
    int rlo, rhi;
    warp_level_range(bc, rlo, rhi);
    for (int r = 0; r <= MAX_LEVEL; r++) {
        unsigned m = (r >= rlo && r <= rhi) ? __ballot_sync(0xffffffffu, has_level(bc, r)) : 0u;
        if (lane == 0) s_wc[r][warp] = __popc(m);
    }
    int g = bc.ngrp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (lane == 0) s_wc[GROUP_ROW][warp] = (unsigned)g;
    __syncthreads();
    if (tid < NROWS) {
        unsigned s = 0;
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
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_write(const unsigned long long *__restrict__ sk, const uint8_t *__restrict__ sysid, int n,
              int nleaf, int ncrit, const unsigned *__restrict__ blockcount, int nblocks, long long ccap,
              DevState *st,
              uint2 *cell_body, uint2 *cell_link, uint8_t *cell_level, uint32_t *cell_parent,
              uint32_t *cell_done, uint32_t *cell_cb, uint2 *groups) {
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
    BuildShared b = load_build_shared(smem_u64, sk, sysid, n, base, nleaf, ncrit);
    const int t = base + tid;
    const int send = system_end(st, sysid, t, n);
    BodyCells bc = analyse_body(b, t, n, nleaf, ncrit, sk, send);
    const unsigned lt = (1u << lane) - 1u;
    int rlo, rhi;
    warp_level_range(bc, rlo, rhi);

    for (int r = 0; r <= MAX_LEVEL; r++) {
        unsigned m = (r >= rlo && r <= rhi) ? __ballot_sync(0xffffffffu, has_level(bc, r)) : 0u;
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
    if (warp < NROWS) {                          // exclusive prefix across warps per row
        unsigned v = s_wc[warp][lane], x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncwarp();
        s_wc[warp][lane] = x - v;
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
                int cnt = run_end_win(b, sk, send, t, r) - t;
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
            int e = run_end_win(b, sk, send, t, bc.lg);
            groups[g] = make_uint2((unsigned)t, (unsigned)(e - t));
        } else {
            int e = run_end_win(b, sk, send, t, bc.hi);
            for (int k = 0; k < bc.ngrp; k++) {
                int b0 = t + k * ncrit;
                groups[g + k] = make_uint2((unsigned)b0, (unsigned)min(ncrit, e - b0));
            }
        }
    }
}

// Pass 4 (one thread per internal cell): child count from the cb of the next
// cell of the same level, parent pointers of the children, and the body
// count from the descent along last children to a leaf.
__global__ void k_build_link(const DevState *__restrict__ st, const uint32_t *__restrict__ cell_cb,
                             const uint8_t *__restrict__ cell_level, uint2 *cell_link,
                             uint2 *cell_body, uint32_t *cell_parent) {
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st->ncells || (st->status & ST_TIMEOUT)) return;
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
    k_build_write<<<c.nbblocks, BUILD_THREADS, smem, c.stream>>>(
        c.keys, c.sysid, n, c.nleaf, c.ncrit, c.blockcount, c.nbblocks, c.ccap, c.st, c.cell_body,
        c.cell_link, c.cell_level, c.cell_parent, c.cell_done, c.cell_cb, c.groups);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unsigned grid = (unsigned)((c.ccap + 255) / 256);
    k_build_link<<<grid, 256, 0, c.stream>>>(c.st, c.cell_cb, c.cell_level, c.cell_link, c.cell_body,
                                             c.cell_parent);
    return cudaGetLastError();
}

}  // namespace bonsai
