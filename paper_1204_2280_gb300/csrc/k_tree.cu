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

// First index > t whose level-`level` key prefix differs from k[t] (or n):
// galloping then bisection.
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

// Number of distinct level-(l+1) octants among sorted keys sk[b..e) that
// share their level-l prefix.
__device__ int count_children(const unsigned long long *__restrict__ sk, int b, int e, int l) {
    unsigned d0 = digit_at(sk[b], l + 1), d1 = digit_at(sk[e - 1], l + 1);
    int nch = 1, pos = b;
    for (unsigned o = d0 + 1; o <= d1; o++) {
        int lo = pos, hi = e;                 // first index with digit >= o
        while (lo < hi) {
            int mid = lo + ((hi - lo) >> 1);
            if (digit_at(sk[mid], l + 1) < o) lo = mid + 1; else hi = mid;
        }
        if (lo < e && digit_at(sk[lo], l + 1) == o) nch++;
        pos = lo;
    }
    return nch;
}

struct BodyCells {
    bool has;
    int lo, hi, ngrp, lg;   // lg: group level (>hi: oversize leaf cut in chunks)
};

// Per-body analysis shared by the count and write kernels.  s_k holds keys
// [base - W, base + BUILD_THREADS + W); keys outside [0, n) are never read.
__device__ BodyCells analyse_body(const unsigned long long *s_k, int W, int base, int t, int n,
                                  int nleaf, int ncrit, const unsigned long long *__restrict__ sk) {
    BodyCells r{false, 0, -1, 0, 0};
    if (t >= n) return r;
    auto K = [&](int j) { return s_k[j - base + W]; };
    int l0 = (t == 0) ? 0 : key_cpl(K(t - 1), K(t)) + 1;
    if (l0 > MAX_LEVEL) return r;
    auto D = [&](int j, int w) { return (j >= 0 && j + w < n) ? key_cpl(K(j), K(j + w)) : -1; };
    if (l0 > 0) {
        int e = -1;
        for (int j = max(0, t - nleaf); j <= t; j++) e = max(e, D(j, nleaf));
        if (e < l0 - 1) return r;
    }
    r.has = true;
    r.lo = l0;
    r.hi = max(l0, min(D(t, nleaf) + 1, MAX_LEVEL));
    int lg = max(l0, D(t, ncrit) + 1);
    r.lg = lg;
    if (lg <= r.hi) {
        bool starts = (lg > l0) || l0 == 0;
        if (!starts) {
            int e = -1;
            for (int j = max(0, t - ncrit); j <= t; j++) e = max(e, D(j, ncrit));
            starts = e >= l0 - 1;
        }
        r.ngrp = starts ? 1 : 0;
    } else {
        int cnt = run_end(sk, n, t, r.hi) - t;
        r.ngrp = (cnt + ncrit - 1) / ncrit;
    }
    return r;
}

__device__ void load_key_window(unsigned long long *s_k, const unsigned long long *__restrict__ sk,
                                int n, int base, int W) {
    for (int i = threadIdx.x; i < BUILD_THREADS + 2 * W; i += blockDim.x) {
        int j = base - W + i;
        s_k[i] = (j >= 0 && j < n) ? sk[j] : 0ull;
    }
}

// Pass 1: per block, the number of cells of each level and of groups.
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_count(const unsigned long long *__restrict__ sk, int n, int nleaf, int ncrit,
              unsigned *blockcount, int nblocks, const DevState *__restrict__ st) {
    extern __shared__ unsigned long long s_k[];
    if (st->status & ST_TIMEOUT) return;        // keys not sorted: skip the build
    __shared__ unsigned s_wc[NROWS][32];
    const int W = max(nleaf, ncrit);
    const int base = blockIdx.x * BUILD_THREADS, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    load_key_window(s_k, sk, n, base, W);
    __syncthreads();
    BodyCells bc = analyse_body(s_k, W, base, base + tid, n, nleaf, ncrit, sk);
    for (int r = 0; r <= MAX_LEVEL; r++) {
        unsigned b = __ballot_sync(0xffffffffu, bc.has && bc.lo <= r && r <= bc.hi);
        if (lane == 0) s_wc[r][warp] = __popc(b);
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

// Pass 3: write every cell, its children links and parent pointers, and the
// groups.
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_write(const unsigned long long *__restrict__ sk, int n, int nleaf, int ncrit,
              const unsigned *__restrict__ blockcount, int nblocks, long long ccap, DevState *st,
              uint2 *cell_body, uint2 *cell_link, uint8_t *cell_level, uint32_t *cell_parent,
              uint32_t *cell_done, uint2 *groups) {
    extern __shared__ unsigned long long s_k[];
    __shared__ unsigned s_wc[NROWS][32];
    __shared__ unsigned s_base[NROWS];
    __shared__ int s_ok;
    const int W = max(nleaf, ncrit);
    const int base = blockIdx.x * BUILD_THREADS, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (st->status & ST_TIMEOUT) return;        // keys not sorted: skip the build
    load_key_window(s_k, sk, n, base, W);
    if (tid == 0) {
        unsigned run = 0;
        for (int r = 0; r <= MAX_LEVEL; r++) {
            s_base[r] = run + blockcount[(size_t)r * nblocks + blockIdx.x];
            run += st->row_total[r];
        }
        s_base[GROUP_ROW] = blockcount[(size_t)GROUP_ROW * nblocks + blockIdx.x];
        s_ok = (long long)run <= ccap;
        if (blockIdx.x == 0) {
            st->ncells = run;
            st->ngroups = st->row_total[GROUP_ROW];
            if (!s_ok) atomicOr(&st->status, ST_CAPACITY);
        }
    }
    __syncthreads();
    if (!s_ok) return;
    const int t = base + tid;
    BodyCells bc = analyse_body(s_k, W, base, t, n, nleaf, ncrit, sk);
    const unsigned lt = (1u << lane) - 1u;

    // Warp-level counts per row, then exclusive prefix across warps.
    for (int r = 0; r <= MAX_LEVEL; r++) {
        unsigned b = __ballot_sync(0xffffffffu, bc.has && bc.lo <= r && r <= bc.hi);
        if (lane == 0) s_wc[r][warp] = __popc(b);
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
    if (warp < NROWS) {
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

    // Cells of this body, level by level (warp-uniform loop for the ballots).
    unsigned prev_c = 0;
    int prev_nch = 0;
    for (int r = 0; r <= MAX_LEVEL; r++) {
        bool mine = bc.has && bc.lo <= r && r <= bc.hi;
        unsigned b = __ballot_sync(0xffffffffu, mine);
        if (!mine) continue;
        unsigned c = s_base[r] + s_wc[r][warp] + __popc(b & lt);
        if (r > bc.lo) {                         // link the parent made at r-1
            cell_link[prev_c] = make_uint2(c, (unsigned)prev_nch);
            for (int k = 0; k < prev_nch; k++) cell_parent[c + k] = prev_c;
        }
        int e = run_end(sk, n, t, r);
        int cnt = e - t;
        cell_body[c] = make_uint2((unsigned)t, (unsigned)cnt);
        cell_level[c] = (uint8_t)r;
        cell_done[c] = 0u;
        if (r == 0) cell_parent[c] = 0xffffffffu;
        if (r == bc.hi) {
            cell_link[c] = make_uint2((unsigned)t, (unsigned)cnt | LEAF_BIT);
        } else {
            prev_nch = count_children(sk, t, e, r);
        }
        prev_c = c;
    }
    // Groups in key order.
    if (bc.ngrp > 0) {
        unsigned g = s_base[GROUP_ROW] + s_wc[GROUP_ROW][warp] + (unsigned)gx;
        if (bc.lg <= bc.hi) {
            int e = run_end(sk, n, t, bc.lg);
            groups[g] = make_uint2((unsigned)t, (unsigned)(e - t));
        } else {
            int e = run_end(sk, n, t, bc.hi);
            for (int k = 0; k < bc.ngrp; k++) {
                int b0 = t + k * ncrit;
                groups[g + k] = make_uint2((unsigned)b0, (unsigned)min(ncrit, e - b0));
            }
        }
    }
}

cudaError_t launch_build(Ctx &c) {
    int n = (int)c.n;
    int W = c.nleaf > c.ncrit ? c.nleaf : c.ncrit;
    size_t smem = (size_t)(BUILD_THREADS + 2 * W) * sizeof(unsigned long long);
    k_build_count<<<c.nbblocks, BUILD_THREADS, smem, c.stream>>>(c.keys, n, c.nleaf, c.ncrit,
                                                                 c.blockcount, c.nbblocks, c.st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_build_scan<<<NROWS, 1024, 0, c.stream>>>(c.blockcount, c.nbblocks, c.st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_build_write<<<c.nbblocks, BUILD_THREADS, smem, c.stream>>>(
        c.keys, n, c.nleaf, c.ncrit, c.blockcount, c.nbblocks, c.ccap, c.st, c.cell_body,
        c.cell_link, c.cell_level, c.cell_parent, c.cell_done, c.groups);
    return cudaGetLastError();
}

}  // namespace bonsai
