// k_sort.cu -- stable LSD radix sort of (63-bit Morton key, u32 index).
//
// Paper Sect. 2, "sorting": bodies are ordered along the space-filling curve
// by their keys; equal keys keep their input order (stable).  Passes of
// SORT_BITS-bit digits (8 by default: eight passes) cover the 63 key bits.
// Each pass is one "onesweep" launch: the digit histograms of all passes
// come from the key kernel, so a pass reads every key/value once and writes
// it once (24 B per body per pass):
//   1. a tile of 4096 keys is taken in ticket order (atomic counter), loaded
//      warp-striped and ranked per warp: peers with equal digits by ballots,
//      counts by shared-memory atomics (stable: item order, then lane order,
//      then warp order);
//   2. per digit the tile count is published (each owner thread holds
//      SORT_DPT consecutive digits); the keys/values are reordered
//      by digit in shared memory (tile-local offsets only), which frees their
//      registers for the decoupled look-back that then finds the prefix over
//      earlier tiles (bounded spin; on timeout a status bit is set and the
//      kernel continues, so it always terminates);
//   3. the tile is written out so that consecutive threads write consecutive
//      addresses of a digit run.
#include "common.cuh"

namespace bonsai {

#ifndef SORT_LOOKBACK
#define SORT_LOOKBACK 8           // predecessor tiles read per look-back round trip (16: 3% slower at 2^20, 32: 9%)
#endif
#ifndef SORT_MIN_BLOCKS
#define SORT_MIN_BLOCKS 2         // resident onesweep blocks per SM the register budget allows
#endif

constexpr unsigned FLAG_AGG = 1u << 30;
constexpr unsigned FLAG_INC = 2u << 30;
constexpr unsigned VAL_MASK = (1u << 30) - 1u;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) {
    unsigned v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_volatile(unsigned *p, unsigned v) {
    asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exclusive scan over the threads of a block (one value per thread).
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *s_warp) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    unsigned off = 0;
#pragma unroll
    for (int w = 0; w < SORT_THREADS / 32; w++) off += (w < warp) ? s_warp[w] : 0u;
    __syncthreads();
    return off + x - v;
}

__global__ void __launch_bounds__(SORT_THREADS, SORT_MIN_BLOCKS)
k_onesweep(const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
           unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, int n, int shift,
           const unsigned *__restrict__ ghist, unsigned *status, unsigned *status_next,
           unsigned *ticket, int ntiles, DevState *st, long long max_spin,
           const uint8_t *__restrict__ dsrc) {
    constexpr unsigned R = SORT_RADIX, DMASK = SORT_RADIX - 1;
    extern __shared__ unsigned long long s_keys[];                 // SORT_TILE keys
    uint32_t *s_vals = (uint32_t *)(s_keys + SORT_TILE);          // SORT_TILE values
    __shared__ unsigned s_whist[SORT_THREADS / 32][SORT_RADIX];
    __shared__ unsigned s_dstart[SORT_RADIX], s_goff[SORT_RADIX], s_warp[SORT_THREADS / 32];
    __shared__ unsigned s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (status_next)
        for (int i = blockIdx.x * SORT_THREADS + tid; i < ntiles * (int)R; i += gridDim.x * SORT_THREADS)
            status_next[i] = 0u;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = tid; i < (SORT_THREADS / 32) * (int)R; i += SORT_THREADS) (&s_whist[0][0])[i] = 0u;
    __syncthreads();
    const int tile = (int)s_tile;
    const int wbase = tile * SORT_TILE + warp * (SORT_ITEMS * 32);

    unsigned long long k[SORT_ITEMS];
    uint32_t v[SORT_ITEMS];
    unsigned short rk[SORT_ITEMS];
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        int idx = wbase + it * 32 + lane;
        bool ok = idx < n;
        k[it] = ok ? kin[idx] : ~0ull;
        v[it] = vin ? (ok ? vin[idx] : 0u) : (uint32_t)idx;
    }
    // Digit of each item: SORT_BITS bits of the key, or (dsrc) the byte
    // dsrc[value], the system id of the body's pre-sort position.
    unsigned short dg[SORT_ITEMS];
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++)
        dg[it] = dsrc ? (unsigned short)(wbase + it * 32 + lane < n ? dsrc[v[it]] : 0)
                      : (unsigned short)((k[it] >> shift) & DMASK);
    // Rank within the warp: peers with the same digit by SORT_BITS ballots
    // (one __match_any_sync per item instead measured 28% slower per sort);
    // the lowest peer adds the peer count to the warp's digit counter with a
    // shared-memory atomic that returns the count before it.  A warp's
    // atomics execute in program order, so item order (then lane order) is
    // kept: stable.  All atomics are issued before the first result is used.
    const unsigned lt = lanemask_lt();
    unsigned pe[SORT_ITEMS], old[SORT_ITEMS];
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        const int idx = wbase + it * 32 + lane;
        const unsigned d = idx < n ? (unsigned)dg[it] : R;
        unsigned peers = __ballot_sync(0xffffffffu, d < R);
        if (d >= R) peers = ~peers;
#pragma unroll
        for (int bit = 0; bit < SORT_BITS; bit++) {
            const bool on = (d >> bit) & 1u;
            const unsigned bm = __ballot_sync(0xffffffffu, on);
            peers &= on ? bm : ~bm;
        }
        pe[it] = peers;
        old[it] = (d < R && (peers & lt) == 0u) ? atomicAdd(&s_whist[warp][d], (unsigned)__popc(peers)) : 0u;
    }
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        const unsigned base = __shfl_sync(0xffffffffu, old[it], __ffs(pe[it]) - 1);
        rk[it] = (unsigned short)(base + __popc(pe[it] & lt));
    }
    __syncthreads();

    // Thread t owns the SORT_DPT consecutive digits from d0 = t * SORT_DPT:
    // exclusive prefix over warps, tile counts, then block-wide digit starts.
    const unsigned d0 = (unsigned)tid * SORT_DPT;
    const bool owner = d0 < R;
    unsigned tcount[SORT_DPT], gh[SORT_DPT];
    unsigned tsum = 0, gsum = 0;
#pragma unroll
    for (int q = 0; q < SORT_DPT; q++) {
        unsigned run = 0;
        if (owner) {
#pragma unroll
            for (int w = 0; w < SORT_THREADS / 32; w++) {
                unsigned c = s_whist[w][d0 + q];
                s_whist[w][d0 + q] = run;
                run += c;
            }
        }
        tcount[q] = run;
        gh[q] = owner ? ghist[d0 + q] : 0u;
        tsum += run;
        gsum += gh[q];
    }
    const unsigned dstart0 = block_excl_scan(tsum, s_warp);
    const unsigned gbase0 = block_excl_scan(gsum, s_warp);
    // Testing aid (bonsai_debug_hold_sort_tile): a held tile publishes
    // nothing, so the look-back of the next tile runs into its bounded wait.
    // The positions a tile writes after giving up stay inside the output
    // (its prefix can only fall short of the true one).
    const bool held = st->hold_tile == (unsigned)tile + 1u;
    if (owner) {
        unsigned ds = dstart0;
#pragma unroll
        for (int q = 0; q < SORT_DPT; q++) {
            s_dstart[d0 + q] = ds;
            ds += tcount[q];
            // publish the tile's count first: later tiles look back meanwhile
            if (!held) st_volatile(status + (size_t)tile * R + d0 + q, (tile == 0 ? FLAG_INC : FLAG_AGG) | tcount[q]);
        }
    }
    __syncthreads();

    // Reorder the tile by digit in shared memory (needs only tile-local
    // offsets), so that the look-back below runs with the items' registers
    // free for more loads in flight.
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        int idx = wbase + it * 32 + lane;
        if (idx < n) {
            unsigned dd = dg[it];
            unsigned pos = s_dstart[dd] + s_whist[warp][dd] + rk[it];
            s_keys[pos] = k[it];
            s_vals[pos] = v[it];
        }
    }
    if (owner) {
        unsigned gb = gbase0;
#pragma unroll
        for (int q = 0; q < SORT_DPT; q++) {
            const unsigned d = d0 + q;
            // Decoupled look-back over earlier tiles for digit d.
            unsigned prefix = 0;
            if (tile > 0) {
                // Look back LB tiles per round trip (independent loads), then
                // consume them in order: aggregates are added, an inclusive
                // prefix ends the look-back, an unpublished tile is polled again.
                constexpr int LB = SORT_LOOKBACK;
                int j = tile - 1;
                long long spins = 0;
                bool found = false;
                while (!found) {
                    unsigned sv[LB];
#pragma unroll
                    for (int qq = 0; qq < LB; qq++)
                        sv[qq] = j - qq >= 0 ? ld_volatile(status + (size_t)(j - qq) * R + d) : FLAG_INC;
                    int qq = 0;
                    for (; qq < LB; qq++) {
                        const unsigned f = sv[qq] & ~VAL_MASK;
                        if (f == 0u) break;
                        prefix += sv[qq] & VAL_MASK;
                        if (f == FLAG_INC) { found = true; break; }
                    }
                    if (found) break;
                    if (qq == 0 && ++spins > max_spin) { atomicOr(&st->status, ST_TIMEOUT); break; }
                    j -= qq;
                }
                if (!held) st_volatile(status + (size_t)tile * R + d, FLAG_INC | ((prefix + tcount[q]) & VAL_MASK));
            }
            s_goff[d] = gb + prefix;
            gb += gh[q];
        }
    }
    __syncthreads();
    const int nvalid = min(SORT_TILE, n - tile * SORT_TILE);
    for (int p = tid; p < nvalid; p += SORT_THREADS) {
        unsigned long long key = s_keys[p];
        unsigned dd = dsrc ? (unsigned)dsrc[s_vals[p]] : (unsigned)((key >> shift) & DMASK);
        unsigned g = s_goff[dd] + ((unsigned)p - s_dstart[dd]);
        kout[g] = key;
        vout[g] = s_vals[p];
    }
}

constexpr size_t SORT_DYN_SMEM = (size_t)SORT_TILE * (sizeof(unsigned long long) + sizeof(uint32_t));
extern const size_t SORT_DYN_SMEM_BYTES = SORT_DYN_SMEM;

// SORT_PASSES passes over the key digits; with several systems one more
// stable pass on the system id groups the bodies by system (key order inside
// each).  Buffers alternate so that the result always lands in c.keys /
// c.vals (the key kernel writes to c.keys_alt for an odd number of passes).
cudaError_t launch_sort(Ctx &c) {
    static size_t attr_done[MAX_DEVICES] = {};
    cudaError_t ea = allow_dyn_smem((const void *)k_onesweep, SORT_DYN_SMEM, attr_done);
    if (ea != cudaSuccess) return ea;
    const int n = (int)c.n;
    const int npass = SORT_PASSES + (c.nsys > 1 ? 1 : 0);
    const int start = npass & 1;
    unsigned long long *kb[2] = {c.keys, c.keys_alt};
    uint32_t *vb[2] = {c.vals, c.vals_alt};
    const size_t plane = (size_t)c.ntiles * SORT_RADIX;
    for (int p = 0; p < npass; p++) {
        const int src = (p + start) & 1, dst = src ^ 1;
        k_onesweep<<<c.ntiles, SORT_THREADS, SORT_DYN_SMEM, c.stream>>>(
            kb[src], p == 0 ? nullptr : vb[src], kb[dst], vb[dst], n, p < SORT_PASSES ? SORT_BITS * p : 0,
            c.st->hist + SORT_RADIX * p,
            c.tile_status + plane * p, p + 1 < npass ? c.tile_status + plane * (p + 1) : nullptr,
            c.st->sort_tile + p, c.ntiles, c.st, c.max_spin, p == SORT_PASSES ? c.sysid : nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bonsai
