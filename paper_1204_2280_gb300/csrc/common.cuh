// common.cuh -- internal declarations of libbonsai (not part of the C ABI).
//
// Data layout in HBM (sorted body order unless stated):
//   pos4  float4[N]  (x, y, z, m)          vel4  float4[N] (vx, vy, vz, 0)
//   id    u32[N]     caller index          acc4  float4[N] (ax, ay, az, phi)
//   *_alt            the same, pre-sort copies written by pack / drift
//   keys  u64[N] + sort ping-pong buffers, perm u32[N]
//   cells (capacity C): body uint2 (begin, count), link uint2 (internal:
//     child_begin, nchild; leaf: begin, count | LEAF_BIT), level u8,
//     parent u32, done u32, mono float4 (com, M), quadA float4 (-Q: xx yy zz xy),
//     quadB float2 (-Q: xz yz), test float4 (com, r_open), delta float
//   groups (capacity N): uint2 (begin, count); with sibling packing the
//     unpacked groups (uint2), their levels (u8) and start flags (u8) too
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/bonsai.h"

namespace bonsai {

constexpr int KEY_BITS_PER_AXIS = 21;            // L, Sect. 2 Morton keys
constexpr int MAX_LEVEL = KEY_BITS_PER_AXIS;     // deepest level (root = 0)
constexpr int NROWS = MAX_LEVEL + 2;             // 22 level rows + group row
constexpr int GROUP_ROW = MAX_LEVEL + 1;
constexpr uint32_t LEAF_BIT = 0x80000000u;

#ifndef SORT_THREADS_CFG
#define SORT_THREADS_CFG 256
#endif
#ifndef SORT_ITEMS_CFG
#define SORT_ITEMS_CFG 16
#endif
#ifndef SORT_BITS_CFG
#define SORT_BITS_CFG 8
#endif
constexpr int SORT_THREADS = SORT_THREADS_CFG;          // >= 256 (a multiple of 32)
constexpr int SORT_ITEMS = SORT_ITEMS_CFG;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;   // 4096 keys per tile
constexpr int SORT_BITS = SORT_BITS_CFG;               // digit width of a radix pass
constexpr int SORT_RADIX = 1 << SORT_BITS;             // digit values (>= 256: the system-id pass)
constexpr int SORT_PASSES = (63 + SORT_BITS - 1) / SORT_BITS;   // passes over the 63-bit keys
constexpr int SORT_DPT = SORT_RADIX > SORT_THREADS ? SORT_RADIX / SORT_THREADS : 1;   // digits per owner thread
constexpr int MAX_SYSTEMS = 256;                       // ensemble: one more pass on the system id
constexpr int MLP_IN = 12, MLP_H = 64, MLP_OUT = 3;    // learned correction 12 -> 64 -> 64 -> 3
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;
constexpr int MLP_NNORM = 2 * MLP_IN + 1;              // mu[12], sigma[12], ysig
constexpr int FEAT_STRIDE = 12;                        // walk features per body
constexpr int JUDGE_MAX = 4096;                        // sampled bodies of the direct-sum judge
#ifndef JUDGE_SPLIT_CFG
#define JUDGE_SPLIT_CFG 128
#endif
constexpr int JUDGE_SPLIT = JUDGE_SPLIT_CFG;            // source splits of the judge's direct sum
#ifndef BUILD_THREADS_CFG
#define BUILD_THREADS_CFG 1024
#endif
constexpr int BUILD_THREADS = BUILD_THREADS_CFG;       // threads per build block (multiple of 32, <= 1024)
#ifndef BUILD_BPT_CFG
#define BUILD_BPT_CFG 4
#endif
constexpr int BUILD_BPT = BUILD_BPT_CFG;               // bodies per thread of the build's analysis pass
constexpr int BUILD_BODIES = BUILD_BPT * BUILD_THREADS;   // bodies per build block
constexpr int PACK_THREADS = 1024;                     // unpacked groups per group-packing block
constexpr long long STAGE_MIN_FLOATS = 4096;           // staging area floor (getters stream cells through it)
constexpr int ENTRY_ROW = NROWS;                       // build: entries per block (a row that is not scanned)
constexpr int BUILD_ROWS = NROWS + 1;                  // build: per-block count rows

// Device status bits (ORed by kernels, read and cleared by bonsai_sync).
constexpr unsigned ST_CAPACITY = 1u;
constexpr unsigned ST_TIMEOUT = 2u;
constexpr unsigned ST_NAN = 4u;

struct DevState {
    int dom[6 * MAX_SYSTEMS];         // per system: orderable-int min xyz, max xyz
    float mn[3 * MAX_SYSTEMS];        // per system: domain corner
    float side[MAX_SYSTEMS];          // per system: domain side S
    float scale[MAX_SYSTEMS];         // per system: 2^21 / S
    unsigned sys_off[MAX_SYSTEMS + 1];    // first body of each system (+ n)
    unsigned hist[(SORT_PASSES + 1) * SORT_RADIX]; // digit histograms (+ system sizes)
    unsigned sort_tile[SORT_PASSES + 1];    // tile tickets per pass
    unsigned ncells, ngroups;
    unsigned row_total[NROWS];        // cells per level, groups
    unsigned level_start[MAX_LEVEL + 2]; // first cell of each level; [22] = ncells
    unsigned walk_next;               // group queue heads of the walk instantiations with
    unsigned walk_next2;              // one and two bodies per lane
    unsigned status;
    unsigned long long inter[2];      // n_pc, n_pp totals of the last walk
    double diag[8];
    float judge_p99;                  // learned path: p99 relative error at the judge's samples
    unsigned fallback;                // 1: the judge asked for the fine-theta walk
    unsigned judge_tick;              // learned evaluations since the interval was set
    unsigned judge_on;                // 1: this evaluation is judged
    unsigned long long cyc_active;    // block steps, last cycle: body steps ended (forces taken)
    unsigned long long cyc_inter[2];  // block steps, last cycle: n_pc, n_pp summed over substeps
    unsigned hold_tile;               // testing aid: sort tile hold_tile - 1 never publishes (0: off)
    unsigned blk_next;                // block steps: first substep after the last kick at which a step ends
    unsigned mom_starts;              // multipoles: internal cells whose children are all leaves
};

// The launches of one entry point captured into a CUDA graph and replayed
// while the parameters they were captured with (key) stay the same.
struct CallGraph {
    static constexpr int KEYS = 12;
    cudaGraphExec_t exec = nullptr;
    long long key[KEYS] = {};
    int nkey = 0;              // 0: no call recorded yet
    bool failed = false;       // capture or instantiation failed for this key: direct launches
};

struct Ctx {
    // configuration
    int nleaf = 16, ncrit = 64, walk_warps = 4, list_capacity = 256, use_graph = 1;
    int group_pack = 0;               // 1: consecutive sibling groups packed up to ncrit bodies
    long long max_spin = 1ll << 24;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;                     // forked from stream for concurrent walk launches
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0, num_sms = 0;

    // sizes
    long long n = 0, ncap = 0, ccap = 0;
    long long cells_hint = 0;         // cell count of the last tree the host read (0: none); sizes launches
    int ntiles = 0, nbblocks = 0;     // sort tiles, build blocks
    int nsys = 1;                     // independent systems (contiguous body segments)

    // body arrays
    float4 *pos4 = nullptr, *vel4 = nullptr, *acc4 = nullptr;
    float4 *pos4_alt = nullptr, *vel4_alt = nullptr;
    uint32_t *id = nullptr, *id_alt = nullptr;
    uint8_t *sysid = nullptr;         // system of each body position (same before/after sorting)
    // sort
    unsigned long long *keys = nullptr, *keys_alt = nullptr;
    uint32_t *vals = nullptr, *vals_alt = nullptr;   // vals ends as perm
    unsigned *tile_status = nullptr;                   // (SORT_PASSES + 1) * ntiles * SORT_RADIX
    // build
    unsigned *blockcount = nullptr;  // BUILD_ROWS * nbblocks
    uint4 *build_entries = nullptr;  // per build block, the bodies that start cells (capacity n)
    uint2 *cell_body = nullptr, *cell_link = nullptr;
    uint8_t *cell_level = nullptr;
    uint32_t *cell_parent = nullptr, *cell_done = nullptr, *cell_cb = nullptr;
    uint32_t *cell_start = nullptr;  // multipoles: the internal cells whose children are all leaves
    float4 *mono = nullptr, *quadA = nullptr, *test = nullptr;
    float2 *quadB = nullptr;
    float2 *delta = nullptr;         // per cell: (|com - centre|, side l; after a refit 2 ext)
    float4 *cext = nullptr;          // per cell after a refit: build-time centre, half side ext holding its bodies
    double *shadow = nullptr;        // FP64 moments of the top levels (10 per cell)
    uint2 *groups = nullptr;
    // sibling packing (group_pack = 1): the unpacked groups, their cell level
    // (0xff: a run of an oversize leaf), packed-group start flags, and the
    // number of starts per packing block
    uint2 *groups_raw = nullptr;
    uint8_t *group_lvl = nullptr, *group_flag = nullptr;
    unsigned *group_bcount = nullptr;
    uint2 *counts = nullptr;         // per body (n_pc, n_pp), sorted order
    float *feat = nullptr;           // per body FEAT_STRIDE walk features (learned correction), sorted order
    // staging for host transfers and caller-order outputs
    float *stage = nullptr;          // 7 floats per body, at least STAGE_MIN_FLOATS
    long long stage_floats = 0;      // its size
    DevState *st = nullptr;          // device
    DevState *st_host = nullptr;     // pinned mirror for reads

    // pipeline state
    bool have_bodies = false, built = false, moments_ready = false, have_acc = false;
    long long arena_limit = 0;       // bytes; 0: no cap on the body arena
    bool tree_fresh = false;         // the tree was built from the current positions (no refit since)
    float theta = 0.75f, eps = 0.01f;
    cudaGraphExec_t step_graph = nullptr;
    CallGraph build_graph, mom_graph, forces_graph;   // bonsai_build / _multipoles / _forces
    long long arena_gen = 0;         // bumped whenever the arena is reallocated
    static constexpr int NSTAGE = 8;
    cudaEvent_t ev[NSTAGE + 1] = {};
    bool timed_step = false;         // the last bonsai_step recorded stage events
    bool stage_timing = false;       // bonsai_step records stage events (bonsai_set_stage_timing)
    bool graph_timing = false;       // the captured step graph holds them
    float graph_dt = 0.f, graph_theta = 0.f, graph_eps = 0.f;
    long long graph_n = -1;

    // block time steps: while a cycle's walk runs, block_kmax >= 0 and the
    // walk takes only the bodies whose step ends at substep block_s (their
    // level is vel4.w); -1 otherwise
    int block_kmax = -1;
    unsigned block_s = 0;
    int blk_walked = 0, blk_rebuilt = 0;   // last cycle: substeps walked, substeps rebuilt

    // learned far-field correction (bonsai_set_learned): weights, thetas,
    // judge budget, and the judge's sample and scratch
    const float *mlp_P = nullptr, *mlp_norm = nullptr;
    float theta_coarse = 1.0f, theta_fine = 0.5f, p99_budget = 0.f;
    int judge_every = 1;                 // judge every k-th learned evaluation, 0: never
    uint32_t *judge_targets = nullptr;   // JUDGE_MAX sorted positions
    float4 *judge_partial = nullptr;     // JUDGE_SPLIT x JUDGE_MAX
    float4 *judge_direct = nullptr;      // JUDGE_MAX
    int judge_n = 0;                     // targets in use

    std::string err;
};

// ---- per-device one-time kernel set-up --------------------------------------
constexpr int MAX_DEVICES = 64;

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) applies to the current
// device only, so each call site records, per device, the largest size it
// has already allowed.  Called before any stream capture of the launch.
inline cudaError_t allow_dyn_smem(const void *fn, size_t bytes, size_t (&done)[MAX_DEVICES]) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (bytes <= done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[dev] = bytes;
    return e;
}

// ---- device helpers ------------------------------------------------------

// Monotone map float -> int (signed compare order == float order).
__device__ __forceinline__ int f2ord(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) {
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// Reciprocal square root on the MUFU unit (PTX rsqrt.approx.ftz.f32).  The
// interaction kernels call it on r^2 + eps^2 >= eps^2, a normal float, where
// it returns what rsqrtf returns, without the scaling steps that a
// denormal-preserving build adds around every rsqrtf.
__device__ __forceinline__ float rsqrt_mufu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Number of leading tree levels shared by two keys (level 0 always shared):
// prefix_l(a) == prefix_l(b) iff l <= cpl(a, b).
// Branch-free: with y = 2(a ^ b) + 1 the highest set bit of y is one above
// the highest differing bit h of the keys (bit 0 when they are equal), so
// ceil(bit / 3) is h / 3 + 1 for different keys and 0 for equal ones.
__device__ __forceinline__ int key_cpl(unsigned long long a, unsigned long long b) {
    const unsigned long long y = ((a ^ b) << 1) | 1ull;         // keys use bits 0..62
    const unsigned hb = 63u - (unsigned)__clzll((long long)y);
    return MAX_LEVEL - (int)((hb + 2u) / 3u);
}

// Block time steps: a body of level k (stored as a float) takes forces at
// substep s of a cycle of 2^kmax substeps iff s is a multiple of 2^(kmax - k).
__device__ __forceinline__ bool block_active(float level, unsigned s, int kmax) {
    const unsigned len = 1u << (kmax - (int)level);
    return (s & (len - 1u)) == 0u;
}

// Shared levels of two bodies that may belong to different systems (-1: none).
__device__ __forceinline__ int body_cpl(unsigned long long a, unsigned long long b, uint8_t sa, uint8_t sb) {
    return sa == sb ? key_cpl(a, b) : -1;
}

__device__ __forceinline__ unsigned long long key_prefix(unsigned long long k, int level) {
    return level == 0 ? 0ull : (k >> (3 * (MAX_LEVEL - level)));
}

// ---- launchers (host) ------------------------------------------------------
cudaError_t launch_reset(Ctx &c);
cudaError_t launch_domains(Ctx &c);
cudaError_t launch_fill_sysid(Ctx &c);
cudaError_t launch_pack(Ctx &c, const float *pos, const float *mass, const float *vel);
cudaError_t launch_bbox(Ctx &c);
cudaError_t launch_kick_drift_bbox(Ctx &c, float dt);
cudaError_t launch_drift_bbox(Ctx &c, float dt);
cudaError_t launch_keys(Ctx &c);
cudaError_t launch_sort(Ctx &c);
cudaError_t launch_reorder(Ctx &c);
cudaError_t launch_build(Ctx &c);
cudaError_t launch_internal_counts(Ctx &c);
cudaError_t launch_multipoles(Ctx &c, float theta = 0.f);
cudaError_t launch_multipoles_refit(Ctx &c);
cudaError_t launch_cell_cubes(Ctx &c);
cudaError_t launch_sph_walk(Ctx &c, const float *hs, const float4 *cext, float *rho_s, int32_t *cnt_s);
cudaError_t launch_open_radius(Ctx &c, float theta, const unsigned *gate = nullptr);
cudaError_t launch_walk(Ctx &c, float eps, bool features = false, const unsigned *gate = nullptr);
cudaError_t launch_direct(Ctx &c, const uint32_t *targets, int ntar, float eps, float4 *partial, int nsplit,
                          float4 *out, const unsigned *gate = nullptr);
cudaError_t launch_judge(Ctx &c, const uint32_t *targets, int ntar, const float4 *direct, float budget,
                         const unsigned *gate = nullptr);
cudaError_t launch_mlp_infer(Ctx &c, const float *P, const float *norm);
cudaError_t launch_mlp_rows(cudaStream_t s, const float *P, const float *norm, const float *X, float *Y, int n);
cudaError_t launch_mlp_grad(cudaStream_t s, const float *P, const float *norm, const float *X, const float *Y,
                            const uint32_t *idx, int bsz, float *grad, float *loss);
cudaError_t launch_adamw(cudaStream_t s, float *P, const float *grad, float *m, float *v, float lr, float wd,
                         int step);
cudaError_t launch_gather_features(Ctx &c, const uint32_t *targets, int ntar, float *X, uint32_t *ids);
cudaError_t launch_labels(Ctx &c, const uint32_t *targets, int ntar, const float4 *direct, float *Y);
cudaError_t launch_feature_stats(cudaStream_t s, const float *X, const float *Y, int n, float *norm);
cudaError_t launch_kick(Ctx &c, float dt);
cudaError_t launch_scatter_forces(Ctx &c, float *acc, float *pot);
cudaError_t launch_scatter_bodies(Ctx &c, float *pos, float *vel);
cudaError_t launch_scatter_counts(Ctx &c, uint32_t *npc, uint32_t *npp);
cudaError_t launch_diag(Ctx &c);
cudaError_t launch_tree_export(Ctx &c, unsigned c0, unsigned cnt, int32_t *bb, int32_t *bc, int32_t *cb,
                               int32_t *nc, int32_t *lv);
cudaError_t launch_moments_export(Ctx &c, unsigned c0, unsigned cnt, float *mono, float *quad);

cudaError_t launch_fma_peak(int blocks, int threads, long long iters, float *sink);
cudaError_t launch_judge_targets(Ctx &c);
cudaError_t launch_gated_walk_reset(Ctx &c);
cudaError_t pipeline_learned_forces(Ctx &c, float eps);

}  // namespace bonsai

struct bonsai_ctx {
    bonsai::Ctx c;
};
