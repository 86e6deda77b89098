/*
 * bonsai.h -- C ABI of the GB300 Barnes-Hut tree-code library (libbonsai.so).
 *
 * The library runs the per-step hot path of "Bonsai: A GPU Tree-Code"
 * (Bedorf, Gaburov & Portegies Zwart) entirely on one GPU: Morton keys and
 * radix sort of the bodies along the space-filling curve, reordering
 * ("moving"), octree construction, multipole moments and the group-wise
 * tree-traverse under the opening angle theta (paper Sect. 2 and Fig. 1),
 * plus the shared-time-step leapfrog the paper's block-time-step discussion
 * builds on (Sect. 1 and 3).
 *
 * Conventions (all entry points):
 *  - Return value: BONSAI_OK (0) or a negative BONSAI_ERR_* code; the text of
 *    the last error of a context is returned by bonsai_last_error().  No entry
 *    point aborts the process and no kernel traps.
 *  - Pointers: plain host or device pointers and element counts.  The caller
 *    owns every buffer it passes; the library copies inputs in and writes
 *    outputs out, and keeps no reference to caller memory after a call.
 *    `on_device` = 1 means the pointers are CUDA device pointers on the
 *    context's device, ordered on the context's stream; 0 means host memory
 *    (the call then synchronises the stream before returning).
 *  - Units: G = 1.  Positions, velocities and masses are float32.
 *  - Order: every per-body output is in the caller's body order (the order of
 *    the last bonsai_set_bodies call); the library sorts bodies internally.
 *  - Memory: the context allocates and owns all device memory it uses
 *    (cudaMalloc at create / set_bodies; reused while N does not grow) and
 *    frees it in bonsai_destroy.
 *  - Threads: a context may be used by one host thread at a time.
 */
#ifndef BONSAI_H
#define BONSAI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BONSAI_OK              0
#define BONSAI_ERR_INVALID_ARG (-1)  /* bad pointer, size or parameter        */
#define BONSAI_ERR_OOM         (-2)  /* device allocation failed              */
#define BONSAI_ERR_CUDA        (-3)  /* a CUDA runtime call failed            */
#define BONSAI_ERR_CAPACITY    (-4)  /* a walk list or cell capacity overflow */
#define BONSAI_ERR_TIMEOUT     (-5)  /* a bounded device-side wait gave up    */
#define BONSAI_ERR_NAN         (-6)  /* non-finite positions detected         */
#define BONSAI_ERR_NOT_READY   (-7)  /* stage called before its inputs exist  */

typedef struct bonsai_ctx bonsai_ctx;

/* Tuning knobs; a zero field selects the default shown. */
typedef struct {
    int nleaf;            /* max bodies per leaf cell (16)                    */
    int ncrit;            /* max bodies per walk group, 1..64 (64)            */
    int walk_warps;       /* warps per walk thread block, 1..8 (4)            */
    int list_capacity;    /* walk stack entries per warp, 64..8192 (256)      */
    int use_graph;        /* -1: direct launches; else replay bonsai_step
                             from a CUDA graph (default)                      */
    int group_pack;       /* walk groups: 0 = the cells with at most ncrit
                             bodies whose parent holds more (default);
                             1 = those groups with consecutive siblings (same
                             parent cell) packed greedily, in key order, up
                             to ncrit bodies per group                        */
    int arena_limit_mib;  /* 0: none; else bonsai_set_bodies refuses, with
                             BONSAI_ERR_OOM, a device arena larger than this
                             many MiB (a host-side cap that stands in for an
                             out-of-memory device)                           */
    int reserved;
    long long max_spin;   /* bound on every device-side wait, polls (1<<24)   */
} bonsai_config;

/* Create a context on the current CUDA device.  cfg may be NULL (defaults).
 * cuda_stream is a cudaStream_t (not the legacy NULL stream) to order all
 * work on, or NULL for a blocking stream owned by the context (ordered with
 * the legacy default stream).  *out receives the context (NULL on failure). */
int bonsai_create(bonsai_ctx **out, const bonsai_config *cfg, void *cuda_stream);

/* Free every device resource of the context.  NULL is ignored. */
void bonsai_destroy(bonsai_ctx *ctx);

/* Load N bodies: pos (N x 3, xyz interleaved), mass (N), vel (N x 3, or
 * NULL for zero velocities).  Invalidates the tree and the forces.
 * N must be in [1, 2^26].  Host buffers (on_device = 0) are read before the
 * call returns: page-locked ones directly by a kernel through their device
 * address, others through a copy to the context's staging area. */
int bonsai_set_bodies(bonsai_ctx *ctx, const float *pos, const float *mass,
                      const float *vel, long long n, int on_device);

/* Batched ensemble: the n bodies of the last bonsai_set_bodies form nsys
 * independent systems, system s holding bodies [offsets[s], offsets[s+1])
 * (host array of nsys + 1 entries, offsets[0] = 0, offsets[nsys] = n, no
 * empty system, 1 <= nsys <= 256).  Every stage then runs on all systems at
 * once: per-system domain cubes and keys, one sort by (system, key), one tree
 * build with one root per system, one multipole pass and one persistent walk
 * over the groups of all systems.  Call right after bonsai_set_bodies
 * (bonsai_set_bodies resets to a single system). */
int bonsai_set_systems(bonsai_ctx *ctx, const long long *offsets, int nsys);

/* bonsai_build, bonsai_multipoles and bonsai_forces run their launches
 * directly the first time a configuration is seen (size, systems, tuning
 * knobs, theta and eps), capture them into a CUDA graph the second time and
 * replay that graph while the configuration holds (use_graph = -1: always
 * direct launches); the results are the same bit for bit. */

/* Sect. 2 "sorting", "moving", "tree-construction": domain cube, 63-bit
 * Morton keys (21 bits per axis, x in the lowest bit of each triple), stable
 * LSD radix sort, body reorder, octree (cells with more than nleaf bodies
 * split into their non-empty octants; breadth-first, key order within a
 * level) and walk groups (cells with at most ncrit bodies whose parent has
 * more). */
int bonsai_build(bonsai_ctx *ctx);

/* Sect. 2 "multipole moments": per cell mass, centre of mass and traceless
 * quadrupole Q_ij = sum m (3 y_i y_j - |y|^2 delta_ij), y = x - com, computed
 * from the leaves up (FP64 for the root of each system).  Requires
 * bonsai_build. */
int bonsai_multipoles(bonsai_ctx *ctx);

/* Sect. 2 "tree-traverse": softened accelerations and potentials under the
 * opening angle theta (a cell is opened when the squared distance from its
 * com to the group's bounding box is below (l/theta + delta)^2, l its side,
 * delta the com's offset from its centre) with Plummer softening eps.
 * acc: N x 3, pot: N (either may be NULL), caller order.  Requires
 * bonsai_multipoles.  0 < theta <= 1.15, eps > 0. */
int bonsai_forces(bonsai_ctx *ctx, float theta, float eps, float *acc,
                  float *pot, int on_device);

/* One kick-drift-kick leapfrog step of length dt for all bodies: the first
 * kick uses the accelerations of the last bonsai_forces/bonsai_step (if there
 * are none, they are computed first at that call's theta/eps, default 0.75 /
 * 0.01), then the drift, the full rebuild (keys, sort, reorder, build,
 * multipoles), the walk and the second kick.  No host synchronisation. */
int bonsai_step(bonsai_ctx *ctx, float dt);

/* Block (hierarchical) time steps, paper Sect. 1 and 3: only the bodies
 * whose step ends are walked, and between rebuilds only the moments of the
 * cells are recomputed ("refit"); the paper names the scheme, not its rules,
 * which are these.  Body i steps with dt_max / 2^k, k in [0, max_level] the
 * smallest level with dt_max / 2^k <= eta * sqrt(eps / |a_i|) (decided in
 * float32 as 16^k >= c |a|^2, c = dt_max^4 / (eta^4 eps^2) rounded to float
 * once).  One call advances one cycle of dt_max = 2^max_level substeps of
 * dt_max / 2^max_level, all bodies synchronised at both ends: opening half
 * kicks at the start; per substep a drift of every body and, if some body's
 * step ends there, a rebuild (every rebuild_every-th substep, starting with
 * the first; one scheduled on a substep where no step ends is taken at the
 * next substep where one does) or a refit, a walk of the bodies whose step
 * ends (each group's box is its active bodies' box), and for those the
 * closing half kick, a new level (never coarser than the substep's
 * alignment allows) and the next opening half kick.  A substep where no
 * step ends only drifts.  theta and
 * eps are those of the last bonsai_forces / bonsai_set_params; without
 * forces yet they are computed first.  max_level = 0 is bonsai_step(dt_max).
 * One system only (BONSAI_ERR_INVALID_ARG otherwise); 0 <= max_level <= 20,
 * rebuild_every >= 1.  A refitted cell opens with 2 ext / theta + delta,
 * ext the half side of its build-time cube enlarged to hold its bodies'
 * current positions (a leaf from its bodies, a parent from its children), so
 * a cell that holds a walked body is always opened for that body's group.
 * Synchronises once per walked substep: each kick leaves on the device the
 * next substep at which some body's step ends, and the host reads it (4
 * bytes) to schedule the next walk. */
int bonsai_block_cycle(bonsai_ctx *ctx, float dt_max, int max_level, float eta,
                       int rebuild_every);

/* The level every body would take from its current acceleration under
 * (dt_max, max_level, eta) and the context's eps: levels (N int32, caller
 * order, host buffer).  A query; nothing changes.  Requires forces. */
int bonsai_block_levels(bonsai_ctx *ctx, float dt_max, int max_level, float eta,
                        int32_t *levels);

/* Counters of the last block cycle: out[0] = body steps that ended (forces
 * taken), out[1] / out[2] = body-cell / body-body interactions summed over
 * its substeps.  Synchronises. */
int bonsai_block_stats(bonsai_ctx *ctx, long long out[3]);

/* Schedule of the last block cycle (host counters, no synchronisation):
 * out[0] = substeps walked (those where some body's step ended), out[1] =
 * substeps rebuilt; the other substeps refitted (walked - rebuilt) or only
 * drifted (2^max_level - walked). */
int bonsai_block_substeps(bonsai_ctx *ctx, int32_t out[2]);

/* Neighbour search and SPH density on the octree (paper Sect. 3: the tree
 * also serves neighbour search and smoothed particle hydrodynamics).  h: the
 * smoothing length of every body (N floats, caller order).  The neighbours
 * of body i are the bodies j, i itself included, with |x_j - x_i| < h_i,
 * decided in float32 as r^2 < h_i^2 with dx = x_j - x_i rounded and
 * r^2 = fma(dz, dz, fma(dy, dy, dx*dx)); nngb[i] is their count and
 * rho[i] = sum_j m_j W(|x_j - x_i|, h_i), W the cubic spline kernel of
 * compact support h: 8/(pi h^3) (1 - 6q^2 + 6q^3) for q = r/h <= 1/2,
 * 8/(pi h^3) 2 (1 - q)^3 for 1/2 < q < 1.  The groups and traversal are the
 * gravity walk's; a cell is searched iff its cube comes within the group's
 * largest h of the group's box.  Outputs (N each, caller order, either may be
 * NULL) on the side on_device says; h on the same side.  Needs a tree built
 * from the current positions (bonsai_build or bonsai_step; not after a block
 * cycle that ended on a refit: BONSAI_ERR_NOT_READY).  h > 0 is the caller's
 * to ensure (h <= 0 gives no neighbours). */
int bonsai_sph_density(bonsai_ctx *ctx, const float *h, float *rho, int32_t *nngb,
                       int on_device);

/* Autotuner: times the walk of the current bodies (CUDA events, mean of two
 * walks after one untimed) for every group size ncrit in {16, 32, 48, 64},
 * both group rules (group_pack 0 and 1), walk thread-block width in
 * {2, 4, 8} warps and walk stack capacity (list_capacity) in {128, 256, 512}
 * entries per warp, keeps the fastest choice in the context (rebuilding the
 * tree and groups for it) and leaves forces at (theta, eps) computed.
 * Candidates that overflow the walk stack are skipped.  Any output pointer
 * may be NULL; bonsai_get_config reports the chosen group rule and
 * capacity. */
int bonsai_autotune(bonsai_ctx *ctx, float theta, float eps, int *best_ncrit,
                    int *best_warps, float *best_ms);

/* The context's current tuning knobs (after defaults and any autotuning):
 * every field of *out is filled in (reserved fields 0). */
int bonsai_get_config(const bonsai_ctx *ctx, bonsai_config *out);

/* Sets theta and eps for bonsai_step without computing forces. */
int bonsai_set_params(bonsai_ctx *ctx, float theta, float eps);

/* Copy the current state out in caller order: pos (N x 3), vel (N x 3),
 * either may be NULL. */
int bonsai_get_bodies(bonsai_ctx *ctx, float *pos, float *vel, int on_device);

/* FP64 diagnostics of the current state: out[8] = {K, W, E, Px, Py, Pz,
 * Mtot, Lz} with K = sum m v^2/2, W = sum m phi/2 (phi of the last walk),
 * E = K + W, P = sum m v, Lz = sum m (x v_y - y v_x).  Host output. */
int bonsai_diagnostics(bonsai_ctx *ctx, double out[8]);

/* Synchronise the context's stream and return (and clear) the device status:
 * BONSAI_OK, BONSAI_ERR_CAPACITY, BONSAI_ERR_TIMEOUT or BONSAI_ERR_NAN. */
int bonsai_sync(bonsai_ctx *ctx);

/* on != 0: later bonsai_step calls record CUDA events on the context's
 * stream between their stages (also when the step is replayed from its
 * graph) for bonsai_get_stage_times; 0 (the default): no events.  The nine
 * event nodes cost about 40 us per step at N = 2^20, so timed runs measure
 * steps without them.  Changing it re-captures the step graph. */
int bonsai_set_stage_timing(bonsai_ctx *ctx, int on);

/* Device time of each stage of the last bonsai_step in milliseconds (that
 * step must have run with stage timing on: BONSAI_ERR_NOT_READY otherwise).
 * ms[0] first kick + drift + domain, [1] keys, [2] sort, [3] reorder, [4]
 * tree build, [5] multipoles (with the walk's MAC records), [6] walk, [7]
 * second kick.  Synchronises; writes min(n, 8) values and returns that
 * count (negative on error). */
int bonsai_get_stage_times(bonsai_ctx *ctx, float *ms, int n);

/* ---- introspection (copies to caller-owned HOST buffers; synchronises) -- */

/* Number of bodies, cells and groups of the current tree. */
int bonsai_get_sizes(bonsai_ctx *ctx, long long *n, long long *ncells,
                     long long *ngroups);

/* Domain of the last build: mn[3] (per-axis float minimum) and side[1]
 * (of system 0). */
int bonsai_get_domain(bonsai_ctx *ctx, float mn[3], float side[1]);

/* Domains of all systems: mn (nsys x 3), side (nsys). */
int bonsai_get_domains(bonsai_ctx *ctx, float *mn, float *side);

/* Sorted keys (N) and the sort permutation perm (N): sorted position i holds
 * caller body perm[i]. */
int bonsai_get_keys(bonsai_ctx *ctx, uint64_t *keys, uint32_t *perm);

/* Cells in breadth-first order (ncells each): first body (sorted order),
 * body count, first child (0 for leaves), child count, level. */
int bonsai_get_tree(bonsai_ctx *ctx, int32_t *body_begin, int32_t *body_count,
                    int32_t *child_begin, int32_t *nchild, int32_t *level);

/* Groups in key order (ngroups each): first body (sorted order), count. */
int bonsai_get_groups(bonsai_ctx *ctx, int32_t *begin, int32_t *count);

/* Moments per cell: mono (ncells x 4: com xyz, M), quad (ncells x 6:
 * Qxx Qyy Qzz Qxy Qxz Qyz). */
int bonsai_get_moments(bonsai_ctx *ctx, float *mono, float *quad);

/* Interaction counts of the last walk per body, caller order: n_pc
 * (body-cell) and n_pp (body-body, self excluded); and the totals over all
 * bodies in tot[2].  Any pointer may be NULL. */
int bonsai_get_counts(bonsai_ctx *ctx, uint32_t *n_pc, uint32_t *n_pp,
                      unsigned long long tot[2]);

/* Stable sort of n 63-bit keys that allocates nothing.  No counterpart in
 * the paper: it exists for callers that cannot call cudaMalloc -- latency-
 * critical loops (cudaMalloc/cudaFree may synchronise the whole device), or
 * hosts whose own caching allocator already owns the device memory (a second
 * allocator would fail or fragment it).  keys (n, read only), sorted_keys
 * (n) and perm (n) are caller-owned DEVICE buffers on the current device;
 * sorted_keys[i] = keys[perm[i]], equal keys in input order.  All scratch is
 * one static device array (about 0.9 MiB, held by every GPU that loads the
 * library until exit), so n is limited to 65536 (larger n: INVALID_ARG).
 * The first call on a device looks up that array's device address and sets
 * the sort kernel's shared-memory limit for that device.  Every call reuses
 * the same scratch: calls whose GPU work could overlap (other threads or
 * streams) race and must be serialised by the caller.  Work is ordered on
 * cuda_stream (NULL: the legacy default stream); the call then reads a status
 * word back and synchronises that stream, so it cannot run while the stream
 * is being captured into a CUDA graph.  It returns BONSAI_ERR_TIMEOUT if a
 * bounded device-side wait gave up.  Error text: bonsai_last_error(NULL). */
int bonsai_sort_keys_static(const uint64_t *keys, uint64_t *sorted_keys,
                            uint32_t *perm, long long n, void *cuda_stream);

/* ---- measurement and testing aids (no counterpart in the paper) --------- */

/* FP32 peak microbenchmark for the walk's roofline: `blocks` blocks of
 * `threads` threads on the current device each run `iters` iterations of
 * eight independent chains of packed FP32x2 fused multiply-adds (the
 * instruction the walk's interaction tiles are made of), timed with CUDA
 * events on the legacy default stream.  *ms receives the kernel time and
 * *flop the floating-point operations it performed (blocks x threads x iters
 * x 8 chains x 2 lanes x 2), so the achieved rate is flop / ms.  Synchronises.
 * 1 <= blocks <= 65535, 32 <= threads <= 1024 (a multiple of 32), iters >= 1. */
int bonsai_bench_fma(int blocks, int threads, long long iters, float *ms, double *flop);

/* Testing aid for the bounded device-side waits: while tile >= 0, sort tile
 * `tile` (4096 keys) of every radix-sort pass of this context publishes no
 * count, so the look-back of the tile after it polls max_spin times, gives
 * up and sets the device's timeout status: bonsai_sync then returns
 * BONSAI_ERR_TIMEOUT and the stages after the sort skip their work.  The
 * keys are not sorted then and the bodies, reordered by an invalid
 * permutation, are lost: load them again with bonsai_set_bodies.  Nothing
 * faults (every position written stays inside the sort's buffers).  tile =
 * -1 (the default) turns it off. */
int bonsai_debug_hold_sort_tile(bonsai_ctx *ctx, int tile);

/* ---- learned far-field correction (an extension of the Sect. 2 walk) -----
 * A per-body MLP 12 -> 64 -> 64 -> 3 (ReLU; BF16 weights, inputs and hidden
 * activations, FP32 accumulation; inference on the tensor cores) predicts
 * the residual r = (a_direct - a_tree) / |a_tree| of the coarse-theta walk
 * as coefficients along a body-local frame (e0 = a_tree/|a_tree|, e1 = the
 * part of the body's offset o from its group box's centre orthogonal to e0,
 * e2 = e0 x e1), from 12 rotation-invariant quantities the walk produces:
 * log|a_tree|, log(-phi_tree), log(1 + accepted cells) in the level bins
 * 0-3, 4-6, 7-9, 10-21, log(1 + body-body interactions), log(n_G / (e_G^3 +
 * eps^3)), log((d_G + eps)/eps), |o| / (d_G / 2), cos(o, a_tree), log n_G
 * (e_G / d_G the largest extent / diagonal of the group's box).  Parameters:
 * 5187 floats, rows W[out][in]: W1 64x12, b1 64, W2 64x64, b2 64, W3 3x64,
 * b3 3; normalisation: mu[12], sigma[12], ysig (inputs (x-mu)/sigma, the net
 * predicts r / ysig).  Feature rows X are n x 12 raw (unnormalised) inputs,
 * targets Y n x 3 frame coefficients of r. */
typedef struct bonsai_mlp bonsai_mlp;

/* New MLP on the current device: He-normal weights from `seed`, zero
 * biases, identity normalisation. */
int bonsai_mlp_create(bonsai_mlp **out, unsigned long long seed);
void bonsai_mlp_destroy(bonsai_mlp *m);
const char *bonsai_mlp_last_error(const bonsai_mlp *m);

/* Host copies in/out of the 5187 parameters and 25 normalisation values
 * (either pointer may be NULL). */
int bonsai_mlp_set_params(bonsai_mlp *m, const float *params, const float *norm);
int bonsai_mlp_get_params(bonsai_mlp *m, float *params, float *norm);

/* Normalisation from a training set: per-feature mean and standard
 * deviation of X, RMS of Y. */
int bonsai_mlp_fit_norm(bonsai_mlp *m, const float *X, const float *Y, long long n, int on_device);

/* Raw network outputs (r / ysig) of n feature rows, on the tensor cores. */
int bonsai_mlp_predict(bonsai_mlp *m, const float *X, float *Y, long long n, int on_device);

/* Gradient (5187, host) and value (host) of the loss mean((net(X) -
 * Y/ysig)^2) over the n rows and 3 outputs; forward and backward on the GPU. */
int bonsai_mlp_grad(bonsai_mlp *m, const float *X, const float *Y, long long n, int on_device, float *grad,
                    float *loss);

/* AdamW training (beta 0.9/0.999, decoupled weight decay wd on the weight
 * matrices) for `epochs` passes over the n rows in shuffled batches of
 * `batch`; fits the normalisation first if it was never set.  loss_per_epoch
 * (host, may be NULL) receives the mean batch loss of each epoch. */
int bonsai_mlp_train(bonsai_mlp *m, const float *X, const float *Y, long long n, int on_device, int epochs,
                     int batch, float lr, float wd, unsigned long long seed, float *loss_per_epoch);

/* Training samples from a built context (after bonsai_multipoles): walk at
 * theta with features, direct sum at ntar <= 4096 distinct bodies drawn with
 * `seed`; X (ntar x 12) features, Y (ntar x 3) targets r, ids (ntar, may be
 * NULL) the caller indices of the sampled bodies.  Leaves the theta-walk
 * forces in the context. */
int bonsai_learn_samples(bonsai_ctx *ctx, float theta, float eps, int ntar, unsigned long long seed,
                         float *X, float *Y, uint32_t *ids, int on_device);

/* Judge of the current accelerations: direct sum (FP32 tiles and a FP32
 * reduction over source splits, both Kahan-compensated) at min(n, 4096)
 * bodies spaced evenly in key order and the 99th
 * percentile (numpy's linear interpolation) of |a - a_direct| / |a_direct|. */
int bonsai_judge(bonsai_ctx *ctx, float eps, float *p99);

/* Use the learned correction in bonsai_step and bonsai_forces_learned: walk
 * at theta_coarse with features, add the MLP's correction, judge it; if the
 * judge's p99 exceeds p99_budget, redo the walk at theta_fine (decided on the
 * device, no host synchronisation).  m must stay alive while in use; NULL
 * turns the correction off. */
int bonsai_set_learned(bonsai_ctx *ctx, const bonsai_mlp *m, float theta_coarse, float theta_fine,
                       float p99_budget);

/* Judge only every `every`-th learned evaluation (bonsai_step or
 * bonsai_forces_learned), counted from this call; the p99 and the fallback
 * decision of a judged evaluation hold until the next judged one.  every = 1
 * (the default) judges each evaluation; every = 0 never judges and never falls
 * back.  Resets the count and the fallback flag.  BONSAI_ERR_INVALID_ARG for
 * every < 0. */
int bonsai_set_judge_interval(bonsai_ctx *ctx, int every);

/* One learned force evaluation (requires bonsai_set_learned and
 * bonsai_multipoles); outputs as in bonsai_forces. */
int bonsai_forces_learned(bonsai_ctx *ctx, float eps, float *acc, float *pot, int on_device);

/* The last learned evaluation's judge p99 and whether it fell back. */
int bonsai_get_judge(bonsai_ctx *ctx, float *p99, int *fell_back);

/* Text of the last error of ctx (or, for ctx == NULL, of the last failed
 * bonsai_create, bonsai_sort_keys_static or bonsai_bench_fma of this
 * thread).  Valid until the next call on the context. */
const char *bonsai_last_error(const bonsai_ctx *ctx);

/* Library version string. */
const char *bonsai_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BONSAI_H */
