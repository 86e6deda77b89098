/*
 * bonsai_oracle.c -- plain FP64 CPU oracle of the Bonsai tree-code hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline /
 * reference arm of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Every function is either the plain definition of its result (Morton keys,
 * stable sort, moments about the centre of mass, O(N^2) direct summation,
 * energy) or the steps of the algorithm in the paper's order (level-by-level
 * octree construction, body groups, the group-wise tree walk under the opening
 * angle theta).  Nothing is blocked, fused or reordered for speed; OpenMP only
 * runs independent cells, groups or bodies side by side.
 *
 * Paper: Bedorf, Gaburov & Portegies Zwart, "Bonsai: A GPU Tree-Code",
 * Sect. 1 (Barnes-Hut tree-code, O(N log N) vs O(N^2)), Sect. 2 (sorting along
 * a Morton space-filling curve, moving, tree-construction, multipole moments,
 * tree-traverse with the Barnes (1994) / vector-machine MAC), Fig. 1 and 2.
 * The paper leaves most formulas unstated; the readings used here (key bit
 * order, leaf capacity, group rule, MAC form, quadrupole force, softening) are
 * listed in the repository's design notes and in each function below.
 *
 * Parity pins: every function is checked by the CPU test suite against closed
 * forms, invariants or brute force (tests/test_oracle_*.py).
 *
 * Build: gcc -O2 -std=c11 -fopenmp -fPIC -shared -ffp-contract=off
 * (-ffp-contract=off keeps a*b+c un-fused so results are identical on x86 and
 * Arm hosts; TwoSum below relies on it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_L 21                 /* bits per axis of the Morton key        */
#define ORC_Q ((double)(1 << ORC_L))

/* ------------------------------------------------------------------------ */
/* Exact arithmetic helpers.                                                */
/* ------------------------------------------------------------------------ */

/* Knuth's TwoSum: s + e == a + b exactly (round-to-nearest doubles). */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *e = (a - av) + (b - bv);
    *s = x;
}

/* Smallest power of two strictly greater than the exact value hi - lo
 * (hi >= lo, both float). */
static double pow2_above_diff(float hi, float lo)
{
    double s, e;
    two_sum((double)hi, -(double)lo, &s, &e);
    if (s <= 0.0) return 0.0;
    int ex;
    frexp(s, &ex);                  /* s = m 2^ex, m in [0.5, 1) */
    double p = ldexp(1.0, ex - 1);  /* largest power of two <= s */
    if (s == p) return (e < 0.0) ? p : 2.0 * p;
    return 2.0 * p;
}

/* floor((x - mn) * scale) for the exact real x - mn, scale a power of two. */
static int64_t exact_floor_scaled(float x, float mn, double scale)
{
    double s, e;
    two_sum((double)x, -(double)mn, &s, &e);
    double t = s * scale;           /* exact: scale is a power of two */
    double f = floor(t);
    if (f == t && e < 0.0) f -= 1.0;
    return (int64_t)f;
}

/* ------------------------------------------------------------------------ */
/* Sect. 2 "sorting": the domain cube and the Morton (Z-order) key.          */
/* ------------------------------------------------------------------------ */

/* Domain: per-axis float minimum mn[d]; side S = the smallest power of two
 * strictly greater than the largest per-axis extent max_d - mn_d (never below
 * 2^-64, so a zero extent gives S = 2^-64). */
int oracle_domain(const float *pos, int64_t n, float *mn_out, double *S_out)
{
    if (n <= 0) return -1;
    float mn[3] = {pos[0], pos[1], pos[2]}, mx[3] = {pos[0], pos[1], pos[2]};
    for (int64_t i = 1; i < n; i++)
        for (int d = 0; d < 3; d++) {
            float v = pos[3 * i + d];
            if (v < mn[d]) mn[d] = v;
            if (v > mx[d]) mx[d] = v;
        }
    double S = ldexp(1.0, -64);
    for (int d = 0; d < 3; d++) {
        double p = pow2_above_diff(mx[d], mn[d]);
        if (p > S) S = p;
    }
    for (int d = 0; d < 3; d++) mn_out[d] = mn[d];
    *S_out = S;
    return 0;
}

/* Key: q_d = floor((x_d - mn_d) * 2^21 / S) (exact real arithmetic), clamped
 * to [0, 2^21 - 1]; bit 3b of the key is bit b of q_x, bit 3b+1 of q_y and
 * bit 3b+2 of q_z (x in the lowest bit of each triple). */
uint64_t oracle_interleave(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t k = 0;
    for (int b = 0; b < ORC_L; b++) {
        k |= (uint64_t)((qx >> b) & 1u) << (3 * b);
        k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((qz >> b) & 1u) << (3 * b + 2);
    }
    return k;
}

int oracle_keys(const float *pos, int64_t n, const float *mn, double S,
                uint64_t *keys)
{
    double scale = ORC_Q / S;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        uint32_t q[3];
        for (int d = 0; d < 3; d++) {
            int64_t v = exact_floor_scaled(pos[3 * i + d], mn[d], scale);
            if (v < 0) v = 0;
            if (v > (1 << ORC_L) - 1) v = (1 << ORC_L) - 1;
            q[d] = (uint32_t)v;
        }
        keys[i] = oracle_interleave(q[0], q[1], q[2]);
    }
    return 0;
}

/* Stable sort by key: ties keep their input order. */
typedef struct { uint64_t k; uint32_t i; } kv_t;
static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return (x->i > y->i) - (x->i < y->i);
}

int oracle_sort(const uint64_t *keys, int64_t n, uint32_t *perm)
{
    kv_t *a = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
    if (!a) return -2;
    for (int64_t i = 0; i < n; i++) { a[i].k = keys[i]; a[i].i = (uint32_t)i; }
    qsort(a, (size_t)n, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < n; i++) perm[i] = a[i].i;
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sect. 2 "tree-construction": level-by-level octree from sorted keys.      */
/* ------------------------------------------------------------------------ */

static inline unsigned digit_at(uint64_t key, int level)
{   /* octant digit of a level-`level` cell (level >= 1) */
    return (unsigned)((key >> (3 * (ORC_L - level))) & 7u);
}

/* Octree over sorted keys.  The root (level 0) holds all n bodies.  Walking
 * the levels in order, every cell with more than nleaf bodies and level < 21
 * splits into its non-empty octants, in octant order; other cells are leaves.
 * Cells are stored level by level (breadth first), in key order within a
 * level, so the children of a cell are contiguous.  Leaves get child_begin =
 * nchild = 0.  Returns the cell count, or -1 if cap is too small. */
int64_t oracle_build(const uint64_t *skeys, int64_t n, int nleaf, int64_t cap,
                     int32_t *body_begin, int32_t *body_count,
                     int32_t *child_begin, int32_t *nchild, int32_t *level,
                     int32_t *parent)
{
    if (n <= 0 || cap < 1) return -1;
    int64_t nc = 1;
    body_begin[0] = 0; body_count[0] = (int32_t)n; level[0] = 0; parent[0] = -1;
    int64_t lb = 0, le = 1;
    for (int l = 0; l <= ORC_L; l++) {
        for (int64_t c = lb; c < le; c++) {
            child_begin[c] = 0; nchild[c] = 0;
            if (body_count[c] <= nleaf || l == ORC_L) continue;
            int64_t b = body_begin[c], e = b + body_count[c];
            child_begin[c] = (int32_t)nc;
            int64_t s = b;
            while (s < e) {
                unsigned dg = digit_at(skeys[s], l + 1);
                int64_t t = s + 1;
                while (t < e && digit_at(skeys[t], l + 1) == dg) t++;
                if (nc >= cap) return -1;
                body_begin[nc] = (int32_t)s; body_count[nc] = (int32_t)(t - s);
                level[nc] = l + 1; parent[nc] = (int32_t)c;
                nc++; nchild[c]++;
                s = t;
            }
        }
        lb = le; le = nc;
        if (lb == le) break;
    }
    return nc;
}

/* Groups (Barnes 1990 vector-machine walk): the cells with at most ncrit
 * bodies whose parent holds more than ncrit (the root when n <= ncrit),
 * listed in key order.  A leaf with more than ncrit bodies (possible only for
 * identical keys at the deepest level, or ncrit < nleaf) is cut into
 * consecutive runs of ncrit bodies.
 *
 * pack != 0 (sibling packing, a reading of ours: the paper fixes no group
 * rule): the groups above are then taken in key order, and a group that is a
 * sibling of the previous one (same parent cell) joins the packed group that
 * the previous one belongs to if the sum stays within ncrit bodies; else it
 * starts a new packed group.  The root group and the runs of an oversize
 * leaf never join or absorb a neighbour.  Every packed group is then a run of
 * consecutive children of one cell.  Returns the group count or -1. */
static int cmp_first_int32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t oracle_groups(int64_t ncells, const int32_t *body_begin,
                      const int32_t *body_count, const int32_t *nchild,
                      const int32_t *parent, int ncrit, int pack, int64_t cap,
                      int32_t *g_begin, int32_t *g_count)
{
    int64_t ng = 0;
    int32_t *g_par = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    if (!g_par) return -1;
    for (int64_t c = 0; c < ncells; c++) {
        int is_group = 0;
        if (body_count[c] <= ncrit && (c == 0 || body_count[parent[c]] > ncrit))
            is_group = 1;
        if (is_group) {
            if (ng >= cap) { free(g_par); return -1; }
            g_begin[ng] = body_begin[c]; g_count[ng] = body_count[c];
            g_par[ng] = c == 0 ? -1 : parent[c];
            ng++;
        } else if (nchild[c] == 0 && body_count[c] > ncrit) {
            for (int32_t o = 0; o < body_count[c]; o += ncrit) {
                if (ng >= cap) { free(g_par); return -1; }
                g_begin[ng] = body_begin[c] + o;
                g_count[ng] = (body_count[c] - o < ncrit) ? body_count[c] - o : ncrit;
                g_par[ng] = -1;
                ng++;
            }
        }
    }
    /* key order = order of first body (unique per group, so any sort gives
     * the same order) */
    int32_t *trip = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(ng > 0 ? ng : 1));
    if (!trip) { free(g_par); return -1; }
    for (int64_t i = 0; i < ng; i++) {
        trip[3 * i] = g_begin[i]; trip[3 * i + 1] = g_count[i]; trip[3 * i + 2] = g_par[i];
    }
    qsort(trip, (size_t)ng, 3 * sizeof(int32_t), cmp_first_int32);
    for (int64_t i = 0; i < ng; i++) {
        g_begin[i] = trip[3 * i]; g_count[i] = trip[3 * i + 1]; g_par[i] = trip[3 * i + 2];
    }
    free(trip);
    if (pack && ng > 0) {
        int64_t out = 0;                         /* packed group being filled */
        for (int64_t i = 1; i < ng; i++) {
            int sibling = g_par[i] >= 0 && g_par[i] == g_par[i - 1];
            if (sibling && g_count[out] + g_count[i] <= ncrit) {
                g_count[out] += g_count[i];
            } else {
                out++;
                g_begin[out] = g_begin[i]; g_count[out] = g_count[i];
            }
        }
        ng = out + 1;
    }
    free(g_par);
    return ng;
}

/* ------------------------------------------------------------------------ */
/* Sect. 2 "multipole moments": mass, centre of mass, traceless quadrupole.  */
/* ------------------------------------------------------------------------ */

/* For every cell, straight from its bodies (sorted order):
 *   M = sum m,  com = sum m x / M,
 *   Q_ij = sum m (3 y_i y_j - |y|^2 delta_ij),  y = x - com.
 * Q is stored as (xx, yy, zz, xy, xz, yz). */
int oracle_moments(int64_t ncells, const int32_t *body_begin,
                   const int32_t *body_count, const float *spos,
                   const float *smass, double *M, double *com, double *Q)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < ncells; c++) {
        int64_t b = body_begin[c], e = b + body_count[c];
        double m = 0, cx = 0, cy = 0, cz = 0;
        for (int64_t j = b; j < e; j++) {
            double mj = smass[j];
            m += mj;
            cx += mj * spos[3 * j]; cy += mj * spos[3 * j + 1]; cz += mj * spos[3 * j + 2];
        }
        M[c] = m;
        if (m > 0) { cx /= m; cy /= m; cz /= m; }
        else { cx = spos[3 * b]; cy = spos[3 * b + 1]; cz = spos[3 * b + 2]; }
        com[3 * c] = cx; com[3 * c + 1] = cy; com[3 * c + 2] = cz;
        double q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = b; j < e; j++) {
            double mj = smass[j];
            double y0 = spos[3 * j] - cx, y1 = spos[3 * j + 1] - cy, y2 = spos[3 * j + 2] - cz;
            double y2s = y0 * y0 + y1 * y1 + y2 * y2;
            q[0] += mj * (3 * y0 * y0 - y2s);
            q[1] += mj * (3 * y1 * y1 - y2s);
            q[2] += mj * (3 * y2 * y2 - y2s);
            q[3] += mj * (3 * y0 * y1);
            q[4] += mj * (3 * y0 * y2);
            q[5] += mj * (3 * y1 * y2);
        }
        for (int k = 0; k < 6; k++) Q[6 * c + k] = q[k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Interaction formulas (Plummer-softened, G = 1).                           */
/* ------------------------------------------------------------------------ */

/* Body-body: a += m d / (|d|^2 + eps^2)^(3/2), phi -= m / (|d|^2+eps^2)^(1/2),
 * d = x_j - x_i. */
static inline void pp(double xi, double yi, double zi, double xj, double yj,
                      double zj, double mj, double eps2, double *a, double *phi)
{
    double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    double rinv = 1.0 / sqrt(r2);
    double mr3 = mj * rinv * rinv * rinv;
    a[0] += mr3 * dx; a[1] += mr3 * dy; a[2] += mr3 * dz;
    *phi -= mj * rinv;
}

/* Body-cell, monopole + traceless quadrupole about com, softened by using
 * r = sqrt(|d|^2 + eps^2), d = com - x_i, q = d^T Q d:
 *   phi -= M/r + q / (2 r^5)
 *   a   += M d / r^3 - Q d / r^5 + (5/2) q d / r^7 . */
static inline void pc(double xi, double yi, double zi, const double *cm,
                      double M, const double *Q, double eps2, double *a,
                      double *phi)
{
    double dx = cm[0] - xi, dy = cm[1] - yi, dz = cm[2] - zi;
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    double rinv = 1.0 / sqrt(r2);
    double r2i = rinv * rinv;
    double r3i = rinv * r2i, r5i = r3i * r2i, r7i = r5i * r2i;
    double Qx = Q[0] * dx + Q[3] * dy + Q[4] * dz;
    double Qy = Q[3] * dx + Q[1] * dy + Q[5] * dz;
    double Qz = Q[4] * dx + Q[5] * dy + Q[2] * dz;
    double q = dx * Qx + dy * Qy + dz * Qz;
    double s = M * r3i + 2.5 * q * r7i;
    a[0] += s * dx - r5i * Qx;
    a[1] += s * dy - r5i * Qy;
    a[2] += s * dz - r5i * Qz;
    *phi -= M * rinv + 0.5 * q * r5i;
}

/* Geometric cube of a cell: level l, corner index from the first body's key. */
static void cell_cube(uint64_t key, int l, const float *mn, double S,
                      double *centre, double *side)
{
    uint32_t q[3] = {0, 0, 0};
    for (int b = ORC_L - l; b < ORC_L; b++) {       /* top l bits per axis */
        q[0] |= (uint32_t)((key >> (3 * b)) & 1u) << b;
        q[1] |= (uint32_t)((key >> (3 * b + 1)) & 1u) << b;
        q[2] |= (uint32_t)((key >> (3 * b + 2)) & 1u) << b;
    }
    double h = S / ORC_Q;                           /* finest cell side */
    double l_side = ldexp(S, -l);
    for (int d = 0; d < 3; d++)
        centre[d] = (double)mn[d] + (double)q[d] * h + 0.5 * l_side;
    *side = l_side;
}

/* Opening radius (Barnes 1994 form, as read here): r_open = l/theta + delta,
 * delta = |com - geometric centre|, l = the cell's side. */
int oracle_open_radius(int64_t ncells, const int32_t *body_begin,
                       const int32_t *level, const uint64_t *skeys,
                       const float *mn, double S, const double *com,
                       double theta, double *r_open, const double *ext)
{
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < ncells; c++) {
        double ctr[3], l;
        cell_cube(skeys[body_begin[c]], level[c], mn, S, ctr, &l);
        if (ext) l = 2.0 * ext[c];      /* refit: the cube enlarged to hold the bodies */
        double dx = com[3 * c] - ctr[0], dy = com[3 * c + 1] - ctr[1], dz = com[3 * c + 2] - ctr[2];
        r_open[c] = l / theta + sqrt(dx * dx + dy * dy + dz * dz);
    }
    return 0;
}

/* Block time steps, refit between rebuilds (Sect. 3: only the moments are
 * recomputed): ext[c] = half side of a cube about the cell's build-time
 * geometric centre that holds the cell's bodies at their current positions,
 * at least l/2, bounded from the leaves up -- a leaf from its bodies, an
 * internal cell as max(l/2, max_k |centre_k - centre|_inf + ext_k) over its
 * children.  The opening radius of a refitted cell is then 2 ext / theta +
 * delta: for theta < 2/sqrt(3) a cell holding a body of a group is always
 * opened for that group.  At the build positions every body lies in its
 * cell's cube, so ext = l/2 and the radius is the plain one. */
int oracle_refit_extent(int64_t ncells, const int32_t *body_begin,
                        const int32_t *body_count, const int32_t *child_begin,
                        const int32_t *nchild, const int32_t *level,
                        const uint64_t *skeys, const float *mn, double S,
                        const float *spos, double *ext)
{
    double *ctr = (double *)malloc(sizeof(double) * 3 * (size_t)(ncells > 0 ? ncells : 1));
    if (!ctr) return -1;
    for (int64_t c = 0; c < ncells; c++) {
        double l;
        cell_cube(skeys[body_begin[c]], level[c], mn, S, ctr + 3 * c, &l);
        ext[c] = 0.5 * l;
    }
    for (int64_t c = ncells - 1; c >= 0; c--) {   /* breadth-first order: children after parents */
        double e = ext[c];
        if (nchild[c] == 0) {
            for (int64_t i = body_begin[c]; i < body_begin[c] + body_count[c]; i++)
                for (int d = 0; d < 3; d++) {
                    double t = fabs((double)spos[3 * i + d] - ctr[3 * c + d]);
                    if (t > e) e = t;
                }
        } else {
            for (int k = 0; k < nchild[c]; k++) {
                int64_t ch = child_begin[c] + k;
                double m = 0;
                for (int d = 0; d < 3; d++) {
                    double t = fabs(ctr[3 * ch + d] - ctr[3 * c + d]);
                    if (t > m) m = t;
                }
                if (m + ext[ch] > e) e = m + ext[ch];
            }
        }
        ext[c] = e;
    }
    free(ctr);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sect. 2 "tree-traverse": group-wise walk under the MAC.                   */
/* ------------------------------------------------------------------------ */

/* For every group G (in parallel), starting at the root and going breadth
 * first: a cell c is opened when the squared distance from its com to the
 * axis-aligned box of G's bodies (0 inside) is strictly below r_open(c)^2,
 * else accepted.  Every body of G takes a body-cell interaction with each
 * accepted cell and a body-body interaction with every other body of each
 * opened leaf; opened internal cells queue their children.
 *
 * Outputs per body (sorted order): acc[3], pot, n_pc, n_pp (self excluded).
 * A group is flagged borderline (flag[body] = 1 for its bodies) when some
 * tested cell had |dist - r_open| <= tau_abs + tau_rel * r_open, i.e. a
 * single-precision implementation may take the other decision there.
 * npc_bins (may be NULL, needs level): accepted cells per level bin.
 * active (may be NULL: every body): with block time steps only the active
 * bodies take forces; a group's box is then the box of its active bodies and
 * a group without one is skipped (outputs of inactive bodies untouched). */
int oracle_walk(int64_t n, const float *spos, const float *smass,
                int64_t ncells, const int32_t *body_begin,
                const int32_t *body_count, const int32_t *child_begin,
                const int32_t *nchild, const double *M, const double *com,
                const double *Q, const double *r_open, int64_t ngroups,
                const int32_t *g_begin, const int32_t *g_count, double eps,
                double tau_abs, double tau_rel, double *acc, double *pot,
                int32_t *n_pc, int32_t *n_pp, int8_t *flag,
                const int32_t *level, int32_t *npc_bins, const int8_t *active)
{
    (void)n; (void)ncells;
    double eps2 = eps * eps;
    int err = 0;
    #pragma omp parallel
    {
        int64_t qcap = 1024;
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)qcap);
        int32_t *acc_cells = (int32_t *)malloc(sizeof(int32_t) * (size_t)qcap);
        int32_t *open_leaves = (int32_t *)malloc(sizeof(int32_t) * (size_t)qcap);
        int64_t acap = qcap, lcap = qcap;
        #pragma omp for schedule(dynamic, 4)
        for (int64_t g = 0; g < ngroups; g++) {
            int64_t gb = g_begin[g], ge = gb + g_count[g];
            float bmin[3], bmax[3];
            int64_t first = gb;
            if (active) {
                while (first < ge && !active[first]) first++;
                if (first == ge) continue;               /* no active body */
            }
            for (int d = 0; d < 3; d++) bmin[d] = bmax[d] = spos[3 * first + d];
            for (int64_t i = first; i < ge; i++)
                for (int d = 0; d < 3; d++) {
                    if (active && !active[i]) break;
                    float v = spos[3 * i + d];
                    if (v < bmin[d]) bmin[d] = v;
                    if (v > bmax[d]) bmax[d] = v;
                }
            /* 1. Traverse: collect accepted cells and opened leaves. */
            int64_t qh = 0, qt = 0, na = 0, nl = 0;
            int border = 0;
            queue[qt++] = 0;
            while (qh < qt) {
                int32_t c = queue[qh++];
                const double *cm = com + 3 * c;
                double dist2 = 0;
                for (int d = 0; d < 3; d++) {
                    double t = 0;
                    if (cm[d] < bmin[d]) t = (double)bmin[d] - cm[d];
                    else if (cm[d] > bmax[d]) t = cm[d] - (double)bmax[d];
                    dist2 += t * t;
                }
                double ro = r_open[c];
                if (fabs(sqrt(dist2) - ro) <= tau_abs + tau_rel * ro) border = 1;
                if (dist2 < ro * ro) {                      /* open */
                    if (nchild[c] == 0) {
                        if (nl == lcap) { lcap *= 2; open_leaves = realloc(open_leaves, sizeof(int32_t) * (size_t)lcap); }
                        open_leaves[nl++] = c;
                    } else {
                        if (qt + nchild[c] > qcap) {
                            /* compact the consumed head, grow if needed */
                            memmove(queue, queue + qh, sizeof(int32_t) * (size_t)(qt - qh));
                            qt -= qh; qh = 0;
                            while (qt + nchild[c] > qcap) { qcap *= 2; queue = realloc(queue, sizeof(int32_t) * (size_t)qcap); }
                        }
                        for (int k = 0; k < nchild[c]; k++) queue[qt++] = child_begin[c] + k;
                    }
                } else {                                    /* accept */
                    if (na == acap) { acap *= 2; acc_cells = realloc(acc_cells, sizeof(int32_t) * (size_t)acap); }
                    acc_cells[na++] = c;
                }
            }
            /* Accepted cells by level bin (0-3, 4-6, 7-9, 10-21): an input of
             * the learned correction. */
            int32_t bins[4] = {0, 0, 0, 0};
            if (npc_bins)
                for (int64_t k = 0; k < na; k++) {
                    int32_t lv = level[acc_cells[k]];
                    bins[lv <= 3 ? 0 : lv <= 6 ? 1 : lv <= 9 ? 2 : 3]++;
                }
            /* 2. Evaluate for every body of the group. */
            int32_t npp_group = 0;
            for (int64_t k = 0; k < nl; k++) npp_group += body_count[open_leaves[k]];
            for (int64_t i = gb; i < ge; i++) {
                if (active && !active[i]) continue;
                double xi = spos[3 * i], yi = spos[3 * i + 1], zi = spos[3 * i + 2];
                double a[3] = {0, 0, 0}, phi = 0;
                int32_t self_seen = 0;
                for (int64_t k = 0; k < na; k++) {
                    int32_t c = acc_cells[k];
                    pc(xi, yi, zi, com + 3 * c, M[c], Q + 6 * c, eps2, a, &phi);
                }
                for (int64_t k = 0; k < nl; k++) {
                    int32_t c = open_leaves[k];
                    for (int64_t j = body_begin[c]; j < body_begin[c] + body_count[c]; j++) {
                        if (j == i) { self_seen++; continue; }
                        pp(xi, yi, zi, spos[3 * j], spos[3 * j + 1], spos[3 * j + 2],
                           smass[j], eps2, a, &phi);
                    }
                }
                acc[3 * i] = a[0]; acc[3 * i + 1] = a[1]; acc[3 * i + 2] = a[2];
                pot[i] = phi;
                n_pc[i] = (int32_t)na;
                n_pp[i] = npp_group - self_seen;
                flag[i] = (int8_t)border;
                if (npc_bins)
                    for (int b = 0; b < 4; b++) npc_bins[4 * i + b] = bins[b];
                if (self_seen != 1) {
                    #pragma omp atomic write
                    err = 1;
                }
            }
        }
        free(queue); free(acc_cells); free(open_leaves);
    }
    return err ? -3 : 0;   /* -3: a body's own leaf was accepted (theta too large) */
}

/* ------------------------------------------------------------------------ */
/* Sect. 1: O(N^2) direct summation -- the exact softened result.            */
/* ------------------------------------------------------------------------ */

/* For each target index t = idx[k]: a_t = sum_{j != t} m_j d / (|d|^2+eps^2)^(3/2),
 * phi_t = -sum_{j != t} m_j / (|d|^2+eps^2)^(1/2), d = x_j - x_t. */
int oracle_direct(const float *pos, const float *mass, int64_t n,
                  const int64_t *idx, int64_t nidx, double eps, double *acc,
                  double *pot)
{
    double eps2 = eps * eps;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nidx; k++) {
        int64_t t = idx[k];
        double xi = pos[3 * t], yi = pos[3 * t + 1], zi = pos[3 * t + 2];
        double a[3] = {0, 0, 0}, phi = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == t) continue;
            pp(xi, yi, zi, pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], mass[j],
               eps2, a, &phi);
        }
        acc[3 * k] = a[0]; acc[3 * k + 1] = a[1]; acc[3 * k + 2] = a[2];
        pot[k] = phi;
    }
    return 0;
}

/* Diagnostics: out = {K, W, E, Px, Py, Pz, Mtot, Lz} with
 * K = sum m v^2 / 2, W = sum m phi / 2, E = K + W, P = sum m v,
 * Lz = sum m (x v_y - y v_x). */
int oracle_energy(const float *pos, const float *vel, const float *mass,
                  const double *pot, int64_t n, double *out)
{
    double K = 0, W = 0, P[3] = {0, 0, 0}, Mt = 0, Lz = 0;
    for (int64_t i = 0; i < n; i++) {
        double m = mass[i];
        double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        K += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        W += 0.5 * m * pot[i];
        P[0] += m * vx; P[1] += m * vy; P[2] += m * vz;
        Mt += m;
        Lz += m * ((double)pos[3 * i] * vy - (double)pos[3 * i + 1] * vx);
    }
    out[0] = K; out[1] = W; out[2] = K + W;
    out[3] = P[0]; out[4] = P[1]; out[5] = P[2]; out[6] = Mt; out[7] = Lz;
    return 0;
}

/* Body-cell interaction of one target with one cell (M, com, Q), for tests of
 * the expansion's order of accuracy and of a = -grad(phi). */
int oracle_pc_eval(const double *x, const double *com, double M,
                   const double *Q, double eps, double *a, double *phi)
{
    a[0] = a[1] = a[2] = 0; *phi = 0;
    pc(x[0], x[1], x[2], com, M, Q, eps * eps, a, phi);
    return 0;
}

/* Geometric cube of every cell (centre xyz, side), for tests. */
int oracle_cell_cube(int64_t ncells, const int32_t *body_begin,
                     const int32_t *level, const uint64_t *skeys,
                     const float *mn, double S, double *centre, double *side)
{
    for (int64_t c = 0; c < ncells; c++)
        cell_cube(skeys[body_begin[c]], level[c], mn, S, centre + 3 * c, side + c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sect. 3: the tree also serves neighbour search and smoothed particle     */
/* hydrodynamics.  The plain definitions, O(N^2).                           */
/* ------------------------------------------------------------------------ */

/* Cubic spline kernel of compact support h in three dimensions (Monaghan &
 * Lattanzio 1985, written with q = r/h): W = 8/(pi h^3) (1 - 6q^2 + 6q^3)
 * for q <= 1/2, 8/(pi h^3) 2 (1 - q)^3 for 1/2 < q <= 1, 0 beyond. */
double oracle_sph_kernel(double r, double h)
{
    const double pi = 3.14159265358979323846;
    double q = r / h, s = 8.0 / (pi * h * h * h);
    if (q <= 0.5) return s * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    if (q <= 1.0) { double t = 1.0 - q; return s * 2.0 * t * t * t; }
    return 0.0;
}

/* For every body i: the neighbours are the bodies j (i included) with
 * r^2 < h_i^2, decided in float32 as the GPU decides it (dx = x_j - x_i
 * rounded, r^2 = fma(dz, dz, fma(dy, dy, dx * dx)), h_i^2 rounded); the
 * density is rho_i = sum over the neighbours of m_j W(r_ij, h_i) in float64
 * with r_ij from the float32 positions.  targets (may be NULL: every body):
 * the bodies i computed, outputs in that order. */
int oracle_sph_density(const float *pos, const float *mass, const float *h, int64_t n,
                       const int64_t *targets, int64_t ntar, double *rho, int32_t *nngb)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < ntar; t++) {
        const int64_t i = targets ? targets[t] : t;
        float xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        float h2 = h[i] * h[i];
        double r = 0.0;
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; j++) {
            float dx = pos[3 * j] - xi, dy = pos[3 * j + 1] - yi, dz = pos[3 * j + 2] - zi;
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (!(r2 < h2)) continue;
            double ex = (double)pos[3 * j] - xi, ey = (double)pos[3 * j + 1] - yi, ez = (double)pos[3 * j + 2] - zi;
            r += (double)mass[j] * oracle_sph_kernel(sqrt(ex * ex + ey * ey + ez * ez), (double)h[i]);
            cnt++;
        }
        rho[t] = r;
        nngb[t] = cnt;
    }
    return 0;
}
