/*
 * oracle.c -- the plain, slow CPU oracle of grain-pair seeded straight-line
 * track finding in one emulsion view.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA implementation, and neither imports the other.
 *
 * What it computes, in the order of the paper's Section 2 (tracking algorithm,
 * Fig. 4), with exact integer arithmetic everywhere except the final fit:
 *
 *  0. rank(i): position of grain i in lexicographic (x, y, z) order.  It fixes
 *     a canonical order that does not depend on the input order.
 *  1. Seeds (Section 2, Fig. 4a): every unordered grain pair {a, b} whose
 *     separation lies in the window  seed_min^2 <= |g_b - g_a|^2 < seed_max^2,
 *     in any direction (4 pi).  The pair is oriented lo = lower rank.
 *  2. Count along the seed line (Section 2, Fig. 4b): the number of grains k of
 *     the whole view with  |(g_k - g_lo) x (g_hi - g_lo)|^2 <= r^2 |g_hi - g_lo|^2,
 *     i.e. within distance r of the infinite line; the seed grains count.
 *  3. Threshold (Section 2): seeds with count >= min_hits are candidates.
 *  4. Exclusive association (Section 2): candidates are visited in the order
 *     (count descending, rank lo ascending, rank hi ascending).  A candidate's
 *     unused tube grains U are collected; it becomes a track iff |U| >= min_hits
 *     (the threshold applied again), and then the grains of U are used.
 *  5. Fit (not described in the paper): the orthogonal least-squares line of U
 *     in FP64 -- centroid, principal eigenvector of the scatter matrix by the
 *     cyclic Jacobi method (Golub & Van Loan, Matrix Computations, Sec. 8.5),
 *     oriented so that it points from the lo seed grain towards the hi one --
 *     and the range [tmin, tmax] of member projections, the segment's start
 *     and end (Section 2, Fig. 3).
 *
 * Grains are binned in a uniform 3D cell hash, as the paper's implementation
 * does (Section 3, footnote on 3D hash tables), so that seeds and tubes visit
 * only the relevant cells.  The cell cover of a tube is derived in exact
 * integer arithmetic and contains the whole tube (see tube_scan).  The
 * function or_count_pairs_brute() evaluates step 2 over all grains with no
 * hash at all.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

enum { OR_OK = 0, OR_ERR_INVALID_ARG = -1, OR_ERR_OUT_OF_RANGE = -2, OR_ERR_DUPLICATE = -3,
       OR_ERR_OOM = -6 };

/* Variants (flags): OR_SINGLE_PASS -- every grain goes to the best candidate
 * (candidate order) whose tube holds it, a candidate is a track iff at least
 * min_hits grains went to it; OR_ANGLE_CUT -- a track is kept iff
 * nhits >= cut_base + cut_slope * min(tan theta, cut_tan_max), theta the angle
 * of its seed vector to the z axis (the grain-count cut of Section 3, Fig. 9c). */
enum { OR_SINGLE_PASS = 1, OR_ANGLE_CUT = 2 };

typedef struct {
    int32_t extent[3];
    int32_t seed_min, seed_max;
    int32_t tube_r;
    int32_t min_hits;
    uint32_t flags;
    int32_t cut_base, cut_slope, cut_tan_max, reserved;
} or_params;

typedef struct {
    int64_t n;
    int32_t *xyz;          /* copy of the grains, n x 3 */
    or_params p;
    int32_t cs[3];         /* cell edge per axis */
    int32_t nc[3];         /* cells per axis */
    int64_t ncell;
    int64_t *cell_start;   /* ncell + 1 */
    int32_t *cell_items;   /* grain ids grouped by cell */
    int32_t *rank;         /* rank[i] in lexicographic order */
} or_ctx;

typedef struct {
    int64_t n_seeds, n_cand, n_tracks, tests;
    int32_t *lo, *hi, *nhits;   /* seed grains (input ids) and member count */
    int64_t *moff;              /* n_tracks + 1 offsets into members */
    int32_t *members;           /* input ids, ascending within a track */
    double *c, *u, *t, *lam;    /* 3, 3, 2, 3 per track */
} or_tracks;

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}
static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }
static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------ set-up */

static const or_ctx *g_sort_ctx;
static int cmp_lex(const void *pa, const void *pb) {
    const int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    const int32_t *ga = g_sort_ctx->xyz + 3 * (int64_t)a, *gb = g_sort_ctx->xyz + 3 * (int64_t)b;
    for (int k = 0; k < 3; ++k) {
        if (ga[k] < gb[k]) return -1;
        if (ga[k] > gb[k]) return 1;
    }
    return 0;
}

void or_destroy(or_ctx *c) {
    if (!c) return;
    free(c->xyz); free(c->cell_start); free(c->cell_items); free(c->rank);
    free(c);
}

/* cell[3]: the hash cell edge per axis in coordinate units (> 0). */
or_ctx *or_create(const int32_t *xyz, int64_t n, const or_params *p, const int32_t cell[3],
                  int32_t *status) {
    *status = OR_OK;
    if (n < 0 || !p || !cell || (n > 0 && !xyz)) { *status = OR_ERR_INVALID_ARG; return NULL; }
    for (int k = 0; k < 3; ++k)
        if (p->extent[k] <= 0 || p->extent[k] > (1 << 30) || cell[k] <= 0) {
            *status = OR_ERR_INVALID_ARG; return NULL;
        }
    if (p->seed_min < 0 || p->seed_max < p->seed_min || p->tube_r < 0 || p->tube_r > (1 << 30) ||
        p->min_hits < 1 || (p->flags & ~(uint32_t)(OR_SINGLE_PASS | OR_ANGLE_CUT)) ||
        ((p->flags & OR_ANGLE_CUT) && (p->cut_base < 0 || p->cut_slope < 0 || p->cut_tan_max < 0))) {
        *status = OR_ERR_INVALID_ARG; return NULL;
    }
    if (n > 2147483647LL) { *status = OR_ERR_INVALID_ARG; return NULL; }
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    if (!c) { *status = OR_ERR_OOM; return NULL; }
    c->n = n;
    c->p = *p;
    c->xyz = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    c->rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!c->xyz || !c->rank) { or_destroy(c); *status = OR_ERR_OOM; return NULL; }
    if (n > 0) memcpy(c->xyz, xyz, sizeof(int32_t) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k)
            if (c->xyz[3 * i + k] < 0 || c->xyz[3 * i + k] >= p->extent[k]) {
                or_destroy(c); *status = OR_ERR_OUT_OF_RANGE; return NULL;
            }
    /* step 0: canonical rank, lexicographic (x, y, z) */
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!order) { or_destroy(c); *status = OR_ERR_OOM; return NULL; }
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    g_sort_ctx = c;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_lex);
    for (int64_t r = 0; r < n; ++r) c->rank[order[r]] = (int32_t)r;
    for (int64_t r = 1; r < n; ++r)
        if (cmp_lex(&order[r - 1], &order[r]) == 0) {
            free(order); or_destroy(c); *status = OR_ERR_DUPLICATE; return NULL;
        }
    free(order);
    /* uniform cell hash */
    c->ncell = 1;
    for (int k = 0; k < 3; ++k) {
        c->cs[k] = cell[k];
        c->nc[k] = (int32_t)ceil_div(p->extent[k], cell[k]);
        c->ncell *= c->nc[k];
    }
    c->cell_start = (int64_t *)calloc((size_t)c->ncell + 1, sizeof(int64_t));
    c->cell_items = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!c->cell_start || !c->cell_items) { or_destroy(c); *status = OR_ERR_OOM; return NULL; }
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cid) { or_destroy(c); *status = OR_ERR_OOM; return NULL; }
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *g = c->xyz + 3 * i;
        int64_t ix = g[0] / c->cs[0], iy = g[1] / c->cs[1], iz = g[2] / c->cs[2];
        cid[i] = ix + (int64_t)c->nc[0] * (iy + (int64_t)c->nc[1] * iz);
        c->cell_start[cid[i] + 1] += 1;
    }
    for (int64_t q = 0; q < c->ncell; ++q) c->cell_start[q + 1] += c->cell_start[q];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)c->ncell);
    if (!fill) { free(cid); or_destroy(c); *status = OR_ERR_OOM; return NULL; }
    memcpy(fill, c->cell_start, sizeof(int64_t) * (size_t)c->ncell);
    for (int64_t i = 0; i < n; ++i) c->cell_items[fill[cid[i]]++] = (int32_t)i;
    free(fill);
    free(cid);
    return c;
}

int32_t or_rank(const or_ctx *c, int32_t i) { return c->rank[i]; }

static int64_t cell_index(const or_ctx *c, int64_t ix, int64_t iy, int64_t iz) {
    return ix + (int64_t)c->nc[0] * (iy + (int64_t)c->nc[1] * iz);
}

/* ------------------------------------------------------------ step 1: seeds */

static int in_window(const or_ctx *c, int32_t a, int32_t b) {
    const int32_t *ga = c->xyz + 3 * (int64_t)a, *gb = c->xyz + 3 * (int64_t)b;
    int64_t d2 = 0;
    for (int k = 0; k < 3; ++k) {
        int64_t d = (int64_t)gb[k] - ga[k];
        d2 += d * d;
    }
    return d2 >= (int64_t)c->p.seed_min * c->p.seed_min && d2 < (int64_t)c->p.seed_max * c->p.seed_max;
}

/* Visit the seeds whose lo grain is a: partners b of higher rank in the window,
   found in the cells within seed_max - 1 of g_a along every axis. */
static int64_t seeds_of(const or_ctx *c, int32_t a, int32_t *out_b, int64_t cap) {
    if (c->p.seed_max <= 0) return 0;
    const int32_t *ga = c->xyz + 3 * (int64_t)a;
    int64_t lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = clampi(floor_div((int64_t)ga[k] - (c->p.seed_max - 1), c->cs[k]), 0, c->nc[k] - 1);
        hi[k] = clampi(floor_div((int64_t)ga[k] + (c->p.seed_max - 1), c->cs[k]), 0, c->nc[k] - 1);
    }
    int64_t m = 0;
    for (int64_t iz = lo[2]; iz <= hi[2]; ++iz)
        for (int64_t iy = lo[1]; iy <= hi[1]; ++iy)
            for (int64_t ix = lo[0]; ix <= hi[0]; ++ix) {
                int64_t q = cell_index(c, ix, iy, iz);
                for (int64_t s = c->cell_start[q]; s < c->cell_start[q + 1]; ++s) {
                    int32_t b = c->cell_items[s];
                    if (c->rank[b] > c->rank[a] && in_window(c, a, b)) {
                        if (out_b && m < cap) out_b[m] = b;
                        ++m;
                    }
                }
            }
    return m;
}

typedef struct { int32_t lo, hi, rlo, rhi, count; } seed_rec;

static int cmp_seed_rank(const void *pa, const void *pb) {
    const seed_rec *a = (const seed_rec *)pa, *b = (const seed_rec *)pb;
    if (a->rlo != b->rlo) return a->rlo < b->rlo ? -1 : 1;
    if (a->rhi != b->rhi) return a->rhi < b->rhi ? -1 : 1;
    return 0;
}

/* All seeds, ordered by (rank lo, rank hi).  Returns NULL on OOM. */
static seed_rec *all_seeds(const or_ctx *c, int64_t *n_out) {
    int64_t total = 0;
    int64_t *per = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->n + 1));
    if (!per) return NULL;
    for (int64_t a = 0; a < c->n; ++a) { per[a] = seeds_of(c, (int32_t)a, NULL, 0); total += per[a]; }
    seed_rec *s = (seed_rec *)malloc(sizeof(seed_rec) * (size_t)(total > 0 ? total : 1));
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c->n > 0 ? c->n : 1));
    if (!s || !buf) { free(per); free(s); free(buf); return NULL; }
    int64_t m = 0;
    for (int64_t a = 0; a < c->n; ++a) {
        int64_t k = seeds_of(c, (int32_t)a, buf, c->n);
        for (int64_t j = 0; j < k; ++j) {
            s[m].lo = (int32_t)a; s[m].hi = buf[j];
            s[m].rlo = c->rank[a]; s[m].rhi = c->rank[buf[j]]; s[m].count = 0;
            ++m;
        }
    }
    free(per); free(buf);
    qsort(s, (size_t)m, sizeof(seed_rec), cmp_seed_rank);
    *n_out = m;
    return s;
}

int64_t or_seed_total(const or_ctx *c) {
    int64_t total = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : total)
#endif
    for (int64_t a = 0; a < c->n; ++a) total += seeds_of(c, (int32_t)a, NULL, 0);
    return total;
}

/* Number of seeds whose lo grain is each grain (input ids); returns the total. */
int64_t or_seeds_per_grain(const or_ctx *c, int64_t *out) {
    int64_t total = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : total)
#endif
    for (int64_t a = 0; a < c->n; ++a) {
        out[a] = seeds_of(c, (int32_t)a, NULL, 0);
        total += out[a];
    }
    return total;
}

/* Writes up to cap seeds (input ids, lo = lower rank) ordered by (rank lo,
   rank hi); returns the total number of seeds, or -1 on OOM. */
int64_t or_list_seeds(const or_ctx *c, int32_t *lo, int32_t *hi, int64_t cap) {
    int64_t m = 0;
    seed_rec *s = all_seeds(c, &m);
    if (!s) return -1;
    for (int64_t i = 0; i < m && i < cap; ++i) { lo[i] = s[i].lo; hi[i] = s[i].hi; }
    free(s);
    return m;
}

/* ------------------------------------------------------------ step 2: tube */

/* Exact membership: |(g_k - g_a) x w|^2 <= r^2 |w|^2 with w = g_b - g_a. */
static int in_tube(const int32_t *gk, const int32_t *ga, const int64_t w[3], i128 rhs) {
    int64_t d0 = (int64_t)gk[0] - ga[0], d1 = (int64_t)gk[1] - ga[1], d2 = (int64_t)gk[2] - ga[2];
    i128 c0 = (i128)d1 * w[2] - (i128)d2 * w[1];
    i128 c1 = (i128)d2 * w[0] - (i128)d0 * w[2];
    i128 c2 = (i128)d0 * w[1] - (i128)d1 * w[0];
    return c0 * c0 + c1 * c1 + c2 * c2 <= rhs;
}

/* Range of a coordinate e over the line's foot points whose d-coordinate lies
   in [D0, D1], widened by r:  e(D) = a_e + (D - a_d) w_e / w_d  is monotone in D,
   so its extremes sit at D0 and D1.  Bounds are rounded outwards. */
static void cover_range(int64_t a_e, int64_t a_d, int64_t w_e, int64_t w_d, int64_t D0, int64_t D1,
                        int64_t r, int64_t *lo, int64_t *hi) {
    int64_t n0 = (D0 - a_d) * w_e, n1 = (D1 - a_d) * w_e, den = w_d;
    if (den < 0) { n0 = -n0; n1 = -n1; den = -den; }
    int64_t mn = n0 < n1 ? n0 : n1, mx = n0 < n1 ? n1 : n0;
    *lo = a_e + floor_div(mn, den) - r;
    *hi = a_e + ceil_div(mx, den) + r;
}

/*
 * Count the grains within distance r of the line through g_a and g_b; write
 * their ids to out (if non-NULL, at most cap of them).
 *
 * Cover.  Let d be an axis with the largest |w_d| (so w_d != 0).  The cells are
 * walked one slab of constant d-cell index at a time.  A grain p inside the
 * tube has a foot point q on the line with |p - q| <= r, hence |p_x - q_x| <= r
 * on every axis x.  For p in slab k (k s_d <= p_d <= min((k+1) s_d, E_d) - 1),
 * q_d lies in [k s_d - r, min((k+1) s_d, E_d) - 1 + r]; along the line the other
 * two coordinates of q are linear in q_d, so p_e lies within r of their range
 * over that interval (cover_range).  Every cell of the slab meeting those
 * ranges is visited once, and the exact test decides.
 */
static int64_t tube_scan(const or_ctx *c, int32_t a, int32_t b, int32_t *out, int64_t cap,
                         int64_t *tests) {
    const int32_t *ga = c->xyz + 3 * (int64_t)a, *gb = c->xyz + 3 * (int64_t)b;
    int64_t w[3] = {(int64_t)gb[0] - ga[0], (int64_t)gb[1] - ga[1], (int64_t)gb[2] - ga[2]};
    const int64_t r = c->p.tube_r;
    i128 rhs = (i128)r * r * (i128)(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    int d = 0;
    for (int k = 1; k < 3; ++k) {
        int64_t ak = w[k] < 0 ? -w[k] : w[k], ad = w[d] < 0 ? -w[d] : w[d];
        if (ak > ad) d = k;
    }
    if (w[d] == 0) return 0; /* a == b: not a seed */
    const int e = (d + 1) % 3, f = (d + 2) % 3;
    int64_t count = 0, ntest = 0;
    for (int64_t k = 0; k < c->nc[d]; ++k) {
        int64_t p_lo = k * c->cs[d];
        int64_t p_hi = (k + 1) * (int64_t)c->cs[d];
        if (p_hi > c->p.extent[d]) p_hi = c->p.extent[d];
        p_hi -= 1;
        int64_t D0 = p_lo - r, D1 = p_hi + r;
        int64_t elo, ehi, flo, fhi;
        cover_range(ga[e], ga[d], w[e], w[d], D0, D1, r, &elo, &ehi);
        cover_range(ga[f], ga[d], w[f], w[d], D0, D1, r, &flo, &fhi);
        if (ehi < 0 || elo > c->p.extent[e] - 1 || fhi < 0 || flo > c->p.extent[f] - 1) continue;
        int64_t ce0 = clampi(floor_div(elo, c->cs[e]), 0, c->nc[e] - 1);
        int64_t ce1 = clampi(floor_div(ehi, c->cs[e]), 0, c->nc[e] - 1);
        int64_t cf0 = clampi(floor_div(flo, c->cs[f]), 0, c->nc[f] - 1);
        int64_t cf1 = clampi(floor_div(fhi, c->cs[f]), 0, c->nc[f] - 1);
        for (int64_t ce = ce0; ce <= ce1; ++ce)
            for (int64_t cf = cf0; cf <= cf1; ++cf) {
                int64_t idx[3];
                idx[d] = k; idx[e] = ce; idx[f] = cf;
                int64_t q = cell_index(c, idx[0], idx[1], idx[2]);
                for (int64_t s = c->cell_start[q]; s < c->cell_start[q + 1]; ++s) {
                    int32_t g = c->cell_items[s];
                    ++ntest;
                    if (in_tube(c->xyz + 3 * (int64_t)g, ga, w, rhs)) {
                        if (out && count < cap) out[count] = g;
                        ++count;
                    }
                }
            }
    }
    if (tests) *tests += ntest;
    return count;
}

static int cmp_i32(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Tube members of the seed (a, b), ascending; returns the count (may exceed cap). */
int64_t or_tube_members(const or_ctx *c, int32_t a, int32_t b, int32_t *out, int64_t cap) {
    int64_t m = tube_scan(c, a, b, out, cap, NULL);
    if (out) qsort(out, (size_t)(m < cap ? m : cap), sizeof(int32_t), cmp_i32);
    return m;
}

/* Step 2 with the cell hash, for the given pairs (any orientation). */
void or_count_pairs(const or_ctx *c, const int32_t *a, const int32_t *b, int64_t n, int32_t *counts,
                    int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n; ++s) counts[s] = (int32_t)tube_scan(c, a[s], b[s], NULL, 0, NULL);
    (void)nthreads;
}

/* Step 2 straight from the definition: every grain of the view is tested. */
void or_count_pairs_brute(const or_ctx *c, const int32_t *a, const int32_t *b, int64_t n,
                          int32_t *counts, int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n; ++s) {
        const int32_t *ga = c->xyz + 3 * (int64_t)a[s], *gb = c->xyz + 3 * (int64_t)b[s];
        int64_t w[3] = {(int64_t)gb[0] - ga[0], (int64_t)gb[1] - ga[1], (int64_t)gb[2] - ga[2]};
        i128 rhs = (i128)c->p.tube_r * c->p.tube_r * (i128)(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        int32_t m = 0;
        for (int64_t k = 0; k < c->n; ++k) m += in_tube(c->xyz + 3 * k, ga, w, rhs);
        counts[s] = m;
    }
    (void)nthreads;
}

/* ------------------------------------------------------------ step 5: fit */

/* Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
   (Golub & Van Loan, Sec. 8.5): each rotation in the (p, q) plane is the 2x2
   symmetric Schur decomposition that zeroes A[p][q]; sweeps repeat until the
   off-diagonal mass is negligible.  Columns of V are the eigenvectors. */
static void jacobi3(double A[3][3], double V[3][3]) {
    static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-34 * diag) break;
        for (int m = 0; m < 3; ++m) {
            int p = P[m], q = Q[m];
            if (A[p][q] == 0.0) continue;
            double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
            for (int k = 0; k < 3; ++k) { /* A <- A J */
                double akp = A[k][p], akq = A[k][q];
                A[k][p] = cs * akp - sn * akq;
                A[k][q] = sn * akp + cs * akq;
            }
            for (int k = 0; k < 3; ++k) { /* A <- J^T A */
                double apk = A[p][k], aqk = A[q][k];
                A[p][k] = cs * apk - sn * aqk;
                A[q][k] = sn * apk + cs * aqk;
            }
            for (int k = 0; k < 3; ++k) { /* V <- V J */
                double vkp = V[k][p], vkq = V[k][q];
                V[k][p] = cs * vkp - sn * vkq;
                V[k][q] = sn * vkp + cs * vkq;
            }
        }
    }
}

/* Exposed for the tests: eigenvalues (descending) and matching eigenvectors
   (rows of vec) of a symmetric 3x3 matrix given row-major. */
void or_sym_eigen3(const double *m, double *lam, double *vec) {
    double A[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = m[3 * i + j];
    jacobi3(A, V);
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (A[idx[j]][idx[j]] > A[idx[i]][idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < 3; ++i) {
        lam[i] = A[idx[i]][idx[i]];
        for (int k = 0; k < 3; ++k) vec[3 * i + k] = V[k][idx[i]];
    }
}

static void fit_line(const or_ctx *c, const int32_t *mem, int64_t n, int32_t lo, int32_t hi,
                     double *cen, double *u, double *t, double *lam) {
    double s[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) s[k] += c->xyz[3 * (int64_t)mem[i] + k];
    for (int k = 0; k < 3; ++k) cen[k] = s[k] / (double)n;
    double M[9] = {0};
    for (int64_t i = 0; i < n; ++i) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = c->xyz[3 * (int64_t)mem[i] + k] - cen[k];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[3 * a + b] += d[a] * d[b];
    }
    double vec[9];
    or_sym_eigen3(M, lam, vec);
    for (int k = 0; k < 3; ++k) u[k] = vec[k];
    double nrm = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int k = 0; k < 3; ++k) u[k] /= nrm;
    /* orientation: along the seed, from its lo grain to its hi grain */
    double dot = 0;
    for (int k = 0; k < 3; ++k) dot += u[k] * ((double)c->xyz[3 * (int64_t)hi + k] - c->xyz[3 * (int64_t)lo + k]);
    int flip = dot < 0;
    if (dot == 0) {
        for (int k = 0; k < 3; ++k)
            if (u[k] != 0) { flip = u[k] < 0; break; }
    }
    if (flip)
        for (int k = 0; k < 3; ++k) u[k] = -u[k];
    double tmin = INFINITY, tmax = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double v = 0;
        for (int k = 0; k < 3; ++k) v += (c->xyz[3 * (int64_t)mem[i] + k] - cen[k]) * u[k];
        if (v < tmin) tmin = v;
        if (v > tmax) tmax = v;
    }
    t[0] = tmin; t[1] = tmax;
}

/* ------------------------------------------------------------ steps 3-5 */

static int cmp_cand(const void *pa, const void *pb) {
    const seed_rec *a = (const seed_rec *)pa, *b = (const seed_rec *)pb;
    if (a->count != b->count) return a->count > b->count ? -1 : 1;   /* count descending */
    if (a->rlo != b->rlo) return a->rlo < b->rlo ? -1 : 1;             /* rank lo ascending */
    if (a->rhi != b->rhi) return a->rhi < b->rhi ? -1 : 1;             /* rank hi ascending */
    return 0;
}

void or_tracks_free(or_tracks *t) {
    if (!t) return;
    free(t->lo); free(t->hi); free(t->nhits); free(t->moff); free(t->members);
    free(t->c); free(t->u); free(t->t); free(t->lam);
    memset(t, 0, sizeof(*t));
}

/* The whole method.  Seeds and counts may optionally be returned (keep_seeds):
   then seed_lo/seed_hi/seed_count receive n_seeds entries ordered by (rank lo,
   rank hi) and must be freed with free(). */
/* The grain-count cut (Section 3, Fig. 9c) as the plain inequality
 * nhits >= cut_base + cut_slope * min(tan theta, cut_tan_max) with
 * tan theta = sqrt(wx^2 + wy^2) / |wz| for the seed vector w = g_hi - g_lo,
 * decided exactly: squares of non-negative sides compared in 128 bits. */
static int angle_cut_keeps(const or_ctx *c, int32_t lo, int32_t hi, int64_t nhits) {
    const int32_t *a = c->xyz + 3 * (int64_t)lo, *b = c->xyz + 3 * (int64_t)hi;
    const i128 wx = b[0] - a[0], wy = b[1] - a[1], wz = b[2] - a[2];
    const i128 t2 = wx * wx + wy * wy, z2 = wz * wz;        /* tan^2 theta = t2 / z2 */
    const i128 need = (i128)nhits - c->p.cut_base;          /* must reach cut_slope * min(tan, tmax) */
    if (need < 0) return 0;
    const i128 tm = c->p.cut_tan_max, sl = c->p.cut_slope;
    if (t2 >= tm * tm * z2) return need >= sl * tm;          /* tan theta >= tmax (or wz = 0) */
    return need * need * z2 >= sl * sl * t2;                /* need >= sl * sqrt(t2 / z2) */
}

int or_find_tracks(const or_ctx *c, int nthreads, or_tracks *out, int keep_seeds, int32_t **seed_lo,
                   int32_t **seed_hi, int32_t **seed_count) {
    memset(out, 0, sizeof(*out));
    int64_t ns = 0;
    seed_rec *s = all_seeds(c, &ns);
    if (!s) return OR_ERR_OOM;
    out->n_seeds = ns;
    int64_t tests = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads) reduction(+ : tests)
#endif
    for (int64_t i = 0; i < ns; ++i) s[i].count = (int32_t)tube_scan(c, s[i].lo, s[i].hi, NULL, 0, &tests);
    out->tests = tests;
    if (keep_seeds) {
        *seed_lo = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
        *seed_hi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
        *seed_count = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
        if (!*seed_lo || !*seed_hi || !*seed_count) { free(s); return OR_ERR_OOM; }
        for (int64_t i = 0; i < ns; ++i) {
            (*seed_lo)[i] = s[i].lo; (*seed_hi)[i] = s[i].hi; (*seed_count)[i] = s[i].count;
        }
    }
    /* step 3: threshold */
    int64_t nc = 0;
    for (int64_t i = 0; i < ns; ++i)
        if (s[i].count >= c->p.min_hits) s[nc++] = s[i];
    out->n_cand = nc;
    /* step 4: canonical order, then sequential exclusive association */
    qsort(s, (size_t)nc, sizeof(seed_rec), cmp_cand);
    unsigned char *used = (unsigned char *)calloc((size_t)(c->n > 0 ? c->n : 1), 1);
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c->n > 0 ? c->n : 1));
    int64_t tcap = 16, mcap = 256;
    out->lo = (int32_t *)malloc(sizeof(int32_t) * tcap);
    out->hi = (int32_t *)malloc(sizeof(int32_t) * tcap);
    out->nhits = (int32_t *)malloc(sizeof(int32_t) * tcap);
    out->moff = (int64_t *)malloc(sizeof(int64_t) * (tcap + 1));
    out->members = (int32_t *)malloc(sizeof(int32_t) * mcap);
    if (!used || !buf || !out->lo || !out->hi || !out->nhits || !out->moff || !out->members) {
        free(s); free(used); free(buf); or_tracks_free(out); return OR_ERR_OOM;
    }
    out->moff[0] = 0;
    int64_t nt = 0, nm = 0;
    /* single pass: first[g] = position (candidate order) of the first candidate
     * whose tube holds grain g, or nc */
    int64_t *first = NULL;
    if (c->p.flags & OR_SINGLE_PASS) {
        first = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->n > 0 ? c->n : 1));
        if (!first) { free(s); free(used); free(buf); or_tracks_free(out); return OR_ERR_OOM; }
        for (int64_t g = 0; g < c->n; ++g) first[g] = nc;
        for (int64_t i = 0; i < nc; ++i) {
            int64_t m = tube_scan(c, s[i].lo, s[i].hi, buf, c->n, NULL);
            for (int64_t j = 0; j < m; ++j)
                if (first[buf[j]] > i) first[buf[j]] = i;
        }
    }
    for (int64_t i = 0; i < nc; ++i) {
        int64_t m = tube_scan(c, s[i].lo, s[i].hi, buf, c->n, NULL);
        int64_t u = 0;
        if (first) {   /* the grains that chose this candidate */
            for (int64_t j = 0; j < m; ++j)
                if (first[buf[j]] == i) buf[u++] = buf[j];
            if (u < c->p.min_hits) continue;
        } else {       /* sequential greedy: the grains no earlier track took */
            for (int64_t j = 0; j < m; ++j)
                if (!used[buf[j]]) buf[u++] = buf[j];
            if (u < c->p.min_hits) continue;
            for (int64_t j = 0; j < u; ++j) used[buf[j]] = 1;
        }
        if ((c->p.flags & OR_ANGLE_CUT) && !angle_cut_keeps(c, s[i].lo, s[i].hi, u)) continue;
        qsort(buf, (size_t)u, sizeof(int32_t), cmp_i32);
        if (nt + 1 >= tcap) {
            tcap *= 2;
            out->lo = (int32_t *)realloc(out->lo, sizeof(int32_t) * tcap);
            out->hi = (int32_t *)realloc(out->hi, sizeof(int32_t) * tcap);
            out->nhits = (int32_t *)realloc(out->nhits, sizeof(int32_t) * tcap);
            out->moff = (int64_t *)realloc(out->moff, sizeof(int64_t) * (tcap + 1));
        }
        while (nm + u > mcap) {
            mcap *= 2;
            out->members = (int32_t *)realloc(out->members, sizeof(int32_t) * mcap);
        }
        if (!out->lo || !out->hi || !out->nhits || !out->moff || !out->members) {
            free(s); free(used); free(buf); free(first); or_tracks_free(out); return OR_ERR_OOM;
        }
        out->lo[nt] = s[i].lo; out->hi[nt] = s[i].hi; out->nhits[nt] = (int32_t)u;
        memcpy(out->members + nm, buf, sizeof(int32_t) * (size_t)u);
        nm += u;
        out->moff[++nt] = nm;
    }
    free(first);
    out->n_tracks = nt;
    free(s); free(used); free(buf);
    /* step 5: fit */
    out->c = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    out->u = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    out->t = (double *)malloc(sizeof(double) * 2 * (size_t)(nt > 0 ? nt : 1));
    out->lam = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    if (!out->c || !out->u || !out->t || !out->lam) { or_tracks_free(out); return OR_ERR_OOM; }
    for (int64_t k = 0; k < nt; ++k)
        fit_line(c, out->members + out->moff[k], out->moff[k + 1] - out->moff[k], out->lo[k], out->hi[k],
                 out->c + 3 * k, out->u + 3 * k, out->t + 2 * k, out->lam + 3 * k);
    return OR_OK;
}

/* Fit of an arbitrary member set (input ids), for the tests. */
void or_fit(const or_ctx *c, const int32_t *mem, int64_t n, int32_t lo, int32_t hi, double *cen,
            double *u, double *t, double *lam) {
    fit_line(c, mem, n, lo, hi, cen, u, t, lam);
}

int or_abi_version(void) { return 1; }
