/*
 * rsi_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of what the ray-segment /
 * surface intersection method computes.  It exists so that tests, the
 * smoke check and the CPU-baseline leg of the benchmark have something to
 * compare the CUDA path against.  Nothing in the product path may call it,
 * and it shares no code, header, table or helper with the CUDA library.
 *
 * Contents (each function cites the passage it restates):
 *   - oracle_classify_pair : FP64 Moller-Trumbore segment/triangle test
 *                            (Sec. 1, the Moller-Trumbore reference; Epilogue
 *                            on FP32 vs FP64) with the margin classification
 *                            decisive-hit / decisive-miss / ambiguous.
 *   - oracle_query         : brute force over all N_r x N_t pairs (Sec. 1:
 *                            the exhaustive search the BVH accelerates), in the
 *                            three result forms of Sec. 1 (boolean,
 *                            intercept_count, and barycentric = the nearest
 *                            hit's triangle, t, point and distance).
 *   - oracle_extent / oracle_morton : surface extent and 30/63-bit Morton
 *                            codes of triangle centroids (Sec. 3.2, Sec. 3.3).
 *   - oracle_sort          : stable sort of (key, triangle id) (Sec. 3.2).
 *   - oracle_radix_tree    : binary radix tree over sorted keys, by its
 *                            definition (Sec. 1 cites Karras 2012), indexed
 *                            Karras-style.
 *   - oracle_refit         : bounding boxes of every node (Sec. 4.1, 4.2).
 *
 * Floating point: the query is FP64 (inputs are FP32 and converted exactly).
 * The Morton codes are FP32 round-to-nearest like the method itself (the
 * paper's implementation is entirely 32-bit float, Epilogue), because the
 * code is an integer decided by floating point.  Build with
 * -ffp-contract=off so no multiply-add is fused on any host.
 *
 * Parity status: every function here is pinned by the CPU tests (worked
 * example of Sec. 4.1, closed-box parity, exact rational predicates, a
 * second independent tree construction, library sorts).  The de-duplication
 * of crossing points on ambiguous rays (intercept_count, Sec. 1 "unique
 * intersections") is pinned by convexity where several triangles report one
 * point (a shared vertex or edge of a closed box: one crossing); the merge
 * distance for distinct but close points (1e-9 in t) has no rule in the
 * paper: parity unpinned for that distance.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_TAU 1e-6       /* relative margin of the ambiguity band      */
#define ORACLE_TMERGE 1e-9    /* crossing points closer than this are one   */

enum { PAIR_MISS = 0, PAIR_HIT = 1, PAIR_AMBIGUOUS = 2 };

typedef struct { double x, y, z; } vec3;

static vec3 v_load(const float* p) { vec3 r = {(double)p[0], (double)p[1], (double)p[2]}; return r; }
static vec3 v_sub(vec3 a, vec3 b) { vec3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static vec3 v_add(vec3 a, vec3 b) { vec3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static vec3 v_scale(vec3 a, double s) { vec3 r = {a.x * s, a.y * s, a.z * s}; return r; }
static double v_dot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 v_cross(vec3 a, vec3 b) {
    vec3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}
static double v_norm(vec3 a) { return sqrt(v_dot(a, a)); }
static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Distance from point p to the segment [a, b]. */
static double point_segment_distance(vec3 p, vec3 a, vec3 b) {
    vec3 ab = v_sub(b, a);
    double len2 = v_dot(ab, ab);
    double t = len2 > 0.0 ? clamp01(v_dot(v_sub(p, a), ab) / len2) : 0.0;
    return v_norm(v_sub(p, v_add(a, v_scale(ab, t))));
}

/* Distance between segments [p0,p1] and [q0,q1]: |p0 + s u - q0 - t v| is a
 * convex quadratic on the unit square, so its minimum is the interior
 * critical point (when the lines are not parallel and it lies inside) or on
 * one of the four sides, each side being a point-to-segment distance. */
static double segment_segment_distance(vec3 p0, vec3 p1, vec3 q0, vec3 q1) {
    double best = point_segment_distance(p0, q0, q1);
    double d;
    d = point_segment_distance(p1, q0, q1); if (d < best) best = d;
    d = point_segment_distance(q0, p0, p1); if (d < best) best = d;
    d = point_segment_distance(q1, p0, p1); if (d < best) best = d;
    vec3 u = v_sub(p1, p0), v = v_sub(q1, q0), w0 = v_sub(p0, q0);
    double a = v_dot(u, u), b = v_dot(u, v), c = v_dot(v, v);
    double dd = v_dot(u, w0), e = v_dot(v, w0);
    double den = a * c - b * b;
    if (den > 0.0) {
        double s = (b * e - c * dd) / den;
        double t = (a * e - b * dd) / den;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            vec3 diff = v_sub(v_add(w0, v_scale(u, s)), v_scale(v, t));
            d = v_norm(diff);
            if (d < best) best = d;
        }
    }
    return best;
}

/* Distance from point p to the (non-degenerate) triangle a,b,c: the
 * orthogonal projection if it falls inside, else the nearest edge. */
static double point_triangle_distance(vec3 p, vec3 a, vec3 b, vec3 c) {
    vec3 n = v_cross(v_sub(b, a), v_sub(c, a));
    double nn = v_dot(n, n);
    double h = v_dot(v_sub(p, a), n) / nn;           /* signed height / |n| */
    vec3 proj = v_sub(p, v_scale(n, h));
    /* inside test of the projection by the signs of the sub-triangle normals */
    double s0 = v_dot(v_cross(v_sub(b, a), v_sub(proj, a)), n);
    double s1 = v_dot(v_cross(v_sub(c, b), v_sub(proj, b)), n);
    double s2 = v_dot(v_cross(v_sub(a, c), v_sub(proj, c)), n);
    if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) return fabs(h) * sqrt(nn);
    double best = point_segment_distance(p, a, b);
    double d = point_segment_distance(p, b, c); if (d < best) best = d;
    d = point_segment_distance(p, c, a); if (d < best) best = d;
    return best;
}

/*
 * One segment l = (s, e) against one triangle (a, b, c).
 *
 * Moller-Trumbore (Sec. 1, "Moller-Trumbore algorithm"; Epilogue: the
 * intermediate quantities are dot and cross products):
 *   d = e - s, e1 = b - a, e2 = c - a, p = d x e2, det = e1 . p,
 *   sv = s - a, q = sv x e1,
 *   u = (sv . p) / det, v = (d . q) / det, t = (e2 . q) / det, w = 1 - u - v.
 * The segment meets the triangle iff det != 0, u, v, w >= 0 and 0 <= t <= 1
 * (t is the fraction along the segment from its start point to its end point,
 * Sec. 1 defines a ray as the segment between the two).
 *
 * Margin classification with tau = 1e-6 and det_rel = det/(|d||e1||e2|):
 *   decisive hit : |det_rel| > tau and u, v, w > tau and tau < t < 1 - tau
 *   decisive miss: |det_rel| > tau and one of u, v, w, t < -tau or t > 1+tau,
 *                  or |det_rel| <= tau and dist(segment, triangle) > tau |d|
 *   ambiguous    : anything else.
 * A zero-length segment or a triangle whose normal is exactly zero never
 * hits (decisive miss).
 *
 * out[0..6] = u, v, t, det_rel, distance (only on the parallel branch, else
 * -1), inclusive hit (0/1), w.  Returns the class.
 */
int oracle_classify_pair(const float* s_, const float* e_, const float* a_,
                         const float* b_, const float* c_, double* out) {
    vec3 s = v_load(s_), e = v_load(e_), a = v_load(a_), b = v_load(b_), c = v_load(c_);
    vec3 d = v_sub(e, s);
    vec3 e1 = v_sub(b, a), e2 = v_sub(c, a);
    vec3 n = v_cross(e1, e2);
    double u = 0.0, v = 0.0, t = 0.0, w = 0.0, det_rel = 0.0, dist = -1.0;
    int incl = 0, cls;
    if ((d.x == 0.0 && d.y == 0.0 && d.z == 0.0) ||
        (n.x == 0.0 && n.y == 0.0 && n.z == 0.0)) {
        cls = PAIR_MISS;
    } else {
        vec3 p = v_cross(d, e2);
        double det = v_dot(e1, p);
        vec3 sv = v_sub(s, a);
        vec3 q = v_cross(sv, e1);
        det_rel = det / (v_norm(d) * v_norm(e1) * v_norm(e2));
        if (det != 0.0) {
            u = v_dot(sv, p) / det;
            v = v_dot(d, q) / det;
            t = v_dot(e2, q) / det;
            w = 1.0 - u - v;
            incl = (u >= 0.0 && v >= 0.0 && w >= 0.0 && t >= 0.0 && t <= 1.0);
        }
        const double tau = ORACLE_TAU;
        if (fabs(det_rel) > tau) {
            if (u > tau && v > tau && w > tau && t > tau && t < 1.0 - tau)
                cls = PAIR_HIT;
            else if (u < -tau || v < -tau || w < -tau || t < -tau || t > 1.0 + tau)
                cls = PAIR_MISS;
            else
                cls = PAIR_AMBIGUOUS;
        } else {
            /* nearly parallel: decide by the segment-triangle distance, which
             * is 0 when the closed segment meets the closed triangle and is
             * otherwise attained at a segment end point or a triangle edge */
            if (incl) {
                dist = 0.0;
            } else {
                dist = point_triangle_distance(s, a, b, c);
                double dd = point_triangle_distance(e, a, b, c); if (dd < dist) dist = dd;
                dd = segment_segment_distance(s, e, a, b); if (dd < dist) dist = dd;
                dd = segment_segment_distance(s, e, b, c); if (dd < dist) dist = dd;
                dd = segment_segment_distance(s, e, c, a); if (dd < dist) dist = dd;
            }
            cls = dist > tau * v_norm(d) ? PAIR_MISS : PAIR_AMBIGUOUS;
        }
    }
    if (out) {
        out[0] = u; out[1] = v; out[2] = t; out[3] = det_rel;
        out[4] = dist; out[5] = (double)incl; out[6] = w;
    }
    return cls;
}

static int cmp_double(const void* x, const void* y) {
    double a = *(const double*)x, b = *(const double*)y;
    return (a > b) - (a < b);
}

typedef struct {
    const float *V, *from, *to;
    const int32_t* T;
    int64_t nT, r0, r1;
    uint8_t *hit, *amb_hit, *amb_count;
    int32_t *count, *near_tri;
    float *near_t, *near_point, *near_dist;
} query_job;

/* Per ray, over every triangle (the exhaustive search of Sec. 1):
 *  boolean mode   : hit = some decisive hit, else the inclusive result;
 *                   ambiguous iff no decisive hit and some ambiguous pair
 *                   (a decisive hit settles the boolean answer alone).
 *  intercept_count: ambiguous iff some pair is ambiguous; count = number of
 *                   decisive hits, or on an ambiguous ray the number of
 *                   distinct inclusive crossing points (t merged within 1e-9).
 *  nearest hit    : the barycentric mode (Sec. 1: the intersecting triangle,
 *                   the distance to and the location of the nearest
 *                   intersecting point).  Smallest t over the inclusive hits
 *                   (equal t: the lower triangle index), its triangle, the
 *                   point s + t (e - s) and the distance t |e - s| from the
 *                   start point; -1 / NaN when none.  The ray is flagged
 *                   exactly as in intercept_count (some ambiguous pair). */
static void* query_worker(void* arg) {
    query_job* J = (query_job*)arg;
    double* ts = (double*)malloc(sizeof(double) * (size_t)(J->nT > 0 ? J->nT : 1));
    double out[7];
    for (int64_t r = J->r0; r < J->r1; ++r) {
        const float* s = J->from + 3 * r;
        const float* e = J->to + 3 * r;
        int n_hit = 0, n_amb = 0, n_incl = 0;
        double best_t = INFINITY;
        int32_t best_j = -1;
        for (int64_t j = 0; j < J->nT; ++j) {
            const int32_t* tri = J->T + 3 * j;
            int cls = oracle_classify_pair(s, e, J->V + 3 * (int64_t)tri[0], J->V + 3 * (int64_t)tri[1],
                                           J->V + 3 * (int64_t)tri[2], out);
            if (cls == PAIR_HIT) ++n_hit;
            else if (cls == PAIR_AMBIGUOUS) ++n_amb;
            if (out[5] != 0.0) {
                ts[n_incl++] = out[2];
                if (out[2] < best_t) { best_t = out[2]; best_j = (int32_t)j; }
            }
        }
        int amb_count = n_amb > 0;
        int amb_hit = (n_hit == 0) && (n_amb > 0);
        int count;
        if (!amb_count) {
            count = n_hit;
        } else {
            qsort(ts, (size_t)n_incl, sizeof(double), cmp_double);
            count = 0;
            for (int k = 0; k < n_incl; ++k)
                if (k == 0 || ts[k] - ts[k - 1] > ORACLE_TMERGE) ++count;
        }
        if (J->hit) J->hit[r] = (uint8_t)(n_hit > 0 || (amb_hit && n_incl > 0));
        if (J->amb_hit) J->amb_hit[r] = (uint8_t)amb_hit;
        if (J->count) J->count[r] = count;
        if (J->amb_count) J->amb_count[r] = (uint8_t)amb_count;
        if (J->near_tri) J->near_tri[r] = best_j;
        if (J->near_t) J->near_t[r] = best_j >= 0 ? (float)best_t : -1.0f;
        vec3 sv = v_load(s), dv = v_sub(v_load(e), sv);
        if (J->near_point) {
            vec3 pt = v_add(sv, v_scale(dv, best_t));
            J->near_point[3 * r + 0] = best_j >= 0 ? (float)pt.x : NAN;
            J->near_point[3 * r + 1] = best_j >= 0 ? (float)pt.y : NAN;
            J->near_point[3 * r + 2] = best_j >= 0 ? (float)pt.z : NAN;
        }
        if (J->near_dist) J->near_dist[r] = best_j >= 0 ? (float)(best_t * v_norm(dv)) : -1.0f;
    }
    free(ts);
    return NULL;
}

int oracle_num_threads(void) {
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* Returns 0, or -1 on an argument error (index out of range, n < 0). */
int oracle_query(const float* V, int64_t nV, const int32_t* T, int64_t nT,
                 const float* from, const float* to, int64_t nR,
                 uint8_t* hit, uint8_t* amb_hit, int32_t* count, uint8_t* amb_count,
                 int32_t* near_tri, float* near_t, float* near_point, float* near_dist, int nthreads) {
    if (nV < 0 || nT < 0 || nR < 0) return -1;
    for (int64_t j = 0; j < 3 * nT; ++j)
        if (T[j] < 0 || (int64_t)T[j] >= nV) return -1;
    if (nthreads <= 0) nthreads = oracle_num_threads();
    if ((int64_t)nthreads > nR) nthreads = nR > 0 ? (int)nR : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    query_job* jobs = (query_job*)malloc(sizeof(query_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; ++k) {
        query_job j = {V, from, to, T, nT, nR * k / nthreads, nR * (k + 1) / nthreads,
                       hit, amb_hit, amb_count, count, near_tri, near_t, near_point, near_dist};
        jobs[k] = j;
        pthread_create(&th[k], NULL, query_worker, &jobs[k]);
    }
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    free(th);
    free(jobs);
    return 0;
}

/* Class of every pair (ray-major, n_rays x n_triangles bytes): the input of
 * per-triangle checks such as which triangles a segment meets. */
int oracle_pair_classes(const float* V, int64_t nV, const int32_t* T, int64_t nT, const float* from,
                        const float* to, int64_t nR, uint8_t* cls) {
    for (int64_t j = 0; j < 3 * nT; ++j)
        if (T[j] < 0 || (int64_t)T[j] >= nV) return -1;
    for (int64_t r = 0; r < nR; ++r)
        for (int64_t j = 0; j < nT; ++j) {
            const int32_t* tri = T + 3 * j;
            cls[r * nT + j] = (uint8_t)oracle_classify_pair(from + 3 * r, to + 3 * r, V + 3 * (int64_t)tri[0],
                                                            V + 3 * (int64_t)tri[1], V + 3 * (int64_t)tri[2], NULL);
        }
    return 0;
}

/* Surface extent (Sec. 3.3, get_min_max_extent_of_surface): per-axis min and
 * max over all vertices.  Returns -1 if any coordinate is NaN. */
int oracle_extent(const float* V, int64_t nV, float* lo, float* hi) {
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int64_t i = 0; i < nV; ++i)
        for (int a = 0; a < 3; ++a) {
            float x = V[3 * i + a];
            if (x != x) return -1;
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
    return 0;
}

/*
 * Morton codes of triangle locations (Sec. 3.2: the location of every mesh
 * triangle becomes a 64-bit Morton code; Sec. 3.3: the surface extent is
 * computed first).  The location is the centroid ((v0 + v1) + v2) / 3 in FP32
 * round-to-nearest; each axis is normalised to u = (c - lo) / (hi - lo)
 * (0 when hi == lo), clamped to [0, 1], quantised to q = min(floor(u 2^b),
 * 2^b - 1) with b = bits / 3, and the key holds bit i of q_x, q_y, q_z at
 * bits 3i, 3i+1, 3i+2 (z is the high bit of each 3-bit group).
 * bits is 30 (b = 10) or 63 (b = 21).  Returns -1 on bad input.
 */
int oracle_morton(const float* V, int64_t nV, const int32_t* T, int64_t nT, int bits,
                  uint64_t* keys) {
    if (bits != 30 && bits != 63) return -1;
    float lo[3], hi[3];
    if (oracle_extent(V, nV, lo, hi) != 0) return -1;
    const int b = bits / 3;
    const float scale = (float)(1u << b);
    const uint32_t qmax = (1u << b) - 1u;
    for (int64_t j = 0; j < nT; ++j) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            int32_t i0 = T[3 * j], i1 = T[3 * j + 1], i2 = T[3 * j + 2];
            if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nV || i1 >= nV || i2 >= nV) return -1;
            float c = ((V[3 * (int64_t)i0 + a] + V[3 * (int64_t)i1 + a]) + V[3 * (int64_t)i2 + a]) / 3.0f;
            float u = 0.0f;
            if (hi[a] != lo[a]) u = (c - lo[a]) / (hi[a] - lo[a]);
            if (u < 0.0f) u = 0.0f;
            if (u > 1.0f) u = 1.0f;
            uint32_t qq = (uint32_t)(u * scale);
            q[a] = qq > qmax ? qmax : qq;
        }
        uint64_t key = 0;
        for (int i = 0; i < b; ++i)
            for (int a = 0; a < 3; ++a)
                key |= (uint64_t)((q[a] >> i) & 1u) << (3 * i + a);
        keys[j] = key;
    }
    return 0;
}

typedef struct { uint64_t key; int32_t id; } key_id;

static int cmp_key_id(const void* x, const void* y) {
    const key_id* a = (const key_id*)x;
    const key_id* b = (const key_id*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* Sort of the Morton codes with the triangle ids (Sec. 3.2, the numpy
 * argsort), made stable: order by (key, original index). */
int oracle_sort(const uint64_t* keys, int64_t n, uint64_t* sorted_keys, int32_t* perm) {
    key_id* a = (key_id*)malloc(sizeof(key_id) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].key = keys[i]; a[i].id = (int32_t)i; }
    qsort(a, (size_t)n, sizeof(key_id), cmp_key_id);
    for (int64_t i = 0; i < n; ++i) { sorted_keys[i] = a[i].key; perm[i] = a[i].id; }
    free(a);
    return 0;
}

#define ORACLE_LEAF_TAG 0x80000000u

static int highest_bit64(uint64_t x) { int p = -1; while (x) { x >>= 1; ++p; } return p; }

/* Split of the range [a, b] of sorted keys: the last index whose key has a
 * zero at the highest bit where the keys at a and b differ.  Equal keys are
 * told apart by their index (the index is appended below the key bits). */
static int64_t split_of(const uint64_t* k, int64_t a, int64_t b) {
    if (k[a] != k[b]) {
        int p = highest_bit64(k[a] ^ k[b]);
        int64_t g = a;
        while (g + 1 <= b && ((k[g + 1] >> p) & 1u) == 0) ++g;
        return g;
    }
    int p = highest_bit64((uint64_t)(a ^ b));
    int64_t g = a;
    while (g + 1 <= b && (((uint64_t)(g + 1) >> p) & 1u) == 0) ++g;
    return g;
}

static void tree_rec(const uint64_t* k, int64_t a, int64_t b, int64_t node, int64_t n,
                     int32_t* left, int32_t* right, int32_t* parent,
                     int32_t* range_lo, int32_t* range_hi) {
    int64_t g = split_of(k, a, b);
    range_lo[node] = (int32_t)a;
    range_hi[node] = (int32_t)b;
    if (g == a) {
        left[node] = (int32_t)(ORACLE_LEAF_TAG | (uint32_t)g);
        parent[n - 1 + g] = (int32_t)node;
    } else {
        left[node] = (int32_t)g;
        parent[g] = (int32_t)node;
        tree_rec(k, a, g, g, n, left, right, parent, range_lo, range_hi);
    }
    if (g + 1 == b) {
        right[node] = (int32_t)(ORACLE_LEAF_TAG | (uint32_t)(g + 1));
        parent[n - 1 + g + 1] = (int32_t)node;
    } else {
        right[node] = (int32_t)(g + 1);
        parent[g + 1] = (int32_t)node;
        tree_rec(k, g + 1, b, g + 1, n, left, right, parent, range_lo, range_hi);
    }
}

/*
 * Binary radix tree over n sorted keys (Sec. 1: the triangles are held in a
 * binary radix tree, Karras 2012; Sec. 4.2: n - 1 internal nodes are used).
 * It is the unique tree whose every internal node covers a key range [a, b]
 * and splits it at the highest differing bit.  Numbering follows Karras: the
 * root is internal node 0; a node split at g has the left child "g" (internal
 * node g covering [a, g], or leaf g when g == a) and the right child "g + 1"
 * (internal node g+1 covering [g+1, b], or leaf g+1 when g + 1 == b).
 * Children are int32 ids, a leaf tagged by the high bit.  parent[] has the
 * internal nodes first (0..n-2) then the leaves (n-1 .. 2n-2); the root has
 * parent -1.  With n == 1 there is no internal node.
 */
int oracle_radix_tree(const uint64_t* sorted_keys, int64_t n, int32_t* left, int32_t* right,
                      int32_t* parent, int32_t* range_lo, int32_t* range_hi) {
    if (n < 1) return -1;
    for (int64_t i = 0; i < 2 * n - 1; ++i) parent[i] = -1;
    if (n == 1) return 0;
    tree_rec(sorted_keys, 0, n - 1, 0, n, left, right, parent, range_lo, range_hi);
    return 0;
}

static int box_rec(int32_t ref, int64_t n, const int32_t* left, const int32_t* right,
                   const float* V, const int32_t* T, const int32_t* perm, float* box) {
    if ((uint32_t)ref & ORACLE_LEAF_TAG) {
        int64_t j = (int64_t)((uint32_t)ref & ~ORACLE_LEAF_TAG);
        float* bx = box + 6 * (n - 1 + j);
        const int32_t* tri = T + 3 * (int64_t)perm[j];
        for (int a = 0; a < 3; ++a) {
            float x0 = V[3 * (int64_t)tri[0] + a], x1 = V[3 * (int64_t)tri[1] + a], x2 = V[3 * (int64_t)tri[2] + a];
            float mn = x0 < x1 ? x0 : x1; mn = mn < x2 ? mn : x2;
            float mx = x0 > x1 ? x0 : x1; mx = mx > x2 ? mx : x2;
            bx[a] = mn; bx[3 + a] = mx;
        }
        return 0;
    }
    int64_t i = ref;
    int hl = box_rec(left[i], n, left, right, V, T, perm, box);
    int hr = box_rec(right[i], n, left, right, V, T, perm, box);
    const float* bl = (uint32_t)left[i] & ORACLE_LEAF_TAG
                          ? box + 6 * (n - 1 + (int64_t)((uint32_t)left[i] & ~ORACLE_LEAF_TAG)) : box + 6 * (int64_t)left[i];
    const float* br = (uint32_t)right[i] & ORACLE_LEAF_TAG
                          ? box + 6 * (n - 1 + (int64_t)((uint32_t)right[i] & ~ORACLE_LEAF_TAG)) : box + 6 * (int64_t)right[i];
    float* bx = box + 6 * i;
    for (int a = 0; a < 3; ++a) {
        bx[a] = bl[a] < br[a] ? bl[a] : br[a];
        bx[3 + a] = bl[3 + a] > br[3 + a] ? bl[3 + a] : br[3 + a];
    }
    return 1 + (hl > hr ? hl : hr);
}

/* Axis-aligned boxes of every node (Sec. 4.1: each BVH node holds the
 * bounding volume of its subtree; Sec. 4.2: the leaf bounds propagate to the
 * top).  box[6 * node] = (min x, y, z, max x, y, z), internal nodes first
 * then leaves (leaf j holds triangle perm[j]).  Returns the height of the
 * tree (edges on the longest root-to-leaf path). */
int oracle_refit(const float* V, const int32_t* T, const int32_t* perm, int64_t n,
                 const int32_t* left, const int32_t* right, float* box) {
    if (n < 1) return -1;
    if (n == 1) return box_rec((int32_t)ORACLE_LEAF_TAG, n, left, right, V, T, perm, box);
    return box_rec(0, n, left, right, V, T, perm, box);
}
