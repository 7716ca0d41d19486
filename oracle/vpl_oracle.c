/*
 * FP64 CPU oracle for the hybrid close-range VPL method
 * (Jin, Wang, Zheng, Hua, Huo: "A Virtual Point Light Generation Method in
 * Close-Range Area", arXiv 2203.11484).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  It shares no code with the CUDA
 * library; only the test-suite, the smoke check and the benchmark's CPU
 * baseline load it.  Everything is double precision, compiled with
 * -ffp-contract=off so every product and sum is rounded on its own.
 *
 * Paper passages followed (Sec. 3 unless noted):
 *   Eq. 1                 L(y) ~ Le(y) + sum_i G_i V_i L_i  (indirect part only)
 *   close/distant split   one-sided face, inside the field of view, nearer
 *                         than a threshold  -> close range
 *   pipeline (1)-(4)      classify; patch sampling of the close range; instant
 *                         radiosity over the whole scene keeping only hits on
 *                         the distant part; render
 *   Eq. 2                 patch VPL value L_i = G_i V_i L_e, G_i = D cos w/(4 pi r^2)
 *   "Realization"         Morton order of the close triangles, area prefix sum
 *                         f(i), inverse g, K equal-area strata, random points in
 *                         the chosen triangle, each VPL carrying the area of its
 *                         stratum
 *
 * Readings where the paper is silent or garbled (the same ones the GPU path
 * implements, listed with reasons in the design notes):
 *   - "camera" in the definition of w and r in Eq. 2 means the light;
 *   - a patch VPL stores reflected power: albedo x incident power on its area;
 *   - close-range test on the triangle centroid, front-facing to the camera,
 *     and facing the light (no occlusion test);
 *   - integer-quantised areas so that stratum -> triangle is exact;
 *   - instant-radiosity paths start at the first bounce, no roulette, a hit on
 *     a close face stores nothing but the path continues, the first m_far VPLs
 *     in (path, bounce) order are kept and all are divided by the number of
 *     paths P that were needed;
 *   - random numbers: Philox4x64-10 (Salmon et al., SC'11) with counter
 *     (index, sub-index, 0, 0) and key (seed, stream); u = (w >> 40) * 2^-24.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* small FP64 vector algebra (each op rounded separately)                   */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } d3;

static d3 mk(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 add(d3 a, d3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 sub(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 scl(d3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(d3 a, d3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static d3 cross(d3 a, d3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(d3 a) { return sqrt(dot(a, a)); }
static d3 unit(d3 a) { double l = len(a); return mk(a.x / l, a.y / l, a.z / l); }
static d3 ld3(const double *p) { return mk(p[0], p[1], p[2]); }
static d3 lf3(const float *p) { return mk((double)p[0], (double)p[1], (double)p[2]); }
static void st3(double *p, d3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)                        */
/* ------------------------------------------------------------------------ */
ORC_API void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { STREAM_PATCH = 1, STREAM_LIGHT = 2, STREAM_IR = 3, STREAM_DIRECT = 4, STREAM_REJECT = 5 };

static void rng4(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j, uint64_t w[4])
{
    uint64_t ctr[4] = {i, j, 0, 0}, key[2] = {seed, stream};
    orc_philox4x64_10(ctr, key, w);
}

/* top 24 bits of a word as a number in [0, 1) (exact in FP32 and FP64) */
static double u01(uint64_t w) { return (double)(w >> 40) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Morton code: bit i of qx, qy, qz goes to bit 3i+2, 3i+1, 3i                */
/* ------------------------------------------------------------------------ */
ORC_API uint64_t orc_morton63(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t code = 0;
    for (int i = 0; i < 21; i++) {
        code |= (uint64_t)((qx >> i) & 1u) << (3 * i + 2);
        code |= (uint64_t)((qy >> i) & 1u) << (3 * i + 1);
        code |= (uint64_t)((qz >> i) & 1u) << (3 * i);
    }
    return code;
}

static uint32_t quant21(double v, double lo, double hi)
{
    double t = (hi > lo) ? (v - lo) / (hi - lo) : 0.0;
    double q = floor(t * 2097152.0);
    if (q > 2097151.0) q = 2097151.0;
    if (q < 0.0) q = 0.0;
    return (uint32_t)q;
}

/* ------------------------------------------------------------------------ */
/* scene                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    d3 lo, hi;
    int32_t left, right;   /* children (internal) */
    int32_t first, count;  /* triangle range in perm[] (leaf when count > 0) */
} onode;

typedef struct {
    int64_t nt;
    d3 *a, *b, *c, *e1, *e2, *cr, *n, *g;
    double *area, *rho;
    d3 glo, ghi;           /* AABB of all centroids   */
    d3 vlo, vhi;           /* AABB of all vertices    */
    onode *nodes;
    int32_t n_nodes;
    int32_t *perm;
} oscene;

typedef struct {
    double eye[3], fwd[3], up[3];
    double vfov_deg;
    int32_t width, height;
} ocamera;

typedef struct {
    double center[3], normal[3], edge_u[3], edge_v[3], power[3];
    int32_t type;          /* 0 one-sided square area light, 1 isotropic point light */
} olight;

typedef struct {
    double d_close;
    double ray_eps;
    int64_t ir_max_paths;
    uint64_t seed;
    int32_t m_close, m_far, max_bounces, light_samples;
    int32_t vis_mode;      /* 0 BVH, 1 brute force */
    int32_t close_rule;    /* 0 centroid, 1 centroid or any vertex (see is_close) */
    int32_t patch_rule;    /* 0 a point per stratum, 1 set sum for strata over several faces */
} ogen;

/* ---- FP64 BVH: top-down median split, boxes padded so that the set of
 *      candidate triangles is always a superset of the true hits ---------- */
static const d3 *g_sort_g;
static int g_sort_axis;
static int cmp_axis(const void *pa, const void *pb)
{
    int32_t ia = *(const int32_t *)pa, ib = *(const int32_t *)pb;
    const d3 *A = &g_sort_g[ia], *B = &g_sort_g[ib];
    double va = g_sort_axis == 0 ? A->x : g_sort_axis == 1 ? A->y : A->z;
    double vb = g_sort_axis == 0 ? B->x : g_sort_axis == 1 ? B->y : B->z;
    if (va < vb) return -1;
    if (va > vb) return 1;
    return ia < ib ? -1 : (ia > ib);
}

static int32_t build_rec(oscene *s, int32_t first, int32_t count, double pad)
{
    int32_t id = s->n_nodes++;
    onode *nd = &s->nodes[id];
    d3 lo = mk(INFINITY, INFINITY, INFINITY), hi = mk(-INFINITY, -INFINITY, -INFINITY);
    d3 clo = lo, chi = hi;
    for (int32_t k = first; k < first + count; k++) {
        int32_t t = s->perm[k];
        d3 v[3] = {s->a[t], add(s->a[t], s->e1[t]), add(s->a[t], s->e2[t])};
        for (int q = 0; q < 3; q++) {
            lo = mk(dmin(lo.x, v[q].x), dmin(lo.y, v[q].y), dmin(lo.z, v[q].z));
            hi = mk(dmax(hi.x, v[q].x), dmax(hi.y, v[q].y), dmax(hi.z, v[q].z));
        }
        clo = mk(dmin(clo.x, s->g[t].x), dmin(clo.y, s->g[t].y), dmin(clo.z, s->g[t].z));
        chi = mk(dmax(chi.x, s->g[t].x), dmax(chi.y, s->g[t].y), dmax(chi.z, s->g[t].z));
    }
    nd->lo = sub(lo, mk(pad, pad, pad));
    nd->hi = add(hi, mk(pad, pad, pad));
    if (count <= 4) {
        nd->first = first; nd->count = count; nd->left = nd->right = -1;
        return id;
    }
    d3 ext = sub(chi, clo);
    int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
    g_sort_g = s->g;
    g_sort_axis = axis;
    qsort(s->perm + first, (size_t)count, sizeof(int32_t), cmp_axis);
    int32_t half = count / 2;
    nd->first = first; nd->count = 0;
    int32_t l = build_rec(s, first, half, pad);
    int32_t r = build_rec(s, first + half, count - half, pad);
    s->nodes[id].left = l;
    s->nodes[id].right = r;
    return id;
}

ORC_API void *orc_scene_create(const float *verts, int64_t nv, const int32_t *tris,
                               int64_t nt, const float *albedo)
{
    (void)nv;
    oscene *s = (oscene *)calloc(1, sizeof(oscene));
    s->nt = nt;
    s->a = malloc(sizeof(d3) * nt);   s->e1 = malloc(sizeof(d3) * nt);
    s->b = malloc(sizeof(d3) * nt);   s->c = malloc(sizeof(d3) * nt);
    s->e2 = malloc(sizeof(d3) * nt);  s->cr = malloc(sizeof(d3) * nt);
    s->n = malloc(sizeof(d3) * nt);   s->g = malloc(sizeof(d3) * nt);
    s->area = malloc(sizeof(double) * nt);
    s->rho = malloc(sizeof(double) * 3 * nt);
    s->glo = s->vlo = mk(INFINITY, INFINITY, INFINITY);
    s->ghi = s->vhi = mk(-INFINITY, -INFINITY, -INFINITY);
    for (int64_t t = 0; t < nt; t++) {
        d3 a = lf3(verts + 3 * (int64_t)tris[3 * t + 0]);
        d3 b = lf3(verts + 3 * (int64_t)tris[3 * t + 1]);
        d3 c = lf3(verts + 3 * (int64_t)tris[3 * t + 2]);
        d3 e1 = sub(b, a), e2 = sub(c, a);
        d3 cr = cross(e1, e2);
        double l = len(cr);
        s->a[t] = a; s->b[t] = b; s->c[t] = c; s->e1[t] = e1; s->e2[t] = e2; s->cr[t] = cr;
        s->n[t] = l > 0.0 ? mk(cr.x / l, cr.y / l, cr.z / l) : mk(0, 0, 0);
        s->area[t] = 0.5 * l;
        d3 g = add(add(a, b), c);
        s->g[t] = mk(g.x / 3.0, g.y / 3.0, g.z / 3.0);
        for (int k = 0; k < 3; k++) s->rho[3 * t + k] = (double)albedo[3 * t + k];
        d3 gg = s->g[t];
        s->glo = mk(dmin(s->glo.x, gg.x), dmin(s->glo.y, gg.y), dmin(s->glo.z, gg.z));
        s->ghi = mk(dmax(s->ghi.x, gg.x), dmax(s->ghi.y, gg.y), dmax(s->ghi.z, gg.z));
        d3 vv[3] = {a, b, c};
        for (int q = 0; q < 3; q++) {
            s->vlo = mk(dmin(s->vlo.x, vv[q].x), dmin(s->vlo.y, vv[q].y), dmin(s->vlo.z, vv[q].z));
            s->vhi = mk(dmax(s->vhi.x, vv[q].x), dmax(s->vhi.y, vv[q].y), dmax(s->vhi.z, vv[q].z));
        }
    }
    /* BVH */
    s->perm = malloc(sizeof(int32_t) * (nt > 0 ? nt : 1));
    for (int64_t t = 0; t < nt; t++) s->perm[t] = (int32_t)t;
    s->nodes = malloc(sizeof(onode) * (2 * (nt > 0 ? nt : 1)));
    s->n_nodes = 0;
    double pad = 1e-9 * (len(sub(s->vhi, s->vlo)) + 1.0);
    if (nt > 0) build_rec(s, 0, (int32_t)nt, pad);
    return s;
}

ORC_API void orc_scene_destroy(void *p)
{
    oscene *s = (oscene *)p;
    if (!s) return;
    free(s->a); free(s->b); free(s->c); free(s->e1); free(s->e2); free(s->cr); free(s->n); free(s->g);
    free(s->area); free(s->rho); free(s->nodes); free(s->perm);
    free(s);
}

ORC_API void orc_scene_info(void *p, double out[14])
{
    oscene *s = (oscene *)p;
    st3(out + 0, s->glo); st3(out + 3, s->ghi);
    st3(out + 6, s->vlo); st3(out + 9, s->vhi);
    out[12] = (double)s->n_nodes;
    out[13] = (double)s->nt;
}

/* ------------------------------------------------------------------------ */
/* ray / triangle (Moller-Trumbore, inclusive barycentric bounds)           */
/* ------------------------------------------------------------------------ */
/* returns 1 and t when the line o + t d meets triangle k (either side) */
static int tri_hit(const oscene *s, int64_t k, d3 o, d3 d, double *t_out)
{
    d3 pv = cross(d, s->e2[k]);
    double det = dot(s->e1[k], pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    d3 tv = sub(o, s->a[k]);
    double u = dot(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    d3 qv = cross(tv, s->e1[k]);
    double v = dot(d, qv) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *t_out = dot(s->e2[k], qv) * inv;
    return 1;
}

/* slab test of the ray against a (padded) box, interval [t0, t1] */
static int box_hit(const onode *nd, d3 o, d3 d, double t0, double t1, double *t_enter)
{
    double lo[3] = {nd->lo.x, nd->lo.y, nd->lo.z}, hi[3] = {nd->hi.x, nd->hi.y, nd->hi.z};
    double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    for (int a = 0; a < 3; a++) {
        if (dd[a] == 0.0) {
            if (oo[a] < lo[a] || oo[a] > hi[a]) return 0;
            continue;
        }
        double ta = (lo[a] - oo[a]) / dd[a], tb = (hi[a] - oo[a]) / dd[a];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    *t_enter = t0;
    return 1;
}

/* closest hit with t > tmin; ties broken by the lower triangle index */
static int64_t closest_brute(const oscene *s, d3 o, d3 d, double tmin, double *t_best)
{
    int64_t best = -1;
    double bt = INFINITY, t;
    for (int64_t k = 0; k < s->nt; k++)
        if (tri_hit(s, k, o, d, &t) && t > tmin && t < bt) { bt = t; best = k; }
    *t_best = bt;
    return best;
}

static int64_t closest_bvh(const oscene *s, d3 o, d3 d, double tmin, double *t_best)
{
    int64_t best = -1;
    double bt = INFINITY;
    if (s->nt == 0) { *t_best = bt; return -1; }
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const onode *nd = &s->nodes[stack[--sp]];
        double te;
        if (!box_hit(nd, o, d, tmin, bt, &te)) continue;
        if (nd->count > 0) {
            for (int32_t q = nd->first; q < nd->first + nd->count; q++) {
                int64_t k = s->perm[q];
                double t;
                if (tri_hit(s, k, o, d, &t) && t > tmin &&
                    (t < bt || (t == bt && k < best))) { bt = t; best = k; }
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    *t_best = bt;
    return best;
}

/* segment p -> q blocked by any triangle at t in (0, 1), either side */
static int occluded_brute(const oscene *s, d3 p, d3 q)
{
    d3 d = sub(q, p);
    double t;
    for (int64_t k = 0; k < s->nt; k++)
        if (tri_hit(s, k, p, d, &t) && t > 0.0 && t < 1.0) return 1;
    return 0;
}

static int occluded_bvh(const oscene *s, d3 p, d3 q)
{
    if (s->nt == 0) return 0;
    d3 d = sub(q, p);
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const onode *nd = &s->nodes[stack[--sp]];
        double te;
        if (!box_hit(nd, p, d, 0.0, 1.0, &te)) continue;
        if (nd->count > 0) {
            for (int32_t k = nd->first; k < nd->first + nd->count; k++) {
                double t;
                if (tri_hit(s, s->perm[k], p, d, &t) && t > 0.0 && t < 1.0) return 1;
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return 0;
}

static int64_t closest(const oscene *s, d3 o, d3 d, double tmin, double *t, int vis_mode)
{
    return vis_mode == 1 ? closest_brute(s, o, d, tmin, t) : closest_bvh(s, o, d, tmin, t);
}
static int occluded(const oscene *s, d3 p, d3 q, int vis_mode)
{
    return vis_mode == 1 ? occluded_brute(s, p, q) : occluded_bvh(s, p, q);
}

ORC_API void orc_closest_batch(void *sp, int64_t n, const double *o, const double *d,
                               double tmin, int32_t vis_mode, int64_t *tri, double *t)
{
    const oscene *s = (const oscene *)sp;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++)
        tri[i] = closest(s, ld3(o + 3 * i), ld3(d + 3 * i), tmin, &t[i], vis_mode);
}

ORC_API void orc_occluded_batch(void *sp, int64_t n, const double *p, const double *q,
                                int32_t vis_mode, uint8_t *out)
{
    const oscene *s = (const oscene *)sp;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++)
        out[i] = (uint8_t)occluded(s, ld3(p + 3 * i), ld3(q + 3 * i), vis_mode);
}

/* distance from x to the segment A-B */
static double seg_dist(d3 x, d3 A, d3 B)
{
    d3 ab = sub(B, A);
    double l2 = dot(ab, ab);
    double t = l2 > 0.0 ? dot(sub(x, A), ab) / l2 : 0.0;
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    return len(sub(x, add(A, scl(ab, t))));
}

/* Smallest distance-like margin of segment p->q to flipping its visibility:
 * for every triangle whose plane the segment crosses (or nearly touches), the
 * distance of the crossing point to the triangle's boundary, and the
 * distance of the endpoints to the plane.  A GPU/oracle visibility
 * disagreement is explained when this margin is tiny. */
ORC_API double orc_segment_margin(void *sp, const double *p3, const double *q3)
{
    const oscene *s = (const oscene *)sp;
    d3 p = ld3(p3), q = ld3(q3), d = sub(q, p);
    double best = INFINITY;
    for (int64_t k = 0; k < s->nt; k++) {
        double nl = len(s->cr[k]);
        if (nl == 0.0) continue;
        d3 nn = scl(s->cr[k], 1.0 / nl);
        double sp_ = dot(sub(p, s->a[k]), nn), sq_ = dot(sub(q, s->a[k]), nn);
        /* endpoint close to the plane and over the triangle */
        double dd = dot(d, nn);
        if (fabs(dd) == 0.0) continue;
        double t = -sp_ / dd;
        if (t < -1e-3 || t > 1.0 + 1e-3) {
            continue;
        }
        d3 x = add(p, scl(d, t));
        /* distance of x to the triangle's edges (in-plane, signed inside > 0) */
        d3 v0 = s->a[k], v1 = add(v0, s->e1[k]), v2 = add(v0, s->e2[k]);
        d3 vs[3] = {v0, v1, v2};
        /* distance of x (in the plane) to the triangle's boundary */
        double m_in = INFINITY;
        for (int e = 0; e < 3; e++) m_in = dmin(m_in, seg_dist(x, vs[e], vs[(e + 1) % 3]));
        int inside = 1;
        for (int e = 0; e < 3; e++) {
            d3 A = vs[e], B = vs[(e + 1) % 3];
            if (dot(cross(sub(B, A), sub(x, A)), nn) < 0.0) inside = 0;
        }
        double m = m_in;
        if (inside) {
            double ep = dmin(fabs(sp_), fabs(sq_));
            if (ep < m) m = ep;
        }
        if (m < best) best = m;
    }
    return best;
}

/* How close segment p->q comes to changing its answer against any triangle,
 * measured against what FP32 arithmetic can move.  For each triangle whose
 * plane the segment's line crosses at t in [-1e-3, 1 + 1e-3]:
 *   - when the segment itself crosses the plane (t in [0, 1]), the in-plane
 *     distance m_e of the crossing to the triangle's boundary, against
 *       B_e = (c u (|p|inf + |q|inf + |p - a_k|) + extra) / (cos_k sin_k);
 *   - when the crossing lies inside the triangle, the distance m_p of an end
 *     point to its plane (p when ends & 1, q when ends & 2), against
 *       B_p = (c u (|p|inf + |q|inf + |p - a_k|) + extra) / sin_k.
 * u = 2^-24 (FP32 unit roundoff); cos_k = |cos| of the angle between the
 * segment and the triangle's normal; sin_k = the sine of the triangle's
 * angle at a_k.  Rounding the end points and the products of a
 * Moller-Trumbore test in FP32 moves its barycentric decisions by a few
 * u (|p| + |q| + |p - a|) / sin in barycentric length, which the crossing
 * turns into 1 / cos along the plane, and its segment-parameter decisions
 * by the same over sin in distance from the plane; `extra` is an absolute
 * error the end points already carry (e.g. from earlier FP32 bounces).
 * Returns the smallest ratio m / B: a disagreement between FP32 and FP64 is
 * explained when it is at most 1. */
ORC_API double orc_flip_ratio(void *sp, const double *p3, const double *q3, double c, double extra, int32_t ends)
{
    const oscene *s = (const oscene *)sp;
    const double u = 1.0 / 16777216.0;
    d3 p = ld3(p3), q = ld3(q3), d = sub(q, p);
    double dl = len(d);
    double pinf = dmax(fabs(p.x), dmax(fabs(p.y), fabs(p.z)));
    double qinf = dmax(fabs(q.x), dmax(fabs(q.y), fabs(q.z)));
    double best = INFINITY;
    if (dl == 0.0) return best;
    for (int64_t k = 0; k < s->nt; k++) {
        double nl = len(s->cr[k]);
        if (nl == 0.0) continue;
        d3 nn = scl(s->cr[k], 1.0 / nl);
        double sp_ = dot(sub(p, s->a[k]), nn), sq_ = dot(sub(q, s->a[k]), nn);
        double dd = dot(d, nn);
        if (fabs(dd) == 0.0) continue;
        double t = -sp_ / dd;
        if (t < -1e-3 || t > 1.0 + 1e-3) continue;
        d3 x = add(p, scl(d, t));
        d3 v0 = s->a[k], v1 = add(v0, s->e1[k]), v2 = add(v0, s->e2[k]);
        d3 vs[3] = {v0, v1, v2};
        double me = INFINITY;
        int inside = 1;
        for (int e = 0; e < 3; e++) {
            d3 A = vs[e], B = vs[(e + 1) % 3];
            me = dmin(me, seg_dist(x, A, B));
            if (dot(cross(sub(B, A), sub(x, A)), nn) < 0.0) inside = 0;
        }
        double cosk = fabs(dd) / dl;
        double sink = nl / (len(s->e1[k]) * len(s->e2[k]));
        double base = c * u * (pinf + qinf + len(sub(p, s->a[k]))) + extra;
        double r = (t >= 0.0 && t <= 1.0) ? me / (base / (cosk * sink)) : INFINITY;
        if (inside) {
            double mp = INFINITY;
            if (ends & 1) mp = dmin(mp, fabs(sp_));
            if (ends & 2) mp = dmin(mp, fabs(sq_));
            r = dmin(r, mp / (base / sink));
        }
        if (r < best) best = r;
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* camera frame and close-range classification                              */
/* ------------------------------------------------------------------------ */
typedef struct { d3 e, f, r, u; double tv, th; } frame;

static frame cam_frame(const ocamera *c)
{
    frame F;
    F.e = ld3(c->eye);
    F.f = unit(ld3(c->fwd));
    F.r = unit(cross(F.f, ld3(c->up)));
    F.u = cross(F.r, F.f);
    F.tv = tan(c->vfov_deg * (PI / 180.0) * 0.5);
    F.th = (F.tv * (double)c->width) / (double)c->height;
    return F;
}

/* point p inside the field of view and nearer than d_close */
static int in_view(d3 p, const frame *F, double dc2)
{
    d3 v = sub(p, F->e);
    double z = dot(v, F->f);
    if (!(z > 0.0)) return 0;
    if (!(fabs(dot(v, F->r)) <= z * F->th)) return 0;
    if (!(fabs(dot(v, F->u)) <= z * F->tv)) return 0;
    return dot(v, v) < dc2;
}

/* close/distant split: a one-sided face is close range when it faces the
 * camera, lies inside the field of view and nearer than d_close -- judged at
 * its centroid (rule 0), or at its centroid or any of its vertices (rule 1,
 * the any-vertex reading of "within the field of view") -- and patch
 * sampling further only considers faces that face the light. */
static int is_close(const oscene *s, int64_t t, const frame *F, const olight *L, double dc2, int rule)
{
    d3 g = s->g[t], cr = s->cr[t];
    if (!(dot(cr, sub(F->e, g)) > 0.0)) return 0;
    if (!(in_view(g, F, dc2) ||
          (rule == 1 && (in_view(s->a[t], F, dc2) || in_view(s->b[t], F, dc2) || in_view(s->c[t], F, dc2)))))
        return 0;
    d3 cl = ld3(L->center);
    if (!(dot(cr, sub(cl, g)) > 0.0)) return 0;
    if (L->type == 0 && !(dot(ld3(L->normal), sub(g, cl)) > 0.0)) return 0;
    return 1;
}

ORC_API int64_t orc_classify(void *sp, const ocamera *cam, const olight *L, double d_close, int32_t rule,
                             uint8_t *flags)
{
    const oscene *s = (const oscene *)sp;
    frame F = cam_frame(cam);
    double dc2 = d_close * d_close;
    int64_t n = 0;
    for (int64_t t = 0; t < s->nt; t++) {
        flags[t] = (uint8_t)is_close(s, t, &F, L, dc2, rule);
        n += flags[t];
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* light sampling and hemisphere directions                                 */
/* ------------------------------------------------------------------------ */
static d3 light_point(const olight *L, double s1, double s2)
{
    d3 c = ld3(L->center);
    if (L->type == 1) return c;
    d3 a = scl(ld3(L->edge_u), (2.0 * s1 - 1.0) * 0.5);
    d3 b = scl(ld3(L->edge_v), (2.0 * s2 - 1.0) * 0.5);
    return add(add(c, a), b);
}

/* Direct term L_e(y) of Eq. 1 as light-sample VPLs: sample s is the point
 * of the square light at Philox (seed, STREAM_DIRECT) counter (s, 0) words
 * w0, w1 -> (s1, s2), with the light's normal and power P / S.  Gathered
 * with Eq. 1's sum, S such VPLs give the Monte Carlo estimate
 * (rho/pi) * (1/S) sum_s P cos_i cos_y / (pi d^2) V of the light's one-sided
 * Lambertian emission (radiance P / (pi A_L)) reflected at y.  Tag -1 - s.
 * Returns -1 for a point light (no normal: its direct term is not this sum). */
ORC_API int64_t orc_light_vpls(const olight *L, int64_t S, uint64_t seed, double *pos, double *nrm, double *flux,
                               int64_t *tag)
{
    if (L->type == 1) return -1;
    d3 nl = ld3(L->normal);
    for (int64_t k = 0; k < S; k++) {
        uint64_t w[4];
        rng4(seed, STREAM_DIRECT, (uint64_t)k, 0, w);
        d3 y = light_point(L, u01(w[0]), u01(w[1]));
        pos[3 * k] = y.x;
        pos[3 * k + 1] = y.y;
        pos[3 * k + 2] = y.z;
        nrm[3 * k] = nl.x;
        nrm[3 * k + 1] = nl.y;
        nrm[3 * k + 2] = nl.z;
        for (int c = 0; c < 3; c++) flux[3 * k + c] = L->power[c] / (double)S;
        tag[k] = -1 - k;
    }
    return S;
}

/* orthonormal basis around unit n (Duff et al., JCGT 2017) */
static void onb(d3 n, d3 *t1, d3 *t2)
{
    double sg = copysign(1.0, n.z);
    double a = -1.0 / (sg + n.z);
    double b = n.x * n.y * a;
    *t1 = mk(1.0 + sg * n.x * n.x * a, sg * b, -sg * n.x);
    *t2 = mk(b, sg + n.y * n.y * a, -n.y);
}

/* cosine-weighted direction about n (Malley's method) */
static d3 cosine_dir(d3 n, double s1, double s2)
{
    d3 t1, t2;
    onb(n, &t1, &t2);
    double r = sqrt(s1), ph = 2.0 * PI * s2;
    return add(add(scl(t1, r * cos(ph)), scl(t2, r * sin(ph))), scl(n, sqrt(1.0 - s1)));
}

static d3 sphere_dir(double s1, double s2)
{
    double z = 1.0 - 2.0 * s1;
    double r = sqrt(dmax(0.0, 1.0 - z * z)), ph = 2.0 * PI * s2;
    return mk(r * cos(ph), r * sin(ph), z);
}

/* ------------------------------------------------------------------------ */
/* one instant-radiosity light path (pipeline step (3)): the rays it casts    */
/* ------------------------------------------------------------------------ */
typedef struct {
    d3 o, d;       /* ray origin and direction                               */
    int64_t k;     /* triangle hit (closest, t > 0), -1 on a miss            */
    double t;      /* its ray parameter                                      */
    int front;     /* 1: front face hit, x is a path vertex; 0: the path ends */
    d3 x;          /* hit point o + t d (front hits)                         */
} irray;

/* Path p: start on the light (Philox key (seed, STREAM_IR), counter (p, 0):
 * words w0, w1 the point, w2, w3 the direction; cosine-weighted about the
 * light's normal, or uniform on the sphere for a point light), then at most
 * max_bounces closest hits; after each front-face hit x on face k the next
 * direction is cosine-weighted about n_k with counter (p, b) and the next
 * ray starts at x + ray_eps n_k.  A miss or a back-face hit (one-sided faces
 * absorb from behind) ends the path.  Writes the rays cast, returns how many. */
static int ir_path(const oscene *s, const olight *L, const ogen *G, int64_t p, irray *out)
{
    uint64_t w[4];
    rng4(G->seed, STREAM_IR, (uint64_t)p, 0, w);
    d3 o, d;
    if (L->type == 1) {
        o = ld3(L->center);
        d = sphere_dir(u01(w[2]), u01(w[3]));
    } else {
        o = light_point(L, u01(w[0]), u01(w[1]));
        d = cosine_dir(ld3(L->normal), u01(w[2]), u01(w[3]));
    }
    int n = 0;
    for (int32_t b = 1; b <= G->max_bounces; b++) {
        double t;
        int64_t k = closest(s, o, d, 0.0, &t, G->vis_mode);
        irray *r = &out[n++];
        r->o = o;
        r->d = d;
        r->k = k;
        r->t = t;
        r->front = 0;
        r->x = mk(0, 0, 0);
        if (k < 0) break;
        if (!(dot(d, s->cr[k]) < 0.0)) break;   /* back face absorbs */
        d3 x = add(o, scl(d, t));
        r->front = 1;
        r->x = x;
        if (b == G->max_bounces) break;
        rng4(G->seed, STREAM_IR, (uint64_t)p, (uint64_t)b, w);
        d = cosine_dir(s->n[k], u01(w[0]), u01(w[1]));
        o = add(x, scl(s->n[k], G->ray_eps));
    }
    return n;
}

/* The rays of light path p (ir_path) for replay by the tests: per ray its
 * origin o[3i..], direction d[3i..], triangle k[i] (-1 miss), t[i] and
 * front[i]; arrays of max_bounces entries.  Returns the number of rays. */
ORC_API int64_t orc_ir_path(void *sp, const olight *L, const ogen *G, int64_t p, double *o, double *d,
                            int64_t *k, double *t, int64_t *front)
{
    const oscene *s = (const oscene *)sp;
    irray *r = malloc(sizeof(irray) * (size_t)(G->max_bounces > 0 ? G->max_bounces : 1));
    int n = ir_path(s, L, G, p, r);
    for (int i = 0; i < n; i++) {
        st3(o + 3 * i, r[i].o);
        st3(d + 3 * i, r[i].d);
        k[i] = r[i].k;
        t[i] = r[i].t;
        front[i] = r[i].front;
    }
    free(r);
    return n;
}

/* ------------------------------------------------------------------------ */
/* VPL generation (pipeline steps (1)-(3))                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_close;     /* |C|                                  */
    int64_t shift_s;     /* S in q_t = llround(A_t 2^S)          */
    uint64_t f_total;    /* f(N) in quantised units              */
    int64_t paths;       /* P                                    */
    int64_t m_far_kept;  /* far VPLs produced (< m_far if exhausted) */
    double a_rep;        /* area represented by one patch VPL    */
    int64_t status;      /* 0 ok, 6 close set empty, 7 paths exhausted */
} oinfo;

typedef struct { uint64_t code; int32_t tri; } mkey;
static int cmp_mkey(const void *pa, const void *pb)
{
    const mkey *a = (const mkey *)pa, *b = (const mkey *)pb;
    if (a->code != b->code) return a->code < b->code ? -1 : 1;
    return a->tri < b->tri ? -1 : (a->tri > b->tri);
}

/* Spatial order of the close-range faces ("Realization": the faces are
 * sorted by the Morton code of their position): the FP64 centroid of each
 * face with mask[t] != 0, normalised into the AABB of the centroids of ALL
 * faces, quantised to 21 bits per axis (quant21), interleaved (orc_morton63)
 * and sorted ascending by (code, triangle index).  keys gets nc entries. */
static void close_order(const oscene *s, const uint8_t *mask, int64_t nc, mkey *keys)
{
    int64_t j = 0;
    for (int64_t t = 0; t < s->nt && j < nc; t++) {
        if (!mask[t]) continue;
        d3 g = s->g[t];
        keys[j].code = orc_morton63(quant21(g.x, s->glo.x, s->ghi.x),
                                    quant21(g.y, s->glo.y, s->ghi.y),
                                    quant21(g.z, s->glo.z, s->ghi.z));
        keys[j].tri = (int32_t)t;
        j++;
    }
    qsort(keys, (size_t)nc, sizeof(mkey), cmp_mkey);
}

/* The order close_order gives the faces with mask[t] != 0 (their triangle
 * indices into out, which holds one entry per set mask byte); returns how
 * many.  The patch sampling of orc_generate walks its strata in this order. */
ORC_API int64_t orc_close_order(void *sp, const uint8_t *mask, int64_t *out)
{
    const oscene *s = (const oscene *)sp;
    int64_t nc = 0;
    for (int64_t t = 0; t < s->nt; t++) nc += mask[t] != 0;
    mkey *keys = malloc(sizeof(mkey) * (size_t)(nc > 0 ? nc : 1));
    close_order(s, mask, nc, keys);
    for (int64_t i = 0; i < nc; i++) out[i] = keys[i].tri;
    free(keys);
    return nc;
}

/* Eq. 2 for a VPL at x (unit normal n, albedo rho, area D): reflected power */
static d3 patch_flux(const oscene *s, const olight *L, const ogen *G, int64_t k, d3 x, d3 n,
                     const double *rho, double D)
{
    d3 cl = ld3(L->center), P = ld3(L->power);
    d3 xo = add(x, scl(n, G->ray_eps));
    double acc = 0.0;
    if (L->type == 1) {
        /* Eq. 2 literally: G = D cos(w) / (4 pi r^2), w and r towards the light */
        d3 dv = sub(cl, x);
        double r = len(dv);
        double cw = dot(n, dv) / r;
        if (cw > 0.0 && !occluded(s, xo, cl, G->vis_mode))
            acc = D * cw / (4.0 * PI * r * r);
    } else {
        /* one-sided Lambertian square of power P: radiance P / (pi A_L);
         * incident power on area D estimated with light_samples points */
        d3 nl = ld3(L->normal);
        for (int32_t sidx = 0; sidx < G->light_samples; sidx++) {
            uint64_t w[4];
            rng4(G->seed, STREAM_LIGHT, (uint64_t)k, (uint64_t)sidx, w);
            d3 y = light_point(L, u01(w[0]), u01(w[1]));
            d3 dv = sub(y, x);
            double r2 = dot(dv, dv), r = sqrt(r2);
            double cw = dot(n, dv) / r;
            double cl_ = -dot(nl, dv) / r;
            if (cw > 0.0 && cl_ > 0.0 && !occluded(s, xo, y, G->vis_mode))
                acc += cw * cl_ / (PI * r2);
        }
        acc = D * acc / (double)G->light_samples;
    }
    return mk(rho[0] * P.x * acc, rho[1] * P.y * acc, rho[2] * P.z * acc);
}

ORC_API int64_t orc_generate(void *sp, const ocamera *cam, const olight *L, const ogen *G,
                             double *pos, double *nrm, double *flux, int64_t *tri,
                             int64_t *tag, oinfo *info)
{
    const oscene *s = (const oscene *)sp;
    memset(info, 0, sizeof(*info));
    const int64_t M = (int64_t)G->m_close + G->m_far;
    for (int64_t i = 0; i < 3 * M; i++) pos[i] = nrm[i] = flux[i] = 0.0;
    for (int64_t i = 0; i < M; i++) { tri[i] = -1; tag[i] = -1; }

    /* (1) close-range faces */
    uint8_t *close = calloc((size_t)(s->nt > 0 ? s->nt : 1), 1);
    int64_t nc = orc_classify(sp, cam, L, G->d_close, G->close_rule, close);
    info->n_close = nc;

    /* (2) patch sampling of the close range */
    if (G->m_close > 0) {
        if (nc == 0) {
            info->status = 6;
        } else {
            /* spatial order: Morton code of the centroid in the AABB of all
             * centroids, ties by triangle index */
            mkey *keys = malloc(sizeof(mkey) * nc);
            close_order(s, close, nc, keys);
            /* integer areas q_t = round(A_t 2^S) with S = 40 - exponent(max A) */
            double amax = 0.0;
            for (int64_t i = 0; i < nc; i++) amax = dmax(amax, s->area[keys[i].tri]);
            int ex;
            frexp(amax, &ex);
            int S = 40 - ex;
            info->shift_s = S;
            /* f(i): area prefix sum over the sorted list, f[0] = 0 */
            uint64_t *f = malloc(sizeof(uint64_t) * (nc + 1));
            f[0] = 0;
            for (int64_t i = 0; i < nc; i++)
                f[i + 1] = f[i] + (uint64_t)llround(ldexp(s->area[keys[i].tri], S));
            uint64_t F = f[nc];
            info->f_total = F;
            const uint64_t K = (uint64_t)G->m_close;
            double a_rep = ldexp((double)F, -S) / (double)K;
            info->a_rep = a_rep;
            for (uint64_t k = 0; k < K; k++) {
                uint64_t w[4];
                rng4(G->seed, STREAM_PATCH, k, 0, w);
                /* a point in stratum [kF/K, (k+1)F/K) */
                unsigned __int128 num = ((unsigned __int128)((k << 32) + (w[0] >> 32))) * F;
                uint64_t u = (uint64_t)(num / ((unsigned __int128)K << 32));
                /* g(u): index m with f(m) <= u < f(m+1) */
                int64_t lo = 0, hi = nc;   /* invariant f[lo] <= u < f[hi] */
                while (hi - lo > 1) {
                    int64_t mid = lo + (hi - lo) / 2;
                    if (f[mid] <= u) lo = mid; else hi = mid;
                }
                int64_t t = keys[lo].tri;
                if (G->patch_rule == 1) {
                    /* the faces overlapping the stratum [A, B) of the prefix */
                    uint64_t A = (uint64_t)(((unsigned __int128)k * F) / K);
                    uint64_t B = (uint64_t)(((unsigned __int128)(k + 1) * F) / K);
                    int64_t m0 = lo, m1 = lo;
                    while (m0 > 0 && f[m0] > A) m0--;              /* f[m0] <= A < f[m0 + 1] */
                    while (m1 + 1 < nc && f[m1 + 1] < B) m1++;     /* f[m1] < B <= f[m1 + 1] */
                    if (m1 > m0) {
                        /* set sum: each face's Eq. 2 at its centroid with the
                         * area it gives to the stratum; the VPL at the
                         * area-weighted centroid, normal the area-weighted
                         * normal, face the one giving the most area */
                        d3 fl = mk(0, 0, 0), xs = mk(0, 0, 0), ns = mk(0, 0, 0);
                        double Dsum = 0.0;
                        uint64_t wbest = 0;
                        int64_t tbest = keys[m0].tri;
                        for (int64_t m = m0; m <= m1; m++) {
                            uint64_t lo_m = f[m] > A ? f[m] : A, hi_m = f[m + 1] < B ? f[m + 1] : B;
                            if (hi_m <= lo_m) continue;
                            uint64_t wm = hi_m - lo_m;
                            int64_t tm = keys[m].tri;
                            double Dm = ldexp((double)wm, -S);
                            fl = add(fl, patch_flux(s, L, G, (int64_t)k, s->g[tm], s->n[tm], s->rho + 3 * tm, Dm));
                            xs = add(xs, scl(s->g[tm], Dm));
                            ns = add(ns, scl(s->n[tm], Dm));
                            Dsum += Dm;
                            if (wm > wbest) {
                                wbest = wm;
                                tbest = tm;
                            }
                        }
                        double nl = len(ns);
                        st3(pos + 3 * k, scl(xs, 1.0 / Dsum));
                        st3(nrm + 3 * k, nl > 0.0 ? scl(ns, 1.0 / nl) : s->n[tbest]);
                        st3(flux + 3 * k, fl);
                        tri[k] = tbest;
                        tag[k] = (int64_t)k;
                        continue;
                    }
                }
                /* uniform random point in triangle t */
                double r1 = u01(w[1]), r2 = u01(w[2]);
                double sr = sqrt(r1);
                d3 a = s->a[t], b = add(a, s->e1[t]), c = add(a, s->e2[t]);
                d3 x = add(add(scl(a, 1.0 - sr), scl(b, sr * (1.0 - r2))), scl(c, sr * r2));
                d3 fl = patch_flux(s, L, G, (int64_t)k, x, s->n[t], s->rho + 3 * t, a_rep);
                st3(pos + 3 * k, x);
                st3(nrm + 3 * k, s->n[t]);
                st3(flux + 3 * k, fl);
                tri[k] = t;
                tag[k] = (int64_t)k;
            }
            free(f);
            free(keys);
        }
    }

    /* (3) instant radiosity over the whole scene; only hits on the distant
     * part become VPLs, hits on the close range are discarded but the path
     * goes on */
    if (G->m_far > 0) {
        const int64_t base = G->m_close;
        int64_t kept = 0, p = 0, P = 0;
        const int64_t pmax = G->ir_max_paths;
        irray *rays = malloc(sizeof(irray) * (size_t)(G->max_bounces > 0 ? G->max_bounces : 1));
        while (kept < G->m_far && p < pmax) {
            int n = ir_path(s, L, G, p, rays);
            double thr[3] = {1.0, 1.0, 1.0};
            for (int32_t b = 1; b <= n && kept < G->m_far; b++) {
                const irray *r = &rays[b - 1];
                if (!r->front) break;
                int64_t k = r->k;
                for (int c = 0; c < 3; c++) thr[c] = thr[c] * s->rho[3 * k + c];
                if (!close[k]) {
                    int64_t i = base + kept;
                    st3(pos + 3 * i, r->x);
                    st3(nrm + 3 * i, s->n[k]);
                    st3(flux + 3 * i, mk(thr[0], thr[1], thr[2]));
                    tri[i] = k;
                    tag[i] = p * 16 + b;
                    kept++;
                    P = p + 1;
                }
            }
            p++;
        }
        free(rays);
        if (kept < G->m_far) { info->status = 7; P = pmax; }
        info->paths = P;
        info->m_far_kept = kept;
        d3 pw = ld3(L->power);
        for (int64_t i = 0; i < kept; i++) {
            double *fl = flux + 3 * (base + i);
            fl[0] = pw.x * fl[0] / (double)P;
            fl[1] = pw.y * fl[1] / (double)P;
            fl[2] = pw.z * fl[2] / (double)P;
        }
    }
    free(close);
    return info->status;
}

/* ------------------------------------------------------------------------ */
/* G-buffer: closest front-face hit through each requested pixel centre      */
/* ------------------------------------------------------------------------ */
ORC_API void orc_gbuffer(void *sp, const ocamera *cam, int64_t n, const int64_t *pix,
                         int32_t vis_mode, double *pos, double *nrm, double *rho, int64_t *tri)
{
    const oscene *s = (const oscene *)sp;
    frame F = cam_frame(cam);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; q++) {
        int64_t i = pix[q] % cam->width, j = pix[q] / cam->width;
        double sx = 2.0 * ((double)i + 0.5) / (double)cam->width - 1.0;
        double sy = 1.0 - 2.0 * ((double)j + 0.5) / (double)cam->height;
        d3 d = add(add(F.f, scl(F.r, sx * F.th)), scl(F.u, sy * F.tv));
        double t;
        int64_t k = closest(s, F.e, d, 0.0, &t, vis_mode);
        if (k >= 0 && dot(d, s->cr[k]) < 0.0) {
            st3(pos + 3 * q, add(F.e, scl(d, t)));
            st3(nrm + 3 * q, s->n[k]);
            for (int c = 0; c < 3; c++) rho[3 * q + c] = s->rho[3 * k + c];
            tri[q] = k;
        } else {
            st3(pos + 3 * q, mk(0, 0, 0));
            st3(nrm + 3 * q, mk(0, 0, 0));
            for (int c = 0; c < 3; c++) rho[3 * q + c] = 0.0;
            tri[q] = -1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Gather (Eq. 1, indirect part): every pixel sums all VPLs in index order   */
/* ------------------------------------------------------------------------ */
/* shading factor of one pair without visibility and without the receiver's
 * albedo: cos_i cos_y / (pi max(d^2, d2_min)) */
static double pair_term(d3 y, d3 ny, d3 x, d3 nx, double d2min)
{
    d3 d = sub(x, y);
    double d2 = dot(d, d);
    if (d2 == 0.0) return 0.0;
    double dl = sqrt(d2);
    double cy = dot(ny, d) / dl;
    double ci = -dot(nx, d) / dl;
    if (!(cy > 0.0) || !(ci > 0.0)) return 0.0;
    return ci * cy / (PI * dmax(d2, d2min));
}

ORC_API void orc_gather(void *sp, int64_t n, const double *y, const double *ny,
                        const double *rho, const int64_t *valid, int64_t M, const double *x,
                        const double *nx, const double *phi, double d2min, double eps,
                        int32_t vis_mode, double *out)
{
    const oscene *s = (const oscene *)sp;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; q++) {
        double L[3] = {0.0, 0.0, 0.0};
        if (valid[q] >= 0) {
            d3 yy = ld3(y + 3 * q), nyy = ld3(ny + 3 * q);
            d3 p = add(yy, scl(nyy, eps));
            for (int64_t i = 0; i < M; i++) {
                const double *fi = phi + 3 * i;
                if (fi[0] == 0.0 && fi[1] == 0.0 && fi[2] == 0.0) continue;
                d3 xi = ld3(x + 3 * i), ni = ld3(nx + 3 * i);
                double g = pair_term(yy, nyy, xi, ni, d2min);
                if (g == 0.0) continue;
                if (vis_mode != 2 && occluded(s, p, add(xi, scl(ni, eps)), vis_mode)) continue;
                for (int c = 0; c < 3; c++) L[c] = L[c] + fi[c] * g;
            }
        }
        for (int c = 0; c < 3; c++) out[3 * q + c] = rho[3 * q + c] / PI * L[c];
    }
}

/* Per-pair shading factor and visibility for one receiver, for flip
 * analysis: term[i] (no visibility), vis[i] (1 visible, 0 blocked, -1 not
 * traced because term is zero), margin[i] (orc_segment_margin, only where
 * want_margin[i] != 0). */
/* ------------------------------------------------------------------------ */
/* Rejection-sampled instant radiosity (the comparison method the paper     */
/* cites as r3): the light paths of plain instant radiosity, with no close   */
/* range; every hit is a candidate VPL; its contribution to the image is     */
/* estimated on a pilot grid of pixels (Eq. 1's pair term with visibility,   */
/* the receiver's albedo and the path's albedos, channel mean); a candidate  */
/* is kept with probability p = min(1, c / cbar), cbar the mean over the      */
/* candidates of all ir_max_paths paths, decided by Philox (seed, 5) counter */
/* (path, bounce); the first m_far kept in (path, bounce) order are the      */
/* VPLs, P = last kept path + 1, flux = power x albedos / (P p).             */
/* ------------------------------------------------------------------------ */
ORC_API int64_t orc_generate_rs(void *sp, const ocamera *cam, const olight *L, const ogen *G, int32_t pilot,
                                double d2min, double eps, double *pos, double *nrm, double *flux, int64_t *tri,
                                int64_t *tag, oinfo *info)
{
    const oscene *s = (const oscene *)sp;
    memset(info, 0, sizeof(*info));
    const int64_t M = G->m_far, pmax = G->ir_max_paths, B = G->max_bounces;
    for (int64_t i = 0; i < 3 * M; i++) pos[i] = nrm[i] = flux[i] = 0.0;
    for (int64_t i = 0; i < M; i++) { tri[i] = -1; tag[i] = -1; }
    /* candidates of every path, slot p * B + (b - 1) */
    const int64_t ns = pmax * B;
    d3 *cx = calloc((size_t)(ns > 0 ? ns : 1), sizeof(d3));
    d3 *cn = calloc((size_t)(ns > 0 ? ns : 1), sizeof(d3));
    double *ct = calloc((size_t)(ns > 0 ? 3 * ns : 1), sizeof(double));
    int64_t *ck = malloc(sizeof(int64_t) * (size_t)(ns > 0 ? ns : 1));
    double *cc = calloc((size_t)(ns > 0 ? ns : 1), sizeof(double));
    for (int64_t i = 0; i < ns; i++) ck[i] = -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < pmax; p++) {
        irray rays[64];
        irray *rp = B <= 64 ? rays : malloc(sizeof(irray) * (size_t)B);
        int n = ir_path(s, L, G, p, rp);
        double thr[3] = {1.0, 1.0, 1.0};
        for (int64_t b = 1; b <= n; b++) {
            const irray *r = &rp[b - 1];
            if (!r->front) break;
            int64_t k = r->k;
            for (int c = 0; c < 3; c++) thr[c] = thr[c] * s->rho[3 * k + c];
            int64_t slot = p * B + (b - 1);
            cx[slot] = r->x;
            cn[slot] = s->n[k];
            for (int c = 0; c < 3; c++) ct[3 * slot + c] = thr[c];
            ck[slot] = k;
        }
        if (rp != rays) free(rp);
    }
    /* pilot pixels: a pilot x ph grid over the same view */
    const int64_t pw = pilot, ph0 = ((int64_t)pilot * cam->height + cam->width / 2) / cam->width;
    const int64_t ph = ph0 > 0 ? ph0 : 1; /* round(pilot H / W), at least 1 */
    ocamera pc = *cam;
    pc.width = (int32_t)pw;
    pc.height = (int32_t)ph;
    const int64_t np = pw * ph;
    int64_t *pix = malloc(sizeof(int64_t) * (size_t)np);
    double *py = malloc(sizeof(double) * 3 * (size_t)np), *pn = malloc(sizeof(double) * 3 * (size_t)np);
    double *pr = malloc(sizeof(double) * 3 * (size_t)np);
    int64_t *pt = malloc(sizeof(int64_t) * (size_t)np);
    for (int64_t q = 0; q < np; q++) pix[q] = q;
    orc_gbuffer(sp, &pc, np, pix, G->vis_mode, py, pn, pr, pt);
    d3 P = ld3(L->power);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < ns; i++) {
        if (ck[i] < 0) continue;
        double acc = 0.0;
        d3 q = add(cx[i], scl(cn[i], eps));
        for (int64_t j = 0; j < np; j++) {
            if (pt[j] < 0) continue;
            d3 y = ld3(py + 3 * j), ny = ld3(pn + 3 * j);
            double g = pair_term(y, ny, cx[i], cn[i], d2min);
            if (g == 0.0) continue;
            if (occluded(s, add(y, scl(ny, eps)), q, G->vis_mode)) continue;
            double c = (pr[3 * j] * ct[3 * i] * P.x + pr[3 * j + 1] * ct[3 * i + 1] * P.y +
                        pr[3 * j + 2] * ct[3 * i + 2] * P.z) / 3.0;
            acc += g * c / PI;
        }
        cc[i] = acc;
    }
    double csum = 0.0;
    int64_t nvalid = 0;
    for (int64_t i = 0; i < ns; i++)
        if (ck[i] >= 0) {
            csum += cc[i];
            nvalid++;
        }
    const double cbar = nvalid > 0 ? csum / (double)nvalid : 0.0;
    /* acceptance in (path, bounce) order */
    int64_t kept = 0, Pp = 0;
    double *pk = malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    for (int64_t i = 0; i < ns && kept < M; i++) {
        if (ck[i] < 0) continue;
        int64_t p = i / B, b = i % B + 1;
        uint64_t w[4];
        rng4(G->seed, STREAM_REJECT, (uint64_t)p, (uint64_t)b, w);
        double prob = cbar > 0.0 ? dmin(1.0, cc[i] / cbar) : 1.0;
        if (!(u01(w[0]) < prob)) continue;
        st3(pos + 3 * kept, cx[i]);
        st3(nrm + 3 * kept, cn[i]);
        st3(flux + 3 * kept, mk(ct[3 * i], ct[3 * i + 1], ct[3 * i + 2]));
        tri[kept] = ck[i];
        tag[kept] = p * 16 + b;
        pk[kept] = prob;
        kept++;
        Pp = p + 1;
    }
    if (kept < M) { info->status = 7; Pp = pmax; }
    info->paths = Pp;
    info->m_far_kept = kept;
    for (int64_t i = 0; i < kept; i++) {
        double *fl = flux + 3 * i;
        fl[0] = P.x * fl[0] / ((double)Pp * pk[i]);
        fl[1] = P.y * fl[1] / ((double)Pp * pk[i]);
        fl[2] = P.z * fl[2] / ((double)Pp * pk[i]);
    }
    info->a_rep = cbar; /* here: the mean candidate contribution */
    free(cx); free(cn); free(ct); free(ck); free(cc); free(pix); free(py); free(pn); free(pr); free(pt); free(pk);
    return kept;
}

ORC_API void orc_pairs(void *sp, const double *y, const double *ny, int64_t M, const double *x,
                       const double *nx, double d2min, double eps, int32_t vis_mode,
                       const uint8_t *want_margin, double *term, int8_t *vis, double *margin)
{
    const oscene *s = (const oscene *)sp;
    d3 yy = ld3(y), nyy = ld3(ny);
    d3 p = add(yy, scl(nyy, eps));
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < M; i++) {
        d3 xi = ld3(x + 3 * i), ni = ld3(nx + 3 * i);
        term[i] = pair_term(yy, nyy, xi, ni, d2min);
        d3 q = add(xi, scl(ni, eps));
        vis[i] = term[i] == 0.0 ? -1 : (int8_t)!occluded(s, p, q, vis_mode);
        margin[i] = INFINITY;
        if (want_margin && want_margin[i]) {
            double pp[3] = {p.x, p.y, p.z}, qq[3] = {q.x, q.y, q.z};
            margin[i] = orc_segment_margin(sp, pp, qq);
        }
    }
}

/* threads of the parallel loops from now on (n >= 1) */
ORC_API void orc_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

ORC_API int32_t orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
