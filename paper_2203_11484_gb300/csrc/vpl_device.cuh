// Device-side building blocks shared by the kernels of the VPL library:
// vector helpers, exact FP64 helpers for decisions, Philox4x64-10, Morton
// codes, ray/box and ray/triangle tests, and BVH traversal (single-ray
// closest hit / any hit, and a warp-wide packet any-hit for shadow rays).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vpl.h"

namespace vpl {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStackMax = 96;            // BVH depth is checked against this at build time
constexpr int kTraversalLimit = 1 << 16; // node visits per query before giving up
constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;

// --------------------------------------------------------------------------
// device view of an uploaded scene
// --------------------------------------------------------------------------
struct SceneView {
    int32_t n_tris;
    int32_t n_nodes;
    const float4 *tri;     // 3 per triangle, BVH leaf order: v0 (w = original id bits), e1, e2
    const float4 *nodes;   // 4 per internal node (see bvh.cu)
    const float4 *nrm;     // per original triangle: unit normal (FP32 from FP64)
    const float4 *rho;     // per original triangle: albedo
    const float *verts;    // original FP32 vertices
    const int32_t *idx;    // original triangle indices
    const double *gbox;    // [6] AABB of the FP64 centroids of all triangles (lo xyz, hi xyz)
};

struct LightView {
    float center[3], normal[3], edge_u[3], edge_v[3], power[3];
    int32_t type;
};

__device__ __forceinline__ void latch(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// --------------------------------------------------------------------------
// FP32 vectors
// --------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// --------------------------------------------------------------------------
// FP64 with every operation rounded on its own (no contraction): the
// close-range decisions, Morton codes and areas must equal the reference
// computation bit for bit.
// --------------------------------------------------------------------------
struct D3 { double x, y, z; };
__device__ __forceinline__ D3 dmk(double x, double y, double z) { D3 r = {x, y, z}; return r; }
__device__ __forceinline__ D3 dadd(D3 a, D3 b) { return dmk(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z)); }
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return dmk(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)); }
__device__ __forceinline__ D3 dscl(D3 a, double s) { return dmk(__dmul_rn(a.x, s), __dmul_rn(a.y, s), __dmul_rn(a.z, s)); }
__device__ __forceinline__ double ddot(D3 a, D3 b)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}
__device__ __forceinline__ D3 dcross(D3 a, D3 b)
{
    return dmk(__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)),
               __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
               __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ D3 dvert(const float *v, int32_t i)
{
    return dmk((double)v[3 * (int64_t)i], (double)v[3 * (int64_t)i + 1], (double)v[3 * (int64_t)i + 2]);
}
__device__ __forceinline__ D3 dld(const float *p) { return dmk((double)p[0], (double)p[1], (double)p[2]); }

// triangle quantities used by decisions (same operation order as the FP64 reference)
struct TriD { D3 a, e1, e2, cr, g; double area; };
__device__ __forceinline__ TriD tri_exact(const SceneView &s, int32_t t)
{
    TriD r;
    D3 a = dvert(s.verts, s.idx[3 * (int64_t)t]);
    D3 b = dvert(s.verts, s.idx[3 * (int64_t)t + 1]);
    D3 c = dvert(s.verts, s.idx[3 * (int64_t)t + 2]);
    r.a = a;
    r.e1 = dsub(b, a);
    r.e2 = dsub(c, a);
    r.cr = dcross(r.e1, r.e2);
    r.area = __dmul_rn(0.5, __dsqrt_rn(ddot(r.cr, r.cr)));
    D3 s3 = dadd(dadd(a, b), c);
    r.g = dmk(__ddiv_rn(s3.x, 3.0), __ddiv_rn(s3.y, 3.0), __ddiv_rn(s3.z, 3.0));
    return r;
}

// --------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (i, j, 0, 0),
// key (seed, stream)
// --------------------------------------------------------------------------
enum { kStreamPatch = 1, kStreamLight = 2, kStreamIR = 3 };

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__device__ __forceinline__ void rng4(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j, uint64_t w[4])
{
    w[0] = i; w[1] = j; w[2] = 0; w[3] = 0;
    philox4x64_10(w, seed, stream);
}

// top 24 bits as a number in [0, 1): exact in FP32 and FP64
__device__ __forceinline__ double u01(uint64_t w) { return (double)(w >> 40) * (1.0 / 16777216.0); }

// --------------------------------------------------------------------------
// Morton codes (21 bits per axis, x y z -> bits 3i+2, 3i+1, 3i)
// --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread21(uint64_t x)
{
    x &= 0x1fffffULL;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}
__device__ __forceinline__ uint64_t morton63(uint32_t qx, uint32_t qy, uint32_t qz)
{
    return (spread21(qx) << 2) | (spread21(qy) << 1) | spread21(qz);
}

// --------------------------------------------------------------------------
// rays
// --------------------------------------------------------------------------
struct Ray {
    float3 o, d;     // origin and (unnormalised) direction
    float3 inv, oinv; // 1/d and o/d for the slab test
};

__device__ __forceinline__ float safe_inv(float v)
{
    const float tiny = 1e-20f;
    return 1.0f / (fabsf(v) < tiny ? copysignf(tiny, v) : v);
}

__device__ __forceinline__ Ray make_ray(float3 o, float3 d)
{
    Ray r;
    r.o = o;
    r.d = d;
    r.inv = make_float3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    r.oinv = make_float3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    return r;
}

// Moller-Trumbore, inclusive barycentric bounds, either side; t of the line
__device__ __forceinline__ bool tri_hit(const Ray &r, float4 v0, float4 e1v, float4 e2v, float &t)
{
    float3 e1 = f3(e1v), e2 = f3(e2v);
    float3 pv = cross(r.d, e2);
    float det = dot(e1, pv);
    if (det == 0.0f) return false;
    float inv = 1.0f / det;
    float3 tv = r.o - f3(v0);
    float u = dot(tv, pv) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    float3 qv = cross(tv, e1);
    float v = dot(r.d, qv) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    t = dot(e2, qv) * inv;
    return true;
}

// slab test of both children of a node against [tlo, thi]
// node layout: n0 = (c0 lo.x, c0 hi.x, c0 lo.y, c0 hi.y), n1 = same for c1,
//              n2 = (c0 lo.z, c0 hi.z, c1 lo.z, c1 hi.z),
//              n3 = (child0, child1, leaf count0, leaf count1) as int bits
__device__ __forceinline__ void slab2(const Ray &r, float4 n0, float4 n1, float4 n2, float tlo,
                                      float thi, bool &h0, bool &h1, float &te0, float &te1)
{
    float ax = fmaf(n0.x, r.inv.x, -r.oinv.x), bx = fmaf(n0.y, r.inv.x, -r.oinv.x);
    float ay = fmaf(n0.z, r.inv.y, -r.oinv.y), by = fmaf(n0.w, r.inv.y, -r.oinv.y);
    float az = fmaf(n2.x, r.inv.z, -r.oinv.z), bz = fmaf(n2.y, r.inv.z, -r.oinv.z);
    float lo0 = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), tlo));
    float hi0 = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), thi));
    float cx = fmaf(n1.x, r.inv.x, -r.oinv.x), dx = fmaf(n1.y, r.inv.x, -r.oinv.x);
    float cy = fmaf(n1.z, r.inv.y, -r.oinv.y), dy = fmaf(n1.w, r.inv.y, -r.oinv.y);
    float cz = fmaf(n2.z, r.inv.z, -r.oinv.z), dz = fmaf(n2.w, r.inv.z, -r.oinv.z);
    float lo1 = fmaxf(fmaxf(fminf(cx, dx), fminf(cy, dy)), fmaxf(fminf(cz, dz), tlo));
    float hi1 = fminf(fminf(fmaxf(cx, dx), fmaxf(cy, dy)), fminf(fmaxf(cz, dz), thi));
    h0 = lo0 <= hi0;
    h1 = lo1 <= hi1;
    te0 = lo0;
    te1 = lo1;
}

__device__ __forceinline__ void load_node(const float4 *nodes, int node, float4 &n0, float4 &n1,
                                          float4 &n2, float4 &n3)
{
    const float4 *p = nodes + 4 * (int64_t)node;
    n0 = __ldg(p);
    n1 = __ldg(p + 1);
    n2 = __ldg(p + 2);
    n3 = __ldg(p + 3);
}

// closest hit with t in (tmin, inf); ties to the lower original triangle id.
// Returns the original triangle id or -1.
static __device__ __noinline__ int closest_hit(const SceneView &s, const Ray &r, float tmin, float &tbest,
                                        int *status)
{
    int stack[kStackMax];
    int sp = 0, node = 0, best = -1, steps = 0;
    tbest = __int_as_float(0x7f800000);
    while (true) {
        float4 n0, n1, n2, n3;
        load_node(s.nodes, node, n0, n1, n2, n3);
        bool h0, h1;
        float t0, t1;
        slab2(r, n0, n1, n2, tmin, tbest, h0, h1, t0, t1);
        int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        if (h0 && c0 < 0) {
            int first = ~c0, cnt = __float_as_int(n3.z);
            for (int k = first; k < first + cnt; k++) {
                float4 v0 = __ldg(s.tri + 3 * k), e1 = __ldg(s.tri + 3 * k + 1), e2 = __ldg(s.tri + 3 * k + 2);
                float t;
                int id = __float_as_int(v0.w);
                if (tri_hit(r, v0, e1, e2, t) && t > tmin && (t < tbest || (t == tbest && id < best))) {
                    tbest = t;
                    best = id;
                }
            }
            h0 = false;
        }
        if (h1 && c1 < 0) {
            int first = ~c1, cnt = __float_as_int(n3.w);
            for (int k = first; k < first + cnt; k++) {
                float4 v0 = __ldg(s.tri + 3 * k), e1 = __ldg(s.tri + 3 * k + 1), e2 = __ldg(s.tri + 3 * k + 2);
                float t;
                int id = __float_as_int(v0.w);
                if (tri_hit(r, v0, e1, e2, t) && t > tmin && (t < tbest || (t == tbest && id < best))) {
                    tbest = t;
                    best = id;
                }
            }
            h1 = false;
        }
        if (h0 && h1) {
            int nearc = t0 <= t1 ? c0 : c1, farc = t0 <= t1 ? c1 : c0;
            if (sp >= kStackMax) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
            stack[sp++] = farc;
            node = nearc;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
        if (++steps > kTraversalLimit) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
    }
    return best;
}

// any hit at t in (0, 1) of the segment r.o -> r.o + r.d (single ray)
static __device__ __noinline__ bool occluded1(const SceneView &s, const Ray &r, int *status)
{
    int stack[kStackMax];
    int sp = 0, node = 0, steps = 0;
    while (true) {
        float4 n0, n1, n2, n3;
        load_node(s.nodes, node, n0, n1, n2, n3);
        bool h0, h1;
        float t0, t1;
        slab2(r, n0, n1, n2, 0.0f, 1.0f, h0, h1, t0, t1);
        int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        if (h0 && c0 < 0) {
            int first = ~c0, cnt = __float_as_int(n3.z);
            for (int k = first; k < first + cnt; k++) {
                float t;
                if (tri_hit(r, __ldg(s.tri + 3 * k), __ldg(s.tri + 3 * k + 1), __ldg(s.tri + 3 * k + 2), t) &&
                    t > 0.0f && t < 1.0f)
                    return true;
            }
            h0 = false;
        }
        if (h1 && c1 < 0) {
            int first = ~c1, cnt = __float_as_int(n3.w);
            for (int k = first; k < first + cnt; k++) {
                float t;
                if (tri_hit(r, __ldg(s.tri + 3 * k), __ldg(s.tri + 3 * k + 1), __ldg(s.tri + 3 * k + 2), t) &&
                    t > 0.0f && t < 1.0f)
                    return true;
            }
            h1 = false;
        }
        if (h0 && h1) {
            if (sp >= kStackMax) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); return false; }
            stack[sp++] = t0 <= t1 ? c1 : c0;
            node = t0 <= t1 ? c0 : c1;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (sp == 0) return false;
            node = stack[--sp];
        }
        if (++steps > kTraversalLimit) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); return false; }
    }
}

// all-triangle variants (tiny scenes)
__device__ __forceinline__ int closest_brute(const SceneView &s, const Ray &r, float tmin, float &tbest)
{
    int best = -1;
    tbest = __int_as_float(0x7f800000);
    for (int k = 0; k < s.n_tris; k++) {
        float4 v0 = __ldg(s.tri + 3 * k);
        float t;
        int id = __float_as_int(v0.w);
        if (tri_hit(r, v0, __ldg(s.tri + 3 * k + 1), __ldg(s.tri + 3 * k + 2), t) && t > tmin &&
            (t < tbest || (t == tbest && id < best))) {
            tbest = t;
            best = id;
        }
    }
    return best;
}

__device__ __forceinline__ bool occluded_brute(const SceneView &s, const Ray &r)
{
    for (int k = 0; k < s.n_tris; k++) {
        float t;
        if (tri_hit(r, __ldg(s.tri + 3 * k), __ldg(s.tri + 3 * k + 1), __ldg(s.tri + 3 * k + 2), t) &&
            t > 0.0f && t < 1.0f)
            return true;
    }
    return false;
}

// --------------------------------------------------------------------------
// warp-wide packet traversal for shadow segments.  All 32 lanes call it
// together; lanes with want == false ride along.  The traversal stack is
// warp-uniform and lives in registers spread over the lanes (entry e in
// lane e % 32, slot e / 32), so pushes are a predicated move and pops a
// shuffle.  Node and triangle loads are the same address in every lane
// (one transaction, broadcast).
// --------------------------------------------------------------------------
struct WarpCounters {
    uint32_t visits, tests; // per lane: nodes visited / triangles tested by its own ray
    uint32_t steps;         // per warp: packet traversal steps (same in every lane)
};

template <bool COUNT>
__device__ __forceinline__ void leaf_any(const SceneView &s, const Ray &r, int first, int cnt,
                                         bool mask, bool &occl, WarpCounters &wc)
{
    for (int k = first; k < first + cnt; k++) {
        float4 v0 = __ldg(s.tri + 3 * k), e1 = __ldg(s.tri + 3 * k + 1), e2 = __ldg(s.tri + 3 * k + 2);
        if (mask && !occl) {
            float t;
            if (COUNT) wc.tests++;
            if (tri_hit(r, v0, e1, e2, t) && t > 0.0f && t < 1.0f) occl = true;
        }
    }
}

template <bool COUNT>
__device__ __forceinline__ bool warp_occluded(const SceneView &s, bool want, const Ray &r, int *status,
                                              WarpCounters &wc)
{
    const int lane = threadIdx.x & 31;
    bool occl = false;
    if (__ballot_sync(kFull, want) == 0) return false;
    int slot0 = 0, slot1 = 0, slot2 = 0; // stack entries held by this lane
    int sp = 0, node = 0, steps = 0;
    while (true) {
        float4 n0, n1, n2, n3;
        load_node(s.nodes, node, n0, n1, n2, n3);
        bool live = want && !occl;
        bool h0, h1;
        float t0, t1;
        slab2(r, n0, n1, n2, 0.0f, 1.0f, h0, h1, t0, t1);
        h0 = h0 && live;
        h1 = h1 && live;
        if (COUNT) {
            wc.steps++;
            if (live) wc.visits++;
        }
        int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        if (c0 < 0) {
            if (__any_sync(kFull, h0)) leaf_any<COUNT>(s, r, ~c0, __float_as_int(n3.z), h0, occl, wc);
            h0 = false;
        }
        if (c1 < 0) {
            if (__any_sync(kFull, h1)) leaf_any<COUNT>(s, r, ~c1, __float_as_int(n3.w), h1, occl, wc);
            h1 = false;
        }
        h0 = h0 && !occl;
        h1 = h1 && !occl;
        unsigned b0 = __ballot_sync(kFull, h0), b1 = __ballot_sync(kFull, h1);
        if (b0 && b1) {
            // visit first the child that most of the lanes needing both enter first
            unsigned both = b0 & b1;
            unsigned near0 = __ballot_sync(kFull, h0 && h1 && t0 <= t1);
            bool first0 = 2 * __popc(near0) >= __popc(both);
            int nearc = first0 ? c0 : c1, farc = first0 ? c1 : c0;
            if (sp >= kStackMax) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
            if (lane == (sp & 31)) {
                if (sp < 32) slot0 = farc; else if (sp < 64) slot1 = farc; else slot2 = farc;
            }
            sp++;
            node = nearc;
        } else if (b0) {
            node = c0;
        } else if (b1) {
            node = c1;
        } else {
            if (sp == 0 || __ballot_sync(kFull, want && !occl) == 0) break;
            sp--;
            int v = sp < 32 ? slot0 : (sp < 64 ? slot1 : slot2);
            node = __shfl_sync(kFull, v, sp & 31);
        }
        if (++steps > kTraversalLimit) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
    }
    return occl;
}

template <bool COUNT>
__device__ __forceinline__ bool warp_occluded_brute(const SceneView &s, bool want, const Ray &r,
                                                    WarpCounters &wc)
{
    bool occl = false;
    for (int k = 0; k < s.n_tris; k++) {
        if (__ballot_sync(kFull, want && !occl) == 0) break;
        if (COUNT) wc.steps++;
        float4 v0 = __ldg(s.tri + 3 * k), e1 = __ldg(s.tri + 3 * k + 1), e2 = __ldg(s.tri + 3 * k + 2);
        if (want && !occl) {
            float t;
            if (COUNT) wc.tests++;
            if (tri_hit(r, v0, e1, e2, t) && t > 0.0f && t < 1.0f) occl = true;
        }
    }
    return occl;
}

} // namespace vpl
