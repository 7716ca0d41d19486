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
constexpr int kDepthMax = 96;            // binary hierarchy depth, checked when a scene is built
constexpr int kStackMax = 160;           // >= 3 x levels of the 4-wide tree (<= 53) + 1
constexpr int kTraversalLimit = 1 << 16; // node visits per query before giving up
#ifndef VPL_BEAM
#define VPL_BEAM 1                       // shadow packets take the beam walk when they can
#endif
#ifndef VPL_BEAM_PAD
#define VPL_BEAM_PAD 3.814697265625e-06f // beam boxes widened by this x (|q| + |E|): 2^-18
#endif
#ifndef VPL_BEAM_WIDTH
#define VPL_BEAM_WIDTH 0.1f              // widest beam (spread of directions / length) walked as one
#endif
constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;

// --------------------------------------------------------------------------
// device view of an uploaded scene
// --------------------------------------------------------------------------
struct SceneView {
    int32_t n_tris;
    int32_t n_nodes;
    const float4 *tri;     // 3 per triangle, BVH leaf order: v0 (w = original id bits), e1, e2
    const float4 *nodes;   // 8 per 4-wide node (see Node4)
    const float4 *bnodes;  // the same nodes per child, 8 per node (beam walk)
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
// FP32 vectors.  Every operation has its rounding spelled out (fmaf where a
// product feeds a sum), so the compiler cannot fuse differently in the
// several instantiations of a kernel: a segment's visibility and a pair's
// shading terms come out bit for bit the same in every gather variant.
// --------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b)
{
    return make_float3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}
__device__ __forceinline__ float3 operator-(float3 a, float3 b)
{
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float3 operator*(float3 a, float s)
{
    return make_float3(__fmul_rn(a.x, s), __fmul_rn(a.y, s), __fmul_rn(a.z, s));
}
// a * s + b with one rounding per component
__device__ __forceinline__ float3 fma3(float3 a, float s, float3 b)
{
    return make_float3(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y), fmaf(a.z, s, b.z));
}
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, __fmul_rn(a.z, b.z))); }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return make_float3(fmaf(a.y, b.z, -__fmul_rn(a.z, b.y)), fmaf(a.z, b.x, -__fmul_rn(a.x, b.z)),
                       fmaf(a.x, b.y, -__fmul_rn(a.y, b.x)));
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
struct TriD { D3 a, b, c, e1, e2, cr, g; double area; };
__device__ __forceinline__ TriD tri_exact(const SceneView &s, int32_t t)
{
    TriD r;
    D3 a = dvert(s.verts, s.idx[3 * (int64_t)t]);
    D3 b = dvert(s.verts, s.idx[3 * (int64_t)t + 1]);
    D3 c = dvert(s.verts, s.idx[3 * (int64_t)t + 2]);
    r.a = a;
    r.b = b;
    r.c = c;
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
enum { kStreamPatch = 1, kStreamLight = 2, kStreamIR = 3, kStreamDirect = 4, kStreamReject = 5 };

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
    return __frcp_rn(fabsf(v) < tiny ? copysignf(tiny, v) : v); // correctly rounded, as 1.0f / v
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
    float u = __fmul_rn(dot(tv, pv), inv);
    if (u < 0.0f || u > 1.0f) return false;
    float3 qv = cross(tv, e1);
    float v = __fmul_rn(dot(r.d, qv), inv);
    if (v < 0.0f || __fadd_rn(u, v) > 1.0f) return false;
    t = __fmul_rn(dot(e2, qv), inv);
    return true;
}

// Moller-Trumbore for a shadow segment, without the division: the
// barycentric and segment bounds are compared against |det| after the signs
// are made positive (u in [0, |det|], v >= 0, u + v <= |det|, t in
// (0, |det|) -- the tests of tri_hit scaled by |det|); either side blocks.
__device__ __forceinline__ bool seg_block(const Ray &r, float4 v0, float4 e1v, float4 e2v)
{
    const float3 e1 = f3(e1v), e2 = f3(e2v);
    const float3 pv = cross(r.d, e2);
    const float det = dot(e1, pv);
    if (det == 0.0f) return false;
    const float sg = det < 0.0f ? -1.0f : 1.0f, ad = fabsf(det);
    const float3 tv = r.o - f3(v0);
    const float u = __fmul_rn(dot(tv, pv), sg);
    if (u < 0.0f || u > ad) return false;
    const float3 qv = cross(tv, e1);
    const float v = __fmul_rn(dot(r.d, qv), sg);
    if (v < 0.0f || __fadd_rn(u, v) > ad) return false;
    const float t = __fmul_rn(dot(e2, qv), sg);
    return t > 0.0f && t < ad;
}

// --------------------------------------------------------------------------
// 4-wide BVH nodes (8 float4 = 128 B): rows 0-5 lo.x / hi.x / lo.y / hi.y /
// lo.z / hi.z of the four child slots; row 6 (ibase, lbase, masks, runs)
// with masks bits 0-3 = leaf slots, bits 4-7 = internal slots; row 7 unused.
// A node's internal children are nodes ibase, ibase + 1, ... in slot order;
// leaf slot k holds the triangle slots lbase + off_k ... + cnt_k - 1 (byte k
// of runs: off_k in bits 0-3, cnt_k in bits 4-6); an empty slot holds a box
// no segment reaches.
// --------------------------------------------------------------------------
constexpr int kEmptyRef = (int)0x80000000;
// The same node per child (bnodes, same index, 8 float4 = 128 B): slot k in
// rows 2k = (lo.x, lo.y, lo.z, ref) and 2k + 1 = (hi.x, hi.y, hi.z, cnt),
// ref >= 0 an internal node, ~triangle slot for a leaf of cnt triangles,
// kEmptyRef none.  A lane reads its own child's box and reference with two
// 16-byte loads, the four lanes of a node one 128-byte line.

struct Node4 {
    float4 lx, hx, ly, hy, lz, hz;
    int ibase, lbase;           // first internal child node / first leaf triangle slot
    unsigned leafmask, intmask; // bit k: slot k holds a leaf / an internal node
    unsigned runs;              // byte k: leaf slot k's offset from lbase (bits 0-3), triangles (4-6)
    int ref[4], cnt[4];         // decoded per slot (load_node4 only)
};

// child bases and slot masks (row 6)
__device__ __forceinline__ void load_node4_meta(const float4 *p, Node4 &n)
{
    const float4 r = __ldg(p + 6);
    n.ibase = __float_as_int(r.x);
    n.lbase = __float_as_int(r.y);
    const unsigned m = __float_as_uint(r.z);
    n.leafmask = m & 15u;
    n.intmask = (m >> 4) & 15u;
    n.runs = __float_as_uint(r.w);
}

// whole node, with each slot's reference decoded: >= 0 internal node,
// < 0 leaf (~triangle slot, cnt 1), kEmptyRef none
__device__ __forceinline__ void load_node4(const float4 *nodes, int node, Node4 &n)
{
    const float4 *p = nodes + 8 * (int64_t)node;
    n.lx = __ldg(p);
    n.hx = __ldg(p + 1);
    n.ly = __ldg(p + 2);
    n.hy = __ldg(p + 3);
    n.lz = __ldg(p + 4);
    n.hz = __ldg(p + 5);
    load_node4_meta(p, n);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned below = (1u << k) - 1u;
        if ((n.leafmask >> k) & 1u) {
            n.ref[k] = ~(n.lbase + (int)((n.runs >> (8 * k)) & 15u));
            n.cnt[k] = (int)((n.runs >> (8 * k + 4)) & 7u);
        } else if ((n.intmask >> k) & 1u) {
            n.ref[k] = n.ibase + __popc(n.intmask & below);
            n.cnt[k] = 0;
        } else {
            n.ref[k] = kEmptyRef;
            n.cnt[k] = 0;
        }
    }
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// two FP32 FMAs in one instruction (f32x2, sm_100 and later); each lane is an
// ordinary round-to-nearest fma, so results equal fmaf element by element
__device__ __forceinline__ unsigned long long pack2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float4 fma4(const float4 &v, unsigned long long s2, unsigned long long c2)
{
    unsigned long long lo, hi;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(lo) : "l"(pack2(v.x, v.y)), "l"(s2), "l"(c2));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(hi) : "l"(pack2(v.z, v.w)), "l"(s2), "l"(c2));
    float4 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(lo));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.z), "=f"(r.w) : "l"(hi));
    return r;
}

__device__ __forceinline__ float comp(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// slab test of child k of a node against [tlo, thi]; te = entry parameter
__device__ __forceinline__ bool slab(const Ray &r, const Node4 &n, int k, float tlo, float thi, float &te)
{
    float ax = fmaf(comp(n.lx, k), r.inv.x, -r.oinv.x), bx = fmaf(comp(n.hx, k), r.inv.x, -r.oinv.x);
    float ay = fmaf(comp(n.ly, k), r.inv.y, -r.oinv.y), by = fmaf(comp(n.hy, k), r.inv.y, -r.oinv.y);
    float az = fmaf(comp(n.lz, k), r.inv.z, -r.oinv.z), bz = fmaf(comp(n.hz, k), r.inv.z, -r.oinv.z);
    float lo = fmax3(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), tlo));
    float hi = fmin3(fmaxf(ax, bx), fmaxf(ay, by), fminf(fmaxf(az, bz), thi));
    te = lo;
    return lo <= hi;
}

__device__ __forceinline__ void cswap(float &ta, int &ra, float &tb, int &rb)
{
    if (tb < ta) {
        float t = ta; ta = tb; tb = t;
        int q = ra; ra = rb; rb = q;
    }
}

// closest hit with t in (tmin, inf); ties to the lower original triangle id.
// Returns the original triangle id or -1.
static __device__ __noinline__ int closest_hit(const SceneView &s, const Ray &r, float tmin, float &tbest,
                                               int *status)
{
    int stack[kStackMax];
    int sp = 0, node = 0, best = -1, steps = 0;
    const float kInf = __int_as_float(0x7f800000);
    tbest = kInf;
    while (true) {
        Node4 n;
        load_node4(s.nodes, node, n);
        float te[4];
        int rf[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            rf[k] = n.ref[k];
            bool h = rf[k] != kEmptyRef && slab(r, n, k, tmin, tbest, te[k]);
            if (h && rf[k] < 0) {
                for (int q = ~rf[k]; q < ~rf[k] + n.cnt[k]; q++) {
                    float4 v0 = __ldg(s.tri + 3 * q);
                    float t;
                    int id = __float_as_int(v0.w);
                    if (tri_hit(r, v0, __ldg(s.tri + 3 * q + 1), __ldg(s.tri + 3 * q + 2), t) && t > tmin &&
                        (t < tbest || (t == tbest && id < best))) {
                        tbest = t;
                        best = id;
                    }
                }
                h = false;
            }
            if (!h) {          // only internal children that the ray enters stay
                te[k] = kInf;
                rf[k] = kEmptyRef;
            }
        }
        // nearest internal child next, the others pushed farthest first
        cswap(te[0], rf[0], te[1], rf[1]);
        cswap(te[2], rf[2], te[3], rf[3]);
        cswap(te[0], rf[0], te[2], rf[2]);
        cswap(te[1], rf[1], te[3], rf[3]);
        cswap(te[1], rf[1], te[2], rf[2]);
        bool overflow = false;
#pragma unroll
        for (int k = 3; k >= 1; k--)
            if (rf[k] != kEmptyRef && te[k] <= tbest) {
                if (sp >= kStackMax) overflow = true;
                else stack[sp++] = rf[k];
            }
        if (overflow) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
        if (rf[0] != kEmptyRef && te[0] <= tbest) {
            node = rf[0];
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
        Node4 n;
        load_node4(s.nodes, node, n);
        int next = -1;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float te;
            int rf = n.ref[k];
            if (rf == kEmptyRef || !slab(r, n, k, 0.0f, 1.0f, te)) continue;
            if (rf < 0) {
                for (int q = ~rf; q < ~rf + n.cnt[k]; q++)
                    if (seg_block(r, __ldg(s.tri + 3 * q), __ldg(s.tri + 3 * q + 1), __ldg(s.tri + 3 * q + 2)))
                        return true;
            } else if (next < 0) {
                next = rf;
            } else {
                if (sp >= kStackMax) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); return false; }
                stack[sp++] = rf;
            }
        }
        if (next >= 0) {
            node = next;
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
    for (int k = 0; k < s.n_tris; k++)
        if (seg_block(r, __ldg(s.tri + 3 * k), __ldg(s.tri + 3 * k + 1), __ldg(s.tri + 3 * k + 2))) return true;
    return false;
}

// --------------------------------------------------------------------------
// warp-wide packet traversal for shadow segments.  All 32 lanes call it
// together; lanes with want == false ride along.  Node and triangle loads are
// the same address in every lane (one transaction, broadcast).  Per node each
// lane forms a 4-bit mask of the children its segment enters; one OR-reduction
// over the warp gives the children any lane needs.  Leaf children are tested
// at once, each lane its own (divergent loads, one leaf per lane and round);
// among internal children the packet visits them in slot order (the
// builder puts the largest box first): it descends into the first and pushes
// the others on a warp-uniform stack in shared memory (`stk`, kStackMax
// entries per warp) with the next slot on top.  A distance-ordered descent
// saves a few node visits but costs more than it saves in per-node work.
// --------------------------------------------------------------------------
struct WarpCounters {
    uint32_t visits, tests; // per lane: nodes visited / triangles tested by its own ray
    uint32_t steps;         // per warp: packet traversal steps (same in every lane)
};

// The packet walk proper; ORIENTED (all live segments share direction
// signs) and the general case are separate instantiations, so each keeps
// only the ray values its slab test reads.
template <bool COUNT, bool ORIENTED>
__device__ __forceinline__ bool packet_walk(const SceneView &s, bool want, const Ray &r, bool occl, int &cache,
                                            int &cache2, int *stk, int *status, WarpCounters &wc, int fx, int fy,
                                            int fz)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long sx2 = pack2(r.inv.x, r.inv.x), cx2 = pack2(-r.oinv.x, -r.oinv.x);
    const unsigned long long sy2 = pack2(r.inv.y, r.inv.y), cy2 = pack2(-r.oinv.y, -r.oinv.y);
    const unsigned long long sz2 = pack2(r.inv.z, r.inv.z), cz2 = pack2(-r.oinv.z, -r.oinv.z);
    // lanes with nothing to test get plane offsets of 3e38: every entry
    // parameter is huge, so their slab tests fail without a predicate
    unsigned long long kx2 = cx2, ky2 = cy2, kz2 = cz2;
    if (!(want && !occl)) kx2 = ky2 = kz2 = pack2(3.0e38f, 3.0e38f);
    // the entry-plane row of each axis, as an address from which each node's row follows
    const float4 *bx = s.nodes + fx, *by = s.nodes + fy, *bz = s.nodes + fz;
    int sp = 0, node = 0, steps = 0;
    while (true) {
        Node4 n;
        const bool live = want && !occl;
        unsigned hits = 0;     // children this lane's segment enters
        if (ORIENTED) {
            const float4 *p = s.nodes + 8 * (int64_t)node;
            // entry rows from the walk's per-axis bases; each exit row is the
            // other row of its 32-byte pair (node rows are 128-byte aligned)
            const float4 *pex = bx + 8 * (int64_t)node, *pey = by + 8 * (int64_t)node, *pez = bz + 8 * (int64_t)node;
            const float4 *pxx = (const float4 *)((uintptr_t)pex ^ 16u), *pxy = (const float4 *)((uintptr_t)pey ^ 16u),
                         *pxz = (const float4 *)((uintptr_t)pez ^ 16u);
            // plane crossings of all four children, two per instruction
            const float4 ex = fma4(__ldg(pex), sx2, kx2), xx = fma4(__ldg(pxx), sx2, kx2);
            const float4 ey = fma4(__ldg(pey), sy2, ky2), xy = fma4(__ldg(pxy), sy2, ky2);
            const float4 ez = fma4(__ldg(pez), sz2, kz2), xz = fma4(__ldg(pxz), sz2, kz2);
            load_node4_meta(p, n);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float te = fmax3(comp(ex, k), comp(ey, k), fmaxf(comp(ez, k), 0.0f));
                const float tx = fmin3(comp(xx, k), comp(xy, k), fminf(comp(xz, k), 1.0f));
                if (te <= tx) hits |= 1u << k;
            }
        } else {
            load_node4(s.nodes, node, n);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float te;
                // empty slots hold a box no segment of a scene reaches: no test needed
                if (live && slab(r, n, k, 0.0f, 1.0f, te)) hits |= 1u << k;
            }
        }
        const unsigned leafmask = n.leafmask;
        if (COUNT) {
            wc.steps++;
            if (live) wc.visits++;
        }
        unsigned any = __reduce_or_sync(kFull, hits);
        if (any & leafmask) {
            // each lane tests the leaves its own segment enters, one per
            // round: the rounds are the most leaves any one lane enters,
            // not all the leaves any lane enters
            unsigned todo = hits & leafmask;
            while (__any_sync(kFull, todo != 0 && !occl)) {
                if (todo != 0 && !occl) {
                    const int k = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const unsigned run = n.runs >> (8 * k);
                    const int q0 = n.lbase + (int)(run & 15u), q1 = q0 + (int)((run >> 4) & 7u);
                    for (int q = q0; q < q1 && !occl; q++) {
                        if (COUNT) wc.tests++;
                        if (seg_block(r, __ldg(s.tri + 3 * q), __ldg(s.tri + 3 * q + 1), __ldg(s.tri + 3 * q + 2))) {
                            occl = true;
                            cache2 = cache;
                            cache = q;
                            kx2 = ky2 = kz2 = pack2(3.0e38f, 3.0e38f);
                        }
                    }
                }
            }
            if (__ballot_sync(kFull, want && !occl) == 0) break;
            any = __reduce_or_sync(kFull, occl ? 0u : hits);
        }
        unsigned need = any & n.intmask;
        if (need) {
            const int pick = __ffs(need) - 1;
            need &= need - 1;
            if (sp + __popc(need) > kStackMax) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
            // lanes 0-3 push the other children at once, lowest slot on top
            const int mk = lane & 3;
            if (lane < 4 && ((need >> mk) & 1u))
                stk[sp + __popc(need >> (mk + 1))] = n.ibase + __popc(n.intmask & ((1u << mk) - 1u));
            sp += __popc(need);
            node = n.ibase + __popc(n.intmask & ((1u << pick) - 1u));
        } else {
            if (sp == 0) break;
            __syncwarp();
            node = stk[--sp];
        }
        if (++steps > kTraversalLimit) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
    }
    __syncwarp();
    return occl;
}

// --------------------------------------------------------------------------
// Beam walk for shadow packets whose segments all end at one point.  The 32
// segments of a packet run from the pixels' points o_l to the same VPL point
// q, so every point of them is q + s e with s in [0, 1] and e = o_l - q in
// the box E = [El, Eh] (per axis, over the live lanes).  When no axis of E
// contains 0, a child box B can meet a segment only if
//     max(0, max_a min_e s_in_a(e)) <= min(1, min_a max_e s_out_a(e)),
// and since (P - q_a) / e_a is monotonic in e_a on E_a, each extreme is one
// of the two products with 1/El_a and 1/Eh_a.  That test is one per child
// box for the whole packet, not one per lane: each step takes up to
// kBeamNodes nodes off the stack, four lanes per node, one lane per child
// (its box and reference read from the per-child layout, bnodes).
// The boxes are widened by delta = 2^-18 (|q| + |E|) in the test, far more
// than the FP32 rounding of the test and of the per-lane slab tests, so it
// never drops a box a lane's own segment enters.  Leaf children the beam
// keeps are tested per lane exactly as in packet_walk (the same slab test on
// the lane's own segment, then its triangles), and a segment that enters a
// leaf box enters every ancestor box (the FP32 slab test is monotonic under
// box inclusion), so each lane tests the same triangles as in packet_walk
// and the answer is the same bit for bit.  A packet whose E spreads over
// more than VPL_BEAM_WIDTH of its length (a tile across a depth edge) keeps
// the per-lane walk: its beam would cover far more of the scene than its
// segments.
// --------------------------------------------------------------------------
constexpr int kBeamNodes = 8;    // nodes tested per step (four lanes each)
constexpr int kBeamStack = 512;  // per-warp stack entries of the beam walk
constexpr int kWalkStack = kBeamStack > kStackMax ? kBeamStack : kStackMax;
// per-warp shared slice of the beam walk: 9 float pairs of constants
// (+2 floats so that each warp's slice stays 16-byte aligned)
constexpr int kBeamConst = 20;
static_assert(kBeamConst % 4 == 0, "16-byte aligned per-warp slices");
static_assert(kBeamNodes >= 1 && kBeamNodes <= 8, "a warp holds at most eight groups of four lanes");

// float <-> int with the same order (for warp min / max reductions)
__device__ __forceinline__ int f2ord(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// (a, a) * (r1, r2) + (c1, c2) -> min and max of the two lanes
__device__ __forceinline__ void fma_pair(float a, unsigned long long r12, unsigned long long c12, float &lo, float &hi)
{
    unsigned long long v;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(v) : "l"(pack2(a, a)), "l"(r12), "l"(c12));
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
    lo = fminf(x, y);
    hi = fmaxf(x, y);
}

// plane constants of the beam test: reciprocals of E's ends (r*) and the
// terms -(q -+ delta) r of the widened entry (n*) and exit (x*) planes
__device__ __forceinline__ void beam_setup(float3 q, float3 El, float3 Eh, unsigned long long &rx,
                                           unsigned long long &ry, unsigned long long &rz, unsigned long long &nx,
                                           unsigned long long &xx, unsigned long long &ny, unsigned long long &xy,
                                           unsigned long long &nz, unsigned long long &xz)
{
    const float r1x = __frcp_rn(El.x), r2x = __frcp_rn(Eh.x);
    const float r1y = __frcp_rn(El.y), r2y = __frcp_rn(Eh.y);
    const float r1z = __frcp_rn(El.z), r2z = __frcp_rn(Eh.z);
    const float emax = fmaxf(fmaxf(fmaxf(fabsf(El.x), fabsf(Eh.x)), fmaxf(fabsf(El.y), fabsf(Eh.y))),
                             fmaxf(fabsf(El.z), fabsf(Eh.z)));
    const float delta = VPL_BEAM_PAD * (fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fabsf(q.z)) + emax);
    const float dx = El.x > 0.0f ? delta : -delta, dy = El.y > 0.0f ? delta : -delta,
                dz = El.z > 0.0f ? delta : -delta;
    rx = pack2(r1x, r2x);
    ry = pack2(r1y, r2y);
    rz = pack2(r1z, r2z);
    nx = pack2(-(q.x + dx) * r1x, -(q.x + dx) * r2x);
    xx = pack2(-(q.x - dx) * r1x, -(q.x - dx) * r2x);
    ny = pack2(-(q.y + dy) * r1y, -(q.y + dy) * r2y);
    xy = pack2(-(q.y - dy) * r1y, -(q.y - dy) * r2y);
    nz = pack2(-(q.z + dz) * r1z, -(q.z + dz) * r2z);
    xz = pack2(-(q.z - dz) * r1z, -(q.z - dz) * r2z);
}

// E over the lanes with lv set: min and max of e = -d per axis
__device__ __forceinline__ void beam_extent(bool lv, const Ray &r, float3 &El, float3 &Eh)
{
    const float ex = -r.d.x, ey = -r.d.y, ez = -r.d.z;
    El = make_float3(ord2f(__reduce_min_sync(kFull, lv ? f2ord(ex) : 0x7fffffff)),
                     ord2f(__reduce_min_sync(kFull, lv ? f2ord(ey) : 0x7fffffff)),
                     ord2f(__reduce_min_sync(kFull, lv ? f2ord(ez) : 0x7fffffff)));
    Eh = make_float3(ord2f(__reduce_max_sync(kFull, lv ? f2ord(ex) : (int)0x80000000)),
                     ord2f(__reduce_max_sync(kFull, lv ? f2ord(ey) : (int)0x80000000)),
                     ord2f(__reduce_max_sync(kFull, lv ? f2ord(ez) : (int)0x80000000)));
}

// fx, fy, fz: the per-lane walk's entry rows (odd: the hi plane, the
// segments run towards -axis); E lo / hi over live lanes, per axis, with no
// axis containing 0; nbuf: the warp's kBeamConst floats of shared memory
template <bool COUNT>
__device__ __forceinline__ bool beam_walk(const SceneView &s, bool want, const Ray &r, bool occl, int &cache,
                                       int &cache2, int *stk, float *nbuf, int *status, WarpCounters &wc, float3 q,
                                       float3 El, float3 Eh, int fx, int fy, int fz)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, k = lane & 3;
    const bool hx = fx & 1, hy = fy & 1, hz = fz & 1; // entry plane is the hi plane
    // the beam: reciprocals of E's ends, box widening, plane constants
    unsigned long long rx, ry, rz, nx, xx, ny, xy, nz, xz;
    beam_setup(q, El, Eh, rx, ry, rz, nx, xx, ny, xy, nz, xz);
    // the constants are the same in every lane: kept in the warp's shared
    // slice (read back as broadcasts) instead of 18 registers per lane
    unsigned long long *bc = reinterpret_cast<unsigned long long *>(nbuf);
    if (lane == 0) {
        bc[0] = rx; bc[1] = nx; bc[2] = xx; bc[3] = ry; bc[4] = ny; bc[5] = xy; bc[6] = rz; bc[7] = nz; bc[8] = xz;
    }
    __syncwarp();
    // per-lane exact slab terms (the same arithmetic as packet_walk<ORIENTED>)
    const float sx = r.inv.x, sy = r.inv.y, sz = r.inv.z;
    const float kx = -r.oinv.x, ky = -r.oinv.y, kz = -r.oinv.z;
    // The walk starts from the root's internal children, all pushed: their
    // boxes lie in the root's, which holds every triangle, so testing them
    // would only cull what the next step's tests of their children cull
    // anyway (the beam test is monotonic under box inclusion), one step
    // later.  A root with a leaf child (a scene of a few triangles) is
    // walked from the root.
    int sp;
    {
        const int rref = lane < 4 ? __float_as_int(__ldg(s.bnodes + 2 * lane).w) : kEmptyRef;
        const unsigned rl = __ballot_sync(kFull, rref < 0 && rref != kEmptyRef);
        const unsigned ri = __ballot_sync(kFull, rref >= 0);
        if (rl) {
            if (lane == 0) stk[0] = 0;
            sp = 1;
        } else {
            sp = __popc(ri);
            if (rref >= 0) stk[sp - 1 - __popc(ri & ((1u << lane) - 1u))] = rref;
        }
    }
    __syncwarp();
    int steps = 0;
    while (true) {
        // up to kBeamNodes nodes, while their pushes (<= 4 each) fit the stack
        const int F = sp + 3 * kBeamNodes <= kBeamStack ? (sp < kBeamNodes ? sp : kBeamNodes) : 1;
        const bool act = g < F;
        const int node = act ? stk[sp - 1 - g] : 0;
        sp -= F;
        __syncwarp();
        // lane k of a node's four reads child k (its box and reference) from
        // the per-child layout: the four lanes read the node's 128-byte line
        const float4 *p = s.bnodes + 8 * (int64_t)node + 2 * k;
        const float4 blo = __ldg(p), bhi = __ldg(p + 1);
        const int ref = __float_as_int(blo.w), tcnt = __float_as_int(bhi.w);
        const bool isint = ref >= 0, isleaf = ref < 0 && ref != kEmptyRef;
        // this lane's child: the per-lane walk's entry (en*) and exit (ex*) planes
        const float enx = hx ? bhi.x : blo.x, exx = hx ? blo.x : bhi.x;
        const float eny = hy ? bhi.y : blo.y, exy = hy ? blo.y : bhi.y;
        const float enz = hz ? bhi.z : blo.z, exz = hz ? blo.z : bhi.z;
        bool hit = false;
        if (act && (isleaf || isint)) {
            // seen from q, the segment enters through the per-lane exit plane
            float a0, a1, b0, b1, c0, c1, t;
            fma_pair(exx, bc[0], bc[1], a0, t);
            fma_pair(enx, bc[0], bc[2], t, a1);
            fma_pair(exy, bc[3], bc[4], b0, t);
            fma_pair(eny, bc[3], bc[5], t, b1);
            fma_pair(exz, bc[6], bc[7], c0, t);
            fma_pair(enz, bc[6], bc[8], t, c1);
            const float sin_ = fmax3(a0, b0, fmaxf(c0, 0.0f));
            const float sout = fmin3(a1, b1, fminf(c1, 1.0f));
            hit = sin_ <= sout;
        }
        const unsigned lh = __ballot_sync(kFull, hit && isleaf), ih = __ballot_sync(kFull, hit && isint);
        if (COUNT) {
            wc.steps++;
            if (want && !occl) wc.visits += F;
        }
        // leaves the beam keeps: each live lane first finds those its own
        // segment enters (the exact per-lane slab test), then tests their
        // triangles one leaf per round, every lane on its own leaf
        if (lh) {
            unsigned mine = 0, todo = lh;
            while (todo) {
                const int j = __ffs(todo) - 1;
                todo &= todo - 1;
                const float ax = __shfl_sync(kFull, enx, j), bx = __shfl_sync(kFull, exx, j);
                const float ay = __shfl_sync(kFull, eny, j), by = __shfl_sync(kFull, exy, j);
                const float az = __shfl_sync(kFull, enz, j), bz = __shfl_sync(kFull, exz, j);
                const float te = fmax3(fmaf(ax, sx, kx), fmaf(ay, sy, ky), fmaxf(fmaf(az, sz, kz), 0.0f));
                const float tx = fmin3(fmaf(bx, sx, kx), fmaf(by, sy, ky), fminf(fmaf(bz, sz, kz), 1.0f));
                if (te <= tx) mine |= 1u << j;
            }
            if (!(want && !occl)) mine = 0;
            while (__any_sync(kFull, mine != 0)) {
                const bool has = mine != 0;
                const int j = has ? __ffs(mine) - 1 : lane;
                mine &= mine - 1;
                const int lref = __shfl_sync(kFull, ref, j);
                const int lcnt = __shfl_sync(kFull, tcnt, j);
                if (has && !occl) {
                    const int q0 = ~lref, q1 = q0 + lcnt;
                    for (int t = q0; t < q1 && !occl; t++) {
                        if (COUNT) wc.tests++;
                        if (seg_block(r, __ldg(s.tri + 3 * t), __ldg(s.tri + 3 * t + 1), __ldg(s.tri + 3 * t + 2))) {
                            occl = true;
                            cache2 = cache;
                            cache = t;
                        }
                    }
                }
                if (occl) mine = 0;
            }
        }
        if (lh && __ballot_sync(kFull, want && !occl) == 0) break;
        if (ih) {
            const int n_push = __popc(ih);
            if (sp + n_push > kBeamStack) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
            // the first node's first child ends on top
            if (hit && isint) stk[sp + n_push - 1 - __popc(ih & ((1u << lane) - 1u))] = ref;
            sp += n_push;
        }
        if (sp == 0) break;
        __syncwarp();
        if (++steps > kTraversalLimit) { latch(status, VPL_ERR_TRAVERSAL_LIMIT); break; }
    }
    __syncwarp();
    return occl;
}

// `cache`, `cache2` (per lane) are the triangle slots of the last two
// triangles that blocked one of this lane's segments (most recent first), or
// -1.  They are tested before the traversal: neighbouring VPLs are usually
// hidden by the same triangle.  The answer is the same with or without them
// (a segment is blocked when any triangle blocks it).
// q: the end point every lane's segment shares (r.o + r.d up to rounding);
// beam: narrow packets may take the beam walk (else the per-lane walk only)
template <bool COUNT>
__device__ __forceinline__ bool warp_occluded(const SceneView &s, bool want, const Ray &r, float3 q, int &cache,
                                              int &cache2, int *stk, float *nbuf, int *status, WarpCounters &wc,
                                              bool beam)
{
    bool occl = false;
    if (want && cache >= 0) {
        if (COUNT) wc.tests++;
        if (seg_block(r, __ldg(s.tri + 3 * cache), __ldg(s.tri + 3 * cache + 1), __ldg(s.tri + 3 * cache + 2)))
            occl = true;
    }
    if (want && !occl && cache2 >= 0) {
        if (COUNT) wc.tests++;
        if (seg_block(r, __ldg(s.tri + 3 * cache2), __ldg(s.tri + 3 * cache2 + 1), __ldg(s.tri + 3 * cache2 + 2))) {
            occl = true;
            const int x = cache; cache = cache2; cache2 = x;
        }
    }
    unsigned alive = __ballot_sync(kFull, want && !occl);
    if (alive == 0) return occl;
    // Direction signs of the live segments, per axis.  When every live segment
    // of the packet points the same way along an axis, the entry plane of that
    // axis is the same box face for all of them, so the packet loads the near
    // and far rows by address and skips the per-lane min/max that orders the
    // two plane crossings (the usual case: 32 pixels of a small tile seen from
    // one VPL).  Otherwise it takes the general slab test.
    const unsigned nx = __ballot_sync(kFull, want && !occl && signbit(r.inv.x));
    const unsigned ny = __ballot_sync(kFull, want && !occl && signbit(r.inv.y));
    const unsigned nz = __ballot_sync(kFull, want && !occl && signbit(r.inv.z));
    const bool oriented = (nx == 0 || nx == alive) && (ny == 0 || ny == alive) && (nz == 0 || nz == alive);
    const int fx = nx ? 1 : 0, fy = ny ? 3 : 2, fz = nz ? 5 : 4; // row of each axis' entry plane
#if VPL_BEAM
    // the counting instantiation keeps the per-lane walk: its counters are
    // the work of each ray's own traversal (the algorithmic work of the
    // roofline), which the beam walk's conservative test would inflate
    if (!COUNT && beam && oriented) {
        // e = o - q = -d over the live lanes, per axis
        float3 El, Eh;
        beam_extent(want && !occl, r, El, Eh);
        // no axis of E may contain 0 (every segment crosses each axis' planes
        // one way), and the beam must be narrow: the spread of E against its
        // length, else (a tile across a depth edge) the box of directions
        // covers far more of the scene than the segments do
        const float spread = fmaxf(fmaxf(Eh.x - El.x, Eh.y - El.y), Eh.z - El.z);
        const float reach = fmaxf(fmaxf(fmaxf(fabsf(El.x), fabsf(Eh.x)), fmaxf(fabsf(El.y), fabsf(Eh.y))),
                                  fmaxf(fabsf(El.z), fabsf(Eh.z)));
        // every |e_a| at least 1e-30 (|q| + 1): the plane constants (q -+ delta) / e
        // of the test stay finite, so no extreme is lost to an overflow
        const float emin = fminf(fminf(fminf(fabsf(El.x), fabsf(Eh.x)), fminf(fabsf(El.y), fabsf(Eh.y))),
                                 fminf(fabsf(El.z), fabsf(Eh.z)));
        const float qmax = fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fabsf(q.z));
        if (El.x * Eh.x > 0.0f && El.y * Eh.y > 0.0f && El.z * Eh.z > 0.0f && spread <= VPL_BEAM_WIDTH * reach &&
            emin >= 1e-30f * (qmax + 1.0f))
            return beam_walk<COUNT>(s, want, r, occl, cache, cache2, stk, nbuf, status, wc, q, El, Eh, fx, fy, fz);
    }
#endif
    return oriented ? packet_walk<COUNT, true>(s, want, r, occl, cache, cache2, stk, status, wc, fx, fy, fz)
                    : packet_walk<COUNT, false>(s, want, r, occl, cache, cache2, stk, status, wc, fx, fy, fz);
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
            if (COUNT) wc.tests++;
            if (seg_block(r, v0, e1, e2)) occl = true;
        }
    }
    return occl;
}

} // namespace vpl
