// Primary-ray G-buffer and the per-pixel indirect gather (Eq. 1 indirect
// term, Sec. 3 pipeline step (4)), plus the diagnostic kernels.
//
// Gather organisation: a warp owns an 8 x 4 pixel tile (tile_w x 32 / tile_w)
// and walks the whole VPL list in VPL tiles of 16, 32 or 64 (vpl_tile).  Each
// VPL tile is read with coalesced float4 loads into a per-warp slice of
// shared memory and then broadcast VPL by VPL to all 32 lanes, so the 32 shadow segments of one step all end at the same VPL and
// start from neighbouring pixels: the warp traverses the BVH as one packet
// (warp_occluded).  Tiles are handed out dynamically (an atomic counter) to a
// grid of resident blocks.  Each pixel sums its VPLs in one thread, in the
// order of the permutation v_order (the Morton order of the VPL positions
// that the gather entry points sort; the given order when there is none), so
// the result does not depend on tiling or batching.
#include <mutex>

#include "vpl_internal.h"

namespace vpl {

constexpr int kGatherWarps = 4;
constexpr int kMaxVplTile = 64; // the largest VPL tile a warp stages
// resident blocks per SM the gather is compiled for (register budget
// 65536 / (128 * blocks)); a build-time tuning knob.  With the beam walk's
// constants in shared memory the kernel fits 80 registers without spills:
// 6 blocks measured fastest (53.7 ms against 54.4 at 5 and 54.2 at 7)
#ifndef VPL_GATHER_MIN_BLOCKS
#define VPL_GATHER_MIN_BLOCKS 6
#endif

__device__ __forceinline__ float4 load_attr(const void *base, int64_t i, int fmt)
{
    if (fmt == VPL_FORMAT_FP16) {
        const __half2 *p = reinterpret_cast<const __half2 *>(base) + 2 * i;
        float2 a = __half22float2(p[0]), b = __half22float2(p[1]);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    return __ldg(reinterpret_cast<const float4 *>(base) + i);
}

__device__ __forceinline__ void store_attr_g(void *base, int64_t i, float4 v, int fmt)
{
    if (fmt == VPL_FORMAT_FP16) {
        __half2 *p = reinterpret_cast<__half2 *>(base) + 2 * i;
        p[0] = __floats2half2_rn(v.x, v.y);
        p[1] = __floats2half2_rn(v.z, v.w);
    } else {
        reinterpret_cast<float4 *>(base)[i] = v;
    }
}

// ==========================================================================
// G-buffer: closest hit through each pixel centre; empty on miss / back face
// ==========================================================================
__global__ void __launch_bounds__(128) gbuffer_kernel(SceneView s, CamArgs c, int brute, float4 *pos, void *nrm,
                                                      void *alb, int fmt, int *status)
{
    int x = blockIdx.x * 16 + (threadIdx.x & 15), y = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (x >= c.width || y >= c.height) return;
    int64_t p = (int64_t)y * c.width + x;
    float sx = 2.0f * ((float)x + 0.5f) / (float)c.width - 1.0f;
    float sy = 1.0f - 2.0f * ((float)y + 0.5f) / (float)c.height;
    float3 f = make_float3(c.f[0], c.f[1], c.f[2]), r = make_float3(c.r[0], c.r[1], c.r[2]),
           u = make_float3(c.u[0], c.u[1], c.u[2]);
    float3 d = f + r * (sx * c.th) + u * (sy * c.tv);
    Ray ray = make_ray(make_float3(c.eye[0], c.eye[1], c.eye[2]), d);
    float t;
    int k = brute ? closest_brute(s, ray, 0.0f, t) : closest_hit(s, ray, 0.0f, t, status);
    if (k >= 0) {
        float4 n = __ldg(s.nrm + k);
        if (dot(d, f3(n)) < 0.0f) {
            float3 hp = ray.o + d * t;
            pos[p] = make_float4(hp.x, hp.y, hp.z, __int_as_float(k));
            store_attr_g(nrm, p, make_float4(n.x, n.y, n.z, 0.0f), fmt);
            float4 a = __ldg(s.rho + k);
            store_attr_g(alb, p, make_float4(a.x, a.y, a.z, 0.0f), fmt);
            return;
        }
    }
    pos[p] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));
    store_attr_g(nrm, p, make_float4(0, 0, 0, 0), fmt);
    store_attr_g(alb, p, make_float4(0, 0, 0, 0), fmt);
}

cudaError_t gbuffer_build(const Exec &ex, const SceneView &s, const CamArgs &c, bool brute, float4 *pos,
                          void *nrm, void *alb, int fmt)
{
    if ((int64_t)c.width * c.height == 0) return cudaSuccess;
    dim3 grid((c.width + 15) / 16, (c.height + 7) / 8);
    gbuffer_kernel<<<grid, 128, 0, ex.stream>>>(s, c, brute ? 1 : 0, pos, nrm, alb, fmt, ex.status);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

// ==========================================================================
// gather
// ==========================================================================
struct GatherExtra {
    int *tile_counter;
    int n_tiles, tiles_x, tile_shift; // tile_w = 1 << tile_shift pixels, tile_h = 32 / tile_w
    const ViewDesc *views;            // BATCH: view table sorted by tile_begin
    int n_views;
    unsigned long long *counters;     // COUNT
    const int32_t *dbg_pixels;        // DEBUG: pixel list, else null
    int64_t n_dbg;
    int8_t *dbg_vis;
    const uint32_t *v_order;          // VPLs in this order (per view from vpl_begin), else as given
    const uint32_t *tile_order;       // tiles taken in this order, else in scan order
    unsigned *tile_cost;              // when set: SM cycles each tile took (cost-sampling pass)
};

template <int VIS, int PREC, bool COUNT, bool DEBUG, bool BATCH>
__global__ void __launch_bounds__(kGatherWarps * 32, VPL_GATHER_MIN_BLOCKS) gather_kernel(SceneView s, GatherArgs a, GatherExtra e, int *status)
{
    __shared__ float4 stage[kGatherWarps][3][kMaxVplTile];
    __shared__ int stack[kGatherWarps][kWalkStack]; // per-warp traversal stacks
    __shared__ __align__(16) float nodebuf[kGatherWarps][kBeamConst]; // per-warp beam constants
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gfmt = PREC == VPL_PREC_FP32 ? VPL_FORMAT_FP32 : VPL_FORMAT_FP16;
    const float eps = a.ray_eps, d2min = a.d2_min;
    // VPLs staged per warp at a time (16, 32 or 64; the ABI checks the value)
    const int vt = a.vpl_tile >= 1 && a.vpl_tile <= kMaxVplTile ? a.vpl_tile : kMaxVplTile;
    const bool beam = a.walk == 0; // narrow shadow packets take the beam walk
    WarpCounters wc = {0u, 0u, 0u};
    unsigned long long n_pairs = 0, n_rays = 0, n_blocked = 0;
    while (true) {
        int tile = 0;
        if (lane == 0) tile = atomicAdd(e.tile_counter, 1);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= e.n_tiles) break;
        // cost order and the cost-sampling pass: single-view gathers only
        constexpr bool kOrdered = !COUNT && !DEBUG && !BATCH;
        if (kOrdered && e.tile_order) tile = (int)__ldg(e.tile_order + tile);
        const long long clk0 = kOrdered && e.tile_cost ? clock64() : 0;
        // the view this tile belongs to
        int width = a.width, height = a.height, M = a.count, tiles_x = e.tiles_x, lt = tile;
        const float4 *g_pos = a.g_pos, *v_pos = a.v_pos;
        const void *g_nrm = a.g_nrm, *g_alb = a.g_alb, *v_nrm = a.v_nrm, *v_flux = a.v_flux;
        float4 *out = a.out;
        int vbeg = 0;
        if (BATCH) {
            int lo = 0, hi = e.n_views;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (e.views[mid].tile_begin <= tile) lo = mid; else hi = mid;
            }
            const ViewDesc *vd = e.views + lo;
            width = vd->width;
            height = vd->height;
            M = vd->count;
            tiles_x = vd->tiles_x;
            lt = tile - vd->tile_begin;
            g_pos = vd->g_pos;
            g_nrm = vd->g_nrm;
            g_alb = vd->g_alb;
            v_pos = vd->v_pos;
            v_nrm = vd->v_nrm;
            v_flux = vd->v_flux;
            out = vd->out;
            vbeg = vd->vpl_begin;
        }
        const uint32_t *ord = e.v_order ? e.v_order + vbeg : nullptr;
        int64_t p;
        bool inb; // pixel exists (in the image / in the debug list)
        if (DEBUG) {
            int64_t q = (int64_t)tile * 32 + lane;
            inb = q < e.n_dbg;
            p = inb ? e.dbg_pixels[q] : 0;
            if (inb && (p < 0 || p >= (int64_t)width * height)) { // a pixel the image does not have
                latch(status, VPL_ERR_INVALID_ARG);
                inb = false;
                p = 0;
            }
        } else {
            const int tw = 1 << e.tile_shift, th = 32 >> e.tile_shift;
            const int px = (lt % tiles_x) * tw + (lane & (tw - 1));
            const int py = (lt / tiles_x) * th + (lane >> e.tile_shift);
            inb = px < width && py < height;
            p = inb ? (int64_t)py * width + px : 0;
        }
        float4 gp = inb ? __ldg(g_pos + p) : make_float4(0, 0, 0, __int_as_float(-1));
        const bool valid = inb && __float_as_int(gp.w) >= 0;
        float4 gn = valid ? load_attr(g_nrm, p, gfmt) : make_float4(0, 0, 0, 0);
        const float3 y = f3(gp), ny = f3(gn);
        const float3 o = fma3(ny, eps, y);
        int occ_cache = -1, occ_cache2 = -1;   // last blocking triangles of this pixel
        float ax = 0.0f, ay = 0.0f, az = 0.0f; // running sums
        float cx = 0.0f, cy_ = 0.0f, cz = 0.0f; // Kahan compensation
        for (int base = 0; base < M; base += vt) {
            // a BVH walk that hit its limit ends the launch early (the method's
            // own degenerate cases, such as an empty close range, do not)
            int st = lane == 0 ? *(volatile int *)status : 0;
            if (__shfl_sync(kFull, st, 0) == VPL_ERR_TRAVERSAL_LIMIT) break;
            for (int l = lane; l < vt; l += 32) {
                const int i = base + l;
                if (i < M) {
                    const int src = ord ? (int)__ldg(ord + i) : i;
                    const float4 vp = __ldg(v_pos + src);
                    float4 vf = load_attr(v_flux, src, gfmt);
                    if (gfmt == VPL_FORMAT_FP16) { // FP16 colour x FP32 magnitude (pos.w)
                        vf.x *= vp.w;
                        vf.y *= vp.w;
                        vf.z *= vp.w;
                    }
                    // a VPL without flux is staged with a zero normal: its
                    // cosine is never positive, so no pixel wants it
                    const bool lit = vf.x != 0.0f || vf.y != 0.0f || vf.z != 0.0f;
                    stage[wid][0][l] = vp;
                    stage[wid][1][l] = lit ? load_attr(v_nrm, src, gfmt) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    stage[wid][2][l] = vf;
                }
            }
            __syncwarp();
            const int cnt = min(vt, M - base);
            for (int j = 0; j < cnt; j++) {
                const float4 xp = stage[wid][0][j], xn = stage[wid][1][j];
                const float3 d = f3(xp) - y;
                const float d2 = dot(d, d);
                const float cosy = dot(ny, d), cosi = -dot(f3(xn), d);
                const bool want = valid && cosy > 0.0f && cosi > 0.0f && d2 > 0.0f;
                bool vis = true;
                // most VPLs light none of a tile's pixels (a cosine or the
                // flux is zero): the shadow rays are skipped warp-uniformly
                if (VIS == VPL_VIS_BVH) {
                    if (__any_sync(kFull, want)) {
                        const float3 q = fma3(f3(xn), eps, f3(xp));
                        vis = !warp_occluded<COUNT>(s, want, make_ray(o, q - o), q, occ_cache, occ_cache2,
                                                    stack[wid], nodebuf[wid], status, wc, beam);
                    }
                } else if (VIS == VPL_VIS_BRUTE) {
                    if (__any_sync(kFull, want)) {
                        const float3 q = fma3(f3(xn), eps, f3(xp));
                        vis = !warp_occluded_brute<COUNT>(s, want, make_ray(o, q - o), wc);
                    }
                }
                if (COUNT) {
                    n_pairs += valid ? 1 : 0;
                    n_rays += want ? 1 : 0;
                    n_blocked += (want && !vis) ? 1 : 0;
                }
                if (DEBUG && inb) {
                    const int64_t v = ord ? (int64_t)__ldg(ord + base + j) : base + j; // as given
                    e.dbg_vis[((int64_t)tile * 32 + lane) * M + v] = want ? (vis ? 1 : 0) : -1;
                }
                if (want && vis) {
                    const float4 xf = stage[wid][2][j]; // the flux only where the pair contributes
                    const float g = __fdividef(cosi * cosy, d2 * fmaxf(d2, d2min));
                    if (PREC == VPL_PREC_FP16_KAHAN) {
                        float yv = fmaf(xf.x, g, -cx), t = __fadd_rn(ax, yv);
                        cx = __fsub_rn(__fsub_rn(t, ax), yv); ax = t;
                        yv = fmaf(xf.y, g, -cy_); t = __fadd_rn(ay, yv);
                        cy_ = __fsub_rn(__fsub_rn(t, ay), yv); ay = t;
                        yv = fmaf(xf.z, g, -cz); t = __fadd_rn(az, yv);
                        cz = __fsub_rn(__fsub_rn(t, az), yv); az = t;
                    } else {
                        ax = fmaf(xf.x, g, ax);
                        ay = fmaf(xf.y, g, ay);
                        az = fmaf(xf.z, g, az);
                    }
                }
            }
            __syncwarp();
        }
        if (kOrdered && e.tile_cost && lane == 0) {
            const long long c = clock64() - clk0;
            e.tile_cost[tile] = (unsigned)(c < 0 ? 0 : c > 0xffffffffLL ? 0xffffffffLL : c);
        }
        if (!DEBUG && inb && out) {
            float4 rho = valid ? load_attr(g_alb, p, gfmt) : make_float4(0, 0, 0, 0);
            const float k = 1.0f / (kPi * kPi);
            out[p] = make_float4(rho.x * ax * k, rho.y * ay * k, rho.z * az * k, 0.0f);
        }
    }
    if (COUNT) {
        unsigned long long v[6] = {n_pairs, n_rays, (unsigned long long)wc.visits, (unsigned long long)wc.tests,
                                   n_blocked, lane == 0 ? (unsigned long long)wc.steps : 0ULL};
        for (int k = 0; k < 6; k++) {
            unsigned long long x = v[k];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(kFull, x, off);
            if (lane == 0) atomicAdd(e.counters + k, x);
        }
    }
}

template <int VIS, int PREC, bool COUNT, bool DEBUG, bool BATCH>
static cudaError_t launch_gather(const Exec &ex, const SceneView &s, const GatherArgs &a, GatherExtra e)
{
    auto kern = gather_kernel<VIS, PREC, COUNT, DEBUG, BATCH>;
    int dev = 0, sms = 0, per_sm = 0;
    VPL_TRY(cudaGetDevice(&dev));
    VPL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VPL_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGatherWarps * 32, 0));
    if (per_sm < 1) per_sm = 1;
    if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
    int64_t want = (e.n_tiles + kGatherWarps - 1) / kGatherWarps;
    int64_t cap = (int64_t)sms * per_sm;
    unsigned grid = (unsigned)(want < cap ? want : cap);
    if (grid == 0) grid = 1;
    kern<<<grid, kGatherWarps * 32, 0, ex.stream>>>(s, a, e, ex.status);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

template <bool COUNT, bool DEBUG, bool BATCH>
static cudaError_t dispatch(const Exec &ex, const SceneView &s, const GatherArgs &a, GatherExtra e)
{
#define VPL_CASE(V, P)                                                                  \
    if (a.visibility == V && a.precision == P) return launch_gather<V, P, COUNT, DEBUG, BATCH>(ex, s, a, e);
    VPL_CASE(VPL_VIS_BVH, VPL_PREC_FP32)
    VPL_CASE(VPL_VIS_BRUTE, VPL_PREC_FP32)
    VPL_CASE(VPL_VIS_NONE, VPL_PREC_FP32)
    VPL_CASE(VPL_VIS_BVH, VPL_PREC_FP16_KAHAN)
    VPL_CASE(VPL_VIS_BVH, VPL_PREC_FP16_PLAIN)
    VPL_CASE(VPL_VIS_BRUTE, VPL_PREC_FP16_KAHAN)
    VPL_CASE(VPL_VIS_BRUTE, VPL_PREC_FP16_PLAIN)
    VPL_CASE(VPL_VIS_NONE, VPL_PREC_FP16_KAHAN)
    VPL_CASE(VPL_VIS_NONE, VPL_PREC_FP16_PLAIN)
#undef VPL_CASE
    return cudaErrorInvalidValue;
}

int tile_shift_of(int tile_w)
{
    switch (tile_w) {
    case 4: return 2;
    case 16: return 4;
    case 32: return 5;
    default: return 3; // 8 x 4
    }
}

static GatherExtra single_view_extra(const GatherArgs &a, int *counter)
{
    GatherExtra e;
    e.tile_counter = counter;
    e.tile_shift = tile_shift_of(a.tile_w);
    const int tw = 1 << e.tile_shift, th = 32 >> e.tile_shift;
    e.tiles_x = (a.width + tw - 1) / tw;
    e.n_tiles = e.tiles_x * ((a.height + th - 1) / th);
    e.views = nullptr;
    e.n_views = 0;
    e.counters = nullptr;
    e.dbg_pixels = nullptr;
    e.n_dbg = 0;
    e.dbg_vis = nullptr;
    e.v_order = nullptr;
    e.tile_order = nullptr;
    e.tile_cost = nullptr;
    return e;
}

// ---------------------------------------------------------------------------
// VPL order of a gather.  The image is the same sum in any order (up to FP32
// rounding); the order only steers speed: consecutive VPLs close in space
// send each warp's shadow packets through the same part of the BVH and let
// the per-pixel occluder cache hit.  Order = 42-bit Morton code (14 bits per
// axis) of the VPL position in the scene box, ties by index (a stable sort);
// in a batch each view's VPLs are ordered on their own (view index above the
// code).
// ---------------------------------------------------------------------------
__global__ void vpl_order_keys_kernel(const double *gbox, const float4 *v_pos, const ViewDesc *views, int n_views,
                                      int64_t total, uint64_t *keys, uint32_t *vals)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int view = 0;
    int64_t local = g;
    const float4 *vp = v_pos;
    if (views) {
        int lo = 0, hi = n_views;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (views[mid].vpl_begin <= g) lo = mid; else hi = mid;
        }
        view = lo;
        local = g - views[lo].vpl_begin;
        vp = views[lo].v_pos;
    }
    const float4 p = __ldg(vp + local);
    const float c[3] = {p.x, p.y, p.z};
    uint32_t q[3];
    for (int a = 0; a < 3; a++) {
        const float lo = (float)gbox[a], ext = (float)gbox[3 + a] - lo;
        const float u = ext > 0.0f ? (c[a] - lo) / ext : 0.0f;
        q[a] = (uint32_t)fminf(fmaxf(floorf(u * 16384.0f), 0.0f), 16383.0f);
    }
    keys[g] = ((uint64_t)view << 42) | morton63(q[0], q[1], q[2]);
    vals[g] = (uint32_t)local;
}

static cudaError_t vpl_order(const Exec &ex, const SceneView &s, const float4 *v_pos, const ViewDesc *views,
                             int n_views, int64_t total, Tmp &order)
{
    Tmp keys;
    VPL_TRY(keys.alloc(ex, sizeof(uint64_t) * total));
    VPL_TRY(order.alloc(ex, sizeof(uint32_t) * total));
    vpl_order_keys_kernel<<<grid_for(total, 256), 256, 0, ex.stream>>>(s.gbox, v_pos, views, n_views, total,
                                                                       keys.as<uint64_t>(), order.as<uint32_t>());
    VPL_LAUNCHED(ex);
    int bits = 42;
    while (bits < 64 && ((int64_t)1 << (bits - 42)) < n_views) bits++;
    return radix_sort_pairs(ex, keys.as<uint64_t>(), order.as<uint32_t>(), nullptr, total, bits);
}

// ---------------------------------------------------------------------------
// Tile order of a single-view gather.  The persistent grid takes tiles from a
// queue; tiles differ in cost by an order of magnitude or more (a tile whose
// pixels see most VPLs unblocked walks the BVH for nearly every VPL), and a
// costly tile taken late sets the end of the launch.  With tile_order 2 (or
// 0 and a large VPL set) a first pass gathers a sample of the VPLs into no
// image and records the SM cycles each tile took; the main pass then takes
// the tiles most costly first (ties in scan order).  The order changes speed
// only: each pixel is summed by one thread over the same VPLs in the same
// order either way.
// ---------------------------------------------------------------------------
#ifndef VPL_COST_SAMPLE
#define VPL_COST_SAMPLE 64
#endif
constexpr int kCostSample = VPL_COST_SAMPLE; // sample VPLs per tile in the cost pass (build-time knob)
constexpr int kCostOrderAuto = 8192;    // tile_order 0: cost order from this many VPLs on

__global__ void sample_order_kernel(const uint32_t *order, int64_t stride, int64_t n, uint32_t *sub)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sub[i] = order ? order[i * stride] : (uint32_t)(i * stride);
}

__global__ void cost_keys_kernel(const unsigned *cost, int n, uint64_t *keys, uint32_t *vals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = 0xffffffffULL - cost[i]; // ascending keys: most costly first
    vals[i] = (uint32_t)i;
}

static cudaError_t cost_order(const Exec &ex, const SceneView &s, const GatherArgs &a, const GatherExtra &e,
                              int *counter, Tmp &tiles)
{
    const int64_t stride = (a.count + kCostSample - 1) / kCostSample;
    const int64_t n_sample = (a.count + stride - 1) / stride;
    Tmp sub, cost, keys;
    VPL_TRY(sub.alloc(ex, sizeof(uint32_t) * n_sample));
    VPL_TRY(cost.alloc(ex, sizeof(unsigned) * e.n_tiles));
    VPL_TRY(keys.alloc(ex, sizeof(uint64_t) * e.n_tiles));
    VPL_TRY(tiles.alloc(ex, sizeof(uint32_t) * e.n_tiles));
    VPL_TRY(cudaMemsetAsync(cost.p, 0, sizeof(unsigned) * e.n_tiles, ex.stream));
    sample_order_kernel<<<grid_for(n_sample, 256), 256, 0, ex.stream>>>(e.v_order, stride, n_sample,
                                                                         sub.as<uint32_t>());
    VPL_LAUNCHED(ex);
    GatherArgs as = a;
    as.count = (int32_t)n_sample;
    as.out = nullptr; // the sample pass writes no image
    GatherExtra es = e;
    es.tile_counter = counter;
    es.v_order = sub.as<uint32_t>();
    es.tile_cost = cost.as<unsigned>();
    VPL_TRY(cudaMemsetAsync(counter, 0, sizeof(int), ex.stream));
    VPL_TRY((dispatch<false, false, false>(ex, s, as, es)));
    cost_keys_kernel<<<grid_for(e.n_tiles, 256), 256, 0, ex.stream>>>(cost.as<unsigned>(), e.n_tiles,
                                                                       keys.as<uint64_t>(), tiles.as<uint32_t>());
    VPL_LAUNCHED(ex);
    return radix_sort_pairs(ex, keys.as<uint64_t>(), tiles.as<uint32_t>(), nullptr, e.n_tiles, 32);
}

static cudaError_t run_gather(const Exec &ex, const SceneView &s, const GatherArgs &a, bool count,
                              unsigned long long *counters, const int32_t *pixels, int64_t n_pixels, int8_t *vis)
{
    const int64_t npx = (int64_t)a.width * a.height;
    if (pixels == nullptr && npx == 0) return cudaSuccess;
    if (pixels != nullptr && n_pixels == 0) return cudaSuccess;
    Tmp ctr, order, tiles;
    VPL_TRY(ctr.alloc(ex, 2 * sizeof(int)));
    VPL_TRY(cudaMemsetAsync(ctr.p, 0, sizeof(int), ex.stream));
    GatherExtra e = single_view_extra(a, ctr.as<int>());
    if (a.count > 1) {
        VPL_TRY(vpl_order(ex, s, a.v_pos, nullptr, 1, a.count, order));
        e.v_order = order.as<uint32_t>();
    }
    const bool by_cost = a.tile_order == 2 || (a.tile_order == 0 && a.count >= kCostOrderAuto);
    if (!count && !pixels && by_cost && a.count > 0 && e.n_tiles > 1) {
        VPL_TRY(cost_order(ex, s, a, e, ctr.as<int>() + 1, tiles));
        e.tile_order = tiles.as<uint32_t>();
    }
    if (pixels) e.n_tiles = (int)((n_pixels + 31) / 32);
    e.counters = counters;
    e.dbg_pixels = pixels;
    e.n_dbg = n_pixels;
    e.dbg_vis = vis;
    if (pixels) return dispatch<false, true, false>(ex, s, a, e);
    if (count) return dispatch<true, false, false>(ex, s, a, e);
    return dispatch<false, false, false>(ex, s, a, e);
}

// many views in one persistent launch: tiles of all views in one queue
cudaError_t gather_batch(const Exec &ex, const SceneView &s, const GatherArgs &a, const ViewDesc *views, int n_views,
                         int n_tiles, int tile_shift, int *counter, int64_t n_vpls)
{
    if (n_tiles == 0) return cudaSuccess;
    VPL_TRY(cudaMemsetAsync(counter, 0, sizeof(int), ex.stream));
    GatherExtra e = single_view_extra(a, counter);
    Tmp order;
    if (n_vpls > 1) {
        VPL_TRY(vpl_order(ex, s, nullptr, views, n_views, n_vpls, order));
        e.v_order = order.as<uint32_t>();
    }
    e.views = views;
    e.n_views = n_views;
    e.n_tiles = n_tiles;
    e.tile_shift = tile_shift;
    return dispatch<false, false, true>(ex, s, a, e);
}

cudaError_t gather(const Exec &ex, const SceneView &s, const GatherArgs &a)
{
    return run_gather(ex, s, a, false, nullptr, nullptr, 0, nullptr);
}

cudaError_t gather_counters(const Exec &ex, const SceneView &s, const GatherArgs &a, unsigned long long *counters)
{
    VPL_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * 6, ex.stream));
    return run_gather(ex, s, a, true, counters, nullptr, 0, nullptr);
}

cudaError_t gather_visibility(const Exec &ex, const SceneView &s, const GatherArgs &a, const int32_t *pixels,
                              int64_t n_pixels, int8_t *vis)
{
    return run_gather(ex, s, a, false, nullptr, pixels, n_pixels, vis);
}

// ==========================================================================
// gather that allocates nothing
// ==========================================================================
// For callers that may not allocate device memory while they run, the
// tile counter of the dynamic scheduler lives in this file-scope array (256
// bytes, held by every device that loads the library until the process
// exits) instead of the context's memory pool.  All such calls share it.
constexpr int kNoAllocScratchInts = 64;
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocScratchInts];
constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static int *g_noalloc_addr[kNoAllocMaxDevices] = {};

cudaError_t gather_noalloc(const Exec &ex, const SceneView &s, const GatherArgs &a)
{
    const int64_t npx = (int64_t)a.width * a.height;
    if (npx == 0) return cudaSuccess;
    int dev = 0;
    VPL_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    int *scratch = nullptr;
    {
        // once per device, with that device current: host code only knows a
        // stand-in for the array, the kernel needs its device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            VPL_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_addr[dev] = static_cast<int *>(p);
        }
        scratch = g_noalloc_addr[dev];
    }
    // the array keeps the previous call's counter: start this one at zero
    VPL_TRY(cudaMemsetAsync(scratch, 0, sizeof(int), ex.stream));
    return dispatch<false, false, false>(ex, s, a, single_view_extra(a, scratch));
}

int64_t gather_noalloc_max_tiles() { return (int64_t)1 << 30; }

// ==========================================================================
// diagnostics
// ==========================================================================
__global__ void philox_kernel(const uint64_t *ctr, const uint64_t *key, int64_t n, uint64_t *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox4x64_10(c, key[2 * i], key[2 * i + 1]);
    for (int k = 0; k < 4; k++) out[4 * i + k] = c[k];
}

cudaError_t debug_philox(const Exec &ex, const uint64_t *ctr, const uint64_t *key, int64_t n, uint64_t *out)
{
    if (n == 0) return cudaSuccess;
    philox_kernel<<<grid_for(n, 256), 256, 0, ex.stream>>>(ctr, key, n, out);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

__global__ void rays_kernel(SceneView s, int mode, int brute, const float4 *a, const float4 *b, int64_t n,
                            int32_t *out_tri, float *out_t, int *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 p = f3(a[i]), q = f3(b[i]);
    if (mode == 0) {
        Ray r = make_ray(p, q - p);
        bool bl = brute ? occluded_brute(s, r) : occluded1(s, r, status);
        out_tri[i] = bl ? 1 : 0;
    } else {
        Ray r = make_ray(p, q);
        float t;
        int k = brute ? closest_brute(s, r, 0.0f, t) : closest_hit(s, r, 0.0f, t, status);
        out_tri[i] = k;
        if (out_t) out_t[i] = k >= 0 ? t : 0.0f;
    }
}

cudaError_t debug_rays(const Exec &ex, const SceneView &s, int mode, int brute, const float4 *a, const float4 *b,
                       int64_t n, int32_t *out_tri, float *out_t)
{
    if (n == 0) return cudaSuccess;
    rays_kernel<<<grid_for(n, 128), 128, 0, ex.stream>>>(s, mode, brute, a, b, n, out_tri, out_t, ex.status);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

} // namespace vpl
