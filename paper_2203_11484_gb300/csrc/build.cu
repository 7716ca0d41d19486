// Scene upload kernels: per-triangle preparation, device prefix sums, a
// stable LSD radix sort over 63-bit Morton codes and the BVH: a binary
// hierarchy by locally-ordered clustering of the Morton-ordered triangles
// (the Karras 2012 linear hierarchy with boxes fitted bottom-up is the
// fallback and a build option), collapsed into 4-wide nodes.  The BVH is not part
// of the paper; it is the acceleration structure behind every ray query of
// the method (G-buffer, light paths, Eq. 2 and Eq. 1 visibility).
#include "vpl_internal.h"

namespace vpl {

// ==========================================================================
// exclusive prefix sum (reduce / scan partials / scan tiles)
// ==========================================================================
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T *warp_tot, T &block_total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T n = __shfl_up_sync(kFull, ti, o);
            if (lane >= o) ti += n;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t; // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) warp_tot[kScanThreads / 32] = ti;
    }
    __syncthreads();
    T r = warp_tot[w] + inc - v;
    block_total = warp_tot[kScanThreads / 32];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const T *in, const int *n_dev, int64_t n_max, T *partial)
{
    __shared__ T wt[kScanThreads / 32 + 1];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T s = 0;
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    T tot;
    block_exclusive<T>(s, wt, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(T *partial, int64_t n_tiles)
{
    __shared__ T wt[kScanThreads / 32 + 1];
    T carry = 0;
    for (int64_t b = 0; b < n_tiles; b += kScanThreads) {
        int64_t i = b + threadIdx.x;
        T v = i < n_tiles ? partial[i] : T(0);
        T tot;
        T ex = block_exclusive<T>(v, wt, tot);
        if (i < n_tiles) partial[i] = carry + ex;
        carry += tot;
    }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const T *in, T *out, const int *n_dev, int64_t n_max, const T *partial)
{
    __shared__ T wt[kScanThreads / 32 + 1];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base > n) return;
    T v[kScanItems];
    T s = 0;
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        v[k] = i < n ? in[i] : T(0);
        s += v[k];
    }
    T tot;
    T run = block_exclusive<T>(s, wt, tot) + partial[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    // the tile holding position n writes the total
    if (threadIdx.x == 0 && n >= base && n < base + kScanTile) out[n] = partial[blockIdx.x] + tot;
}

template <typename T>
cudaError_t exclusive_scan(const Exec &ex, const T *in, T *out, const int *n_dev, int64_t n_max)
{
    int64_t tiles = n_max / kScanTile + 1; // +1: position n_max needs a tile too
    Tmp part;
    VPL_TRY(part.alloc(ex, sizeof(T) * tiles));
    scan_reduce_kernel<T><<<(unsigned)tiles, kScanThreads, 0, ex.stream>>>(in, n_dev, n_max, part.as<T>());
    VPL_LAUNCHED(ex);
    scan_partials_kernel<T><<<1, kScanThreads, 0, ex.stream>>>(part.as<T>(), tiles);
    VPL_LAUNCHED(ex);
    scan_down_kernel<T><<<(unsigned)tiles, kScanThreads, 0, ex.stream>>>(in, out, n_dev, n_max, part.as<T>());
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

template cudaError_t exclusive_scan<uint32_t>(const Exec &, const uint32_t *, uint32_t *, const int *, int64_t);
template cudaError_t exclusive_scan<unsigned long long>(const Exec &, const unsigned long long *, unsigned long long *,
                                                        const int *, int64_t);

// ==========================================================================
// stable LSD radix sort, 8 bits per pass
// ==========================================================================
constexpr int kSortThreads = 256, kSortItems = 4, kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *keys, const int *n_dev, int64_t n_max, int shift,
                                  uint32_t *tile_hist, int n_tiles)
{
    __shared__ uint32_t h[256];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; r++) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    tile_hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout,
                                     const int *n_dev, int64_t n_max, int shift,
                                     const uint32_t *tile_off, int n_tiles)
{
    __shared__ uint32_t wc[kSortThreads / 32][256];
    __shared__ uint32_t run[256];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    if (base >= n) return;
    run[threadIdx.x] = tile_off[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
    for (int r = 0; r < kSortItems; r++) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        uint32_t val = valid ? vin[i] : 0;
        uint32_t digit = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
#pragma unroll
        for (int q = 0; q < kSortThreads / 32; q++) wc[q][threadIdx.x] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(kFull, digit);
        unsigned lower = peers & ((1u << lane) - 1u);
        uint32_t rank = __popc(lower);
        if (valid && lower == 0) wc[w][digit] = __popc(peers);
        __syncthreads();
        uint32_t acc = 0;
#pragma unroll
        for (int q = 0; q < kSortThreads / 32; q++) {
            uint32_t c = wc[q][threadIdx.x];
            wc[q][threadIdx.x] = acc;
            acc += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = run[digit] + wc[w][digit] + rank;
            kout[dst] = key;
            vout[dst] = val;
        }
        __syncthreads();
        run[threadIdx.x] += acc;
        __syncthreads();
    }
}

cudaError_t radix_sort_pairs(const Exec &ex, uint64_t *keys, uint32_t *vals, const int *n_dev, int64_t n_max,
                             int key_bits)
{
    if (n_max <= 0) return cudaSuccess;
    const int n_tiles = (int)((n_max + kSortTile - 1) / kSortTile);
    Tmp k2, v2, hist, off;
    VPL_TRY(k2.alloc(ex, sizeof(uint64_t) * n_max));
    VPL_TRY(v2.alloc(ex, sizeof(uint32_t) * n_max));
    VPL_TRY(hist.alloc(ex, sizeof(uint32_t) * 256 * n_tiles));
    VPL_TRY(off.alloc(ex, sizeof(uint32_t) * (256 * (int64_t)n_tiles + 1)));
    uint64_t *ka = keys, *kb = k2.as<uint64_t>();
    uint32_t *va = vals, *vb = v2.as<uint32_t>();
    const int passes = ((key_bits + 15) / 16) * 2; // even: the result ends where it started
    for (int shift = 0; shift < 8 * passes && shift < 64; shift += 8) {
        radix_hist_kernel<<<n_tiles, kSortThreads, 0, ex.stream>>>(ka, n_dev, n_max, shift, hist.as<uint32_t>(), n_tiles);
        VPL_LAUNCHED(ex);
        VPL_TRY(exclusive_scan<uint32_t>(ex, hist.as<uint32_t>(), off.as<uint32_t>(), nullptr, 256 * (int64_t)n_tiles));
        radix_scatter_kernel<<<n_tiles, kSortThreads, 0, ex.stream>>>(ka, va, kb, vb, n_dev, n_max, shift,
                                                                      off.as<uint32_t>(), n_tiles);
        VPL_LAUNCHED(ex);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // an even number of passes: the result is back in keys / vals
    return cudaSuccess;
}

// ==========================================================================
// scene preparation
// ==========================================================================
// order-preserving integer images of doubles / floats for atomic min / max
__device__ __forceinline__ unsigned long long dkey(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dunkey(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k));
}
__device__ __forceinline__ unsigned fkey(float v)
{
    unsigned b = __float_as_uint(v);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float funkey(unsigned k) { return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k); }

struct BoxKeys {
    unsigned long long glo[3], ghi[3];
    unsigned vlo[3], vhi[3];
};

__global__ void init_box_keys_kernel(BoxKeys *bk)
{
    for (int a = 0; a < 3; a++) {
        bk->glo[a] = ~0ULL;
        bk->ghi[a] = 0ULL;
        bk->vlo[a] = ~0u;
        bk->vhi[a] = 0u;
    }
}

// vertex indices out of range are reported and replaced by 0 in the
// library's copy, so that no later kernel reads outside the vertex array
__global__ void validate_kernel(int32_t *tris, int64_t n_tris, int64_t n_verts, int *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    for (int k = 0; k < 3; k++) {
        int32_t v = tris[3 * t + k];
        if (v < 0 || v >= n_verts) {
            latch(status, VPL_ERR_INVALID_ARG);
            tris[3 * t + k] = 0;
        }
    }
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// per-triangle normal and albedo; the centroid and vertex boxes are reduced
// over each warp first, so each warp makes one atomic per bound
__global__ void prep_kernel(const float *verts, const int32_t *tris, const float *albedo, int64_t n_tris,
                            int64_t n_verts, float4 *nrm, float4 *rho, BoxKeys *bk)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long glo[3] = {~0ULL, ~0ULL, ~0ULL}, ghi[3] = {0ULL, 0ULL, 0ULL};
    unsigned vlo[3] = {~0u, ~0u, ~0u}, vhi[3] = {0u, 0u, 0u};
    if (t < n_tris) {
        const int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
        if (i0 < 0 || i0 >= n_verts || i1 < 0 || i1 >= n_verts || i2 < 0 || i2 >= n_verts) {
            nrm[t] = make_float4(0, 0, 0, 0);
            rho[t] = make_float4(0, 0, 0, 0);
        } else {
            D3 a = dvert(verts, i0), b = dvert(verts, i1), c = dvert(verts, i2);
            D3 cr = dcross(dsub(b, a), dsub(c, a));
            double l = __dsqrt_rn(ddot(cr, cr));
            D3 n = l > 0.0 ? dmk(__ddiv_rn(cr.x, l), __ddiv_rn(cr.y, l), __ddiv_rn(cr.z, l)) : dmk(0, 0, 0);
            nrm[t] = make_float4((float)n.x, (float)n.y, (float)n.z, 0.0f);
            rho[t] = make_float4(albedo[3 * t], albedo[3 * t + 1], albedo[3 * t + 2], 0.0f);
            D3 s = dadd(dadd(a, b), c);
            const double g[3] = {__ddiv_rn(s.x, 3.0), __ddiv_rn(s.y, 3.0), __ddiv_rn(s.z, 3.0)};
            for (int ax = 0; ax < 3; ax++) {
                glo[ax] = ghi[ax] = dkey(g[ax]);
                const float v0 = verts[3 * (int64_t)i0 + ax], v1 = verts[3 * (int64_t)i1 + ax],
                            v2 = verts[3 * (int64_t)i2 + ax];
                vlo[ax] = fkey(fminf(v0, fminf(v1, v2)));
                vhi[ax] = fkey(fmaxf(v0, fmaxf(v1, v2)));
            }
        }
    }
    for (int ax = 0; ax < 3; ax++) {
        const unsigned long long lo = warp_min64(glo[ax]), hi = warp_max64(ghi[ax]);
        const unsigned flo = __reduce_min_sync(kFull, vlo[ax]), fhi = __reduce_max_sync(kFull, vhi[ax]);
        if ((threadIdx.x & 31) == 0 && hi >= lo) { // some lane of the warp had a valid triangle
            atomicMin(&bk->glo[ax], lo);
            atomicMax(&bk->ghi[ax], hi);
            atomicMin(&bk->vlo[ax], flo);
            atomicMax(&bk->vhi[ax], fhi);
        }
    }
}

__global__ void finish_boxes_kernel(const BoxKeys *bk, double *gbox, float *vbox)
{
    for (int a = 0; a < 3; a++) {
        gbox[a] = dunkey(bk->glo[a]);
        gbox[3 + a] = dunkey(bk->ghi[a]);
        vbox[a] = funkey(bk->vlo[a]);
        vbox[3 + a] = funkey(bk->vhi[a]);
    }
}

// 63-bit Morton code of the FP32 centroid in the vertex AABB
__global__ void bvh_keys_kernel(const float *verts, const int32_t *tris, int64_t n_tris, const float *vbox,
                                uint64_t *keys, uint32_t *vals)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    uint32_t q[3];
    for (int ax = 0; ax < 3; ax++) {
        float c = (verts[3 * (int64_t)tris[3 * t] + ax] + verts[3 * (int64_t)tris[3 * t + 1] + ax] +
                   verts[3 * (int64_t)tris[3 * t + 2] + ax]) * (1.0f / 3.0f);
        float ext = vbox[3 + ax] - vbox[ax];
        float u = ext > 0.0f ? (c - vbox[ax]) / ext : 0.0f;
        float f = floorf(u * 2097152.0f);
        q[ax] = (uint32_t)fminf(fmaxf(f, 0.0f), 2097151.0f);
    }
    keys[t] = morton63(q[0], q[1], q[2]);
    vals[t] = (uint32_t)t;
}

// Karras (2012): one thread per internal node finds its key range and split
__device__ __forceinline__ int delta(const uint64_t *k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    uint64_t a = k[i], b = k[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz(i ^ j);
}

__global__ void karras_kernel(const uint64_t *keys, int n, int *child, int *parent_int, int *parent_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gam = i + s * d + (d < 0 ? -1 : 0);
    int lo = min(i, j), hi = max(i, j);
    int c0 = (lo == gam) ? ~gam : gam;
    int c1 = (hi == gam + 1) ? ~(gam + 1) : gam + 1;
    child[2 * i] = c0;
    child[2 * i + 1] = c1;
    if (c0 < 0) parent_leaf[~c0] = i; else parent_int[c0] = i;
    if (c1 < 0) parent_leaf[~c1] = i; else parent_int[c1] = i;
    if (i == 0) parent_int[0] = -1;
}

// triangles in leaf order and their (padded) boxes
__global__ void leaves_kernel(const float *verts, const int32_t *tris, const uint32_t *order, int64_t n_tris,
                              const float *vbox, float4 *tri, float *leafbox)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_tris) return;
    uint32_t t = order[k];
    float3 v[3];
    for (int q = 0; q < 3; q++) {
        int64_t vi = tris[3 * (int64_t)t + q];
        v[q] = make_float3(verts[3 * vi], verts[3 * vi + 1], verts[3 * vi + 2]);
    }
    tri[3 * k] = make_float4(v[0].x, v[0].y, v[0].z, __int_as_float((int)t));
    float3 e1 = v[1] - v[0], e2 = v[2] - v[0];
    tri[3 * k + 1] = make_float4(e1.x, e1.y, e1.z, 0.0f);
    tri[3 * k + 2] = make_float4(e2.x, e2.y, e2.z, 0.0f);
    // pad by a few ulps of the largest coordinate so that flat boxes of
    // axis-aligned faces never lose a hit to rounding in the slab test
    float m = 0.0f;
    for (int a = 0; a < 6; a++) m = fmaxf(m, fabsf(vbox[a]));
    float pad = m * 1e-6f + 1e-30f;
    float *b = leafbox + 6 * k;
    b[0] = fminf(v[0].x, fminf(v[1].x, v[2].x)) - pad;
    b[1] = fminf(v[0].y, fminf(v[1].y, v[2].y)) - pad;
    b[2] = fminf(v[0].z, fminf(v[1].z, v[2].z)) - pad;
    b[3] = fmaxf(v[0].x, fmaxf(v[1].x, v[2].x)) + pad;
    b[4] = fmaxf(v[0].y, fmaxf(v[1].y, v[2].y)) + pad;
    b[5] = fmaxf(v[0].z, fmaxf(v[1].z, v[2].z)) + pad;
}

__device__ __forceinline__ void load_box(const float *p, float b[6])
{
    for (int a = 0; a < 6; a++) b[a] = __ldcg(p + a);
}

// bottom-up boxes: the second thread to reach a node merges its children
__global__ void bounds_kernel(int n, const int *child, const int *parent_int, const int *parent_leaf,
                              const float *leafbox, float *nodebox, int *visits, int *status)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int node = parent_leaf[k];
    for (int steps = 0; node >= 0; steps++) {
        if (steps > 4 * kStackMax) { // a well-formed hierarchy is never this deep
            latch(status, VPL_ERR_TRAVERSAL_LIMIT);
            return;
        }
        __threadfence();
        if (atomicAdd(&visits[node], 1) == 0) return;
        int c0 = child[2 * node], c1 = child[2 * node + 1];
        float b0[6], b1[6];
        load_box(c0 < 0 ? leafbox + 6 * (int64_t)(~c0) : nodebox + 6 * (int64_t)c0, b0);
        load_box(c1 < 0 ? leafbox + 6 * (int64_t)(~c1) : nodebox + 6 * (int64_t)c1, b1);
        float *o = nodebox + 6 * (int64_t)node;
        for (int a = 0; a < 3; a++) {
            __stcg(o + a, fminf(b0[a], b1[a]));
            __stcg(o + 3 + a, fmaxf(b0[3 + a], b1[3 + a]));
        }
        node = parent_int[node];
    }
}

// ==========================================================================
// binary hierarchy by parallel locally-ordered clustering (Meister and
// Bittner 2018): clusters in Morton order, each finds the cluster within +-R
// positions whose union box has the smallest surface area; mutual nearest
// neighbours merge; the survivors are compacted in order; repeat until one
// cluster is left.  Internal nodes are numbered downwards from T-2, so the
// last merge -- the root -- is node 0.
// ==========================================================================
#ifndef VPL_PLOC_R
#define VPL_PLOC_R 32
#endif
constexpr int kPlocR = VPL_PLOC_R; // neighbour search radius
constexpr int kPlocThreads = 256;

struct PlocCtl {
    int n_cur;     // clusters left
    int node_next; // internal nodes made so far
};

__device__ __forceinline__ float union_area(const float *a, const float *b)
{
    const float dx = fmaxf(a[3], b[3]) - fminf(a[0], b[0]);
    const float dy = fmaxf(a[4], b[4]) - fminf(a[1], b[1]);
    const float dz = fmaxf(a[5], b[5]) - fminf(a[2], b[2]);
    return dx * dy + dy * dz + dz * dx;
}

__global__ void ploc_init_kernel(int n, const float *leafbox, int *cref, float *cbox, int *parent_int, PlocCtl *ctl)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ctl->n_cur = n;
        ctl->node_next = 0;
    }
    if (i < n - 1) parent_int[i] = -1;
    if (i >= n) return;
    cref[i] = ~i;
    for (int a = 0; a < 6; a++) cbox[6 * (int64_t)i + a] = leafbox[6 * (int64_t)i + a];
}

__global__ void __launch_bounds__(kPlocThreads) ploc_nn_kernel(const PlocCtl *ctl, const float *cbox, int *nn)
{
    __shared__ float tile[(kPlocThreads + 2 * kPlocR) * 6];
    const int n = ctl->n_cur;
    const int base = blockIdx.x * kPlocThreads;
    if (n <= 1 || base >= n) return;
    const int lo = base - kPlocR;
    for (int k = threadIdx.x; k < kPlocThreads + 2 * kPlocR; k += kPlocThreads) {
        const int c = lo + k;
        for (int a = 0; a < 6; a++) tile[6 * k + a] = (c >= 0 && c < n) ? cbox[6 * (int64_t)c + a] : 0.0f;
    }
    __syncthreads();
    const int i = base + threadIdx.x;
    if (i >= n) return;
    const float *bi = tile + 6 * (threadIdx.x + kPlocR);
    const int j0 = max(0, i - kPlocR), j1 = min(n - 1, i + kPlocR);
    // j ascends and only a strictly smaller area replaces: ties keep the lower
    // index, so the lowest cluster of the globally smallest pair always finds
    // a mutual partner and every pass merges at least once
    int bj = j0 == i ? i + 1 : j0;
    float best = union_area(bi, tile + 6 * (bj - lo));
    for (int j = bj + 1; j <= j1; j++) {
        if (j == i) continue;
        const float a = union_area(bi, tile + 6 * (j - lo));
        if (a < best) {
            best = a;
            bj = j;
        }
    }
    nn[i] = bj;
}

// flags packed as keep << 32 | make: one scan gives both prefix sums
__global__ void ploc_flags_kernel(const PlocCtl *ctl, const int *nn, unsigned long long *flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = ctl->n_cur;
    if (i >= n) return;
    const int j = n > 1 ? nn[i] : -1;
    const bool mutual = j >= 0 && nn[j] == i;
    const bool make = mutual && i < j, keep = !(mutual && i > j);
    flags[i] = ((unsigned long long)(keep ? 1u : 0u) << 32) | (make ? 1u : 0u);
}

__global__ void ploc_merge_kernel(int T, const PlocCtl *ctl, const int *nn, const unsigned long long *flags,
                                  const unsigned long long *off, const int *cref_in, const float *cbox_in,
                                  int *cref_out, float *cbox_out, int *child, float *nodebox, int *parent_int,
                                  int *parent_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = ctl->n_cur;
    if (i >= n) return;
    const unsigned long long f = flags[i];
    if (!(f >> 32)) return; // merged into a lower cluster
    const int pos = (int)(off[i] >> 32);
    if (f & 1ull) {
        const int j = nn[i];
        const int id = (T - 2) - (ctl->node_next + (int)(off[i] & 0xffffffffull));
        const int a = cref_in[i], b = cref_in[j];
        child[2 * (int64_t)id] = a;
        child[2 * (int64_t)id + 1] = b;
        if (a < 0) parent_leaf[~a] = id; else parent_int[a] = id;
        if (b < 0) parent_leaf[~b] = id; else parent_int[b] = id;
        const float *p = cbox_in + 6 * (int64_t)i, *q = cbox_in + 6 * (int64_t)j;
        float *o = nodebox + 6 * (int64_t)id, *c = cbox_out + 6 * (int64_t)pos;
        for (int k = 0; k < 3; k++) {
            o[k] = c[k] = fminf(p[k], q[k]);
            o[3 + k] = c[3 + k] = fmaxf(p[3 + k], q[3 + k]);
        }
        cref_out[pos] = id;
    } else {
        cref_out[pos] = cref_in[i];
        for (int k = 0; k < 6; k++) cbox_out[6 * (int64_t)pos + k] = cbox_in[6 * (int64_t)i + k];
    }
}

__global__ void ploc_ctl_kernel(PlocCtl *ctl, const unsigned long long *off)
{
    const unsigned long long tot = off[ctl->n_cur];
    ctl->node_next += (int)(tot & 0xffffffffull);
    ctl->n_cur = (int)(tot >> 32);
}

// The last passes, from at most kTailMax clusters down to one, in a single
// block: the same three steps per pass (nearest neighbours, mutual-pair
// flags with a block scan, merge and compaction), with block barriers in
// place of kernel boundaries.
constexpr int kTailThreads = 1024, kTailItems = 4, kTailMax = kTailThreads * kTailItems;

__global__ void __launch_bounds__(kTailThreads) ploc_tail_kernel(int T, PlocCtl *ctl, int cur, int *cref0,
                                                                 float *cbox0, int *cref1, float *cbox1, int *nn,
                                                                 int *child, float *nodebox, int *parent_int,
                                                                 int *parent_leaf)
{
    __shared__ int wk[kTailThreads / 32], wm[kTailThreads / 32];
    __shared__ int tot[2];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int n = ctl->n_cur, made = ctl->node_next;
    for (int pass = 0; n > 1 && pass < kTailMax; pass++) { // each pass merges at least one pair
        const int *rin = cur ? cref1 : cref0;
        const float *bin = cur ? cbox1 : cbox0;
        int *rout = cur ? cref0 : cref1;
        float *bout = cur ? cbox0 : cbox1;
        for (int i = tid; i < n; i += kTailThreads) {
            const float *bi = bin + 6 * (int64_t)i;
            const int j0 = max(0, i - kPlocR), j1 = min(n - 1, i + kPlocR);
            int bj = j0 == i ? i + 1 : j0;
            float best = union_area(bi, bin + 6 * (int64_t)bj);
            for (int j = bj + 1; j <= j1; j++) {
                if (j == i) continue;
                const float a = union_area(bi, bin + 6 * (int64_t)j);
                if (a < best) {
                    best = a;
                    bj = j;
                }
            }
            nn[i] = bj;
        }
        __syncthreads();
        // items tid * kTailItems + k, in order: flags and their block scan
        int keep[kTailItems], make[kTailItems], sk = 0, sm = 0;
        for (int k = 0; k < kTailItems; k++) {
            const int i = tid * kTailItems + k;
            keep[k] = make[k] = 0;
            if (i < n) {
                const int j = nn[i];
                const bool mutual = nn[j] == i;
                make[k] = mutual && i < j;
                keep[k] = !(mutual && i > j);
            }
            sk += keep[k];
            sm += make[k];
        }
        int ik = sk, im = sm;
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(kFull, ik, o), b = __shfl_up_sync(kFull, im, o);
            if (lane >= o) {
                ik += a;
                im += b;
            }
        }
        if (lane == 31) {
            wk[w] = ik;
            wm[w] = im;
        }
        __syncthreads();
        if (w == 0) {
            int a = wk[lane], b = wm[lane]; // kTailThreads / 32 == 32 warps
            int ia = a, ib = b;
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(kFull, ia, o), y = __shfl_up_sync(kFull, ib, o);
                if (lane >= o) {
                    ia += x;
                    ib += y;
                }
            }
            wk[lane] = ia - a;
            wm[lane] = ib - b;
            if (lane == 31) {
                tot[0] = ia;
                tot[1] = ib;
            }
        }
        __syncthreads();
        int pk = wk[w] + ik - sk, pm = wm[w] + im - sm; // exclusive offsets of this thread's first item
        for (int k = 0; k < kTailItems; k++) {
            const int i = tid * kTailItems + k;
            if (i < n && keep[k]) {
                if (make[k]) {
                    const int j = nn[i];
                    const int id = (T - 2) - (made + pm);
                    const int a = rin[i], b = rin[j];
                    child[2 * (int64_t)id] = a;
                    child[2 * (int64_t)id + 1] = b;
                    if (a < 0) parent_leaf[~a] = id; else parent_int[a] = id;
                    if (b < 0) parent_leaf[~b] = id; else parent_int[b] = id;
                    const float *p = bin + 6 * (int64_t)i, *q = bin + 6 * (int64_t)j;
                    float *o = nodebox + 6 * (int64_t)id, *c = bout + 6 * (int64_t)pk;
                    for (int x = 0; x < 3; x++) {
                        o[x] = c[x] = fminf(p[x], q[x]);
                        o[3 + x] = c[3 + x] = fmaxf(p[3 + x], q[3 + x]);
                    }
                    rout[pk] = id;
                } else {
                    rout[pk] = rin[i];
                    for (int x = 0; x < 6; x++) bout[6 * (int64_t)pk + x] = bin[6 * (int64_t)i + x];
                }
            }
            pk += keep[k];
            pm += make[k];
        }
        __syncthreads();
        n = tot[0];
        made += tot[1];
        cur ^= 1;
        __syncthreads(); // tot is rewritten by the next pass
    }
    if (tid == 0) {
        ctl->n_cur = n;
        ctl->node_next = made;
    }
}

// Runs merge passes until one cluster is left; *done stays false if a check
// sees no merge over a whole batch of passes (only non-finite boxes can do
// that), and the caller then builds the Karras hierarchy instead.
static cudaError_t ploc_build(const Exec &ex, int T, const float *leafbox, int *child, float *nodebox,
                              int *parent_int, int *parent_leaf, bool *done)
{
    const int B = kPlocThreads, kBatch = 8;
    *done = false;
    Tmp cref[2], cbox[2], nn, flags, off, ctl;
    for (int k = 0; k < 2; k++) {
        VPL_TRY(cref[k].alloc(ex, sizeof(int) * T));
        VPL_TRY(cbox[k].alloc(ex, sizeof(float) * 6 * T));
    }
    VPL_TRY(nn.alloc(ex, sizeof(int) * T));
    VPL_TRY(flags.alloc(ex, sizeof(unsigned long long) * T));
    VPL_TRY(off.alloc(ex, sizeof(unsigned long long) * (T + 1)));
    VPL_TRY(ctl.alloc(ex, sizeof(PlocCtl)));
    PlocCtl *c = ctl.as<PlocCtl>();
    ploc_init_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(T, leafbox, cref[0].as<int>(), cbox[0].as<float>(),
                                                           parent_int, c);
    VPL_LAUNCHED(ex);
    int cur = 0, left = T;
    while (left > 1) {
        if (left <= kTailMax) {
            ploc_tail_kernel<<<1, kTailThreads, 0, ex.stream>>>(T, c, cur, cref[0].as<int>(), cbox[0].as<float>(),
                                                               cref[1].as<int>(), cbox[1].as<float>(), nn.as<int>(),
                                                               child, nodebox, parent_int, parent_leaf);
            VPL_LAUNCHED(ex);
        } else {
            // grids sized by the last count read back (an upper bound)
            const unsigned g = grid_for(left, B);
            for (int it = 0; it < kBatch; it++) {
                ploc_nn_kernel<<<g, B, 0, ex.stream>>>(c, cbox[cur].as<float>(), nn.as<int>());
                VPL_LAUNCHED(ex);
                ploc_flags_kernel<<<g, B, 0, ex.stream>>>(c, nn.as<int>(), flags.as<unsigned long long>());
                VPL_LAUNCHED(ex);
                VPL_TRY(exclusive_scan<unsigned long long>(ex, flags.as<unsigned long long>(),
                                                           off.as<unsigned long long>(), &c->n_cur, left));
                ploc_merge_kernel<<<g, B, 0, ex.stream>>>(T, c, nn.as<int>(), flags.as<unsigned long long>(),
                                                          off.as<unsigned long long>(), cref[cur].as<int>(),
                                                          cbox[cur].as<float>(), cref[1 - cur].as<int>(),
                                                          cbox[1 - cur].as<float>(), child, nodebox, parent_int,
                                                          parent_leaf);
                VPL_LAUNCHED(ex);
                ploc_ctl_kernel<<<1, 1, 0, ex.stream>>>(c, off.as<unsigned long long>());
                VPL_LAUNCHED(ex);
                cur = 1 - cur;
            }
        }
        int now = 0;
        VPL_TRY(cudaMemcpyAsync(&now, &c->n_cur, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
        VPL_TRY(cudaStreamSynchronize(ex.stream));
        if (now >= left) return cudaSuccess; // no progress
        left = now;
    }
    *done = true;
    return cudaSuccess;
}

static cudaError_t lbvh_build(const Exec &ex, const uint64_t *keys, int n, const float *leafbox, int *child,
                              float *nodebox, int *parent_int, int *parent_leaf)
{
    const int B = 256;
    Tmp visits;
    VPL_TRY(visits.alloc(ex, sizeof(int) * (n - 1)));
    VPL_TRY(cudaMemsetAsync(visits.p, 0, sizeof(int) * (n - 1), ex.stream));
    karras_kernel<<<grid_for(n - 1, B), B, 0, ex.stream>>>(keys, n, child, parent_int, parent_leaf);
    VPL_LAUNCHED(ex);
    bounds_kernel<<<grid_for(n, B), B, 0, ex.stream>>>(n, child, parent_int, parent_leaf, leafbox, nodebox,
                                                       visits.as<int>(), ex.status);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

// ==========================================================================
// 4-wide nodes, built top down one level per launch.  A node starts from the
// two children of its binary node; while it has fewer than four slots it
// opens an internal slot into that node's two children: the one with the
// largest box surface (surface rule) or, in the even rule, each of the two
// starting slots once (every binary node at even depth becomes a node).  The
// slots are then put in order of box surface, largest first: the packet
// shadow walk visits internal children in slot order.  A node's internal
// children get consecutive node indices from `ibase` and its leaf children
// consecutive triangle slots from `lbase` (both in slot order), so a child is
// found from its base and its rank among the node's children of its kind;
// the triangles are moved into those slots at the end.  Node indices are
// handed out in allocation order (root 0, then breadth first); the result
// does not depend on that order, only on the slot contents and their order.
// Each node is written in two layouts with the same index: per axis (Node4,
// for the per-ray and per-lane walks) and per child (two float4 per slot,
// for the beam walk; see BeamNode).
// ==========================================================================
constexpr int kCollapseLevels = (kStackMax - 1) / 3; // each level pushes <= 3 stack entries

__device__ __forceinline__ float box_area(const float *b)
{
    const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return dx * dy + dy * dz + dz * dx;
}

__global__ void collapse_init_kernel(int2 *queue, int *count, int *next)
{
    queue[0] = make_int2(0, 0);
    count[0] = 1; // nodes of the current level (count[1]: of the next)
    count[1] = 0;
    next[0] = 1;  // internal nodes handed out
    next[1] = 0;  // triangle slots handed out
}

#ifndef VPL_LEAF_MAX
#define VPL_LEAF_MAX 2
#endif
constexpr int kLeafMax = VPL_LEAF_MAX; // triangles per leaf slot
static_assert(kLeafMax >= 1 && kLeafMax <= 4, "a node's leaf runs are addressed with 4-bit offsets");

// Leaves of the binary subtree under c in depth-first order, if there are at
// most kLeafMax of them (c < 0: the one leaf ~c); else -1.
__device__ __forceinline__ int small_subtree(const int *child, int c, int *tris)
{
    if (c < 0) {
        tris[0] = ~c;
        return 1;
    }
    if (kLeafMax < 2) return -1;
    int stack[kLeafMax + 1], sp = 0, n = 0;
    stack[sp++] = c;
    while (sp > 0) {
        const int x = stack[--sp];
        if (x < 0) {
            if (n == kLeafMax) return -1;
            tris[n++] = ~x;
            continue;
        }
        if (sp + 2 > kLeafMax + 1) return -1; // more than kLeafMax leaves below
        stack[sp++] = child[2 * x + 1];
        stack[sp++] = child[2 * x];
    }
    return n;
}

template <bool EVEN>
__global__ void collapse_level_kernel(int level, const int2 *qin, int2 *qout, int *count, int *next,
                                      const int *child, const float *leafbox, const float *nodebox, float4 *nodes,
                                      float4 *bnodes, int *leaf_src)
{
    const int n_in = count[level & 1];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_in; q += gridDim.x * blockDim.x) {
        const int2 w = qin[q];
        int slot[4] = {child[2 * w.x], child[2 * w.x + 1], 0, 0};
        int tris[kLeafMax];
        // a slot is a leaf when its subtree has at most kLeafMax triangles
        bool leaf[4] = {small_subtree(child, slot[0], tris) > 0, small_subtree(child, slot[1], tris) > 0, false,
                        false};
        int m = 2;
        if (EVEN) {
            for (int k = 0; k < 2; k++)
                if (!leaf[k]) {
                    const int c = slot[k];
                    slot[k] = child[2 * c];
                    slot[m] = child[2 * c + 1];
                    leaf[k] = small_subtree(child, slot[k], tris) > 0;
                    leaf[m] = small_subtree(child, slot[m], tris) > 0;
                    m++;
                }
        } else {
            while (m < 4) {
                int pick = -1;
                float best = -1.0f;
                for (int k = 0; k < m; k++)
                    if (!leaf[k]) {
                        const float a = box_area(nodebox + 6 * (int64_t)slot[k]);
                        if (pick < 0 || a > best) {
                            pick = k;
                            best = a;
                        }
                    }
                if (pick < 0) break;
                const int c = slot[pick];
                slot[pick] = child[2 * c];
                slot[m] = child[2 * c + 1];
                leaf[pick] = small_subtree(child, slot[pick], tris) > 0;
                leaf[m] = small_subtree(child, slot[m], tris) > 0;
                m++;
            }
        }
        // slot order: box surface, largest first (stable)
        float area[4];
        for (int k = 0; k < m; k++)
            area[k] = box_area(slot[k] < 0 ? leafbox + 6 * (int64_t)(~slot[k]) : nodebox + 6 * (int64_t)slot[k]);
        for (int i = 1; i < m; i++)
            for (int j = i; j > 0 && area[j] > area[j - 1]; j--) {
                float ta = area[j]; area[j] = area[j - 1]; area[j - 1] = ta;
                int ts = slot[j]; slot[j] = slot[j - 1]; slot[j - 1] = ts;
                bool tl = leaf[j]; leaf[j] = leaf[j - 1]; leaf[j - 1] = tl;
            }
        int n_int = 0, n_tri = 0;
        for (int k = 0; k < m; k++) {
            if (leaf[k]) n_tri += small_subtree(child, slot[k], tris);
            else n_int++;
        }
        const int ibase = n_int ? atomicAdd(&next[0], n_int) : 0;
        const int lbase = n_tri ? atomicAdd(&next[1], n_tri) : 0;
        const int pos = n_int ? atomicAdd(&count[(level + 1) & 1], n_int) : 0;
        // empty slots: a point box at (3e38, -3e38, 3e38), which no segment or
        // ray of a scene reaches
        float lo[3][4], hi[3][4];
        unsigned leafmask = 0, intmask = 0, runs = 0;
        int ji = 0, jl = 0;
        int ref[4], cnt[4]; // per slot, for the per-child layout
        for (int k = 0; k < 4; k++) {
            const float *b = nullptr;
            ref[k] = kEmptyRef;
            cnt[k] = 0;
            if (k < m && leaf[k]) {
                b = slot[k] < 0 ? leafbox + 6 * (int64_t)(~slot[k]) : nodebox + 6 * (int64_t)slot[k];
                const int n = small_subtree(child, slot[k], tris);
                runs |= (unsigned)(jl | (n << 4)) << (8 * k); // offset in the node's run, count
                ref[k] = ~(lbase + jl);
                cnt[k] = n;
                for (int i = 0; i < n; i++) leaf_src[lbase + jl++] = tris[i];
                leafmask |= 1u << k;
            } else if (k < m) {
                b = nodebox + 6 * (int64_t)slot[k];
                qout[pos + ji] = make_int2(slot[k], ibase + ji);
                ref[k] = ibase + ji;
                ji++;
                intmask |= 1u << k;
            }
            for (int a = 0; a < 3; a++) {
                lo[a][k] = b ? b[a] : (a == 1 ? -3.0e38f : 3.0e38f);
                hi[a][k] = b ? b[3 + a] : (a == 1 ? -3.0e38f : 3.0e38f);
            }
        }
        float4 *bo = bnodes + 8 * (int64_t)w.y;
        for (int k = 0; k < 4; k++) {
            bo[2 * k] = make_float4(lo[0][k], lo[1][k], lo[2][k], __int_as_float(ref[k]));
            bo[2 * k + 1] = make_float4(hi[0][k], hi[1][k], hi[2][k], __int_as_float(cnt[k]));
        }
        float4 *o = nodes + 8 * (int64_t)w.y;
        o[0] = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
        o[1] = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
        o[2] = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
        o[3] = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
        o[4] = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
        o[5] = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
        o[6] = make_float4(__int_as_float(ibase), __int_as_float(lbase), __uint_as_float(leafmask | (intmask << 4)),
                           __uint_as_float(runs));
        o[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

// triangles into the slots the nodes gave their leaves
__global__ void place_tris_kernel(int T, const int *leaf_src, const float4 *tri_in, float4 *tri_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    const int k = leaf_src[i];
    for (int c = 0; c < 3; c++) tri_out[3 * (int64_t)i + c] = tri_in[3 * (int64_t)k + c];
}

// Runs the levels with the given rule.  The surface rule stops after
// kCollapseLevels levels and leaves *done false if internal nodes are left (a
// tree too deep for the traversal stack); the even rule runs until every
// node is written (at most kCollapseLevels levels when the binary depth is
// within kDepthMax, which the build checks).
static cudaError_t collapse4(const Exec &ex, int T, bool even, const int *child, const float *leafbox,
                             const float *nodebox, float4 *nodes, float4 *bnodes, int *leaf_src, bool *done)
{
    *done = false;
    Tmp qa, qb, cnt, next;
    VPL_TRY(qa.alloc(ex, sizeof(int2) * T));
    VPL_TRY(qb.alloc(ex, sizeof(int2) * T));
    VPL_TRY(cnt.alloc(ex, sizeof(int) * 2));
    VPL_TRY(next.alloc(ex, sizeof(int) * 2));
    collapse_init_kernel<<<1, 1, 0, ex.stream>>>(qa.as<int2>(), cnt.as<int>(), next.as<int>());
    VPL_LAUNCHED(ex);
    const unsigned grid = grid_for(T, 256) < 1216u ? grid_for(T, 256) : 1216u;
    for (int l = 0;; l++) {
        const Tmp &in = (l & 1) ? qb : qa, &out = (l & 1) ? qa : qb;
        VPL_TRY(cudaMemsetAsync(cnt.as<int>() + ((l + 1) & 1), 0, sizeof(int), ex.stream));
        if (even)
            collapse_level_kernel<true><<<grid, 256, 0, ex.stream>>>(l, in.as<int2>(), out.as<int2>(), cnt.as<int>(),
                                                                     next.as<int>(), child, leafbox, nodebox, nodes,
                                                                     bnodes, leaf_src);
        else
            collapse_level_kernel<false><<<grid, 256, 0, ex.stream>>>(l, in.as<int2>(), out.as<int2>(),
                                                                      cnt.as<int>(), next.as<int>(), child, leafbox,
                                                                      nodebox, nodes, bnodes, leaf_src);
        VPL_LAUNCHED(ex);
        const bool last = !even && l + 1 == kCollapseLevels;
        if (last || (l + 1) % 16 == 0) {
            int left = 0;
            VPL_TRY(cudaMemcpyAsync(&left, cnt.as<int>() + ((l + 1) & 1), sizeof(int), cudaMemcpyDeviceToHost,
                                    ex.stream));
            VPL_TRY(cudaStreamSynchronize(ex.stream));
            if (left == 0) {
                *done = true;
                break;
            }
            if (last) break;
        }
    }
    return cudaSuccess;
}

// one triangle: a root with the leaf (slot 0) in slot 0 and three empty slots
__global__ void single_root_kernel(const float *leafbox, float4 *nodes, float4 *bnodes)
{
    const float *a = leafbox;
    const float f = 3.0e38f;
    nodes[0] = make_float4(a[0], f, f, f);
    nodes[1] = make_float4(a[3], f, f, f);
    nodes[2] = make_float4(a[1], -f, -f, -f);
    nodes[3] = make_float4(a[4], -f, -f, -f);
    nodes[4] = make_float4(a[2], f, f, f);
    nodes[5] = make_float4(a[5], f, f, f);
    nodes[6] = make_float4(__int_as_float(0), __int_as_float(0), __uint_as_float(1u), __uint_as_float(1u << 4));
    nodes[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bnodes[0] = make_float4(a[0], a[1], a[2], __int_as_float(~0));
    bnodes[1] = make_float4(a[3], a[4], a[5], __int_as_float(1));
    for (int k = 1; k < 4; k++) {
        bnodes[2 * k] = make_float4(f, -f, f, __int_as_float(kEmptyRef));
        bnodes[2 * k + 1] = make_float4(f, -f, f, __int_as_float(0));
    }
}

__global__ void depth_kernel(int n, const int *parent_int, const int *parent_leaf, int *depth, int *status)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int d = 0, node = n > 1 ? parent_leaf[k] : 0;
    while (node >= 0 && d <= 4 * kStackMax) {
        d++;
        node = n > 1 ? parent_int[node] : -1;
    }
    atomicMax(depth, d);
    if (d > kDepthMax) latch(status, VPL_ERR_TRAVERSAL_LIMIT);
}

cudaError_t build_scene(const Exec &ex, const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                        const float *albedo, SceneBuffers *sb)
{
    const int B = 256;
    const int64_t T = n_tris;
    const int n = (int)T;
    sb->n_tris = T;
    sb->n_verts = n_verts;
    size_t bytes = 0;
    auto dalloc = [&](void **p, size_t sz) -> cudaError_t {
        bytes += sz;
        return cudaMalloc(p, sz ? sz : 16);
    };
    VPL_TRY(dalloc((void **)&sb->verts, sizeof(float) * 3 * n_verts));
    VPL_TRY(dalloc((void **)&sb->idx, sizeof(int32_t) * 3 * T));
    VPL_TRY(dalloc((void **)&sb->tri, sizeof(float4) * 3 * T));
    VPL_TRY(dalloc((void **)&sb->nodes, sizeof(float4) * 8 * (T > 1 ? T - 1 : 1)));
    VPL_TRY(dalloc((void **)&sb->bnodes, sizeof(float4) * 8 * (T > 1 ? T - 1 : 1)));
    VPL_TRY(dalloc((void **)&sb->nrm, sizeof(float4) * T));
    VPL_TRY(dalloc((void **)&sb->rho, sizeof(float4) * T));
    VPL_TRY(dalloc((void **)&sb->gbox, sizeof(double) * 6));
    VPL_TRY(dalloc((void **)&sb->vbox, sizeof(float) * 6));
    VPL_TRY(dalloc((void **)&sb->depth, sizeof(int)));
    sb->bytes = bytes;
    VPL_TRY(cudaMemcpyAsync(sb->verts, verts, sizeof(float) * 3 * n_verts, cudaMemcpyDefault, ex.stream));
    VPL_TRY(cudaMemcpyAsync(sb->idx, tris, sizeof(int32_t) * 3 * T, cudaMemcpyDefault, ex.stream));
    Tmp alb, bk, keys, vals, leafbox, nodebox, child, pint, pleaf;
    VPL_TRY(alb.alloc(ex, sizeof(float) * 3 * T));
    VPL_TRY(cudaMemcpyAsync(alb.p, albedo, sizeof(float) * 3 * T, cudaMemcpyDefault, ex.stream));
    VPL_TRY(bk.alloc(ex, sizeof(BoxKeys)));
    VPL_TRY(cudaMemsetAsync(sb->depth, 0, sizeof(int), ex.stream));

    validate_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(sb->idx, T, n_verts, ex.status);
    VPL_LAUNCHED(ex);
    init_box_keys_kernel<<<1, 1, 0, ex.stream>>>(bk.as<BoxKeys>());
    VPL_LAUNCHED(ex);
    prep_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(sb->verts, sb->idx, alb.as<float>(), T, n_verts, sb->nrm,
                                                     sb->rho, bk.as<BoxKeys>());
    VPL_LAUNCHED(ex);
    finish_boxes_kernel<<<1, 1, 0, ex.stream>>>(bk.as<BoxKeys>(), sb->gbox, sb->vbox);
    VPL_LAUNCHED(ex);

    VPL_TRY(keys.alloc(ex, sizeof(uint64_t) * T));
    VPL_TRY(vals.alloc(ex, sizeof(uint32_t) * T));
    bvh_keys_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(sb->verts, sb->idx, T, sb->vbox, keys.as<uint64_t>(),
                                                         vals.as<uint32_t>());
    VPL_LAUNCHED(ex);
    VPL_TRY(radix_sort_pairs(ex, keys.as<uint64_t>(), vals.as<uint32_t>(), nullptr, T));

    VPL_TRY(leafbox.alloc(ex, sizeof(float) * 6 * T));
    Tmp trim;
    VPL_TRY(trim.alloc(ex, sizeof(float4) * 3 * T));
    leaves_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(sb->verts, sb->idx, vals.as<uint32_t>(), T, sb->vbox,
                                                       trim.as<float4>(), leafbox.as<float>());
    VPL_LAUNCHED(ex);
    VPL_TRY(pleaf.alloc(ex, sizeof(int) * T));
    VPL_TRY(pint.alloc(ex, sizeof(int) * (T > 1 ? T - 1 : 1)));
    if (T == 1) {
        single_root_kernel<<<1, 1, 0, ex.stream>>>(leafbox.as<float>(), sb->nodes, sb->bnodes);
        VPL_LAUNCHED(ex);
        VPL_TRY(cudaMemcpyAsync(sb->tri, trim.p, sizeof(float4) * 3, cudaMemcpyDeviceToDevice, ex.stream));
    } else {
        VPL_TRY(nodebox.alloc(ex, sizeof(float) * 6 * (T - 1)));
        VPL_TRY(child.alloc(ex, sizeof(int) * 2 * (T - 1)));
        bool built = false;
#if !VPL_BVH_LBVH
        VPL_TRY(ploc_build(ex, n, leafbox.as<float>(), child.as<int>(), nodebox.as<float>(), pint.as<int>(),
                           pleaf.as<int>(), &built));
#endif
        if (!built)
            VPL_TRY(lbvh_build(ex, keys.as<uint64_t>(), n, leafbox.as<float>(), child.as<int>(), nodebox.as<float>(),
                               pint.as<int>(), pleaf.as<int>()));
        Tmp leaf_src;
        VPL_TRY(leaf_src.alloc(ex, sizeof(int) * T));
        bool packed = false;
#if !VPL_BVH_EVEN_COLLAPSE
        VPL_TRY(collapse4(ex, n, false, child.as<int>(), leafbox.as<float>(), nodebox.as<float>(), sb->nodes,
                          sb->bnodes, leaf_src.as<int>(), &packed));
#endif
        if (!packed)
            VPL_TRY(collapse4(ex, n, true, child.as<int>(), leafbox.as<float>(), nodebox.as<float>(), sb->nodes,
                              sb->bnodes, leaf_src.as<int>(), &packed));
        place_tris_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(n, leaf_src.as<int>(), trim.as<float4>(), sb->tri);
        VPL_LAUNCHED(ex);
    }
    depth_kernel<<<grid_for(T, B), B, 0, ex.stream>>>(n, pint.as<int>(), pleaf.as<int>(), sb->depth, ex.status);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

} // namespace vpl
