// Host-side declarations shared by the translation units of libvpl.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vpl_device.cuh"

namespace vpl {

// Everything a launcher needs: the stream, the context's launch counter,
// its device status word and the stream-ordered pool for temporaries.
struct Exec {
    cudaStream_t stream;
    int64_t *launches;
    int *status;
    cudaMemPool_t pool;
    bool timing;
};

#define VPL_LAUNCHED(ex)                                 \
    do {                                                 \
        ++*(ex).launches;                                \
        cudaError_t e_ = cudaGetLastError();             \
        if (e_ != cudaSuccess) return e_;                \
    } while (0)

#define VPL_TRY(x)                                       \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return e_;                \
    } while (0)

// stream-ordered temporary from the context's pool, released on the same
// stream when it goes out of scope
struct Tmp {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    Tmp() = default;
    Tmp(const Tmp &) = delete;
    Tmp &operator=(const Tmp &) = delete;
    ~Tmp() { if (p) cudaFreeAsync(p, s); }
    cudaError_t alloc(const Exec &ex, size_t bytes)
    {
        s = ex.stream;
        return cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, ex.pool, ex.stream);
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block > 0 ? (n + block - 1) / block : 1); }

// ---- build.cu --------------------------------------------------------------
// exclusive prefix sum; out has n + 1 entries, out[n] = total.  The count
// is read from n_dev on the device when given (n_max bounds the launch),
// else n_max is the count.
template <typename T>
cudaError_t exclusive_scan(const Exec &ex, const T *in, T *out, const int *n_dev, int64_t n_max);

// stable LSD radix sort of (key, value) pairs on bits [0, key_bits) (keys
// must be zero above); the result ends in keys/vals.  Count from n_dev when
// given.
cudaError_t radix_sort_pairs(const Exec &ex, uint64_t *keys, uint32_t *vals, const int *n_dev,
                             int64_t n_max, int key_bits = 64);

struct SceneBuffers {
    int64_t n_tris = 0, n_verts = 0;
    float4 *tri = nullptr, *nodes = nullptr, *bnodes = nullptr, *nrm = nullptr, *rho = nullptr;
    float *verts = nullptr;
    int32_t *idx = nullptr;
    double *gbox = nullptr; // [6]: centroid AABB lo xyz, hi xyz (FP64)
    float *vbox = nullptr;  // [6]: vertex AABB lo xyz, hi xyz
    int *depth = nullptr;   // [1]: longest root-to-leaf path
    size_t bytes = 0;
};

cudaError_t build_scene(const Exec &ex, const float *verts, int64_t n_verts, const int32_t *tris,
                        int64_t n_tris, const float *albedo, SceneBuffers *sb);

// ---- generate.cu -------------------------------------------------------------
struct GenArgs {
    double d_close;
    float ray_eps;
    int32_t m_close, m_far, max_bounces, light_samples;
    int32_t close_rule; // 0 centroid, 1 centroid or any vertex
    int32_t patch_rule; // 0 a point per stratum, 1 set sum over the stratum's faces
    int64_t max_paths;
    uint64_t seed;
    // camera frame in FP64 (computed on the host)
    double eye[3], f[3], r[3], u[3], tv, th;
    LightView light;
};

struct GenInfoDev {
    int n_close;
    int pad0;
    int64_t shift_s;
    unsigned long long f_total;
    int64_t paths;
    int64_t m_far_kept;
};

cudaError_t generate_vpls(const Exec &ex, const SceneView &s, const GenArgs &g, float4 *pos,
                          void *nrm, void *flux, int format, GenInfoDev *report);
cudaError_t light_vpls(const Exec &ex, const LightView &L, int n, uint64_t seed, float4 *pos, void *nrm, void *flux,
                       int fmt);
struct CamArgs;
cudaError_t generate_rs(const Exec &ex, const SceneView &s, const GenArgs &g, const CamArgs &pilot, float d2min,
                        float eps, float4 *pos, void *nrm, void *flux, int fmt, GenInfoDev *report);

// ---- gather.cu -----------------------------------------------------------------
struct CamArgs {
    float eye[3], f[3], r[3], u[3];
    float tv, th;
    int32_t width, height;
};

struct GatherArgs {
    int32_t width, height, count;
    float d2_min, ray_eps;
    int32_t precision, visibility;
    int32_t tile_w;        // pixel tile width of a warp (4, 8, 16, 32; 0 = 8)
    int32_t blocks_per_sm; // resident blocks per SM of the persistent grid (0 = occupancy limit)
    int32_t vpl_tile;      // VPLs staged per warp at a time: 16, 32 or 64
    int32_t walk;          // 0: beam walk for narrow shadow packets, 1: per-lane packet walk only
    int32_t tile_order;    // 0 auto, 1 scan order, 2 costliest tiles first (single-view gathers)
    const float4 *g_pos;
    const void *g_nrm, *g_alb;
    const float4 *v_pos;
    const void *v_nrm, *v_flux;
    float4 *out;
};

// one view of a batched gather (a device table built by vpl_batch_create,
// views in order of their first tile)
struct ViewDesc {
    int32_t width, height, count, tiles_x;
    int32_t tile_begin, vpl_begin, pad1, pad2; // first tile / first entry in the batch's VPL order array
    const float4 *g_pos;
    const void *g_nrm, *g_alb;
    const float4 *v_pos;
    const void *v_nrm, *v_flux;
    float4 *out;
    const void *pad3;
};

int tile_shift_of(int tile_w);
cudaError_t gather_batch(const Exec &ex, const SceneView &s, const GatherArgs &a, const ViewDesc *views, int n_views,
                         int n_tiles, int tile_shift, int *counter, int64_t n_vpls);

cudaError_t gbuffer_build(const Exec &ex, const SceneView &s, const CamArgs &c, bool brute,
                          float4 *pos, void *nrm, void *alb, int format);
cudaError_t gather(const Exec &ex, const SceneView &s, const GatherArgs &a);
// the same launch with its scratch in static device memory (no allocation)
cudaError_t gather_noalloc(const Exec &ex, const SceneView &s, const GatherArgs &a);
int64_t gather_noalloc_max_tiles();
cudaError_t gather_counters(const Exec &ex, const SceneView &s, const GatherArgs &a,
                            unsigned long long *counters_dev);
cudaError_t gather_visibility(const Exec &ex, const SceneView &s, const GatherArgs &a,
                              const int32_t *pixels, int64_t n_pixels, int8_t *vis);
cudaError_t debug_philox(const Exec &ex, const uint64_t *ctr, const uint64_t *key, int64_t n,
                         uint64_t *out);
cudaError_t debug_rays(const Exec &ex, const SceneView &s, int mode, int brute, const float4 *a,
                       const float4 *b, int64_t n, int32_t *out_tri, float *out_t);

} // namespace vpl
