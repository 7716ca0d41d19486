/*
 * vpl.h -- C ABI of the GB300 renderer for the hybrid close-range VPL method
 * (Jin, Wang, Zheng, Hua, Huo, "A Virtual Point Light Generation Method in
 * Close-Range Area", arXiv 2203.11484).
 *
 * Pipeline (Sec. 3, "overall flow" steps (1)-(4)):
 *   (1) find the close-range faces from the camera position and orientation;
 *   (2) patch-based VPLs on the close range (Eq. 2 and the "Realization"
 *       paragraph: Morton order, area prefix sum f, inverse g, equal-area
 *       strata, random points in triangles);
 *   (3) sparse instant radiosity over the whole scene, keeping only the hits
 *       on the distant part;
 *   (4) render with all VPLs: the indirect term of Eq. 1, sum over VPLs of
 *       G_i V_i L_i, with V found by shadow rays through a device BVH.
 *
 * Conventions (all entry points):
 *  - Return value: a vpl_status.  Argument errors are detected on the host and
 *    returned at once; nothing is enqueued then.  Errors found by kernels
 *    (traversal limits, an empty close set, too few light paths) are latched
 *    in a per-context device status word and returned by vpl_sync.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *    work is enqueued asynchronously on it; buffers must stay valid until the
 *    stream has passed the call.
 *  - Memory: scene data (triangles, BVH) is owned by the context from
 *    vpl_scene_upload until vpl_scene_release / vpl_destroy.  G-buffers, VPL
 *    sets and images are caller-owned device memory.  Temporary buffers come
 *    from the device's stream-ordered memory pool (cudaMallocAsync) on the
 *    call's stream.
 *  - Positions are in scene units; triangles are one-sided, front side where
 *    (b - a) x (c - a) points (counter-clockwise winding).
 *  - A context is bound to one device and is not thread-safe; use one per
 *    host thread.
 *
 * Device layouts (structure of arrays, 16-byte float4 / 8-byte half4 rows):
 *  G-buffer row p = y * width + x:
 *    pos[p]    float4 (x, y, z, triangle id as int bits; -1 = empty pixel)
 *    nrm[p]    float4 (unit geometric normal, 0)      | half4 in FP16 format
 *    albedo[p] float4 (r, g, b, 0)                    | half4 in FP16 format
 *  VPL row i (patch VPLs first in stratum order, then distant VPLs in
 *  (path, bounce) order), FP32 format:
 *    pos[i]    float4 (x, y, z, triangle id as int bits)
 *    nrm[i]    float4 (unit normal, tag as int bits)
 *              tag = stratum k for patch VPLs, 16 * path + bounce otherwise
 *    flux[i]   float4 (reflected power r, g, b, 0)
 *  FP16 format (32 bytes a row):
 *    pos[i]    float4 (x, y, z, m) with m = max(r, g, b) in FP32
 *    nrm[i]    half4 (unit normal, 0)
 *    flux[i]   half4 (r / m, g / m, b / m, 0): colour in FP16, magnitude in FP32
 *  Image: float4 (r, g, b, 0) per pixel, same row order as the G-buffer.
 */
#ifndef VPL_H
#define VPL_H

#include <stdint.h>

#if defined(__GNUC__)
#define VPL_API __attribute__((visibility("default")))
#else
#define VPL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vpl_ctx vpl_ctx;
typedef uint64_t vpl_scene_id;
typedef void *vpl_stream; /* cudaStream_t */

typedef enum {
    VPL_OK = 0,
    VPL_ERR_INVALID_ARG = 1,      /* bad pointer, size or parameter            */
    VPL_ERR_OOM = 2,              /* device allocation failed                   */
    VPL_ERR_CUDA = 3,             /* CUDA runtime error (see vpl_last_error)    */
    VPL_ERR_TRAVERSAL_LIMIT = 4,  /* a BVH walk hit its step or stack limit     */
    VPL_ERR_NOT_FOUND = 5,        /* unknown scene id                           */
    VPL_ERR_EMPTY_CLOSE = 6,      /* m_close > 0 but no face is close range     */
    VPL_ERR_PATHS_EXHAUSTED = 7,  /* ir_max_paths paths gave fewer than m_far   */
    VPL_ERR_UNSUPPORTED = 8       /* combination not built into this library    */
} vpl_status;

enum { VPL_LIGHT_AREA = 0, VPL_LIGHT_POINT = 1 };
enum { VPL_RULE_ANY_VERTEX = 1, VPL_RULE_SET_SUM = 2 };
enum { VPL_PREC_FP32 = 0, VPL_PREC_FP16_KAHAN = 1, VPL_PREC_FP16_PLAIN = 2 };
enum { VPL_VIS_BVH = 0, VPL_VIS_BRUTE = 1, VPL_VIS_NONE = 2 };
enum { VPL_FORMAT_FP32 = 0, VPL_FORMAT_FP16 = 1 };

/* Light (Sec. 3.1 uses point lights; a one-sided square area light is the
 * other supported emitter).  Area light: centre, unit normal of the emitting
 * side, full edge vectors, total power (W per channel), Lambertian, radiance
 * power / (pi * area).  Point light: centre and power, isotropic. */
typedef struct {
    float center[3], normal[3], edge_u[3], edge_v[3], power[3];
    int32_t type;
} vpl_light;

/* Pinhole camera: eye, viewing direction (any length), up hint, vertical
 * field of view in degrees; the horizontal one follows from width/height.
 * Pixel (x, y), y = 0 at the top, looks through
 * forward + (2(x+0.5)/W - 1) tan(hfov/2) right + (1 - 2(y+0.5)/H) tan(vfov/2) up. */
typedef struct {
    float eye[3], forward[3], up[3];
    float vfov_deg;
    int32_t width, height;
} vpl_camera;

/* VPL generation (Sec. 3, pipeline steps (1)-(3)).
 *  d_close       close-range distance threshold (camera to face centroid)
 *  rules         readings of the paper, as bits (0 = the defaults):
 *                VPL_RULE_ANY_VERTEX: a face is "inside the field of view
 *                and nearer than d_close" at its centroid or any vertex (else
 *                at its centroid; both decide in FP64, exactly);
 *                VPL_RULE_SET_SUM: a stratum that spans several close faces
 *                gives one VPL at their area-weighted centroid with the sum
 *                of their Eq. 2 terms, each at the face's centroid with the
 *                area it gives the stratum, tagged with the face giving the
 *                most area (else a random point of the face at the
 *                stratum's jittered point)
 *  ray_eps       offset along normals of secondary-ray origins (scene units)
 *  m_close       patch VPLs on the close range (the paper's K)
 *  m_far         instant-radiosity VPLs on the distant part
 *  max_bounces   surface hits per light path that may store a VPL
 *  light_samples points on an area light per patch VPL for Eq. 2
 *  ir_max_paths  upper bound on light paths traced (0 = 16 m_far + 4096)
 *  seed          Philox4x64-10 key word 0 */
typedef struct {
    double d_close;
    float ray_eps;
    int32_t m_close, m_far, max_bounces, light_samples;
    int32_t rules;
    int64_t ir_max_paths;
    uint64_t seed;
} vpl_gen_params;

/* Gather (Eq. 1, indirect part).
 *  d2_min     lower clamp of the squared distance in the geometry term
 *  ray_eps    offset of both shadow-ray end points along their normals
 *  precision  VPL_PREC_*: FP32, or FP16 attributes with Kahan / plain FP32 sums
 *  visibility VPL_VIS_*: BVH shadow rays, all-triangle test, or none (V = 1)
 *  tile_w     pixel tile of one warp: tile_w x (32 / tile_w), tile_w in
 *             {4, 8, 16, 32}; 0 = 8 (8 x 4)
 *  blocks_per_sm  cap on resident blocks per SM of the persistent grid
 *             (0 = as many as fit)
 *  vpl_tile   VPLs a warp stages in shared memory at a time (the VPL side
 *             of the pixel-tile x VPL-tile blocking): 16, 32 or 64; 0 = 64.
 *  walk       shadow-packet traversal of the BVH visibility: 0 = the beam
 *             walk for packets whose segments form a narrow beam (one
 *             conservative test per child box for the whole packet, exact
 *             per-lane tests at the leaves) and the per-lane packet walk for
 *             the others; 1 = the per-lane packet walk for every packet.
 *  tile_order order in which the persistent grid takes the pixel tiles of a
 *             single-view gather: 1 = scan order; 2 = most costly first, the
 *             cost of each tile measured by a first pass over a sample of
 *             the VPLs (64 per tile, every ceil(count / 64)-th in the gather's
 *             VPL order), so that the slowest tiles do not start last and set
 *             the end of the launch; 0 = cost order when the VPL set has at
 *             least 8192 VPLs (the sample pass then costs under 1/128 of the
 *             gather), else scan order.  Batched gathers and
 *             vpl_gather_noalloc always take scan order.
 *             tile_w, blocks_per_sm, vpl_tile, walk and tile_order change
 *             speed only, never the result (every pixel sums its VPLs in the
 *             same order and every segment gets the same answer from either
 *             walk). */
typedef struct {
    float d2_min, ray_eps;
    int32_t precision, visibility;
    int32_t tile_w, blocks_per_sm;
    int32_t vpl_tile;
    int32_t walk;
    int32_t tile_order;
} vpl_gather_params;

/* caller-owned device buffers (see the layouts above) */
typedef struct {
    void *pos, *nrm, *flux;
    int32_t count;
    int32_t format; /* VPL_FORMAT_* of nrm and flux */
} vpl_vpl_set;

typedef struct {
    void *pos, *nrm, *albedo;
    int32_t width, height;
    int32_t format; /* VPL_FORMAT_* of nrm and albedo */
    int32_t reserved;
} vpl_gbuffer;

typedef struct {
    int64_t n_tris;
    int64_t n_nodes;      /* internal BVH nodes                      */
    int64_t depth;        /* longest root-to-leaf path               */
    int64_t device_bytes; /* bytes held for this scene               */
    float bounds_lo[3], bounds_hi[3];
} vpl_scene_info;

/* statistics of the last vpl_generate on a context */
typedef struct {
    int64_t n_close;   /* close-range faces |C|                     */
    int64_t shift_s;   /* areas quantised as round(A * 2^S)        */
    uint64_t f_total;  /* f(N): total quantised close-range area   */
    int64_t paths;     /* light paths P that the kept VPLs needed  */
    int64_t m_far_kept;
    int64_t status;    /* vpl_status of that call's device checks  */
} vpl_gen_info;

/* Context on `device` (a CUDA ordinal).  *out is NULL on failure. */
VPL_API int vpl_create(vpl_ctx **out, int device);
VPL_API void vpl_destroy(vpl_ctx *ctx);
/* Text of the last error on this context ("" when none).  Owned by ctx. */
VPL_API const char *vpl_last_error(const vpl_ctx *ctx);

/* Copies a triangle scene to the device and builds its BVH (not in the
 * paper: the acceleration structure behind every ray query).
 *  verts  float[n_verts][3], tris int32[n_tris][3] (indices into verts),
 *  albedo float[n_tris][3] diffuse reflectance per face, light: the emitter.
 *  verts/tris/albedo may be host or device pointers.  Requires n_tris >= 1
 *  and indices in [0, n_verts); returns the new scene's id in *out.
 *  Unlike the other calls it waits on `stream` a few times while the BVH is
 *  built (the host reads the cluster count back), so it returns after the
 *  build, and it must not be called while `stream` is being captured. */
VPL_API int vpl_scene_upload(vpl_ctx *ctx, const float *verts, int64_t n_verts, const int32_t *tris,
                     int64_t n_tris, const float *albedo, const vpl_light *light,
                     vpl_stream stream, vpl_scene_id *out);
VPL_API int vpl_scene_release(vpl_ctx *ctx, vpl_scene_id scene);
/* Synchronises the stream last used by the scene's upload. */
VPL_API int vpl_scene_query(vpl_ctx *ctx, vpl_scene_id scene, vpl_scene_info *out);

/* Primary rays: closest front-face hit per pixel centre (the points y of
 * Eq. 1).  A miss or a back-face hit leaves the pixel empty. */
VPL_API int vpl_gbuffer_build(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam,
                      const vpl_gbuffer *out, vpl_stream stream);

/* Steps (1)-(3): out->count must equal m_close + m_far. */
VPL_API int vpl_generate(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam,
                 const vpl_gen_params *gen, const vpl_vpl_set *vpls, vpl_stream stream);
/* Synchronises the device and reports the numbers of the generation that
 * finished last (vpl_generate or vpl_render; with calls in flight on several
 * streams, whichever of them wrote its record last). */
VPL_API int vpl_generate_info(vpl_ctx *ctx, vpl_gen_info *out);

/* Rejection-sampled instant radiosity, the comparison method the paper cites
 * (Sec. 2, r3): VPLs of light paths that contribute little to the image are
 * rejected.  The light paths are those of plain instant radiosity (no close
 * range; gen->m_close must be 0, vpls->count == gen->m_far); every surface
 * hit is a candidate whose contribution c to the image is estimated on a
 * pilot grid of pilot x round(pilot * height / width) pixels over the same
 * view (Eq. 1's pair term with visibility, d2_min and ray_eps as in the
 * gather, the receiver's and the path's albedos, mean over the channels, in
 * FP64); a candidate is kept with probability p = min(1, c / cbar), cbar the
 * mean c over the candidates of all ir_max_paths paths, when the top 24 bits
 * of Philox4x64-10 word 0 at key (seed, 5), counter (path, bounce, 0, 0) fall
 * below p; the first m_far kept in (path, bounce) order are the VPLs, P = last
 * kept path + 1, flux = power x albedos / (P p) (unbiased).  Tags and the
 * report of vpl_generate_info as for vpl_generate; too few kept candidates
 * latch VPL_ERR_PATHS_EXHAUSTED. */
VPL_API int vpl_generate_rs(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam,
                            const vpl_gen_params *gen, int32_t pilot, float d2_min, float ray_eps,
                            const vpl_vpl_set *vpls, vpl_stream stream);

/* Direct term L_e(y) of Eq. 1 (the light's own contribution, which the VPL
 * sum leaves out) as n light-sample VPLs written to vpls (count == n, either
 * format): sample k is the point c + (2 s1 - 1) edge_u / 2 + (2 s2 - 1)
 * edge_v / 2 of the scene's square light, with s1, s2 the top 24 bits of
 * Philox4x64-10 words 0 and 1 at key (seed, 4), counter (k, 0, 0, 0), the
 * light's normal, flux power / n and tag -1 - k.  vpl_gather of these rows
 * gives (rho/pi) (1/n) sum_k power cos_k cos_y V / (pi d^2), the Monte Carlo
 * estimate of the one-sided Lambertian emitter (radiance power / (pi A))
 * reflected at y; gathering them together with the indirect VPLs (rows of
 * one set) gives the composite L(y) of Eq. 1.  A point light has no
 * emitting normal for this sum: VPL_ERR_UNSUPPORTED. */
VPL_API int vpl_light_vpls(vpl_ctx *ctx, vpl_scene_id scene, int32_t n, uint64_t seed,
                           const vpl_vpl_set *vpls, vpl_stream stream);

/* Step (4): out_rgba (device float4[width*height]) receives, per pixel,
 * (rho/pi) * sum_i flux_i cos_i cos_y / (pi max(d^2, d2_min)) * V_i.
 * The sum runs over the VPLs in the Morton order of their positions (a
 * stable sort made on the stream for each call; it only changes FP32
 * rounding, and makes neighbouring shadow rays of a warp share BVH work).
 * In cost order (params->tile_order) the call first gathers a sample of the
 * VPLs into no image to time each pixel tile, then sorts the tiles.  Scratch
 * (the VPL order; in cost order the tile costs and tile order, 16 B per tile)
 * comes from the context's stream-ordered memory pool. */
VPL_API int vpl_gather(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf,
               const vpl_vpl_set *vpls, const vpl_gather_params *params, float *out_rgba,
               vpl_stream stream);

/* vpl_gather for callers that must not allocate device memory.  The paper has
 * no counterpart to this entry point.  It exists for callers that reserve
 * their device memory up front and may not allocate while they run -- a
 * render loop working inside a fixed memory budget owned by its host
 * application, or code where an allocation could block on or synchronise
 * with other work on the device.  Arguments, results and errors are those of
 * vpl_gather; the caller passes every input and output buffer, and this call
 * makes no cudaMalloc/cudaFree, pool or other allocating call.  It sums the
 * VPLs in the order given (sorting them would need scratch), so its image
 * equals vpl_gather's up to FP32 rounding, not bit for bit, and it is slower.
 * Its one piece of scratch, the tile counter of the gather's dynamic
 * scheduler, sits in a 256-byte static device array of the library that
 * every GPU which loads libvpl holds until the process exits.  The first
 * call on each device looks up that array's device address with the
 * context's device current; make that first call before any stream capture.
 * Each call clears the counter before its launch; all calls share the array,
 * so calls that overlap on the GPU (other streams, other contexts on the same
 * device) race on it and must be ordered by the caller.  Images of more than
 * 2^30 tiles of 32 pixels in the tile shape of params->tile_w return
 * VPL_ERR_INVALID_ARG.  The looked-up address is kept for the life of the
 * process: after the application resets a device (cudaDeviceReset), this
 * entry point must not be called on that device again. */
VPL_API int vpl_gather_noalloc(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf,
                               const vpl_vpl_set *vpls, const vpl_gather_params *params,
                               float *out_rgba, vpl_stream stream);

/* Batched step (4): many views, each with its own G-buffer, VPL set and
 * image (resolutions and VPL counts may differ), gathered by ONE persistent
 * launch whose warps take 32-pixel tiles of all views from one queue, views
 * with the most VPLs first.  vpl_batch_create copies a device table of the
 * views (synchronously; the buffers must stay allocated while the batch is
 * used) and fixes the tile width (tile_w as in vpl_gather_params, 0 = 8);
 * vpl_gather_batch then enqueues the VPL sort of all views (pool memory on
 * the stream), a memset and one gather kernel; it can be captured in a CUDA
 * graph.  Each pixel's sum runs in the view's VPL order (as in vpl_gather)
 * within one thread: images equal those of vpl_gather per view.  Calls with
 * the same batch must not overlap on the GPU (they share its tile counter).
 * At most 2^22 views and 2^31 - 1 VPLs in all. */
typedef uint64_t vpl_batch_id;
VPL_API int vpl_batch_create(vpl_ctx *ctx, int32_t n_views, const vpl_gbuffer *gbufs,
                             const vpl_vpl_set *vpls, float *const *out_rgba, int32_t tile_w,
                             vpl_batch_id *out);
VPL_API int vpl_batch_destroy(vpl_ctx *ctx, vpl_batch_id batch);
VPL_API int vpl_gather_batch(vpl_ctx *ctx, vpl_scene_id scene, vpl_batch_id batch,
                             const vpl_gather_params *params, vpl_stream stream);

/* The batched gather without a persistent batch: the view table is built on
 * the host and copied to pool memory on `stream` by this call, so it costs no
 * device-wide synchronisation (the serving loop's path; not capturable).
 * Arguments as vpl_batch_create plus the gather parameters. */
VPL_API int vpl_gather_views(vpl_ctx *ctx, vpl_scene_id scene, int32_t n_views,
                             const vpl_gbuffer *gbufs, const vpl_vpl_set *vpls,
                             float *const *out_rgba, const vpl_gather_params *params,
                             vpl_stream stream);

/* Steps (1)-(4) with library-held temporaries: G-buffer, VPLs, gather. */
VPL_API int vpl_render(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam,
               const vpl_gen_params *gen, const vpl_gather_params *params, float *out_rgba,
               vpl_stream stream);

/* Waits for `stream`, then returns and clears the context's device status
 * (VPL_OK or the first vpl_status a kernel latched). */
VPL_API int vpl_sync(vpl_ctx *ctx, vpl_stream stream);

/* ---- diagnostics used by the tests and the benchmark ------------------- */

/* Philox4x64-10 blocks: out[4i..4i+3] = philox(ctr[4i..4i+3], key[2i..2i+1]);
 * all three are device arrays of uint64. */
VPL_API int vpl_debug_philox(vpl_ctx *ctx, const uint64_t *ctr, const uint64_t *key, int64_t n,
                     uint64_t *out, vpl_stream stream);
/* Ray queries on a scene through the device BVH (or all triangles when
 * brute != 0).  a, b: device float4[n] (xyz used).
 *  mode 0: segment a -> b, out_tri[i] = 1 when blocked at t in (0,1), else 0
 *  mode 1: ray a + t b, t > 0; out_tri[i] = closest original triangle id or -1,
 *          out_t[i] = its t (may be NULL in mode 0). */
VPL_API int vpl_debug_rays(vpl_ctx *ctx, vpl_scene_id scene, int32_t mode, int32_t brute,
                   const float *a, const float *b, int64_t n, int32_t *out_tri, float *out_t,
                   vpl_stream stream);
/* Visibility bits of the gather for chosen pixels: vis[k * count + i] =
 * 1 visible, 0 blocked, -1 not traced (zero shading term or zero flux), for
 * pixel pixels[k] (row index) and VPL i.  pixels, vis: device int32 / int8.
 * Pixels k * 32 .. k * 32 + 31 of the list form one packet, as the 32
 * pixels of one tile do in vpl_gather.  A pixel index outside the G-buffer
 * sets VPL_ERR_INVALID_ARG in the device status (vpl_sync) and its row is
 * left unwritten. */
VPL_API int vpl_debug_visibility(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf,
                         const vpl_vpl_set *vpls, const vpl_gather_params *params,
                         const int32_t *pixels, int64_t n_pixels, int8_t *vis,
                         vpl_stream stream);
/* Per-call stage timing with CUDA events on the call's stream (off by
 * default).  vpl_stage_times writes up to n floats (ms) of the last render /
 * gather: [0] scene build, [1] G-buffer, [2] generation, [3] gather. */
VPL_API int vpl_set_timing(vpl_ctx *ctx, int32_t on);
VPL_API int vpl_stage_times(vpl_ctx *ctx, float *ms, int32_t n);
/* Kernel launches enqueued by this context since its creation. */
VPL_API int64_t vpl_launch_count(const vpl_ctx *ctx);
/* Bytes of the context's stream-ordered pool (the library's temporaries):
 * out[0] in use now, out[1] the most in use at once since the context was
 * created or since the last call with reset_high != 0 (which first sets the
 * mark to the bytes in use now), out[2] reserved from the device.  Host-side
 * query; it waits for nothing, so synchronise the streams whose calls should
 * be counted first.  Not in the paper: a diagnostic of memory admission. */
VPL_API int vpl_pool_stats(vpl_ctx *ctx, int32_t reset_high, uint64_t out[3]);
/* Work counters of one gather launch (not timed): out[0] pairs with a
 * non-empty receiver, [1] pairs with a non-zero shading term (shadow rays),
 * [2] BVH node visits summed over rays, [3] triangle tests summed over rays,
 * [4] blocked rays, [5] warp-wide packet traversal steps.  The counts are
 * those of each ray's own traversal (the per-lane packet walk, whose node
 * visits and triangle tests each ray needs); vpl_gather itself may walk
 * shadow packets with one conservative test per node for the whole packet,
 * which gives the same visibility with other step counts. */
VPL_API int vpl_gather_counters(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf,
                                const vpl_vpl_set *vpls, const vpl_gather_params *params,
                                uint64_t out[6], vpl_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* VPL_H */
