// The C ABI of libvpl (declared in include/vpl.h): contexts, the scene
// registry, argument checks, the camera frame, and the order of launches of
// each pipeline step.  Host code here is compiled with -ffp-contract=off: the
// camera frame feeds the exact FP64 close-range decisions.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "vpl_internal.h"

using namespace vpl;

namespace {

struct SceneRec {
    SceneBuffers b;
    vpl_light light;
};

void free_scene(SceneBuffers &b)
{
    void *ps[] = {b.tri, b.nodes, b.bnodes, b.nrm, b.rho, b.verts, b.idx, b.gbox, b.vbox, b.depth};
    for (void *p : ps)
        if (p) cudaFree(p);
    b = SceneBuffers();
}

} // namespace

struct vpl_ctx {
    int device = 0;
    std::string err;
    int *d_status = nullptr;
    GenInfoDev *d_info = nullptr;
    std::map<uint64_t, SceneRec *> scenes;
    uint64_t next_id = 1;
    int64_t launches = 0;
    bool timing = false;
    cudaEvent_t ev[6] = {};
    bool ev_valid[6] = {};
    cudaMemPool_t pool = nullptr;
    struct Batch {
        ViewDesc *views = nullptr; // device table, sorted by first tile
        int *counter = nullptr;    // the launch's tile counter
        int n_views = 0, n_tiles = 0, tile_shift = 3;
        int64_t n_vpls = 0;        // VPLs of all views
    };
    std::map<uint64_t, Batch> batches;
    uint64_t next_batch = 1;
};

namespace {

const double kPiHost = 3.14159265358979323846;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(vpl_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(vpl_ctx *ctx, cudaError_t e, const char *where)
{
    cudaGetLastError(); // clear a sticky launch error so later calls are not confused
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? VPL_ERR_OOM : VPL_ERR_CUDA, m);
}

#define CK(ctx, expr, where)                                     \
    do {                                                         \
        cudaError_t e__ = (expr);                                \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, where); \
    } while (0)

Exec exec_of(vpl_ctx *ctx, vpl_stream stream)
{
    Exec e;
    e.stream = (cudaStream_t)stream;
    e.launches = &ctx->launches;
    e.status = ctx->d_status;
    e.pool = ctx->pool;
    e.timing = ctx->timing;
    return e;
}

void mark(vpl_ctx *ctx, int k, vpl_stream stream)
{
    if (!ctx->timing) return;
    cudaEventRecord(ctx->ev[k], (cudaStream_t)stream);
    ctx->ev_valid[k] = true;
}

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int check_light(vpl_ctx *ctx, const vpl_light *L)
{
    if (!L) return fail(ctx, VPL_ERR_INVALID_ARG, "light is NULL");
    if (L->type != VPL_LIGHT_AREA && L->type != VPL_LIGHT_POINT)
        return fail(ctx, VPL_ERR_INVALID_ARG, "light.type must be 0 (area) or 1 (point)");
    if (!finite3(L->center) || !finite3(L->normal) || !finite3(L->edge_u) || !finite3(L->edge_v) ||
        !finite3(L->power))
        return fail(ctx, VPL_ERR_INVALID_ARG, "light fields must be finite");
    for (int c = 0; c < 3; c++)
        if (L->power[c] < 0.0f) return fail(ctx, VPL_ERR_INVALID_ARG, "light.power must be >= 0");
    return VPL_OK;
}

struct Frame {
    double e[3], f[3], r[3], u[3], tv, th;
};

double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// camera frame: f = forward/|forward|, r = unit(f x up), u = r x f,
// tan(vfov/2) and tan(hfov/2) = tan(vfov/2) W / H
int camera_frame(vpl_ctx *ctx, const vpl_camera *c, Frame *F)
{
    if (!c) return fail(ctx, VPL_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 0 || c->height < 0 || (int64_t)c->width * c->height > (int64_t)1 << 31)
        return fail(ctx, VPL_ERR_INVALID_ARG, "camera width/height out of range");
    if (!(c->vfov_deg > 0.0f && c->vfov_deg < 180.0f))
        return fail(ctx, VPL_ERR_INVALID_ARG, "camera vfov_deg must lie in (0, 180)");
    if (!finite3(c->eye) || !finite3(c->forward) || !finite3(c->up))
        return fail(ctx, VPL_ERR_INVALID_ARG, "camera vectors must be finite");
    double fw[3] = {(double)c->forward[0], (double)c->forward[1], (double)c->forward[2]};
    double up[3] = {(double)c->up[0], (double)c->up[1], (double)c->up[2]};
    double l = std::sqrt(dot3(fw, fw));
    if (!(l > 0.0)) return fail(ctx, VPL_ERR_INVALID_ARG, "camera forward is zero");
    for (int a = 0; a < 3; a++) {
        F->e[a] = (double)c->eye[a];
        F->f[a] = fw[a] / l;
    }
    double rr[3];
    cross3(F->f, up, rr);
    double lr = std::sqrt(dot3(rr, rr));
    if (!(lr > 0.0)) return fail(ctx, VPL_ERR_INVALID_ARG, "camera up is parallel to forward");
    for (int a = 0; a < 3; a++) F->r[a] = rr[a] / lr;
    cross3(F->r, F->f, F->u);
    F->tv = std::tan((double)c->vfov_deg * (kPiHost / 180.0) * 0.5);
    F->th = c->height > 0 ? (F->tv * (double)c->width) / (double)c->height : F->tv;
    return VPL_OK;
}

SceneRec *find_scene(vpl_ctx *ctx, vpl_scene_id id)
{
    auto it = ctx->scenes.find(id);
    return it == ctx->scenes.end() ? nullptr : it->second;
}

SceneView view_of(const SceneRec *s)
{
    SceneView v;
    v.n_tris = (int32_t)s->b.n_tris;
    v.n_nodes = (int32_t)(s->b.n_tris > 1 ? s->b.n_tris - 1 : 1);
    v.tri = s->b.tri;
    v.nodes = s->b.nodes;
    v.bnodes = s->b.bnodes;
    v.nrm = s->b.nrm;
    v.rho = s->b.rho;
    v.verts = s->b.verts;
    v.idx = s->b.idx;
    v.gbox = s->b.gbox;
    return v;
}

LightView light_of(const vpl_light &L)
{
    LightView v;
    memcpy(v.center, L.center, sizeof v.center);
    memcpy(v.normal, L.normal, sizeof v.normal);
    memcpy(v.edge_u, L.edge_u, sizeof v.edge_u);
    memcpy(v.edge_v, L.edge_v, sizeof v.edge_v);
    memcpy(v.power, L.power, sizeof v.power);
    v.type = L.type;
    return v;
}

int check_gbuffer(vpl_ctx *ctx, const vpl_gbuffer *g, const vpl_camera *cam)
{
    if (!g) return fail(ctx, VPL_ERR_INVALID_ARG, "gbuffer is NULL");
    if (g->width < 0 || g->height < 0) return fail(ctx, VPL_ERR_INVALID_ARG, "gbuffer size negative");
    if (cam && (g->width != cam->width || g->height != cam->height))
        return fail(ctx, VPL_ERR_INVALID_ARG, "gbuffer size differs from the camera's");
    if (g->format != VPL_FORMAT_FP32 && g->format != VPL_FORMAT_FP16)
        return fail(ctx, VPL_ERR_INVALID_ARG, "gbuffer format must be 0 (FP32) or 1 (FP16)");
    if ((int64_t)g->width * g->height > 0 && (!g->pos || !g->nrm || !g->albedo))
        return fail(ctx, VPL_ERR_INVALID_ARG, "gbuffer pointers must be non-NULL");
    return VPL_OK;
}

int check_vpls(vpl_ctx *ctx, const vpl_vpl_set *v)
{
    if (!v) return fail(ctx, VPL_ERR_INVALID_ARG, "vpl set is NULL");
    if (v->count < 0) return fail(ctx, VPL_ERR_INVALID_ARG, "vpl count negative");
    if (v->format != VPL_FORMAT_FP32 && v->format != VPL_FORMAT_FP16)
        return fail(ctx, VPL_ERR_INVALID_ARG, "vpl format must be 0 (FP32) or 1 (FP16)");
    if (v->count > 0 && (!v->pos || !v->nrm || !v->flux))
        return fail(ctx, VPL_ERR_INVALID_ARG, "vpl pointers must be non-NULL");
    return VPL_OK;
}

int check_gather(vpl_ctx *ctx, const vpl_gather_params *p, int gfmt, int vfmt)
{
    if (!p) return fail(ctx, VPL_ERR_INVALID_ARG, "gather params are NULL");
    if (p->visibility < 0 || p->visibility > 2) return fail(ctx, VPL_ERR_INVALID_ARG, "visibility must be 0, 1 or 2");
    if (p->precision < 0 || p->precision > 2) return fail(ctx, VPL_ERR_INVALID_ARG, "precision must be 0, 1 or 2");
    if (!(p->d2_min >= 0.0f) || !std::isfinite(p->d2_min)) return fail(ctx, VPL_ERR_INVALID_ARG, "d2_min must be >= 0");
    if (!(p->ray_eps >= 0.0f) || !std::isfinite(p->ray_eps)) return fail(ctx, VPL_ERR_INVALID_ARG, "ray_eps must be >= 0");
    if (p->tile_w != 0 && p->tile_w != 4 && p->tile_w != 8 && p->tile_w != 16 && p->tile_w != 32)
        return fail(ctx, VPL_ERR_INVALID_ARG, "tile_w must be 0, 4, 8, 16 or 32");
    if (p->blocks_per_sm < 0) return fail(ctx, VPL_ERR_INVALID_ARG, "blocks_per_sm must be >= 0");
    if (p->vpl_tile != 0 && p->vpl_tile != 16 && p->vpl_tile != 32 && p->vpl_tile != 64)
        return fail(ctx, VPL_ERR_INVALID_ARG, "vpl_tile must be 0, 16, 32 or 64");
    if (p->walk != 0 && p->walk != 1) return fail(ctx, VPL_ERR_INVALID_ARG, "walk must be 0 or 1");
    if (p->tile_order < 0 || p->tile_order > 2) return fail(ctx, VPL_ERR_INVALID_ARG, "tile_order must be 0, 1 or 2");
    int want = p->precision == VPL_PREC_FP32 ? VPL_FORMAT_FP32 : VPL_FORMAT_FP16;
    if (gfmt != want || vfmt != want)
        return fail(ctx, VPL_ERR_INVALID_ARG, "buffer formats must be FP32 for precision 0 and FP16 otherwise");
    return VPL_OK;
}

int check_gen(vpl_ctx *ctx, const vpl_gen_params *g)
{
    if (!g) return fail(ctx, VPL_ERR_INVALID_ARG, "gen params are NULL");
    if (g->m_close < 0 || g->m_far < 0) return fail(ctx, VPL_ERR_INVALID_ARG, "m_close / m_far must be >= 0");
    if (g->max_bounces < 1 || g->max_bounces > 15) return fail(ctx, VPL_ERR_INVALID_ARG, "max_bounces must be 1..15");
    if (g->light_samples < 1) return fail(ctx, VPL_ERR_INVALID_ARG, "light_samples must be >= 1");
    if (g->rules & ~(VPL_RULE_ANY_VERTEX | VPL_RULE_SET_SUM)) return fail(ctx, VPL_ERR_INVALID_ARG, "unknown rule bits");
    if (!(g->d_close >= 0.0) || !std::isfinite(g->d_close)) return fail(ctx, VPL_ERR_INVALID_ARG, "d_close must be >= 0");
    if (!(g->ray_eps >= 0.0f) || !std::isfinite(g->ray_eps)) return fail(ctx, VPL_ERR_INVALID_ARG, "ray_eps must be >= 0");
    if (g->ir_max_paths < 0 || g->ir_max_paths > ((int64_t)1 << 26))
        return fail(ctx, VPL_ERR_INVALID_ARG, "ir_max_paths must be in [0, 2^26]");
    if ((int64_t)g->m_close + g->m_far > ((int64_t)1 << 30)) return fail(ctx, VPL_ERR_INVALID_ARG, "too many VPLs");
    return VPL_OK;
}

GenArgs gen_args(const Frame &F, const vpl_gen_params *g, const vpl_light &L)
{
    GenArgs a;
    a.d_close = g->d_close;
    a.ray_eps = g->ray_eps;
    a.m_close = g->m_close;
    a.m_far = g->m_far;
    a.max_bounces = g->max_bounces;
    a.light_samples = g->light_samples;
    a.close_rule = (g->rules & VPL_RULE_ANY_VERTEX) ? 1 : 0;
    a.patch_rule = (g->rules & VPL_RULE_SET_SUM) ? 1 : 0;
    a.max_paths = g->ir_max_paths > 0 ? g->ir_max_paths : 16 * (int64_t)g->m_far + 4096;
    a.seed = g->seed;
    for (int k = 0; k < 3; k++) {
        a.eye[k] = F.e[k];
        a.f[k] = F.f[k];
        a.r[k] = F.r[k];
        a.u[k] = F.u[k];
    }
    a.tv = F.tv;
    a.th = F.th;
    a.light = light_of(L);
    return a;
}

CamArgs cam_args(const Frame &F, const vpl_camera *c)
{
    CamArgs a;
    for (int k = 0; k < 3; k++) {
        a.eye[k] = (float)F.e[k];
        a.f[k] = (float)F.f[k];
        a.r[k] = (float)F.r[k];
        a.u[k] = (float)F.u[k];
    }
    a.tv = (float)F.tv;
    a.th = (float)F.th;
    a.width = c->width;
    a.height = c->height;
    return a;
}

GatherArgs gather_args(const vpl_gbuffer *g, const vpl_vpl_set *v, const vpl_gather_params *p, float *out)
{
    GatherArgs a;
    a.width = g->width;
    a.height = g->height;
    a.count = v->count;
    a.d2_min = p->d2_min;
    a.ray_eps = p->ray_eps;
    a.precision = p->precision;
    a.visibility = p->visibility;
    a.tile_w = p->tile_w;
    a.blocks_per_sm = p->blocks_per_sm;
    a.vpl_tile = p->vpl_tile ? p->vpl_tile : 64;
    a.walk = p->walk;
    a.tile_order = p->tile_order;
    a.g_pos = (const float4 *)g->pos;
    a.g_nrm = g->nrm;
    a.g_alb = g->albedo;
    a.v_pos = (const float4 *)v->pos;
    a.v_nrm = v->nrm;
    a.v_flux = v->flux;
    a.out = (float4 *)out;
    return a;
}

} // namespace

extern "C" {

int vpl_create(vpl_ctx **out, int device)
{
    if (!out) return VPL_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return device < 0 || (n > 0 && device >= n) ? VPL_ERR_INVALID_ARG : VPL_ERR_CUDA;
    }
    DeviceGuard g(device);
    vpl_ctx *ctx = new vpl_ctx();
    ctx->device = device;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->d_info, sizeof(GenInfoDev)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_info, 0, sizeof(GenInfoDev)) != cudaSuccess ||
        cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        vpl_destroy(ctx);
        return VPL_ERR_CUDA;
    }
    uint64_t keep = ~0ULL;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (auto &e : ctx->ev) cudaEventCreate(&e);
    *out = ctx;
    return VPL_OK;
}

void vpl_destroy(vpl_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->batches) {
        cudaFree(kv.second.views);
        cudaFree(kv.second.counter);
    }
    ctx->batches.clear();
    for (auto &kv : ctx->scenes) {
        free_scene(kv.second->b);
        delete kv.second;
    }
    ctx->scenes.clear();
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_info) cudaFree(ctx->d_info);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
}

const char *vpl_last_error(const vpl_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int vpl_scene_upload(vpl_ctx *ctx, const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                     const float *albedo, const vpl_light *light, vpl_stream stream, vpl_scene_id *out)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    if (!out) return fail(ctx, VPL_ERR_INVALID_ARG, "out is NULL");
    *out = 0;
    if (!verts || !tris || !albedo) return fail(ctx, VPL_ERR_INVALID_ARG, "scene arrays must be non-NULL");
    if (n_tris < 1 || n_tris > ((int64_t)1 << 30)) return fail(ctx, VPL_ERR_INVALID_ARG, "n_tris must be in [1, 2^30]");
    if (n_verts < 1 || n_verts > ((int64_t)1 << 31) - 1) return fail(ctx, VPL_ERR_INVALID_ARG, "n_verts out of range");
    int rc = check_light(ctx, light);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    SceneRec *s = new SceneRec();
    s->light = *light;
    Exec ex = exec_of(ctx, stream);
    mark(ctx, 0, stream);
    cudaError_t e = build_scene(ex, verts, n_verts, tris, n_tris, albedo, &s->b);
    mark(ctx, 1, stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize((cudaStream_t)stream);
        free_scene(s->b);
        delete s;
        return cuda_fail(ctx, e, "vpl_scene_upload");
    }
    uint64_t id = ctx->next_id++;
    ctx->scenes[id] = s;
    *out = id;
    return VPL_OK;
}

int vpl_scene_release(vpl_ctx *ctx, vpl_scene_id scene)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize(); // work in flight may still read the scene
    free_scene(s->b);
    delete s;
    ctx->scenes.erase(scene);
    return VPL_OK;
}

int vpl_scene_query(vpl_ctx *ctx, vpl_scene_id scene, vpl_scene_info *out)
{
    if (!ctx || !out) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    DeviceGuard g(ctx->device);
    CK(ctx, cudaDeviceSynchronize(), "vpl_scene_query");
    int depth = 0;
    float box[6];
    CK(ctx, cudaMemcpy(&depth, s->b.depth, sizeof depth, cudaMemcpyDeviceToHost), "vpl_scene_query");
    CK(ctx, cudaMemcpy(box, s->b.vbox, sizeof box, cudaMemcpyDeviceToHost), "vpl_scene_query");
    out->n_tris = s->b.n_tris;
    out->n_nodes = s->b.n_tris > 1 ? s->b.n_tris - 1 : 1;
    out->depth = depth;
    out->device_bytes = (int64_t)s->b.bytes;
    memcpy(out->bounds_lo, box, sizeof out->bounds_lo);
    memcpy(out->bounds_hi, box + 3, sizeof out->bounds_hi);
    return VPL_OK;
}

int vpl_gbuffer_build(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam, const vpl_gbuffer *out,
                      vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    Frame F;
    int rc = camera_frame(ctx, cam, &F);
    if (rc) return rc;
    if ((rc = check_gbuffer(ctx, out, cam))) return rc;
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    CK(ctx, gbuffer_build(ex, view_of(s), cam_args(F, cam), false, (float4 *)out->pos, out->nrm, out->albedo,
                          out->format),
       "vpl_gbuffer_build");
    return VPL_OK;
}

int vpl_generate(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam, const vpl_gen_params *gen,
                 const vpl_vpl_set *vpls, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    Frame F;
    int rc = camera_frame(ctx, cam, &F);
    if (rc) return rc;
    if ((rc = check_gen(ctx, gen))) return rc;
    if ((rc = check_vpls(ctx, vpls))) return rc;
    if (vpls->count != gen->m_close + gen->m_far)
        return fail(ctx, VPL_ERR_INVALID_ARG, "vpl set count must equal m_close + m_far");
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    CK(ctx, generate_vpls(ex, view_of(s), gen_args(F, gen, s->light), (float4 *)vpls->pos, vpls->nrm, vpls->flux,
                          vpls->format, ctx->d_info),
       "vpl_generate");
    return VPL_OK;
}

int vpl_generate_rs(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam, const vpl_gen_params *gen, int32_t pilot,
                    float d2_min, float ray_eps, const vpl_vpl_set *vpls, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    Frame F;
    int rc = camera_frame(ctx, cam, &F);
    if (rc) return rc;
    if ((rc = check_gen(ctx, gen))) return rc;
    if ((rc = check_vpls(ctx, vpls))) return rc;
    if (gen->m_close != 0) return fail(ctx, VPL_ERR_INVALID_ARG, "rejection sampling makes far VPLs only: m_close must be 0");
    if (vpls->count != gen->m_far) return fail(ctx, VPL_ERR_INVALID_ARG, "vpl set count must equal m_far");
    if (pilot < 1 || pilot > 1024) return fail(ctx, VPL_ERR_INVALID_ARG, "pilot must be in [1, 1024]");
    if (!(d2_min >= 0.0f) || !std::isfinite(d2_min) || !(ray_eps >= 0.0f) || !std::isfinite(ray_eps))
        return fail(ctx, VPL_ERR_INVALID_ARG, "d2_min and ray_eps must be finite and >= 0");
    vpl_camera pc = *cam;
    pc.width = pilot;
    const int64_t ph = ((int64_t)pilot * cam->height + cam->width / 2) / cam->width;
    pc.height = (int32_t)(ph > 0 ? ph : 1);
    Frame PF;
    if ((rc = camera_frame(ctx, &pc, &PF))) return rc;
    DeviceGuard g(ctx->device);
    CK(ctx, generate_rs(exec_of(ctx, stream), view_of(s), gen_args(F, gen, s->light), cam_args(PF, &pc), d2_min,
                        ray_eps, (float4 *)vpls->pos, vpls->nrm, vpls->flux, vpls->format, ctx->d_info),
       "vpl_generate_rs");
    return VPL_OK;
}

int vpl_light_vpls(vpl_ctx *ctx, vpl_scene_id scene, int32_t n, uint64_t seed, const vpl_vpl_set *vpls,
                   vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    int rc = check_vpls(ctx, vpls);
    if (rc) return rc;
    if (n < 0 || vpls->count != n) return fail(ctx, VPL_ERR_INVALID_ARG, "vpl set count must equal n >= 0");
    if (s->light.type != VPL_LIGHT_AREA)
        return fail(ctx, VPL_ERR_UNSUPPORTED, "light samples need an area light (a point light has no normal)");
    DeviceGuard g(ctx->device);
    CK(ctx, light_vpls(exec_of(ctx, stream), light_of(s->light), n, seed, (float4 *)vpls->pos, vpls->nrm, vpls->flux,
                       vpls->format),
       "vpl_light_vpls");
    return VPL_OK;
}

int vpl_generate_info(vpl_ctx *ctx, vpl_gen_info *out)
{
    if (!ctx || !out) return VPL_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(ctx, cudaDeviceSynchronize(), "vpl_generate_info");
    GenInfoDev d;
    int st = 0;
    CK(ctx, cudaMemcpy(&d, ctx->d_info, sizeof d, cudaMemcpyDeviceToHost), "vpl_generate_info");
    CK(ctx, cudaMemcpy(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost), "vpl_generate_info");
    out->n_close = d.n_close;
    out->shift_s = d.shift_s;
    out->f_total = d.f_total;
    out->paths = d.paths;
    out->m_far_kept = d.m_far_kept;
    out->status = st;
    return VPL_OK;
}

int vpl_gather(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf, const vpl_vpl_set *vpls,
               const vpl_gather_params *params, float *out_rgba, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    int rc = check_gbuffer(ctx, gbuf, nullptr);
    if (rc) return rc;
    if ((rc = check_vpls(ctx, vpls))) return rc;
    if ((rc = check_gather(ctx, params, gbuf->format, vpls->format))) return rc;
    if ((int64_t)gbuf->width * gbuf->height > 0 && !out_rgba) return fail(ctx, VPL_ERR_INVALID_ARG, "out_rgba is NULL");
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    for (int k = 2; k < 4; k++) ctx->ev_valid[k] = false;
    mark(ctx, 4, stream);
    CK(ctx, gather(ex, view_of(s), gather_args(gbuf, vpls, params, out_rgba)), "vpl_gather");
    mark(ctx, 5, stream);
    return VPL_OK;
}

int vpl_gather_noalloc(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf, const vpl_vpl_set *vpls,
                       const vpl_gather_params *params, float *out_rgba, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    int rc = check_gbuffer(ctx, gbuf, nullptr);
    if (rc) return rc;
    if ((rc = check_vpls(ctx, vpls))) return rc;
    if ((rc = check_gather(ctx, params, gbuf->format, vpls->format))) return rc;
    if ((int64_t)gbuf->width * gbuf->height > 0 && !out_rgba) return fail(ctx, VPL_ERR_INVALID_ARG, "out_rgba is NULL");
    const int tsh = tile_shift_of(params->tile_w);
    const int64_t tw = (int64_t)1 << tsh, th = 32 >> tsh;
    const int64_t tiles = (((int64_t)gbuf->width + tw - 1) / tw) * (((int64_t)gbuf->height + th - 1) / th);
    if (tiles > gather_noalloc_max_tiles())
        return fail(ctx, VPL_ERR_INVALID_ARG,
                    "vpl_gather_noalloc: image has more than 2^30 tiles of 32 pixels in the chosen tile shape, "
                    "the most its static tile counter supports");
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    // timed like vpl_gather (the events are created with the context)
    for (int k = 2; k < 4; k++) ctx->ev_valid[k] = false;
    mark(ctx, 4, stream);
    CK(ctx, gather_noalloc(ex, view_of(s), gather_args(gbuf, vpls, params, out_rgba)), "vpl_gather_noalloc");
    mark(ctx, 5, stream);
    return VPL_OK;
}

} // extern "C"

namespace {
// host view table of a batch: views with the most VPLs first, tile ranges
// in that order
int build_view_table(vpl_ctx *ctx, int32_t n_views, const vpl_gbuffer *gbufs, const vpl_vpl_set *vpls,
                     float *const *out_rgba, int32_t tile_w, std::vector<ViewDesc> &h, int64_t &tiles,
                     int64_t &n_vpls)
{
    if (n_views < 1 || !gbufs || !vpls || !out_rgba) return fail(ctx, VPL_ERR_INVALID_ARG, "bad batch arrays");
    if (n_views > (1 << 22)) return fail(ctx, VPL_ERR_INVALID_ARG, "a batch holds at most 2^22 views");
    if (tile_w != 0 && tile_w != 4 && tile_w != 8 && tile_w != 16 && tile_w != 32)
        return fail(ctx, VPL_ERR_INVALID_ARG, "tile_w must be 0, 4, 8, 16 or 32");
    int fmt = gbufs[0].format;
    for (int i = 0; i < n_views; i++) {
        int rc = check_gbuffer(ctx, &gbufs[i], nullptr);
        if (rc) return rc;
        if ((rc = check_vpls(ctx, &vpls[i]))) return rc;
        if (gbufs[i].format != fmt || vpls[i].format != fmt)
            return fail(ctx, VPL_ERR_INVALID_ARG, "all views of a batch need one format");
        if ((int64_t)gbufs[i].width * gbufs[i].height > 0 && !out_rgba[i])
            return fail(ctx, VPL_ERR_INVALID_ARG, "out_rgba[i] is NULL");
    }
    const int tsh = tile_shift_of(tile_w);
    const int64_t tw = (int64_t)1 << tsh, th = 32 >> tsh;
    std::vector<int> order(n_views);
    for (int i = 0; i < n_views; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return vpls[a].count > vpls[b].count; });
    h.assign(n_views, ViewDesc());
    tiles = 0;
    n_vpls = 0;
    for (int k = 0; k < n_views; k++) {
        const int i = order[k];
        ViewDesc &d = h[k];
        memset(&d, 0, sizeof d);
        d.width = gbufs[i].width;
        d.height = gbufs[i].height;
        d.count = vpls[i].count;
        d.tiles_x = (int32_t)((gbufs[i].width + tw - 1) / tw);
        d.tile_begin = (int32_t)tiles;
        d.vpl_begin = (int32_t)n_vpls;
        n_vpls += vpls[i].count;
        if (n_vpls > INT32_MAX) return fail(ctx, VPL_ERR_INVALID_ARG, "batch has more than 2^31 - 1 VPLs");
        d.g_pos = (const float4 *)gbufs[i].pos;
        d.g_nrm = gbufs[i].nrm;
        d.g_alb = gbufs[i].albedo;
        d.v_pos = (const float4 *)vpls[i].pos;
        d.v_nrm = vpls[i].nrm;
        d.v_flux = vpls[i].flux;
        d.out = (float4 *)out_rgba[i];
        tiles += (int64_t)d.tiles_x * ((gbufs[i].height + th - 1) / th);
        if (tiles > ((int64_t)1 << 30)) return fail(ctx, VPL_ERR_INVALID_ARG, "batch has more than 2^30 tiles");
    }
    return VPL_OK;
}
} // namespace

extern "C" {

int vpl_gather_views(vpl_ctx *ctx, vpl_scene_id scene, int32_t n_views, const vpl_gbuffer *gbufs,
                     const vpl_vpl_set *vpls, float *const *out_rgba, const vpl_gather_params *params,
                     vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    const int fmt = params && params->precision != VPL_PREC_FP32 ? VPL_FORMAT_FP16 : VPL_FORMAT_FP32;
    int rc = check_gather(ctx, params, fmt, fmt);
    if (rc) return rc;
    std::vector<ViewDesc> h;
    int64_t tiles = 0;
    int64_t n_vpls = 0;
    if ((rc = build_view_table(ctx, n_views, gbufs, vpls, out_rgba, params->tile_w, h, tiles, n_vpls))) return rc;
    if (gbufs[0].format != fmt) return fail(ctx, VPL_ERR_INVALID_ARG, "buffer format does not match the precision");
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    Tmp table, counter;
    CK(ctx, table.alloc(ex, sizeof(ViewDesc) * n_views), "vpl_gather_views");
    CK(ctx, counter.alloc(ex, sizeof(int)), "vpl_gather_views");
    CK(ctx, cudaMemcpyAsync(table.p, h.data(), sizeof(ViewDesc) * n_views, cudaMemcpyHostToDevice, ex.stream),
       "vpl_gather_views");
    GatherArgs a;
    memset(&a, 0, sizeof a);
    a.d2_min = params->d2_min;
    a.ray_eps = params->ray_eps;
    a.precision = params->precision;
    a.visibility = params->visibility;
    a.blocks_per_sm = params->blocks_per_sm;
    a.vpl_tile = params->vpl_tile ? params->vpl_tile : 64;
    a.walk = params->walk;
    a.tile_order = params->tile_order;
    CK(ctx, gather_batch(ex, view_of(s), a, table.as<ViewDesc>(), n_views, (int)tiles,
                         tile_shift_of(params->tile_w), counter.as<int>(), n_vpls),
       "vpl_gather_views");
    return VPL_OK;
}

int vpl_batch_create(vpl_ctx *ctx, int32_t n_views, const vpl_gbuffer *gbufs, const vpl_vpl_set *vpls,
                     float *const *out_rgba, int32_t tile_w, vpl_batch_id *out)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    if (!out) return fail(ctx, VPL_ERR_INVALID_ARG, "out is NULL");
    *out = 0;
    std::vector<ViewDesc> h;
    int64_t tiles = 0;
    int64_t n_vpls = 0;
    int rc = build_view_table(ctx, n_views, gbufs, vpls, out_rgba, tile_w, h, tiles, n_vpls);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    vpl_ctx::Batch b;
    b.n_views = n_views;
    b.n_vpls = n_vpls;
    b.n_tiles = (int)tiles;
    b.tile_shift = tile_shift_of(tile_w);
    CK(ctx, cudaMalloc(&b.views, sizeof(ViewDesc) * n_views), "vpl_batch_create");
    if (cudaMalloc(&b.counter, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(b.views, h.data(), sizeof(ViewDesc) * n_views, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(b.views);
        if (b.counter) cudaFree(b.counter);
        return cuda_fail(ctx, cudaErrorMemoryAllocation, "vpl_batch_create");
    }
    const uint64_t id = ctx->next_batch++;
    ctx->batches[id] = b;
    *out = id;
    return VPL_OK;
}

int vpl_batch_destroy(vpl_ctx *ctx, vpl_batch_id batch)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    auto it = ctx->batches.find(batch);
    if (it == ctx->batches.end()) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown batch id");
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(it->second.views);
    cudaFree(it->second.counter);
    ctx->batches.erase(it);
    return VPL_OK;
}

int vpl_gather_batch(vpl_ctx *ctx, vpl_scene_id scene, vpl_batch_id batch, const vpl_gather_params *params,
                     vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    auto it = ctx->batches.find(batch);
    if (it == ctx->batches.end()) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown batch id");
    const int fmt = params && params->precision != VPL_PREC_FP32 ? VPL_FORMAT_FP16 : VPL_FORMAT_FP32;
    int rc = check_gather(ctx, params, fmt, fmt);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    GatherArgs a;
    memset(&a, 0, sizeof a);
    a.d2_min = params->d2_min;
    a.ray_eps = params->ray_eps;
    a.precision = params->precision;
    a.visibility = params->visibility;
    a.blocks_per_sm = params->blocks_per_sm;
    a.vpl_tile = params->vpl_tile ? params->vpl_tile : 64;
    a.walk = params->walk;
    a.tile_order = params->tile_order;
    const vpl_ctx::Batch &b = it->second;
    CK(ctx, gather_batch(exec_of(ctx, stream), view_of(s), a, b.views, b.n_views, b.n_tiles, b.tile_shift, b.counter,
                         b.n_vpls),
       "vpl_gather_batch");
    return VPL_OK;
}

int vpl_render(vpl_ctx *ctx, vpl_scene_id scene, const vpl_camera *cam, const vpl_gen_params *gen,
               const vpl_gather_params *params, float *out_rgba, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    Frame F;
    int rc = camera_frame(ctx, cam, &F);
    if (rc) return rc;
    if ((rc = check_gen(ctx, gen))) return rc;
    const int fmt = params && params->precision != VPL_PREC_FP32 ? VPL_FORMAT_FP16 : VPL_FORMAT_FP32;
    if ((rc = check_gather(ctx, params, fmt, fmt))) return rc;
    const int64_t npx = (int64_t)cam->width * cam->height;
    if (npx > 0 && !out_rgba) return fail(ctx, VPL_ERR_INVALID_ARG, "out_rgba is NULL");
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    const int64_t M = (int64_t)gen->m_close + gen->m_far;
    Tmp gpos, gnrm, galb, vpos, vnrm, vflux;
    const size_t attr = fmt == VPL_FORMAT_FP16 ? 8 : 16; // half4 or float4 rows
    CK(ctx, gpos.alloc(ex, sizeof(float4) * npx), "vpl_render");
    CK(ctx, gnrm.alloc(ex, attr * npx), "vpl_render");
    CK(ctx, galb.alloc(ex, attr * npx), "vpl_render");
    CK(ctx, vpos.alloc(ex, sizeof(float4) * M), "vpl_render");
    CK(ctx, vnrm.alloc(ex, attr * M), "vpl_render");
    CK(ctx, vflux.alloc(ex, attr * M), "vpl_render");
    vpl_gbuffer gb = {gpos.p, gnrm.p, galb.p, cam->width, cam->height, fmt, 0};
    vpl_vpl_set vs = {vpos.p, vnrm.p, vflux.p, (int32_t)M, fmt};
    SceneView v = view_of(s);
    mark(ctx, 2, stream);
    CK(ctx, gbuffer_build(ex, v, cam_args(F, cam), params->visibility == VPL_VIS_BRUTE, gpos.as<float4>(), gnrm.p,
                          galb.p, fmt),
       "vpl_render gbuffer");
    mark(ctx, 3, stream);
    CK(ctx, generate_vpls(ex, v, gen_args(F, gen, s->light), vpos.as<float4>(), vnrm.p, vflux.p, fmt,
                          ctx->d_info),
       "vpl_render generate");
    mark(ctx, 4, stream);
    CK(ctx, gather(ex, v, gather_args(&gb, &vs, params, out_rgba)), "vpl_render gather");
    mark(ctx, 5, stream);
    return VPL_OK;
}

int vpl_sync(vpl_ctx *ctx, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(ctx, cudaStreamSynchronize((cudaStream_t)stream), "vpl_sync");
    int st = 0;
    CK(ctx, cudaMemcpy(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost), "vpl_sync");
    if (st != 0) {
        CK(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)), "vpl_sync");
        const char *what = st == VPL_ERR_TRAVERSAL_LIMIT   ? "a BVH walk hit its step or stack limit"
                           : st == VPL_ERR_EMPTY_CLOSE     ? "no close-range face for m_close > 0"
                           : st == VPL_ERR_PATHS_EXHAUSTED ? "ir_max_paths light paths gave fewer than m_far VPLs"
                           : st == VPL_ERR_INVALID_ARG     ? "an index (vertex or debug pixel) was out of range"
                                                           : "device error";
        ctx->err = what;
    }
    return st;
}

int vpl_debug_philox(vpl_ctx *ctx, const uint64_t *ctr, const uint64_t *key, int64_t n, uint64_t *out,
                     vpl_stream stream)
{
    if (!ctx || n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(ctx, VPL_ERR_INVALID_ARG, "bad philox args");
    DeviceGuard g(ctx->device);
    CK(ctx, debug_philox(exec_of(ctx, stream), ctr, key, n, out), "vpl_debug_philox");
    return VPL_OK;
}

int vpl_debug_rays(vpl_ctx *ctx, vpl_scene_id scene, int32_t mode, int32_t brute, const float *a, const float *b,
                   int64_t n, int32_t *out_tri, float *out_t, vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    if ((mode != 0 && mode != 1) || n < 0 || (n > 0 && (!a || !b || !out_tri)))
        return fail(ctx, VPL_ERR_INVALID_ARG, "bad ray query args");
    DeviceGuard g(ctx->device);
    CK(ctx, debug_rays(exec_of(ctx, stream), view_of(s), mode, brute, (const float4 *)a, (const float4 *)b, n, out_tri,
                       out_t),
       "vpl_debug_rays");
    return VPL_OK;
}

int vpl_debug_visibility(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf, const vpl_vpl_set *vpls,
                         const vpl_gather_params *params, const int32_t *pixels, int64_t n_pixels, int8_t *vis,
                         vpl_stream stream)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    int rc = check_gbuffer(ctx, gbuf, nullptr);
    if (rc) return rc;
    if ((rc = check_vpls(ctx, vpls))) return rc;
    if ((rc = check_gather(ctx, params, gbuf->format, vpls->format))) return rc;
    if (n_pixels < 0 || (n_pixels > 0 && (!pixels || !vis))) return fail(ctx, VPL_ERR_INVALID_ARG, "bad pixel list");
    DeviceGuard g(ctx->device);
    CK(ctx, gather_visibility(exec_of(ctx, stream), view_of(s), gather_args(gbuf, vpls, params, nullptr), pixels,
                              n_pixels, vis),
       "vpl_debug_visibility");
    return VPL_OK;
}

int vpl_set_timing(vpl_ctx *ctx, int32_t on)
{
    if (!ctx) return VPL_ERR_INVALID_ARG;
    ctx->timing = on != 0;
    return VPL_OK;
}

int vpl_stage_times(vpl_ctx *ctx, float *ms, int32_t n)
{
    if (!ctx || (n > 0 && !ms)) return VPL_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const int pairs[4][2] = {{0, 1}, {2, 3}, {3, 4}, {4, 5}};
    for (int k = 0; k < n && k < 4; k++) {
        ms[k] = -1.0f;
        int a = pairs[k][0], b = pairs[k][1];
        if (ctx->ev_valid[a] && ctx->ev_valid[b]) {
            CK(ctx, cudaEventSynchronize(ctx->ev[b]), "vpl_stage_times");
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, ctx->ev[a], ctx->ev[b]) == cudaSuccess) ms[k] = t;
            else cudaGetLastError();
        }
    }
    return VPL_OK;
}

int64_t vpl_launch_count(const vpl_ctx *ctx) { return ctx ? ctx->launches : -1; }

int vpl_pool_stats(vpl_ctx *ctx, int32_t reset_high, uint64_t out[3])
{
    if (!ctx || !out) return VPL_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    unsigned long long used = 0, high = 0, reserved = 0;
    if (reset_high) {
        unsigned long long zero = 0;
        CK(ctx, cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &zero), "vpl_pool_stats");
    }
    CK(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used), "vpl_pool_stats");
    CK(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &high), "vpl_pool_stats");
    CK(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrReservedMemCurrent, &reserved), "vpl_pool_stats");
    out[0] = used;
    out[1] = high;
    out[2] = reserved;
    return VPL_OK;
}

int vpl_gather_counters(vpl_ctx *ctx, vpl_scene_id scene, const vpl_gbuffer *gbuf, const vpl_vpl_set *vpls,
                        const vpl_gather_params *params, uint64_t out[6], vpl_stream stream)
{
    if (!ctx || !out) return VPL_ERR_INVALID_ARG;
    SceneRec *s = find_scene(ctx, scene);
    if (!s) return fail(ctx, VPL_ERR_NOT_FOUND, "unknown scene id");
    int rc = check_gbuffer(ctx, gbuf, nullptr);
    if (rc) return rc;
    if ((rc = check_vpls(ctx, vpls))) return rc;
    if ((rc = check_gather(ctx, params, gbuf->format, vpls->format))) return rc;
    DeviceGuard g(ctx->device);
    Exec ex = exec_of(ctx, stream);
    unsigned long long *d = nullptr;
    CK(ctx, cudaMallocFromPoolAsync((void **)&d, sizeof(unsigned long long) * 6, ctx->pool, ex.stream),
       "vpl_gather_counters");
    cudaError_t e = gather_counters(ex, view_of(s), gather_args(gbuf, vpls, params, nullptr), d);
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ex.stream);
    cudaFreeAsync(d, ex.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ex.stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "vpl_gather_counters");
    for (int k = 0; k < 6; k++) out[k] = h[k];
    return VPL_OK;
}

} // extern "C"
