// VPL generation (Sec. 3, pipeline steps (1)-(3)):
//   (1) close-range faces from the camera (one-sided, inside the field of
//       view, nearer than d_close; patch sampling further needs the face to
//       face the light);
//   (2) patch VPLs: the close faces in Morton order of their centroids, the
//       area prefix sum f, K equal-area strata [kF/K, (k+1)F/K), a jittered
//       point per stratum mapped back through g = f^-1, a uniform random
//       point in the selected triangle, and its value from Eq. 2 with D the
//       area one VPL represents;
//   (3) sparse instant radiosity: light paths whose hits on distant faces
//       become VPLs while hits on close faces are discarded.
// Decisions (close set, Morton codes, quantised areas, strata) are computed
// in FP64 with every operation rounded separately, so they are exact and
// reproducible; geometry is FP64 and visibility uses the FP32 BVH.
#include "vpl_internal.h"

namespace vpl {

constexpr int kGenThreads = 128;

// point p inside the field of view and nearer than d_close
__device__ __forceinline__ bool in_view(const D3 &p, const GenArgs &g)
{
    D3 e = dmk(g.eye[0], g.eye[1], g.eye[2]);
    D3 f = dmk(g.f[0], g.f[1], g.f[2]), r = dmk(g.r[0], g.r[1], g.r[2]), u = dmk(g.u[0], g.u[1], g.u[2]);
    D3 v = dsub(p, e);
    double z = ddot(v, f);
    if (!(z > 0.0)) return false;                                  // in front
    if (!(fabs(ddot(v, r)) <= __dmul_rn(z, g.th))) return false;   // horizontal field of view
    if (!(fabs(ddot(v, u)) <= __dmul_rn(z, g.tv))) return false;   // vertical field of view
    return ddot(v, v) < __dmul_rn(g.d_close, g.d_close);           // nearer than d_close
}

// close range: faces the camera, in view and range at its centroid (rule 0)
// or at its centroid or any vertex (rule 1), and faces the light
__device__ __forceinline__ bool is_close(const TriD &T, const GenArgs &g)
{
    D3 e = dmk(g.eye[0], g.eye[1], g.eye[2]);
    if (!(ddot(T.cr, dsub(e, T.g)) > 0.0)) return false;          // faces the camera
    if (!(in_view(T.g, g) || (g.close_rule == 1 && (in_view(T.a, g) || in_view(T.b, g) || in_view(T.c, g)))))
        return false;
    D3 cl = dld(g.light.center);
    if (!(ddot(T.cr, dsub(cl, T.g)) > 0.0)) return false;          // faces the light
    if (g.light.type == VPL_LIGHT_AREA && !(ddot(dld(g.light.normal), dsub(T.g, cl)) > 0.0)) return false;
    return true;
}

__global__ void classify_kernel(SceneView s, GenArgs g, uint32_t *flag)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s.n_tris) return;
    flag[t] = is_close(tri_exact(s, t), g) ? 1u : 0u;
}

__global__ void compact_kernel(int n, const uint32_t *flag, const uint32_t *pos, uint32_t *list)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && flag[t]) list[pos[t]] = (uint32_t)t;
}

__device__ __forceinline__ uint32_t quant21(double v, double lo, double hi)
{
    double t = (hi > lo) ? __ddiv_rn(__dsub_rn(v, lo), __dsub_rn(hi, lo)) : 0.0;
    double q = floor(__dmul_rn(t, 2097152.0));
    if (q > 2097151.0) q = 2097151.0;
    if (q < 0.0) q = 0.0;
    return (uint32_t)q;
}

// Morton key of each close face's centroid in the AABB of all centroids
__global__ void close_keys_kernel(SceneView s, const double *gbox, const uint32_t *list, const int *n_close,
                                  uint64_t *keys, uint32_t *vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_close) return;
    uint32_t t = list[i];
    TriD T = tri_exact(s, (int)t);
    keys[i] = morton63(quant21(T.g.x, gbox[0], gbox[3]), quant21(T.g.y, gbox[1], gbox[4]),
                       quant21(T.g.z, gbox[2], gbox[5]));
    vals[i] = t;
}

__global__ void area_kernel(SceneView s, const uint32_t *sorted, const int *n_close, double *area,
                            unsigned long long *amax_bits)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_close) return;
    double a = tri_exact(s, (int)sorted[i]).area;
    area[i] = a;
    atomicMax(amax_bits, (unsigned long long)__double_as_longlong(a)); // a >= 0: bits order like values
}

// q_i = round(A_i 2^S), S = 40 - exponent(max A): integer areas, so that
// f and the strata are exact
__global__ void quant_kernel(const double *area, const int *n_close, const unsigned long long *amax_bits,
                             unsigned long long *q, GenInfoDev *info)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int ex;
    frexp(__longlong_as_double((long long)*amax_bits), &ex);
    int S = 40 - ex;
    if (i == 0) info->shift_s = S;
    if (i >= *n_close) return;
    q[i] = (unsigned long long)llround(ldexp(area[i], S));
}

__global__ void close_info_kernel(const int *n_close, const unsigned long long *F, GenInfoDev *info)
{
    info->n_close = *n_close;
    info->f_total = F[*n_close];
}

// floor(a F / (K 2^32)) for a < K 2^32, F < 2^61, K < 2^31: 128-bit product,
// then long division in 32-bit digits
__device__ __forceinline__ uint64_t stratum_point(uint64_t a, uint64_t F, uint64_t K)
{
    uint64_t lo = a * F, hi = __umul64hi(a, F);
    uint64_t q_lo = (hi << 32) | (lo >> 32); // floor(N / 2^32), low 64 bits
    uint64_t q_hi = hi >> 32;                // and bits 64..95
    uint64_t cur = q_hi, r = cur % K;
    cur = (r << 32) | (q_lo >> 32);
    uint64_t d1 = cur / K;
    r = cur % K;
    cur = (r << 32) | (q_lo & 0xffffffffULL);
    uint64_t d0 = cur / K;
    return (d1 << 32) + d0;
}

// One VPL row.  FP32 format: pos (x, y, z, triangle), nrm (n, tag), flux
// (r, g, b, 0).  FP16 format: pos (x, y, z, m) with m = max(r, g, b) in FP32,
// nrm half4 (n, 0), flux half4 (r/m, g/m, b/m, 0): FP16 holds the colour, FP32
// the magnitude, so fluxes of any size keep an 11-bit mantissa.
__device__ __forceinline__ void store_vpl(float4 *pos, void *nrm, void *flux, int64_t i, float3 x, int tri,
                                          float3 n, int tag, float3 phi, int fmt)
{
    if (fmt == VPL_FORMAT_FP16) {
        const float m = fmaxf(phi.x, fmaxf(phi.y, phi.z));
        const float inv = m > 0.0f ? 1.0f / m : 0.0f;
        pos[i] = make_float4(x.x, x.y, x.z, m);
        __half2 *pn = reinterpret_cast<__half2 *>(nrm) + 2 * i;
        pn[0] = __floats2half2_rn(n.x, n.y);
        pn[1] = __floats2half2_rn(n.z, 0.0f);
        __half2 *pf = reinterpret_cast<__half2 *>(flux) + 2 * i;
        pf[0] = __floats2half2_rn(phi.x * inv, phi.y * inv);
        pf[1] = __floats2half2_rn(phi.z * inv, 0.0f);
    } else {
        pos[i] = make_float4(x.x, x.y, x.z, __int_as_float(tri));
        reinterpret_cast<float4 *>(nrm)[i] = make_float4(n.x, n.y, n.z, __int_as_float(tag));
        reinterpret_cast<float4 *>(flux)[i] = make_float4(phi.x, phi.y, phi.z, 0.0f);
    }
}

__device__ __forceinline__ D3 light_point(const LightView &L, double s1, double s2)
{
    D3 c = dld(L.center);
    if (L.type == VPL_LIGHT_POINT) return c;
    D3 a = dscl(dld(L.edge_u), (2.0 * s1 - 1.0) * 0.5);
    D3 b = dscl(dld(L.edge_v), (2.0 * s2 - 1.0) * 0.5);
    return dadd(dadd(c, a), b);
}

// segment p -> q blocked? (FP32 BVH)
__device__ __forceinline__ bool seg_blocked(const SceneView &s, D3 p, D3 q, int *status)
{
    float3 o = make_float3((float)p.x, (float)p.y, (float)p.z);
    float3 d = make_float3((float)(q.x - p.x), (float)(q.y - p.y), (float)(q.z - p.z));
    return occluded1(s, make_ray(o, d), status);
}

// (2): one thread per stratum k
// Eq. 2 for a VPL k at x (unit normal n) representing area D: the light's
// power reaching D, as a factor of the power (times the albedo it is the
// reflected flux); point light literally, area light by light_samples points
__device__ __forceinline__ double eq2_factor(const SceneView &s, const GenArgs &g, int k, D3 x, D3 n, double D,
                                            int *status)
{
    const LightView &L = g.light;
    D3 cl = dld(L.center);
    D3 xo = dadd(x, dscl(n, (double)g.ray_eps));
    double acc = 0.0;
    if (L.type == VPL_LIGHT_POINT) {
        D3 dv = dsub(cl, x);
        double r = sqrt(ddot(dv, dv));
        double cw = ddot(n, dv) / r;
        if (cw > 0.0 && !seg_blocked(s, xo, cl, status)) acc = D * cw / (4.0 * kPiD * r * r);
    } else {
        D3 nL = dld(L.normal);
        for (int j = 0; j < g.light_samples; j++) {
            uint64_t v[4];
            rng4(g.seed, kStreamLight, (uint64_t)k, (uint64_t)j, v);
            D3 y = light_point(L, u01(v[0]), u01(v[1]));
            D3 dv = dsub(y, x);
            double r2s = ddot(dv, dv), r = sqrt(r2s);
            double cw = ddot(n, dv) / r;
            double cL = -ddot(nL, dv) / r;
            if (cw > 0.0 && cL > 0.0 && !seg_blocked(s, xo, y, status)) acc += cw * cL / (kPiD * r2s);
        }
        acc = D * acc / (double)g.light_samples;
    }
    return acc;
}

__global__ void patch_kernel(SceneView s, GenArgs g, const uint32_t *sorted, const unsigned long long *F,
                             const int *n_close, const GenInfoDev *info, float4 *pos, void *nrm, void *flux,
                             int fmt, int *status)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.m_close) return;
    const int nc = *n_close;
    if (nc == 0) {
        const float3 z = make_float3(0.0f, 0.0f, 0.0f);
        store_vpl(pos, nrm, flux, k, z, -1, z, k, z, fmt);
        if (k == 0) latch(status, VPL_ERR_EMPTY_CLOSE);
        return;
    }
    const uint64_t Ftot = F[nc];
    uint64_t w[4];
    rng4(g.seed, kStreamPatch, (uint64_t)k, 0, w);
    // a jittered point of stratum k, then g(u): f(m) <= u < f(m+1)
    uint64_t u = stratum_point(((uint64_t)k << 32) + (w[0] >> 32), Ftot, (uint64_t)g.m_close);
    int lo = 0, hi = nc;
    while (hi - lo > 1) {
        int mid = lo + (hi - lo) / 2;
        if (F[mid] <= u) lo = mid; else hi = mid;
    }
    const int t = (int)sorted[lo];
    if (g.patch_rule == 1) {
        // the faces overlapping the stratum [A, B) of the prefix
        const uint64_t A = stratum_point((uint64_t)k << 32, Ftot, (uint64_t)g.m_close);
        const uint64_t B = stratum_point((uint64_t)(k + 1) << 32, Ftot, (uint64_t)g.m_close);
        int m0 = lo, m1 = lo;
        while (m0 > 0 && F[m0] > A) m0--;
        while (m1 + 1 < nc && F[m1 + 1] < B) m1++;
        if (m1 > m0) {
            // set sum: each face's Eq. 2 at its centroid with the area it
            // gives the stratum; the VPL at the area-weighted centroid with
            // the area-weighted normal, tagged with the face giving most area
            const int S = (int)info->shift_s;
            double fl[3] = {0.0, 0.0, 0.0};
            D3 xs = dmk(0, 0, 0), ns = dmk(0, 0, 0);
            double Dsum = 0.0;
            uint64_t wbest = 0;
            int tbest = (int)sorted[m0];
            D3 nbest = dmk(0, 0, 0);
            for (int m = m0; m <= m1; m++) {
                const uint64_t a = F[m] > A ? F[m] : A, b = F[m + 1] < B ? F[m + 1] : B;
                if (b <= a) continue;
                const uint64_t wm = b - a;
                const int tm = (int)sorted[m];
                const TriD Tm = tri_exact(s, tm);
                const double nlm = __dsqrt_rn(ddot(Tm.cr, Tm.cr));
                const D3 nm = dmk(__ddiv_rn(Tm.cr.x, nlm), __ddiv_rn(Tm.cr.y, nlm), __ddiv_rn(Tm.cr.z, nlm));
                const double Dm = ldexp((double)wm, -S);
                const double accm = eq2_factor(s, g, k, Tm.g, nm, Dm, status);
                const float4 rho = __ldg(s.rho + tm);
                fl[0] = __dadd_rn(fl[0], __dmul_rn(__dmul_rn((double)rho.x, (double)g.light.power[0]), accm));
                fl[1] = __dadd_rn(fl[1], __dmul_rn(__dmul_rn((double)rho.y, (double)g.light.power[1]), accm));
                fl[2] = __dadd_rn(fl[2], __dmul_rn(__dmul_rn((double)rho.z, (double)g.light.power[2]), accm));
                xs = dadd(xs, dscl(Tm.g, Dm));
                ns = dadd(ns, dscl(nm, Dm));
                Dsum = __dadd_rn(Dsum, Dm);
                if (wm > wbest) {
                    wbest = wm;
                    tbest = tm;
                    nbest = nm;
                }
            }
            const double nl = __dsqrt_rn(ddot(ns, ns));
            const D3 x = dscl(xs, __ddiv_rn(1.0, Dsum));
            const D3 n = nl > 0.0 ? dscl(ns, __ddiv_rn(1.0, nl)) : nbest;
            store_vpl(pos, nrm, flux, k, make_float3((float)x.x, (float)x.y, (float)x.z), tbest,
                      make_float3((float)n.x, (float)n.y, (float)n.z), k,
                      make_float3((float)fl[0], (float)fl[1], (float)fl[2]), fmt);
            return;
        }
    }
    TriD T = tri_exact(s, t);
    // uniform point in the triangle (square-root warp)
    double r1 = u01(w[1]), r2 = u01(w[2]);
    double sr = __dsqrt_rn(r1);
    D3 A = T.a, Bv = dadd(T.a, T.e1), C = dadd(T.a, T.e2);
    D3 x = dadd(dadd(dscl(A, __dsub_rn(1.0, sr)), dscl(Bv, __dmul_rn(sr, __dsub_rn(1.0, r2)))),
                dscl(C, __dmul_rn(sr, r2)));
    double nl = __dsqrt_rn(ddot(T.cr, T.cr));
    D3 n = dmk(__ddiv_rn(T.cr.x, nl), __ddiv_rn(T.cr.y, nl), __ddiv_rn(T.cr.z, nl));
    // Eq. 2 with D = area represented by one VPL
    const double D = ldexp((double)Ftot, -(int)info->shift_s) / (double)g.m_close;
    const double acc = eq2_factor(s, g, k, x, n, D, status);
    float4 rho = __ldg(s.rho + t);
    const LightView &L = g.light;
    store_vpl(pos, nrm, flux, k, make_float3((float)x.x, (float)x.y, (float)x.z), t,
              make_float3((float)n.x, (float)n.y, (float)n.z), k,
              make_float3((float)((double)rho.x * L.power[0] * acc), (float)((double)rho.y * L.power[1] * acc),
                          (float)((double)rho.z * L.power[2] * acc)),
              fmt);
}

// orthonormal basis around a unit vector (Duff et al., JCGT 2017) and
// cosine-weighted directions (Malley's method)
__device__ __forceinline__ D3 cosine_dir(D3 n, double s1, double s2)
{
    double sg = copysign(1.0, n.z);
    double a = -1.0 / (sg + n.z);
    double b = n.x * n.y * a;
    D3 t1 = dmk(1.0 + sg * n.x * n.x * a, sg * b, -sg * n.x);
    D3 t2 = dmk(b, sg + n.y * n.y * a, -n.y);
    double r = sqrt(s1), ph = 2.0 * kPiD * s2;
    double sp, cp;
    sincos(ph, &sp, &cp);
    return dadd(dadd(dscl(t1, r * cp), dscl(t2, r * sp)), dscl(n, sqrt(1.0 - s1)));
}

__device__ __forceinline__ D3 sphere_dir(double s1, double s2)
{
    double z = 1.0 - 2.0 * s1;
    double r = sqrt(fmax(0.0, 1.0 - z * z)), ph = 2.0 * kPiD * s2;
    double sp, cp;
    sincos(ph, &sp, &cp);
    return dmk(r * cp, r * sp, z);
}

// (3): one thread per light path; hits on distant faces become candidate
// VPLs in slot p * B + (bounce - 1)
__global__ void ir_walk_kernel(SceneView s, GenArgs g, const uint32_t *close_flag, int64_t n_paths,
                               float4 *c_pos, float4 *c_nrm, double *c_thr, uint32_t *c_valid, int *status)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_paths) return;
    const int B = g.max_bounces;
    for (int b = 0; b < B; b++) c_valid[p * B + b] = 0u;
    const LightView &L = g.light;
    uint64_t w[4];
    rng4(g.seed, kStreamIR, (uint64_t)p, 0, w);
    D3 o, d;
    if (L.type == VPL_LIGHT_POINT) {
        o = dld(L.center);
        d = sphere_dir(u01(w[2]), u01(w[3]));
    } else {
        o = light_point(L, u01(w[0]), u01(w[1]));
        d = cosine_dir(dld(L.normal), u01(w[2]), u01(w[3]));
    }
    double thr[3] = {1.0, 1.0, 1.0};
    float3 of = make_float3((float)o.x, (float)o.y, (float)o.z);
    for (int b = 1; b <= B; b++) {
        Ray r = make_ray(of, make_float3((float)d.x, (float)d.y, (float)d.z));
        float t;
        int k = closest_hit(s, r, 0.0f, t, status);
        if (k < 0) break;
        float4 nk4 = __ldg(s.nrm + k);
        float3 nk = f3(nk4);
        if (!(dot(r.d, nk) < 0.0f)) break; // the back of a one-sided face absorbs
        float3 x = r.o + r.d * t;
        float4 rho = __ldg(s.rho + k);
        thr[0] = thr[0] * (double)rho.x;
        thr[1] = thr[1] * (double)rho.y;
        thr[2] = thr[2] * (double)rho.z;
        if (!close_flag || !close_flag[k]) {
            int64_t slot = p * B + (b - 1);
            c_pos[slot] = make_float4(x.x, x.y, x.z, __int_as_float(k));
            c_nrm[slot] = make_float4(nk.x, nk.y, nk.z, __int_as_float((int)(p * 16 + b)));
            c_thr[3 * slot] = thr[0];
            c_thr[3 * slot + 1] = thr[1];
            c_thr[3 * slot + 2] = thr[2];
            c_valid[slot] = 1u;
        }
        if (b == B) break;
        rng4(g.seed, kStreamIR, (uint64_t)p, (uint64_t)b, w);
        D3 nd = dmk((double)nk.x, (double)nk.y, (double)nk.z);
        d = cosine_dir(nd, u01(w[0]), u01(w[1]));
        of = x + nk * g.ray_eps;
    }
}

// P = (path of the m_far-th kept candidate) + 1
__global__ void ir_paths_kernel(const uint32_t *c_valid, const uint32_t *rank, int64_t n_slots, int B, int m_far,
                                int64_t n_paths, GenInfoDev *info, int *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        uint32_t total = rank[n_slots];
        info->m_far_kept = total < (uint32_t)m_far ? (int64_t)total : (int64_t)m_far;
        if (total < (uint32_t)m_far) {
            info->paths = n_paths;
            latch(status, VPL_ERR_PATHS_EXHAUSTED);
        }
    }
    if (i < n_slots && c_valid[i] && rank[i] == (uint32_t)(m_far - 1)) info->paths = i / B + 1;
}

__global__ void ir_emit_kernel(GenArgs g, const float4 *c_pos, const float4 *c_nrm, const double *c_thr,
                               const uint32_t *c_valid, const uint32_t *rank, int64_t n_slots,
                               const GenInfoDev *info, float4 *pos, void *nrm, void *flux, int fmt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots || !c_valid[i] || rank[i] >= (uint32_t)g.m_far) return;
    const int64_t v = g.m_close + rank[i];
    const double P = (double)info->paths;
    const float4 cp = c_pos[i], cn = c_nrm[i];
    store_vpl(pos, nrm, flux, v, f3(cp), __float_as_int(cp.w), f3(cn), __float_as_int(cn.w),
              make_float3((float)(g.light.power[0] * c_thr[3 * i] / P), (float)(g.light.power[1] * c_thr[3 * i + 1] / P),
                          (float)(g.light.power[2] * c_thr[3 * i + 2] / P)),
              fmt);
}

// far VPL rows that no path filled (only when the path budget ran out)
__global__ void far_tail_kernel(GenArgs g, const GenInfoDev *info, float4 *pos, void *nrm, void *flux, int fmt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.m_far || i < info->m_far_kept) return;
    const float3 z = make_float3(0.0f, 0.0f, 0.0f);
    store_vpl(pos, nrm, flux, g.m_close + i, z, -1, z, -1, z, fmt);
}

// ---------------------------------------------------------------------------
// Rejection-sampled instant radiosity (the comparison method the paper cites
// as r3): the light paths of plain instant radiosity with no close range;
// every hit is a candidate; its contribution c to the image is estimated on a
// pilot grid of pixels (Eq. 1's pair term with visibility, the receiver's and
// the path's albedos, channel mean, FP64); a candidate is kept with
// probability p = min(1, c / cbar), cbar the mean over all candidates, decided
// by Philox (seed, 5) counter (path, bounce); the first m_far kept in (path,
// bounce) order are the VPLs, P = last kept path + 1, flux = power x albedos
// / (P p).
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;

// block per candidate slot, threads over the pilot pixels (fixed-order sums)
__global__ void __launch_bounds__(kRsThreads) rs_contrib_kernel(SceneView s, GenArgs g, const float4 *c_pos,
                                                                const float4 *c_nrm, const double *c_thr,
                                                                const uint32_t *c_valid, const float4 *p_pos,
                                                                const float4 *p_nrm, const float4 *p_alb, int np,
                                                                float d2min, float eps, double *contrib, int *status)
{
    __shared__ double part[kRsThreads];
    const int64_t slot = blockIdx.x;
    if (!c_valid[slot]) {
        if (threadIdx.x == 0) contrib[slot] = 0.0;
        return;
    }
    const float4 cx = c_pos[slot], cn4 = c_nrm[slot];
    const D3 x = dmk(cx.x, cx.y, cx.z), nx = dmk(cn4.x, cn4.y, cn4.z);
    const float3 q = fma3(f3(cn4), eps, f3(cx));
    const double w[3] = {c_thr[3 * slot] * (double)g.light.power[0], c_thr[3 * slot + 1] * (double)g.light.power[1],
                         c_thr[3 * slot + 2] * (double)g.light.power[2]};
    double acc = 0.0;
    for (int j = threadIdx.x; j < np; j += kRsThreads) {
        const float4 py = p_pos[j];
        if (__float_as_int(py.w) < 0) continue;
        const float4 pn = p_nrm[j];
        const D3 y = dmk(py.x, py.y, py.z), ny = dmk(pn.x, pn.y, pn.z);
        const D3 d = dsub(x, y);
        const double d2 = ddot(d, d);
        if (d2 == 0.0) continue;
        const double dl = __dsqrt_rn(d2);
        const double cy = ddot(ny, d) / dl, ci = -ddot(nx, d) / dl;
        if (!(cy > 0.0) || !(ci > 0.0)) continue;
        const float3 o = fma3(f3(pn), eps, f3(py));
        if (occluded1(s, make_ray(o, q - o), status)) continue;
        const double gterm = ci * cy / (kPiD * fmax(d2, (double)d2min));
        const float4 a = p_alb[j];
        const double c = ((double)a.x * w[0] + (double)a.y * w[1] + (double)a.z * w[2]) / 3.0;
        acc += gterm * c / kPiD;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kRsThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) contrib[slot] = part[0];
}

// fixed-order sums of the contributions and counts of valid candidates
__global__ void __launch_bounds__(kRsThreads) rs_sum_kernel(const double *contrib, const uint32_t *c_valid,
                                                            int64_t n, double *psum, unsigned long long *pcnt)
{
    __shared__ double ps[kRsThreads];
    __shared__ unsigned long long pc[kRsThreads];
    double a = 0.0;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * kRsThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRsThreads)
        if (c_valid[i]) {
            a += contrib[i];
            c++;
        }
    ps[threadIdx.x] = a;
    pc[threadIdx.x] = c;
    __syncthreads();
    for (int h = kRsThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            ps[threadIdx.x] += ps[threadIdx.x + h];
            pc[threadIdx.x] += pc[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        psum[blockIdx.x] = ps[0];
        pcnt[blockIdx.x] = pc[0];
    }
}

// cbar: the partial sums added in a fixed order
__global__ void rs_mean_kernel(const double *psum, const unsigned long long *pcnt, int nparts, double *cbar)
{
    double sum = 0.0;
    unsigned long long cnt = 0;
    for (int k = 0; k < nparts; k++) {
        sum += psum[k];
        cnt += pcnt[k];
    }
    *cbar = cnt ? sum / (double)cnt : 0.0;
}

__global__ void rs_accept_kernel(GenArgs g, const double *contrib, uint32_t *c_valid, const double *cbar_p, int64_t n,
                                 double *prob)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !c_valid[i]) return;
    const double cbar = *cbar_p;
    const double pr = cbar > 0.0 ? fmin(1.0, contrib[i] / cbar) : 1.0;
    const int64_t B = g.max_bounces, p = i / B, b = i % B + 1;
    uint64_t w[4];
    rng4(g.seed, kStreamReject, (uint64_t)p, (uint64_t)b, w);
    prob[i] = pr;
    c_valid[i] = u01(w[0]) < pr ? 1u : 0u;
}

__global__ void rs_emit_kernel(GenArgs g, const float4 *c_pos, const float4 *c_nrm, const double *c_thr,
                               const uint32_t *c_valid, const uint32_t *rank, const double *prob, int64_t n_slots,
                               const GenInfoDev *info, float4 *pos, void *nrm, void *flux, int fmt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots || !c_valid[i] || rank[i] >= (uint32_t)g.m_far) return;
    const int64_t v = rank[i];
    const double d = (double)info->paths * prob[i];
    const float4 cp = c_pos[i], cn = c_nrm[i];
    store_vpl(pos, nrm, flux, v, f3(cp), __float_as_int(cp.w), f3(cn), __float_as_int(cn.w),
              make_float3((float)(g.light.power[0] * c_thr[3 * i] / d), (float)(g.light.power[1] * c_thr[3 * i + 1] / d),
                          (float)(g.light.power[2] * c_thr[3 * i + 2] / d)),
              fmt);
}

cudaError_t generate_rs(const Exec &ex, const SceneView &s, const GenArgs &g, const CamArgs &pilot, float d2min,
                        float eps, float4 *pos, void *nrm, void *flux, int fmt, GenInfoDev *report)
{
    const int TB = kGenThreads;
    Tmp rec;
    VPL_TRY(rec.alloc(ex, sizeof(GenInfoDev)));
    GenInfoDev *info = rec.as<GenInfoDev>();
    VPL_TRY(cudaMemsetAsync(info, 0, sizeof(GenInfoDev), ex.stream));
    if (g.m_far > 0) {
        const int64_t n_paths = g.max_paths, n_slots = n_paths * g.max_bounces;
        const int np = pilot.width * pilot.height;
        Tmp cp, cn, ct, cv, rk, pp, pn, pa, cc, pr, ps, pc;
        VPL_TRY(cp.alloc(ex, sizeof(float4) * n_slots));
        VPL_TRY(cn.alloc(ex, sizeof(float4) * n_slots));
        VPL_TRY(ct.alloc(ex, sizeof(double) * 3 * n_slots));
        VPL_TRY(cv.alloc(ex, sizeof(uint32_t) * n_slots));
        VPL_TRY(rk.alloc(ex, sizeof(uint32_t) * (n_slots + 1)));
        VPL_TRY(pp.alloc(ex, sizeof(float4) * np));
        VPL_TRY(pn.alloc(ex, sizeof(float4) * np));
        VPL_TRY(pa.alloc(ex, sizeof(float4) * np));
        VPL_TRY(cc.alloc(ex, sizeof(double) * n_slots));
        VPL_TRY(pr.alloc(ex, sizeof(double) * n_slots));
        const int nparts = 256;
        VPL_TRY(ps.alloc(ex, sizeof(double) * (nparts + 1))); // partial sums, then cbar
        VPL_TRY(pc.alloc(ex, sizeof(unsigned long long) * nparts));
        ir_walk_kernel<<<grid_for(n_paths, TB), TB, 0, ex.stream>>>(s, g, nullptr, n_paths, cp.as<float4>(),
                                                                    cn.as<float4>(), ct.as<double>(),
                                                                    cv.as<uint32_t>(), ex.status);
        VPL_LAUNCHED(ex);
        VPL_TRY(gbuffer_build(ex, s, pilot, false, pp.as<float4>(), pn.p, pa.p, VPL_FORMAT_FP32));
        rs_contrib_kernel<<<(unsigned)n_slots, kRsThreads, 0, ex.stream>>>(
            s, g, cp.as<float4>(), cn.as<float4>(), ct.as<double>(), cv.as<uint32_t>(), pp.as<float4>(),
            pn.as<float4>(), pa.as<float4>(), np, d2min, eps, cc.as<double>(), ex.status);
        VPL_LAUNCHED(ex);
        rs_sum_kernel<<<nparts, kRsThreads, 0, ex.stream>>>(cc.as<double>(), cv.as<uint32_t>(), n_slots,
                                                            ps.as<double>(), pc.as<unsigned long long>());
        VPL_LAUNCHED(ex);
        rs_mean_kernel<<<1, 1, 0, ex.stream>>>(ps.as<double>(), pc.as<unsigned long long>(), nparts,
                                               ps.as<double>() + nparts);
        VPL_LAUNCHED(ex);
        rs_accept_kernel<<<grid_for(n_slots, 256), 256, 0, ex.stream>>>(g, cc.as<double>(), cv.as<uint32_t>(),
                                                                        ps.as<double>() + nparts, n_slots,
                                                                        pr.as<double>());
        VPL_LAUNCHED(ex);
        VPL_TRY(exclusive_scan<uint32_t>(ex, cv.as<uint32_t>(), rk.as<uint32_t>(), nullptr, n_slots));
        ir_paths_kernel<<<grid_for(n_slots, 256), 256, 0, ex.stream>>>(cv.as<uint32_t>(), rk.as<uint32_t>(), n_slots,
                                                                       g.max_bounces, g.m_far, n_paths, info,
                                                                       ex.status);
        VPL_LAUNCHED(ex);
        rs_emit_kernel<<<grid_for(n_slots, 256), 256, 0, ex.stream>>>(g, cp.as<float4>(), cn.as<float4>(),
                                                                      ct.as<double>(), cv.as<uint32_t>(),
                                                                      rk.as<uint32_t>(), pr.as<double>(), n_slots,
                                                                      info, pos, nrm, flux, fmt);
        VPL_LAUNCHED(ex);
        far_tail_kernel<<<grid_for(g.m_far, 256), 256, 0, ex.stream>>>(g, info, pos, nrm, flux, fmt);
        VPL_LAUNCHED(ex);
    }
    if (report) VPL_TRY(cudaMemcpyAsync(report, info, sizeof(GenInfoDev), cudaMemcpyDeviceToDevice, ex.stream));
    return cudaSuccess;
}

// Direct term L_e(y) of Eq. 1 as light-sample VPLs: sample k is the point of
// the square light at Philox (seed, stream 4) counter (k, 0) words 0 and 1,
// with the light's normal and power P / n; tag -1 - k.  Gathered like the
// indirect VPLs, n of them estimate the light's one-sided Lambertian emission
// reflected at each pixel.
__global__ void light_vpls_kernel(LightView L, int n, uint64_t seed, float4 *pos, void *nrm, void *flux, int fmt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint64_t w[4];
    rng4(seed, kStreamDirect, (uint64_t)k, 0, w);
    const D3 y = light_point(L, u01(w[0]), u01(w[1]));
    store_vpl(pos, nrm, flux, k, make_float3((float)y.x, (float)y.y, (float)y.z), -1,
              make_float3(L.normal[0], L.normal[1], L.normal[2]), -1 - k,
              make_float3((float)((double)L.power[0] / n), (float)((double)L.power[1] / n),
                          (float)((double)L.power[2] / n)),
              fmt);
}

cudaError_t light_vpls(const Exec &ex, const LightView &L, int n, uint64_t seed, float4 *pos, void *nrm, void *flux,
                       int fmt)
{
    if (n <= 0) return cudaSuccess;
    light_vpls_kernel<<<grid_for(n, 256), 256, 0, ex.stream>>>(L, n, seed, pos, nrm, flux, fmt);
    VPL_LAUNCHED(ex);
    return cudaSuccess;
}

cudaError_t generate_vpls(const Exec &ex, const SceneView &s, const GenArgs &g, float4 *pos, void *nrm,
                          void *flux, int fmt, GenInfoDev *report)
{
    const int T = s.n_tris;
    const int TB = kGenThreads;
    // the kernels below read back what earlier ones wrote here, so each call
    // has its own record (calls on other streams may run at the same time);
    // it is copied to `report` at the end
    Tmp rec;
    VPL_TRY(rec.alloc(ex, sizeof(GenInfoDev)));
    GenInfoDev *info = rec.as<GenInfoDev>();
    VPL_TRY(cudaMemsetAsync(info, 0, sizeof(GenInfoDev), ex.stream));
    Tmp flag, fpos;
    VPL_TRY(flag.alloc(ex, sizeof(uint32_t) * T));
    VPL_TRY(fpos.alloc(ex, sizeof(uint32_t) * (T + 1)));
    classify_kernel<<<grid_for(T, TB), TB, 0, ex.stream>>>(s, g, flag.as<uint32_t>());
    VPL_LAUNCHED(ex);
    VPL_TRY(exclusive_scan<uint32_t>(ex, flag.as<uint32_t>(), fpos.as<uint32_t>(), nullptr, T));
    const int *n_close = reinterpret_cast<const int *>(fpos.as<uint32_t>() + T);

    if (g.m_close > 0) {
        Tmp list, keys, vals, area, amax, q, F;
        VPL_TRY(list.alloc(ex, sizeof(uint32_t) * T));
        VPL_TRY(keys.alloc(ex, sizeof(uint64_t) * T));
        VPL_TRY(vals.alloc(ex, sizeof(uint32_t) * T));
        VPL_TRY(area.alloc(ex, sizeof(double) * T));
        VPL_TRY(amax.alloc(ex, sizeof(unsigned long long)));
        VPL_TRY(q.alloc(ex, sizeof(unsigned long long) * T));
        VPL_TRY(F.alloc(ex, sizeof(unsigned long long) * (T + 1)));
        VPL_TRY(cudaMemsetAsync(amax.p, 0, sizeof(unsigned long long), ex.stream));
        compact_kernel<<<grid_for(T, 256), 256, 0, ex.stream>>>(T, flag.as<uint32_t>(), fpos.as<uint32_t>(),
                                                                list.as<uint32_t>());
        VPL_LAUNCHED(ex);
        close_keys_kernel<<<grid_for(T, TB), TB, 0, ex.stream>>>(s, s.gbox, list.as<uint32_t>(), n_close,
                                                                 keys.as<uint64_t>(), vals.as<uint32_t>());
        VPL_LAUNCHED(ex);
        VPL_TRY(radix_sort_pairs(ex, keys.as<uint64_t>(), vals.as<uint32_t>(), n_close, T));
        area_kernel<<<grid_for(T, TB), TB, 0, ex.stream>>>(s, vals.as<uint32_t>(), n_close, area.as<double>(),
                                                           amax.as<unsigned long long>());
        VPL_LAUNCHED(ex);
        quant_kernel<<<grid_for(T, 256), 256, 0, ex.stream>>>(area.as<double>(), n_close,
                                                              amax.as<unsigned long long>(),
                                                              q.as<unsigned long long>(), info);
        VPL_LAUNCHED(ex);
        VPL_TRY(exclusive_scan<unsigned long long>(ex, q.as<unsigned long long>(), F.as<unsigned long long>(),
                                                   n_close, T));
        close_info_kernel<<<1, 1, 0, ex.stream>>>(n_close, F.as<unsigned long long>(), info);
        VPL_LAUNCHED(ex);
        patch_kernel<<<grid_for(g.m_close, TB), TB, 0, ex.stream>>>(s, g, vals.as<uint32_t>(),
                                                                    F.as<unsigned long long>(), n_close, info, pos,
                                                                    nrm, flux, fmt, ex.status);
        VPL_LAUNCHED(ex);
    } else {
        Tmp F0;
        VPL_TRY(F0.alloc(ex, sizeof(unsigned long long) * (T + 1)));
        VPL_TRY(cudaMemsetAsync(F0.p, 0, sizeof(unsigned long long) * (T + 1), ex.stream));
        close_info_kernel<<<1, 1, 0, ex.stream>>>(n_close, F0.as<unsigned long long>(), info);
        VPL_LAUNCHED(ex);
    }

    if (g.m_far > 0) {
        const int64_t n_paths = g.max_paths;
        const int64_t n_slots = n_paths * g.max_bounces;
        Tmp cp, cn, ct, cv, rk;
        VPL_TRY(cp.alloc(ex, sizeof(float4) * n_slots));
        VPL_TRY(cn.alloc(ex, sizeof(float4) * n_slots));
        VPL_TRY(ct.alloc(ex, sizeof(double) * 3 * n_slots));
        VPL_TRY(cv.alloc(ex, sizeof(uint32_t) * n_slots));
        VPL_TRY(rk.alloc(ex, sizeof(uint32_t) * (n_slots + 1)));
        ir_walk_kernel<<<grid_for(n_paths, TB), TB, 0, ex.stream>>>(s, g, flag.as<uint32_t>(), n_paths,
                                                                    cp.as<float4>(), cn.as<float4>(), ct.as<double>(),
                                                                    cv.as<uint32_t>(), ex.status);
        VPL_LAUNCHED(ex);
        VPL_TRY(exclusive_scan<uint32_t>(ex, cv.as<uint32_t>(), rk.as<uint32_t>(), nullptr, n_slots));
        ir_paths_kernel<<<grid_for(n_slots, 256), 256, 0, ex.stream>>>(cv.as<uint32_t>(), rk.as<uint32_t>(), n_slots,
                                                                       g.max_bounces, g.m_far, n_paths, info,
                                                                       ex.status);
        VPL_LAUNCHED(ex);
        ir_emit_kernel<<<grid_for(n_slots, 256), 256, 0, ex.stream>>>(g, cp.as<float4>(), cn.as<float4>(),
                                                                      ct.as<double>(), cv.as<uint32_t>(),
                                                                      rk.as<uint32_t>(), n_slots, info, pos, nrm,
                                                                      flux, fmt);
        VPL_LAUNCHED(ex);
        far_tail_kernel<<<grid_for(g.m_far, 256), 256, 0, ex.stream>>>(g, info, pos, nrm, flux, fmt);
        VPL_LAUNCHED(ex);
    }
    if (report) VPL_TRY(cudaMemcpyAsync(report, info, sizeof(GenInfoDev), cudaMemcpyDeviceToDevice, ex.stream));
    return cudaSuccess;
}

} // namespace vpl
