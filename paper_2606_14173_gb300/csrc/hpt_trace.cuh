#pragma once
// Persistent wave-path-tracing kernel for sm_103a (template; instantiated per variant).
//
// One thread owns one (job, wavelength, pixel) work item at a time and loops over its N
// coherent samples; each loop iteration traces exactly one ray (coherent segment, NEE shadow
// ray or BSDF bounce) so that the warp's lanes traverse the BVH together whatever stage their
// own path is in.  Lanes that finish an item fetch the next one with one warp-aggregated
// atomic.  Accumulators of the K holograms (Kahan-compensated complex sums, Eq. 5) live in
// shared memory; the traversal stack too.
//
// Stages follow Sec. 4 of the paper (s1 cone sampling, s2 world transform of Eq. 3, s3
// tracing, s4 delta / non-delta lobe selection, s5 incoherent radiance of Eq. 1, s6-s7 the
// virtual image point and its distance, s8 facet phase, s9 Path-Reuse accumulation).
#include <cstdint>
#include <cfloat>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "hpt_internal.h"
#include "hpt_real.cuh"

namespace hpt {

#define INC_OFFSET 1e-7f        // incoherent origin offset along the geometric normal (m)
#define COH_TMIN 1e-9           // coherent continuation minimum distance (m)
#define SHADOW_SHRINK 1e-5f
#define NEAR_MARGIN 1e-4f       // barycentric band treated as "near an edge" on coherent rays
#define TIE_REL 2e-6f           // relative distance band treated as a tie on coherent rays
#define WATERTIGHT_EPS 2e-5f    // barycentric slack of float tests on incoherent rays
#define PI_F 3.14159265358979f
#define INV_PI_F 0.318309886183791f

// ------------------------------------------------------------------------------ small math
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return a * rsqrtf(dot3(a, a)); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

template <class R> struct R3 {
    R x, y, z;
};
template <class R> __device__ __forceinline__ R3<R> neg(R3<R> a) { R3<R> v; v.x = -a.x; v.y = -a.y; v.z = -a.z; return v; }
template <class R> __device__ __forceinline__ R3<R> r3(R x, R y, R z) { R3<R> v; v.x = x; v.y = y; v.z = z; return v; }
template <class R> __device__ __forceinline__ R3<R> operator+(R3<R> a, R3<R> b) { return r3<R>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class R> __device__ __forceinline__ R3<R> operator-(R3<R> a, R3<R> b) { return r3<R>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class R> __device__ __forceinline__ R3<R> scale(R3<R> a, R s) { return r3<R>(a.x * s, a.y * s, a.z * s); }
template <class R> __device__ __forceinline__ R rdot(R3<R> a, R3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> __device__ __forceinline__ float3 tof3(R3<R> a)
{
    return f3(RealOps<R>::to_f(a.x), RealOps<R>::to_f(a.y), RealOps<R>::to_f(a.z));
}
template <class R> __device__ __forceinline__ R3<R> fromf3(float3 a)
{
    return r3<R>(RealOps<R>::f(a.x), RealOps<R>::f(a.y), RealOps<R>::f(a.z));
}

// ------------------------------------------------------------------- Philox4x32-10 (SC'11)
__device__ __forceinline__ uint4 philox(uint4 c, unsigned k0, unsigned k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
__device__ __forceinline__ float u24(unsigned x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// path draws: counter (pixel, sample, vertex<<8 | group, lambda<<16 | 0xFFFF)
__device__ __forceinline__ float4 path_draw(const DevJob &J, unsigned pix, unsigned s, unsigned v, unsigned g, unsigned lam)
{
    uint4 o = philox(make_uint4(pix, s, (v << 8) | g, (lam << 16) | 0xFFFFu), J.seed_lo, J.seed_hi);
    return make_float4(u24(o.x), u24(o.y), u24(o.z), u24(o.w));
}

// ------------------------------------------------------------------------------- traversal
struct HitF {
    float t, u, v;
    int tri;
};

struct Counters {
    unsigned rays, boxes, tris, refines, fallbacks, shadows, bounces, samples;
};

// Closest (or any) hit of a float ray against the BVH.  TRACK: record in t_near the smallest
// distance of a triangle met within NEAR_MARGIN of an edge, or of two hits tied within TIE_REL,
// so that the caller can re-decide the hit in double precision.
template <bool STATS>
__device__ __forceinline__ bool traverse(const DevScene &sc, float3 o, float3 d, float tmax, int skip, float eps_w,
                                         bool TRACK, bool ANYHIT, HitF &h, float &t_near, int *stk, int &status,
                                         Counters &cnt)
{
    const float big = 1e30f;
    float3 inv = f3(fabsf(d.x) > 1e-20f ? 1.0f / d.x : copysignf(1e20f, d.x),
                    fabsf(d.y) > 1e-20f ? 1.0f / d.y : copysignf(1e20f, d.y),
                    fabsf(d.z) > 1e-20f ? 1.0f / d.z : copysignf(1e20f, d.z));
    float3 ood = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    h.t = tmax;
    h.tri = -1;
    h.u = h.v = 0.0f;
    if (TRACK) t_near = big;
    const float cull = TRACK ? (1.0f + 4.0f * TIE_REL) : 1.0f;
    const float4 *__restrict__ nodes = sc.nodes;
    const float4 *__restrict__ tris = sc.tri4;
    int sp = 0;
    int node = 0;
    for (;;) {
        // descend inner nodes
        while (node >= 0) {
            const float4 *np = nodes + 4 * node;
            float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
            float tl = h.t * cull;
            float a0 = n0.x * inv.x - ood.x, b0 = n0.y * inv.x - ood.x;
            float a1 = n0.z * inv.y - ood.y, b1 = n0.w * inv.y - ood.y;
            float a2 = n2.x * inv.z - ood.z, b2 = n2.y * inv.z - ood.z;
            float c0min = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), 0.0f));
            float c0max = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), tl));
            float e0 = n1.x * inv.x - ood.x, f0 = n1.y * inv.x - ood.x;
            float e1 = n1.z * inv.y - ood.y, f1 = n1.w * inv.y - ood.y;
            float e2 = n2.z * inv.z - ood.z, f2 = n2.w * inv.z - ood.z;
            float c1min = fmaxf(fmaxf(fminf(e0, f0), fminf(e1, f1)), fmaxf(fminf(e2, f2), 0.0f));
            float c1max = fminf(fminf(fmaxf(e0, f0), fmaxf(e1, f1)), fminf(fmaxf(e2, f2), tl));
            if (STATS) cnt.boxes += 2;
            bool h0 = c0min <= c0max, h1 = c1min <= c1max;
            int l0 = __float_as_int(n3.x), l1 = __float_as_int(n3.y);
            if (!h0 && !h1) {
                if (sp == 0) return h.tri >= 0;
                node = stk[(--sp) * BLOCK];
            } else {
                node = h0 ? l0 : l1;
                if (h0 && h1) {
                    int other = l1;
                    if (c1min < c0min) { node = l1; other = l0; }
                    if (sp < STACK) stk[(sp++) * BLOCK] = other;
                    else status |= ST_STACK_OVERFLOW;
                }
            }
        }
        // leaf: ~(start << 8 | count)
        int code = ~node;
        int start = code >> 8, count = code & 255;
        for (int i = start; i < start + count; ++i) {
            const float4 *tp = tris + 3 * i;
            float4 A = __ldg(tp), E1 = __ldg(tp + 1), E2 = __ldg(tp + 2);
            int id = __float_as_int(A.w);
            if (STATS) cnt.tris++;
            if (id == skip) continue;
            float3 e1 = xyz(E1), e2 = xyz(E2);
            float3 pv = cross3(d, e2);
            float det = dot3(e1, pv);
            float idet = __frcp_rn(det);
            float3 tv = o - xyz(A);
            float u = dot3(tv, pv) * idet;
            float3 qv = cross3(tv, e1);
            float v = dot3(d, qv) * idet;
            float t = dot3(e2, qv) * idet;
            if (TRACK) {
                float m = fminf(fminf(u, v), 1.0f - u - v);
                if (fabsf(m) < NEAR_MARGIN && t > 0.0f && t < t_near) t_near = t;
            }
            bool inside = (u >= -eps_w) && (v >= -eps_w) && (u + v <= 1.0f + eps_w) && (t > 0.0f);
            if (!inside) continue;
            if (ANYHIT) {
                if (t < tmax) { h.t = t; h.tri = id; return true; }
                continue;
            }
            if (TRACK && h.tri >= 0 && fabsf(t - h.t) <= TIE_REL * h.t) t_near = fminf(t_near, fmaxf(t, h.t));
            if (t < h.t || (t == h.t && id < h.tri)) {
                h.t = t; h.u = u; h.v = v; h.tri = id;
            }
        }
        if (sp == 0) break;
        node = stk[(--sp) * BLOCK];
    }
    return h.tri >= 0;
}

// Double-precision closest hit used when the float traversal of a coherent ray was not
// conclusive.  Exact triangle edges (from the float32 vertices), Moller-Trumbore in double,
// ties to the lower triangle id -- the decision rule of the definition.
static __device__ __noinline__ int traverse_fp64(const DevScene &sc, double ox, double oy, double oz, double dx, double dy,
                                          double dz, double tmin, int skip, double *t_out, int *stk, int &status)
{
    double ix = fabs(dx) > 1e-300 ? 1.0 / dx : 1e300, iy = fabs(dy) > 1e-300 ? 1.0 / dy : 1e300,
           iz = fabs(dz) > 1e-300 ? 1.0 / dz : 1e300;
    double best = 1e300;
    int best_id = -1;
    int sp = 0, node = 0;
    for (;;) {
        while (node >= 0) {
            const float4 *np = sc.nodes + 4 * node;
            float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
            double lo0[3] = {n0.x, n0.z, n2.x}, hi0[3] = {n0.y, n0.w, n2.y};
            double lo1[3] = {n1.x, n1.z, n2.z}, hi1[3] = {n1.y, n1.w, n2.w};
            double o[3] = {ox, oy, oz}, iv[3] = {ix, iy, iz};
            double t0a = 0.0, t0b = best * (1.0 + 1e-9), t1a = 0.0, t1b = best * (1.0 + 1e-9);
            for (int k = 0; k < 3; ++k) {
                double a = (lo0[k] - o[k]) * iv[k], b = (hi0[k] - o[k]) * iv[k];
                t0a = fmax(t0a, fmin(a, b)); t0b = fmin(t0b, fmax(a, b));
                a = (lo1[k] - o[k]) * iv[k]; b = (hi1[k] - o[k]) * iv[k];
                t1a = fmax(t1a, fmin(a, b)); t1b = fmin(t1b, fmax(a, b));
            }
            bool h0 = t0a <= t0b, h1 = t1a <= t1b;
            int l0 = __float_as_int(n3.x), l1 = __float_as_int(n3.y);
            if (!h0 && !h1) {
                if (sp == 0) { *t_out = best; return best_id; }
                node = stk[(--sp) * BLOCK];
            } else {
                node = h0 ? l0 : l1;
                if (h0 && h1) {
                    int other = l1;
                    if (t1a < t0a) { node = l1; other = l0; }
                    if (sp < STACK) stk[(sp++) * BLOCK] = other;
                    else status |= ST_FALLBACK_STACK;
                }
            }
        }
        int code = ~node;
        int start = code >> 8, count = code & 255;
        for (int i = start; i < start + count; ++i) {
            int id = __float_as_int(__ldg(sc.tri4 + 3 * i).w);
            if (id == skip) continue;
            uint4 ix4 = __ldg(sc.tri_attr + id);
            const float *p0 = sc.verts + 3 * ix4.x, *p1 = sc.verts + 3 * ix4.y, *p2 = sc.verts + 3 * ix4.z;
            double v0x = p0[0], v0y = p0[1], v0z = p0[2];
            double e1x = (double)p1[0] - v0x, e1y = (double)p1[1] - v0y, e1z = (double)p1[2] - v0z;
            double e2x = (double)p2[0] - v0x, e2y = (double)p2[1] - v0y, e2z = (double)p2[2] - v0z;
            double px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
            double det = e1x * px + e1y * py + e1z * pz;
            if (det == 0.0) continue;
            double id_ = 1.0 / det;
            double tx = ox - v0x, ty = oy - v0y, tz = oz - v0z;
            double u = (tx * px + ty * py + tz * pz) * id_;
            double qx = ty * e1z - tz * e1y, qy = tz * e1x - tx * e1z, qz = tx * e1y - ty * e1x;
            double v = (dx * qx + dy * qy + dz * qz) * id_;
            double t = (e2x * qx + e2y * qy + e2z * qz) * id_;
            if (u < 0.0 || v < 0.0 || u + v > 1.0 || !(t > tmin)) continue;
            if (t < best || (t == best && id < best_id)) { best = t; best_id = id; }
        }
        if (sp == 0) break;
        node = stk[(--sp) * BLOCK];
    }
    *t_out = best;
    return best_id;
}

// ------------------------------------------------------------------------ surface and BSDFs
struct Surf {
    float3 p, ng, ns;   // point, unit geometric normal (winding), unit shading normal
    float u, v;         // texture coordinates
    int tri, mat;
};

__device__ __forceinline__ Surf make_surf(const DevScene &sc, int tri, float3 p, float b1, float b2)
{
    Surf S;
    uint4 ix = __ldg(sc.tri_attr + tri);
    S.p = p;
    S.tri = tri;
    S.mat = (int)ix.w;
    S.ng = xyz(__ldg(sc.tri_ng + tri));
    float b0 = 1.0f - b1 - b2;
    const float *n0 = sc.normals + 3 * ix.x, *n1 = sc.normals + 3 * ix.y, *n2 = sc.normals + 3 * ix.z;
    float3 n = f3(b0 * n0[0] + b1 * n1[0] + b2 * n2[0], b0 * n0[1] + b1 * n1[1] + b2 * n2[1],
                  b0 * n0[2] + b1 * n1[2] + b2 * n2[2]);
    S.ns = normalize3(n);
    const float *t0 = sc.uvs + 2 * ix.x, *t1 = sc.uvs + 2 * ix.y, *t2 = sc.uvs + 2 * ix.z;
    S.u = b0 * t0[0] + b1 * t1[0] + b2 * t2[0];
    S.v = b0 * t0[1] + b1 * t1[1] + b2 * t2[1];
    return S;
}

__device__ __forceinline__ float tex_lookup(const DevScene &sc, int tex, float u, float v, int ch)
{
    int off = __ldg(sc.tex_info + 3 * tex), w = __ldg(sc.tex_info + 3 * tex + 1), hgt = __ldg(sc.tex_info + 3 * tex + 2);
    float x = u * (float)w - 0.5f, y = v * (float)hgt - 0.5f;
    float fx0 = floorf(x), fy0 = floorf(y);
    float fx = x - fx0, fy = y - fy0;
    int x0 = (int)fx0, y0 = (int)fy0, x1 = x0 + 1, y1 = y0 + 1;
    x0 = min(max(x0, 0), w - 1); x1 = min(max(x1, 0), w - 1);
    y0 = min(max(y0, 0), hgt - 1); y1 = min(max(y1, 0), hgt - 1);
    const float *d = sc.tex + off;
    float a = __ldg(d + (y0 * w + x0) * 3 + ch), b = __ldg(d + (y0 * w + x1) * 3 + ch);
    float c = __ldg(d + (y1 * w + x0) * 3 + ch), e = __ldg(d + (y1 * w + x1) * 3 + ch);
    return (a * (1.0f - fx) + b * fx) * (1.0f - fy) + (c * (1.0f - fx) + e * fx) * fy;
}

__device__ __forceinline__ float albedo_of(const DevScene &sc, const MatDev &M, const Surf &S, int ch)
{
    float a = M.albedo[ch];
    return M.tex >= 0 ? a * tex_lookup(sc, M.tex, S.u, S.v, ch) : a;
}

__device__ __forceinline__ float emitted(const DevScene &sc, const MatDev &M, const Surf &S, float3 wo, int ch)
{
    float Le = M.Le[ch];
    if (Le == 0.0f || dot3(wo, S.ng) <= 0.0f) return 0.0f;
    if (M.emit_tex && M.tex >= 0) Le *= tex_lookup(sc, M.tex, S.u, S.v, ch);
    return Le;
}

__device__ __forceinline__ float cache_lookup(const DevScene &sc, float3 p, int ch)
{
    int R = sc.cache_res;
    float g[3] = {p.x, p.y, p.z}, f[3];
    int i0[3], i1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float lo = sc.cache_bmin[k], hi = sc.cache_bmax[k];
        float gg = (g[k] - lo) / (hi - lo) * (float)R - 0.5f;
        float fl = floorf(gg);
        f[k] = gg - fl;
        int a = (int)fl, b = a + 1;
        i0[k] = min(max(a, 0), R - 1);
        i1[k] = min(max(b, 0), R - 1);
    }
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
        float w = ((c & 1) ? f[0] : 1.0f - f[0]) * ((c & 2) ? f[1] : 1.0f - f[1]) * ((c & 4) ? f[2] : 1.0f - f[2]);
        unsigned short hb = __ldg(sc.cache + (((size_t)iz * R + iy) * R + ix) * 3 + ch);
        acc += w * __half2float(__ushort_as_half(hb));
    }
    return acc;
}

// orthonormal basis around a unit normal (Duff et al., JCGT 2017)
__device__ __forceinline__ void make_frame(float3 n, float3 &t, float3 &b)
{
    float sg = n.z >= 0.0f ? 1.0f : -1.0f;
    float a = -1.0f / (sg + n.z);
    float c = n.x * n.y * a;
    t = f3(1.0f + sg * n.x * n.x * a, sg * c, -sg * n.x);
    b = f3(c, sg + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float fresnel_dielectric(float ci, float n_i, float n_t)
{
    float eta = n_i / n_t;
    float s2 = eta * eta * (1.0f - ci * ci);
    if (s2 >= 1.0f) return 1.0f;
    float ct = sqrtf(1.0f - s2);
    float rs = (n_i * ci - n_t * ct) / (n_i * ci + n_t * ct);
    float rp = (n_t * ci - n_i * ct) / (n_t * ci + n_i * ct);
    return 0.5f * (rs * rs + rp * rp);
}

__device__ __forceinline__ float ggx_D(float a, float3 h)
{
    if (h.z <= 0.0f) return 0.0f;
    float a2 = a * a;
    float q = (h.x * h.x + h.y * h.y) / a2 + h.z * h.z;
    return 1.0f / (PI_F * a2 * q * q);
}
__device__ __forceinline__ float ggx_G1(float a, float3 w)
{
    if (w.z <= 0.0f) return 0.0f;
    float t2 = (w.x * w.x + w.y * w.y) / (w.z * w.z);
    float lam = 0.5f * (-1.0f + sqrtf(1.0f + a * a * t2));
    return 1.0f / (1.0f + lam);
}
__device__ __forceinline__ float schlick(float F0, float c)
{
    float m = 1.0f - c;
    float m2 = m * m;
    return F0 + (1.0f - F0) * m2 * m2 * m;
}

// BSDF value and sampling pdf of a non-delta material (world-frame directions)
__device__ __forceinline__ void bsdf_eval(const DevScene &sc, const MatDev &M, const Surf &S, float3 ns, float3 wo,
                                          float3 wi, int ch, float &f, float &pdf)
{
    f = 0.0f;
    pdf = 0.0f;
    float a = albedo_of(sc, M, S, ch);
    if (M.kind == 0) {
        float c = dot3(wi, ns);
        if (c <= 0.0f) return;
        f = a * INV_PI_F;
        pdf = c * INV_PI_F;
    } else if (M.kind == 1) {
        float3 t, b;
        make_frame(ns, t, b);
        float3 lo = f3(dot3(wo, t), dot3(wo, b), dot3(wo, ns));
        float3 li = f3(dot3(wi, t), dot3(wi, b), dot3(wi, ns));
        if (lo.z <= 0.0f || li.z <= 0.0f) return;
        float al = M.rough * M.rough;
        float3 h = normalize3(lo + li);
        float D = ggx_D(al, h);
        float G1o = ggx_G1(al, lo), G1i = ggx_G1(al, li);
        float F = schlick(a, dot3(li, h));
        f = F * D * G1o * G1i / (4.0f * lo.z * li.z);
        pdf = G1o * D / (4.0f * lo.z);
    }
}

// ----------------------------------------------------------------------------- lane state
enum : int { S_NEED_ITEM = 0, S_COH = 1, S_SHADOW = 2, S_BOUNCE = 3, S_DONE = 4 };

template <class R> struct Lane {
    // work item
    const DevJob *J;
    int lam, ch, px, py, s;
    unsigned pix;
    int state;
    // coherent chain (s3, s4): origin, direction, optical path length, medium index
    R3<R> co, cd;
    R opl;
    float n_cur, beta_c, cos_t;
    int cv;
    // at the real image point P (s5-s8)
    bool hasP;
    float f_turns, base_pre;
    int cell[3];
    // incoherent path (Eq. 1)
    float L, beta, prev_pdf, t_prev;
    int v;
    bool prev_delta, inc_first;
    float nee_val;
    bool has_bounce;
    float3 bdir, borg;
    float b_beta, b_pdf;
    int bskip;
    // ray in flight
    float3 ro, rd;
    float rtmax;
    int rskip;
    // surface waiting for vertex processing
    Surf surf;
    float3 wo;
};

// what the main loop does next with a lane
enum : int { A_COH = 0, A_SHADOW = 1, A_BOUNCE = 2, A_VERTEX = 3, A_FINISH = 4 };

// s1 + s2: pixel centre, uniform direction in the cone theta <= asin(lambda / 2p), world space
template <class R> __device__ __forceinline__ void start_sample(Lane<R> &st)
{
    using RO = RealOps<R>;
    const DevJob &J = *st.J;
    float4 u = path_draw(J, st.pix, (unsigned)st.s, 0u, 0u, (unsigned)st.lam);
    R x = RO::mulf(RO::rc(J.pitch), (float)st.px + 0.5f - 0.5f * (float)J.W);
    R y = RO::mulf(RO::rc(J.pitch), (float)st.py + 0.5f - 0.5f * (float)J.H);
    R s1 = RO::mulf(RO::rc(J.h_cone[st.lam]), u.x);          // 1 - cos(theta)
    R ct = RO::f(1.0f) - s1;
    R sn = RO::sqrt_(s1 * (RO::f(2.0f) - s1));
    R sp, cp;
    RO::sincos2pi(u.y, J.sincos_tab, sp, cp);
    R3<R> dh = r3<R>(sn * cp, sn * sp, ct);
    st.cos_t = RO::to_f(ct);
    if (J.t_identity) {
        st.co = r3<R>(x, y, RO::f(0.0f));
        st.cd = dh;
    } else {
        // T = [Rm | t]: world origin = Rm^T (x - t), world direction = Rm^T d
        R qx = x - RO::rc(J.t[0]), qy = y - RO::rc(J.t[1]), qz = -RO::rc(J.t[2]);
        R3<R> c0 = r3<R>(RO::rc(J.R[0]), RO::rc(J.R[3]), RO::rc(J.R[6]));
        R3<R> c1 = r3<R>(RO::rc(J.R[1]), RO::rc(J.R[4]), RO::rc(J.R[7]));
        R3<R> c2 = r3<R>(RO::rc(J.R[2]), RO::rc(J.R[5]), RO::rc(J.R[8]));
        R3<R> q = r3<R>(qx, qy, qz);
        st.co = r3<R>(rdot(c0, q), rdot(c1, q), rdot(c2, q));
        st.cd = r3<R>(rdot(c0, dh), rdot(c1, dh), rdot(c2, dh));
    }
    st.opl = RO::f(0.0f);
    st.n_cur = 1.0f;
    st.beta_c = 1.0f;
    st.cv = 0;
    st.hasP = false;
    st.L = 0.0f;
    st.ro = tof3(st.co);
    st.rd = tof3(st.cd);
    st.rskip = -1;
    st.rtmax = 1e30f;
    st.state = S_COH;
}

// deterministic point emitters of the pixel: a e^{i k r} cos(theta) / r inside the cone
template <class R>
__device__ __noinline__ float2 point_field(const DevJob *Jp, int lam, int px, int py, int *stk, int &status)
{
    using RO = RealOps<R>;
    const DevJob &J = *Jp;
    const DevScene &sc = J.sc;
    float2 acc = make_float2(0.0f, 0.0f);
    R x = RO::mulf(RO::rc(J.pitch), (float)px + 0.5f - 0.5f * (float)J.W);
    R y = RO::mulf(RO::rc(J.pitch), (float)py + 0.5f - 0.5f * (float)J.H);
    for (int e = 0; e < sc.n_points; ++e) {
        const double *pe = sc.points + 4 * e;
        R3<R> pw = r3<R>(RO::fromd(pe[0]), RO::fromd(pe[1]), RO::fromd(pe[2]));
        R3<R> q;
        R3<R> O;
        if (J.t_identity) {
            q = r3<R>(pw.x - x, pw.y - y, pw.z);
            O = r3<R>(x, y, RO::f(0.0f));
        } else {
            R3<R> rw0 = r3<R>(RO::rc(J.R[0]), RO::rc(J.R[1]), RO::rc(J.R[2]));
            R3<R> rw1 = r3<R>(RO::rc(J.R[3]), RO::rc(J.R[4]), RO::rc(J.R[5]));
            R3<R> rw2 = r3<R>(RO::rc(J.R[6]), RO::rc(J.R[7]), RO::rc(J.R[8]));
            q = r3<R>(rdot(rw0, pw) + RO::rc(J.t[0]) - x, rdot(rw1, pw) + RO::rc(J.t[1]) - y,
                      rdot(rw2, pw) + RO::rc(J.t[2]));
            R qx = x - RO::rc(J.t[0]), qy = y - RO::rc(J.t[1]), qz = -RO::rc(J.t[2]);
            R3<R> c0 = r3<R>(RO::rc(J.R[0]), RO::rc(J.R[3]), RO::rc(J.R[6]));
            R3<R> c1 = r3<R>(RO::rc(J.R[1]), RO::rc(J.R[4]), RO::rc(J.R[7]));
            R3<R> c2 = r3<R>(RO::rc(J.R[2]), RO::rc(J.R[5]), RO::rc(J.R[8]));
            R3<R> qq = r3<R>(qx, qy, qz);
            O = r3<R>(rdot(c0, qq), rdot(c1, qq), rdot(c2, qq));
        }
        R r = RO::sqrt_(rdot(q, q));
        float rf = RO::to_f(r);
        float ct = RO::to_f(q.z) / rf;
        if (ct < J.cos_max[lam]) continue;
        float3 Of = tof3(O);
        float3 dw = tof3(pw - O);
        float dist = sqrtf(dot3(dw, dw));
        HitF h;
        float tn;
        Counters dummy;
        if (traverse<false>(sc, Of, dw * (1.0f / dist), dist * (1.0f - SHADOW_SHRINK), -1, WATERTIGHT_EPS, false, true,
                            h, tn, stk, status, dummy))
            continue;
        float turns = RO::frac_f(r * RO::rc(J.inv_lambda[lam]));
        float sn, cs;
        sincospif(2.0f * turns, &sn, &cs);
        float a = (float)pe[3] * ct / rf;
        acc.x += a * cs;
        acc.y += a * sn;
    }
    return acc;
}

// s8 + s9: facet phases of the K holograms and the Kahan-compensated Path-Reuse sums (Eq. 5);
// then the next sample, or the output of a finished item.
template <class R, bool STATS>
__device__ __forceinline__ int finish_sample(Lane<R> &st, float *acc, int *stk, int &status, Counters &cnt)
{
    const DevJob &J = *st.J;
    if (STATS) cnt.samples++;
    if (st.hasP && st.L > 0.0f) {
        float base = sqrtf(st.beta_c * st.L) * st.base_pre;
        const int K = J.K, off = J.hologram_offset;
        uint4 ph = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < K) {
                int m = off + j;
                float u = 0.0f;
                if (J.phase_mode == 0) {
                    if (j == 0 || (m & 3) == 0)
                        ph = philox(make_uint4((unsigned)st.cell[0], (unsigned)st.cell[1], (unsigned)st.cell[2],
                                               ((unsigned)st.lam << 16) | ((unsigned)m >> 2)),
                                    J.pseed_lo, J.pseed_hi);
                    unsigned w = (m & 3) == 0 ? ph.x : ((m & 3) == 1 ? ph.y : ((m & 3) == 2 ? ph.z : ph.w));
                    u = u24(w);
                }
                float sn, cs;
                sincospif(2.0f * (st.f_turns + u), &sn, &cs);
                // (1/(i lambda)) folded into base: multiply the phasor by -i
                float xr = base * sn, xi = -base * cs;
                float *a = acc + (j * 4) * BLOCK;
                float yr = xr - a[2 * BLOCK], tr = a[0] + yr;
                a[2 * BLOCK] = (tr - a[0]) - yr;
                a[0] = tr;
                float yi = xi - a[3 * BLOCK], ti = a[BLOCK] + yi;
                a[3 * BLOCK] = (ti - a[BLOCK]) - yi;
                a[BLOCK] = ti;
            }
        }
    }
    st.s++;
    if (st.s < J.spp) {
        start_sample(st);
        return S_COH;
    }
    // item complete: U_m = sum / N (+ point emitters)
    float2 pf = make_float2(0.0f, 0.0f);
    if (J.sc.n_points > 0) pf = point_field<R>(st.J, st.lam, st.px, st.py, stk, status);
    const float inv_n = 1.0f / (float)J.spp;
    for (int j = 0; j < J.K; ++j) {
        const float *a = acc + (j * 4) * BLOCK;
        float re = (a[0] - a[2 * BLOCK]) * inv_n + pf.x;
        float im = (a[BLOCK] - a[3 * BLOCK]) * inv_n + pf.y;
        size_t o = ((size_t)(st.lam * J.K + j) * J.H + st.py) * J.W + st.px;
        J.out[o] = make_float2(re, im);
    }
    return S_NEED_ITEM;
}

// Sets the ray for the stored BSDF continuation.
template <class R> __device__ __forceinline__ void take_bounce(Lane<R> &st)
{
    st.ro = st.borg;
    st.rd = st.bdir;
    st.rtmax = 1e30f;
    st.rskip = st.bskip;
    st.beta = st.b_beta;
    st.prev_pdf = st.b_pdf;
    st.prev_delta = false;
}

// s5: one vertex of the incoherent path: emission (MIS-weighted), then a delta continuation, or
// the ambient cache, or NEE to a rectangular light plus a BSDF-sampled continuation.
template <class R>
__device__ __forceinline__ int vertex(Lane<R> &st)
{
    const Surf &S = st.surf;
    const float3 wo = st.wo;
    const DevJob &J = *st.J;
    const DevScene &sc = J.sc;
    const MatDev M = sc.mats[S.mat];
    const int ch = st.ch;
    float Le = emitted(sc, M, S, wo, ch);
    if (Le > 0.0f) {
        float w = 1.0f;
        if (!st.prev_delta && M.kind == 4 && M.light >= 0 && sc.n_lights > 0) {
            const LightDev &Lt = sc.lights[M.light];
            float cl = dot3(wo, f3(Lt.n[0], Lt.n[1], Lt.n[2]));
            float pl = st.t_prev * st.t_prev / (cl * Lt.area) / (float)sc.n_lights;
            w = st.prev_pdf * st.prev_pdf / (st.prev_pdf * st.prev_pdf + pl * pl);
        }
        st.L += st.beta * Le * w;
    }
    if (M.kind == 4) return A_FINISH;
    float3 ng = S.ng, ns = S.ns;
    const bool front = dot3(wo, ng) > 0.0f;
    const float4 u = path_draw(J, st.pix, (unsigned)st.s, (unsigned)st.v, 0u, (unsigned)st.lam);
    if (M.kind == 2 || M.kind == 3) {
        if (st.v >= J.max_depth) return A_FINISH;
        float3 wi;
        if (M.kind == 2) {
            if (!front) { ng = -ng; ns = -ns; }
            float c = dot3(wo, ns);
            if (c <= 0.0f) return A_FINISH;
            wi = ns * (2.0f * c) - wo;
            if (dot3(wi, ng) <= 0.0f) return A_FINISH;
            st.beta *= albedo_of(sc, M, S, ch);
        } else {
            float n_i = front ? 1.0f : M.ior, n_t = front ? M.ior : 1.0f;
            float3 n = front ? ns : -ns, g = front ? ng : -ng;
            float ci = dot3(wo, n);
            if (ci <= 0.0f) return A_FINISH;
            float F = fresnel_dielectric(ci, n_i, n_t);
            if (u.x < F) {
                wi = n * (2.0f * ci) - wo;
                if (dot3(wi, g) <= 0.0f) return A_FINISH;
            } else {
                float eta = n_i / n_t;
                float ct = sqrtf(fmaxf(0.0f, 1.0f - eta * eta * (1.0f - ci * ci)));
                wi = wo * (-eta) + n * (eta * ci - ct);
                if (dot3(wi, g) >= 0.0f) return A_FINISH;
                st.beta *= eta * eta;
            }
        }
        st.prev_delta = true;
        st.inc_first = false;
        st.ro = S.p + (dot3(wi, S.ng) > 0.0f ? S.ng : -S.ng) * INC_OFFSET;
        st.rd = wi;
        st.rtmax = 1e30f;
        st.rskip = S.tri;
        return A_BOUNCE;
    }
    // non-delta (Lambert, GGX)
    if (!front) { ng = -ng; ns = -ns; }
    if (dot3(wo, ns) <= 0.0f) return A_FINISH;
    if (J.use_cache && sc.cache_res > 0 && !st.inc_first) {
        st.L += st.beta * albedo_of(sc, M, S, ch) * INV_PI_F * cache_lookup(sc, S.p, ch);
        return A_FINISH;
    }
    const float3 org = S.p + ng * INC_OFFSET;
    bool shadow = false;
    float3 wl = f3(0.0f, 0.0f, 1.0f);
    float smax = 0.0f;
    if (sc.n_lights > 0) {
        int li = 0;
        if (sc.n_lights > 1) {
            float4 u2 = path_draw(J, st.pix, (unsigned)st.s, (unsigned)st.v, 1u, (unsigned)st.lam);
            li = min((int)(u2.x * (float)sc.n_lights), sc.n_lights - 1);
        }
        const LightDev &Lt = sc.lights[li];
        float3 y = f3(Lt.corner[0], Lt.corner[1], Lt.corner[2]) + f3(Lt.eu[0], Lt.eu[1], Lt.eu[2]) * u.x +
                   f3(Lt.ev[0], Lt.ev[1], Lt.ev[2]) * u.y;
        float3 dv = y - org;
        float dist = sqrtf(dot3(dv, dv));
        wl = dv * (1.0f / dist);
        float cl = -dot3(wl, f3(Lt.n[0], Lt.n[1], Lt.n[2]));
        float Ll = Lt.Le[ch];
        if (cl > 0.0f && dot3(wl, ng) > 0.0f && dot3(wl, ns) > 0.0f && Ll > 0.0f) {
            float f, pb;
            bsdf_eval(sc, M, S, ns, wo, wl, ch, f, pb);
            float pl = dist * dist / (cl * Lt.area) / (float)sc.n_lights;
            if (f > 0.0f) {
                float wm = st.v < J.max_depth ? pl * pl / (pl * pl + pb * pb) : 1.0f;
                st.nee_val = st.beta * f * dot3(wl, ns) * Ll * wm / pl;
                shadow = true;
                smax = dist * (1.0f - SHADOW_SHRINK);
            }
        }
    }
    st.has_bounce = false;
    if (st.v < J.max_depth) {
        float3 t, b;
        make_frame(ns, t, b);
        float3 wi;
        float weight = 0.0f, pb = 0.0f;
        bool ok = false;
        if (M.kind == 0) {
            float rr = sqrtf(u.z), s_, c_;
            sincospif(2.0f * u.w, &s_, &c_);
            float z = sqrtf(1.0f - u.z);
            wi = t * (rr * c_) + b * (rr * s_) + ns * z;
            ok = dot3(wi, ng) > 0.0f;
            weight = albedo_of(sc, M, S, ch);
            pb = z * INV_PI_F;
        } else {
            float al = M.rough * M.rough;
            float3 lo = f3(dot3(wo, t), dot3(wo, b), dot3(wo, ns));
            if (lo.z > 0.0f) {
                float3 vh = normalize3(f3(al * lo.x, al * lo.y, lo.z));
                float l2 = vh.x * vh.x + vh.y * vh.y;
                float3 T1 = l2 > 0.0f ? f3(-vh.y, vh.x, 0.0f) * rsqrtf(l2) : f3(1.0f, 0.0f, 0.0f);
                float3 T2 = cross3(vh, T1);
                float rr = sqrtf(u.z), s_, c_;
                sincospif(2.0f * u.w, &s_, &c_);
                float t1 = rr * c_, t2 = rr * s_;
                float sm = 0.5f * (1.0f + vh.z);
                t2 = (1.0f - sm) * sqrtf(fmaxf(0.0f, 1.0f - t1 * t1)) + sm * t2;
                float tz = sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
                float3 nh = T1 * t1 + T2 * t2 + vh * tz;
                float3 ne = normalize3(f3(al * nh.x, al * nh.y, fmaxf(0.0f, nh.z)));
                float c = dot3(lo, ne);
                float3 li = ne * (2.0f * c) - lo;
                if (li.z > 0.0f) {
                    float a = albedo_of(sc, M, S, ch);
                    weight = schlick(a, dot3(li, ne)) * ggx_G1(al, li);
                    pb = ggx_G1(al, lo) * ggx_D(al, ne) / (4.0f * lo.z);
                    wi = t * li.x + b * li.y + ns * li.z;
                    ok = dot3(wi, ng) > 0.0f;
                }
            }
        }
        if (ok) {
            st.has_bounce = true;
            st.bdir = wi;
            st.borg = S.p + (dot3(wi, S.ng) > 0.0f ? S.ng : -S.ng) * INC_OFFSET;
            st.b_beta = st.beta * weight;
            st.b_pdf = pb;
            st.bskip = S.tri;
        }
    }
    st.inc_first = false;
    if (shadow) {
        st.ro = org;
        st.rd = wl;
        st.rtmax = smax;
        st.rskip = S.tri;
        return A_SHADOW;
    }
    if (st.has_bounce) {
        take_bounce(st);
        return A_BOUNCE;
    }
    return A_FINISH;
}

// s3 + s4 for a coherent segment: decide the hit (float traversal, double re-decision when not
// conclusive), refine the distance in the coherent arithmetic, then either the real image
// point P (non-delta) or the next delta segment.
template <class R, bool STATS>
__device__ __forceinline__ int coherent_hit(Lane<R> &st, const HitF &hit, float t_near, int *stk, int &status,
                                           Counters &cnt)
{
    using RO = RealOps<R>;
    const DevJob &J = *st.J;
    const DevScene &sc = J.sc;
    int tri = hit.tri;
    if (t_near < 1e29f && (tri < 0 || t_near <= hit.t * (1.0f + 10.0f * TIE_REL))) {
        if (STATS) cnt.fallbacks++;
        double tt;
        tri = traverse_fp64(sc, RO::to_d(st.co.x), RO::to_d(st.co.y), RO::to_d(st.co.z), RO::to_d(st.cd.x),
                            RO::to_d(st.cd.y), RO::to_d(st.cd.z), st.cv > 0 ? COH_TMIN : 0.0, st.rskip, &tt, stk,
                            status);
    }
    if (tri < 0) return A_FINISH;
    if (STATS) cnt.refines++;
    // distance along the ray to the triangle's plane n . x = d0
    const int rb = tri * REF_N;
    R3<R> n = r3<R>(RO::load(sc.ref64, sc.refdf, rb), RO::load(sc.ref64, sc.refdf, rb + 1),
                    RO::load(sc.ref64, sc.refdf, rb + 2));
    R d0 = RO::load(sc.ref64, sc.refdf, rb + 3);
    R t = (d0 - rdot(n, st.co)) / rdot(n, st.cd);
    R3<R> P = st.co + scale(st.cd, t);
    st.opl = st.opl + RO::mulf(t, st.n_cur);     // OPL = sum n_i L_i (Sec. 4.2)
    st.cv++;
    const uint4 ix = __ldg(sc.tri_attr + tri);
    const int kind = sc.mats[ix.w].kind;
    float3 ng = xyz(__ldg(sc.tri_ng + tri));
    const float3 v0 = f3(sc.verts[3 * ix.x], sc.verts[3 * ix.x + 1], sc.verts[3 * ix.x + 2]);
    const R3<R> dP = P - fromf3<R>(v0);
    const float3 dPf = tof3(dP);
    const float3 m1f = f3(RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 4)), RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 5)),
                          RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 6)));
    const float3 m2f = f3(RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 7)), RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 8)),
                          RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 9)));
    st.surf = make_surf(sc, tri, tof3(P), dot3(m1f, dPf), dot3(m2f, dPf));
    const Surf &S = st.surf;
    if (kind != 2 && kind != 3) {
        // P: first non-delta hit = the real image point.  For a rigid T the virtual image point
        // Q = T (O + d_OPL v) lies at distance r = d_OPL from the pixel along the sampled
        // hologram-space direction, so cos(theta) is that direction's z component.
        const float3 dl = tof3(st.cd);
        const float cosP = fabsf(dot3(dl, ng));
        st.f_turns = RO::frac_f(st.opl * RO::rc(J.inv_lambda[st.lam]));
        st.base_pre = st.cos_t * RO::to_f(st.opl) / (J.pdf_w[st.lam] * cosP * J.lambda_f[st.lam]);
        const R ih = RO::rc(J.inv_facet);
        st.cell[0] = RO::floor_i(P.x * ih);
        st.cell[1] = RO::floor_i(P.y * ih);
        st.cell[2] = RO::floor_i(P.z * ih);
        st.hasP = true;
        st.L = 0.0f;
        st.beta = 1.0f;
        st.v = st.cv;
        st.prev_delta = true;
        st.inc_first = true;
        st.prev_pdf = 0.0f;
        st.t_prev = 0.0f;
        st.wo = -dl;
        return A_VERTEX;
    }
    if (st.cv >= J.max_depth) return A_FINISH;
    // delta vertex: interpolated shading normal and the new direction in the coherent arithmetic
    const MatDev M = sc.mats[ix.w];
    R b1 = rdot(r3<R>(RO::load(sc.ref64, sc.refdf, rb + 4), RO::load(sc.ref64, sc.refdf, rb + 5),
                      RO::load(sc.ref64, sc.refdf, rb + 6)), dP);
    R b2 = rdot(r3<R>(RO::load(sc.ref64, sc.refdf, rb + 7), RO::load(sc.ref64, sc.refdf, rb + 8),
                      RO::load(sc.ref64, sc.refdf, rb + 9)), dP);
    R b0 = RO::f(1.0f) - b1 - b2;
    const float *n0 = sc.normals + 3 * ix.x, *n1 = sc.normals + 3 * ix.y, *n2 = sc.normals + 3 * ix.z;
    R3<R> ns = r3<R>(RO::mulf(b0, n0[0]) + RO::mulf(b1, n1[0]) + RO::mulf(b2, n2[0]),
                     RO::mulf(b0, n0[1]) + RO::mulf(b1, n1[1]) + RO::mulf(b2, n2[1]),
                     RO::mulf(b0, n0[2]) + RO::mulf(b1, n1[2]) + RO::mulf(b2, n2[2]));
    ns = scale(ns, RO::f(1.0f) / RO::sqrt_(rdot(ns, ns)));
    const R3<R> wo = neg(st.cd);
    const bool front = dot3(tof3(wo), ng) > 0.0f;
    R3<R> wi;
    if (kind == 2) {
        if (!front) { ns = neg(ns); ng = -ng; }
        R c = rdot(wo, ns);
        if (!(RO::to_f(c) > 0.0f)) return A_FINISH;
        wi = scale(ns, RO::mulf(c, 2.0f)) - wo;
        if (dot3(tof3(wi), ng) <= 0.0f) return A_FINISH;
        st.beta_c *= albedo_of(sc, M, S, st.ch);
    } else {
        const float n_i = front ? 1.0f : M.ior, n_t = front ? M.ior : 1.0f;
        const R3<R> nn = front ? ns : neg(ns);
        const float3 g = front ? ng : -ng;
        R ci = rdot(wo, nn);
        const float cif = RO::to_f(ci);
        if (!(cif > 0.0f)) return A_FINISH;
        const float F = fresnel_dielectric(cif, n_i, n_t);
        const float4 u = path_draw(J, st.pix, (unsigned)st.s, (unsigned)st.cv, 0u, (unsigned)st.lam);
        if (u.x < F) {
            wi = scale(nn, RO::mulf(ci, 2.0f)) - wo;
            if (dot3(tof3(wi), g) <= 0.0f) return A_FINISH;
        } else {
            R eta = RO::f(n_i) / RO::f(n_t);
            R ct = RO::sqrt_(RO::f(1.0f) - eta * eta * (RO::f(1.0f) - ci * ci));
            wi = scale(nn, eta * ci - ct) - scale(wo, eta);
            if (dot3(tof3(wi), g) >= 0.0f) return A_FINISH;
            st.beta_c *= RO::to_f(eta * eta);
            st.n_cur = n_t;
        }
    }
    st.co = P;
    st.cd = wi;
    st.ro = tof3(P);
    st.rd = tof3(wi);
    st.rskip = tri;
    st.rtmax = 1e30f;
    return A_COH;
}

// ------------------------------------------------------------------------------ the kernel
template <class R, bool STATS>
__global__ void __launch_bounds__(BLOCK) trace_kernel(const JobTable *__restrict__ table,
                                                      SlotScratch *__restrict__ scratch)
{
    __shared__ int s_stack[STACK * BLOCK];
    __shared__ float s_acc[KMAX * 4 * BLOCK];
    const int tid = threadIdx.x;
    const int lane_id = tid & 31;
    int *stk = s_stack + tid;
    float *acc = s_acc + tid;    // acc[(m * 4 + c) * BLOCK]: sum re, sum im, comp re, comp im
    const long long total = table->total_items;
    const int n_jobs = table->n_jobs;
    int status = 0;
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    Lane<R> st;
    st.state = S_NEED_ITEM;
    st.J = table->jobs;

    for (;;) {
        // fetch work items: one atomic per warp for all lanes that need one
        const bool need = st.state == S_NEED_ITEM;
        const unsigned want = __ballot_sync(0xFFFFFFFFu, need);
        if (want) {
            const int leader = __ffs(want) - 1;
            unsigned long long base = 0;
            if (lane_id == leader) base = atomicAdd(&scratch->next_item, (unsigned long long)__popc(want));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (need) {
                const long long item = (long long)base + __popc(want & ((1u << lane_id) - 1u));
                if (item >= total) {
                    st.state = S_DONE;
                } else {
                    int j = 0;
                    while (j + 1 < n_jobs && table->jobs[j + 1].item_start <= item) ++j;
                    const DevJob *J = table->jobs + j;
                    const long long loc = item - J->item_start;
                    const long long per_lam = (long long)J->n_tiles * 32;
                    const int lam = (int)(loc / per_lam);
                    const int rem = (int)(loc - (long long)lam * per_lam);
                    const int tile = rem >> 5, l = rem & 31;
                    const int tx = tile % J->n_tiles_x, ty = tile / J->n_tiles_x;
                    const int px = tx * TILE_W + (l & (TILE_W - 1)), py = ty * TILE_H + l / TILE_W;
                    if (px < J->W && py < J->H && lam < J->n_lambda) {
                        st.J = J;
                        st.lam = lam;
                        st.ch = J->channel[lam];
                        st.px = px;
                        st.py = py;
                        st.pix = (unsigned)(py * J->W + px);
                        for (int m = 0; m < KMAX * 4; ++m) acc[m * BLOCK] = 0.0f;
                        st.s = 0;
                        start_sample(st);
                    }
                }
            }
        }
        if (__all_sync(0xFFFFFFFFu, st.state == S_DONE)) break;
        if (st.state == S_NEED_ITEM || st.state == S_DONE) continue;

        // trace exactly one ray per lane
        HitF hit;
        float t_near = 1e30f;
        const bool coh = st.state == S_COH, shadow = st.state == S_SHADOW;
        if (STATS) { cnt.rays++; cnt.shadows += shadow; cnt.bounces += (st.state == S_BOUNCE); }
        const bool any = traverse<STATS>(st.J->sc, st.ro, st.rd, st.rtmax, st.rskip, coh ? 0.0f : WATERTIGHT_EPS, coh,
                                         shadow, hit, t_near, stk, status, cnt);
        int act;
        if (coh) {
            act = coherent_hit<R, STATS>(st, hit, t_near, stk, status, cnt);
        } else if (shadow) {
            if (!any) st.L += st.nee_val;
            act = A_FINISH;
            if (st.has_bounce) {
                take_bounce(st);
                act = A_BOUNCE;
            }
        } else if (hit.tri < 0) {
            act = A_FINISH;
        } else {
            st.v++;
            st.t_prev = hit.t;
            st.surf = make_surf(st.J->sc, hit.tri, st.ro + st.rd * hit.t, hit.u, hit.v);
            st.wo = -st.rd;
            act = A_VERTEX;
        }
        if (act == A_VERTEX) act = vertex(st);
        if (act == A_FINISH) {
            st.state = finish_sample<R, STATS>(st, acc, stk, status, cnt);
        } else {
            st.state = act == A_COH ? S_COH : (act == A_SHADOW ? S_SHADOW : S_BOUNCE);
        }
    }
    if (STATS) {
        unsigned v[8] = {cnt.samples, cnt.rays, cnt.boxes, cnt.tris, cnt.refines, cnt.fallbacks, cnt.shadows, cnt.bounces};
        for (int k = 0; k < 8; ++k) {
            unsigned long long x = v[k];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, off);
            if (lane_id == 0) atomicAdd(&scratch->counters[k], x);
        }
    }
    if (status) atomicOr(&scratch->status, (unsigned)status);
}

}  // namespace hpt
