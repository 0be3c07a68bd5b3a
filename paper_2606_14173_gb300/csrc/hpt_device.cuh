#pragma once
// Device building blocks of the wave path tracer: small vector math, the Philox4x32-10
// counter-based generator, float BVH traversal with near-edge tracking, the double-precision
// re-decision of a coherent hit, surface attributes, textures, the ambient cache and BSDFs.
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
#define WATERTIGHT_EPS 2e-5f    // most barycentric slack of float tests on incoherent rays (per
                                // triangle: a band of 1e-6 x the scene's largest coordinate)
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
// the same products with every rounding spelled out (fixed FMA contraction), so that a result does
// not depend on how the compiler contracts the surrounding code of a given build
__device__ __forceinline__ float dot3_rn(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, __fmul_rn(a.z, b.z))); }
__device__ __forceinline__ float3 cross3_rn(float3 a, float3 b)
{
    return f3(fmaf(a.y, b.z, -__fmul_rn(a.z, b.y)), fmaf(a.z, b.x, -__fmul_rn(a.x, b.z)), fmaf(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
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

// Triangles whose float test was within its error band (near an edge, or tied in distance):
// the closest hit among them is re-decided in the coherent arithmetic.
constexpr int NCAND = 4;
struct Cands {
    float t[NCAND];
    int id[NCAND];
    int n;          // > NCAND: overflow
    __device__ __forceinline__ void add(float tt, int i)
    {
        for (int k = 0; k < NCAND; ++k)
            if (k < n && id[k] == i) return;
        if (n < NCAND) {
            t[n] = tt;
            id[n] = i;
        }
        ++n;
    }
};

struct Counters {
    unsigned rays, boxes, tris, refines, fallbacks, shadows, bounces, samples;
};


#ifndef HPT_NODE_LD256
#define HPT_NODE_LD256 1
#endif
// 32 bytes through the read-only path in one instruction (p 32-byte aligned): a node of the BVH is
// two of them instead of four 16-byte loads, which halves the L1 sector accesses of a node visit
__device__ __forceinline__ void ldg256(const float4 *p, float4 &a, float4 &b)
{
#if HPT_NODE_LD256
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
#else
    a = __ldg(p);
    b = __ldg(p + 1);
#endif
}

// Closest (or any) hit of a float ray against the BVH.  TRACK: collect the triangles met within
// NEAR_MARGIN of an edge, or tied in distance within TIE_REL, no farther than the float winner,
// so that the caller can re-decide the hit in the coherent arithmetic.  The traversal stack has
// slimit entries (stride SSTRIDE); a deeper tree sets ST_STACK_OVERFLOW.

template <bool STATS, int SSTRIDE>
__device__ __forceinline__ bool traverse(const DevScene &sc, float3 o, float3 d, float tmax, int skip, float eps_w,
                                         bool TRACK, bool ANYHIT, HitF &h, Cands &cand, int *stk, int slimit,
                                         int &status, Counters &cnt, bool primary = false)
{
    const float big = 1e30f;
    float3 inv = f3(fabsf(d.x) > 1e-20f ? 1.0f / d.x : copysignf(1e20f, d.x),
                    fabsf(d.y) > 1e-20f ? 1.0f / d.y : copysignf(1e20f, d.y),
                    fabsf(d.z) > 1e-20f ? 1.0f / d.z : copysignf(1e20f, d.z));
    float3 ood = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    h.t = tmax;
    h.tri = -1;
    h.u = h.v = 0.0f;
    (void)big;
    if (TRACK) cand.n = 0;
    const float cull = TRACK ? (1.0f + 4.0f * TIE_REL) : 1.0f;
    // the pixels' first rays walk the tree built for their direction; the closest hit and the
    // candidates do not depend on the tree
    const float4 *__restrict__ nodes = primary ? sc.nodes_p : sc.nodes;
    const float4 *__restrict__ tris = primary ? sc.tri4_p : sc.tri4;
    const int n_nodes = primary ? sc.n_nodes_p : sc.n_nodes, n_tri4 = primary ? sc.n_tri4_p : sc.n_tri4;
    (void)n_nodes;
    (void)n_tri4;
    int sp = 0;
    int node = 0;
    // Speculative descent (Aila and Laine 2009): a leaf met while none is pending is postponed
    // and the descent continues until every active lane of the warp holds a leaf; then the
    // lanes test their leaves together.  Culling uses the closest hit known so far, so only the
    // order of the visits changes: the closest hit (ties to the lower id) is the same, and the
    // candidates of a coherent ray, re-decided exactly, lead to the same decision.
    const int SENT = 0x7FFFFFFF;    // stack exhausted
    int LEAF = 0;                   // pending leaf (< 0); 0 = none (the root is never a leaf)
    for (;;) {
        while (node >= 0 && node != SENT) {
            if (!HPT_IN(node, n_nodes)) {
                status |= ST_BOUNDS;
                node = SENT;
                break;
            }
            float tl = h.t * cull;
            const float4 *np = nodes + 4 * node;
            float4 n0, n1, n2, n3;
            ldg256(np, n0, n1);
            ldg256(np + 2, n2, n3);
            float a0 = n0.x * inv.x - ood.x, b0 = n0.y * inv.x - ood.x;
            float a1 = n0.z * inv.y - ood.y, b1 = n0.w * inv.y - ood.y;
            float a2 = n2.x * inv.z - ood.z, b2 = n2.y * inv.z - ood.z;
            float e0 = n1.x * inv.x - ood.x, f0 = n1.y * inv.x - ood.x;
            float e1 = n1.z * inv.y - ood.y, f1 = n1.w * inv.y - ood.y;
            float e2 = n2.z * inv.z - ood.z, f2 = n2.w * inv.z - ood.z;
            int l0 = __float_as_int(n3.x), l1 = __float_as_int(n3.y);
            float c0min = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), 0.0f));
            float c0max = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), tl));
            float c1min = fmaxf(fmaxf(fminf(e0, f0), fminf(e1, f1)), fmaxf(fminf(e2, f2), 0.0f));
            float c1max = fminf(fminf(fmaxf(e0, f0), fmaxf(e1, f1)), fminf(fmaxf(e2, f2), tl));
            if (STATS) cnt.boxes += 2;
            bool h0 = c0min <= c0max, h1 = c1min <= c1max;
            if (!h0 && !h1) {
                node = sp > 0 ? stk[(--sp) * SSTRIDE] : SENT;
            } else {
                node = h0 ? l0 : l1;
                if (h0 && h1) {
                    int other = l1;
                    if (c1min < c0min) { node = l1; other = l0; }
                    if (sp < slimit) stk[(sp++) * SSTRIDE] = other;
                    else status |= ST_STACK_OVERFLOW;
                }
            }
            if (node < 0 && LEAF == 0) {
                LEAF = node;
                node = sp > 0 ? stk[(--sp) * SSTRIDE] : SENT;
            }
            if (!__any_sync(__activemask(), LEAF == 0)) break;
        }
        while (LEAF < 0) {
            // leaf: ~(start << 8 | count)
            int code = ~LEAF;
            int start = code >> 8, count = code & 255;
            if (count > 0 && !HPT_IN(start + count - 1, n_tri4)) {
                status |= ST_BOUNDS;
                count = 0;
            }
            for (int i = start; i < start + count; ++i) {
                const float4 *tp = tris + 3 * i;
                float4 A = __ldg(tp), E1 = __ldg(tp + 1), E2 = __ldg(tp + 2);
                int id = __float_as_int(A.w);
                if (STATS) cnt.tris++;
                if (id == skip) continue;
                if (!HPT_IN(id, sc.n_tris)) {
                    status |= ST_BOUNDS;
                    continue;
                }
                float3 e1 = xyz(E1), e2 = xyz(E2);
                float3 pv = cross3_rn(d, e2);
                float det = dot3_rn(e1, pv);
                float idet = __fdividef(1.0f, det);
                float3 tv = o - xyz(A);
                float u = __fmul_rn(dot3_rn(tv, pv), idet);
                float3 qv = cross3_rn(tv, e1);
                float v = __fmul_rn(dot3_rn(d, qv), idet);
                float t = __fmul_rn(dot3_rn(e2, qv), idet);
                if (TRACK) {
                    const float m = fminf(fminf(u, v), 1.0f - u - v);
                    if (fabsf(m) < NEAR_MARGIN && t > 0.0f && t <= h.t * (1.0f + 10.0f * TIE_REL)) cand.add(t, id);
                }
                // the slack of a float test closes cracks between neighbours; per triangle it is a
                // band of fixed width in space (E1.w), so that large triangles do not grow far
                // past their outer edges
                const float ew = eps_w > 0.0f ? E1.w : 0.0f;
                bool inside = (u >= -ew) && (v >= -ew) && (u + v <= 1.0f + ew) && (t > 0.0f);
                if (!inside) continue;
                if (ANYHIT) {
                    if (t < tmax) { h.t = t; h.tri = id; return true; }
                    continue;
                }
                if (TRACK && h.tri >= 0 && fabsf(t - h.t) <= TIE_REL * h.t) {
                    cand.add(h.t, h.tri);
                    cand.add(t, id);
                }
                if (t < h.t || (t == h.t && id < h.tri)) {
                    h.t = t; h.u = u; h.v = v; h.tri = id;
                }
            }
            LEAF = 0;
            if (node < 0) {
                LEAF = node;
                node = sp > 0 ? stk[(--sp) * SSTRIDE] : SENT;
            }
        }
        if (node == SENT) break;
    }
    return h.tri >= 0;
}

// Double-precision closest hit used when the float traversal of a coherent ray was not
// conclusive.  Exact triangle edges (from the float32 vertices), Moller-Trumbore in double,
// ties to the lower triangle id -- the decision rule of the definition.
//
// The box tests need not be exact, only conservative: every box the double ray meets at some t
// in [0, best] must be visited, and which boxes are visited changes the work, never the winner.
// They run in float against the boxes widened by w = 2^-17 (|o|_inf + M), M the largest
// coordinate magnitude of the scene's bounds.  For a point X = o + t d inside the bounds, the
// float ray (o and d rounded to float) passes within 2^-24 (|o|_inf + |X - o|_inf) <=
// 2^-24 (2 |o|_inf + M) of X, and the slab arithmetic (the rounded reciprocal, the rounded
// origin products, one FMA) errs by a few units of 2^-24 (|o|_inf + M) in space; w covers both
// with a margin of about 8.  Culling uses the double best rounded up to float with a margin of
// 2^-16.  (GB300 runs float at 64 times the double rate; the boxes are most of the work.)
template <int SSTRIDE>
__device__ __noinline__ int traverse_fp64(const DevScene &sc, double ox, double oy, double oz, double dx, double dy,
                                          double dz, double tmin, int skip, double *t_out, int *stk, int slimit,
                                          int &status)
{
    const float3 of = f3((float)ox, (float)oy, (float)oz);
    const float3 dfl = f3((float)dx, (float)dy, (float)dz);
    float M;
    {
        const float4 r0 = __ldg(sc.nodes), r1 = __ldg(sc.nodes + 1), r2 = __ldg(sc.nodes + 2);
        M = fmaxf(fmaxf(fmaxf(fabsf(r0.x), fabsf(r0.y)), fmaxf(fabsf(r0.z), fabsf(r0.w))),
                  fmaxf(fmaxf(fabsf(r1.x), fabsf(r1.y)), fmaxf(fabsf(r1.z), fabsf(r1.w))));
        M = fmaxf(M, fmaxf(fmaxf(fabsf(r2.x), fabsf(r2.y)), fmaxf(fabsf(r2.z), fabsf(r2.w))));
    }
    const float w = (fmaxf(fmaxf(fabsf(of.x), fabsf(of.y)), fabsf(of.z)) + M) * 0x1p-17f;
    const float3 inv = f3(fabsf(dfl.x) > 1e-20f ? 1.0f / dfl.x : copysignf(1e20f, dfl.x),
                          fabsf(dfl.y) > 1e-20f ? 1.0f / dfl.y : copysignf(1e20f, dfl.y),
                          fabsf(dfl.z) > 1e-20f ? 1.0f / dfl.z : copysignf(1e20f, dfl.z));
    // lower planes moved down by w, upper planes up by w: (lo - w - o) inv = lo inv - (o + w) inv
    const float3 oa = f3((of.x + w) * inv.x, (of.y + w) * inv.y, (of.z + w) * inv.z);
    const float3 ob = f3((of.x - w) * inv.x, (of.y - w) * inv.y, (of.z - w) * inv.z);
    double best = 1e300;
    int best_id = -1;
    float tl = 1e30f;
    int sp = 0, node = 0;
    for (;;) {
        while (node >= 0) {
            if (!HPT_IN(node, sc.n_nodes)) {
                status |= ST_BOUNDS;
                *t_out = best;
                return best_id;
            }
            // 16-byte loads: ptxas of CUDA 13.0 fails on the 32-byte form in this non-inlined function
            const float4 *np = sc.nodes + 4 * node;
            const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
            const float a0 = fmaf(n0.x, inv.x, -oa.x), b0 = fmaf(n0.y, inv.x, -ob.x);
            const float a1 = fmaf(n0.z, inv.y, -oa.y), b1 = fmaf(n0.w, inv.y, -ob.y);
            const float a2 = fmaf(n2.x, inv.z, -oa.z), b2 = fmaf(n2.y, inv.z, -ob.z);
            const float e0 = fmaf(n1.x, inv.x, -oa.x), f0 = fmaf(n1.y, inv.x, -ob.x);
            const float e1 = fmaf(n1.z, inv.y, -oa.y), f1 = fmaf(n1.w, inv.y, -ob.y);
            const float e2 = fmaf(n2.z, inv.z, -oa.z), f2 = fmaf(n2.w, inv.z, -ob.z);
            const int l0 = __float_as_int(n3.x), l1 = __float_as_int(n3.y);
            const float t0a = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), 0.0f));
            const float t0b = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), tl));
            const float t1a = fmaxf(fmaxf(fminf(e0, f0), fminf(e1, f1)), fmaxf(fminf(e2, f2), 0.0f));
            const float t1b = fminf(fminf(fmaxf(e0, f0), fmaxf(e1, f1)), fminf(fmaxf(e2, f2), tl));
            const bool h0 = t0a <= t0b, h1 = t1a <= t1b;
            if (!h0 && !h1) {
                if (sp == 0) { *t_out = best; return best_id; }
                node = stk[(--sp) * SSTRIDE];
            } else {
                node = h0 ? l0 : l1;
                if (h0 && h1) {
                    int other = l1;
                    if (t1a < t0a) { node = l1; other = l0; }
                    if (sp < slimit) stk[(sp++) * SSTRIDE] = other;
                    else status |= ST_FALLBACK_STACK;
                }
            }
        }
        int code = ~node;
        int start = code >> 8, count = code & 255;
        if (count > 0 && !HPT_IN(start + count - 1, sc.n_tri4)) {
            status |= ST_BOUNDS;
            count = 0;
        }
        for (int i = start; i < start + count; ++i) {
            int id = __float_as_int(__ldg(sc.tri4 + 3 * i).w);
            if (id == skip) continue;
            if (!HPT_IN(id, sc.n_tris)) {
                status |= ST_BOUNDS;
                continue;
            }
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
            if (t < best || (t == best && id < best_id)) {
                best = t;
                best_id = id;
                tl = __double2float_ru(best) * (1.0f + 0x1p-16f);
            }
        }
        if (sp == 0) break;
        node = stk[(--sp) * SSTRIDE];
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

// BSDF value and sampling pdf of a non-delta material (world-frame directions); a = albedo
__device__ __forceinline__ void bsdf_eval(const MatDev &M, float a, float3 ns, float3 wo, float3 wi, float &f,
                                          float &pdf)
{
    f = 0.0f;
    pdf = 0.0f;
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

}  // namespace hpt
