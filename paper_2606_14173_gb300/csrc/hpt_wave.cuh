// Wavefront kernels of the wave path tracer (templated on the coherent arithmetic R).
//
// A wave holds the paths of consecutive (wavelength, pixel) work items with all of their N
// samples; path p of a segment is sample s = p / n_items of item p % n_items, so adjacent paths
// belong to adjacent pixels.  Per wave:
//   k_gen                 s1, s2: pixel centre and a direction in the SLM cone, to world space
//   (k_trace, k_shade) x (max_depth + 1)
//     k_trace             s3: closest hit of coherent and incoherent rays, any hit of shadow rays
//                         (float BVH; when the float test of a coherent ray was within its error
//                         band of an edge or a tie, the hit is re-decided among the candidates in
//                         the coherent arithmetic)
//     k_shade             s3-s5: coherent refinement and delta lobes (R arithmetic), the real
//                         image point P, incoherent vertices with NEE and BSDF sampling (Eq. 1)
//   k_accum               s6-s9: per pixel and wavelength, the K facet phases and the
//                         Kahan-compensated Path-Reuse sums (Eq. 5) in sample order
// Queues are compacted with one atomic per warp.  Each path owns its state slots, so the order
// in which queues are filled does not change any result.
#pragma once
#include "hpt_device.cuh"

namespace hpt {

// an 8-byte coherent slot: a double, or a double-float as its two floats' bits
template <class R> struct RS;
template <> struct RS<double> {
    static __device__ __forceinline__ double from(unsigned a, unsigned b) { return __hiloint2double((int)b, (int)a); }
    static __device__ __forceinline__ void to(double v, unsigned &a, unsigned &b)
    {
        a = (unsigned)__double2loint(v);
        b = (unsigned)__double2hiint(v);
    }
};
template <> struct RS<df> {
    static __device__ __forceinline__ df from(unsigned a, unsigned b) { return mkdf(__uint_as_float(a), __uint_as_float(b)); }
    static __device__ __forceinline__ void to(df v, unsigned &a, unsigned &b)
    {
        a = __float_as_uint(v.hi);
        b = __float_as_uint(v.lo);
    }
};

// the coherent state of path p: origin, direction and optical path length
template <class R>
__device__ __forceinline__ void coh_load(const PathBufs &pb, int p, R3<R> &o, R3<R> &d, R &opl)
{
    const uint4 a = pb.cs0[p], b = pb.cs1[p], c = pb.cs2[p];
    const uint2 e = pb.cs3[p];
    o = r3<R>(RS<R>::from(a.x, a.y), RS<R>::from(a.z, a.w), RS<R>::from(b.x, b.y));
    d = r3<R>(RS<R>::from(b.z, b.w), RS<R>::from(c.x, c.y), RS<R>::from(c.z, c.w));
    opl = RS<R>::from(e.x, e.y);
}

template <class R>
__device__ __forceinline__ void coh_store(const PathBufs &pb, int p, const R3<R> &o, const R3<R> &d, R opl)
{
    uint4 a, b, c;
    uint2 e;
    RS<R>::to(o.x, a.x, a.y);
    RS<R>::to(o.y, a.z, a.w);
    RS<R>::to(o.z, b.x, b.y);
    RS<R>::to(d.x, b.z, b.w);
    RS<R>::to(d.y, c.x, c.y);
    RS<R>::to(d.z, c.z, c.w);
    RS<R>::to(opl, e.x, e.y);
    pb.cs0[p] = a;
    pb.cs1[p] = b;
    pb.cs2[p] = c;
    pb.cs3[p] = e;
}

enum : int { VF_V = 0xFF, VF_PREV_DELTA = 1 << 8, VF_INC_FIRST = 1 << 9, VF_HASP = 1 << 10, VF_BAKE = 1 << 11 };
constexpr int Q_FINALIZE = (int)0x80000000;

struct PathId {
    const DevJob *J;
    int lam, ch, px, py, s;
    unsigned pix;
    bool valid;
};

__device__ __forceinline__ int seg_of_path(const WaveDesc &wd, int p)
{
    int k = 0;
    while (k + 1 < wd.n_seg && wd.seg[k + 1].path_offset <= p) ++k;
    return k;
}

__device__ __forceinline__ void decode_item(const DevJob *J, long long item, PathId &id)
{
    const long long per_lam = (long long)J->n_tiles * 32;
    const int lam = (int)(item / per_lam);
    const int rem = (int)(item - (long long)lam * per_lam);
    const int tile = rem >> 5, l = rem & 31;
    const int tx = tile % J->n_tiles_x, ty = tile / J->n_tiles_x;
    id.J = J;
    id.lam = lam;
    id.px = tx * TILE_W + (l & (TILE_W - 1));
    id.py = ty * TILE_H + l / TILE_W;
    id.valid = id.px < J->W && id.py < J->H && lam < J->n_lambda;
    id.ch = J->channel[lam < 3 ? lam : 2];
    id.pix = (unsigned)(id.py * J->W + id.px);
}

__device__ __forceinline__ PathId path_id(const JobTable *jt, const WaveDesc &wd, int p)
{
    const WaveSeg &g = wd.seg[seg_of_path(wd, p)];
    const int loc = p - g.path_offset;
    const int s = loc / g.item_count, il = loc - s * g.item_count;
    PathId id;
    decode_item(jt->jobs + g.job, g.item_begin + il, id);
    id.s = s;
    return id;
}

// append val to a queue: one atomic per group of converged lanes
__device__ __forceinline__ void enqueue(int *q, int *count, int val)
{
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(m, base, leader);
    q[base + __popc(m & ((1u << lane) - 1u))] = val;
}

__device__ __forceinline__ void flush_counters(const Counters &cnt, SlotScratch *scr)
{
    const unsigned v[8] = {cnt.samples, cnt.rays, cnt.boxes, cnt.tris, cnt.refines, cnt.fallbacks, cnt.shadows, cnt.bounces};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        unsigned long long x = v[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, off);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&scr->counters[k], x);
    }
}

// ------------------------------------------------------------------------------- s1 + s2
template <class R>
__global__ void __launch_bounds__(GEN_BLOCK) k_gen(const JobTable *__restrict__ jt, const WaveDesc wd, PathBufs pb,
                                                   SlotScratch *__restrict__ scr)
{
    using RO = RealOps<R>;
    const int p = blockIdx.x * GEN_BLOCK + threadIdx.x;
    if (p >= wd.n_paths) return;
    const PathId id = path_id(jt, wd, p);
    pb.amp[p] = 0.0f;
    if (id.J->kind == 1) {
        // cache bake (a wave of bake jobs only): every path starts as an incoherent ray from its
        // cell centre in a direction uniform on the sphere, drawn at vertex 0
        if (p == 0) scr->qcount[0][1] = wd.n_paths;
        pb.q[1][0][p] = id.valid ? p : (p | Q_FINALIZE);
        pb.inc[p] = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
        pb.inc2[p] = make_float2(0.0f, __int_as_float(0));
        if (!id.valid) return;
        const DevJob &J = *id.J;
        const float4 u = path_draw(J, id.pix, (unsigned)id.s, 0u, 0u, (unsigned)id.lam);
        const float ct = 1.0f - 2.0f * u.x, st = 2.0f * sqrtf(u.x * (1.0f - u.x));
        float sp, cp;
        sincospif(2.0f * u.y, &sp, &cp);
        const int iy = id.py % J.W, iz = id.py / J.W;
        const float3 x = f3(J.bake_lo[0] + ((float)id.px + 0.5f) * J.bake_h[0], J.bake_lo[1] + ((float)iy + 0.5f) * J.bake_h[1],
                            J.bake_lo[2] + ((float)iz + 0.5f) * J.bake_h[2]);
        pb.ray_o[p] = make_float4(x.x, x.y, x.z, 1e30f);
        pb.ray_d[p] = make_float4(st * cp, st * sp, ct, __int_as_float(-1));
        pb.inc2[p] = make_float2(0.0f, __int_as_float(VF_PREV_DELTA | VF_BAKE));
        return;
    }
    // the first coherent queue is the identity; paths of pixels outside a ragged SLM are marked
    if (p == 0) scr->qcount[0][0] = wd.n_paths;
    pb.q[0][0][p] = id.valid ? p : (p | Q_FINALIZE);
    if (!id.valid) return;
    const DevJob &J = *id.J;
    const float4 u = path_draw(J, id.pix, (unsigned)id.s, 0u, 0u, (unsigned)id.lam);
    const R x = RO::mulf(RO::rc(J.pitch), (float)id.px + 0.5f - 0.5f * (float)J.W);
    const R y = RO::mulf(RO::rc(J.pitch), (float)id.py + 0.5f - 0.5f * (float)J.H);
    const R s1 = RO::mulf(RO::rc(J.h_cone[id.lam]), u.x);    // 1 - cos(theta)
    const R ct = RO::f(1.0f) - s1;
    const R sn = RO::sqrt_(s1 * (RO::f(2.0f) - s1));
    R sp, cp;
    RO::sincos2pi(u.y, J.sincos_tab, sp, cp);
    const R3<R> dh = r3<R>(sn * cp, sn * sp, ct);
    R3<R> co, cd;
    if (J.t_identity) {
        co = r3<R>(x, y, RO::f(0.0f));
        cd = dh;
    } else {
        // T = [Rm | t]: world origin Rm^T (x - t), world direction Rm^T d (Eq. 3, rigid T)
        const R3<R> q = r3<R>(x - RO::rc(J.t[0]), y - RO::rc(J.t[1]), -RO::rc(J.t[2]));
        const R3<R> c0 = r3<R>(RO::rc(J.R[0]), RO::rc(J.R[3]), RO::rc(J.R[6]));
        const R3<R> c1 = r3<R>(RO::rc(J.R[1]), RO::rc(J.R[4]), RO::rc(J.R[7]));
        const R3<R> c2 = r3<R>(RO::rc(J.R[2]), RO::rc(J.R[5]), RO::rc(J.R[8]));
        co = r3<R>(rdot(c0, q), rdot(c1, q), rdot(c2, q));
        cd = r3<R>(rdot(c0, dh), rdot(c1, dh), rdot(c2, dh));
    }
    coh_store<R>(pb, p, co, cd, RO::f(0.0f));
    pb.coh4[p] = make_float4(1.0f, 1.0f, RO::to_f(ct), __int_as_float(0));
    pb.inc2[p] = make_float2(0.0f, __int_as_float(0));
    const float3 of = tof3(co), df_ = tof3(cd);
    pb.ray_o[p] = make_float4(of.x, of.y, of.z, 1e30f);
    pb.ray_d[p] = make_float4(df_.x, df_.y, df_.z, __int_as_float(-1));
}

// ------------------------------------------------------------------------------------ s3
template <class R> __device__ __forceinline__ bool r_less(R a, R b);
template <> __device__ __forceinline__ bool r_less<double>(double a, double b) { return a < b; }
template <> __device__ __forceinline__ bool r_less<df>(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
template <class R> __device__ __forceinline__ bool r_nonneg(R a);
template <> __device__ __forceinline__ bool r_nonneg<double>(double a) { return a >= 0.0; }
template <> __device__ __forceinline__ bool r_nonneg<df>(df a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo >= 0.0f); }

// Plane intersection and barycentric inside test of one triangle in the coherent arithmetic
// (the decision rule of the definition: closed triangle, distance beyond tmin).
template <class R>
__device__ __forceinline__ bool exact_hit(const DevScene &sc, int tri, const R3<R> &co, const R3<R> &cd, R tmin, R &t)
{
    using RO = RealOps<R>;
    const int rb = tri * REF_N;
    const R3<R> n = r3<R>(RO::load(sc.ref64, sc.refdf, rb), RO::load(sc.ref64, sc.refdf, rb + 1),
                          RO::load(sc.ref64, sc.refdf, rb + 2));
    const R den = rdot(n, cd);
    if (RO::to_f(den) == 0.0f) return false;
    t = (RO::load(sc.ref64, sc.refdf, rb + 3) - rdot(n, co)) / den;
    if (!r_less<R>(tmin, t)) return false;
    const uint4 ix = __ldg(sc.tri_attr + tri);
    const R3<R> dP = (co + scale(cd, t)) - fromf3<R>(f3(sc.verts[3 * ix.x], sc.verts[3 * ix.x + 1], sc.verts[3 * ix.x + 2]));
    const R b1 = rdot(r3<R>(RO::load(sc.ref64, sc.refdf, rb + 4), RO::load(sc.ref64, sc.refdf, rb + 5),
                            RO::load(sc.ref64, sc.refdf, rb + 6)), dP);
    const R b2 = rdot(r3<R>(RO::load(sc.ref64, sc.refdf, rb + 7), RO::load(sc.ref64, sc.refdf, rb + 8),
                            RO::load(sc.ref64, sc.refdf, rb + 9)), dP);
    return r_nonneg<R>(b1) && r_nonneg<R>(b2) && r_nonneg<R>(RO::f(1.0f) - b1 - b2);
}

// resident blocks per SM the trace and shading kernels are compiled for (bounds their registers)
#ifndef HPT_SHADE_MINB
#define HPT_SHADE_MINB 8            // 64 registers: 50 % occupancy beats the spill-free 96 (31 %)
#endif
#ifndef HPT_SHADE_INC_MINB
#define HPT_SHADE_INC_MINB HPT_SHADE_MINB   // the incoherent shading kernel
#endif
#ifndef HPT_TRACE_MINB
#define HPT_TRACE_MINB 8
#endif
#ifndef HPT_TRACE_INC_MINB
#define HPT_TRACE_INC_MINB 8        // the incoherent / shadow-ray trace kernel
#endif
#ifndef HPT_ACCUM_MINB
#define HPT_ACCUM_MINB 1
#endif

// COH = true: the coherent queue of the iteration (closest hit with the re-decision of uncertain
// hits in the coherent arithmetic); false: the incoherent and shadow queues (float closest / any
// hit only), so that the second kernel carries none of the coherent code and its registers.
template <class R, bool STATS, bool COH>
__global__ void __launch_bounds__(TRACE_BLOCK, COH ? HPT_TRACE_MINB : HPT_TRACE_INC_MINB)
    k_trace(const JobTable *__restrict__ jt, const WaveDesc wd, PathBufs pb, SlotScratch *__restrict__ scr, int it)
{
    using RO = RealOps<R>;
    extern __shared__ int s_stack[];          // wd.stack_n traversal stack entries per thread
    int *stk = s_stack + threadIdx.x;
    const int slimit = wd.stack_n;
    const int nc = COH ? scr->qcount[it][0] : 0;
    const int ni = COH ? 0 : scr->qcount[it][1], ns = COH ? 0 : scr->qcount[it][2];
    const int total = nc + ni + ns;
    const int par = it & 1;
    int status = 0;
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int idx = blockIdx.x * TRACE_BLOCK + threadIdx.x; idx < total; idx += gridDim.x * TRACE_BLOCK) {
        int kind, qi;
        if (COH) { kind = 0; qi = idx; }
        else if (idx < ni) { kind = 1; qi = idx; }
        else { kind = 2; qi = idx - ni; }
        if (!HPT_IN(qi, pb.capacity)) {
            status |= ST_BOUNDS;
            continue;
        }
        const int e = pb.q[kind][par][qi];
        if (kind < 2 && (e & Q_FINALIZE)) continue;   // no ray: a path that only waits for its shadow ray, or none
        const int p = e;
        if (!HPT_IN(p, wd.n_paths)) {
            status |= ST_BOUNDS;
            continue;
        }
        const DevScene &sc = jt->jobs[wd.seg[seg_of_path(wd, p)].job].sc;
        const float4 o4 = pb.ray_o[p], d4 = pb.ray_d[p];
        const int skip = __float_as_int(d4.w);
        HitF h;
        Cands cand;
        if (STATS) cnt.rays++;
        if (kind == 2) {
            if (STATS) cnt.shadows++;
            const float4 s4 = pb.sh_d[p];
            const bool any = traverse<STATS, TRACE_BLOCK>(sc, xyz(o4), xyz(s4), s4.w, skip, WATERTIGHT_EPS, false, true, h,
                                                          cand, stk, slimit, status, cnt);
            pb.occl[p] = any ? 1 : 0;
        } else if (kind == 1) {
            if (STATS) cnt.bounces++;
            traverse<STATS, TRACE_BLOCK>(sc, xyz(o4), xyz(d4), 1e30f, skip, WATERTIGHT_EPS, false, false, h, cand, stk,
                                         slimit, status, cnt);
            pb.hit[p] = make_float4(h.t, h.u, h.v, __int_as_float(h.tri));
        } else if constexpr (COH) {
            traverse<STATS, TRACE_BLOCK>(sc, xyz(o4), xyz(d4), 1e30f, skip, 0.0f, true, false, h, cand, stk, slimit,
                                         status, cnt, it == 0);
            int tri = h.tri;
            if (cand.n > 0) {
                // the float test was within its error band: decide among the candidates (and the
                // float winner) in the coherent arithmetic; a full double traversal only when the
                // list overflowed or no candidate holds
                if (STATS) cnt.refines++;
                R3<R> co, cd;
                R opl_unused;
                coh_load<R>(pb, p, co, cd, opl_unused);
                const bool cont = __float_as_int(pb.coh4[p].w) > 0;   // a continuation after a delta vertex
                const R tmin = cont ? RO::fromd(COH_TMIN) : RO::f(0.0f);
                int best = -1;
                R bt = RO::f(0.0f);
                if (cand.n <= NCAND) {
                    for (int k = -1; k < cand.n; ++k) {
                        const int id = k < 0 ? h.tri : cand.id[k];
                        if (id < 0 || id == skip) continue;
                        R tk;
                        if (exact_hit<R>(sc, id, co, cd, tmin, tk) &&
                            (best < 0 || r_less<R>(tk, bt) || (!r_less<R>(bt, tk) && id < best))) {
                            best = id;
                            bt = tk;
                        }
                    }
                }
                if (best >= 0) {
                    tri = best;
                } else {
                    if (STATS) cnt.fallbacks++;
                    double tt;
                    tri = traverse_fp64<TRACE_BLOCK>(sc, RO::to_d(co.x), RO::to_d(co.y), RO::to_d(co.z), RO::to_d(cd.x),
                                                     RO::to_d(cd.y), RO::to_d(cd.z), cont ? COH_TMIN : 0.0, skip,
                                                     &tt, stk, slimit, status);
                }
            }
            pb.hit[p] = make_float4(h.t, 0.0f, 0.0f, __int_as_float(tri));
        }
    }
    if (STATS) flush_counters(cnt, scr);
    if (status) atomicOr(&scr->status, (unsigned)status);
}

// ------------------------------------------------------------------------------- s3 - s5
struct IncState {
    float L, beta, ppdf, tprev, nee;
    int vfl;
};

// One vertex of the incoherent path (Eq. 1): MIS-weighted emission, then a delta continuation,
// or the ambient cache, or NEE to a rectangular light plus a BSDF-sampled continuation.  Rays
// are appended to the next iteration's queues; returns true when the path ends here.
__device__ __forceinline__ bool vertex(const PathId &id, IncState &st, const Surf &S, float3 wo, const PathBufs &pb,
                                       int p, int *const *qn, int *qcn)
{
    const DevJob &J = *id.J;
    const DevScene &sc = J.sc;
    const MatDev M = sc.mats[S.mat];
    const int ch = id.ch;
    const int v = st.vfl & VF_V;
    const bool prev_delta = st.vfl & VF_PREV_DELTA;
    const float Le = emitted(sc, M, S, wo, ch);
    if (Le > 0.0f) {
        float w = 1.0f;
        if (!prev_delta && M.kind == 4 && M.light >= 0 && sc.n_lights > 0) {
            const LightDev &Lt = sc.lights[M.light];
            const float cl = dot3(wo, f3(Lt.n[0], Lt.n[1], Lt.n[2]));
            const float pl = st.tprev * st.tprev / (cl * Lt.area) / (float)sc.n_lights;
            w = st.ppdf * st.ppdf / (st.ppdf * st.ppdf + pl * pl);
        }
        st.L += st.beta * Le * w;
    }
    if (M.kind == 4) return true;
    float3 ng = S.ng, ns = S.ns;
    const bool front = dot3(wo, ng) > 0.0f;
    const float4 u = path_draw(J, id.pix, (unsigned)id.s, (unsigned)v, 0u, (unsigned)id.lam);
    if (M.kind == 2 || M.kind == 3) {
        if (v >= J.max_depth) return true;
        float3 wi;
        if (M.kind == 2) {
            if (!front) { ng = -ng; ns = -ns; }
            const float c = dot3(wo, ns);
            if (c <= 0.0f) return true;
            wi = ns * (2.0f * c) - wo;
            if (dot3(wi, ng) <= 0.0f) return true;
            st.beta *= albedo_of(sc, M, S, ch);
        } else {
            const float n_i = front ? 1.0f : M.ior, n_t = front ? M.ior : 1.0f;
            const float3 n = front ? ns : -ns, g = front ? ng : -ng;
            const float ci = dot3(wo, n);
            if (ci <= 0.0f) return true;
            const float F = fresnel_dielectric(ci, n_i, n_t);
            if (u.x < F) {
                wi = n * (2.0f * ci) - wo;
                if (dot3(wi, g) <= 0.0f) return true;
            } else {
                const float eta = n_i / n_t;
                const float ct = sqrtf(fmaxf(0.0f, 1.0f - eta * eta * (1.0f - ci * ci)));
                wi = wo * (-eta) + n * (eta * ci - ct);
                if (dot3(wi, g) >= 0.0f) return true;
                st.beta *= eta * eta;
            }
        }
        st.vfl = (st.vfl | VF_PREV_DELTA) & ~VF_INC_FIRST;
        st.nee = 0.0f;
        const float3 o = S.p + (dot3(wi, S.ng) > 0.0f ? S.ng : -S.ng) * INC_OFFSET;
        pb.ray_o[p] = make_float4(o.x, o.y, o.z, 1e30f);
        pb.ray_d[p] = make_float4(wi.x, wi.y, wi.z, __int_as_float(S.tri));
        enqueue(qn[1], &qcn[1], p);
        return false;
    }
    // non-delta (Lambert, GGX)
    if (!front) { ng = -ng; ns = -ns; }
    if (dot3(wo, ns) <= 0.0f) return true;
    if (J.use_cache && sc.cache_res > 0 && !(st.vfl & VF_INC_FIRST)) {
        st.L += st.beta * albedo_of(sc, M, S, ch) * INV_PI_F * cache_lookup(sc, S.p, ch);
        return true;
    }
    const float3 org = S.p + ng * INC_OFFSET;
    const float alb = albedo_of(sc, M, S, ch);
    bool shadow = false;
    st.nee = 0.0f;
    if (sc.n_lights > 0) {
        int li = 0;
        if (sc.n_lights > 1) {
            const float4 u2 = path_draw(J, id.pix, (unsigned)id.s, (unsigned)v, 1u, (unsigned)id.lam);
            li = min((int)(u2.x * (float)sc.n_lights), sc.n_lights - 1);
        }
        const LightDev &Lt = sc.lights[li];
        const float3 y = f3(Lt.corner[0], Lt.corner[1], Lt.corner[2]) + f3(Lt.eu[0], Lt.eu[1], Lt.eu[2]) * u.x +
                         f3(Lt.ev[0], Lt.ev[1], Lt.ev[2]) * u.y;
        const float3 dv = y - org;
        const float dist = sqrtf(dot3(dv, dv));
        const float3 wl = dv * (1.0f / dist);
        const float cl = -dot3(wl, f3(Lt.n[0], Lt.n[1], Lt.n[2]));
        const float Ll = Lt.Le[ch];
        if (cl > 0.0f && dot3(wl, ng) > 0.0f && dot3(wl, ns) > 0.0f && Ll > 0.0f) {
            float f, pbs;
            bsdf_eval(M, alb, ns, wo, wl, f, pbs);
            const float pl = dist * dist / (cl * Lt.area) / (float)sc.n_lights;
            if (f > 0.0f) {
                const float wm = v < J.max_depth ? pl * pl / (pl * pl + pbs * pbs) : 1.0f;
                st.nee = st.beta * f * dot3(wl, ns) * Ll * wm / pl;
                shadow = true;
                pb.sh_d[p] = make_float4(wl.x, wl.y, wl.z, dist * (1.0f - SHADOW_SHRINK));
            }
        }
    }
    bool bounce = false;
    float3 wi = f3(0.0f, 0.0f, 1.0f);
    if (v < J.max_depth) {
        float3 t, b;
        make_frame(ns, t, b);
        float weight = 0.0f, pbs = 0.0f;
        if (M.kind == 0) {
            const float rr = sqrtf(u.z);
            float s_, c_;
            sincospif(2.0f * u.w, &s_, &c_);
            const float z = sqrtf(1.0f - u.z);
            wi = t * (rr * c_) + b * (rr * s_) + ns * z;
            bounce = dot3(wi, ng) > 0.0f;
            weight = alb;
            pbs = z * INV_PI_F;
        } else {
            const float al = M.rough * M.rough;
            const float3 lo = f3(dot3(wo, t), dot3(wo, b), dot3(wo, ns));
            if (lo.z > 0.0f) {
                const float3 vh = normalize3(f3(al * lo.x, al * lo.y, lo.z));
                const float l2 = vh.x * vh.x + vh.y * vh.y;
                const float3 T1 = l2 > 0.0f ? f3(-vh.y, vh.x, 0.0f) * rsqrtf(l2) : f3(1.0f, 0.0f, 0.0f);
                const float3 T2 = cross3(vh, T1);
                const float rr = sqrtf(u.z);
                float s_, c_;
                sincospif(2.0f * u.w, &s_, &c_);
                const float t1 = rr * c_;
                float t2 = rr * s_;
                const float sm = 0.5f * (1.0f + vh.z);
                t2 = (1.0f - sm) * sqrtf(fmaxf(0.0f, 1.0f - t1 * t1)) + sm * t2;
                const float tz = sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
                const float3 nh = T1 * t1 + T2 * t2 + vh * tz;
                const float3 ne = normalize3(f3(al * nh.x, al * nh.y, fmaxf(0.0f, nh.z)));
                const float c = dot3(lo, ne);
                const float3 li = ne * (2.0f * c) - lo;
                if (li.z > 0.0f) {
                    weight = schlick(alb, dot3(li, ne)) * ggx_G1(al, li);
                    pbs = ggx_G1(al, lo) * ggx_D(al, ne) / (4.0f * lo.z);
                    wi = t * li.x + b * li.y + ns * li.z;
                    bounce = dot3(wi, ng) > 0.0f;
                }
            }
        }
        if (bounce) {
            st.beta *= weight;
            st.ppdf = pbs;
        }
    }
    st.vfl &= ~(VF_INC_FIRST | VF_PREV_DELTA);
    if (!shadow && !bounce) return true;
    // both rays leave from the same side of a reflecting surface: one origin serves both
    pb.ray_o[p] = make_float4(org.x, org.y, org.z, 1e30f);
    pb.ray_d[p] = make_float4(wi.x, wi.y, wi.z, __int_as_float(S.tri));
    if (shadow) enqueue(qn[2], &qcn[2], p);
    if (bounce) enqueue(qn[1], &qcn[1], p);
    else enqueue(qn[1], &qcn[1], p | Q_FINALIZE);
    return false;
}

// COH = true: the coherent entries of the iteration; false: the incoherent ones (two kernels,
// so that each carries only its half of the shading code)
template <class R, bool STATS, bool COH>
__global__ void __launch_bounds__(SHADE_BLOCK, COH ? HPT_SHADE_MINB : HPT_SHADE_INC_MINB) k_shade(const JobTable *__restrict__ jt, const WaveDesc wd, PathBufs pb,
                                                       SlotScratch *__restrict__ scr, int it)
{
    using RO = RealOps<R>;
    const int total = scr->qcount[it][COH ? 0 : 1];
    const int par = it & 1, nx = par ^ 1;
    int *const qn[3] = {pb.q[0][nx], pb.q[1][nx], pb.q[2][nx]};
    int *qcn = scr->qcount[it + 1];
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned status = 0;
    for (int idx = blockIdx.x * SHADE_BLOCK + threadIdx.x; idx < total; idx += gridDim.x * SHADE_BLOCK) {
        if (!HPT_IN(idx, pb.capacity)) {
            status |= ST_BOUNDS;
            break;
        }
        const int e = pb.q[COH ? 0 : 1][par][idx];
        if (COH && (e & Q_FINALIZE)) continue;
        const int p = e & 0x7FFFFFFF;
        if (!HPT_IN(p, wd.n_paths)) {
            status |= ST_BOUNDS;
            continue;
        }
        const PathId id = path_id(jt, wd, p);
        const DevJob &J = *id.J;
        const DevScene &sc = J.sc;
        IncState st;
        Surf S;
        float3 wo = f3(0.0f, 0.0f, 1.0f);
        bool do_vertex = false;
        if constexpr (COH) {
            const int tri = __float_as_int(pb.hit[p].w);
            if (tri >= 0 && !HPT_IN(tri, sc.n_tris)) {
                status |= ST_BOUNDS;
                continue;
            }
            if (tri >= 0) {
                R3<R> co, cd;
                R opl;
                coh_load<R>(pb, p, co, cd, opl);
                const float4 c4 = pb.coh4[p];
                const float ncur = c4.x;
                // distance to the triangle's plane n . x = d0 in the coherent arithmetic
                const int rb = tri * REF_N;
                const R3<R> n = r3<R>(RO::load(sc.ref64, sc.refdf, rb), RO::load(sc.ref64, sc.refdf, rb + 1),
                                      RO::load(sc.ref64, sc.refdf, rb + 2));
                const R d0 = RO::load(sc.ref64, sc.refdf, rb + 3);
                const R t = (d0 - rdot(n, co)) / rdot(n, cd);
                const R3<R> P = co + scale(cd, t);
                opl = opl + RO::mulf(t, ncur);        // OPL = sum n_i L_i (Sec. 4.2)
                const int cv = __float_as_int(c4.w) + 1;
                const uint4 ix = __ldg(sc.tri_attr + tri);
                const int kind = sc.mats[ix.w].kind;
                float3 ng = xyz(__ldg(sc.tri_ng + tri));
                const float3 v0 = f3(sc.verts[3 * ix.x], sc.verts[3 * ix.x + 1], sc.verts[3 * ix.x + 2]);
                const R3<R> dP = P - fromf3<R>(v0);
                const float3 dPf = tof3(dP);
                const float3 m1f = f3(RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 4)),
                                      RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 5)),
                                      RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 6)));
                const float3 m2f = f3(RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 7)),
                                      RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 8)),
                                      RO::to_f(RO::load(sc.ref64, sc.refdf, rb + 9)));
                const float3 Pf = tof3(P);
                const float bb1 = dot3(m1f, dPf), bb2 = dot3(m2f, dPf);
                S = make_surf(sc, tri, Pf, bb1, bb2);
                if (kind != 2 && kind != 3) {
                    // P, the real image point.  For a rigid T the virtual image point
                    // Q = T (O + d_OPL v) lies at distance r = d_OPL from the pixel along the
                    // sampled hologram-space direction, whose z component is cos(theta).
                    const float3 dl = tof3(cd);
                    const float cosP = fabsf(dot3(dl, ng));
                    const R ih = RO::rc(J.inv_facet);
                    pb.fturn[p] = RO::frac_f(opl * RO::rc(J.inv_lambda[id.lam]));
                    if (J.phase_mode == 2) {
                        // Eq. 4: the GRF sample under Q = x + d_OPL dh on the hologram plane
                        // (rigid T), dh the sampled hologram-space direction, redrawn here
                        const float4 u0 = path_draw(J, id.pix, (unsigned)id.s, 0u, 0u, (unsigned)id.lam);
                        const R s1 = RO::mulf(RO::rc(J.h_cone[id.lam]), u0.x);
                        const R sn = RO::sqrt_(s1 * (RO::f(2.0f) - s1));
                        R sp, cp;
                        RO::sincos2pi(u0.y, J.sincos_tab, sp, cp);
                        const R xq = RO::mulf(RO::rc(J.pitch), (float)id.px + 0.5f - 0.5f * (float)J.W) + opl * (sn * cp);
                        const R yq = RO::mulf(RO::rc(J.pitch), (float)id.py + 0.5f - 0.5f * (float)J.H) + opl * (sn * sp);
                        int jx = RO::floor_i(RO::addf(xq * RO::rc(J.inv_pitch), 0.5f * (float)J.grf_nx)) % J.grf_nx;
                        int jy = RO::floor_i(RO::addf(yq * RO::rc(J.inv_pitch), 0.5f * (float)J.grf_ny)) % J.grf_ny;
                        pb.cx[p] = jx < 0 ? jx + J.grf_nx : jx;
                        pb.cy[p] = jy < 0 ? jy + J.grf_ny : jy;
                        pb.cz[p] = 0;
                    } else {
                        pb.cx[p] = RO::floor_i(P.x * ih);
                        pb.cy[p] = RO::floor_i(P.y * ih);
                        pb.cz[p] = RO::floor_i(P.z * ih);
                    }
                    // Eq. 2 with the obliquity factor cos(theta) (unless omitted)
                    pb.basep[p] = (J.obliquity ? c4.z : 1.0f) * RO::to_f(opl) /
                                  (J.pdf_w[id.lam] * cosP * J.lambda_f[id.lam]);
                    // the incoherent part starts at P: handed to this iteration's incoherent
                    // shading as a hit at distance 0 from P (vertex count cv after its increment),
                    // so that the coherent kernel carries no BSDF / NEE code
                    pb.inc[p] = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
                    pb.inc2[p] = make_float2(0.0f, __int_as_float((cv - 1) | VF_PREV_DELTA | VF_INC_FIRST | VF_HASP));
                    pb.ray_o[p] = make_float4(Pf.x, Pf.y, Pf.z, 1e30f);
                    pb.ray_d[p] = make_float4(dl.x, dl.y, dl.z, __int_as_float(tri));
                    pb.hit[p] = make_float4(0.0f, bb1, bb2, __int_as_float(tri));
                    enqueue(pb.q[1][par], &scr->qcount[it][1], p);
                } else if (cv < J.max_depth) {
                    // delta vertex: shading normal and the new direction in the coherent arithmetic
                    const MatDev M = sc.mats[ix.w];
                    const R b1 = rdot(r3<R>(RO::load(sc.ref64, sc.refdf, rb + 4), RO::load(sc.ref64, sc.refdf, rb + 5),
                                            RO::load(sc.ref64, sc.refdf, rb + 6)), dP);
                    const R b2 = rdot(r3<R>(RO::load(sc.ref64, sc.refdf, rb + 7), RO::load(sc.ref64, sc.refdf, rb + 8),
                                            RO::load(sc.ref64, sc.refdf, rb + 9)), dP);
                    const R b0 = RO::f(1.0f) - b1 - b2;
                    const float *n0 = sc.normals + 3 * ix.x, *n1 = sc.normals + 3 * ix.y, *n2 = sc.normals + 3 * ix.z;
                    R3<R> ns = r3<R>(RO::mulf(b0, n0[0]) + RO::mulf(b1, n1[0]) + RO::mulf(b2, n2[0]),
                                     RO::mulf(b0, n0[1]) + RO::mulf(b1, n1[1]) + RO::mulf(b2, n2[1]),
                                     RO::mulf(b0, n0[2]) + RO::mulf(b1, n1[2]) + RO::mulf(b2, n2[2]));
                    ns = scale(ns, RO::f(1.0f) / RO::sqrt_(rdot(ns, ns)));
                    const R3<R> wo_r = neg(cd);
                    const bool front = dot3(tof3(wo_r), ng) > 0.0f;
                    R3<R> wi = cd;
                    bool ok = true;
                    float betac = c4.y, nnew = ncur;
                    if (kind == 2) {
                        if (!front) { ns = neg(ns); ng = -ng; }
                        const R c = rdot(wo_r, ns);
                        if (!(RO::to_f(c) > 0.0f)) ok = false;
                        else {
                            wi = scale(ns, RO::mulf(c, 2.0f)) - wo_r;
                            ok = dot3(tof3(wi), ng) > 0.0f;
                            betac *= albedo_of(sc, M, S, id.ch);
                        }
                    } else {
                        const float n_i = front ? 1.0f : M.ior, n_t = front ? M.ior : 1.0f;
                        const R3<R> nn = front ? ns : neg(ns);
                        const float3 g = front ? ng : -ng;
                        const R ci = rdot(wo_r, nn);
                        const float cif = RO::to_f(ci);
                        if (!(cif > 0.0f)) ok = false;
                        else {
                            const float F = fresnel_dielectric(cif, n_i, n_t);
                            const float4 u = path_draw(J, id.pix, (unsigned)id.s, (unsigned)cv, 0u, (unsigned)id.lam);
                            if (u.x < F) {
                                wi = scale(nn, RO::mulf(ci, 2.0f)) - wo_r;
                                ok = dot3(tof3(wi), g) > 0.0f;
                            } else {
                                const R eta = RO::f(n_i) / RO::f(n_t);
                                const R ct = RO::sqrt_(RO::f(1.0f) - eta * eta * (RO::f(1.0f) - ci * ci));
                                wi = scale(nn, eta * ci - ct) - scale(wo_r, eta);
                                ok = dot3(tof3(wi), g) < 0.0f;
                                betac *= RO::to_f(eta * eta);
                                nnew = n_t;
                            }
                        }
                    }
                    if (ok) {
                        coh_store<R>(pb, p, P, wi, opl);
                        pb.coh4[p] = make_float4(nnew, betac, c4.z, __int_as_float(cv));
                        const float3 pf = tof3(P), wf = tof3(wi);
                        pb.ray_o[p] = make_float4(pf.x, pf.y, pf.z, 1e30f);
                        pb.ray_d[p] = make_float4(wf.x, wf.y, wf.z, __int_as_float(tri));
                        enqueue(qn[0], &qcn[0], p);
                    }
                }
            }
        } else {
            const float4 s4 = pb.inc[p];
            const float2 s2 = pb.inc2[p];
            st.L = s4.x;
            st.beta = s4.y;
            st.ppdf = s4.z;
            st.tprev = s4.w;
            st.nee = s2.x;
            st.vfl = __float_as_int(s2.y);
            // the NEE of the previous vertex lands first, as in the sequential estimator
            if (st.nee > 0.0f && !pb.occl[p]) st.L += st.nee;
            st.nee = 0.0f;
            if (!(e & Q_FINALIZE)) {
                const float4 h = pb.hit[p];
                const int tri = __float_as_int(h.w);
                if (tri >= 0 && !HPT_IN(tri, sc.n_tris)) {
                    status |= ST_BOUNDS;
                    continue;
                }
                if (tri >= 0) {
                    const float4 o4 = pb.ray_o[p], d4 = pb.ray_d[p];
                    st.vfl = (st.vfl & ~VF_V) | ((st.vfl & VF_V) + 1);
                    st.tprev = h.x;
                    S = make_surf(sc, tri, xyz(o4) + xyz(d4) * h.x, h.y, h.z);
                    wo = -xyz(d4);
                    do_vertex = true;
                }
            }
            if (!do_vertex) {
                if (STATS) cnt.samples++;
                pb.amp[p] = (st.vfl & VF_BAKE) ? st.L
                            : (st.vfl & VF_HASP) ? pb.basep[p] * sqrtf(pb.coh4[p].y * st.L) : 0.0f;
            }
        }
        if (do_vertex) {
            const bool done = vertex(id, st, S, wo, pb, p, qn, qcn);
            if (done) {
                if (STATS) cnt.samples++;
                pb.amp[p] = (st.vfl & VF_BAKE) ? st.L
                            : (st.vfl & VF_HASP) ? pb.basep[p] * sqrtf(pb.coh4[p].y * st.L) : 0.0f;
            } else {
                pb.inc[p] = make_float4(st.L, st.beta, st.ppdf, st.tprev);
                pb.inc2[p] = make_float2(st.nee, __int_as_float(st.vfl));
            }
        }
    }
    if (STATS) flush_counters(cnt, scr);
    if (HPT_CHECKED && status) atomicOr(&scr->status, status);
}

// ------------------------------------------------------------------------------- s6 - s9
template <class R>
__device__ __noinline__ float2 point_field(const DevJob *Jp, int lam, int px, int py, int *stk, int &status)
{
    using RO = RealOps<R>;
    const DevJob &J = *Jp;
    const DevScene &sc = J.sc;
    float2 acc = make_float2(0.0f, 0.0f);
    const R x = RO::mulf(RO::rc(J.pitch), (float)px + 0.5f - 0.5f * (float)J.W);
    const R y = RO::mulf(RO::rc(J.pitch), (float)py + 0.5f - 0.5f * (float)J.H);
    for (int e = 0; e < sc.n_points; ++e) {
        const double *pe = sc.points + 4 * e;
        const R3<R> pw = r3<R>(RO::fromd(pe[0]), RO::fromd(pe[1]), RO::fromd(pe[2]));
        R3<R> q, O;
        if (J.t_identity) {
            q = r3<R>(pw.x - x, pw.y - y, pw.z);
            O = r3<R>(x, y, RO::f(0.0f));
        } else {
            const R3<R> rw0 = r3<R>(RO::rc(J.R[0]), RO::rc(J.R[1]), RO::rc(J.R[2]));
            const R3<R> rw1 = r3<R>(RO::rc(J.R[3]), RO::rc(J.R[4]), RO::rc(J.R[5]));
            const R3<R> rw2 = r3<R>(RO::rc(J.R[6]), RO::rc(J.R[7]), RO::rc(J.R[8]));
            q = r3<R>(rdot(rw0, pw) + RO::rc(J.t[0]) - x, rdot(rw1, pw) + RO::rc(J.t[1]) - y,
                      rdot(rw2, pw) + RO::rc(J.t[2]));
            const R3<R> qq = r3<R>(x - RO::rc(J.t[0]), y - RO::rc(J.t[1]), -RO::rc(J.t[2]));
            const R3<R> c0 = r3<R>(RO::rc(J.R[0]), RO::rc(J.R[3]), RO::rc(J.R[6]));
            const R3<R> c1 = r3<R>(RO::rc(J.R[1]), RO::rc(J.R[4]), RO::rc(J.R[7]));
            const R3<R> c2 = r3<R>(RO::rc(J.R[2]), RO::rc(J.R[5]), RO::rc(J.R[8]));
            O = r3<R>(rdot(c0, qq), rdot(c1, qq), rdot(c2, qq));
        }
        const R r = RO::sqrt_(rdot(q, q));
        const float rf = RO::to_f(r);
        const float ct = RO::to_f(q.z) / rf;
        if (ct < J.cos_max[lam]) continue;
        const float3 Of = tof3(O);
        const float3 dw = tof3(pw - O);
        const float dist = sqrtf(dot3(dw, dw));
        HitF h;
        Cands cand;
        Counters dummy;
        if (traverse<false, ACCUM_BLOCK>(sc, Of, dw * (1.0f / dist), dist * (1.0f - SHADOW_SHRINK), -1, WATERTIGHT_EPS,
                                         false, true, h, cand, stk, TSTACK, status, dummy))
            continue;
        const float turns = RO::frac_f(r * RO::rc(J.inv_lambda[lam]));
        float sn, cs;
        sincospif(2.0f * turns, &sn, &cs);
        const float a = (float)pe[3] * (J.obliquity ? ct : 1.0f) / rf;
        acc.x += a * cs;
        acc.y += a * sn;
    }
    return acc;
}

template <class R>
__global__ void __launch_bounds__(ACCUM_BLOCK, HPT_ACCUM_MINB) k_accum(const JobTable *__restrict__ jt, const WaveDesc wd, PathBufs pb,
                                                       SlotScratch *__restrict__ scr)
{
    __shared__ int s_stack[TSTACK * ACCUM_BLOCK];
    const int i = blockIdx.x * ACCUM_BLOCK + threadIdx.x;
    if (i >= wd.n_items) return;
    int k = 0, first = 0;
    while (k + 1 < wd.n_seg && first + wd.seg[k].item_count <= i) {
        first += wd.seg[k].item_count;
        ++k;
    }
    const WaveSeg &g = wd.seg[k];
    const int il = i - first;
    PathId id;
    decode_item(jt->jobs + g.job, g.item_begin + il, id);
    if (!id.valid) return;
    const DevJob &J = *id.J;
    if (J.kind == 1) {
        // cache bake: E = pi / N sum of the arriving radiance, Kahan-compensated in sample order
        float a = 0.0f, c = 0.0f;
        for (int s = 0; s < g.spp; ++s) {
            const float y = pb.amp[g.path_offset + s * g.item_count + il] - c, t = a + y;
            c = (t - a) - y;
            a = t;
        }
        J.bake_out[(size_t)id.pix * 3 + id.lam] = 3.14159265f * (a - c) / (float)g.spp;
        return;
    }
    const int K = J.K, off = J.hologram_offset, spp = g.spp;
    float ar[KMAX], ai[KMAX], cr[KMAX], ci[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) ar[j] = ai[j] = cr[j] = ci[j] = 0.0f;
    for (int s = 0; s < spp; ++s) {
        const int p = g.path_offset + s * g.item_count + il;
        if (!HPT_IN(p, wd.n_paths)) {
            atomicOr(&scr->status, ST_BOUNDS);
            break;
        }
        const float amp = pb.amp[p];
        if (amp == 0.0f) continue;
        const float ft = pb.fturn[p];
        const unsigned c0 = (unsigned)pb.cx[p], c1 = (unsigned)pb.cy[p], c2 = (unsigned)pb.cz[p];
        uint4 ph = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < K) {
                const int m = off + j;
                float u = 0.0f;
                if (J.phase_mode == 0) {
                    // s8: facet phase of hologram m, one Philox draw per four holograms
                    if (j == 0 || (m & 3) == 0)
                        ph = philox(make_uint4(c0, c1, c2, ((unsigned)id.lam << 16) | ((unsigned)m >> 2)), J.pseed_lo,
                                    J.pseed_hi);
                    const unsigned w = (m & 3) == 0 ? ph.x : ((m & 3) == 1 ? ph.y : ((m & 3) == 2 ? ph.z : ph.w));
                    u = u24(w);
                } else if (J.phase_mode == 2) {
                    // Eq. 4: phi_m sampled from the hologram's GRF map at the cell of Q
                    u = __ldg(J.grf + ((size_t)j * J.grf_ny + c1) * J.grf_nx + c0) * 0.159154943f;
                }
                float sn, cs;
                sincospif(2.0f * (ft + u), &sn, &cs);
                // s9: (1/(i lambda)) is folded into the amplitude: multiply the phasor by -i
                const float xr = amp * sn, xi = -amp * cs;
                const float yr = xr - cr[j], tr = ar[j] + yr;
                cr[j] = (tr - ar[j]) - yr;
                ar[j] = tr;
                const float yi = xi - ci[j], ti = ai[j] + yi;
                ci[j] = (ti - ai[j]) - yi;
                ai[j] = ti;
            }
        }
    }
    float2 pf = make_float2(0.0f, 0.0f);
    if (J.sc.n_points > 0) {
        int status = 0;
        pf = point_field<R>(id.J, id.lam, id.px, id.py, s_stack + threadIdx.x, status);
        if (status) atomicOr(&scr->status, (unsigned)status);
    }
    const float inv_n = 1.0f / (float)spp;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j < K) {
            const size_t o = ((size_t)(id.lam * K + j) * J.H + id.py) * J.W + id.px;
            J.out[o] = make_float2((ar[j] - cr[j]) * inv_n + pf.x, (ai[j] - ci[j]) * inv_n + pf.y);
        }
    }
}

}  // namespace hpt
