/* FP64 CPU oracle of the wave path tracer -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision restatement of the method of
 * "HoloPathTracer: Fast and Accurate Wave Path Tracing for Holography"
 * (ACM TOG 45(4), 2026).  Each function names the passage it follows.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * CUDA library shares no code with it.
 *
 * Readings taken where the paper is silent:
 *  - estimator weight: A = sqrt(beta * L); contribution
 *      (1/(i lambda)) * A * cos(theta) / (r * pdf_A) * exp(i (k r + phi_m))
 *    with pdf_A = pdf_omega * |cos theta_P| / r^2 (area measure at P);
 *  - directions uniform in solid angle inside the cone theta <= asin(lambda/2p);
 *  - ray origin = pixel centre; one incoherent estimate per coherent sample;
 *  - every scattering vertex counts toward max_depth; depth 1 = emission + NEE
 *    at the first vertex; a delta chain that reaches max_depth contributes 0;
 *    NEE at the last vertex takes full weight (no BSDF continuation exists);
 *  - random facet phase: cubic world cells of edge facet_size, hashed with a
 *    Philox draw keyed by phase_seed;
 *  - smooth (interpolated) shading normals; geometric normals for sidedness,
 *    offsets and the area Jacobian; bilinear textures; trilinear cache;
 *  - incoherent ray origins are offset 1e-7 m along the geometric normal; the
 *    coherent chain restarts exactly at the hit point (t > 1e-9 m) so that the
 *    optical path length is not perturbed; the hit triangle is excluded.
 *  Parity unpinned: the absolute brightness convention against the paper's
 *  figures (the paper prints no field values).
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define INC_OFFSET 1e-7      /* metres, incoherent origin offset            */
#define COH_TMIN 1e-9        /* metres, coherent-chain minimum distance      */
#define SHADOW_SHRINK 1e-5   /* shadow rays stop at (1 - SHADOW_SHRINK) dist */
#define EDGE_FLAG 1e-5       /* barycentric margin reported as "near edge"   */

enum { M_LAMBERT = 0, M_GGX = 1, M_MIRROR = 2, M_DIELECTRIC = 3, M_EMITTER = 4 };

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 nrm(v3 a) { return scl(a, 1.0 / len(a)); }
static double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:   */
/* ten rounds of two 32x32->64 multiplies with a Weyl-sequence key schedule. */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* draw stream of the path: counter (pixel, sample, vertex<<8 | group, lambda<<16 | 0xFFFF) */
static void path_draw(const or_render *r, int lam, int64_t pix, int s, int v, int group, double u[4])
{
    uint32_t c[4] = {(uint32_t)pix, (uint32_t)s, ((uint32_t)v << 8) | (uint32_t)group,
                     ((uint32_t)lam << 16) | 0xFFFFu};
    uint32_t k[2] = {(uint32_t)r->seed, (uint32_t)(r->seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(c, k, o);
    for (int i = 0; i < 4; i++) u[i] = u24(o[i]);
}

/* facet phase draw (Sec. 4.3 stand-in): counter (cell x, y, z, lambda<<16 | m>>2), lane m&3 */
static double phase_draw(const or_render *r, int lam, const int64_t cell[3], int m)
{
    uint32_t c[4] = {(uint32_t)cell[0], (uint32_t)cell[1], (uint32_t)cell[2],
                     ((uint32_t)lam << 16) | ((uint32_t)m >> 2)};
    uint32_t k[2] = {(uint32_t)r->phase_seed, (uint32_t)(r->phase_seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(c, k, o);
    return u24(o[m & 3]);
}

/* Eq. 4: phase of hologram m (relative to hologram_offset) at the image point's position
   (x_Q, y_Q) on the hologram plane: the sample of the periodic GRF grid, of the SLM's pitch,
   whose cell [j - n/2, j + 1 - n/2) * pitch contains it.  Returned in turns. */
static double grf_phase(const or_render *r, double qx, double qy, int m)
{
    const int64_t nx = r->grf_nx, ny = r->grf_ny;
    const double inv_p = 1.0 / r->pitch;
    int64_t jx = (int64_t)floor(qx * inv_p + 0.5 * (double)nx) % nx;
    int64_t jy = (int64_t)floor(qy * inv_p + 0.5 * (double)ny) % ny;
    if (jx < 0) jx += nx;
    if (jy < 0) jy += ny;
    return r->grf_phi[((int64_t)m * ny + jy) * nx + jx] / (2.0 * PI);
}

void or_grf_phases(uint64_t seed, int32_t m, int32_t nx, int32_t ny, double *xi)
{
    const uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t iy = 0; iy < ny; iy++)
        for (int32_t ix = 0; ix < nx; ix++) {
            uint32_t c[4] = {(uint32_t)ix, (uint32_t)iy, (uint32_t)m, 0x47524600u}, o[4];
            or_philox4x32_10(c, k, o);
            xi[(int64_t)iy * nx + ix] = 2.0 * PI * u24(o[0]);
        }
}

/* ------------------------------------------------------------------------ */
/* binary16 -> double, from the IEEE 754 layout                              */
/* ------------------------------------------------------------------------ */
double or_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1024.0 + m, e - 25);
    return sign ? -v : v;
}

/* ------------------------------------------------------------------------ */
/* scene + median-split BVH (the oracle's own, FP64 boxes)                   */
/* ------------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3]; int left, right, first, count; } bnode;

typedef struct {
    or_scene s;
    int nt;
    v3 *V0, *E1, *E2;     /* per triangle, exact doubles of the float32 vertices */
    int *order;           /* triangle ids in leaf order */
    bnode *nodes;
    int nn;
    double light_area[8];
    v3 light_n[8];
} oracle_t;

static void tri_bounds(const oracle_t *o, int t, double lo[3], double hi[3])
{
    v3 p[3] = {o->V0[t], add(o->V0[t], o->E1[t]), add(o->V0[t], o->E2[t])};
    for (int k = 0; k < 3; k++) {
        lo[k] = hi[k] = comp(p[0], k);
        for (int j = 1; j < 3; j++) {
            double c = comp(p[j], k);
            if (c < lo[k]) lo[k] = c;
            if (c > hi[k]) hi[k] = c;
        }
    }
}

static double *g_sort_key;
static int cmp_key(const void *a, const void *b)
{
    double ka = g_sort_key[*(const int *)a], kb = g_sort_key[*(const int *)b];
    return ka < kb ? -1 : (ka > kb ? 1 : (*(const int *)a - *(const int *)b));
}

static int build_node(oracle_t *o, int first, int count, double *cent)
{
    int id = o->nn++;
    bnode *n = &o->nodes[id];
    for (int k = 0; k < 3; k++) { n->lo[k] = INFINITY; n->hi[k] = -INFINITY; }
    for (int i = first; i < first + count; i++) {
        double lo[3], hi[3];
        tri_bounds(o, o->order[i], lo, hi);
        for (int k = 0; k < 3; k++) {
            if (lo[k] < n->lo[k]) n->lo[k] = lo[k];
            if (hi[k] > n->hi[k]) n->hi[k] = hi[k];
        }
    }
    for (int k = 0; k < 3; k++) {   /* pad so that FP64 rounding never culls a hit */
        double m = fmax(fabs(n->lo[k]), fabs(n->hi[k])) * 1e-12 + 1e-300;
        n->lo[k] -= m; n->hi[k] += m;
    }
    n->left = n->right = -1;
    n->first = first; n->count = count;
    if (count <= 4) return id;
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; i++)
        for (int k = 0; k < 3; k++) {
            double c = cent[3 * o->order[i] + k];
            if (c < clo[k]) clo[k] = c;
            if (c > chi[k]) chi[k] = c;
        }
    int ax = 0;
    for (int k = 1; k < 3; k++) if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
    double *key = malloc(sizeof(double) * o->nt);
    for (int i = first; i < first + count; i++) key[o->order[i]] = cent[3 * o->order[i] + ax];
    g_sort_key = key;
    qsort(o->order + first, count, sizeof(int), cmp_key);
    free(key);
    int half = count / 2;
    int l = build_node(o, first, half, cent);
    int r = build_node(o, first + half, count - half, cent);
    o->nodes[id].left = l;
    o->nodes[id].right = r;
    o->nodes[id].count = 0;
    return id;
}

void *or_build(const or_scene *s)
{
    oracle_t *o = calloc(1, sizeof(oracle_t));
    o->s = *s;
    o->nt = s->nt;
    o->V0 = malloc(sizeof(v3) * (s->nt + 1));
    o->E1 = malloc(sizeof(v3) * (s->nt + 1));
    o->E2 = malloc(sizeof(v3) * (s->nt + 1));
    o->order = malloc(sizeof(int) * (s->nt + 1));
    double *cent = malloc(sizeof(double) * 3 * (s->nt + 1));
    for (int t = 0; t < s->nt; t++) {
        const float *a = s->verts + 3 * s->tris[3 * t], *b = s->verts + 3 * s->tris[3 * t + 1],
                    *c = s->verts + 3 * s->tris[3 * t + 2];
        v3 A = mk(a[0], a[1], a[2]), B = mk(b[0], b[1], b[2]), C = mk(c[0], c[1], c[2]);
        o->V0[t] = A; o->E1[t] = sub(B, A); o->E2[t] = sub(C, A);
        o->order[t] = t;
        for (int k = 0; k < 3; k++) cent[3 * t + k] = (comp(A, k) + comp(B, k) + comp(C, k)) / 3.0;
    }
    o->nodes = malloc(sizeof(bnode) * (2 * s->nt + 2));
    o->nn = 0;
    if (s->nt > 0) build_node(o, 0, s->nt, cent);
    free(cent);
    for (int l = 0; l < s->nl && l < 8; l++) {
        const float *L = s->lights + 12 * l;
        v3 eu = mk(L[3], L[4], L[5]), ev = mk(L[6], L[7], L[8]);
        v3 n = cross(eu, ev);
        o->light_area[l] = len(n);
        o->light_n[l] = nrm(n);
    }
    return o;
}

void or_free(void *h)
{
    oracle_t *o = h;
    if (!o) return;
    free(o->V0); free(o->E1); free(o->E2); free(o->order); free(o->nodes);
    free(o);
}

/* ------------------------------------------------------------------------ */
/* ray queries: plane intersection + barycentric inside test, FP64           */
/* ------------------------------------------------------------------------ */
typedef struct { double t; int tri; double b1, b2; int near; } hit_t;

static int tri_test(const oracle_t *o, int t, v3 org, v3 dir, double tmin, double tmax,
                    double *tt, double *b1, double *b2, double *margin)
{
    v3 n = cross(o->E1[t], o->E2[t]);
    double den = dot(n, dir);
    *tt = -INFINITY;
    *margin = -INFINITY;
    if (den == 0.0) return 0;
    double th = dot(n, sub(o->V0[t], org)) / den;
    *tt = th;
    if (!(th > tmin) || !(th < tmax)) return 0;
    v3 q = sub(add(org, scl(dir, th)), o->V0[t]);
    double nn = dot(n, n);
    double c1 = dot(cross(q, o->E2[t]), n) / nn;
    double c2 = dot(cross(o->E1[t], q), n) / nn;
    double c0 = 1.0 - c1 - c2;
    double m = fmin(c0, fmin(c1, c2));
    *margin = m;
    *tt = th; *b1 = c1; *b2 = c2;
    return m >= 0.0;
}

static int box_hit(const bnode *n, v3 org, v3 dir, double tmin, double tmax)
{
    double t0 = tmin, t1 = tmax;
    for (int k = 0; k < 3; k++) {
        double oc = comp(org, k), dc = comp(dir, k);
        if (dc == 0.0) {
            if (oc < n->lo[k] || oc > n->hi[k]) return 0;
            continue;
        }
        double a = (n->lo[k] - oc) / dc, b = (n->hi[k] - oc) / dc;
        if (a > b) { double x = a; a = b; b = x; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* closest hit with ties to the lower triangle id; 'skip' is excluded.
 * 'near' is set when a candidate at or before the final distance lies within
 * EDGE_FLAG of a triangle edge (these are the samples where a float32 kernel
 * may legitimately pick another triangle). */
static int closest(const oracle_t *o, v3 org, v3 dir, double tmin, double tmax, int skip,
                   int brute, hit_t *h)
{
    h->t = tmax; h->tri = -1; h->near = 0;
    double near_t = INFINITY;
    int stack[128], sp = 0;
    if (o->nn == 0) return 0;
    if (brute) {
        for (int t = 0; t < o->nt; t++) {
            if (t == skip) continue;
            double tt, b1, b2, m;
            int ok = tri_test(o, t, org, dir, tmin, INFINITY, &tt, &b1, &b2, &m);
            if (tt > tmin && fabs(m) < EDGE_FLAG && tt < near_t) near_t = tt;
            if (ok && (tt < h->t || (tt == h->t && t < h->tri))) { h->t = tt; h->tri = t; h->b1 = b1; h->b2 = b2; }
        }
    } else {
        stack[sp++] = 0;
        while (sp) {
            const bnode *n = &o->nodes[stack[--sp]];
            if (!box_hit(n, org, dir, tmin, h->t * (1.0 + 1e-9))) continue;
            if (n->count > 0) {
                for (int i = n->first; i < n->first + n->count; i++) {
                    int t = o->order[i];
                    if (t == skip) continue;
                    double tt, b1, b2, m;
                    int ok = tri_test(o, t, org, dir, tmin, INFINITY, &tt, &b1, &b2, &m);
                    if (tt > tmin && fabs(m) < EDGE_FLAG && tt < near_t) near_t = tt;
                    if (ok && tt < tmax && (tt < h->t || (tt == h->t && t < h->tri))) {
                        h->t = tt; h->tri = t; h->b1 = b1; h->b2 = b2;
                    }
                }
            } else {
                stack[sp++] = n->left;
                stack[sp++] = n->right;
            }
        }
    }
    if (h->tri >= 0 && near_t <= h->t * (1.0 + 1e-6)) h->near = 1;
    return h->tri >= 0;
}

/* any hit with tmin < t < tmax, skipping 'skip' */
static int occluded(const oracle_t *o, v3 org, v3 dir, double tmax, int skip, int64_t *nearf)
{
    int stack[128], sp = 0;
    if (o->nn == 0) return 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode *n = &o->nodes[stack[--sp]];
        if (!box_hit(n, org, dir, 0.0, tmax)) continue;
        if (n->count > 0) {
            for (int i = n->first; i < n->first + n->count; i++) {
                int t = o->order[i];
                if (t == skip) continue;
                double tt, b1, b2, m;
                int ok = tri_test(o, t, org, dir, 0.0, tmax, &tt, &b1, &b2, &m);
                if (tt > 0.0 && tt < tmax && fabs(m) < EDGE_FLAG) *nearf = 1;
                if (ok) return 1;
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    return 0;
}

int or_closest_hit(void *h, const double o_[3], const double d_[3], double tmin, double tmax,
                   int brute, double *t, int32_t *tri)
{
    hit_t hh;
    int r = closest((const oracle_t *)h, mk(o_[0], o_[1], o_[2]), mk(d_[0], d_[1], d_[2]), tmin, tmax,
                    -1, brute, &hh);
    *t = r ? hh.t : INFINITY;
    *tri = r ? hh.tri : -1;
    return r;
}

/* ------------------------------------------------------------------------ */
/* surface attributes at a hit                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    v3 p, ng, ns;       /* point, unit geometric normal (winding), unit shading normal */
    double u, v;        /* texture coordinates */
    int tri, mat;
} surf_t;

static surf_t surface(const oracle_t *o, int tri, v3 p, double b1, double b2)
{
    const or_scene *s = &o->s;
    surf_t S;
    S.p = p; S.tri = tri; S.mat = (int)s->tri_mat[tri];
    S.ng = nrm(cross(o->E1[tri], o->E2[tri]));
    double b0 = 1.0 - b1 - b2;
    const uint32_t *ix = s->tris + 3 * tri;
    v3 n = mk(0, 0, 0);
    double u = 0, v = 0, w[3] = {b0, b1, b2};
    for (int k = 0; k < 3; k++) {
        const float *nk = s->normals + 3 * ix[k];
        n = add(n, scl(mk(nk[0], nk[1], nk[2]), w[k]));
        u += w[k] * s->uvs[2 * ix[k]];
        v += w[k] * s->uvs[2 * ix[k] + 1];
    }
    S.ns = nrm(n);
    S.u = u; S.v = v;
    return S;
}

/* bilinear texture lookup, clamp to edge, texel centres at (i + 1/2)/w */
static double tex_lookup(const or_scene *s, int tex, double u, double v, int ch)
{
    const int32_t *ti = s->tex_info + 3 * tex;
    int off = ti[0], w = ti[1], hgt = ti[2];
    double x = u * w - 0.5, y = v * hgt - 0.5;
    double fx0 = floor(x), fy0 = floor(y);
    double fx = x - fx0, fy = y - fy0;
    int x0 = (int)fx0, y0 = (int)fy0, x1 = x0 + 1, y1 = y0 + 1;
    x0 = x0 < 0 ? 0 : (x0 > w - 1 ? w - 1 : x0);
    x1 = x1 < 0 ? 0 : (x1 > w - 1 ? w - 1 : x1);
    y0 = y0 < 0 ? 0 : (y0 > hgt - 1 ? hgt - 1 : y0);
    y1 = y1 < 0 ? 0 : (y1 > hgt - 1 ? hgt - 1 : y1);
    const float *d = s->tex_data + off;
    double a = d[(y0 * w + x0) * 3 + ch], b = d[(y0 * w + x1) * 3 + ch];
    double c = d[(y1 * w + x0) * 3 + ch], e = d[(y1 * w + x1) * 3 + ch];
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + e * fx) * fy;
}

static double albedo(const or_scene *s, const surf_t *S, int ch)
{
    double a = s->mat_albedo[3 * S->mat + ch];
    int t = s->mat_tex[S->mat];
    return t >= 0 ? a * tex_lookup(s, t, S->u, S->v, ch) : a;
}

/* emitted radiance toward wo; one-sided (front = winding normal side) */
static double emitted(const or_scene *s, const surf_t *S, v3 wo, int ch)
{
    double Le = s->mat_Le[3 * S->mat + ch];
    if (Le == 0.0 || dot(wo, S->ng) <= 0.0) return 0.0;
    if (s->mat_emit_tex[S->mat] && s->mat_tex[S->mat] >= 0)
        Le *= tex_lookup(s, s->mat_tex[S->mat], S->u, S->v, ch);
    return Le;
}

/* trilinear lookup in the ambient cache, values at cell centres */
static double cache_lookup(const or_scene *s, v3 p, int ch)
{
    int R = s->cache_res;
    double g[3], f[3];
    int i0[3], i1[3];
    for (int k = 0; k < 3; k++) {
        double lo = s->cache_bmin[k], hi = s->cache_bmax[k];
        g[k] = (comp(p, k) - lo) / (hi - lo) * R - 0.5;
        double fl = floor(g[k]);
        f[k] = g[k] - fl;
        int a = (int)fl, b = a + 1;
        i0[k] = a < 0 ? 0 : (a > R - 1 ? R - 1 : a);
        i1[k] = b < 0 ? 0 : (b > R - 1 ? R - 1 : b);
    }
    double acc = 0.0;
    for (int c = 0; c < 8; c++) {
        int ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
        double w = ((c & 1) ? f[0] : 1 - f[0]) * ((c & 2) ? f[1] : 1 - f[1]) * ((c & 4) ? f[2] : 1 - f[2]);
        acc += w * or_half_to_double(s->cache_E[(((size_t)iz * R + iy) * R + ix) * 3 + ch]);
    }
    return acc;
}

/* the two lookups of a built scene, exposed for the pins */
double or_tex_lookup(void *h, int32_t tex, double u, double v, int32_t ch)
{
    const oracle_t *o = h;
    return tex_lookup(&o->s, tex, u, v, ch);
}

double or_cache_lookup(void *h, const double p[3], int32_t ch)
{
    const oracle_t *o = h;
    return cache_lookup(&o->s, mk(p[0], p[1], p[2]), ch);
}

/* ------------------------------------------------------------------------ */
/* BSDFs                                                                     */
/* ------------------------------------------------------------------------ */
/* orthonormal basis around a unit normal (Duff et al., JCGT 2017) */
void or_frame(const double n[3], double t[3], double b[3])
{
    double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double c = n[0] * n[1] * a;
    t[0] = 1.0 + sg * n[0] * n[0] * a; t[1] = sg * c; t[2] = -sg * n[0];
    b[0] = c; b[1] = sg + n[1] * n[1] * a; b[2] = -n[1];
}

typedef struct { v3 t, b, n; } frame_t;
static frame_t make_frame(v3 n)
{
    double nn[3] = {n.x, n.y, n.z}, t[3], b[3];
    or_frame(nn, t, b);
    frame_t F = {mk(t[0], t[1], t[2]), mk(b[0], b[1], b[2]), n};
    return F;
}
static v3 to_local(const frame_t *F, v3 w) { return mk(dot(w, F->t), dot(w, F->b), dot(w, F->n)); }
static v3 to_world(const frame_t *F, v3 w) { return add(add(scl(F->t, w.x), scl(F->b, w.y)), scl(F->n, w.z)); }

/* unpolarised Fresnel reflectance of a smooth dielectric interface */
double or_fresnel_dielectric(double cos_i, double n_i, double n_t)
{
    double eta = n_i / n_t;
    double s2 = eta * eta * (1.0 - cos_i * cos_i);
    if (s2 >= 1.0) return 1.0;
    double cos_t = sqrt(1.0 - s2);
    double rs = (n_i * cos_i - n_t * cos_t) / (n_i * cos_i + n_t * cos_t);
    double rp = (n_t * cos_i - n_i * cos_t) / (n_t * cos_i + n_i * cos_t);
    return 0.5 * (rs * rs + rp * rp);
}

/* GGX (Trowbridge-Reitz) normal distribution, local frame, h unit */
static double ggx_D(double alpha, v3 h)
{
    if (h.z <= 0.0) return 0.0;
    double a2 = alpha * alpha;
    double q = (h.x * h.x + h.y * h.y) / a2 + h.z * h.z;
    return 1.0 / (PI * a2 * q * q);
}

/* Smith masking for GGX: G1 = 1 / (1 + Lambda) */
static double ggx_G1(double alpha, v3 w)
{
    if (w.z <= 0.0) return 0.0;
    double t2 = (w.x * w.x + w.y * w.y) / (w.z * w.z);
    double lam = 0.5 * (-1.0 + sqrt(1.0 + alpha * alpha * t2));
    return 1.0 / (1.0 + lam);
}

static double schlick(double F0, double c)
{
    double m = 1.0 - c;
    return F0 + (1.0 - F0) * m * m * m * m * m;
}

/* f and the visible-normal sampling pdf, local frame (Heitz, JCGT 2018) */
void or_ggx_eval(double alpha, double F0, const double wo_[3], const double wi_[3], double *f, double *pdf)
{
    v3 wo = mk(wo_[0], wo_[1], wo_[2]), wi = mk(wi_[0], wi_[1], wi_[2]);
    *f = 0.0; *pdf = 0.0;
    if (wo.z <= 0.0 || wi.z <= 0.0) return;
    v3 h = nrm(add(wo, wi));
    double D = ggx_D(alpha, h);
    double G1o = ggx_G1(alpha, wo), G1i = ggx_G1(alpha, wi);
    double F = schlick(F0, dot(wi, h));
    *f = F * D * G1o * G1i / (4.0 * wo.z * wi.z);
    *pdf = G1o * D / (4.0 * wo.z);
}

/* sample a visible normal, reflect; weight = f cos / pdf = F * G1(wi) */
int or_ggx_sample(double alpha, double F0, const double wo_[3], double u0, double u1,
                  double wi_[3], double *weight, double *pdf)
{
    v3 wo = mk(wo_[0], wo_[1], wo_[2]);
    *weight = 0.0; *pdf = 0.0;
    if (wo.z <= 0.0) return 0;
    v3 vh = nrm(mk(alpha * wo.x, alpha * wo.y, wo.z));
    double l2 = vh.x * vh.x + vh.y * vh.y;
    v3 T1 = l2 > 0.0 ? scl(mk(-vh.y, vh.x, 0.0), 1.0 / sqrt(l2)) : mk(1.0, 0.0, 0.0);
    v3 T2 = cross(vh, T1);
    double rr = sqrt(u0), ph = 2.0 * PI * u1;
    double t1 = rr * cos(ph), t2 = rr * sin(ph);
    double sm = 0.5 * (1.0 + vh.z);
    t2 = (1.0 - sm) * sqrt(1.0 - t1 * t1) + sm * t2;
    double tz = sqrt(fmax(0.0, 1.0 - t1 * t1 - t2 * t2));
    v3 nh = add(add(scl(T1, t1), scl(T2, t2)), scl(vh, tz));
    v3 ne = nrm(mk(alpha * nh.x, alpha * nh.y, fmax(0.0, nh.z)));
    double c = dot(wo, ne);
    v3 wi = sub(scl(ne, 2.0 * c), wo);
    wi_[0] = wi.x; wi_[1] = wi.y; wi_[2] = wi.z;
    if (wi.z <= 0.0) return 0;
    *weight = schlick(F0, dot(wi, ne)) * ggx_G1(alpha, wi);
    *pdf = ggx_G1(alpha, wo) * ggx_D(alpha, ne) / (4.0 * wo.z);
    return 1;
}

/* BSDF value (times nothing) and pdf for a non-delta material, world frame */
static void bsdf_eval(const or_scene *s, const surf_t *S, v3 ns, v3 wo, v3 wi, int ch, double *f, double *pdf)
{
    int type = s->mat_type[S->mat];
    double a = albedo(s, S, ch);
    *f = 0.0; *pdf = 0.0;
    if (type == M_LAMBERT) {
        double c = dot(wi, ns);
        if (c <= 0.0) return;
        *f = a / PI;
        *pdf = c / PI;
    } else if (type == M_GGX) {
        frame_t F = make_frame(ns);
        v3 lo = to_local(&F, wo), li = to_local(&F, wi);
        double r = s->mat_rough[S->mat];
        double wo_[3] = {lo.x, lo.y, lo.z}, wi_[3] = {li.x, li.y, li.z};
        or_ggx_eval(r * r, a, wo_, wi_, f, pdf);
    }
}

/* ------------------------------------------------------------------------ */
/* Stage s1: uniform direction in the SLM diffraction cone (Sec. 4.1, 4.2)   */
/* theta_max = asin(lambda / 2p); 1 - cos(theta) = u0 * 2 sin^2(theta_max/2) */
/* ------------------------------------------------------------------------ */
void or_cone_dir(double lambda, double pitch, double u0, double u1, double d[3], double *pdf)
{
    double thmax = asin(lambda / (2.0 * pitch));
    double sh = sin(0.5 * thmax);
    double h = 2.0 * sh * sh;           /* 1 - cos(theta_max) without cancellation */
    double s = u0 * h;                  /* 1 - cos(theta) */
    double ct = 1.0 - s;
    double st = sqrt(s * (2.0 - s));
    double ph = 2.0 * PI * u1;
    d[0] = st * cos(ph);
    d[1] = st * sin(ph);
    d[2] = ct;
    *pdf = 1.0 / (2.0 * PI * h);
}

/* rigid transform helpers: T maps world to hologram space (Eq. 3) */
static v3 xf_point(const double T[16], v3 p)
{
    return mk(T[0] * p.x + T[1] * p.y + T[2] * p.z + T[3], T[4] * p.x + T[5] * p.y + T[6] * p.z + T[7],
              T[8] * p.x + T[9] * p.y + T[10] * p.z + T[11]);
}
static v3 inv_xf_point(const double T[16], v3 q)   /* R^T (q - t) */
{
    v3 d = mk(q.x - T[3], q.y - T[7], q.z - T[11]);
    return mk(T[0] * d.x + T[4] * d.y + T[8] * d.z, T[1] * d.x + T[5] * d.y + T[9] * d.z,
              T[2] * d.x + T[6] * d.y + T[10] * d.z);
}
static v3 inv_xf_dir(const double T[16], v3 d)
{
    return mk(T[0] * d.x + T[4] * d.y + T[8] * d.z, T[1] * d.x + T[5] * d.y + T[9] * d.z,
              T[2] * d.x + T[6] * d.y + T[10] * d.z);
}

/* ------------------------------------------------------------------------ */
/* Stage s5: incoherent radiance at the real image point P (Eq. 1)           */
/* path tracing with next-event estimation to rectangular lights and         */
/* power-heuristic MIS; every vertex counts toward max_depth.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const oracle_t *o;
    const or_render *r;
    int lam, ch, s;
    int64_t pix;
    int64_t flags;
    int nrays;
    int want_cond;   /* estimate the conditioning of the incoherent part (flags bit 4, sens) */
    double dA, Lmax; /* last sample: bound on |sqrt(L') - sqrt(L)| under float32-sized moves of
                        P, and the largest L' the probes saw */
    double sens;     /* pixel: bound on the field change from its delta-chain samples */
} ctx_t;

static double light_pdf_at(const oracle_t *o, int li, double dist, double cos_l)
{
    return dist * dist / (cos_l * o->light_area[li]) / (double)o->s.nl;
}

static double radiance(ctx_t *C, surf_t S, v3 wo, int v)
{
    const oracle_t *o = C->o;
    const or_scene *s = &o->s;
    const or_render *r = C->r;
    const int ch = C->ch;
    double L = 0.0, beta = 1.0, prev_pdf = 0.0, t_prev = 0.0;
    int prev_delta = 1, first = 1;
    for (;;) {
        int type = s->mat_type[S.mat];
        /* emission, MIS-weighted when the previous vertex also sampled this light */
        double Le = emitted(s, &S, wo, ch);
        if (Le > 0.0) {
            double w = 1.0;
            int li = s->mat_light[S.mat];
            if (!prev_delta && type == M_EMITTER && li >= 0 && s->nl > 0) {
                double cl = dot(wo, o->light_n[li]);
                double pl = light_pdf_at(o, li, t_prev, cl);
                w = prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);
            }
            L += beta * Le * w;
        }
        if (type == M_EMITTER) break;

        /* orient normals toward the side wo comes from */
        v3 ng = S.ng, ns = S.ns;
        int front = dot(wo, ng) > 0.0;
        v3 wi;
        double u[4];
        path_draw(r, C->lam, C->pix, C->s, v, 0, u);
        if (type == M_MIRROR || type == M_DIELECTRIC) {
            if (v >= r->max_depth) break;
            C->flags |= 2;   /* the incoherent path met a mirror or dielectric */
            if (type == M_MIRROR) {
                if (!front) { ng = scl(ng, -1); ns = scl(ns, -1); }
                double c = dot(wo, ns);
                if (c <= 0.0) break;
                wi = sub(scl(ns, 2.0 * c), wo);
                if (dot(wi, ng) <= 0.0) break;
                beta *= albedo(s, &S, ch);
            } else {
                double ior = s->mat_ior[S.mat];
                double n_i = front ? 1.0 : ior, n_t = front ? ior : 1.0;
                v3 n = front ? ns : scl(ns, -1);
                v3 g = front ? ng : scl(ng, -1);
                double ci = dot(wo, n);
                if (ci <= 0.0) break;
                double F = or_fresnel_dielectric(ci, n_i, n_t);
                if (u[0] < F) {
                    wi = sub(scl(n, 2.0 * ci), wo);
                    if (dot(wi, g) <= 0.0) break;
                } else {
                    double eta = n_i / n_t;
                    double ct = sqrt(1.0 - eta * eta * (1.0 - ci * ci));
                    wi = add(scl(wo, -eta), scl(n, eta * ci - ct));
                    if (dot(wi, g) >= 0.0) break;
                    beta *= eta * eta;
                }
            }
            prev_delta = 1;
        } else {
            if (!front) { ng = scl(ng, -1); ns = scl(ns, -1); }
            if (dot(wo, ns) <= 0.0) break;
            if (r->use_cache && s->cache_res > 0 && !first) {
                /* ambient cache past the first bounce: Lambertian read-out of cached irradiance */
                L += beta * albedo(s, &S, ch) / PI * cache_lookup(s, S.p, ch);
                break;
            }
            v3 org = add(S.p, scl(ng, INC_OFFSET));
            /* next-event estimation */
            if (s->nl > 0) {
                int li = 0;
                if (s->nl > 1) {
                    double u2[4];
                    path_draw(r, C->lam, C->pix, C->s, v, 1, u2);
                    li = (int)(u2[0] * s->nl);
                    if (li >= s->nl) li = s->nl - 1;
                }
                const float *Lr = s->lights + 12 * li;
                v3 y = add(add(mk(Lr[0], Lr[1], Lr[2]), scl(mk(Lr[3], Lr[4], Lr[5]), u[0])),
                           scl(mk(Lr[6], Lr[7], Lr[8]), u[1]));
                v3 dvec = sub(y, org);
                double dist = len(dvec);
                v3 wl = scl(dvec, 1.0 / dist);
                double cl = -dot(wl, o->light_n[li]);
                double Ll = Lr[9 + ch];
                if (cl > 0.0 && dot(wl, ng) > 0.0 && dot(wl, ns) > 0.0 && Ll > 0.0) {
                    double f, pb;
                    bsdf_eval(s, &S, ns, wo, wl, ch, &f, &pb);
                    double pl = light_pdf_at(o, li, dist, cl);
                    if (f > 0.0) {
                        C->nrays++;
                        /* power heuristic only when a BSDF continuation exists (v < max_depth) */
                        double wm = v < r->max_depth ? pl * pl / (pl * pl + pb * pb) : 1.0;
                        if (!occluded(o, org, wl, dist * (1.0 - SHADOW_SHRINK), S.tri, &C->flags))
                            L += beta * f * dot(wl, ns) * Ll * wm / pl;
                    }
                }
            }
            if (v >= r->max_depth) break;
            /* BSDF sampling */
            double pb;
            if (type == M_LAMBERT) {
                frame_t F = make_frame(ns);
                double rr = sqrt(u[2]), ph = 2.0 * PI * u[3];
                double z = sqrt(1.0 - u[2]);
                wi = to_world(&F, mk(rr * cos(ph), rr * sin(ph), z));
                if (dot(wi, ng) <= 0.0) break;
                beta *= albedo(s, &S, ch);
                pb = z / PI;
            } else { /* GGX */
                frame_t F = make_frame(ns);
                v3 lo = to_local(&F, wo);
                double wo_[3] = {lo.x, lo.y, lo.z}, wi_[3], wgt;
                double rg = s->mat_rough[S.mat];
                if (!or_ggx_sample(rg * rg, albedo(s, &S, ch), wo_, u[2], u[3], wi_, &wgt, &pb)) break;
                wi = to_world(&F, mk(wi_[0], wi_[1], wi_[2]));
                if (dot(wi, ng) <= 0.0) break;
                beta *= wgt;
            }
            prev_delta = 0;
            prev_pdf = pb;
        }
        /* continue the incoherent path */
        v3 org = add(S.p, scl(dot(wi, S.ng) > 0.0 ? S.ng : scl(S.ng, -1), INC_OFFSET));
        hit_t h;
        C->nrays++;
        if (!closest(o, org, wi, 0.0, INFINITY, S.tri, 0, &h)) break;
        if (h.near) C->flags |= 1;
        v++;
        t_prev = h.t;
        wo = scl(wi, -1);
        S = surface(o, h.tri, add(org, scl(wi, h.t)), h.b1, h.b2);
        first = 0;
    }
    return L;
}

/* Conditioning of the incoherent part of a sample.
 * The incoherent radiance L(P) is evaluated in float32 by a fast path, so the
 * question is how much a rounding-sized change of the image point P moves L.
 * Mostly it barely does, but reflection and refraction at curved mirrors and
 * lenses (and near-specular GGX) magnify a displacement of the incoming ray,
 * so after a few of them a later hit can move across a texture or lighting
 * gradient, or the path can change branch.  Two probes, with the same random
 * numbers:
 *   - P moved by COND_STEP (relative to |P|, about one float32 ulp) along both
 *     tangents: the local sensitivity; the sample is ill-conditioned when the
 *     relative change of L exceeds COND_KAPPA times the relative step;
 *   - P moved by COND_SPREAD steps the other way along both tangents: branch
 *     changes within the reach of float32 rounding, which the local probe misses.
 * The amplitude change sqrt(L') - sqrt(L), the local one scaled by COND_SPREAD,
 * bounds what the sample may contribute to a disagreement; it is capped by
 * sqrt(L) + sqrt(L'max), the change when the path flips to the neighbouring
 * branch.  COND_SPREAD is the float32 budget of an incoherent path expressed as a
 * move of its image point: the rounding of P to float32 (half an ulp), then at
 * each of at most three incoherent vertices (depth 4) a few ulps of direction
 * error (square root, sine and cosine, frame) carried over a hit distance of
 * the order of |P|, and a few ulps of hit-point error: about 10 ulps per vertex,
 * 32 in all. */
#define COND_STEP   1.2e-7
#define COND_KAPPA  30.0
#define COND_SPREAD 32.0

static int sample_ill_conditioned(ctx_t *C, surf_t S, v3 wo, int v, double L)
{
    double t[3], b[3], n[3] = {S.ng.x, S.ng.y, S.ng.z};
    or_frame(n, t, b);
    double scale = fmax(fabs(S.p.x), fmax(fabs(S.p.y), fabs(S.p.z)));
    int64_t flags = C->flags;
    int nrays = C->nrays;
    int ill = 0;
    double dlin = 0.0, dbig = 0.0, a0 = sqrt(fmax(L, 0.0));
    C->Lmax = L;
    for (int k = 0; k < 4; k++) {
        const double *d = (k & 1) ? b : t;
        const double e = k < 2 ? COND_STEP * scale : -COND_SPREAD * COND_STEP * scale;
        surf_t S2 = S;
        S2.p = add(S.p, scl(mk(d[0], d[1], d[2]), e));
        double L2 = radiance(C, S2, wo, v);
        double da = fabs(sqrt(fmax(L2, 0.0)) - a0);
        if (k < 2) {
            if (fabs(L2 - L) > COND_KAPPA * COND_STEP * fmax(fabs(L), 1e-300)) ill = 1;
            dlin = fmax(dlin, COND_SPREAD * da);
        } else {
            dbig = fmax(dbig, da);
        }
        C->Lmax = fmax(C->Lmax, L2);
    }
    C->dA = fmax(dlin, dbig);
    C->flags = flags;
    C->nrays = nrays;
    return ill;
}

/* ------------------------------------------------------------------------ */
/* One coherent sample: stages s1-s9 of Sec. 4 for pixel 'pix', sample 's'.  */
/* Returns 1 and fills the sample record when the path reaches a real image */
/* point P, 0 when it contributes nothing (miss, depth exhausted).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double A, beta, L, opl, r, cos_t, cos_p, base, sens;
    double qx, qy;   /* Q on the hologram plane */
    v3 P;
    int vP, tri;
    int64_t cell[3];
} samp_t;

static int coherent_sample(ctx_t *C, samp_t *out)
{
    const oracle_t *o = C->o;
    const or_scene *s = &o->s;
    const or_render *r = C->r;
    const double lambda = r->lambda[C->lam];
    const int64_t W = r->W, H = r->H;
    const int64_t i = C->pix % W, j = C->pix / W;
    /* s1: pixel centre and a direction in the cone */
    v3 x = mk(((double)i + 0.5 - 0.5 * (double)W) * r->pitch, ((double)j + 0.5 - 0.5 * (double)H) * r->pitch, 0.0);
    double u[4], dh[3], pdf_w;
    path_draw(r, C->lam, C->pix, C->s, 0, 0, u);
    or_cone_dir(lambda, r->pitch, u[0], u[1], dh, &pdf_w);
    /* s2: to world space */
    v3 O = inv_xf_point(r->T, x);
    v3 vdir = inv_xf_dir(r->T, mk(dh[0], dh[1], dh[2]));
    v3 org = O, dir = vdir;
    double opl = 0.0, n_cur = 1.0, beta = 1.0;
    int v = 0, skip = -1;
    /* s3/s4: coherent delta chain, accumulating OPL = sum n_i L_i */
    for (;;) {
        hit_t h;
        C->nrays++;
        if (!closest(o, org, dir, skip < 0 ? 0.0 : COH_TMIN, INFINITY, skip, 0, &h)) return 0;
        if (h.near) C->flags |= 1;
        v++;
        v3 P = add(org, scl(dir, h.t));
        opl += n_cur * h.t;
        surf_t S = surface(o, h.tri, P, h.b1, h.b2);
        int type = s->mat_type[S.mat];
        if (type != M_MIRROR && type != M_DIELECTRIC) {
            /* P: first non-delta hit = the real image point */
            v3 wo = scl(dir, -1);
            double L = radiance(C, S, wo, v);
            int cond = C->want_cond;
            if (cond && sample_ill_conditioned(C, S, wo, v, L)) C->flags |= 4;
            /* s6: virtual image point P' = O + d_OPL v, Q = T P' */
            v3 Pv = add(O, scl(vdir, opl));
            v3 Q = xf_point(r->T, Pv);
            v3 rq = sub(Q, x);
            double rr = len(rq);
            double cos_t = rq.z / rr;
            double cos_p = fabs(dot(dir, S.ng));
            out->beta = beta;
            out->L = L;
            out->A = sqrt(beta * L);
            out->opl = opl;
            out->r = rr;
            out->cos_t = cos_t;
            out->cos_p = cos_p;
            /* RS estimator (Eq. 2) with the area-measure pdf of the sampled point */
            double pdf_A = pdf_w * cos_p / (rr * rr);
            out->base = out->A * (r->omit_obliquity ? 1.0 : cos_t) / (rr * pdf_A * lambda);
            out->sens = 0.0;
            if (cond) {
                double g = sqrt(beta) * fabs(cos_t) / (rr * pdf_A * lambda);
                out->sens = g * fmin(C->dA, sqrt(fmax(L, 0.0)) + sqrt(C->Lmax));
            }
            out->qx = Q.x;
            out->qy = Q.y;
            out->P = P;
            out->vP = v;
            out->tri = h.tri;
            double inv_h = 1.0 / r->facet_size;
            out->cell[0] = (int64_t)floor(P.x * inv_h);
            out->cell[1] = (int64_t)floor(P.y * inv_h);
            out->cell[2] = (int64_t)floor(P.z * inv_h);
            return 1;
        }
        if (v >= r->max_depth) return 0;
        v3 ng = S.ng, ns = S.ns, wo = scl(dir, -1), wi;
        int front = dot(wo, ng) > 0.0;
        if (type == M_MIRROR) {
            if (!front) { ng = scl(ng, -1); ns = scl(ns, -1); }
            double c = dot(wo, ns);
            if (c <= 0.0) return 0;
            wi = sub(scl(ns, 2.0 * c), wo);
            if (dot(wi, ng) <= 0.0) return 0;
            beta *= albedo(s, &S, C->ch);
        } else {
            double ior = s->mat_ior[S.mat];
            double n_i = front ? 1.0 : ior, n_t = front ? ior : 1.0;
            v3 n = front ? ns : scl(ns, -1);
            v3 g = front ? ng : scl(ng, -1);
            double ci = dot(wo, n);
            if (ci <= 0.0) return 0;
            double F = or_fresnel_dielectric(ci, n_i, n_t);
            path_draw(r, C->lam, C->pix, C->s, v, 0, u);
            if (u[0] < F) {
                wi = sub(scl(n, 2.0 * ci), wo);
                if (dot(wi, g) <= 0.0) return 0;
            } else {
                double eta = n_i / n_t;
                double ct = sqrt(1.0 - eta * eta * (1.0 - ci * ci));
                wi = add(scl(wo, -eta), scl(n, eta * ci - ct));
                if (dot(wi, g) >= 0.0) return 0;
                beta *= eta * eta;
                n_cur = n_t;
            }
        }
        org = P;
        dir = wi;
        skip = h.tri;
    }
}

/* deterministic point emitters: a e^{ikr} cos(theta) / r inside the cone, if unoccluded */
static void point_field(ctx_t *C, double *re, double *im)
{
    const oracle_t *o = C->o;
    const or_scene *s = &o->s;
    const or_render *r = C->r;
    const double lambda = r->lambda[C->lam];
    const int64_t W = r->W, H = r->H;
    const int64_t i = C->pix % W, j = C->pix / W;
    v3 x = mk(((double)i + 0.5 - 0.5 * (double)W) * r->pitch, ((double)j + 0.5 - 0.5 * (double)H) * r->pitch, 0.0);
    v3 O = inv_xf_point(r->T, x);
    double cos_max = cos(asin(lambda / (2.0 * r->pitch)));
    *re = *im = 0.0;
    for (int e = 0; e < s->npts; e++) {
        const double *pe = s->points + 4 * e;
        v3 pw = mk(pe[0], pe[1], pe[2]);
        v3 q = sub(xf_point(r->T, pw), x);
        double rr = len(q);
        double ct = q.z / rr;
        if (ct < cos_max) continue;
        v3 dw = sub(pw, O);
        double dist = len(dw);
        int64_t nf = 0;
        if (occluded(o, O, scl(dw, 1.0 / dist), dist * (1.0 - SHADOW_SHRINK), -1, &nf)) continue;
        double turns = fmod(rr / lambda, 1.0);
        double a = pe[3] * (r->omit_obliquity ? 1.0 : ct) / rr;
        *re += a * cos(2.0 * PI * turns);
        *im += a * sin(2.0 * PI * turns);
    }
}

/* one pixel and wavelength: U_m for all m (Eq. 5, Path Reuse) */
static void pixel_field(ctx_t *C, double *ure, double *uim)
{
    const or_render *r = C->r;
    const int K = r->K;
    const double lambda = r->lambda[C->lam];
    for (int m = 0; m < K; m++) ure[m] = uim[m] = 0.0;
    for (int s = 0; s < r->spp; s++) {
        samp_t S;
        C->s = s;
        int64_t fl0 = C->flags;
        C->flags = 0;
        int ok = coherent_sample(C, &S);
        /* per pixel, 16 bits each: samples near a triangle edge or tie, ill-conditioned samples,
           samples whose incoherent path went through a mirror or dielectric */
        C->flags = fl0 + ((C->flags & 1) ? 1 : 0) + ((C->flags & 4) ? ((int64_t)1 << 16) : 0) +
                   ((C->flags & 2) ? ((int64_t)1 << 32) : 0);
        if (ok) C->sens += S.sens;
        if (!ok || S.base == 0.0) continue;
        double turns_r = fmod(S.r / lambda, 1.0);
        for (int m = 0; m < K; m++) {
            double ph = 0.0;
            if (r->phase_mode == 0) ph = phase_draw(r, C->lam, S.cell, r->hologram_offset + m);
            else if (r->phase_mode == 2) ph = grf_phase(r, S.qx, S.qy, m);
            double t = turns_r + ph;
            /* (1/(i lambda)) folded into base; multiply by -i */
            double c = cos(2.0 * PI * t), sn = sin(2.0 * PI * t);
            ure[m] += S.base * sn;
            uim[m] += -S.base * c;
        }
    }
    for (int m = 0; m < K; m++) { ure[m] /= r->spp; uim[m] /= r->spp; }
    C->sens /= r->spp;
    double pre, pim;
    point_field(C, &pre, &pim);
    for (int m = 0; m < K; m++) { ure[m] += pre; uim[m] += pim; }
}

int or_sample(void *h, const or_render *r, int lam, int64_t pixel, int s, double *rec)
{
    const oracle_t *o = h;
    if (r->phase_mode == 2 && (!r->grf_phi || r->grf_nx < 1 || r->grf_ny < 1)) return -1;
    ctx_t C = {o, r, lam, r->channel[lam], s, pixel, 0, 0, 1, 0.0, 0.0, 0.0};
    samp_t S;
    memset(&S, 0, sizeof S);
    memset(rec, 0, sizeof(double) * OR_REC_N);
    int ok = coherent_sample(&C, &S);
    double u[4];
    path_draw(r, lam, pixel, s, 0, 0, u);
    rec[OR_REC_U0] = u[0];
    rec[OR_REC_FLAGS] = C.flags;
    rec[OR_REC_NRAYS] = C.nrays;
    if (!ok) { rec[OR_REC_TRI] = -1; return 0; }
    rec[OR_REC_L] = S.L; rec[OR_REC_BETA] = S.beta; rec[OR_REC_OPL] = S.opl; rec[OR_REC_R] = S.r;
    rec[OR_REC_COS] = S.cos_t; rec[OR_REC_COSP] = S.cos_p; rec[OR_REC_VP] = S.vP;
    rec[OR_REC_PX] = S.P.x; rec[OR_REC_PY] = S.P.y; rec[OR_REC_PZ] = S.P.z; rec[OR_REC_TRI] = S.tri;
    double ph = r->phase_mode == 0 ? phase_draw(r, lam, S.cell, r->hologram_offset)
              : r->phase_mode == 2 ? grf_phase(r, S.qx, S.qy, 0) : 0.0;
    rec[OR_REC_QX] = S.qx;
    rec[OR_REC_QY] = S.qy;
    double t = fmod(S.r / r->lambda[lam], 1.0) + ph;
    rec[OR_REC_RE] = S.base * sin(2.0 * PI * t);
    rec[OR_REC_IM] = -S.base * cos(2.0 * PI * t);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* threaded driver                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const oracle_t *o;
    const or_render *r;
    const int64_t *pixels;
    int64_t n;
    double *out;
    int64_t *flags;
    double *sens;
    int64_t next;
    pthread_mutex_t mu;
} job_t;

static void *worker(void *arg)
{
    job_t *J = arg;
    const or_render *r = J->r;
    double ure[64], uim[64];
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t w = J->next;
        J->next += 16;
        pthread_mutex_unlock(&J->mu);
        int64_t total = J->n * r->n_lambda;
        if (w >= total) break;
        int64_t end = w + 16 < total ? w + 16 : total;
        for (int64_t it = w; it < end; it++) {
            int lam = (int)(it / J->n);
            int64_t pi = it % J->n;
            ctx_t C = {J->o, r, lam, r->channel[lam], 0, J->pixels[pi], 0, 0, J->flags != NULL || J->sens != NULL,
                       0.0, 0.0, 0.0};
            pixel_field(&C, ure, uim);
            for (int m = 0; m < r->K; m++) {
                double *d = J->out + 2 * (((int64_t)lam * r->K + m) * J->n + pi);
                d[0] = ure[m];
                d[1] = uim[m];
            }
            if (J->flags) J->flags[(int64_t)lam * J->n + pi] = C.flags;
            if (J->sens) J->sens[(int64_t)lam * J->n + pi] = C.sens;
        }
    }
    return NULL;
}

int or_trace(void *h, const or_render *r, const int64_t *pixels, int64_t n_pixels,
             double *out, int64_t *flags, double *sens, int n_threads)
{
    if (!h || !r || r->K < 1 || r->K > 64 || r->n_lambda < 1 || r->n_lambda > 3 || r->spp < 1) return -1;
    if (r->phase_mode == 2 && (!r->grf_phi || r->grf_nx < 1 || r->grf_ny < 1)) return -1;
    for (int64_t i = 0; i < n_pixels; i++)
        if (pixels[i] < 0 || pixels[i] >= (int64_t)r->W * r->H) return -2;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    job_t J;
    memset(&J, 0, sizeof J);
    J.o = h; J.r = r; J.pixels = pixels; J.n = n_pixels; J.out = out; J.flags = flags; J.sens = sens;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t th[256];
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, worker, &J);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ambient cache construction (see oracle.h)                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const oracle_t *o;
    const or_bake_desc *b;
    or_render r;
    const int64_t *cells;
    int64_t n;
    double *E;
    double *sens;    /* optional [n][3]: sensitivity bound of each cell-channel */
    int64_t next;
    pthread_mutex_t mu;
} bake_job_t;

/* radiance arriving at x from direction d (the first hit's incoherent radiance towards x), 0 on a miss */
static double bake_sample(bake_job_t *J, v3 x, v3 d, int c, int64_t pix, int s)
{
    hit_t h;
    if (!closest(J->o, x, d, 0.0, INFINITY, -1, 0, &h)) return 0.0;
    surf_t S = surface(J->o, h.tri, add(x, scl(d, h.t)), h.b1, h.b2);
    ctx_t C = {J->o, &J->r, c, c, s, pix, 0, 0, 0, 0.0, 0.0, 0.0};
    return radiance(&C, S, scl(d, -1.0), 1);
}

static void bake_cell(bake_job_t *J, int64_t cell, double E[3], double sens[3])
{
    const or_bake_desc *b = J->b;
    const int64_t R = b->res;
    const int64_t ix = cell % R, iy = (cell / R) % R, iz = cell / (R * R);
    const int64_t idx[3] = {ix, iy, iz};
    double xc[3];
    for (int k = 0; k < 3; k++) xc[k] = b->bmin[k] + ((double)idx[k] + 0.5) * (b->bmax[k] - b->bmin[k]) / (double)R;
    const v3 x = mk(xc[0], xc[1], xc[2]);
    const int64_t pix = (iy + R * iz) * R + ix;
    const double scale = fmax(fabs(x.x), fmax(fabs(x.y), fabs(x.z)));
    for (int c = 0; c < 3; c++) {
        double acc = 0.0, dev = 0.0;
        for (int s = 0; s < b->spp; s++) {
            double u[4];
            path_draw(&J->r, c, pix, s, 0, 0, u);
            const double ct = 1.0 - 2.0 * u[0], st = 2.0 * sqrt(u[0] * (1.0 - u[0]));
            const v3 d = mk(st * cos(2.0 * PI * u[1]), st * sin(2.0 * PI * u[1]), ct);
            const double L = bake_sample(J, x, d, c, pix, s);
            acc += L;
            if (sens) {
                /* the sample's change when its start point moves by +-COND_SPREAD float32 ulps
                   along two directions across the ray (the float32 budget of the path) */
                double t3[3], b3[3], n3[3] = {d.x, d.y, d.z};
                or_frame(n3, t3, b3);
                double m = 0.0;
                for (int k = 0; k < 4; k++) {
                    const double *e = (k & 1) ? b3 : t3;
                    const double step = ((k & 2) ? -1.0 : 1.0) * COND_SPREAD * COND_STEP * scale;
                    const v3 x2 = add(x, scl(mk(e[0], e[1], e[2]), step));
                    m = fmax(m, fabs(bake_sample(J, x2, d, c, pix, s) - L));
                }
                dev += m;
            }
        }
        E[c] = PI * acc / (double)b->spp;
        if (sens) sens[c] = PI * dev / (double)b->spp;
    }
}

static void *bake_worker(void *arg)
{
    bake_job_t *J = arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t w = J->next;
        J->next += 8;
        pthread_mutex_unlock(&J->mu);
        if (w >= J->n) break;
        int64_t end = w + 8 < J->n ? w + 8 : J->n;
        for (int64_t i = w; i < end; i++) bake_cell(J, J->cells[i], J->E + 3 * i, J->sens ? J->sens + 3 * i : NULL);
    }
    return NULL;
}

int or_bake(void *h, const or_bake_desc *b, const int64_t *cells, int64_t n_cells, double *E, int n_threads)
{
    return or_bake_sens(h, b, cells, n_cells, E, NULL, n_threads);
}

int or_bake_sens(void *h, const or_bake_desc *b, const int64_t *cells, int64_t n_cells, double *E, double *sens,
                 int n_threads)
{
    if (!h || !b || b->res < 1 || b->spp < 1 || b->max_depth < 1) return -1;
    for (int64_t i = 0; i < n_cells; i++)
        if (cells[i] < 0 || cells[i] >= (int64_t)b->res * b->res * b->res) return -2;
    bake_job_t J;
    memset(&J, 0, sizeof J);
    J.o = h; J.b = b; J.cells = cells; J.n = n_cells; J.E = E; J.sens = sens;
    J.r.W = b->res; J.r.H = b->res * b->res; J.r.n_lambda = 3;
    for (int c = 0; c < 3; c++) J.r.channel[c] = c;
    J.r.spp = b->spp; J.r.max_depth = b->max_depth; J.r.K = 1; J.r.seed = b->seed;
    J.r.phase_mode = 1; J.r.use_cache = 0;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, bake_worker, &J);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);
    return 0;
}
