// Internal layouts shared by the host runtime and the device kernels of the wave path tracer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hpt {

constexpr int KMAX = 8;            // holograms per path set (Path Reuse)
#ifndef HPT_LANES
#define HPT_LANES 3   // wave lanes of a trace by default (path-state sets rotating over streams)
#endif
#define HPT_MAX_LANES 4   // most wave lanes a trace may use (hpt_autotune chooses 1 .. 4)
#ifndef HPT_TSTACK
#define HPT_TSTACK 32
#endif
constexpr int TSTACK = HPT_TSTACK; // most traversal stack entries per thread (shared memory)
// the first BVH nodes are laid out breadth-first from the root (the rest depth-first): the
// levels every ray visits first share a few KB of cache lines
constexpr int TOP_ORDER = 255;
constexpr int TRACE_BLOCK = 128;   // threads per block of the trace kernel
constexpr int SHADE_BLOCK = 128;
constexpr int GEN_BLOCK = 256;
constexpr int ACCUM_BLOCK = 128;
constexpr int MAX_JOBS = 64;       // jobs (requests) of one launch group
constexpr int MAX_SEG = 16;        // job segments of one wave
constexpr int MAX_ITER = 66;       // trace/shade iterations of a wave: max_depth + 1 <= 65
constexpr int TILE_W = 8, TILE_H = 4;

// status bits written by the kernels
enum : uint32_t { ST_STACK_OVERFLOW = 1u, ST_BAD_JOB = 2u, ST_FALLBACK_STACK = 4u, ST_BOUNDS = 8u };

// The checked build (-DHPT_CHECKED=1, a separate library for tests): device indices into the
// path state, the queues, the BVH and the triangle arrays are checked before use; a failing
// check sets ST_BOUNDS in the status word and the access is skipped.  In the product build the
// checks compile to nothing.
#ifndef HPT_CHECKED
#define HPT_CHECKED 0
#endif
#define HPT_IN(i, n) (!HPT_CHECKED || (unsigned)(i) < (unsigned)(n))

// A constant needed by the coherent chain in both arithmetics: the double value and
// its double-float split (hi = rn(x), lo = rn(x - hi)).
struct RC {
    double d;
    float hi, lo;
};

struct alignas(16) MatDev {
    int kind, tex, emit_tex, light;
    float albedo[3];
    float rough;
    float ior;
    float Le[3];
};

struct alignas(16) LightDev {
    float corner[3], eu[3], ev[3], Le[3];
    float n[3];       // unit normal (eu x ev)
    float area;
};

// Per-triangle record for the high-precision refinement (indexed by the input triangle id):
// plane n . x = d0 with n = e1 x e2 (unnormalised), and the rows m1, m2 that give the
// barycentrics b1 = m1 . (x - v0), b2 = m2 . (x - v0) of a point on the plane.
constexpr int REF_N = 10;   // n.xyz, d0, m1.xyz, m2.xyz

struct DevScene {
    const float4 *nodes;      // 4 float4 per BVH2 node (child boxes + child links)
    int bvh_depth;            // inner levels above the deepest leaf: traversal stack entries needed
    const float4 *tri4;       // 3 float4 per triangle in leaf order: (v0, id), e1, e2
    // a second tree of the same triangles for the pixels' first rays (along +z of the hologram
    // plane, within the diffraction cone), with its own leaf-order records
    const float4 *nodes_p, *tri4_p;
    int n_nodes_p, n_tri4_p, bvh_depth_p;
    const double *ref64;      // [nt][REF_N]
    const float2 *refdf;      // [nt][REF_N] (hi, lo)
    const uint4 *tri_attr;    // [nt] vertex indices i0, i1, i2, material
    const float4 *tri_ng;     // [nt] unit geometric normal (winding)
    const float *verts;       // [nv][3]
    const float *normals;     // [nv][3]
    const float *uvs;         // [nv][2]
    const MatDev *mats;
    const float *tex;
    const int *tex_info;      // [ntex][3]
    const LightDev *lights;
    const double *points;     // [np][4]
    const unsigned short *cache;   // binary16 [res][res][res][3]
    float cache_bmin[3], cache_bmax[3];
    int cache_res;
    int n_tris, n_nodes, n_lights, n_points;
    int n_tri4;               // triangle records in leaf order (the non-degenerate triangles)
};

struct DevJob {
    DevScene sc;
    float2 *out;                // [n_lambda][K][H][W]
    long long n_items;          // n_lambda * n_tiles * 32
    int W, H, n_lambda, spp, max_depth, K, hologram_offset, phase_mode, use_cache;
    int t_identity;
    int n_tiles_x, n_tiles;
    int channel[3];
    unsigned seed_lo, seed_hi, pseed_lo, pseed_hi;
    float lambda_f[3];
    float pdf_w[3];             // 1 / (2 pi (1 - cos theta_max))
    float cos_max[3];           // cos theta_max (float) for the point-emitter cone mask
    RC lambda[3];
    RC inv_lambda[3];
    RC h_cone[3];               // 1 - cos theta_max = 2 sin^2(theta_max / 2)
    RC pitch;
    RC inv_facet;
    RC R[9];                    // rotation of T (world -> hologram), row-major
    RC t[3];                    // translation of T
    const float4 *sincos_tab;   // cos/sin(2 pi k / 256) as (hi, lo) float pairs, 256 entries
    const float *grf;           // phase mode 2: [K][grf_ny][grf_nx] radians
    int grf_nx, grf_ny;
    RC inv_pitch;
    // kind 1: ambient-cache bake; items are (channel, cell) with the cells laid out as a
    // W = res by H = res^2 image, each path an incoherent ray from the cell centre
    int kind;
    int obliquity;              // 1: cos(theta) of Eq. 2 applied, 0: omitted
    float *bake_out;            // [res^3][3] float
    float bake_lo[3], bake_h[3];
};

struct JobTable {
    int n_jobs;
    int pad;
    DevJob jobs[MAX_JOBS];
};

// A wave: consecutive work items of up to MAX_SEG jobs, with all their samples.  Path p of a
// segment with n items is sample s = (p - path_offset) / n of item item_begin + (p - path_offset) % n.
struct WaveSeg {
    int job;
    int spp;
    long long item_begin;
    int item_count;
    int path_offset;
};

struct WaveDesc {
    int n_seg;
    int n_paths;
    int n_items;
    int stack_n;      // traversal stack entries per thread of the trace kernels (<= TSTACK)
    WaveSeg seg[MAX_SEG];
};

// Structure-of-arrays state of the paths of one wave (capacity paths each).  The coherent
// quantities are 8-byte slots holding a double or a double-float (hi, lo) pair.
struct PathBufs {
    // coherent origin o, direction d, optical path length, as 8-byte slots (double or (hi, lo)
    // floats) packed in 16-byte units: (o.x, o.y), (o.z, d.x), (d.y, d.z), then OPL alone
    uint4 *cs0, *cs1, *cs2;
    uint2 *cs3;
    float4 *coh4;                        // medium index, delta-chain throughput, cos(theta) of the sample,
                                         // coherent vertex count (int bits)
    float4 *inc;                         // incoherent state: radiance L, throughput, last BSDF pdf, last distance
    float2 *inc2;                        // pending NEE contribution, vertex count | flags (int bits)
    float4 *ray_o, *ray_d, *sh_d;        // float ray (origin | tmax, direction | skip), shadow direction | tmax
    float4 *hit;                         // t, u, v, triangle
    int *occl;                           // shadow ray blocked
    float *amp, *fturn, *basep;          // sample record: amplitude factor, frac(r / lambda), estimator weight
    int *cx, *cy, *cz;                   // facet cell of the real image point
    int *q[3][2];                        // queues (coherent, incoherent, shadow) x ping-pong
    int capacity;
};

// traversal stack entries per thread for a BVH of the given depth (inner levels above the
// deepest leaf): a near-first traversal holds at most one entry per level; one spare
inline int stack_entries(int bvh_depth) { return bvh_depth + 1 < 2 ? 2 : (bvh_depth + 1 > TSTACK ? TSTACK : bvh_depth + 1); }
// stack entries for the deeper of a scene's two trees
inline int scene_stack_entries(const DevScene &s) { return stack_entries(s.bvh_depth > s.bvh_depth_p ? s.bvh_depth : s.bvh_depth_p); }

// device-side scratch of one launch slot
struct SlotScratch {
    unsigned int status;            // error bits (sticky until read by hpt_sync)
    unsigned int pad;
    unsigned long long counters[8];
    int qcount[MAX_ITER + 1][3];    // queue lengths per iteration
};

}  // namespace hpt
