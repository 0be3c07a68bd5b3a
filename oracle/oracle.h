/* FP64 CPU oracle of the wave path tracer (test infrastructure only).
 *
 * Plain, slow, double-precision restatement of the method of
 * "HoloPathTracer: Fast and Accurate Wave Path Tracing for Holography"
 * (ACM TOG 45(4), 2026): the nine stages of Sec. 4, the wave-facet model of
 * Sec. 4.1, the coherent/incoherent split and virtual image point of Sec. 4.2,
 * the Path-Reuse accumulation of Eq. 5 (Sec. 4.3), the rendering equation
 * (Eq. 1) for the incoherent amplitude and the Rayleigh-Sommerfeld integral
 * (Eq. 2) as the estimator the per-pixel sum computes.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA library.
 */
#ifndef HPT_ORACLE_H
#define HPT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nv, nt, nm, ntex, nl, npts;
    const float *verts;      /* [nv][3] metres                          */
    const float *normals;    /* [nv][3] per-vertex shading normals      */
    const float *uvs;        /* [nv][2]                                 */
    const uint32_t *tris;    /* [nt][3]                                 */
    const uint32_t *tri_mat; /* [nt]                                    */
    const int32_t *mat_type; /* [nm] 0 lambert 1 ggx 2 mirror 3 dielectric 4 emitter */
    const float *mat_albedo; /* [nm][3] */
    const float *mat_rough;  /* [nm]    */
    const float *mat_ior;    /* [nm]    */
    const float *mat_Le;     /* [nm][3] */
    const int32_t *mat_tex;  /* [nm]    */
    const int32_t *mat_emit_tex; /* [nm] */
    const int32_t *mat_light;    /* [nm] */
    const float *tex_data;   /* texels, RGB row-major */
    const int32_t *tex_info; /* [ntex][3] offset, w, h */
    const float *lights;     /* [nl][12] corner, edge_u, edge_v, Le */
    const double *points;    /* [npts][4] position, amplitude */
    int32_t cache_res;
    const float *cache_bmin, *cache_bmax; /* [3] */
    const uint16_t *cache_E; /* [res][res][res][3] IEEE binary16 bits */
} or_scene;

typedef struct {
    int32_t W, H;
    double pitch;
    int32_t n_lambda;
    double lambda[3];
    int32_t channel[3];
    int32_t spp, max_depth, K, hologram_offset;
    uint64_t seed, phase_seed;
    int32_t phase_mode;      /* 0 hashed facet phase, 1 zero phase */
    double facet_size;
    double T[16];            /* world -> hologram, row-major, rigid */
    int32_t use_cache;
    int32_t grf_nx, grf_ny;  /* phase_mode 2: periodic GRF phase grid (pitch = the SLM pitch) */
    const double *grf_phi;   /* [K][grf_ny][grf_nx] radians, hologram_offset + m for map m */
    int32_t omit_obliquity;  /* 1: leave out the cos(theta) factor of Eq. 2 */
} or_render;

/* per-sample debug record (or_sample) */
enum { OR_REC_L, OR_REC_BETA, OR_REC_OPL, OR_REC_R, OR_REC_COS, OR_REC_COSP, OR_REC_VP,
       OR_REC_PX, OR_REC_PY, OR_REC_PZ, OR_REC_TRI, OR_REC_FLAGS, OR_REC_RE, OR_REC_IM,
       OR_REC_NRAYS, OR_REC_U0, OR_REC_QX, OR_REC_QY, OR_REC_N };

void *or_build(const or_scene *s);
void or_free(void *h);
/* phase_mode: 0 hashed facet phase, 1 zero phase, 2 GRF phase maps (Eq. 4) sampled at the
 * image point's hologram-plane position Q.
 * out: [n_lambda][K][n_pixels][2] complex128.  flags (optional): [n_lambda][n_pixels], three
 * 16-bit sample counts: bits 0-15 samples with a ray query near a triangle edge or tie; bits
 * 16-31 samples whose incoherent part is ill-conditioned (a rounding-sized move of the image
 * point changes its radiance by more than 30x as much, relatively); bits 32-47 samples whose
 * incoherent path met a mirror or dielectric.  sens (optional): [n_lambda][n_pixels], a bound
 * on how far float32-sized moves of the image points can change |U_m| (the same for every m;
 * the phase of a sample does not depend on its radiance).  Conditioning is only estimated
 * when flags or sens are requested.  or_sample's record flags: bit 0 near edge, bit 1 delta
 * in the incoherent path, bit 2 ill-conditioned.  Returns 0 or <0. */
int or_trace(void *h, const or_render *r, const int64_t *pixels, int64_t n_pixels,
             double *out, int64_t *flags, double *sens, int n_threads);
int or_sample(void *h, const or_render *r, int lam, int64_t pixel, int s, double *rec);

/* Ambient cache construction (texture baking, Sec. 4.4; the paper's supplementary S1.4 is not
 * available, this is the reading): for cell (ix, iy, iz) of a res^3 grid over [bmin, bmax],
 * centre x = bmin + (i + 0.5) (bmax - bmin) / res, and channel c,
 *   E_c(x) = pi / spp * sum_s L_c(y_s -> x),
 * directions w_s uniform on the sphere (cos theta = 1 - 2 u0, phi = 2 pi u1 from the path draw of
 * vertex 0 at pixel index (iy + res iz) res + ix, sample s, wavelength index c), y_s the first hit
 * along w_s, L_c the incoherent radiance leaving y_s towards x (emission at full weight, NEE + BSDF
 * with MIS, vertices counted from 1 at y_s up to max_depth, no cache); a miss gives 0.  For
 * isotropic incident radiance this is the irradiance (pi L).  cells: linear indices
 * (iz res + iy) res + ix; E: [n_cells][3].  Returns 0 or < 0. */
typedef struct {
    int32_t res;
    double bmin[3], bmax[3];
    int32_t spp, max_depth;
    uint64_t seed;
} or_bake_desc;
int or_bake(void *h, const or_bake_desc *b, const int64_t *cells, int64_t n_cells, double *E, int n_threads);
/* or_bake plus sens [n_cells][3]: for each cell-channel, pi / spp times the sum over its
 * directions of the largest change of the arriving radiance when the cell centre moves by 32
 * float32 ulps (of its largest coordinate) along either of two directions across the ray, up or
 * down -- the float32 budget of a GPU path, as for the trace's sensitivity bound. */
int or_bake_sens(void *h, const or_bake_desc *b, const int64_t *cells, int64_t n_cells, double *E, double *sens,
                 int n_threads);

/* building blocks exposed for the pins */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_cone_dir(double lambda, double pitch, double u0, double u1, double d[3], double *pdf);
int or_closest_hit(void *h, const double o[3], const double d[3], double tmin, double tmax,
                   int brute, double *t, int32_t *tri);
/* bilinear texture lookup (clamp to edge, texel centres at (i + 1/2) / w) and trilinear
 * ambient-cache lookup (values at cell centres, [z][y][x][c]) of the scene built into h */
double or_tex_lookup(void *h, int32_t tex, double u, double v, int32_t ch);
double or_cache_lookup(void *h, const double p[3], int32_t ch);
double or_fresnel_dielectric(double cos_i, double n_i, double n_t);
void or_ggx_eval(double alpha, double F0, const double wo[3], const double wi[3], double *f, double *pdf);
int or_ggx_sample(double alpha, double F0, const double wo[3], double u0, double u1,
                  double wi[3], double *weight, double *pdf);
void or_frame(const double n[3], double t[3], double b[3]);
double or_half_to_double(uint16_t h);
/* Eq. 4: the random spectral phases xi_m(fx, fy) of GRF map m on an nx x ny frequency grid in
 * FFT order, row-major [ny][nx]: xi = 2 pi u24(Philox4x32-10(ix, iy, m, 0x47524600; seed)). */
void or_grf_phases(uint64_t seed, int32_t m, int32_t nx, int32_t ny, double *xi);

#ifdef __cplusplus
}
#endif
#endif
