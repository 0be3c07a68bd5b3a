/* hpt.h -- C-ABI of the GB300 wave path tracer.
 *
 * The library computes, for every pixel of a spatial light modulator (SLM) and
 * every wavelength, K complex fields U_m (m = 0..K-1) by Monte Carlo wave path
 * tracing, following "HoloPathTracer: Fast and Accurate Wave Path Tracing for
 * Holography" (ACM TOG 45(4), 2026):
 *
 *   - Sec. 4 (nine stages s1-s9): a ray leaves the pixel centre in a random
 *     direction inside the SLM diffraction cone theta <= asin(lambda / 2p)
 *     (Sec. 4.1), is mapped to world space by T^-1 (Eq. 3), follows delta
 *     (mirror / smooth dielectric) lobes coherently while accumulating the
 *     optical path length OPL = sum n_i L_i (Sec. 4.2) and stops at the first
 *     non-delta hit, the real image point P;
 *   - the amplitude at P is sqrt(L), L estimated by incoherent path tracing of
 *     the rendering equation (Eq. 1) with next-event estimation, and, past the
 *     first bounce, optionally read from an ambient radiance cache (Sec. 4.2);
 *   - the virtual image point P' = O + d_OPL v is mapped back by Q = T P' and
 *     its contribution (1/(i lambda)) sqrt(L) cos(theta) / (r pdf_A)
 *     * exp(i (2 pi r / lambda + phi_m)) is summed into U_m, the Monte Carlo
 *     estimate of the Rayleigh-Sommerfeld integral (Eq. 2);
 *   - Path Reuse (Eq. 5, Sec. 4.3): all K holograms share one path set and
 *     differ only in the random facet phase phi_m.
 *
 * Conventions for every entry point:
 *   - units are SI metres; all arrays are row-major and tightly packed;
 *   - host pointers are only read during the call; the library copies what it
 *     keeps; device pointers (out_dev) are owned by the caller;
 *   - calls return HPT_OK (0) or a negative status, never throw, and leave a
 *     message for hpt_last_error();
 *   - one context serves one CUDA device; calls on one context may come from
 *     several host threads (they are serialised internally).
 */
#ifndef HPT_H
#define HPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hpt_status;
enum {
    HPT_OK = 0,
    HPT_ERR_INVALID_ARG = -1,   /* bad pointer, size, NaN/Inf input, out-of-range index   */
    HPT_ERR_OOM = -2,           /* device allocation failed or budget exceeded            */
    HPT_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the cause)     */
    HPT_ERR_TIMEOUT = -4,       /* hpt_wait ran out of time                               */
    HPT_ERR_BUSY = -5,          /* serving queue full / admission refused                 */
    HPT_ERR_NOT_FOUND = -6,     /* unknown scene or request id                            */
    HPT_ERR_UNSUPPORTED = -7,   /* valid request outside what this build supports         */
    HPT_ERR_DEVICE = -8,        /* the kernel reported an internal error (status word)    */
    HPT_ERR_CANCELLED = -9      /* the request was cancelled (hpt_cancel)                 */
};

/* material kinds (Sec. 4.2: mirror and dielectric are delta lobes, the rest non-delta) */
enum { HPT_LAMBERT = 0, HPT_GGX = 1, HPT_MIRROR = 2, HPT_DIELECTRIC = 3, HPT_EMITTER = 4 };
enum { HPT_PHASE_HASH = 0, HPT_PHASE_ZERO = 1, HPT_PHASE_GRF = 2 };
/* arithmetic of the coherent chain (ray origin/direction, hit distance, OPL, phase):
 * FP64 = native double; DF32 = double-float (unevaluated sum of two floats, ~48-bit mantissa) */
enum { HPT_PREC_FP64 = 0, HPT_PREC_DF32 = 1 };

typedef struct hpt_ctx hpt_ctx;

/* context flags */
enum {
    HPT_CTX_NO_GRAPHS = 1,          /* hpt_trace launches every kernel instead of replaying frames   */
    HPT_CTX_FAIL_SERVING_WAVES = 2  /* for tests of the failure path: every serving wave fails to be
                                       issued as if its wave state could not be allocated (OOM)     */
};

typedef struct {
    uint64_t hbm_budget_bytes;  /* serving admission limit for in-flight outputs; 0 = 60 % of
                                   the free HBM at creation                                   */
    int32_t max_inflight;       /* serving: requests admitted and not finished (0 -> 8)       */
    int32_t flags;              /* HPT_CTX_* bits                                              */
    int32_t max_queue;          /* serving: requests waiting for admission before hpt_submit
                                   answers HPT_ERR_BUSY (0 -> 4096)                            */
    int32_t reserved;           /* 0                                                           */
} hpt_ctx_desc;

/* Scene description.  All arrays are host memory, read during hpt_scene_upload only.
 *  verts    float[nv][3]   vertex positions (float32 values; the geometry is exactly these)
 *  normals  float[nv][3]   per-vertex shading normals (interpolated, renormalised)
 *  uvs      float[nv][2]   texture coordinates
 *  tris     uint32[nt][3]  vertex indices; winding gives the geometric normal (e1 x e2)
 *  tri_mat  uint32[nt]     material index
 *  materials: kind, albedo (mirror reflectance / GGX F0 / Lambert albedo), GGX roughness
 *    (alpha = roughness^2), index of refraction, emitted radiance Le (one-sided, toward the
 *    winding normal), albedo texture id (-1 none), emit_tex (Le scaled by the texture),
 *    light (rectangular light this EMITTER surface belongs to, -1 none)
 *  textures: float RGB texels, row-major, tex_info[i] = {offset in floats, width, height};
 *    sampled bilinearly with clamp-to-edge, texel centres at (i + 1/2) / width
 *  lights   float[nl][12]  rectangular lights for next-event estimation:
 *    corner, edge_u, edge_v, Le; they emit toward edge_u x edge_v
 *  points   double[np][4]  deterministic point emitters (position, amplitude a); each adds
 *    a exp(i k r) cos(theta) / r to every hologram of the pixels whose cone contains it
 *  cache    optional ambient radiance cache: res^3 cells over [bmin, bmax], binary16 RGB
 *    irradiance at cell centres, layout [z][y][x][c], read trilinearly                      */
typedef struct {
    int32_t kind;
    float albedo[3];
    float roughness;
    float ior;
    float Le[3];
    int32_t tex;
    int32_t emit_tex;
    int32_t light;
} hpt_material;

typedef struct {
    int32_t nv, nt, nm, ntex, nl, np;
    const float *verts;
    const float *normals;
    const float *uvs;
    const uint32_t *tris;
    const uint32_t *tri_mat;
    const hpt_material *materials;
    const float *tex_data;
    int64_t tex_floats;
    const int32_t *tex_info;
    const float *lights;
    const double *points;
    int32_t cache_res;
    float cache_bmin[3], cache_bmax[3];
    const uint16_t *cache_E;
} hpt_scene_desc;

/* Render description (one hologram set).
 *  W, H, pitch   SLM size in pixels and pixel pitch (m); pixel (i, j) centre is
 *                ((i + 1/2 - W/2) p, (j + 1/2 - H/2) p, 0) in hologram space, normal +z
 *  lambda[c]     wavelengths (m), n_lambda <= 3; channel[c] = RGB channel of the scene read
 *  spp           coherent samples per pixel and wavelength (N)
 *  max_depth     scattering vertices per path (delta vertices included); >= 1
 *  K             holograms from one path set (Path Reuse), 1..8; hologram_offset shifts m
 *  seed          key of the path draws; phase_seed key of the facet phases
 *  phase_mode    HPT_PHASE_HASH: phi_m uniform in [0, 2 pi) per facet cell (edge
 *                facet_size, world space) and hologram; HPT_PHASE_ZERO: phi_m = 0;
 *                HPT_PHASE_GRF: phi_m = grf_phi[m][jy][jx], the band-limited Gaussian
 *                random field of Eq. 4 (hpt_grf_build) at the image point's hologram-plane
 *                position Q = (x_Q, y_Q): jx = floor(x_Q / pitch + grf_nx / 2) mod grf_nx,
 *                likewise jy (m counts from 0 for hologram hologram_offset)
 *  T             world -> hologram transform, row-major 4x4, must be rigid
 *  precision     HPT_PREC_FP64 or HPT_PREC_DF32 (coherent chain arithmetic)
 *  use_cache     read the scene's ambient cache past the first incoherent bounce
 *  grf_phi       HPT_PHASE_GRF only: device pointer, float radians [K][grf_ny][grf_nx],
 *                caller-owned, must stay valid until the trace completes; else NULL
 *  omit_obliquity 0: the obliquity factor cos(theta) of Eq. 2 is applied (default);
 *                1: left out (a point emitter then gives exactly a exp(ikr) / r)           */
typedef struct {
    int32_t W, H;
    double pitch;
    int32_t n_lambda;
    double lambda[3];
    int32_t channel[3];
    int32_t spp, max_depth, K, hologram_offset;
    uint64_t seed, phase_seed;
    int32_t phase_mode;
    double facet_size;
    double T[16];
    int32_t precision;
    int32_t use_cache;
    const float *grf_phi;
    int32_t grf_nx, grf_ny;
    int32_t omit_obliquity;
} hpt_render_desc;

/* Output layout of every trace: complex64 (float re, float im) [n_lambda][K][H][W];
 * out_bytes must be >= 8 * n_lambda * K * H * W. */

/* Create a context on CUDA device 'device'. desc may be NULL (defaults). */
hpt_status hpt_create(hpt_ctx **ctx, int device, const hpt_ctx_desc *desc);
/* Finish all work, free every device allocation of the context. ctx may be NULL. */
void hpt_destroy(hpt_ctx *ctx);
/* Message of the last failing call on this thread ("" if none). Valid until the next call. */
const char *hpt_last_error(void);

/* Copy a scene to the device and build its BVHs (binned SAH over the triangles; a second tree
 * of the same triangles, its SAH weighting the box faces across the hologram plane's z axis, is
 * walked by the pixels' first rays); *scene_id receives a handle. Synchronous. */
hpt_status hpt_scene_upload(hpt_ctx *ctx, const hpt_scene_desc *scene, uint64_t *scene_id);
/* Free a scene after all work using it has finished. */
hpt_status hpt_scene_release(hpt_ctx *ctx, uint64_t scene_id);
/* Bytes of device memory the scene occupies (both BVHs, triangles, attributes, textures, cache);
 * n_nodes and bvh_depth describe the tree of the rays in every direction. */
hpt_status hpt_scene_info(hpt_ctx *ctx, uint64_t scene_id, uint64_t *device_bytes,
                          int32_t *n_nodes, int32_t *bvh_depth);

/* Trace one render description into the caller's device buffer, asynchronously on
 * 'cuda_stream' (a cudaStream_t, NULL = legacy default stream).  All wavelengths and all K
 * holograms are produced by one launch group (waves of generate / trace / shade / accumulate
 * kernels).  The first call with a given launch shape (arithmetic, out_dev, SLM size x
 * wavelengths, spp, max_depth) captures the frame as a CUDA graph; later calls replay it (up to
 * 8 shapes are kept, least recently used first out).  Calls on one context are serialised on
 * one internal stream, linked to cuda_stream by events. */
hpt_status hpt_trace(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                     void *out_dev, size_t out_bytes, void *cuda_stream);
/* Same, end to end with host memory: the result is copied into out_host (pinned or pageable)
 * before the call returns.  Uses a device buffer owned by the context.  Into pinned memory
 * (cudaHostAlloc / cudaHostRegister) the rows of the fields are copied as the waves that
 * complete them finish, on a stream of the context, overlapping the rest of the trace (the
 * frame then runs without a captured graph); into pageable memory the whole frame runs first
 * and one copy follows.  The fields are the same either way. */
hpt_status hpt_trace_host(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                          void *out_host, size_t out_bytes, void *cuda_stream);
/* Block until all work queued by this context has finished; then report (and clear) the
 * kernel status word: HPT_OK, or HPT_ERR_DEVICE with the cause in hpt_last_error(). */
hpt_status hpt_sync(hpt_ctx *ctx);

/* Per-path-sample work counters of one trace (synchronous; for roofline accounting).
 * counters[0..HPT_NCOUNTERS-1]: path samples, rays, box tests, triangle tests,
 * coherent refinements, FP64 fallback traversals, NEE shadow rays, BSDF bounces.
 * The trace runs on separately compiled counting kernels: the fields they write to out_dev
 * meet the parity tolerance but may differ from hpt_trace's in the last bits (the counter
 * updates change the code around them, and with it where the compiler fuses multiply-adds),
 * and through such a rounding difference an incoherent path may occasionally take another
 * branch. */
enum { HPT_NCOUNTERS = 8 };
hpt_status hpt_trace_counters(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                              void *out_dev, size_t out_bytes, uint64_t counters[HPT_NCOUNTERS]);

/* Trace one frame like hpt_trace, without a captured graph, with a CUDA event recorded on the
 * context's wave stream before every launch, and report the device time and number of kernel
 * launches per kernel kind: HPT_K_GEN (primary path generation, with the queue-counter reset),
 * HPT_K_TRACE (BVH traversal of one queue iteration: two launches, coherent rays and incoherent /
 * shadow rays), HPT_K_SHADE (coherent and incoherent shading of one iteration: two launches),
 * HPT_K_ACCUM (Path-Reuse accumulation, Eq. 5).
 * Synchronous; the results in out_dev equal those of hpt_trace.  The paper has no counterpart:
 * this feeds the roofline of each kernel. */
enum { HPT_K_GEN = 0, HPT_K_TRACE = 1, HPT_K_SHADE = 2, HPT_K_ACCUM = 3, HPT_NKERNELS = 4 };
hpt_status hpt_trace_timed(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                           void *out_dev, size_t out_bytes, float kernel_ms[HPT_NKERNELS],
                           uint32_t launches[HPT_NKERNELS]);

/* Launch-shape autotuner (the paper has no counterpart).  Times hpt_trace of a band of 'desc'
 * (its first rows, about 50 M path samples, all wavelengths, spp and K as given) under candidate
 * launch shapes and keeps the fastest, by coordinate descent from the current shape:
 *   paths_per_wave       wave size, 2 M .. 16 M paths (within half of the free HBM);
 *   lanes                wave lanes (path-state sets on their own streams), 1 .. 4;
 *   trace_blocks_per_sm  resident blocks of the trace kernel x 1, 2 or 4 per SM in its grid;
 *   shade_blocks_per_sm  the same for the shading kernels.
 * A candidate replaces the current choice only when it is faster by more than 1 %.  The result
 * is applied to the context (reallocating the wave state and dropping captured frames when the
 * wave size or lane count changes) and kept for the scene's size class (triangle count < 4 k,
 * < 64 k, < 1 M, larger); later hpt_trace / hpt_trace_host calls on a scene of a tuned class
 * switch to that class's shape first.  Results of traces do not depend on the launch shape.
 * Synchronous; *out receives the choice (out may be NULL).  Serving waves keep their own shape. */
enum { HPT_SCENE_CLASSES = 4 };
typedef struct {
    int32_t paths_per_wave;
    int32_t lanes;
    int32_t trace_blocks_per_sm;
    int32_t shade_blocks_per_sm;
    int32_t scene_class;
    int32_t candidates;        /* launch shapes timed */
    double band_ms;            /* band time of the choice (best of the timed repetitions) */
    double band_ms_start;      /* band time of the shape the context had before the call */
    int64_t band_path_samples; /* path samples of the band */
} hpt_tuning;
hpt_status hpt_autotune(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, hpt_tuning *out);

/* ---- wave optics around the tracer: GRF phase maps and angular-spectrum propagation ---- */
/* Eq. 4 (Sec. 4.3): for m = hologram_offset .. hologram_offset + K - 1, the band-limited
 * Gaussian random field r_m = F^-1{ chi exp(i xi_m) } on a periodic nx x ny grid of the given
 * pitch, chi the circular passband |f| <= sin(theta_max)/lambda = 1/(2 pitch) (frequencies
 * kx/(nx pitch), ky/(ny pitch) in FFT order, inside when 4 (kx^2 ny^2 + ky^2 nx^2) <=
 * nx^2 ny^2), xi_m = 2 pi u24(Philox4x32-10(kx mod nx, ky mod ny, m, 0x47524600; phase_seed)),
 * and writes phi_m = arg r_m in radians, float [K][ny][nx], to phi_dev (caller-owned device
 * memory, 4 K nx ny bytes).  nx, ny: powers of two, 2 .. 8192.  Runs on 'stream' (NULL: the
 * legacy default stream); its scratch (8 nx ny bytes and the twiddle tables) comes from the
 * device's stream-ordered pool and is released on the stream.  The paper's own numbers for the
 * grid are not given: the caller chooses it to cover the image points' hologram positions
 * (the field is periodic). */
hpt_status hpt_grf_build(hpt_ctx *ctx, uint64_t phase_seed, int32_t hologram_offset, int32_t K,
                         int32_t nx, int32_t ny, double pitch, float *phi_dev, void *stream);

/* Angular spectrum method (Sec. 3, "Angular Spectrum of Wave Field"; the two-stage scheme of
 * Sec. 5): propagate each of the n_lambda * K complex64 fields [n_lambda][K][H][W] in in_dev
 * by z metres (light travelling from the recording plane towards the SLM: z > 0) and write
 * them to out_dev (same layout; may equal in_dev).  Each field is zero-padded to Wp x Hp,
 * the next powers of two of at least 2W and 2H (centred at ((Wp - W)/2, (Hp - H)/2)), its
 * spectrum multiplied by exp(i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2)) (0 where the root is
 * imaginary), transformed back and cropped to the original window.  lambdas: host array of
 * n_lambda wavelengths (m).  Wp, Hp <= 8192.  Asynchronous on 'stream'.  The zero padding is
 * never stored: the scratch, from the device's stream-ordered pool and released on the
 * stream, is 8 (min(K, 8) Wp H + n_lambda Wp Hp + Wp + Hp) bytes (the K fields of a
 * wavelength go through in groups of up to 8; their spectra stay row-major, the column
 * transforms read and write them in place). */
hpt_status hpt_asm_propagate(hpt_ctx *ctx, const void *in_dev, void *out_dev, int32_t W, int32_t H,
                             int32_t n_lambda, int32_t K, const double *lambdas, double pitch, double z,
                             void *stream);

/* Phase-only encoding with complex supervision (Sec. 2, Sec. 5 "Phase-only Hologram
 * Encoding"): 'iters' gradient steps phi <- phi - lr dL/dphi on the SLM phase phi_dev (float
 * [H][W] radians, device, read as the start and overwritten), L = sum |s A - T|^2 with
 * A = ASM_z(exp(i phi)) (the padded propagation of hpt_asm_propagate), T = target_dev
 * (complex64 [H][W], device) and s = <A, T> / <A, A> the phase-shift-invariant complex scale;
 * dL/dphi = -2 Im(exp(i phi) conj(ASM_-z(conj(s) (s A - T)))).  The supplementary section with
 * the paper's optimiser is not available: plain gradient descent with a fixed step is the
 * reading.  losses: host array of iters doubles (L before each step) or NULL; when given the
 * call waits for the stream.  Reductions: runs of 16 terms per thread in float, the rest in
 * double, in a fixed order. */
hpt_status hpt_phase_encode(hpt_ctx *ctx, const void *target_dev, float *phi_dev, int32_t W, int32_t H,
                            double lambda, double pitch, double z, int32_t iters, float lr, double *losses,
                            void *stream);

/* ---- probes ---------------------------------------------------------------------------- */
/* Measured throughputs of this device for the roofline (the paper has no counterpart):
 * peaks[0] FP32 FMA TFLOP/s, peaks[1] FP64 FMA TFLOP/s (2 flops per FMA, eight independent
 * chains per thread, 8 blocks of 256 threads per SM), peaks[2] L2 read GB/s over a 64 MiB
 * buffer, peaks[3] the SM count.  Synchronous; allocates and frees 64 MiB. */
enum { HPT_NPEAKS = 4 };
hpt_status hpt_probe_peaks(hpt_ctx *ctx, double peaks[HPT_NPEAKS]);

/* ---- ambient cache construction (texture baking, Sec. 4.4) ---------------------------- */
/* The supplementary section that defines the bake is not available; this is the reading.
 * For cell (ix, iy, iz) of a res^3 grid over [bmin, bmax] (centre x = bmin + (i + 0.5)
 * (bmax - bmin) / res) and channel c: E_c(x) = pi / spp * sum_s L_c(y_s -> x), with spp
 * directions w_s uniform on the sphere (cos theta = 1 - 2 u0, phi = 2 pi u1 from the Philox
 * path draw of vertex 0 at pixel index (iy + res iz) res + ix, sample s, wavelength index c,
 * key seed), y_s the first hit along w_s and L_c the incoherent radiance leaving it towards x
 * (emission at full weight, NEE + BSDF sampling with MIS, vertices counted from 1 at y_s up
 * to max_depth, no cache); a miss gives 0.  For isotropic incident light E is the irradiance
 * pi L, the quantity the cache lookup multiplies by albedo / pi.  Writes float [res][res]
 * [res][3] ([z][y][x][c]) to E_dev (caller-owned device memory, E_bytes >= 12 res^3).
 * Asynchronous on 'stream'. */
typedef struct {
    int32_t res;
    float bmin[3], bmax[3];
    int32_t spp, max_depth;
    uint64_t seed;
} hpt_bake_desc;
hpt_status hpt_cache_bake(hpt_ctx *ctx, uint64_t scene_id, const hpt_bake_desc *desc, float *E_dev,
                          size_t E_bytes, void *stream);
/* Upload an ambient cache from host memory: binary16 [res][res][res][3] ([z][y][x][c], IEEE
 * bits) over [bmin, bmax]; the library copies it (res = 0 removes the cache).  Synchronises
 * the device first; HPT_ERR_BUSY while queued requests use the scene. */
hpt_status hpt_cache_upload(hpt_ctx *ctx, uint64_t scene_id, int32_t res, const float bmin[3],
                            const float bmax[3], const uint16_t *E_half_host);
/* Replace the scene's ambient cache by the float grid E_dev [res][res][res][3] over [bmin,
 * bmax] (device memory, converted to binary16 with round to nearest even; res = 0 removes
 * the cache).  Synchronises the device first (traces in flight may read the old cache);
 * HPT_ERR_BUSY while queued requests use the scene. */
hpt_status hpt_scene_set_cache(hpt_ctx *ctx, uint64_t scene_id, int32_t res, const float bmin[3],
                               const float bmax[3], const float *E_dev);

/* ---- serving: continuous batching of render requests ---------------------------------- */
/* Queue a request; the scheduler thread admits it when a slot and memory are free and runs
 * it concurrently with the requests already on the device (the waves of all admitted requests
 * share the device; a request's fields equal those of the same render traced alone).
 *  out_dev != NULL: caller-owned device output (complex64 [n_lambda][K][H][W], out_bytes >= its
 *    size); it must stay valid until the request is done.  Admission counts its bytes against the
 *    context's hbm_budget_bytes.
 *  out_dev == NULL: the library allocates the output when it admits the request, and only while
 *    the device's free memory (cudaMemGetInfo at admission, so scenes, caches and every other
 *    allocation on the device are accounted for) minus a reserve of max(1 GiB, 5 % of the device)
 *    holds it; the request waits in the queue until then.  A request that does not fit even with
 *    nothing else admitted finishes with HPT_ERR_OOM.  Read the result with hpt_request_output and
 *    free it with hpt_request_release.
 * HPT_ERR_BUSY (nothing queued) when max_queue requests already wait for admission. */
hpt_status hpt_submit(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                      void *out_dev, size_t out_bytes, uint64_t *req_id);
/* *done = 1 when the request finished; then returns its final status (HPT_OK, or the error that
 * ended it, e.g. HPT_ERR_DEVICE with the kernels' status bits, HPT_ERR_OOM, HPT_ERR_CUDA or
 * HPT_ERR_CANCELLED, with the message in hpt_last_error()); HPT_OK while it runs. */
hpt_status hpt_poll(hpt_ctx *ctx, uint64_t req_id, int *done);
/* Wait up to timeout_ms (0 = forever) for the request; HPT_ERR_TIMEOUT if not done, else its
 * final status as hpt_poll reports it.  A request is done only when no kernel of it is still
 * running: its output (complete when the status is HPT_OK) may then be read or freed. */
hpt_status hpt_wait(hpt_ctx *ctx, uint64_t req_id, uint32_t timeout_ms);
/* Cancel a request: a queued one is dropped at once, an admitted one gets no further waves and
 * is done when its waves in flight have completed; its final status is HPT_ERR_CANCELLED.  A
 * finished request is left as it is (HPT_OK). */
hpt_status hpt_cancel(hpt_ctx *ctx, uint64_t req_id);
/* Timestamps of a finished request in microseconds since the context was created:
 * t[0] submitted, t[1] admitted (launched; -1 if never admitted), t[2] completed. */
hpt_status hpt_request_times(hpt_ctx *ctx, uint64_t req_id, double t[3]);
/* Copy the library-owned output of a finished request (submitted with out_dev == NULL) to dst
 * (host or device memory, bytes >= its size); synchronous. */
hpt_status hpt_request_output(hpt_ctx *ctx, uint64_t req_id, void *dst, size_t bytes);
/* Forget a finished request and free its library-owned output; its id becomes unknown.  Records
 * of finished requests are otherwise kept until 4096 newer requests have finished, then dropped
 * oldest first (with their library-owned outputs). */
hpt_status hpt_request_release(hpt_ctx *ctx, uint64_t req_id);

/* ---- trace with fixed scratch: an entry point that allocates nothing -------------------
 * The paper has no counterpart; this is an interface for callers that cannot allocate device
 * memory while they run -- for instance a real-time hologram display loop that must not stall
 * on the device-wide synchronisation that cudaMalloc / cudaFree can cause, or a host process
 * whose device memory is handed out up front by another framework's pool, so that a driver
 * allocation in the middle of serving could fail.
 *
 * hpt_trace_fixed_scratch computes exactly what hpt_trace computes (same inputs, same output
 * layout, bitwise the same fields) but takes every scratch buffer of the trace -- the path
 * state of a wave, the ray queues and their counters, the device copy of the render job --
 * from one device array of HPT_FIXED_SCRATCH_BYTES (64 MiB) that the library defines at file
 * scope.  The call issues no cudaMalloc, cudaFree or other allocating routine.  The context,
 * the uploaded scene (device memory allocated earlier by hpt_create / hpt_scene_upload) and
 * out_dev (caller-owned, complex64 [n_lambda][K][H][W], out_bytes >= 8 n_lambda K H W) are its
 * inputs and output.  The work is queued asynchronously on cuda_stream.
 *  - Set-up: hpt_create, with its device current, looks up the array's device address
 *    (cudaGetSymbolAddress), which places the array in that device's memory; the array then
 *    stays there until the process exits.  The entry point itself does no set-up; if the
 *    set-up failed on the context's device it returns HPT_ERR_UNSUPPORTED with the cause.
 *  - Frames of any size are split into waves that fit the array; spp larger than the array's
 *    path capacity (about 300k paths) is rejected with HPT_ERR_INVALID_ARG.
 *  - All calls share the one array and it keeps the last call's contents; each call clears
 *    what must start at zero (the queue counters of every wave).  Calls whose work overlaps on
 *    the GPU (on different streams, or from different contexts on one device) race on the
 *    array: serialise them on one stream.
 *  - The kernels' status bits (e.g. a traversal-stack overflow) accumulate in the array and
 *    are reported, then cleared, by the next hpt_sync on a context of that device.          */
#define HPT_FIXED_SCRATCH_BYTES (64u << 20)
hpt_status hpt_trace_fixed_scratch(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                                   void *out_dev, size_t out_bytes, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
