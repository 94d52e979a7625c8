/*
 * mt_api.h -- C ABI of libmt.so: time-resolved Monte Carlo path tracing on
 * GB300 (sm_103a), after arXiv 2510.25660 ("mitransient").
 *
 * The calls follow the paper's statement of the problem (Sec. 2 listing: load a
 * scene, render it with a sample count and get back a steady image and a
 * transient image; Sec. 4.4: gradients of a scalar loss in backward mode;
 * Sec. 4.5: impulse responses over a relay-wall scan grid).
 *
 * Conventions
 *   - Every function returns mt_status and never throws.  On failure
 *     mt_last_error() returns a thread-local message valid until the next call
 *     on the same thread.
 *   - Argument checks run synchronously.  Kernel faults and device watchdog
 *     timeouts surface at mt_sync() or at the next call on the stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - "host" pointers are read during the call and may be freed afterwards;
 *     "device" pointers are CUDA device memory owned by the caller.
 *   - Time is optical path length (OPL) in metres (speed of light c = 1,
 *     Sec. 3 Eq. 3): time bin k covers [start + k*width, start + (k+1)*width).
 *   - Films are row-major float32 [H][W][T][C], steady images [H][W][C].
 *     The film holds (1/spp) * sum of contributions per bin (Sec. 3 Eq. 9 with
 *     path reuse); with MT_ACCUMULATE it holds unnormalised sums added to its
 *     previous contents (progressive / resumable rendering).
 *   - Handles are not thread-safe per object; distinct handles may be used
 *     from distinct threads.
 */
#ifndef MT_API_H
#define MT_API_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MT_OK = 0,
    MT_ERR_INVALID_ARGUMENT = 1,
    MT_ERR_OUT_OF_MEMORY = 2,
    MT_ERR_CUDA = 3,
    MT_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (error word set by a kernel) */
    MT_ERR_UNSUPPORTED = 5, /* valid request outside what the library implements */
    MT_ERR_INTERNAL = 6
} mt_status;

typedef struct mt_scene_s *mt_scene;
typedef struct mt_film_s *mt_film;

/* Material per triangle (Sec. 4.1 "complex materials").  LAMBERT: f = albedo/pi,
 * two-sided.  GGX_CONDUCTOR: isotropic GGX with alpha = roughness, Smith
 * height-correlated masking, Schlick Fresnel with F0 = albedo, two-sided. */
#define MT_LAMBERT 0u
#define MT_GGX_CONDUCTOR 1u
typedef struct {
    float albedo[3];
    float roughness;
    uint32_t type;
} mt_material;

/* Emitters (delta pulse in time at t = 0, Sec. 3 Eq. 5).  AREA: triangles
 * [first_tri, first_tri + n_tris) emit `radiance` (RGB, W sr^-1 m^-2) from the
 * side of their winding normal (v1-v0)x(v2-v0).  POINT: isotropic point at
 * `position` with intensity `radiance` (W sr^-1); not hit by rays. */
#define MT_EMITTER_AREA 0u
#define MT_EMITTER_POINT 1u
typedef struct {
    uint32_t type;
    uint32_t first_tri;
    uint32_t n_tris;
    float radiance[3];
    float position[3];
} mt_emitter;

/* Pinhole camera; fov_x_deg is the horizontal field of view. */
typedef struct {
    float origin[3];
    float target[3];
    float up[3];
    float fov_x_deg;
} mt_camera;

/* Heterogeneous participating medium filling the box [lo, hi] (Sec. 4.1,
 * "Volumetric scattering"): extinction sigma_t (1/m) on a res[0] x res[1] x
 * res[2] grid, host array laid out [z][y][x], sampled trilinearly with voxel
 * centres at lo + (i + 0.5) (hi - lo) / res; scalar single-scatter albedo and
 * Henyey-Greenstein g; index-matched (eta = 1), invisible boundary. */
typedef struct {
    float lo[3];
    float hi[3];
    int32_t res[3];
    const float *density; /* host */
    float albedo;
    float g;
} mt_medium;

/* film flags */
#define MT_UNWARP 1u       /* drop the camera segment's time of flight (Sec. 3, "Camera warp") */
#define MT_ACCUMULATE 2u   /* add unnormalised sums into the film instead of overwriting it */
#define MT_PIXEL_CENTER 4u /* no pixel jitter: every sample goes through the pixel centre */
#define MT_COUNTERS 8u     /* count node visits / triangle tests / rays (slower; see mt_read_counters) */

/* NLOS relay-wall scan (Sec. 4.5).  CONFOCAL: laser and sensor at the same wall
 * point, one film row per point (n_sensors ignored).  EXHAUSTIVE: every laser
 * against every sensor, film row = laser * n_sensors + sensor.  Paths are
 * laser -> x_l -> y -> x_s -> sensor with y on the hidden triangles
 * [hidden_first, hidden_first + hidden_count); time is the relay-wall clock
 * |x_l - y| + |y - x_s|.  Points are device arrays float32 [n][3]. */
#define MT_CONFOCAL 0u
#define MT_EXHAUSTIVE 1u
typedef struct {
    const float *lasers;  /* device [n_lasers][3] */
    int32_t n_lasers;
    const float *sensors; /* device [n_sensors][3], EXHAUSTIVE only */
    int32_t n_sensors;
    uint32_t mode;
    float wall_normal[3];
    float wall_albedo;
    uint32_t hidden_first;
    uint32_t hidden_count;
} mt_scan;

/* Thread-local message of the last failing call on this thread. */
const char *mt_last_error(void);

/* Load a scene (Sec. 2 listing, "load_dict").  Copies the host arrays tris
 * [n_tris][3][3], materials [n_tris], emitters [n_emitters], the camera and the
 * optional medium into library-owned device memory, builds the SAH BVH and the
 * emitter sampling table on the device, and returns a handle in *out.  The
 * emitter table weights triangles by area * mean radiance at creation time and
 * is kept fixed by mt_scene_set_params.  Errors: INVALID_ARGUMENT (NULL
 * pointers, n_tris < 1, non-finite vertices, invalid materials, emitter ranges
 * out of bounds), OUT_OF_MEMORY, CUDA.  The vertices and materials of scenes
 * of more than 65,536 triangles are checked on the device after the upload
 * (the same errors and messages; nothing stays allocated), smaller ones on the
 * host before any device work.  Synchronises `stream`. */
mt_status mt_scene_create(const float *tris, int64_t n_tris, const mt_material *materials,
                          const mt_emitter *emitters, int32_t n_emitters, const mt_camera *camera,
                          const mt_medium *medium, void *stream, mt_scene *out);

/* Replace per-triangle albedos (device float32 [n_tris][3]), emitter radiances
 * (device float32 [n_emitters][3]) and/or the medium albedo (device float32
 * [1]); NULL leaves a parameter unchanged.  Asynchronous on `stream`. */
mt_status mt_scene_set_params(mt_scene scene, const float *d_albedo, const float *d_radiance,
                              const float *d_medium_albedo, void *stream);

/* Describe a caller-owned film: d_film device float32 [H][W][T][C] and the
 * optional d_steady device float32 [H][W][C] (Sec. 2 listing returns both; the
 * steady image is the time integral including contributions outside the
 * window, Sec. 3 "Path reuse").  C must be 3 for mt_render / mt_render_backward
 * / mt_render_tangent / mt_render_phasor, 1 for mt_render_nlos and 12 for
 * mt_render_polarized.  bin_width > 0, T >= 1. */
mt_status mt_film_create(int32_t H, int32_t W, int32_t T, int32_t C, float start_opl, float bin_width,
                         float *d_film, float *d_steady, uint32_t flags, mt_film *out);

/* Make the film a window of a taller frame: its H rows are rows [row0, row0 + H)
 * of a frame_H x W image (same camera, same per-pixel random numbers), so a
 * frame rendered window by window equals the frame rendered at once (crop
 * rendering; e.g. to copy finished rows to the host while later rows render).
 * Default: frame_H = H, row0 = 0.  Applies to mt_render, mt_render_dump,
 * mt_render_phasor, mt_render_backward, mt_render_tangent and
 * mt_render_polarized; dump records carry frame pixel ids.
 * MT_ERR_INVALID_ARGUMENT if the window does not fit. */
mt_status mt_film_set_window(mt_film film, int32_t frame_H, int32_t row0);

/* Transient path tracing (Sec. 3, transient_path integrator): for each pixel,
 * spp paths with samples sample_offset .. sample_offset + spp - 1 from the
 * Philox stream keyed by `seed`, at most max_depth segments each (1 = emitters
 * seen directly), next-event estimation with power-heuristic MIS (no MIS in a
 * medium), every contribution splatted into the bin of its own optical path
 * length and into the steady image.  Asynchronous on `stream`.  The persistent
 * form (the default) allocates nothing.  The wavefront form (MT_OPT_WAVEFRONT
 * in mt_set_launch) allocates its path pool on the first wavefront render of a
 * scene that needs a larger pool than the scene holds (a render of more paths,
 * up to the pool size of mt_set_wavefront_pool), waits every few iterations
 * until `stream` has finished the iteration two back (the host stays ahead of
 * the GPU; nothing is copied for it), and refuses to run under stream capture
 * when it would allocate (INVALID_ARGUMENT).  Errors: INVALID_ARGUMENT (spp < 1,
 * max_depth outside [1, 64], film C != 3), OUT_OF_MEMORY (path pool), CUDA. */
mt_status mt_render(mt_scene scene, mt_film film, int32_t spp, uint64_t seed, int32_t max_depth,
                    uint64_t sample_offset, void *stream);

/* mt_render, with the film and steady image copied to host memory band by band
 * as the bands finish: host_film [H][W][T][3] and host_steady [H][W][3] (NULL
 * exactly when the film has no steady image), caller-owned and page-locked for
 * the copies to overlap the render.  The film's rows are cut into bands of
 * band_rows rows (the last one shorter); in the wavefront form with its state in
 * queue order, paths start in pixel order, so the top bands finish first: after
 * every traversal pass a one-block pass flags each band whose paths have all
 * finished and whose shadow rays have all been traced, and its copy is queued
 * on copy_stream behind that iteration; the bands left at the end follow the
 * render's last stage.  Any other form copies every band after the whole
 * render.  Returns once every copy is queued (synchronise copy_stream before
 * reading the host arrays).  As with mt_render, the render clears the film on
 * `stream`: order it after earlier readers of the film (e.g. the copies of an
 * earlier call on the same film, by making `stream` wait for copy_stream).
 * Errors: those of mt_render, and
 * INVALID_ARGUMENT (NULL host_film, host_steady given without a steady image or
 * missing with one, band_rows < 1, more than 4096 bands, copy_stream equal to
 * stream), OUT_OF_MEMORY (per-band counters). */
mt_status mt_render_to_host(mt_scene scene, mt_film film, int32_t spp, uint64_t seed, int32_t max_depth,
                            uint64_t sample_offset, int32_t band_rows, float *host_film, float *host_steady,
                            void *stream, void *copy_stream);

/* Relay-wall impulse responses H(x_l, x_s, t) for all scan pairs in one
 * persistent launch (Sec. 4.5): spp hidden-surface samples per pair (shared by
 * all sensors of a laser in EXHAUSTIVE mode), film rows = pairs, C = 1, H * W
 * must equal the number of pairs.  Asynchronous; allocates nothing after the
 * first call for a scene (scratch grows to the largest exhaustive grid seen). */
mt_status mt_render_nlos(mt_scene scene, mt_film film, const mt_scan *scan, int32_t spp, uint64_t seed,
                         uint64_t sample_offset, void *stream);

/* Frequency-space rendering (Sec. 4.3, Eq. 12): the paths of mt_render, each
 * contribution C adding C * exp(-i * 2 pi * opl / lambda_k) for the K
 * wavelengths d_lambdas (device float32 [K], metres; opl is the optical path
 * length, so 1/lambda is the modulation frequency in 1/m).  The film must have
 * T = 2K and C = 3 and is laid out [H][W][K][2][3]: the real RGB then the
 * imaginary RGB per wavelength, times 1/spp (unnormalised with MT_ACCUMULATE);
 * the film's start and width are ignored; the steady image is the usual one.
 * Asynchronous; allocates nothing. */
mt_status mt_render_phasor(mt_scene scene, mt_film film, const float *d_lambdas, int32_t K, int32_t spp,
                           uint64_t seed, int32_t max_depth, uint64_t sample_offset, void *stream);

/* Transient polarization (Sec. 4.2, "Transient polarization tracking"): the
 * same paths as mt_render with a Stokes vector (S0 intensity, S1 = I_x - I_y,
 * S2 = I(+45) - I(-45), S3 circular) per colour channel.  The film has C = 12,
 * laid out [H][W][T][4 Stokes][3 colours], and its steady image [H][W][4][3]
 * is required.  x is the camera's horizontal axis, y = k x x for light
 * travelling along k.  Emitters are unpolarised, Lambert surfaces depolarise,
 * GGX conductors reflect with the Fresnel Mueller matrix of the complex index
 * 1 + i kappa, kappa = 2 sqrt(F0 / (1 - F0)) (normal-incidence reflectance
 * F0 = albedo, clamped to 0.999) at the microfacet, so S0 of a conductor
 * differs from mt_render's Schlick value.  Scattering delays and the emission
 * pulse apply.  MT_ERR_UNSUPPORTED for scenes with a medium; other errors as
 * mt_render. */
mt_status mt_render_polarized(mt_scene scene, mt_film film, int32_t spp, uint64_t seed, int32_t max_depth,
                              uint64_t sample_offset, void *stream);

/* Forward-mode derivative (Sec. 4.4, forward mode): the film of
 * dI/dtheta . dtheta for one direction dtheta in parameter space, i.e. the
 * time-resolved derivative of the image along that direction, with the same
 * paths as mt_render (same seed and sample_offset).  Parameters as in
 * mt_render_backward: d_dalbedo device float32 [n_tris][3] (input triangle
 * order) or NULL, d_dradiance device float32 [n_emitters][3] or NULL, dmedium
 * the medium-albedo component (ignored without a medium).  The film (C = 3)
 * and its steady image receive the tangent; same flags, ownership and errors
 * as mt_render.  Each contribution C adds C * sum_v ratio_v * dtheta_v over
 * its vertices plus Cbar * dLe: exact for the estimator (no finite
 * differences), the transpose of mt_render_backward. */
mt_status mt_render_tangent(mt_scene scene, mt_film film, const float *d_dalbedo, const float *d_dradiance,
                            float dmedium, int32_t spp, uint64_t seed, int32_t max_depth, uint64_t sample_offset,
                            void *stream);

/* Backward mode by path replay (Sec. 4.4, Eqs. 13-15): regenerate every path of
 * mt_render(scene, film, spp, seed, max_depth, sample_offset) from its Philox
 * key and add dL/dalbedo (device [n_tris][3]), dL/dradiance (device
 * [n_emitters][3]) and dL/dmedium_albedo (device [1], nullable) given
 * d_grad_film = dL/dfilm (device, film layout) and the optional d_grad_steady.
 * Gradients are ADDED to the outputs.  Requires albedos > 0.  Asynchronous. */
mt_status mt_render_backward(mt_scene scene, mt_film film, const float *d_grad_film,
                             const float *d_grad_steady, int32_t spp, uint64_t seed, int32_t max_depth,
                             uint64_t sample_offset, float *d_grad_albedo, float *d_grad_radiance,
                             float *d_grad_medium_albedo, void *stream);

/* Synchronise `stream` and report device-side errors raised since the last
 * call (traversal stack overflow -> INTERNAL, bounded waits -> TIMEOUT).  The
 * scene names the device error word that the kernels of its renders set (each
 * scene has its own), so errors of one scene do not surface on another. */
mt_status mt_sync(mt_scene scene, void *stream);

/* Counters accumulated by launches on this scene since the last reset:
 * out[0] path vertices, out[1] paths, out[2] contributions, out[3] rays,
 * out[4] bytes of BVH nodes fetched*, out[5] triangle tests*, out[6] splats into shared
 * memory, out[7] splats into global memory (* only with MT_COUNTERS).
 * Synchronises `stream`; reset != 0 zeroes them afterwards. */
mt_status mt_read_counters(mt_scene scene, uint64_t *out, int32_t reset, void *stream);

/* Device time of the wavefront stages of renders launched with
 * MT_OPT_STAGE_TIMING since the last reset (out has 5 entries): out[0] ms in
 * queue setup, camera-ray generation (and ray sorting), out[1] ms in the
 * traversal pass (k_wf_trace: extension rays, then the shadow rays the
 * previous shading pass queued; k_wf_extend in the backward, polarized and
 * dump forms), out[2] ms in shading (k_wf_shade), out[3] ms in shadow passes
 * of their own (k_wf_shadow in the backward, polarized and dump forms, and
 * for the last shading pass), out[4] iterations.  The
 * values are complete when the renders have returned (they synchronise their
 * stream).  reset != 0 zeroes them afterwards. */
mt_status mt_stage_times(mt_scene scene, double *out, int32_t reset);

/* Scattering delays (Sec. 4.1): light arriving at a surface point of triangle
 * i is re-emitted after a delay dt ~ Exp(mean tau[i]), so every contribution
 * formed at or after that vertex arrives later; the delay density has unit
 * area, so steady-state values do not change.  d_tau: device float32
 * [n_tris] (input triangle order), means in metres of light travel (c = 1),
 * each finite and >= 0 (0 = instantaneous); copied into the scene.  NULL
 * removes the delays.  Applies to mt_render (all forms), mt_render_phasor,
 * mt_render_dump and mt_render_backward; NLOS captures ignore it.
 * Synchronises `stream`; MT_ERR_INVALID_ARGUMENT (scene unchanged) on a bad
 * value. */
mt_status mt_scene_set_delays(mt_scene scene, const float *d_tau, void *stream);

/* Emission pulse p(t) shared by all emitters, L_e(x, t) = L_e(x) p(t) (Sec. 3,
 * Eq. 5 with a pulse of unit area in place of the delta): every contribution
 * carries its own emission time drawn from p.  DELTA: t = 0 (default); BOX:
 * uniform on [0, a), a > 0; GAUSSIAN: mean a, deviation b > 0; EXPONENTIAL:
 * mean a > 0 (metres of light travel).  Same scope as mt_scene_set_delays.
 * MT_ERR_INVALID_ARGUMENT (scene unchanged) on bad parameters. */
#define MT_PULSE_DELTA 0u
#define MT_PULSE_BOX 1u
#define MT_PULSE_GAUSSIAN 2u
#define MT_PULSE_EXPONENTIAL 3u
mt_status mt_scene_set_pulse(mt_scene scene, uint32_t shape, float a, float b);

/* Scene statistics (out has 8 entries): out[0] n_tris, out[1] BVH internal
 * nodes, out[2] BVH depth, out[3] SAH cost x 1000 (sum of node areas / root
 * area, with unit traversal and intersection costs), out[4] light units,
 * out[5] scene bytes on the device, out[6] BVH build time in microseconds,
 * out[7] kernels launched by render calls on this scene so far. */
mt_status mt_scene_stats(mt_scene scene, int64_t *out);

/* Launch configuration used by the next launches of this scene (set by the
 * autotuner; 0 keeps a field at its default), per kind: MT_LAUNCH_RENDER,
 * MT_LAUNCH_BACKWARD, MT_LAUNCH_NLOS (scan-point grids) and
 * MT_LAUNCH_NLOS_EXHAUSTIVE (laser x sensor grids, whose scene default is 32
 * sensors per tile with priv_bins = 0: the lanes of a warp take consecutive
 * sensors and one hidden sample):
 *   threads      threads per CTA (32..256, multiple of 32)
 *   tile         RENDER/BACKWARD: pixels of one image row owned by one warp at
 *                a time; NLOS: scan rows owned by one CTA at a time
 *   ctas_per_sm  cap on resident CTAs per SM (0 = occupancy maximum)
 *   priv_bins    time bins per pixel (scan row) accumulated in shared memory
 *                before one write to HBM; later bins are added to the film in
 *                global memory directly.  -1 = as many as fit (default),
 *                0 = none.
 *   options      MT_OPT_* bits (below). */
mt_status mt_set_launch(mt_scene scene, int32_t kind, int32_t threads, int32_t tile, int32_t ctas_per_sm,
                        int32_t priv_bins, uint32_t options);
/* options: MT_OPT_AGGREGATE = lanes of a warp that add to the same film bin
 * combine their values with warp shuffles first and issue one atomic.
 * MT_OPT_NO_GRAPH (NLOS) = enqueue the kernels directly instead of replaying
 * the cached CUDA graph.  MT_OPT_REFILL(k) (RENDER/BACKWARD, k = 1..32) = a
 * warp starts new paths only once at least k of its lanes are idle (default 1:
 * every idle lane is refilled at once).  MT_OPT_WAVEFRONT (RENDER and
 * BACKWARD; forward, phasor, tangent, polarized and backward renders, with or
 * without a medium) = render in wavefront form: a pool of up to 4M paths in
 * device memory (one 128-B record per path plus queues and shadow-ray records,
 * about 200 B per path; polarized renders add 208 B, backward renders 48 B per
 * vertex; allocated by the first such render of a scene, which therefore must
 * not be captured in a graph) with separate kernels for camera rays, the
 * traversal pass (extension rays, then the previous shading pass's shadow
 * rays), shading and, for backward and polarized renders, a shadow pass of its
 * own; each warp claims rays from a queue; films are zeroed and written with
 * global atomics (tile, priv_bins and the refill option do not apply); the
 * call synchronises `stream` every few iterations.
 * MT_OPT_DYNAMIC_FETCH (with MT_OPT_WAVEFRONT) = traversal lanes whose ray is
 * done take the next queued ray instead of waiting for their warp, as soon as
 * MT_OPT_REFILL(k) lanes of the warp are idle (k = 0: 8; k > 32: 32).
 * MT_OPT_WIDE_BVH (with MT_OPT_WAVEFRONT) = extension and shadow rays traverse
 * the scene's 8-wide BVH (80-byte nodes, 8-bit child planes in a per-node
 * frame) instead of the binary one; hits are the same.
 * MT_OPT_SORT_RAYS (with MT_OPT_WAVEFRONT) = before each extension pass the
 * queued rays are sorted by direction octant and the Morton code of their
 * origin, so that a warp traces similar rays (the film is the same).
 * MT_OPT_STAGE_TIMING (with MT_OPT_WAVEFRONT) = CUDA events on the render
 * stream at every stage boundary; read the totals with mt_stage_times (the
 * extension stage holds the whole traversal pass, shadow rays included, in the
 * forms whose shadow rays are traced there).
 * MT_OPT_SORT_SHADOW (with MT_OPT_WAVEFRONT) = shadow rays are traced in the
 * order of (direction cell, origin Morton code) (the film is the same). */
/* Paths in flight of the wavefront form: its path pool holds at most
 * max_paths paths (0 = the default 4,194,304; otherwise 32 .. 4,194,304).
 * A render of more paths than the pool holds starts new paths in the slots
 * that finished paths free, so every path is traced exactly once and the
 * result does not depend on the pool size (up to the order of floating-point
 * additions).  A smaller pool takes less device memory (about 200 B per path,
 * see MT_OPT_WAVEFRONT) and refills more often.  Takes effect at the next
 * wavefront render, which allocates a pool of this size if the scene holds a
 * smaller one (a larger pool already held is reused, only max_paths slots of
 * it).  Dividing max_paths by the threads of one wavefront launch (8 CTAs of
 * 256 threads per SM) gives the paths per thread the autotuner searches over.
 * INVALID_ARGUMENT outside the range. */
mt_status mt_set_wavefront_pool(mt_scene scene, int64_t max_paths);

#define MT_OPT_AGGREGATE 1u
#define MT_OPT_NO_GRAPH 2u
#define MT_OPT_WAVEFRONT 4u
#define MT_OPT_DYNAMIC_FETCH 8u
#define MT_OPT_WIDE_BVH 16u
#define MT_OPT_SORT_RAYS 32u
#define MT_OPT_STAGE_TIMING 64u
#define MT_OPT_SORT_SHADOW 128u
#define MT_OPT_REFILL(k) ((uint32_t)(k) << 8)
#define MT_LAUNCH_RENDER 0
#define MT_LAUNCH_BACKWARD 1
#define MT_LAUNCH_NLOS 2            /* scan points (confocal grids) */
#define MT_LAUNCH_NLOS_EXHAUSTIVE 3 /* laser x sensor grids; default 32 sensors per tile, no privatisation */

void mt_scene_destroy(mt_scene scene);
void mt_film_destroy(mt_film film);

/* ---- parity probes: the same device code as the renderer, on fixed inputs ---- */

/* Philox4x32-10 (Salmon et al., SC'11) of n counters (device uint32 [n][4]) under
 * key (seed_lo, seed_hi) into device uint32 [n][4]. */
mt_status mt_probe_philox(uint64_t seed, const uint32_t *d_counters, int64_t n, uint32_t *d_out, void *stream);

/* Closest hits of n rays (device float32 [n][6] = origin, unit direction) with
 * t in (0, tmax): device int32 [n] triangle index (-1 = miss, ties to the
 * smaller index) and device float32 [n] distance.  Bit 0 of any_hit set
 * instead writes 1/0 occlusion into d_tri; bit 1 set traverses the 8-wide BVH
 * (MT_OPT_WIDE_BVH) instead of the binary one; other bits are invalid. */
mt_status mt_probe_trace(mt_scene scene, const float *d_rays, int64_t n, float tmax, int32_t any_hit,
                         int32_t *d_tri, float *d_t, void *stream);

/* Time-bin index floor((opl - start) / width) of n optical path lengths
 * (device float32 [n]) into device int32 [n], -1 outside [0, T). */
mt_status mt_probe_bins(const float *d_opl, int64_t n, float start, float width, int32_t T, int32_t *d_bin,
                        void *stream);

/* One contribution record of the per-path dump. */
typedef struct {
    int32_t pixel, sample, depth, kind, tri, bin;
    float opl;
    float c[3];
} mt_contrib;

/* mt_render, additionally writing every contribution (kind 0 = emission found
 * by the path, 1 = next-event estimate, 2 = NLOS connection) into d_dump
 * (capacity `cap`); *d_count (device int64) receives the total number of
 * contributions, which may exceed cap.  For NLOS pass a scan (non-NULL). */
mt_status mt_render_dump(mt_scene scene, mt_film film, const mt_scan *scan, int32_t spp, uint64_t seed,
                         int32_t max_depth, uint64_t sample_offset, mt_contrib *d_dump, int64_t cap,
                         int64_t *d_count, void *stream);

/* ---- microbenchmarks for the memory/atomic roofline ----
 * Rates the tracer's access patterns can reach on this GPU, measured with CUDA
 * events on `stream` (second of two runs):
 *   MT_MICRO_GATHER32    random 32-byte loads from d_buf (bytes long; L2
 *                        resident when smaller than L2), *out_rate in GB/s
 *   MT_MICRO_RED_GLOBAL  red.global.add.f32 at random addresses of d_buf, Gop/s
 *   MT_MICRO_RED_SHARED  shared-memory atomicAdd.f32 into a 48 KB histogram per
 *                        CTA, Gop/s (d_buf is only a sink)
 * iters = accesses per thread.  d_buf must be device memory of >= 4096 bytes;
 * its contents are overwritten by MT_MICRO_RED_GLOBAL.  Synchronises. */
#define MT_MICRO_GATHER32 0
#define MT_MICRO_RED_GLOBAL 1
#define MT_MICRO_RED_SHARED 2
mt_status mt_microbench(int32_t kind, void *d_buf, int64_t bytes, int32_t iters, double *out_rate, void *stream);

/* ---- allocation-free variant ----
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory at the time they render.  mt_render_nlos
 * allocates (with cudaMalloc) a hidden-surface table the first time it sees a
 * hidden triangle range and grows a per-scene sample buffer the first time it
 * sees a larger exhaustive grid.  That fails or is unwelcome for applications
 * whose device memory is reserved up front by their own allocator or a fixed
 * budget (a cudaMalloc outside that pool can fail once the budget is taken),
 * and for render loops that must not stall on an allocation.
 * mt_render_nlos_noalloc computes the same impulse responses as mt_render_nlos
 * (same arguments, same launch configuration and options, same result up to
 * the order of floating-point additions) but keeps its per-call scratch in one
 * static device array of 5.27 MiB compiled into libmt.so, which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc or
 * cudaFree.
 *   - Limits: at most 65,536 hidden triangles and, for EXHAUSTIVE scans,
 *     n_lasers * spp <= 131,072; larger requests return
 *     MT_ERR_INVALID_ARGUMENT with a message naming the limit.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) for that device; make that first call before any
 *     stream capture.
 *   - Each call rebuilds the hidden-surface table (with its guide table) in the
 *     array with four small kernels on `stream`; the capture kernels read the
 *     hidden area from the array, so the call does not synchronise `stream`.
 *     A hidden range of zero total area gives a zero film (mt_render_nlos
 *     rejects it).
 *   - All calls share the array and leave their contents in it: calls that
 *     overlap on the GPU (for example on two streams, or from two threads)
 *     race and corrupt each other's results; serialise them.
 *   - The scene still comes from mt_scene_create and the film, steady image
 *     and scan points are the caller's. */
mt_status mt_render_nlos_noalloc(mt_scene scene, mt_film film, const mt_scan *scan, int32_t spp, uint64_t seed,
                                 uint64_t sample_offset, void *stream);

#ifdef __cplusplus
}
#endif
#endif
