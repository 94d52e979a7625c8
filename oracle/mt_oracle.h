/*
 * mt_oracle.h -- plain, slow, single-threaded FP64 CPU oracle for time-resolved
 * Monte Carlo path tracing (arXiv 2510.25660, "mitransient").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load or call this library.  It shares no
 * code, header, table or constant generator with the CUDA path: everything
 * here (Philox, BVH, intersection, sampling, estimator) is written out again
 * from the published definitions, in double precision.
 *
 * What it computes (paper sections):
 *   - light paths x0 -> ... -> xk and the transient path integral (Sec. 3, Eqs. 1-2)
 *   - time of flight as optical path length, sum of eta * |x_i - x_{i+1}| with
 *     c = 1, so the time axis is in metres (Sec. 3, Eqs. 3-4)
 *   - delta-pulse emission, rectangular time-gated sensor (Sec. 3, Eqs. 5-6)
 *   - impulse response without scattering delays (Sec. 3, Eq. 8)
 *   - Monte Carlo estimator (1/N) sum C/p (Sec. 3, Eq. 9)
 *   - path reuse: bin = floor((tof - b_start) / b_width) (Sec. 3, "Path reuse")
 *   - camera unwarping: drop the last segment's tof (Sec. 3, "Camera warp")
 *   - transient volumetric path tracing with tof inside media (Sec. 4.1)
 *   - backward-mode gradients of a scalar loss (Sec. 4.4, Eqs. 13-15)
 *   - relay-wall NLOS impulse responses H(x_l, x_s, t) (Sec. 4.5)
 *   - frequency-space (phasor) rendering, C * exp(-i 2 pi tof / lambda) (Sec. 4.3)
 * Where the paper is silent (estimator details, sampling maps, RNG layout)
 * the oracle follows the readings listed in the project's design notes; each
 * function below states the one it uses.
 */
#ifndef MT_ORACLE_H
#define MT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mo_scene mo_scene;

/* flags (same bit meaning as the public film flags) */
#define MO_UNWARP 1u
#define MO_ACCUMULATE 2u
#define MO_PIXEL_CENTER 4u

/* estimator strategy, oracle-only (MIS consistency checks) */
#define MO_STRAT_MIS 0
#define MO_STRAT_NEE_ONLY 1
#define MO_STRAT_BSDF_ONLY 2

typedef struct {
    int32_t pixel;    /* film row index (pixel or scan pair) */
    int32_t sample;   /* sample index including sample_offset */
    int32_t depth;    /* vertex index the contribution is attached to */
    int32_t kind;     /* 0 = emission found by the path, 1 = next-event estimate, 2 = NLOS */
    int32_t tri;      /* triangle hit (kind 0) / emitter triangle (kind 1) / hidden triangle (kind 2); -1 point */
    int32_t bin;      /* time bin, may lie outside [0, T) */
    double opl;       /* optical path length in metres */
    double c[3];      /* contribution (already divided by the sampling pdf) */
} mo_contrib;

typedef struct {
    int32_t H, W, T;
    double start, width;
    uint32_t flags;
    int32_t spp;
    uint64_t seed;
    int32_t max_depth;
    uint64_t sample_offset;
    int32_t x0, x1, y0, y1; /* pixel crop [x0,x1) x [y0,y1) */
    int32_t strategy;
} mo_args;

mo_scene *mo_scene_create(const float *tris, int64_t n, const float *albedo, const float *rough,
                          const uint32_t *mtype, int32_t n_em, const int32_t *em_type,
                          const int32_t *em_first, const int32_t *em_n, const double *em_radiance,
                          const double *em_pos, const double *camera /* origin3 target3 up3 fov_x_deg */,
                          const float *density /* [rz][ry][rx] or NULL */, const int32_t *res /* rx ry rz */,
                          const double *medium /* lo3 hi3 albedo g */);
void mo_scene_destroy(mo_scene *s);
/* Replace albedos / emitter radiances / medium albedo; sampling tables are kept. */
void mo_scene_set_params(mo_scene *s, const double *albedo, const double *radiance, double medium_albedo);

#define MO_PULSE_DELTA 0
#define MO_PULSE_BOX 1
#define MO_PULSE_GAUSSIAN 2
#define MO_PULSE_EXPONENTIAL 3
/* per-triangle exponential scattering-delay means in metres (copied; NULL clears); 1 on a bad value */
int mo_scene_set_delays(mo_scene *s, const double *tau);
/* emission pulse shared by all emitters; 1 on bad parameters */
int mo_scene_set_pulse(mo_scene *s, int type, double a, double b);

void mo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void mo_philox_batch(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *out);

int64_t mo_intersect(const mo_scene *s, const double *o, const double *d, double tmax, int brute,
                     double *t_out);
int mo_occluded(const mo_scene *s, const double *o, const double *d, double tmax, int brute);
void mo_camera_ray(const mo_scene *s, int32_t W, int32_t H, int32_t px, int32_t py, double jx, double jy,
                   double *o, double *d);

/* BSDF in world space around geometric normal ng (flipped toward wo inside). */
double mo_bsdf_eval(uint32_t type, const double *albedo, double rough, const double *ng, const double *wo,
                    const double *wi, double *f_out, double *pdf_out);
int mo_bsdf_sample(uint32_t type, const double *albedo, double rough, const double *ng, const double *wo,
                   double u0, double u1, double *wi_out, double *weight_out, double *pdf_out);
double mo_hg_eval(double g, double cos_theta);
void mo_hg_sample(double g, const double *dir, double u0, double u1, double *wi_out);
double mo_density(const mo_scene *s, const double *p);
double mo_majorant(const mo_scene *s);
double mo_track(const mo_scene *s, const double *o, const double *d, double dist, uint64_t seed, uint32_t key_a,
                uint32_t key_b, int method);

int mo_render(const mo_scene *s, const mo_args *a, double *film, double *steady, double *dropped,
              mo_contrib *dump, int64_t dump_cap, int64_t *n_dump, uint64_t *counters);
int mo_render_phasor(const mo_scene *s, const mo_args *a, const double *lambdas, int32_t K, double *phasor,
                     double *steady);
/* Stokes film [crop px][T][4][3] and steady [crop px][4][3] (transient polarization) */
int mo_render_polarized(const mo_scene *s, const mo_args *a, double *film, double *steady);
/* conductor extinction coefficient of the polarized GGX model for a normal-incidence reflectance F0 */
double mo_conductor_kappa(double F0);
int mo_render_tangent(const mo_scene *s, const mo_args *a, const double *dalb, const double *drad, double dmed,
                      double *tfilm, double *tsteady);
int mo_render_backward(const mo_scene *s, const mo_args *a, const double *grad_film,
                       const double *grad_steady, double *grad_albedo, double *grad_radiance,
                       double *grad_medium_albedo);
int mo_render_nlos(const mo_scene *s, int32_t hidden_first, int32_t hidden_n, const double *wall_normal,
                   double wall_albedo, const float *lasers, int32_t n_l, const float *sensors, int32_t n_s,
                   int32_t exhaustive, int64_t pair0, int64_t pair1, int32_t T, double start, double width,
                   int32_t spp, uint64_t seed, uint64_t sample_offset, uint32_t flags, double *film,
                   double *steady, mo_contrib *dump, int64_t dump_cap, int64_t *n_dump, uint64_t *counters);

#ifdef __cplusplus
}
#endif
#endif
