/*
 * mt_oracle.c -- FP64 single-threaded CPU oracle (test infrastructure only).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this.  It is written straight from the paper's formulation (arXiv
 * 2510.25660, Sec. 3 and Sec. 4) plus the readings recorded in the design notes
 * for what the paper leaves open; it shares nothing with the CUDA path.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared mt_oracle.c -o libmt_oracle.so -lm
 */
#include "mt_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846
#define MO_MAX_DEPTH 64
#define MO_TRACK_STEPS 1024 /* free-flight steps per segment before a path is dropped */

/* ------------------------------------------------------------------------- */
/* vectors                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 nrm(v3 a) { double l = len(a); return scl(a, 1.0 / l); }
static double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static v3 ld(const double *p) { return mk(p[0], p[1], p[2]); }
static void st(double *p, v3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
static double maxabs(v3 p) { double m = fabs(p.x); if (fabs(p.y) > m) m = fabs(p.y); if (fabs(p.z) > m) m = fabs(p.z); return m; }

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the       */
/* multiply-hi/lo S-box with a Weyl-sequence key schedule.                    */
/* ------------------------------------------------------------------------- */
void mo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void mo_philox_batch(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *out) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; i++) mo_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* four uniforms in [0,1) from counter (a, b, c, d): top 24 bits * 2^-24 */
static void rng4(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d, double u[4]) {
    uint32_t ctr[4] = {a, b, c, d}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, o[4];
    mo_philox4x32_10(ctr, key, o);
    for (int i = 0; i < 4; i++) u[i] = (double)(o[i] >> 8) * (1.0 / 16777216.0);
}

#define G_NEE 0u
#define G_SCATTER 1u
#define G_TRACK 0x100u
#define G_RATIO 0x10000u
#define G_DELAY 0x20000u /* scattering delay at a surface vertex */
#define G_PULSE 0x20010u /* emission time of a contribution (+ kind) */

/* ------------------------------------------------------------------------- */
/* scene                                                                      */
/* ------------------------------------------------------------------------- */
typedef struct { double lo[3], hi[3]; int32_t left, right, first, count; } onode;

struct mo_scene {
    int64_t n;
    v3 *v0, *v1, *v2, *ng;
    double *area;
    double *albedo; /* n*3 */
    double *rough;
    uint32_t *type;
    int32_t *tri_em;    /* emitter index or -1 */
    double *tri_lpdf;   /* pick probability / area (area-measure light pdf), 0 if not emissive */
    /* emitters */
    int32_t n_em;
    int32_t *em_type, *em_first, *em_n;
    double *em_rad; /* n_em*3, current */
    v3 *em_pos;
    /* light units: area-emitter triangles and point emitters */
    int64_t n_units;
    int64_t *unit_tri; /* -1 for a point emitter */
    int32_t *unit_em;
    double *unit_cdf;  /* normalised, inclusive */
    double *unit_p;    /* pick probability */
    /* camera */
    v3 cam_o, cam_f, cam_r, cam_u;
    double tan_half;
    /* bvh */
    onode *nodes;
    int64_t n_nodes;
    int64_t *order;
    /* medium */
    int has_medium;
    int32_t res[3];
    double *dens;
    v3 m_lo, m_hi;
    double m_albedo, m_g, m_major;
    /* time-resolved materials and sources (Sec. 4.1, scattering delays; Sec. 3, emission L_e(t)) */
    double *delay;      /* per triangle: mean of an exponential scattering delay (m), NULL = none */
    int pulse_type;     /* MO_PULSE_* */
    double pulse_a, pulse_b;
};

static double cen(const mo_scene *s, int64_t i, int ax) {
    return (comp(s->v0[i], ax) + comp(s->v1[i], ax) + comp(s->v2[i], ax)) / 3.0;
}

/* quickselect: order[lo..hi) partially sorted so that position k holds the
 * k-th smallest centroid along ax (ties broken by triangle index) */
static int less_c(const mo_scene *s, int64_t a, int64_t b, int ax) {
    double ca = cen(s, a, ax), cb = cen(s, b, ax);
    return ca < cb || (ca == cb && a < b);
}
static void select_k(const mo_scene *s, int64_t *o, int64_t lo, int64_t hi, int64_t k, int ax) {
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t piv = o[mid];
        int64_t i = lo, j = hi - 1;
        /* Hoare-style partition around pivot value */
        while (i <= j) {
            while (less_c(s, o[i], piv, ax)) i++;
            while (less_c(s, piv, o[j], ax)) j--;
            if (i <= j) { int64_t t = o[i]; o[i] = o[j]; o[j] = t; i++; j--; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

static void build_bvh(mo_scene *s) {
    int64_t n = s->n;
    s->order = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) s->order[i] = i;
    int64_t cap = 2 * n + 1;
    s->nodes = (onode *)calloc((size_t)cap, sizeof(onode));
    s->n_nodes = 1;
    typedef struct { int64_t node, first, count; } job;
    job *stack = (job *)malloc(sizeof(job) * 128);
    int sp = 0;
    stack[sp++] = (job){0, 0, n};
    while (sp > 0) {
        job jb = stack[--sp];
        onode *nd = &s->nodes[jb.node];
        double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
        double clo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, chi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
        for (int64_t k = jb.first; k < jb.first + jb.count; k++) {
            int64_t i = s->order[k];
            v3 vs[3] = {s->v0[i], s->v1[i], s->v2[i]};
            for (int a = 0; a < 3; a++) {
                for (int v = 0; v < 3; v++) {
                    double c = comp(vs[v], a);
                    if (c < lo[a]) lo[a] = c;
                    if (c > hi[a]) hi[a] = c;
                }
                double c = cen(s, i, a);
                if (c < clo[a]) clo[a] = c;
                if (c > chi[a]) chi[a] = c;
            }
        }
        for (int a = 0; a < 3; a++) {
            /* pad so that rounding in the slab test never drops a contained hit */
            double pad = 1e-9 * (1.0 + fabs(lo[a]) + fabs(hi[a]));
            nd->lo[a] = lo[a] - pad;
            nd->hi[a] = hi[a] + pad;
        }
        if (jb.count <= 4) {
            nd->first = (int32_t)jb.first; nd->count = (int32_t)jb.count; nd->left = nd->right = -1;
            continue;
        }
        int ax = 0;
        double ext = chi[0] - clo[0];
        for (int a = 1; a < 3; a++) if (chi[a] - clo[a] > ext) { ext = chi[a] - clo[a]; ax = a; }
        int64_t half = jb.count / 2;
        select_k(s, s->order, jb.first, jb.first + jb.count, jb.first + half, ax);
        int64_t L = s->n_nodes++, R = s->n_nodes++;
        nd->left = (int32_t)L; nd->right = (int32_t)R; nd->count = 0; nd->first = -1;
        stack[sp++] = (job){R, jb.first + half, jb.count - half};
        stack[sp++] = (job){L, jb.first, half};
    }
    free(stack);
}

static void setup_lights(mo_scene *s, const double *create_rad) {
    int64_t nu = 0;
    for (int e = 0; e < s->n_em; e++) nu += (s->em_type[e] == 0) ? s->em_n[e] : 1;
    s->n_units = nu;
    s->unit_tri = (int64_t *)malloc(sizeof(int64_t) * (nu ? nu : 1));
    s->unit_em = (int32_t *)malloc(sizeof(int32_t) * (nu ? nu : 1));
    s->unit_cdf = (double *)malloc(sizeof(double) * (nu ? nu : 1));
    s->unit_p = (double *)malloc(sizeof(double) * (nu ? nu : 1));
    double *w = (double *)malloc(sizeof(double) * (nu ? nu : 1));
    int64_t k = 0;
    double tot = 0.0;
    for (int e = 0; e < s->n_em; e++) {
        double mean = (create_rad[3 * e] + create_rad[3 * e + 1] + create_rad[3 * e + 2]) / 3.0;
        if (s->em_type[e] == 0) {
            for (int32_t t = 0; t < s->em_n[e]; t++) {
                int64_t tri = s->em_first[e] + t;
                s->unit_tri[k] = tri; s->unit_em[k] = e; w[k] = s->area[tri] * mean; tot += w[k]; k++;
            }
        } else {
            s->unit_tri[k] = -1; s->unit_em[k] = e; w[k] = mean; tot += w[k]; k++;
        }
    }
    double acc = 0.0;
    for (int64_t i = 0; i < nu; i++) {
        acc += w[i];
        s->unit_cdf[i] = tot > 0 ? acc / tot : 0.0;
        s->unit_p[i] = tot > 0 ? w[i] / tot : 0.0;
    }
    if (nu > 0 && tot > 0) s->unit_cdf[nu - 1] = 1.0;
    for (int64_t i = 0; i < nu; i++)
        if (s->unit_tri[i] >= 0 && s->area[s->unit_tri[i]] > 0)
            s->tri_lpdf[s->unit_tri[i]] = s->unit_p[i] / s->area[s->unit_tri[i]];
    free(w);
}

mo_scene *mo_scene_create(const float *tris, int64_t n, const float *albedo, const float *rough,
                          const uint32_t *mtype, int32_t n_em, const int32_t *em_type,
                          const int32_t *em_first, const int32_t *em_n, const double *em_radiance,
                          const double *em_pos, const double *camera, const float *density,
                          const int32_t *res, const double *medium) {
    mo_scene *s = (mo_scene *)calloc(1, sizeof(mo_scene));
    s->n = n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    s->v0 = (v3 *)malloc(sizeof(v3) * nn); s->v1 = (v3 *)malloc(sizeof(v3) * nn);
    s->v2 = (v3 *)malloc(sizeof(v3) * nn); s->ng = (v3 *)malloc(sizeof(v3) * nn);
    s->area = (double *)malloc(sizeof(double) * nn);
    s->albedo = (double *)malloc(sizeof(double) * 3 * nn);
    s->rough = (double *)malloc(sizeof(double) * nn);
    s->type = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    s->tri_em = (int32_t *)malloc(sizeof(int32_t) * nn);
    s->tri_lpdf = (double *)calloc(nn, sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        const float *t = tris + 9 * i;
        s->v0[i] = mk(t[0], t[1], t[2]);
        s->v1[i] = mk(t[3], t[4], t[5]);
        s->v2[i] = mk(t[6], t[7], t[8]);
        v3 c = cross(sub(s->v1[i], s->v0[i]), sub(s->v2[i], s->v0[i]));
        double l = len(c);
        s->area[i] = 0.5 * l;
        s->ng[i] = l > 0 ? scl(c, 1.0 / l) : mk(0, 0, 1);
        for (int k = 0; k < 3; k++) s->albedo[3 * i + k] = albedo[3 * i + k];
        s->rough[i] = rough[i];
        s->type[i] = mtype[i];
        s->tri_em[i] = -1;
    }
    s->n_em = n_em;
    size_t ne = (size_t)(n_em > 0 ? n_em : 1);
    s->em_type = (int32_t *)malloc(sizeof(int32_t) * ne);
    s->em_first = (int32_t *)malloc(sizeof(int32_t) * ne);
    s->em_n = (int32_t *)malloc(sizeof(int32_t) * ne);
    s->em_rad = (double *)malloc(sizeof(double) * 3 * ne);
    s->em_pos = (v3 *)malloc(sizeof(v3) * ne);
    for (int e = 0; e < n_em; e++) {
        s->em_type[e] = em_type[e]; s->em_first[e] = em_first[e]; s->em_n[e] = em_n[e];
        for (int k = 0; k < 3; k++) s->em_rad[3 * e + k] = em_radiance[3 * e + k];
        s->em_pos[e] = ld(em_pos + 3 * e);
        if (em_type[e] == 0)
            for (int32_t t = 0; t < em_n[e]; t++) s->tri_em[em_first[e] + t] = e;
    }
    setup_lights(s, em_radiance);
    /* camera: forward, right = forward x up, true up = right x forward */
    s->cam_o = ld(camera);
    s->cam_f = nrm(sub(ld(camera + 3), s->cam_o));
    s->cam_r = nrm(cross(s->cam_f, ld(camera + 6)));
    s->cam_u = cross(s->cam_r, s->cam_f);
    s->tan_half = tan(camera[9] * PI_D / 360.0);
    build_bvh(s);
    if (density && res && medium) {
        s->has_medium = 1;
        s->res[0] = res[0]; s->res[1] = res[1]; s->res[2] = res[2];
        size_t nv = (size_t)res[0] * res[1] * res[2];
        s->dens = (double *)malloc(sizeof(double) * nv);
        double mx = 0.0;
        for (size_t i = 0; i < nv; i++) { s->dens[i] = density[i]; if (s->dens[i] > mx) mx = s->dens[i]; }
        s->m_major = mx;
        s->m_lo = ld(medium); s->m_hi = ld(medium + 3);
        s->m_albedo = medium[6]; s->m_g = medium[7];
    }
    return s;
}

void mo_scene_destroy(mo_scene *s) {
    if (!s) return;
    free(s->v0); free(s->v1); free(s->v2); free(s->ng); free(s->area); free(s->albedo); free(s->rough);
    free(s->type); free(s->tri_em); free(s->tri_lpdf); free(s->em_type); free(s->em_first); free(s->em_n);
    free(s->em_rad); free(s->em_pos); free(s->unit_tri); free(s->unit_em); free(s->unit_cdf); free(s->unit_p);
    free(s->nodes); free(s->order); free(s->dens); free(s->delay); free(s);
}

/* Scattering delays: the light leaving surface vertex x_i is re-emitted a time
 * dt_i after it arrived, dt_i ~ Exp(mean tau(x_i)) (Sec. 4.1: the time of
 * flight gains the sum of the delays along the path; rho(x, dt) = rho(x)
 * times the delay density, so steady-state values are unchanged). */
int mo_scene_set_delays(mo_scene *s, const double *tau) {
    free(s->delay);
    s->delay = NULL;
    if (!tau) return 0;
    for (int64_t i = 0; i < s->n; i++)
        if (!(tau[i] >= 0.0) || !isfinite(tau[i])) return 1;
    s->delay = (double *)malloc(sizeof(double) * (size_t)s->n);
    if (!s->delay) return 1;
    memcpy(s->delay, tau, sizeof(double) * (size_t)s->n);
    return 0;
}

/* Emission L_e(x, t) = L_e(x) p(t) with a unit-area pulse p (Eq. 5 generalised):
 * DELTA p = delta(t); BOX uniform on [0, a); GAUSSIAN mean a, deviation b;
 * EXPONENTIAL mean a. */
int mo_scene_set_pulse(mo_scene *s, int type, double a, double b) {
    if (type < MO_PULSE_DELTA || type > MO_PULSE_EXPONENTIAL || !isfinite(a) || !isfinite(b)) return 1;
    if ((type == MO_PULSE_BOX || type == MO_PULSE_EXPONENTIAL) && !(a > 0.0)) return 1;
    if (type == MO_PULSE_GAUSSIAN && !(b > 0.0)) return 1;
    s->pulse_type = type;
    s->pulse_a = a;
    s->pulse_b = b;
    return 0;
}

/* one draw of the emission time from u[0], u[1] */
static double pulse_time(const mo_scene *s, const double u[4]) {
    switch (s->pulse_type) {
    case MO_PULSE_BOX: return s->pulse_a * u[0];
    case MO_PULSE_GAUSSIAN:  /* Box-Muller */
        return s->pulse_a + s->pulse_b * sqrt(-2.0 * log(1.0 - u[0])) * cos(2.0 * PI_D * u[1]);
    case MO_PULSE_EXPONENTIAL: return -s->pulse_a * log(1.0 - u[0]);
    default: return 0.0;
    }
}

void mo_scene_set_params(mo_scene *s, const double *albedo, const double *radiance, double medium_albedo) {
    if (albedo) memcpy(s->albedo, albedo, sizeof(double) * 3 * (size_t)s->n);
    if (radiance) memcpy(s->em_rad, radiance, sizeof(double) * 3 * (size_t)s->n_em);
    if (!isnan(medium_albedo)) s->m_albedo = medium_albedo;
}

/* ------------------------------------------------------------------------- */
/* intersection: Moller-Trumbore in FP64, edges inclusive; closest hit breaks */
/* ties in t toward the smaller triangle index.                              */
/* ------------------------------------------------------------------------- */
static int tri_hit(const mo_scene *s, int64_t i, v3 o, v3 d, double *t) {
    v3 e1 = sub(s->v1[i], s->v0[i]), e2 = sub(s->v2[i], s->v0[i]);
    v3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 sv = sub(o, s->v0[i]);
    double u = dot(sv, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    v3 q = cross(sv, e1);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *t = dot(e2, q) * inv;
    return 1;
}

static int box_hit(const onode *nd, v3 o, v3 d, double tmax, double *tnear) {
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; a++) {
        double oa = comp(o, a), da = comp(d, a);
        if (da == 0.0) {
            if (oa < nd->lo[a] || oa > nd->hi[a]) return 0;
            continue;
        }
        double ta = (nd->lo[a] - oa) / da, tb = (nd->hi[a] - oa) / da;
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    *tnear = t0;
    return 1;
}

static int64_t closest(const mo_scene *s, v3 o, v3 d, double tmax, int brute, double *tout) {
    int64_t best = -1;
    double bt = tmax;
    if (brute) {
        for (int64_t i = 0; i < s->n; i++) {
            double t;
            if (tri_hit(s, i, o, d, &t) && t > 0.0 && (t < bt || (t == bt && best >= 0 && i < best))) {
                if (t < tmax) { bt = t; best = i; }
            }
        }
    } else if (s->n > 0) {
        int64_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const onode *nd = &s->nodes[stack[--sp]];
            double tn;
            if (!box_hit(nd, o, d, bt, &tn)) continue;
            if (nd->left < 0) {
                for (int k = 0; k < nd->count; k++) {
                    int64_t i = s->order[nd->first + k];
                    double t;
                    if (tri_hit(s, i, o, d, &t) && t > 0.0 && t < tmax &&
                        (t < bt || (t == bt && (best < 0 || i < best)))) { bt = t; best = i; }
                }
            } else {
                stack[sp++] = nd->right;
                stack[sp++] = nd->left;
            }
        }
    }
    *tout = bt;
    return best;
}

static int occluded(const mo_scene *s, v3 o, v3 d, double tmax, int brute) {
    if (brute) {
        for (int64_t i = 0; i < s->n; i++) {
            double t;
            if (tri_hit(s, i, o, d, &t) && t > 0.0 && t < tmax) return 1;
        }
        return 0;
    }
    if (s->n == 0) return 0;
    int64_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode *nd = &s->nodes[stack[--sp]];
        double tn;
        if (!box_hit(nd, o, d, tmax, &tn)) continue;
        if (nd->left < 0) {
            for (int k = 0; k < nd->count; k++) {
                double t;
                if (tri_hit(s, s->order[nd->first + k], o, d, &t) && t > 0.0 && t < tmax) return 1;
            }
        } else {
            stack[sp++] = nd->right;
            stack[sp++] = nd->left;
        }
    }
    return 0;
}

int64_t mo_intersect(const mo_scene *s, const double *o, const double *d, double tmax, int brute, double *t_out) {
    return closest(s, ld(o), ld(d), tmax, brute, t_out);
}
int mo_occluded(const mo_scene *s, const double *o, const double *d, double tmax, int brute) {
    return occluded(s, ld(o), ld(d), tmax, brute);
}

/* ray-origin offset: 1e-4 * max(1, |p|_inf) along the side normal */
static double eps_of(v3 p) { double m = maxabs(p); return 1e-4 * (m > 1.0 ? m : 1.0); }
static v3 offset(v3 p, v3 n_side) { return add(p, scl(n_side, eps_of(p))); }

/* ------------------------------------------------------------------------- */
/* camera: pinhole, horizontal field of view, box pixel filter                */
/* ------------------------------------------------------------------------- */
static void cam_ray(const mo_scene *s, int W, int H, int px, int py, double jx, double jy, v3 *o, v3 *d) {
    double sx = (2.0 * (px + jx) / W - 1.0) * s->tan_half;
    double sy = (1.0 - 2.0 * (py + jy) / H) * s->tan_half * ((double)H / (double)W);
    *o = s->cam_o;
    *d = nrm(add(s->cam_f, add(scl(s->cam_r, sx), scl(s->cam_u, sy))));
}
void mo_camera_ray(const mo_scene *s, int32_t W, int32_t H, int32_t px, int32_t py, double jx, double jy,
                   double *o, double *d) {
    v3 a, b;
    cam_ray(s, W, H, px, py, jx, jy, &a, &b);
    st(o, a); st(d, b);
}

/* ------------------------------------------------------------------------- */
/* local frames and BSDFs                                                     */
/* ------------------------------------------------------------------------- */
/* orthonormal basis from a unit normal (Duff et al., JCGT 2017), with the sign
 * taken as +1 for n.z >= 0 (negative zero counts as positive) */
static void basis(v3 n, v3 *t, v3 *b) {
    double sg = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n.z);
    double c = n.x * n.y * a;
    *t = mk(1.0 + sg * n.x * n.x * a, sg * c, -sg * n.x);
    *b = mk(c, sg + n.y * n.y * a, -n.y);
}
static v3 to_local(v3 w, v3 t, v3 b, v3 n) { return mk(dot(w, t), dot(w, b), dot(w, n)); }
static v3 to_world(v3 l, v3 t, v3 b, v3 n) { return add(add(scl(t, l.x), scl(b, l.y)), scl(n, l.z)); }

static double ggx_alpha(double r) { return r < 1e-4 ? 1e-4 : r; }
static double ggx_D(double a, v3 h) {
    double a2 = a * a, c2 = h.z * h.z;
    double k = c2 * (a2 - 1.0) + 1.0;
    return a2 / (PI_D * k * k);
}
static double ggx_lambda(double a, v3 w) {
    double s2 = w.x * w.x + w.y * w.y;
    return 0.5 * (-1.0 + sqrt(1.0 + a * a * s2 / (w.z * w.z)));
}

/* f(wo, wi) for local directions (z = shading normal); returns f per channel
 * and the solid-angle pdf of the sampling routine below */
static void bsdf_local(uint32_t type, const double *alb, double rough, v3 wo, v3 wi, double f[3], double *pdf) {
    f[0] = f[1] = f[2] = 0.0;
    *pdf = 0.0;
    if (wo.z <= 0.0 || wi.z <= 0.0) return;
    if (type == 0) {
        for (int k = 0; k < 3; k++) f[k] = alb[k] / PI_D;
        *pdf = wi.z / PI_D;
        return;
    }
    double a = ggx_alpha(rough);
    v3 h = nrm(add(wo, wi));
    double D = ggx_D(a, h);
    double lo = ggx_lambda(a, wo), li = ggx_lambda(a, wi);
    double G2 = 1.0 / (1.0 + lo + li), G1o = 1.0 / (1.0 + lo);
    double c = dot(wi, h);
    double m = pow(1.0 - c, 5.0);
    for (int k = 0; k < 3; k++) {
        double F = alb[k] + (1.0 - alb[k]) * m;
        f[k] = D * G2 * F / (4.0 * wo.z * wi.z);
    }
    *pdf = G1o * D / (4.0 * wo.z);
}

/* d f_c / d albedo_c divided by f_c: 1/albedo (Lambert), (1-m)/F (Schlick F0) */
static void bsdf_dratio(uint32_t type, const double *alb, v3 wo, v3 wi, double r[3]) {
    if (type == 0) {
        for (int k = 0; k < 3; k++) r[k] = 1.0 / alb[k];
        return;
    }
    v3 h = nrm(add(wo, wi));
    double m = pow(1.0 - dot(wi, h), 5.0);
    for (int k = 0; k < 3; k++) r[k] = (1.0 - m) / (alb[k] + (1.0 - alb[k]) * m);
}

/* sample wi; returns 0 if the sample is invalid (below the surface) */
static int bsdf_sample_local(uint32_t type, double rough, v3 wo, double u0, double u1, v3 *wi) {
    if (type == 0) {
        double r = sqrt(u0), ph = 2.0 * PI_D * u1;
        *wi = mk(r * cos(ph), r * sin(ph), sqrt(fmax(0.0, 1.0 - u0)));
        return wi->z > 0.0;
    }
    /* visible-normal sampling of GGX (Heitz, JCGT 2018) */
    double a = ggx_alpha(rough);
    v3 vh = nrm(mk(a * wo.x, a * wo.y, wo.z));
    double l2 = vh.x * vh.x + vh.y * vh.y;
    v3 T1 = l2 > 0.0 ? scl(mk(-vh.y, vh.x, 0.0), 1.0 / sqrt(l2)) : mk(1.0, 0.0, 0.0);
    v3 T2 = cross(vh, T1);
    double r = sqrt(u0), ph = 2.0 * PI_D * u1;
    double t1 = r * cos(ph), t2 = r * sin(ph);
    double sh = 0.5 * (1.0 + vh.z);
    t2 = (1.0 - sh) * sqrt(fmax(0.0, 1.0 - t1 * t1)) + sh * t2;
    v3 nh = add(add(scl(T1, t1), scl(T2, t2)), scl(vh, sqrt(fmax(0.0, 1.0 - t1 * t1 - t2 * t2))));
    v3 ne = nrm(mk(a * nh.x, a * nh.y, fmax(0.0, nh.z)));
    *wi = sub(scl(ne, 2.0 * dot(wo, ne)), wo);
    return wi->z > 0.0;
}

static v3 side_normal(v3 ng, v3 w) { return dot(ng, w) >= 0.0 ? ng : scl(ng, -1.0); }

double mo_bsdf_eval(uint32_t type, const double *albedo, double rough, const double *ng, const double *wo,
                    const double *wi, double *f_out, double *pdf_out) {
    v3 n = side_normal(ld(ng), ld(wo)), t, b;
    basis(n, &t, &b);
    double f[3], pdf;
    bsdf_local(type, albedo, rough, to_local(ld(wo), t, b, n), to_local(ld(wi), t, b, n), f, &pdf);
    for (int k = 0; k < 3; k++) f_out[k] = f[k];
    *pdf_out = pdf;
    return f[0];
}

int mo_bsdf_sample(uint32_t type, const double *albedo, double rough, const double *ng, const double *wo,
                   double u0, double u1, double *wi_out, double *weight_out, double *pdf_out) {
    v3 n = side_normal(ld(ng), ld(wo)), t, b;
    basis(n, &t, &b);
    v3 wol = to_local(ld(wo), t, b, n), wil;
    if (!bsdf_sample_local(type, rough, wol, u0, u1, &wil)) return 0;
    double f[3], pdf;
    bsdf_local(type, albedo, rough, wol, wil, f, &pdf);
    st(wi_out, to_world(wil, t, b, n));
    for (int k = 0; k < 3; k++) weight_out[k] = pdf > 0 ? f[k] * wil.z / pdf : 0.0;
    *pdf_out = pdf;
    return pdf > 0.0;
}

/* Henyey-Greenstein: cos_theta is between propagation directions */
double mo_hg_eval(double g, double c) {
    double d = 1.0 + g * g - 2.0 * g * c;
    return (1.0 - g * g) / (4.0 * PI_D * d * sqrt(d));
}
static v3 hg_sample(double g, v3 dir, double u0, double u1) {
    double c;
    if (fabs(g) < 1e-3) c = 1.0 - 2.0 * u0;
    else {
        double q = (1.0 - g * g) / (1.0 - g + 2.0 * g * u0);
        c = (1.0 + g * g - q * q) / (2.0 * g);
    }
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double sn = sqrt(fmax(0.0, 1.0 - c * c)), ph = 2.0 * PI_D * u1;
    v3 t, b;
    basis(dir, &t, &b);
    return to_world(mk(sn * cos(ph), sn * sin(ph), c), t, b, dir);
}
void mo_hg_sample(double g, const double *dir, double u0, double u1, double *wi_out) {
    st(wi_out, hg_sample(g, ld(dir), u0, u1));
}

/* ------------------------------------------------------------------------- */
/* medium: trilinear density on voxel centres, clamped at the border          */
/* ------------------------------------------------------------------------- */
static double dens(const mo_scene *s, v3 p) {
    double g[3];
    for (int a = 0; a < 3; a++) {
        double lo = comp(s->m_lo, a), hi = comp(s->m_hi, a);
        g[a] = (comp(p, a) - lo) / (hi - lo) * s->res[a] - 0.5;
    }
    int i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; a++) {
        double fl = floor(g[a]);
        f[a] = g[a] - fl;
        int i = (int)fl;
        i0[a] = i < 0 ? 0 : (i > s->res[a] - 1 ? s->res[a] - 1 : i);
        i1[a] = i + 1 < 0 ? 0 : (i + 1 > s->res[a] - 1 ? s->res[a] - 1 : i + 1);
    }
    double acc = 0.0;
    for (int c = 0; c < 8; c++) {
        int ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
        double w = ((c & 1) ? f[0] : 1.0 - f[0]) * ((c & 2) ? f[1] : 1.0 - f[1]) * ((c & 4) ? f[2] : 1.0 - f[2]);
        acc += w * s->dens[((size_t)iz * s->res[1] + iy) * s->res[0] + ix];
    }
    return acc;
}
double mo_density(const mo_scene *s, const double *p) { return s->has_medium ? dens(s, ld(p)) : 0.0; }
double mo_majorant(const mo_scene *s) { return s->has_medium ? s->m_major : 0.0; }

/* parametric overlap of the ray with the medium box, clipped to [0, tmax] */
static int medium_span(const mo_scene *s, v3 o, v3 d, double tmax, double *a, double *b) {
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; k++) {
        double ok = comp(o, k), dk = comp(d, k), lo = comp(s->m_lo, k), hi = comp(s->m_hi, k);
        if (dk == 0.0) {
            if (ok < lo || ok > hi) return 0;
            continue;
        }
        double ta = (lo - ok) / dk, tb = (hi - ok) / dk;
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t0 >= t1) return 0;
    *a = t0; *b = t1;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* forward / backward estimator (Sec. 3 Eq. 9 with path reuse)                */
/* ------------------------------------------------------------------------- */
typedef struct {
    const mo_scene *s;
    const mo_args *a;
    int backward;
    /* forward outputs (crop-relative) */
    double *film, *steady, *dropped;
    double *phasor; const double *lambdas; int32_t K; /* frequency-space film (Sec. 4.3) */
    mo_contrib *dump; int64_t dump_cap, n_dump;
    /* backward inputs/outputs */
    const double *gfilm, *gsteady;
    double *galb, *grad, *gmed;
    /* forward-mode derivative: tangent direction of the parameters; film and
     * steady then receive dC = sum over vertices of C * ratio * dtheta + Cbar * dLe */
    int tangent;
    const double *dalb, *drad;
    double dmed;
    uint64_t cnt[4];
} ctx_t;

typedef struct {
    int32_t tri[MO_MAX_DEPTH + 1];     /* scattering vertex triangle, -1 = medium vertex */
    double ratio[MO_MAX_DEPTH + 1][3]; /* d factor / factor for the continuation direction */
} vlist_t;

/* Deposit one contribution c (cbar = c without the emitter radiance) into the
 * transient film and the steady image, or, in backward mode, push g * dC/dtheta
 * into the gradients.  nv scattering vertices precede it; own_ratio (if not
 * NULL) replaces the continuation ratio of vertex nv (a next-event estimate
 * uses its own direction at the last vertex). */
static void deposit(ctx_t *cx, int32_t pix_full, int32_t lp, int32_t sample, int depth, int kind, int32_t tri,
                    double opl, const double c[3], const double cbar[3], int32_t em, const vlist_t *vl, int nv,
                    const double *own_ratio) {
    const mo_args *a = cx->a;
    if (cx->s->pulse_type != MO_PULSE_DELTA) {
        /* the source emitted this contribution's light at a time drawn from the pulse */
        double u[4];
        rng4(a->seed, (uint32_t)pix_full, (uint32_t)sample, (uint32_t)depth, G_PULSE + (uint32_t)kind, u);
        opl += pulse_time(cx->s, u);
    }
    double x = (opl - a->start) / a->width;
    double fb = floor(x);
    int32_t bin = (fb < -1e9) ? -1000000000 : (fb > 1e9 ? 1000000000 : (int32_t)fb);
    int in = bin >= 0 && bin < a->T;
    cx->cnt[2]++;
    if (cx->tangent) {
        /* C is a product of per-vertex factors: dC = C * sum_v (dfactor_v / factor_v) dtheta_v,
         * plus Cbar dLe for the emitter (C is linear in its radiance) */
        double dc[3];
        for (int k = 0; k < 3; k++) {
            double sum = 0.0;
            for (int v = 1; v <= nv; v++) {
                const double *r = (v == nv && own_ratio) ? own_ratio : vl->ratio[v];
                double dth = vl->tri[v] >= 0 ? (cx->dalb ? cx->dalb[(int64_t)vl->tri[v] * 3 + k] : 0.0) : cx->dmed;
                sum += r[k] * dth;
            }
            dc[k] = c[k] * sum + (em >= 0 && cx->drad ? cbar[k] * cx->drad[(int64_t)em * 3 + k] : 0.0);
        }
        for (int k = 0; k < 3; k++) {
            if (in) cx->film[((int64_t)lp * a->T + bin) * 3 + k] += dc[k];
            if (cx->steady) cx->steady[(int64_t)lp * 3 + k] += dc[k];
        }
        return;
    }
    if (!cx->backward) {
        /* frequency space (Sec. 4.3, Eq. 12): C * exp(-i * 2 pi * tof / lambda) per wavelength */
        for (int32_t q = 0; q < cx->K; q++) {
            double ph = 2.0 * PI_D * opl / cx->lambdas[q];
            double cr = cos(ph), si = sin(ph);
            for (int k = 0; k < 3; k++) {
                cx->phasor[(((int64_t)lp * cx->K + q) * 2 + 0) * 3 + k] += c[k] * cr;
                cx->phasor[(((int64_t)lp * cx->K + q) * 2 + 1) * 3 + k] -= c[k] * si;
            }
        }
        for (int k = 0; k < 3; k++) {
            if (in) cx->film[((int64_t)lp * a->T + bin) * 3 + k] += c[k];
            else if (cx->dropped) cx->dropped[(int64_t)lp * 3 + k] += c[k];
            if (cx->steady) cx->steady[(int64_t)lp * 3 + k] += c[k];
        }
        if (cx->dump && cx->n_dump < cx->dump_cap) {
            mo_contrib *r = &cx->dump[cx->n_dump];
            r->pixel = pix_full; r->sample = sample; r->depth = depth; r->kind = kind; r->tri = tri;
            r->bin = bin; r->opl = opl;
            for (int k = 0; k < 3; k++) r->c[k] = c[k];
        }
        if (cx->dump) cx->n_dump++;
        return;
    }
    double g[3];
    for (int k = 0; k < 3; k++) {
        g[k] = in ? cx->gfilm[((int64_t)lp * a->T + bin) * 3 + k] : 0.0;
        if (cx->gsteady) g[k] += cx->gsteady[(int64_t)lp * 3 + k];
    }
    for (int v = 1; v <= nv; v++) {
        const double *r = (v == nv && own_ratio) ? own_ratio : vl->ratio[v];
        if (vl->tri[v] >= 0) {
            for (int k = 0; k < 3; k++) cx->galb[(int64_t)vl->tri[v] * 3 + k] += g[k] * c[k] * r[k];
        } else if (cx->gmed) {
            for (int k = 0; k < 3; k++) *cx->gmed += g[k] * c[k] * r[k];
        }
    }
    if (em >= 0)
        for (int k = 0; k < 3; k++) cx->grad[(int64_t)em * 3 + k] += g[k] * cbar[k];
}

static int64_t pick_unit(const mo_scene *s, double u) {
    int64_t lo = 0, hi = s->n_units - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (u < s->unit_cdf[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static v3 tri_point(const mo_scene *s, int64_t tri, double u1, double u2) {
    double su = sqrt(u1);
    double b0 = 1.0 - su, b1 = u2 * su, b2 = 1.0 - b0 - b1;
    return add(add(scl(s->v0[tri], b0), scl(s->v1[tri], b1)), scl(s->v2[tri], b2));
}

/* ratio-tracking transmittance along [0, dist] of the ray, 1 outside media */
static double transmittance(const mo_scene *s, v3 o, v3 d, double dist, uint64_t seed, uint32_t p,
                            uint32_t smp, uint32_t depth, int *ok) {
    *ok = 1;
    double a, b;
    if (!s->has_medium || !medium_span(s, o, d, dist, &a, &b)) return 1.0;
    double T = 1.0, t = a;
    for (uint32_t j = 0;; j++) {
        if (j >= MO_TRACK_STEPS) { *ok = 0; return 0.0; }
        double u[4];
        rng4(seed, p, smp, depth, G_RATIO + j, u);
        t += -log(1.0 - u[0]) / s->m_major;
        if (t >= b) break;
        T *= 1.0 - dens(s, add(o, scl(d, t))) / s->m_major;
    }
    return T;
}

/* Transmittance estimates along [0, dist] of a ray (test hook): method 0 =
 * ratio tracking (returns T), method 1 = delta tracking (returns 1 if the
 * ray crosses without a real collision, else 0). */
double mo_track(const mo_scene *s, const double *o, const double *d, double dist, uint64_t seed, uint32_t key_a,
                uint32_t key_b, int method) {
    int ok;
    if (method == 0) return transmittance(s, ld(o), ld(d), dist, seed, key_a, key_b, 0, &ok);
    double a, b;
    v3 O = ld(o), D = ld(d);
    if (!s->has_medium || !medium_span(s, O, D, dist, &a, &b)) return 1.0;
    double t = a, u[4];
    for (uint32_t j = 0; j < MO_TRACK_STEPS; j++) {
        rng4(seed, key_a, key_b, 0, G_TRACK + j, u);
        t += -log(1.0 - u[0]) / s->m_major;
        if (t >= b) return 1.0;
        if (u[1] < dens(s, add(O, scl(D, t))) / s->m_major) return 0.0;
    }
    return 0.0;
}

static double mis2(double a, double b) { return a * a / (a * a + b * b); }

/* Trace one path for full-film pixel (px, py), sample index smp. */
static void trace_path(ctx_t *cx, int32_t px, int32_t py, int32_t lp, uint32_t smp) {
    const mo_scene *s = cx->s;
    const mo_args *a = cx->a;
    uint32_t pix = (uint32_t)(py * a->W + px);
    uint64_t seed = a->seed;
    double u[4];
    rng4(seed, pix, smp, 0, 0, u);
    double jx = (a->flags & MO_PIXEL_CENTER) ? 0.5 : u[0];
    double jy = (a->flags & MO_PIXEL_CENTER) ? 0.5 : u[1];
    v3 o, d;
    cam_ray(s, a->W, a->H, px, py, jx, jy, &o, &d);
    double beta[3] = {1.0, 1.0, 1.0};
    double opl = 0.0;
    double prev_pdf = 0.0;  /* solid-angle pdf of the direction that produced this ray */
    int media = s->has_medium;
    int strat = a->strategy;
    vlist_t vl;
    vl.tri[0] = -2;
    cx->cnt[3]++;
    for (int depth = 1; depth <= a->max_depth; depth++) {
        double th;
        int64_t hit = closest(s, o, d, INFINITY, 0, &th);
        cx->cnt[1]++;
        /* participating medium: delta tracking along [0, th] (Sec. 4.1) */
        if (media) {
            double ma, mb;
            double tsurf = hit >= 0 ? th : 1e30;
            if (medium_span(s, o, d, tsurf, &ma, &mb)) {
                double t = ma;
                int collided = 0;
                for (uint32_t j = 0;; j++) {
                    if (j >= MO_TRACK_STEPS) return;
                    rng4(seed, pix, smp, (uint32_t)(depth - 1), G_TRACK + j, u);
                    t += -log(1.0 - u[0]) / s->m_major;
                    if (t >= mb) break;
                    if (u[1] < dens(s, add(o, scl(d, t))) / s->m_major) { collided = 1; break; }
                }
                if (collided) {
                    /* real collision: medium vertex */
                    cx->cnt[0]++;
                    v3 x = add(o, scl(d, t));
                    if (!(depth == 1 && (a->flags & MO_UNWARP))) opl += t;
                    for (int k = 0; k < 3; k++) beta[k] *= s->m_albedo;
                    vl.tri[depth] = -1;
                    for (int k = 0; k < 3; k++) vl.ratio[depth][k] = 1.0 / s->m_albedo;
                    if (depth == a->max_depth) return;
                    /* next-event estimate through the medium (ratio tracking) */
                    if (s->n_units > 0 && strat != MO_STRAT_BSDF_ONLY) {
                        rng4(seed, pix, smp, (uint32_t)depth, G_NEE, u);
                        int64_t un = pick_unit(s, u[0]);
                        int32_t em = s->unit_em[un];
                        v3 y, ny = mk(0, 0, 0);
                        int is_pt = s->unit_tri[un] < 0;
                        if (is_pt) y = s->em_pos[em];
                        else { y = tri_point(s, s->unit_tri[un], u[1], u[2]); ny = s->ng[s->unit_tri[un]]; }
                        v3 dl = sub(y, x);
                        double dist = len(dl);
                        v3 wi = scl(dl, 1.0 / dist);
                        double cy = is_pt ? 1.0 : -dot(ny, wi);
                        if (cy > 0.0 && dist > 0.0) {
                            double tmax = dist - (is_pt ? 0.0 : eps_of(y));
                            cx->cnt[1]++;
                            if (!occluded(s, x, wi, tmax, 0)) {
                                int ok;
                                double Tr = transmittance(s, x, wi, tmax, seed, pix, smp, (uint32_t)depth, &ok);
                                if (ok && Tr != 0.0) {
                                    double ph = mo_hg_eval(s->m_g, dot(d, wi));
                                    double geo = is_pt ? 1.0 / (dist * dist) : cy / (dist * dist) / (s->unit_p[un] / s->area[s->unit_tri[un]]);
                                    if (is_pt) geo /= s->unit_p[un];
                                    double c[3], cb[3];
                                    for (int k = 0; k < 3; k++) {
                                        cb[k] = beta[k] * ph * Tr * geo;
                                        c[k] = cb[k] * s->em_rad[3 * em + k];
                                    }
                                    deposit(cx, (int32_t)pix, lp, (int32_t)smp, depth, 1,
                                            (int32_t)s->unit_tri[un], opl + dist, c, cb, em, &vl, depth, NULL);
                                }
                            }
                        }
                    }
                    rng4(seed, pix, smp, (uint32_t)depth, G_SCATTER, u);
                    v3 wi = hg_sample(s->m_g, d, u[0], u[1]);
                    o = x; d = wi;
                    continue;
                }
            }
        }
        if (hit < 0) return;
        cx->cnt[0]++;
        v3 x = add(o, scl(d, th));
        if (!(depth == 1 && (a->flags & MO_UNWARP))) opl += th;
        v3 wo = scl(d, -1.0);
        v3 ng = s->ng[hit];
        /* emission found by the path: one-sided, front face = winding normal */
        int32_t em = s->tri_em[hit];
        if (em >= 0 && dot(ng, wo) > 0.0) {
            double w = 1.0;
            int count = 1;
            if (depth > 1) {
                if (media || strat == MO_STRAT_NEE_ONLY) count = 0;
                else if (strat == MO_STRAT_MIS) {
                    double pl = s->tri_lpdf[hit] * th * th / dot(ng, wo);
                    w = mis2(prev_pdf, pl);
                }
            }
            if (count) {
                double c[3], cb[3];
                for (int k = 0; k < 3; k++) { cb[k] = beta[k] * w; c[k] = cb[k] * s->em_rad[3 * em + k]; }
                deposit(cx, (int32_t)pix, lp, (int32_t)smp, depth, 0, (int32_t)hit, opl, c, cb, em, &vl, depth - 1, NULL);
            }
        }
        if (depth == a->max_depth) return;
        if (s->delay && s->delay[hit] > 0.0) {
            /* scattering delay of this vertex: every contribution formed here or later carries it */
            rng4(seed, pix, smp, (uint32_t)depth, G_DELAY, u);
            opl += -s->delay[hit] * log(1.0 - u[0]);
        }
        v3 n = side_normal(ng, wo), t, b;
        basis(n, &t, &b);
        v3 wol = to_local(wo, t, b, n);
        const double *alb = s->albedo + 3 * hit;
        uint32_t ty = s->type[hit];
        double rgh = s->rough[hit];
        vl.tri[depth] = (int32_t)hit;
        /* next-event estimation (with power-heuristic MIS) */
        if (s->n_units > 0 && strat != MO_STRAT_BSDF_ONLY) {
            rng4(seed, pix, smp, (uint32_t)depth, G_NEE, u);
            int64_t un = pick_unit(s, u[0]);
            int32_t eml = s->unit_em[un];
            int is_pt = s->unit_tri[un] < 0;
            v3 y, ny = mk(0, 0, 0);
            if (is_pt) y = s->em_pos[eml];
            else { y = tri_point(s, s->unit_tri[un], u[1], u[2]); ny = s->ng[s->unit_tri[un]]; }
            v3 xo = offset(x, n);
            v3 dl = sub(y, xo);
            double dist = len(dl);
            v3 wi = scl(dl, 1.0 / dist);
            double cx_ = dot(n, wi);
            double cy = is_pt ? 1.0 : -dot(ny, wi);
            if (cx_ > 0.0 && cy > 0.0) {
                double tmax = dist - (is_pt ? 0.0 : eps_of(y));
                cx->cnt[1]++;
                if (!occluded(s, xo, wi, tmax, 0)) {
                    int ok = 1;
                    double Tr = media ? transmittance(s, xo, wi, tmax, seed, pix, smp, (uint32_t)depth, &ok) : 1.0;
                    if (ok && Tr != 0.0) {
                        v3 wil = to_local(wi, t, b, n);
                        double f[3], pb;
                        bsdf_local(ty, alb, rgh, wol, wil, f, &pb);
                        double geo, w = 1.0;
                        if (is_pt) geo = 1.0 / (dist * dist) / s->unit_p[un];
                        else {
                            double pA = s->unit_p[un] / s->area[s->unit_tri[un]];
                            geo = cy / (dist * dist) / pA;
                            if (!media && strat == MO_STRAT_MIS) w = mis2(pA * dist * dist / cy, pb);
                        }
                        double c[3], cb[3], own[3];
                        for (int k = 0; k < 3; k++) {
                            cb[k] = beta[k] * f[k] * cx_ * geo * w * Tr;
                            c[k] = cb[k] * s->em_rad[3 * eml + k];
                        }
                        bsdf_dratio(ty, alb, wol, wil, own);
                        if (c[0] != 0.0 || c[1] != 0.0 || c[2] != 0.0 || cx->backward)
                            deposit(cx, (int32_t)pix, lp, (int32_t)smp, depth, 1, (int32_t)s->unit_tri[un],
                                    opl + dist, c, cb, eml, &vl, depth, own);
                    }
                }
            }
        }
        /* continue by sampling the BSDF */
        rng4(seed, pix, smp, (uint32_t)depth, G_SCATTER, u);
        v3 wil;
        if (!bsdf_sample_local(ty, rgh, wol, u[0], u[1], &wil)) return;
        double f[3], pb;
        bsdf_local(ty, alb, rgh, wol, wil, f, &pb);
        if (pb <= 0.0) return;
        for (int k = 0; k < 3; k++) beta[k] *= f[k] * wil.z / pb;
        bsdf_dratio(ty, alb, wol, wil, vl.ratio[depth]);
        prev_pdf = pb;
        v3 wi = to_world(wil, t, b, n);
        o = offset(x, n);
        d = wi;
    }
}

static int run(ctx_t *cx) {
    const mo_args *a = cx->a;
    if (a->x0 < 0 || a->x1 > a->W || a->y0 < 0 || a->y1 > a->H || a->x0 > a->x1 || a->y0 > a->y1) return 1;
    if (a->max_depth > MO_MAX_DEPTH || a->max_depth < 1 || a->spp < 0 || a->T < 0) return 1;
    int cw = a->x1 - a->x0;
    for (int py = a->y0; py < a->y1; py++)
        for (int px = a->x0; px < a->x1; px++) {
            int32_t lp = (py - a->y0) * cw + (px - a->x0);
            for (int32_t sI = 0; sI < a->spp; sI++)
                trace_path(cx, px, py, lp, (uint32_t)(a->sample_offset + (uint64_t)sI));
        }
    return 0;
}

int mo_render(const mo_scene *s, const mo_args *a, double *film, double *steady, double *dropped,
              mo_contrib *dump, int64_t dump_cap, int64_t *n_dump, uint64_t *counters) {
    ctx_t cx;
    memset(&cx, 0, sizeof(cx));
    cx.s = s; cx.a = a; cx.film = film; cx.steady = steady; cx.dropped = dropped;
    cx.dump = dump; cx.dump_cap = dump_cap;
    int64_t npx = (int64_t)(a->x1 - a->x0) * (a->y1 - a->y0);
    if (!(a->flags & MO_ACCUMULATE)) {
        memset(film, 0, sizeof(double) * (size_t)(npx * a->T * 3));
        if (steady) memset(steady, 0, sizeof(double) * (size_t)(npx * 3));
        if (dropped) memset(dropped, 0, sizeof(double) * (size_t)(npx * 3));
    }
    /* accumulate into scratch so that ACCUMULATE adds unnormalised sums */
    int rc = run(&cx);
    if (rc) return rc;
    if (!(a->flags & MO_ACCUMULATE) && a->spp > 0) {
        double inv = 1.0 / a->spp;
        for (int64_t i = 0; i < npx * a->T * 3; i++) film[i] *= inv;
        if (steady) for (int64_t i = 0; i < npx * 3; i++) steady[i] *= inv;
        if (dropped) for (int64_t i = 0; i < npx * 3; i++) dropped[i] *= inv;
    }
    if (n_dump) *n_dump = cx.n_dump;
    if (counters) for (int k = 0; k < 4; k++) counters[k] += cx.cnt[k];
    return 0;
}

/* Frequency-space rendering (Sec. 4.3, Eq. 12): the same paths, each
 * contribution adding C * exp(-i * 2 pi * tof / lambda_k) for K wavelengths
 * (lambda in metres, tof as optical path length).  phasor is [px][K][2][3]
 * (real RGB, imaginary RGB), normalised by 1/spp unless MO_ACCUMULATE. */
int mo_render_phasor(const mo_scene *s, const mo_args *a0, const double *lambdas, int32_t K, double *phasor,
                     double *steady) {
    mo_args a = *a0;
    a.T = 0; /* no time bins: every contribution goes to the phasors and the steady image */
    ctx_t cx;
    memset(&cx, 0, sizeof(cx));
    double dummy = 0.0;
    cx.s = s; cx.a = &a; cx.film = &dummy; cx.steady = steady;
    cx.phasor = phasor; cx.lambdas = lambdas; cx.K = K;
    int64_t npx = (int64_t)(a.x1 - a.x0) * (a.y1 - a.y0);
    if (K < 1) return 1;
    for (int32_t q = 0; q < K; q++) if (!(lambdas[q] > 0.0)) return 1;
    if (!(a.flags & MO_ACCUMULATE)) {
        memset(phasor, 0, sizeof(double) * (size_t)(npx * K * 6));
        if (steady) memset(steady, 0, sizeof(double) * (size_t)(npx * 3));
    }
    int rc = run(&cx);
    if (rc) return rc;
    if (!(a.flags & MO_ACCUMULATE) && a.spp > 0) {
        double inv = 1.0 / a.spp;
        for (int64_t i = 0; i < npx * K * 6; i++) phasor[i] *= inv;
        if (steady) for (int64_t i = 0; i < npx * 3; i++) steady[i] *= inv;
    }
    return 0;
}

/* Backward (Sec. 4.4): for L(I) with dL/dI = grad_film (and grad_steady), each
 * contribution C_k of a path is a product of per-vertex factors, so
 * dL/dtheta = (1/N) sum_k g_k * C_k * (d factor / factor) over the vertices
 * that carry theta; radiance enters linearly. The 1/N factor of Eq. 9 is
 * applied here unless MO_ACCUMULATE is set. Gradients are accumulated. */
int mo_render_backward(const mo_scene *s, const mo_args *a, const double *grad_film,
                       const double *grad_steady, double *grad_albedo, double *grad_radiance,
                       double *grad_medium_albedo) {
    ctx_t cx;
    memset(&cx, 0, sizeof(cx));
    cx.s = s; cx.a = a; cx.backward = 1;
    cx.gfilm = grad_film; cx.gsteady = grad_steady;
    int64_t n = s->n, ne = s->n_em;
    double *ga = (double *)calloc((size_t)(n * 3 + 1), sizeof(double));
    double *gr = (double *)calloc((size_t)(ne * 3 + 1), sizeof(double));
    double gm = 0.0;
    cx.galb = ga; cx.grad = gr; cx.gmed = &gm;
    int rc = run(&cx);
    if (rc) { free(ga); free(gr); return rc; }
    double sc = (!(a->flags & MO_ACCUMULATE) && a->spp > 0) ? 1.0 / a->spp : 1.0;
    for (int64_t i = 0; i < n * 3; i++) grad_albedo[i] += ga[i] * sc;
    for (int64_t i = 0; i < ne * 3; i++) grad_radiance[i] += gr[i] * sc;
    if (grad_medium_albedo) *grad_medium_albedo += gm * sc;
    free(ga); free(gr);
    return 0;
}

/* Forward-mode derivative (Sec. 4.4, forward mode): the film of
 * dI/dtheta . dtheta for one tangent direction over per-triangle albedos
 * (dalb [n][3], NULL = 0), emitter radiances (drad [n_em][3], NULL = 0) and
 * the medium albedo (dmed).  tfilm / tsteady are crop-sized like mo_render's
 * film / steady and are overwritten (accumulated with MO_ACCUMULATE). */
int mo_render_tangent(const mo_scene *s, const mo_args *a, const double *dalb, const double *drad, double dmed,
                      double *tfilm, double *tsteady) {
    ctx_t cx;
    memset(&cx, 0, sizeof(cx));
    cx.s = s; cx.a = a; cx.tangent = 1;
    cx.dalb = dalb; cx.drad = drad; cx.dmed = dmed;
    cx.film = tfilm; cx.steady = tsteady;
    int64_t npx = (int64_t)(a->x1 - a->x0) * (a->y1 - a->y0);
    if (!(a->flags & MO_ACCUMULATE)) {
        memset(tfilm, 0, sizeof(double) * (size_t)(npx * a->T * 3));
        if (tsteady) memset(tsteady, 0, sizeof(double) * (size_t)(npx * 3));
    }
    int rc = run(&cx);
    if (rc) return rc;
    if (!(a->flags & MO_ACCUMULATE) && a->spp > 0) {
        double sc = 1.0 / a->spp;
        for (int64_t i = 0; i < npx * a->T * 3; i++) tfilm[i] *= sc;
        if (tsteady) for (int64_t i = 0; i < npx * 3; i++) tsteady[i] *= sc;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Transient polarization (Sec. 4.2, "Transient polarization tracking"):      */
/* a Stokes vector (S0..S3) per colour channel and time bin.                  */
/*                                                                            */
/* Conventions: a Stokes vector of light propagating along k is given in a    */
/* reference frame x (unit, perpendicular to k), y = k x x; S1 = I_x - I_y,   */
/* S2 = I(+45) - I(-45).  Expressing it in a frame x' = cos(t) x + sin(t) y   */
/* multiplies it by R(t) (rows 1, 2 rotated by 2t).  The throughput of a path */
/* is a 4x4 Mueller matrix per channel mapping light leaving the current      */
/* vertex toward the camera (in the segment's frame) to the Stokes vector the */
/* camera measures (frame x = the camera's horizontal axis).  Emitters emit   */
/* unpolarised light.  Lambert is an ideal depolariser; the GGX conductor     */
/* reflects at its microfacet with the Fresnel Mueller matrix of a complex    */
/* index 1 + i kappa, kappa = 2 sqrt(F0 / (1 - F0)) (normal-incidence         */
/* reflectance F0), in the s/p frames of the scattering plane.                */
/* ------------------------------------------------------------------------- */
typedef struct { double m[4][4]; } mat4;

static mat4 m4_ident(double v) {
    mat4 r;
    memset(&r, 0, sizeof(r));
    for (int i = 0; i < 4; i++) r.m[i][i] = v;
    return r;
}
static mat4 m4_mul(const mat4 *a, const mat4 *b) {
    mat4 r;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double acc = 0.0;
            for (int k = 0; k < 4; k++) acc += a->m[i][k] * b->m[k][j];
            r.m[i][j] = acc;
        }
    return r;
}
static mat4 m4_scale(const mat4 *a, double v) {
    mat4 r;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) r.m[i][j] = a->m[i][j] * v;
    return r;
}
/* Stokes rotation into a frame turned by t about the propagation direction */
static mat4 m4_rot(double t) {
    mat4 r = m4_ident(1.0);
    double c = cos(2.0 * t), s = sin(2.0 * t);
    r.m[1][1] = c; r.m[1][2] = s;
    r.m[2][1] = -s; r.m[2][2] = c;
    return r;
}
/* angle t with x_to = cos t x_from + sin t (k x x_from) */
static double frame_angle(v3 k, v3 x_from, v3 x_to) {
    return atan2(dot(x_to, cross(k, x_from)), dot(x_to, x_from));
}
/* unit vector perpendicular to the plane of a and b, or to a alone when they are parallel */
static v3 plane_normal(v3 a, v3 b) {
    v3 c = cross(a, b);
    double l = len(c);
    if (l > 1e-12) return scl(c, 1.0 / l);
    v3 t, bb;
    basis(a, &t, &bb);
    return t;
}
/* Fresnel reflection Mueller matrix at incidence cosine ci, index 1 + i kappa, in s/p frames */
static mat4 fresnel_mueller(double ci, double kappa) {
    double complex N = 1.0 + I * kappa;
    double s2 = 1.0 - ci * ci;
    double complex ct = csqrt(1.0 - s2 / (N * N));
    double complex rs = (ci - N * ct) / (ci + N * ct);
    double complex rp = (N * ci - ct) / (N * ci + ct);
    double Rs = creal(rs * conj(rs)), Rp = creal(rp * conj(rp));
    double complex X = rs * conj(rp);
    mat4 m;
    memset(&m, 0, sizeof(m));
    m.m[0][0] = m.m[1][1] = 0.5 * (Rs + Rp);
    m.m[0][1] = m.m[1][0] = 0.5 * (Rs - Rp);
    m.m[2][2] = m.m[3][3] = creal(X);
    m.m[2][3] = cimag(X);
    m.m[3][2] = -cimag(X);
    return m;
}
double mo_conductor_kappa(double F0) {
    double f = F0 < 0.0 ? 0.0 : (F0 > 0.999 ? 0.999 : F0);
    return 2.0 * sqrt(f / (1.0 - f));
}
/* Mueller matrix of one surface vertex for light arriving along -wi (world) and
 * leaving along -d toward the camera, in the frame s = plane normal of (wi, d)
 * for both; scalar factors D G2 / (4 cos cos) included, cosine and pdf not */
static void vertex_mueller(uint32_t ty, const double *alb, double rgh, v3 wol, v3 wil, mat4 M[3]) {
    if (ty == 0) {
        for (int c = 0; c < 3; c++) { memset(&M[c], 0, sizeof(mat4)); M[c].m[0][0] = alb[c] / PI_D; }
        return;
    }
    double a = ggx_alpha(rgh);
    v3 h = nrm(add(wol, wil));
    double D = ggx_D(a, h);
    double G2 = 1.0 / (1.0 + ggx_lambda(a, wol) + ggx_lambda(a, wil));
    double k = D * G2 / (4.0 * wol.z * wil.z);
    double cd = dot(wil, h);
    for (int c = 0; c < 3; c++) {
        mat4 F = fresnel_mueller(cd, mo_conductor_kappa(alb[c]));
        M[c] = m4_scale(&F, k);
    }
}

typedef struct {
    const mo_scene *s;
    const mo_args *a;
    double *film, *steady; /* [px][T][4][3], [px][4][3] */
} pctx_t;

static void pol_deposit(pctx_t *cx, int32_t pix_full, int32_t lp, int32_t sample, int depth, int kind, double opl,
                        const double S[3][4]) {
    const mo_args *a = cx->a;
    if (cx->s->pulse_type != MO_PULSE_DELTA) {
        double u[4];
        rng4(a->seed, (uint32_t)pix_full, (uint32_t)sample, (uint32_t)depth, G_PULSE + (uint32_t)kind, u);
        opl += pulse_time(cx->s, u);
    }
    double fb = floor((opl - a->start) / a->width);
    int in = fb >= 0.0 && fb < (double)a->T;
    for (int k = 0; k < 4; k++)
        for (int c = 0; c < 3; c++) {
            if (in) cx->film[(((int64_t)lp * a->T + (int64_t)fb) * 4 + k) * 3 + c] += S[c][k];
            cx->steady[((int64_t)lp * 4 + k) * 3 + c] += S[c][k];
        }
}

/* the same estimator as trace_path (surfaces only), with Mueller throughput */
static void trace_path_pol(pctx_t *cx, int32_t px, int32_t py, int32_t lp, uint32_t smp) {
    const mo_scene *s = cx->s;
    const mo_args *a = cx->a;
    uint32_t pix = (uint32_t)(py * a->W + px);
    uint64_t seed = a->seed;
    double u[4];
    rng4(seed, pix, smp, 0, 0, u);
    double jx = (a->flags & MO_PIXEL_CENTER) ? 0.5 : u[0];
    double jy = (a->flags & MO_PIXEL_CENTER) ? 0.5 : u[1];
    v3 o, d;
    cam_ray(s, a->W, a->H, px, py, jx, jy, &o, &d);
    mat4 P[3];
    for (int c = 0; c < 3; c++) P[c] = m4_ident(1.0);
    v3 xf = nrm(sub(s->cam_r, scl(d, dot(s->cam_r, d))));  /* frame of the current segment */
    double opl = 0.0, prev_pdf = 0.0;
    for (int depth = 1; depth <= a->max_depth; depth++) {
        double th;
        int64_t hit = closest(s, o, d, INFINITY, 0, &th);
        if (hit < 0) return;
        v3 x = add(o, scl(d, th));
        if (!(depth == 1 && (a->flags & MO_UNWARP))) opl += th;
        v3 wo = scl(d, -1.0);
        v3 ng = s->ng[hit];
        int32_t em = s->tri_em[hit];
        if (em >= 0 && dot(ng, wo) > 0.0) {
            double w = 1.0;
            if (depth > 1) {
                double pl = s->tri_lpdf[hit] * th * th / dot(ng, wo);
                w = mis2(prev_pdf, pl);
            }
            double S[3][4];
            for (int c = 0; c < 3; c++)
                for (int k = 0; k < 4; k++) S[c][k] = P[c].m[k][0] * s->em_rad[3 * em + c] * w;
            pol_deposit(cx, (int32_t)pix, lp, (int32_t)smp, depth, 0, opl, S);
        }
        if (depth == a->max_depth) return;
        if (s->delay && s->delay[hit] > 0.0) {
            rng4(seed, pix, smp, (uint32_t)depth, G_DELAY, u);
            opl += -s->delay[hit] * log(1.0 - u[0]);
        }
        v3 n = side_normal(ng, wo), t, b;
        basis(n, &t, &b);
        v3 wol = to_local(wo, t, b, n);
        const double *alb = s->albedo + 3 * hit;
        uint32_t ty = s->type[hit];
        double rgh = s->rough[hit];
        if (s->n_units > 0) {
            rng4(seed, pix, smp, (uint32_t)depth, G_NEE, u);
            int64_t un = pick_unit(s, u[0]);
            int32_t eml = s->unit_em[un];
            int is_pt = s->unit_tri[un] < 0;
            v3 y, ny = mk(0, 0, 0);
            if (is_pt) y = s->em_pos[eml];
            else { y = tri_point(s, s->unit_tri[un], u[1], u[2]); ny = s->ng[s->unit_tri[un]]; }
            v3 xo = offset(x, n);
            v3 dl = sub(y, xo);
            double dist = len(dl);
            v3 wi = scl(dl, 1.0 / dist);
            double cx_ = dot(n, wi), cy = is_pt ? 1.0 : -dot(ny, wi);
            if (cx_ > 0.0 && cy > 0.0) {
                double tmax = dist - (is_pt ? 0.0 : eps_of(y));
                if (!occluded(s, xo, wi, tmax, 0)) {
                    v3 wil = to_local(wi, t, b, n);
                    double f[3], pb;
                    bsdf_local(ty, alb, rgh, wol, wil, f, &pb);
                    if (pb > 0.0 || ty == 0) {
                        double geo, w = 1.0;
                        if (is_pt) geo = 1.0 / (dist * dist) / s->unit_p[un];
                        else {
                            double pA = s->unit_p[un] / s->area[s->unit_tri[un]];
                            geo = cy / (dist * dist) / pA;
                            w = mis2(pA * dist * dist / cy, pb);
                        }
                        mat4 Mv[3];
                        vertex_mueller(ty, alb, rgh, wol, wil, Mv);
                        v3 sv = plane_normal(wi, d);
                        mat4 R = m4_rot(frame_angle(wo, sv, xf));
                        double S[3][4];
                        for (int c = 0; c < 3; c++) {
                            mat4 A = m4_mul(&P[c], &R);
                            mat4 B = m4_mul(&A, &Mv[c]);
                            double k = cx_ * geo * w * s->em_rad[3 * eml + c];
                            for (int q = 0; q < 4; q++) S[c][q] = B.m[q][0] * k;
                        }
                        pol_deposit(cx, (int32_t)pix, lp, (int32_t)smp, depth, 1, opl + dist, S);
                    }
                }
            }
        }
        rng4(seed, pix, smp, (uint32_t)depth, G_SCATTER, u);
        v3 wil;
        if (!bsdf_sample_local(ty, rgh, wol, u[0], u[1], &wil)) return;
        double f[3], pb;
        bsdf_local(ty, alb, rgh, wol, wil, f, &pb);
        if (pb <= 0.0) return;
        v3 wi = to_world(wil, t, b, n);
        mat4 Mv[3];
        vertex_mueller(ty, alb, rgh, wol, wil, Mv);
        v3 sv = plane_normal(wi, d);
        mat4 R = m4_rot(frame_angle(wo, sv, xf));
        for (int c = 0; c < 3; c++) {
            mat4 A = m4_mul(&P[c], &R);
            mat4 B = m4_mul(&A, &Mv[c]);
            P[c] = m4_scale(&B, wil.z / pb);
        }
        xf = sv;
        prev_pdf = pb;
        o = offset(x, n);
        d = wi;
    }
}

/* Stokes film [crop px][T][4][3] and steady [crop px][4][3] (divided by spp
 * unless MO_ACCUMULATE); scenes with a medium are rejected (returns 1). */
int mo_render_polarized(const mo_scene *s, const mo_args *a, double *film, double *steady) {
    if (s->has_medium) return 1;
    if (a->x0 < 0 || a->x1 > a->W || a->y0 < 0 || a->y1 > a->H || a->x0 > a->x1 || a->y0 > a->y1) return 1;
    if (a->max_depth > MO_MAX_DEPTH || a->max_depth < 1 || a->spp < 0 || a->T < 0) return 1;
    pctx_t cx = {s, a, film, steady};
    int64_t npx = (int64_t)(a->x1 - a->x0) * (a->y1 - a->y0);
    if (!(a->flags & MO_ACCUMULATE)) {
        memset(film, 0, sizeof(double) * (size_t)(npx * a->T * 12));
        memset(steady, 0, sizeof(double) * (size_t)(npx * 12));
    }
    int cw = a->x1 - a->x0;
    for (int py = a->y0; py < a->y1; py++)
        for (int px = a->x0; px < a->x1; px++) {
            int32_t lp = (py - a->y0) * cw + (px - a->x0);
            for (int32_t sI = 0; sI < a->spp; sI++)
                trace_path_pol(&cx, px, py, lp, (uint32_t)(a->sample_offset + (uint64_t)sI));
        }
    if (!(a->flags & MO_ACCUMULATE) && a->spp > 0) {
        double sc = 1.0 / a->spp;
        for (int64_t i = 0; i < npx * a->T * 12; i++) film[i] *= sc;
        for (int64_t i = 0; i < npx * 12; i++) steady[i] *= sc;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* NLOS relay-wall capture (Sec. 4.5): third-bounce transport                 */
/*   laser -> x_l -> y -> x_s -> sensor with y drawn uniformly by area on     */
/*   the hidden mesh; the clock is the relay-wall clock |x_l-y| + |y-x_s|.    */
/* ------------------------------------------------------------------------- */
int mo_render_nlos(const mo_scene *s, int32_t hidden_first, int32_t hidden_n, const double *wall_normal,
                   double wall_albedo, const float *lasers, int32_t n_l, const float *sensors, int32_t n_s,
                   int32_t exhaustive, int64_t pair0, int64_t pair1, int32_t T, double start, double width,
                   int32_t spp, uint64_t seed, uint64_t sample_offset, uint32_t flags, double *film,
                   double *steady, mo_contrib *dump, int64_t dump_cap, int64_t *n_dump, uint64_t *counters) {
    if (hidden_n <= 0 || hidden_first < 0 || hidden_first + hidden_n > s->n) return 1;
    int64_t npairs = exhaustive ? (int64_t)n_l * n_s : n_l;
    if (pair0 < 0 || pair1 > npairs || pair0 > pair1) return 1;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)hidden_n);
    double tot = 0.0;
    for (int32_t i = 0; i < hidden_n; i++) { tot += s->area[hidden_first + i]; cdf[i] = tot; }
    for (int32_t i = 0; i < hidden_n; i++) cdf[i] /= tot;
    cdf[hidden_n - 1] = 1.0;
    v3 nw = ld(wall_normal);
    double fw = wall_albedo / PI_D;
    int64_t nd = 0;
    uint64_t cnt[4] = {0, 0, 0, 0};
    int64_t np = pair1 - pair0;
    if (!(flags & MO_ACCUMULATE)) {
        memset(film, 0, sizeof(double) * (size_t)(np * T));
        if (steady) memset(steady, 0, sizeof(double) * (size_t)np);
    }
    for (int64_t pr = pair0; pr < pair1; pr++) {
        int32_t li = exhaustive ? (int32_t)(pr / n_s) : (int32_t)pr;
        int32_t si = exhaustive ? (int32_t)(pr % n_s) : (int32_t)pr;
        const float *lp = lasers + 3 * li;
        const float *sp = exhaustive ? sensors + 3 * si : lasers + 3 * li;
        v3 xl = mk(lp[0], lp[1], lp[2]), xs = mk(sp[0], sp[1], sp[2]);
        int64_t row = pr - pair0;
        for (int32_t j = 0; j < spp; j++) {
            uint32_t smp = (uint32_t)(sample_offset + (uint64_t)j);
            double u[4];
            rng4(seed, (uint32_t)li, smp, 0, 0, u);
            int32_t lo = 0, hi = hidden_n - 1;
            while (lo < hi) { int32_t m = (lo + hi) / 2; if (u[0] < cdf[m]) hi = m; else lo = m + 1; }
            int64_t tri = hidden_first + lo;
            v3 y = tri_point(s, tri, u[1], u[2]);
            cnt[3]++;
            v3 d1v = sub(y, xl), d2v = sub(xs, y);
            double d1 = len(d1v), d2 = len(d2v);
            if (d1 <= 0.0 || d2 <= 0.0) continue;
            v3 w1 = scl(d1v, 1.0 / d1), w2 = scl(d2v, 1.0 / d2);
            double cl = dot(nw, w1), cs = -dot(nw, w2);
            v3 ny = side_normal(s->ng[tri], scl(w1, -1.0));
            double cy1 = -dot(ny, w1), cy2 = dot(ny, w2);
            if (cl <= 0.0 || cs <= 0.0 || cy1 <= 0.0 || cy2 <= 0.0) continue;
            /* visibility x_l -> y (laser side), y -> x_s (sensor side) */
            v3 xlo = offset(xl, nw);
            v3 r1 = sub(y, xlo);
            double l1 = len(r1);
            cnt[1]++;
            if (occluded(s, xlo, scl(r1, 1.0 / l1), l1 - eps_of(y), 0)) continue;
            if (exhaustive) {
                v3 yo = offset(y, ny);
                v3 r2 = sub(xs, yo);
                double l2 = len(r2);
                cnt[1]++;
                if (occluded(s, yo, scl(r2, 1.0 / l2), l2 - eps_of(xs), 0)) continue;
            }
            const double *al = s->albedo + 3 * tri;
            double fh = (al[0] + al[1] + al[2]) / 3.0 / PI_D;
            double H = fw * cl * fh * cy1 * cy2 / (d1 * d1 * d2 * d2) * cs * fw * tot;
            double opl = d1 + d2;
            double x = (opl - start) / width;
            double fb = floor(x);
            int32_t bin = (fb < -1e9) ? -1000000000 : (fb > 1e9 ? 1000000000 : (int32_t)fb);
            cnt[2]++;
            if (bin >= 0 && bin < T) film[row * T + bin] += H;
            if (steady) steady[row] += H;
            if (dump) {
                if (nd < dump_cap) {
                    mo_contrib *r = &dump[nd];
                    r->pixel = (int32_t)pr; r->sample = (int32_t)smp; r->depth = 2; r->kind = 2;
                    r->tri = (int32_t)tri; r->bin = bin; r->opl = opl;
                    r->c[0] = H; r->c[1] = r->c[2] = 0.0;
                }
                nd++;
            }
        }
    }
    if (!(flags & MO_ACCUMULATE) && spp > 0) {
        double inv = 1.0 / spp;
        for (int64_t i = 0; i < np * T; i++) film[i] *= inv;
        if (steady) for (int64_t i = 0; i < np; i++) steady[i] *= inv;
    }
    if (n_dump) *n_dump = nd;
    if (counters) for (int k = 0; k < 4; k++) counters[k] += cnt[k];
    free(cdf);
    return 0;
}
