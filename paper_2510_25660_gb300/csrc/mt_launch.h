// mt_launch.h -- parameter blocks passed from the C-ABI layer to the kernels.
#pragma once
#include <cstddef>
#include <cstdint>

#include "../../include/mt_api.h"
#include "mt_common.cuh"

#define MT_MAX_BWD_DEPTH 16

struct RenderParams {
    int32_t H, W, T, D;        // film size; D = bins per pixel privatised in shared memory
    int32_t H_full, row0;      // the film holds rows [row0, row0 + H) of an H_full x W frame
    uint32_t pix_base;         // row0 * W: frame pixel id of the film's first pixel
    float start, width, scale; // time window (OPL metres) and 1/spp (1 when accumulating)
    uint32_t flags;
    int32_t spp, max_depth;
    uint32_t sample_offset;
    uint32_t k0, k1;           // Philox key = seed
    int32_t tile_px, n_tiles, tiles_per_row;  // tile = tile_px pixels of one row, owned by one warp
    float *film, *steady;
    const float *gfilm, *gsteady;
    float *galb, *grad, *gmed;
    mt_contrib *dump;
    long long dump_cap;
    unsigned long long *dump_count;
    int *tile_counter;
    int32_t n_em_smem;         // emitters whose radiance gradients are summed in shared memory
    int32_t aggregate;         // warp-aggregated splats
    int32_t refill_min;        // idle lanes needed before a warp starts new paths (1..32)
    const float *lambdas;      // frequency-space film: K wavelengths (m); the film has T = 2K
    int32_t K;
    const float *dalb, *drad;  // forward-mode derivative: tangent of albedos [n][3] and radiances [e][3] (or null)
    float dmed;                // and of the medium albedo
};

struct NlosParams {
    int32_t T, D;
    float start, width, scale;
    uint32_t flags;
    int32_t spp, mode;
    uint32_t sample_offset, k0, k1;
    const float *lasers, *sensors;
    int32_t n_l, n_s;
    float3 nw;
    float fw;                  // wall albedo / pi
    int32_t hidden_first, hidden_n;
    const uint32_t *hcdf;      // ceil(cdf * 2^24) over hidden triangles (original order)
    // optional guide table (MT_HGUIDE_N + 1 entries): hguide[g] = smallest i with (g << 12) < hcdf[i]
    // (hidden_n if none), so the pick of a 24-bit key lies in [hguide[key >> 12], hguide[(key >> 12) + 1]];
    // nullptr = search the whole table
    const uint32_t *hguide;
    float hidden_area;
    const float *hidden_area_dev;  // if set, the hidden area is read from here instead of hidden_area
    int32_t tile, n_tiles;
    float *film, *steady;
    float4 *ysamp;             // exhaustive: 2 per (laser, sample): (y, |x_l - y|), (side normal, partial weight or 0)
    int32_t *ysamp_tri;        // exhaustive: hidden triangle of each sample
    mt_contrib *dump;
    long long dump_cap;
    unsigned long long *dump_count;
    int *tile_counter;
    int32_t aggregate;         // warp-aggregated splats
};

// Path pool layout of the wavefront form.  MT_WF_AOS = 1: one 128-byte record
// per slot, float4 words [o, d, beta, meta, hit, sig, -, -], so the state of a
// path shares cache lines (a shading step reads two and a half 32-byte sectors
// and a new path writes two whole sectors); 0: one array per field.
#ifndef MT_WF_AOS
#define MT_WF_AOS 1
#endif
#define MT_WF_REC (MT_WF_AOS ? 8 : 1)  // float4 words between the fields of consecutive slots

// one field of the path pool, indexed by slot
template <class T>
struct PoolField {
    T *base;
    __host__ __device__ __forceinline__ T &operator[](size_t slot) const { return base[slot * MT_WF_REC]; }
    __host__ __device__ __forceinline__ explicit operator bool() const { return base != nullptr; }
};

#define MT_WF_POOL_DEFAULT (1u << 22)  // paths in flight of the wavefront form unless set per scene

#define MT_HGUIDE_N 4096  // guide-table buckets over the 24-bit keys of the hidden-triangle pick

struct WfParams {
    int32_t H, W, T;
    int32_t H_full, row0;          // film window in the frame (see RenderParams)
    uint32_t pix_base;
    float start, width, scale;
    uint32_t flags;
    int32_t spp, max_depth;
    uint32_t sample_offset, k0, k1;
    unsigned long long total_paths;
    uint32_t P;                    // paths in flight (pool size)
    float *film, *steady;
    PoolField<float4> o, d, beta;  // path state: origin + OPL, direction + pdf of the last BSDF sample, throughput
    PoolField<uint4> meta;         // pixel, sample index, depth
    PoolField<int4> hit;           // leaf-order triangle, original triangle, t bits
    uint32_t *qa, *qb, *free_q;    // extension queues and the free-slot stack
    // Queue-ordered path state (qmode = 1; the forward forms without ray sorting or dynamic fetch): the
    // path at position i of this iteration's extension queue has its state at ps_o[i], ps_d[i], ps_b[i],
    // ps_m[i] (ps_sig[i] for the forward-mode derivative) and its hit at ps_h[i]; shading writes each continuing
    // path to the next iteration's arrays (_n) at its position in the next queue, so every stage reads
    // and writes the state in queue order and no slot index or free-slot stack is involved.
    int32_t qmode;
    float4 *ps_o, *ps_d, *ps_b, *ps_sig;
    uint4 *ps_m;
    float4 *ps_o_n, *ps_d_n, *ps_b_n, *ps_sig_n;
    uint4 *ps_m_n;
    int4 *ps_h;
    float4 *sh_o, *sh_d, *sh_c;    // shadow rays: origin + tmax, direction + OPL, contribution + pixel
    uint4 *sh_m;                   // shadow ray record: sample, depth, emitter triangle
    uint32_t *counters;            // queue counts and cursors
    unsigned long long *next_path;
    struct WfIter *iter;
    mt_contrib *dump;
    long long dump_cap;
    unsigned long long *dump_count;
    unsigned long long *splat_count;  // MT_COUNTERS: film and steady-image splats (each C atomics), else null
    int32_t dynamic_fetch;         // 0: off; else idle lanes of a warp that trigger a fetch (1..32)
    int32_t wide;                  // traverse the 8-wide BVH
    const float *lambdas;          // frequency-space film: K wavelengths (m), the film has T = 2K; K = 0: bins
    int32_t K;
    // forward-mode derivative: per-path prefix sum of ratio * dtheta over the vertices so far, and the tangent
    PoolField<float4> sig;
    const float *dalb, *drad;
    float dmed;
    // path replay (backward): vertex records [vertex][slot] (a: ratio of the continuation + triangle bits,
    // b: sum of g * C of contributions made at the vertex, c: own next-event term), the queue of paths
    // that ended in this iteration, gradient inputs and outputs
    int32_t bwd;
    float4 *rec_a, *rec_b, *rec_c;
    uint32_t *fin_q;
    const float *gfilm, *gsteady;
    float *galb, *grad, *gmed;
    float4 *sh_cb;                 // backward shadow records: own ratio of the next-event direction
    // polarization: per path a 4x4 Mueller throughput per colour (12 float4 rows) and the frame vector
    // of its current segment; shadow records carry a Stokes vector per colour (3 float4); the film is
    // [H][W][T][4][3]
    float4 *mueller, *xframe, *sh_s;
    // ray reordering: extension rays sorted by (direction octant, origin Morton code)
    int32_t sort_rays;
    uint32_t *sort_keys, *sort_keys_out, *sort_q;  // [P] each; sort_q = the sorted queue
    uint32_t *sh_perm;             // shadow rays in sorted order (record indices), null = queue order
    void *sort_tmp;
    size_t sort_tmp_bytes;
    uint32_t *done_flag;  // mapped host word: the setup stage stores done_token in it once the queues
    uint32_t done_token;  // have drained, else 0 (null: no flag); the token differs per render
    // streamed output (null: off): finished paths per band of band_rows film rows, bands flagged as
    // complete, and the mapped host words per band that receive done_token and the flagging iteration
    unsigned long long *band_done;
    uint32_t *band_mark, *band_flag;
    uint32_t band_rows, n_bands;
};

size_t mt_wf_sort_bytes(uint32_t P);

mt_status mt_launch_polarized(const DevScene &s, int32_t H, int32_t W, int32_t T, int32_t H_full, int32_t row0,
                              float start, float width, float scale, uint32_t flags, int32_t spp, int32_t max_depth,
                              uint32_t sample_offset, uint32_t k0, uint32_t k1, float *film, float *steady,
                              int num_sms, cudaStream_t st);

// Per-stage device time of wavefront renders, from CUDA events recorded on the
// render stream at the stage boundaries of every iteration.
struct WfTiming {
    cudaEvent_t *ev = nullptr;  // pool of n_ev events
    int n_ev = 0;
    double ms[4] = {0, 0, 0, 0};  // setup + generate (+ sort), extend, shade, shadow
    long long iters = 0;
};
void mt_wf_timing_free(WfTiming *t);

struct LaunchCfg {
    int threads, tile, ctas_per_sm, num_sms;
    size_t smem_bytes;
    int priv;  // bins per pixel (scan row) kept in shared memory: -1 = as many as fit, 0 = none
    int options;  // MT_OPT_* bits
};

mt_status mt_launch_render(const DevScene &s, const RenderParams &p, const LaunchCfg &cfg, int mode, bool counters,
                           cudaStream_t st);
mt_status mt_launch_nlos(const DevScene &s, const NlosParams &p, const LaunchCfg &cfg, bool dump, bool counters,
                         cudaStream_t st);
// Completion checks of wavefront renders without draining the stream: the setup
// stage writes the "queues drained" flag into mapped host memory and the host
// reads it after waiting on the event of an iteration a few launches back, so
// the GPU always has queued work and no copy-engine transfer is involved.
struct WfSync {
    uint32_t *done_h = nullptr;  // mapped pinned word (host view)
    uint32_t *done_d = nullptr;  // its device view
    cudaEvent_t ev[8] = {};      // end of iteration i: ev[i % 8]
    uint32_t token = 0;          // of the last render (a render still queued may write its own)
    bool ready = false;
};
mt_status mt_wf_sync_init(WfSync *w);
void mt_wf_sync_free(WfSync *w);

// Streamed output of a wavefront render (mt_render_to_host): shading counts the
// finished paths of each band of film rows, a one-block pass after every
// traversal pass flags the bands whose paths have all finished and whose shadow
// rays have all been traced, in mapped host memory, and the host queues each
// flagged band's copy on `copy` behind the event of the iteration that flagged
// it; the bands left at the end are copied behind the render's last stage.
struct WfStreamOut {
    cudaStream_t copy = nullptr;
    float *h_film = nullptr, *h_steady = nullptr;
    const float *d_film = nullptr, *d_steady = nullptr;
    size_t film_row_bytes = 0, steady_row_bytes = 0;
    uint32_t H = 0, band_rows = 0, n_bands = 0;
    unsigned long long *band_done = nullptr;  // device [n_bands]
    uint32_t *band_mark = nullptr;            // device [n_bands]
    uint32_t *flag_h = nullptr, *flag_d = nullptr;  // mapped host [2][n_bands] (host and device views):
                                                    // the render token of a flagged band, then its iteration
    char *issued = nullptr;                   // host [n_bands]: copy queued
    bool used = false;                        // the render streamed its bands
};

mt_status mt_launch_wavefront(const DevScene &s, const WfParams &p, int num_sms, bool dump, bool counters,
                              cudaStream_t st, long long *launches, WfTiming *timing = nullptr,
                              WfSync *sync = nullptr, WfStreamOut *out = nullptr);
