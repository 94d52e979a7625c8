// mt_api.cu -- the C ABI of libmt (declared in include/mt_api.h).
//
// Host-side orchestration only: argument validation, device memory of scenes,
// launch configuration and error reporting.  Every step of the rendering path
// runs in the kernels of mt_render.cu / mt_nlos.cu / mt_bvh.cu or in the small
// set-up kernels below.
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>

#include "mt_common.cuh"
#include <thread>

#include "mt_internal.h"
#include "mt_launch.h"
#include "mt_trace.cuh"

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------
namespace mt {
static thread_local std::string g_err;
void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}
const char *get_error() { return g_err.c_str(); }

static std::atomic<long long> g_alloc_count{0};
static long long fault_at() {
    static long long v = [] {
        const char *e = getenv("MT_FAULT_INJECT");
        if (!e || strncmp(e, "alloc:", 6) != 0) return -1LL;
        return atoll(e + 6);
    }();
    return v;
}

mt_status alloc_device(void **p, size_t bytes, const char *what) {
    const long long k = ++g_alloc_count;
    if (fault_at() > 0 && k == fault_at()) {
        set_error("injected allocation failure (%s, %zu bytes)", what, bytes);
        return MT_ERR_OUT_OF_MEMORY;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MT_ERR_OUT_OF_MEMORY : MT_ERR_CUDA;
    }
    return MT_OK;
}

mt_status alloc_device_async(void **p, size_t bytes, const char *what, cudaStream_t st) {
    const long long k = ++g_alloc_count;
    if (fault_at() > 0 && k == fault_at()) {
        set_error("injected allocation failure (%s, %zu bytes)", what, bytes);
        return MT_ERR_OUT_OF_MEMORY;
    }
    static std::once_flag once;
    std::call_once(once, [] {
        // keep freed blocks of this process's default pool for the next scene build
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = 8ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocAsync of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MT_ERR_OUT_OF_MEMORY : MT_ERR_CUDA;
    }
    return MT_OK;
}
}  // namespace mt

struct mt_film_s {
    int32_t H, W, T, C;
    float start, width;
    float *film, *steady;
    uint32_t flags;
    int32_t H_full, row0;  // window: rows [row0, row0 + H) of an H_full x W frame
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
};

struct mt_scene_s {
    mt::AllocList al;
    DevScene dev{};
    int num_sms = 0;
    int smem_optin = 0;
    int64_t n_tris = 0;
    int32_t n_em = 0;
    BvhResult bvh;
    LaunchCfg cfg[4];
    // scratch
    int *tile_counter = nullptr;   // [4]
    uint32_t *err = nullptr;
    unsigned long long *counters = nullptr;
    float *m_params = nullptr;
    // NLOS state
    int32_t h_first = -1, h_count = -1, h_cap = 0;
    uint32_t *hcdf = nullptr;
    uint32_t *hguide = nullptr;  // MT_HGUIDE_N + 1 entries over hcdf
    double *hprefix = nullptr;   // running sums of the hidden areas (table build)
    float *harea = nullptr;
    float h_area = 0.f;
    float4 *ysamp = nullptr;
    int32_t *ysamp_tri = nullptr;
    long long ysamp_cap = 0;
    GraphCache nlos_graph;
    cudaStream_t cap_stream = nullptr;  // private stream the NLOS graph is captured on
    // wavefront path pool
    long long launches = 0;  // kernels launched by this scene's render calls
    uint32_t wf_cap = 0;       // slots of the shadow-ray records and queue counters
    uint32_t wf_slot_cap = 0;  // slots of the slot-indexed path pool and its queues
    uint32_t wf_q_cap = 0;     // entries of the queue-ordered path state
    float4 *wf_qs = nullptr;   // queue-ordered state: 2 x (o, d, beta, meta, tangent sums) + hits
    uint32_t wf_pool_max = MT_WF_POOL_DEFAULT;  // paths in flight (mt_set_wavefront_pool)
    float4 *wf_o = nullptr, *wf_d = nullptr, *wf_beta = nullptr, *wf_sh_o = nullptr, *wf_sh_d = nullptr,
           *wf_sh_c = nullptr;
    uint4 *wf_meta = nullptr, *wf_sh_m = nullptr;
    int4 *wf_hit = nullptr;
    uint32_t *wf_qa = nullptr, *wf_qb = nullptr, *wf_free = nullptr, *wf_counters = nullptr;
    float4 *wf_sig = nullptr;  // forward-mode prefix sums of the path pool
    float4 *wf_rec = nullptr;   // path replay: vertex records (3 x [max_depth + 1][P])
    uint32_t *wf_fin = nullptr;
    float4 *wf_shown = nullptr;
    size_t wf_rec_cap = 0;      // float4s per record array
    float4 *wf_mueller = nullptr, *wf_xframe = nullptr, *wf_shs = nullptr;  // polarization state of the pool
    uint32_t wf_pol_cap = 0;
    uint32_t *wf_sk = nullptr, *wf_sko = nullptr, *wf_sq = nullptr, *wf_shperm = nullptr;  // ray reordering
    char *wf_stmp = nullptr;
    size_t wf_stmp_bytes = 0;
    uint32_t wf_sort_cap = 0;
    WfTiming wf_timing;  // stage times of wavefront renders (MT_OPT_STAGE_TIMING)
    WfSync wf_sync;      // completion flag and events of wavefront renders
    WfStreamOut *wf_out = nullptr;  // set by mt_render_to_host for the duration of its render
    unsigned long long *so_done = nullptr;  // its per-band buffers (so_cap bands)
    uint32_t *so_mark = nullptr, *so_flag_h = nullptr, *so_flag_d = nullptr;
    char *so_issued = nullptr;
    uint32_t so_cap = 0;
    float *delay_buf = nullptr;  // per-triangle scattering-delay means (mt_scene_set_delays)
    int *check_flag = nullptr;   // validation result of mt_scene_set_delays
    unsigned long long *wf_next = nullptr;
    void *wf_iter = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------
namespace {

// non-finite vertex coordinates and invalid materials (the host checks, on the
// device): sets *bad
__global__ void k_check_inputs(const uint32_t *tri_bits, size_t n_floats, const mt_material *m, int n, int *bad) {
    bool ok = true;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_floats; i += stride)
        ok &= (__ldg(&tri_bits[i]) & 0x7F800000u) != 0x7F800000u;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n; i += stride) {
        const mt_material x = m[i];
        for (int k = 0; k < 3; ++k) ok &= x.albedo[k] >= 0.f && x.albedo[k] < INFINITY;
        ok &= x.type == MT_LAMBERT || x.type == MT_GGX_CONDUCTOR;
        ok &= x.type != MT_GGX_CONDUCTOR || (x.roughness > 0.f && x.roughness <= 1.f);
    }
    if (!ok) atomicOr(bad, 1);
}

__global__ void k_pack_mats(const mt_material *m, int n, float4 *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const mt_material a = m[i];
        out[i] = make_float4(a.albedo[0], a.albedo[1], a.albedo[2], a.type == MT_GGX_CONDUCTOR ? a.roughness : -1.0f);
    }
}

__global__ void k_set_albedo(const float *alb, int n, float4 *mats, const int32_t *leaf_of, float4 *shrec) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 m = mats[i];
        const float4 v = make_float4(alb[3 * i], alb[3 * i + 1], alb[3 * i + 2], m.w);
        mats[i] = v;
        shrec[2 * (size_t)leaf_of[i] + 1] = v;
    }
}

// shading records in leaf order: normal of the winding + light unit, material
__global__ void k_shading_records(const float4 *tris, const float4 *mats, const int32_t *tri_unit, int n,
                                  float4 *shrec) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float4 p0 = tris[3 * k], p1 = tris[3 * k + 1], p2 = tris[3 * k + 2];
        const int orig = __float_as_int(p0.w);
        const float3 ng = normalize(cross(xyz(p1) - xyz(p0), xyz(p2) - xyz(p0)));
        shrec[2 * (size_t)k] = make_float4(ng.x, ng.y, ng.z, __int_as_float(tri_unit[orig]));
        shrec[2 * (size_t)k + 1] = mats[orig];
    }
}

__global__ void k_set_radiance(const float *rad, int n, float4 *em) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        em[i] = make_float4(rad[3 * i], rad[3 * i + 1], rad[3 * i + 2], 0.f);
}

__global__ void k_check_delays(const float *tau, int n, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (!(tau[i] >= 0.0f) || !isfinite(tau[i])) atomicOr(bad, 1);
}

__global__ void k_leaf_of(const float4 *tris, int n, int32_t *leaf_of) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        leaf_of[__float_as_int(tris[3 * k].w)] = k;
}

// double-precision area of a triangle, evaluated without contraction
__device__ double tri_area_d(const float *t) {
    const double ax = __dsub_rn((double)t[3], (double)t[0]), ay = __dsub_rn((double)t[4], (double)t[1]),
                 az = __dsub_rn((double)t[5], (double)t[2]);
    const double bx = __dsub_rn((double)t[6], (double)t[0]), by = __dsub_rn((double)t[7], (double)t[1]),
                 bz = __dsub_rn((double)t[8], (double)t[2]);
    const double cx = __dsub_rn(__dmul_rn(ay, bz), __dmul_rn(az, by));
    const double cy = __dsub_rn(__dmul_rn(az, bx), __dmul_rn(ax, bz));
    const double cz = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
    const double l2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
    return __dmul_rn(0.5, __dsqrt_rn(l2));
}

// Emitter sampling table: units (area-emitter triangles, point emitters)
// weighted by area * mean radiance; the normalised running sum is kept in
// double and stored as ceil(cdf * 2^24) so that comparing the top 24 bits of a
// Philox output against it is the comparison u < cdf.
__global__ void k_setup_units(const float *tris, const int32_t *unit_tri, const int32_t *unit_em, int nu,
                              const mt_emitter *em, LightUnit *units, uint32_t *cdf, int32_t *tri_unit) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double tot = 0.0;
    for (int i = 0; i < nu; ++i) {
        const mt_emitter e = em[unit_em[i]];
        const double mean = __ddiv_rn(__dadd_rn(__dadd_rn((double)e.radiance[0], (double)e.radiance[1]),
                                                (double)e.radiance[2]), 3.0);
        const double a = unit_tri[i] >= 0 ? tri_area_d(tris + 9 * (size_t)unit_tri[i]) : 1.0;
        tot = __dadd_rn(tot, unit_tri[i] >= 0 ? __dmul_rn(a, mean) : mean);
    }
    double acc = 0.0;
    for (int i = 0; i < nu; ++i) {
        const mt_emitter e = em[unit_em[i]];
        const double mean = __ddiv_rn(__dadd_rn(__dadd_rn((double)e.radiance[0], (double)e.radiance[1]),
                                                (double)e.radiance[2]), 3.0);
        const int t = unit_tri[i];
        const double a = t >= 0 ? tri_area_d(tris + 9 * (size_t)t) : 0.0;
        const double w = t >= 0 ? __dmul_rn(a, mean) : mean;
        acc = __dadd_rn(acc, w);
        double c = tot > 0.0 ? __ddiv_rn(acc, tot) : 0.0;
        if (i == nu - 1 && tot > 0.0) c = 1.0;
        const double q = ceil(c * 16777216.0);
        cdf[i] = (uint32_t)(q > 16777216.0 ? 16777216.0 : q);
        LightUnit u;
        const float pick = tot > 0.0 ? (float)__ddiv_rn(w, tot) : 0.0f;
        if (t >= 0) {
            const float *v = tris + 9 * (size_t)t;
            const float3 v0 = f3(v[0], v[1], v[2]), v1 = f3(v[3], v[4], v[5]), v2 = f3(v[6], v[7], v[8]);
            const float3 n = normalize(cross(v1 - v0, v2 - v0));
            u.v0 = make_float4(v0.x, v0.y, v0.z, (float)a);
            u.v1 = make_float4(v1.x, v1.y, v1.z, pick);
            u.v2 = make_float4(v2.x, v2.y, v2.z, __int_as_float(unit_em[i]));
            u.n = make_float4(n.x, n.y, n.z, __int_as_float(t));
            tri_unit[t] = i;
        } else {
            u.v0 = make_float4(e.position[0], e.position[1], e.position[2], 0.f);
            u.v1 = make_float4(0.f, 0.f, 0.f, pick);
            u.v2 = make_float4(0.f, 0.f, 0.f, __int_as_float(unit_em[i]));
            u.n = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        }
        units[i] = u;
    }
}

// hidden-surface area table for NLOS (same construction, weight = area)
// guide[g] = smallest i with (g << 12) < cdf[i], or n if none (g = 0..MT_HGUIDE_N)
__global__ void k_hidden_guide(const uint32_t *cdf, int n, uint32_t *guide) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= MT_HGUIDE_N; g += gridDim.x * blockDim.x) {
        const uint32_t key = (uint32_t)g << 12;
        int lo = 0, hi = n;  // answer in [0, n]
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (key < cdf[mid]) hi = mid;
            else lo = mid + 1;
        }
        guide[g] = (uint32_t)lo;
    }
}

// hidden-surface area table in three passes whose result equals one sequential
// loop in double: the areas in parallel, their running sum in index order by one
// thread (the only order-dependent step), then the quantised CDF in parallel.
__global__ void k_hidden_area(const float4 *t4, const int32_t *leaf_of, int first, int n, double *area) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = leaf_of[first + i];
        const float4 a = t4[3 * k], b = t4[3 * k + 1], c = t4[3 * k + 2];
        const float v[9] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z};
        area[i] = tri_area_d(v);
    }
}

// in place: area[i] -> area[0] + ... + area[i] (left to right, rounded once per addition)
__global__ void k_hidden_prefix(double *acc, int n) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double s = 0.0;
    int i = 0;
    for (; i + 8 <= n; i += 8) {
        double v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = acc[i + j];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            s = __dadd_rn(s, v[j]);
            acc[i + j] = s;
        }
    }
    for (; i < n; ++i) {
        s = __dadd_rn(s, acc[i]);
        acc[i] = s;
    }
}

// cdf[i] = ceil(prefix[i] / total * 2^24), the last entry 2^24; total area as float
__global__ void k_hidden_cdf(const double *prefix, int n, uint32_t *cdf, float *area_out) {
    const double tot = prefix[n - 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double cc = i == n - 1 ? 1.0 : __ddiv_rn(prefix[i], tot);
        const double q = ceil(cc * 16777216.0);
        cdf[i] = (uint32_t)(q > 16777216.0 ? 16777216.0 : q);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *area_out = (float)tot;
}

struct CamOut {
    float o[3], f[3], r[3], u[3], tan_half;
};

__global__ void k_camera(mt_camera c, CamOut *out) {
    const double o[3] = {c.origin[0], c.origin[1], c.origin[2]};
    double f[3] = {c.target[0] - o[0], c.target[1] - o[1], c.target[2] - o[2]};
    double l = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int k = 0; k < 3; ++k) f[k] /= l;
    const double up[3] = {c.up[0], c.up[1], c.up[2]};
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    l = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int k = 0; k < 3; ++k) r[k] /= l;
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    for (int k = 0; k < 3; ++k) {
        out->o[k] = (float)o[k];
        out->f[k] = (float)f[k];
        out->r[k] = (float)r[k];
        out->u[k] = (float)u[k];
    }
    out->tan_half = (float)tan((double)c.fov_x_deg * 3.14159265358979323846 / 360.0);
}

__global__ void k_max(const float *v, size_t n, unsigned int *out) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}

__global__ void k_probe_philox(uint32_t k0, uint32_t k1, const uint4 *c, long long n, uint4 *o) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        o[i] = philox4x32_10(c[i], k0, k1);
}

__global__ void k_probe_trace(const DevScene s, const float *rays, long long n, float tmax, int any, int32_t *tri,
                              float *tt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float *r = rays + 6 * i;
        const RayT ray = make_ray(s, f3(r[0], r[1], r[2]), f3(r[3], r[4], r[5]));
        TraceCnt c{0, 0};
        const bool wide = any & 2;
        float t;
        int orig;
        if (any & 1) {
            tri[i] = (wide ? trace_wide<true, false>(s, ray, tmax, t, orig, c) >= 0 : trace_any<false>(s, ray, tmax, c))
                         ? 1
                         : 0;
        } else {
            const int k = wide ? trace_wide<false, false>(s, ray, tmax, t, orig, c)
                               : trace_closest<false>(s, ray, tmax, t, orig, c);
            tri[i] = k >= 0 ? orig : -1;
            if (tt) tt[i] = k >= 0 ? t : INFINITY;
        }
    }
}

__global__ void k_probe_bins(const float *opl, long long n, float start, float width, int T, int32_t *bin) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = (opl[i] - start) / width;
        bin[i] = (x >= 0.f && x < (float)T) ? (int)x : -1;
    }
}

int grid_for(long long n, int threads, int num_sms) {
    return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, (long long)num_sms * 32));
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define MT_CHECK_ARG(cond, ...)            \
    do {                                   \
        if (!(cond)) {                     \
            mt::set_error(__VA_ARGS__);    \
            return MT_ERR_INVALID_ARGUMENT; \
        }                                  \
    } while (0)

extern "C" {

const char *mt_last_error(void) { return mt::get_error(); }

static mt_status scene_create_impl(const float *tris, int64_t n, const mt_material *mats, const mt_emitter *ems,
                                   int32_t n_em, const mt_camera *cam, const mt_medium *med, cudaStream_t st,
                                   mt_scene_s *sc, bool check_on_device) {
    int dev = 0;
    MT_CUDA_TRY(cudaGetDevice(&dev));
    MT_CUDA_TRY(cudaDeviceGetAttribute(&sc->num_sms, cudaDevAttrMultiProcessorCount, dev));
    MT_CUDA_TRY(cudaDeviceGetAttribute(&sc->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    sc->n_tris = n;
    sc->n_em = n_em;
    auto &al = sc->al;
    float *d_tris;
    mt_material *d_mats;
    mt_emitter *d_em;
    MT_TRY(al.alloc(&d_tris, (size_t)n * 9, "triangles"));
    MT_TRY(al.alloc(&d_mats, (size_t)n, "materials"));
    MT_TRY(al.alloc(&d_em, (size_t)std::max(1, n_em), "emitters"));
    MT_CUDA_TRY(cudaMemcpyAsync(d_tris, tris, (size_t)n * 9 * sizeof(float), cudaMemcpyHostToDevice, st));
    MT_CUDA_TRY(cudaMemcpyAsync(d_mats, mats, (size_t)n * sizeof(mt_material), cudaMemcpyHostToDevice, st));
    if (n_em > 0) MT_CUDA_TRY(cudaMemcpyAsync(d_em, ems, (size_t)n_em * sizeof(mt_emitter), cudaMemcpyHostToDevice, st));
    if (check_on_device) {  // the triangles and materials are checked where they now are, before the build
        int *dbad, hbad = 0;
        MT_TRY(al.alloc(&dbad, 1, "input check"));
        MT_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), st));
        k_check_inputs<<<grid_for(n * 9, 256, sc->num_sms), 256, 0, st>>>(
            reinterpret_cast<const uint32_t *>(d_tris), (size_t)n * 9, d_mats, (int)n, dbad);
        MT_CUDA_TRY(cudaGetLastError());
        MT_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad) {
            mt::set_error("non-finite vertex coordinates or invalid materials");
            return MT_ERR_INVALID_ARGUMENT;
        }
    }
    MT_TRY(mt_build_bvh(d_tris, (int32_t)n, st, al, &sc->bvh));
    DevScene &D = sc->dev;
    D.nodes = sc->bvh.nodes;
    D.wnodes = sc->bvh.wnodes;
    D.tris = sc->bvh.tris;
    D.n_tris = (int32_t)n;
    D.n_em = n_em;
    for (int k = 0; k < 3; ++k) {
        (&D.q_lo.x)[k] = sc->bvh.q_lo[k];
        (&D.q_scale.x)[k] = sc->bvh.q_scale[k];
    }
    float4 *mats4, *emrad;
    int32_t *tri_unit, *leaf_of;
    MT_TRY(al.alloc(&mats4, (size_t)n, "packed materials"));
    MT_TRY(al.alloc(&tri_unit, (size_t)n, "triangle light units"));
    MT_TRY(al.alloc(&leaf_of, (size_t)n, "leaf order"));
    MT_TRY(al.alloc(&emrad, (size_t)std::max(1, n_em), "emitter radiance"));
    const int g = grid_for(n, 256, sc->num_sms);
    k_pack_mats<<<g, 256, 0, st>>>(d_mats, (int)n, mats4);
    k_leaf_of<<<g, 256, 0, st>>>(sc->bvh.tris, (int)n, leaf_of);
    MT_CUDA_TRY(cudaMemsetAsync(tri_unit, 0xFF, (size_t)n * sizeof(int32_t), st));
    // light units (index bookkeeping on the host, arithmetic on the device)
    std::vector<int32_t> ut, ue;
    std::vector<float> rad(3 * (size_t)std::max(1, n_em), 0.f);
    for (int e = 0; e < n_em; ++e) {
        for (int k = 0; k < 3; ++k) rad[3 * e + k] = ems[e].radiance[k];
        if (ems[e].type == MT_EMITTER_AREA) {
            for (uint32_t t = 0; t < ems[e].n_tris; ++t) {
                ut.push_back((int32_t)(ems[e].first_tri + t));
                ue.push_back(e);
            }
        } else {
            ut.push_back(-1);
            ue.push_back(e);
        }
    }
    const int nu = (int)ut.size();
    int32_t *d_ut, *d_ue;
    LightUnit *units;
    uint32_t *cdf;
    MT_TRY(al.alloc(&d_ut, std::max(1, nu), "light units"));
    MT_TRY(al.alloc(&d_ue, std::max(1, nu), "light units"));
    MT_TRY(al.alloc(&units, std::max(1, nu), "light units"));
    MT_TRY(al.alloc(&cdf, std::max(1, nu), "light cdf"));
    if (nu > 0) {
        MT_CUDA_TRY(cudaMemcpyAsync(d_ut, ut.data(), nu * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        MT_CUDA_TRY(cudaMemcpyAsync(d_ue, ue.data(), nu * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        k_setup_units<<<1, 1, 0, st>>>(d_tris, d_ut, d_ue, nu, d_em, units, cdf, tri_unit);
    }
    // radiance rows -> float4
    {
        float *tmp;
        MT_TRY(al.alloc(&tmp, rad.size(), "radiance staging"));
        MT_CUDA_TRY(cudaMemcpyAsync(tmp, rad.data(), rad.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        k_set_radiance<<<1, 64, 0, st>>>(tmp, std::max(1, n_em), emrad);
    }
    float4 *shrec;
    MT_TRY(al.alloc(&shrec, (size_t)2 * n, "shading records"));
    k_shading_records<<<g, 256, 0, st>>>(sc->bvh.tris, mats4, tri_unit, (int)n, shrec);
    D.mats = mats4;
    D.tri_unit = tri_unit;
    D.leaf_of = leaf_of;
    D.shrec = shrec;
    D.units = units;
    D.unit_cdf = cdf;
    D.n_units = nu;
    D.em_rad = emrad;
    // camera
    CamOut *dcam, hcam;
    MT_TRY(al.alloc(&dcam, 1, "camera"));
    k_camera<<<1, 1, 0, st>>>(*cam, dcam);
    MT_CUDA_TRY(cudaMemcpyAsync(&hcam, dcam, sizeof(CamOut), cudaMemcpyDeviceToHost, st));
    // medium
    MT_TRY(al.alloc(&sc->m_params, 2, "medium parameters"));
    float mp[2] = {med ? med->albedo : 0.f, med ? med->g : 0.f};
    MT_CUDA_TRY(cudaMemcpyAsync(sc->m_params, mp, sizeof(mp), cudaMemcpyHostToDevice, st));
    D.m_params = sc->m_params;
    D.has_medium = med != nullptr;
    unsigned int hmax = 0;
    if (med) {
        const size_t nv = (size_t)med->res[0] * med->res[1] * med->res[2];
        float *dens;
        unsigned int *dmax;
        MT_TRY(al.alloc(&dens, nv, "density grid"));
        MT_TRY(al.alloc(&dmax, 1, "majorant"));
        MT_CUDA_TRY(cudaMemcpyAsync(dens, med->density, nv * sizeof(float), cudaMemcpyHostToDevice, st));
        MT_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(unsigned int), st));
        k_max<<<grid_for((long long)nv, 256, sc->num_sms), 256, 0, st>>>(dens, nv, dmax);
        MT_CUDA_TRY(cudaMemcpyAsync(&hmax, dmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        D.dens = dens;
        D.rx = med->res[0];
        D.ry = med->res[1];
        D.rz = med->res[2];
        D.m_lo = make_float3(med->lo[0], med->lo[1], med->lo[2]);
        D.m_hi = make_float3(med->hi[0], med->hi[1], med->hi[2]);
    }
    // scratch
    MT_TRY(al.alloc(&sc->tile_counter, 4, "tile counters"));
    MT_TRY(al.alloc(&sc->err, 1, "error word"));
    MT_TRY(al.alloc(&sc->counters, 8, "counters"));
    MT_CUDA_TRY(cudaMemsetAsync(sc->err, 0, sizeof(uint32_t), st));
    MT_CUDA_TRY(cudaMemsetAsync(sc->counters, 0, 8 * sizeof(unsigned long long), st));
    MT_CUDA_TRY(cudaGetLastError());
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    if (med) {
        float mj;
        memcpy(&mj, &hmax, 4);
        D.m_major = mj;
        if (!(mj > 0.f)) {
            mt::set_error("medium density must have a positive maximum");
            return MT_ERR_INVALID_ARGUMENT;
        }
    }
    D.cam_o = make_float3(hcam.o[0], hcam.o[1], hcam.o[2]);
    D.cam_f = make_float3(hcam.f[0], hcam.f[1], hcam.f[2]);
    D.cam_r = make_float3(hcam.r[0], hcam.r[1], hcam.r[2]);
    D.cam_u = make_float3(hcam.u[0], hcam.u[1], hcam.u[2]);
    D.tan_half = hcam.tan_half;
    D.err = sc->err;
    D.counters = sc->counters;
    for (int k = 0; k < 4; ++k) sc->cfg[k] = LaunchCfg{256, 0, 0, sc->num_sms, 0, -1, 0};
    // exhaustive NLOS grids: 32 sensors per tile with every splat in global memory (measured 130 ms
    // against 190 ms at the automatic 6-row tiles with shared-memory histograms)
    sc->cfg[MT_LAUNCH_NLOS_EXHAUSTIVE] = LaunchCfg{256, 32, 0, sc->num_sms, 0, 0, 0};
    return MT_OK;
}

// true when no float has an all-ones exponent (no infinity or NaN)
// Run f(begin, end) over [0, n) on up to 8 host threads (one for small n); true when
// every part returned true.
extern "C++" {
template <class F>
static bool parallel_all(int64_t n, F f) {
    const int64_t min_part = 1 << 20;
    const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(8, n / min_part));
    if (parts == 1) return f(0, n);
    std::vector<std::thread> th;
    std::vector<char> ok((size_t)parts, 1);
    for (int t = 0; t < parts; ++t)
        th.emplace_back([&, t] { ok[t] = f(n * t / parts, n * (t + 1) / parts) ? 1 : 0; });
    for (auto &x : th) x.join();
    for (char c : ok)
        if (!c) return false;
    return true;
}
}  // extern "C++"

#define MT_MAX_BANDS 4096  // bands of mt_render_to_host

#ifndef MT_HOST_CHECK_TRIS
#define MT_HOST_CHECK_TRIS (1 << 16)
#endif

static bool all_finite(const float *v, size_t n) {
    const uint32_t *b = reinterpret_cast<const uint32_t *>(v);
    return parallel_all((int64_t)n, [b](int64_t lo, int64_t hi) {
        uint32_t bad = 0;
        for (int64_t i = lo; i < hi; ++i) bad |= (uint32_t)((b[i] & 0x7F800000u) == 0x7F800000u);
        return bad == 0;
    });
}

static bool materials_ok(const mt_material *m, int64_t n) {
    return parallel_all(n, [m](int64_t lo, int64_t hi) {
        uint32_t bad = 0;
        for (int64_t i = lo; i < hi; ++i) {
            const mt_material &x = m[i];
            bad |= (uint32_t)!(x.albedo[0] >= 0.f && x.albedo[0] < INFINITY);
            bad |= (uint32_t)!(x.albedo[1] >= 0.f && x.albedo[1] < INFINITY);
            bad |= (uint32_t)!(x.albedo[2] >= 0.f && x.albedo[2] < INFINITY);
            bad |= (uint32_t)(x.type != MT_LAMBERT && x.type != MT_GGX_CONDUCTOR);
            bad |= (uint32_t)(x.type == MT_GGX_CONDUCTOR && !(x.roughness > 0.f && x.roughness <= 1.f));
        }
        return bad == 0;
    });
}

// vertices finite and materials valid, else INVALID_ARGUMENT naming the first offending triangle
static mt_status check_tris_materials(const float *tris, int64_t n_tris, const mt_material *materials) {
    // branch-free passes first (vectorisable); the offending element is located only on failure
    if (!all_finite(tris, (size_t)n_tris * 9)) {
        for (int64_t i = 0; i < n_tris * 9; ++i)
            MT_CHECK_ARG(std::isfinite(tris[i]), "non-finite vertex coordinate at triangle %lld", (long long)(i / 9));
    }
    if (!materials_ok(materials, n_tris)) {
        for (int64_t i = 0; i < n_tris; ++i) {
            const mt_material &m = materials[i];
            MT_CHECK_ARG(m.type == MT_LAMBERT || m.type == MT_GGX_CONDUCTOR,
                         "triangle %lld: unknown material type %u", (long long)i, m.type);
            for (int k = 0; k < 3; ++k)
                MT_CHECK_ARG(std::isfinite(m.albedo[k]) && m.albedo[k] >= 0.f, "triangle %lld: bad albedo",
                             (long long)i);
            MT_CHECK_ARG(m.type != MT_GGX_CONDUCTOR || (m.roughness > 0.f && m.roughness <= 1.f),
                         "triangle %lld: GGX roughness must lie in (0, 1]", (long long)i);
        }
    }
    return MT_OK;
}

mt_status mt_scene_create(const float *tris, int64_t n_tris, const mt_material *materials, const mt_emitter *emitters,
                          int32_t n_emitters, const mt_camera *camera, const mt_medium *medium, void *stream,
                          mt_scene *out) {
    MT_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MT_CHECK_ARG(tris != nullptr && materials != nullptr && camera != nullptr, "tris, materials and camera must not be NULL");
    MT_CHECK_ARG(n_tris >= 1 && n_tris < (1LL << 29), "n_tris = %lld outside [1, 2^29)", (long long)n_tris);
    MT_CHECK_ARG(n_emitters >= 0 && (n_emitters == 0 || emitters != nullptr), "bad emitter list");
    // scenes of up to MT_HOST_CHECK_TRIS triangles are checked here; larger ones on the device
    // after the upload (scanning 1.16M triangles on the host took 3.4 ms)
    const bool check_on_device = n_tris > MT_HOST_CHECK_TRIS;
    if (!check_on_device) MT_TRY(check_tris_materials(tris, n_tris, materials));
    for (int e = 0; e < n_emitters; ++e) {
        const mt_emitter &em = emitters[e];
        MT_CHECK_ARG(em.type == MT_EMITTER_AREA || em.type == MT_EMITTER_POINT, "emitter %d: unknown type", e);
        for (int k = 0; k < 3; ++k)
            MT_CHECK_ARG(std::isfinite(em.radiance[k]) && em.radiance[k] >= 0.f, "emitter %d: bad radiance", e);
        if (em.type == MT_EMITTER_AREA)
            MT_CHECK_ARG(em.n_tris >= 1 && (int64_t)em.first_tri + em.n_tris <= n_tris,
                         "emitter %d: triangle range out of bounds", e);
        else
            for (int k = 0; k < 3; ++k) MT_CHECK_ARG(std::isfinite(em.position[k]), "emitter %d: bad position", e);
    }
    if (medium) {
        MT_CHECK_ARG(medium->density != nullptr && medium->res[0] > 0 && medium->res[1] > 0 && medium->res[2] > 0,
                     "medium: bad grid");
        for (int k = 0; k < 3; ++k) MT_CHECK_ARG(medium->hi[k] > medium->lo[k], "medium: empty box");
        MT_CHECK_ARG(medium->albedo > 0.f && medium->albedo <= 1.f && std::fabs(medium->g) < 1.f,
                     "medium: albedo must lie in (0, 1] and |g| < 1");
        const size_t nv = (size_t)medium->res[0] * medium->res[1] * medium->res[2];
        for (size_t i = 0; i < nv; ++i)
            MT_CHECK_ARG(std::isfinite(medium->density[i]) && medium->density[i] >= 0.f, "medium: bad density");
    }
    MT_CHECK_ARG(std::isfinite(camera->fov_x_deg) && camera->fov_x_deg > 0.f && camera->fov_x_deg < 180.f,
                 "camera: fov_x_deg must lie in (0, 180)");
    mt_scene_s *sc = new (std::nothrow) mt_scene_s();
    if (!sc) {
        mt::set_error("host allocation failed");
        return MT_ERR_OUT_OF_MEMORY;
    }
    const mt_status st = scene_create_impl(tris, n_tris, materials, emitters, n_emitters, camera, medium,
                                           (cudaStream_t)stream, sc, check_on_device);
    if (st != MT_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        sc->al.free_all();
        delete sc;
        if (st == MT_ERR_INVALID_ARGUMENT && check_on_device) {
            const mt_status where = check_tris_materials(tris, n_tris, materials);  // names the element
            (void)where;
        }
        // return the build's pooled temporaries too: a failed creation keeps nothing
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
            cudaMemPoolTrimTo(pool, 0);
        cudaGetLastError();
        return st;
    }
    *out = sc;
    return MT_OK;
}

void mt_scene_destroy(mt_scene s) {
    if (!s) return;
    cudaDeviceSynchronize();
    if (s->nlos_graph.exec) cudaGraphExecDestroy(s->nlos_graph.exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    mt_wf_timing_free(&s->wf_timing);
    mt_wf_sync_free(&s->wf_sync);
    if (s->so_flag_h) cudaFreeHost(s->so_flag_h);
    free(s->so_issued);
    s->al.free_all();
    delete s;
}

mt_status mt_scene_set_params(mt_scene s, const float *d_albedo, const float *d_radiance,
                              const float *d_medium_albedo, void *stream) {
    MT_CHECK_ARG(s != nullptr, "scene is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (d_albedo)
        k_set_albedo<<<grid_for(s->n_tris, 256, s->num_sms), 256, 0, st>>>(
            d_albedo, (int)s->n_tris, const_cast<float4 *>(s->dev.mats), s->dev.leaf_of,
            const_cast<float4 *>(s->dev.shrec));
    if (d_radiance && s->n_em > 0)
        k_set_radiance<<<1, 64, 0, st>>>(d_radiance, s->n_em, const_cast<float4 *>(s->dev.em_rad));
    if (d_medium_albedo)
        MT_CUDA_TRY(cudaMemcpyAsync(s->m_params, d_medium_albedo, sizeof(float), cudaMemcpyDeviceToDevice, st));
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

mt_status mt_scene_set_delays(mt_scene s, const float *d_tau, void *stream) {
    MT_CHECK_ARG(s != nullptr, "scene is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (!d_tau) {
        s->dev.delay = nullptr;
        return MT_OK;
    }
    if (!s->delay_buf) MT_TRY(s->al.alloc(&s->delay_buf, (size_t)s->n_tris, "scattering delays"));
    if (!s->check_flag) MT_TRY(s->al.alloc(&s->check_flag, 1, "scattering delays"));
    int *dbad = s->check_flag;
    MT_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), st));
    k_check_delays<<<grid_for(s->n_tris, 256, s->num_sms), 256, 0, st>>>(d_tau, (int)s->n_tris, dbad);
    MT_CUDA_TRY(cudaGetLastError());
    int hbad = 0;
    MT_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    MT_CHECK_ARG(hbad == 0, "scattering delays must be finite and >= 0");
    MT_CUDA_TRY(cudaMemcpyAsync(s->delay_buf, d_tau, (size_t)s->n_tris * sizeof(float), cudaMemcpyDeviceToDevice, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));  // the caller may release d_tau on return
    s->dev.delay = s->delay_buf;
    return MT_OK;
}

mt_status mt_scene_set_pulse(mt_scene s, uint32_t shape, float a, float b) {
    MT_CHECK_ARG(s != nullptr, "scene is NULL");
    MT_CHECK_ARG(shape <= MT_PULSE_EXPONENTIAL, "unknown pulse shape %u", shape);
    MT_CHECK_ARG(std::isfinite(a) && std::isfinite(b), "pulse parameters must be finite");
    MT_CHECK_ARG(!((shape == MT_PULSE_BOX || shape == MT_PULSE_EXPONENTIAL) && !(a > 0.f)), "pulse width must be > 0");
    MT_CHECK_ARG(!(shape == MT_PULSE_GAUSSIAN && !(b > 0.f)), "pulse deviation must be > 0");
    s->dev.pulse_type = (int32_t)shape;
    s->dev.pulse_a = a;
    s->dev.pulse_b = b;
    return MT_OK;
}

mt_status mt_film_create(int32_t H, int32_t W, int32_t T, int32_t C, float start_opl, float bin_width, float *d_film,
                         float *d_steady, uint32_t flags, mt_film *out) {
    MT_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MT_CHECK_ARG(H >= 1 && W >= 1 && T >= 1, "film size H=%d W=%d T=%d must be positive", H, W, T);
    MT_CHECK_ARG(C == 1 || C == 3 || C == 12, "C must be 1, 3 or 12 (Stokes x colour)");
    MT_CHECK_ARG(std::isfinite(start_opl) && std::isfinite(bin_width) && bin_width > 0.f, "bad time window");
    MT_CHECK_ARG(d_film != nullptr, "film pointer is NULL");
    MT_CHECK_ARG((flags & ~(MT_UNWARP | MT_ACCUMULATE | MT_PIXEL_CENTER | MT_COUNTERS)) == 0, "unknown flags 0x%x", flags);
    MT_CHECK_ARG((int64_t)H * W < (1LL << 31), "too many pixels");
    mt_film_s *f = new (std::nothrow) mt_film_s{H, W, T, C, start_opl, bin_width, d_film, d_steady, flags, H, 0};
    if (!f) return MT_ERR_OUT_OF_MEMORY;
    *out = f;
    return MT_OK;
}

mt_status mt_film_set_window(mt_film f, int32_t frame_H, int32_t row0) {
    MT_CHECK_ARG(f != nullptr, "film is NULL");
    MT_CHECK_ARG(row0 >= 0 && frame_H >= 1 && (int64_t)row0 + f->H <= frame_H,
                 "window rows [%d, %d) do not fit a frame of %d rows", row0, row0 + f->H, frame_H);
    MT_CHECK_ARG((int64_t)frame_H * f->W < (1LL << 31), "too many pixels");
    f->H_full = frame_H;
    f->row0 = row0;
    return MT_OK;
}

void mt_film_destroy(mt_film f) { delete f; }

static void seed_key(uint64_t seed, uint32_t &k0, uint32_t &k1) {
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
}

// pick tile size and privatisation depth for a film within the shared-memory budget
static LaunchCfg render_cfg(const mt_scene_s *s, int kind, int32_t W, int32_t T, int C, int extra_floats, int &D) {
    LaunchCfg c = s->cfg[kind];
    const size_t budget = (size_t)std::min(s->smem_optin, 220 * 1024) - 1024;
    int tile = c.tile > 0 ? c.tile : 0;
    if (tile == 0) {
        // default: aim for >= 48 KB histograms, up to 32 pixels
        const size_t per_px = (size_t)T * C * 4;
        tile = (int)std::max<size_t>(1, std::min<size_t>(32, (96 * 1024) / std::max<size_t>(per_px, 1)));
        if (kind == MT_LAUNCH_RENDER || kind == MT_LAUNCH_BACKWARD) tile = std::min(tile, W);
    }
    size_t fixed = ((size_t)tile * (C == 3 ? 3 : 1) + extra_floats) * 4 + 64;
    size_t avail = budget > fixed ? budget - fixed : 0;
    D = (int)std::min<size_t>((size_t)T, avail / ((size_t)tile * C * 4));
    if (c.priv >= 0) D = std::min(D, c.priv);
    if (D < 1) D = 0;
    c.tile = tile;
    c.smem_bytes = (((size_t)tile * D * C + (size_t)tile * (C == 3 ? 3 : 1) + extra_floats) * 4 + 15) & ~(size_t)15;
    return c;
}

// warp-owned tiles of k_render: `tile` pixels per warp (default: enough pixels
// for 64 paths), D = bins per pixel privatised in the warp's shared-memory
// slice (priv < 0: as many as fit in ~100 KB per CTA; bins >= D go to global
// memory with red.add)
static LaunchCfg warp_tile_cfg(const mt_scene_s *s, int kind, int32_t W, int32_t T, int32_t spp, int extra_floats,
                               int &D) {
    LaunchCfg c = s->cfg[kind];
    const int warps = c.threads / 32;
    int tile = c.tile > 0 ? c.tile : std::max(1, (64 + spp - 1) / spp);
    tile = std::max(1, std::min(tile, W));
    const size_t cap = (size_t)std::min(s->smem_optin, 220 * 1024) - 1024;
    const size_t budget = std::min(cap, (size_t)100 * 1024);
    const size_t fixed = (size_t)extra_floats * 4 + 64;
    const size_t per_warp = budget > fixed ? (budget - fixed) / warps : 0;
    long long fit = ((long long)(per_warp / 4) - 3LL * tile) / (3LL * tile);
    if (fit < 0) fit = 0;
    long long d = c.priv < 0 ? std::min<long long>(T, fit) : std::min<long long>(std::min<long long>(c.priv, T), fit);
    if (c.priv > 0 && d < c.priv) {  // an explicit depth may use the whole opt-in budget
        const size_t per_warp_cap = cap > fixed ? (cap - fixed) / warps : 0;
        const long long fit_cap = ((long long)(per_warp_cap / 4) - 3LL * tile) / (3LL * tile);
        d = std::max<long long>(0, std::min<long long>(std::min<long long>(c.priv, T), fit_cap));
    }
    D = (int)d;
    c.tile = tile;
    c.smem_bytes = (((size_t)warps * tile * (3 * (size_t)D + 3) + extra_floats) * 4 + 15) & ~(size_t)15;
    return c;
}

static mt_status check_err_word(mt_scene s) {
    uint32_t e = 0;
    MT_CUDA_TRY(cudaMemcpy(&e, s->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) {
        MT_CUDA_TRY(cudaMemset(s->err, 0, sizeof(e)));
        if (e & MT_EFLAG_STACK) {
            mt::set_error("device: traversal stack overflow");
            return MT_ERR_INTERNAL;
        }
        mt::set_error("device: bounded wait or tracking loop gave up (flags 0x%x)", e);
        return MT_ERR_TIMEOUT;
    }
    return MT_OK;
}

// forward render in wavefront form: a pool of paths in device memory
static mt_status render_wavefront(mt_scene s, mt_film f, const RenderParams &rp, const LaunchCfg &cfg, bool dump,
                                  cudaStream_t st, bool tangent = false, bool backward = false,
                                  bool polarized = false) {
    const unsigned long long total = (unsigned long long)f->H * f->W * rp.spp;
    const uint32_t P = (uint32_t)std::min<unsigned long long>(total, s->wf_pool_max);
    // path state in queue order unless a form keeps per-path records by slot (replay, polarization)
    // or reorders the queue (ray sorting, dynamic fetch)
    const bool dyn = (cfg.options & MT_OPT_DYNAMIC_FETCH) && !dump && !s->dev.has_medium && !backward;
    const bool qmode = !backward && !polarized && !dyn && !((cfg.options & MT_OPT_SORT_RAYS) && !dump);
    if (P > s->wf_cap || (qmode ? P > s->wf_q_cap : P > s->wf_slot_cap)) {
        cudaStreamCaptureStatus cs;
        MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        MT_CHECK_ARG(cs == cudaStreamCaptureStatusNone,
                     "the first wavefront render of this size must not be captured (it sizes the path pool)");
    }
    if (P > s->wf_cap) {
        auto &al = s->al;
        MT_TRY(al.alloc(&s->wf_sh_o, P, "shadow queue"));
        MT_TRY(al.alloc(&s->wf_sh_d, P, "shadow queue"));
        MT_TRY(al.alloc(&s->wf_sh_c, P, "shadow queue"));
        MT_TRY(al.alloc(&s->wf_sh_m, P, "shadow queue"));
        if (!s->wf_counters) {
            MT_TRY(al.alloc(&s->wf_counters, 16, "path queue counters"));
            MT_TRY(al.alloc(&s->wf_next, 1, "path queue counters"));
            MT_TRY(al.alloc((char **)&s->wf_iter, 64, "path queue counters"));
        }
        s->wf_cap = P;
    }
    if (qmode && P > s->wf_q_cap) {
        MT_TRY(s->al.alloc(&s->wf_qs, (size_t)11 * P, "queue-ordered path state"));
        s->wf_q_cap = P;
    }
    if (!qmode && P > s->wf_slot_cap) {
        auto &al = s->al;
#if MT_WF_AOS
        MT_TRY(al.alloc(&s->wf_o, (size_t)MT_WF_REC * P, "path pool"));
        s->wf_d = s->wf_o + 1;
        s->wf_beta = s->wf_o + 2;
        s->wf_meta = (uint4 *)(s->wf_o + 3);
        s->wf_hit = (int4 *)(s->wf_o + 4);
        s->wf_sig = s->wf_o + 5;
#else
        MT_TRY(al.alloc(&s->wf_o, P, "path pool"));
        MT_TRY(al.alloc(&s->wf_d, P, "path pool"));
        MT_TRY(al.alloc(&s->wf_beta, P, "path pool"));
        MT_TRY(al.alloc(&s->wf_meta, P, "path pool"));
        MT_TRY(al.alloc(&s->wf_hit, P, "path pool"));
        MT_TRY(al.alloc(&s->wf_sig, P, "path tangent sums"));
#endif
        MT_TRY(al.alloc(&s->wf_qa, P, "path queues"));
        MT_TRY(al.alloc(&s->wf_qb, P, "path queues"));
        MT_TRY(al.alloc(&s->wf_free, P, "path queues"));
        s->wf_slot_cap = P;
    }
    if (backward) {
        const size_t need = (size_t)(rp.max_depth + 1) * P;
        if (need > s->wf_rec_cap) {
            cudaStreamCaptureStatus cs;
            MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
            MT_CHECK_ARG(cs == cudaStreamCaptureStatusNone,
                         "the first wavefront backward pass of this size must not be captured (it sizes the records)");
            auto &al = s->al;
            MT_TRY(al.alloc(&s->wf_rec, 3 * need, "path replay vertex records"));
            if (!s->wf_fin) {
                MT_TRY(al.alloc(&s->wf_fin, (size_t)MT_WF_POOL_DEFAULT, "path replay queue"));
                MT_TRY(al.alloc(&s->wf_shown, (size_t)MT_WF_POOL_DEFAULT, "path replay shadow records"));
            }
            s->wf_rec_cap = need;
        }
    }
    if (polarized && P > s->wf_pol_cap) {
        cudaStreamCaptureStatus cs;
        MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        MT_CHECK_ARG(cs == cudaStreamCaptureStatusNone,
                     "the first polarized wavefront render of this size must not be captured (it sizes the pool)");
        auto &al = s->al;
        MT_TRY(al.alloc(&s->wf_mueller, (size_t)12 * P, "path Mueller matrices"));
        MT_TRY(al.alloc(&s->wf_xframe, P, "path Stokes frames"));
        MT_TRY(al.alloc(&s->wf_shs, (size_t)3 * P, "shadow Stokes records"));
        s->wf_pol_cap = P;
    }
    // the polarized stages read neither ray order
    const bool sort_rays = (cfg.options & MT_OPT_SORT_RAYS) != 0 && !polarized;
    const bool sort_shadow = (cfg.options & MT_OPT_SORT_SHADOW) != 0 && !dump && !polarized;
    if ((sort_rays || sort_shadow) && P > s->wf_sort_cap) {
        cudaStreamCaptureStatus cs;
        MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        MT_CHECK_ARG(cs == cudaStreamCaptureStatusNone,
                     "the first sorted wavefront render of this size must not be captured (it sizes the sort)");
        auto &al = s->al;
        MT_TRY(al.alloc(&s->wf_sk, P, "ray sort keys"));
        MT_TRY(al.alloc(&s->wf_sko, P, "ray sort keys"));
        MT_TRY(al.alloc(&s->wf_sq, P, "ray sort queue"));
        s->wf_stmp_bytes = mt_wf_sort_bytes(P);
        MT_TRY(al.alloc(&s->wf_stmp, s->wf_stmp_bytes, "ray sort scratch"));
        MT_TRY(al.alloc(&s->wf_shperm, P, "shadow ray order"));
        s->wf_sort_cap = P;
    }
    WfParams w{};
    w.H = rp.H;
    w.W = rp.W;
    w.H_full = rp.H_full;
    w.row0 = rp.row0;
    w.pix_base = rp.pix_base;
    w.T = rp.T;
    w.start = rp.start;
    w.width = rp.width;
    w.scale = rp.scale;
    w.flags = rp.flags;
    w.spp = rp.spp;
    w.max_depth = rp.max_depth;
    w.sample_offset = rp.sample_offset;
    w.k0 = rp.k0;
    w.k1 = rp.k1;
    w.total_paths = total;
    w.P = P;
    w.film = rp.film;
    w.steady = rp.steady;
    w.o.base = s->wf_o;
    w.d.base = s->wf_d;
    w.beta.base = s->wf_beta;
    w.meta.base = s->wf_meta;
    w.hit.base = s->wf_hit;
    w.qa = s->wf_qa;
    w.qb = s->wf_qb;
    w.free_q = s->wf_free;
    w.qmode = qmode ? 1 : 0;
    if (qmode) {
        float4 *q = s->wf_qs;  // 11 arrays of P float4: o, d, beta, meta, sig (current), the same (next), hits
        w.ps_o = q;
        w.ps_d = q + (size_t)P;
        w.ps_b = q + (size_t)2 * P;
        w.ps_m = (uint4 *)(q + (size_t)3 * P);
        w.ps_sig = tangent ? q + (size_t)4 * P : nullptr;
        w.ps_o_n = q + (size_t)5 * P;
        w.ps_d_n = q + (size_t)6 * P;
        w.ps_b_n = q + (size_t)7 * P;
        w.ps_m_n = (uint4 *)(q + (size_t)8 * P);
        w.ps_sig_n = tangent ? q + (size_t)9 * P : nullptr;
        w.ps_h = (int4 *)(q + (size_t)10 * P);
    }
    w.sh_o = s->wf_sh_o;
    w.sh_d = s->wf_sh_d;
    w.sh_c = s->wf_sh_c;
    w.sh_m = s->wf_sh_m;
    w.counters = s->wf_counters;
    w.next_path = s->wf_next;
    w.iter = (struct WfIter *)s->wf_iter;
    w.dump = rp.dump;
    w.dump_cap = rp.dump_cap;
    w.dump_count = rp.dump_count;
    w.splat_count = (f->flags & MT_COUNTERS) ? s->counters + 7 : nullptr;
    // the refill field of the options word doubles as the fetch threshold
    const int fetch_k = (int)((cfg.options >> 8) & 0xFFu);
    w.dynamic_fetch = (cfg.options & MT_OPT_DYNAMIC_FETCH) ? (fetch_k ? std::min(fetch_k, 32) : 8) : 0;
    w.wide = (cfg.options & MT_OPT_WIDE_BVH) ? 1 : 0;
    w.lambdas = rp.lambdas;
    w.K = rp.lambdas ? rp.K : 0;
    w.sig.base = tangent ? s->wf_sig : nullptr;
    w.dalb = rp.dalb;
    w.drad = rp.drad;
    w.dmed = rp.dmed;
    w.bwd = backward ? 1 : 0;
    if (backward) {
        const size_t cap = s->wf_rec_cap;
        w.rec_a = s->wf_rec;
        w.rec_b = s->wf_rec + cap;
        w.rec_c = s->wf_rec + 2 * cap;
        w.fin_q = s->wf_fin;
        w.sh_cb = s->wf_shown;
        w.gfilm = rp.gfilm;
        w.gsteady = rp.gsteady;
        w.galb = rp.galb;
        w.grad = rp.grad;
        w.gmed = rp.gmed;
    }
    w.sort_rays = sort_rays ? 1 : 0;
    w.sort_keys = s->wf_sk;
    w.sort_keys_out = s->wf_sko;
    w.sort_q = s->wf_sq;
    w.sort_tmp = s->wf_stmp;
    w.sort_tmp_bytes = s->wf_stmp_bytes;
    w.sh_perm = sort_shadow ? s->wf_shperm : nullptr;
    if (polarized) {
        w.mueller = s->wf_mueller;
        w.xframe = s->wf_xframe;
        w.sh_s = s->wf_shs;
    }
    // a backward pass reads dL/dfilm from the film; polarized films (C = 12) are cleared by the caller
    if (!(rp.flags & MT_ACCUMULATE) && !backward && !polarized) {
        MT_CUDA_TRY(cudaMemsetAsync(f->film, 0, (size_t)f->H * f->W * f->T * 3 * sizeof(float), st));
        if (f->steady) MT_CUDA_TRY(cudaMemsetAsync(f->steady, 0, (size_t)f->H * f->W * 3 * sizeof(float), st));
    }
    long long n = 0;
    WfTiming *tm = (cfg.options & MT_OPT_STAGE_TIMING) ? &s->wf_timing : nullptr;
    MT_TRY(mt_wf_sync_init(&s->wf_sync));
    const mt_status r = mt_launch_wavefront(s->dev, w, s->num_sms, dump, (f->flags & MT_COUNTERS) != 0, st, &n, tm,
                                            &s->wf_sync, s->wf_out);
    s->launches += n + 1;
    return r;
}

static mt_status render_common(mt_scene s, mt_film f, int32_t spp, uint64_t seed, int32_t max_depth,
                               uint64_t sample_offset, int mode, const float *gfilm, const float *gsteady,
                               float *galb, float *grad, float *gmed, mt_contrib *dump, int64_t cap,
                               int64_t *dcount, cudaStream_t st, const float *lambdas = nullptr, int32_t K = 0,
                               const float *dalb = nullptr, const float *drad = nullptr, float dmed = 0.f) {
    MT_CHECK_ARG(s != nullptr && f != nullptr, "scene or film is NULL");
    MT_CHECK_ARG(f->C == 3, "path-traced films have C = 3");
    MT_CHECK_ARG(spp >= 1, "spp must be >= 1");
    MT_CHECK_ARG(max_depth >= 1 && max_depth <= MT_MAX_DEPTH, "max_depth must lie in [1, %d]", MT_MAX_DEPTH);
    MT_CHECK_ARG(sample_offset + (uint64_t)spp <= 0xFFFFFFFFull, "sample indices must fit in 32 bits");
    MT_CHECK_ARG((int64_t)f->W * spp < (1LL << 31), "tile path count overflows");
    if (mode == 2) {
        MT_CHECK_ARG(max_depth <= MT_MAX_BWD_DEPTH, "backward supports max_depth <= %d", MT_MAX_BWD_DEPTH);
        MT_CHECK_ARG(gfilm != nullptr && galb != nullptr && grad != nullptr, "gradient buffers must not be NULL");
    }
    const int kind = mode == 2 ? MT_LAUNCH_BACKWARD : MT_LAUNCH_RENDER;
    const int n_em_smem = (mode == 2 && s->n_em <= 64) ? s->n_em : 0;
    int D;
    LaunchCfg cfg = warp_tile_cfg(s, kind, f->W, f->T, spp, n_em_smem * 3, D);
    RenderParams p{};
    p.H = f->H;
    p.W = f->W;
    p.H_full = f->H_full;
    p.row0 = f->row0;
    p.pix_base = (uint32_t)f->row0 * (uint32_t)f->W;
    p.T = f->T;
    p.D = D;
    p.start = f->start;
    p.width = f->width;
    const bool acc = f->flags & MT_ACCUMULATE;
    p.scale = acc ? 1.0f : 1.0f / (float)spp;
    p.flags = f->flags;
    p.spp = spp;
    p.max_depth = max_depth;
    p.sample_offset = (uint32_t)sample_offset;
    seed_key(seed, p.k0, p.k1);
    p.tile_px = cfg.tile;
    p.tiles_per_row = (f->W + cfg.tile - 1) / cfg.tile;
    p.n_tiles = p.tiles_per_row * f->H;
    p.film = f->film;
    p.steady = f->steady;
    p.gfilm = gfilm;
    p.gsteady = gsteady;
    p.galb = galb;
    p.grad = grad;
    p.gmed = gmed;
    p.dump = dump;
    p.dump_cap = cap;
    p.dump_count = (unsigned long long *)dcount;
    p.tile_counter = s->tile_counter;
    p.n_em_smem = n_em_smem;
    p.aggregate = (cfg.options & MT_OPT_AGGREGATE) ? 1 : 0;
    p.refill_min = std::max(1, std::min(32, (cfg.options >> 8) & 0xFF));
    p.lambdas = lambdas;
    p.K = K;
    p.dalb = dalb;
    p.drad = drad;
    p.dmed = dmed;
    if (mode != 2 && D < f->T && !acc) {
        MT_CUDA_TRY(cudaMemsetAsync(f->film, 0, (size_t)f->H * f->W * f->T * 3 * sizeof(float), st));
    }
    if (dump) MT_CUDA_TRY(cudaMemsetAsync(dcount, 0, sizeof(int64_t), st));
    if ((mode == 0 || mode == 1 || mode == 2 || mode == 3 || mode == 4) && (cfg.options & MT_OPT_WAVEFRONT))
        return render_wavefront(s, f, p, cfg, mode == 1, st, mode == 4, mode == 2);
    MT_CUDA_TRY(cudaMemsetAsync(s->tile_counter, 0, sizeof(int), st));
    s->launches += 1;
    return mt_launch_render(s->dev, p, cfg, mode, (f->flags & MT_COUNTERS) != 0, st);
}

mt_status mt_render(mt_scene s, mt_film f, int32_t spp, uint64_t seed, int32_t max_depth, uint64_t sample_offset,
                    void *stream) {
    return render_common(s, f, spp, seed, max_depth, sample_offset, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, 0, nullptr, (cudaStream_t)stream);
}

mt_status mt_render_to_host(mt_scene s, mt_film f, int32_t spp, uint64_t seed, int32_t max_depth,
                            uint64_t sample_offset, int32_t band_rows, float *host_film, float *host_steady,
                            void *stream, void *copy_stream) {
    MT_CHECK_ARG(s != nullptr && f != nullptr, "scene or film is NULL");
    MT_CHECK_ARG(host_film != nullptr, "host_film is NULL");
    MT_CHECK_ARG((host_steady != nullptr) == (f->steady != nullptr),
                 "host_steady must be given exactly when the film has a steady image");
    MT_CHECK_ARG(f->C == 3, "path-traced films have C = 3");
    MT_CHECK_ARG(band_rows >= 1, "band_rows must be >= 1");
    const uint32_t n_bands = (uint32_t)((f->H + band_rows - 1) / band_rows);
    MT_CHECK_ARG(n_bands <= MT_MAX_BANDS, "at most %d bands (band_rows too small for %d rows)", MT_MAX_BANDS, f->H);
    cudaStream_t st = (cudaStream_t)stream, cp = (cudaStream_t)copy_stream;
    MT_CHECK_ARG(cp != st, "copy_stream must differ from stream");
    if (n_bands > s->so_cap) {
        // no capacity until every buffer below exists again, so a call after a failed
        // allocation here grows them anew instead of using a released host flag array
        s->so_cap = 0;
        auto &al = s->al;
        MT_TRY(al.alloc(&s->so_done, n_bands, "streamed output"));
        MT_TRY(al.alloc(&s->so_mark, n_bands, "streamed output"));
        if (s->so_flag_h) {
            MT_CUDA_TRY(cudaDeviceSynchronize());  // band passes of an earlier render may still write it
            cudaFreeHost(s->so_flag_h);
        }
        s->so_flag_h = nullptr;
        void *h = nullptr, *d = nullptr;
        MT_CUDA_TRY(cudaHostAlloc(&h, 2 * n_bands * sizeof(uint32_t), cudaHostAllocMapped));
        memset(h, 0, 2 * n_bands * sizeof(uint32_t));
        s->so_flag_h = (uint32_t *)h;
        MT_CUDA_TRY(cudaHostGetDevicePointer(&d, h, 0));
        s->so_flag_d = (uint32_t *)d;
        char *iss = (char *)realloc(s->so_issued, n_bands);
        if (!iss) {
            mt::set_error("streamed output: out of host memory");
            return MT_ERR_OUT_OF_MEMORY;
        }
        s->so_issued = iss;
        s->so_cap = n_bands;
    }
    WfStreamOut out;
    out.copy = cp;
    out.h_film = host_film;
    out.h_steady = host_steady;
    out.d_film = f->film;
    out.d_steady = f->steady;
    out.film_row_bytes = (size_t)f->W * f->T * 3 * sizeof(float);
    out.steady_row_bytes = (size_t)f->W * 3 * sizeof(float);
    out.H = (uint32_t)f->H;
    out.band_rows = (uint32_t)band_rows;
    out.n_bands = n_bands;
    out.band_done = s->so_done;
    out.band_mark = s->so_mark;
    out.flag_h = s->so_flag_h;
    out.flag_d = s->so_flag_d;
    out.issued = s->so_issued;
    s->wf_out = &out;
    const mt_status r = render_common(s, f, spp, seed, max_depth, sample_offset, 0, nullptr, nullptr, nullptr, nullptr,
                                      nullptr, nullptr, 0, nullptr, st);
    s->wf_out = nullptr;
    MT_TRY(r);
    if (!out.used) {  // another form: every band behind the whole render
        cudaEvent_t ev;
        MT_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        MT_CUDA_TRY(cudaEventRecord(ev, st));
        MT_CUDA_TRY(cudaStreamWaitEvent(cp, ev, 0));
        cudaEventDestroy(ev);
        MT_CUDA_TRY(cudaMemcpyAsync(host_film, f->film, (size_t)f->H * out.film_row_bytes, cudaMemcpyDeviceToHost, cp));
        if (host_steady)
            MT_CUDA_TRY(cudaMemcpyAsync(host_steady, f->steady, (size_t)f->H * out.steady_row_bytes,
                                        cudaMemcpyDeviceToHost, cp));
    }
    return MT_OK;
}

mt_status mt_render_polarized(mt_scene s, mt_film f, int32_t spp, uint64_t seed, int32_t max_depth,
                              uint64_t sample_offset, void *stream) {
    MT_CHECK_ARG(s != nullptr && f != nullptr, "scene or film is NULL");
    MT_CHECK_ARG(f->C == 12, "polarized films have C = 12 (4 Stokes components x 3 colours)");
    MT_CHECK_ARG(f->steady != nullptr, "polarized renders need the steady Stokes image");
    MT_CHECK_ARG(spp >= 1, "spp must be >= 1");
    MT_CHECK_ARG(max_depth >= 1 && max_depth <= MT_MAX_DEPTH, "max_depth must lie in [1, %d]", MT_MAX_DEPTH);
    MT_CHECK_ARG(sample_offset + (uint64_t)spp <= 0xFFFFFFFFull, "sample indices must fit in 32 bits");
    if (s->dev.has_medium) {
        mt::set_error("polarization tracking does not support participating media");
        return MT_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool acc = f->flags & MT_ACCUMULATE;
    if (!acc) {
        MT_CUDA_TRY(cudaMemsetAsync(f->film, 0, (size_t)f->H * f->W * f->T * 12 * sizeof(float), st));
        MT_CUDA_TRY(cudaMemsetAsync(f->steady, 0, (size_t)f->H * f->W * 12 * sizeof(float), st));
    }
    uint32_t k0, k1;
    seed_key(seed, k0, k1);
    const LaunchCfg &cfg = s->cfg[MT_LAUNCH_RENDER];
    if (cfg.options & MT_OPT_WAVEFRONT) {  // the render configuration selects the form
        RenderParams p{};
        p.H = f->H;
        p.W = f->W;
        p.H_full = f->H_full;
        p.row0 = f->row0;
        p.pix_base = (uint32_t)f->row0 * (uint32_t)f->W;
        p.T = f->T;
        p.start = f->start;
        p.width = f->width;
        p.scale = acc ? 1.0f : 1.0f / (float)spp;
        p.flags = f->flags;
        p.spp = spp;
        p.max_depth = max_depth;
        p.sample_offset = (uint32_t)sample_offset;
        p.k0 = k0;
        p.k1 = k1;
        p.film = f->film;
        p.steady = f->steady;
        return render_wavefront(s, f, p, cfg, false, st, false, false, true);
    }
    s->launches += 1;
    return mt_launch_polarized(s->dev, f->H, f->W, f->T, f->H_full, f->row0, f->start, f->width,
                               acc ? 1.0f : 1.0f / (float)spp,
                               f->flags, spp, max_depth, (uint32_t)sample_offset, k0, k1, f->film, f->steady,
                               s->num_sms, st);
}

mt_status mt_render_phasor(mt_scene s, mt_film f, const float *d_lambdas, int32_t K, int32_t spp, uint64_t seed,
                           int32_t max_depth, uint64_t sample_offset, void *stream) {
    MT_CHECK_ARG(s != nullptr && f != nullptr, "scene or film is NULL");
    MT_CHECK_ARG(d_lambdas != nullptr && K >= 1, "need K >= 1 wavelengths");
    MT_CHECK_ARG(f->T == 2 * K && f->C == 3, "phasor films have T = 2K (real, imaginary) and C = 3");
    return render_common(s, f, spp, seed, max_depth, sample_offset, 3, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, 0, nullptr, (cudaStream_t)stream, d_lambdas, K);
}

mt_status mt_render_tangent(mt_scene s, mt_film f, const float *d_dalbedo, const float *d_dradiance, float dmedium,
                            int32_t spp, uint64_t seed, int32_t max_depth, uint64_t sample_offset, void *stream) {
    MT_CHECK_ARG(s != nullptr && f != nullptr, "scene or film is NULL");
    MT_CHECK_ARG(std::isfinite(dmedium), "medium-albedo tangent must be finite");
    MT_CHECK_ARG(f->C == 3, "tangent films have C = 3");
    return render_common(s, f, spp, seed, max_depth, sample_offset, 4, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, 0, nullptr, (cudaStream_t)stream, nullptr, 0, d_dalbedo, d_dradiance,
                         s->dev.has_medium ? dmedium : 0.f);
}

mt_status mt_render_backward(mt_scene s, mt_film f, const float *d_grad_film, const float *d_grad_steady, int32_t spp,
                             uint64_t seed, int32_t max_depth, uint64_t sample_offset, float *d_grad_albedo,
                             float *d_grad_radiance, float *d_grad_medium_albedo, void *stream) {
    return render_common(s, f, spp, seed, max_depth, sample_offset, 2, d_grad_film, d_grad_steady, d_grad_albedo,
                         d_grad_radiance, d_grad_medium_albedo, nullptr, 0, nullptr, (cudaStream_t)stream);
}

// argument checks shared by every NLOS entry point
static mt_status nlos_check(mt_scene s, mt_film f, const mt_scan *sc, int32_t spp, uint64_t sample_offset) {
    MT_CHECK_ARG(s != nullptr && f != nullptr && sc != nullptr, "scene, film or scan is NULL");
    MT_CHECK_ARG(f->C == 1, "NLOS films have C = 1");
    MT_CHECK_ARG(sc->mode == MT_CONFOCAL || sc->mode == MT_EXHAUSTIVE, "unknown scan mode");
    MT_CHECK_ARG(sc->lasers != nullptr && sc->n_lasers >= 1, "no laser points");
    MT_CHECK_ARG(sc->mode == MT_CONFOCAL || (sc->sensors != nullptr && sc->n_sensors >= 1), "no sensor points");
    const long long rows = sc->mode == MT_EXHAUSTIVE ? (long long)sc->n_lasers * sc->n_sensors : sc->n_lasers;
    MT_CHECK_ARG((long long)f->H * f->W == rows, "film H*W = %lld must equal the number of scan pairs %lld",
                 (long long)f->H * f->W, rows);
    MT_CHECK_ARG(sc->hidden_count >= 1 && (int64_t)sc->hidden_first + sc->hidden_count <= s->n_tris,
                 "hidden triangle range out of bounds");
    MT_CHECK_ARG(spp >= 1 && sample_offset + (uint64_t)spp <= 0xFFFFFFFFull, "bad spp / sample_offset");
    const float nl = std::sqrt(sc->wall_normal[0] * sc->wall_normal[0] + sc->wall_normal[1] * sc->wall_normal[1] +
                               sc->wall_normal[2] * sc->wall_normal[2]);
    MT_CHECK_ARG(std::fabs(nl - 1.0f) < 1e-3f, "wall normal must be a unit vector");
    return MT_OK;
}

// Hidden-surface sampling table of triangles [first, first + n) into cdf [n] and
// guide [MT_HGUIDE_N + 1], with prefix [n] doubles of scratch and the total area
// (float) written to *area; asynchronous on st.
static mt_status hidden_table(mt_scene s, int first, int n, uint32_t *cdf, uint32_t *guide, double *prefix,
                              float *area, cudaStream_t st) {
    const int g = grid_for(n, 256, s->num_sms);
    k_hidden_area<<<g, 256, 0, st>>>(s->dev.tris, s->dev.leaf_of, first, n, prefix);
    k_hidden_prefix<<<1, 1, 0, st>>>(prefix, n);
    k_hidden_cdf<<<g, 256, 0, st>>>(prefix, n, cdf, area);
    k_hidden_guide<<<(MT_HGUIDE_N + 256) / 256, 256, 0, st>>>(cdf, n, guide);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

// Launch parameters of an NLOS capture over the given sampling table and scratch
// (area_dev: device copy of the hidden area read by the kernels, or null to use
// `area`); shared by the allocating and the allocation-free entry points.
static void nlos_fill(mt_scene s, mt_film f, const mt_scan *sc, int32_t spp, uint64_t seed, uint64_t sample_offset,
                      const uint32_t *cdf, const uint32_t *guide, float area, const float *area_dev, float4 *ysamp,
                      int32_t *ysamp_tri, int *tile_counter, NlosParams &p, LaunchCfg &cfg) {
    const long long rows = sc->mode == MT_EXHAUSTIVE ? (long long)sc->n_lasers * sc->n_sensors : sc->n_lasers;
    int D;
    cfg = render_cfg(s, sc->mode == MT_EXHAUSTIVE ? MT_LAUNCH_NLOS_EXHAUSTIVE : MT_LAUNCH_NLOS, (int)rows, f->T, 1, 0,
                     D);
    p = NlosParams{};
    p.T = f->T;
    p.D = D;
    p.start = f->start;
    p.width = f->width;
    const bool acc = f->flags & MT_ACCUMULATE;
    p.scale = acc ? 1.0f : 1.0f / (float)spp;
    p.flags = f->flags;
    p.spp = spp;
    p.mode = (int32_t)sc->mode;
    p.sample_offset = (uint32_t)sample_offset;
    seed_key(seed, p.k0, p.k1);
    p.lasers = sc->lasers;
    p.sensors = sc->sensors;
    p.n_l = sc->n_lasers;
    p.n_s = sc->mode == MT_EXHAUSTIVE ? sc->n_sensors : 0;
    p.nw = make_float3(sc->wall_normal[0], sc->wall_normal[1], sc->wall_normal[2]);
    p.fw = sc->wall_albedo / MT_PI;
    p.hidden_first = (int32_t)sc->hidden_first;
    p.hidden_n = (int32_t)sc->hidden_count;
    p.hcdf = cdf;
    p.hguide = guide;
    p.hidden_area = area;
    p.hidden_area_dev = area_dev;
    p.tile = cfg.tile;
    if (sc->mode == MT_EXHAUSTIVE) p.n_tiles = sc->n_lasers * ((sc->n_sensors + cfg.tile - 1) / cfg.tile);
    else p.n_tiles = (int)((rows + cfg.tile - 1) / cfg.tile);
    p.film = f->film;
    p.steady = f->steady;
    p.ysamp = ysamp;
    p.ysamp_tri = ysamp_tri;
    p.tile_counter = tile_counter;
    p.aggregate = (cfg.options & MT_OPT_AGGREGATE) ? 1 : 0;
}

static mt_status nlos_prepare(mt_scene s, mt_film f, const mt_scan *sc, int32_t spp, uint64_t seed,
                              uint64_t sample_offset, NlosParams &p, LaunchCfg &cfg, cudaStream_t st) {
    MT_TRY(nlos_check(s, f, sc, spp, sample_offset));
    if (s->h_first != (int32_t)sc->hidden_first || s->h_count != (int32_t)sc->hidden_count) {
        cudaStreamCaptureStatus cs;
        MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        MT_CHECK_ARG(cs == cudaStreamCaptureStatusNone,
                     "the first NLOS call for a hidden range must not be captured (it builds the sampling table)");
        if (s->h_cap < (int32_t)sc->hidden_count) {
            s->h_first = -1;
            MT_TRY(s->al.alloc(&s->hcdf, sc->hidden_count, "hidden cdf"));
            MT_TRY(s->al.alloc(&s->hprefix, sc->hidden_count, "hidden area sums"));
            s->h_cap = (int32_t)sc->hidden_count;
        }
        if (!s->hguide) MT_TRY(s->al.alloc(&s->hguide, (size_t)MT_HGUIDE_N + 1, "hidden cdf guide"));
        if (!s->harea) MT_TRY(s->al.alloc(&s->harea, 1, "hidden area"));
        MT_TRY(hidden_table(s, (int)sc->hidden_first, (int)sc->hidden_count, s->hcdf, s->hguide, s->hprefix,
                            s->harea, st));
        float area = 0.f;
        MT_CUDA_TRY(cudaMemcpyAsync(&area, s->harea, sizeof(float), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        s->h_first = -1;  // a failure below leaves no table behind
        MT_CHECK_ARG(area > 0.f, "the hidden triangles have no area");
        s->h_area = area;
        s->h_first = (int32_t)sc->hidden_first;
        s->h_count = (int32_t)sc->hidden_count;
    }
    if (sc->mode == MT_EXHAUSTIVE) {
        const long long need = (long long)sc->n_lasers * spp;
        if (need > s->ysamp_cap) {
            cudaStreamCaptureStatus cs;
            MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
            MT_CHECK_ARG(cs == cudaStreamCaptureStatusNone,
                         "the first exhaustive NLOS call of this size must not be captured (it sizes its scratch)");
            MT_TRY(s->al.alloc(&s->ysamp, (size_t)need * 2, "nlos hidden samples"));
            MT_TRY(s->al.alloc(&s->ysamp_tri, (size_t)need, "nlos hidden samples"));
            s->ysamp_cap = need;
        }
    }
    nlos_fill(s, f, sc, spp, seed, sample_offset, s->hcdf, s->hguide, s->h_area, nullptr, s->ysamp, s->ysamp_tri,
              s->tile_counter + 1, p, cfg);
    return MT_OK;
}

static mt_status nlos_enqueue(mt_scene s, mt_film f, const NlosParams &p, const LaunchCfg &cfg, bool dump,
                              cudaStream_t st) {
    if (p.D < p.T && !(p.flags & MT_ACCUMULATE))
        MT_CUDA_TRY(cudaMemsetAsync(p.film, 0, (size_t)f->H * f->W * f->T * sizeof(float), st));
    if (dump) MT_CUDA_TRY(cudaMemsetAsync(p.dump_count, 0, sizeof(int64_t), st));
    MT_CUDA_TRY(cudaMemsetAsync(p.tile_counter, 0, sizeof(int), st));
    s->launches += p.mode == MT_EXHAUSTIVE ? 2 : 1;
    return mt_launch_nlos(s->dev, p, cfg, dump, (f->flags & MT_COUNTERS) != 0, st);
}

mt_status mt_render_nlos(mt_scene s, mt_film f, const mt_scan *scan, int32_t spp, uint64_t seed,
                         uint64_t sample_offset, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    NlosParams p;
    LaunchCfg cfg;
    MT_TRY(nlos_prepare(s, f, scan, spp, seed, sample_offset, p, cfg, st));
    cudaStreamCaptureStatus cs;
    MT_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || (f->flags & MT_COUNTERS) || (cfg.options & MT_OPT_NO_GRAPH))
        return nlos_enqueue(s, f, p, cfg, false, st);
    // replay a cached graph of [zero counters, (sample pass,) connection pass];
    // re-capture when any launch parameter changed
    std::vector<unsigned char> key(sizeof(NlosParams) + sizeof(LaunchCfg) + sizeof(mt_film_s));
    memcpy(key.data(), &p, sizeof(NlosParams));
    memcpy(key.data() + sizeof(NlosParams), &cfg, sizeof(LaunchCfg));
    memcpy(key.data() + sizeof(NlosParams) + sizeof(LaunchCfg), f, sizeof(mt_film_s));
    GraphCache &gc = s->nlos_graph;
    if (!gc.exec || gc.key != key) {
        if (!s->cap_stream) MT_CUDA_TRY(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g;
        const long long launches = s->launches;  // counted when the graph runs
        MT_CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        const mt_status es = nlos_enqueue(s, f, p, cfg, false, s->cap_stream);
        s->launches = launches;
        const cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
        if (es != MT_OK) {
            if (ce == cudaSuccess) cudaGraphDestroy(g);
            return es;
        }
        MT_CUDA_TRY(ce);
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        MT_CUDA_TRY(ie);
        gc.key = key;
    }
    MT_CUDA_TRY(cudaGraphLaunch(gc.exec, st));
    s->launches += scan->mode == MT_EXHAUSTIVE ? 2 : 1;
    return MT_OK;
}

mt_status mt_render_dump(mt_scene s, mt_film f, const mt_scan *scan, int32_t spp, uint64_t seed, int32_t max_depth,
                         uint64_t sample_offset, mt_contrib *d_dump, int64_t cap, int64_t *d_count, void *stream) {
    MT_CHECK_ARG(d_dump != nullptr && d_count != nullptr && cap >= 0, "dump buffers must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (scan) {
        NlosParams p;
        LaunchCfg cfg;
        MT_TRY(nlos_prepare(s, f, scan, spp, seed, sample_offset, p, cfg, st));
        p.dump = d_dump;
        p.dump_cap = cap;
        p.dump_count = (unsigned long long *)d_count;
        return nlos_enqueue(s, f, p, cfg, true, st);
    }
    return render_common(s, f, spp, seed, max_depth, sample_offset, 1, nullptr, nullptr, nullptr, nullptr, nullptr,
                         d_dump, cap, d_count, st);
}

mt_status mt_sync(mt_scene s, void *stream) {
    MT_CHECK_ARG(s != nullptr, "scene is NULL");
    MT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    MT_CUDA_TRY(cudaGetLastError());
    return check_err_word(s);
}

mt_status mt_stage_times(mt_scene s, double *out, int32_t reset) {
    MT_CHECK_ARG(s != nullptr && out != nullptr, "bad arguments");
    for (int k = 0; k < 4; ++k) out[k] = s->wf_timing.ms[k];
    out[4] = (double)s->wf_timing.iters;
    if (reset) {
        for (int k = 0; k < 4; ++k) s->wf_timing.ms[k] = 0.0;
        s->wf_timing.iters = 0;
    }
    return MT_OK;
}

mt_status mt_read_counters(mt_scene s, uint64_t *out, int32_t reset, void *stream) {
    MT_CHECK_ARG(s != nullptr && out != nullptr, "NULL argument");
    MT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    MT_CUDA_TRY(cudaMemcpy(out, s->counters, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (reset) MT_CUDA_TRY(cudaMemset(s->counters, 0, 8 * sizeof(uint64_t)));
    return MT_OK;
}

mt_status mt_scene_stats(mt_scene s, int64_t *out) {
    MT_CHECK_ARG(s != nullptr && out != nullptr, "NULL argument");
    out[0] = s->n_tris;
    out[1] = s->bvh.n_nodes;
    out[2] = s->bvh.depth;
    out[3] = (int64_t)llround(s->bvh.sah * 1000.0);
    out[4] = s->dev.n_units;
    out[5] = (int64_t)s->bvh.n_nodes * 32 + (int64_t)s->bvh.n_wnodes * 80 + s->n_tris * 48 + s->n_tris * 24;
    out[6] = (int64_t)llround(s->bvh.build_us);
    out[7] = s->launches;
    return MT_OK;
}

mt_status mt_set_launch(mt_scene s, int32_t kind, int32_t threads, int32_t tile, int32_t ctas_per_sm,
                        int32_t priv_bins, uint32_t options) {
    MT_CHECK_ARG(s != nullptr, "scene is NULL");
    MT_CHECK_ARG(kind >= 0 && kind <= MT_LAUNCH_NLOS_EXHAUSTIVE, "unknown launch kind");
    MT_CHECK_ARG(threads == 0 || (threads >= 32 && threads <= 256 && threads % 32 == 0), "threads must be 32..256, x32");
    MT_CHECK_ARG(tile >= 0 && tile <= 4096 && ctas_per_sm >= 0 && ctas_per_sm <= 32, "bad tile / ctas_per_sm");
    MT_CHECK_ARG(priv_bins >= -1, "priv_bins must be >= -1");
    MT_CHECK_ARG((options & ~(MT_OPT_AGGREGATE | MT_OPT_NO_GRAPH | MT_OPT_WAVEFRONT | MT_OPT_DYNAMIC_FETCH |
                              MT_OPT_WIDE_BVH | MT_OPT_SORT_RAYS | MT_OPT_STAGE_TIMING | MT_OPT_SORT_SHADOW |
                              0xFF00u)) == 0,
                 "unknown launch options 0x%x", options);
    LaunchCfg &c = s->cfg[kind];
    c.threads = threads ? threads : 256;
    c.tile = tile;
    c.ctas_per_sm = ctas_per_sm;
    c.priv = priv_bins;
    c.options = (int)options;
    return MT_OK;
}

mt_status mt_set_wavefront_pool(mt_scene s, int64_t max_paths) {
    MT_CHECK_ARG(s != nullptr, "scene is NULL");
    MT_CHECK_ARG(max_paths == 0 || (max_paths >= 32 && max_paths <= (int64_t)MT_WF_POOL_DEFAULT),
                 "max_paths must be 0 or lie in [32, %u]", MT_WF_POOL_DEFAULT);
    s->wf_pool_max = max_paths == 0 ? MT_WF_POOL_DEFAULT : (uint32_t)max_paths;
    return MT_OK;
}

mt_status mt_probe_philox(uint64_t seed, const uint32_t *d_counters, int64_t n, uint32_t *d_out, void *stream) {
    MT_CHECK_ARG(d_counters != nullptr && d_out != nullptr && n >= 0, "bad arguments");
    if (n == 0) return MT_OK;
    uint32_t k0, k1;
    seed_key(seed, k0, k1);
    k_probe_philox<<<grid_for(n, 256, 152), 256, 0, (cudaStream_t)stream>>>(k0, k1, (const uint4 *)d_counters, n,
                                                                           (uint4 *)d_out);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

mt_status mt_probe_trace(mt_scene s, const float *d_rays, int64_t n, float tmax, int32_t any_hit, int32_t *d_tri,
                         float *d_t, void *stream) {
    MT_CHECK_ARG(s != nullptr && d_rays != nullptr && d_tri != nullptr && n >= 0 && (any_hit & ~3) == 0,
                 "bad arguments");
    if (n == 0) return MT_OK;
    k_probe_trace<<<grid_for(n, 128, s->num_sms), 128, 0, (cudaStream_t)stream>>>(s->dev, d_rays, n, tmax, any_hit,
                                                                                 d_tri, d_t);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

mt_status mt_probe_bins(const float *d_opl, int64_t n, float start, float width, int32_t T, int32_t *d_bin,
                        void *stream) {
    MT_CHECK_ARG(d_opl != nullptr && d_bin != nullptr && n >= 0 && width > 0.f && T >= 1, "bad arguments");
    if (n == 0) return MT_OK;
    k_probe_bins<<<grid_for(n, 256, 152), 256, 0, (cudaStream_t)stream>>>(d_opl, n, start, width, T, d_bin);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// NLOS capture that allocates nothing: the per-call scratch (tile counter,
// hidden-surface table with its guide table, running area sums, per-laser
// hidden samples) lives in one static device array compiled into the library
// instead of scene-owned buffers.
// ---------------------------------------------------------------------------
#define MT_NOALLOC_MAX_HIDDEN (1 << 16)
#define MT_NOALLOC_MAX_SAMPLES (1 << 17)
namespace {
constexpr size_t na_up(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_HDR = 256;                                         // tile counter at 0, hidden area at 16
constexpr size_t NA_CDF = (size_t)MT_NOALLOC_MAX_HIDDEN * 4;           // u32 table per hidden triangle
constexpr size_t NA_GUIDE = na_up(((size_t)MT_HGUIDE_N + 1) * 4);      // guide table over the u32 table
constexpr size_t NA_PREFIX = (size_t)MT_NOALLOC_MAX_HIDDEN * 8;        // running area sums (double)
constexpr size_t NA_YS = (size_t)MT_NOALLOC_MAX_SAMPLES * 32;          // two float4 per (laser, sample)
constexpr size_t NA_YT = (size_t)MT_NOALLOC_MAX_SAMPLES * 4;           // hidden triangle per (laser, sample)
constexpr size_t NA_BYTES = NA_HDR + NA_CDF + NA_GUIDE + NA_PREFIX + NA_YS + NA_YT;  // 5.27 MiB
}  // namespace

static __device__ __align__(256) unsigned char g_mt_noalloc_scratch[NA_BYTES];
static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[256];

// device address of the static array for the current device (looked up once per device)
static mt_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    MT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        mt::set_error("device ordinal %d out of range", dev);
        return MT_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        MT_CUDA_TRY(cudaGetSymbolAddress(&p, g_mt_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return MT_OK;
}

extern "C" mt_status mt_render_nlos_noalloc(mt_scene s, mt_film f, const mt_scan *sc, int32_t spp, uint64_t seed,
                                            uint64_t sample_offset, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    MT_TRY(nlos_check(s, f, sc, spp, sample_offset));
    MT_CHECK_ARG(sc->hidden_count <= (uint32_t)MT_NOALLOC_MAX_HIDDEN,
                 "mt_render_nlos_noalloc: %u hidden triangles exceed the static scratch limit of %d",
                 sc->hidden_count, MT_NOALLOC_MAX_HIDDEN);
    MT_CHECK_ARG(sc->mode != MT_EXHAUSTIVE || (long long)sc->n_lasers * spp <= (long long)MT_NOALLOC_MAX_SAMPLES,
                 "mt_render_nlos_noalloc: n_lasers * spp = %lld exceeds the static scratch limit of %d",
                 (long long)sc->n_lasers * spp, MT_NOALLOC_MAX_SAMPLES);
    unsigned char *base = nullptr;
    MT_TRY(noalloc_scratch(&base));
    int *tile_counter = reinterpret_cast<int *>(base);
    float *d_area = reinterpret_cast<float *>(base + 16);
    size_t off = NA_HDR;
    uint32_t *cdf = reinterpret_cast<uint32_t *>(base + off);
    off += NA_CDF;
    uint32_t *guide = reinterpret_cast<uint32_t *>(base + off);
    off += NA_GUIDE;
    double *prefix = reinterpret_cast<double *>(base + off);
    off += NA_PREFIX;
    float4 *ys = reinterpret_cast<float4 *>(base + off);
    off += NA_YS;
    int32_t *yt = reinterpret_cast<int32_t *>(base + off);
    // the sampling table is rebuilt in the array on every call; the kernels read
    // the hidden area from the array, so nothing is read back to the host
    MT_TRY(hidden_table(s, (int)sc->hidden_first, (int)sc->hidden_count, cdf, guide, prefix, d_area, st));
    NlosParams p;
    LaunchCfg cfg;
    nlos_fill(s, f, sc, spp, seed, sample_offset, cdf, guide, 0.f, d_area, ys, yt, tile_counter, p, cfg);
    s->launches += 4;  // the table build
    return nlos_enqueue(s, f, p, cfg, false, st);
}
