// mt_common.cuh -- shared device code of libmt: Philox RNG, vector math,
// sampling maps, BSDFs and the device view of a scene.
//
// Every function here is FP32 device code for sm_103a.  The estimator follows
// arXiv 2510.25660 Sec. 3 (paths, time of flight as optical path length,
// impulse response without scattering delays, Monte Carlo estimator, path
// reuse); the sampling maps and random-number layout are this library's
// readings of what the paper leaves open, stated next to each function.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MT_PI 3.14159265358979323846f
#define MT_MAX_DEPTH 64
#define MT_STACK 64
#define MT_TRACK_STEPS 1024

// device error word bits
#define MT_EFLAG_STACK 1u
#define MT_EFLAG_TIMEOUT 2u
#define MT_EFLAG_TRACK 4u

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float length(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float3 normalize(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
__device__ __forceinline__ float maxabs3(float3 p) { return fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter layout:
// (pixel or scan index, sample index, vertex index, group); key = seed.
// Uniforms are the top 24 bits times 2^-24, exact in float, in [0, 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

#define G_NEE 0u
#define G_SCATTER 1u
#define G_TRACK 0x100u
#define G_RATIO 0x10000u
#define G_DELAY 0x20000u  // scattering delay at a surface vertex
#define G_PULSE 0x20010u  // emission time of a contribution (+ kind)

struct Rng {
    uint32_t k0, k1;
    __device__ __forceinline__ uint4 raw(uint32_t a, uint32_t b, uint32_t c, uint32_t d) const {
        return philox4x32_10(make_uint4(a, b, c, d), k0, k1);
    }
};

// ---------------------------------------------------------------------------
// frames and sampling maps
// ---------------------------------------------------------------------------
// Orthonormal basis from a unit vector (Duff et al., JCGT 2017); n.z >= 0 (and
// -0) takes the positive branch.
__device__ __forceinline__ void onb(float3 n, float3 &t, float3 &b) {
    const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + n.z);
    const float c = n.x * n.y * a;
    t = f3(1.0f + sg * n.x * n.x * a, sg * c, -sg * n.x);
    b = f3(c, sg + n.y * n.y * a, -n.y);
}
__device__ __forceinline__ float3 to_local(float3 w, float3 t, float3 b, float3 n) {
    return f3(dot(w, t), dot(w, b), dot(w, n));
}
__device__ __forceinline__ float3 to_world(float3 l, float3 t, float3 b, float3 n) {
    return t * l.x + b * l.y + n * l.z;
}
// ray-origin offset along the side normal: 1e-4 * max(1, |p|_inf)
__device__ __forceinline__ float eps_of(float3 p) { return 1e-4f * fmaxf(1.0f, maxabs3(p)); }

// uniform point on a triangle: b0 = 1 - sqrt(u1), b1 = u2 sqrt(u1)
__device__ __forceinline__ float3 tri_point(float3 v0, float3 v1, float3 v2, float u1, float u2) {
    const float su = sqrtf(u1);
    const float b0 = 1.0f - su, b1 = u2 * su, b2 = 1.0f - b0 - b1;
    return v0 * b0 + v1 * b1 + v2 * b2;
}

// ---------------------------------------------------------------------------
// BSDFs in the local frame (z = side normal).  Lambert: albedo/pi with cosine
// sampling.  GGX conductor: D GGX, Smith height-correlated G2, Schlick F with
// F0 = albedo, visible-normal sampling (Heitz, JCGT 2018).
// ---------------------------------------------------------------------------
struct Mat {
    float3 alb;
    float rough; // < 0 marks Lambert
};

__device__ __forceinline__ float ggx_lambda(float a2, float3 w) {
    const float s2 = w.x * w.x + w.y * w.y;
    return 0.5f * (-1.0f + sqrtf(1.0f + a2 * s2 / (w.z * w.z)));
}

// f (per channel) and the solid-angle pdf of bsdf_sample for (wo, wi)
__device__ __forceinline__ void bsdf_eval(const Mat &m, float3 wo, float3 wi, float3 &f, float &pdf) {
    f = f3(0.f, 0.f, 0.f);
    pdf = 0.f;
    if (wo.z <= 0.f || wi.z <= 0.f) return;
    if (m.rough < 0.f) {
        f = m.alb * (1.0f / MT_PI);
        pdf = wi.z * (1.0f / MT_PI);
        return;
    }
    const float a = fmaxf(m.rough, 1e-4f), a2 = a * a;
    const float3 h = normalize(wo + wi);
    // 1 - h.z^2 (a^2 - 1) written as (h.x^2 + h.y^2) + a^2 h.z^2: no cancellation for small a in FP32
    const float k = (h.x * h.x + h.y * h.y) + a2 * (h.z * h.z);
    const float D = a2 / (MT_PI * k * k);
    const float lo = ggx_lambda(a2, wo), li = ggx_lambda(a2, wi);
    const float G2 = 1.0f / (1.0f + lo + li), G1o = 1.0f / (1.0f + lo);
    const float c = 1.0f - dot(wi, h);
    const float c2 = c * c, m5 = c2 * c2 * c;
    const float3 F = f3(m.alb.x + (1.f - m.alb.x) * m5, m.alb.y + (1.f - m.alb.y) * m5, m.alb.z + (1.f - m.alb.z) * m5);
    f = F * (D * G2 / (4.0f * wo.z * wi.z));
    pdf = G1o * D / (4.0f * wo.z);
}

// d f_c / d albedo_c divided by f_c
__device__ __forceinline__ float3 bsdf_dratio(const Mat &m, float3 wo, float3 wi) {
    if (m.rough < 0.f) return f3(1.0f / m.alb.x, 1.0f / m.alb.y, 1.0f / m.alb.z);
    const float3 h = normalize(wo + wi);
    const float c = 1.0f - dot(wi, h);
    const float c2 = c * c, m5 = c2 * c2 * c;
    return f3((1.f - m5) / (m.alb.x + (1.f - m.alb.x) * m5), (1.f - m5) / (m.alb.y + (1.f - m.alb.y) * m5),
              (1.f - m5) / (m.alb.z + (1.f - m.alb.z) * m5));
}

__device__ __forceinline__ bool bsdf_sample(const Mat &m, float3 wo, float u0, float u1, float3 &wi) {
    if (m.rough < 0.f) {
        const float r = sqrtf(u0), ph = 2.0f * MT_PI * u1;
        float s, c;
        sincosf(ph, &s, &c);
        wi = f3(r * c, r * s, sqrtf(fmaxf(0.f, 1.0f - u0)));
        return wi.z > 0.f;
    }
    const float a = fmaxf(m.rough, 1e-4f);
    const float3 vh = normalize(f3(a * wo.x, a * wo.y, wo.z));
    const float l2 = vh.x * vh.x + vh.y * vh.y;
    const float3 T1 = l2 > 0.f ? f3(-vh.y, vh.x, 0.f) * rsqrtf(l2) : f3(1.f, 0.f, 0.f);
    const float3 T2 = cross(vh, T1);
    const float r = sqrtf(u0), ph = 2.0f * MT_PI * u1;
    float s, c;
    sincosf(ph, &s, &c);
    const float t1 = r * c;
    float t2 = r * s;
    const float sh = 0.5f * (1.0f + vh.z);
    t2 = (1.0f - sh) * sqrtf(fmaxf(0.f, 1.0f - t1 * t1)) + sh * t2;
    const float3 nh = T1 * t1 + T2 * t2 + vh * sqrtf(fmaxf(0.f, 1.0f - t1 * t1 - t2 * t2));
    const float3 ne = normalize(f3(a * nh.x, a * nh.y, fmaxf(0.f, nh.z)));
    wi = ne * (2.0f * dot(wo, ne)) - wo;
    return wi.z > 0.f;
}

// Henyey-Greenstein phase function; cos_theta between propagation directions
__device__ __forceinline__ float hg_eval(float g, float c) {
    const float d = 1.0f + g * g - 2.0f * g * c;
    return (1.0f - g * g) / (4.0f * MT_PI * d * sqrtf(d));
}
__device__ __forceinline__ float3 hg_sample(float g, float3 dir, float u0, float u1) {
    float c;
    if (fabsf(g) < 1e-3f) c = 1.0f - 2.0f * u0;
    else {
        const float q = (1.0f - g * g) / (1.0f - g + 2.0f * g * u0);
        c = (1.0f + g * g - q * q) / (2.0f * g);
    }
    c = fminf(1.0f, fmaxf(-1.0f, c));
    const float sn = sqrtf(fmaxf(0.f, 1.0f - c * c)), ph = 2.0f * MT_PI * u1;
    float s, co;
    sincosf(ph, &s, &co);
    float3 t, b;
    onb(dir, t, b);
    return to_world(f3(sn * co, sn * s, c), t, b, dir);
}

// ---------------------------------------------------------------------------
// device view of a scene (passed by value to kernels)
// ---------------------------------------------------------------------------
struct LightUnit {
    float4 v0;  // xyz, w = area
    float4 v1;  // xyz, w = pick probability
    float4 v2;  // xyz, w = emitter index (int bits)
    float4 n;   // unit winding normal, w = original triangle index (int bits), -1 for a point emitter
};

// L2 eviction priorities (PTX createpolicy / .L2::cache_hint, sm_80 and later),
// off by default: loading BVH nodes and triangle records (~76 MB for 1.16M
// triangles, less than the 129 MB L2) as evict-last made the 512x512x256-spp
// forward render of that scene slower (102.8 against 98.5 ms), and streaming the
// film atomics as evict-first changed nothing (98.5 ms).
#ifndef MT_L2_KEEP_BVH
#define MT_L2_KEEP_BVH 0
#endif
#ifndef MT_L2_STREAM_FILM
#define MT_L2_STREAM_FILM 0
#endif

__device__ __forceinline__ unsigned long long l2_policy_keep() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_policy_stream() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ldg_keep(const uint4 *a) {
#if MT_L2_KEEP_BVH
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(a), "l"(l2_policy_keep()));
    return r;
#else
    return __ldg(a);
#endif
}
__device__ __forceinline__ float4 ldg_keep(const float4 *a) {
#if MT_L2_KEEP_BVH
    float4 r;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(a), "l"(l2_policy_keep()));
    return r;
#else
    return __ldg(a);
#endif
}
// fire-and-forget float add into global memory, evict-first in L2
__device__ __forceinline__ void red_add_stream(float *a, float v) {
#if MT_L2_STREAM_FILM
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(l2_policy_stream())
                 : "memory");
#else
    atomicAdd(a, v);
#endif
}

struct DevScene {
    const uint4 *nodes;    // 2 x uint4 per internal node
    const uint4 *wnodes;   // 5 x uint4 per 8-wide node (root = node 0)
    const float4 *tris;    // 3 x float4 per leaf-ordered triangle, v0.w = original index
    const float4 *mats;    // per original triangle: albedo, w = GGX roughness or -1 (Lambert)
    const int32_t *tri_unit; // per original triangle: light unit or -1
    const int32_t *leaf_of;  // per original triangle: its leaf-order index
    // per leaf-ordered triangle, the two float4 a shading step reads (one 32-byte sector):
    // geometric normal (winding) + light unit (int bits, -1 = none), material as in mats
    const float4 *shrec;
    const uint32_t *unit_cdf; // ceil(cdf * 2^24)
    const LightUnit *units;
    const float4 *em_rad;  // per emitter: radiance (rgb)
    int32_t n_units;
    int32_t n_tris;
    int32_t n_em;
    int32_t has_medium;
    // time-resolved materials and sources (Sec. 4.1 scattering delays; Sec. 3 emission pulse)
    const float *delay;    // per original triangle: exponential delay mean (m), nullptr = none
    int32_t pulse_type;    // MT_PULSE_*
    float pulse_a, pulse_b;
    float3 cam_o, cam_f, cam_r, cam_u;
    float tan_half;
    float3 q_lo, q_scale;  // BVH plane quantisation: plane = q_lo + q * q_scale
    // medium
    const float *dens;     // [z][y][x]
    int32_t rx, ry, rz;
    float3 m_lo, m_hi;
    float m_major;
    const float *m_params; // device [2]: albedo, g
    uint32_t *err;
    unsigned long long *counters; // 8 counters
};

__device__ __forceinline__ void raise_err(const DevScene &s, uint32_t bit) { atomicOr(s.err, bit); }

// ---------------------------------------------------------------------------
// participating medium (Sec. 4.1): trilinear density, box overlap, ratio tracking
// ---------------------------------------------------------------------------
__device__ __forceinline__ float density_at(const DevScene &s, float3 p) {
    const float gx = (p.x - s.m_lo.x) / (s.m_hi.x - s.m_lo.x) * s.rx - 0.5f;
    const float gy = (p.y - s.m_lo.y) / (s.m_hi.y - s.m_lo.y) * s.ry - 0.5f;
    const float gz = (p.z - s.m_lo.z) / (s.m_hi.z - s.m_lo.z) * s.rz - 0.5f;
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
    const int x0 = min(max(ix, 0), s.rx - 1), x1 = min(max(ix + 1, 0), s.rx - 1);
    const int y0 = min(max(iy, 0), s.ry - 1), y1 = min(max(iy + 1, 0), s.ry - 1);
    const int z0 = min(max(iz, 0), s.rz - 1), z1 = min(max(iz + 1, 0), s.rz - 1);
    auto D = [&](int x, int y, int z) { return __ldg(&s.dens[((size_t)z * s.ry + y) * s.rx + x]); };
    const float c00 = D(x0, y0, z0) * (1.f - fx) + D(x1, y0, z0) * fx;
    const float c10 = D(x0, y1, z0) * (1.f - fx) + D(x1, y1, z0) * fx;
    const float c01 = D(x0, y0, z1) * (1.f - fx) + D(x1, y0, z1) * fx;
    const float c11 = D(x0, y1, z1) * (1.f - fx) + D(x1, y1, z1) * fx;
    const float c0 = c00 * (1.f - fy) + c10 * fy, c1 = c01 * (1.f - fy) + c11 * fy;
    return c0 * (1.f - fz) + c1 * fz;
}

// overlap of the ray with the medium box, clipped to [0, tmax]
__device__ __forceinline__ bool medium_span(const DevScene &s, float3 o, float3 d, float tmax, float &a, float &b) {
    float t0 = 0.f, t1 = tmax;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    const float lo[3] = {s.m_lo.x, s.m_lo.y, s.m_lo.z}, hi[3] = {s.m_hi.x, s.m_hi.y, s.m_hi.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (dd[k] == 0.f) {
            if (oo[k] < lo[k] || oo[k] > hi[k]) return false;
            continue;
        }
        float ta = (lo[k] - oo[k]) / dd[k], tb = (hi[k] - oo[k]) / dd[k];
        if (ta > tb) {
            const float x = ta;
            ta = tb;
            tb = x;
        }
        t0 = fmaxf(t0, ta);
        t1 = fminf(t1, tb);
    }
    if (t0 >= t1) return false;
    a = t0;
    b = t1;
    return true;
}

// ratio-tracking transmittance over [0, dist]; ok = false if the step cap was hit
__device__ __forceinline__ float transmittance(const DevScene &s, const Rng &rng, float3 o, float3 d, float dist,
                                               uint32_t pix, uint32_t smp, uint32_t depth, bool &ok) {
    ok = true;
    float a, b;
    if (!medium_span(s, o, d, dist, a, b)) return 1.0f;
    float T = 1.0f, t = a;
    const float inv = 1.0f / s.m_major;
    for (uint32_t j = 0;; ++j) {
        if (j >= MT_TRACK_STEPS) {
            ok = false;
            return 0.f;
        }
        const uint4 R = rng.raw(pix, smp, depth, G_RATIO + j);
        t += -logf(1.0f - u24(R.x)) * inv;
        if (t >= b) break;
        T *= 1.0f - density_at(s, o + d * t) * inv;
    }
    return T;
}

// exponential draw of mean `mean` from one Philox word (1 - u > 0)
__device__ __forceinline__ float exp_draw(float mean, uint32_t x) { return -mean * logf(1.0f - u24(x)); }

// scattering delay of a surface vertex on original triangle `orig` (0 without delays)
__device__ __forceinline__ float vertex_delay(const DevScene &s, int orig, uint32_t pix, uint32_t smp, uint32_t depth,
                                              uint32_t k0, uint32_t k1) {
    if (!s.delay) return 0.0f;
    const float tau = __ldg(&s.delay[orig]);
    if (!(tau > 0.0f)) return 0.0f;
    return exp_draw(tau, philox4x32_10(make_uint4(pix, smp, depth, G_DELAY), k0, k1).x);
}

// emission time of one contribution (kind 0 = found at vertex `depth`, 1 = next-event there):
// box [0, a), Gaussian (a, b) by Box-Muller, exponential of mean a; 0 for a delta pulse
__device__ __forceinline__ float pulse_time(const DevScene &s, uint32_t pix, uint32_t smp, uint32_t depth, int kind,
                                            uint32_t k0, uint32_t k1) {
    if (s.pulse_type == 0) return 0.0f;
    const uint4 R = philox4x32_10(make_uint4(pix, smp, depth, G_PULSE + (uint32_t)kind), k0, k1);
    switch (s.pulse_type) {
    case 1: return s.pulse_a * u24(R.x);
    case 2: return s.pulse_a + s.pulse_b * sqrtf(-2.0f * logf(1.0f - u24(R.x))) * cospif(2.0f * u24(R.y));
    case 3: return exp_draw(s.pulse_a, R.x);
    default: return 0.0f;
    }
}

// Add v to addr[0..n) (shared or global memory).  With aggregate set, the
// lanes of the warp that target the same address first sum their values with
// shuffles and only the group's first lane issues the atomics.
template <int N, bool AGG>
__device__ __forceinline__ void splat_add(float *addr, const float *v) {
    if (AGG) {
        const unsigned active = __activemask();
        const unsigned peers = __match_any_sync(active, (unsigned long long)addr);
        if (peers != (1u << (threadIdx.x & 31))) {
            float sum[N];
#pragma unroll
            for (int k = 0; k < N; ++k) sum[k] = 0.f;
            unsigned m = peers;
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
#pragma unroll
                for (int k = 0; k < N; ++k) sum[k] += __shfl_sync(peers, v[k], src);
            }
            if ((threadIdx.x & 31) == __ffs(peers) - 1) {
#pragma unroll
                for (int k = 0; k < N; ++k) atomicAdd(addr + k, sum[k]);
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) atomicAdd(addr + k, v[k]);
}
