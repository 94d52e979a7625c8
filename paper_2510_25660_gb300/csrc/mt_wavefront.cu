// mt_wavefront.cu -- wavefront form of the forward transient path tracer.
//
// The same estimator as k_render (arXiv 2510.25660 Sec. 3: paths, optical
// path length, next-event estimation with power-heuristic MIS, path reuse into
// time bins), reorganised so that every traversal kernel sees only one kind of
// ray: up to P paths are in flight in device memory and each iteration runs
//   k_wf_setup     bookkeeping of queue counts, how many new paths to start
//   k_wf_generate  camera rays for new paths behind the continuing ones
//   k_wf_trace     closest hits of all queued extension rays, then the shadow
//                  rays of the previous shading pass (k_wf_extend and
//                  k_wf_shadow separately in the replay, polarized and dump
//                  forms)
//   k_wf_shade     emission found by the path, next-event sample (a shadow ray
//                  carrying its contribution), BSDF sample, continuation
// Warps claim rays 32 at a time from a queue cursor, so lanes stay busy until
// the queue drains; appends to the queues are warp-aggregated.  New paths get
// consecutive ids (pixel-major), so camera rays of a warp share a pixel.
// The state of the forward forms is kept in queue order (the path at queue
// position i has its record at index i of per-field arrays, and shading
// writes a continuing path to its position in the next queue), so every stage
// streams it; the path replay and polarization keep per-slot records in a
// pool indexed through the queues, with a stack of free slots.
// Contributions go to the film with global atomics (no per-tile ownership).
#include <cub/cub.cuh>

#include "mt_common.cuh"
#include "mt_internal.h"
#include "mt_launch.h"
#include "mt_trace.cuh"
#include "mt_polar.cuh"

struct WfIter {
    uint32_t cont, n_new, free_before;
    unsigned long long base;
};

namespace {

// counters[] layout
// C_SH_N: shadow rays queued by the previous iteration's shading, which the
// fused traversal pass of this iteration traces after its extension rays
// C_CONT: continuing paths at the head of this iteration's queue (new paths follow)
enum { C_CUR = 0, C_NEXT = 1, C_SHADOW = 2, C_FREE = 3, C_EXT_CUR = 4, C_SH_CUR = 5, C_DONE = 6, C_FIN = 7, C_SH_N = 8,
       C_CONT = 9 };
#define MT_WF_COUNTERS 16
// 1: extension (closest-hit) and shadow (any-hit) rays of the wavefront
// passes traced by the warp-cooperative hybrid traversal (trace_hybrid)
#ifndef MT_HYBRID_EXT
#define MT_HYBRID_EXT 0
#endif
#ifndef MT_HYBRID_SH
#define MT_HYBRID_SH 0
#endif
// > 0: warps whose 32 queue positions all hold camera rays of new paths
// traverse as a packet while at least this many of their rays enter a node
#ifndef MT_PACKET_CAMERA
#define MT_PACKET_CAMERA 0
#endif
#ifndef MT_WF_FUSE
#define MT_WF_FUSE 1  // 0: a shadow pass of its own after every shading pass
#endif

__device__ __forceinline__ float mis2w(float a, float b) { return a * a / (a * a + b * b); }

__device__ __forceinline__ int pick_unit_wf(const DevScene &s, uint32_t u) {
    int lo = 0, hi = s.n_units - 1;
    const uint32_t key = u >> 8;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key < __ldg(&s.unit_cdf[mid])) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// warp-aggregated append of one entry per participating lane; returns the slot
__device__ __forceinline__ uint32_t wf_append(uint32_t *count, bool want) {
    // every lane of the warp calls this together (shade loops in whole warps)
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    if (!want) return 0;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// 256-bit global loads and stores (sm_100-class) for the 32-byte halves of a
// path record, (o, d) and (beta, meta), when the pool is a record per slot, per
// use: generation stores, extension-ray loads, shading loads, shading stores.
// Measured on the 512x512x256-spp render of the 1.16M-triangle scene: generation
// 3.65 -> 2.2 ms, loads neutral to slightly faster, shading stores 13.7 -> 15.0
// ms (off).
#ifndef MT_WF_V8_GEN
#define MT_WF_V8_GEN MT_WF_AOS
#endif
#ifndef MT_WF_V8_EXT
#define MT_WF_V8_EXT MT_WF_AOS
#endif
#ifndef MT_WF_V8_SHADE_LD
#define MT_WF_V8_SHADE_LD MT_WF_AOS
#endif
#ifndef MT_WF_V8_SHADE_ST
#define MT_WF_V8_SHADE_ST 0
#endif

template <bool V8>
__device__ __forceinline__ void ld_pair(const float4 *a, const float4 *b, float4 &x, float4 &y) {
    if (V8) {  // b == a + 1 in a record
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w), "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
                 : "l"(a));
    } else {
        x = *a;
        y = *b;
    }
}

template <bool V8>
__device__ __forceinline__ void st_pair(float4 *a, float4 *b, float4 x, float4 y) {
    if (V8) {
        asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(a), "f"(x.x), "f"(x.y), "f"(x.z),
                     "f"(x.w), "f"(y.x), "f"(y.y), "f"(y.z), "f"(y.w)
                     : "memory");
    } else {
        *a = x;
        *b = y;
    }
}

__device__ __forceinline__ float4 u4f(uint4 v) {
    return make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w));
}
__device__ __forceinline__ uint4 f4u(float4 v) {
    return make_uint4(__float_as_uint(v.x), __float_as_uint(v.y), __float_as_uint(v.z), __float_as_uint(v.w));
}

// frequency space (Sec. 4.3, Eq. 12): C exp(-i 2 pi opl / lambda); "bin" 2q real, 2q + 1 imaginary.
// Out of line so that its registers do not weigh on the time-binned path.  lp = film pixel.
__device__ __noinline__ void wf_splat_phasor(const WfParams &p, uint32_t lp, float opl, float3 c) {
    for (int q = 0; q < p.K; ++q) {
        float sn, cs;
        sincospif(2.0f * opl / __ldg(&p.lambdas[q]), &sn, &cs);
        float *h = p.film + ((size_t)lp * p.T + 2 * q) * 3;
        red_add_stream(h, c.x * cs);
        red_add_stream(h + 1, c.y * cs);
        red_add_stream(h + 2, c.z * cs);
        red_add_stream(h + 3, -c.x * sn);
        red_add_stream(h + 4, -c.y * sn);
        red_add_stream(h + 5, -c.z * sn);
    }
}

// pix is the frame pixel id; the film holds the window that starts at p.pix_base
__device__ __forceinline__ void wf_splat(const WfParams &p, uint32_t pix, float opl, float3 c) {
    const uint32_t lp = pix - p.pix_base;
    const float x = (opl - p.start) / p.width;
    if (p.splat_count)  // counting pass only: splats of this contribution into global memory
        atomicAdd(p.splat_count, (unsigned long long)((p.K > 0 ? 2 * p.K : (x >= 0.f && x < (float)p.T ? 1 : 0)) +
                                                      (p.steady ? 1 : 0)));
    if (p.K > 0) {
        wf_splat_phasor(p, lp, opl, c);
    } else if (x >= 0.f && x < (float)p.T) {
        float *h = p.film + ((size_t)lp * p.T + (int)x) * 3;
        red_add_stream(h, c.x);
        red_add_stream(h + 1, c.y);
        red_add_stream(h + 2, c.z);
    }
    if (p.steady) {
        float *g = p.steady + (size_t)lp * 3;
        red_add_stream(g, c.x);
        red_add_stream(g + 1, c.y);
        red_add_stream(g + 2, c.z);
    }
}

__device__ __forceinline__ void wf_dump(const WfParams &p, uint32_t pix, uint32_t smp, int depth, int kind, int tri,
                                        float opl, float3 c) {
    const unsigned long long slot = atomicAdd(p.dump_count, 1ull);
    if ((long long)slot < p.dump_cap) {
        const float x = (opl - p.start) / p.width;
        mt_contrib r;
        r.pixel = (int32_t)pix;
        r.sample = (int32_t)smp;
        r.depth = depth;
        r.kind = kind;
        r.tri = tri;
        r.bin = (x >= 0.f && x < (float)p.T) ? (int)x : (int)floorf(x);
        r.opl = opl;
        r.c[0] = c.x / p.scale;
        r.c[1] = c.y / p.scale;
        r.c[2] = c.z / p.scale;
        p.dump[slot] = r;
    }
}

// dL/dfilm at the bin of a contribution at `opl` plus dL/dsteady (backward)
__device__ __forceinline__ float3 wf_grad_at(const WfParams &p, uint32_t pix, float opl) {
    const uint32_t lp = pix - p.pix_base;
    float3 g = p.gsteady ? f3(p.gsteady[lp * 3], p.gsteady[lp * 3 + 1], p.gsteady[lp * 3 + 2]) : f3(0.f, 0.f, 0.f);
    const float x = (opl - p.start) / p.width;
    if (x >= 0.f && x < (float)p.T) {
        const float *h = p.gfilm + ((size_t)lp * p.T + (int)x) * 3;
        g = g + f3(h[0], h[1], h[2]);
    }
    return g;
}

#define MT_WF_EM_SMEM 64  // emitters whose radiance gradients a CTA sums in shared memory

__device__ __forceinline__ void em_grad_add(const WfParams &p, float *em_acc, int n_em, int em, float3 v) {
    if (n_em <= MT_WF_EM_SMEM) {
        atomicAdd(&em_acc[em * 3], v.x);
        atomicAdd(&em_acc[em * 3 + 1], v.y);
        atomicAdd(&em_acc[em * 3 + 2], v.z);
    } else {
        atomicAdd(&p.grad[em * 3], v.x);
        atomicAdd(&p.grad[em * 3 + 1], v.y);
        atomicAdd(&p.grad[em * 3 + 2], v.z);
    }
}

__device__ __forceinline__ void em_grad_flush(const WfParams &p, const float *em_acc, int n_em) {
    __syncthreads();
    if (n_em <= MT_WF_EM_SMEM)
        for (int k = threadIdx.x; k < n_em * 3; k += blockDim.x)
            if (em_acc[k] != 0.f) atomicAdd(&p.grad[k], em_acc[k]);
}

// Paths that ended in this iteration (after their shadow rays were traced):
// suffix sums over the vertex records turn the per-vertex sums of g * C into
// the albedo and medium-albedo gradients (Sec. 4.4 path replay), then the slot
// returns to the free stack.
// Scenes of at most MT_FIN_SMEM_TRIS triangles sum the albedo gradients of a CTA
// in shared memory and add them to global memory once: on a 36-triangle scene
// every vertex of a warp adds to the same few entries, whose global atomics
// then serialise (38.9 ms of a 101-ms backward pass in a medium).
#ifndef MT_FIN_SMEM_TRIS
#define MT_FIN_SMEM_TRIS 4096
#endif
__global__ void __launch_bounds__(256) k_wf_finalize(const DevScene s, const WfParams p) {
    extern __shared__ float s_galb[];  // [3 n_tris] when n_tris <= MT_FIN_SMEM_TRIS
    const bool smem = s.n_tris <= MT_FIN_SMEM_TRIS;
    if (smem) {
        for (int k = threadIdx.x; k < 3 * s.n_tris; k += blockDim.x) s_galb[k] = 0.f;
        __syncthreads();
    }
    const uint32_t n = p.counters[C_FIN];
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t n_round = ((n + 31u) / 32u) * 32u;
    float gm = 0.f;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_round; q += stride) {
        const bool valid = q < n;
        uint32_t slot = 0;
        if (valid) {
            slot = p.fin_q[q];
            const int end = (int)p.meta[slot].w;
            float3 P = f3(0.f, 0.f, 0.f);
            for (int i = end; i >= 1; --i) {
                const size_t r = (size_t)i * p.P + slot;
                const float4 a = p.rec_a[r], b = p.rec_b[r], c = p.rec_c[r];
                const float3 gi = mul(P, xyz(a)) + xyz(c);
                const int tri = __float_as_int(a.w);
                if (tri >= 0) {
                    if (gi.x != 0.f || gi.y != 0.f || gi.z != 0.f) {
                        float *g = smem ? s_galb + 3 * tri : p.galb + (size_t)tri * 3;
                        atomicAdd(g, gi.x);
                        atomicAdd(g + 1, gi.y);
                        atomicAdd(g + 2, gi.z);
                    }
                } else {
                    gm += gi.x + gi.y + gi.z;
                }
                P = P + xyz(b);
            }
        }
        const uint32_t fs = wf_append(&p.counters[C_FREE], valid);
        if (valid) p.free_q[fs] = slot;
    }
    for (int o = 16; o > 0; o >>= 1) gm += __shfl_xor_sync(0xffffffffu, gm, o);
    if ((threadIdx.x & 31) == 0 && gm != 0.f && p.gmed) atomicAdd(p.gmed, gm);
    if (smem) {  // the CTA's sums, once
        __syncthreads();
        for (int k = threadIdx.x; k < 3 * s.n_tris; k += blockDim.x)
            if (s_galb[k] != 0.f) atomicAdd(&p.galb[k], s_galb[k]);
    }
}

template <typename T>
__device__ __forceinline__ void warp_count(unsigned long long *dst, T v) {
    unsigned long long x = v;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(dst, x);
}

__global__ void k_wf_setup(WfParams p, WfIter *it) {
    uint32_t *c = p.counters;
    const uint32_t cont = c[C_NEXT], freec = p.qmode ? p.P - cont : c[C_FREE];
    const unsigned long long base = *p.next_path;
    const unsigned long long remain = base < p.total_paths ? p.total_paths - base : 0ull;
    const uint32_t n_new = (uint32_t)min((unsigned long long)freec, remain);
    it->cont = cont;
    c[C_CONT] = cont;
    it->n_new = n_new;
    it->free_before = freec;
    it->base = base;
    c[C_CUR] = cont + n_new;
    c[C_NEXT] = 0;
    c[C_SH_N] = c[C_SHADOW];
    c[C_SHADOW] = 0;
    c[C_FREE] = freec - n_new;
    c[C_EXT_CUR] = 0;
    c[C_SH_CUR] = 0;
    c[C_FIN] = 0;
    c[C_DONE] = (cont + n_new == 0) ? 1u : 0u;
    if (p.done_flag) {  // read by the host once this iteration's event has completed
        *(volatile uint32_t *)p.done_flag = c[C_DONE] ? p.done_token : 0u;
        __threadfence_system();
    }
    *p.next_path = base + n_new;
}

__global__ void __launch_bounds__(256) k_wf_generate(const DevScene s, const WfParams p, const WfIter *itp,
                                                     uint32_t *qcur) {
    const WfIter it = *itp;
    uint32_t paths = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < it.n_new; i += gridDim.x * blockDim.x) {
        const uint32_t slot = p.qmode ? 0u : p.free_q[it.free_before - 1 - i];
        const unsigned long long j = it.base + i;
        const uint32_t lpix = (uint32_t)(j / p.spp);
        const uint32_t smp = p.sample_offset + (uint32_t)(j - (unsigned long long)lpix * p.spp);
        const uint32_t pix = lpix + p.pix_base;  // frame pixel id
        const uint4 R = philox4x32_10(make_uint4(pix, smp, 0u, 0u), p.k0, p.k1);
        const bool center = p.flags & MT_PIXEL_CENTER;
        const float jx = center ? 0.5f : u24(R.x), jy = center ? 0.5f : u24(R.y);
        const uint32_t py = pix / (uint32_t)p.W, px = pix - py * (uint32_t)p.W;
        const float sx = (2.0f * ((float)px + jx) / (float)p.W - 1.0f) * s.tan_half;
        const float sy =
            (1.0f - 2.0f * ((float)py + jy) / (float)p.H_full) * s.tan_half * ((float)p.H_full / (float)p.W);
        const float3 d = normalize(s.cam_f + s.cam_r * sx + s.cam_u * sy);
        if (p.qmode) {  // the new path's state at its position in this iteration's queue
            const uint32_t q = it.cont + i;
            p.ps_o[q] = make_float4(s.cam_o.x, s.cam_o.y, s.cam_o.z, 0.f);
            p.ps_d[q] = make_float4(d.x, d.y, d.z, 0.f);
            p.ps_b[q] = make_float4(1.f, 1.f, 1.f, 0.f);
            p.ps_m[q] = make_uint4(pix, smp, 1u, 0u);
            if (p.ps_sig) p.ps_sig[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            paths++;
            continue;
        }
        st_pair<MT_WF_V8_GEN>(&p.o[slot], &p.d[slot], make_float4(s.cam_o.x, s.cam_o.y, s.cam_o.z, 0.f),
                make_float4(d.x, d.y, d.z, 0.f));
        if (p.sig) p.sig[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p.mueller) {  // frame = the camera's horizontal axis (P = identity is implied at depth 1)
            const float3 xf = normalize(s.cam_r - d * dot(s.cam_r, d));
            p.xframe[slot] = make_float4(xf.x, xf.y, xf.z, 0.f);
        }
        st_pair<MT_WF_V8_GEN>(&p.beta[slot], (float4 *)&p.meta[slot], make_float4(1.f, 1.f, 1.f, 0.f),
                u4f(make_uint4(pix, smp, 1u, 0u)));
        qcur[it.cont + i] = slot;
        paths++;
    }
    warp_count(&s.counters[1], paths);
}

// Resident CTAs per SM the traversal stages are compiled for (6 x 256 threads
// caps them at 40 registers; the few spilled values cost less than the
// occupancy they buy: measured 98 ms against 107 ms at 53 registers and 4 CTAs
// per SM for the 512x512x256-spp forward render of the 1.16M-triangle scene).
#ifndef MT_WF_TRACE_MINB
#define MT_WF_TRACE_MINB 6
#endif

// hit record: (leaf-order triangle or -1, original triangle, t bits, 1 if the
// path scatters in the medium at t before reaching that surface)
template <bool WIDE, bool CNT, bool MEDIA>
__device__ __forceinline__ void ext_rays(const DevScene &s, const WfParams &p, const uint32_t *qcur, TraceCnt &tc,
                                         uint32_t &rays) {
    const uint32_t n = p.counters[C_CUR], cont = p.counters[C_CONT];
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&p.counters[C_EXT_CUR], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const uint32_t i = base + lane;
        const bool live = i < n;
        const uint32_t slot = !live ? 0u : (p.qmode ? i : qcur[i]);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f), d = make_float4(0.f, 0.f, 1.f, 0.f);
        if (live) {
            if (p.qmode) {
                o = p.ps_o[i];
                d = p.ps_d[i];
            } else {
                ld_pair<MT_WF_V8_EXT>(&p.o[slot], &p.d[slot], o, d);
            }
        }
        const RayT r = make_ray(s, xyz(o), xyz(d));
        float t;
        int orig;
        int k;
        if (WIDE) {
            k = live ? trace_wide<false, CNT>(s, r, INFINITY, t, orig, tc) : -1;
        } else if (MT_HYBRID_EXT || (MT_PACKET_CAMERA && p.qmode && base >= cont)) {
            // the whole warp traverses together (in queue order, positions from `cont` on hold the
            // camera rays of new paths, consecutive samples of one pixel)
            k = trace_hybrid<false, CNT>(s, r, live, INFINITY, t, orig, tc,
                                         MT_HYBRID_EXT ? MT_HYBRID_MIN : MT_PACKET_CAMERA);
        } else {
            k = live ? trace_closest<CNT>(s, r, INFINITY, t, orig, tc) : -1;
        }
        if (live) {
            int collided = 0;
            if (MEDIA) {
                // delta tracking over the part of the segment inside the medium (Sec. 4.1)
                float ma, mb;
                if (medium_span(s, xyz(o), xyz(d), k >= 0 ? t : 1e30f, ma, mb)) {
                    const uint4 m = p.qmode ? p.ps_m[i] : p.meta[slot];
                    const float inv = 1.0f / s.m_major;
                    float tt = ma;
                    for (uint32_t j = 0;; ++j) {
                        if (j >= MT_TRACK_STEPS) {
                            raise_err(s, MT_EFLAG_TRACK);
                            k = -1;  // the path is dropped
                            break;
                        }
                        const uint4 R = philox4x32_10(make_uint4(m.x, m.y, m.z - 1u, G_TRACK + j), p.k0, p.k1);
                        tt += -logf(1.0f - u24(R.x)) * inv;
                        if (tt >= mb) break;
                        if (u24(R.y) < density_at(s, xyz(o) + xyz(d) * tt) * inv) {
                            collided = 1;
                            t = tt;
                            break;
                        }
                    }
                }
            }
            if (p.qmode) p.ps_h[i] = make_int4(k, orig, __float_as_int(t), collided);
            else p.hit[slot] = make_int4(k, orig, __float_as_int(t), collided);
            rays++;
        }
    }
}

template <bool WIDE, bool CNT, bool MEDIA>
__global__ void __launch_bounds__(256, MT_WF_TRACE_MINB) k_wf_extend(const DevScene s, const WfParams p, const uint32_t *qcur) {
    TraceCnt tc{0, 0};
    uint32_t rays = 0;
    ext_rays<WIDE, CNT, MEDIA>(s, p, qcur, tc, rays);
    warp_count(&s.counters[3], rays);
    if (CNT) {
        warp_count(&s.counters[4], tc.nodes);
        warp_count(&s.counters[5], tc.tris);
    }
}

// 9 bits -> every third bit of 27
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x1FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Key widths of the ray sorts (radix passes of 8 bits each): Morton bits per
// axis of the extension-ray origin grid, of the shadow-ray origin grid, and
// bits per octahedral coordinate of the shadow-ray direction.
#ifndef MT_SORT_EXT_B
#define MT_SORT_EXT_B 9
#endif
#ifndef MT_SORT_SH_B
#define MT_SORT_SH_B 7
#endif
#ifndef MT_SORT_SH_D
#define MT_SORT_SH_D 4
#endif
#define MT_SORT_EXT_BITS (3 + 3 * MT_SORT_EXT_B)
#define MT_SORT_SH_BITS (3 * MT_SORT_SH_B + 2 * MT_SORT_SH_D)

// Sort keys of the queued extension rays: direction octant (3 bits) above the
// Morton code of the origin on a 2^B x 2^B x 2^B grid over the scene box.
// Entries past the queue's end get the largest key and sort to the back.
__global__ void k_wf_sort_keys(const DevScene s, const WfParams p, const uint32_t *qcur) {
    const uint32_t n = p.counters[C_CUR];
    constexpr float G = (float)(1 << MT_SORT_EXT_B);
    const float gx = G / (65536.0f * s.q_scale.x), gy = G / (65536.0f * s.q_scale.y),
                gz = G / (65536.0f * s.q_scale.z);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p.P; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const uint32_t slot = qcur[i];
            const float4 o = p.o[slot], d = p.d[slot];
            const uint32_t cx = (uint32_t)fminf(fmaxf((o.x - s.q_lo.x) * gx, 0.0f), G - 1.0f);
            const uint32_t cy = (uint32_t)fminf(fmaxf((o.y - s.q_lo.y) * gy, 0.0f), G - 1.0f);
            const uint32_t cz = (uint32_t)fminf(fmaxf((o.z - s.q_lo.z) * gz, 0.0f), G - 1.0f);
            const uint32_t oct = (d.x < 0.0f ? 1u : 0u) | (d.y < 0.0f ? 2u : 0u) | (d.z < 0.0f ? 4u : 0u);
            p.sort_keys[i] =
                (oct << (3 * MT_SORT_EXT_B)) | spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
        } else {
            p.sort_keys[i] = 0xFFFFFFFFu;
        }
    }
}

// ---------------------------------------------------------------------------
// Transient polarization in wavefront form (Sec. 4.2): the estimator of the
// path-per-thread kernel k_render_pol (mt_polar.cu) with each path's Mueller
// throughput (3 colours x 4 rows) and segment frame kept in the path pool.
// Shade adds emission Stokes vectors and queues next-event rays with their
// Stokes contributions; the shadow stage splats those that are unoccluded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void wf_splat_stokes(const WfParams &p, uint32_t pix, float opl, const float S[3][4]) {
    const uint32_t lp = pix - p.pix_base;
    const float x = (opl - p.start) / p.width;
    const bool in = x >= 0.f && x < (float)p.T;
    float *f = in ? p.film + ((size_t)lp * p.T + (int)x) * 12 : nullptr;
    float *st = p.steady + (size_t)lp * 12;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = S[c][k];
            if (v != 0.f) {
                if (in) atomicAdd(f + k * 3 + c, v);
                atomicAdd(st + k * 3 + c, v);
            }
        }
}

__device__ __forceinline__ void load_mueller(const WfParams &p, uint32_t slot, Mueller &P) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 v = p.mueller[(size_t)slot * 12 + c * 4 + r];
            P.m[c][4 * r] = v.x;
            P.m[c][4 * r + 1] = v.y;
            P.m[c][4 * r + 2] = v.z;
            P.m[c][4 * r + 3] = v.w;
        }
}

__device__ __forceinline__ void store_mueller(const WfParams &p, uint32_t slot, const Mueller &P) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r)
            p.mueller[(size_t)slot * 12 + c * 4 + r] =
                make_float4(P.m[c][4 * r], P.m[c][4 * r + 1], P.m[c][4 * r + 2], P.m[c][4 * r + 3]);
}

// GGX microfacet factor D G2 / (4 cos_o cos_i) and the cosine of the microfacet
// incidence (conductor branch of the Mueller BSDF)
__device__ __forceinline__ float ggx_factor(float rough, float3 wol, float3 wil, float &cd) {
    const float a = fmaxf(rough, 1e-4f), a2 = a * a;
    const float3 hh = normalize(wol + wil);
    const float kd = (hh.x * hh.x + hh.y * hh.y) + a2 * (hh.z * hh.z);
    const float D = a2 / (MT_PI * kd * kd);
    const float G2 = 1.0f / (1.0f + ggx_lambda(a2, wol) + ggx_lambda(a2, wil));
    cd = dot(wil, hh);
    return D * G2 / (4.0f * wol.z * wil.z);
}

__global__ void __launch_bounds__(128) k_wf_shade_pol(const DevScene s, const WfParams p, const uint32_t *qcur,
                                                     uint32_t *qnext) {
    const uint32_t n = p.counters[C_CUR];
    uint32_t verts = 0, contribs = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t n_round = ((n + 31u) / 32u) * 32u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        const uint32_t slot = valid ? qcur[i] : 0u;
        bool cont = false, shadow = false, done = false;
        float4 sh_o = make_float4(0, 0, 0, 0), sh_d = sh_o, sh_c = sh_o;
        float S_nee[3][4];
        if (valid) {
            const float4 o4 = p.o[slot], d4 = p.d[slot];
            const uint4 m = p.meta[slot];
            const int4 h = p.hit[slot];
            const uint32_t pix = m.x, smp = m.y;
            const int depth = (int)m.z;
            float opl = o4.w;
            const float3 d = xyz(d4);
            if (h.x < 0) {
                done = true;
            } else {
                verts++;
                Mueller P;
                if (depth == 1) {  // a camera ray: identity per colour (not stored)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int e = 0; e < 16; ++e) P.m[c][e] = (e % 5 == 0) ? 1.f : 0.f;
                } else {
                    load_mueller(p, slot, P);
                }
                const float3 xf = xyz(p.xframe[slot]);
                const int k = h.x, orig = h.y;
                const float th = __int_as_float(h.z);
                const float3 x = xyz(o4) + d * th;
                if (!(depth == 1 && (p.flags & MT_UNWARP))) opl += th;
                const float4 sn = __ldg(&s.shrec[2 * (size_t)k]);  // normal + light unit
                const float3 ng = xyz(sn);
                const float3 wo = -d;
                const float cwo = dot(ng, wo);
                const int unit = __float_as_int(sn.w);
                if (unit >= 0 && cwo > 0.f) {  // emission: column 0 of P (unpolarised emitter)
                    const LightUnit U = s.units[unit];
                    float w = 1.0f;
                    if (depth > 1) w = mis2w(d4.w, (U.v1.w / U.v0.w) * th * th / cwo);
                    const float4 Le = s.em_rad[__float_as_int(U.v2.w)];
                    const float le[3] = {Le.x, Le.y, Le.z};
                    float S[3][4];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int q = 0; q < 4; ++q) S[c][q] = P.m[c][4 * q] * le[c] * w * p.scale;
                    wf_splat_stokes(p, pix, opl + pulse_time(s, pix, smp, (uint32_t)depth, 0, p.k0, p.k1), S);
                    contribs++;
                }
                if (depth == p.max_depth) {
                    done = true;
                } else {
                    opl += vertex_delay(s, orig, pix, smp, (uint32_t)depth, p.k0, p.k1);
                    const float3 nn = cwo >= 0.f ? ng : -ng;
                    float3 tb, bb;
                    onb(nn, tb, bb);
                    const float3 wol = to_local(wo, tb, bb, nn);
                    const float4 mm = __ldg(&s.shrec[2 * (size_t)k + 1]);
                    const Mat mat{xyz(mm), mm.w};
                    const float alb[3] = {mm.x, mm.y, mm.z};
                    if (s.n_units > 0) {  // next-event estimate, queued for the shadow stage
                        const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_NEE), p.k0, p.k1);
                        const LightUnit U = s.units[pick_unit_wf(s, R.x)];
                        const int em = __float_as_int(U.v2.w);
                        const bool is_pt = __float_as_int(U.n.w) < 0;
                        const float3 y = is_pt ? xyz(U.v0)
                                               : tri_point(xyz(U.v0), xyz(U.v1), xyz(U.v2), u24(R.y), u24(R.z));
                        const float3 xo = x + nn * eps_of(x);
                        const float3 dl = y - xo;
                        const float dist = sqrtf(dot(dl, dl));
                        const float3 wi = dl * (1.0f / dist);
                        const float cx = dot(nn, wi);
                        const float cy = is_pt ? 1.0f : -dot(xyz(U.n), wi);
                        if (cx > 0.f && cy > 0.f && dist > 0.f) {
                            const float3 wil = to_local(wi, tb, bb, nn);
                            float3 fc;
                            float pb;
                            bsdf_eval(mat, wol, wil, fc, pb);
                            const float pick = U.v1.w;
                            float geo, w = 1.0f;
                            if (is_pt) geo = 1.0f / (dist * dist) / pick;
                            else {
                                const float pA = pick / U.v0.w;
                                geo = cy / (dist * dist) / pA;
                                w = mis2w(pA * dist * dist / cy, pb);
                            }
                            const float4 Le = s.em_rad[em];
                            const float le[3] = {Le.x, Le.y, Le.z};
                            if (mat.rough < 0.f) {
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const float kk = alb[c] * (1.0f / MT_PI) * cx * geo * w * le[c] * p.scale;
#pragma unroll
                                    for (int q = 0; q < 4; ++q) S_nee[c][q] = P.m[c][4 * q] * kk;
                                }
                            } else {
                                // column 0 of (P R(t)) M_F, t the turn from the scattering plane to the frame
                                const float t = frame_angle(wo, plane_normal(wi, d), xf);
                                float s2, c2;
                                sincosf(2.0f * t, &s2, &c2);
                                float cd;
                                const float kf = ggx_factor(mat.rough, wol, wil, cd) * cx * geo * w * p.scale;
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const float4 F = fresnel_abcd(cd, conductor_kappa(alb[c]));
#pragma unroll
                                    for (int q = 0; q < 4; ++q) {
                                        const float q0 = P.m[c][4 * q];
                                        const float q1 = P.m[c][4 * q + 1] * c2 - P.m[c][4 * q + 2] * s2;
                                        S_nee[c][q] = (q0 * F.x + q1 * F.y) * kf * le[c];
                                    }
                                }
                            }
                            bool nonzero = false;
#pragma unroll
                            for (int c = 0; c < 3; ++c)
#pragma unroll
                                for (int q = 0; q < 4; ++q) nonzero |= S_nee[c][q] != 0.f;
                            if (nonzero) {
                                shadow = true;
                                sh_o = make_float4(xo.x, xo.y, xo.z, dist - (is_pt ? 0.0f : eps_of(y)));
                                sh_d = make_float4(wi.x, wi.y, wi.z,
                                                   opl + dist + pulse_time(s, pix, smp, (uint32_t)depth, 1, p.k0,
                                                                           p.k1));
                                sh_c = make_float4(0.f, 0.f, 0.f, __int_as_float((int)pix));
                            }
                        }
                    }
                    // continue by sampling the BSDF
                    const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_SCATTER), p.k0, p.k1);
                    float3 wil;
                    if (bsdf_sample(mat, wol, u24(R.x), u24(R.y), wil)) {
                        float3 f;
                        float pb;
                        bsdf_eval(mat, wol, wil, f, pb);
                        if (pb > 0.f) {
                            const float3 wi = to_world(wil, tb, bb, nn);
                            const float3 sv = plane_normal(wi, d);
                            rotate_columns(P, frame_angle(wo, sv, xf));
                            if (mat.rough < 0.f) {  // ideal depolariser
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const float kk = alb[c] * (1.0f / MT_PI) * wil.z / pb;
#pragma unroll
                                    for (int q = 0; q < 4; ++q) {
                                        P.m[c][4 * q] *= kk;
                                        P.m[c][4 * q + 1] = 0.f;
                                        P.m[c][4 * q + 2] = 0.f;
                                        P.m[c][4 * q + 3] = 0.f;
                                    }
                                }
                            } else {  // P <- P M_F (Fresnel Mueller of the microfacet) x GGX factor / pdf
                                float cd;
                                const float kf = ggx_factor(mat.rough, wol, wil, cd) * wil.z / pb;
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const float4 F = fresnel_abcd(cd, conductor_kappa(alb[c]));
#pragma unroll
                                    for (int q = 0; q < 4; ++q) {
                                        float *row = &P.m[c][4 * q];
                                        const float r0 = row[0], r1 = row[1], r2 = row[2], r3 = row[3];
                                        row[0] = (r0 * F.x + r1 * F.y) * kf;
                                        row[1] = (r0 * F.y + r1 * F.x) * kf;
                                        row[2] = (r2 * F.z - r3 * F.w) * kf;
                                        row[3] = (r2 * F.w + r3 * F.z) * kf;
                                    }
                                }
                            }
                            store_mueller(p, slot, P);
                            p.xframe[slot] = make_float4(sv.x, sv.y, sv.z, 0.f);
                            const float3 no = x + nn * eps_of(x);
                            p.o[slot] = make_float4(no.x, no.y, no.z, opl);
                            p.d[slot] = make_float4(wi.x, wi.y, wi.z, pb);
                            p.meta[slot] = make_uint4(pix, smp, (uint32_t)(depth + 1), 0u);
                            cont = true;
                        }
                    }
                    if (!cont) done = true;
                }
            }
        }
        const uint32_t qs = wf_append(&p.counters[C_NEXT], cont);
        if (cont) qnext[qs] = slot;
        const uint32_t fs = wf_append(&p.counters[C_FREE], done);
        if (done) p.free_q[fs] = slot;
        const uint32_t ss = wf_append(&p.counters[C_SHADOW], shadow);
        if (shadow) {
            p.sh_o[ss] = sh_o;
            p.sh_d[ss] = sh_d;
            p.sh_c[ss] = sh_c;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                p.sh_s[(size_t)ss * 3 + c] = make_float4(S_nee[c][0], S_nee[c][1], S_nee[c][2], S_nee[c][3]);
        }
    }
    warp_count(&s.counters[0], verts);
    warp_count(&s.counters[2], contribs);
}

// unoccluded next-event rays add their Stokes records (warps claim 32 rays at a time)
__global__ void __launch_bounds__(256, 4) k_wf_shadow_pol(const DevScene s, const WfParams p) {
    const uint32_t n = p.counters[C_SHADOW];
    const int lane = threadIdx.x & 31;
    TraceCnt tc{0, 0};
    uint32_t rays = 0, contribs = 0;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&p.counters[C_SH_CUR], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const uint32_t i = base + lane;
        if (i < n) {
            const float4 o = p.sh_o[i], d = p.sh_d[i];
            rays++;
            if (!trace_any<false>(s, make_ray(s, xyz(o), xyz(d)), o.w, tc)) {
                float S[3][4];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 v = p.sh_s[(size_t)i * 3 + c];
                    S[c][0] = v.x;
                    S[c][1] = v.y;
                    S[c][2] = v.z;
                    S[c][3] = v.w;
                }
                wf_splat_stokes(p, (uint32_t)__float_as_int(p.sh_c[i].w), d.w, S);
                contribs++;
            }
        }
    }
    warp_count(&s.counters[3], rays);
    warp_count(&s.counters[2], contribs);
}

// Sort keys of the queued shadow rays: an octahedral cell of the direction
// (2 x MT_SORT_SH_D bits) above the Morton code of the origin on a 2^B per
// axis grid (3 x MT_SORT_SH_B bits); the values are record indices.
__global__ void k_wf_shadow_keys(const DevScene s, const WfParams p) {
    const uint32_t n = p.counters[C_SHADOW];
    constexpr float G = (float)(1 << MT_SORT_SH_B), GD = (float)(1 << MT_SORT_SH_D);
    const float gx = G / (65536.0f * s.q_scale.x), gy = G / (65536.0f * s.q_scale.y),
                gz = G / (65536.0f * s.q_scale.z);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p.P; i += gridDim.x * blockDim.x) {
        uint32_t key = 0xFFFFFFFFu;
        if (i < n) {
            const float4 o = p.sh_o[i], d = p.sh_d[i];
            const uint32_t cx = (uint32_t)fminf(fmaxf((o.x - s.q_lo.x) * gx, 0.0f), G - 1.0f);
            const uint32_t cy = (uint32_t)fminf(fmaxf((o.y - s.q_lo.y) * gy, 0.0f), G - 1.0f);
            const uint32_t cz = (uint32_t)fminf(fmaxf((o.z - s.q_lo.z) * gz, 0.0f), G - 1.0f);
            const float l1 = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
            float u = d.x / l1, v = d.y / l1;
            if (d.z < 0.0f) {
                const float uu = (1.0f - fabsf(v)) * (u < 0.0f ? -1.0f : 1.0f);
                v = (1.0f - fabsf(u)) * (v < 0.0f ? -1.0f : 1.0f);
                u = uu;
            }
            const uint32_t du = (uint32_t)fminf(fmaxf((u + 1.0f) * (0.5f * GD), 0.0f), GD - 1.0f);
            const uint32_t dv = (uint32_t)fminf(fmaxf((v + 1.0f) * (0.5f * GD), 0.0f), GD - 1.0f);
            key = (du << (3 * MT_SORT_SH_B + MT_SORT_SH_D)) | (dv << (3 * MT_SORT_SH_B)) | spread3(cx) |
                  (spread3(cy) << 1) | (spread3(cz) << 2);
        }
        p.sort_keys[i] = key;
        p.sort_q[i] = i;
    }
}

// Extension and shadow rays with dynamic fetch: a lane whose ray is done
// takes the next queue entry as soon as at least p.dynamic_fetch lanes of its
// warp are idle, so a warp does not wait for its longest ray.  Between two
// fetch decisions every busy lane advances MT_WF_STEPS nodes or leaves.
#define MT_WF_STEPS 8

template <bool SHADOW, bool CNT>
__global__ void __launch_bounds__(256) k_wf_trace_dyn(const DevScene s, const WfParams p, const uint32_t *qcur) {
    const uint32_t n = p.counters[SHADOW ? C_SHADOW : C_CUR];
    uint32_t *cursor = &p.counters[SHADOW ? C_SH_CUR : C_EXT_CUR];
    const int lane = threadIdx.x & 31;
    TraceCnt tc{0, 0};
    uint32_t rays = 0, contribs = 0;
    uint2 st[MT_STACK];
    TravState ts;
    RayT r;
    float tmax = INFINITY;
    uint32_t item = 0;
    bool active = false, exhausted = false;
    for (;;) {
        const unsigned idle = __ballot_sync(0xffffffffu, !active);
        if (!exhausted && idle && (__popc(idle) >= p.dynamic_fetch || idle == 0xffffffffu)) {
            const int leader = __ffs(idle) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(cursor, (uint32_t)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (base + __popc(idle) >= n) exhausted = true;
            if (!active) {
                const uint32_t i = base + __popc(idle & ((1u << lane) - 1u));
                if (i < n) {
                    item = SHADOW ? i : qcur[i];
                    float4 o, d;
                    if (SHADOW) {
                        o = p.sh_o[i];
                        d = p.sh_d[i];
                        tmax = o.w;
                    } else {
                        o = p.o[item];
                        d = p.d[item];
                        tmax = INFINITY;
                    }
                    r = make_ray(s, xyz(o), xyz(d));
                    trav_init(ts, tmax);
                    active = true;
                    rays++;
                }
            }
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (exhausted) break;
            continue;
        }
        if (active) {
            for (int k = 0; k < MT_WF_STEPS; ++k) {
                if (trav_step<SHADOW, CNT>(s, r, tmax, ts, st, tc)) {
                    active = false;
                    break;
                }
            }
            if (!active) {
                if (SHADOW) {
                    if (ts.best_k < 0) {  // unoccluded: splat the carried contribution
                        const float4 c = p.sh_c[item];
                        const float4 d = p.sh_d[item];
                        wf_splat(p, (uint32_t)__float_as_int(c.w), d.w, xyz(c));
                        contribs++;
                    }
                } else {
                    p.hit[item] = make_int4(ts.best_k, ts.best_id, __float_as_int(ts.tbest), 0);
                }
            }
        }
    }
    warp_count(&s.counters[3], rays);
    if (SHADOW) warp_count(&s.counters[2], contribs);
    if (CNT) {
        warp_count(&s.counters[4], tc.nodes);
        warp_count(&s.counters[5], tc.tris);
    }
}

// the shading stage at 3 CTAs per SM (80 registers, no spills)
#ifndef MT_WF_SHADE_MINB
#define MT_WF_SHADE_MINB 3
#endif

__device__ __forceinline__ float3 drad_of(const WfParams &p, int em) {
    return p.drad ? f3(p.drad[em * 3], p.drad[em * 3 + 1], p.drad[em * 3 + 2]) : f3(0.f, 0.f, 0.f);
}

// TAN: forward-mode derivative (Sec. 4.4): every contribution C is replaced by
// C * (sum of ratio * dtheta over its vertices) + Cbar * dLe (the film becomes
// the tangent film); the prefix sum of a path lives in p.sig (slot-indexed pool) or
// p.ps_sig (queue-ordered state).
// BWD: path replay (Sec. 4.4): each vertex records the ratio of its
// continuation and the sum of g * C of the contributions made there (light found
// here; the next-event term is added by the shadow stage), paths that end go to
// the finalize queue; radiance gradients are summed per CTA.
template <bool DUMP, bool MEDIA, bool TAN, bool BWD>
__global__ void __launch_bounds__(256, MT_WF_SHADE_MINB) k_wf_shade(const DevScene s, const WfParams p, const uint32_t *qcur,
                                                  uint32_t *qnext) {
    __shared__ float em_acc[BWD ? MT_WF_EM_SMEM * 3 : 1];
    if (BWD) {
        for (int k = threadIdx.x; k < MT_WF_EM_SMEM * 3; k += blockDim.x) em_acc[k] = 0.f;
        __syncthreads();
    }
    const uint32_t n = p.counters[C_CUR];
    uint32_t verts = 0, contribs = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (warp-level appends)
    const uint32_t n_round = ((n + 31u) / 32u) * 32u;
    const bool qord = !BWD && p.qmode;  // queue-ordered state (the replay keeps its records per slot)
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        bool valid = i < n;
        const uint32_t slot = valid && !qord ? qcur[i] : 0u;
        bool cont = false, shadow = false, done = false;
        float4 sh_o = make_float4(0, 0, 0, 0), sh_d = sh_o, sh_c = sh_o, sh_own = sh_o;
        int end = 0;  // BWD: the path's last vertex
        float3 Sv = f3(0.f, 0.f, 0.f), rv = f3(0.f, 0.f, 0.f);  // BWD: record of this vertex
        int rtri = -2;
        uint4 sh_m = make_uint4(0, 0, 0, 0);
        float4 o4 = sh_o, d4 = sh_o, b4 = sh_o;
        uint4 m = sh_m;
        // state of the continuing path, written once its position in the next queue is known
        float4 n_o = sh_o, n_d = sh_o, n_b = sh_o;
        uint4 n_m = sh_m;
        float3 n_sig = f3(0.f, 0.f, 0.f);
        if (valid) {
            int4 h;
            if (qord) {
                o4 = p.ps_o[i];
                d4 = p.ps_d[i];
                b4 = p.ps_b[i];
                m = p.ps_m[i];
                h = p.ps_h[i];
            } else {
                ld_pair<MT_WF_V8_SHADE_LD>(&p.o[slot], &p.d[slot], o4, d4);
                float4 mf;
                ld_pair<MT_WF_V8_SHADE_LD>(&p.beta[slot], (const float4 *)&p.meta[slot], b4, mf);
                m = f4u(mf);
                h = p.hit[slot];
            }
            const uint32_t pix = m.x, smp = m.y;
            const int depth = (int)m.z;
            float opl = o4.w;
            float3 beta = xyz(b4);
            const float3 dir = xyz(d4);
            float3 sig = f3(0.f, 0.f, 0.f);
            if (TAN) sig = xyz(qord ? p.ps_sig[i] : p.sig[slot]);
            end = depth - 1;
            if (MEDIA && h.w) {
                // scattering in the medium: albedo, next-event estimate through the medium
                // (phase function, no MIS; the shadow stage applies the transmittance),
                // Henyey-Greenstein continuation
                verts++;
                rtri = -1;
                end = depth;
                const float th = __int_as_float(h.z);
                const float3 x = xyz(o4) + dir * th;
                if (!(depth == 1 && (p.flags & MT_UNWARP))) opl += th;
                beta = beta * s.m_params[0];
                if (depth == p.max_depth) {
                    done = true;
                } else {
                    if (s.n_units > 0) {
                        const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_NEE), p.k0, p.k1);
                        const int un = pick_unit_wf(s, R.x);
                        const LightUnit U = s.units[un];
                        const int em = __float_as_int(U.v2.w);
                        const bool is_pt = __float_as_int(U.n.w) < 0;
                        const float3 y = is_pt ? xyz(U.v0)
                                               : tri_point(xyz(U.v0), xyz(U.v1), xyz(U.v2), u24(R.y), u24(R.z));
                        const float3 dl = y - x;
                        const float dist = sqrtf(dot(dl, dl));
                        const float3 wi = dl * (1.0f / dist);
                        const float cy = is_pt ? 1.0f : -dot(xyz(U.n), wi);
                        if (cy > 0.f && dist > 0.f) {
                            const float ph = hg_eval(s.m_params[1], dot(dir, wi));
                            const float pick = U.v1.w;
                            const float geo = is_pt ? 1.0f / (dist * dist) / pick : cy / (dist * dist) / (pick / U.v0.w);
                            const float3 cb = beta * (ph * geo * p.scale);
                            float3 c = mul(cb, xyz(s.em_rad[em]));
                            const bool nonzero = c.x != 0.f || c.y != 0.f || c.z != 0.f;
                            if (TAN) {
                                const float dr = p.dmed / s.m_params[0];
                                c = mul(c, sig + f3(dr, dr, dr)) + mul(cb, drad_of(p, em));
                            }
                            if (nonzero) {
                                shadow = true;
                                sh_o = make_float4(x.x, x.y, x.z, dist - (is_pt ? 0.0f : eps_of(y)));
                                sh_d = make_float4(wi.x, wi.y, wi.z,
                                                   opl + dist + pulse_time(s, pix, smp, (uint32_t)depth, 1, p.k0,
                                                                           p.k1));
                                if (BWD) {
                                    const float ia = 1.0f / s.m_params[0];
                                    sh_c = make_float4(cb.x, cb.y, cb.z, __int_as_float((int)pix));
                                    sh_m = make_uint4(smp, (uint32_t)depth, (uint32_t)em, slot);
                                    sh_own = make_float4(ia, ia, ia, 0.f);
                                } else {
                                    sh_c = make_float4(c.x, c.y, c.z, __int_as_float((int)pix));
                                    sh_m = make_uint4(smp, (uint32_t)depth, (uint32_t)__float_as_int(U.n.w), 0u);
                                }
                            }
                        }
                    }
                    const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_SCATTER), p.k0, p.k1);
                    const float3 nd = hg_sample(s.m_params[1], dir, u24(R.x), u24(R.y));
                    if (TAN) {
                        const float dr = p.dmed / s.m_params[0];
                        sig = sig + f3(dr, dr, dr);
                        n_sig = sig;
                    }
                    if (BWD) {
                        const float ia = 1.0f / s.m_params[0];
                        rv = f3(ia, ia, ia);
                    }
                    n_o = make_float4(x.x, x.y, x.z, opl);
                    n_d = make_float4(nd.x, nd.y, nd.z, 0.f);
                    n_b = make_float4(beta.x, beta.y, beta.z, 0.f);
                    n_m = make_uint4(pix, smp, (uint32_t)(depth + 1), 0u);
                    cont = true;
                }
            } else if (h.x < 0) {
                done = true;
            } else {
                verts++;
                rtri = h.y;
                end = depth;
                const int k = h.x, orig = h.y;
                const float th = __int_as_float(h.z);
                const float3 x = xyz(o4) + dir * th;
                if (!(depth == 1 && (p.flags & MT_UNWARP))) opl += th;
                const float4 sn = __ldg(&s.shrec[2 * (size_t)k]);  // normal + light unit
                const float3 ng = xyz(sn);
                const float3 wo = -dir;
                const float cwo = dot(ng, wo);
                const int unit = __float_as_int(sn.w);
                // with a medium, emission found by the path counts only at the camera vertex
                if (unit >= 0 && cwo > 0.f && (!MEDIA || depth == 1)) {
                    const LightUnit U = s.units[unit];
                    float w = 1.0f;
                    if (depth > 1) w = mis2w(d4.w, (U.v1.w / U.v0.w) * th * th / cwo);
                    const int em = __float_as_int(U.v2.w);
                    const float3 cb = beta * (w * p.scale);
                    float3 c = mul(cb, xyz(s.em_rad[em]));
                    if (TAN) c = mul(c, sig) + mul(cb, drad_of(p, em));
                    const float oc = opl + pulse_time(s, pix, smp, (uint32_t)depth, 0, p.k0, p.k1);
                    if (BWD) {
                        const float3 g = wf_grad_at(p, pix, oc);
                        Sv = Sv + mul(g, c);
                        em_grad_add(p, em_acc, s.n_em, em, mul(g, cb));
                    } else {
                        wf_splat(p, pix, oc, c);
                    }
                    contribs++;
                    if (DUMP) wf_dump(p, pix, smp, depth, 0, orig, oc, c);
                }
                if (depth == p.max_depth) {
                    done = true;
                } else {
                    // scattering delay of this vertex: every later contribution carries it
                    opl += vertex_delay(s, orig, pix, smp, (uint32_t)depth, p.k0, p.k1);
                    const float3 nn = cwo >= 0.f ? ng : -ng;
                    float3 tb, bb;
                    onb(nn, tb, bb);
                    const float3 wol = to_local(wo, tb, bb, nn);
                    const float4 mm = __ldg(&s.shrec[2 * (size_t)k + 1]);
                    const Mat mat{xyz(mm), mm.w};
                    // next-event estimate: a shadow ray carrying its contribution
                    if (s.n_units > 0) {
                        const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_NEE), p.k0, p.k1);
                        const int un = pick_unit_wf(s, R.x);
                        const LightUnit U = s.units[un];
                        const int em = __float_as_int(U.v2.w);
                        const bool is_pt = __float_as_int(U.n.w) < 0;
                        const float3 y = is_pt ? xyz(U.v0)
                                               : tri_point(xyz(U.v0), xyz(U.v1), xyz(U.v2), u24(R.y), u24(R.z));
                        const float3 xo = x + nn * eps_of(x);
                        const float3 dl = y - xo;
                        const float dist = sqrtf(dot(dl, dl));
                        const float3 wi = dl * (1.0f / dist);
                        const float cx = dot(nn, wi);
                        const float cy = is_pt ? 1.0f : -dot(xyz(U.n), wi);
                        if (cx > 0.f && cy > 0.f && dist > 0.f) {
                            float3 f;
                            float pb;
                            bsdf_eval(mat, wol, to_local(wi, tb, bb, nn), f, pb);
                            const float pick = U.v1.w;
                            float geo, w = 1.0f;
                            if (is_pt) geo = 1.0f / (dist * dist) / pick;
                            else {
                                const float pA = pick / U.v0.w;
                                geo = cy / (dist * dist) / pA;
                                if (!MEDIA) w = mis2w(pA * dist * dist / cy, pb);
                            }
                            const float3 cb = mul(beta, f) * (cx * geo * w * p.scale);
                            float3 c = mul(cb, xyz(s.em_rad[em]));
                            const bool nonzero = c.x != 0.f || c.y != 0.f || c.z != 0.f;
                            if (TAN) {
                                const float3 dv = p.dalb ? f3(p.dalb[orig * 3], p.dalb[orig * 3 + 1],
                                                              p.dalb[orig * 3 + 2])
                                                         : f3(0.f, 0.f, 0.f);
                                const float3 own = mul(bsdf_dratio(mat, wol, to_local(wi, tb, bb, nn)), dv);
                                c = mul(c, sig + own) + mul(cb, drad_of(p, em));
                            }
                            if (nonzero) {
                                shadow = true;
                                sh_o = make_float4(xo.x, xo.y, xo.z, dist - (is_pt ? 0.0f : eps_of(y)));
                                sh_d = make_float4(wi.x, wi.y, wi.z,
                                                   opl + dist + pulse_time(s, pix, smp, (uint32_t)depth, 1, p.k0,
                                                                           p.k1));
                                if (BWD) {
                                    const float3 own = bsdf_dratio(mat, wol, to_local(wi, tb, bb, nn));
                                    sh_c = make_float4(cb.x, cb.y, cb.z, __int_as_float((int)pix));
                                    sh_m = make_uint4(smp, (uint32_t)depth, (uint32_t)em, slot);
                                    sh_own = make_float4(own.x, own.y, own.z, 0.f);
                                } else {
                                    sh_c = make_float4(c.x, c.y, c.z, __int_as_float((int)pix));
                                    sh_m = make_uint4(smp, (uint32_t)depth, (uint32_t)__float_as_int(U.n.w), 0u);
                                }
                            }
                        }
                    }
                    // continue by sampling the BSDF
                    const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_SCATTER), p.k0, p.k1);
                    float3 wil;
                    if (bsdf_sample(mat, wol, u24(R.x), u24(R.y), wil)) {
                        float3 f;
                        float pb;
                        bsdf_eval(mat, wol, wil, f, pb);
                        if (pb > 0.f) {
                            beta = mul(beta, f) * (wil.z / pb);
                            if (BWD) rv = bsdf_dratio(mat, wol, wil);
                            if (TAN) {
                                const float3 dv = p.dalb ? f3(p.dalb[orig * 3], p.dalb[orig * 3 + 1],
                                                              p.dalb[orig * 3 + 2])
                                                         : f3(0.f, 0.f, 0.f);
                                sig = sig + mul(bsdf_dratio(mat, wol, wil), dv);
                                n_sig = sig;
                            }
                            const float3 no = x + nn * eps_of(x);
                            const float3 nd = to_world(wil, tb, bb, nn);
                            n_o = make_float4(no.x, no.y, no.z, opl);
                            n_d = make_float4(nd.x, nd.y, nd.z, pb);
                            n_b = make_float4(beta.x, beta.y, beta.z, 0.f);
                            n_m = make_uint4(pix, smp, (uint32_t)(depth + 1), 0u);
                            cont = true;
                        }
                    }
                    if (!cont) done = true;
                }
            }
        }
        if (BWD && valid && end >= 1 && end == (int)m.z) {
            // the record of this vertex (the shadow stage adds its next-event term)
            const size_t r = (size_t)m.z * p.P + slot;
            p.rec_a[r] = make_float4(rv.x, rv.y, rv.z, __int_as_float(rtri));
            p.rec_b[r] = make_float4(Sv.x, Sv.y, Sv.z, 0.f);
            p.rec_c[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const uint32_t qs = wf_append(&p.counters[C_NEXT], cont);
        if (cont) {
            if (qord) {
                p.ps_o_n[qs] = n_o;
                p.ps_d_n[qs] = n_d;
                p.ps_b_n[qs] = n_b;
                p.ps_m_n[qs] = n_m;
                if (TAN) p.ps_sig_n[qs] = make_float4(n_sig.x, n_sig.y, n_sig.z, 0.f);
            } else {
                qnext[qs] = slot;
                st_pair<MT_WF_V8_SHADE_ST>(&p.o[slot], &p.d[slot], n_o, n_d);
                st_pair<MT_WF_V8_SHADE_ST>(&p.beta[slot], (float4 *)&p.meta[slot], n_b, u4f(n_m));
                if (TAN) p.sig[slot] = make_float4(n_sig.x, n_sig.y, n_sig.z, 0.f);
            }
        }
        if (!qord) {  // the slot of a finished path returns to the free stack (replay: to the finalize queue)
            const uint32_t fs = wf_append(&p.counters[BWD ? C_FIN : C_FREE], done);
            if (done) {
                if (BWD) {
                    p.fin_q[fs] = slot;
                    p.meta[slot] = make_uint4(m.x, m.y, m.z, (uint32_t)end);
                } else {
                    p.free_q[fs] = slot;
                }
            }
        }
        const uint32_t ss = wf_append(&p.counters[C_SHADOW], shadow);
        if (shadow) {
            p.sh_o[ss] = sh_o;
            p.sh_d[ss] = sh_d;
            p.sh_c[ss] = sh_c;
            if (DUMP || MEDIA || BWD) p.sh_m[ss] = sh_m;  // read only by these forms' shadow stages
            if (BWD) p.sh_cb[ss] = sh_own;
        }
        if (!BWD && p.band_done) {  // streamed output: a finished path counts toward its band of film rows
            const unsigned dm = __ballot_sync(0xffffffffu, done);
            if (done) {
                const uint32_t band = (m.x / (uint32_t)p.W - (uint32_t)p.row0) / p.band_rows;
                const unsigned peers = __match_any_sync(dm, band);
                if ((threadIdx.x & 31) == __ffs(peers) - 1)
                    atomicAdd(&p.band_done[band], (unsigned long long)__popc(peers));
            }
        }
        (void)valid;
    }
    warp_count(&s.counters[0], verts);
    warp_count(&s.counters[2], contribs);
    if (BWD) em_grad_flush(p, em_acc, s.n_em);
}

template <bool DUMP, bool CNT, bool WIDE, bool MEDIA, bool BWD>
__device__ __forceinline__ void sh_rays(const DevScene &s, const WfParams &p, uint32_t n, float *em_acc,
                                        TraceCnt &tc, uint32_t &rays, uint32_t &contribs) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&p.counters[C_SH_CUR], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const uint32_t q = base + lane;
#if MT_HYBRID_SH
        // the warp traverses together (lanes past the queue's end carry no ray)
        const bool live = q < n;
        const uint32_t i = !live ? 0u : (p.sh_perm ? __ldg(&p.sh_perm[q]) : q);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f), d = make_float4(0.f, 0.f, 1.f, 0.f);
        if (live) {
            o = p.sh_o[i];
            d = p.sh_d[i];
        }
        const RayT r = make_ray(s, xyz(o), xyz(d));
        float t_unused;
        int id_unused;
        const bool occluded = WIDE ? (live && trace_wide<true, CNT>(s, r, o.w, t_unused, id_unused, tc) >= 0)
                                   : trace_hybrid<true, CNT>(s, r, live, o.w, t_unused, id_unused, tc) >= 0;
        if (live) {
            rays++;
#else
        if (q < n) {
            const uint32_t i = p.sh_perm ? __ldg(&p.sh_perm[q]) : q;
            const float4 o = p.sh_o[i], d = p.sh_d[i];
            const RayT r = make_ray(s, xyz(o), xyz(d));
            rays++;
            float t_unused;
            int id_unused;
            const bool occluded = WIDE ? trace_wide<true, CNT>(s, r, o.w, t_unused, id_unused, tc) >= 0
                                       : trace_any<CNT>(s, r, o.w, tc);
#endif
            if (!occluded) {
                const float4 c = p.sh_c[i];
                const uint32_t pix = (uint32_t)__float_as_int(c.w);
                float3 cv = xyz(c);
                bool keep = true;
                if (MEDIA) {
                    // ratio-tracking transmittance of the shadow segment (Sec. 4.1)
                    const uint4 m = p.sh_m[i];
                    bool ok;
                    const float Tr = transmittance(s, Rng{p.k0, p.k1}, xyz(o), xyz(d), o.w, pix, m.x, m.y, ok);
                    if (!ok) raise_err(s, MT_EFLAG_TRACK);
                    keep = ok && Tr != 0.f;
                    cv = cv * Tr;
                }
                if (keep && BWD) {
                    // path replay: the next-event contribution of vertex m.y of the path in slot m.w
                    // (the record holds Cbar; C = Cbar * L_e)
                    const uint4 m = p.sh_m[i];
                    const float3 cc = mul(cv, xyz(s.em_rad[m.z]));
                    const float3 g = wf_grad_at(p, pix, d.w);
                    const float3 gc = mul(g, cc);
                    const size_t r = (size_t)m.y * p.P + m.w;
                    const float4 b = p.rec_b[r], c2 = p.rec_c[r];
                    const float3 own = mul(gc, xyz(p.sh_cb[i]));
                    p.rec_b[r] = make_float4(b.x + gc.x, b.y + gc.y, b.z + gc.z, b.w);
                    p.rec_c[r] = make_float4(c2.x + own.x, c2.y + own.y, c2.z + own.z, c2.w);
                    em_grad_add(p, em_acc, s.n_em, (int)m.z, mul(g, cv));
                    contribs++;
                } else if (keep) {
                    wf_splat(p, pix, d.w, cv);
                    contribs++;
                    if (DUMP) {
                        const uint4 m = p.sh_m[i];
                        wf_dump(p, pix, m.x, (int)m.y, 1, (int)m.z, d.w, cv);
                    }
                }
            }
        }
    }
}

// shadow rays of this iteration's shading; n_idx names the counter that holds their number
template <bool DUMP, bool CNT, bool WIDE, bool MEDIA, bool BWD>
__global__ void __launch_bounds__(256, MT_WF_TRACE_MINB) k_wf_shadow(const DevScene s, const WfParams p, int n_idx) {
    __shared__ float em_acc[BWD ? MT_WF_EM_SMEM * 3 : 1];
    if (BWD) {
        for (int k = threadIdx.x; k < MT_WF_EM_SMEM * 3; k += blockDim.x) em_acc[k] = 0.f;
        __syncthreads();
    }
    TraceCnt tc{0, 0};
    uint32_t rays = 0, contribs = 0;
    sh_rays<DUMP, CNT, WIDE, MEDIA, BWD>(s, p, p.counters[n_idx], em_acc, tc, rays, contribs);
    warp_count(&s.counters[3], rays);
    warp_count(&s.counters[2], contribs);
    if (CNT) {
        warp_count(&s.counters[4], tc.nodes);
        warp_count(&s.counters[5], tc.tris);
    }
    if (BWD) em_grad_flush(p, em_acc, s.n_em);
}

// Fused traversal pass: the extension rays of this iteration, then the shadow
// rays that the previous iteration's shading queued (they are independent of
// each other), so that warps that find the extension queue drained trace
// shadow rays instead of idling in the tail of the pass.
template <bool WIDE, bool CNT, bool MEDIA, bool DUMP>
__global__ void __launch_bounds__(256, MT_WF_TRACE_MINB) k_wf_trace(const DevScene s, const WfParams p, const uint32_t *qcur) {
    TraceCnt tc{0, 0};
    uint32_t rays = 0, contribs = 0;
    ext_rays<WIDE, CNT, MEDIA>(s, p, qcur, tc, rays);
    sh_rays<DUMP, CNT, WIDE, MEDIA, false>(s, p, p.counters[C_SH_N], nullptr, tc, rays, contribs);
    warp_count(&s.counters[3], rays);
    warp_count(&s.counters[2], contribs);
    if (CNT) {
        warp_count(&s.counters[4], tc.nodes);
        warp_count(&s.counters[5], tc.tris);
    }
}

// streamed output: flag the bands whose paths have all finished (by the last
// shading pass, whose shadow rays the traversal pass before this one traced)
__global__ void k_wf_bands(const WfParams p, uint32_t iter) {
    for (uint32_t k = threadIdx.x; k < p.n_bands; k += blockDim.x) {
        if (p.band_mark[k]) continue;
        const uint32_t rows = min(p.band_rows, (uint32_t)p.H - k * p.band_rows);
        const unsigned long long need = (unsigned long long)rows * (unsigned long long)p.W * (unsigned long long)p.spp;
        if (p.band_done[k] == need) {
            p.band_mark[k] = 1u;
            *(volatile uint32_t *)&p.band_flag[p.n_bands + k] = iter;  // the flagging iteration, then
            __threadfence_system();
            *(volatile uint32_t *)&p.band_flag[k] = p.done_token;   // this render's token
        }
    }
    __threadfence_system();
}

__global__ void k_wf_init(uint32_t *free_q, uint32_t P, uint32_t *counters, unsigned long long *next_path) {
    if (free_q)  // slot-indexed pool only
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) free_q[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k < MT_WF_COUNTERS; ++k) counters[k] = 0;
        counters[C_FREE] = P;
        *next_path = 0ull;
    }
}

}  // namespace

size_t mt_wf_sort_bytes(uint32_t P) {
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                    (const uint32_t *)nullptr, (uint32_t *)nullptr, (int)P, 0, 32);
    return bytes;
}

mt_status mt_wf_sync_init(WfSync *w) {
    if (w->ready) return MT_OK;
    void *h = nullptr;
    MT_CUDA_TRY(cudaHostAlloc(&h, 64, cudaHostAllocMapped));
    w->done_h = (uint32_t *)h;
    *(volatile uint32_t *)w->done_h = 0u;
    void *d = nullptr;
    MT_CUDA_TRY(cudaHostGetDevicePointer(&d, h, 0));
    w->done_d = (uint32_t *)d;
    for (int i = 0; i < 8; ++i) MT_CUDA_TRY(cudaEventCreateWithFlags(&w->ev[i], cudaEventDisableTiming));
    w->ready = true;
    return MT_OK;
}

void mt_wf_sync_free(WfSync *w) {
    for (int i = 0; i < 8; ++i)
        if (w->ev[i]) cudaEventDestroy(w->ev[i]);
    if (w->done_h) cudaFreeHost(w->done_h);
    *w = WfSync{};
}

void mt_wf_timing_free(WfTiming *t) {
    for (int i = 0; i < t->n_ev; ++i) cudaEventDestroy(t->ev[i]);
    free(t->ev);
    t->ev = nullptr;
    t->n_ev = 0;
}

namespace {

// event k of iteration it (five boundaries per iteration), growing the pool
mt_status wf_event(WfTiming *t, unsigned long long it, int k, cudaStream_t st) {
    const long long idx = (long long)it * 5 + k;
    if (idx >= t->n_ev) {
        const int n = (int)std::max<long long>(idx + 1, 2 * (long long)t->n_ev + 40);
        cudaEvent_t *ev = (cudaEvent_t *)realloc(t->ev, sizeof(cudaEvent_t) * n);
        if (!ev) {
            mt::set_error("stage timing: out of host memory");
            return MT_ERR_OUT_OF_MEMORY;
        }
        t->ev = ev;
        for (int i = t->n_ev; i < n; ++i) {
            if (cudaEventCreate(&t->ev[i]) != cudaSuccess) {
                t->n_ev = i;
                mt::set_error("stage timing: cudaEventCreate failed");
                return MT_ERR_CUDA;
            }
            t->n_ev = i + 1;
        }
    }
    MT_CUDA_TRY(cudaEventRecord(t->ev[idx], st));
    return MT_OK;
}

// add the stage times of iterations [0, n) once the stream has drained
mt_status wf_accumulate(WfTiming *t, unsigned long long n) {
    for (unsigned long long it = 0; it < n; ++it) {
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            MT_CUDA_TRY(cudaEventElapsedTime(&ms, t->ev[it * 5 + k], t->ev[it * 5 + k + 1]));
            t->ms[k] += ms;
        }
    }
    t->iters += (long long)n;
    return MT_OK;
}

}  // namespace

// queue the copies of the bands the host sees flagged (each behind the event of
// the iteration that flagged it, which the event ring still holds), or, with
// all_left, of every band not yet queued behind `last`
static mt_status stream_out_bands(WfStreamOut *out, const WfSync *sync, cudaEvent_t last, bool all_left) {
    for (uint32_t k = 0; k < out->n_bands; ++k) {
        if (out->issued[k]) continue;
        // a band pass of an earlier render still queued writes that render's token, never this one's
        const bool f = *(volatile uint32_t *)&out->flag_h[k] == sync->token;
        if (!f && !all_left) continue;
        const uint32_t it = f ? *(volatile uint32_t *)&out->flag_h[out->n_bands + k] : 0u;
        MT_CUDA_TRY(cudaStreamWaitEvent(out->copy, f ? sync->ev[it & 7u] : last, 0));
        const uint32_t r0 = k * out->band_rows, rows = std::min(out->band_rows, out->H - r0);
        MT_CUDA_TRY(cudaMemcpyAsync((char *)out->h_film + r0 * out->film_row_bytes,
                                    (const char *)out->d_film + r0 * out->film_row_bytes, rows * out->film_row_bytes,
                                    cudaMemcpyDeviceToHost, out->copy));
        if (out->h_steady)
            MT_CUDA_TRY(cudaMemcpyAsync((char *)out->h_steady + r0 * out->steady_row_bytes,
                                        (const char *)out->d_steady + r0 * out->steady_row_bytes,
                                        rows * out->steady_row_bytes, cudaMemcpyDeviceToHost, out->copy));
        out->issued[k] = 1;
    }
    return MT_OK;
}

mt_status mt_launch_wavefront(const DevScene &s, const WfParams &p0, int num_sms, bool dump, bool counters,
                              cudaStream_t st, long long *launches, WfTiming *timing, WfSync *sync,
                              WfStreamOut *out) {
    WfParams p = p0;
    p.done_flag = sync && sync->ready ? sync->done_d : nullptr;
    if (p.done_flag) {
        sync->token = sync->token == 0xFFFFFFFFu ? 1u : sync->token + 1u;  // never 0
        p.done_token = sync->token;
    }
    // streamed output: the forward form in queue order with the fused traversal pass
    const bool streamed = out && p.done_flag && p.qmode && MT_WF_FUSE && !p.bwd && !p.mueller && !dump &&
                          !(p.dynamic_fetch && !s.has_medium);
    if (streamed) {
        for (uint32_t k = 0; k < out->n_bands; ++k) out->issued[k] = 0;
        MT_CUDA_TRY(cudaMemsetAsync(out->band_done, 0, out->n_bands * sizeof(unsigned long long), st));
        MT_CUDA_TRY(cudaMemsetAsync(out->band_mark, 0, out->n_bands * sizeof(uint32_t), st));
        p.band_done = out->band_done;
        p.band_mark = out->band_mark;
        p.band_flag = out->flag_d;
        p.band_rows = out->band_rows;
        p.n_bands = out->n_bands;
        out->used = true;
    }
    const int grid = num_sms * 8;
    k_wf_init<<<std::max(1, std::min(grid, (int)((p.P + 255) / 256))), 256, 0, st>>>(p.qmode ? nullptr : p.free_q, p.P, p.counters,
                                                                                    p.next_path);
    MT_CUDA_TRY(cudaGetLastError());
    uint32_t *qa = p.qa, *qb = p.qb;
    // fused form: trace the shadow rays whose count the last setup moved to C_SH_N
    auto shadow_tail = [&]() -> mt_status {
        const bool media = s.has_medium != 0;
        const bool dyn = p.dynamic_fetch && !dump && !media && !p.bwd;
        const bool wide = p.wide && !media && !p.bwd;
        if (!MT_WF_FUSE || p.bwd || p.mueller || dyn || dump) return MT_OK;
        if (media) {
            if (counters) k_wf_shadow<false, true, false, true, false><<<grid, 256, 0, st>>>(s, p, C_SH_N);
            else k_wf_shadow<false, false, false, true, false><<<grid, 256, 0, st>>>(s, p, C_SH_N);
        } else if (wide) {
            if (counters) k_wf_shadow<false, true, true, false, false><<<grid, 256, 0, st>>>(s, p, C_SH_N);
            else k_wf_shadow<false, false, true, false, false><<<grid, 256, 0, st>>>(s, p, C_SH_N);
        } else {
            if (counters) k_wf_shadow<false, true, false, false, false><<<grid, 256, 0, st>>>(s, p, C_SH_N);
            else k_wf_shadow<false, false, false, false, false><<<grid, 256, 0, st>>>(s, p, C_SH_N);
        }
        MT_CUDA_TRY(cudaGetLastError());
        *launches += 2;
        return MT_OK;
    };
    // an upper bound on iterations: every path needs at most max_depth extension rays
    const unsigned long long bound =
        (p.total_paths + p.P - 1) / p.P * (unsigned long long)(p.max_depth + 1) + (unsigned long long)p.max_depth + 2;
    for (unsigned long long iter = 0; iter < bound; ++iter) {
        if (timing) MT_TRY(wf_event(timing, iter, 0, st));
        k_wf_setup<<<1, 1, 0, st>>>(p, p.iter);
        k_wf_generate<<<grid, 256, 0, st>>>(s, p, p.iter, qa);
        const bool media = s.has_medium != 0;
        const bool dyn = p.dynamic_fetch && !dump && !media && !p.bwd;
        const bool wide = p.wide && !media && !p.bwd;  // the medium and replay forms traverse the binary tree
        // shadow rays traced in the next iteration's extension pass (the replay needs its shadow
        // terms before the finalize stage, polarization and dynamic fetch have kernels of their own)
        const bool fused = MT_WF_FUSE && !p.bwd && !p.mueller && !dyn && !dump;
        const uint32_t *qext = qa;
        if (p.sort_rays && !dump) {
            k_wf_sort_keys<<<grid, 256, 0, st>>>(s, p, qa);
            size_t bytes = p.sort_tmp_bytes;
            MT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(p.sort_tmp, bytes, p.sort_keys, p.sort_keys_out, qa, p.sort_q,
                                                        (int)p.P, 0, MT_SORT_EXT_BITS, st));
            qext = p.sort_q;
            *launches += 1;
        }
        if (timing) MT_TRY(wf_event(timing, iter, 1, st));
        if (dyn) {
            if (counters) k_wf_trace_dyn<false, true><<<grid, 256, 0, st>>>(s, p, qa);
            else k_wf_trace_dyn<false, false><<<grid, 256, 0, st>>>(s, p, qa);
        } else if (fused) {
            if (media) {
                if (counters) k_wf_trace<false, true, true, false><<<grid, 256, 0, st>>>(s, p, qext);
                else k_wf_trace<false, false, true, false><<<grid, 256, 0, st>>>(s, p, qext);
            } else if (wide) {
                if (counters) k_wf_trace<true, true, false, false><<<grid, 256, 0, st>>>(s, p, qext);
                else k_wf_trace<true, false, false, false><<<grid, 256, 0, st>>>(s, p, qext);
            } else {
                if (counters) k_wf_trace<false, true, false, false><<<grid, 256, 0, st>>>(s, p, qext);
                else k_wf_trace<false, false, false, false><<<grid, 256, 0, st>>>(s, p, qext);
            }
        } else if (media) {
            if (counters) k_wf_extend<false, true, true><<<grid, 256, 0, st>>>(s, p, qext);
            else k_wf_extend<false, false, true><<<grid, 256, 0, st>>>(s, p, qext);
        } else if (wide) {
            if (counters) k_wf_extend<true, true, false><<<grid, 256, 0, st>>>(s, p, qext);
            else k_wf_extend<true, false, false><<<grid, 256, 0, st>>>(s, p, qext);
        } else {
            if (counters) k_wf_extend<false, true, false><<<grid, 256, 0, st>>>(s, p, qext);
            else k_wf_extend<false, false, false><<<grid, 256, 0, st>>>(s, p, qext);
        }
        if (streamed) {
            k_wf_bands<<<1, 256, 0, st>>>(p, (uint32_t)iter);
            *launches += 1;
        }
        if (timing) MT_TRY(wf_event(timing, iter, 2, st));
        if (p.mueller) {
            k_wf_shade_pol<<<grid * 2, 128, 0, st>>>(s, p, qa, qb);
        } else if (p.bwd) {
            if (media) k_wf_shade<false, true, false, true><<<grid, 256, 0, st>>>(s, p, qa, qb);
            else k_wf_shade<false, false, false, true><<<grid, 256, 0, st>>>(s, p, qa, qb);
        } else if (p.sig || p.ps_sig) {  // forward-mode derivative
            if (media) k_wf_shade<false, true, true, false><<<grid, 256, 0, st>>>(s, p, qa, qb);
            else k_wf_shade<false, false, true, false><<<grid, 256, 0, st>>>(s, p, qa, qb);
        } else if (media) {
            if (dump) k_wf_shade<true, true, false, false><<<grid, 256, 0, st>>>(s, p, qa, qb);
            else k_wf_shade<false, true, false, false><<<grid, 256, 0, st>>>(s, p, qa, qb);
        } else {
            if (dump) k_wf_shade<true, false, false, false><<<grid, 256, 0, st>>>(s, p, qa, qb);
            else k_wf_shade<false, false, false, false><<<grid, 256, 0, st>>>(s, p, qa, qb);
        }
        if (p.sh_perm) {
            k_wf_shadow_keys<<<grid, 256, 0, st>>>(s, p);
            size_t bytes = p.sort_tmp_bytes;
            MT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(p.sort_tmp, bytes, p.sort_keys, p.sort_keys_out, p.sort_q,
                                                        p.sh_perm, (int)p.P, 0, MT_SORT_SH_BITS, st));
            *launches += 1;
        }
        if (timing) MT_TRY(wf_event(timing, iter, 3, st));
        if (fused) {
            // traced by the next iteration's extension pass
        } else if (p.mueller) {
            k_wf_shadow_pol<<<grid, 256, 0, st>>>(s, p);
        } else if (p.bwd) {
            if (media) {
                if (counters) k_wf_shadow<false, true, false, true, true><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
                else k_wf_shadow<false, false, false, true, true><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            } else {
                if (counters) k_wf_shadow<false, true, false, false, true><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
                else k_wf_shadow<false, false, false, false, true><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            }
            k_wf_finalize<<<grid, 256, s.n_tris <= MT_FIN_SMEM_TRIS ? 3 * (size_t)s.n_tris * sizeof(float) : 0, st>>>(s, p);
            *launches += 1;
        } else if (dyn) {
            if (counters) k_wf_trace_dyn<true, true><<<grid, 256, 0, st>>>(s, p, qa);
            else k_wf_trace_dyn<true, false><<<grid, 256, 0, st>>>(s, p, qa);
        } else if (media) {
            if (dump) {
                if (counters) k_wf_shadow<true, true, false, true, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
                else k_wf_shadow<true, false, false, true, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            } else {
                if (counters) k_wf_shadow<false, true, false, true, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
                else k_wf_shadow<false, false, false, true, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            }
        } else if (wide) {
            if (dump) {
                if (counters) k_wf_shadow<true, true, true, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
                else k_wf_shadow<true, false, true, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            } else {
                if (counters) k_wf_shadow<false, true, true, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
                else k_wf_shadow<false, false, true, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            }
        } else if (dump) {
            if (counters) k_wf_shadow<true, true, false, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            else k_wf_shadow<true, false, false, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
        } else {
            if (counters) k_wf_shadow<false, true, false, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
            else k_wf_shadow<false, false, false, false, false><<<grid, 256, 0, st>>>(s, p, C_SHADOW);
        }
        MT_CUDA_TRY(cudaGetLastError());
        if (timing) MT_TRY(wf_event(timing, iter, 4, st));
        *launches += fused ? 4 : 5;
        uint32_t *t = qa;
        qa = qb;
        qb = t;
        if (p.qmode) {  // the next iteration reads the state shading wrote
            std::swap(p.ps_o, p.ps_o_n);
            std::swap(p.ps_d, p.ps_d_n);
            std::swap(p.ps_b, p.ps_b_n);
            std::swap(p.ps_m, p.ps_m_n);
            std::swap(p.ps_sig, p.ps_sig_n);
        }
        // check for completion: with the mapped flag every second iteration, on the event of the
        // iteration two back (the drained state persists, so a later iteration's flag is as good),
        // which leaves two iterations queued and at most three empty ones at the end; else every
        // fourth, with one small read-back that drains the stream
        if (p.done_flag) MT_CUDA_TRY(cudaEventRecord(sync->ev[iter & 7], st));
        if ((p.done_flag ? (iter & 1) == 1 : (iter & 3) == 3) || iter + 1 == bound) {
            uint32_t done = 0;
            if (p.done_flag && iter >= 2) {
                MT_CUDA_TRY(cudaEventSynchronize(sync->ev[(iter - 2) & 7]));
                done = *(volatile uint32_t *)sync->done_h == p.done_token ? 1u : 0u;
                if (streamed) MT_TRY(stream_out_bands(out, sync, nullptr, false));
            } else {
                MT_CUDA_TRY(cudaMemcpyAsync(&done, p.counters + C_DONE, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
                MT_CUDA_TRY(cudaStreamSynchronize(st));
            }
            if (done) {
                // shadow rays of the last shading pass (none once the queues have drained, but the
                // fused form never leaves queued rays behind)
                k_wf_setup<<<1, 1, 0, st>>>(p, p.iter);
                MT_TRY(shadow_tail());
                if (streamed) {  // the bands not flagged yet, behind the last stage
                    MT_CUDA_TRY(cudaEventRecord(sync->ev[(iter + 1) & 7], st));
                    MT_TRY(stream_out_bands(out, sync, sync->ev[(iter + 1) & 7], true));
                }
                if (!timing) return MT_OK;
                MT_CUDA_TRY(cudaStreamSynchronize(st));  // the stage events of every iteration have completed
                return wf_accumulate(timing, iter + 1);
            }
        }
    }
    if (timing) {
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        MT_TRY(wf_accumulate(timing, bound));
    }
    // one more setup decides whether anything is left
    k_wf_setup<<<1, 1, 0, st>>>(p, p.iter);
    *launches += 1;
    MT_TRY(shadow_tail());
    if (streamed) {
        MT_CUDA_TRY(cudaEventRecord(sync->ev[bound & 7], st));
        MT_TRY(stream_out_bands(out, sync, sync->ev[bound & 7], true));
    }
    uint32_t done = 0;
    MT_CUDA_TRY(cudaMemcpyAsync(&done, p.counters + C_DONE, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    if (!done) {
        mt::set_error("wavefront render did not drain its queues within the iteration bound");
        return MT_ERR_INTERNAL;
    }
    return MT_OK;
}
