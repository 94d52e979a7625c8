// mt_render.cu -- persistent transient path-tracing megakernel.
//
// One launch renders a whole (H, W, T) film (arXiv 2510.25660 Sec. 3):
//   * CTAs pull pixel tiles from a global counter; a tile is tile_px
//     consecutive pixels of one row, so its film rows are one contiguous span.
//   * The tile's time histograms live in shared memory (bins [0, D) of every
//     pixel; bins >= D go straight to global memory with red.add) and are
//     written to HBM once per tile with coalesced stores (path reuse:
//     every contribution lands in the bin of its own optical path length).
//   * Warps keep all 32 lanes busy: a lane whose path ended takes the next
//     path of the tile (warp-aggregated claim on a shared counter), so every
//     loop iteration advances 32 paths by one vertex.
//   * Each vertex traces an extension ray (closest hit) and a shadow ray (any
//     hit) for next-event estimation with power-heuristic MIS; in a medium
//     (Sec. 4.1) free flights use delta tracking and shadow rays ratio
//     tracking, and their lengths add to the optical path length.
//   * MODE_BWD replays the same paths from their Philox keys (Sec. 4.4,
//     path replay): contributions gather dL/dfilm from the tile (staged in
//     shared memory), per-vertex sums are kept in local memory and the
//     per-triangle albedo gradients are scattered once per vertex at path end.
#include "mt_common.cuh"
#include "mt_internal.h"
#include "mt_launch.h"
#include "mt_trace.cuh"

namespace {

constexpr int MODE_FWD = 0, MODE_DUMP = 1, MODE_BWD = 2, MODE_PHASOR = 3, MODE_TAN = 4;

// CTAs of 256 threads the register allocation must leave room for per SM: 4
// (64 registers) measured fastest on GB300 for the large scene (205 ms against
// 227 ms at 2), the extra warps hiding more gather latency than the spills cost
#ifndef MT_RENDER_MINB
#define MT_RENDER_MINB 4
#endif
// with a participating medium the free-flight and ratio-tracking loops need
// more registers: 2 CTAs per SM (128 registers) measured 479 ms against 553 ms
// at 4 for the 256x256x128-spp, depth-16 render of the medium-filled box
#ifndef MT_RENDER_MINB_MEDIA
#define MT_RENDER_MINB_MEDIA 2
#endif
// the path replay keeps per-vertex records
#ifndef MT_RENDER_MINB_BWD
#define MT_RENDER_MINB_BWD 4
#endif
#define MT_MINB_OF(MODE, MEDIA) ((MEDIA) ? MT_RENDER_MINB_MEDIA : ((MODE) == MODE_BWD ? MT_RENDER_MINB_BWD : MT_RENDER_MINB))

struct VRec {
    int32_t tri;   // original triangle index, -1 for a medium vertex
    float3 r;      // d(factor)/factor of the continuation
    float3 S;      // sum of g*C of contributions attached to this vertex
    float3 own;    // own-direction gradient term of this vertex's next-event estimate
};

struct PathState {
    float3 o, d, beta;
    float opl, prev_pdf;
    int depth, lp;
    uint32_t pix, smp;
    float3 acc;     // steady-image sum of this path (forward)
    float3 sig;     // forward-mode derivative: sum over earlier vertices of ratio * dtheta
    float3 dv;      // forward-mode derivative: dtheta of the current vertex
};

struct Counters {
    uint32_t vertices = 0, paths = 0, contribs = 0, rays = 0, smem_splats = 0, gmem_splats = 0;
    TraceCnt tc{0, 0};
};

__device__ __forceinline__ float mis2(float a, float b) { return a * a / (a * a + b * b); }

__device__ __forceinline__ int pick_unit(const DevScene &s, uint32_t u) {
    int lo = 0, hi = s.n_units - 1;
    const uint32_t key = u >> 8;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key < __ldg(&s.unit_cdf[mid])) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <int MODE, bool MEDIA, bool CNT, bool AGG>
struct Tracer {
    const DevScene &s;
    const RenderParams &p;
    float *hist, *steady_s, *em_acc;
    float &med_acc;
    Counters &cnt;
    VRec *vr;  // backward only
    Rng rng;

    // one contribution c (cb = c without radiance) of emitter em at OPL opl;
    // kind 0 = found by the path at vertex `vert`, kind 1 = next-event at `vert`
    __device__ __forceinline__ void deposit(PathState &ps, int vert, int kind, int tri, float opl, float3 c,
                                            float3 cb, int em, float3 own_r) {
        // the source emitted this contribution's light at a time drawn from its pulse
        opl += pulse_time(s, gp(ps), ps.smp, (uint32_t)vert, kind, rng.k0, rng.k1);
        const float x = (opl - p.start) / p.width;
        const bool in = x >= 0.f && x < (float)p.T;
        const int bin = in ? (int)x : -1;
        c = c * p.scale;
        cb = cb * p.scale;
        cnt.contribs++;
        if (MODE == MODE_TAN) {
            // forward-mode derivative (Sec. 4.4): dC = C * (sum of ratio * dtheta over the
            // vertices, the next-event's own term included) + Cbar * dLe; splatted like C
            float3 dc = mul(c, ps.sig + own_r);
            if (p.drad) dc = dc + mul(cb, f3(p.drad[em * 3], p.drad[em * 3 + 1], p.drad[em * 3 + 2]));
            c = dc;
        }
        if (MODE == MODE_PHASOR) {
            // frequency space (Sec. 4.3, Eq. 12): C exp(-i 2 pi opl / lambda) per wavelength;
            // "bin" 2q holds the real part, 2q + 1 the imaginary part
            for (int q = 0; q < p.K; ++q) {
                float sn, cs;
                sincospif(2.0f * opl / __ldg(&p.lambdas[q]), &sn, &cs);
                const float re[3] = {c.x * cs, c.y * cs, c.z * cs};
                const float im[3] = {-c.x * sn, -c.y * sn, -c.z * sn};
                if (2 * q + 1 < p.D) {
                    splat_add<3, AGG>(hist + ((size_t)ps.lp * p.D + 2 * q) * 3, re);
                    splat_add<3, AGG>(hist + ((size_t)ps.lp * p.D + 2 * q + 1) * 3, im);
                } else {
                    splat_add<3, AGG>(p.film + ((size_t)ps.pix * p.T + 2 * q) * 3, re);
                    splat_add<3, AGG>(p.film + ((size_t)ps.pix * p.T + 2 * q + 1) * 3, im);
                }
            }
            ps.acc = ps.acc + c;
            (void)in;
            (void)bin;
        } else if (MODE != MODE_BWD) {
            if (in) {
                const float cv[3] = {c.x, c.y, c.z};
                if (bin < p.D) {
                    splat_add<3, AGG>(hist + ((size_t)ps.lp * p.D + bin) * 3, cv);
                    cnt.smem_splats++;
                } else {
                    splat_add<3, AGG>(p.film + ((size_t)ps.pix * p.T + bin) * 3, cv);
                    cnt.gmem_splats++;
                }
            }
            ps.acc = ps.acc + c;
            if (MODE == MODE_DUMP) {
                const unsigned long long slot = atomicAdd(p.dump_count, 1ull);
                if ((long long)slot < p.dump_cap) {
                    mt_contrib r;
                    r.pixel = (int32_t)gp(ps);
                    r.sample = (int32_t)ps.smp;
                    r.depth = vert;
                    r.kind = kind;
                    r.tri = tri;
                    r.bin = in ? bin : (int)floorf(x);
                    r.opl = opl;
                    r.c[0] = c.x / p.scale;
                    r.c[1] = c.y / p.scale;
                    r.c[2] = c.z / p.scale;
                    p.dump[slot] = r;
                }
            }
        } else {
            float3 g = f3(steady_s[ps.lp * 3], steady_s[ps.lp * 3 + 1], steady_s[ps.lp * 3 + 2]);
            if (in) {
                const float *h = bin < p.D ? hist + ((size_t)ps.lp * p.D + bin) * 3
                                           : p.gfilm + ((size_t)ps.pix * p.T + bin) * 3;
                g = g + f3(h[0], h[1], h[2]);
            }
            const float3 gc = mul(g, c);
            VRec &v = vr[vert];
            if (kind == 0) v.S = v.S + gc;
            else {
                v.S = v.S + gc;
                v.own = v.own + mul(gc, own_r);
            }
            const float3 gr = mul(g, cb);
            if (p.n_em_smem > 0) {
                atomicAdd(&em_acc[em * 3], gr.x);
                atomicAdd(&em_acc[em * 3 + 1], gr.y);
                atomicAdd(&em_acc[em * 3 + 2], gr.z);
            } else {
                atomicAdd(&p.grad[em * 3], gr.x);
                atomicAdd(&p.grad[em * 3 + 1], gr.y);
                atomicAdd(&p.grad[em * 3 + 2], gr.z);
            }
        }
    }

    // frame pixel id of the path (Philox counters, dump records); ps.pix indexes the film
    __device__ __forceinline__ uint32_t gp(const PathState &ps) const { return ps.pix + p.pix_base; }

    __device__ __forceinline__ void begin(PathState &ps, int j, int pix0, int x0, int ty) {
        ps.lp = j / p.spp;
        const int sI = j - ps.lp * p.spp;
        ps.pix = (uint32_t)(pix0 + ps.lp);
        ps.smp = p.sample_offset + (uint32_t)sI;
        const uint4 R = rng.raw(gp(ps), ps.smp, 0, 0);
        const bool center = p.flags & MT_PIXEL_CENTER;
        const float jx = center ? 0.5f : u24(R.x), jy = center ? 0.5f : u24(R.y);
        const int px = x0 + ps.lp;
        const float sx = (2.0f * ((float)px + jx) / (float)p.W - 1.0f) * s.tan_half;
        const float sy =
            (1.0f - 2.0f * ((float)(ty + p.row0) + jy) / (float)p.H_full) * s.tan_half * ((float)p.H_full / (float)p.W);
        ps.o = s.cam_o;
        ps.d = normalize(s.cam_f + s.cam_r * sx + s.cam_u * sy);
        ps.beta = f3(1.f, 1.f, 1.f);
        ps.opl = 0.f;
        ps.prev_pdf = 0.f;
        ps.depth = 1;
        ps.acc = f3(0.f, 0.f, 0.f);
        ps.sig = f3(0.f, 0.f, 0.f);
        ps.dv = f3(0.f, 0.f, 0.f);
        cnt.paths++;
        if (MODE == MODE_BWD) vr[0].tri = -2;
    }

    __device__ __forceinline__ void end(PathState &ps) {
        if (MODE != MODE_BWD) {
            if (ps.acc.x != 0.f || ps.acc.y != 0.f || ps.acc.z != 0.f) {
                atomicAdd(&steady_s[ps.lp * 3], ps.acc.x);
                atomicAdd(&steady_s[ps.lp * 3 + 1], ps.acc.y);
                atomicAdd(&steady_s[ps.lp * 3 + 2], ps.acc.z);
            }
        } else {
            // suffix sums: vertex i receives the contributions of later vertices
            float3 P = f3(0.f, 0.f, 0.f);
            for (int i = ps.depth; i >= 1; --i) {
                const VRec &v = vr[i];
                if (v.tri == -2) continue;
                const float3 gi = mul(P, v.r) + v.own;
                if (v.tri >= 0) {
                    if (gi.x != 0.f || gi.y != 0.f || gi.z != 0.f) {
                        float *g = p.galb + (size_t)v.tri * 3;
                        atomicAdd(g, gi.x);
                        atomicAdd(g + 1, gi.y);
                        atomicAdd(g + 2, gi.z);
                    }
                } else {
                    med_acc_add(gi.x + gi.y + gi.z);
                }
                P = P + v.S;
            }
        }
    }

    __device__ __forceinline__ void med_acc_add(float v) {
        if (v != 0.f) atomicAdd(&med_acc, v);
    }

    __device__ __forceinline__ void reset_vertex(int i) {
        if (MODE == MODE_BWD) {
            vr[i].tri = -2;
            vr[i].r = f3(0.f, 0.f, 0.f);
            vr[i].S = f3(0.f, 0.f, 0.f);
            vr[i].own = f3(0.f, 0.f, 0.f);
        }
    }

    // next-event estimate from x (surface: side normal n and frame, or medium)
    __device__ __forceinline__ void nee(PathState &ps, float3 x, bool surface, float3 n, float3 tb, float3 bb,
                                        float3 wol, const Mat &m) {
        const uint4 R = rng.raw(gp(ps), ps.smp, (uint32_t)ps.depth, G_NEE);
        const int un = pick_unit(s, R.x);
        const LightUnit U = s.units[un];
        const int em = __float_as_int(U.v2.w);
        const bool is_pt = __float_as_int(U.n.w) < 0;
        const float3 y = is_pt ? xyz(U.v0) : tri_point(xyz(U.v0), xyz(U.v1), xyz(U.v2), u24(R.y), u24(R.z));
        const float3 xo = surface ? x + n * eps_of(x) : x;
        const float3 dl = y - xo;
        const float dist = sqrtf(dot(dl, dl));
        const float3 wi = dl * (1.0f / dist);
        const float cx = surface ? dot(n, wi) : 1.0f;
        const float cy = is_pt ? 1.0f : -dot(xyz(U.n), wi);
        if (!(cx > 0.f && cy > 0.f && dist > 0.f)) return;
        const float tmax = dist - (is_pt ? 0.0f : eps_of(y));
        cnt.rays++;
        const RayT sr = make_ray(s, xo, wi);
        if (trace_any<CNT>(s, sr, tmax, cnt.tc)) return;
        float Tr = 1.0f;
        if (MEDIA) {
            bool ok;
            Tr = transmittance(s, rng, xo, wi, tmax, gp(ps), ps.smp, (uint32_t)ps.depth, ok);
            if (!ok) {
                raise_err(s, MT_EFLAG_TRACK);
                return;
            }
            if (Tr == 0.f) return;
        }
        const float pick = U.v1.w;
        float3 fc;
        float3 own = f3(0.f, 0.f, 0.f);
        float w = 1.0f, geo;
        if (surface) {
            const float3 wil = to_local(wi, tb, bb, n);
            float pb;
            bsdf_eval(m, wol, wil, fc, pb);
            fc = fc * cx;
            if (is_pt) geo = 1.0f / (dist * dist) / pick;
            else {
                const float pA = pick / U.v0.w;
                geo = cy / (dist * dist) / pA;
                if (!MEDIA) w = mis2(pA * dist * dist / cy, pb);
            }
            if (MODE == MODE_BWD) own = bsdf_dratio(m, wol, wil);
            if (MODE == MODE_TAN) own = mul(bsdf_dratio(m, wol, wil), ps.dv);
        } else {
            const float ph = hg_eval(s.m_params[1], dot(ps.d, wi));
            fc = f3(ph, ph, ph);
            geo = is_pt ? 1.0f / (dist * dist) / pick : cy / (dist * dist) / (pick / U.v0.w);
            if (MODE == MODE_BWD) {
                const float ia = 1.0f / s.m_params[0];
                own = f3(ia, ia, ia);
            }
            if (MODE == MODE_TAN) own = ps.dv;  // (1 / albedo) * dalbedo, set at the vertex
        }
        const float k = geo * w * Tr;
        const float3 cb = mul(ps.beta, fc) * k;
        const float4 Le = s.em_rad[em];
        const float3 c = mul(cb, xyz(Le));
        if (c.x == 0.f && c.y == 0.f && c.z == 0.f) return;
        deposit(ps, ps.depth, 1, __float_as_int(U.n.w), ps.opl + dist, c, cb, em, own);
    }

    // advance the path by one vertex; returns false when it ends
    __device__ bool step(PathState &ps) {
        if (MODE == MODE_BWD) reset_vertex(ps.depth);
        const RayT r = make_ray(s, ps.o, ps.d);
        float th;
        int orig;
        cnt.rays++;
        const int k = trace_closest<CNT>(s, r, INFINITY, th, orig, cnt.tc);
        if (MEDIA) {
            float ma, mb;
            const float tsurf = k >= 0 ? th : 1e30f;
            if (medium_span(s, ps.o, ps.d, tsurf, ma, mb)) {
                float t = ma;
                bool collided = false;
                const float inv = 1.0f / s.m_major;
                for (uint32_t j = 0;; ++j) {
                    if (j >= MT_TRACK_STEPS) {
                        raise_err(s, MT_EFLAG_TRACK);
                        return false;
                    }
                    const uint4 R = rng.raw(gp(ps), ps.smp, (uint32_t)(ps.depth - 1), G_TRACK + j);
                    t += -logf(1.0f - u24(R.x)) * inv;
                    if (t >= mb) break;
                    if (u24(R.y) < density_at(s, ps.o + ps.d * t) * inv) {
                        collided = true;
                        break;
                    }
                }
                if (collided) {
                    cnt.vertices++;
                    const float3 x = ps.o + ps.d * t;
                    if (!(ps.depth == 1 && (p.flags & MT_UNWARP))) ps.opl += t;
                    const float alb = s.m_params[0];
                    ps.beta = ps.beta * alb;
                    if (MODE == MODE_BWD) {
                        vr[ps.depth].tri = -1;
                        const float ia = 1.0f / alb;
                        vr[ps.depth].r = f3(ia, ia, ia);
                    }
                    if (MODE == MODE_TAN) {
                        const float dr = p.dmed / alb;
                        ps.dv = f3(dr, dr, dr);
                    }
                    if (ps.depth == p.max_depth) return false;
                    if (s.n_units > 0) nee(ps, x, false, f3(0, 0, 1), f3(1, 0, 0), f3(0, 1, 0), f3(0, 0, 1), Mat{});
                    const uint4 R = rng.raw(gp(ps), ps.smp, (uint32_t)ps.depth, G_SCATTER);
                    ps.d = hg_sample(s.m_params[1], ps.d, u24(R.x), u24(R.y));
                    if (MODE == MODE_TAN) ps.sig = ps.sig + ps.dv;
                    ps.o = x;
                    ps.depth++;
                    return true;
                }
            }
        }
        if (k < 0) return false;
        cnt.vertices++;
        const float3 x = ps.o + ps.d * th;
        if (!(ps.depth == 1 && (p.flags & MT_UNWARP))) ps.opl += th;
        const float4 p0 = ldg_keep(&s.tris[3 * k]), p1 = ldg_keep(&s.tris[3 * k + 1]), p2 = ldg_keep(&s.tris[3 * k + 2]);
        const float3 ng = normalize(cross(xyz(p1) - xyz(p0), xyz(p2) - xyz(p0)));
        const float3 wo = -ps.d;
        const float cwo = dot(ng, wo);
        const int unit = __ldg(&s.tri_unit[orig]);
        // the vertex is recorded before anything can end the path here, so that light
        // found at the last vertex still reaches the earlier vertices' gradients
        if (MODE == MODE_BWD) vr[ps.depth].tri = orig;
        if (unit >= 0 && cwo > 0.f && (ps.depth == 1 || !MEDIA)) {
            const LightUnit U = s.units[unit];
            float w = 1.0f;
            if (ps.depth > 1) {
                const float pl = (U.v1.w / U.v0.w) * th * th / cwo;
                w = mis2(ps.prev_pdf, pl);
            }
            const int em = __float_as_int(U.v2.w);
            const float3 cb = ps.beta * w;
            const float3 c = mul(cb, xyz(s.em_rad[em]));
            deposit(ps, ps.depth, 0, orig, ps.opl, c, cb, em, f3(0.f, 0.f, 0.f));
        }
        if (ps.depth == p.max_depth) return false;
        // scattering delay of this vertex: every later contribution carries it
        ps.opl += vertex_delay(s, orig, gp(ps), ps.smp, (uint32_t)ps.depth, rng.k0, rng.k1);
        const float3 n = cwo >= 0.f ? ng : -ng;
        float3 tb, bb;
        onb(n, tb, bb);
        const float3 wol = to_local(wo, tb, bb, n);
        const float4 mm = __ldg(&s.mats[orig]);
        const Mat m{xyz(mm), mm.w};
        if (MODE == MODE_TAN)
            ps.dv = p.dalb ? f3(p.dalb[orig * 3], p.dalb[orig * 3 + 1], p.dalb[orig * 3 + 2]) : f3(0.f, 0.f, 0.f);
        if (s.n_units > 0) nee(ps, x, true, n, tb, bb, wol, m);
        const uint4 R = rng.raw(gp(ps), ps.smp, (uint32_t)ps.depth, G_SCATTER);
        float3 wil;
        if (!bsdf_sample(m, wol, u24(R.x), u24(R.y), wil)) return false;
        float3 f;
        float pb;
        bsdf_eval(m, wol, wil, f, pb);
        if (!(pb > 0.f)) return false;
        ps.beta = mul(ps.beta, f) * (wil.z / pb);
        if (MODE == MODE_BWD) vr[ps.depth].r = bsdf_dratio(m, wol, wil);
        if (MODE == MODE_TAN) ps.sig = ps.sig + mul(bsdf_dratio(m, wol, wil), ps.dv);
        ps.prev_pdf = pb;
        ps.o = x + n * eps_of(x);
        ps.d = to_world(wil, tb, bb, n);
        ps.depth++;
        return true;
    }
};

template <int MODE, bool MEDIA, bool CNT, bool AGG>
__global__ void __launch_bounds__(256, MT_MINB_OF(MODE, MEDIA)) k_render(const DevScene s, const RenderParams p) {
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // each warp owns a slice: its tile's histograms (tile_px x D x 3) and steady sums (tile_px x 3)
    const int slice = p.tile_px * (p.D * 3 + 3);
    float *hist = smem + (size_t)warp * slice;
    float *steady_s = hist + p.tile_px * p.D * 3;
    float *em_acc = smem + (size_t)nwarps * slice;  // shared by the CTA (backward)
    __shared__ float s_med;
    Counters cnt;
    VRec vrec[MODE == MODE_BWD ? MT_MAX_BWD_DEPTH + 1 : 1];
    if (MODE == MODE_BWD) {
        for (int i = threadIdx.x; i < p.n_em_smem * 3; i += blockDim.x) em_acc[i] = 0.f;
        if (threadIdx.x == 0) s_med = 0.f;
        __syncthreads();
    }
    Tracer<MODE, MEDIA, CNT, AGG> tr{s, p, hist, steady_s, em_acc, s_med, cnt, vrec, Rng{p.k0, p.k1}};
    for (;;) {
        // the warp claims its next tile
        int tile = 0;
        if (lane == 0) tile = atomicAdd(p.tile_counter, 1);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= p.n_tiles) break;
        const int ty = tile / p.tiles_per_row, tx = tile - ty * p.tiles_per_row;
        const int x0 = tx * p.tile_px;
        const int npx = min(p.tile_px, p.W - x0);
        const int pix0 = ty * p.W + x0;
        // stage the tile: zero the histograms, or load dL/dfilm for replay
        if (MODE != MODE_BWD) {
            for (int i = lane; i < slice; i += 32) hist[i] = 0.f;
        } else {
            for (int i = lane; i < npx * p.D * 3; i += 32) {
                const int lp = i / (p.D * 3), r = i - lp * p.D * 3;
                hist[i] = __ldg(&p.gfilm[((size_t)(pix0 + lp) * p.T) * 3 + r]);
            }
            for (int i = lane; i < p.tile_px * 3; i += 32)
                steady_s[i] = (p.gsteady && i < npx * 3) ? __ldg(&p.gsteady[(size_t)pix0 * 3 + i]) : 0.f;
        }
        __syncwarp();
        // paths of the tile; a lane whose path ended takes the next one
        const int n_paths = npx * p.spp;
        int next = 0;
        PathState ps;
        bool active = false;
        for (;;) {
            if (next < n_paths) {
                const unsigned need = __ballot_sync(0xffffffffu, !active);
                if (__popc(need) >= p.refill_min || need == 0xffffffffu) {
                    if (!active) {
                        const int j = next + __popc(need & ((1u << lane) - 1u));
                        if (j < n_paths) {
                            tr.begin(ps, j, pix0, x0, ty);
                            active = true;
                        }
                    }
                    next += __popc(need);
                }
            }
            if (!__any_sync(0xffffffffu, active)) break;
            if (active) {
                if (!tr.step(ps)) {
                    tr.end(ps);
                    active = false;
                }
            }
        }
        __syncwarp();
        if (MODE != MODE_BWD) {
            // write the tile: bins < D of every pixel, then the steady image
            const bool acc = p.flags & MT_ACCUMULATE;
            if (p.D == p.T) {
                const size_t n = (size_t)npx * p.T * 3;
                float *dst = p.film + (size_t)pix0 * p.T * 3;
                if (((n | (size_t)pix0 * p.T * 3 | (size_t)slice) & 3) == 0 && (((uintptr_t)p.film) & 15) == 0) {
                    float4 *d4 = reinterpret_cast<float4 *>(dst);
                    const float4 *s4 = reinterpret_cast<const float4 *>(hist);
                    for (size_t i = lane; i < n / 4; i += 32) {
                        float4 v = s4[i];
                        if (acc) {
                            const float4 o = d4[i];
                            v = make_float4(v.x + o.x, v.y + o.y, v.z + o.z, v.w + o.w);
                        }
                        d4[i] = v;
                    }
                } else {
                    for (size_t i = lane; i < n; i += 32) dst[i] = acc ? dst[i] + hist[i] : hist[i];
                }
            } else if (p.D > 0) {
                const int row = p.D * 3;
                for (int i = lane; i < npx * row; i += 32) {
                    const int lp = i / row, r = i - lp * row;
                    float *d = p.film + (size_t)(pix0 + lp) * p.T * 3 + r;
                    *d = acc ? *d + hist[i] : hist[i];
                }
            }
            if (p.steady)
                for (int i = lane; i < npx * 3; i += 32) {
                    float *d = p.steady + (size_t)pix0 * 3 + i;
                    *d = acc ? *d + steady_s[i] : steady_s[i];
                }
        }
        __syncwarp();
    }
    if (MODE == MODE_BWD) {
        __syncthreads();
        for (int i = threadIdx.x; i < p.n_em_smem * 3; i += blockDim.x)
            if (em_acc[i] != 0.f) atomicAdd(&p.grad[i], em_acc[i]);
        if (threadIdx.x == 0 && p.gmed && s_med != 0.f) atomicAdd(p.gmed, s_med);
    }
    // counters: one atomic per warp and counter
    unsigned long long v[8] = {cnt.vertices, cnt.paths, cnt.contribs, cnt.rays, cnt.tc.nodes, cnt.tc.tris,
                               cnt.smem_splats, cnt.gmem_splats};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        unsigned long long x = v[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(&s.counters[c], x);
    }
}

template <int MODE, bool MEDIA, bool CNT, bool AGG>
mt_status launch_one(const DevScene &s, const RenderParams &p, const LaunchCfg &cfg, cudaStream_t st) {
    auto kern = k_render<MODE, MEDIA, CNT, AGG>;
    const size_t smem = cfg.smem_bytes;
    MT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    MT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.threads, smem));
    if (per_sm < 1) {
        mt::set_error("render kernel does not fit: %d threads, %zu bytes of shared memory", cfg.threads, smem);
        return MT_ERR_UNSUPPORTED;
    }
    if (cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, cfg.ctas_per_sm);
    const int warps = cfg.threads / 32;
    const int grid = std::max(1, std::min((p.n_tiles + warps - 1) / warps, per_sm * cfg.num_sms));
    kern<<<grid, cfg.threads, smem, st>>>(s, p);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

template <int MODE, bool MEDIA, bool CNT>
mt_status launch_agg(const DevScene &s, const RenderParams &p, const LaunchCfg &cfg, cudaStream_t st) {
    // the backward pass splats nothing; only forward kernels get the aggregating variant
    if (MODE != MODE_BWD && p.aggregate) return launch_one<MODE, MEDIA, CNT, true>(s, p, cfg, st);
    return launch_one<MODE, MEDIA, CNT, false>(s, p, cfg, st);
}

}  // namespace

mt_status mt_launch_render(const DevScene &s, const RenderParams &p, const LaunchCfg &cfg, int mode, bool counters,
                           cudaStream_t st) {
    const bool media = s.has_medium;
#define MT_DISPATCH(M)                                                                 \
    if (media) return counters ? launch_agg<M, true, true>(s, p, cfg, st) : launch_agg<M, true, false>(s, p, cfg, st); \
    return counters ? launch_agg<M, false, true>(s, p, cfg, st) : launch_agg<M, false, false>(s, p, cfg, st);
    if (mode == 0) { MT_DISPATCH(MODE_FWD) }
    if (mode == 1) { MT_DISPATCH(MODE_DUMP) }
    if (mode == 3) { MT_DISPATCH(MODE_PHASOR) }
    if (mode == 4) {
        // forward-mode derivative: no counting or aggregating variants
        return media ? launch_one<MODE_TAN, true, false, false>(s, p, cfg, st)
                     : launch_one<MODE_TAN, false, false, false>(s, p, cfg, st);
    }
    MT_DISPATCH(MODE_BWD)
#undef MT_DISPATCH
}
