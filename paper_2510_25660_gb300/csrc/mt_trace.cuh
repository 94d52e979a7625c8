// mt_trace.cuh -- BVH traversal and ray/triangle intersection (device code).
//
// Visibility V and segment lengths of the path integral (arXiv 2510.25660,
// Sec. 3 Eqs. 3 and 8) come from these queries.
//
// Node layout (32 bytes = one L2 sector, fetched by one 256-bit load): one
// 32-bit word per child and axis holds that axis' lower plane (low half) and
// upper plane (high half):
//   a.x = child 0 x   a.y = child 0 y   a.z = child 0 z   a.w = child 1 x
//   b.x = child 1 y   b.y = child 1 z   b.z = child 0 reference   b.w = child 1 reference
// Planes are 16-bit fixed point in the scene box, rounded outward by two steps
// (plane = q_lo + q * q_scale), so boxes are conservative.  A reference with
// bit 31 clear is an internal node index; with bit 31 set it is a leaf of
// ((ref >> 29) & 3) + 1 triangles starting at (ref & 0x1FFFFFFF); 0xFFFFFFFF
// is an empty child.  Triangles are 48-byte records (three float4 vertices,
// v0.w holding the original triangle index as int bits) in leaf order.
#pragma once
#include "mt_common.cuh"

#define MT_EMPTY_REF 0xFFFFFFFFu

// An empty child also has inverted planes (lower 65535, upper 0 on every axis),
// which the slab test rejects for either direction sign, so the traversal does
// not need to look at its reference.
#ifndef MT_CHECK_EMPTY
#define MT_CHECK_EMPTY 0
#endif
#define MT_LIVE(ref) (!MT_CHECK_EMPTY || (ref) != MT_EMPTY_REF)

struct RayT {
    float3 o, d;
    float3 sa, sb;   // slab: t = (2^23 + q) * sa + sb for a quantised plane q
    float3 inv;      // 1 / direction (zero components replaced by +-1e-20)
    uint32_t oct;    // bit k set: direction component k is negative
    uint32_t sel_n[3];  // byte-permute selector of the near plane per axis (far = near ^ 0x22)
    int kx, ky, kz;  // watertight test axes (Woop, Benthin, Wald, JCGT 2013)
    float Sx, Sy, Sz;
};

__device__ __forceinline__ float comp3(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ RayT make_ray(const DevScene &s, float3 o, float3 d) {
    RayT r;
    r.o = o;
    r.d = d;
    // zero direction components are replaced by +-1e-20 for the slab test only
    const float dx = fabsf(d.x) < 1e-20f ? copysignf(1e-20f, d.x) : d.x;
    const float dy = fabsf(d.y) < 1e-20f ? copysignf(1e-20f, d.y) : d.y;
    const float dz = fabsf(d.z) < 1e-20f ? copysignf(1e-20f, d.z) : d.z;
    const float ix = 1.0f / dx, iy = 1.0f / dy, iz = 1.0f / dz;
    r.inv = f3(ix, iy, iz);
    r.oct = (dx < 0.0f ? 1u : 0u) | (dy < 0.0f ? 2u : 0u) | (dz < 0.0f ? 4u : 0u);
    r.sa = f3(s.q_scale.x * ix, s.q_scale.y * iy, s.q_scale.z * iz);
    // the 2^23 offset of the exponent trick below is folded into sb; the two
    // 2^23 * sa terms cancel exactly inside the FMA, leaving one rounding of sb
    // (at most half a quantisation step, inside the two-step padding)
    r.sb = f3((s.q_lo.x - o.x) * ix - 8388608.0f * r.sa.x, (s.q_lo.y - o.y) * iy - 8388608.0f * r.sa.y,
              (s.q_lo.z - o.z) * iz - 8388608.0f * r.sa.z);
    const float dd[3] = {dx, dy, dz};
#pragma unroll
    for (int k = 0; k < 3; ++k) r.sel_n[k] = dd[k] >= 0.0f ? 0x7610u : 0x7632u;  // low half = lower plane
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (comp3(d, kz) < 0.0f) {
        const int t = kx;
        kx = ky;
        ky = t;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    const float dk = comp3(d, kz);
    r.Sx = comp3(d, kx) / dk;
    r.Sy = comp3(d, ky) / dk;
    r.Sz = 1.0f / dk;
    return r;
}

// 16-bit fixed point q -> the float 2^23 + q (exact) by writing q under the
// exponent of 2^23 with one byte permute
__device__ __forceinline__ float q_plane(uint32_t word, uint32_t sel) {
    return __int_as_float(__byte_perm(word, 0x4B000000u, sel));
}

// One binary node (32 bytes, 32-byte aligned) in one 256-bit read-only load
// (sm_100-class); MT_NODE_V8 = 0: two 128-bit loads.
#ifndef MT_NODE_V8
#define MT_NODE_V8 1
#endif
__device__ __forceinline__ void ldg_node(const uint4 *p, uint4 &a, uint4 &b) {
#if MT_NODE_V8 && !MT_L2_KEEP_BVH
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
        : "l"(p));
#else
    a = ldg_keep(p);
    b = ldg_keep(p + 1);
#endif
}

// Packed arithmetic of sm_100-class GPUs: fma.rn.f32x2 (two independent FMAs,
// each rounded once, in one instruction) and three-input min/max.  Each lane
// gets the same values as the scalar forms, so switching MT_SLAB_PACKED off
// (scalar FMAs and two-input min/max) changes no result, only the count of
// issued instructions per node.
#ifndef MT_SLAB_PACKED
#define MT_SLAB_PACKED 1
#endif

__device__ __forceinline__ void fma_x2(float ax, float ay, float bx, float by, float cx, float cy, float &dx,
                                       float &dy) {
#if MT_SLAB_PACKED
    asm("{\n\t.reg .b64 a, b, c, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmov.b64 c, {%6, %7};\n\t"
        "fma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(dx), "=f"(dy)
        : "f"(ax), "f"(ay), "f"(bx), "f"(by), "f"(cx), "f"(cy));
#else
    dx = fmaf(ax, bx, cx);
    dy = fmaf(ay, by, cy);
#endif
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
#if MT_SLAB_PACKED
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
#else
    return fmaxf(fmaxf(a, b), c);
#endif
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
#if MT_SLAB_PACKED
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
#else
    return fminf(fminf(a, b), c);
#endif
}

// entry / exit distance of one child box; wx, wy, wz are its three axis words
__device__ __forceinline__ void slab(const RayT &r, uint32_t wx, uint32_t wy, uint32_t wz, float tmax, float &tn,
                                     float &tf) {
    float nx, ny, fx, fy;
    fma_x2(q_plane(wx, r.sel_n[0]), q_plane(wy, r.sel_n[1]), r.sa.x, r.sa.y, r.sb.x, r.sb.y, nx, ny);
    fma_x2(q_plane(wx, r.sel_n[0] ^ 0x22u), q_plane(wy, r.sel_n[1] ^ 0x22u), r.sa.x, r.sa.y, r.sb.x, r.sb.y, fx,
           fy);
    const float nz = fmaf(q_plane(wz, r.sel_n[2]), r.sa.z, r.sb.z);
    const float fz = fmaf(q_plane(wz, r.sel_n[2] ^ 0x22u), r.sa.z, r.sb.z);
    tn = fmaxf(max3f(nx, ny, nz), 0.0f);
    tf = fminf(min3f(fx, fy, fz), tmax);
}

// entry / exit distances of both child boxes of a binary node (a, b = its two
// 128-bit halves); with MT_SLAB_PAIR_Z the z planes of the two children share
// packed FMAs as the x and y planes of one child do (same results)
#ifndef MT_SLAB_PAIR_Z
#define MT_SLAB_PAIR_Z 0
#endif
__device__ __forceinline__ void slab2(const RayT &r, const uint4 &a, const uint4 &b, float tmax, float &tn0,
                                      float &tf0, float &tn1, float &tf1) {
#if MT_SLAB_PAIR_Z
    const uint32_t sx = r.sel_n[0], sy = r.sel_n[1], sz = r.sel_n[2];
    float nx0, ny0, fx0, fy0, nx1, ny1, fx1, fy1, nz0, nz1, fz0, fz1;
    fma_x2(q_plane(a.x, sx), q_plane(a.y, sy), r.sa.x, r.sa.y, r.sb.x, r.sb.y, nx0, ny0);
    fma_x2(q_plane(a.x, sx ^ 0x22u), q_plane(a.y, sy ^ 0x22u), r.sa.x, r.sa.y, r.sb.x, r.sb.y, fx0, fy0);
    fma_x2(q_plane(a.w, sx), q_plane(b.x, sy), r.sa.x, r.sa.y, r.sb.x, r.sb.y, nx1, ny1);
    fma_x2(q_plane(a.w, sx ^ 0x22u), q_plane(b.x, sy ^ 0x22u), r.sa.x, r.sa.y, r.sb.x, r.sb.y, fx1, fy1);
    fma_x2(q_plane(a.z, sz), q_plane(b.y, sz), r.sa.z, r.sa.z, r.sb.z, r.sb.z, nz0, nz1);
    fma_x2(q_plane(a.z, sz ^ 0x22u), q_plane(b.y, sz ^ 0x22u), r.sa.z, r.sa.z, r.sb.z, r.sb.z, fz0, fz1);
    tn0 = fmaxf(max3f(nx0, ny0, nz0), 0.0f);
    tf0 = fminf(min3f(fx0, fy0, fz0), tmax);
    tn1 = fmaxf(max3f(nx1, ny1, nz1), 0.0f);
    tf1 = fminf(min3f(fx1, fy1, fz1), tmax);
#else
    slab(r, a.x, a.y, a.z, tmax, tn0, tf0);
    slab(r, a.w, b.x, b.y, tmax, tn1, tf1);
#endif
}

// Watertight ray/triangle test.  The edge functions are evaluated without
// contraction so that a shared edge gives exactly opposite values in its two
// triangles (no gaps).  Returns true with t = T/det when the ray crosses the
// triangle (edges inclusive) at t > 0.
__device__ __forceinline__ bool tri_hit(const RayT &r, float3 v0, float3 v1, float3 v2, float &t) {
    const float3 A = v0 - r.o, B = v1 - r.o, C = v2 - r.o;
    const float Akz = comp3(A, r.kz), Bkz = comp3(B, r.kz), Ckz = comp3(C, r.kz);
    const float Ax = comp3(A, r.kx) - r.Sx * Akz, Ay = comp3(A, r.ky) - r.Sy * Akz;
    const float Bx = comp3(B, r.kx) - r.Sx * Bkz, By = comp3(B, r.ky) - r.Sy * Bkz;
    const float Cx = comp3(C, r.kx) - r.Sx * Ckz, Cy = comp3(C, r.ky) - r.Sy * Ckz;
    const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    const float det = U + V + W;
    if (det == 0.f) return false;
    const float T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
    if (det > 0.f ? T <= 0.f : T >= 0.f) return false;
    t = T / det;
    return true;
}

struct TraceCnt {
    uint32_t nodes, tris;  // bytes of BVH nodes fetched, triangle records tested
};

// MT_LEAF_STEP bit 0 (closest hit), bit 1 (any hit): a leaf's triangles are
// tested one per iteration of the traversal loop (the leaf reference advances
// to the next triangle: first + 1, count - 1), so that in a warp whose lanes
// meet leaves at different steps the diverging leaf work of one step is one
// triangle test instead of up to four, while the other lanes go on with their
// nodes.  The nodes visited, their order and the triangles tested are the
// same, so are the hits.  Measured on the 1.16M-triangle scene (fused
// traversal pass of the 512x512x256-spp render): 67.36 ms with the leaf's
// triangles in an inner loop, 66.54 (closest hit only), 66.24 (any hit
// only), 65.35 ms (both).
#ifndef MT_LEAF_STEP
#define MT_LEAF_STEP 3
#endif
#define MT_LEAF_MORE 0x60000000u                // count - 1 field of a leaf reference
#define MT_LEAF_NEXT (1u - 0x20000000u)         // first + 1, count - 1 (mod 2^32)

// MT_SMEM_STACK > 0: the first MT_SMEM_STACK entries of each thread's traversal
// stack live in shared memory (CTAs of at most 256 threads), deeper ones in
// local memory
#ifndef MT_SMEM_STACK
#define MT_SMEM_STACK 0
#endif

// Closest hit with t in (0, tmax); ties in t go to the smaller original index.
// Returns the leaf-order triangle index (or -1) and writes t and the original index.
template <bool CNT>
__device__ __forceinline__ int trace_closest_simple(const DevScene &s, const RayT &r, float tmax, float &t_out,
                                                    int &orig_out, TraceCnt &cnt) {
    float tbest = tmax;
    int best_k = -1, best_id = 0x7fffffff;
    uint2 st[MT_STACK];  // (reference, entry distance bits)
#if MT_SMEM_STACK
    __shared__ uint2 s_st[MT_SMEM_STACK][256];
#define MT_ST_PUT(i, v) do { if ((i) < MT_SMEM_STACK) s_st[i][threadIdx.x] = (v); else st[i] = (v); } while (0)
#define MT_ST_GET(i) ((i) < MT_SMEM_STACK ? s_st[i][threadIdx.x] : st[i])
#else
#define MT_ST_PUT(i, v) (st[i] = (v))
#define MT_ST_GET(i) (st[i])
#endif
    int sp = 0;
    uint32_t ref = 0;
    for (;;) {
        if (!(ref & 0x80000000u)) {
            uint4 a, b;
            ldg_node(&s.nodes[2 * ref], a, b);
            if (CNT) cnt.nodes += 32;
            float tn0, tf0, tn1, tf1;
            slab2(r, a, b, tbest, tn0, tf0, tn1, tf1);
            const bool h0 = tn0 <= tf0 && MT_LIVE(b.z);
            const bool h1 = tn1 <= tf1 && MT_LIVE(b.w);
            if (h0 && h1) {
                const bool f0 = tn0 <= tn1;
                if (sp < MT_STACK) {
                    MT_ST_PUT(sp, make_uint2(f0 ? b.w : b.z, __float_as_uint(f0 ? tn1 : tn0)));
                    ++sp;
                } else {
                    raise_err(s, MT_EFLAG_STACK);
                }
                ref = f0 ? b.z : b.w;
                continue;
            }
            if (h0) { ref = b.z; continue; }
            if (h1) { ref = b.w; continue; }
        } else {
#if MT_LEAF_STEP & 1
            // one triangle of the leaf per iteration; the rest stay in `ref`
            const int k = (int)(ref & 0x1FFFFFFFu);
            const float4 p0 = ldg_keep(&s.tris[3 * k]);
            const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
            const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
            if (CNT) cnt.tris++;
            float t;
            if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
                const int id = __float_as_int(p0.w);
                if (t < tbest || (t == tbest && id < best_id)) {
                    tbest = t;
                    best_k = k;
                    best_id = id;
                }
            }
            if (ref & MT_LEAF_MORE) {
                ref += MT_LEAF_NEXT;
                continue;
            }
#else
            const int first = (int)(ref & 0x1FFFFFFFu), n = (int)((ref >> 29) & 3u) + 1;
            for (int k = first; k < first + n; ++k) {
                const float4 p0 = ldg_keep(&s.tris[3 * k]);
                const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
                const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
                if (CNT) cnt.tris++;
                float t;
                if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
                    const int id = __float_as_int(p0.w);
                    if (t < tbest || (t == tbest && id < best_id)) {
                        tbest = t;
                        best_k = k;
                        best_id = id;
                    }
                }
            }
#endif
        }
        // pop the next entry whose entry distance does not exceed the best hit
        for (;;) {
            if (sp == 0) {
                t_out = tbest;
                orig_out = best_id;
                return best_k;
            }
            --sp;
            const uint2 e = MT_ST_GET(sp);
            if (__uint_as_float(e.y) <= tbest) {
                ref = e.x;
                break;
            }
        }
    }
}

#undef MT_ST_PUT
#undef MT_ST_GET

// Any hit with t in (0, tmax).
template <bool CNT>
__device__ __forceinline__ bool trace_any_simple(const DevScene &s, const RayT &r, float tmax, TraceCnt &cnt) {
    uint32_t st_ref[MT_STACK];
#if MT_SMEM_STACK
    __shared__ uint32_t s_st1[MT_SMEM_STACK][256];
#endif
    int sp = 0;
    uint32_t ref = 0;
    for (;;) {
        if (!(ref & 0x80000000u)) {
            uint4 a, b;
            ldg_node(&s.nodes[2 * ref], a, b);
            if (CNT) cnt.nodes += 32;
            float tn0, tf0, tn1, tf1;
            slab2(r, a, b, tmax, tn0, tf0, tn1, tf1);
            const bool h0 = tn0 <= tf0 && MT_LIVE(b.z);
            const bool h1 = tn1 <= tf1 && MT_LIVE(b.w);
            if (h0 && h1) {
                const bool f0 = tn0 <= tn1;
                if (sp < MT_STACK) {
#if MT_SMEM_STACK
                    if (sp < MT_SMEM_STACK) s_st1[sp][threadIdx.x] = f0 ? b.w : b.z;
                    else st_ref[sp] = f0 ? b.w : b.z;
#else
                    st_ref[sp] = f0 ? b.w : b.z;
#endif
                    ++sp;
                } else {
                    raise_err(s, MT_EFLAG_STACK);
                }
                ref = f0 ? b.z : b.w;
                continue;
            }
            if (h0) { ref = b.z; continue; }
            if (h1) { ref = b.w; continue; }
        } else {
#if MT_LEAF_STEP & 2
            const int k = (int)(ref & 0x1FFFFFFFu);
            const float4 p0 = ldg_keep(&s.tris[3 * k]);
            const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
            const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
            if (CNT) cnt.tris++;
            float t;
            if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) return true;
            if (ref & MT_LEAF_MORE) {
                ref += MT_LEAF_NEXT;
                continue;
            }
#else
            const int first = (int)(ref & 0x1FFFFFFFu), n = (int)((ref >> 29) & 3u) + 1;
            for (int k = first; k < first + n; ++k) {
                const float4 p0 = ldg_keep(&s.tris[3 * k]);
                const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
                const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
                if (CNT) cnt.tris++;
                float t;
                if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) return true;
            }
#endif
        }
        if (sp == 0) return false;
        --sp;
#if MT_SMEM_STACK
        ref = sp < MT_SMEM_STACK ? s_st1[sp][threadIdx.x] : st_ref[sp];
#else
        ref = st_ref[sp];
#endif
    }
}

// ---------------------------------------------------------------------------
// "While-while" traversal with speculative leaf postponing (Aila & Laine,
// HPG 2009): a lane keeps descending internal nodes after it met a leaf, which
// it postpones, until every lane of the warp holds a leaf; then the lanes test
// their leaves' triangles together.  Only the visiting order changes: the
// closest hit is still the smallest (t, original index).
// ---------------------------------------------------------------------------
#define MT_DONE 0xFFFFFFFEu
#define MT_IS_LEAF(r) (((r) & 0x80000000u) != 0u)

template <bool ANY, bool CNT>
__device__ __forceinline__ int trace_ww(const DevScene &s, const RayT &r, float tmax, float &t_out, int &orig_out,
                                        TraceCnt &cnt) {
    float tbest = tmax;
    int best_k = -1, best_id = 0x7fffffff;
    uint32_t st_ref[MT_STACK];
    float st_t[MT_STACK];
    int sp = 0;
    uint32_t ref = 0, leaf = MT_DONE;
    auto pop = [&]() -> uint32_t {
        while (sp > 0) {
            --sp;
            if (ANY || st_t[sp] <= tbest) return st_ref[sp];
        }
        return MT_DONE;
    };
    while (ref != MT_DONE) {
        // internal nodes; the first leaf met is postponed
        while (ref != MT_DONE && !MT_IS_LEAF(ref)) {
            uint4 a, b;
            ldg_node(&s.nodes[2 * ref], a, b);
            if (CNT) cnt.nodes += 32;
            float tn0, tf0, tn1, tf1;
            slab(r, a.x, a.y, a.z, tbest, tn0, tf0);
            slab(r, a.w, b.x, b.y, tbest, tn1, tf1);
            const bool h0 = tn0 <= tf0 && MT_LIVE(b.z);
            const bool h1 = tn1 <= tf1 && MT_LIVE(b.w);
            if (h0 && h1) {
                const bool f0 = tn0 <= tn1;
                if (sp < MT_STACK) {
                    st_ref[sp] = f0 ? b.w : b.z;
                    st_t[sp] = f0 ? tn1 : tn0;
                    ++sp;
                } else {
                    raise_err(s, MT_EFLAG_STACK);
                }
                ref = f0 ? b.z : b.w;
            } else if (h0) {
                ref = b.z;
            } else if (h1) {
                ref = b.w;
            } else {
                ref = pop();
            }
            if (ref != MT_DONE && MT_IS_LEAF(ref) && leaf == MT_DONE) {
                leaf = ref;
                ref = pop();
            }
            if (!__any_sync(__activemask(), leaf == MT_DONE)) break;
        }
        // leaves: the postponed one, then the current reference while it is a leaf
        for (;;) {
            if (leaf == MT_DONE) {
                if (ref != MT_DONE && MT_IS_LEAF(ref)) {
                    leaf = ref;
                    ref = pop();
                } else {
                    break;
                }
            }
            const int first = (int)(leaf & 0x1FFFFFFFu), n = (int)((leaf >> 29) & 3u) + 1;
            leaf = MT_DONE;
            for (int k = first; k < first + n; ++k) {
                const float4 p0 = ldg_keep(&s.tris[3 * k]);
                const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
                const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
                if (CNT) cnt.tris++;
                float t;
                if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
                    if (ANY) return 1;
                    const int id = __float_as_int(p0.w);
                    if (t < tbest || (t == tbest && id < best_id)) {
                        tbest = t;
                        best_k = k;
                        best_id = id;
                    }
                }
            }
        }
    }
    if (ANY) return 0;
    t_out = tbest;
    orig_out = best_id;
    return best_k;
}

// ---------------------------------------------------------------------------
// Single-loop traversal with batched leaves: a lane that reaches a leaf keeps
// it pending and goes on with the next node from its stack; the pending leaves
// of a warp are tested together once at least MT_PP_K lanes hold one (or no
// lane has a node left to visit), so that the triangle tests of a few lanes do
// not stall the node tests of the others in every iteration.  Only the visiting
// order changes (closest hit: the smallest (t, original index) over all tested
// triangles; the pop test against a not yet lowered best distance only visits
// more nodes), so the hits are those of trace_closest_simple / trace_any_simple.
// ---------------------------------------------------------------------------
#ifndef MT_PP_K
#define MT_PP_K 16
#endif

template <bool ANY, bool CNT>
__device__ __forceinline__ int trace_pp(const DevScene &s, const RayT &r, float tmax, float &t_out, int &orig_out,
                                        TraceCnt &cnt) {
    float tbest = tmax;
    int best_k = -1, best_id = 0x7fffffff;
    uint2 st[MT_STACK];  // (reference, entry distance bits)
    int sp = 0;
    uint32_t ref = 0, leaf = MT_DONE;
    for (;;) {
        if (ref != MT_DONE && !MT_IS_LEAF(ref)) {
            uint4 a, b;
            ldg_node(&s.nodes[2 * ref], a, b);
            if (CNT) cnt.nodes += 32;
            float tn0, tf0, tn1, tf1;
            slab2(r, a, b, tbest, tn0, tf0, tn1, tf1);
            const bool h0 = tn0 <= tf0 && MT_LIVE(b.z);
            const bool h1 = tn1 <= tf1 && MT_LIVE(b.w);
            if (h0 && h1) {
                const bool f0 = tn0 <= tn1;
                if (sp < MT_STACK) {
                    st[sp] = make_uint2(f0 ? b.w : b.z, __float_as_uint(f0 ? tn1 : tn0));
                    ++sp;
                } else {
                    raise_err(s, MT_EFLAG_STACK);
                }
                ref = f0 ? b.z : b.w;
            } else if (h0) {
                ref = b.z;
            } else if (h1) {
                ref = b.w;
            } else {
                ref = MT_DONE;
                while (sp > 0) {
                    --sp;
                    const uint2 e = st[sp];
                    if (ANY || __uint_as_float(e.y) <= tbest) {
                        ref = e.x;
                        break;
                    }
                }
            }
        }
        if (leaf == MT_DONE && ref != MT_DONE && MT_IS_LEAF(ref)) {  // keep the leaf pending
            leaf = ref;
            ref = MT_DONE;
            while (sp > 0) {
                --sp;
                const uint2 e = st[sp];
                if (ANY || __uint_as_float(e.y) <= tbest) {
                    ref = e.x;
                    break;
                }
            }
        }
        const unsigned act = __activemask();
        const unsigned pend = __ballot_sync(act, leaf != MT_DONE);
        const unsigned busy = __ballot_sync(act, ref != MT_DONE && !MT_IS_LEAF(ref));
        if (__popc(pend) >= MT_PP_K || busy == 0u) {
            if (leaf != MT_DONE) {
                const int first = (int)(leaf & 0x1FFFFFFFu), n = (int)((leaf >> 29) & 3u) + 1;
                leaf = MT_DONE;
                for (int k = first; k < first + n; ++k) {
                    const float4 p0 = ldg_keep(&s.tris[3 * k]);
                    const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
                    const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
                    if (CNT) cnt.tris++;
                    float t;
                    if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
                        if (ANY) return 1;
                        const int id = __float_as_int(p0.w);
                        if (t < tbest || (t == tbest && id < best_id)) {
                            tbest = t;
                            best_k = k;
                            best_id = id;
                        }
                    }
                }
            }
        }
        if (ref == MT_DONE && leaf == MT_DONE) break;
    }
    if (ANY) return -1;
    t_out = tbest;
    orig_out = best_id;
    return best_k;
}

// while-while traversal measured slower than the single loop on GB300 for the
// large scene (269 ms against 244 ms per render), so it is off by default
#ifndef MT_TRAVERSAL_WW
#define MT_TRAVERSAL_WW 0
#endif

// 1: closest-hit queries with batched leaves (trace_pp), 2: any-hit queries too
#ifndef MT_TRAVERSAL_PP
#define MT_TRAVERSAL_PP 0
#endif

template <bool CNT>
__device__ __forceinline__ int trace_closest(const DevScene &s, const RayT &r, float tmax, float &t_out,
                                             int &orig_out, TraceCnt &cnt) {
#if MT_TRAVERSAL_WW
    return trace_ww<false, CNT>(s, r, tmax, t_out, orig_out, cnt);
#elif MT_TRAVERSAL_PP
    return trace_pp<false, CNT>(s, r, tmax, t_out, orig_out, cnt);
#else
    return trace_closest_simple<CNT>(s, r, tmax, t_out, orig_out, cnt);
#endif
}

template <bool CNT>
__device__ __forceinline__ bool trace_any(const DevScene &s, const RayT &r, float tmax, TraceCnt &cnt) {
#if MT_TRAVERSAL_WW
    float t;
    int id;
    return trace_ww<true, CNT>(s, r, tmax, t, id, cnt) != 0;
#elif MT_TRAVERSAL_PP >= 2
    float t;
    int id;
    return trace_pp<true, CNT>(s, r, tmax, t, id, cnt) > 0;
#else
    return trace_any_simple<CNT>(s, r, tmax, cnt);
#endif
}

// ---------------------------------------------------------------------------
// Warp-cooperative traversal: the 32 rays of a warp walk the top of the tree
// as one packet and the rest one ray per lane (hybrid packet / single-ray
// traversal, Benthin, Wald, Woop, Ernst and Mark, IEEE TVCG 2012).  While at
// least MT_HYBRID_MIN of the warp's rays enter the current node, the warp
// visits it together: one node load serves every lane, the stack index is the
// same in every lane (so stack entries are coalesced in local memory), and the
// warp descends first into the child that more of its rays reach first, with
// each lane's own entry distance kept on the stack for culling.  A node that
// fewer rays enter is handed to their lanes, which traverse its subtree alone
// on top of the warp's stack; then the warp pops its next entry.  Only the
// visiting order differs from trace_closest_simple / trace_any_simple: the
// closest hit is the smallest (t, original index) all the same, and the any-hit
// answer is the same.  All 32 lanes call it together, converged; a lane with
// live = false carries no ray and gets -1.  It is an option (MT_HYBRID_EXT,
// MT_HYBRID_SH, MT_PACKET_CAMERA in the wavefront passes): on the 1.16M-triangle
// scene it was slower than one ray per lane at every threshold, even for warps
// of camera rays through one pixel (the packet's visiting order culls less,
// and the votes cost more than the shared node loads save).
// ---------------------------------------------------------------------------
#ifndef MT_HYBRID_MIN
#define MT_HYBRID_MIN 8
#endif

// the triangles of one leaf against one ray; ANY: true on the first hit
template <bool ANY, bool CNT>
__device__ __forceinline__ bool leaf_tris(const DevScene &s, const RayT &r, uint32_t ref, float tmax, float &tbest,
                                          int &best_k, int &best_id, TraceCnt &cnt) {
    const int first = (int)(ref & 0x1FFFFFFFu), n = (int)((ref >> 29) & 3u) + 1;
    for (int k = first; k < first + n; ++k) {
        const float4 p0 = ldg_keep(&s.tris[3 * k]);
        const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
        const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
        if (CNT) cnt.tris++;
        float t;
        if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
            if (ANY) return true;
            const int id = __float_as_int(p0.w);
            if (t < tbest || (t == tbest && id < best_id)) {
                tbest = t;
                best_k = k;
                best_id = id;
            }
        }
    }
    return false;
}

// one ray through the subtree at `ref`, its stack entries above index sp0;
// ANY: true on the first hit
template <bool ANY, bool CNT>
__device__ __forceinline__ bool trav_subtree(const DevScene &s, const RayT &r, uint32_t ref, uint2 *st, const int sp0,
                                             float tmax, float &tbest, int &best_k, int &best_id, TraceCnt &cnt) {
    int sp = sp0;
    for (;;) {
        if (!(ref & 0x80000000u)) {
            uint4 a, b;
            ldg_node(&s.nodes[2 * ref], a, b);
            if (CNT) cnt.nodes += 32;
            float tn0, tf0, tn1, tf1;
            slab2(r, a, b, tbest, tn0, tf0, tn1, tf1);
            const bool h0 = tn0 <= tf0 && MT_LIVE(b.z);
            const bool h1 = tn1 <= tf1 && MT_LIVE(b.w);
            if (h0 && h1) {
                const bool f0 = tn0 <= tn1;
                if (sp < MT_STACK) {
                    st[sp] = make_uint2(f0 ? b.w : b.z, __float_as_uint(f0 ? tn1 : tn0));
                    ++sp;
                } else {
                    raise_err(s, MT_EFLAG_STACK);
                }
                ref = f0 ? b.z : b.w;
                continue;
            }
            if (h0) { ref = b.z; continue; }
            if (h1) { ref = b.w; continue; }
        } else if (leaf_tris<ANY, CNT>(s, r, ref, tmax, tbest, best_k, best_id, cnt)) {
            return true;
        }
        for (;;) {
            if (sp == sp0) return false;
            --sp;
            const uint2 e = st[sp];
            if (__uint_as_float(e.y) <= tbest) {
                ref = e.x;
                break;
            }
        }
    }
}

template <bool ANY, bool CNT>
__device__ __forceinline__ int trace_hybrid(const DevScene &s, const RayT &r, const bool live, float tmax,
                                            float &t_out, int &orig_out, TraceCnt &cnt,
                                            const int min_rays = MT_HYBRID_MIN) {
    float tbest = tmax;
    int best_k = -1, best_id = 0x7fffffff;
    bool found = false;  // ANY: this lane's ray is occluded
    uint2 st[MT_STACK];  // (reference, this lane's entry distance bits; +inf: its ray misses the node)
    int sp = 0;          // the same in every lane
    uint32_t ref = 0;    // the same in every lane
    bool act = live;     // this lane's ray enters node `ref`
    for (;;) {
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (__popc(m) < min_rays) {
            // few rays (or none) enter the node: each traverses its subtree alone
            if (act && trav_subtree<ANY, CNT>(s, r, ref, st, sp, tmax, tbest, best_k, best_id, cnt)) found = true;
        } else if (!(ref & 0x80000000u)) {
            uint4 a, b;
            ldg_node(&s.nodes[2 * ref], a, b);
            if (CNT && act) cnt.nodes += 32;
            float tn0, tf0, tn1, tf1;
            slab2(r, a, b, tbest, tn0, tf0, tn1, tf1);
            const bool h0 = act && tn0 <= tf0 && MT_LIVE(b.z);
            const bool h1 = act && tn1 <= tf1 && MT_LIVE(b.w);
            const unsigned m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
            if (m0 | m1) {
                // child 0 first if it is the nearer (or only) child for at least half of the rays entering either
                const unsigned n0 = __ballot_sync(0xffffffffu, h0 && !(h1 && tn1 < tn0));
                const bool go0 = m0 && (!m1 || 2 * __popc(n0) >= __popc(m0 | m1));
                if (m0 && m1) {
                    if (sp < MT_STACK) {
                        const bool ho = go0 ? h1 : h0;
                        st[sp] = make_uint2(go0 ? b.w : b.z, ho ? __float_as_uint(go0 ? tn1 : tn0) : 0x7F800000u);
                        ++sp;
                    } else {
                        raise_err(s, MT_EFLAG_STACK);
                    }
                }
                ref = go0 ? b.z : b.w;
                act = go0 ? h0 : h1;
                continue;
            }
        } else if (act && leaf_tris<ANY, CNT>(s, r, ref, tmax, tbest, best_k, best_id, cnt)) {
            found = true;
        }
        // the warp's next entry that one of its rays still enters
        if (ANY && !__any_sync(0xffffffffu, live && !found)) break;
        bool more = false;
        while (sp > 0) {
            --sp;
            const uint2 e = st[sp];
            act = !found && __uint_as_float(e.y) <= tbest;
            if (__any_sync(0xffffffffu, act)) {
                ref = e.x;
                more = true;
                break;
            }
        }
        if (!more) break;
    }
    t_out = tbest;
    orig_out = best_id;
    return ANY ? (found ? 1 : -1) : best_k;
}

// ---------------------------------------------------------------------------
// Traversal as a per-lane state machine, one node or leaf per call, for
// kernels whose lanes fetch a new ray as soon as their current one is done
// (persistent threads with dynamic ray fetch, Aila & Laine, HPG 2009).
// ---------------------------------------------------------------------------
struct TravState {
    uint32_t ref;
    int sp;
    float tbest;
    int best_k, best_id;
};

__device__ __forceinline__ void trav_init(TravState &ts, float tmax) {
    ts.ref = 0;
    ts.sp = 0;
    ts.tbest = tmax;
    ts.best_k = -1;
    ts.best_id = 0x7fffffff;
}

// Advance by one node or one leaf; returns true when the traversal is over
// (for ANY: also when a hit is found, signalled by best_k = 1).
template <bool ANY, bool CNT>
__device__ __forceinline__ bool trav_step(const DevScene &s, const RayT &r, float tmax, TravState &ts, uint2 *st,
                                          TraceCnt &cnt) {
    if (!(ts.ref & 0x80000000u)) {
        uint4 a, b;
        ldg_node(&s.nodes[2 * ts.ref], a, b);
        if (CNT) cnt.nodes += 32;
        float tn0, tf0, tn1, tf1;
        slab(r, a.x, a.y, a.z, ts.tbest, tn0, tf0);
        slab(r, a.w, b.x, b.y, ts.tbest, tn1, tf1);
        const bool h0 = tn0 <= tf0 && MT_LIVE(b.z);
        const bool h1 = tn1 <= tf1 && MT_LIVE(b.w);
        if (h0 && h1) {
            const bool f0 = tn0 <= tn1;
            if (ts.sp < MT_STACK) {
                st[ts.sp] = make_uint2(f0 ? b.w : b.z, __float_as_uint(f0 ? tn1 : tn0));
                ++ts.sp;
            } else {
                raise_err(s, MT_EFLAG_STACK);
            }
            ts.ref = f0 ? b.z : b.w;
            return false;
        }
        if (h0) {
            ts.ref = b.z;
            return false;
        }
        if (h1) {
            ts.ref = b.w;
            return false;
        }
    } else {
        const int first = (int)(ts.ref & 0x1FFFFFFFu), n = (int)((ts.ref >> 29) & 3u) + 1;
        for (int k = first; k < first + n; ++k) {
            const float4 p0 = ldg_keep(&s.tris[3 * k]);
            const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
            const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
            if (CNT) cnt.tris++;
            float t;
            if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
                if (ANY) {
                    ts.best_k = 1;
                    return true;
                }
                const int id = __float_as_int(p0.w);
                if (t < ts.tbest || (t == ts.tbest && id < ts.best_id)) {
                    ts.tbest = t;
                    ts.best_k = k;
                    ts.best_id = id;
                }
            }
        }
    }
    while (ts.sp > 0) {
        --ts.sp;
        const uint2 e = st[ts.sp];
        if (ANY || __uint_as_float(e.y) <= ts.tbest) {
            ts.ref = e.x;
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// 8-wide BVH with compressed child boxes (after Ylitie, Karras and Laine,
// "Efficient incoherent ray traversal on GPUs through compressed wide BVHs",
// HPG 2017; the node layout below is this library's own).
//
// Node = 80 bytes = five uint4:
//   w0.xyz  frame origin p (float), w0.w = ex | ey << 8 | ez << 16 | imask << 24
//           (biased float exponents of the per-axis step 2^e; imask bit i set:
//           child slot i is an internal node)
//   w1.x    index of the first internal child; the internal child in slot i
//           is w1.x + popc(imask & ((1 << i) - 1))
//   w1.y    first triangle of this node's leaf children
//   w1.z/w  one meta byte per slot (slots 0-3 / 4-7): a leaf child has
//           0x80 | (count - 1) << 5 | offset, triangles w1.y + offset ...
//   w2.xy qlo_x[8]  w2.zw qlo_y[8]  w3.xy qlo_z[8]  w3.zw qhi_x[8]
//   w4.xy qhi_y[8]  w4.zw qhi_z[8]   (one byte per slot, little-endian)
// A plane is p + q * 2^e, rounded outward by two steps; an empty slot has
// lower planes 255 and upper planes 0 and is never hit.  Slot bit k of a child
// says it lies on the upper side of the node along axis k, so visiting slots
// in increasing order of slot ^ oct(ray) is roughly front to back.
// ---------------------------------------------------------------------------
#define MT_WIDE_WORDS 5

// reorder the bits of an 8-bit mask so that bit k holds bit (k ^ m)
__device__ __forceinline__ uint32_t perm_xor8(uint32_t x, uint32_t m) {
    if (m & 1u) x = ((x & 0x55u) << 1) | ((x >> 1) & 0x55u);
    if (m & 2u) x = ((x & 0x33u) << 2) | ((x >> 2) & 0x33u);
    if (m & 4u) x = ((x & 0x0Fu) << 4) | ((x >> 4) & 0x0Fu);
    return x;
}

// byte i of the 8-byte pair (lo, hi) as the float 2^23 + q
__device__ __forceinline__ float q8(uint32_t lo, uint32_t hi, int i) {
    return __int_as_float(__byte_perm(i < 4 ? lo : hi, 0x4B000000u, 0x7440u | (uint32_t)(i & 3)));
}

// Hit mask of the eight child boxes of node w0..w4 against (0, tmax].
__device__ __forceinline__ uint32_t wide_hits(const RayT &r, const uint4 &w0, const uint4 &w2, const uint4 &w3,
                                              const uint4 &w4, float tmax) {
    // per-axis frame: t = (2^23 + q) * a + b with the 2^23 offset folded into b
    const float ax = __int_as_float((int)((w0.w & 0xFFu) << 23)) * r.inv.x;
    const float ay = __int_as_float((int)(((w0.w >> 8) & 0xFFu) << 23)) * r.inv.y;
    const float az = __int_as_float((int)(((w0.w >> 16) & 0xFFu) << 23)) * r.inv.z;
    const float bx = fmaf(-8388608.0f, ax, (__uint_as_float(w0.x) - r.o.x) * r.inv.x);
    const float by = fmaf(-8388608.0f, ay, (__uint_as_float(w0.y) - r.o.y) * r.inv.y);
    const float bz = fmaf(-8388608.0f, az, (__uint_as_float(w0.z) - r.o.z) * r.inv.z);
    // near planes: the lower ones for a positive direction component
    const bool nx = r.oct & 1u, ny = r.oct & 2u, nz = r.oct & 4u;
    const uint32_t nx0 = nx ? w3.z : w2.x, nx1 = nx ? w3.w : w2.y, fx0 = nx ? w2.x : w3.z, fx1 = nx ? w2.y : w3.w;
    const uint32_t ny0 = ny ? w4.x : w2.z, ny1 = ny ? w4.y : w2.w, fy0 = ny ? w2.z : w4.x, fy1 = ny ? w2.w : w4.y;
    const uint32_t nz0 = nz ? w4.z : w3.x, nz1 = nz ? w4.w : w3.y, fz0 = nz ? w3.x : w4.z, fz1 = nz ? w3.y : w4.w;
    uint32_t hits = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float tnx = fmaf(q8(nx0, nx1, i), ax, bx), tfx = fmaf(q8(fx0, fx1, i), ax, bx);
        const float tny = fmaf(q8(ny0, ny1, i), ay, by), tfy = fmaf(q8(fy0, fy1, i), ay, by);
        const float tnz = fmaf(q8(nz0, nz1, i), az, bz), tfz = fmaf(q8(fz0, fz1, i), az, bz);
        const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, 0.0f));
        const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tmax));
        hits |= (tn <= tf ? 1u : 0u) << i;
    }
    return hits;
}

// Closest hit (ANY = false: returns the triangle index or -1, writes t and the
// original index; ties in t go to the smaller original index) or any hit
// (ANY = true: returns 1 on a hit, else -1) with t in (0, tmax).
template <bool ANY, bool CNT>
__device__ __forceinline__ int trace_wide(const DevScene &s, const RayT &r, float tmax, float &t_out, int &orig_out,
                                          TraceCnt &cnt) {
    float tbest = tmax;
    int best_k = -1, best_id = 0x7fffffff;
    uint2 st[MT_STACK];  // (first internal child, imask << 8 | remaining visit-order mask)
    int sp = 0;
    uint32_t node = 0;
    for (;;) {
        const uint4 *np = s.wnodes + MT_WIDE_WORDS * (size_t)node;
        const uint4 w0 = ldg_keep(np), w1 = ldg_keep(np + 1), w2 = ldg_keep(np + 2), w3 = ldg_keep(np + 3), w4 = ldg_keep(np + 4);
        if (CNT) cnt.nodes += 80;
        const uint32_t hits = wide_hits(r, w0, w2, w3, w4, tbest);
        const uint32_t imask = w0.w >> 24;
        uint32_t leaves = hits & ~imask;
        while (leaves) {
            const int slot = __ffs(leaves) - 1;
            leaves &= leaves - 1u;
            const uint32_t meta = ((slot < 4 ? w1.z : w1.w) >> (8 * (slot & 3))) & 0xFFu;
            const int first = (int)w1.y + (int)(meta & 31u), last = first + (int)((meta >> 5) & 3u);
            for (int k = first; k <= last; ++k) {
                const float4 p0 = ldg_keep(&s.tris[3 * k]);
                const float4 p1 = ldg_keep(&s.tris[3 * k + 1]);
                const float4 p2 = ldg_keep(&s.tris[3 * k + 2]);
                if (CNT) cnt.tris++;
                float t;
                if (tri_hit(r, xyz(p0), xyz(p1), xyz(p2), t) && t < tmax) {
                    if (ANY) return 1;
                    const int id = __float_as_int(p0.w);
                    if (t < tbest || (t == tbest && id < best_id)) {
                        tbest = t;
                        best_k = k;
                        best_id = id;
                    }
                }
            }
        }
        uint32_t order = perm_xor8(hits & imask, r.oct);
        uint32_t base = w1.x, im = imask;
        if (!order) {
            // pop the next group that still has children to visit
            if (sp == 0) break;
            const uint2 g = st[sp - 1];
            base = g.x;
            im = g.y >> 8;
            order = g.y & 0xFFu;
            --sp;
        }
        const int k = __ffs(order) - 1;
        order &= order - 1u;
        const uint32_t slot = (uint32_t)k ^ r.oct;
        node = base + __popc(im & ((1u << slot) - 1u));
        if (order) {
            if (sp < MT_STACK) {
                st[sp] = make_uint2(base, (im << 8) | order);
                ++sp;
            } else {
                raise_err(s, MT_EFLAG_STACK);
            }
        }
    }
    t_out = tbest;
    orig_out = best_id;
    return best_k;
}
