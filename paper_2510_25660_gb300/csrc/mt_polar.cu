// mt_polar.cu -- transient polarization tracking (arXiv 2510.25660 Sec. 4.2,
// "Transient polarization tracking"): the same path estimator as k_render
// (NEE with power-heuristic MIS, path reuse into time bins, scattering delays,
// emission pulses) with a Stokes vector (S0..S3) per colour channel instead of
// an intensity.
//
// A path carries a 4x4 Mueller matrix P per colour that maps light leaving its
// current vertex toward the camera (in the frame of that segment) to what the
// camera measures.  Frames: a Stokes vector of light travelling along k is
// given in a reference vector x perpendicular to k, y = k x x, S1 = I_x - I_y,
// S2 = I(+45) - I(-45); the camera's frame is its horizontal axis; the frame
// of the segment leaving a vertex is the normal s of the scattering plane
// (incident and exitant direction).  Going from frame s to frame x multiplies
// by the rotation R(t) (t the angle from s to x about k), which mixes columns
// 1 and 2 of P.  Lambert is an ideal depolariser (only M00 = albedo / pi);
// the GGX conductor reflects at its microfacet with the Fresnel Mueller matrix
// of a complex index 1 + i kappa, kappa = 2 sqrt(F0 / (1 - F0)) (normal-
// incidence reflectance F0 = albedo), times D G2 / (4 cos cos).  Emitters are
// unpolarised, so a contribution is column 0 of the accumulated matrix.
//
// One path per thread in a persistent grid; contributions go to the Stokes
// film [H][W][T][4][3] and the steady Stokes image [H][W][4][3] with global
// atomics (a feature kernel: no shared-memory privatisation).
#include "mt_common.cuh"
#include "mt_internal.h"
#include "mt_launch.h"
#include "mt_trace.cuh"
#include "mt_polar.cuh"

namespace {

struct PolParams {
    int32_t H, W, T;
    int32_t H_full, row0;  // film window: rows [row0, row0 + H) of an H_full x W frame
    float start, width, scale;
    uint32_t flags;
    int32_t spp, max_depth;
    uint32_t sample_offset, k0, k1;
    float *film, *steady;
};

__device__ __forceinline__ void pol_deposit(const DevScene &s, const PolParams &p, uint32_t pix, uint32_t smp,
                                            int depth, int kind, float opl, const float S[3][4]) {
    opl += pulse_time(s, pix, smp, (uint32_t)depth, kind, p.k0, p.k1);
    const float x = (opl - p.start) / p.width;
    const bool in = x >= 0.f && x < (float)p.T;
    const uint32_t lp = pix - (uint32_t)p.row0 * (uint32_t)p.W;  // film pixel of frame pixel pix
    float *f = in ? p.film + ((size_t)lp * p.T + (int)x) * 12 : nullptr;
    float *st = p.steady + (size_t)lp * 12;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = S[c][k] * p.scale;
            if (v != 0.f) {
                if (in) atomicAdd(f + k * 3 + c, v);
                atomicAdd(st + k * 3 + c, v);
            }
        }
}

__global__ void __launch_bounds__(128) k_render_pol(const DevScene s, const PolParams p) {
    const long long n_paths = (long long)p.H * p.W * p.spp;
    TraceCnt tc{0, 0};
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_paths;
         j += (long long)gridDim.x * blockDim.x) {
        const uint32_t lpix = (uint32_t)(j / p.spp);
        const uint32_t smp = p.sample_offset + (uint32_t)(j - (long long)lpix * p.spp);
        const uint32_t pix = lpix + (uint32_t)p.row0 * (uint32_t)p.W;  // frame pixel id
        const int px = (int)(pix % (uint32_t)p.W), py = (int)(pix / (uint32_t)p.W);
        const uint4 R0 = philox4x32_10(make_uint4(pix, smp, 0u, 0u), p.k0, p.k1);
        const bool center = p.flags & MT_PIXEL_CENTER;
        const float jx = center ? 0.5f : u24(R0.x), jy = center ? 0.5f : u24(R0.y);
        const float sx = (2.0f * ((float)px + jx) / (float)p.W - 1.0f) * s.tan_half;
        const float sy =
            (1.0f - 2.0f * ((float)py + jy) / (float)p.H_full) * s.tan_half * ((float)p.H_full / (float)p.W);
        float3 o = s.cam_o;
        float3 d = normalize(s.cam_f + s.cam_r * sx + s.cam_u * sy);
        Mueller P;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int e = 0; e < 16; ++e) P.m[c][e] = (e % 5 == 0) ? 1.0f : 0.0f;
        float3 xf = normalize(s.cam_r - d * dot(s.cam_r, d));
        float opl = 0.f, prev_pdf = 0.f;
        for (int depth = 1; depth <= p.max_depth; ++depth) {
            const RayT r = make_ray(s, o, d);
            float th;
            int orig;
            const int k = trace_closest<false>(s, r, INFINITY, th, orig, tc);
            if (k < 0) break;
            const float3 x = o + d * th;
            if (!(depth == 1 && (p.flags & MT_UNWARP))) opl += th;
            const float4 p0 = __ldg(&s.tris[3 * k]), p1 = __ldg(&s.tris[3 * k + 1]), p2 = __ldg(&s.tris[3 * k + 2]);
            const float3 ng = normalize(cross(xyz(p1) - xyz(p0), xyz(p2) - xyz(p0)));
            const float3 wo = -d;
            const float cwo = dot(ng, wo);
            const int unit = __ldg(&s.tri_unit[orig]);
            if (unit >= 0 && cwo > 0.f) {
                const LightUnit U = s.units[unit];
                float w = 1.0f;
                if (depth > 1) {
                    const float pl = (U.v1.w / U.v0.w) * th * th / cwo;
                    w = prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);
                }
                const float4 Le = s.em_rad[__float_as_int(U.v2.w)];
                const float le[3] = {Le.x, Le.y, Le.z};
                float S[3][4];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int q = 0; q < 4; ++q) S[c][q] = P.m[c][4 * q] * le[c] * w;
                pol_deposit(s, p, pix, smp, depth, 0, opl, S);
            }
            if (depth == p.max_depth) break;
            opl += vertex_delay(s, orig, pix, smp, (uint32_t)depth, p.k0, p.k1);
            const float3 n = cwo >= 0.f ? ng : -ng;
            float3 tb, bb;
            onb(n, tb, bb);
            const float3 wol = to_local(wo, tb, bb, n);
            const float4 mm = __ldg(&s.mats[orig]);
            const Mat m{xyz(mm), mm.w};
            const float alb[3] = {mm.x, mm.y, mm.z};
            // next-event estimate
            if (s.n_units > 0) {
                const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_NEE), p.k0, p.k1);
                int lo = 0, hi = s.n_units - 1;
                const uint32_t key = R.x >> 8;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (key < __ldg(&s.unit_cdf[mid])) hi = mid;
                    else lo = mid + 1;
                }
                const LightUnit U = s.units[lo];
                const int em = __float_as_int(U.v2.w);
                const bool is_pt = __float_as_int(U.n.w) < 0;
                const float3 y = is_pt ? xyz(U.v0) : tri_point(xyz(U.v0), xyz(U.v1), xyz(U.v2), u24(R.y), u24(R.z));
                const float3 xo = x + n * eps_of(x);
                const float3 dl = y - xo;
                const float dist = sqrtf(dot(dl, dl));
                const float3 wi = dl * (1.0f / dist);
                const float cx = dot(n, wi);
                const float cy = is_pt ? 1.0f : -dot(xyz(U.n), wi);
                if (cx > 0.f && cy > 0.f && dist > 0.f) {
                    const float tmax = dist - (is_pt ? 0.0f : eps_of(y));
                    if (!trace_any<false>(s, make_ray(s, xo, wi), tmax, tc)) {
                        const float3 wil = to_local(wi, tb, bb, n);
                        float3 fc;
                        float pb;
                        bsdf_eval(m, wol, wil, fc, pb);
                        const float pick = U.v1.w;
                        float geo, w = 1.0f;
                        if (is_pt) geo = 1.0f / (dist * dist) / pick;
                        else {
                            const float pA = pick / U.v0.w;
                            geo = cy / (dist * dist) / pA;
                            const float a = pA * dist * dist / cy;
                            w = a * a / (a * a + pb * pb);
                        }
                        const float4 Le = s.em_rad[em];
                        const float le[3] = {Le.x, Le.y, Le.z};
                        const float t = frame_angle(wo, plane_normal(wi, d), xf);
                        float s2, c2;
                        sincosf(2.0f * t, &s2, &c2);
                        float S[3][4];
                        if (m.rough < 0.f) {
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float kk = alb[c] * (1.0f / MT_PI) * cx * geo * w * le[c];
#pragma unroll
                                for (int q = 0; q < 4; ++q) S[c][q] = P.m[c][4 * q] * kk;
                            }
                        } else {
                            const float a = fmaxf(m.rough, 1e-4f), a2 = a * a;
                            const float3 h = normalize(wol + wil);
                            const float kd = (h.x * h.x + h.y * h.y) + a2 * (h.z * h.z);
                            const float D = a2 / (MT_PI * kd * kd);
                            const float G2 = 1.0f / (1.0f + ggx_lambda(a2, wol) + ggx_lambda(a2, wil));
                            const float kf = D * G2 / (4.0f * wol.z * wil.z) * cx * geo * w;
                            const float cd = dot(wil, h);
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float4 F = fresnel_abcd(cd, conductor_kappa(alb[c]));
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    // column 0 of (P R(t)) M_F
                                    const float q0 = P.m[c][4 * q];
                                    const float q1 = P.m[c][4 * q + 1] * c2 - P.m[c][4 * q + 2] * s2;
                                    S[c][q] = (q0 * F.x + q1 * F.y) * kf * le[c];
                                }
                            }
                        }
                        pol_deposit(s, p, pix, smp, depth, 1, opl + dist, S);
                    }
                }
            }
            // continue by sampling the BSDF
            const uint4 R = philox4x32_10(make_uint4(pix, smp, (uint32_t)depth, G_SCATTER), p.k0, p.k1);
            float3 wil;
            if (!bsdf_sample(m, wol, u24(R.x), u24(R.y), wil)) break;
            float3 f;
            float pb;
            bsdf_eval(m, wol, wil, f, pb);
            if (!(pb > 0.f)) break;
            const float3 wi = to_world(wil, tb, bb, n);
            const float3 sv = plane_normal(wi, d);
            rotate_columns(P, frame_angle(wo, sv, xf));
            if (m.rough < 0.f) {
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
            } else {
                const float a = fmaxf(m.rough, 1e-4f), a2 = a * a;
                const float3 h = normalize(wol + wil);
                const float kd = (h.x * h.x + h.y * h.y) + a2 * (h.z * h.z);
                const float D = a2 / (MT_PI * kd * kd);
                const float G2 = 1.0f / (1.0f + ggx_lambda(a2, wol) + ggx_lambda(a2, wil));
                const float kf = D * G2 / (4.0f * wol.z * wil.z) * wil.z / pb;
                const float cd = dot(wil, h);
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
            xf = sv;
            prev_pdf = pb;
            o = x + n * eps_of(x);
            d = wi;
        }
    }
}

}  // namespace

mt_status mt_launch_polarized(const DevScene &s, int32_t H, int32_t W, int32_t T, int32_t H_full, int32_t row0,
                              float start, float width, float scale, uint32_t flags, int32_t spp, int32_t max_depth,
                              uint32_t sample_offset, uint32_t k0, uint32_t k1, float *film, float *steady,
                              int num_sms, cudaStream_t st) {
    PolParams p{H, W, T, H_full, row0, start, width, scale, flags, spp, max_depth, sample_offset, k0, k1, film, steady};
    const long long n = (long long)H * W * spp;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 127) / 128, (long long)num_sms * 8));
    k_render_pol<<<grid, 128, 0, st>>>(s, p);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}
