// mt_polar.cuh -- device helpers of transient polarization tracking (arXiv
// 2510.25660 Sec. 4.2): complex arithmetic, the Fresnel Mueller entries of a
// conductor, Stokes reference frames and the per-colour Mueller throughput of
// a path.  Used by the path-per-thread kernel (mt_polar.cu) and the wavefront
// stages (mt_wavefront.cu).
#pragma once
#include "mt_common.cuh"

namespace {

struct cf {
    float re, im;
};
__device__ __forceinline__ cf cmul(cf a, cf b) { return cf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf cdiv(cf a, cf b) {
    const float d = b.re * b.re + b.im * b.im;
    return cf{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// principal square root (imaginary part takes the sign of z.im)
__device__ __forceinline__ cf csqrt_p(cf z) {
    const float r = hypotf(z.re, z.im);
    return cf{sqrtf(fmaxf(0.0f, 0.5f * (r + z.re))), copysignf(sqrtf(fmaxf(0.0f, 0.5f * (r - z.re))), z.im)};
}

// Fresnel reflection of an interface from vacuum into 1 + i kappa at incidence
// cosine ci: Mueller entries a = (Rs + Rp)/2, b = (Rs - Rp)/2, c = Re rs rp*, d = Im rs rp*
__device__ __forceinline__ float4 fresnel_abcd(float ci, float kappa) {
    const cf N = {1.0f, kappa};
    const cf N2 = cmul(N, N);
    const cf q = cdiv(cf{1.0f - ci * ci, 0.0f}, N2);
    const cf ct = csqrt_p(cf{1.0f - q.re, -q.im});
    const cf Nct = cmul(N, ct), Nci = cf{ci, kappa * ci};
    const cf rs = cdiv(cf{ci - Nct.re, -Nct.im}, cf{ci + Nct.re, Nct.im});
    const cf rp = cdiv(cf{Nci.re - ct.re, Nci.im - ct.im}, cf{Nci.re + ct.re, Nci.im + ct.im});
    const float Rs = rs.re * rs.re + rs.im * rs.im, Rp = rp.re * rp.re + rp.im * rp.im;
    // rs * conj(rp)
    const float xr = rs.re * rp.re + rs.im * rp.im, xi = rs.im * rp.re - rs.re * rp.im;
    return make_float4(0.5f * (Rs + Rp), 0.5f * (Rs - Rp), xr, xi);
}

__device__ __forceinline__ float conductor_kappa(float f0) {
    const float f = fminf(fmaxf(f0, 0.0f), 0.999f);
    return 2.0f * sqrtf(f / (1.0f - f));
}

// unit normal of the plane of a and b (or any unit vector perpendicular to a)
__device__ __forceinline__ float3 plane_normal(float3 a, float3 b) {
    const float3 c = cross(a, b);
    const float l = sqrtf(dot(c, c));
    if (l > 1e-6f) return c * (1.0f / l);
    float3 t, bb;
    onb(a, t, bb);
    return t;
}

// angle t with x_to = cos t x_from + sin t (k x x_from)
__device__ __forceinline__ float frame_angle(float3 k, float3 x_from, float3 x_to) {
    return atan2f(dot(x_to, cross(k, x_from)), dot(x_to, x_from));
}

struct Mueller {
    float m[3][16];  // per colour, row-major 4x4
};

// P <- P R(t): columns 1 and 2 turn by 2t
__device__ __forceinline__ void rotate_columns(Mueller &P, float t) {
    float s2, c2;
    sincosf(2.0f * t, &s2, &c2);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float p1 = P.m[c][4 * i + 1], p2 = P.m[c][4 * i + 2];
            P.m[c][4 * i + 1] = p1 * c2 - p2 * s2;
            P.m[c][4 * i + 2] = p1 * s2 + p2 * c2;
        }
}

}  // namespace
