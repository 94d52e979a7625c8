// mt_nlos.cu -- relay-wall NLOS impulse responses (arXiv 2510.25660 Sec. 4.5).
//
// Third-bounce transport laser -> x_l -> y -> x_s -> sensor with y drawn
// uniformly by area on the hidden triangles; the clock is the relay-wall
// clock |x_l - y| + |y - x_s|.  With unit laser power at x_l and Lambertian
// wall (albedo rho_w) and hidden surface (rho_h):
//   H = (rho_w/pi) cos_l (rho_h/pi) cos_y1 cos_y2 (rho_w/pi) cos_s
//       / (|x_l - y|^2 |y - x_s|^2) * A_hidden * V(x_l, y) V(y, x_s)
// per sample.  All scan pairs are one persistent launch: CTAs pull tiles of
// consecutive film rows (scan points, or sensors of one laser), keep the rows'
// time histograms in shared memory and write them to HBM once.  In the
// exhaustive grid the hidden samples of a laser are drawn once (visibility
// x_l -> y included) by k_nlos_ysample and shared by all its sensors.
#include "mt_common.cuh"
#include "mt_internal.h"
#include "mt_launch.h"
#include "mt_trace.cuh"

namespace {

// smallest i with key < hcdf[i] (the last index if none); the guide table only
// narrows the bracket the same search runs in, so the pick is unchanged
__device__ __forceinline__ int pick_hidden(const NlosParams &p, uint32_t u) {
    int lo = 0, hi = p.hidden_n - 1;
    const uint32_t key = u >> 8;
    if (p.hguide) {
        const uint32_t g = key >> 12;
        lo = min((int)__ldg(&p.hguide[g]), p.hidden_n - 1);
        hi = min((int)__ldg(&p.hguide[g + 1]), p.hidden_n - 1);
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key < __ldg(&p.hcdf[mid])) hi = mid;
        else lo = mid + 1;
    }
    return p.hidden_first + lo;
}

struct HiddenSample {
    float3 y, ny;
    float d1, partial;  // partial = fw cos_l fh cos_y1 / d1^2 * A (0 if invalid or occluded)
    float cl, cy1;
    int tri;
};

template <bool CNT>
__device__ __forceinline__ HiddenSample sample_hidden(const DevScene &s, const NlosParams &p, int l, uint32_t smp,
                                                      float3 xl, TraceCnt &tc, uint32_t &rays) {
    HiddenSample h;
    const uint4 R = philox4x32_10(make_uint4((uint32_t)l, smp, 0u, 0u), p.k0, p.k1);
    const int tri = pick_hidden(p, R.x);
    const int k = __ldg(&s.leaf_of[tri]);
    const float3 v0 = xyz(ldg_keep(&s.tris[3 * k])), v1 = xyz(ldg_keep(&s.tris[3 * k + 1])), v2 = xyz(ldg_keep(&s.tris[3 * k + 2]));
    h.tri = tri;
    h.y = tri_point(v0, v1, v2, u24(R.y), u24(R.z));
    h.partial = 0.f;
    h.cl = h.cy1 = 0.f;
    const float3 ng = normalize(cross(v1 - v0, v2 - v0));
    const float3 d1v = h.y - xl;
    h.d1 = sqrtf(dot(d1v, d1v));
    if (!(h.d1 > 0.f)) return h;
    const float3 w1 = d1v * (1.0f / h.d1);
    h.ny = dot(ng, -w1) >= 0.f ? ng : -ng;
    const float cl = dot(p.nw, w1), cy1 = -dot(h.ny, w1);
    h.cl = cl;
    h.cy1 = cy1;
    if (!(cl > 0.f && cy1 > 0.f)) return h;
    const float3 xlo = xl + p.nw * eps_of(xl);
    const float3 r1 = h.y - xlo;
    const float l1 = sqrtf(dot(r1, r1));
    rays++;
    const RayT ray = make_ray(s, xlo, r1 * (1.0f / l1));
    if (trace_any<CNT>(s, ray, l1 - eps_of(h.y), tc)) return h;
    const float4 m = __ldg(&s.mats[tri]);
    const float fh = (m.x + m.y + m.z) * (1.0f / 3.0f) * (1.0f / MT_PI);
    const float area = p.hidden_area_dev ? __ldg(p.hidden_area_dev) : p.hidden_area;
    h.partial = p.fw * cl * fh * cy1 / (h.d1 * h.d1) * area;
    return h;
}

// exhaustive pass 1: hidden samples of every laser, shared by its sensors
template <bool CNT>
__global__ void __launch_bounds__(256) k_nlos_ysample(const DevScene s, const NlosParams p) {
    uint32_t rays = 0;
    TraceCnt tc{0, 0};
    const long long total = (long long)p.n_l * p.spp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(i / p.spp);
        const uint32_t smp = p.sample_offset + (uint32_t)(i - (long long)l * p.spp);
        const float3 xl = f3(p.lasers[3 * l], p.lasers[3 * l + 1], p.lasers[3 * l + 2]);
        const HiddenSample h = sample_hidden<CNT>(s, p, l, smp, xl, tc, rays);
        p.ysamp[2 * i] = make_float4(h.y.x, h.y.y, h.y.z, h.d1);
        p.ysamp[2 * i + 1] = make_float4(h.ny.x, h.ny.y, h.ny.z, h.partial);
        p.ysamp_tri[i] = h.tri;
    }
    unsigned long long v[3] = {rays, tc.nodes, tc.tris};
    const int c_idx[3] = {3, 4, 5};
    for (int c = 0; c < 3; ++c) {
        unsigned long long x = v[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s.counters[c_idx[c]], x);
    }
}

template <bool DUMP, bool CNT>
__global__ void __launch_bounds__(256) k_nlos(const DevScene s, const NlosParams p) {
    extern __shared__ float4 smem4[];
    float *hist = reinterpret_cast<float *>(smem4);
    float *steady_s = hist + (size_t)p.tile * p.D;
    __shared__ int s_tile;
    uint32_t conns = 0, contribs = 0, rays = 0;
    TraceCnt tc{0, 0};
    const bool exh = p.mode == MT_EXHAUSTIVE;
    const long long rows = exh ? (long long)p.n_l * p.n_s : p.n_l;
    const int tiles_per_laser = exh ? (p.n_s + p.tile - 1) / p.tile : 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(p.tile_counter, 1);
        for (int i = threadIdx.x; i < p.tile * (p.D + 1); i += blockDim.x) hist[i] = 0.f;
        __syncthreads();
        const int tile = s_tile;
        if (tile >= p.n_tiles) break;
        // rows [row0, row0 + nrows) of the film; laser l for the exhaustive grid
        long long row0;
        int nrows, l = 0, s0 = 0;
        if (exh) {
            l = tile / tiles_per_laser;
            s0 = (tile - l * tiles_per_laser) * p.tile;
            nrows = min(p.tile, p.n_s - s0);
            row0 = (long long)l * p.n_s + s0;
        } else {
            row0 = (long long)tile * p.tile;
            nrows = (int)min((long long)p.tile, rows - row0);
        }
        const int work = nrows * p.spp;
        // the exhaustive grid goes sensor-fastest: the lanes of a warp take consecutive sensors of the
        // tile and share one hidden sample, so their shadow rays leave the same point y (262 -> 190 ms
        // at 2-row tiles, 130 ms at 32-row tiles for 16x16 lasers x 64x64 sensors x 1024 samples);
        // scan points go sample-fastest
        for (int j = threadIdx.x; j < work; j += blockDim.x) {
            const int r = exh ? j % nrows : j / p.spp;
            const int sj = exh ? j / nrows : j - r * p.spp;
            const uint32_t smp = p.sample_offset + (uint32_t)sj;
            conns++;
            float H = 0.f, opl = 0.f;
            int tri = -1;
            if (!exh) {
                const int li = (int)row0 + r;
                const float3 xl = f3(p.lasers[3 * li], p.lasers[3 * li + 1], p.lasers[3 * li + 2]);
                const HiddenSample h = sample_hidden<CNT>(s, p, li, smp, xl, tc, rays);
                tri = h.tri;
                if (h.partial > 0.f) {
                    // confocal: x_s = x_l, the same segment both ways
                    H = h.partial * h.cy1 * h.cl * p.fw / (h.d1 * h.d1);
                    opl = 2.0f * h.d1;
                }
            } else {
                const int si = s0 + r;
                const float3 xs = f3(p.sensors[3 * si], p.sensors[3 * si + 1], p.sensors[3 * si + 2]);
                const size_t yi = (size_t)l * p.spp + sj;
                const float4 ya = p.ysamp[2 * yi], yb = p.ysamp[2 * yi + 1];
                tri = DUMP ? p.ysamp_tri[yi] : -1;
                if (yb.w > 0.f) {
                    const float3 y = xyz(ya), ny = xyz(yb);
                    const float3 d2v = xs - y;
                    const float d2 = sqrtf(dot(d2v, d2v));
                    if (d2 > 0.f) {
                        const float3 w2 = d2v * (1.0f / d2);
                        const float cs = -dot(p.nw, w2), cy2 = dot(ny, w2);
                        if (cs > 0.f && cy2 > 0.f) {
                            const float3 yo = y + ny * eps_of(y);
                            const float3 r2 = xs - yo;
                            const float l2 = sqrtf(dot(r2, r2));
                            rays++;
                            const RayT ray = make_ray(s, yo, r2 * (1.0f / l2));
                            if (!trace_any<CNT>(s, ray, l2 - eps_of(xs), tc)) {
                                H = yb.w * cy2 * cs * p.fw / (d2 * d2);
                                opl = ya.w + d2;
                            }
                        }
                    }
                }
            }
            if (H > 0.f) {
                contribs++;
                const float x = (opl - p.start) / p.width;
                const bool in = x >= 0.f && x < (float)p.T;
                const int bin = in ? (int)x : -1;
                const float v = H * p.scale;
                if (in) {
                    if (p.aggregate) {
                        if (bin < p.D) splat_add<1, true>(&hist[r * p.D + bin], &v);
                        else splat_add<1, true>(&p.film[(size_t)(row0 + r) * p.T + bin], &v);
                    } else {
                        if (bin < p.D) atomicAdd(&hist[r * p.D + bin], v);
                        else atomicAdd(&p.film[(size_t)(row0 + r) * p.T + bin], v);
                    }
                }
                atomicAdd(&steady_s[r], v);
                if (DUMP) {
                    const unsigned long long slot = atomicAdd(p.dump_count, 1ull);
                    if ((long long)slot < p.dump_cap) {
                        mt_contrib c;
                        c.pixel = (int32_t)(row0 + r);
                        c.sample = (int32_t)smp;
                        c.depth = 2;
                        c.kind = 2;
                        c.tri = tri;
                        c.bin = in ? bin : (int)floorf(x);
                        c.opl = opl;
                        c.c[0] = H;
                        c.c[1] = 0.f;
                        c.c[2] = 0.f;
                        p.dump[slot] = c;
                    }
                }
            }
        }
        __syncthreads();
        const bool acc = p.flags & MT_ACCUMULATE;
        if (p.D == p.T) {
            const size_t n = (size_t)nrows * p.T;
            float *dst = p.film + (size_t)row0 * p.T;
            if (((n | (size_t)row0 * p.T) & 3) == 0 && (((uintptr_t)p.film) & 15) == 0) {
                float4 *d4 = reinterpret_cast<float4 *>(dst);
                const float4 *s4 = reinterpret_cast<const float4 *>(hist);
                for (size_t i = threadIdx.x; i < n / 4; i += blockDim.x) {
                    float4 v = s4[i];
                    if (acc) {
                        const float4 o = d4[i];
                        v = make_float4(v.x + o.x, v.y + o.y, v.z + o.z, v.w + o.w);
                    }
                    d4[i] = v;
                }
            } else {
                for (size_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = acc ? dst[i] + hist[i] : hist[i];
            }
        } else {
            for (int i = threadIdx.x; i < nrows * p.D; i += blockDim.x) {
                const int r = i / p.D, b = i - r * p.D;
                float *d = p.film + (size_t)(row0 + r) * p.T + b;
                *d = acc ? *d + hist[i] : hist[i];
            }
        }
        if (p.steady)
            for (int i = threadIdx.x; i < nrows; i += blockDim.x)
                p.steady[row0 + i] = acc ? p.steady[row0 + i] + steady_s[i] : steady_s[i];
        __syncthreads();
    }
    unsigned long long v[5] = {conns, contribs, rays, tc.nodes, tc.tris};
    const int c_idx[5] = {1, 2, 3, 4, 5};
    for (int c = 0; c < 5; ++c) {
        unsigned long long x = v[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s.counters[c_idx[c]], x);
    }
}

template <bool DUMP, bool CNT>
mt_status launch_nlos(const DevScene &s, const NlosParams &p, const LaunchCfg &cfg, cudaStream_t st) {
    if (p.mode == MT_EXHAUSTIVE) {
        const long long total = (long long)p.n_l * p.spp;
        const int grid = (int)std::min<long long>((total + 255) / 256, (long long)cfg.num_sms * 16);
        k_nlos_ysample<CNT><<<grid, 256, 0, st>>>(s, p);
        MT_CUDA_TRY(cudaGetLastError());
    }
    auto kern = k_nlos<DUMP, CNT>;
    MT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem_bytes));
    int per_sm = 0;
    MT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.threads, cfg.smem_bytes));
    if (per_sm < 1) {
        mt::set_error("nlos kernel does not fit: %d threads, %zu bytes of shared memory", cfg.threads, cfg.smem_bytes);
        return MT_ERR_UNSUPPORTED;
    }
    if (cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, cfg.ctas_per_sm);
    const int grid = std::max(1, std::min(p.n_tiles, per_sm * cfg.num_sms));
    kern<<<grid, cfg.threads, cfg.smem_bytes, st>>>(s, p);
    MT_CUDA_TRY(cudaGetLastError());
    return MT_OK;
}

}  // namespace

mt_status mt_launch_nlos(const DevScene &s, const NlosParams &p, const LaunchCfg &cfg, bool dump, bool counters,
                         cudaStream_t st) {
    if (dump) return counters ? launch_nlos<true, true>(s, p, cfg, st) : launch_nlos<true, false>(s, p, cfg, st);
    return counters ? launch_nlos<false, true>(s, p, cfg, st) : launch_nlos<false, false>(s, p, cfg, st);
}
