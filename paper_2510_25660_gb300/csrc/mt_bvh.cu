// mt_bvh.cu -- SAH BVH builder on the device.
//
// Top-down binned SAH (32 bins per axis, unit traversal and intersection
// costs).  Nodes with more than SMALL_T (256) triangles are split level by level,
// each level binning fixed-size chunks of the node's index range in many CTAs
// (shared-memory bins merged with global atomics), choosing the split with one
// warp per node and partitioning stably per chunk (the partition also gathers
// the children's centroid bounds).  Smaller nodes are built completely by one
// CTA each with an explicit stack and CTA-local node ids.  Leaves hold at most four
// triangles; a node of two to four triangles becomes a leaf when that is
// cheaper under the SAH.  The binary tree is then collapsed into an 8-wide
// tree (each wide node takes a binary node's two children and keeps replacing
// the internal child of largest surface area by its two children while it has
// fewer than eight), the triangles are reordered so that the leaf children of
// every wide node are contiguous, and both trees are written: binary nodes of
// 32 bytes holding both children's boxes as outward-rounded 16-bit planes in
// the scene box, wide nodes of 80 bytes with 8-bit planes in a per-node frame,
// and 48-byte triangle records shared by the two.
#include <cub/cub.cuh>

#include <chrono>
#include <cmath>

#include "mt_common.cuh"
#include "mt_internal.h"
#include "mt_trace.cuh"

namespace {

constexpr int NB = 32;          // bins per axis
// SAH cost of one traversal step relative to one triangle test (leaf decision).
// A triangle test (48-byte record, watertight test) costs more than a node test
// on GB300: 0.5 measured 96.8 ms against 97.6 ms at 1.0 and 107-109 ms at 2-3
// for the 512x512x256-spp forward render of the 1.16M-triangle scene.
#ifndef MT_SAH_CT
#define MT_SAH_CT 0.5f
#endif
// The tree does not depend on this threshold (the same binned SAH decisions are
// taken either way); a CTA steps through its subtree node by node, so smaller
// subtrees shorten the longest CTA: 12.8 ms against 17.7 ms at 2048 for the
// 1.16M-triangle scene.
#ifndef MT_BVH_SMALL_T
#define MT_BVH_SMALL_T 256
#endif
constexpr int SMALL_T = MT_BVH_SMALL_T;  // nodes at or below this size are built by one CTA
constexpr int CHUNK = 4096;     // index positions binned/partitioned per CTA for large nodes
// bins hold counts and boxes only: the children's centroid bounds come from the partition
// pass, which reads every centroid anyway (six more atomics per bin and axis otherwise)
constexpr int BIN_INTS = 7;     // count, box lo3 hi3 (ordered ints)
constexpr int ilog2_ceil(int v) { return v <= 1 ? 0 : 1 + ilog2_ceil((v + 1) / 2); }
// a subtree CTA pushes the larger child below the smaller one and pops the smaller first, so an
// entry waits on the stack only below a descent into a child of at most half its parent's
// triangles: fewer than ceil(log2 SMALL_T) entries wait below the two just pushed
constexpr int SMALL_STACK = ilog2_ceil(SMALL_T) + 4;

struct BNode {
    float lo[3], hi[3];
    int32_t left, right;   // child build ids, -1 for a leaf
    int32_t first, count;  // index range
};

struct Task {
    int32_t node, first, count, depth;
    float clo[3], chi[3];  // centroid bounds
    float box_lo[3], box_hi[3];
};

struct Decision {
    int32_t axis;     // -1: object median without reordering
    int32_t split;    // bins <= split go left
    int32_t nL;
    int32_t cntL, cntR; // partition cursors
    float llo[3], lhi[3], rlo[3], rhi[3];   // child boxes
    float lclo[3], lchi[3], rclo[3], rchi[3]; // child centroid bounds
    int32_t cb[12];  // the same as ordered ints while the partition pass gathers them
};

struct Chunk {
    int32_t task, begin, end;
};

__device__ __forceinline__ int f2o(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// surface area of a box with every operation rounded on its own (no contraction), so that
// each caller gets the same value for the same box
__device__ __forceinline__ float area_of(const float *lo, const float *hi) {
    const float dx = fmaxf(0.f, __fsub_rn(hi[0], lo[0])), dy = fmaxf(0.f, __fsub_rn(hi[1], lo[1])),
                dz = fmaxf(0.f, __fsub_rn(hi[2], lo[2]));
    return __fmul_rn(2.0f, __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx)));
}

// SAH cost of a split, SA_L n_L + SA_R n_R (no contraction: binned and per-triangle
// evaluations of the same split agree to the bit)
__device__ __forceinline__ float split_sah(const float *llo, const float *lhi, int nl, const float *rlo,
                                           const float *rhi, int nr) {
    return __fadd_rn(__fmul_rn(area_of(llo, lhi), (float)nl), __fmul_rn(area_of(rlo, rhi), (float)nr));
}

// bin of a centroid coordinate; identical in the binning and partition passes
__device__ __forceinline__ int bin_of(float c, float lo, float hi) {
    const float ext = hi - lo;
    if (!(ext > 0.f)) return 0;
    const float k = (float)NB / ext;
    int b = (int)((c - lo) * k);
    return b < 0 ? 0 : (b > NB - 1 ? NB - 1 : b);
}

__device__ __forceinline__ void bins_init(int *bins) {
    for (int i = threadIdx.x; i < 3 * NB; i += blockDim.x) {
        int *b = bins + i * BIN_INTS;
        b[0] = 0;
        for (int k = 0; k < 3; ++k) {
            b[1 + k] = f2o(INFINITY);
            b[4 + k] = f2o(-INFINITY);
        }
    }
}

__device__ __forceinline__ void bins_add(int *bins, const float4 lo, const float4 hi, const float4 c, const float *clo,
                                         const float *chi) {
    const float cc[3] = {c.x, c.y, c.z};
    for (int a = 0; a < 3; ++a) {
        const int bi = bin_of(cc[a], clo[a], chi[a]);
        int *b = bins + (a * NB + bi) * BIN_INTS;
        atomicAdd(&b[0], 1);
        atomicMin(&b[1], f2o(lo.x));
        atomicMin(&b[2], f2o(lo.y));
        atomicMin(&b[3], f2o(lo.z));
        atomicMax(&b[4], f2o(hi.x));
        atomicMax(&b[5], f2o(hi.y));
        atomicMax(&b[6], f2o(hi.z));
    }
}

// One warp sweeps the NB bins of one axis; returns (cost, split) of the best
// split (cost = SA_L*nL + SA_R*nR) to all lanes; cost = inf if none is valid.
__device__ __forceinline__ void sweep_axis(const int *bins_axis, float &best_cost, int &best_split) {
    const int lane = threadIdx.x & 31;
    const int *b = bins_axis + lane * BIN_INTS;
    int cnt = b[0];
    float lo[3] = {o2f(b[1]), o2f(b[2]), o2f(b[3])}, hi[3] = {o2f(b[4]), o2f(b[5]), o2f(b[6])};
    // inclusive prefix from the left
    int pc = cnt;
    float plo[3] = {lo[0], lo[1], lo[2]}, phi[3] = {hi[0], hi[1], hi[2]};
    for (int o = 1; o < 32; o <<= 1) {
        const int c2 = __shfl_up_sync(0xffffffffu, pc, o);
        float l2[3], h2[3];
        for (int k = 0; k < 3; ++k) {
            l2[k] = __shfl_up_sync(0xffffffffu, plo[k], o);
            h2[k] = __shfl_up_sync(0xffffffffu, phi[k], o);
        }
        if (lane >= o) {
            pc += c2;
            for (int k = 0; k < 3; ++k) {
                plo[k] = fminf(plo[k], l2[k]);
                phi[k] = fmaxf(phi[k], h2[k]);
            }
        }
    }
    // inclusive suffix from the right
    int sc = cnt;
    float slo[3] = {lo[0], lo[1], lo[2]}, shi[3] = {hi[0], hi[1], hi[2]};
    for (int o = 1; o < 32; o <<= 1) {
        const int c2 = __shfl_down_sync(0xffffffffu, sc, o);
        float l2[3], h2[3];
        for (int k = 0; k < 3; ++k) {
            l2[k] = __shfl_down_sync(0xffffffffu, slo[k], o);
            h2[k] = __shfl_down_sync(0xffffffffu, shi[k], o);
        }
        if (lane + o < 32) {
            sc += c2;
            for (int k = 0; k < 3; ++k) {
                slo[k] = fminf(slo[k], l2[k]);
                shi[k] = fmaxf(shi[k], h2[k]);
            }
        }
    }
    // right side of a split after bin `lane` is the suffix starting at lane+1
    const int rc = __shfl_down_sync(0xffffffffu, sc, 1);
    float rlo[3], rhi[3];
    for (int k = 0; k < 3; ++k) {
        rlo[k] = __shfl_down_sync(0xffffffffu, slo[k], 1);
        rhi[k] = __shfl_down_sync(0xffffffffu, shi[k], 1);
    }
    float cost = INFINITY;
    if (lane < 31 && pc > 0 && rc > 0) cost = split_sah(plo, phi, pc, rlo, rhi, rc);
    int split = lane;
    for (int o = 16; o > 0; o >>= 1) {
        const float c2 = __shfl_xor_sync(0xffffffffu, cost, o);
        const int s2 = __shfl_xor_sync(0xffffffffu, split, o);
        if (c2 < cost || (c2 == cost && s2 < split)) {
            cost = c2;
            split = s2;
        }
    }
    best_cost = cost;
    best_split = split;
}

// block-wide exclusive scan of one int per thread; returns the total
__device__ __forceinline__ int block_exscan(int v, int *s_warp, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    const int before = w > 0 ? s_warp[w - 1] : 0;
    total = s_warp[nw - 1];
    __syncthreads();
    return before + x - v;
}

// centroid bounds of the two sides of a partition, as ordered ints:
// [0, 3) left lower, [3, 6) left upper, [6, 9) right lower, [9, 12) right upper
struct SideBounds {
    int v[12];
    __device__ __forceinline__ void init() {
        for (int k = 0; k < 12; ++k) v[k] = f2o((k / 3) & 1 ? -INFINITY : INFINITY);
    }
    __device__ __forceinline__ void add(const float4 c, bool left) {
        const int o[3] = {f2o(c.x), f2o(c.y), f2o(c.z)};
        const int b = left ? 0 : 6;
        for (int k = 0; k < 3; ++k) {
            v[b + k] = min(v[b + k], o[k]);
            v[b + 3 + k] = max(v[b + 3 + k], o[k]);
        }
    }
    // warp reduction, then lane 0 merges into s (shared, initialised like init())
    __device__ __forceinline__ void merge_into(int *s) const {
        for (int k = 0; k < 12; ++k) {
            const int r = (k / 3) & 1 ? __reduce_max_sync(0xffffffffu, v[k]) : __reduce_min_sync(0xffffffffu, v[k]);
            if ((threadIdx.x & 31) == 0) {
                if ((k / 3) & 1) atomicMax(&s[k], r);
                else atomicMin(&s[k], r);
            }
        }
    }
};

__device__ __forceinline__ void cb_to_decision(const int *cb, Decision &d) {
    for (int k = 0; k < 3; ++k) {
        d.lclo[k] = o2f(cb[k]);
        d.lchi[k] = o2f(cb[3 + k]);
        d.rclo[k] = o2f(cb[6 + k]);
        d.rchi[k] = o2f(cb[9 + k]);
    }
}

// ---------------------------------------------------------------------------
__global__ void k_prim_bounds(const float *tris, int n, float4 *plo, float4 *phi, float4 *cen, int *gbox) {
    __shared__ int sb[12];
    if (threadIdx.x < 12) sb[threadIdx.x] = (threadIdx.x % 6) < 3 ? f2o(INFINITY) : f2o(-INFINITY);
    __syncthreads();
    float l[6] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
    float h[6] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float *t = tris + 9 * (size_t)i;
        float lo[3], hi[3], c[3];
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(t[k], fminf(t[3 + k], t[6 + k]));
            hi[k] = fmaxf(t[k], fmaxf(t[3 + k], t[6 + k]));
            c[k] = (t[k] + t[3 + k] + t[6 + k]) * (1.0f / 3.0f);
            l[k] = fminf(l[k], lo[k]);
            h[k] = fmaxf(h[k], hi[k]);
            l[3 + k] = fminf(l[3 + k], c[k]);
            h[3 + k] = fmaxf(h[3 + k], c[k]);
        }
        plo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
        phi[i] = make_float4(hi[0], hi[1], hi[2], 0.f);
        cen[i] = make_float4(c[0], c[1], c[2], 0.f);
    }
    for (int k = 0; k < 6; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            l[k] = fminf(l[k], __shfl_xor_sync(0xffffffffu, l[k], o));
            h[k] = fmaxf(h[k], __shfl_xor_sync(0xffffffffu, h[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&sb[k], f2o(l[k]));
            atomicMax(&sb[3 + k], f2o(h[k]));
            atomicMin(&sb[6 + k], f2o(l[3 + k]));
            atomicMax(&sb[9 + k], f2o(h[3 + k]));
        }
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        if ((threadIdx.x % 6) < 3) atomicMin(&gbox[threadIdx.x], sb[threadIdx.x]);
        else atomicMax(&gbox[threadIdx.x], sb[threadIdx.x]);
    }
}

__global__ void k_iota(int *idx, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) idx[i] = i;
}

__global__ void k_bin_chunks(const Chunk *chunks, const Task *tasks, const int *idx, const float4 *plo,
                             const float4 *phi, const float4 *cen, int *gbins) {
    __shared__ int bins[3 * NB * BIN_INTS];
    const Chunk ch = chunks[blockIdx.x];
    const Task tk = tasks[ch.task];
    bins_init(bins);
    __syncthreads();
    for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
        const int p = idx[i];
        bins_add(bins, plo[p], phi[p], cen[p], tk.clo, tk.chi);
    }
    __syncthreads();
    int *g = gbins + (size_t)ch.task * 3 * NB * BIN_INTS;
    for (int i = threadIdx.x; i < 3 * NB; i += blockDim.x) {
        const int *b = bins + i * BIN_INTS;
        if (b[0] == 0) continue;
        int *d = g + i * BIN_INTS;
        atomicAdd(&d[0], b[0]);
        for (int k = 0; k < 3; ++k) {
            atomicMin(&d[1 + k], b[1 + k]);
            atomicMax(&d[4 + k], b[4 + k]);
        }
    }
}

__global__ void k_init_bins(int *gbins, int n_tasks) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tasks * 3 * NB; i += gridDim.x * blockDim.x) {
        int *b = gbins + (size_t)i * BIN_INTS;
        b[0] = 0;
        for (int k = 0; k < 3; ++k) {
            b[1 + k] = f2o(INFINITY);
            b[4 + k] = f2o(-INFINITY);
        }
    }
}

// decide a split from bins (one warp); writes *dec (lane 0); returns via dec
__device__ void decide(const int *bins, const Task &tk, Decision *dec) {
    const int lane = threadIdx.x & 31;
    float bc = INFINITY;
    int ba = -1, bs = 0;
    for (int a = 0; a < 3; ++a) {
        float c;
        int s;
        sweep_axis(bins + a * NB * BIN_INTS, c, s);
        if (c < bc) {
            bc = c;
            ba = a;
            bs = s;
        }
    }
    Decision d;
    d.cntL = 0;
    d.cntR = 0;
    if (ba < 0) {
        d.axis = -1;
        d.split = 0;
        d.nL = tk.count / 2;
        for (int k = 0; k < 3; ++k) {
            d.llo[k] = d.rlo[k] = tk.box_lo[k];
            d.lhi[k] = d.rhi[k] = tk.box_hi[k];
            d.lclo[k] = d.rclo[k] = tk.clo[k];
            d.lchi[k] = d.rchi[k] = tk.chi[k];
        }
    } else {
        // lane i holds bin i of the split axis: the children's counts and boxes are warp
        // reductions over the bins on either side (min / max of the ordered ints, so the same
        // values as a sequential union)
        static_assert(NB == 32, "one bin per lane");
        const int *b = bins + (ba * NB + lane) * BIN_INTS;
        const int cnt = b[0];
        const bool left = lane <= bs, has = cnt > 0;
        d.axis = ba;
        d.split = bs;
        d.nL = __reduce_add_sync(0xffffffffu, left ? cnt : 0);
        const int up = f2o(INFINITY), dn = f2o(-INFINITY);  // an empty bin holds these
        for (int k = 0; k < 3; ++k) {
            const int blo = has ? b[1 + k] : up, bhi = has ? b[4 + k] : dn;
            d.llo[k] = o2f(__reduce_min_sync(0xffffffffu, left ? blo : up));
            d.lhi[k] = o2f(__reduce_max_sync(0xffffffffu, left ? bhi : dn));
            d.rlo[k] = o2f(__reduce_min_sync(0xffffffffu, left ? up : blo));
            d.rhi[k] = o2f(__reduce_max_sync(0xffffffffu, left ? dn : bhi));
            d.cb[k] = d.cb[6 + k] = up;  // the centroid bounds are gathered by the partition pass
            d.cb[3 + k] = d.cb[9 + k] = dn;
        }
    }
    if (lane == 0) *dec = d;
}

__global__ void k_choose(const Task *tasks, const int *gbins, Decision *decs) {
    decide(gbins + (size_t)blockIdx.x * 3 * NB * BIN_INTS, tasks[blockIdx.x], &decs[blockIdx.x]);
}

__global__ void k_partition_chunks(const Chunk *chunks, const Task *tasks, Decision *decs, const int *idx,
                                   const float4 *cen, int *tmp) {
    __shared__ int s_warp[32];
    __shared__ int s_base[2];
    __shared__ int s_cb[12];
    const Chunk ch = chunks[blockIdx.x];
    const Task tk = tasks[ch.task];
    Decision *dec = &decs[ch.task];
    const int axis = dec->axis;
    if (axis < 0) return;
    const int split = dec->split, nL = dec->nL;
    SideBounds sb;
    sb.init();
    if (threadIdx.x == 0)
        for (int k = 0; k < 12; ++k) s_cb[k] = sb.v[k];
    for (int base = ch.begin; base < ch.end; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int p = 0, left = 0;
        const bool valid = i < ch.end;
        if (valid) {
            p = idx[i];
            const float4 c = cen[p];
            const float cc = axis == 0 ? c.x : (axis == 1 ? c.y : c.z);
            left = bin_of(cc, tk.clo[axis], tk.chi[axis]) <= split;
            sb.add(c, left);
        }
        int totL;
        const int rankL = block_exscan(valid && left, s_warp, totL);
        const int nvalid = min((int)blockDim.x, ch.end - base);
        if (threadIdx.x == 0) {
            s_base[0] = atomicAdd(&dec->cntL, totL);
            s_base[1] = atomicAdd(&dec->cntR, nvalid - totL);
        }
        __syncthreads();
        if (valid) {
            const int rankR = (int)threadIdx.x - rankL;
            const int dst = left ? tk.first + s_base[0] + rankL : tk.first + nL + s_base[1] + rankR;
            tmp[dst] = p;
        }
        __syncthreads();
    }
    sb.merge_into(s_cb);
    __syncthreads();
    if (threadIdx.x < 12) {
        const int k = threadIdx.x;
        if ((k / 3) & 1) atomicMax(&dec->cb[k], s_cb[k]);
        else atomicMin(&dec->cb[k], s_cb[k]);
    }
}

__global__ void k_copy_chunks(const Chunk *chunks, const Decision *decs, int *idx, const int *tmp) {
    const Chunk ch = chunks[blockIdx.x];
    if (decs[ch.task].axis < 0) return;
    for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) idx[i] = tmp[i];
}

// child s (0 left, 1 right) of task tk under split d, with node id `id`: its task and its node, a leaf
__device__ __forceinline__ void child_of(const Task &tk, const Decision &d, int s, int id, Task &t, BNode &nd) {
    t.node = id;
    t.first = s == 0 ? tk.first : tk.first + d.nL;
    t.count = s == 0 ? d.nL : tk.count - d.nL;
    t.depth = tk.depth + 1;
    for (int k = 0; k < 3; ++k) {
        t.box_lo[k] = s == 0 ? d.llo[k] : d.rlo[k];
        t.box_hi[k] = s == 0 ? d.lhi[k] : d.rhi[k];
        t.clo[k] = s == 0 ? d.lclo[k] : d.rclo[k];
        t.chi[k] = s == 0 ? d.lchi[k] : d.rchi[k];
        nd.lo[k] = t.box_lo[k];
        nd.hi[k] = t.box_hi[k];
    }
    nd.left = nd.right = -1;
    nd.first = t.first;
    nd.count = t.count;
}

__device__ void make_child_tasks(const Task &tk, const Decision &d, int base, BNode *nodes, Task *c) {
    for (int s = 0; s < 2; ++s) {
        BNode nd;
        child_of(tk, d, s, base + s, c[s], nd);
        nodes[base + s] = nd;
    }
    nodes[tk.node].left = base;
    nodes[tk.node].right = base + 1;
}

__global__ void k_children(const Task *tasks, int n_tasks, const Decision *decs, BNode *nodes, int *counters,
                           Task *next, Task *small) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tasks) return;
    const Task tk = tasks[i];
    const int base = atomicAdd(&counters[0], 2);
    Task c[2];
    Decision d = decs[i];
    if (d.axis >= 0) cb_to_decision(d.cb, d);
    make_child_tasks(tk, d, base, nodes, c);
    for (int s = 0; s < 2; ++s) {
        if (c[s].count > SMALL_T) next[atomicAdd(&counters[1], 1)] = c[s];
        else small[atomicAdd(&counters[2], 1)] = c[s];
        atomicMax(&counters[3], c[s].depth);
    }
}

// a task of at most four triangles becomes a leaf when that costs no more than its split
__device__ __forceinline__ bool leaf_better(const Task &tk, const Decision &d) {
    const float sa = area_of(tk.box_lo, tk.box_hi);
    const float split_cost =
        __fadd_rn(__fmul_rn(MT_SAH_CT, sa), split_sah(d.llo, d.lhi, d.nL, d.rlo, d.rhi, tk.count - d.nL));
    return tk.count <= 4 && __fmul_rn(sa, (float)tk.count) <= split_cost;
}

// The binned SAH decision (bins_add, then decide) of a task of at most 32
// triangles, one triangle per lane of a warp, without bins.  Every split that
// binning can choose is the largest occupied bin of its left side (equal-cost
// splits between two occupied bins go to the smallest index), i.e. the bin of
// some triangle: each lane prices the split at its triangle's bin, on all three
// axes in one pass over the triangles (one shuffle of the three bins packed in
// one word and six of the box per triangle), from the same box unions and in
// the same operations, and the warp takes the smallest (cost, split), then the
// first axis of smallest cost, as decide does.  A lane that priced the chosen
// split holds the children's boxes.  bb returns this lane's bins, side its side
// of the chosen split (1: left).
__device__ void decide_small(const Task &tk, const float lo[3], const float hi[3], const float cc[3], bool v,
                             int bb[3], Decision &d, bool &side) {
    for (int a = 0; a < 3; ++a) bb[a] = v ? bin_of(cc[a], tk.clo[a], tk.chi[a]) : NB;
    const int packed = bb[0] | (bb[1] << 6) | (bb[2] << 12);  // bins 0..NB fit six bits
    int nl[3] = {0, 0, 0};
    float L[3][6], R[3][6];  // per axis: lower corner, upper corner of the left / right side
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            L[a][k] = R[a][k] = INFINITY;
            L[a][3 + k] = R[a][3 + k] = -INFINITY;
        }
    for (int j = 0; j < tk.count; ++j) {
        const int pj = __shfl_sync(0xffffffffu, packed, j);
        float bl[3], bh[3];
        for (int k = 0; k < 3; ++k) {
            bl[k] = __shfl_sync(0xffffffffu, lo[k], j);
            bh[k] = __shfl_sync(0xffffffffu, hi[k], j);
        }
        for (int a = 0; a < 3; ++a) {
            const bool inl = ((pj >> (6 * a)) & 63) <= bb[a];
            nl[a] += inl ? 1 : 0;
            for (int k = 0; k < 3; ++k) {
                if (inl) {
                    L[a][k] = fminf(L[a][k], bl[k]);
                    L[a][3 + k] = fmaxf(L[a][3 + k], bh[k]);
                } else {
                    R[a][k] = fminf(R[a][k], bl[k]);
                    R[a][3 + k] = fmaxf(R[a][3 + k], bh[k]);
                }
            }
        }
    }
    float bc = INFINITY;
    int ba = -1, bs = 0;
    for (int a = 0; a < 3; ++a) {
        const int s = bb[a];
        float cost = INFINITY;
        int split = v ? s : NB;
        if (v && s < NB - 1 && nl[a] > 0 && tk.count - nl[a] > 0)
            cost = split_sah(&L[a][0], &L[a][3], nl[a], &R[a][0], &R[a][3], tk.count - nl[a]);
        for (int o = 16; o > 0; o >>= 1) {
            const float c2 = __shfl_xor_sync(0xffffffffu, cost, o);
            const int s2 = __shfl_xor_sync(0xffffffffu, split, o);
            if (c2 < cost || (c2 == cost && s2 < split)) {
                cost = c2;
                split = s2;
            }
        }
        if (cost < bc) {
            bc = cost;
            ba = a;
            bs = split;
        }
    }
    d.cntL = 0;
    d.cntR = 0;
    if (ba < 0) {
        d.axis = -1;
        d.split = 0;
        d.nL = tk.count / 2;
        side = false;
        for (int k = 0; k < 3; ++k) {
            d.llo[k] = d.rlo[k] = tk.box_lo[k];
            d.lhi[k] = d.rhi[k] = tk.box_hi[k];
            d.lclo[k] = d.rclo[k] = tk.clo[k];
            d.lchi[k] = d.rchi[k] = tk.chi[k];
        }
        return;
    }
    const int bsel = ba == 0 ? bb[0] : (ba == 1 ? bb[1] : bb[2]);
    const bool left = v && bsel <= bs, right = v && !left;
    side = left;
    d.axis = ba;
    d.split = bs;
    d.nL = __popc(__ballot_sync(0xffffffffu, left));
    // the lowest lane that priced (ba, bs): its unions are the children's boxes
    const int src = __ffs(__ballot_sync(0xffffffffu, v && bsel == bs)) - 1;
    for (int k = 0; k < 6; ++k) {
        const float l = ba == 0 ? L[0][k] : (ba == 1 ? L[1][k] : L[2][k]);
        const float r = ba == 0 ? R[0][k] : (ba == 1 ? R[1][k] : R[2][k]);
        const float lv = __shfl_sync(0xffffffffu, l, src), rv = __shfl_sync(0xffffffffu, r, src);
        if (k < 3) {
            d.llo[k] = lv;
            d.rlo[k] = rv;
        } else {
            d.lhi[k - 3] = lv;
            d.rhi[k - 3] = rv;
        }
    }
    // centroid bounds of either side: reductions over ordered ints
    for (int k = 0; k < 3; ++k) {
        const int o = f2o(cc[k]);
        d.lclo[k] = o2f(__reduce_min_sync(0xffffffffu, left ? o : f2o(INFINITY)));
        d.lchi[k] = o2f(__reduce_max_sync(0xffffffffu, left ? o : f2o(-INFINITY)));
        d.rclo[k] = o2f(__reduce_min_sync(0xffffffffu, right ? o : f2o(INFINITY)));
        d.rchi[k] = o2f(__reduce_max_sync(0xffffffffu, right ? o : f2o(-INFINITY)));
    }
}

// One CTA builds the whole subtree of a small task, node by node with an
// explicit stack.  The nodes below the task's root get local ids in the CTA's
// own region of `loc` (two slots per triangle of the task: a subtree of c
// triangles has at most 2c - 2 nodes below its root, since every split leaves
// both sides non-empty) and move to `nodes` with one allocation once the
// subtree is complete, so no node step waits on a global atomic.
// Threads of the CTA (any multiple of 32): one warp, so the barriers between
// its node steps cost little (11.0 ms against 12.8 ms at 128 threads for the
// 1.16M-triangle scene; the same tree).
#ifndef MT_BVH_SMALL_THREADS
#define MT_BVH_SMALL_THREADS 32
#endif
__global__ void __launch_bounds__(MT_BVH_SMALL_THREADS) k_build_small(const Task *small, BNode *nodes, BNode *loc_all,
                                                                      int *idx, int *tmp, const float4 *plo,
                                                                      const float4 *phi, const float4 *cen,
                                                                      int *counters) {
    __shared__ int bins[3 * NB * BIN_INTS];
    __shared__ Task stack[SMALL_STACK];
    __shared__ int s_sp, s_next, s_link[2], s_maxd, s_base;
    __shared__ Decision s_dec;
    __shared__ int s_leaf;
    __shared__ int s_warp[32];
    __shared__ Task s_tk;
    const Task root = small[blockIdx.x];
    BNode *loc = loc_all + 2 * (size_t)root.first;
    const int cap = 2 * root.count - 2;
    if (threadIdx.x == 0) {
        stack[0] = root;
        s_sp = 1;
        s_next = 0;
        s_link[0] = s_link[1] = -1;
        s_maxd = root.depth;
    }
    // thread 0: the two children of tk under split d, written as leaves with the next local ids,
    // linked to tk and pushed larger first (the smaller is built first)
    auto split_node = [&](const Task &tk, const Decision &d) {
        if (s_next + 2 > cap) {  // unreachable: both sides of a split are non-empty
            atomicOr(&counters[4], 2);
            return;
        }
        const int lb = s_next;
        s_next = lb + 2;
        Task c[2];
        for (int q = 0; q < 2; ++q) {
            BNode nd;
            child_of(tk, d, q, lb + q, c[q], nd);
            loc[lb + q] = nd;
        }
        if (tk.depth == root.depth) {  // the root keeps its global id
            s_link[0] = lb;
            s_link[1] = lb + 1;
        } else {
            loc[tk.node].left = lb;
            loc[tk.node].right = lb + 1;
        }
        s_maxd = max(s_maxd, tk.depth + 1);
        if (s_sp + 2 <= SMALL_STACK) {
            const int big = c[1].count >= c[0].count ? 1 : 0;
            stack[s_sp++] = c[big];
            stack[s_sp++] = c[1 - big];
        } else {
            atomicOr(&counters[4], 1);  // stack overflow: the children stay leaves
        }
    };
    for (;;) {
        __syncthreads();
        const int sp_now = s_sp;  // every thread reads before thread 0 pops
        __syncthreads();
        if (sp_now == 0) break;
        if (threadIdx.x == 0) s_tk = stack[--s_sp];
        __syncthreads();
        const Task tk = s_tk;
        if (tk.count <= 1) continue;  // a leaf: its node was written as one
        if (MT_BVH_SMALL_THREADS == 32 && tk.count <= 32) {
            // a triangle per lane: the same decision as binning, without bins or barriers
            const bool v = threadIdx.x < tk.count;
            const int p = v ? idx[tk.first + threadIdx.x] : 0;
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, cc[3] = {0.f, 0.f, 0.f};
            if (v) {
                const float4 l4 = plo[p], h4 = phi[p], c4 = cen[p];
                lo[0] = l4.x, lo[1] = l4.y, lo[2] = l4.z;
                hi[0] = h4.x, hi[1] = h4.y, hi[2] = h4.z;
                cc[0] = c4.x, cc[1] = c4.y, cc[2] = c4.z;
            }
            int bb[3];
            Decision d;
            bool side;
            decide_small(tk, lo, hi, cc, v, bb, d, side);
            if (leaf_better(tk, d)) continue;
            if (d.axis >= 0) {  // stable partition in place: left triangles first, each side in order
                const unsigned ml = __ballot_sync(0xffffffffu, side), mr = __ballot_sync(0xffffffffu, v && !side);
                const unsigned lt = (1u << threadIdx.x) - 1u;
                const int dst = side ? tk.first + __popc(ml & lt) : tk.first + d.nL + __popc(mr & lt);
                __syncwarp();
                if (v) idx[dst] = p;
                __syncwarp();
            }
            if (threadIdx.x == 0) split_node(tk, d);
            continue;
        }
        bins_init(bins);
        __syncthreads();
        for (int i = tk.first + threadIdx.x; i < tk.first + tk.count; i += blockDim.x) {
            const int p = idx[i];
            bins_add(bins, plo[p], phi[p], cen[p], tk.clo, tk.chi);
        }
        __syncthreads();
        if (threadIdx.x < 32) decide(bins, tk, &s_dec);
        __syncthreads();
        if (threadIdx.x == 0) s_leaf = leaf_better(tk, s_dec);
        __syncthreads();
        if (s_leaf) continue;
        const int axis = s_dec.axis;
        if (axis >= 0) {
            const int split = s_dec.split, nL = s_dec.nL;
            int cL = 0, cR = 0;
            SideBounds sb;
            sb.init();
            for (int base = tk.first; base < tk.first + tk.count; base += blockDim.x) {
                const int i = base + threadIdx.x;
                const bool valid = i < tk.first + tk.count;
                int p = 0, left = 0;
                if (valid) {
                    p = idx[i];
                    const float4 c = cen[p];
                    const float cc = axis == 0 ? c.x : (axis == 1 ? c.y : c.z);
                    left = bin_of(cc, tk.clo[axis], tk.chi[axis]) <= split;
                    sb.add(c, left);
                }
                int totL;
                const int rankL = block_exscan(valid && left, s_warp, totL);
                const int nvalid = min((int)blockDim.x, tk.first + tk.count - base);
                if (valid) {
                    const int rankR = (int)threadIdx.x - rankL;
                    tmp[left ? tk.first + cL + rankL : tk.first + nL + cR + rankR] = p;
                }
                cL += totL;
                cR += nvalid - totL;
            }
            sb.merge_into(s_dec.cb);  // decide initialised s_dec.cb
            __syncthreads();
            for (int i = tk.first + threadIdx.x; i < tk.first + tk.count; i += blockDim.x) idx[i] = tmp[i];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (s_dec.axis >= 0) cb_to_decision(s_dec.cb, s_dec);
            split_node(tk, s_dec);
        }
        __syncthreads();
    }
    // one allocation for the subtree, then its nodes move to their global ids
    if (threadIdx.x == 0) {
        const int u = s_next;
        const int base = u > 0 ? atomicAdd(&counters[0], u) : 0;
        if (u > 0) {
            nodes[root.node].left = base + s_link[0];
            nodes[root.node].right = base + s_link[1];
        }
        atomicMax(&counters[3], s_maxd);
        s_base = base;
    }
    __syncthreads();
    const int u = s_next, base = s_base;
    for (int i = threadIdx.x; i < u; i += blockDim.x) {
        BNode nd = loc[i];
        if (nd.left >= 0) {
            nd.left += base;
            nd.right += base;
        }
        nodes[base + i] = nd;
    }
}

__global__ void k_internal_flags(const BNode *nodes, int n, int *flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flags[i] = nodes[i].left >= 0 ? 1 : 0;
}

// planes rounded outward and padded by two quantisation steps: (v - lo) / sc evaluated in
// float with directed rounding (toward -inf for a lower plane, +inf for an upper one, with
// the reciprocal of sc rounded the same way), so the plane never moves inward
__device__ __forceinline__ uint32_t qfloor(float v, float lo, float sc) {
    float q = floorf(__fmul_rd(__fsub_rd(v, lo), __frcp_rd(sc))) - 2.0f;
    q = q < 0.0f ? 0.0f : (q > 65535.0f ? 65535.0f : q);
    return (uint32_t)q;
}
__device__ __forceinline__ uint32_t qceil(float v, float lo, float sc) {
    float q = ceilf(__fmul_ru(__fsub_ru(v, lo), __frcp_ru(sc))) + 2.0f;
    q = q < 0.0f ? 0.0f : (q > 65535.0f ? 65535.0f : q);
    return (uint32_t)q;
}

__device__ __forceinline__ uint32_t child_ref(const BNode *nodes, const int *map, int c) {
    const BNode &n = nodes[c];
    if (n.left >= 0) return (uint32_t)map[c];
    if (n.count <= 0) return MT_EMPTY_REF;
    return 0x80000000u | ((uint32_t)(n.count - 1) << 29) | (uint32_t)n.first;
}

__device__ __forceinline__ void quant_box(const BNode &n, const float *qlo, const float *qs, uint32_t *q) {
    const bool empty = n.left < 0 && n.count <= 0;  // inverted planes: never hit
    for (int k = 0; k < 3; ++k) {
        q[k] = empty ? 65535u : qfloor(n.lo[k], qlo[k], qs[k]);
        q[3 + k] = empty ? 0u : qceil(n.hi[k], qlo[k], qs[k]);
    }
}

__global__ void k_emit(const BNode *nodes, int n, const int *map, const int *flags, uint4 *out, float qlx, float qly,
                       float qlz, float qsx, float qsy, float qsz) {
    const float qlo[3] = {qlx, qly, qlz}, qs[3] = {qsx, qsy, qsz};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        const BNode &nd = nodes[i];
        uint32_t a[6], b[6];
        quant_box(nodes[nd.left], qlo, qs, a);
        quant_box(nodes[nd.right], qlo, qs, b);
        const int m = map[i];
        // a[k] = lower plane, a[3 + k] = upper plane of axis k
        out[2 * m] = make_uint4(a[0] | (a[3] << 16), a[1] | (a[4] << 16), a[2] | (a[5] << 16), b[0] | (b[3] << 16));
        out[2 * m + 1] = make_uint4(b[1] | (b[4] << 16), b[2] | (b[5] << 16), child_ref(nodes, map, nd.left),
                                    child_ref(nodes, map, nd.right));
    }
}

// Depth-first preorder of the internal nodes (a node, its left subtree, its
// right subtree), so that a node's left child is stored right after it and a
// descent into it usually reads the cache line its parent arrived in.  Walks
// up the tree are bounded by MT_BVH_WALK steps (the tree depth is checked to be
// below the traversal stack first); a longer walk sets bit 1 of *bad.
#ifndef MT_BVH_DFS
#define MT_BVH_DFS 1
#endif
#define MT_BVH_WALK 256

__device__ __forceinline__ bool bn_internal(const BNode *nodes, int i) { return nodes[i].left >= 0; }

__global__ void k_parents(const BNode *nodes, int n, int *parent) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const BNode &b = nodes[i];
        if (b.left >= 0) {
            parent[b.left] = i;
            parent[b.right] = i;
        }
    }
}

// internal-node counts of every subtree, bottom-up: a walk starts at each
// internal node without internal children and climbs while it is the last of
// its parent's internal children to arrive
__global__ void k_subtree_sizes(const BNode *nodes, int n, const int *parent, int *cnt, int *arrive, int *bad) {
    volatile int *vc = cnt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!bn_internal(nodes, i) || bn_internal(nodes, nodes[i].left) || bn_internal(nodes, nodes[i].right)) continue;
        int node = i;
        vc[node] = 1;
        for (int step = 0;; ++step) {
            if (step >= MT_BVH_WALK) {
                atomicOr(bad, 2);
                break;
            }
            const int p = parent[node];
            if (p < 0) break;
            const int l = nodes[p].left, r = nodes[p].right;
            const bool il = bn_internal(nodes, l), ir = bn_internal(nodes, r);
            const int need = (il ? 1 : 0) + (ir ? 1 : 0);
            __threadfence();
            if (atomicAdd(&arrive[p], 1) + 1 < need) break;  // the other child's walk finishes p
            __threadfence();
            vc[p] = 1 + (il ? vc[l] : 0) + (ir ? vc[r] : 0);
            node = p;
        }
    }
}

// preorder rank of every internal node: the sum, over its ancestors, of one
// (the ancestor) plus the left sibling's subtree where the path turns right
__global__ void k_preorder(const BNode *nodes, int n, const int *parent, const int *cnt, int *map, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!bn_internal(nodes, i)) continue;
        int pre = 0, node = i;
        for (int step = 0;; ++step) {
            if (step >= MT_BVH_WALK) {
                atomicOr(bad, 2);
                break;
            }
            const int p = parent[node];
            if (p < 0) break;
            const int l = nodes[p].left;
            pre += 1 + ((node != l && bn_internal(nodes, l)) ? cnt[l] : 0);
            node = p;
        }
        map[i] = pre;
    }
}

__global__ void k_emit_root_leaf(const BNode *nodes, uint4 *out, float qlx, float qly, float qlz, float qsx, float qsy,
                                 float qsz) {
    const float qlo[3] = {qlx, qly, qlz}, qs[3] = {qsx, qsy, qsz};
    uint32_t a[6];
    quant_box(nodes[0], qlo, qs, a);
    const uint32_t ref = 0x80000000u | ((uint32_t)(nodes[0].count - 1) << 29) | (uint32_t)nodes[0].first;
    // child 1 is empty: lower plane 65535 above upper plane 0 on every axis
    out[0] = make_uint4(a[0] | (a[3] << 16), a[1] | (a[4] << 16), a[2] | (a[5] << 16), 0xFFFFu);
    out[1] = make_uint4(0xFFFFu, 0xFFFFu, ref, MT_EMPTY_REF);
}

// One thread per wide node of the current level: collapse the binary subtree
// below binary node wsrc[w] into up to eight children, give the children
// slots by position, quantise their boxes, allocate the internal children
// (wsrc of the next level), place the leaf triangles, record the new triangle
// order in perm and point the binary leaves at it.  The triangles of every
// wide subtree occupy one range in depth-first order: the subtree of wide node
// w starts at wstart[w] with the leaf children of w (in slot order), followed
// by the subtrees of its internal children in slot order, so the order does
// not depend on which thread runs first.
__global__ void k_wide_collapse(BNode *nodes, const int *idx, int n_tris, int begin, int end, int *wsrc, int *wstart,
                                uint4 *wnodes, int *wcount, int *perm, int e_min) {
    for (int w = begin + blockIdx.x * blockDim.x + threadIdx.x; w < end; w += gridDim.x * blockDim.x) {
        const int b = wsrc[w];
        int ch[8];
        int n = 0;
        if (nodes[b].left < 0) {
            ch[n++] = b;  // the root is a leaf
        } else {
            ch[n++] = nodes[b].left;
            ch[n++] = nodes[b].right;
        }
        while (n < 8) {
            int best = -1;
            float ba = -1.0f;
            for (int i = 0; i < n; ++i) {
                const BNode &c = nodes[ch[i]];
                if (c.left < 0) continue;
                const float a = area_of(c.lo, c.hi);
                if (a > ba) {
                    ba = a;
                    best = i;
                }
            }
            if (best < 0) break;
            const int c = ch[best];
            ch[best] = nodes[c].left;
            ch[n++] = nodes[c].right;
        }
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        float cc[8][3];  // child centroids relative to the node centre (only rank the slot choices)
        for (int i = 0; i < n; ++i) {
            const BNode &c = nodes[ch[i]];
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], (double)c.lo[k]);
                hi[k] = fmax(hi[k], (double)c.hi[k]);
            }
        }
        for (int i = 0; i < n; ++i) {
            const BNode &c = nodes[ch[i]];
            for (int k = 0; k < 3; ++k) cc[i][k] = 0.5f * (c.lo[k] + c.hi[k]) - (float)(0.5 * (lo[k] + hi[k]));
        }
        // per-axis step 2^e >= extent / 250 (and >= 2^e_min); origin two steps below
        int e[3];
        double inv_step[3];
        float p[3];
        for (int k = 0; k < 3; ++k) {
            const double ext = hi[k] - lo[k];
            int ek = e_min;
            if (ext > 0.0) ek = max(e_min, ilogb(ext / 250.0) - 1);  // at most the answer: the loop ends it
            while (ek < 127 && ldexp(250.0, ek) < ext) ++ek;
            e[k] = ek;
            inv_step[k] = ldexp(1.0, -ek);  // exact: the planes below divide by a power of two
            p[k] = (float)(lo[k] - 2.0 * ldexp(1.0, ek));
        }
        // slots: greedily pair the child and corner whose centroid offset
        // points most toward that corner
        int slot_child[8];
        for (int q = 0; q < 8; ++q) slot_child[q] = -1;
        bool used[8] = {false, false, false, false, false, false, false, false};
        for (int round = 0; round < n; ++round) {
            float bestc = INFINITY;
            int bi = -1, bq = -1;
            for (int i = 0; i < n; ++i) {
                if (used[i]) continue;
                for (int q = 0; q < 8; ++q) {
                    if (slot_child[q] >= 0) continue;
                    float c = 0.0f;
                    for (int k = 0; k < 3; ++k) {
                        const float off = cc[i][k];
                        c -= ((q >> k) & 1) ? off : -off;
                    }
                    if (c < bestc) {
                        bestc = c;
                        bi = i;
                        bq = q;
                    }
                }
            }
            used[bi] = true;
            slot_child[bq] = bi;
        }
        int n_int = 0, n_leaf_tris = 0;
        for (int i = 0; i < n; ++i) {
            if (nodes[ch[i]].left >= 0) ++n_int;
            else n_leaf_tris += max(0, nodes[ch[i]].count);
        }
        const int base = n_int ? atomicAdd(&wcount[0], n_int) : 0;
        const int tbase = wstart[w];
        if (n_leaf_tris) atomicAdd(&wcount[1], n_leaf_tris);  // the host checks that all triangles are placed
        int tnext = tbase + n_leaf_tris;  // the first internal child's subtree follows the leaf triangles
        uint32_t imask = 0, meta[2] = {0, 0}, ql[3][2] = {{0, 0}, {0, 0}, {0, 0}}, qh[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        int r_int = 0, off = 0;
        for (int q = 0; q < 8; ++q) {
            const int sh = 8 * (q & 3), h = q >> 2;
            if (slot_child[q] < 0) {
                for (int k = 0; k < 3; ++k) ql[k][h] |= 255u << sh;
                continue;
            }
            const int c = ch[slot_child[q]];
            BNode &cn = nodes[c];
            if (cn.left < 0 && cn.count <= 0) {  // an empty leaf stays an empty slot
                for (int k = 0; k < 3; ++k) ql[k][h] |= 255u << sh;
                continue;
            }
            for (int k = 0; k < 3; ++k) {
                double a = floor(((double)cn.lo[k] - (double)p[k]) * inv_step[k]) - 2.0;
                double z = ceil(((double)cn.hi[k] - (double)p[k]) * inv_step[k]) + 2.0;
                a = a < 0.0 ? 0.0 : a;
                z = z > 255.0 ? 255.0 : z;  // unreachable: extent / step <= 250
                ql[k][h] |= (uint32_t)a << sh;
                qh[k][h] |= (uint32_t)z << sh;
            }
            if (cn.left >= 0) {
                imask |= 1u << q;
                wstart[base + r_int] = tnext;
                tnext += cn.count;
                wsrc[base + r_int++] = c;
            } else {
                if (tbase < 0 || tbase + off + cn.count > n_tris) {  // inconsistent counts: the host check fails
                    atomicAdd(&wcount[1], n_tris + 1);
                    continue;
                }
                meta[h] |= (0x80u | ((uint32_t)(cn.count - 1) << 5) | (uint32_t)off) << sh;
                for (int j = 0; j < cn.count; ++j) perm[tbase + off + j] = idx[cn.first + j];
                cn.first = tbase + off;
                off += cn.count;
            }
        }
        uint4 *o = wnodes + MT_WIDE_WORDS * (size_t)w;
        o[0] = make_uint4(__float_as_uint(p[0]), __float_as_uint(p[1]), __float_as_uint(p[2]),
                          (uint32_t)(e[0] + 127) | ((uint32_t)(e[1] + 127) << 8) | ((uint32_t)(e[2] + 127) << 16) |
                              (imask << 24));
        o[1] = make_uint4((uint32_t)base, (uint32_t)tbase, meta[0], meta[1]);
        o[2] = make_uint4(ql[0][0], ql[0][1], ql[1][0], ql[1][1]);
        o[3] = make_uint4(ql[2][0], ql[2][1], qh[0][0], qh[0][1]);
        o[4] = make_uint4(qh[1][0], qh[1][1], qh[2][0], qh[2][1]);
    }
}

// every internal child index in range, leaf triangles inside [0, n)
__global__ void k_wide_validate(const uint4 *w, int nw, int n, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        const uint4 a = w[MT_WIDE_WORDS * (size_t)i], b = w[MT_WIDE_WORDS * (size_t)i + 1];
        const uint32_t imask = a.w >> 24;
        if (imask && ((uint64_t)b.x + __popc(imask) > (uint64_t)nw || b.x == 0u)) atomicOr(bad, 4);
        for (int q = 0; q < 8; ++q) {
            const uint32_t m = ((q < 4 ? b.z : b.w) >> (8 * (q & 3))) & 0xFFu;
            if (!(imask >> q & 1u) && (m & 0x80u)) {
                const uint64_t last = (uint64_t)b.y + (m & 31u) + ((m >> 5) & 3u);
                if (last >= (uint64_t)n) atomicOr(bad, 8);
            }
        }
    }
}

__global__ void k_reorder(const float *tris, const int *idx, int n, float4 *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int p = idx[k];
        const float *t = tris + 9 * (size_t)p;
        out[3 * k] = make_float4(t[0], t[1], t[2], __int_as_float(p));
        out[3 * k + 1] = make_float4(t[3], t[4], t[5], 0.f);
        out[3 * k + 2] = make_float4(t[6], t[7], t[8], 0.f);
    }
}

__global__ void k_sah(const BNode *nodes, int n, double inv_root, double *acc) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const BNode &nd = nodes[i];
        const double a = area_of(nd.lo, nd.hi) * inv_root;
        s += nd.left >= 0 ? a : a * nd.count;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// every child reference in range and every triangle in exactly one leaf slot
__global__ void k_validate(const uint4 *nodes, int n_int, int n, int *bad, unsigned long long *leaf_sum) {
    unsigned long long cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_int; i += gridDim.x * blockDim.x) {
        const uint4 a = nodes[2 * i], b = nodes[2 * i + 1];
        const uint32_t refs[2] = {b.z, b.w};
        // an empty child must have inverted planes on every axis (the traversal relies on it)
        const uint32_t words[2][3] = {{a.x, a.y, a.z}, {a.w, b.x, b.y}};
        for (int c = 0; c < 2; ++c) {
            const uint32_t r = refs[c];
            if (r == MT_EMPTY_REF) {
                for (int k = 0; k < 3; ++k)
                    if ((words[c][k] & 0xFFFFu) <= (words[c][k] >> 16)) atomicOr(bad, 16);
                continue;
            }
            if (!(r & 0x80000000u)) {
                if (r >= (uint32_t)n_int || r == 0u) atomicOr(bad, 1);
            } else {
                const uint32_t first = r & 0x1FFFFFFFu, k = ((r >> 29) & 3u) + 1u;
                if ((unsigned long long)first + k > (unsigned long long)n) atomicOr(bad, 2);
                cnt += k;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(leaf_sum, cnt);
}

}  // namespace

mt_status mt_build_bvh(const float *d_tris, int32_t n, cudaStream_t st, mt::AllocList &al, BvhResult *out) {
    auto t0 = std::chrono::steady_clock::now();
    mt::AllocList tmpal;  // temporaries: stream-ordered, returned to the pool when the build ends
    tmpal.stream_ordered = true;
    tmpal.stream = st;
    struct Guard {
        mt::AllocList &a;
        ~Guard() { a.free_all(); }
    } guard{tmpal};
    float4 *plo, *phi, *cen;
    int *idx, *tmp, *gbox, *counters, *flags, *map;
    BNode *nodes;
    Task *taskA, *taskB, *small;
    const int max_nodes = 2 * n + 2;
    MT_TRY(tmpal.alloc(&plo, n, "bvh prim boxes"));
    MT_TRY(tmpal.alloc(&phi, n, "bvh prim boxes"));
    MT_TRY(tmpal.alloc(&cen, n, "bvh centroids"));
    MT_TRY(tmpal.alloc(&idx, n, "bvh index"));
    MT_TRY(tmpal.alloc(&tmp, n, "bvh index"));
    MT_TRY(tmpal.alloc(&gbox, 12, "bvh box"));
    MT_TRY(tmpal.alloc(&counters, 8, "bvh counters"));
    MT_TRY(tmpal.alloc(&nodes, max_nodes, "bvh build nodes"));
    MT_TRY(tmpal.alloc(&flags, max_nodes, "bvh flags"));
    MT_TRY(tmpal.alloc(&map, max_nodes, "bvh map"));
    const int max_tasks = n / SMALL_T + 4;
    MT_TRY(tmpal.alloc(&taskA, max_tasks, "bvh tasks"));
    MT_TRY(tmpal.alloc(&taskB, max_tasks, "bvh tasks"));
    MT_TRY(tmpal.alloc(&small, n + 2, "bvh small tasks"));

    // scene box and centroid box
    {
        int init[12];
        for (int k = 0; k < 12; ++k) {
            const float v = (k % 6) < 3 ? INFINITY : -INFINITY;
            int i;
            memcpy(&i, &v, 4);
            init[k] = i >= 0 ? i : i ^ 0x7FFFFFFF;
        }
        MT_CUDA_TRY(cudaMemcpyAsync(gbox, init, sizeof(init), cudaMemcpyHostToDevice, st));
    }
    const int nb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    k_prim_bounds<<<nb, 256, 0, st>>>(d_tris, n, plo, phi, cen, gbox);
    k_iota<<<nb, 256, 0, st>>>(idx, n);
    MT_CUDA_TRY(cudaMemsetAsync(counters, 0, 8 * sizeof(int), st));
    int hbox[12];
    MT_CUDA_TRY(cudaMemcpyAsync(hbox, gbox, sizeof(hbox), cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    float box[12];
    for (int k = 0; k < 12; ++k) {
        int i = hbox[k];
        i = i >= 0 ? i : i ^ 0x7FFFFFFF;
        memcpy(&box[k], &i, 4);
    }
    Task root;
    root.node = 0;
    root.first = 0;
    root.count = n;
    root.depth = 0;
    for (int k = 0; k < 3; ++k) {
        root.box_lo[k] = box[k];
        root.box_hi[k] = box[3 + k];
        root.clo[k] = box[6 + k];
        root.chi[k] = box[9 + k];
        out->scene_lo[k] = box[k];
        out->scene_hi[k] = box[3 + k];
    }
    {
        BNode rn;
        for (int k = 0; k < 3; ++k) {
            rn.lo[k] = box[k];
            rn.hi[k] = box[3 + k];
        }
        rn.left = rn.right = -1;
        rn.first = 0;
        rn.count = n;
        MT_CUDA_TRY(cudaMemcpyAsync(nodes, &rn, sizeof(rn), cudaMemcpyHostToDevice, st));
    }
    int hc[8] = {1, 0, 0, 0, 0, 0, 0, 0};
    std::vector<Task> large;
    if (n > SMALL_T) large.push_back(root);
    else {
        MT_CUDA_TRY(cudaMemcpyAsync(small, &root, sizeof(Task), cudaMemcpyHostToDevice, st));
        hc[2] = 1;
    }
    MT_CUDA_TRY(cudaMemcpyAsync(counters, hc, sizeof(hc), cudaMemcpyHostToDevice, st));

    int *gbins = nullptr;
    Decision *decs = nullptr;
    Chunk *dchunks = nullptr;
    const int max_chunks = n / CHUNK + max_tasks + 4;
    MT_TRY(tmpal.alloc(&gbins, (size_t)max_tasks * 3 * NB * BIN_INTS, "bvh bins"));
    MT_TRY(tmpal.alloc(&decs, max_tasks, "bvh decisions"));
    MT_TRY(tmpal.alloc(&dchunks, max_chunks, "bvh chunks"));
    std::vector<Chunk> chunks;
    while (!large.empty()) {
        const int nt = (int)large.size();
        chunks.clear();
        for (int t = 0; t < nt; ++t)
            for (int b = large[t].first; b < large[t].first + large[t].count; b += CHUNK)
                chunks.push_back(Chunk{t, b, std::min(b + CHUNK, large[t].first + large[t].count)});
        const int nc = (int)chunks.size();
        MT_CUDA_TRY(cudaMemcpyAsync(taskA, large.data(), nt * sizeof(Task), cudaMemcpyHostToDevice, st));
        MT_CUDA_TRY(cudaMemcpyAsync(dchunks, chunks.data(), nc * sizeof(Chunk), cudaMemcpyHostToDevice, st));
        k_init_bins<<<std::min(1024, (nt * 3 * NB + 255) / 256), 256, 0, st>>>(gbins, nt);
        k_bin_chunks<<<nc, 512, 0, st>>>(dchunks, taskA, idx, plo, phi, cen, gbins);
        k_choose<<<nt, 32, 0, st>>>(taskA, gbins, decs);
        k_partition_chunks<<<nc, 512, 0, st>>>(dchunks, taskA, decs, idx, cen, tmp);
        k_copy_chunks<<<nc, 512, 0, st>>>(dchunks, decs, idx, tmp);
        MT_CUDA_TRY(cudaMemsetAsync(counters + 1, 0, sizeof(int), st));
        k_children<<<(nt + 127) / 128, 128, 0, st>>>(taskA, nt, decs, nodes, counters, taskB, small);
        MT_CUDA_TRY(cudaGetLastError());
        MT_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        large.resize(hc[1]);
        if (hc[1] > 0) {
            MT_CUDA_TRY(cudaMemcpyAsync(large.data(), taskB, hc[1] * sizeof(Task), cudaMemcpyDeviceToHost, st));
            MT_CUDA_TRY(cudaStreamSynchronize(st));
        }
    }
    if (hc[2] > 0) {
        BNode *loc;
        MT_TRY(tmpal.alloc(&loc, (size_t)2 * n, "bvh subtree nodes"));
        k_build_small<<<hc[2], MT_BVH_SMALL_THREADS, 0, st>>>(small, nodes, loc, idx, tmp, plo, phi, cen, counters);
    }
    MT_CUDA_TRY(cudaGetLastError());
    MT_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    if (hc[4]) {
        mt::set_error("BVH build stack overflow");
        return MT_ERR_INTERNAL;
    }
    const int n_build = hc[0];
    out->depth = hc[3] + 1;
    if (out->depth > MT_STACK - 2) {
        mt::set_error("BVH depth %d exceeds the traversal stack (%d)", out->depth, MT_STACK);
        return MT_ERR_UNSUPPORTED;
    }

    // quantisation frame: scene box mapped into [3, 65532] so that the
    // outward-rounded, two-step padded planes never clamp
    double ext[3], mx = 0.0;
    for (int k = 0; k < 3; ++k) {
        ext[k] = (double)box[3 + k] - (double)box[k];
        mx = std::max(mx, ext[k]);
    }
    for (int k = 0; k < 3; ++k) {
        const double e = std::max(std::max(ext[k], 1e-4 * mx), 1e-12) * (1.0 + 1.0 / 1024.0);
        out->q_scale[k] = (float)(e / 65529.0);
        out->q_lo[k] = (float)((double)box[k] - 3.0 * (double)out->q_scale[k]);
    }

    // 8-wide tree, level by level; the leaves' triangle ranges move to the
    // wide order (perm) before the binary nodes are written
    {
        int *wsrc, *wstart, *wcount, *perm, *dbad;
        uint4 *wtmp;
        const int max_w = std::max(1, n_build);
        MT_TRY(tmpal.alloc(&wsrc, max_w, "wide bvh sources"));
        MT_TRY(tmpal.alloc(&wstart, max_w, "wide bvh triangle ranges"));
        MT_TRY(tmpal.alloc(&wtmp, (size_t)MT_WIDE_WORDS * max_w, "wide bvh nodes"));
        MT_TRY(tmpal.alloc(&wcount, 2, "wide bvh counters"));
        MT_TRY(tmpal.alloc(&perm, n, "wide bvh order"));
        MT_TRY(tmpal.alloc(&dbad, 1, "wide bvh check"));
        const int hw[2] = {1, 0}, zero = 0;
        MT_CUDA_TRY(cudaMemcpyAsync(wcount, hw, sizeof(hw), cudaMemcpyHostToDevice, st));
        MT_CUDA_TRY(cudaMemcpyAsync(wsrc, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        MT_CUDA_TRY(cudaMemcpyAsync(wstart, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        // smallest step: 2^-16 of the largest scene extent, far above the
        // rounding of the slab distances
        double mxe = 0.0;
        for (int k = 0; k < 3; ++k) mxe = std::max(mxe, (double)box[3 + k] - (double)box[k]);
        int e_min = -126;
        if (mxe > 0.0) e_min = std::max(-126, (int)std::ceil(std::log2(mxe)) - 16);
        int begin = 0, end = 1, levels = 0, hcount[2] = {1, 0};
        while (begin < end) {
            const int nl = end - begin;
            k_wide_collapse<<<std::min(4096, (nl + 127) / 128), 128, 0, st>>>(nodes, idx, n, begin, end, wsrc, wstart, wtmp,
                                                                              wcount, perm, e_min);
            MT_CUDA_TRY(cudaGetLastError());
            MT_CUDA_TRY(cudaMemcpyAsync(hcount, wcount, sizeof(hcount), cudaMemcpyDeviceToHost, st));
            MT_CUDA_TRY(cudaStreamSynchronize(st));
            begin = end;
            end = hcount[0];
            if (++levels > MT_STACK || end > max_w) {
                mt::set_error("wide BVH collapse did not terminate (%d levels, %d nodes)", levels, end);
                return MT_ERR_INTERNAL;
            }
        }
        if (hcount[1] != n) {
            mt::set_error("wide BVH holds %d of %d triangles", hcount[1], n);
            return MT_ERR_INTERNAL;
        }
        out->n_wnodes = end;
        MT_TRY(al.alloc(&out->wnodes, (size_t)MT_WIDE_WORDS * end, "wide bvh nodes"));
        MT_CUDA_TRY(cudaMemcpyAsync(out->wnodes, wtmp, (size_t)MT_WIDE_WORDS * end * sizeof(uint4),
                                    cudaMemcpyDeviceToDevice, st));
        MT_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), st));
        k_wide_validate<<<std::min(1024, (end + 255) / 256), 256, 0, st>>>(out->wnodes, end, n, dbad);
        int hbad = 0;
        MT_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad) {
            mt::set_error("wide BVH validation failed (flags %d)", hbad);
            return MT_ERR_INTERNAL;
        }
        std::swap(idx, perm);  // perm is freed with the other temporaries
    }

    // internal nodes -> dense compact nodes
    k_internal_flags<<<std::min(1024, (n_build + 255) / 256), 256, 0, st>>>(nodes, n_build, flags);
    size_t scan_bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, flags, map, n_build, st);
    void *scan_tmp = nullptr;
    MT_TRY(tmpal.alloc((char **)&scan_tmp, scan_bytes, "bvh scan"));
    MT_CUDA_TRY(cub::DeviceScan::ExclusiveSum(scan_tmp, scan_bytes, flags, map, n_build, st));
    int last_map = 0, last_flag = 0;
    MT_CUDA_TRY(cudaMemcpyAsync(&last_map, map + n_build - 1, 4, cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaMemcpyAsync(&last_flag, flags + n_build - 1, 4, cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    int n_int = last_map + last_flag;
    const bool root_leaf = n_int == 0;
    if (root_leaf) n_int = 1;
#if MT_BVH_DFS
    if (!root_leaf) {  // renumber the internal nodes in depth-first preorder (root stays 0)
        int *parent, *cnt, *arrive, *dbad;
        MT_TRY(tmpal.alloc(&parent, n_build, "bvh parents"));
        MT_TRY(tmpal.alloc(&cnt, n_build, "bvh subtree sizes"));
        MT_TRY(tmpal.alloc(&arrive, n_build, "bvh subtree sizes"));
        MT_TRY(tmpal.alloc(&dbad, 1, "bvh order check"));
        MT_CUDA_TRY(cudaMemsetAsync(parent, 0xFF, (size_t)n_build * sizeof(int), st));
        MT_CUDA_TRY(cudaMemsetAsync(arrive, 0, (size_t)n_build * sizeof(int), st));
        MT_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), st));
        const int g = std::min(2048, (n_build + 255) / 256);
        k_parents<<<g, 256, 0, st>>>(nodes, n_build, parent);
        k_subtree_sizes<<<g, 256, 0, st>>>(nodes, n_build, parent, cnt, arrive, dbad);
        k_preorder<<<g, 256, 0, st>>>(nodes, n_build, parent, cnt, map, dbad);
        MT_CUDA_TRY(cudaGetLastError());
        int hbad = 0, hroot = 0;
        MT_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaMemcpyAsync(&hroot, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad || hroot != n_int) {
            mt::set_error("BVH depth-first order failed (flags %d, %d of %d internal nodes)", hbad, hroot, n_int);
            return MT_ERR_INTERNAL;
        }
    }
#endif
    MT_TRY(al.alloc(&out->nodes, (size_t)2 * n_int, "bvh nodes"));
    MT_TRY(al.alloc(&out->tris, (size_t)3 * n, "bvh triangles"));
    if (root_leaf)
        k_emit_root_leaf<<<1, 1, 0, st>>>(nodes, out->nodes, out->q_lo[0], out->q_lo[1], out->q_lo[2],
                                          out->q_scale[0], out->q_scale[1], out->q_scale[2]);
    else
        k_emit<<<std::min(2048, (n_build + 255) / 256), 256, 0, st>>>(nodes, n_build, map, flags, out->nodes,
                                                                      out->q_lo[0], out->q_lo[1], out->q_lo[2],
                                                                      out->q_scale[0], out->q_scale[1],
                                                                      out->q_scale[2]);
    k_reorder<<<std::min(2048, (n + 255) / 256), 256, 0, st>>>(d_tris, idx, n, out->tris);
    {
        int *dbad;
        unsigned long long *dsum;
        MT_TRY(tmpal.alloc(&dbad, 1, "bvh check"));
        MT_TRY(tmpal.alloc(&dsum, 1, "bvh check"));
        MT_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), st));
        MT_CUDA_TRY(cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), st));
        k_validate<<<std::min(1024, (n_int + 255) / 256), 256, 0, st>>>(out->nodes, n_int, n, dbad, dsum);
        int hbad = 0;
        unsigned long long hsum = 0;
        MT_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaMemcpyAsync(&hsum, dsum, sizeof(hsum), cudaMemcpyDeviceToHost, st));
        MT_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad || hsum != (unsigned long long)n) {
            mt::set_error("BVH validation failed (flags %d, %llu leaf slots for %d triangles)", hbad, hsum, n);
            return MT_ERR_INTERNAL;
        }
    }
    double *dsah;
    MT_TRY(tmpal.alloc(&dsah, 1, "bvh sah"));
    MT_CUDA_TRY(cudaMemsetAsync(dsah, 0, sizeof(double), st));
    float rlo[3] = {box[0], box[1], box[2]}, rhi[3] = {box[3], box[4], box[5]};
    const double ra = 2.0 * ((double)(rhi[0] - rlo[0]) * (rhi[1] - rlo[1]) + (double)(rhi[1] - rlo[1]) * (rhi[2] - rlo[2]) +
                             (double)(rhi[2] - rlo[2]) * (rhi[0] - rlo[0]));
    k_sah<<<std::min(1024, (n_build + 255) / 256), 256, 0, st>>>(nodes, n_build, ra > 0 ? 1.0 / ra : 0.0, dsah);
    MT_CUDA_TRY(cudaGetLastError());
    MT_CUDA_TRY(cudaMemcpyAsync(&out->sah, dsah, sizeof(double), cudaMemcpyDeviceToHost, st));
    MT_CUDA_TRY(cudaStreamSynchronize(st));
    out->n_nodes = n_int;
    out->build_us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    return MT_OK;
}
