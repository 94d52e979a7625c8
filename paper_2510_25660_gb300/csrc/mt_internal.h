// mt_internal.h -- host-side helpers shared by the libmt translation units:
// thread-local error messages, checked CUDA calls and device allocation with
// optional host-side fault injection (MT_FAULT_INJECT=alloc:<n> makes the n-th
// device allocation of the process fail, 1-based; used by the fault tests,
// which never fault a GPU).
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mt_api.h"

namespace mt {

void set_error(const char *fmt, ...);
const char *get_error();

mt_status alloc_device(void **p, size_t bytes, const char *what);
// stream-ordered allocation from the device's default memory pool (which keeps
// freed memory for reuse), for temporaries used on one stream only
mt_status alloc_device_async(void **p, size_t bytes, const char *what, cudaStream_t st);

struct AllocList {
    std::vector<void *> ptrs;
    bool stream_ordered = false;  // allocate and free on `stream` (temporaries)
    cudaStream_t stream = nullptr;
    template <class T>
    mt_status alloc(T **p, size_t count, const char *what) {
        void *q = nullptr;
        const size_t bytes = count * sizeof(T) + (count == 0 ? 16 : 0);
        mt_status st = stream_ordered ? alloc_device_async(&q, bytes, what, stream) : alloc_device(&q, bytes, what);
        if (st != MT_OK) return st;
        ptrs.push_back(q);
        *p = (T *)q;
        return MT_OK;
    }
    void free_all() {
        for (void *p : ptrs) {
            if (stream_ordered) cudaFreeAsync(p, stream);
            else cudaFree(p);
        }
        ptrs.clear();
    }
    size_t bytes = 0;
};

}  // namespace mt

#define MT_CUDA_TRY(call)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            mt::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return MT_ERR_CUDA;                                                                    \
        }                                                                                          \
    } while (0)

#define MT_TRY(call)                      \
    do {                                  \
        mt_status s_ = (call);            \
        if (s_ != MT_OK) return s_;       \
    } while (0)

// BVH build products (device pointers owned by the caller's AllocList)
struct BvhResult {
    uint4 *nodes = nullptr;     // 2 per internal node
    uint4 *wnodes = nullptr;    // 5 per 8-wide node
    int32_t n_wnodes = 0;
    float4 *tris = nullptr;     // 3 per triangle, leaf order
    int32_t n_nodes = 0;
    int32_t depth = 0;
    double sah = 0.0;
    float q_lo[3] = {0, 0, 0}, q_scale[3] = {1, 1, 1};
    float scene_lo[3], scene_hi[3];
    double build_us = 0.0;
};

mt_status mt_build_bvh(const float *d_tris, int32_t n, cudaStream_t st, mt::AllocList &al, BvhResult *out);
