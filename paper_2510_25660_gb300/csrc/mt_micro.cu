// mt_micro.cu -- microbenchmarks for the memory/atomic roofline of the tracer.
//
// The render kernel's traffic is dominated by 32-byte node and 48-byte
// triangle fetches at data-dependent addresses (mostly L2 hits) and by film
// atomics; the measured HBM copy bandwidth alone does not bound it.  These
// kernels measure, on the GPU in use, the rates those access patterns can reach:
//   MT_MICRO_GATHER32  random 32-byte sector loads from a buffer (L2 resident
//                      when it is smaller than L2), GB/s
//   MT_MICRO_RED_GLOBAL  red.global.add.f32 at random addresses of a buffer, Gop/s
//   MT_MICRO_RED_SHARED  shared-memory atomicAdd.f32 at random addresses of a
//                      48 KB histogram per CTA, Gop/s
#include "mt_common.cuh"
#include "mt_internal.h"

namespace {

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    // integer mix (Wang-style shifts and multiplies); only used to scatter addresses
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

__global__ void k_gather32(const uint4 *buf, uint64_t n_sectors, int iters, uint32_t *sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0, h = hash32(tid * 0x9E3779B9u + 1u);
    for (int i = 0; i < iters; ++i) {
        h = hash32(h + (uint32_t)i);
        const uint64_t sct = ((uint64_t)h * n_sectors) >> 32;
        const uint4 a = __ldg(&buf[2 * sct]);
        const uint4 b = __ldg(&buf[2 * sct + 1]);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
    }
    if (acc == 0x12345678u) sink[0] = acc;
}

__global__ void k_red_global(float *buf, uint64_t n, int iters) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(tid + 7u);
    for (int i = 0; i < iters; ++i) {
        h = hash32(h + (uint32_t)i);
        atomicAdd(&buf[((uint64_t)h * n) >> 32], 1.0f);
    }
}

__global__ void k_red_shared(int iters, float *sink) {
    __shared__ float hist[12288];
    for (int i = threadIdx.x; i < 12288; i += blockDim.x) hist[i] = 0.f;
    __syncthreads();
    uint32_t h = hash32(blockIdx.x * blockDim.x + threadIdx.x + 3u);
    for (int i = 0; i < iters; ++i) {
        h = hash32(h + (uint32_t)i);
        atomicAdd(&hist[((uint64_t)h * 12288u) >> 32], 1.0f);
    }
    __syncthreads();
    if (threadIdx.x == 0 && hist[0] == -1.0f) sink[0] = hist[1];
}

}  // namespace

extern "C" mt_status mt_microbench(int32_t kind, void *d_buf, int64_t bytes, int32_t iters, double *out_rate,
                                   void *stream) {
    if (!out_rate || iters < 1 || !d_buf || bytes < 4096) {
        mt::set_error("mt_microbench: bad arguments");
        return MT_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    MT_CUDA_TRY(cudaGetDevice(&dev));
    MT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    MT_CUDA_TRY(cudaEventCreate(&e0));
    MT_CUDA_TRY(cudaEventCreate(&e1));
    double units = 0.0;
    for (int rep = 0; rep < 2; ++rep) {  // first run warms caches and clocks
        MT_CUDA_TRY(cudaEventRecord(e0, st));
        if (kind == MT_MICRO_GATHER32) {
            k_gather32<<<blocks, threads, 0, st>>>((const uint4 *)d_buf, (uint64_t)bytes / 32, iters,
                                                   (uint32_t *)d_buf);
            units = (double)blocks * threads * iters * 32.0;
        } else if (kind == MT_MICRO_RED_GLOBAL) {
            k_red_global<<<blocks, threads, 0, st>>>((float *)d_buf, (uint64_t)bytes / 4, iters);
            units = (double)blocks * threads * iters;
        } else if (kind == MT_MICRO_RED_SHARED) {
            k_red_shared<<<blocks, threads, 0, st>>>(iters, (float *)d_buf);
            units = (double)blocks * threads * iters;
        } else {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            mt::set_error("mt_microbench: unknown kind %d", kind);
            return MT_ERR_INVALID_ARGUMENT;
        }
        MT_CUDA_TRY(cudaGetLastError());
        MT_CUDA_TRY(cudaEventRecord(e1, st));
    }
    MT_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    MT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out_rate = units / (ms * 1e-3) / 1e9;  // GB/s or Gop/s
    return MT_OK;
}
