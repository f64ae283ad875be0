// Per-message launch of a Mandelbrot message (the comparator of the drain):
// one kernel launch per image job, one thread per pixel, the same escape-count
// function as the drain (mandel.cuh).  Each block adds its count sum to
// scratch; the last block to finish writes the reply (pixels, sum) and
// resets the scratch words for the next launch.
#include <cuda_runtime.h>

#include "common.cuh"
#include "factor.cuh"
#include "kernels.h"
#include "layout.h"
#include "mandel.cuh"

namespace cafgpu {
namespace {

constexpr uint32_t kMandelOneThreads = 256;

__global__ void __launch_bounds__(kMandelOneThreads) k_mandel_one(MandelDesc d, uint32_t pixels, uint64_t reply_addr,
                                                                  uint32_t reply_token, unsigned long long *sum,
                                                                  uint32_t *blocks_done, DevCtl *ctl) {
    const uint32_t p = blockIdx.x * kMandelOneThreads + threadIdx.x;
    uint32_t k = 0;
    if (p < pixels) {
        float cx, cy;
        mandel_c(d, p, cx, cy);
        k = mandel_count(cx, cy, d.max_iter);
        reinterpret_cast<uint32_t *>(d.out)[p] = k;
    }
    unsigned long long s = k;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    __shared__ unsigned long long ws[kMandelOneThreads / 32];
    __shared__ uint32_t last;
    if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
#pragma unroll
        for (uint32_t w = 0; w < kMandelOneThreads / 32; ++w) t += ws[w];
        if (t) atomicAdd(sum, t);
        __threadfence();   // this block's pixel stores and sum before the count
        last = atomicAdd(blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long total = atomicExch(sum, 0ull);
        *blocks_done = 0;
        write_reply(reply_addr, 0, pixels, total, 0, reply_token);
        add_u64(&ctl->messages, 1);
        __threadfence();
    }
}

}  // namespace

cudaError_t launch_mandel_one(const MandelDesc &d, uint64_t reply_addr, uint32_t reply_token,
                              unsigned long long *sum, uint32_t *blocks_done, DevCtl *ctl, cudaStream_t stream) {
    const uint32_t pixels = d.width * d.rows;
    const uint32_t grid = (pixels + kMandelOneThreads - 1) / kMandelOneThreads;
    k_mandel_one<<<grid, kMandelOneThreads, 0, stream>>>(d, pixels, reply_addr, reply_token, sum, blocks_done, ctl);
    return cudaGetLastError();
}

}  // namespace cafgpu
