// caf_gpu_measure_mul_rates: measured throughput of the integer multiplies
// the factorization payload is made of, on the current GPU.
//
// The divisibility test (factor.cuh) is two 32-bit low multiplies and one
// high multiply (mul.hi) per (n, p) pair.  Its roofline peak is quoted as the
// nominal 32-bit multiply rate of the SM (64 per clock); this entry point
// measures what the hardware sustains for each instruction form and for the
// test's own chain, so a report can state the ceiling the test can reach.
// Each thread runs 8 independent chains for a fixed number of iterations and
// stores one word; nothing else is read or written.
//
// caf_gpu_measure_fp32_rate does the same for the float32 multiplies and adds
// (rounded one by one) of the Mandelbrot escape iteration (mandel.cuh).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/caf_gpu.h"

namespace cafgpu {
namespace {

constexpr int kChains = 8;
constexpr int kThreadsPerBlock = 256;

template <int kMode>
__global__ void __launch_bounds__(kThreadsPerBlock) k_mul_rate(uint32_t *out, uint32_t iters, uint32_t seed) {
    uint32_t x[kChains];
    const uint32_t a = seed | 1u, b = seed * 7u + threadIdx.x;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 13u + (uint32_t)i * 101u + blockIdx.x;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (kMode == 0) {
                x[i] = x[i] * a + b;                        // low multiply-add
            } else if (kMode == 1) {
                x[i] = __umulhi(x[i], a) + b;               // high multiply
            } else {
                const uint32_t m0 = x[i] * a;               // the test: low, high, low
                const uint32_t n1 = __umulhi(m0, b) + (uint32_t)i;
                x[i] = n1 * a;
            }
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- x * a + b as a rounded multiply and a rounded add (two operations);
// with a = 0.999 and b = 0.001 every chain stays near 1 (no overflow, no
// subnormals).
__global__ void __launch_bounds__(kThreadsPerBlock) k_fp32_rate(float *out, uint32_t iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 0.001f * (float)(threadIdx.x + i);
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __fadd_rn(__fmul_rn(x[i], a), b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int kMode>
int time_mode(uint32_t *d, int blocks, uint32_t iters, int muls_per_step, double *rate) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CAF_GPU_ECUDA;
    k_mul_rate<kMode><<<blocks, kThreadsPerBlock>>>(d, iters / 8, 3u);   // warm-up
    cudaEventRecord(e0);
    k_mul_rate<kMode><<<blocks, kThreadsPerBlock>>>(d, iters, 3u);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || ms <= 0.f) return CAF_GPU_ECUDA;
    *rate = (double)blocks * kThreadsPerBlock * iters * kChains * muls_per_step / (ms * 1e-3);
    return 0;
}

}  // namespace
}  // namespace cafgpu

extern "C" int caf_gpu_measure_mul_rates(double *rates) {
    using namespace cafgpu;
    if (!rates) return CAF_GPU_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return CAF_GPU_ECUDA;
    const int blocks = sms * 8;
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * (size_t)blocks * kThreadsPerBlock) != cudaSuccess) return CAF_GPU_ECUDA;
    const uint32_t iters = 20000;
    int r = time_mode<0>(d, blocks, iters, 1, &rates[0]);
    if (!r) r = time_mode<1>(d, blocks, iters, 1, &rates[1]);
    if (!r) r = time_mode<2>(d, blocks, iters, 3, &rates[2]);
    cudaFree(d);
    return r;
}

extern "C" int caf_gpu_measure_fp32_rate(double *ops_per_s) {
    using namespace cafgpu;
    if (!ops_per_s) return CAF_GPU_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return CAF_GPU_ECUDA;
    const int blocks = sms * 8;
    float *d = nullptr;
    if (cudaMalloc(&d, sizeof(float) * (size_t)blocks * kThreadsPerBlock) != cudaSuccess) return CAF_GPU_ECUDA;
    const uint32_t iters = 40000;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int r = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = CAF_GPU_ECUDA;
    float ms = 0.f;
    if (!r) {
        k_fp32_rate<<<blocks, kThreadsPerBlock>>>(d, iters / 8, 0.999f, 0.001f);   // warm-up
        cudaEventRecord(e0);
        k_fp32_rate<<<blocks, kThreadsPerBlock>>>(d, iters, 0.999f, 0.001f);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) r = CAF_GPU_ECUDA;
        if (!r) cudaEventElapsedTime(&ms, e0, e1);
        if (!r && ms <= 0.f) r = CAF_GPU_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (!r) *ops_per_s = (double)blocks * kThreadsPerBlock * iters * kChains * 2.0 / (ms * 1e-3);
    return r;
}
