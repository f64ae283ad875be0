// caf_gpu_measure_latency: measured latencies of the memory operations a
// mailbox hop is made of, on the current GPU.
//
// A token passed along a ring of actors (Sec. 5, "Mixed Operations Under
// Work Load") is a chain of dependent steps -- each hop reads the mailbox
// words the previous hop wrote, takes a ticket with a returning atomic and
// publishes with release stores and fences -- so its time per hop is a sum of
// L2 round trips, not a bandwidth.  This entry point measures those round
// trips, so a hop time can be stated as a multiple of them:
//
//   ns[0]  a returning atomic add on a global word (one thread, each add's
//          address depends on the previous result: one L2 round trip each);
//   ns[1]  an acquire load of a line in L2 (one thread, a dependent chain
//          through a table of 4096 words: one L2 round trip each);
//   ns[2]  a relaxed store followed by fence.sc.gpu (one thread, in a loop);
//   ns[3]  one-way flag handoff between two SMs: a release store seen by an
//          acquire-polling thread on another SM, half of a ping-pong round
//          trip.  The two CTAs of the ping-pong are launched cooperatively
//          (co-resident) and each takes more than half an SM's shared memory,
//          so they run on different SMs.  Every wait is bounded: a wait that
//          gives up sets a flag, both CTAs leave, and the call returns ECUDA.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/caf_gpu.h"
#include "common.cuh"

namespace cafgpu {
namespace {

constexpr uint32_t kChainIters = 20000;
constexpr uint32_t kPingIters = 20000;
constexpr uint32_t kTableWords = 4096;
constexpr uint32_t kPingSmem = 160 * 1024;   // > half of an SM's shared memory: one CTA per SM
constexpr uint64_t kPingWaitNs = 200000000;  // 200 ms per wait, then give up

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// out[0] = atomic chain ns, out[1] = acquire-load chain ns, out[2] = store+fence ns (per step).
__global__ void k_chains(uint32_t *words, uint32_t *table, uint64_t *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    // warm the table into L2 (acquire loads are served by L2, not L1)
    uint32_t x = 0;
    for (uint32_t i = 0; i < kTableWords; ++i) x += ld_acquire_gpu(&table[i]);
    // returning atomics, each address taken from the previous result
    uint64_t t0 = globaltimer();
    uint32_t a = x & 7u;
    for (uint32_t i = 0; i < kChainIters; ++i) a = atomicAdd(&words[a & 7u], 1u) & 7u;
    uint64_t t1 = globaltimer();
    out[0] = t1 - t0;
    // dependent acquire loads through the table (a single cycle visits every word)
    uint32_t p = a & (kTableWords - 1);
    t0 = globaltimer();
    for (uint32_t i = 0; i < kChainIters; ++i) p = ld_acquire_gpu(&table[p]);
    t1 = globaltimer();
    out[1] = t1 - t0;
    // store + fence.sc
    t0 = globaltimer();
    for (uint32_t i = 0; i < kChainIters; ++i) {
        st_relaxed_u32(&words[8 + (p & 7u)], i);
        asm volatile("fence.sc.gpu;" ::: "memory");
    }
    t1 = globaltimer();
    out[2] = t1 - t0;
    words[16] = p;   // keep the chains
}

// Ping-pong between thread 0 of CTA 0 and thread 0 of CTA 1 on flags[0] (CTA
// 0 -> 1) and flags[32] (1 -> 0).  flags[64] is the give-up flag; out[3] the
// time of kPingIters round trips measured by CTA 0; out[4], out[5] the SM ids.
__global__ void k_ping(uint32_t *flags, uint64_t *out) {
    extern __shared__ uint8_t ping_smem[];
    if (threadIdx.x != 0) return;
    ping_smem[0] = 1;
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    out[4 + blockIdx.x] = smid;
    uint32_t *to = &flags[blockIdx.x == 0 ? 0 : 32];
    uint32_t *from = &flags[blockIdx.x == 0 ? 32 : 0];
    uint32_t *quit = &flags[64];
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1; i <= kPingIters; ++i) {
        if (blockIdx.x == 0) st_release_gpu(to, i);
        const uint64_t deadline = globaltimer() + kPingWaitNs;
        uint32_t spins = 0;
        while (ld_acquire_gpu(from) != i) {
            if ((++spins & 255u) == 0 && (globaltimer() > deadline || ld_acquire_gpu(quit) != 0)) {
                atomicExch(quit, 1u);
                return;
            }
        }
        if (blockIdx.x == 1) st_release_gpu(to, i);
    }
    if (blockIdx.x == 0) out[3] = globaltimer() - t0;
}

}  // namespace
}  // namespace cafgpu

extern "C" int caf_gpu_measure_latency(double *ns) {
    using namespace cafgpu;
    if (!ns) return CAF_GPU_EINVAL;
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return CAF_GPU_ECUDA;
    uint32_t *words = nullptr, *table = nullptr, *flags = nullptr;
    uint64_t *out = nullptr;
    int r = 0;
    if (cudaMalloc(&words, 64 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&table, kTableWords * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&flags, 128 * sizeof(uint32_t)) != cudaSuccess || cudaMalloc(&out, 8 * sizeof(uint64_t)) != cudaSuccess)
        r = CAF_GPU_ECUDA;
    if (!r) {
        // table[i] = i + 1337 (mod 4096): one cycle through every word, strided
        // so consecutive loads touch different lines
        uint32_t host[kTableWords];
        for (uint32_t i = 0; i < kTableWords; ++i) host[i] = (i + 1337u) & (kTableWords - 1);
        if (cudaMemcpy(table, host, sizeof host, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(words, 0, 64 * sizeof(uint32_t)) != cudaSuccess ||
            cudaMemset(flags, 0, 128 * sizeof(uint32_t)) != cudaSuccess ||
            cudaMemset(out, 0, 8 * sizeof(uint64_t)) != cudaSuccess)
            r = CAF_GPU_ECUDA;
    }
    if (!r) {
        k_chains<<<1, 32>>>(words, table, out);
        if (cudaGetLastError() != cudaSuccess) r = CAF_GPU_ECUDA;
    }
    if (!r && cudaFuncSetAttribute(k_ping, cudaFuncAttributeMaxDynamicSharedMemorySize, kPingSmem) != cudaSuccess)
        r = CAF_GPU_ECUDA;
    if (!r) {
        void *args[] = {&flags, &out};
        if (cudaLaunchCooperativeKernel((const void *)k_ping, dim3(2), dim3(32), args, kPingSmem, nullptr) !=
            cudaSuccess)
            r = CAF_GPU_ECUDA;
    }
    uint64_t h[8] = {};
    uint32_t quit = 0;
    if (!r && (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(h, out, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess ||
               cudaMemcpy(&quit, flags + 64, sizeof quit, cudaMemcpyDeviceToHost) != cudaSuccess))
        r = CAF_GPU_ECUDA;
    if (!r && (quit != 0 || h[3] == 0 || h[4] == h[5])) r = CAF_GPU_ECUDA;
    if (!r) {
        ns[0] = (double)h[0] / kChainIters;
        ns[1] = (double)h[1] / kChainIters;
        ns[2] = (double)h[2] / kChainIters;
        ns[3] = (double)h[3] / (2.0 * kPingIters);
    }
    cudaFree(words);
    cudaFree(table);
    cudaFree(flags);
    cudaFree(out);
    return r;
}
