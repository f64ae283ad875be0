// caf_gpu_factor_static: factorization of a batch of numbers without any
// device allocation by the library.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// whose allocator owns all of the GPU's memory (a stray cudaMalloc there can
// fail, or fragment the pool the framework manages), latency-critical paths
// that cannot afford cudaMalloc's device-wide synchronisation, and programs
// that forbid dynamic allocation once they have started.  They cannot create
// a caf_gpu runtime either, since that allocates its arenas.  This entry
// point needs nothing from them but the input and output arrays.
//
// The kernel is the one-launch-per-message factorization (several CTAs share
// one number and agree on the smallest divisor through a per-number word in
// global memory) applied to a batch, with the divisors generated on the fly
// (2, then every odd d) instead of read from a prime table, because the table
// would have to be allocated.  Its only scratch -- two words per number --
// lives in the file-scope array g_static_words below.  That array is part of
// the library image: every GPU that loads the library holds its 32 KB until
// the process exits.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/caf_gpu.h"
#include "common.cuh"
#include "factor.cuh"

namespace cafgpu {
namespace {

constexpr uint32_t kStaticCtasPerMsg = 4;
constexpr uint32_t kStaticThreads = 256;
constexpr uint32_t kStaticNone = 0xFFFFFFFFu;
static_assert(CAF_GPU_FACTOR_STATIC_MAX == 4096, "scratch size follows the header's limit");

struct StaticWords {
    uint32_t divisor;    // smallest odd divisor found so far (atomicMin); kStaticNone if none
    uint32_t ctas_done;  // CTAs of this number that have finished
};

// Scratch shared by every call in the process.  Host code may not use this
// name as an address (it is a host-side stand-in); the launch below passes the
// device address obtained with cudaGetSymbolAddress.
__device__ __align__(256) StaticWords g_static_words[CAF_GPU_FACTOR_STATIC_MAX];

// Put the words of numbers [0, count) in their rest state.
__global__ void k_static_clear(StaticWords *w, uint32_t count) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        w[i].divisor = kStaticNone;
        w[i].ctas_done = 0;
    }
}

// d^-1 mod 2^32 for odd d: d*d == 1 (mod 8) gives 3 correct bits, and each
// Newton step x <- x(2 - d x) doubles them (6, 12, 24, 48).
__device__ __forceinline__ uint32_t inverse_mod_2_32(uint32_t d) {
    uint32_t x = d;
    x *= 2u - d * x;
    x *= 2u - d * x;
    x *= 2u - d * x;
    x *= 2u - d * x;
    return x;
}

// kStaticCtasPerMsg CTAs per number.  Warp g of a number tests the chunks of
// 32 consecutive odd candidates g, g + G, ... (G warps per number) and stops
// once a divisor below its chunk is known.  Divisibility: the same two-step
// Montgomery test as the drain, with the final check written as
// umulhi(m1, d) == 0 (m1 * d < 2^32) since floor((2^32-1)/d) is not tabled.
__global__ void __launch_bounds__(kStaticThreads) k_factor_static(const uint64_t *d_n, uint32_t count,
                                                                  Reply *rep, StaticWords *w) {
    const uint32_t msg = blockIdx.x / kStaticCtasPerMsg;
    if (msg >= count) return;
    const uint32_t part = blockIdx.x % kStaticCtasPerMsg;
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t warps = kStaticCtasPerMsg * (kStaticThreads / 32);
    const uint32_t gw = part * (kStaticThreads / 32) + warp;
    const uint64_t n = d_n[msg];
    const bool valid = n < (1ull << 62);
    const bool even = n >= 4 && !(n & 1u);
    const uint64_t root = (valid && !even && n >= 9) ? isqrt_u64(n) : 0;
    const uint64_t ncand = root >= 3 ? (root - 3) / 2 + 1 : 0;   // odd d in [3, root]
    const uint32_t nl = 0u - (uint32_t)n;
    const uint32_t ch = (uint32_t)(n >> 32) + ((uint32_t)n != 0u ? 1u : 0u);
    for (uint64_t c = (uint64_t)gw * 32; c < ncand; c += (uint64_t)warps * 32) {
        const uint32_t first = (uint32_t)(3 + 2 * c);
        if (*((volatile uint32_t *)&w[msg].divisor) < first) break;
        const uint64_t i = c + lane;
        bool hit = false;
        uint32_t d = 0;
        if (i < ncand) {
            d = (uint32_t)(3 + 2 * i);
            const uint32_t dinv = inverse_mod_2_32(d);
            const uint32_t m0 = nl * dinv;
            const uint32_t n1 = __umulhi(m0, d) + ch;
            hit = __umulhi(n1 * dinv, d) == 0u;
        }
        const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, hit ? d : kStaticNone);
        if (mn != kStaticNone) {
            if (lane == 0) atomicMin(reinterpret_cast<unsigned int *>(&w[msg].divisor), mn);
            break;
        }
    }
    __syncthreads();
    __shared__ uint32_t last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(reinterpret_cast<unsigned int *>(&w[msg].ctas_done), 1u) == kStaticCtasPerMsg - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const uint32_t dv = *((volatile uint32_t *)&w[msg].divisor);
        int32_t status;
        uint64_t r0, r1;
        if (!valid) {
            status = CAF_GPU_REPLY_REJECTED;
            r0 = r1 = 0;
        } else if (even) {
            status = CAF_GPU_REPLY_OK;
            r0 = 2;
            r1 = n >> 1;
        } else if (dv != kStaticNone) {
            status = CAF_GPU_REPLY_OK;
            r0 = dv;
            r1 = n / dv;
        } else {
            status = CAF_GPU_REPLY_NOFACTOR;
            r0 = 1;
            r1 = n;
        }
        write_reply((uint64_t)&rep[msg], status, r0, r1, 0, 1u);
        // leave the words at rest for the next call
        w[msg].divisor = kStaticNone;
        w[msg].ctas_done = 0;
    }
}

// Device address of g_static_words, looked up once per device with that
// device current.
std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
StaticWords *g_static_addr[kMaxDevices] = {};

int static_words(StaticWords **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CAF_GPU_ECUDA;
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_words) != cudaSuccess || !p) return CAF_GPU_ECUDA;
        g_static_addr[dev] = static_cast<StaticWords *>(p);
    }
    *out = g_static_addr[dev];
    return 0;
}

}  // namespace
}  // namespace cafgpu

extern "C" int caf_gpu_factor_static(const uint64_t *d_n, uint32_t count, caf_gpu_dreply *d_replies,
                                     void *stream) {
    using namespace cafgpu;
    if (count == 0) return CAF_GPU_OK;
    if (!d_n || !d_replies) return CAF_GPU_EINVAL;
    if (count > CAF_GPU_FACTOR_STATIC_MAX) return CAF_GPU_EINVAL;
    StaticWords *w = nullptr;
    int r = static_words(&w);
    if (r) return r;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_static_clear<<<(count + 255) / 256, 256, 0, s>>>(w, count);
    k_factor_static<<<count * kStaticCtasPerMsg, kStaticThreads, 0, s>>>(d_n, count,
                                                                         reinterpret_cast<Reply *>(d_replies), w);
    return cudaGetLastError() == cudaSuccess ? CAF_GPU_OK : CAF_GPU_ECUDA;
}
