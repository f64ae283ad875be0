// GEMM kernels outside the persistent drain: one launch per GEMM message
// (the per-message-launch form), each CTA one 128 x 128 output tile.
#include <cuda_runtime.h>

#include "common.cuh"
#include "factor.cuh"
#include "gemm_tc.cuh"
#include "kernels.h"
#include "layout.h"

namespace cafgpu {

// scratch[0] counts the CTAs of this launch that have finished; the last one
// writes the reply and puts the counter back to 0.
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_one(const float *A, const float *B, float *C, uint32_t n, uint32_t split, uint64_t reply_addr,
               uint32_t reply_token, uint32_t *scratch, uint64_t limit_ns, DevCtl *ctl) {
    extern __shared__ uint8_t gemm_raw[];
    GemmSmem &S = gemm_smem(gemm_raw);
    const uint32_t tiles_n = (n + kGemmBN - 1) / kGemmBN;
    const uint32_t tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
    gemm_cta_init(S);
    GemmCounters K{0, 0, 0};
    const bool ok = gemm_tile(A, B, C, n, tm, tn, split != 0, S.ops, S.bars, K, limit_ns, CtaSyncAll{});
    gemm_cta_exit(S);
    __shared__ uint32_t last;
    if (threadIdx.x == 0) {
        if (!ok) raise_error(ctl, kErrGemm, 14);
        __threadfence();
        last = atomicAdd(scratch, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        write_reply(reply_addr, ok ? 0 : 3, 0, n, 0, reply_token);
        scratch[0] = 0;
        add_u64(&ctl->messages, 1);
        add_u64(&ctl->gemm_tiles, gridDim.x);
    }
}

cudaError_t launch_gemm_one(const float *A, const float *B, float *C, uint32_t n, bool split, uint64_t reply_addr,
                            uint32_t reply_token, uint32_t *scratch, uint64_t limit_ns, DevCtl *ctl,
                            cudaStream_t stream) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_one, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const uint32_t t = (n + kGemmBN - 1) / kGemmBN;
    k_gemm_one<<<t * t, kGemmThreads, kGemmSmemBytes, stream>>>(A, B, C, n, split ? 1u : 0u, reply_addr,
                                                                reply_token, scratch, limit_ns, ctl);
    return cudaGetLastError();
}

}  // namespace cafgpu
