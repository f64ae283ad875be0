// GEMM kernels outside the persistent drain: one launch per GEMM message
// (the per-message-launch form), each CTA one 128 x 128 output tile; and the
// host side of the tensor maps the tile engine stages its operands with.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "factor.cuh"
#include "gemm_tc.cuh"
#include "kernels.h"
#include "layout.h"

namespace cafgpu {

// scratch[0] counts the CTAs of this launch that have finished; the last one
// writes the reply and puts the counter back to 0.  use_tma: tma_a / tma_b
// describe A and B (else the converters read them directly).
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_one(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b,
               uint32_t use_tma, const float *A, const float *B, float *C, uint32_t n, uint32_t split,
               uint64_t reply_addr, uint32_t reply_token, uint32_t *scratch, uint64_t limit_ns, DevCtl *ctl) {
    extern __shared__ uint8_t gemm_raw[];
    GemmSmem &S = gemm_smem(gemm_raw);
    const uint32_t tiles_n = (n + kGemmBN - 1) / kGemmBN;
    gemm_cta_init(S);
    GemmCounters K{0, 0, 0, 0};
    const GemmArgs g{A, B, C, use_tma ? &tma_a : nullptr, use_tma ? &tma_b : nullptr,
                     n, blockIdx.x / tiles_n, blockIdx.x % tiles_n, split != 0};
    const bool ok = gemm_tile(g, S.ops, S.bars, K, limit_ns, CtaSyncAll{});
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

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

int gemm_encode_tmap(void *out128, const void *base, uint32_t n, bool is_a) {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    std::memset(out128, 0, 128);
    if (!g_encode || n == 0) return -1;
    const cuuint64_t dims[2] = {n, n};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 4u};
    const cuuint32_t box_a[2] = {32, kGemmBM}, box_b[2] = {kGemmBN, kGemmBK};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r =
        g_encode(static_cast<CUtensorMap *>(out128), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base),
                 dims, strides, is_a ? box_a : box_b, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 is_a ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

bool gemm_tma_ok(const void *A, const void *B, uint32_t n) {
    return (n & 3u) == 0 && ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) == 0;
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
    CUtensorMap ta, tb;
    const bool tma = gemm_tma_ok(A, B, n) && gemm_encode_tmap(&ta, A, n, true) == 0 &&
                     gemm_encode_tmap(&tb, B, n, false) == 0;
    if (!tma) {
        std::memset(&ta, 0, sizeof ta);
        std::memset(&tb, 0, sizeof tb);
    }
    const uint32_t t = (n + kGemmBN - 1) / kGemmBN;
    k_gemm_one<<<t * t, kGemmThreads, kGemmSmemBytes, stream>>>(ta, tb, tma ? 1u : 0u, A, B, C, n, split ? 1u : 0u,
                                                                reply_addr, reply_token, scratch, limit_ns, ctl);
    return cudaGetLastError();
}

}  // namespace cafgpu
