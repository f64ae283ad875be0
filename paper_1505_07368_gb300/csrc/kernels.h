// Host-side launch wrappers for the kernels in drain.cu.  Each enqueues on
// `stream` and returns the launch status.
#pragma once

#include <cuda_runtime.h>

#include "layout.h"

namespace cafgpu {

cudaError_t launch_drain(const DrainParams &p, unsigned grid, cudaStream_t stream);
// CTAs of the drain kernel that fit on one SM at once (GEMM layout or not).
cudaError_t drain_occupancy(bool gemm, bool split, int *ctas_per_sm);
cudaError_t launch_reset_ctl(DevCtl *ctl, cudaStream_t stream);
cudaError_t launch_mark(DevCtl *ctl, cudaStream_t stream);
cudaError_t launch_factor_one(uint64_t n, const uint32_t *primes, const uint32_t *pinv,
                              const uint32_t *plim, uint32_t nprimes, uint64_t reply_addr,
                              uint32_t reply_token, uint64_t tag, uint32_t *scratch, DevCtl *ctl,
                              unsigned grid, cudaStream_t stream);
cudaError_t launch_token_one(ActorDesc *actors, uint32_t a, uint32_t kind, int32_t v,
                             uint64_t reply_addr, uint32_t reply_token, IngressEntry *outbox,
                             DevCtl *ctl, cudaStream_t stream);
cudaError_t launch_reset_actors(ActorDesc *actors, uint32_t n_actors, cudaStream_t stream);
// FORK actor pool: `count` free records from actor index `base`, mailboxes from slot `slot0`.
cudaError_t launch_fork_pool_init(ActorDesc *actors, uint32_t base, uint32_t count, uint64_t slot0,
                                  cudaStream_t stream);
// One GEMM message, C = A * B (n x n FP32), BF16 or split-BF16x3 on tcgen05;
// scratch[0] must be 0 at rest.
cudaError_t launch_gemm_one(const float *A, const float *B, float *C, uint32_t n, bool split, uint64_t reply_addr,
                            uint32_t reply_token, uint32_t *scratch, uint64_t limit_ns, DevCtl *ctl,
                            cudaStream_t stream);
// Tensor map (128 bytes, zeroed first) of an n x n row-major FP32 operand as
// the GEMM tile engine stages it: A (is_a) as boxes of 32 k x 128 rows with
// the 128-byte swizzle, B as boxes of 128 columns x 64 k.  Returns 0, or -1
// when the driver's encoder is unavailable or rejects the map.
int gemm_encode_tmap(void *out128, const void *base, uint32_t n, bool is_a);
// A and B can be staged through tensor maps (n % 4 == 0, 16-byte aligned).
bool gemm_tma_ok(const void *A, const void *B, uint32_t n);
// One Mandelbrot message (per-message backend): one thread per pixel; sum and
// blocks_done are scratch words, zero at rest and left zero.
cudaError_t launch_mandel_one(const MandelDesc &d, uint64_t reply_addr, uint32_t reply_token,
                              unsigned long long *sum, uint32_t *blocks_done, DevCtl *ctl, cudaStream_t stream);
cudaError_t launch_debug_wait(const uint32_t *flag, uint64_t limit_ns, DevCtl *ctl, HostCtl *hctl,
                              cudaStream_t stream);
// Prime table of the odd primes <= limit.  Allocates *primes/*pinv/*plim
// (cudaMalloc, padded with zeros by `pad` entries) and returns their count.
cudaError_t build_prime_table(uint64_t limit, uint32_t pad, uint32_t **primes, uint32_t **pinv,
                              uint32_t **plim, uint32_t *count, cudaStream_t stream);

}  // namespace cafgpu
