// Self-test of the failure path of the tensor-core kernels: a bounded wait
// that expires.  One CTA allocates 32 TMEM columns, waits (with the same
// bounded mbarrier wait the correlation kernels use, here limited to the
// caller's microseconds) on a barrier that nothing arrives on, and then takes
// their abort path: the wait sets the CTA's abort flag, the CTA frees its
// TMEM, sets the context's device error word and returns.  No kernel hangs
// and nothing faults; sfoc_ctx_sync then reports SFOC_ERR_TIMEOUT.
#include <stdint.h>

#include "internal.h"
#include "tc_ptx.h"

namespace sfoc {

namespace {

using namespace tcx;

__global__ void __launch_bounds__(32, 1) k_wait_selftest(int* __restrict__ err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const uint32_t bar = smem_u32(&s_bar);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);  // one arrival expected; none comes
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)), "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0) (void)mbar_wait_limit(bar, 0, &s_abort, limit_ns);
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (s_abort && threadIdx.x == 0) atomicExch(err, 1);
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

}  // namespace

cudaError_t launch_wait_selftest(int* err, int limit_us, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, (uint64_t)limit_us * 1000ull);
    return cudaGetLastError();
}

}  // namespace sfoc
