// Shared-memory descriptors, mbarrier waits, TMA copies and tcgen05
// wrappers for the tensor-core correlation kernels (sm_103a), and the
// tensor-map encoders for the chunked BF16 cube layouts.  Internal to this
// library's tensor-core translation units.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "internal.h"

namespace sfoc {
namespace tcx {

constexpr int kM = 128;                                 // MMA M
constexpr unsigned long long kWaitNs = 2000000000ull;   // bounded waits: about 2 s of %globaltimer
constexpr unsigned long long kDrainNs = 200000000ull;   // waits for copies in flight after an abort
constexpr int kTcSmemMax = 225 * 1024;                  // dynamic shared memory (static shared memory needs the rest)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait of at most limit_ns; on expiry it sets *s_abort and returns
// false, as it does once another role has aborted.
__device__ inline bool mbar_wait_limit(uint32_t bar, uint32_t parity, int* s_abort, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*reinterpret_cast<volatile int*>(s_abort)) return false;
        if (globaltimer() - t0 > limit_ns) {
            atomicExch(s_abort, 1);
            return false;
        }
    }
}

// The kernels' bounded wait (about 2 s).
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, int* s_abort) {
    return mbar_wait_limit(bar, parity, s_abort, kWaitNs);
}

// Bounded wait that ignores the abort flag (used to let copies land).
__device__ inline void mbar_wait_short(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > kDrainNs) return;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major, no-swizzle shared-memory matrix descriptor (tcgen05 format).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout SWIZZLE_NONE
}

// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major.
__host__ __device__ inline uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 4-D bf16 view {8 channels, d1, d2, 2 chunks} of a chunked cube layout.
bool make_map(CUtensorMap* map, const void* base, uint64_t d1, uint64_t d2, uint32_t b1, uint32_t b2, uint32_t b3);
// The same view in 128-byte runs of 8 pixels along d1 (see k_corr_tc.cu).
bool make_map_rows8(CUtensorMap* map, const void* base, uint64_t d1, uint64_t d2, uint32_t b1, uint32_t b2);

}  // namespace tcx

// band form of the tensor-core correlation (k_corr_band.cu): whether it
// runs for (m, R), the MMAs it issues per point, its class (kernel
// instance NQ, 0 = unsupported), the job's tensor maps, and the launch
bool corr_band_supported(int m, int R);
long long corr_band_mmas(int m, int R);
int corr_band_class(int m, int R);
bool corr_band_maps(MatchJob& j);
cudaError_t launch_corr_band(const MatchJob& one, const ItemSet& is, int NQ, const int* ms, const int* Rs, int cnt,
                             int* err_flag, int sms, cudaStream_t st);

}  // namespace sfoc
