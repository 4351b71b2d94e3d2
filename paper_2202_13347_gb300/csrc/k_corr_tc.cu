// Correlation R_ST (Eq. 10 of arXiv 2202.13347) as a tcgen05 BF16 implicit
// GEMM with FP32 accumulation in tensor memory (sm_103a).
//
// Out[dy][dx] = sum_{c,y,u} S[c][y][u+dx] * T[c][y-dy][u]
//   S: reference window (m+2R)^2 around p (cube rows/cols from p - h - R),
//   T: template m^2 from the sensed cube (zero outside [0, m)^2).
// As a GEMM D[r][n] = sum_k A[r][k] B[n][k] with
//   r = dx (M = 128 rows, rows > 2R are discarded),
//   n = 2R - dy (N = roundup(2R+1, 16) columns),
//   k = (y, u, channel), 16 channels per instruction (12 + 4 zero pad).
// Both operands are K-major, no swizzle: one "core matrix" row is the 16 B
// chunk of 8 channels of one pixel, so
//   A row r  = window pixel (y, u + r)  -> in a row-major pixel layout the
//              rows of A are consecutive 16 B chunks: a shift in dx is a
//              16 B offset of the descriptor start address;
//   B row n  = template pixel (y - 2R + n, u) -> in a column-major pixel
//              layout consecutive n are consecutive 16 B chunks (Toeplitz
//              along y by address arithmetic, no copies).
// The two chunks of an instruction (channels 0-7 and 8-15) sit in two
// planes, LBO apart; 8-row groups are SBO = 128 B apart.
//
// Staging: per K stage (8 window rows x 16 template columns) the A slab
// (8 x (16+2R) pixels) and the B slab (16 columns x (8+N-1) template rows)
// are copied with cp.async (16 B, zero-fill outside the window/template)
// into one of NB ring buffers.  One thread issues the MMAs of a stage and
// commits them to that buffer's mbarrier; the buffer is refilled once that
// barrier fires.  Persistent CTAs walk the points; the accumulator is read
// back with tcgen05.ld and written as the numerator map of Eq. 9 (raw R_ST;
// the NCC stage subtracts R_S R_T / mnz in FP64).
//
// Every wait is bounded (about 2 s of %globaltimer); on expiry the CTA sets
// the context's device error word, drains its copies, frees its TMEM and
// returns.
#include <stdint.h>

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kThreads = 256;
constexpr int kY = 8;    // window rows per stage
constexpr int kU = 16;   // template columns per stage
constexpr int kM = 128;  // MMA M (dx rows)
constexpr unsigned long long kWaitNs = 2000000000ull;

struct TcGeom {
    int m, R, P1, Lw, Npad, AW, J, NB, tmem_cols, acc_stride;
    int a_bytes, b_bytes, stage_bytes;  // per buffer (both channel chunks)
};

__host__ __device__ inline TcGeom tc_geom(int m, int R) {
    TcGeom g;
    g.m = m;
    g.R = R;
    g.P1 = 2 * R + 1;
    g.Lw = m + 2 * R;
    g.Npad = (g.P1 + 15) / 16 * 16;
    g.AW = kU + 2 * R;
    g.J = kY + g.Npad - 1;
    g.a_bytes = 2 * kY * g.AW * 16;
    g.b_bytes = 2 * kU * g.J * 16;
    g.stage_bytes = g.a_bytes + g.b_bytes;
    int nb = (224 * 1024) / g.stage_bytes;
    g.NB = nb > 4 ? 4 : nb;
    g.acc_stride = (g.Npad + 31) / 32 * 32;  // second accumulator starts on a 32-column boundary
    int c = 32;
    while (c < 2 * g.acc_stride) c <<= 1;   // two accumulators
    g.tmem_cols = c;
    return g;
}

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

// Bounded wait; returns false (and sets *s_abort) when the limit expires.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* s_abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*reinterpret_cast<volatile int*>(s_abort)) return false;
        if (globaltimer() - t0 > kWaitNs) {
            atomicExch(s_abort, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
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

// Number of 16-column accumulator chunks a thread drains: warps w and w+4
// share a 32-lane quarter and take alternate chunks.
template <int NQ>
__global__ void __launch_bounds__(kThreads, 1) k_corr_tc(const __nv_bfloat16* __restrict__ rm, int Hr, int Wr,
                                                         const __nv_bfloat16* __restrict__ cm, int Hs, int Ws,
                                                         const int32_t* __restrict__ pts, int n, int m, int R,
                                                         const PointStat* __restrict__ stats,
                                                         float* __restrict__ maps, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_empty[4];     // MMAs of the stage in buffer b are complete
    __shared__ __align__(8) uint64_t s_acc_free[2];  // accumulator a has been drained
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const TcGeom g = tc_geom(m, R);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int h = template_half(m);
    const int nyb = (g.Lw + kY - 1) / kY, nub = (m + kU - 1) / kU;
    const int T = nyb * nub;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t idesc = idesc_bf16(kM, g.Npad);
    const int nchunk = g.Npad / 16;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&s_empty[i]), 1);
        for (int i = 0; i < 2; ++i) mbar_init(smem_u32(&s_acc_free[i]), kThreads / 32);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    uint32_t g_stage = 0;  // stages issued by this CTA so far (ring-buffer and accumulator phases)
    bool aborted = false;
    const size_t rplane = (size_t)Hr * Wr * 8, splane = (size_t)Ws * Hs * 8;

    for (int k = blockIdx.x; k < n && !aborted; k += gridDim.x) {
        const PointStat st = stats[k];
        if (st.status != SFOC_PT_OK) continue;  // uniform across the CTA
        const int ty0 = pts[2 * k + 1] - h, tx0 = pts[2 * k] - h;
        const int wy0 = ty0 - R, wx0 = tx0 - R;

        // loads stage s of this point into ring buffer gs % NB
        auto load_stage = [&](int s, uint32_t gs) -> bool {
            const uint32_t buf = gs % g.NB;
            if (gs >= (uint32_t)g.NB) {
                if (!mbar_wait(smem_u32(&s_empty[buf]), ((gs / g.NB) - 1) & 1, &s_abort)) return false;
            }
            const int yb = s / nub, ub = s - yb * nub;
            const int y0 = yb * kY, u0 = ub * kU;
            const uint32_t a_s = sbase + buf * g.stage_bytes;
            const uint32_t b_s = a_s + g.a_bytes;
            const int na = 2 * kY * g.AW;
            for (int i = tid; i < na; i += kThreads) {
                int cg = i / (kY * g.AW);
                int rr = i - cg * kY * g.AW;
                int yl = rr / g.AW, xl = rr - yl * g.AW;
                int y = y0 + yl, x = u0 + xl;
                bool v = y < g.Lw && x < g.Lw;
                const __nv_bfloat16* src = v ? rm + cg * rplane + ((size_t)(wy0 + y) * Wr + (wx0 + x)) * 8 : rm;
                cp_async16(a_s + i * 16, src, v);
            }
            const int nbk = 2 * kU * g.J;
            for (int i = tid; i < nbk; i += kThreads) {
                int cg = i / (kU * g.J);
                int rr = i - cg * kU * g.J;
                int ul = rr / g.J, jl = rr - ul * g.J;
                int u = u0 + ul, j = y0 - 2 * R + jl;
                bool v = u < m && j >= 0 && j < m;
                const __nv_bfloat16* src = v ? cm + cg * splane + ((size_t)(tx0 + u) * Hs + (ty0 + j)) * 8 : cm;
                cp_async16(b_s + i * 16, src, v);
            }
            return true;
        };

        // FP32 register sums of the per-stage accumulators (round to nearest):
        // the tensor core's own accumulation truncates, so each hardware
        // partial sum covers one stage only.
        float acc[NQ][16];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[q][i] = 0.f;

        // drains the accumulator of global stage gs into acc[] and frees it
        auto drain = [&](uint32_t gs) -> bool {
            if (!mbar_wait(smem_u32(&s_empty[gs % g.NB]), (gs / g.NB) & 1, &s_abort)) return false;
            tc_fence_after();
            const uint32_t abase = tmem + ((uint32_t)(quarter * 32) << 16) + (gs & 1) * g.acc_stride;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int chunk = half + 2 * q;
                if (chunk < nchunk) {
                    float v[16];
                    tmem_ld16(abase + chunk * 16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[q][i] += v[i];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&s_acc_free[gs & 1])) : "memory");
            return true;
        };

        const uint32_t gbase = g_stage;
        const int NB = g.NB;
        for (int s = 0; s < NB - 1; ++s) {
            if (s < T && !load_stage(s, gbase + s)) aborted = true;
            cp_async_commit();
        }
        for (int c = 0; c < T; ++c) {
            if (NB == 2) cp_async_wait<0>();
            else if (NB == 3) cp_async_wait<1>();
            else cp_async_wait<2>();
            fence_proxy_async();
            __syncthreads();
            if (s_abort) aborted = true;
            if (aborted) break;
            const uint32_t gs = gbase + c;
            if (tid == 0) {
                // accumulator gs & 1 must have been drained (stage gs - 2)
                bool ok = true;
                if (gs >= 2) ok = mbar_wait(smem_u32(&s_acc_free[gs & 1]), ((gs >> 1) - 1) & 1, &s_abort);
                if (ok) {
                    tc_fence_after();
                    const uint32_t buf = gs % NB;
                    const int yb = c / nub, ub = c - yb * nub;
                    const int y0 = yb * kY, u0 = ub * kU;
                    const uint32_t a_s = sbase + buf * g.stage_bytes;
                    const uint32_t b_s = a_s + g.a_bytes;
                    const uint32_t a_lbo = kY * g.AW * 16, b_lbo = kU * g.J * 16;
                    const uint32_t dacc = tmem + (gs & 1) * g.acc_stride;
                    uint32_t first = 1;
                    for (int yl = 0; yl < kY; ++yl) {
                        if (y0 + yl >= g.Lw) break;
                        for (int ul = 0; ul < kU; ++ul) {
                            if (u0 + ul >= m) break;
                            uint64_t da = smem_desc(a_s + (yl * g.AW + ul) * 16, a_lbo, 128);
                            uint64_t db = smem_desc(b_s + (ul * g.J + yl) * 16, b_lbo, 128);
                            mma_bf16(dacc, da, db, idesc, first ? 0u : 1u);
                            first = 0;
                        }
                    }
                    mma_commit(smem_u32(&s_empty[buf]));
                }
            }
            // drain the previous stage while this one runs on the tensor cores
            if (c >= 1 && !drain(gs - 1)) aborted = true;
            const int s = c + NB - 1;
            if (s < T && !aborted && !load_stage(s, gbase + s)) aborted = true;
            cp_async_commit();
        }
        g_stage = gbase + T;
        if (!aborted && T >= 1 && !drain(gbase + T - 1)) aborted = true;
        __syncthreads();
        if (s_abort) aborted = true;
        if (aborted) break;
        {
            const int r = quarter * 32 + lane;  // dx
            float* out = maps + (size_t)k * g.P1 * g.P1;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int chunk = half + 2 * q;
                if (chunk < nchunk) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        int nn = chunk * 16 + i;
                        int dy = 2 * R - nn;
                        if (r < g.P1 && dy >= 0) out[dy * g.P1 + r] = acc[q][i];
                    }
                }
            }
        }
    }

    if (aborted || s_abort) {
        if (tid == 0) atomicExch(err, 1);
    }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                     : "memory");
    }
}

}  // namespace

// The kernel always takes the whole opt-in shared memory of an SM (it runs
// one CTA per SM): the ring buffers plus slack that keeps every descriptor
// address inside the allocation.
size_t corr_tc_smem_bytes(int m, int R) {
    TcGeom g = tc_geom(m, R);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t need = (size_t)g.NB * g.stage_bytes + 1024;
    size_t have = optin > 4096 ? (size_t)optin - 1024 : need;
    return need > have ? need : have;
}

cudaError_t launch_corr_tc(const Cube& ref, const Cube& sen, const int32_t* pts, int n, int m, int R,
                           const PointStat* stats, float* maps, int* err_flag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (ref.dtype != SFOC_DTYPE_BF16 || sen.dtype != SFOC_DTYPE_BF16 || ref.z != 12) return cudaErrorNotSupported;
    if (2 * R + 1 > kM || m > kMaxTemplate) return cudaErrorNotSupported;
    TcGeom g = tc_geom(m, R);
    if (g.NB < 2) return cudaErrorNotSupported;
    size_t smem = corr_tc_smem_bytes(m, R);
    cudaError_t e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = n < sms ? n : sms;
    const int nq = (g.Npad / 16 + 1) / 2;
#define SFOC_TC_CASE(NQ)                                                                                          \
    e = cudaFuncSetAttribute(k_corr_tc<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
    if (e != cudaSuccess) return e;                                                                               \
    k_corr_tc<NQ><<<grid, kThreads, smem, st>>>(ref.rm, ref.H, ref.W, sen.cm, sen.H, sen.W, pts, n, m, R, stats, \
                                                maps, err_flag);
    if (nq <= 1) { SFOC_TC_CASE(1) }
    else if (nq <= 2) { SFOC_TC_CASE(2) }
    else if (nq <= 3) { SFOC_TC_CASE(3) }
    else { SFOC_TC_CASE(4) }
#undef SFOC_TC_CASE
    return cudaGetLastError();
}

}  // namespace sfoc
