// Correlation R_ST (Eq. 10 of arXiv 2202.13347), band form of the tcgen05
// BF16 implicit GEMM with FP32 accumulation in tensor memory (sm_103a).
// Every wait is bounded (about 2 s of %globaltimer); on expiry the CTA sets
// the context's device error word, every role leaves its loop (the drain
// warps run on to the end without waiting, so that their named barriers
// stay matched), the producer waits (bounded) for its copies in flight,
// TMEM is freed and the kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "internal.h"
#include "tc_ptx.h"

namespace sfoc {

namespace {

using namespace tcx;
// ---------------------------------------------------------------------------
// Band form.  The window's rows are taken in bands of 16 and the offsets dx
// in groups of 8; one accumulator per (band y0 = 16 b, offset group e):
//   D[8g + r][n] = sum_{u, c} S[c][y0 + g][u + 8e + r] T[c][y0 - 2R + n][u]
// M = 128 = 16 window rows x 8 offsets.  An A row is one 16-byte chunk of
// the row-major window tile, so the 8 rows of a core matrix are 8
// consecutive offsets (a 16-byte step, as in the Toeplitz form) and the
// core-matrix groups step by one window row (SBO = the tile's row pitch).
// N = roundup(16 + 2R, 16) template rows from y0 - 2R: every template row
// that meets a row of the band at some dy in [0, 2R].
// K = (template column u, 16 channels): one MMA per (band, offset group, u).
// Per point this issues ceil((m + 2R)/16) ceil((2R+1)/8) m MMAs of N rows,
// each reading a 4 KB A and a 32N-byte B from shared memory, against the
// column form's (2R+1) m MMAs of 7 KB: about 3/4 of its operand traffic.
// An accumulator is 128 lanes x N columns, so the two 256-column halves of
// TMEM hold consecutive groups: the MMAs of one group run while the other
// half is drained.  Each group reloads its template rows (one slab of
// kBandQ columns per stage) and its window tile (16 rows, 8 GE + m - 1
// columns), a third of the column form's copies per point.
//
// Diagonal sums.  Out[dy][dx] collects D[8g + r][n] with y0 + g - (y0 - 2R
// + n) = dy, i.e. n = 2R + g - dy.  A drain thread owns one TMEM lane, i.e.
// one (g, r): g = 4q + g' with q the warp's lane quarter and g' = lane / 8.
// It shifts its row left by g' (two select steps), after which column j of
// every lane of the warp with the same r holds dy = 2R + 4q - j; two
// butterfly steps over the lanes 8 and 16 apart add the four rows g' and
// leave each lane a quarter of the columns, kept as running sums over the
// bands of one offset-group set.  Template rows outside [0, m) are zeroed
// before the shift; window rows past m + 2R only reach dy > 2R.  After the
// last band the eight drain warps' sums meet in shared memory and are added
// in a fixed order, so the result does not depend on timing.
// Roles: warp 0 copies, warps 1-3 issue the MMAs (accumulator e of a group
// goes to warp 1 + e mod 3: an issuing thread stalls for a few hundred
// clocks at every stage's barrier, and with the short N <= 96 MMAs the
// tensor pipe's queue runs dry meanwhile unless another thread has MMAs
// queued), warps 4-7 drain the even groups (TMEM half 0), warps 8-11 the
// odd ones (half 1).  Each accumulator spans m MMAs, like the column form's.
// ---------------------------------------------------------------------------
constexpr int kBandQ = 8;  // template columns per stage
constexpr int kBandMaxTS = 4;
constexpr int kBandThreads = 384;
constexpr int kBandDrain = 256;
constexpr int kBandMaxNQ = 6;  // N <= 96, i.e. R <= 40
constexpr int kBandIssuers = 3;  // MMA-issuing warps (1 .. kBandIssuers)
constexpr int kBandSmemFloor = 120 * 1024;  // dynamic shared memory of a launch: at least this

__host__ __device__ constexpr int band_ge_max(int nq) { return nq <= 3 ? 5 : 16 / nq; }

struct BandGeom {
    int m, R, P1, Lw;
    int N, NQ;      // template rows per MMA (roundup(16 + 2R, 16)) and N / 16
    int nE, GE;     // offset groups of 8; accumulators per group (<= band_ge_max)
    int nEG, nYB;   // offset-group sets, bands of 16 window rows
    int nS;         // stages (template slabs) per group
    int Xw;         // window tile width in pixels: roundup(8 GE + m - 1, 8)
    int trows;      // template rows per slab column: roundup(16 + 2R, 8)
    int tile_bytes, slab_bytes, TS;
    int tile_off, slab_off, part_off, smem;
};

__host__ __device__ inline BandGeom band_geom(int m, int R) {
    BandGeom b;
    b.m = m;
    b.R = R;
    b.P1 = 2 * R + 1;
    b.Lw = m + 2 * R;
    b.N = (16 + 2 * R + 15) / 16 * 16;
    b.NQ = b.N / 16;
    b.nE = (b.P1 + 7) / 8;
    // as few offset-group sets as TMEM allows, of near-equal size
    const int gm = band_ge_max(b.NQ);
    b.nEG = (b.nE + gm - 1) / gm;
    b.GE = (b.nE + b.nEG - 1) / b.nEG;
    b.nYB = (b.Lw + 15) / 16;
    b.nS = (m + kBandQ - 1) / kBandQ;
    b.Xw = (8 * b.GE + m - 1 + 7) / 8 * 8;
    b.trows = (16 + 2 * R + 7) / 8 * 8;
    b.tile_bytes = 2 * 16 * b.Xw * 16;
    b.slab_bytes = 2 * kBandQ * b.trows * 16;
    b.tile_off = 0;
    b.slab_off = 2 * b.tile_bytes;
    const int part_bytes = 4 * b.GE * b.P1 * 8 * 4;  // per quarter q: GE x P1 x 8 offsets
    // an MMA on the last column of a slab reads N - trows rows past it; the
    // partial-sum buffer follows the slabs, plus a guard for the last slot
    const int guard = (b.N - b.trows) * 16 + 128;
    int ts = (kTcSmemMax - b.slab_off - part_bytes - guard) / b.slab_bytes;
    b.TS = ts > kBandMaxTS ? kBandMaxTS : ts;
    b.part_off = b.slab_off + (b.TS > 0 ? b.TS : 0) * b.slab_bytes;
    b.smem = b.part_off + part_bytes + guard;
    return b;
}

__host__ inline bool band_supported(int m, int R) {
    const BandGeom b = band_geom(m, R);
    return b.NQ <= kBandMaxNQ && b.TS >= 2 && b.Xw <= 256 && b.trows <= 256 && b.smem <= kTcSmemMax;
}

enum {
    BD_WFULL = 0,               // window tile slots (2)
    BD_WEMPTY = 2,
    BD_TFULL = 4,               // template slabs (kBandMaxTS)
    BD_TEMPTY = BD_TFULL + kBandMaxTS,
    BD_AFULL = BD_TEMPTY + kBandMaxTS,  // TMEM halves (2)
    BD_AEMPTY = BD_AFULL + 2,
    BD_FIN = BD_AEMPTY + 2,
    BD_N
};

// One stage of the band form: template columns u0 + q (q < nq) of the slab
// at dB against the window tile at dAu = tile + u0, for GG accumulators
// kBandIssuers apart (one issuer's share of the group),
// as straight-line code (an MMA that is predicated off still costs about
// as much issue time as one that runs).  FIRST: the stage of u0 = 0, whose
// first MMA per accumulator overwrites it.
template <int N, int GG, bool FIRST>
__device__ __forceinline__ void band_stage(uint32_t dacc, uint64_t dAu, uint64_t dB, uint32_t tcol, uint32_t idesc,
                                           int nq) {
    if (nq == kBandQ) {
#pragma unroll
        for (int q = 0; q < kBandQ; ++q)
#pragma unroll
            for (int e = 0; e < GG; ++e)
                mma_bf16(dacc + (uint32_t)(e * kBandIssuers * N), dAu + (uint64_t)(q + 8 * kBandIssuers * e),
                         dB + (uint64_t)(q * tcol), idesc,
                         (FIRST && q == 0) ? 0u : 1u);
    } else {
#pragma unroll
        for (int q = 0; q < kBandQ; ++q)
            if (q < nq) {
#pragma unroll
                for (int e = 0; e < GG; ++e)
                    mma_bf16(dacc + (uint32_t)(e * kBandIssuers * N), dAu + (uint64_t)(q + 8 * kBandIssuers * e),
                         dB + (uint64_t)(q * tcol), idesc,
                             (FIRST && q == 0) ? 0u : 1u);
            }
    }
}

template <int N, int GG>
__device__ __forceinline__ void band_stage_any(bool first, uint32_t dacc, uint64_t dAu, uint64_t dB, uint32_t tcol,
                                               uint32_t idesc, int nq) {
    if (first)
        band_stage<N, GG, true>(dacc, dAu, dB, tcol, idesc, nq);
    else
        band_stage<N, GG, false>(dacc, dAu, dB, tcol, idesc, nq);
}

// 16 TMEM columns of this warp's 32 lanes into v[0..15] (no wait)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory layout of one launch, fixed for all its items: two window
// tile slots, TS template slab slots and the partial-sum buffer, each slot
// as large as the largest item of the launch needs.  An item's own geometry
// (band_geom of its m, R) sets what is copied into a slot and how the MMAs
// read it.
struct BandLaunch {
    int TS;            // template slab slots
    int tile_stride;   // bytes per window tile slot
    int slab_stride;   // bytes per template slab slot
    int part_off;      // partial-sum buffer
    int smem;          // dynamic shared memory of the launch
};

// Items: the points of `one`, or (job, point) pairs of a batch; item kk goes
// to CTA kk mod grid (a batch lists its items by decreasing cost).  The
// window tile map is the job's tm[0] (row-major layout rm), the template
// slab map its tm[1] (column-major layout cm).
template <int NQ>
__global__ void __launch_bounds__(kBandThreads, 1)
    k_corr_tc_band(const __grid_constant__ MatchJob one, const MatchJob* __restrict__ jobs,
                   const int2* __restrict__ items, int n_items, const BandLaunch BL, int* __restrict__ err) {
    constexpr int N = NQ * 16;
    constexpr int N4 = N / 4;
    constexpr int GEM = band_ge_max(NQ);
    constexpr int GEI = (GEM + kBandIssuers - 1) / kBandIssuers;  // accumulators per issuer
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar[BD_N];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bars = smem_u32(&s_bar[0]);
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(BD_WFULL + i), 1);
            mbar_init(bar(BD_WEMPTY + i), kBandIssuers);
            mbar_init(bar(BD_AFULL + i), kBandIssuers);
            mbar_init(bar(BD_AEMPTY + i), 4);  // the four warps of the draining team
        }
        for (int i = 0; i < BL.TS; ++i) {
            mbar_init(bar(BD_TFULL + i), 1);
            mbar_init(bar(BD_TEMPTY + i), kBandIssuers);
        }
        mbar_init(bar(BD_FIN), kBandIssuers);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // per-CTA running counts of groups and stages, advanced alike by every role
    uint32_t gc = 0, tc = 0;
    uint32_t t_issued = 0, w_issued = 0;
    bool ok = true;

    const uint32_t TS = (uint32_t)BL.TS;
    const uint32_t slab_off = 2u * (uint32_t)BL.tile_stride;
    for (int kk = blockIdx.x; kk < n_items; kk += gridDim.x) {
        if (warp < 4 && *reinterpret_cast<volatile int*>(&s_abort)) break;  // the drain warps never leave early
        int k;
        const MatchJob& J = item_job(one, jobs, items, kk, &k);
        const PointStat st = J.stats[k];
        if (st.status != SFOC_PT_OK) continue;  // uniform across the CTA
        const int m = J.m, R = J.R;
        const BandGeom g = band_geom(m, R);
        const int h = template_half(m);
        const int ty0 = J.pts[2 * k + 1] - h, tx0 = J.pts[2 * k] - h;
        const int wy0 = ty0 - R, wx0 = tx0 - R;
        if (warp == 0) {
            // ---------------- TMA producer ----------------
            if (lane == 0) {
                uint32_t gp = gc, tp = tc;
                for (int eg = 0; eg < g.nEG && ok; ++eg) {
                    const int e0 = eg * g.GE;
                    for (int yb = 0; yb < g.nYB && ok; ++yb, ++gp) {
                        const uint32_t slot = gp & 1u;
                        if (gp >= 2) ok = mbar_wait(bar(BD_WEMPTY + slot), ((gp >> 1) - 1) & 1, &s_abort);
                        if (!ok) break;
                        mbar_expect_tx(bar(BD_WFULL + slot), (uint32_t)g.tile_bytes);
                        tma_load_4d(sbase + slot * (uint32_t)BL.tile_stride, &J.tm[0], 0, wx0 + 8 * e0, wy0 + 16 * yb, 0,
                                    bar(BD_WFULL + slot));
                        ++w_issued;
                        for (int s = 0; s < g.nS && ok; ++s, ++tp) {
                            const uint32_t ts = tp % TS;
                            if (tp >= TS)
                                ok = mbar_wait(bar(BD_TEMPTY + ts), ((tp / TS) - 1) & 1, &s_abort);
                            if (!ok) break;
                            // a run of 8 rows that starts above the image is zero filled whole, so
                            // the slab starts at row 0 at the latest (the issuer compensates)
                            const int r0 = ty0 + 16 * yb - 2 * R;
                            mbar_expect_tx(bar(BD_TFULL + ts), (uint32_t)g.slab_bytes);
                            tma_load_4d(sbase + slab_off + ts * (uint32_t)BL.slab_stride, &J.tm[1], 0, r0 < 0 ? 0 : r0,
                                        tx0 + s * kBandQ, 0, bar(BD_TFULL + ts));
                            ++t_issued;
                        }
                    }
                }
            }
        } else if (warp >= 1 && warp <= kBandIssuers) {
            // ---------------- MMA issuers ----------------
            // issuer i (warp 1 + i) owns the accumulators e of the group with
            // e mod kBandIssuers == i, so every accumulator's MMAs come from one
            // thread in a fixed order; every issuer takes every stage's waits
            // and commit every barrier a stage or group releases
            if (lane == 0) {
                const int iss = warp - 1;
                const uint64_t da0 = smem_desc(sbase, 16u * g.Xw * 16u, (uint32_t)g.Xw * 16u);
                const uint64_t db0 = smem_desc(sbase + slab_off, (uint32_t)(kBandQ * g.trows * 16), 128);
                const uint32_t tile_step = (uint32_t)BL.tile_stride >> 4, slab_step = (uint32_t)BL.slab_stride >> 4;
                const uint32_t tcol = (uint32_t)g.trows;  // slab column stride in 16-byte units
                uint32_t gi = gc;
                uint32_t ts = tc % TS, tph = (tc / TS) & 1u;
                for (int eg = 0; eg < g.nEG && ok; ++eg) {
                    const int Gg = g.nE - eg * g.GE < g.GE ? g.nE - eg * g.GE : g.GE;
                    for (int yb = 0; yb < g.nYB && ok; ++yb, ++gi) {
                        const uint32_t half = gi & 1u;
                        if (gi >= 2) ok = mbar_wait(bar(BD_AEMPTY + half), ((gi >> 1) - 1) & 1, &s_abort);
                        if (ok) ok = mbar_wait(bar(BD_WFULL + half), (gi >> 1) & 1, &s_abort);
                        if (!ok) break;
                        tc_fence_after();  // the drain's TMEM reads come before these MMAs
                        const uint64_t dA = da0 + (uint64_t)(half * tile_step);
                        const uint32_t dacc = tmem + half * 256u;
                        // B row n is template row 16 yb - 2R + n; a slab clamped to image row 0
                        // holds it clamp rows further on (rows before the slab only meet
                        // template rows i < 0, which the drain drops)
                        const int r0 = ty0 + 16 * yb - 2 * R;
                        const uint32_t clamp = r0 < 0 ? (uint32_t)(-r0) : 0u;
                        // the band meets template rows [nlo, nhi) of its N; its MMAs cover only
                        // the 16-row-aligned span around them (accumulator columns outside it
                        // keep an earlier group's values, which the drain zeroes)
                        const int ilo = 16 * yb - 2 * R;
                        const int nlo = ilo < 0 ? -ilo : 0;
                        const int nhi = m - ilo < N ? m - ilo : N;
                        const int n0 = nlo & ~15;
                        const int n1 = ((nhi + 15) & ~15) < N ? ((nhi + 15) & ~15) : N;
                        const uint32_t idesc_b = idesc_bf16(kM, n1 - n0);
                        // this issuer's accumulators e = iss, iss + kBandIssuers, ...
                        const int Gi = Gg > iss ? (Gg - iss + kBandIssuers - 1) / kBandIssuers : 0;
                        const uint32_t dacc_i = dacc + (uint32_t)n0 + (uint32_t)(iss * N);
                        for (int s = 0; s < g.nS; ++s) {
                            ok = mbar_wait(bar(BD_TFULL + ts), tph, &s_abort);
                            if (!ok) break;
                            tc_fence_after();
                            const uint64_t dB = db0 + (uint64_t)(ts * slab_step) - (uint64_t)clamp + (uint64_t)n0;
                            const int u0 = s * kBandQ;
                            const int nq = m - u0 < kBandQ ? m - u0 : kBandQ;
                            const uint64_t dAu = dA + (uint64_t)u0;
                            switch (Gi) {  // outside the run of MMAs
                                case 0: break;
                                case 1: band_stage_any<N, 1>(s == 0, dacc_i, dAu + (uint64_t)(8 * iss), dB, tcol, idesc_b, nq); break;
                                case 2: band_stage_any<N, GEI < 2 ? GEI : 2>(s == 0, dacc_i, dAu + (uint64_t)(8 * iss), dB, tcol, idesc_b, nq); break;
                                default: band_stage_any<N, GEI < 3 ? GEI : 3>(s == 0, dacc_i, dAu + (uint64_t)(8 * iss), dB, tcol, idesc_b, nq); break;
                            }
                            mma_commit(bar(BD_TEMPTY + ts));
                            if (++ts == TS) { ts = 0; tph ^= 1u; }
                        }
                        if (!ok) break;
                        mma_commit(bar(BD_WEMPTY + half));
                        mma_commit(bar(BD_AFULL + half));
                    }
                }
            }
        } else if (warp >= 4) {
            // ---------------- drain: diagonal sums ----------------
            const int t = tid - 128;  // 0 .. kBandDrain-1
            const int team = t >> 7;
            const int q = warp & 3;
            const int gq = lane >> 3, r = lane & 7;
            const bool b0 = (gq & 1) != 0, b1 = (gq & 2) != 0;
            const int joff = (b0 ? N / 2 : 0) + (b1 ? N4 : 0);
            float* part = reinterpret_cast<float*>(smem + BL.part_off);
            float* out = J.maps + (size_t)k * g.P1 * g.P1;
            const uint32_t lbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)team * 256u;
            uint32_t gd = gc;
            for (int eg = 0; eg < g.nEG; ++eg) {
                const int e0 = eg * g.GE;
                const int Gg = g.nE - e0 < g.GE ? g.nE - e0 : g.GE;
                float sums[GEM][N4];
#pragma unroll
                for (int e = 0; e < GEM; ++e)
#pragma unroll
                    for (int p = 0; p < N4; ++p) sums[e][p] = 0.f;
                for (int yb = 0; yb < g.nYB; ++yb, ++gd) {
                    if ((int)(gd & 1u) != team) continue;
                    // lane 0 takes the bounded wait; the warp follows its verdict
                    int okw = 0;
                    if (lane == 0 && ok) okw = mbar_wait(bar(BD_AFULL + team), (gd >> 1) & 1, &s_abort) ? 1 : 0;
                    okw = __shfl_sync(0xffffffffu, okw, 0);
                    if (!okw) {
                        ok = false;
                        continue;
                    }
                    mbar_wait(bar(BD_AFULL + team), (gd >> 1) & 1, &s_abort);  // completed: acquire for this lane
                    tc_fence_after();
                    // template rows i = 16 yb - 2R + n outside [0, m) are zeroed
                    const int ilo = 16 * yb - 2 * R;
                    const int nlo = ilo < 0 ? -ilo : 0;
                    const int nhi = m - ilo < N ? m - ilo : N;
#pragma unroll
                    for (int e = 0; e < GEM; ++e) {
                        if (e < Gg) {
                            float v[N];
#pragma unroll
                            for (int c = 0; c < NQ; ++c) tmem_ld16_nowait(lbase + (uint32_t)(e * N + 16 * c), v + 16 * c);
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                            if (e == Gg - 1) {  // every accumulator of the group read: release the TMEM half
                                tc_fence_before();
                                __syncwarp();
                                if (lane == 0) mbar_arrive(bar(BD_AEMPTY + team));
                            }
                            if (nlo > 0 || nhi < N) {
#pragma unroll
                                for (int j = 0; j < N; ++j) v[j] = (j >= nlo && j < nhi) ? v[j] : 0.f;
                            }
                            // shift left by g' = 2 b1 + b0
#pragma unroll
                            for (int j = 0; j < N; ++j) v[j] = b0 ? (j + 1 < N ? v[j + 1] : 0.f) : v[j];
#pragma unroll
                            for (int j = 0; j < N; ++j) v[j] = b1 ? (j + 2 < N ? v[j + 2] : 0.f) : v[j];
                            // add the four rows g': lanes 8 apart, then 16 apart
#pragma unroll
                            for (int p = 0; p < N / 2; ++p) {
                                const float lo = v[p], hi = v[p + N / 2];
                                const float snd = b0 ? lo : hi;
                                v[p] = (b0 ? hi : lo) + __shfl_xor_sync(0xffffffffu, snd, 8);
                            }
#pragma unroll
                            for (int p = 0; p < N4; ++p) {
                                const float lo = v[p], hi = v[p + N4];
                                const float snd = b1 ? lo : hi;
                                sums[e][p] += (b1 ? hi : lo) + __shfl_xor_sync(0xffffffffu, snd, 16);
                            }
                        }
                    }
                }
                // sums of this offset-group set: column j = joff + p is dy = 2R + 4q - j.
                // The two teams hold the same entries (each over its own bands): team 0
                // writes them per quarter q, team 1 adds its own in place (a fixed
                // order), then the four quarters are summed
                for (int tm = 0; tm < 2; ++tm) {
                    if (team == tm) {
#pragma unroll
                        for (int e = 0; e < GEM; ++e) {
                            if (e < Gg) {
#pragma unroll
                                for (int p = 0; p < N4; ++p) {
                                    const int dy = 2 * R + 4 * q - joff - p;
                                    if ((unsigned)dy < (unsigned)g.P1) {
                                        float* slot = &part[((q * g.GE + e) * g.P1 + dy) * 8 + r];
                                        *slot = tm == 0 ? sums[e][p] : *slot + sums[e][p];
                                    }
                                }
                            }
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(kBandDrain) : "memory");
                }
                for (int idx = t; idx < Gg * g.P1 * 8; idx += kBandDrain) {
                    const int e = idx / (g.P1 * 8);
                    const int rem = idx - e * g.P1 * 8;
                    const int dy = rem >> 3, rr = rem & 7;
                    const int dx = 8 * (e0 + e) + rr;
                    if (dx < g.P1) {
                        float s = 0.f;
#pragma unroll
                        for (int w = 0; w < 4; ++w) s += part[((w * g.GE + e) * g.P1 + dy) * 8 + rr];
                        out[dy * g.P1 + dx] = s;
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(kBandDrain) : "memory");
            }
        }
        gc += (uint32_t)(g.nEG * g.nYB);
        tc += (uint32_t)(g.nEG * g.nYB * g.nS);
        if (!ok) atomicExch(&s_abort, 1);
    }

    if (*reinterpret_cast<volatile int*>(&s_abort)) {
        if (warp == 0 && lane == 0) {  // let every copy in flight land
            for (uint32_t i = 0; i < (uint32_t)BL.TS && i < t_issued; ++i) {
                const uint32_t ti = t_issued - 1 - i;
                mbar_wait_short(bar(BD_TFULL + ti % BL.TS), (ti / BL.TS) & 1);
            }
            for (uint32_t i = 0; i < 2u && i < w_issued; ++i) {
                const uint32_t wi = w_issued - 1 - i;
                mbar_wait_short(bar(BD_WFULL + (wi & 1u)), (wi >> 1) & 1);
            }
        }
        if (warp >= 1 && warp <= kBandIssuers && lane == 0) {  // and every MMA issued
            mma_commit(bar(BD_FIN));
            mbar_wait_short(bar(BD_FIN), 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_abort && tid == 0) atomicExch(err, 1);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

}  // namespace

bool corr_band_supported(int m, int R) { return band_supported(m, R); }

long long corr_band_mmas(int m, int R) {
    const BandGeom b = band_geom(m, R);
    return (long long)b.nYB * b.nE * m;
}

int corr_band_class(int m, int R) { return band_supported(m, R) ? band_geom(m, R).NQ : 0; }

// The job's tensor maps for the band form: window tiles of 16 rows x Xw
// pixels of rm = [2][H][W][8] (tm[0]) and template slabs of kBandQ columns
// x trows rows of cm = [2][W][H][8] (tm[1]), both in 128-byte runs of 8
// pixels.
bool corr_band_maps(MatchJob& j) {
    const BandGeom bg = band_geom(j.m, j.R);
    return make_map_rows8(&j.tm[0], j.rrm, (uint64_t)j.Wr, (uint64_t)j.Hr, (uint32_t)bg.Xw, 16) &&
           make_map_rows8(&j.tm[1], j.scm, (uint64_t)j.Hs, (uint64_t)j.Ws, (uint32_t)bg.trows, kBandQ);
}

namespace {

// launch layout for items whose (m, R) lie in [*, max_m] x [*, max_R] of one
// class: every slot as large as the class's largest need
bool band_launch(int NQ, const int* ms, const int* Rs, int cnt, BandLaunch* out) {
    int tile = 0, slab = 0, part = 0, guard = 0;
    for (int i = 0; i < cnt; ++i) {
        const BandGeom g = band_geom(ms[i], Rs[i]);
        if (g.NQ != NQ) return false;
        tile = g.tile_bytes > tile ? g.tile_bytes : tile;
        slab = g.slab_bytes > slab ? g.slab_bytes : slab;
        const int pb = 4 * g.GE * g.P1 * 8 * 4;
        part = pb > part ? pb : part;
        const int gd = (g.N - g.trows) * 16 + 128;
        guard = gd > guard ? gd : guard;
    }
    BandLaunch L;
    const int fixed = 2 * tile + part + guard;
    int ts = (kTcSmemMax - fixed) / (slab > 0 ? slab : 1);
    L.TS = ts > kBandMaxTS ? kBandMaxTS : ts;
    L.tile_stride = tile;
    L.slab_stride = slab;
    L.part_off = 2 * tile + L.TS * slab;
    L.smem = L.part_off + part + guard;
    if (L.smem < kBandSmemFloor) L.smem = kBandSmemFloor;
    *out = L;
    return L.TS >= 2 && L.smem <= kTcSmemMax;
}

}  // namespace

// One launch over `is` (single pair: its points); every job of the launch
// in band class NQ with its tensor maps set (corr_band_maps).  ms / Rs: the
// distinct (m, R) of the launch's jobs (their layout bounds).
cudaError_t launch_corr_band(const MatchJob& one, const ItemSet& is, int NQ, const int* ms, const int* Rs, int cnt,
                             int* err_flag, int sms, cudaStream_t st) {
    const int n = is.items ? is.n : one.n;
    if (n <= 0) return cudaSuccess;
    BandLaunch BL;
    if (!band_launch(NQ, ms, Rs, cnt, &BL)) return cudaErrorNotSupported;
    const int grid = n < sms ? n : sms;
    // one CTA per SM: the kernel allocates all 512 TMEM columns, so a second
    // CTA on the SM would block in tcgen05.alloc until the first one's whole
    // persistent loop ended; more than half of the SM's shared memory rules
    // a second CTA out (BandLaunch.smem is at least kBandSmemFloor)
    cudaError_t e = cudaErrorNotSupported;
#define SFOC_BAND_CASE(NQV)                                                                                   \
    case NQV:                                                                                                 \
        e = cudaFuncSetAttribute(k_corr_tc_band<NQV>, cudaFuncAttributeMaxDynamicSharedMemorySize, BL.smem); \
        if (e != cudaSuccess) return e;                                                                       \
        k_corr_tc_band<NQV><<<grid, kBandThreads, BL.smem, st>>>(one, is.jobs, is.items, n, BL, err_flag);     \
        return cudaGetLastError();
    switch (NQ) {
        SFOC_BAND_CASE(1)
        SFOC_BAND_CASE(2)
        SFOC_BAND_CASE(3)
        SFOC_BAND_CASE(4)
        SFOC_BAND_CASE(5)
        SFOC_BAND_CASE(6)
        default: break;
    }
#undef SFOC_BAND_CASE
    return e;
}

}  // namespace sfoc
