// Correlation R_ST (Eq. 10 of arXiv 2202.13347) as a tcgen05 BF16 implicit
// GEMM with FP32 accumulation in tensor memory (sm_103a).
//
// Out[dy][dx] = sum_{c,y,u} S[c][y][u+dx] * T[c][y-dy][u]
//   S: reference window (m+2R)^2 around p (rows/cols from p - h - R),
//   T: template m^2 from the sensed cube, zero outside [0, m)^2.
// GEMM form D[r][n] = sum_k A[r][k] B[n][k]:
//   r = dx (M = 128 rows; rows > 2R are discarded),
//   n = 2R - dy (N = roundup(2R+1, 16)),
//   k = (y, u, channel); one instruction covers one (y, u) and 16 channels
//   (12 + 4 zero pad) as two 8-channel chunks LBO apart.
// Both operands are K-major without swizzle.  A core-matrix row is the 16 B
// chunk of 8 channels of one pixel, so
//   A row r = window pixel (y, u + r): in the row-major pixel layout rows are
//             consecutive chunks, a shift in dx is a 16 B step of the
//             descriptor start;
//   B row n = template pixel (y - 2R + n, u): in the column-major layout
//             consecutive n are consecutive chunks (Toeplitz along y through
//             address arithmetic, no copies).
//
// Data movement, per point:
//   template column block (U columns x (m+2R+N-1) rows, i.e. the template
//   plus the rows above and below it): TMA loads, then two warps zero the
//   rows outside [0, m); reused for every window row of the point;
//   window slab (8 rows x (U+2R) columns): one 4-D TMA load per K stage into
//   a ring of NA buffers.
// Warp roles (256 threads):
//   warp 0 lane 0  TMA producer          warp 1 lane 0  MMA issuer
//   warps 2-3      template zero rows    warps 4-7      TMEM drain + output
// The MMAs of one K stage (8 window rows x U template columns) go to one of
// two TMEM accumulators; the drain warps add it into FP32 registers with
// round-to-nearest while the next stage runs.  (The tensor core truncates
// as it accumulates: a single accumulator over ~10^4 MMAs biased R_ST by
// about -5e-5 relative; per-stage partial sums keep that near 2e-6.)
// Each MMA's N is trimmed to the 16-column band where the Toeplitz operand
// is non-zero for its window row; the first MMA of a stage is full width so
// that it initialises the whole accumulator.
//
// Every wait is bounded (about 2 s of %globaltimer); on expiry the CTA sets
// the context's device error word, every role leaves its loop, the producer
// waits (bounded) for its copies still in flight, TMEM is freed and the
// kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <type_traits>

#include "internal.h"
#include "tc_ptx.h"

namespace sfoc {

namespace {

using namespace tcx;

constexpr int kThreads = 256;
constexpr int kY = 8;    // window rows per stage
constexpr int kMaxNA = 6;

struct TcGeom {
    int m, R, P1, Lw, Npad, U, AW, JB, JS, NA, tmem_cols, acc_stride;
    int a_bytes, b_bytes;   // one window slab / one template column block (both chunks)
    int a_off, b_off;       // shared-memory offsets of the A ring and the B pair
    int smem;               // dynamic shared memory used (incl. a 2 KB guard)
};

__host__ __device__ inline TcGeom tc_geom(int m, int R, int U) {
    TcGeom g;
    g.m = m;
    g.R = R;
    g.P1 = 2 * R + 1;
    g.Lw = m + 2 * R;
    g.Npad = (g.P1 + 15) / 16 * 16;
    g.U = U;
    g.AW = U + 2 * R;
    g.JB = g.Lw + g.Npad - 1;
    g.JS = (g.JB + 7) / 8 * 8;  // column stride: every TMA destination 128-byte aligned
    g.a_bytes = 2 * kY * g.AW * 16;
    g.b_bytes = 2 * U * g.JS * 16;
    const int budget = 224 * 1024 - 2048;
    int na = (budget - 2 * g.b_bytes) / g.a_bytes;
    g.NA = na > kMaxNA ? kMaxNA : na;
    g.a_off = 0;
    g.b_off = g.NA * g.a_bytes;
    g.smem = g.b_off + 2 * g.b_bytes + 2048;
    g.acc_stride = (g.Npad + 31) / 32 * 32;
    int c = 32;
    while (c < 2 * g.acc_stride) c <<= 1;
    g.tmem_cols = c;
    return g;
}

// barrier slots
enum {
    BA_FULL = 0,
    BA_EMPTY = kMaxNA,
    BB_FULL = 2 * kMaxNA,
    BB_READY = BB_FULL + 2,
    BB_EMPTY = BB_READY + 2,
    BACC_FULL = BB_EMPTY + 2,
    BACC_EMPTY = BACC_FULL + 2,
    NBAR = BACC_EMPTY + 2
};

// NQ = number of 16-column accumulator chunks (Npad / 16), UC = template
// columns per column block (8, or 4 for the largest windows)
// One pair (`one`): its window slab map tm[0], template column maps tm[1]
// (rows [0, 256)) and tm[2] (rows past 256).
template <int NQ, int UC>
__global__ void __launch_bounds__(kThreads, 1)
    k_corr_tc(const __grid_constant__ MatchJob one, int* __restrict__ err) {
    const CUtensorMap& tmA = one.tm[0];
    const CUtensorMap& tmB = one.tm[1];
    const CUtensorMap& tmB2 = one.tm[2];
    const int32_t* __restrict__ pts = one.pts;
    const int n = one.n, m = one.m, R = one.R;
    const PointStat* __restrict__ stats = one.stats;
    float* __restrict__ maps = one.maps;
    constexpr int U = UC;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar[NBAR];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const TcGeom g = tc_geom(m, R, U);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int h = template_half(m);
    const int nyb = (g.Lw + kY - 1) / kY, nub = (m + U - 1) / U;
    const int T = nyb * nub;
    const uint32_t sbase = smem_u32(smem);
    uint32_t bars = smem_u32(&s_bar[0]);
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };

    if (tid == 0) {
        for (int i = 0; i < kMaxNA; ++i) {
            mbar_init(bar(BA_FULL + i), 1);
            mbar_init(bar(BA_EMPTY + i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(BB_FULL + i), 1);
            mbar_init(bar(BB_READY + i), 2);    // the two zeroing warps
            mbar_init(bar(BB_EMPTY + i), 1);
            mbar_init(bar(BACC_FULL + i), 1);
            mbar_init(bar(BACC_EMPTY + i), 4);  // the four drain warps
        }
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

    uint32_t gs = 0;        // K stages of this CTA so far
    uint32_t gb = 0;        // template column blocks of this CTA so far
    uint32_t a_issued = 0;  // producer: window slabs issued
    uint32_t b_issued = 0;  // producer: column blocks issued

    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        if (*reinterpret_cast<volatile int*>(&s_abort)) break;
        const PointStat st = stats[k];
        if (st.status != SFOC_PT_OK) continue;  // uniform across the CTA
        const int ty0 = pts[2 * k + 1] - h, tx0 = pts[2 * k] - h;
        const int wy0 = ty0 - R, wx0 = tx0 - R;
        bool ok = true;

        if (warp == 0) {
            // ---------------- TMA producer ----------------
            if (lane == 0) {
                for (int s = 0; s < T && ok; ++s) {
                    const int ub = s / nyb, yb = s - ub * nyb;
                    const uint32_t ga = gs + s;
                    if (yb == 0) {
                        const uint32_t gk = gb + ub, bb = gk & 1;
                        if (gk >= 2) ok = mbar_wait(bar(BB_EMPTY + bb), ((gk >> 1) - 1) & 1, &s_abort);
                        if (!ok) break;
                        const uint32_t bdst = sbase + g.b_off + bb * g.b_bytes;
                        mbar_expect_tx(bar(BB_FULL + bb), g.b_bytes);
                        for (int cg = 0; cg < 2; ++cg)
                            for (int ul = 0; ul < U; ++ul) {
                                const uint32_t cdst = bdst + (cg * U + ul) * g.JS * 16;
                                const int cx = tx0 + ub * U + ul, cy = ty0 - 2 * R;
                                tma_load_4d(cdst, &tmB, 0, cy, cx, cg, bar(BB_FULL + bb));
                                if (g.JS > 256) tma_load_4d(cdst + 256 * 16, &tmB2, 0, cy + 256, cx, cg, bar(BB_FULL + bb));
                            }
                        ++b_issued;
                    }
                    const uint32_t slot = ga % g.NA;
                    if (ga >= (uint32_t)g.NA) ok = mbar_wait(bar(BA_EMPTY + slot), ((ga / g.NA) - 1) & 1, &s_abort);
                    if (!ok) break;
                    mbar_expect_tx(bar(BA_FULL + slot), g.a_bytes);
                    tma_load_4d(sbase + g.a_off + slot * g.a_bytes, &tmA, 0, wx0 + ub * U, wy0 + yb * kY, 0,
                                bar(BA_FULL + slot));
                    ++a_issued;
                }
            }
        } else if (warp == 1) {
            // ---------------- MMA issuer ----------------
            if (lane == 0) {
                const uint32_t a_lbo = kY * g.AW * 16, b_lbo = UC * g.JS * 16;
                const uint32_t id_full = idesc_bf16(kM, g.Npad);
                // non-zero band of B rows for window row y: j = y - 2R + n in [0, m),
                // rounded out to 16 rows
                auto n0_tab = [&](int y) {
                    int nlo = 2 * R - y;
                    nlo = nlo < 0 ? 0 : nlo;
                    return (nlo / 16) * 16;
                };
                auto id_tab = [&](int y) {
                    int nhi = m + 2 * R - y;
                    nhi = nhi > g.Npad ? g.Npad : nhi;
                    const int n1 = (nhi + 15) / 16 * 16;
                    return idesc_bf16(kM, n1 - n0_tab(y));
                };
                for (int s = 0; s < T && ok; ++s) {
                    const int ub = s / nyb, yb = s - ub * nyb;
                    const uint32_t ga = gs + s, slot = ga % g.NA, acc = ga & 1;
                    const uint32_t gk = gb + ub, bb = gk & 1;
                    if (yb == 0) ok = mbar_wait(bar(BB_READY + bb), (gk >> 1) & 1, &s_abort);
                    if (ok) ok = mbar_wait(bar(BA_FULL + slot), (ga / g.NA) & 1, &s_abort);
                    if (ok && ga >= 2) ok = mbar_wait(bar(BACC_EMPTY + acc), ((ga >> 1) - 1) & 1, &s_abort);
                    if (!ok) break;
                    tc_fence_after();
                    // descriptors advance in 16-byte units by plain integer adds
                    const uint64_t da0 = smem_desc(sbase + g.a_off + slot * g.a_bytes, a_lbo, 128);
                    const uint64_t db0 = smem_desc(sbase + g.b_off + bb * g.b_bytes, b_lbo, 128);
                    const uint32_t dacc = tmem + acc * g.acc_stride;
                    const int y0 = yb * kY, u0 = ub * UC;
                    const int ulim = m - u0 < UC ? m - u0 : UC;
                    const int ylim = g.Lw - y0 < kY ? g.Lw - y0 : kY;
                    // first MMA of the stage: full width, overwrites the accumulator
                    mma_bf16(dacc, da0, db0 + (uint64_t)y0, id_full, 0u);
#pragma unroll
                    for (int yl = 0; yl < kY; ++yl) {
                        if (yl < ylim) {
                            const int y = y0 + yl;
                            const int n0 = yl == 0 ? 0 : n0_tab(y);
                            const uint32_t id = yl == 0 ? id_full : id_tab(y);
                            const uint64_t da = da0 + (uint64_t)(yl * g.AW);
                            const uint64_t db = db0 + (uint64_t)(y + n0);
                            const uint32_t dd = dacc + (uint32_t)n0;
#pragma unroll
                            for (int ul = 0; ul < UC; ++ul) {
                                if ((yl > 0 || ul > 0) && ul < ulim)
                                    mma_bf16(dd, da + (uint64_t)ul, db + (uint64_t)(ul * g.JS), id, 1u);
                            }
                        }
                    }
                    mma_commit(bar(BA_EMPTY + slot));
                    mma_commit(bar(BACC_FULL + acc));
                    if (yb == nyb - 1) mma_commit(bar(BB_EMPTY + bb));
                }
            }
        } else if (warp < 4) {
            // ---------------- template zero rows ----------------
            const int t = tid - 64;  // 0..63
            for (int ub = 0; ub < nub && ok; ++ub) {
                const uint32_t gk = gb + ub, bb = gk & 1;
                ok = mbar_wait(bar(BB_FULL + bb), (gk >> 1) & 1, &s_abort);
                if (!ok) break;
                uint8_t* b = smem + g.b_off + bb * g.b_bytes;
                const int nz_lo = 2 * R;               // rows j < 0
                const int nz_hi = g.JS - (m + 2 * R);  // rows j >= m, incl. the stride padding
                const int per_col = nz_lo + nz_hi;
                const int total = 2 * U * per_col;
                for (int i = t; i < total; i += 64) {
                    const int col = i / per_col, rr = i - col * per_col;
                    const int jl = rr < nz_lo ? rr : m + 2 * R + (rr - nz_lo);
                    *reinterpret_cast<uint4*>(b + ((size_t)col * g.JS + jl) * 16) = make_uint4(0, 0, 0, 0);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(BB_READY + bb));
            }
        } else {
            // ---------------- TMEM drain + output ----------------
            const int quarter = warp & 3;
            float accr[NQ][16];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int i = 0; i < 16; ++i) accr[q][i] = 0.f;
            for (int s = 0; s < T && ok; ++s) {
                const uint32_t ga = gs + s, acc = ga & 1;
                ok = mbar_wait(bar(BACC_FULL + acc), (ga >> 1) & 1, &s_abort);
                if (!ok) break;
                tc_fence_after();
                const uint32_t abase = tmem + ((uint32_t)(quarter * 32) << 16) + acc * g.acc_stride;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    float v[16];
                    tmem_ld16(abase + q * 16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) accr[q][i] += v[i];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(BACC_EMPTY + acc));
            }
            if (ok) {
                const int r = quarter * 32 + lane;  // dx
                float* out = maps + (size_t)k * g.P1 * g.P1;
                if (r < g.P1) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int dy = 2 * R - (q * 16 + i);
                            if (dy >= 0) out[dy * g.P1 + r] = accr[q][i];
                        }
                }
            }
        }
        gs += T;
        gb += nub;
        if (!ok) atomicExch(&s_abort, 1);
    }

    if (warp == 0 && lane == 0 && *reinterpret_cast<volatile int*>(&s_abort)) {
        // let every copy this CTA issued land before the CTA leaves
        for (uint32_t i = 0; i < (uint32_t)g.NA && i < a_issued; ++i) {
            const uint32_t ga = a_issued - 1 - i;
            mbar_wait_short(bar(BA_FULL + ga % g.NA), (ga / g.NA) & 1);
        }
        for (uint32_t i = 0; i < 2 && i < b_issued; ++i) {
            const uint32_t gk = b_issued - 1 - i;
            mbar_wait_short(bar(BB_FULL + (gk & 1)), (gk >> 1) & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_abort && tid == 0) atomicExch(err, 1);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Column form (window at most 128 rows tall).
//
// For a group of G offsets dx = d0 .. d0+G-1, TMEM accumulator g holds
//   D_g[y][i] = sum_{u, c} S[c][y][u + dx] T[c][i][u]
// with M = window row y (128 rows), N = template row i (m rounded up to 16)
// and K = (template column u, 16 channels): one MMA per (dx, u).  Then
//   Out[dy][dx] = sum_{i < m} D_g[i + dy][i],
// a sum along a diagonal, done by the drain warps through shared memory.
// Template rows i >= m (image rows below the template, or the copy's zero
// fill) only reach accumulator columns i >= m, which no diagonal sum reads,
// so they need no clearing.  Per point this issues (2R+1) m MMAs of
// N = roundup(m, 16) instead of the (m+2R) m narrow MMAs of the Toeplitz form.
//
// Operands come from the column-major pixel layout (cm) in slabs of kColQ
// image columns, one 4-D tensor copy each.  The copy engine moves about one
// innermost-dimension row per cycle, so the map's innermost dimension is 8
// consecutive pixels of one 8-channel chunk (128 contiguous bytes), its
// second dimension the pixel row with a 16-byte stride, traversed with an
// element stride of 8: a box row is then 8 pixels starting at any row.
//   template slab s of a group: template columns 8s .. 8s+7, roundup(m, 8)
//                               rows each;
//   window slab b of a group:   window columns d0 + 8b .. d0 + 8b + 7,
//                               roundup(m + 2R, 8) rows each.
// Columns past the region are loaded too (or zero filled past the image);
// rows past the region read on into the next image column (the cube buffers
// carry padding for the last one).  None of it reaches a used accumulator
// entry: an MMA reads 128 window rows and roundup(m, 16) template rows from
// a column's start, and rows past the region only feed accumulator rows
// y >= m + 2R or columns i >= m, which no diagonal sum reads.
// The issuer works in stages of kColQ template columns: it waits once for
// the stage's slabs, then issues the stage's kColQ x G MMAs as straight code
// from precomputed descriptors (control flow between tcgen05.mma
// instructions costs far more issue time than integer work) and commits
// once.  A relay warp turns each stage commit into the releases of the
// stage's slabs.  Each accumulator spans m MMAs, so the tensor core's
// truncating accumulation stays small.
// ---------------------------------------------------------------------------
constexpr int kColMaxG = 16;
constexpr int kColQ = 8;   // template columns per stage and columns per slab
constexpr int kColMaxWS = 4;
constexpr int kColMaxTS = 2;
constexpr int kColSmemMax = kTcSmemMax;
// Stage-done barriers.  The issuer can run at most TS stages ahead of the
// relay (a template slab is reused only after the relay freed it), so with
// more barriers than that no barrier completes twice before the relay has
// seen the first phase.
constexpr int kColNS = 8;
constexpr int kColDB = 4;  // TMEM chunks of 16 columns per drain load batch
// 12 warps: 0 TMA producer, 1 and 3 MMA issuers, 2 release relay,
// 4..11 drain (two teams of four, one warp per TMEM lane quarter each)
constexpr int kColThreads = 384;
constexpr int kColDrain = 256;

struct ColGeom {
    int m, R, P1, Lw, Npad, G;
    int wrows, trows;          // rows loaded per window / template column (multiples of 8)
    int WS, TS;                // window / template slab ring sizes
    int ws_bytes, ts_bytes;    // slab sizes
    int NB;                    // band buffers (accumulators drained before the sums)
    int bk_bytes;              // one band buffer (with 32 dummy slots)
    int t_off, w_off, bk_off;  // shared-memory offsets
    int part_off;              // partial diagonal sums: NB x kColDrain floats
    int bk_stride;             // band buffer row stride in floats (odd: no bank conflicts)
    int smem;
};

__host__ __device__ inline ColGeom col_geom(int m, int R) {
    ColGeom c;
    c.m = m;
    c.R = R;
    c.P1 = 2 * R + 1;
    c.Lw = m + 2 * R;
    c.Npad = (m + 15) / 16 * 16;
    int G = 512 / c.Npad;
    G = G > c.P1 ? c.P1 : G;
    c.G = G > kColMaxG ? kColMaxG : G;
    // a stage reads `span` window slabs; one more is in flight, and one
    // template slab besides the stage's own (a copy lands in ~1.2K cycles,
    // a stage takes ~3K)
    const int span = (kColQ + c.G - 2) / kColQ + 1;
    c.WS = span + 1;
    c.TS = kColMaxTS;
    c.wrows = (c.Lw + 7) / 8 * 8;
    c.trows = (m + 7) / 8 * 8;
    c.ws_bytes = 2 * kColQ * c.wrows * 16;
    c.ts_bytes = 2 * kColQ * c.trows * 16;
    c.t_off = 0;
    c.w_off = c.TS * c.ts_bytes;
    c.bk_stride = c.m | 1;
    c.bk_off = c.w_off + c.WS * c.ws_bytes;
    c.bk_bytes = ((c.P1 * c.bk_stride + 32) * 4 + 127) / 128 * 128;
    // an MMA on the last window slab may read up to 2048 - 16 wrows bytes
    // past it (template slabs are followed by the window slabs)
    const int guard = 2048 - 16 * c.wrows;
    int nb = (kColSmemMax - c.bk_off - guard) / (c.bk_bytes + kColDrain * 4);
    nb = nb > c.G ? c.G : nb;
    c.NB = nb < 1 ? 1 : nb;
    c.part_off = c.bk_off + c.NB * c.bk_bytes;
    c.smem = c.part_off + c.NB * kColDrain * 4 + guard;
    // one CTA per SM: the CTA allocates all 512 TMEM columns
    c.smem = c.smem < 120 * 1024 ? 120 * 1024 : c.smem;
    return c;
}

enum {
    CB_WEMPTY = 0,
    CB_TFULL = kColMaxWS,  // per stage: the template slab and the window slabs loaded with it
    CB_TEMPTY = CB_TFULL + kColMaxTS,
    CB_STG = CB_TEMPTY + kColMaxTS,
    CB_AFULL = CB_STG + kColNS,
    CB_AEMPTY,  // per accumulator: its contents read by every drain warp
    CB_FIN = CB_AEMPTY + kColMaxG,
    CB_N
};

// Shared-memory layout of one column-form launch, fixed for all its items:
// TS template slab slots and WS window slab slots (both counts set by the
// class's G), each as large as the launch's largest item needs, then the
// band buffers and partial sums, whose number (NB) each item derives from
// the room left (col_item).
struct ColLaunch {
    int WS, TS;
    int ts_stride, ws_stride;  // bytes per template / window slab slot
    int w_off, bk_off;
    int smem;
};

// An item's geometry inside a launch: its own slab shapes and band buffers,
// the launch's slots and offsets.
__host__ __device__ inline ColGeom col_item(int m, int R, const ColLaunch& L) {
    ColGeom c = col_geom(m, R);
    c.WS = L.WS;
    c.TS = L.TS;
    c.t_off = 0;
    c.w_off = L.w_off;
    c.bk_off = L.bk_off;
    const int guard = 2048 - 16 * c.wrows;
    int nb = (L.smem - c.bk_off - guard) / (c.bk_bytes + kColDrain * 4);
    nb = nb > c.G ? c.G : nb;
    c.NB = nb < 1 ? 1 : nb;
    c.part_off = c.bk_off + c.NB * c.bk_bytes;
    c.smem = L.smem;
    return c;
}

// Items: the points of `one`, or (job, point) pairs of a batch whose jobs
// all have col_geom(m, R).G == G; item kk goes to CTA kk mod grid.  The
// window slab map is the job's tm[0], the template slab map its tm[1] (both
// over the column-major layout cm).
template <int G>
__global__ void __launch_bounds__(kColThreads, 1)
    k_corr_tc_col(const __grid_constant__ MatchJob one, const MatchJob* __restrict__ jobs,
                  const int2* __restrict__ items, int n_items, const ColLaunch CL, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar[CB_N];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_go;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bars = smem_u32(&s_bar[0]);
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };

    if (tid == 0) {
        for (int i = 0; i < CL.WS; ++i) mbar_init(bar(CB_WEMPTY + i), 1);
        for (int i = 0; i < CL.TS; ++i) {
            mbar_init(bar(CB_TFULL + i), 1);
            mbar_init(bar(CB_TEMPTY + i), 1);
        }
        for (int i = 0; i < kColNS; ++i) mbar_init(bar(CB_STG + i), 2);  // both issuers
        mbar_init(bar(CB_AFULL), 2);
        for (int i = 0; i < kColMaxG; ++i) mbar_init(bar(CB_AEMPTY + i), kColDrain / 32);  // every drain warp
        mbar_init(bar(CB_FIN), 2);
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

    // per-CTA running counts (window slabs, template slabs = stages, groups),
    // advanced identically by every role
    uint32_t wsc = 0, tsc = 0, grp = 0;
    uint32_t t_issued = 0;

    for (int kk = blockIdx.x; kk < n_items; kk += gridDim.x) {
        if (*reinterpret_cast<volatile int*>(&s_abort)) break;
        int k;
        const MatchJob& J = item_job(one, jobs, items, kk, &k);
        const PointStat st = J.stats[k];
        if (st.status != SFOC_PT_OK) continue;  // uniform across the CTA
        const int m = J.m, R = J.R;
        const ColGeom g = col_item(m, R, CL);
        const int nstage = (m + kColQ - 1) / kColQ;  // stages (template slabs) per group
        const int h = template_half(m);
        const int ty0 = J.pts[2 * k + 1] - h, tx0 = J.pts[2 * k] - h;
        const int wy0 = ty0 - R, wx0 = tx0 - R;
        bool ok = true;
        if (warp == 0) {
            // ---------------- TMA producer ----------------
            if (lane == 0) {
                uint32_t wv = wsc, tv = tsc;
                for (int d0 = 0; d0 < g.P1 && ok; d0 += G) {
                    const int Gg = g.P1 - d0 < G ? g.P1 - d0 : G;
                    const int nws = (m + Gg - 1 + kColQ - 1) / kColQ;
                    int wl = 0;  // window slabs of the group loaded
                    for (int s = 0; s < nstage && ok; ++s) {
                        // stage s: template slab s and the window slabs up to
                        // the last one it reads, all completing on the
                        // template slot's barrier (one wait per stage)
                        int last = (s * kColQ + kColQ - 1 + Gg - 1) / kColQ;
                        last = last > nws - 1 ? nws - 1 : last;
                        if (s == nstage - 1) last = nws - 1;
                        const uint32_t tslot = tv % g.TS;
                        if (tv >= (uint32_t)g.TS)
                            ok = mbar_wait(bar(CB_TEMPTY + tslot), ((tv / g.TS) - 1) & 1, &s_abort);
                        for (uint32_t wi = wv; ok && wi < wv + (uint32_t)(last + 1 - wl); ++wi)
                            if (wi >= (uint32_t)g.WS)
                                ok = mbar_wait(bar(CB_WEMPTY + wi % g.WS), ((wi / g.WS) - 1) & 1, &s_abort);
                        if (!ok) break;
                        const uint32_t full = bar(CB_TFULL + tslot);
                        mbar_expect_tx(full, (uint32_t)g.ts_bytes + (uint32_t)(last + 1 - wl) * (uint32_t)g.ws_bytes);
                        tma_load_4d(sbase + g.t_off + tslot * (uint32_t)CL.ts_stride, &J.tm[1], 0, ty0, tx0 + s * kColQ, 0,
                                    full);
                        ++tv;
                        ++t_issued;
                        for (; wl <= last; ++wl, ++wv)
                            tma_load_4d(sbase + g.w_off + (wv % g.WS) * (uint32_t)CL.ws_stride, &J.tm[0], 0, wy0,
                                        wx0 + d0 + wl * kColQ, 0, full);
                    }
                }
            }
        } else if (warp == 1 || warp == 3) {
            // ---------------- MMA issuers ----------------
            // warp 1 issues the even accumulators gi of a group, warp 3 the odd
            // ones: each accumulator's MMAs come from one thread in a fixed
            // order, and while one thread stalls at a stage barrier the other
            // keeps the tensor pipe's queue fed.  Both take every wait and
            // commit every stage and group barrier.
            auto issue = [&](auto iss_c) {
                constexpr int ISS = decltype(iss_c)::value;
                const uint32_t idesc = idesc_bf16(kM, g.Npad);
                const uint32_t wcol = (uint32_t)g.wrows;  // window column stride in 16-byte units
                const uint32_t tcol = (uint32_t)g.trows;  // template column stride in 16-byte units
                const uint64_t da_base = smem_desc(sbase + g.w_off, kColQ * g.wrows * 16u, 128);
                const uint64_t db_base = smem_desc(sbase + g.t_off, kColQ * g.trows * 16u, 128);
                const uint32_t w_step = (uint32_t)CL.ws_stride >> 4, t_step = (uint32_t)CL.ts_stride >> 4;
                uint32_t dD[G];
#pragma unroll
                for (int gi = 0; gi < G; ++gi) dD[gi] = tmem + (uint32_t)(gi * g.Npad);
                constexpr int kSpan = (kColQ + G - 2) / kColQ + 1;  // window slabs one stage reads
                uint32_t stg = tsc % kColNS;                         // stage-done barrier of the next stage
                // ring positions kept as running slot / parity pairs (no
                // divisions on the issue path)
                uint32_t gg = grp;
                uint32_t ts = tsc % g.TS, tph = (tsc / g.TS) & 1;  // template slab of the next stage
                uint32_t ws = wsc % g.WS, wph = (wsc / g.WS) & 1;  // window slab 0 of the current group
                for (int d0 = 0; d0 < g.P1 && ok; d0 += G, ++gg) {
                    const int Gg = g.P1 - d0 < G ? g.P1 - d0 : G;
                    const int nws = (m + Gg - 1 + kColQ - 1) / kColQ;
                    uint32_t wcur = ws;  // slot of window slab s
                    for (int s = 0; s < nstage && ok; ++s) {
                        const int u0 = s * kColQ;
                        const int nq = m - u0 < kColQ ? m - u0 : kColQ;
                        // the stage's template slab and every window slab it
                        // reads complete on this barrier or an earlier stage's
                        ok = mbar_wait(bar(CB_TFULL + ts), tph, &s_abort);
                        if (!ok) break;
                        // descriptors: window slabs s .. s+kSpan-1, template slab ts
                        uint64_t dW[kSpan];
#pragma unroll
                        for (int e = 0; e < kSpan; ++e) {
                            uint32_t sl = wcur + (uint32_t)e;
                            if (sl >= (uint32_t)g.WS) sl -= (uint32_t)g.WS;
                            dW[e] = da_base + (uint64_t)(sl * w_step);
                        }
                        const uint64_t dT = db_base + (uint64_t)(ts * t_step);
                        const uint32_t acc0 = u0 > 0 ? 1u : 0u;
                        if (s == 0) {
                            // the group's first stage accumulator by accumulator: each
                            // starts once the drain has read the previous group's
                            // contents of it (the drain releases them one by one)
#pragma unroll
                            for (int gi = 0; gi < G; ++gi) {
                                if ((gi & 1) == ISS && gi < Gg) {
                                    if (gg >= 1) {
                                        ok = mbar_wait(bar(CB_AEMPTY + gi), (gg - 1) & 1, &s_abort);
                                        if (!ok) break;
                                        tc_fence_after();  // the drain's TMEM reads come before these MMAs
                                    }
#pragma unroll
                                    for (int q = 0; q < kColQ; ++q)
                                        if (q < nq)
                                            mma_bf16(dD[gi],
                                                     dW[(q + gi) / kColQ] + (uint64_t)(((q + gi) % kColQ) * wcol),
                                                     dT + (uint64_t)(q * tcol), idesc, q > 0 ? 1u : 0u);
                                }
                            }
                            if (!ok) break;
                        } else if (nq == kColQ && Gg == G) {
#pragma unroll
                            for (int q = 0; q < kColQ; ++q)
#pragma unroll
                                for (int gi = 0; gi < G; ++gi)
                                    if ((gi & 1) == ISS)
                                        mma_bf16(dD[gi], dW[(q + gi) / kColQ] + (uint64_t)(((q + gi) % kColQ) * wcol),
                                                 dT + (uint64_t)(q * tcol), idesc, q > 0 ? 1u : acc0);
                        } else {
#pragma unroll
                            for (int q = 0; q < kColQ; ++q)
                                if (q < nq) {
#pragma unroll
                                    for (int gi = 0; gi < G; ++gi)
                                        if ((gi & 1) == ISS && gi < Gg)
                                            mma_bf16(dD[gi],
                                                     dW[(q + gi) / kColQ] + (uint64_t)(((q + gi) % kColQ) * wcol),
                                                     dT + (uint64_t)(q * tcol), idesc, q > 0 ? 1u : acc0);
                                }
                        }
                        if (s == nstage - 1) mma_commit(bar(CB_AFULL));
                        mma_commit(bar(CB_STG + stg));
                        if (++stg == (uint32_t)kColNS) stg = 0;
                        if (++ts == (uint32_t)g.TS) { ts = 0; tph ^= 1u; }
                        if (++wcur == (uint32_t)g.WS) wcur = 0;
                    }
                    // the next group's window slab 0 follows this group's last slab
                    for (int b2 = 0; b2 < nws; ++b2)
                        if (++ws == (uint32_t)g.WS) { ws = 0; wph ^= 1u; }
                }
            };
            if (lane == 0) {
                if (warp == 1)
                    issue(std::integral_constant<int, 0>{});
                else
                    issue(std::integral_constant<int, 1>{});
            }
        } else if (warp == 2) {
            // ---------------- slab release relay ----------------
            if (lane == 0) {
                uint32_t wv = wsc, tv = tsc;
                for (int d0 = 0; d0 < g.P1 && ok; d0 += G) {
                    const int Gg = g.P1 - d0 < G ? g.P1 - d0 : G;
                    const int nws = (m + Gg - 1 + kColQ - 1) / kColQ;
                    for (int s = 0; s < nstage && ok; ++s, ++tv) {
                        ok = mbar_wait(bar(CB_STG + tv % kColNS), (tv / kColNS) & 1, &s_abort);
                        if (!ok) break;
                        // template slab s; window slab s (its last reader is
                        // stage s); at the group's end every remaining slab
                        mbar_arrive(bar(CB_TEMPTY + tv % g.TS));
                        const int hi = s == nstage - 1 ? nws : s + 1;
                        for (int b = s; b < hi; ++b) mbar_arrive(bar(CB_WEMPTY + (wv + (uint32_t)b) % g.WS));
                    }
                    wv += (uint32_t)nws;
                }
            }
        } else if (warp >= 4) {
            // ---------------- drain: diagonal sums ----------------
            // Thread t holds accumulator row y (its TMEM lane) and stores the
            // band entries D[y][c], 0 <= y - c < 2R+1, c < m, skewed into
            // bk[y - c][c] (one buffer per accumulator of a round); the two
            // teams split each warp's 16-column chunks.  Then nparts threads
            // per dy sum row dy of each buffer.
            const int t = tid - 128;  // 0 .. kColDrain-1
            const int team = (warp - 4) >> 2;
            const int quarter = warp & 3;
            const int y = quarter * 32 + lane;
            const int Sb = g.bk_stride;
            int nparts = kColDrain / g.P1;
            nparts = nparts > 8 ? 8 : nparts;
            const int dy = t % g.P1, part = t / g.P1;
            const int c0 = part * m / nparts, c1 = (part + 1) * m / nparts;
            // 16-column chunks that hold band entries of this warp's rows,
            // split between the teams
            int clo = quarter * 32 - 2 * R;
            clo = clo < 0 ? 0 : clo / 16;
            int chi = quarter * 32 + 31;
            chi = chi > m - 1 ? m - 1 : chi;
            chi = chi / 16;
            {
                const int nch = chi - clo + 1, h0 = (nch + 1) / 2;
                if (team == 0) chi = clo + h0 - 1;
                else clo = clo + h0;
            }
            const int dummy = g.P1 * Sb + lane;  // per-lane slot for entries outside the band
            float* pbuf = reinterpret_cast<float*>(smem + g.part_off);
            float* out = J.maps + (size_t)k * g.P1 * g.P1;
            const uint32_t lbase = tmem + ((uint32_t)(quarter * 32) << 16);
            uint32_t gg = grp;
            for (int d0 = 0; d0 < g.P1 && ok; d0 += G, ++gg) {
                const int Gg = g.P1 - d0 < G ? g.P1 - d0 : G;
                // one thread takes the bounded wait; the named barrier below
                // is then reached by every drain warp in bounded time
                if (t == 0) {
                    s_go = mbar_wait(bar(CB_AFULL), gg & 1, &s_abort) ? 1 : 0;
                }
                asm volatile("bar.sync 1, %0;" ::"r"(kColDrain) : "memory");
                ok = s_go != 0;
                if (!ok) break;
                mbar_wait(bar(CB_AFULL), gg & 1, &s_abort);  // completed already: acquire for this thread
                tc_fence_after();
                // accumulators this group left unused are released at once
                for (int gi = Gg; gi < G; ++gi)
                    if (lane == 0) mbar_arrive(bar(CB_AEMPTY + gi));
                // rounds of NB accumulators: every accumulator of a round is
                // read from TMEM and stored to its band buffer back to back,
                // each released to the issuer as soon as every warp has read
                // it; the diagonal sums run while the next group's MMAs do
                for (int r0 = 0; r0 < Gg; r0 += g.NB) {
                    const int nb = Gg - r0 < g.NB ? Gg - r0 : g.NB;
                    for (int gl = 0; gl < nb; ++gl) {
                        const int gi = r0 + gl;
                        float* bk = reinterpret_cast<float*>(smem + g.bk_off + gl * g.bk_bytes);
                        // this warp's chunks, kColDB at a time: one batch of
                        // loads and one wait per batch
                        for (int cb = clo; cb <= chi; cb += kColDB) {
                            uint32_t r[kColDB * 16];
#pragma unroll
                            for (int k2 = 0; k2 < kColDB; ++k2) {
                                if (cb + k2 <= chi) {
                                    asm volatile(
                                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"
                                        "%11,%12,%13,%14,%15}, [%16];"
                                        : "=r"(r[k2 * 16 + 0]), "=r"(r[k2 * 16 + 1]), "=r"(r[k2 * 16 + 2]),
                                          "=r"(r[k2 * 16 + 3]), "=r"(r[k2 * 16 + 4]), "=r"(r[k2 * 16 + 5]),
                                          "=r"(r[k2 * 16 + 6]), "=r"(r[k2 * 16 + 7]), "=r"(r[k2 * 16 + 8]),
                                          "=r"(r[k2 * 16 + 9]), "=r"(r[k2 * 16 + 10]), "=r"(r[k2 * 16 + 11]),
                                          "=r"(r[k2 * 16 + 12]), "=r"(r[k2 * 16 + 13]), "=r"(r[k2 * 16 + 14]),
                                          "=r"(r[k2 * 16 + 15])
                                        : "r"(lbase + (uint32_t)(gi * g.Npad + (cb + k2) * 16)));
                                }
                            }
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                            if (cb + kColDB > chi) {  // this warp's part of accumulator gi read: release it
                                tc_fence_before();
                                __syncwarp();
                                if (lane == 0) mbar_arrive(bar(CB_AEMPTY + gi));
                            }
                            // band entries to bk[y - col][col]; the others to
                            // this lane's dummy slot (branch-free stores)
#pragma unroll
                            for (int k2 = 0; k2 < kColDB; ++k2) {
                                if (cb + k2 <= chi) {
                                    const int col0 = (cb + k2) * 16;
#pragma unroll
                                    for (int j = 0; j < 16; ++j) {
                                        const int col = col0 + j, d = y - col;
                                        const bool in = (unsigned)d < (unsigned)g.P1 && col < m;
                                        bk[in ? d * Sb + col : dummy] = __uint_as_float(r[k2 * 16 + j]);
                                    }
                                }
                            }
                        }
                        if (clo > chi) {  // a warp without band entries still releases it
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(bar(CB_AEMPTY + gi));
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(kColDrain) : "memory");
                    if (part < nparts) {  // row dy of each band buffer, eight independent chains
                        for (int gl = 0; gl < nb; ++gl) {
                            const float* row =
                                reinterpret_cast<const float*>(smem + g.bk_off + gl * g.bk_bytes) + dy * Sb;
                            float sa[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) sa[e] = 0.f;
                            int c = c0;
                            for (; c + 8 <= c1; c += 8) {
                                float v[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[e] = row[c + e];
#pragma unroll
                                for (int e = 0; e < 8; ++e) sa[e] += v[e];
                            }
#pragma unroll
                            for (int e = 0; e < 7; ++e)
                                if (c + e < c1) sa[e] += row[c + e];
                            pbuf[gl * kColDrain + part * g.P1 + dy] =
                                ((sa[0] + sa[1]) + (sa[2] + sa[3])) + ((sa[4] + sa[5]) + (sa[6] + sa[7]));
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(kColDrain) : "memory");
                    for (int idx = t; idx < nb * g.P1; idx += kColDrain) {  // offsets d0 + r0 .. d0 + r0 + nb - 1
                        const int gl = idx / g.P1, dyy = idx - gl * g.P1;
                        const float* pb = pbuf + gl * kColDrain;
                        float sum = 0.f;
                        for (int p = 0; p < nparts; ++p) sum += pb[p * g.P1 + dyy];
                        out[dyy * g.P1 + d0 + r0 + gl] = sum;
                    }
                }
            }
        }
        for (int d0 = 0; d0 < g.P1; d0 += G) {
            const int Gg = g.P1 - d0 < G ? g.P1 - d0 : G;
            wsc += (uint32_t)((m + Gg - 1 + kColQ - 1) / kColQ);
            tsc += (uint32_t)nstage;
            ++grp;
        }
        if (!ok) atomicExch(&s_abort, 1);
    }

    if (*reinterpret_cast<volatile int*>(&s_abort)) {
        if (warp == 0 && lane == 0) {  // let every copy in flight land (all complete on template barriers)
            for (uint32_t i = 0; i < (uint32_t)CL.TS && i < t_issued; ++i) {
                const uint32_t ti = t_issued - 1 - i;
                mbar_wait_short(bar(CB_TFULL + ti % CL.TS), (ti / CL.TS) & 1);
            }
        }
        if ((warp == 1 || warp == 3) && lane == 0) {  // and every MMA issued
            mma_commit(bar(CB_FIN));
            mbar_wait_short(bar(CB_FIN), 0);
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

int pick_U(int m, int R) {
    TcGeom g = tc_geom(m, R, 8);
    if (g.NA >= 3) return 8;
    return 4;
}

}  // namespace

namespace tcx {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 4-D bf16 view {8 channels, d1, d2, 2 chunks} of a chunked cube layout.
bool make_map(CUtensorMap* map, const void* base, uint64_t d1, uint64_t d2, uint32_t b1, uint32_t b2, uint32_t b3) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {8, d1, d2, 2};
    cuuint64_t strides[3] = {16, 16 * d1, 16 * d1 * d2};
    cuuint32_t box[4] = {8, b1, b2, b3};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 4-D bf16 view of a chunked cube [2][d2][d1][8] (d1 = H, d2 = W for the
// column-major layout cm; d1 = W, d2 = H for the row-major layout rm) whose
// innermost dimension is 8 pixels x 8 channels (128 contiguous bytes) and
// whose second dimension is the pixel index along d1 (16-byte stride)
// traversed with stride 8: a box {64, b1, b2, 2} loads, per line of d2 and
// chunk, b1 consecutive pixels from any start as b1/8 runs of 128 bytes.
// The last run of a line may read up to 7 pixels past it (the cube buffers
// are padded for the last line).
bool make_map_rows8(CUtensorMap* map, const void* base, uint64_t d1, uint64_t d2, uint32_t b1, uint32_t b2) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {64, d1, d2, 2};
    cuuint64_t strides[3] = {16, 16 * d1, 16 * d1 * d2};
    cuuint32_t box[4] = {64, b1, b2, 2};
    cuuint32_t es[4] = {1, 8, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace tcx

size_t corr_tc_smem_bytes(int m, int R) { return (size_t)tc_geom(m, R, pick_U(m, R)).smem; }

namespace {

bool col_ok(int m, int R) { return m + 2 * R <= kM && 2 * R + 1 <= kM && col_geom(m, R).smem <= kColSmemMax; }

bool toeplitz_ok(int m, int R) {
    if (2 * R + 1 > kM || m > kMaxTemplate) return false;
    const TcGeom g = tc_geom(m, R, pick_U(m, R));
    return g.NA >= 2 && g.JS <= 512 && g.AW <= 256;
}

// launch layout of a column-form class: slots as large as its largest item
bool col_launch(int G, const int* ms, const int* Rs, int cnt, ColLaunch* out) {
    int tsb = 0, wsb = 0, need = 0;
    for (int i = 0; i < cnt; ++i) {
        const ColGeom g = col_geom(ms[i], Rs[i]);
        if (g.G != G) return false;
        tsb = g.ts_bytes > tsb ? g.ts_bytes : tsb;
        wsb = g.ws_bytes > wsb ? g.ws_bytes : wsb;
    }
    ColLaunch L;
    L.TS = kColMaxTS;
    L.WS = (kColQ + G - 2) / kColQ + 2;
    L.ts_stride = tsb;
    L.ws_stride = wsb;
    L.w_off = L.TS * tsb;
    L.bk_off = L.w_off + L.WS * wsb;
    L.smem = kColSmemMax;
    // every item needs one band buffer and its partial sums, and the read
    // guard past the last window slab
    for (int i = 0; i < cnt; ++i) {
        const ColGeom g = col_geom(ms[i], Rs[i]);
        const int n1 = L.bk_off + g.bk_bytes + kColDrain * 4 + (2048 - 16 * g.wrows);
        need = n1 > need ? n1 : need;
    }
    *out = L;
    return need <= L.smem && L.WS <= kColMaxWS;
}

}  // namespace

int corr_tc_class(int form, int m, int R) {
    switch (form) {
        case 1: return toeplitz_ok(m, R) ? 1 : 0;  // per pair (its geometry decides the instance)
        case 2: return col_ok(m, R) ? col_geom(m, R).G : 0;
        case 3: return corr_band_class(m, R);
        default: return 0;
    }
}

int corr_tc_auto_form(int m, int R) {
    // every form's MMAs cost about the same (M = 128, K = 16 and N <= 96 are
    // bound by shared-memory operand reads), so the form that issues fewer
    // per point wins: the column form (2R+1) m, the band form
    // ceil((m+2R)/16) ceil((2R+1)/8) m; the Toeplitz form ((m+2R) m narrow
    // ones) only when neither of the others runs
    const bool c = col_ok(m, R), b = corr_band_supported(m, R);
    if (b && (!c || corr_band_mmas(m, R) < (long long)(2 * R + 1) * m)) return 3;
    if (c) return 2;
    return toeplitz_ok(m, R) ? 1 : 0;
}

bool corr_tc_maps(int form, MatchJob& j) {
    if (form == 3) return corr_band_maps(j);
    if (form == 2) {
        // slabs of 8 columns x 2 chunks, rows in 128-byte runs of 8 pixels
        const ColGeom c = col_geom(j.m, j.R);
        return make_map_rows8(&j.tm[0], j.rcm, (uint64_t)j.Hr, (uint64_t)j.Wr, (uint32_t)c.wrows, kColQ) &&
               make_map_rows8(&j.tm[1], j.scm, (uint64_t)j.Hs, (uint64_t)j.Ws, (uint32_t)c.trows, kColQ);
    }
    if (form == 1) {
        // A: window slab, box {8, AW, 8 rows, 2 chunks} over rm = [2][H][W][8]
        // B: one template column, box {8, rows, 1, 1} over cm = [2][W][H][8];
        //    rows [0, 256) through tm[1] and [256, JS) through tm[2] when JS > 256
        const TcGeom g = tc_geom(j.m, j.R, pick_U(j.m, j.R));
        const uint32_t brow = g.JS < 256 ? (uint32_t)g.JS : 256u;
        const uint32_t brow2 = g.JS > 256 ? (uint32_t)(g.JS - 256) : 8u;
        return make_map(&j.tm[0], j.rrm, (uint64_t)j.Wr, (uint64_t)j.Hr, (uint32_t)g.AW, kY, 2) &&
               make_map(&j.tm[1], j.scm, (uint64_t)j.Hs, (uint64_t)j.Ws, brow, 1, 1) &&
               make_map(&j.tm[2], j.scm, (uint64_t)j.Hs, (uint64_t)j.Ws, brow2, 1, 1);
    }
    return false;
}

// One launch of a tensor-core form over `is` (items == nullptr: the points
// of `one`; the Toeplitz form only runs that way).  Every job of the launch
// has class `cls` of the form and its tensor maps set (corr_tc_maps); ms /
// Rs list the distinct (m, R) of its jobs.
cudaError_t launch_corr_tc(int form, int cls, const MatchJob& one, const ItemSet& is, const int* ms, const int* Rs,
                           int cnt, int* err_flag, cudaStream_t st) {
    const int n = is.items ? is.n : one.n;
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n < sms ? n : sms;
    if (form == 3) return launch_corr_band(one, is, cls, ms, Rs, cnt, err_flag, sms, st);
    if (form == 2) {
        ColLaunch CL;
        if (!col_launch(cls, ms, Rs, cnt, &CL)) return cudaErrorNotSupported;
        cudaError_t e = cudaErrorNotSupported;
#define SFOC_COL_CASE(GV)                                                                                       \
    case GV:                                                                                                    \
        e = cudaFuncSetAttribute(k_corr_tc_col<GV>, cudaFuncAttributeMaxDynamicSharedMemorySize, CL.smem);      \
        if (e != cudaSuccess) return e;                                                                         \
        k_corr_tc_col<GV><<<grid, kColThreads, CL.smem, st>>>(one, is.jobs, is.items, n, CL, err_flag);          \
        return cudaGetLastError();
        switch (cls) {
            SFOC_COL_CASE(1)
            SFOC_COL_CASE(2)
            SFOC_COL_CASE(3)
            SFOC_COL_CASE(4)
            SFOC_COL_CASE(5)
            SFOC_COL_CASE(6)
            SFOC_COL_CASE(7)
            SFOC_COL_CASE(8)
            SFOC_COL_CASE(9)
            SFOC_COL_CASE(10)
            SFOC_COL_CASE(11)
            SFOC_COL_CASE(12)
            SFOC_COL_CASE(13)
            SFOC_COL_CASE(14)
            SFOC_COL_CASE(15)
            SFOC_COL_CASE(16)
            default: break;
        }
#undef SFOC_COL_CASE
        return e;
    }
    if (form != 1 || is.items || !toeplitz_ok(one.m, one.R)) return cudaErrorNotSupported;
    const int m = one.m, R = one.R;
    const int U = pick_U(m, R);
    const TcGeom g = tc_geom(m, R, U);
    const int nq = g.Npad / 16;
    const size_t smem = (size_t)g.smem;
    cudaError_t e;
#define SFOC_TC_CASE(NQ, UC)                                                                               \
    e = cudaFuncSetAttribute(k_corr_tc<NQ, UC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
    if (e != cudaSuccess) return e;                                                                        \
    k_corr_tc<NQ, UC><<<grid, kThreads, smem, st>>>(one, err_flag);
#define SFOC_TC_NQ(UC)                  \
    switch (nq) {                       \
        case 1: SFOC_TC_CASE(1, UC) break; \
        case 2: SFOC_TC_CASE(2, UC) break; \
        case 3: SFOC_TC_CASE(3, UC) break; \
        case 4: SFOC_TC_CASE(4, UC) break; \
        case 5: SFOC_TC_CASE(5, UC) break; \
        case 6: SFOC_TC_CASE(6, UC) break; \
        case 7: SFOC_TC_CASE(7, UC) break; \
        default: SFOC_TC_CASE(8, UC) break; \
    }
    if (U == 8) {
        SFOC_TC_NQ(8)
    } else {
        SFOC_TC_NQ(4)
    }
#undef SFOC_TC_NQ
#undef SFOC_TC_CASE
    return cudaGetLastError();
}

}  // namespace sfoc
