// NCC assembly, peak picking and sub-pixel refinement (Eq. 9, 12, 16 of
// arXiv 2202.13347; Sec. 3.2.2 takes the most similar position as the CP).
//
// k_template_stats  per point (one CTA): bounds check, then R_T and R_TT
//                   (Eq. 12) as sums of the sensed cube's channel-summed
//                   planes over the template, each pixel rounded to 2^-28
//                   units exactly as the integral images round it and added
//                   in 64-bit integers: the same exact values a lookup in
//                   integral images of the sensed cube would give, without
//                   building them.
// k_ncc_argmax      per point (one CTA): for every offset, R_S and R_SS from
//                   the reference integral images (4 lookups each, exact
//                   64-bit fixed point); the two steps that cancel are taken
//                   in exact 128-bit integers: mnz R_SS - R_S^2 (the
//                   variance times mnz) and, for the uncentred correlation
//                   forms, R_S R_T (the mean correction of the numerator);
//                   each is rounded to FP32 once, then NCC = num / sqrt(vS vT)
//                   in FP32; a warp-shuffle argmax with the (NCC desc, dy
//                   asc, dx asc) order and a 3-point parabola per axis.  No
//                   FP64 per offset: GB300 runs it at a small fraction of its
//                   FP32 rate, and 64 x 64-bit integer products cost a few
//                   integer multiply-adds.
#include <math.h>
#include <string.h>

#include "internal.h"

namespace sfoc {

namespace {

typedef unsigned long long u64;

// a non-negative 128-bit integer to FP32 (two roundings: relative error
// below 2^-23)
__device__ __forceinline__ float u128_to_float(unsigned __int128 v) {
    const u64 hi = (u64)(v >> 64), lo = (u64)v;
    return fmaf(__ull2float_rn(hi), 18446744073709551616.f, __ull2float_rn(lo));
}

// window sum (Eq. 16) in 2^-28 units; exact (the planes wrap modulo 2^64)
__device__ __forceinline__ long long rect(const u64* P, size_t ip, int y0, int x0, int y1, int x1) {
    return (long long)(P[(size_t)y1 * ip + x1] - P[(size_t)y0 * ip + x1] - P[(size_t)y1 * ip + x0] +
                       P[(size_t)y0 * ip + x0]);
}

constexpr int kStatThreads = 128;

__global__ void __launch_bounds__(kStatThreads)
    k_template_stats(const __grid_constant__ MatchJob one, const MatchJob* __restrict__ jobs,
                     const int2* __restrict__ items) {
    __shared__ u64 s_acc[kStatThreads / 32][2];
    int k;
    const MatchJob& J = item_job(one, jobs, items, blockIdx.x, &k);
    const float* __restrict__ s1 = J.ss1;
    const float* __restrict__ s2 = J.ss2;
    const size_t pitch = J.spitch;
    const int Hs = J.Hs, Ws = J.Ws, Hr = J.Hr, Wr = J.Wr, m = J.m, R = J.R, z = J.z;
    const int32_t* __restrict__ pts = J.pts;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = template_half(m);
    const int px = pts[2 * k], py = pts[2 * k + 1];
    const int ty0 = py - h, tx0 = px - h;
    const bool ok = ty0 >= 0 && tx0 >= 0 && ty0 + m <= Hs && tx0 + m <= Ws && ty0 - R >= 0 && tx0 - R >= 0 &&
                    ty0 + m + R <= Hr && tx0 + m + R <= Wr;
    u64 a1 = 0, a2 = 0;  // modulo 2^64, like the integral images
    if (ok) {
        // (row, column) pairs of the template taken 4 at a time per thread, so
        // that several loads are in flight before the first sum needs one
        const int ncol = (m + 31) >> 5;          // column blocks of 32 per row
        const int ntask = m * ncol;               // (row, column block) tasks
        for (int t0 = warp; t0 < ntask; t0 += 4 * (kStatThreads / 32)) {
            float v1[4], v2[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u * (kStatThreads / 32);
                const int r = t / ncol, c = (t - r * ncol) * 32 + lane;
                const bool in = t < ntask && c < m;
                const size_t at = (size_t)(ty0 + (in ? r : 0)) * pitch + tx0 + (in ? c : 0);
                v1[u] = in ? s1[at] : 0.f;
                v2[u] = in ? s2[at] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u * (kStatThreads / 32);
                const int r = t / ncol, c = (t - r * ncol) * 32 + lane;
                if (t < ntask && c < m) {
                    a1 += int_quant(v1[u]);
                    a2 += int_quant(v2[u]);
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
        a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
        s_acc[warp][0] = a1;
        s_acc[warp][1] = a2;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    PointStat s;
    s.RT = s.RTT = 0.0;
    s.tmean = 0.f;
    if (!ok) {
        s.status = SFOC_PT_OUT_OF_BOUNDS;
    } else {
        u64 t1 = 0, t2 = 0;
        for (int w = 0; w < kStatThreads / 32; ++w) {
            t1 += s_acc[w][0];
            t2 += s_acc[w][1];
        }
        const long long rt = (long long)t1, rtt = (long long)t2;
        const double N = (double)m * m * z;
        if (rt >= kIntNonFiniteMin || rtt >= kIntNonFiniteMin) {
            s.RT = s.RTT = NAN;
            s.status = SFOC_PT_NAN;
        } else {
            s.RT = int_units_to_double(rt);
            s.RTT = int_units_to_double(rtt);
            s.tmean = (float)(s.RT / N);
            const double vT = s.RTT - s.RT * s.RT / N;
            s.status = vT <= 1e-6 * N ? SFOC_PT_FLAT_TEMPLATE : SFOC_PT_OK;
        }
    }
    J.stats[k] = s;
}

// argmax key: larger value wins, ties go to the smaller index
__device__ __forceinline__ bool better(float v, int i, float bv, int bi) {
    return v > bv || (v == bv && i < bi);
}

constexpr int kNccThreads = 256;

__global__ void __launch_bounds__(kNccThreads) k_ncc_argmax(const __grid_constant__ MatchJob one,
                                                            const MatchJob* __restrict__ jobs,
                                                            const int2* __restrict__ items) {
    extern __shared__ float s_map[];  // P1 * P1
    __shared__ float s_bv[kNccThreads / 32];
    __shared__ int s_bi[kNccThreads / 32];
    __shared__ int s_nan;
    int k;
    const MatchJob& J = item_job(one, jobs, items, blockIdx.x, &k);
    const u64* __restrict__ Pr = J.rint;
    const int Hr = J.Hr, m = J.m, R = J.R, z = J.z, centered = J.centered;
    const size_t ipr = J.ripitch;
    const int32_t* __restrict__ pts = J.pts;
    const float* __restrict__ num = J.maps;
    float* __restrict__ out_maps = J.out_maps;
    fastncc_result* __restrict__ out = J.out;
    const int P1 = 2 * R + 1, P = P1 * P1;
    const PointStat st = J.stats[k];
    if (threadIdx.x == 0) s_nan = 0;
    fastncc_result res;
    res.dx = res.dy = 0;
    res.ncc = 0.f;
    res.sub_dx = res.sub_dy = 0.f;
    res.status = st.status;
    if (st.status != SFOC_PT_OK) {
        if (out_maps)
            for (int i = threadIdx.x; i < P; i += blockDim.x) out_maps[(size_t)k * P + i] = 0.f;
        if (threadIdx.x == 0) out[k] = res;
        return;
    }
    __syncthreads();
    const long long Ni = (long long)m * m * z;
    const double N = (double)Ni;
    const float flat = (float)(1e-6 * N);
    const float vTf = (float)(st.RTT - st.RT * st.RT / N);
    // 2^-56 / mnz: a product of two window sums in 2^-28 units, divided by mnz
    const float sc = (float)(1.0 / (72057594037927936.0 * N));
    const long long rt = (long long)(st.RT * 268435456.0);  // R_T in 2^-28 units (exact)
    const int h = template_half(m);
    const int ty0 = pts[2 * k + 1] - h, tx0 = pts[2 * k] - h;
    const u64* P1p = Pr;
    const u64* P2p = Pr + (size_t)(Hr + 1) * ipr;
    const float* nk = num + (size_t)k * P;
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    int has_nan = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int iy = i / P1, ix = i - iy * P1;
        const int wy = ty0 + iy - R, wx = tx0 + ix - R;
        const long long rs = rect(P1p, ipr, wy, wx, wy + m, wx + m);
        const long long rss = rect(P2p, ipr, wy, wx, wy + m, wx + m);
        const float n32 = nk[i];
        float v;
        if (rs >= kIntNonFiniteMin || rss >= kIntNonFiniteMin || n32 != n32) {
            v = NAN;
        } else {
            // mnz R_SS - R_S^2, exact (units 2^-56); negative only through the
            // per-pixel rounding of a flat window
            const __int128 d = ((__int128)(Ni * rss) << 28) - (__int128)rs * rs;
            const float vS = d > 0 ? u128_to_float((unsigned __int128)d) * sc : 0.f;
            float nm = n32;
            if (!centered) {
                const __int128 p = (__int128)rs * rt;  // R_S R_T, exact
                const float pf = p >= 0 ? u128_to_float((unsigned __int128)p) : -u128_to_float((unsigned __int128)(-p));
                nm = fmaf(-pf, sc, n32);
            }
            v = vS <= flat ? 0.f : nm / sqrtf(vS * vTf);
        }
        s_map[i] = v;
        if (out_maps) out_maps[(size_t)k * P + i] = v;
        if (v != v) { has_nan = 1; continue; }
        if (better(v, i, bv, bi)) { bv = v; bi = i; }
    }
    // warp argmax
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_down_sync(full, bv, o);
        int oi = __shfl_down_sync(full, bi, o);
        if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    has_nan = __any_sync(full, has_nan);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_bv[wid] = bv;
        s_bi[wid] = bi;
        if (has_nan) atomicOr(&s_nan, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bv = s_bv[0];
        bi = s_bi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (better(s_bv[w], s_bi[w], bv, bi)) { bv = s_bv[w]; bi = s_bi[w]; }
        if (bi == 0x7fffffff) {  // every score NaN
            res.status = SFOC_PT_NAN;
        } else {
            int iy = bi / P1, ix = bi - iy * P1;
            res.dy = iy - R;
            res.dx = ix - R;
            res.ncc = (float)bv;
            bool edge = false;
            double ddx = 0.0, ddy = 0.0;
            auto parab = [](double cm, double c0, double cp) {  // from the FP32 map values
                double den = cm - 2.0 * c0 + cp;
                if (!(den < 0.0)) return 0.0;
                double d = (cm - cp) / (2.0 * den);
                return d > 0.5 ? 0.5 : (d < -0.5 ? -0.5 : d);
            };
            if (ix > 0 && ix < P1 - 1) ddx = parab(s_map[bi - 1], bv, s_map[bi + 1]);
            else edge = true;
            if (iy > 0 && iy < P1 - 1) ddy = parab(s_map[bi - P1], bv, s_map[bi + P1]);
            else edge = true;
            if (ddx != ddx) ddx = 0.0;
            if (ddy != ddy) ddy = 0.0;
            res.sub_dx = (float)(res.dx + ddx);
            res.sub_dy = (float)(res.dy + ddy);
            res.status = s_nan ? SFOC_PT_NAN : (edge ? SFOC_PT_PEAK_ON_EDGE : SFOC_PT_OK);
        }
        out[k] = res;
    }
}

}  // namespace

cudaError_t launch_template_stats(const MatchJob& one, const ItemSet& is, cudaStream_t st) {
    const int n = is.items ? is.n : one.n;
    if (n <= 0) return cudaSuccess;
    k_template_stats<<<n, kStatThreads, 0, st>>>(one, is.jobs, is.items);
    return cudaGetLastError();
}

cudaError_t launch_ncc_argmax(const MatchJob& one, const ItemSet& is, cudaStream_t st) {
    const int n = is.items ? is.n : one.n;
    if (n <= 0) return cudaSuccess;
    const int R = is.items ? is.max_R : one.R;
    const int P1 = 2 * R + 1;
    size_t smem = sizeof(float) * (size_t)P1 * P1;
    cudaError_t e = cudaFuncSetAttribute(k_ncc_argmax, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_ncc_argmax<<<n, kNccThreads, smem, st>>>(one, is.jobs, is.items);
    return cudaGetLastError();
}

MatchJob make_job(const Cube& ref, const Cube& sen, const int32_t* pts, int n, int m, int R, PointStat* stats,
                  float* maps, float* out_maps, fastncc_result* out) {
    MatchJob j;
    memset(&j, 0, sizeof(j));
    j.rf32 = ref.f32;
    j.rrm = ref.rm;
    j.rcm = ref.cm;
    j.rint = ref.integ;
    j.rpitch = ref.pitch;
    j.rplane = ref.pitch * (size_t)ref.H;
    j.ripitch = ref.ipitch;
    j.Hr = ref.H;
    j.Wr = ref.W;
    j.sf32 = sen.f32;
    j.ss1 = sen.s1;
    j.ss2 = sen.s2;
    j.srm = sen.rm;
    j.scm = sen.cm;
    j.spitch = sen.pitch;
    j.splane = sen.pitch * (size_t)sen.H;
    j.Hs = sen.H;
    j.Ws = sen.W;
    j.z = ref.z;
    j.m = m;
    j.R = R;
    j.n = n;
    j.pts = pts;
    j.stats = stats;
    j.maps = maps;
    j.out_maps = out_maps;
    j.out = out;
    return j;
}

}  // namespace sfoc
