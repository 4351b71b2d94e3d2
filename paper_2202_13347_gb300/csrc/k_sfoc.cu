// SFOC descriptor kernels (Sec. 2.1 of arXiv 2202.13347).
//
// k_sfoc_steer   separable Gaussian-derivative bases (Eq. 2, 3, 5), steering
//                (Eq. 6, 7), |.| and the sum over scales -> F planes.
// k_sfoc_smooth  three parallel dilated Gaussian smoothings per channel,
//                summed, group-wise L2 normalisation and stacking, plus the
//                per-pixel sum planes used by the integral images (Eq. 14).
//
// Both kernels stage a 2-D tile with its clamped halo in shared memory and
// do the horizontal pass into shared planes, then the vertical pass per
// output pixel.  Borders clamp to the edge in every convolution.
#include <cuda_bf16.h>
#include <string.h>

#include <type_traits>

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kTW = 32;          // output tile width (one warp across)
constexpr int kTH = 32;          // output tile height
constexpr int kThreads = 256;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Row stride (floats) of the smoothing input tile: room for the tile, its
// halo and the 8-wide load blocks' overrun, a multiple of 4 floats (float4
// rows) with an odd number of float4s, so that the two rows a quarter-warp
// reads in the horizontal pass fall in different banks.
__host__ __device__ inline int smooth_row_stride(int maxhal) {
    int fw = (32 + 2 * maxhal + 8 + 3) / 4 * 4;
    if ((fw / 4) % 2 == 0) fw += 4;
    return fw;
}

// even taps: t0 x[0] + sum_q t[q] (x[-q] + x[+q]); `x` points at the centre, stride s
__device__ __forceinline__ float conv_even(const float* x, int s, const float* t, int K) {
    float acc = t[0] * x[0];
#pragma unroll
    for (int q = 1; q <= kMaxDerivRadius; ++q)
        if (q <= K) acc = fmaf(t[q], x[-q * s] + x[q * s], acc);
    return acc;
}

// odd taps under convolution: sum_q t[q] x[c - q] = sum_{q>0} t[q] (x[-q] - x[+q])
__device__ __forceinline__ float conv_odd(const float* x, int s, const float* t, int K) {
    float acc = 0.f;
#pragma unroll
    for (int q = 1; q <= kMaxDerivRadius; ++q)
        if (q <= K) acc = fmaf(t[q], x[-q * s] - x[q * s], acc);
    return acc;
}

// image samples to intensities: float as is; uint16 scaled to [0, 1] by
// v / 65535 (correctly rounded division)
__device__ __forceinline__ float to_unit(float v) { return v; }
__device__ __forceinline__ float to_unit(uint16_t v) { return (float)v / 65535.f; }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_sfoc_steer(const T* __restrict__ img, int H, int W, size_t pitch,
                                                          float* __restrict__ F, size_t fpitch, size_t fplane,
                                                          SteerTaps tp) {
    extern __shared__ float sm[];
    const int hal = tp.halo;
    const int IW = kTW + 2 * hal, IH = kTH + 2 * hal;
    float* s_img = sm;
    float* s_h = s_img + IH * IW;
    const int plane = IH * kTW;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;

    for (int i = threadIdx.x; i < IH * IW; i += kThreads) {
        int r = i / IW, c = i - r * IW;
        int gy = clampi(y0 + r - hal, 0, H - 1), gx = clampi(x0 + c - hal, 0, W - 1);
        s_img[i] = to_unit(__ldg(img + (size_t)gy * pitch + gx));
    }
    __syncthreads();

    // horizontal passes.  planes: 2s = a1_s (odd), 2s+1 = g1_s (even);
    // second group: 2ns = a2 (even), 2ns+1 = g2 (even), 2ns+2 = c2x (odd)
    const int ns = tp.ns;
    for (int i = threadIdx.x; i < IH * kTW; i += kThreads) {
        int r = i / kTW, c = i - r * kTW;
        const float* x = s_img + r * IW + c + hal;
        for (int s = 0; s < ns; ++s) {
            s_h[(2 * s) * plane + i] = conv_odd(x, 1, tp.a1[s], tp.K1[s]);
            s_h[(2 * s + 1) * plane + i] = conv_even(x, 1, tp.g1[s], tp.K1[s]);
        }
        if (tp.second) {
            s_h[(2 * ns) * plane + i] = conv_even(x, 1, tp.a2, tp.K2);
            s_h[(2 * ns + 1) * plane + i] = conv_even(x, 1, tp.g2, tp.K2);
            s_h[(2 * ns + 2) * plane + i] = conv_odd(x, 1, tp.c2x, tp.K2);
        }
    }
    __syncthreads();

    for (int i = threadIdx.x; i < kTH * kTW; i += kThreads) {
        int r = i / kTW, c = i - r * kTW;
        int gy = y0 + r, gx = x0 + c;
        if (gy >= H || gx >= W) continue;
        const int off = (r + hal) * kTW + c;
        float Ix[kMaxScales], Iy[kMaxScales];
        for (int s = 0; s < ns; ++s) {
            Ix[s] = conv_even(s_h + (2 * s) * plane + off, kTW, tp.g1[s], tp.K1[s]);      // a1(x) g(y)
            Iy[s] = conv_odd(s_h + (2 * s + 1) * plane + off, kTW, tp.a1[s], tp.K1[s]);   // g(x) a1(y)
        }
        float* out = F + (size_t)gy * fpitch + gx;
        for (int k = 0; k < tp.no; ++k) {
            float f = 0.f;
            for (int s = 0; s < ns; ++s) {
                float v = fmaf(tp.ct[k], Ix[s], tp.st[k] * Iy[s]);
                f += tp.rectify ? fabsf(v) : v;
            }
            out[(size_t)k * fplane] = f;
        }
        if (tp.second) {
            float Ixx = conv_even(s_h + (2 * ns) * plane + off, kTW, tp.g2, tp.K2);      // a2(x) g2(y)
            float Iyy = conv_even(s_h + (2 * ns + 1) * plane + off, kTW, tp.a2, tp.K2);  // g2(x) a2(y)
            float Ixy = conv_odd(s_h + (2 * ns + 2) * plane + off, kTW, tp.c2y, tp.K2);  // c(x) c(y)
            for (int k = 0; k < tp.no; ++k) {
                float c2 = tp.ct[k] * tp.ct[k], s2 = tp.st[k] * tp.st[k], cs = 2.f * tp.st[k] * tp.ct[k];
                float v = fmaf(c2, Ixx, fmaf(s2, Iyy, -cs * Ixy));
                out[(size_t)(tp.no + k) * fplane] = tp.rectify ? fabsf(v) : v;
            }
        }
    }
}

// Steering with the radii at compile time (three first-order scales of
// radii KA, KB, KC and the second-order radius KS; the paper's scales give
// 2, 3, 3 and 5).  Same arithmetic per output as k_sfoc_steer, register
// blocked: a thread of the horizontal pass loads one row span once (float4)
// and produces all nine basis planes for 8 columns; a thread of the
// vertical pass loads each plane's column span once and produces 4 rows.
template <int K>
__device__ __forceinline__ float ceven(const float* x, const float* t) {
    float acc = t[0] * x[0];
#pragma unroll
    for (int q = 1; q <= K; ++q) acc = fmaf(t[q], x[-q] + x[q], acc);
    return acc;
}
template <int K>
__device__ __forceinline__ float codd(const float* x, const float* t) {
    float acc = 0.f;
#pragma unroll
    for (int q = 1; q <= K; ++q) acc = fmaf(t[q], x[-q] - x[q], acc);
    return acc;
}

// Three CTAs per SM: the 80-register cap (a few spilled values) hides the
// tile loads better than two CTAs at 127 registers did (0.207 -> 0.179 ms
// per step for the two 2048 x 2048 images).
// One image (`one`, CTA = tile in row-major tile order) or a batch (device
// table `jobs`, CTAs of image j from begin[j]).
template <typename T, int KA, int KB, int KC, int KS>
__global__ void __launch_bounds__(kThreads, 3) k_sfoc_steer_ct(const __grid_constant__ ImgJob one,
                                                             const ImgJob* __restrict__ jobs,
                                                             const int* __restrict__ begin, int n_jobs,
                                                             SteerTaps tp) {
    constexpr int HAL = KS > KA ? (KS > KB ? (KS > KC ? KS : KC) : (KB > KC ? KB : KC))
                                : (KA > KB ? (KA > KC ? KA : KC) : (KB > KC ? KB : KC));
    constexpr int IH = kTH + 2 * HAL, IW = kTW + 2 * HAL;
    constexpr int NV = (8 + 2 * HAL + 3) / 4;            // float4 per horizontal span
    constexpr int IWP = ((24 + 4 * NV + 3) / 4 % 2) ? (24 + 4 * NV + 3) / 4 * 4 : (24 + 4 * NV + 3) / 4 * 4 + 4;
    constexpr int NP = 9;                                 // basis planes
    __shared__ __align__(16) float s_img[IH * IWP];
    extern __shared__ float4 sm4[];
    float* s_h = reinterpret_cast<float*>(sm4);          // NP x IH x kTW
    __shared__ float s_t[NP][kMaxDerivRadius + 1];        // taps of the nine 1-D factors
    int tile;
    const ImgJob& J = img_job(one, jobs, begin, n_jobs, &tile);
    const T* __restrict__ img = static_cast<const T*>(J.img);
    const int H = J.H, W = J.W;
    const size_t pitch = J.pitch, fpitch = J.fpitch, fplane = J.fpitch * (size_t)J.H;
    float* __restrict__ F = J.F;
    const int ntx = (W + kTW - 1) / kTW;
    const int tby = tile / ntx;
    const int x0 = (tile - tby * ntx) * kTW, y0 = tby * kTH;
    if (threadIdx.x < NP * (kMaxDerivRadius + 1)) {
        const int pl = threadIdx.x / (kMaxDerivRadius + 1), q = threadIdx.x % (kMaxDerivRadius + 1);
        const float* src = pl < 6 ? ((pl & 1) ? tp.g1[pl >> 1] : tp.a1[pl >> 1])
                                  : (pl == 6 ? tp.a2 : (pl == 7 ? tp.g2 : tp.c2x));
        s_t[pl][q] = src[q];
    }
    for (int i = threadIdx.x; i < IH * IW; i += kThreads) {
        const int r = i / IW, c = i - r * IW;
        const int gy = clampi(y0 + r - HAL, 0, H - 1), gx = clampi(x0 + c - HAL, 0, W - 1);
        s_img[r * IWP + c] = to_unit(__ldg(img + (size_t)gy * pitch + gx));
    }
    __syncthreads();
    // horizontal: task = (row, 8-column block); planes 2s = a1_s (odd),
    // 2s+1 = g1_s (even), 6 = a2 (even), 7 = g2 (even), 8 = c2x (odd)
    for (int task = threadIdx.x; task < IH * 4; task += kThreads) {
        const int rr = task >> 2, cb = (task & 3) * 8;
        const float4* x4 = reinterpret_cast<const float4*>(s_img + rr * IWP + cb);
        float in[NV * 4];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float4 f = x4[v];
            in[4 * v] = f.x;
            in[4 * v + 1] = f.y;
            in[4 * v + 2] = f.z;
            in[4 * v + 3] = f.w;
        }
        float o[NP][8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float* x = in + HAL + c;
            o[0][c] = codd<KA>(x, s_t[0]);
            o[1][c] = ceven<KA>(x, s_t[1]);
            o[2][c] = codd<KB>(x, s_t[2]);
            o[3][c] = ceven<KB>(x, s_t[3]);
            o[4][c] = codd<KC>(x, s_t[4]);
            o[5][c] = ceven<KC>(x, s_t[5]);
            o[6][c] = ceven<KS>(x, s_t[6]);
            o[7][c] = ceven<KS>(x, s_t[7]);
            o[8][c] = codd<KS>(x, s_t[8]);
        }
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) {
            float4* dst = reinterpret_cast<float4*>(s_h + (pl * IH + rr) * kTW + cb);
            dst[0] = make_float4(o[pl][0], o[pl][1], o[pl][2], o[pl][3]);
            dst[1] = make_float4(o[pl][4], o[pl][5], o[pl][6], o[pl][7]);
        }
    }
    __syncthreads();
    // vertical: thread = (column, 4-row block)
    const int col = threadIdx.x & 31, rb = (threadIdx.x >> 5) * 4;
    float Ix[3][4], Iy[3][4], Ixx[4], Iyy[4], Ixy[4];
    auto vpass = [&](int pl, auto kr, auto odd, const float* t, float (&out)[4]) {
        constexpr int K = decltype(kr)::value;
        float in[4 + 2 * K];
        const float* x = s_h + (pl * IH + rb + HAL - K) * kTW + col;
#pragma unroll
        for (int i = 0; i < 4 + 2 * K; ++i) in[i] = x[i * kTW];
#pragma unroll
        for (int j = 0; j < 4; ++j) out[j] = decltype(odd)::value ? codd<K>(in + K + j, t) : ceven<K>(in + K + j, t);
    };
    using F0 = std::integral_constant<bool, false>;
    using T1 = std::integral_constant<bool, true>;
    vpass(0, std::integral_constant<int, KA>(), F0(), tp.g1[0], Ix[0]);  // a1(x) g(y)
    vpass(1, std::integral_constant<int, KA>(), T1(), tp.a1[0], Iy[0]);  // g(x) a1(y)
    vpass(2, std::integral_constant<int, KB>(), F0(), tp.g1[1], Ix[1]);
    vpass(3, std::integral_constant<int, KB>(), T1(), tp.a1[1], Iy[1]);
    vpass(4, std::integral_constant<int, KC>(), F0(), tp.g1[2], Ix[2]);
    vpass(5, std::integral_constant<int, KC>(), T1(), tp.a1[2], Iy[2]);
    vpass(6, std::integral_constant<int, KS>(), F0(), tp.g2, Ixx);       // a2(x) g2(y)
    vpass(7, std::integral_constant<int, KS>(), F0(), tp.a2, Iyy);       // g2(x) a2(y)
    vpass(8, std::integral_constant<int, KS>(), T1(), tp.c2y, Ixy);      // c(x) c(y)
    const int gx = x0 + col;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gy = y0 + rb + j;
        if (gy >= H || gx >= W) continue;
        float* out = F + (size_t)gy * fpitch + gx;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float f = 0.f;
#pragma unroll
            for (int sc = 0; sc < 3; ++sc) {
                float v = fmaf(tp.ct[k], Ix[sc][j], tp.st[k] * Iy[sc][j]);
                f += tp.rectify ? fabsf(v) : v;
            }
            out[(size_t)k * fplane] = f;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float c2 = tp.ct[k] * tp.ct[k], s2 = tp.st[k] * tp.st[k], cs = 2.f * tp.st[k] * tp.ct[k];
            float v = fmaf(c2, Ixx[j], fmaf(s2, Iyy[j], -cs * Ixy[j]));
            out[(size_t)(6 + k) * fplane] = tp.rectify ? fabsf(v) : v;
        }
    }
}

// Smoothing (Sec. 2.1): per channel, the F tile with the group's halo
// (clamped) is staged in shared memory; the horizontal pass of each rate
// runs register-blocked (a thread loads one row segment once and produces 8
// outputs for every rate) into shared planes; the vertical pass runs
// register-blocked too (8 rows of one column per thread) and sums the rates
// in registers.  The six channels of a group stay in registers, are
// normalised there and written out: F32 planar, or the bf16 chunks (chunk
// g = the six channels of group g and two zeros) in both pixel orders,
// plus the per-pixel sum planes.  Tiles are 32 columns x 64 rows.
constexpr int kSTW = 32, kSTH = 64, kSRows = 8;
constexpr int kPRows = 4;  // rows per thread of the paired vertical pass (2 columns x 4 rows)

template <int KD>
__device__ __forceinline__ void smooth_channel(const float* __restrict__ Fk, size_t fpitch, int H, int W, int x0,
                                               int y0, int hal, int n_dil, const int* s_dil, const float* t,
                                               float* s_F, int FW, float* s_h, int HR, float (&Dk)[kSRows]) {
    const int IW = kSTW + 2 * hal, IH = kSTH + 2 * hal;
    const int nd = KD > 0 ? n_dil : 1;  // radius 0: the group is unsmoothed, D = F (no sum over rates)
    __syncthreads();  // previous channel done with s_F / s_h
    // load: 8 threads per row, 8 consecutive columns each
    for (int rr = threadIdx.x >> 3; rr < IH; rr += kThreads >> 3) {
        const int yy = clampi(y0 + rr - hal, 0, H - 1);
        const float* row = Fk + (size_t)yy * fpitch;
        const int cb = (threadIdx.x & 7) * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cc = cb + c;
            if (cc < IW) s_F[rr * FW + cc] = __ldg(row + clampi(x0 + cc - hal, 0, W - 1));
        }
    }
    __syncthreads();
    // horizontal: task = (row, 8-column block); 4 blocks per row
    for (int task = threadIdx.x; task < IH * 4; task += kThreads) {
        const int rr = task >> 2, cb = (task & 3) * 8;
        const float* x = s_F + rr * FW + cb;  // x[c + hal] is column cb + c
        for (int ri = 0; ri < nd; ++ri) {
            const int rate = s_dil[ri];
            float o[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) o[c] = t[0] * x[c + hal];
#pragma unroll
            for (int q = 1; q <= KD; ++q) {
                const float tq = t[q];
#pragma unroll
                for (int c = 0; c < 8; ++c) o[c] = fmaf(tq, x[c + hal - q * rate] + x[c + hal + q * rate], o[c]);
            }
            float4* dst = reinterpret_cast<float4*>(s_h + (ri * HR + rr) * kSTW + cb);
            dst[0] = make_float4(o[0], o[1], o[2], o[3]);
            dst[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
    __syncthreads();
    // vertical: task = (column, 8-row block): 32 x 8 = 256 tasks
    const int col = threadIdx.x & 31, rb = (threadIdx.x >> 5) * kSRows;
#pragma unroll
    for (int j = 0; j < kSRows; ++j) Dk[j] = 0.f;
    for (int ri = 0; ri < nd; ++ri) {
        const int rate = s_dil[ri];
        const float* x = s_h + (ri * HR + rb + hal) * kSTW + col;  // x[j * kSTW] is output row rb + j
#pragma unroll
        for (int j = 0; j < kSRows; ++j) {
            float a = t[0] * x[j * kSTW];
#pragma unroll
            for (int q = 1; q <= KD; ++q) a = fmaf(t[q], x[(j - q * rate) * kSTW] + x[(j + q * rate) * kSTW], a);
            Dk[j] += a;
        }
    }
}

// The paper's dilation rates 1, 2, 3 at compile time: every thread loads
// its input span into registers once (float4 rows in the horizontal pass,
// one column in the vertical pass) and applies all three rates from there,
// instead of reading shared memory once per tap and rate.  Same arithmetic,
// same order of operations per output as smooth_channel.
// Input tile layout of the compile-time path: shared column j of a row holds
// image column x0 - OFF + j, OFF = hal rounded up to 4, so every row starts
// on a 16-byte boundary in global and shared memory.
template <int HAL>
struct TileGeom {
    static constexpr int OFF = (HAL + 3) / 4 * 4;
    static constexpr int NL = (OFF + kSTW + HAL + 3) / 4;  // float4 per row (covers the halo)
    static constexpr int IH = kSTH + 2 * HAL;
};

// Asynchronous copy of one channel's input tile into shared memory, one
// commit group per tile.  Interior tiles copy whole rows as 16-byte pieces;
// tiles at the image border copy element by element with clamped indices.
template <int HAL>
__device__ __forceinline__ void tile_load_async(const float* __restrict__ Fk, size_t fpitch, int H, int W, int x0,
                                                int y0, float* dst, int FW) {
    using TG = TileGeom<HAL>;
    const int xs = x0 - TG::OFF;
    const bool interior = xs >= 0 && xs + 4 * TG::NL <= W && y0 - HAL >= 0 && y0 + kSTH + HAL <= H;
    if (interior) {
        const float* src0 = Fk + (size_t)(y0 - HAL) * fpitch + xs;
        for (int i = threadIdx.x; i < TG::IH * TG::NL; i += kThreads) {
            const int rr = i / TG::NL, v = i - rr * TG::NL;
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + rr * FW + 4 * v);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src0 + (size_t)rr * fpitch + 4 * v)
                         : "memory");
        }
    } else {
        constexpr int IW = kSTW + 2 * HAL;
        for (int i = threadIdx.x; i < TG::IH * IW; i += kThreads) {
            const int rr = i / IW, cc = i - rr * IW;  // tile column cc = image column x0 - HAL + cc
            const int yy = clampi(y0 + rr - HAL, 0, H - 1), xx = clampi(x0 + cc - HAL, 0, W - 1);
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + rr * FW + (TG::OFF - HAL) + cc);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(Fk + (size_t)yy * fpitch + xx)
                         : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One channel with the tile already in s_F (the caller waited for its copy
// and synchronised the block).
template <int KD>
__device__ __forceinline__ void smooth_channel_123(const float* t, const float* s_F, int FW, float* s_h, int HR,
                                                   float2 (&Dk)[kPRows]) {
    constexpr int hal = 3 * KD;
    constexpr int IH = kSTH + 2 * hal;
    float tq[KD + 1];
#pragma unroll
    for (int q = 0; q <= KD; ++q) tq[q] = t[q];
    // horizontal: task = (row, 4-column block); the block's inputs are
    // shared columns cb + OFF - hal .. cb + OFF + 3 + hal.  Blocks of 4 give
    // 8 (64 + 2 hal) tasks for the 256 threads, which fill their last round
    // better than 4 (64 + 2 hal) blocks of 8 did (0.689 -> 0.652 ms of
    // smoothing per 2048 x 2048 step)
    constexpr int OFF = TileGeom<hal>::OFF;
    constexpr int CW = 4;  // columns per task
    constexpr int NV = (OFF + CW + hal + 3) / 4;
    for (int task = threadIdx.x; task < IH * (kSTW / CW); task += kThreads) {
        const int rr = task / (kSTW / CW), cb = (task % (kSTW / CW)) * CW;
        const float4* x4 = reinterpret_cast<const float4*>(s_F + rr * FW + cb);
        float in[NV * 4];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float4 f = x4[v];
            in[4 * v] = f.x;
            in[4 * v + 1] = f.y;
            in[4 * v + 2] = f.z;
            in[4 * v + 3] = f.w;
        }
#pragma unroll
        for (int r = 1; r <= 3; ++r) {
            float o[CW];
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                float a = tq[0] * in[OFF + c];
#pragma unroll
                for (int q = 1; q <= KD; ++q) a = fmaf(tq[q], in[OFF + c - q * r] + in[OFF + c + q * r], a);
                o[c] = a;
            }
            float4* dst = reinterpret_cast<float4*>(s_h + ((r - 1) * HR + rr) * kSTW + cb);
#pragma unroll
            for (int c = 0; c < CW; c += 4) dst[c / 4] = make_float4(o[c], o[c + 1], o[c + 2], o[c + 3]);
        }
    }
    __syncthreads();
    // vertical: thread = (column pair, 4-row block); each value is a float2
    // over two adjacent columns, so every filter step is one paired FP32
    // instruction (per lane the same rounding as the scalar form)
    const int cp = threadIdx.x & 15, rb = (threadIdx.x >> 4) * kPRows;
    float2 tq2[KD + 1];
#pragma unroll
    for (int q = 0; q <= KD; ++q) tq2[q] = make_float2(tq[q], tq[q]);
#pragma unroll
    for (int j = 0; j < kPRows; ++j) Dk[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 1; r <= 3; ++r) {
        constexpr int kMaxSpan = kPRows + 2 * KD * 3;
        const int span = kPRows + 2 * KD * r;
        const float2* x = reinterpret_cast<const float2*>(s_h + ((r - 1) * HR + rb + hal - KD * r) * kSTW) + cp;
        float2 in[kMaxSpan];
#pragma unroll
        for (int i = 0; i < kMaxSpan; ++i)
            if (i < span) in[i] = x[i * (kSTW / 2)];
#pragma unroll
        for (int j = 0; j < kPRows; ++j) {
            float2 a = __fmul2_rn(tq2[0], in[KD * r + j]);
#pragma unroll
            for (int q = 1; q <= KD; ++q)
                a = __ffma2_rn(tq2[q], __fadd2_rn(in[KD * r + j - q * r], in[KD * r + j + q * r]), a);
            Dk[j] = __fadd2_rn(Dk[j], a);
        }
    }
}

// Normalises one pixel's group of `no` smoothed values d[k] (Sec. 2.1) and
// writes it out: F32 planes, or the bf16 chunk in both pixel orders; adds
// the stored values to the per-pixel sums a1 (g) and a2 (g^2).
template <int NO, int KO>
__device__ __forceinline__ void write_pixel(int g, int no, const float* d, float eps, int gy, int gx, int H, int W,
                                            float* __restrict__ c32, size_t cpitch, size_t cplane,
                                            __nv_bfloat16* __restrict__ rm, __nv_bfloat16* __restrict__ cm,
                                            float& a1, float& a2) {
    const bool bf = rm != nullptr;
    float n2 = 0.f;
#pragma unroll
    for (int k = 0; k < KO; ++k)
        if (k < no) n2 = fmaf(d[k], d[k], n2);
    const float den = sqrtf(n2) + eps;
    const float inv = den > 0.f ? 1.f / den : 0.f;  // NaN stays NaN through d * inv
    const bool in = gy < H && gx < W;
    float vs[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        if (k >= no) break;
        float v = (den > 0.f || den != den) ? d[k] * inv : 0.f;
        if (bf) v = __bfloat162float(__float2bfloat16_rn(v));
        vs[k] = v;
        a1 += v;
        a2 = fmaf(v, v, a2);
        if (c32 && in) c32[(size_t)(g * no + k) * cplane + (size_t)gy * cpitch + gx] = v;
    }
    if constexpr (NO == 6) {
        if (bf && in) {  // chunk g: the six channels, then two zeros
            auto pack = [](float lo, float hi) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
                return *reinterpret_cast<const unsigned*>(&h);
            };
            const uint4 chunk = make_uint4(pack(vs[0], vs[1]), pack(vs[2], vs[3]), pack(vs[4], vs[5]), 0u);
            const size_t npx = (size_t)H * W;
            const size_t pix = (size_t)gy * W + gx, cpx = (size_t)gx * H + gy;
            *reinterpret_cast<uint4*>(rm + ((size_t)g * npx + pix) * 8) = chunk;
            *reinterpret_cast<uint4*>(cm + ((size_t)g * npx + cpx) * 8) = chunk;
        }
    }
}

// One group of `no` channels with radius and rates at run time: smooth each
// channel, normalise the group in registers and write it out.
template <int NO>
__device__ __forceinline__ void smooth_group(int g, const float* __restrict__ F, size_t fpitch, size_t fplane, int H,
                                             int W, const SmoothTaps& tp, const int* s_dil, const float* t,
                                             float* s_F, int FW, float* s_h, int HR, int x0,
                                             int y0, float* __restrict__ c32, size_t cpitch, size_t cplane,
                                             __nv_bfloat16* __restrict__ rm, __nv_bfloat16* __restrict__ cm,
                                             float (&a1)[kSRows], float (&a2)[kSRows]) {
    constexpr int KO = NO > 0 ? NO : kMaxOrient;
    const int no = NO > 0 ? NO : tp.no;
    const int col = threadIdx.x & 31, rb = (threadIdx.x >> 5) * kSRows;
    const int gx = x0 + col;
    float D[KO][kSRows];
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        if (k >= no) break;
        const float* Fk = F + (size_t)(g * no + k) * fplane;
        {
            const int hal = tp.halo[g], Kd = tp.Kd[g];
            switch (Kd) {
                case 0: smooth_channel<0>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
                case 1: smooth_channel<1>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
                case 2: smooth_channel<2>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
                case 3: smooth_channel<3>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
                case 4: smooth_channel<4>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
                case 5: smooth_channel<5>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
                default: smooth_channel<6>(Fk, fpitch, H, W, x0, y0, hal, tp.n_dil, s_dil, t, s_F, FW, s_h, HR, D[k]); break;
            }
        }
    }
    // group normalisation in registers; write this group
#pragma unroll
    for (int j = 0; j < kSRows; ++j) {
        float d[KO];
#pragma unroll
        for (int k = 0; k < KO; ++k) d[k] = D[k][j];
        write_pixel<NO, KO>(g, no, d, tp.eps, y0 + rb + j, gx, H, W, c32, cpitch, cplane, rm, cm, a1[j], a2[j]);
    }
}

// One group with radius KDG and the rates 1, 2, 3 at compile time: tiles
// double-buffered with asynchronous copies, paired vertical pass; a thread
// owns 2 columns x kPRows rows of every channel.
template <int NO, int KDG>
__device__ __forceinline__ void smooth_group_123(int g, const float* __restrict__ F, size_t fpitch, size_t fplane,
                                                 int H, int W, float eps, const float* t, float* s_F,
                                                 float* s_F2, int FW, float* s_h, int HR, int x0, int y0,
                                                 float* __restrict__ c32, size_t cpitch, size_t cplane,
                                                 __nv_bfloat16* __restrict__ rm, __nv_bfloat16* __restrict__ cm,
                                                 float (&a1)[kPRows][2], float (&a2)[kPRows][2]) {
    constexpr int KO = NO;
    const int cp = threadIdx.x & 15, rb = (threadIdx.x >> 4) * kPRows;
    const int gx = x0 + 2 * cp;
    float2 D[KO][kPRows];
    __syncthreads();  // the previous group is done with both tile buffers (and the taps are written)
    tile_load_async<3 * KDG>(F + (size_t)(g * NO) * fplane, fpitch, H, W, x0, y0, s_F, FW);
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        const float* Fk = F + (size_t)(g * NO + k) * fplane;
        // tile k is in buffer k & 1; prefetch tile k+1 into the other one (its
        // last reader, channel k-1's horizontal pass, is behind the barrier
        // that ended that pass)
        if (k + 1 < KO) {
            tile_load_async<3 * KDG>(Fk + fplane, fpitch, H, W, x0, y0, (k & 1) ? s_F : s_F2, FW);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();  // tile k visible; every thread is done with channel k-1
        smooth_channel_123<KDG>(t, (k & 1) ? s_F2 : s_F, FW, s_h, HR, D[k]);
    }
#pragma unroll
    for (int j = 0; j < kPRows; ++j) {
        float d0[KO], d1[KO];
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            d0[k] = D[k][j].x;
            d1[k] = D[k][j].y;
        }
        const int gy = y0 + rb + j;
        write_pixel<NO, KO>(g, NO, d0, eps, gy, gx, H, W, c32, cpitch, cplane, rm, cm, a1[j][0], a2[j][0]);
        write_pixel<NO, KO>(g, NO, d1, eps, gy, gx + 1, H, W, c32, cpitch, cplane, rm, cm, a1[j][1], a2[j][1]);
    }
}

// The paper's dilation rates 1, 2, 3 with smoothing radius KDG at compile
// time, one group g per launch: the kernel holds only one group's code (its
// instruction footprint is what limits the fully unrolled passes) and fits
// two CTAs per SM.  The second group's launch continues the per-pixel sums
// from the stored planes, adding in the same order as one launch would.
// One image (`one`, CTA = tile in row-major tile order) or a batch (device
// table `jobs`, CTAs of image j from begin[j]).
template <int NO, int KDG>
__global__ void __launch_bounds__(kThreads, 2)
    k_sfoc_smooth_grp(const __grid_constant__ ImgJob one, const ImgJob* __restrict__ jobs,
                      const int* __restrict__ begin, int n_jobs, SmoothTaps tp, int g) {
    extern __shared__ float sm[];
    int tile;
    const ImgJob& J = img_job(one, jobs, begin, n_jobs, &tile);
    const float* __restrict__ F = J.F;
    const size_t fpitch = J.fpitch, fplane = J.fpitch * (size_t)J.H;
    const int H = J.H, W = J.W;
    float* __restrict__ c32 = J.c32;
    const size_t cpitch = J.cpitch, cplane = J.cpitch * (size_t)J.H;
    __nv_bfloat16* __restrict__ rm = J.rm;
    __nv_bfloat16* __restrict__ cm = J.cm;
    float* __restrict__ s1 = J.s1;
    float* __restrict__ s2 = J.s2;
    __shared__ float s_tap[kMaxSmoothRadius + 1];
    if (threadIdx.x == 0) {  // constant indices: the parameter block stays in the constant bank
#pragma unroll
        for (int q = 0; q <= kMaxSmoothRadius; ++q) s_tap[q] = g ? tp.g[1][q] : tp.g[0][q];
    }
    constexpr int hal = 3 * KDG;
    const int FW = smooth_row_stride(hal);
    constexpr int HR = kSTH + 2 * hal;
    float* s_F = sm;                   // HR x FW
    float* s_h = s_F + HR * FW;        // 3 x HR x kSTW
    float* s_F2 = s_h + 3 * HR * kSTW;  // second input tile buffer
    const int ntx = (W + kSTW - 1) / kSTW;
    const int tby = tile / ntx;
    const int x0 = (tile - tby * ntx) * kSTW, y0 = tby * kSTH;
    const int cp = threadIdx.x & 15, rb = (threadIdx.x >> 4) * kPRows;

    float a1[kPRows][2], a2[kPRows][2];
#pragma unroll
    for (int j = 0; j < kPRows; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int gy = y0 + rb + j, gx = x0 + 2 * cp + e;
            const bool in = g > 0 && gy < H && gx < W;
            a1[j][e] = in ? s1[(size_t)gy * cpitch + gx] : 0.f;
            a2[j][e] = in ? s2[(size_t)gy * cpitch + gx] : 0.f;
        }
    smooth_group_123<NO, KDG>(g, F, fpitch, fplane, H, W, tp.eps, s_tap, s_F, s_F2, FW, s_h, HR, x0, y0, c32, cpitch,
                              cplane, rm, cm, a1, a2);
#pragma unroll
    for (int j = 0; j < kPRows; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int gy = y0 + rb + j, gx = x0 + 2 * cp + e;
            if (gy < H && gx < W) {
                s1[(size_t)gy * cpitch + gx] = a1[j][e];
                s2[(size_t)gy * cpitch + gx] = a2[j][e];
            }
        }
}

// Any radii and rates at run time.
template <int NO>
__global__ void __launch_bounds__(kThreads, 1)
    k_sfoc_smooth(const float* __restrict__ F, size_t fpitch, size_t fplane, int H, int W, SmoothTaps tp,
                  float* __restrict__ c32, size_t cpitch, size_t cplane, __nv_bfloat16* __restrict__ rm,
                  __nv_bfloat16* __restrict__ cm, float* __restrict__ s1, float* __restrict__ s2) {
    extern __shared__ float sm[];
    __shared__ float s_tap[2][kMaxSmoothRadius + 1];  // taps in shared memory: no local copy of the params
    __shared__ int s_dil[kMaxDil];
    if (threadIdx.x < 2 * (kMaxSmoothRadius + 1)) {
        const int gg = threadIdx.x / (kMaxSmoothRadius + 1), q = threadIdx.x % (kMaxSmoothRadius + 1);
        s_tap[gg][q] = tp.g[gg][q];
    }
    if (threadIdx.x < kMaxDil) s_dil[threadIdx.x] = tp.dil[threadIdx.x];
    const int maxhal = max(tp.halo[0], tp.halo[1]);
    const int FW = smooth_row_stride(maxhal);
    const int HR = kSTH + 2 * maxhal;
    float* s_F = sm;             // HR x FW
    float* s_h = s_F + HR * FW;  // n_dil x HR x kSTW
    const int x0 = blockIdx.x * kSTW, y0 = blockIdx.y * kSTH;
    const int col = threadIdx.x & 31, rb = (threadIdx.x >> 5) * kSRows;
    const int gx = x0 + col;
    const int no = NO > 0 ? NO : tp.no;
    const int ng = tp.z / no;

    float a1[kSRows], a2[kSRows];
#pragma unroll
    for (int j = 0; j < kSRows; ++j) a1[j] = a2[j] = 0.f;
    for (int g = 0; g < ng; ++g)
        smooth_group<NO>(g, F, fpitch, fplane, H, W, tp, s_dil, s_tap[g], s_F, FW, s_h, HR, x0, y0, c32, cpitch,
                         cplane, rm, cm, a1, a2);
#pragma unroll
    for (int j = 0; j < kSRows; ++j) {
        const int gy = y0 + rb + j;
        if (gy < H && gx < W) {
            s1[(size_t)gy * cpitch + gx] = a1[j];
            s2[(size_t)gy * cpitch + gx] = a2[j];
        }
    }
}

bool smooth_is_paper(const SmoothTaps& tp) {
    return tp.no == 6 && tp.z == 12 && tp.n_dil == 3 && tp.dil[0] == 1 && tp.dil[1] == 2 && tp.dil[2] == 3 &&
           tp.Kd[0] == 3 && tp.Kd[1] == 5;
}

__global__ void k_cube_export_bf16(const __nv_bfloat16* __restrict__ rm, int H, int W, int z, float* __restrict__ out) {
    size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * z; i += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(i / n);
        size_t p = i - (size_t)k * n;
        int chunk = k / 6, j = k % 6;  // chunk g = the six channels of group g + two zeros
        out[i] = __bfloat162float(rm[((size_t)chunk * n + p) * 8 + j]);
    }
}

__global__ void k_cube_export_f32(const float* __restrict__ c32, int H, int W, int z, size_t pitch, float* __restrict__ out) {
    size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * z; i += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(i / n);
        size_t p = i - (size_t)k * n;
        int y = (int)(p / W), x = (int)(p - (size_t)y * W);
        out[i] = c32[((size_t)k * H + y) * pitch + x];
    }
}

bool steer_is_paper(const SteerTaps& tp) {
    return tp.ns == 3 && tp.K1[0] == 2 && tp.K1[1] == 3 && tp.K1[2] == 3 && tp.second && tp.K2 == 5 && tp.no == 6;
}

template <typename T>
cudaError_t launch_steer_any(const T* img, int H, int W, size_t pitch, float* F, size_t fpitch, const SteerTaps& tp,
                             cudaStream_t st) {
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
    // the paper's scales (0.6, 0.8, 1.0 and 1.5 at 3 sigma: radii 2, 3, 3, 5), six orientations
    if (steer_is_paper(tp)) {
        auto kern = k_sfoc_steer_ct<T, 2, 3, 3, 5>;
        const size_t smem = sizeof(float) * 9 * (size_t)(kTH + 10) * kTW;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ImgJob one;
        memset(&one, 0, sizeof(one));
        one.img = img;
        one.pitch = pitch;
        one.H = H;
        one.W = W;
        one.F = F;
        one.fpitch = fpitch;
        kern<<<grid.x * grid.y, kThreads, smem, st>>>(one, nullptr, nullptr, 0, tp);
        return cudaGetLastError();
    }
    const int hal = tp.halo;
    const int IH = kTH + 2 * hal, IW = kTW + 2 * hal;
    const int np = 2 * tp.ns + (tp.second ? 3 : 0);
    size_t smem = sizeof(float) * ((size_t)IH * IW + (size_t)np * IH * kTW);
    cudaError_t e = cudaFuncSetAttribute(k_sfoc_steer<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sfoc_steer<T><<<grid, kThreads, smem, st>>>(img, H, W, pitch, F, fpitch, fpitch * (size_t)H, tp);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sfoc_steer(const float* img, int H, int W, size_t pitch, float* F, size_t fpitch,
                              const SteerTaps& tp, int /*z_first*/, cudaStream_t st) {
    return launch_steer_any(img, H, W, pitch, F, fpitch, tp, st);
}

cudaError_t launch_sfoc_steer(const uint16_t* img, int H, int W, size_t pitch, float* F, size_t fpitch,
                              const SteerTaps& tp, int /*z_first*/, cudaStream_t st) {
    return launch_steer_any(img, H, W, pitch, F, fpitch, tp, st);
}

int smooth_launch_count(const SmoothTaps& tp) { return smooth_is_paper(tp) ? 2 : 1; }

namespace {

// the two group launches of the paper's smoothing (sigma_d 1.0 / 1.5, rates
// 1, 2, 3) over `ctas` CTAs
cudaError_t launch_smooth_paper(const ImgJob& one, const ImgJob* jobs, const int* begin, int n_jobs, int ctas,
                                const SmoothTaps& tp, cudaStream_t st) {
    auto run = [&](auto kern, int g, int hal) -> cudaError_t {
        const int HR = kSTH + 2 * hal, FW = smooth_row_stride(hal);
        const size_t smem = sizeof(float) * (2 * (size_t)HR * FW + 3 * (size_t)HR * kSTW);
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e2 == cudaSuccess)
            e2 = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared);
        if (e2 != cudaSuccess) return e2;
        kern<<<ctas, kThreads, smem, st>>>(one, jobs, begin, n_jobs, tp, g);
        return cudaGetLastError();
    };
    cudaError_t e = run(k_sfoc_smooth_grp<6, 3>, 0, 9);
    if (e == cudaSuccess) e = run(k_sfoc_smooth_grp<6, 5>, 1, 15);
    return e;
}

}  // namespace

bool sfoc_batch_supported(const SteerTaps& st, const SmoothTaps& sm) { return steer_is_paper(st) && smooth_is_paper(sm); }

void sfoc_batch_tiles(int H, int W, int* steer_ctas, int* smooth_ctas) {
    *steer_ctas = ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
    *smooth_ctas = ((W + kSTW - 1) / kSTW) * ((H + kSTH - 1) / kSTH);
}

cudaError_t launch_sfoc_batch(const ImgJob* jobs, int n_jobs, const int* steer_begin, int steer_ctas,
                              const int* smooth_begin, int smooth_ctas, const SteerTaps& st, const SmoothTaps& sm,
                              cudaStream_t s) {
    if (n_jobs <= 0) return cudaSuccess;
    if (!sfoc_batch_supported(st, sm)) return cudaErrorNotSupported;
    ImgJob none;
    memset(&none, 0, sizeof(none));
    auto kern = k_sfoc_steer_ct<float, 2, 3, 3, 5>;
    const size_t smem = sizeof(float) * 9 * (size_t)(kTH + 10) * kTW;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<steer_ctas, kThreads, smem, s>>>(none, jobs, steer_begin, n_jobs, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_smooth_paper(none, jobs, smooth_begin, n_jobs, smooth_ctas, sm, s);
}

cudaError_t launch_sfoc_smooth(const float* F, size_t fpitch, int H, int W, const SmoothTaps& tp, Cube& c,
                               cudaStream_t st) {
    dim3 grid((W + kSTW - 1) / kSTW, (H + kSTH - 1) / kSTH);
    cudaError_t e;
    if (smooth_is_paper(tp)) {  // sigma_d 1.0 / 1.5 with rates 1, 2, 3 (Sec. 2.1): one launch per group
        ImgJob one;
        memset(&one, 0, sizeof(one));
        one.H = H;
        one.W = W;
        one.F = const_cast<float*>(F);
        one.fpitch = fpitch;
        one.c32 = c.f32;
        one.cpitch = c.pitch;
        one.rm = c.rm;
        one.cm = c.cm;
        one.s1 = c.s1;
        one.s2 = c.s2;
        return launch_smooth_paper(one, nullptr, nullptr, 0, (int)(grid.x * grid.y), tp, st);
    }
    const int maxhal = tp.halo[0] > tp.halo[1] ? tp.halo[0] : tp.halo[1];
    const int HR = kSTH + 2 * maxhal, FW = smooth_row_stride(maxhal);
    size_t smem = sizeof(float) * ((size_t)HR * FW + (size_t)tp.n_dil * HR * kSTW);
    if (tp.no == 6) {
        e = cudaFuncSetAttribute(k_sfoc_smooth<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sfoc_smooth<6><<<grid, kThreads, smem, st>>>(F, fpitch, fpitch * (size_t)H, H, W, tp, c.f32, c.pitch,
                                                       c.pitch * (size_t)H, c.rm, c.cm, c.s1, c.s2);
    } else {
        if (c.rm) return cudaErrorNotSupported;  // bf16 layouts need 12 channels
        e = cudaFuncSetAttribute(k_sfoc_smooth<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sfoc_smooth<0><<<grid, kThreads, smem, st>>>(F, fpitch, fpitch * (size_t)H, H, W, tp, c.f32, c.pitch,
                                                       c.pitch * (size_t)H, c.rm, c.cm, c.s1, c.s2);
    }
    return cudaGetLastError();
}

cudaError_t launch_cube_export(const Cube& c, float* out, cudaStream_t st) {
    int blocks = 152 * 8;
    if (c.dtype == SFOC_DTYPE_BF16)
        k_cube_export_bf16<<<blocks, 256, 0, st>>>(c.rm, c.H, c.W, c.z, out);
    else
        k_cube_export_f32<<<blocks, 256, 0, st>>>(c.f32, c.H, c.W, c.z, c.pitch, out);
    return cudaGetLastError();
}

}  // namespace sfoc
