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

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kTW = 32;          // output tile width (one warp across)
constexpr int kTH = 32;          // output tile height
constexpr int kThreads = 256;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

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

__global__ void __launch_bounds__(kThreads) k_sfoc_steer(const float* __restrict__ img, int H, int W,
                                                          size_t pitch, float* __restrict__ F, size_t fpitch,
                                                          size_t fplane, SteerTaps tp) {
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
        s_img[i] = __ldg(img + (size_t)gy * pitch + gx);
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

// Smoothing: per channel, load the F tile with the group's halo (clamped),
// horizontal dilated passes for each rate into shared planes, vertical
// passes summed over rates into s_D.  Then normalise each group per pixel.
constexpr int kMaxSmoothHalo = kMaxDil * kMaxSmoothRadius;  // 18

__global__ void __launch_bounds__(kThreads) k_sfoc_smooth(const float* __restrict__ F, size_t fpitch,
                                                           size_t fplane, int H, int W, SmoothTaps tp,
                                                           float* __restrict__ c32, size_t cpitch, size_t cplane,
                                                           __nv_bfloat16* __restrict__ rm,
                                                           __nv_bfloat16* __restrict__ cm,
                                                           float* __restrict__ s1, float* __restrict__ s2) {
    extern __shared__ float sm[];
    const int maxhal = max(tp.halo[0], tp.halo[1]);
    const int FW = kTW + 2 * maxhal;
    float* s_F = sm;                                  // (kTH + 2 maxhal) x FW
    float* s_h = s_F + (kTH + 2 * maxhal) * FW;       // n_dil x (kTH + 2 maxhal) x kTW
    float* s_D = s_h + tp.n_dil * (kTH + 2 * maxhal) * kTW;  // z x kTH x kTW
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;

    for (int k = 0; k < tp.z; ++k) {
        const int g = k < tp.no ? 0 : 1;
        const int hal = tp.halo[g];
        const int IW = kTW + 2 * hal, IH = kTH + 2 * hal;
        const float* Fk = F + (size_t)k * fplane;
        __syncthreads();  // previous channel done with s_F / s_h
        for (int i = threadIdx.x; i < IH * IW; i += kThreads) {
            int r = i / IW, c = i - r * IW;
            int gy = clampi(y0 + r - hal, 0, H - 1), gx = clampi(x0 + c - hal, 0, W - 1);
            s_F[r * FW + c] = __ldg(Fk + (size_t)gy * fpitch + gx);
        }
        __syncthreads();
        const float* t = tp.g[g];
        const int Kd = tp.Kd[g];
        for (int i = threadIdx.x; i < IH * kTW; i += kThreads) {
            int r = i / kTW, c = i - r * kTW;
            const float* x = s_F + r * FW + c + hal;
            for (int ri = 0; ri < tp.n_dil; ++ri) {
                const int rate = tp.dil[ri];
                float acc = t[0] * x[0];
#pragma unroll
                for (int q = 1; q <= kMaxSmoothRadius; ++q)
                    if (q <= Kd) acc = fmaf(t[q], x[-q * rate] + x[q * rate], acc);
                s_h[(ri * (kTH + 2 * maxhal) + r) * kTW + c] = acc;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTH * kTW; i += kThreads) {
            int r = i / kTW, c = i - r * kTW;
            float acc = 0.f;
            for (int ri = 0; ri < tp.n_dil; ++ri) {
                const int rate = tp.dil[ri];
                const float* x = s_h + (ri * (kTH + 2 * maxhal) + r + hal) * kTW + c;
                float a = t[0] * x[0];
#pragma unroll
                for (int q = 1; q <= kMaxSmoothRadius; ++q)
                    if (q <= Kd) a = fmaf(t[q], x[-q * rate * kTW] + x[q * rate * kTW], a);
                acc += a;
            }
            s_D[(k * kTH + r) * kTW + c] = acc;
        }
    }
    __syncthreads();

    // group normalisation, per pixel; values stay in s_D (rounded to bf16
    // when the cube is bf16, so the sum planes describe the stored values)
    const bool bf = rm != nullptr;
    for (int i = threadIdx.x; i < kTH * kTW; i += kThreads) {
        int r = i / kTW, c = i - r * kTW;
        int gy = y0 + r, gx = x0 + c;
        float a1 = 0.f, a2 = 0.f;
        const int ng = tp.z / tp.no;
        for (int g = 0; g < ng; ++g) {
            float n2 = 0.f;
            for (int k = 0; k < tp.no; ++k) {
                float v = s_D[((g * tp.no + k) * kTH + r) * kTW + c];
                n2 = fmaf(v, v, n2);
            }
            float inv = 1.f / (sqrtf(n2) + tp.eps);
            if (!(sqrtf(n2) + tp.eps > 0.f)) inv = 0.f;
            for (int k = 0; k < tp.no; ++k) {
                float* p = &s_D[((g * tp.no + k) * kTH + r) * kTW + c];
                float v = *p * inv;
                if (bf) v = __bfloat162float(__float2bfloat16_rn(v));
                *p = v;
                a1 += v;
                a2 = fmaf(v, v, a2);
            }
        }
        if (gy < H && gx < W) {
            s1[(size_t)gy * cpitch + gx] = a1;
            s2[(size_t)gy * cpitch + gx] = a2;
            if (c32)
                for (int k = 0; k < tp.z; ++k) c32[(size_t)k * cplane + (size_t)gy * cpitch + gx] = s_D[(k * kTH + r) * kTW + c];
        }
    }
    if (!bf) return;
    __syncthreads();
    // bf16 chunked layouts: chunk 0 = channels 0..7, chunk 1 = 8..11 + zeros
    auto pack = [&](int r, int c, int chunk) -> uint4 {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int k = chunk * 8 + j;
            v[j] = __float2bfloat16_rn(k < tp.z ? s_D[(k * kTH + r) * kTW + c] : 0.f);
        }
        return *reinterpret_cast<uint4*>(v);
    };
    for (int i = threadIdx.x; i < 2 * kTH * kTW; i += kThreads) {
        int chunk = i / (kTH * kTW);
        int j = i - chunk * kTH * kTW;
        {   // row-major: consecutive threads -> consecutive x
            int r = j / kTW, c = j - r * kTW;
            int gy = y0 + r, gx = x0 + c;
            if (gy < H && gx < W)
                *reinterpret_cast<uint4*>(rm + (((size_t)chunk * H + gy) * W + gx) * 8) = pack(r, c, chunk);
        }
        {   // column-major: consecutive threads -> consecutive y
            int c = j / kTH, r = j - c * kTH;
            int gy = y0 + r, gx = x0 + c;
            if (gy < H && gx < W)
                *reinterpret_cast<uint4*>(cm + (((size_t)chunk * W + gx) * H + gy) * 8) = pack(r, c, chunk);
        }
    }
}

__global__ void k_cube_export_bf16(const __nv_bfloat16* __restrict__ rm, int H, int W, int z, float* __restrict__ out) {
    size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * z; i += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(i / n);
        size_t p = i - (size_t)k * n;
        int chunk = k / 8, j = k % 8;
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

}  // namespace

cudaError_t launch_sfoc_steer(const float* img, int H, int W, size_t pitch, float* F, size_t fpitch,
                              const SteerTaps& tp, int /*z_first*/, cudaStream_t st) {
    const int hal = tp.halo;
    const int IH = kTH + 2 * hal, IW = kTW + 2 * hal;
    const int np = 2 * tp.ns + (tp.second ? 3 : 0);
    size_t smem = sizeof(float) * ((size_t)IH * IW + (size_t)np * IH * kTW);
    cudaError_t e = cudaFuncSetAttribute(k_sfoc_steer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
    k_sfoc_steer<<<grid, kThreads, smem, st>>>(img, H, W, pitch, F, fpitch, fpitch * (size_t)H, tp);
    return cudaGetLastError();
}

cudaError_t launch_sfoc_smooth(const float* F, size_t fpitch, int H, int W, const SmoothTaps& tp, Cube& c,
                               cudaStream_t st) {
    const int maxhal = tp.halo[0] > tp.halo[1] ? tp.halo[0] : tp.halo[1];
    const int IH = kTH + 2 * maxhal, IW = kTW + 2 * maxhal;
    size_t smem = sizeof(float) * ((size_t)IH * IW + (size_t)tp.n_dil * IH * kTW + (size_t)tp.z * kTH * kTW);
    cudaError_t e = cudaFuncSetAttribute(k_sfoc_smooth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
    k_sfoc_smooth<<<grid, kThreads, smem, st>>>(F, fpitch, fpitch * (size_t)H, H, W, tp, c.f32, c.pitch,
                                                c.pitch * (size_t)H, c.rm, c.cm, c.s1, c.s2);
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
