// Plain FP32 correlation R_ST (Eq. 10 of arXiv 2202.13347) on CUDA cores.
//
// One CTA per point.  For each channel the search window S_c ((m+2R)^2) and
// the zero-mean template T_c - mean(T) (m^2) are staged in shared memory; a
// thread owns 8 consecutive dx of one dy and slides along the template row
// with float4 loads (12 window values and 4 template values feed 32 FMAs).
// Correlating against the zero-mean template gives the numerator of Eq. 9
// directly, sum S (T - T_bar) = R_ST - R_S R_T / mnz, without the
// cancellation of the two large terms.
#include "internal.h"

namespace sfoc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int roundup(int v, int a) { return (v + a - 1) / a * a; }

template <int TPT>
__global__ void __launch_bounds__(kThreads) k_corr_f32(const __grid_constant__ MatchJob one,
                                                        const MatchJob* __restrict__ jobs,
                                                        const int2* __restrict__ items) {
    extern __shared__ __align__(16) float sm[];
    int k;
    const MatchJob& J = item_job(one, jobs, items, blockIdx.x, &k);
    const PointStat st = J.stats[k];
    if (st.status != SFOC_PT_OK) return;  // the NCC stage ignores this map
    const float* __restrict__ ref = J.rf32;
    const float* __restrict__ sen = J.sf32;
    const size_t rpitch = J.rpitch, rplane = J.rplane, spitch = J.spitch, splane = J.splane;
    const int32_t* __restrict__ pts = J.pts;
    const int m = J.m, R = J.R, z = J.z;
    const int P1 = 2 * R + 1;
    const int Lw = m + 2 * R;
    const int mp = roundup(m, 4);
    const int Xt = roundup(P1, 8);
    const int Ls = Xt + mp;
    const int ntx = Xt / 8;
    const int ntile = P1 * ntx;
    float* S = sm;              // Lw x Ls
    float* T = sm + Lw * Ls;    // m x mp
    const int h = template_half(m);
    const int ty0 = pts[2 * k + 1] - h, tx0 = pts[2 * k] - h;
    const float tmean = st.tmean;

    float acc[TPT][8];
#pragma unroll
    for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int d = 0; d < 8; ++d) acc[j][d] = 0.f;

    for (int c = 0; c < z; ++c) {
        __syncthreads();
        const float* rc = ref + (size_t)c * rplane;
        for (int i = threadIdx.x; i < Lw * Ls; i += kThreads) {
            int r = i / Ls, x = i - r * Ls;
            S[i] = x < Lw ? __ldg(rc + (size_t)(ty0 - R + r) * rpitch + (tx0 - R + x)) : 0.f;
        }
        const float* sc = sen + (size_t)c * splane;
        for (int i = threadIdx.x; i < m * mp; i += kThreads) {
            int r = i / mp, u = i - r * mp;
            T[i] = u < m ? __ldg(sc + (size_t)(ty0 + r) * spitch + (tx0 + u)) - tmean : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int t = threadIdx.x + j * kThreads;
            if (t < ntile) {
                const int dy = t / ntx, dx0 = (t - dy * ntx) * 8;
                for (int i = 0; i < m; ++i) {
                    const float* srow = S + (i + dy) * Ls + dx0;
                    const float* trow = T + i * mp;
                    for (int u0 = 0; u0 < mp; u0 += 4) {
                        float4 a = *reinterpret_cast<const float4*>(srow + u0);
                        float4 b = *reinterpret_cast<const float4*>(srow + u0 + 4);
                        float4 e = *reinterpret_cast<const float4*>(srow + u0 + 8);
                        float4 tv = *reinterpret_cast<const float4*>(trow + u0);
                        float s[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, e.x, e.y, e.z, e.w};
                        float tq[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int d = 0; d < 8; ++d) acc[j][d] = fmaf(s[q + d], tq[q], acc[j][d]);
                    }
                }
            }
        }
    }
    float* out = J.maps + (size_t)k * P1 * P1;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        const int t = threadIdx.x + j * kThreads;
        if (t < ntile) {
            const int dy = t / ntx, dx0 = (t - dy * ntx) * 8;
#pragma unroll
            for (int d = 0; d < 8; ++d)
                if (dx0 + d < P1) out[dy * P1 + dx0 + d] = acc[j][d];
        }
    }
}

size_t smem_bytes(int m, int R) {
    int P1 = 2 * R + 1, Lw = m + 2 * R;
    int mp = (m + 3) / 4 * 4, Xt = (P1 + 7) / 8 * 8;
    return sizeof(float) * ((size_t)Lw * (Xt + mp) + (size_t)m * mp);
}

}  // namespace

int corr_f32_class(int R) {
    const int P1 = 2 * R + 1;
    const int tpt = (P1 * ((P1 + 7) / 8) + kThreads - 1) / kThreads;
    return tpt <= 1 ? 1 : tpt <= 2 ? 2 : tpt <= 4 ? 4 : tpt <= 8 ? 8 : 0;
}

bool corr_f32_supported(int m, int R) { return corr_f32_class(R) > 0 && smem_bytes(m, R) <= 227 * 1024; }

// tpt: threads-per-tile class, at least corr_f32_class of the largest R
cudaError_t launch_corr_f32(const MatchJob& one, const ItemSet& is, int tpt, cudaStream_t st) {
    const int n = is.items ? is.n : one.n;
    if (n <= 0) return cudaSuccess;
    const int m = is.items ? is.max_m : one.m, R = is.items ? is.max_R : one.R;
    if (!corr_f32_supported(m, R) || tpt < corr_f32_class(R)) return cudaErrorInvalidValue;
    size_t smem = smem_bytes(m, R);
    cudaError_t e;
#define SFOC_CORR_CASE(N)                                                                                      \
    e = cudaFuncSetAttribute(k_corr_f32<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
    if (e != cudaSuccess) return e;                                                                            \
    k_corr_f32<N><<<n, kThreads, smem, st>>>(one, is.jobs, is.items);
    if (tpt <= 1) { SFOC_CORR_CASE(1) }
    else if (tpt <= 2) { SFOC_CORR_CASE(2) }
    else if (tpt <= 4) { SFOC_CORR_CASE(4) }
    else if (tpt <= 8) { SFOC_CORR_CASE(8) }
    else return cudaErrorInvalidValue;
#undef SFOC_CORR_CASE
    return cudaGetLastError();
}

}  // namespace sfoc
