// Correlation R_ST (Eq. 10 of arXiv 2202.13347) by the discrete Fourier
// transform, Eq. 13: per point and channel the window S_c and the zero-mean
// template T_c - mean(T) are zero-padded to L x L (L >= m + 2R, so the
// circular correlation equals the linear one at every offset in [0, 2R]),
// their spectra multiplied (one conjugated) and summed over the channels,
// and one inverse transform gives the numerator of Eq. 9 at every offset.
// FP32 throughout, from the F32 cube; one CTA per point.
//
// Transforms.  A length-L transform (L = 8E) is done by a group of 8
// threads: thread t holds x[t + 8j] (j < E), takes the E-point DFT over j in
// registers, multiplies by W_L^{t k1}, and after an 8 x 8 transpose through
// a padded shared-memory scratch takes the 8-point DFT over t.  The output
// X[t + 8m] lands in the same stride-8 layout, so rows and columns of the
// L x L array chain without reordering.
// Channel c: z = S_c + i (T_c - mean) is transformed once (rows, then
// columns); the spectra of the two real inputs follow from Z[k] and
// conj(Z[-k]):  X = (Z[k] + conj Z[-k]) / 2,  Y = (Z[k] - conj Z[-k]) / 2i.
// Columns are taken in conjugate pairs (c, L - c) (and the two
// self-conjugate columns 0 and L/2 together), so a group holds both Z[k]
// and Z[-k]; the products X conj(Y) for the half spectrum kx in [0, L/2]
// are summed over the channels in registers (the Nyquist column kx = L/2 in
// shared memory).  Inverse: columns kx in [0, L/2], then for each of the
// 2R + 1 wanted rows the Hermitian-extended row.
#include <math.h>

#include <type_traits>

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kScP = 9;  // transpose scratch row pitch (float2): conflict-free columns

// One group of 8 threads per conjugate column pair: L/2 groups.
template <int L>
struct FftShape {
    static constexpr int E = L / 8;
    static constexpr int G = L / 2;                     // groups of 8 threads
    static constexpr int T = 8 * G;                     // threads
    static constexpr int ZP = L + 2;                    // row pitch of the L x L array (float2)
    // scratch per group (float2): 8 rows per array, both arrays of the dual
    // transform (16 rows), or E rows of one; consecutive groups 64 B apart mod 128
    static constexpr int SG = (E < 16 ? 16 : E) * kScP + 8;
    static constexpr size_t smem = sizeof(float2) * ((size_t)L * ZP + (size_t)G * SG + 8 * E + L);
};

// cos(2 pi q / 16) for q in [0, 16)
__device__ __forceinline__ constexpr float cos16(int q) {
    constexpr float c1 = 0.92387953251128674f, c2 = 0.70710678118654752f, c3 = 0.38268343236508977f;
    switch (q & 15) {
        case 0: return 1.f;
        case 1: return c1;
        case 2: return c2;
        case 3: return c3;
        case 4: return 0.f;
        case 5: return -c3;
        case 6: return -c2;
        case 7: return -c1;
        case 8: return -1.f;
        case 9: return -c1;
        case 10: return -c2;
        case 11: return -c3;
        case 12: return 0.f;
        case 13: return c3;
        case 14: return c2;
        default: return c1;
    }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// x * exp(SIGN 2 pi i k / N), k and N compile-time after unrolling (N divides 16)
template <int SIGN>
__device__ __forceinline__ float2 twiddle(float2 x, int k, int N) {
    const int q = (k * (16 / N)) & 15;
    if (q == 0) return x;
    if (q == 8) return make_float2(-x.x, -x.y);
    if (q == 4) return SIGN < 0 ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
    if (q == 12) return SIGN < 0 ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    const float c = cos16(q), s = SIGN * cos16(q - 4);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
}

// in-place N-point DFT, sum_j v[j] exp(SIGN 2 pi i j k / N), natural order
template <int N, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[N]) {
#pragma unroll
    for (int s = N / 2; s >= 1; s >>= 1) {
#pragma unroll
        for (int b = 0; b < N; b += 2 * s) {
#pragma unroll
            for (int j = 0; j < s; ++j) {
                const float2 a = v[b + j], c = v[b + j + s];
                v[b + j] = cadd(a, c);
                v[b + j + s] = twiddle<SIGN>(csub(a, c), j * (N / (2 * s)), N);
            }
        }
    }
    // decimation in frequency leaves X[k] at the bit-reversed position of k
    float2 o[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        int r = 0;
#pragma unroll
        for (int bit = 1, rb = N / 2; bit < N; bit <<= 1, rb >>= 1)
            if (i & bit) r |= rb;
        o[r] = v[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = o[i];
}

// Length-L transform by the 8 threads of a group (t = thread in group):
// v[j] = x[t + 8j] on entry, v[m] = X[t + 8m] on return.  tw[8 k1 + t] =
// exp(-2 pi i t k1 / L).  Every thread of the warp must call it together.
template <int E, int SIGN>
__device__ __forceinline__ void group_fft(float2 (&v)[E], int t, float2* sc, const float2* tw) {
    dft<E, SIGN>(v);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) {
        float2 w = tw[8 * k1 + t];
        if (SIGN > 0) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) sc[k1 * kScP + t] = v[k1];
    __syncwarp();
    float2 w8[E / 8][8];
#pragma unroll
    for (int a = 0; a < E / 8; ++a)
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) w8[a][tt] = sc[(t + 8 * a) * kScP + tt];
    __syncwarp();
#pragma unroll
    for (int a = 0; a < E / 8; ++a) {
        dft<8, SIGN>(w8[a]);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) v[a + (E / 8) * k2] = w8[a][k2];
    }
}

// The second half of group_fft: after the twiddles, the 8 x 8 transposes
// through the group's scratch and the 8-point DFTs over t.
template <int E, int SIGN>
__device__ __forceinline__ void group_fft_tail(float2 (&v)[E], int t, float2* sc) {
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) sc[k1 * kScP + t] = v[k1];
    __syncwarp();
    float2 w8[E / 8][8];
#pragma unroll
    for (int a = 0; a < E / 8; ++a)
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) w8[a][tt] = sc[(t + 8 * a) * kScP + tt];
    __syncwarp();
#pragma unroll
    for (int a = 0; a < E / 8; ++a) {
        dft<8, SIGN>(w8[a]);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) v[a + (E / 8) * k2] = w8[a][k2];
    }
}

// Two independent length-L transforms by one group (the column pair): the
// E-point DFTs interleave and each twiddle feeds both; the transposes run
// one array after the other (every input of an array is in the scratch
// before any of its outputs is written back).
template <int E, int SIGN>
__device__ __forceinline__ void group_fft2(float2 (&va)[E], float2 (&vb)[E], int t, float2* sc, const float2* tw) {
    dft<E, SIGN>(va);
    dft<E, SIGN>(vb);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) {
        float2 w = tw[8 * k1 + t];
        if (SIGN > 0) w.y = -w.y;
        va[k1] = cmul(va[k1], w);
        vb[k1] = cmul(vb[k1], w);
    }
    group_fft_tail<E, SIGN>(va, t, sc);
    group_fft_tail<E, SIGN>(vb, t, sc);
}

// X conj(Y) from a = Z[k] and b = conj(Z[-k]) of z = x + i y
__device__ __forceinline__ float2 cross_spectrum(float2 a, float2 b) {
    const float2 s = cadd(a, b), d = csub(a, b);
    return make_float2(0.25f * fmaf(s.x, d.y, -s.y * d.x), 0.25f * fmaf(s.x, d.x, s.y * d.y));
}

// Rows of one item's window (or template) in a cube: `p` points at channel
// 0, row 0, column 0 of the region; row(c, y) is channel c, region row y.
// F32 cubes: planar, `pitch` elements per row, `plane` per channel.  BF16
// cubes: the row-major chunks (chunk c / 6, lane c % 6 of a pixel's 8),
// widened to FP32 as read; `pitch` = 8 W elements per row, `plane` = 8 H W
// per chunk.
struct CubeF32 {
    const float* p;
    size_t plane;
    unsigned pitch;
    __device__ __forceinline__ const float* row(int c, int y) const {
        return p + (size_t)c * plane + (size_t)y * pitch;
    }
    __device__ __forceinline__ static float at(const float* r, int x) { return r[x]; }
};
struct CubeBF16 {
    const __nv_bfloat16* p;
    size_t plane;
    unsigned pitch;
    __device__ __forceinline__ const __nv_bfloat16* row(int c, int y) const {
        const int g = c / 6;
        return p + (size_t)g * plane + (size_t)y * pitch + (c - 6 * g);
    }
    __device__ __forceinline__ static float at(const __nv_bfloat16* r, int x) { return __bfloat162float(r[8 * x]); }
};

// Items: the points of `one` (items == nullptr) or (job, point) pairs of a
// batch; with a queue the CTAs take items from an atomic counter (points of
// uneven cost balance across the SMs), else item k goes to CTA k mod grid.
// BF: the jobs' cubes are BF16 (12 channels), read from the row-major layout.
template <int L, bool BF>
__global__ void __launch_bounds__(FftShape<L>::T, 1)
    k_corr_fft(const __grid_constant__ MatchJob one, const MatchJob* __restrict__ jobs,
               const int2* __restrict__ items, int n_items, int* __restrict__ queue) {
    using Sh = FftShape<L>;
    constexpr int E = Sh::E, ZP = Sh::ZP, kFftGroups = Sh::G, kFftThreads = Sh::T;
    extern __shared__ __align__(16) float2 fsm[];
    __shared__ int s_item;
    typedef typename std::conditional<BF, CubeBF16, CubeF32>::type SrcT;
    __shared__ SrcT s_src[2];  // the item's window and template rows
    __shared__ float* s_out;
    __shared__ int s_par[4];   // the item's m, m + 2R, 2R + 1, channels
    __shared__ float s_tmean;  // the item's template mean
    float2* Z = fsm;                                       // L x ZP
    float2* scr = Z + (size_t)L * ZP;                      // kFftGroups x SG
    float2* tw = scr + (size_t)kFftGroups * Sh::SG;        // 8E twiddles W_L^{t k1} at 8 k1 + t
    float2* P64 = tw + 8 * E;                              // Nyquist column of the channel sum

    const int tid = threadIdx.x;
    const int grp = tid >> 3, t = tid & 7;
    const int lane = tid & 31, gbase = lane & ~7;
    float2* sc = scr + grp * Sh::SG;
    const float inv_area = 1.f / ((float)L * (float)L);
    // the row a group transforms in the row passes: within a block of 8 rows
    // per warp pair, the two groups of a half-warp take rows 4 apart, so their
    // 64-bit accesses to Z rows (pitch ZP = L + 2: 4 banks apart per row)
    // fall on disjoint banks
    const int yrow = 8 * (grp >> 3) + 2 * ((grp >> 2) & 1) + ((grp >> 1) & 1) + 4 * (grp & 1);
    // partner of row t + 8m is row -(t + 8m): thread (8 - t) mod 8, index
    // (E - m) mod E for t = 0, E - 1 - m otherwise
    const int tpart = gbase + ((8 - t) & 7);

    for (int p = tid; p < 8 * E; p += kFftThreads) {
        double s, c;
        sincospi(-2.0 * ((p & 7) * (p >> 3)) / L, &s, &c);
        tw[p] = make_float2((float)c, (float)s);
    }
    for (int i = tid; i < L * ZP; i += kFftThreads) Z[i] = make_float2(0.f, 0.f);
    __syncthreads();
    // rows of Z at or past zhi are zero; an item's row passes write the rows
    // below its m + 2R, every other row it reads must be zero
    int zhi = 0;

    for (int next = blockIdx.x;;) {
        int kk;
        if (queue) {
            if (tid == 0) s_item = atomicAdd(queue, 1);
            __syncthreads();
            kk = s_item;
            __syncthreads();  // read by all before thread 0 takes the next one
        } else {
            kk = next;
            next += gridDim.x;
        }
        if (kk >= n_items) break;
        int k;
        const MatchJob& J = item_job(one, jobs, items, kk, &k);
        const PointStat st = J.stats[k];
        if (st.status != SFOC_PT_OK) continue;  // uniform across the CTA
        typedef typename std::conditional<BF, CubeBF16, CubeF32>::type Src;
        const int m = J.m, R = J.R, z = J.z;
        const int P1 = 2 * R + 1, Lw = m + 2 * R;
        const int h = template_half(m);
        if (zhi > Lw) {  // rows [Lw, zhi) of an earlier, taller window
            for (int i = tid; i < (zhi - Lw) * ZP; i += kFftThreads) Z[(size_t)Lw * ZP + i] = make_float2(0.f, 0.f);
            __syncthreads();
        }
        zhi = Lw;
        // the item's window and template rows and its output, in shared memory:
        // read again after each barrier, they hold no registers across the
        // column passes (whose transforms set the kernel's register peak)
        if (tid == 0) {
            const int ty0 = J.pts[2 * k + 1] - h, tx0 = J.pts[2 * k] - h;
            const int wy0 = ty0 - R, wx0 = tx0 - R;
            if constexpr (BF) {
                s_src[0] = CubeBF16{J.rrm + ((size_t)wy0 * J.Wr + wx0) * 8, (size_t)8 * J.Hr * J.Wr, 8u * (unsigned)J.Wr};
                s_src[1] = CubeBF16{J.srm + ((size_t)ty0 * J.Ws + tx0) * 8, (size_t)8 * J.Hs * J.Ws, 8u * (unsigned)J.Ws};
            } else {
                s_src[0] = CubeF32{J.rf32 + (size_t)wy0 * J.rpitch + wx0, J.rplane, (unsigned)J.rpitch};
                s_src[1] = CubeF32{J.sf32 + (size_t)ty0 * J.spitch + tx0, J.splane, (unsigned)J.spitch};
            }
            s_out = J.maps + (size_t)k * P1 * P1;
            s_par[0] = m;
            s_par[1] = Lw;
            s_par[2] = P1;
            s_par[3] = z;
            s_tmean = st.tmean;
        }
        __syncthreads();

        float2 acc[E];  // channel sum of X conj(Y) on column pr of this group's pair
#pragma unroll
        for (int j = 0; j < E; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int i = tid; i < L; i += kFftThreads) P64[i] = make_float2(0.f, 0.f);

        for (int c = 0; c < s_par[3]; ++c) {
            const Src Sc = s_src[0], Tc = s_src[1];
            const int m = s_par[0], Lw = s_par[1];
            const float tmean = s_tmean;
            // ---- rows: z = S + i (T - mean), zero outside the window / template
            for (int y0 = 0; y0 < Lw; y0 += kFftGroups) {
                const int y = y0 + yrow;
                const bool rs = y < Lw, rt = y < m;
                const auto srow = Sc.row(c, rs ? y : 0);
                const auto trow = Tc.row(c, rt ? y : 0);
                float2 v[E];
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int x = t + 8 * j;
                    v[j].x = (rs && x < Lw) ? Src::at(srow, x) : 0.f;
                    v[j].y = (rt && x < m) ? Src::at(trow, x) - tmean : 0.f;
                }
                group_fft<E, -1>(v, t, sc, tw);
                if (rs) {
#pragma unroll
                    for (int j = 0; j < E; ++j) Z[(size_t)y * ZP + t + 8 * j] = v[j];
                }
            }
            __syncthreads();
            // ---- columns in conjugate pairs, cross spectrum into the sums
            {
                const int pr = grp;  // pair pr: columns (pr, L - pr); pair 0: (0, L/2)
                const int c1 = pr, c2 = pr == 0 ? L / 2 : L - pr;
                float2 a[E], b[E];
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    a[j] = Z[(size_t)(t + 8 * j) * ZP + c1];
                    b[j] = Z[(size_t)(t + 8 * j) * ZP + c2];
                }
                group_fft2<E, -1>(a, b, t, sc, tw);
                // Z[-k] of column c1 lives in column c2 (in column c1 itself for
                // pair 0).  Row -(t + 8j) is held by thread (8 - t) mod 8 at index
                // E - 1 - j; for t = 0 by the thread itself at index (E - j) mod E.
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const float2 sb = make_float2(__shfl_sync(0xffffffffu, b[E - 1 - j].x, tpart),
                                                  __shfl_sync(0xffffffffu, b[E - 1 - j].y, tpart));
                    const float2 pb = t == 0 ? b[(E - j) & (E - 1)] : sb;
                    if (pr != 0) acc[j] = cadd(acc[j], cross_spectrum(a[j], make_float2(pb.x, -pb.y)));
                }
                if (pr == 0) {  // lanes 0-7 of warp 0: columns 0 and L/2 each pair with themselves
#pragma unroll
                    for (int j = 0; j < E; ++j) {
                        const float2 sa = make_float2(__shfl_sync(0xffu, a[E - 1 - j].x, tpart),
                                                      __shfl_sync(0xffu, a[E - 1 - j].y, tpart));
                        const float2 sb = make_float2(__shfl_sync(0xffu, b[E - 1 - j].x, tpart),
                                                      __shfl_sync(0xffu, b[E - 1 - j].y, tpart));
                        const float2 pa = t == 0 ? a[(E - j) & (E - 1)] : sa;
                        const float2 pb = t == 0 ? b[(E - j) & (E - 1)] : sb;
                        acc[j] = cadd(acc[j], cross_spectrum(a[j], make_float2(pa.x, -pa.y)));
                        P64[t + 8 * j] = cadd(P64[t + 8 * j], cross_spectrum(b[j], make_float2(pb.x, -pb.y)));
                    }
                }
            }
            __syncthreads();
        }

        const int P1i = s_par[2];
        // ---- inverse along the columns kx in [0, L/2]: rows y < 2R + 1 of Q in Z
        {
            const int pr = grp;
            group_fft<E, 1>(acc, t, sc, tw);
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (t + 8 * j < P1i) Z[(size_t)(t + 8 * j) * ZP + pr] = acc[j];
        }
        {
            float2 v[E];
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = P64[t + 8 * j];
            group_fft<E, 1>(v, t, sc, tw);  // every group computes it (uniform); group 0 stores it
            if (grp == 0) {
#pragma unroll
                for (int j = 0; j < E; ++j)
                    if (t + 8 * j < P1i) Z[(size_t)(t + 8 * j) * ZP + L / 2] = v[j];
            }
        }
        __syncthreads();
        // ---- inverse along the rows (Hermitian extension), real part
        float* out = s_out;
        for (int y0 = 0; y0 < P1i; y0 += kFftGroups) {
            const int y = y0 + yrow;
            const int yy = y < P1i ? y : 0;
            float2 v[E];
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int kx = t + 8 * j;
                const float2 q = Z[(size_t)yy * ZP + (kx <= L / 2 ? kx : L - kx)];
                v[j] = kx <= L / 2 ? q : make_float2(q.x, -q.y);
            }
            group_fft<E, 1>(v, t, sc, tw);
            if (y < P1i) {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int x = t + 8 * j;
                    if (x < P1i) out[(size_t)y * P1i + x] = v[j].x * inv_area;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

bool corr_fft_supported(int m, int R) { return m + 2 * R <= 128; }

int corr_fft_side(int m, int R) { return m + 2 * R <= 64 ? 64 : 128; }

// L: the transform side (64 or 128, at least the largest m + 2R of the items)
cudaError_t launch_corr_fft(const MatchJob& one, const ItemSet& is, int L, bool bf16, cudaStream_t st) {
    const int n = is.items ? is.n : one.n;
    if (n <= 0) return cudaSuccess;
    const int lw = is.items ? is.max_lw : one.m + 2 * one.R;
    if ((L != 64 && L != 128) || lw > L) return cudaErrorNotSupported;
    if (!is.items && (bf16 ? (one.rrm == nullptr || one.srm == nullptr || one.z != 12)
                           : (one.rf32 == nullptr || one.sf32 == nullptr)))
        return cudaErrorNotSupported;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
#define SFOC_FFT_LAUNCH(LV, BV)                                                                                   \
    {                                                                                                             \
        const int smem = (int)FftShape<LV>::smem;                                                                 \
        e = cudaFuncSetAttribute(k_corr_fft<LV, BV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);         \
        if (e != cudaSuccess) return e;                                                                           \
        const int grid = n < sms ? n : sms;                                                                       \
        k_corr_fft<LV, BV><<<grid, FftShape<LV>::T, smem, st>>>(one, is.jobs, is.items, n, is.queue);             \
    }
    if (L == 64) {
        if (bf16) SFOC_FFT_LAUNCH(64, true) else SFOC_FFT_LAUNCH(64, false)
    } else {
        if (bf16) SFOC_FFT_LAUNCH(128, true) else SFOC_FFT_LAUNCH(128, false)
    }
#undef SFOC_FFT_LAUNCH
    return cudaGetLastError();
}

}  // namespace sfoc
