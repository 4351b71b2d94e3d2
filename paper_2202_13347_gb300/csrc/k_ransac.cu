// Outlier rejection over the control points (Sec. 3.2.3 of arXiv
// 2202.13347): RANSAC with a projective (or affine) model, FP64.
//
//   x' = (h0 x + h1 y + h2) / (h6 x + h7 y + 1),  y' = (h3 x + h4 y + h5) / (h6 x + h7 y + 1)
//   (affine: h6 = h7 = 0).
// Coordinates are normalised first (the valid points' centroid to the
// origin, their mean distance from it to sqrt(2)), every model is solved
// there and mapped back to pixels.  A hypothesis is the exact solution on a
// minimal sample (4 points; affine 3) whose indices the caller supplies (the
// random draws); a singular sample (pivot below 1e-12) scores -1.  The score
// is the number of valid points within `threshold` pixels of the model's
// image; the best score wins, ties to the lower index.  The winner's inliers
// are refitted by least squares (two equations per point, normal equations)
// and recounted, `refits` times.
//
//   k_ransac_frames  one block: the two normalising frames (fixed-order sums)
//   k_ransac_hyp     one warp per 8 hypotheses: each of 8 lanes solves one,
//                    then the warp counts inliers for each model in turn
//   k_ransac_final   one block: argmax, refits (normal equations reduced in a
//                    fixed order: warp shuffles, then the warps in order)
#include <math.h>

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kRsThreads = 256;
constexpr int kHpw = 8;  // hypotheses per warp (one warp per CTA)

struct Frames {
    double s[3];  // source: scale, cx, cy  (p -> s (p - c))
    double d[3];  // destination
    int n_valid;
};

__device__ __forceinline__ bool is_valid(const uint8_t* valid, int i) { return !valid || valid[i] != 0; }

// sum over the block of v (fixed order: strided per thread, shuffles, warps in order)
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRsThreads) k_ransac_frames(const double* __restrict__ src,
                                                              const double* __restrict__ dst,
                                                              const uint8_t* __restrict__ valid, int n,
                                                              Frames* __restrict__ out) {
    __shared__ double sh[kRsThreads / 32];
    double c = 0.0, sx = 0.0, sy = 0.0, dx = 0.0, dy = 0.0;
    for (int i = threadIdx.x; i < n; i += kRsThreads)
        if (is_valid(valid, i)) {
            c += 1.0;
            sx += src[2 * i];
            sy += src[2 * i + 1];
            dx += dst[2 * i];
            dy += dst[2 * i + 1];
        }
    const double cnt = block_sum(c, sh);
    const double mx = cnt > 0 ? block_sum(sx, sh) / cnt : 0.0, my = cnt > 0 ? block_sum(sy, sh) / cnt : 0.0;
    const double nx = cnt > 0 ? block_sum(dx, sh) / cnt : 0.0, ny = cnt > 0 ? block_sum(dy, sh) / cnt : 0.0;
    double ds = 0.0, dd = 0.0;
    for (int i = threadIdx.x; i < n; i += kRsThreads)
        if (is_valid(valid, i)) {
            ds += hypot(src[2 * i] - mx, src[2 * i + 1] - my);
            dd += hypot(dst[2 * i] - nx, dst[2 * i + 1] - ny);
        }
    const double ms = cnt > 0 ? block_sum(ds, sh) / cnt : 0.0, md = cnt > 0 ? block_sum(dd, sh) / cnt : 0.0;
    if (threadIdx.x == 0) {
        out->s[0] = ms > 0.0 ? sqrt(2.0) / ms : 1.0;
        out->s[1] = mx;
        out->s[2] = my;
        out->d[0] = md > 0.0 ? sqrt(2.0) / md : 1.0;
        out->d[1] = nx;
        out->d[2] = ny;
        out->n_valid = (int)cnt;
    }
}

// the two equations of one correspondence (normalised coordinates)
__device__ __forceinline__ void eq_rows(bool proj, double x, double y, double xp, double yp, double* r1, double* r2) {
    r1[0] = x; r1[1] = y; r1[2] = 1.0; r1[3] = 0.0; r1[4] = 0.0; r1[5] = 0.0;
    r2[0] = 0.0; r2[1] = 0.0; r2[2] = 0.0; r2[3] = x; r2[4] = y; r2[5] = 1.0;
    r1[6] = proj ? -x * xp : 0.0; r1[7] = proj ? -y * xp : 0.0;
    r2[6] = proj ? -x * yp : 0.0; r2[7] = proj ? -y * yp : 0.0;
}

// Gaussian elimination with partial pivoting, n <= 8 (A row-major, b: rhs);
// false when a pivot falls below 1e-12
__device__ bool solve_small(double* A, double* b, int n, double* x) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * 8 + c]) > fabs(A[p * 8 + c])) p = r;
        if (fabs(A[p * 8 + c]) < 1e-12) return false;
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                const double t = A[c * 8 + k];
                A[c * 8 + k] = A[p * 8 + k];
                A[p * 8 + k] = t;
            }
            const double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * 8 + c] / A[c * 8 + c];
            for (int k = c; k < n; ++k) A[r * 8 + k] -= f * A[c * 8 + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * 8 + k] * x[k];
        x[r] = s / A[r * 8 + r];
    }
    return true;
}

// pixel model from the normalised solution: H = Dinv Hn S, scaled to H[8] = 1
__device__ bool to_pixels(const double* h, bool proj, const Frames& F, double* H) {
    const double Hn[9] = {h[0], h[1], h[2], h[3], h[4], h[5], proj ? h[6] : 0.0, proj ? h[7] : 0.0, 1.0};
    const double S[9] = {F.s[0], 0.0, -F.s[0] * F.s[1], 0.0, F.s[0], -F.s[0] * F.s[2], 0.0, 0.0, 1.0};
    const double Di[9] = {1.0 / F.d[0], 0.0, F.d[1], 0.0, 1.0 / F.d[0], F.d[2], 0.0, 0.0, 1.0};
    double M[9], R[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Hn[i * 3 + k] * S[k * 3 + j];
            M[i * 3 + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Di[i * 3 + k] * M[k * 3 + j];
            R[i * 3 + j] = s;
        }
    if (fabs(R[8]) < 1e-300) return false;
    for (int i = 0; i < 9; ++i) H[i] = R[i] / R[8];
    return true;
}

__device__ __forceinline__ bool inlier(const double* H, const double* src, const double* dst, int i, double t2) {
    const double x = src[2 * i], y = src[2 * i + 1];
    const double w = H[6] * x + H[7] * y + H[8];
    if (w == 0.0) return false;
    const double ex = (H[0] * x + H[1] * y + H[2]) / w - dst[2 * i];
    const double ey = (H[3] * x + H[4] * y + H[5]) / w - dst[2 * i + 1];
    return ex * ex + ey * ey <= t2;
}

// One warp (CTA) per kHpw hypotheses: lane l < kHpw solves hypothesis
// h0 + l, then the warp counts inliers for each of the models in turn.
__global__ void __launch_bounds__(32)
    k_ransac_hyp(const double* __restrict__ src, const double* __restrict__ dst, const uint8_t* __restrict__ valid,
                 int n, int proj, const int32_t* __restrict__ samples, int n_hyp, double t2,
                 const Frames* __restrict__ frames, int32_t* __restrict__ scores, double* __restrict__ models) {
    __shared__ double sH[kHpw][9];
    __shared__ int sok[kHpw];
    const int lane = threadIdx.x & 31;
    const int h0 = blockIdx.x * kHpw;
    const bool pj = proj != 0;
    const int k = pj ? 4 : 3, nu = pj ? 8 : 6;
    if (lane < kHpw) {
        const int h = h0 + lane;
        bool ok = false;
        if (h < n_hyp) {
            const Frames F = *frames;
            double A[64], b[8], x[8], r1[8], r2[8];
            bool in_range = true;
            for (int j = 0; j < k; ++j) {
                const int i0 = samples[(size_t)h * k + j];
                in_range = in_range && i0 >= 0 && i0 < n;
                const int i = (i0 >= 0 && i0 < n) ? i0 : 0;  // an index outside [0, n) voids the hypothesis
                const double sx = F.s[0] * (src[2 * i] - F.s[1]), sy = F.s[0] * (src[2 * i + 1] - F.s[2]);
                const double dx = F.d[0] * (dst[2 * i] - F.d[1]), dy = F.d[0] * (dst[2 * i + 1] - F.d[2]);
                eq_rows(pj, sx, sy, dx, dy, r1, r2);
                for (int c = 0; c < nu; ++c) {
                    A[(2 * j) * 8 + c] = r1[c];
                    A[(2 * j + 1) * 8 + c] = r2[c];
                }
                b[2 * j] = dx;
                b[2 * j + 1] = dy;
            }
            ok = in_range && solve_small(A, b, nu, x) && to_pixels(x, pj, F, sH[lane]);
        }
        sok[lane] = ok ? 1 : 0;
    }
    __syncwarp();
    const int nh = n_hyp - h0 < kHpw ? n_hyp - h0 : kHpw;
    for (int q = 0; q < nh; ++q) {
        int c = 0;
        if (sok[q]) {
            double H[9];
#pragma unroll
            for (int r = 0; r < 9; ++r) H[r] = sH[q][r];
            for (int i = lane; i < n; i += 32) c += (is_valid(valid, i) && inlier(H, src, dst, i, t2)) ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) scores[h0 + q] = sok[q] ? c : -1;
    }
    if (lane < nh)
        for (int r = 0; r < 9; ++r) models[(size_t)(h0 + lane) * 9 + r] = sok[lane] ? sH[lane][r] : 0.0;
}

constexpr int kNE = 44;  // unique entries of the 8 x 8 normal matrix (36) and the right side (8)

__global__ void __launch_bounds__(kRsThreads)
    k_ransac_final(const double* __restrict__ src, const double* __restrict__ dst, const uint8_t* __restrict__ valid,
                   int n, int proj, int n_hyp, double t2, int refits, const Frames* __restrict__ frames,
                   const int32_t* __restrict__ scores, const double* __restrict__ models, double* __restrict__ H_out,
                   uint8_t* __restrict__ mask, int32_t* __restrict__ info) {
    __shared__ int s_best, s_score[kRsThreads], s_idx[kRsThreads];
    __shared__ double sH[9];
    __shared__ double s_part[kRsThreads / 32][kNE];
    __shared__ int s_cnt[kRsThreads / 32];
    __shared__ int s_ok;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const bool pj = proj != 0;
    const int k = pj ? 4 : 3, nu = pj ? 8 : 6;
    // argmax: highest score, then lowest index
    int bs = -2, bi = -1;
    for (int h = tid; h < n_hyp; h += kRsThreads)
        if (scores[h] > bs) {
            bs = scores[h];
            bi = h;
        }
    s_score[tid] = bs;
    s_idx[tid] = bi;
    __syncthreads();
    if (tid == 0) {
        int b = -1, v = -1;
        for (int t = 0; t < kRsThreads; ++t)
            if (s_idx[t] >= 0 && (s_score[t] > v || (s_score[t] == v && s_idx[t] < b))) {
                v = s_score[t];
                b = s_idx[t];
            }
        s_best = v >= 0 ? b : -1;  // every hypothesis singular: no winner
        for (int q = 0; q < 9; ++q) sH[q] = s_best >= 0 ? models[(size_t)s_best * 9 + q] : ((q % 4 == 0) ? 1.0 : 0.0);
    }
    __syncthreads();
    const int best = s_best;
    auto recount = [&]() -> int {
        double H[9];
        for (int q = 0; q < 9; ++q) H[q] = sH[q];
        int c = 0;
        for (int i = tid; i < n; i += kRsThreads) {
            const bool in = best >= 0 && is_valid(valid, i) && inlier(H, src, dst, i, t2);
            mask[i] = in ? 1 : 0;
            c += in ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        __syncthreads();
        if (lane == 0) s_cnt[w] = c;
        __syncthreads();
        int t = 0;
        for (int q = 0; q < kRsThreads / 32; ++q) t += s_cnt[q];
        __syncthreads();
        return t;
    };
    int cnt = recount();
    const Frames F = *frames;
    for (int it = 0; it < refits && best >= 0 && cnt >= k; ++it) {
        // normal equations over this thread's inliers (the mask it wrote itself)
        double e[kNE];
#pragma unroll
        for (int q = 0; q < kNE; ++q) e[q] = 0.0;
        for (int i = tid; i < n; i += kRsThreads) {
            if (!mask[i]) continue;
            double r1[8], r2[8];
            const double sx = F.s[0] * (src[2 * i] - F.s[1]), sy = F.s[0] * (src[2 * i + 1] - F.s[2]);
            const double dx = F.d[0] * (dst[2 * i] - F.d[1]), dy = F.d[0] * (dst[2 * i + 1] - F.d[2]);
            eq_rows(pj, sx, sy, dx, dy, r1, r2);
            int q = 0;
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = a; c < 8; ++c) e[q++] += r1[a] * r1[c] + r2[a] * r2[c];
#pragma unroll
            for (int a = 0; a < 8; ++a) e[q++] += r1[a] * dx + r2[a] * dy;
        }
#pragma unroll
        for (int q = 0; q < kNE; ++q) {
            double v = e[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) s_part[w][q] = v;
        }
        __syncthreads();
        if (tid == 0) {
            double tot[kNE];
            for (int q = 0; q < kNE; ++q) {
                double v = 0.0;
                for (int ww = 0; ww < kRsThreads / 32; ++ww) v += s_part[ww][q];
                tot[q] = v;
            }
            double M[64], v[8], x[8], Hr[9];
            int q = 0;
            for (int a = 0; a < 8; ++a)
                for (int c = a; c < 8; ++c) {
                    M[a * 8 + c] = tot[q];
                    M[c * 8 + a] = tot[q];
                    ++q;
                }
            for (int a = 0; a < 8; ++a) v[a] = tot[q++];
            s_ok = solve_small(M, v, nu, x) && to_pixels(x, pj, F, Hr);
            if (s_ok)
                for (int r = 0; r < 9; ++r) sH[r] = Hr[r];
        }
        __syncthreads();
        if (!s_ok) break;
        cnt = recount();
    }
    if (tid == 0) {
        for (int q = 0; q < 9; ++q) H_out[q] = sH[q];
        info[0] = best;
        info[1] = best >= 0 ? cnt : 0;
    }
}

// Rectification (Sec. 3.2.3): out(x, y) = bilinear sample of the sensed
// image at H^-1 (x, y); outside [0, W-1] x [0, H-1] the fill value.  The
// mapping is FP64 (coordinates of 10^4 px keep their sub-pixel part), the
// blend FP32.  Each CTA inverts H (the adjugate scaled by its last entry);
// a singular model gives an all-fill image.
__global__ void k_rectify(const float* __restrict__ img, int H, int W, size_t pitch, const double* __restrict__ Hm,
                          float fill, int out_h, int out_w, float* __restrict__ out) {
    __shared__ double s_inv[9];
    __shared__ int s_ok;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const double a = Hm[0], b = Hm[1], c = Hm[2], d = Hm[3], e = Hm[4], f = Hm[5], g = Hm[6], h = Hm[7],
                     i = Hm[8];
        double inv[9] = {e * i - f * h, c * h - b * i, b * f - c * e, f * g - d * i, a * i - c * g,
                         c * d - a * f, d * h - e * g, b * g - a * h, a * e - b * d};
        const double det = a * inv[0] + b * inv[3] + c * inv[6];
        s_ok = det != 0.0 && inv[8] != 0.0;
        for (int k = 0; k < 9; ++k) s_inv[k] = s_ok ? inv[k] / inv[8] : 0.0;
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= out_w || y >= out_h) return;
    float v = fill;
    const double w = s_inv[6] * x + s_inv[7] * y + s_inv[8];
    if (s_ok && w != 0.0) {
        const double rw = 1.0 / w;  // one division per pixel (FP64 is slow on this part)
        const double u = (s_inv[0] * x + s_inv[1] * y + s_inv[2]) * rw;
        const double t = (s_inv[3] * x + s_inv[4] * y + s_inv[5]) * rw;
        if (u >= 0.0 && t >= 0.0 && u <= W - 1 && t <= H - 1) {
            int u0 = (int)floor(u), t0 = (int)floor(t);
            u0 = min(u0, max(W - 2, 0));
            t0 = min(t0, max(H - 2, 0));
            const int u1 = min(u0 + 1, W - 1), t1 = min(t0 + 1, H - 1);
            const float fu = (float)(u - u0), ft = (float)(t - t0);
            const float p00 = img[(size_t)t0 * pitch + u0], p01 = img[(size_t)t0 * pitch + u1];
            const float p10 = img[(size_t)t1 * pitch + u0], p11 = img[(size_t)t1 * pitch + u1];
            const float r0 = fmaf(fu, p01 - p00, p00), r1 = fmaf(fu, p11 - p10, p10);
            v = fmaf(ft, r1 - r0, r0);
        }
    }
    out[(size_t)y * out_w + x] = v;
}

__global__ void k_results_to_points(const int32_t* __restrict__ pts, const fastncc_result* __restrict__ res, int n,
                                    double* __restrict__ src, double* __restrict__ dst, uint8_t* __restrict__ valid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const fastncc_result r = res[i];
    const double x = pts[2 * i], y = pts[2 * i + 1];
    src[2 * i] = x;
    src[2 * i + 1] = y;
    dst[2 * i] = x + (double)r.sub_dx;  // the refined offset (dx plus its parabola correction)
    dst[2 * i + 1] = y + (double)r.sub_dy;
    valid[i] = r.status == SFOC_PT_OK ? 1 : 0;
}

}  // namespace

size_t ransac_workspace_bytes(int n_hyp) {
    return (sizeof(Frames) + 255) / 256 * 256 + (sizeof(int32_t) * (size_t)n_hyp + 255) / 256 * 256 +
           sizeof(double) * 9 * (size_t)n_hyp;
}

cudaError_t launch_ransac(const double* src, const double* dst, const uint8_t* valid, int n, int proj,
                          const int32_t* samples, int n_hyp, double threshold, int refits, double* H_out,
                          uint8_t* mask, int32_t* info, int32_t* scores_out, void* ws, cudaStream_t st, int* launches) {
    char* p = static_cast<char*>(ws);
    Frames* frames = reinterpret_cast<Frames*>(p);
    p += (sizeof(Frames) + 255) / 256 * 256;
    int32_t* scores = scores_out ? scores_out : reinterpret_cast<int32_t*>(p);
    p += (sizeof(int32_t) * (size_t)n_hyp + 255) / 256 * 256;
    double* models = reinterpret_cast<double*>(p);
    const double t2 = threshold * threshold;
    k_ransac_frames<<<1, kRsThreads, 0, st>>>(src, dst, valid, n, frames);
    int nl = 1;
    if (n_hyp > 0) {
        k_ransac_hyp<<<(n_hyp + kHpw - 1) / kHpw, 32, 0, st>>>(src, dst, valid, n, proj, samples, n_hyp, t2, frames,
                                                                scores, models);
        ++nl;
    }
    k_ransac_final<<<1, kRsThreads, 0, st>>>(src, dst, valid, n, proj, n_hyp, t2, refits, frames, scores, models,
                                             H_out, mask, info);
    ++nl;
    if (launches) *launches = nl;
    return cudaGetLastError();
}

cudaError_t launch_rectify(const float* img, int H, int W, size_t pitch, const double* Hm, float fill, int out_h,
                           int out_w, float* out, cudaStream_t st) {
    dim3 blk(32, 8), grid((unsigned)((out_w + 31) / 32), (unsigned)((out_h + 7) / 8));
    k_rectify<<<grid, blk, 0, st>>>(img, H, W, pitch, Hm, fill, out_h, out_w, out);
    return cudaGetLastError();
}

cudaError_t launch_results_to_points(const int32_t* pts, const fastncc_result* res, int n, double* src, double* dst,
                                     uint8_t* valid, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_results_to_points<<<(n + 255) / 256, 256, 0, st>>>(pts, res, n, src, dst, valid);
    return cudaGetLastError();
}

}  // namespace sfoc
