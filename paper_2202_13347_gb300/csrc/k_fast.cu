// Block-based FAST interest points (Sec. 3.1.1 of arXiv 2202.13347): the
// FAST operator per block of a partition of the image, so that the points
// spread evenly.
//
// Segment test FAST-9 on the 16 pixels of the radius-3 circle; the score of
// a pixel is the largest threshold for which it is still a corner (the
// largest over the 16 arcs of 9 contiguous circle pixels of the arc's
// smallest difference to the centre, brighter or darker), taken in FP32 as
// the image is stored; it is a corner when the score exceeds t.  Pixels
// closer than 3 to the border score 0.  A corner survives 3 x 3
// non-maximum suppression when its score is at least every neighbour's and
// above those before it in raster order.  Each block (grid_y x grid_x
// partition, rows [by H / grid_y, (by + 1) H / grid_y), columns likewise)
// keeps its strongest surviving corner at least `margin` from the border,
// ties to the smaller y, then x.
//
// One CTA per block, walking the block in sub-tiles of up to 64 x 64
// outputs: the image with a 4-pixel halo is staged in shared memory, the
// scores of the sub-tile and a 1-pixel ring (for the suppression) are
// computed there, then each thread keeps its best candidate and the CTA
// reduces.
#include "internal.h"

namespace sfoc {

namespace {

constexpr int kFastThreads = 256;
constexpr int kSub = 64;             // outputs per sub-tile side
constexpr int kIn = kSub + 8;        // staged image side (4-pixel halo)
constexpr int kSc = kSub + 2;        // scores side (1-pixel ring)

__constant__ int c_cdx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
__constant__ int c_cdy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

// candidate order: higher score, then smaller y, then smaller x
__device__ __forceinline__ bool better(float s, int y, int x, float bs, int by, int bx) {
    if (bx < 0) return x >= 0;
    if (x < 0) return false;
    if (s != bs) return s > bs;
    return y < by || (y == by && x < bx);
}

__global__ void __launch_bounds__(kFastThreads)
    k_fast_blocks(const float* __restrict__ img, int H, int W, size_t pitch, float t, int grid_y, int grid_x,
                  int margin, int32_t* __restrict__ points, float* __restrict__ scores) {
    __shared__ float s_img[kIn][kIn + 1];
    __shared__ float s_sc[kSc][kSc + 1];
    __shared__ float r_s[kFastThreads];
    __shared__ int r_y[kFastThreads], r_x[kFastThreads];
    const int bx = blockIdx.x, by = blockIdx.y;
    const int y0 = (int)((long long)by * H / grid_y), y1 = (int)((long long)(by + 1) * H / grid_y);
    const int x0 = (int)((long long)bx * W / grid_x), x1 = (int)((long long)(bx + 1) * W / grid_x);
    float best_s = 0.f;
    int best_y = -1, best_x = -1;
    for (int sy0 = y0; sy0 < y1; sy0 += kSub)
        for (int sx0 = x0; sx0 < x1; sx0 += kSub) {
            const int sy1 = min(sy0 + kSub, y1), sx1 = min(sx0 + kSub, x1);
            __syncthreads();  // the previous sub-tile's readers are done
            for (int i = threadIdx.x; i < kIn * kIn; i += kFastThreads) {
                const int ly = i / kIn, lx = i - ly * kIn;
                const int gy = sy0 - 4 + ly, gx = sx0 - 4 + lx;
                s_img[ly][lx] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? img[(size_t)gy * pitch + gx] : 0.f;
            }
            __syncthreads();
            const int nsy = sy1 - sy0 + 2, nsx = sx1 - sx0 + 2;
            for (int i = threadIdx.x; i < nsy * nsx; i += kFastThreads) {
                const int ly = i / nsx, lx = i - ly * nsx;
                const int gy = sy0 - 1 + ly, gx = sx0 - 1 + lx;
                float sc = 0.f;
                if (gy >= 3 && gy < H - 3 && gx >= 3 && gx < W - 3) {
                    const int iy = ly + 3, ix = lx + 3;  // staged position of (gy, gx)
                    const float c = s_img[iy][ix];
                    float d[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) d[k] = s_img[iy + c_cdy[k]][ix + c_cdx[k]] - c;
                    // smallest and largest difference over every arc of 9 (cyclic),
                    // by doubling: windows of 2, 4, 8, then one more pixel
                    float lo[16], hi[16], l2[16], h2[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        lo[k] = fminf(d[k], d[(k + 1) & 15]);
                        hi[k] = fmaxf(d[k], d[(k + 1) & 15]);
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        l2[k] = fminf(lo[k], lo[(k + 2) & 15]);
                        h2[k] = fmaxf(hi[k], hi[(k + 2) & 15]);
                    }
                    float bright = -INFINITY, dark = INFINITY;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float mn = fminf(fminf(l2[k], l2[(k + 4) & 15]), d[(k + 8) & 15]);
                        const float mx = fmaxf(fmaxf(h2[k], h2[(k + 4) & 15]), d[(k + 8) & 15]);
                        bright = fmaxf(bright, mn);   // brighter arc: its smallest rise
                        dark = fminf(dark, mx);       // darker arc: minus its smallest drop
                    }
                    const float best = fmaxf(bright, -dark);
                    sc = best > t ? best : 0.f;
                }
                s_sc[ly][lx] = sc;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < (sy1 - sy0) * (sx1 - sx0); i += kFastThreads) {
                const int ly = i / (sx1 - sx0), lx = i - ly * (sx1 - sx0);
                const int gy = sy0 + ly, gx = sx0 + lx;
                if (gy < margin || gy >= H - margin || gx < margin || gx >= W - margin) continue;
                const float v = s_sc[ly + 1][lx + 1];
                if (!(v > 0.f)) continue;
                bool keep = true;
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy) continue;
                        const int ny = gy + dy, nx = gx + dx;
                        if (ny < 0 || ny >= H || nx < 0 || nx >= W) continue;
                        const float u = s_sc[ly + 1 + dy][lx + 1 + dx];
                        const bool before = dy < 0 || (dy == 0 && dx < 0);
                        keep = keep && (before ? v > u : v >= u);
                    }
                if (keep && better(v, gy, gx, best_s, best_y, best_x)) {
                    best_s = v;
                    best_y = gy;
                    best_x = gx;
                }
            }
        }
    r_s[threadIdx.x] = best_s;
    r_y[threadIdx.x] = best_y;
    r_x[threadIdx.x] = best_x;
    __syncthreads();
    for (int o = kFastThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const int j = threadIdx.x + o;
            if (better(r_s[j], r_y[j], r_x[j], r_s[threadIdx.x], r_y[threadIdx.x], r_x[threadIdx.x])) {
                r_s[threadIdx.x] = r_s[j];
                r_y[threadIdx.x] = r_y[j];
                r_x[threadIdx.x] = r_x[j];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int b = by * grid_x + bx;
        points[2 * b] = r_x[0];
        points[2 * b + 1] = r_y[0];
        scores[b] = r_x[0] >= 0 ? r_s[0] : 0.f;
    }
}

}  // namespace

cudaError_t launch_fast_blocks(const float* img, int H, int W, size_t pitch, float t, int grid_y, int grid_x,
                               int margin, int32_t* points, float* scores, cudaStream_t st) {
    dim3 grid((unsigned)grid_x, (unsigned)grid_y);
    k_fast_blocks<<<grid, kFastThreads, 0, st>>>(img, H, W, pitch, t, grid_y, grid_x, margin, points, scores);
    return cudaGetLastError();
}

}  // namespace sfoc
