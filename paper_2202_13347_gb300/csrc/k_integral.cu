// Integral feature images (Eq. 14-16 of arXiv 2202.13347) in FP64.
//
// The two channel-summed planes s1 = sum_c g and s2 = sum_c g^2 of a cube
// are turned into exclusive prefix planes P[y][x] = sum over rows < y and
// columns < x, of size (H+1) x (W+1), so any window sum costs four lookups
// (Eq. 16).  Window sums of up to 10^8 pixels lose too much in FP32, hence
// FP64 everywhere here.
//
// Three steps over 64 x 64 tiles:
//   k_int_tilesums  per tile: column sums and row sums (reads s1, s2 once)
//   k_int_lines     P on the tile grid lines: running sums over the tiles
//                   above (left), then a scan along the line
//   k_int_final     per tile: local 2-D prefix + the grid-line values
// HBM traffic is ~8 B/px read twice + 16 B/px written.
#include "internal.h"

namespace sfoc {

namespace {

constexpr int kT = 64;

struct IntLayout {
    int H, W, nty, ntx;
    double* colsum;  // [2][nty][W]   column sums per tile row (then exclusive prefix over tile rows)
    double* rowsum;  // [2][ntx][H]   row sums per tile column (then exclusive prefix over tile columns)
    double* top;     // [2][nty][W+1] P[y0(ty)][x]
    double* left;    // [2][ntx][H+1] P[y][x0(tx)]
};

IntLayout layout(int H, int W, void* scratch) {
    IntLayout L;
    L.H = H;
    L.W = W;
    L.nty = (H + kT - 1) / kT;
    L.ntx = (W + kT - 1) / kT;
    double* p = static_cast<double*>(scratch);
    L.colsum = p;
    p += 2 * (size_t)L.nty * W;
    L.rowsum = p;
    p += 2 * (size_t)L.ntx * H;
    L.top = p;
    p += 2 * (size_t)L.nty * (W + 1);
    L.left = p;
    return L;
}

__global__ void __launch_bounds__(256) k_int_tilesums(const float* __restrict__ s1, const float* __restrict__ s2,
                                                       size_t pitch, IntLayout L) {
    __shared__ double t[kT][kT + 1];
    const int ty = blockIdx.y, tx = blockIdx.x;
    const int y0 = ty * kT, x0 = tx * kT;
    for (int p = 0; p < 2; ++p) {
        const float* s = p ? s2 : s1;
        __syncthreads();
        for (int i = threadIdx.x; i < kT * kT; i += 256) {
            int r = i / kT, c = i % kT;
            int y = y0 + r, x = x0 + c;
            t[r][c] = (y < L.H && x < L.W) ? (double)s[(size_t)y * pitch + x] : 0.0;
        }
        __syncthreads();
        const int role = threadIdx.x / kT, j = threadIdx.x % kT;  // roles 0,1: columns; 2,3: rows (half each)
        if (role == 0) {
            double acc = 0.0;
            for (int r = 0; r < kT; ++r) acc += t[r][j];
            if (x0 + j < L.W) L.colsum[((size_t)p * L.nty + ty) * L.W + x0 + j] = acc;
        } else if (role == 1) {
            double acc = 0.0;
            for (int c = 0; c < kT; ++c) acc += t[j][c];
            if (y0 + j < L.H) L.rowsum[((size_t)p * L.ntx + tx) * L.H + y0 + j] = acc;
        }
    }
}

// Exclusive running sums over tile rows (per column) and tile columns (per row).
__global__ void k_int_carry(IntLayout L) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t ncol = 2 * (size_t)L.W, nrow = 2 * (size_t)L.H;
    if (i < ncol) {
        int p = (int)(i / L.W), x = (int)(i % L.W);
        double run = 0.0;
        for (int ty = 0; ty < L.nty; ++ty) {
            double* q = &L.colsum[((size_t)p * L.nty + ty) * L.W + x];
            double v = *q;
            *q = run;
            run += v;
        }
    } else if (i < ncol + nrow) {
        i -= ncol;
        int p = (int)(i / L.H), y = (int)(i % L.H);
        double run = 0.0;
        for (int tx = 0; tx < L.ntx; ++tx) {
            double* q = &L.rowsum[((size_t)p * L.ntx + tx) * L.H + y];
            double v = *q;
            *q = run;
            run += v;
        }
    }
}

// Block-wide exclusive scan of n values: out[0] = 0, out[k] = sum in[0..k-1].
__device__ void block_scan_excl(const double* in, double* out, int n) {
    __shared__ double warp_tot[32];
    __shared__ double carry;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n + 1; base += blockDim.x) {
        int k = base + threadIdx.x;      // out index
        double v = (k >= 1 && k - 1 < n) ? in[k - 1] : 0.0;
        // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        if (wid == 0) {
            double w = lane < nw ? warp_tot[lane] : 0.0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                double u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            if (lane < nw) warp_tot[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        double off = carry + (wid > 0 ? warp_tot[wid - 1] : 0.0);
        if (k <= n) out[k] = v + off;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = off + v;
        __syncthreads();
    }
}

// blocks [0, 2*nty): horizontal lines; [2*nty, 2*nty + 2*ntx): vertical lines
__global__ void __launch_bounds__(256) k_int_lines(IntLayout L) {
    int b = blockIdx.x;
    if (b < 2 * L.nty) {
        int p = b / L.nty, ty = b % L.nty;
        block_scan_excl(&L.colsum[((size_t)p * L.nty + ty) * L.W], &L.top[((size_t)p * L.nty + ty) * (L.W + 1)], L.W);
    } else {
        b -= 2 * L.nty;
        int p = b / L.ntx, tx = b % L.ntx;
        block_scan_excl(&L.rowsum[((size_t)p * L.ntx + tx) * L.H], &L.left[((size_t)p * L.ntx + tx) * (L.H + 1)], L.H);
    }
}

__global__ void __launch_bounds__(256) k_int_final(const float* __restrict__ s1, const float* __restrict__ s2,
                                                    size_t pitch, IntLayout L, double* __restrict__ P,
                                                    size_t ipitch) {
    __shared__ double t[kT][kT + 1];
    const int ty = blockIdx.y, tx = blockIdx.x, p = blockIdx.z;
    const int y0 = ty * kT, x0 = tx * kT;
    const float* s = p ? s2 : s1;
    double* Pp = P + (size_t)p * (L.H + 1) * ipitch;
    for (int i = threadIdx.x; i < kT * kT; i += 256) {
        int r = i / kT, c = i % kT;
        int y = y0 + r, x = x0 + c;
        t[r][c] = (y < L.H && x < L.W) ? (double)s[(size_t)y * pitch + x] : 0.0;
    }
    __syncthreads();
    // row prefix (64 rows, 4 threads per row would need shuffles; one thread per row is fine: 64 adds)
    if (threadIdx.x < kT) {
        double a = 0.0;
        for (int c = 0; c < kT; ++c) { a += t[threadIdx.x][c]; t[threadIdx.x][c] = a; }
    }
    __syncthreads();
    if (threadIdx.x < kT) {
        double a = 0.0;
        for (int r = 0; r < kT; ++r) { a += t[r][threadIdx.x]; t[r][threadIdx.x] = a; }
    }
    __syncthreads();
    const double* top = &L.top[((size_t)p * L.nty + ty) * (L.W + 1)];
    const double* left = &L.left[((size_t)p * L.ntx + tx) * (L.H + 1)];
    const double corner = top[x0];
    for (int i = threadIdx.x; i < kT * kT; i += 256) {
        int r = i / kT, c = i % kT;
        int y = y0 + r, x = x0 + c;
        if (y < L.H && x < L.W) Pp[(size_t)(y + 1) * ipitch + (x + 1)] = top[x + 1] + (left[y + 1] - corner) + t[r][c];
    }
    // zero first row / column
    if (ty == 0)
        for (int c = threadIdx.x; c < kT; c += 256)
            if (x0 + c < L.W) Pp[x0 + c + 1] = 0.0;
    if (tx == 0)
        for (int r = threadIdx.x; r < kT; r += 256)
            if (y0 + r < L.H) Pp[(size_t)(y0 + r + 1) * ipitch] = 0.0;
    if (tx == 0 && ty == 0 && threadIdx.x == 0) Pp[0] = 0.0;
}

}  // namespace

size_t integral_scratch_bytes(int H, int W) {
    size_t nty = (H + kT - 1) / kT, ntx = (W + kT - 1) / kT;
    return sizeof(double) * (2 * nty * W + 2 * ntx * H + 2 * nty * (W + 1) + 2 * ntx * (H + 1));
}

cudaError_t launch_integral(const Cube& c, void* scratch, cudaStream_t st, int* launches) {
    IntLayout L = layout(c.H, c.W, scratch);
    dim3 g2(L.ntx, L.nty);
    k_int_tilesums<<<g2, 256, 0, st>>>(c.s1, c.s2, c.pitch, L);
    size_t nthreads = 2 * (size_t)L.W + 2 * (size_t)L.H;
    k_int_carry<<<(unsigned)((nthreads + 255) / 256), 256, 0, st>>>(L);
    k_int_lines<<<2 * L.nty + 2 * L.ntx, 256, 0, st>>>(L);
    dim3 g3(L.ntx, L.nty, 2);
    k_int_final<<<g3, 256, 0, st>>>(c.s1, c.s2, c.pitch, L, c.integ, c.ipitch);
    if (launches) *launches += 4;
    return cudaGetLastError();
}

}  // namespace sfoc
