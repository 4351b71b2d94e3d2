// Integral feature images (Eq. 14-16 of arXiv 2202.13347), exact.
//
// The two channel-summed planes s1 = sum_c g and s2 = sum_c g^2 of a cube
// are turned into exclusive prefix planes P[y][x] = sum over rows < y and
// columns < x, of size (H+1) x (W+1), so any window sum costs four lookups
// (Eq. 16).  Each pixel value is rounded once to a multiple of 2^-28 and
// the prefixes are integer sums in 64 bits, so every window sum is exact
// (its only error is the per-pixel rounding, at most 2^-29 per pixel) and
// no floating-point adds are needed: GB300's FP64 rate is a small fraction
// of its FP32 and integer rates.  The sums wrap modulo 2^64, which leaves
// window differences exact.  A non-finite value enters as 2^46; window
// sums of valid values stay below 2^45 (see internal.h), so a window sum at
// or above 2^45 marks a window with a non-finite value.
//
// Three steps over 64 x 64 tiles:
//   k_int_tilesums  per tile: column sums and row sums (reads s1, s2 once)
//   k_int_lines     P on the tile grid lines: running sums over the tiles
//                   above (left), then a scan along the line
//   k_int_final     per tile: local 2-D prefix + the grid-line values
// HBM traffic is ~8 B/px read twice + 16 B/px written.
#include <math.h>

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kT = 64;
typedef unsigned long long u64;

__device__ __forceinline__ u64 quant(float v) { return int_quant(v); }

struct IntLayout {
    int H, W, nty, ntx;
    u64* colsum;  // [2][nty][W]   column sums per tile row (then exclusive prefix over tile rows)
    u64* rowsum;  // [2][ntx][H]   row sums per tile column (then exclusive prefix over tile columns)
    u64* top;     // [2][nty][W+1] P[y0(ty)][x]
    u64* left;    // [2][ntx][H+1] P[y][x0(tx)]
};

IntLayout layout(int H, int W, void* scratch) {
    IntLayout L;
    L.H = H;
    L.W = W;
    L.nty = (H + kT - 1) / kT;
    L.ntx = (W + kT - 1) / kT;
    u64* p = static_cast<u64*>(scratch);
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
    __shared__ u64 t[kT][kT + 1];
    const int ty = blockIdx.y, tx = blockIdx.x;
    const int y0 = ty * kT, x0 = tx * kT;
    for (int p = 0; p < 2; ++p) {
        const float* s = p ? s2 : s1;
        __syncthreads();
        for (int i = threadIdx.x; i < kT * kT; i += 256) {
            int r = i / kT, c = i % kT;
            int y = y0 + r, x = x0 + c;
            t[r][c] = (y < L.H && x < L.W) ? quant(s[(size_t)y * pitch + x]) : 0ull;
        }
        __syncthreads();
        const int role = threadIdx.x / kT, j = threadIdx.x % kT;  // roles 0,1: columns; 2,3: rows (half each)
        if (role == 0) {
            u64 acc = 0;
            for (int r = 0; r < kT; ++r) acc += t[r][j];
            if (x0 + j < L.W) L.colsum[((size_t)p * L.nty + ty) * L.W + x0 + j] = acc;
        } else if (role == 1) {
            u64 acc = 0;
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
        u64 run = 0;
        for (int ty = 0; ty < L.nty; ++ty) {
            u64* q = &L.colsum[((size_t)p * L.nty + ty) * L.W + x];
            u64 v = *q;
            *q = run;
            run += v;
        }
    } else if (i < ncol + nrow) {
        i -= ncol;
        int p = (int)(i / L.H), y = (int)(i % L.H);
        u64 run = 0;
        for (int tx = 0; tx < L.ntx; ++tx) {
            u64* q = &L.rowsum[((size_t)p * L.ntx + tx) * L.H + y];
            u64 v = *q;
            *q = run;
            run += v;
        }
    }
}

// Block-wide exclusive scan of n values: out[0] = 0, out[k] = sum in[0..k-1].
__device__ void block_scan_excl(const u64* in, u64* out, int n) {
    __shared__ u64 warp_tot[32];
    __shared__ u64 carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n + 1; base += blockDim.x) {
        int k = base + threadIdx.x;      // out index
        u64 v = (k >= 1 && k - 1 < n) ? in[k - 1] : 0ull;
        // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u64 u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        if (wid == 0) {
            u64 w = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                u64 u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            if (lane < nw) warp_tot[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        u64 off = carry + (wid > 0 ? warp_tot[wid - 1] : 0ull);
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
                                                    size_t pitch, IntLayout L, u64* __restrict__ P, size_t ipitch) {
    __shared__ u64 t[kT][kT + 1];
    const int ty = blockIdx.y, tx = blockIdx.x, p = blockIdx.z;
    const int y0 = ty * kT, x0 = tx * kT;
    const float* s = p ? s2 : s1;
    u64* Pp = P + (size_t)p * (L.H + 1) * ipitch;
    for (int i = threadIdx.x; i < kT * kT; i += 256) {
        int r = i / kT, c = i % kT;
        int y = y0 + r, x = x0 + c;
        t[r][c] = (y < L.H && x < L.W) ? quant(s[(size_t)y * pitch + x]) : 0ull;
    }
    __syncthreads();
    // row prefix, then column prefix (one thread per row / column: 64 integer adds)
    if (threadIdx.x < kT) {
        u64 a = 0;
        for (int c = 0; c < kT; ++c) { a += t[threadIdx.x][c]; t[threadIdx.x][c] = a; }
    }
    __syncthreads();
    if (threadIdx.x < kT) {
        u64 a = 0;
        for (int r = 0; r < kT; ++r) { a += t[r][threadIdx.x]; t[r][threadIdx.x] = a; }
    }
    __syncthreads();
    const u64* top = &L.top[((size_t)p * L.nty + ty) * (L.W + 1)];
    const u64* left = &L.left[((size_t)p * L.ntx + tx) * (L.H + 1)];
    const u64 corner = top[x0];
    for (int i = threadIdx.x; i < kT * kT; i += 256) {
        int r = i / kT, c = i % kT;
        int y = y0 + r, x = x0 + c;
        if (y < L.H && x < L.W) Pp[(size_t)(y + 1) * ipitch + (x + 1)] = top[x + 1] + (left[y + 1] - corner) + t[r][c];
    }
    // zero first row / column
    if (ty == 0)
        for (int c = threadIdx.x; c < kT; c += 256)
            if (x0 + c < L.W) Pp[x0 + c + 1] = 0;
    if (tx == 0)
        for (int r = threadIdx.x; r < kT; r += 256)
            if (y0 + r < L.H) Pp[(size_t)(y0 + r + 1) * ipitch] = 0;
    if (tx == 0 && ty == 0 && threadIdx.x == 0) Pp[0] = 0;
}

// ---- FP64 export: the prefix planes as doubles, NaN where the prefix
// rectangle holds a non-finite value (counted here, outside the hot path)
__global__ void k_nf_rows(const float* __restrict__ s1, const float* __restrict__ s2, size_t pitch, int H, int W,
                          int* __restrict__ C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * H) return;
    const int p = i / H, y = i - p * H;
    const float* s = (p ? s2 : s1) + (size_t)y * pitch;
    int* row = C + ((size_t)p * (H + 1) + y + 1) * (W + 1);
    int run = 0;
    row[0] = 0;
    for (int x = 0; x < W; ++x) {
        run += isfinite(s[x]) ? 0 : 1;
        row[x + 1] = run;
    }
}

__global__ void k_nf_cols(int H, int W, int* __restrict__ C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * (W + 1)) return;
    const int p = i / (W + 1), x = i - p * (W + 1);
    int* c = C + (size_t)p * (H + 1) * (W + 1) + x;
    c[0] = 0;
    int run = 0;
    for (int y = 1; y <= H; ++y) {
        run += c[(size_t)y * (W + 1)];
        c[(size_t)y * (W + 1)] = run;
    }
}

__global__ void k_int_to_f64(const u64* __restrict__ P, size_t ipitch, const int* __restrict__ C, int H, int W,
                             double* __restrict__ out) {
    const size_t n = 2 * (size_t)(H + 1) * (W + 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pr = i / (W + 1);
        const int x = (int)(i - pr * (W + 1));
        const double v = (double)(long long)P[pr * ipitch + x] * (1.0 / kIntScale);
        out[i] = C[i] ? NAN : v;
    }
}

}  // namespace

size_t integral_export_scratch_bytes(int H, int W) { return sizeof(int) * 2 * (size_t)(H + 1) * (W + 1); }

cudaError_t launch_integral_export(const Cube& c, void* scratch, double* out, cudaStream_t st) {
    int* C = static_cast<int*>(scratch);
    k_nf_rows<<<(2 * c.H + 127) / 128, 128, 0, st>>>(c.s1, c.s2, c.pitch, c.H, c.W, C);
    k_nf_cols<<<(2 * (c.W + 1) + 127) / 128, 128, 0, st>>>(c.H, c.W, C);
    k_int_to_f64<<<152 * 8, 256, 0, st>>>(c.integ, c.ipitch, C, c.H, c.W, out);
    return cudaGetLastError();
}

size_t integral_scratch_bytes(int H, int W) {
    size_t nty = (H + kT - 1) / kT, ntx = (W + kT - 1) / kT;
    return sizeof(u64) * (2 * nty * W + 2 * ntx * H + 2 * nty * (W + 1) + 2 * ntx * (H + 1));
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
