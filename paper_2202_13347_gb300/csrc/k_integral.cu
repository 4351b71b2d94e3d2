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
#include <string.h>

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

// One cube's integral images: its sum planes, scratch layout and output.
struct IntJob {
    IntLayout L;
    const float* s1;
    const float* s2;
    size_t pitch;
    u64* P;
    size_t ipitch;
};

// CTAs of each of the four kernels for one cube
struct IntCtas {
    int tiles, carry, lines, fin;
};

IntCtas int_ctas(int H, int W) {
    const int nty = (H + kT - 1) / kT, ntx = (W + kT - 1) / kT;
    IntCtas c;
    c.tiles = ntx * nty;
    c.carry = (2 * W + 2 * H + 255) / 256;
    c.lines = 2 * nty + 2 * ntx;
    c.fin = 2 * ntx * nty;
    return c;
}

// the job of this CTA (single: `one`, the CTA index as is) and the CTA's
// index within it (binary search of the prefix `begin` of n entries)
__device__ __forceinline__ const IntJob& int_job(const IntJob& one, const IntJob* jobs, const int* begin, int n,
                                                 int* local) {
    const int bid = blockIdx.x;
    if (!jobs) {
        *local = bid;
        return one;
    }
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= bid) lo = mid;
        else hi = mid - 1;
    }
    *local = bid - begin[lo];
    return jobs[lo];
}

__global__ void __launch_bounds__(256) k_int_tilesums(const __grid_constant__ IntJob one, const IntJob* __restrict__ jobs,
                                                       const int* __restrict__ begin, int n_jobs) {
    __shared__ u64 t[kT][kT + 1];
    int local;
    const IntJob& J = int_job(one, jobs, begin, n_jobs, &local);
    const IntLayout& L = J.L;
    const float* __restrict__ s1 = J.s1;
    const float* __restrict__ s2 = J.s2;
    const size_t pitch = J.pitch;
    const int ty = local / L.ntx, tx = local - (local / L.ntx) * L.ntx;
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
__global__ void k_int_carry(const __grid_constant__ IntJob one, const IntJob* __restrict__ jobs,
                            const int* __restrict__ begin, int n_jobs) {
    int local;
    const IntJob& J = int_job(one, jobs, begin, n_jobs, &local);
    const IntLayout& L = J.L;
    size_t i = local * (size_t)blockDim.x + threadIdx.x;
    size_t ncol = 2 * (size_t)L.W, nrow = 2 * (size_t)L.H;
    // a line's values in groups of 8 loaded before any of them is replaced,
    // so the loads of a group overlap (one memory latency per group)
    auto carry = [](u64* __restrict__ base, size_t stride, int n) {
        u64 run = 0;
        for (int t0 = 0; t0 < n; t0 += 8) {
            u64 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = t0 + k < n ? base[(size_t)(t0 + k) * stride] : 0ull;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (t0 + k < n) {
                    base[(size_t)(t0 + k) * stride] = run;
                    run += v[k];
                }
        }
    };
    if (i < ncol) {
        const int p = (int)(i / L.W), x = (int)(i % L.W);
        carry(&L.colsum[(size_t)p * L.nty * L.W + x], (size_t)L.W, L.nty);
    } else if (i < ncol + nrow) {
        i -= ncol;
        const int p = (int)(i / L.H), y = (int)(i % L.H);
        carry(&L.rowsum[(size_t)p * L.ntx * L.H + y], (size_t)L.H, L.ntx);
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
__global__ void __launch_bounds__(256) k_int_lines(const __grid_constant__ IntJob one, const IntJob* __restrict__ jobs,
                                                    const int* __restrict__ begin, int n_jobs) {
    int b;
    const IntJob& J = int_job(one, jobs, begin, n_jobs, &b);
    const IntLayout& L = J.L;
    if (b < 2 * L.nty) {
        int p = b / L.nty, ty = b % L.nty;
        block_scan_excl(&L.colsum[((size_t)p * L.nty + ty) * L.W], &L.top[((size_t)p * L.nty + ty) * (L.W + 1)], L.W);
    } else {
        b -= 2 * L.nty;
        int p = b / L.ntx, tx = b % L.ntx;
        block_scan_excl(&L.rowsum[((size_t)p * L.ntx + tx) * L.H], &L.left[((size_t)p * L.ntx + tx) * (L.H + 1)], L.H);
    }
}

__global__ void __launch_bounds__(256) k_int_final(const __grid_constant__ IntJob one, const IntJob* __restrict__ jobs,
                                                    const int* __restrict__ begin, int n_jobs) {
    __shared__ u64 t[kT][kT + 1];
    int local;
    const IntJob& J = int_job(one, jobs, begin, n_jobs, &local);
    const IntLayout& L = J.L;
    const float* __restrict__ s1 = J.s1;
    const float* __restrict__ s2 = J.s2;
    const size_t pitch = J.pitch, ipitch = J.ipitch;
    u64* __restrict__ P = J.P;
    const int ntiles = L.ntx * L.nty;
    const int p = local >= ntiles ? 1 : 0;
    const int tl = local - p * ntiles;
    const int ty = tl / L.ntx, tx = tl - (tl / L.ntx) * L.ntx;
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

namespace {

IntJob int_job_of(const Cube& c, void* scratch) {
    IntJob j;
    j.L = layout(c.H, c.W, scratch);
    j.s1 = c.s1;
    j.s2 = c.s2;
    j.pitch = c.pitch;
    j.P = c.integ;
    j.ipitch = c.ipitch;
    return j;
}

}  // namespace

cudaError_t launch_integral(const Cube& c, void* scratch, cudaStream_t st, int* launches) {
    const IntJob one = int_job_of(c, scratch);
    const IntCtas n = int_ctas(c.H, c.W);
    k_int_tilesums<<<n.tiles, 256, 0, st>>>(one, nullptr, nullptr, 0);
    k_int_carry<<<n.carry, 256, 0, st>>>(one, nullptr, nullptr, 0);
    k_int_lines<<<n.lines, 256, 0, st>>>(one, nullptr, nullptr, 0);
    k_int_final<<<n.fin, 256, 0, st>>>(one, nullptr, nullptr, 0);
    if (launches) *launches += 4;
    return cudaGetLastError();
}

// Batched form.  The table blob holds n IntJob entries and four prefix
// arrays (n + 1 ints each: tiles, carry, lines, final CTAs), in that order.
size_t integral_batch_blob_bytes(int n) {
    return ((sizeof(IntJob) * (size_t)n + 15) / 16) * 16 + 4 * sizeof(int) * (size_t)(n + 1);
}

void integral_batch_blob(const Cube* const* cubes, int n, char* scratch, void* blob, int* ctas4) {
    IntJob* jobs = static_cast<IntJob*>(blob);
    int* pre = reinterpret_cast<int*>(static_cast<char*>(blob) + ((sizeof(IntJob) * (size_t)n + 15) / 16) * 16);
    int acc[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        const Cube& c = *cubes[i];
        jobs[i] = int_job_of(c, scratch);
        scratch += (integral_scratch_bytes(c.H, c.W) + 255) / 256 * 256;
        const IntCtas k = int_ctas(c.H, c.W);
        const int v[4] = {k.tiles, k.carry, k.lines, k.fin};
        for (int q = 0; q < 4; ++q) {
            pre[q * (n + 1) + i] = acc[q];
            acc[q] += v[q];
        }
    }
    for (int q = 0; q < 4; ++q) {
        pre[q * (n + 1) + n] = acc[q];
        ctas4[q] = acc[q];
    }
}

size_t integral_batch_scratch_bytes(const Cube* const* cubes, int n) {
    size_t b = 0;
    for (int i = 0; i < n; ++i) b += (integral_scratch_bytes(cubes[i]->H, cubes[i]->W) + 255) / 256 * 256;
    return b;
}

cudaError_t launch_integral_batch(const void* d_blob, int n, const int* ctas4, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const IntJob* jobs = static_cast<const IntJob*>(d_blob);
    const int* pre =
        reinterpret_cast<const int*>(static_cast<const char*>(d_blob) + ((sizeof(IntJob) * (size_t)n + 15) / 16) * 16);
    IntJob none;
    memset(&none, 0, sizeof(none));
    k_int_tilesums<<<ctas4[0], 256, 0, st>>>(none, jobs, pre, n);
    k_int_carry<<<ctas4[1], 256, 0, st>>>(none, jobs, pre + (n + 1), n);
    k_int_lines<<<ctas4[2], 256, 0, st>>>(none, jobs, pre + 2 * (n + 1), n);
    k_int_final<<<ctas4[3], 256, 0, st>>>(none, jobs, pre + 3 * (n + 1), n);
    return cudaGetLastError();
}

}  // namespace sfoc
