// Internal declarations of the SFOC / Fast-NCC_SFOC CUDA library (sm_103a).
// Shared only between this library's own translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sfoc.h"

namespace sfoc {

// ---- limits -----------------------------------------------------------
constexpr int kMaxScales = 4;
constexpr int kMaxDerivRadius = 9;   // ceil(3 sigma) <= 9
constexpr int kMaxSmoothRadius = 6;  // ceil(3 sigma_d) <= 6
constexpr int kMaxDil = 3;
constexpr int kMaxOrient = 8;
constexpr int kMaxZ = 16;
constexpr int kMaxTemplate = 128;
constexpr int kMaxRadius = 63;

// ---- filter taps (computed on the host in double, stored as float) -----
// A separable 2-D kernel a(x) b(y) is applied as a horizontal pass with a
// and a vertical pass with b; "odd" taps satisfy t(-q) = -t(q) and "even"
// taps t(-q) = t(q), so only q = 0..K are stored.
struct SteerTaps {
    int ns;                                   // first-order scales
    int K1[kMaxScales];                       // radius per scale
    float a1[kMaxScales][kMaxDerivRadius + 1];  // odd: -q/(2 pi s^4) exp(-q^2/2s^2)
    float g1[kMaxScales][kMaxDerivRadius + 1];  // even: exp(-q^2/2s^2)
    int K2;                                   // second-order radius (0 = no second group)
    float a2[kMaxDerivRadius + 1];            // even, zero-mean second-derivative factor
    float g2[kMaxDerivRadius + 1];            // even Gaussian factor
    float c2x[kMaxDerivRadius + 1];           // odd: q exp(-q^2/2s^2) / (2 pi s^6)
    float c2y[kMaxDerivRadius + 1];           // odd: q exp(-q^2/2s^2)
    int no;                                   // orientations
    float ct[kMaxOrient], st[kMaxOrient];     // cos/sin of theta_k = k pi / no
    int rectify;
    int second;                               // 1: compute the second-order group
    int halo;                                 // max radius
};

struct SmoothTaps {
    int n_dil;
    int dil[kMaxDil];
    int Kd[2];                                // smoothing radius per group
    float g[2][kMaxSmoothRadius + 1];         // normalised even taps per group
    int halo[2];                              // max rate * Kd per group
    int no;                                   // channels per group
    int z;                                    // channels
    float eps;
};

// ---- cube --------------------------------------------------------------
// F32 cube: planar [z][H][pitch] float.
// BF16 cube (z = 12): two 8-channel chunks per pixel, chunk g = the six
// channels of group g and two zeros, stored twice:
//   rm: [2][H][W][8] (pixels row-major)     - Toeplitz-form windows
//   cm: [2][W][H][8] (pixels column-major)  - templates; column-form windows
// Both buffers carry 256 bytes of padding past the end (copies in 128-byte
// runs of pixels may read up to 7 pixels past the last column).
struct Cube {
    int H = 0, W = 0, z = 0, dtype = SFOC_DTYPE_F32;
    size_t pitch = 0;          // elements per row of f32 planes / sum planes
    float* f32 = nullptr;      // [z][H][pitch]
    __nv_bfloat16* rm = nullptr;
    __nv_bfloat16* cm = nullptr;
    float* s1 = nullptr;       // [H][pitch] sum over channels of g
    float* s2 = nullptr;       // [H][pitch] sum over channels of g^2
    unsigned long long* integ = nullptr;  // [2][H+1][ipitch] exclusive prefix of s1, s2 in units of 2^-28
    size_t ipitch = 0;
    bool integ_valid = false;
    int device = 0;
};

struct TileSums;  // integral-image scratch layout (k_integral.cu)

// One image of an SFOC launch: the input, its steering planes F and the
// cube it builds.  A single-image launch passes one by value; a batched
// launch passes a device table and the prefix `begin` of the launch's CTAs
// per image (n_jobs + 1 entries), so one launch covers the tiles of every
// image.
struct ImgJob {
    const void* img;   // float or uint16 samples
    size_t pitch;
    int H, W;
    float* F;          // z steering planes [z][H][fpitch]
    size_t fpitch;
    float* c32;        // F32 cube [z][H][cpitch] or nullptr
    size_t cpitch;
    __nv_bfloat16* rm; // BF16 cube layouts or nullptr
    __nv_bfloat16* cm;
    float* s1;         // per-pixel sums [H][cpitch]
    float* s2;
};

// The image of this CTA and its tile index within it.
__device__ __forceinline__ const ImgJob& img_job(const ImgJob& one, const ImgJob* jobs, const int* begin, int n_jobs,
                                                 int* tile) {
    const int bid = blockIdx.x;
    if (!jobs) {
        *tile = bid;
        return one;
    }
    int lo = 0, hi = n_jobs - 1;  // the last image whose first CTA is at or before this one
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= bid) lo = mid;
        else hi = mid - 1;
    }
    *tile = bid - begin[lo];
    return jobs[lo];
}

// ---- kernel launchers (return cudaError_t of the launch) ----------------
cudaError_t launch_sfoc_steer(const float* img, int H, int W, size_t pitch, float* F, size_t fpitch,
                              const SteerTaps& tp, int z_first, cudaStream_t st);
cudaError_t launch_sfoc_steer(const uint16_t* img, int H, int W, size_t pitch, float* F, size_t fpitch,
                              const SteerTaps& tp, int z_first, cudaStream_t st);
cudaError_t launch_sfoc_smooth(const float* F, size_t fpitch, int H, int W, const SmoothTaps& tp, Cube& c,
                               cudaStream_t st);
// Batched build of several float images with the paper's radii and rates
// (sfoc_batch_supported): one steering launch and one smoothing launch per
// group over the tiles of all images (device table `jobs`, n_jobs entries).
// steer_begin / smooth_begin: device prefix sums of each kernel's CTAs per
// image (sfoc_batch_tiles gives the counts).
bool sfoc_batch_supported(const SteerTaps& st, const SmoothTaps& sm);
void sfoc_batch_tiles(int H, int W, int* steer_ctas, int* smooth_ctas);
cudaError_t launch_sfoc_batch(const ImgJob* jobs, int n_jobs, const int* steer_begin, int steer_ctas,
                              const int* smooth_begin, int smooth_ctas, const SteerTaps& st, const SmoothTaps& sm,
                              cudaStream_t s);
int smooth_launch_count(const SmoothTaps& tp);  // kernels launch_sfoc_smooth launches
cudaError_t launch_cube_export(const Cube& c, float* out, cudaStream_t st);

// Integral planes in fixed point: a value v counts as round(v * 2^28), sums
// are 64-bit integers modulo 2^64 (window differences exact).  Valid window
// sums stay below 2^45: at most 128^2 pixels of |s1| <= 2 sqrt(8) < 5.7 (two
// unit-norm groups of at most 8 channels) or s2 <= 2, i.e. < 2^44.6 units.
// A non-finite value enters as kIntNonFinite, so a window sum >= 2^45 holds
// one (a window has at most 128^2 = 2^14 pixels, so even one made only of
// such values sums to 2^60 at most, well below 2^63).
constexpr float kIntScale = 268435456.f;                  // 2^28
constexpr long long kIntNonFinite = 1ll << 46;
constexpr long long kIntNonFiniteMin = 1ll << 45;
__host__ __device__ inline double int_units_to_double(long long v) { return (double)v * (1.0 / 268435456.0); }
// one pixel value in those units (the integral images and the template sums
// round every pixel with this one function)
__device__ __forceinline__ unsigned long long int_quant(float v) {
    if (!isfinite(v)) return (unsigned long long)kIntNonFinite;
    return (unsigned long long)__float2ll_rn(v * kIntScale);
}

size_t integral_scratch_bytes(int H, int W);
cudaError_t launch_integral(const Cube& c, void* scratch, cudaStream_t st, int* launches);
// batched integral images of n cubes: a table blob (integral_batch_blob_bytes,
// filled on the host by integral_batch_blob with each cube's scratch carved
// from `scratch`, integral_batch_scratch_bytes in all) and one launch of each
// of the four kernels over all cubes; ctas4 = the kernels' CTA counts
size_t integral_batch_blob_bytes(int n);
size_t integral_batch_scratch_bytes(const Cube* const* cubes, int n);
void integral_batch_blob(const Cube* const* cubes, int n, char* scratch, void* blob, int* ctas4);
cudaError_t launch_integral_batch(const void* d_blob, int n, const int* ctas4, cudaStream_t st);
size_t integral_export_scratch_bytes(int H, int W);
cudaError_t launch_integral_export(const Cube& c, void* scratch, double* out, cudaStream_t st);

struct PointStat {
    double RT, RTT;       // template sums (Eq. 12) from the sensed integral images
    float tmean;          // R_T / mnz (for the zero-mean template)
    int status;           // SFOC_PT_*
};

// ---- work descriptions shared by single-pair and batched launches -------
// One image pair of a match: both cubes, the pair's points, m and R, and
// where its per-point scratch and results go.  A single-pair launch passes
// one job by value (a __grid_constant__ kernel parameter, so its tensor maps
// can be used by TMA in place); a batched launch passes a device table of
// jobs and a list of items (job, point), so one launch covers the points of
// every pair.  The tensor maps are those of the correlation form the job's
// class runs (unused by the other kernels).
struct MatchJob {  // aligned as its tensor maps (128 bytes)
    CUtensorMap tm[3];
    // reference (searched) cube
    const float* rf32;
    const __nv_bfloat16* rrm;
    const __nv_bfloat16* rcm;
    const unsigned long long* rint;
    size_t rpitch, rplane, ripitch;
    int Hr, Wr;
    // sensed (template) cube
    const float* sf32;
    const float* ss1;
    const float* ss2;
    const __nv_bfloat16* srm;
    const __nv_bfloat16* scm;
    size_t spitch, splane;
    int Hs, Ws;
    int z, m, R, n;
    int centered;           // 1: the correlation gives the zero-mean numerator of Eq. 9 (FP32 forms)
    const int32_t* pts;     // n x (x, y)
    PointStat* stats;       // n
    float* maps;            // n x (2R+1)^2 correlation maps (scratch)
    float* out_maps;        // optional n x (2R+1)^2 NCC maps
    fastncc_result* out;    // n
};

// The items of a launch: nullptr = the points 0 .. n-1 of `one`.
struct ItemSet {
    const MatchJob* jobs = nullptr;  // device table
    const int2* items = nullptr;     // device list of (job, point)
    int n = 0;                       // items
    int* queue = nullptr;            // device counter for dynamic fetching (zeroed before the launch) or nullptr
    int max_m = 0, max_R = 0;        // bounds over the items' jobs (shared-memory sizes)
    int max_lw = 0;                  // largest m + 2R of the items' jobs
};

__device__ __forceinline__ const MatchJob& item_job(const MatchJob& one, const MatchJob* jobs, const int2* items,
                                                     int k, int* point) {
    if (!items) {
        *point = k;
        return one;
    }
    const int2 it = items[k];
    *point = it.y;
    return jobs[it.x];
}

MatchJob make_job(const Cube& ref, const Cube& sen, const int32_t* pts, int n, int m, int R, PointStat* stats,
                  float* maps, float* out_maps, fastncc_result* out);

// Each launcher runs its kernel over the items of `is` (is.items == nullptr:
// the points of `one`).
cudaError_t launch_template_stats(const MatchJob& one, const ItemSet& is, cudaStream_t st);
// direct FP32 correlation: threads-per-tile class of a radius (1, 2, 4 or 8;
// 0 when R is too large), and whether the shared memory of (m, R) fits
int corr_f32_class(int R);
bool corr_f32_supported(int m, int R);
cudaError_t launch_corr_f32(const MatchJob& one, const ItemSet& is, int tpt, cudaStream_t st);
bool corr_fft_supported(int m, int R);
int corr_fft_side(int m, int R);  // smallest transform side that serves (m, R): 64 or 128
// bf16: the jobs' cubes are BF16 (read from the row-major chunk layout rm)
cudaError_t launch_corr_fft(const MatchJob& one, const ItemSet& is, int L, bool bf16, cudaStream_t st);
// tensor-core forms: 1 Toeplitz, 2 column, 3 band.  corr_tc_class: the
// kernel instance a job of (m, R) takes in that form (column: G, band: NQ,
// Toeplitz: 1 = runs, one pair per launch), 0 where the form does not run;
// corr_tc_auto_form: the form IGEMM_TC picks (fewest MMAs), 0 = none;
// corr_tc_maps: sets the job's tensor maps for the form.
int corr_tc_class(int form, int m, int R);
int corr_tc_auto_form(int m, int R);
bool corr_tc_maps(int form, MatchJob& j);
cudaError_t launch_corr_tc(int form, int cls, const MatchJob& one, const ItemSet& is, const int* ms, const int* Rs,
                           int cnt, int* err_flag, cudaStream_t st);
size_t corr_tc_smem_bytes(int m, int R);
cudaError_t launch_ncc_argmax(const MatchJob& one, const ItemSet& is, cudaStream_t st);

// block-based FAST (k_fast.cu)
cudaError_t launch_fast_blocks(const float* img, int H, int W, size_t pitch, float t, int grid_y, int grid_x,
                               int margin, int32_t* points, float* scores, cudaStream_t st);

// outlier rejection (k_ransac.cu)
size_t ransac_workspace_bytes(int n_hyp);
cudaError_t launch_ransac(const double* src, const double* dst, const uint8_t* valid, int n, int proj,
                          const int32_t* samples, int n_hyp, double threshold, int refits, double* H_out,
                          uint8_t* mask, int32_t* info, int32_t* scores_out, void* ws, cudaStream_t st, int* launches);
cudaError_t launch_rectify(const float* img, int H, int W, size_t pitch, const double* Hm, float fill, int out_h,
                           int out_w, float* out, cudaStream_t st);
cudaError_t launch_results_to_points(const int32_t* pts, const fastncc_result* res, int n, double* src, double* dst,
                                     uint8_t* valid, cudaStream_t st);

// peak microbenchmarks (k_peak.cu): FP32 FFMA, paired FFMA2 and FP64 TFLOP/s,
// HBM copy GB/s; synchronous
cudaError_t measure_peaks(cudaStream_t st, int sms, double* fp32, double* fp32x2, double* fp64, double* hbm);

// failure-path self-test (k_selftest.cu): one bounded wait that expires after
// limit_us microseconds and sets *err
cudaError_t launch_wait_selftest(int* err, int limit_us, cudaStream_t st);

// template half-width: rows before the centre
__host__ __device__ inline int template_half(int m) { return (m % 2) ? (m - 1) / 2 : m / 2; }

}  // namespace sfoc
