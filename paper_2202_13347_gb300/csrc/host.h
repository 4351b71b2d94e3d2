// Host-side state and helpers of the library's C ABI (sfoc_api.cu, batch.cu):
// the context and cube objects, argument checks, filter taps, workspace and
// stage timing.  Internal to the library.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace sfoc {

struct BatchPlan;  // batch.cu

// Autotuner: the correlation form measured fastest for (cube dtype, m, R)
// among a family of forms: 0 = every form that runs on the dtype (AUTO),
// 1 = the tensor-core forms only (IGEMM_TC, BF16 cubes).
struct TuneKey {
    int dtype, m, R, family;
    bool operator<(const TuneKey& o) const {
        if (dtype != o.dtype) return dtype < o.dtype;
        if (family != o.family) return family < o.family;
        if (m != o.m) return m < o.m;
        return R < o.R;
    }
};
struct TuneEntry {
    int path;        // sfoc_corr_path of the winner (a concrete form, never AUTO or IGEMM_TC)
    int option;      // FFT: transform side; otherwise 0
    int n_cand;      // candidates timed
    int cand_path[6];
    int cand_option[6];
    float cand_ms[6];  // per-launch milliseconds of each candidate on the sample
    int sample;        // points in the timed sample
};

void destroy_plan(BatchPlan* p);

}  // namespace sfoc

struct sfoc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int64_t launches = 0;
    int* d_err = nullptr;  // device error word set by bounded waits
    // cached cubes and staging for the pair pipeline
    sfoc_cube* pair_ref = nullptr;
    sfoc_cube* pair_sen = nullptr;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // second stream for the sensed image's host copy (overlaps the reference cube)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_copied = nullptr;
    cudaEvent_t ev_switch = nullptr;  // orders a new stream after the previous one
    std::vector<cudaEvent_t> ev_wave;  // host batch: the images of SFOC wave w copied (last: every copy)
    // per-stage timing
    bool timing = false;
    struct Ev {
        int stage, launches;
        cudaEvent_t a, b;
    };
    std::vector<Ev> evs;
    std::vector<cudaEvent_t> pool;
    double acc_ms[SFOC_NUM_STAGES] = {0};
    int64_t acc_n[SFOC_NUM_STAGES] = {0};
    std::vector<float> scope_ms[SFOC_NUM_STAGES];  // each timed scope of a stage, in order
    // autotuner
    bool autotune = true;
    std::map<sfoc::TuneKey, sfoc::TuneEntry> tune;
    // batch plans (tables, owned cubes, captured graphs), most recent last
    std::vector<sfoc::BatchPlan*> plans;
    size_t max_plans = 2;
    int64_t plans_built = 0;  // batch plans built over the context's life
    // device staging of fastncc_register_batch_host (images, points, results)
    void* hstage = nullptr;
    size_t hstage_bytes = 0;
    // host-buffer batch submissions (fastncc_submit_batch_host): their count,
    // and events on the context stream: the last submission's images read by
    // its SFOC launches, and submission t's results copied out (slot t mod
    // kHostRing)
    static constexpr int kHostRing = 4;
    int64_t host_ticket = 0;
    cudaEvent_t ev_hsfoc = nullptr;
    cudaEvent_t ev_hpts = nullptr;  // the point sets of the submission being enqueued copied
    cudaEvent_t ev_hdone[kHostRing] = {};
};

struct sfoc_cube {
    sfoc::Cube c;
};

namespace sfoc {

enum { ST_STEER = 0, ST_SMOOTH = 1, ST_INTEGRAL = 2, ST_STATS = 3, ST_CORR = 4, ST_NCC = 5, ST_OTHER = 6 };

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Brackets the launches of one stage with events (when timing is on and the
// stream is not being captured) and counts them.
struct StageScope {
    sfoc_ctx* c;
    int stage, launches;
    cudaEvent_t a = nullptr;
    StageScope(sfoc_ctx* ctx, int st, int nl);
    ~StageScope();
};

sfoc_status fail(sfoc_ctx* ctx, sfoc_status s, const std::string& msg);
sfoc_status cuda_fail(sfoc_ctx* ctx, cudaError_t e, const char* what);
bool capturing(cudaStream_t s);
// Grows the workspace (never inside a stream capture).  A reallocation
// drops the context's batch plans, whose tables point into the old one.
sfoc_status ensure_ws(sfoc_ctx* ctx, size_t bytes);
sfoc_status check_params(sfoc_ctx* ctx, const sfoc_params& p);
SteerTaps make_steer(const sfoc_params& p);
SmoothTaps make_smooth(const sfoc_params& p);
sfoc_status alloc_cube(sfoc_ctx* ctx, Cube& c, int H, int W, int z, int dtype);
void free_cube_mem(Cube& c);
sfoc_status build_integral(sfoc_ctx* ctx, Cube& c);
inline size_t roundup(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline size_t align256(size_t v) { return roundup(v, 256); }
// the library's SM count of the context's device
int sm_count(int device);

// Correlation dispatch for one pair (the points of `one`): `path` is a
// concrete sfoc_corr_path (DIRECT_F32, FFT, TC_TOEPLITZ, TC_COLUMN,
// TC_BAND), `option` the FFT side (0 = the smallest that serves).  Returns
// cudaErrorNotSupported where the form does not run for the job.
cudaError_t launch_corr_path(sfoc_ctx* ctx, int path, int option, MatchJob& one);
// The concrete form a family takes for (dtype, m, R) without a tuned entry
// (-1: none runs).
int auto_rule(int dtype, int m, int R, int family);
// Measures every form of the family that runs for `one` on its first points
// (their template statistics already computed) and stores the winner;
// returns it.
const TuneEntry* autotune_pair(sfoc_ctx* ctx, int dtype, int family, MatchJob one);
// The concrete form for a match with corr_path `path` (AUTO, IGEMM_TC or a
// concrete one): the tuned entry, measured now when allowed, else the rule.
// *option receives the FFT side (0 otherwise); -1 when no form runs.
int resolve_path(sfoc_ctx* ctx, int path, int dtype, const MatchJob* one, bool may_measure, int* option);
// whether a concrete path computes the zero-mean numerator of Eq. 9
inline bool centered_path(int path) { return path == SFOC_CORR_DIRECT_F32 || path == SFOC_CORR_FFT; }
// whether a concrete path runs on cubes of this dtype
inline bool path_serves(int path, int dtype) {
    if (path == SFOC_CORR_FFT) return true;
    if (path == SFOC_CORR_DIRECT_F32) return dtype == SFOC_DTYPE_F32;
    return dtype == SFOC_DTYPE_BF16;
}

}  // namespace sfoc
