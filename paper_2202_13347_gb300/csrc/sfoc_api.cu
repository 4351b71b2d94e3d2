// C ABI of the SFOC / Fast-NCC_SFOC library (include/sfoc.h).
//
// Host side only: argument checks, filter taps (computed in double from
// the closed forms of Eq. 2, 3, 5 and the dilated Gaussian of Sec. 2.1),
// workspace management and kernel dispatch on the context's stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "host.h"

using namespace sfoc;


namespace {
const double kPi = 3.14159265358979323846;
int radius_of(double sigma, double mult) { return (int)ceil(mult * sigma - 1e-9); }
}  // namespace

namespace sfoc {

sfoc_status fail(sfoc_ctx* ctx, sfoc_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

sfoc_status cuda_fail(sfoc_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    // the error is reported now; a recoverable one (a failed allocation, a
    // refused launch) is also the runtime's "last error", which the launch
    // check of a later call (cudaGetLastError) would otherwise report again
    // although that launch succeeded.  A sticky error stays sticky.
    (void)cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(ctx, SFOC_ERR_OOM, m);
    return fail(ctx, SFOC_ERR_CUDA, m);
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

int sm_count(int device) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

static cudaEvent_t pool_event(sfoc_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

StageScope::StageScope(sfoc_ctx* ctx, int st, int nl) : c(ctx), stage(st), launches(nl) {
    c->launches += nl;
    if (!c->timing || capturing(c->stream)) return;
    a = pool_event(c);
    if (a) cudaEventRecord(a, c->stream);
}

StageScope::~StageScope() {
    if (!a) return;
    cudaEvent_t b = pool_event(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->evs.push_back({stage, launches, a, b});
}

sfoc_status ensure_ws(sfoc_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return SFOC_OK;
    if (capturing(ctx->stream))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "workspace too small inside a stream capture; call sfoc_ctx_reserve first");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    for (BatchPlan* p : ctx->plans) destroy_plan(p);  // their tables point into the old workspace
    ctx->plans.clear();
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t nb = roundup(bytes, 1 << 20);
    e = cudaMalloc(&ctx->ws, nb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(workspace)");
    ctx->ws_bytes = nb;
    return SFOC_OK;
}

sfoc_status check_params(sfoc_ctx* ctx, const sfoc_params& p) {
    if (p.n_scales < 1 || p.n_scales > kMaxScales) return fail(ctx, SFOC_ERR_UNSUPPORTED, "n_scales must be 1..4");
    for (int s = 0; s < p.n_scales; ++s) {
        if (!(p.scales[s] > 0.0)) return fail(ctx, SFOC_ERR_INVALID_ARG, "scales must be > 0");
        if (radius_of(p.scales[s], p.radius_mult) > kMaxDerivRadius)
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "first-order kernel radius > 9");
    }
    if (!(p.radius_mult > 0.0)) return fail(ctx, SFOC_ERR_INVALID_ARG, "radius_mult must be > 0");
    if (!p.first_order_only) {
        if (!(p.sigma2 > 0.0)) return fail(ctx, SFOC_ERR_INVALID_ARG, "sigma2 must be > 0");
        if (radius_of(p.sigma2, p.radius_mult) > kMaxDerivRadius)
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "second-order kernel radius > 9");
    }
    if (p.n_orient < 1 || p.n_orient > kMaxOrient) return fail(ctx, SFOC_ERR_UNSUPPORTED, "n_orient must be 1..8");
    if (p.n_dil < 1 || p.n_dil > kMaxDil) return fail(ctx, SFOC_ERR_UNSUPPORTED, "n_dil must be 1..3");
    for (int r = 0; r < p.n_dil; ++r)
        if (p.dil[r] < 1 || p.dil[r] > 3) return fail(ctx, SFOC_ERR_UNSUPPORTED, "dilation rates must be 1..3");
    double sd[2] = {p.sigma_d1, p.sigma_d2};
    for (int g = 0; g < 2; ++g) {
        if (!(sd[g] >= 0.0)) return fail(ctx, SFOC_ERR_INVALID_ARG, "smoothing STDs must be >= 0 (0: unsmoothed)");
        if (radius_of(sd[g], p.radius_mult) > kMaxSmoothRadius)
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "smoothing radius > 6");
    }
    if (!(p.eps >= 0.0)) return fail(ctx, SFOC_ERR_INVALID_ARG, "eps must be >= 0");
    if (p.cube_dtype != SFOC_DTYPE_F32 && p.cube_dtype != SFOC_DTYPE_BF16)
        return fail(ctx, SFOC_ERR_INVALID_ARG, "cube_dtype must be F32 or BF16");
    if (p.cube_dtype == SFOC_DTYPE_BF16 && (p.n_orient != 6 || p.first_order_only))
        return fail(ctx, SFOC_ERR_UNSUPPORTED, "BF16 cubes need 12 channels (n_orient 6, both groups)");
    return SFOC_OK;
}

SteerTaps make_steer(const sfoc_params& p) {
    SteerTaps t;
    memset(&t, 0, sizeof(t));
    t.ns = p.n_scales;
    int hal = 0;
    for (int s = 0; s < p.n_scales; ++s) {
        double sg = p.scales[s], s2 = sg * sg, s4 = s2 * s2;
        int K = radius_of(sg, p.radius_mult);
        t.K1[s] = K;
        hal = std::max(hal, K);
        for (int q = 0; q <= K; ++q) {
            double e = exp(-(double)q * q / (2.0 * s2));
            t.a1[s][q] = (float)(-(double)q / (2.0 * kPi * s4) * e);
            t.g1[s][q] = (float)e;
        }
    }
    t.second = p.first_order_only ? 0 : 1;
    if (t.second) {
        double sg = p.sigma2, s2 = sg * sg, s4 = s2 * s2, s6 = s4 * s2;
        int K = radius_of(sg, p.radius_mult);
        t.K2 = K;
        hal = std::max(hal, K);
        double a2[kMaxDerivRadius + 1];
        double mean = 0.0;
        for (int q = 0; q <= K; ++q) {
            double e = exp(-(double)q * q / (2.0 * s2));
            a2[q] = -(1.0 / (2.0 * kPi * s4)) * (1.0 - q * q / s2) * e;
            mean += (q == 0 ? 1.0 : 2.0) * a2[q];
            t.g2[q] = (float)e;
            t.c2x[q] = (float)(q * e / (2.0 * kPi * s6));
            t.c2y[q] = (float)(q * e);
        }
        mean /= (2 * K + 1);
        for (int q = 0; q <= K; ++q) t.a2[q] = (float)(a2[q] - mean);
    }
    t.no = p.n_orient;
    for (int k = 0; k < p.n_orient; ++k) {
        t.ct[k] = (float)cos(k * kPi / p.n_orient);
        t.st[k] = (float)sin(k * kPi / p.n_orient);
    }
    t.rectify = p.rectify ? 1 : 0;
    t.halo = hal;
    return t;
}

SmoothTaps make_smooth(const sfoc_params& p) {
    SmoothTaps t;
    memset(&t, 0, sizeof(t));
    t.n_dil = p.n_dil;
    int maxrate = 0;
    for (int r = 0; r < p.n_dil; ++r) {
        t.dil[r] = p.dil[r];
        maxrate = std::max(maxrate, p.dil[r]);
    }
    double sd[2] = {p.sigma_d1, p.sigma_d2};
    for (int g = 0; g < 2; ++g) {
        if (sd[g] == 0.0) {  // smoothing off for this group (Fig. 3 (d)): one unit tap, no rate sum
            t.Kd[g] = 0;
            t.g[g][0] = 1.f;
            t.halo[g] = 0;
            continue;
        }
        int K = radius_of(sd[g], p.radius_mult);
        t.Kd[g] = K;
        double w[kMaxSmoothRadius + 1], sum = 0.0;
        for (int q = 0; q <= K; ++q) {
            w[q] = exp(-(double)q * q / (2.0 * sd[g] * sd[g]));
            sum += (q == 0 ? 1.0 : 2.0) * w[q];
        }
        for (int q = 0; q <= K; ++q) t.g[g][q] = (float)(w[q] / sum);
        t.halo[g] = maxrate * K;
    }
    t.no = p.n_orient;
    t.z = p.first_order_only ? p.n_orient : 2 * p.n_orient;
    if (p.first_order_only) t.halo[1] = 0;
    t.eps = (float)p.eps;
    return t;
}

void free_cube_mem(Cube& c) {
    cudaFree(c.f32);
    cudaFree(c.rm);
    cudaFree(c.cm);
    cudaFree(c.s1);
    cudaFree(c.s2);
    cudaFree(c.integ);
    c.f32 = nullptr;
    c.rm = c.cm = nullptr;
    c.s1 = c.s2 = nullptr;
    c.integ = nullptr;
}

sfoc_status alloc_cube(sfoc_ctx* ctx, Cube& c, int H, int W, int z, int dtype) {
    c.H = H;
    c.W = W;
    c.z = z;
    c.dtype = dtype;
    c.pitch = roundup((size_t)W, 32);
    c.ipitch = (size_t)W + 1;
    c.device = ctx->device;
    cudaError_t e = cudaSuccess;
    size_t plane = c.pitch * (size_t)H;
    if (dtype == SFOC_DTYPE_F32) {
        e = cudaMalloc(&c.f32, sizeof(float) * plane * z);
    } else {
        // + 256 bytes: copies in 128-byte runs of pixels may read up to 112
        // bytes past the last column
        e = cudaMalloc(&c.rm, sizeof(__nv_bfloat16) * 16 * (size_t)H * W + 256);
        if (e == cudaSuccess) e = cudaMalloc(&c.cm, sizeof(__nv_bfloat16) * 16 * (size_t)H * W + 256);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c.s1, sizeof(float) * plane);
    if (e == cudaSuccess) e = cudaMalloc(&c.s2, sizeof(float) * plane);
    if (e == cudaSuccess) e = cudaMalloc(&c.integ, sizeof(unsigned long long) * 2 * (size_t)(H + 1) * c.ipitch);
    if (e != cudaSuccess) {
        free_cube_mem(c);
        return cuda_fail(ctx, e, "cudaMalloc(cube)");
    }
    return SFOC_OK;
}

sfoc_status build_integral(sfoc_ctx* ctx, Cube& c) {
    if (c.integ_valid) return SFOC_OK;
    sfoc_status s = ensure_ws(ctx, integral_scratch_bytes(c.H, c.W));
    if (s != SFOC_OK) return s;
    int nl = 0;
    cudaError_t e;
    {
        StageScope sc(ctx, ST_INTEGRAL, 4);
        e = launch_integral(c, ctx->ws, ctx->stream, &nl);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "integral launch");
    c.integ_valid = true;
    return SFOC_OK;
}

}  // namespace sfoc

namespace sfoc {

cudaError_t launch_corr_path(sfoc_ctx* ctx, int path, int option, MatchJob& one) {
    const ItemSet none;
    const int m = one.m, R = one.R;
    switch (path) {
        case SFOC_CORR_DIRECT_F32: {
            const int c = corr_f32_class(R);
            if (!c || !corr_f32_supported(m, R) || !one.rf32) return cudaErrorNotSupported;
            return launch_corr_f32(one, none, c, ctx->stream);
        }
        case SFOC_CORR_FFT: {
            if (!corr_fft_supported(m, R)) return cudaErrorNotSupported;
            return launch_corr_fft(one, none, option ? option : corr_fft_side(m, R), one.rf32 == nullptr,
                                   ctx->stream);
        }
        case SFOC_CORR_TC_TOEPLITZ:
        case SFOC_CORR_TC_COLUMN:
        case SFOC_CORR_TC_BAND: {
            const int form = path == SFOC_CORR_TC_TOEPLITZ ? 1 : path == SFOC_CORR_TC_COLUMN ? 2 : 3;
            const int cls = corr_tc_class(form, m, R);
            if (!cls || !one.rrm || one.z != 12 || !corr_tc_maps(form, one)) return cudaErrorNotSupported;
            return launch_corr_tc(form, cls, one, none, &m, &R, 1, ctx->d_err, ctx->stream);
        }
        default:
            return cudaErrorNotSupported;
    }
}

int auto_rule(int dtype, int m, int R, int family) {
    if (dtype == SFOC_DTYPE_BF16) {
        switch (corr_tc_auto_form(m, R)) {
            case 3: return SFOC_CORR_TC_BAND;
            case 2: return SFOC_CORR_TC_COLUMN;
            case 1: return SFOC_CORR_TC_TOEPLITZ;
            default: return family == 0 && corr_fft_supported(m, R) ? SFOC_CORR_FFT : -1;
        }
    }
    if (family != 0) return -1;
    if (corr_fft_supported(m, R)) return SFOC_CORR_FFT;
    return corr_f32_supported(m, R) ? SFOC_CORR_DIRECT_F32 : -1;
}

const TuneEntry* autotune_pair(sfoc_ctx* ctx, int dtype, int family, MatchJob one) {
    const int m = one.m, R = one.R;
    TuneEntry t;
    memset(&t, 0, sizeof(t));
    auto add = [&](int path, int option) {
        t.cand_path[t.n_cand] = path;
        t.cand_option[t.n_cand++] = option;
    };
    if (dtype == SFOC_DTYPE_BF16) {
        if (corr_tc_class(3, m, R) > 0) add(SFOC_CORR_TC_BAND, 0);
        if (corr_tc_class(2, m, R) > 0) add(SFOC_CORR_TC_COLUMN, 0);
        if (corr_tc_class(1, m, R) > 0) add(SFOC_CORR_TC_TOEPLITZ, 0);
    }
    if (family == 0 && corr_fft_supported(m, R)) {
        const int side = corr_fft_side(m, R);
        add(SFOC_CORR_FFT, side);
        if (side == 64) add(SFOC_CORR_FFT, 128);  // the larger transform as a tile option
    }
    if (family == 0 && dtype == SFOC_DTYPE_F32 && corr_f32_supported(m, R)) add(SFOC_CORR_DIRECT_F32, 0);
    if (t.n_cand == 0) return nullptr;
    // a sample of up to two waves of points, timed per candidate: one
    // warm-up launch, then the better of two
    const int sms = sm_count(ctx->device);
    one.n = one.n < 2 * sms ? one.n : 2 * sms;
    t.sample = one.n;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    int best = -1;
    for (int c = 0; c < t.n_cand; ++c) {
        t.cand_ms[c] = -1.f;
        if (!ev[0] || !ev[1] || !ev[2]) continue;
        bool ok = launch_corr_path(ctx, t.cand_path[c], t.cand_option[c], one) == cudaSuccess;
        ok = ok && cudaEventRecord(ev[0], ctx->stream) == cudaSuccess;
        ok = ok && launch_corr_path(ctx, t.cand_path[c], t.cand_option[c], one) == cudaSuccess;
        ok = ok && cudaEventRecord(ev[1], ctx->stream) == cudaSuccess;
        ok = ok && launch_corr_path(ctx, t.cand_path[c], t.cand_option[c], one) == cudaSuccess;
        ok = ok && cudaEventRecord(ev[2], ctx->stream) == cudaSuccess;
        ok = ok && cudaEventSynchronize(ev[2]) == cudaSuccess;
        ctx->launches += 3;
        float a = 0.f, b = 0.f;
        if (ok && cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ev[1], ev[2]) == cudaSuccess) {
            t.cand_ms[c] = a < b ? a : b;
            if (best < 0 || t.cand_ms[c] < t.cand_ms[best]) best = c;
        } else {
            (void)cudaGetLastError();  // a refused candidate leaves no error behind
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (best < 0) return nullptr;
    t.path = t.cand_path[best];
    t.option = t.cand_option[best];
    auto& slot = ctx->tune[TuneKey{dtype, m, R, family}];
    slot = t;
    return &slot;
}

int resolve_path(sfoc_ctx* ctx, int path, int dtype, const MatchJob* one, bool may_measure, int* option) {
    *option = 0;
    if (path != SFOC_CORR_AUTO && path != SFOC_CORR_IGEMM_TC) return path_serves(path, dtype) ? path : -1;
    const int family = path == SFOC_CORR_AUTO ? 0 : 1;
    if (family == 1 && dtype != SFOC_DTYPE_BF16) return -1;
    const int m = one->m, R = one->R;
    auto it = ctx->tune.find(TuneKey{dtype, m, R, family});
    const TuneEntry* te = it != ctx->tune.end() ? &it->second : nullptr;
    if (!te && may_measure && ctx->autotune && !capturing(ctx->stream)) te = autotune_pair(ctx, dtype, family, *one);
    if (te) {
        *option = te->option;
        return te->path;
    }
    return auto_rule(dtype, m, R, family);
}

}  // namespace sfoc

namespace {

template <typename T>
sfoc_status build_cube(sfoc_ctx* ctx, const T* d_image, int H, int W, size_t pitch_elems, const double* scales,
                       int n_scales, int n_orient, const sfoc_params* pin, sfoc_cube** out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!d_image || !out) return fail(ctx, SFOC_ERR_INVALID_ARG, "null image or output pointer");
    if (H <= 0 || W <= 0) return fail(ctx, SFOC_ERR_SHAPE, "image must be at least 1 x 1");
    if (pitch_elems < (size_t)W) return fail(ctx, SFOC_ERR_SHAPE, "pitch_elems < W");
    if ((size_t)H * (size_t)W > ((size_t)1 << 31)) return fail(ctx, SFOC_ERR_UNSUPPORTED, "image larger than 2^31 pixels");
    sfoc_params p;
    if (pin) p = *pin;
    else sfoc_params_default(&p);
    if (scales) {
        if (n_scales < 1 || n_scales > kMaxScales) return fail(ctx, SFOC_ERR_UNSUPPORTED, "n_scales must be 1..4");
        p.n_scales = n_scales;
        for (int s = 0; s < n_scales; ++s) p.scales[s] = scales[s];
    }
    if (n_orient > 0) p.n_orient = n_orient;
    sfoc_status s = check_params(ctx, p);
    if (s != SFOC_OK) return s;
    const int z = p.first_order_only ? p.n_orient : 2 * p.n_orient;
    DeviceGuard g(ctx->device);

    sfoc_cube* cube = *out;
    bool reuse = cube && cube->c.H == H && cube->c.W == W && cube->c.z == z && cube->c.dtype == p.cube_dtype &&
                 cube->c.device == ctx->device;
    if (!reuse) {
        cube = new (std::nothrow) sfoc_cube();
        if (!cube) return fail(ctx, SFOC_ERR_OOM, "host allocation");
        s = alloc_cube(ctx, cube->c, H, W, z, p.cube_dtype);
        if (s != SFOC_OK) {
            delete cube;
            return s;
        }
    }
    const size_t fpitch = roundup((size_t)W, 32);
    s = ensure_ws(ctx, sizeof(float) * fpitch * (size_t)H * z);
    if (s != SFOC_OK) {
        if (!reuse) sfoc_cube_free(cube);
        return s;
    }
    float* F = static_cast<float*>(ctx->ws);
    SteerTaps st = make_steer(p);
    SmoothTaps sm = make_smooth(p);
    cudaError_t e;
    {
        StageScope sc(ctx, ST_STEER, 1);
        e = launch_sfoc_steer(d_image, H, W, pitch_elems, F, fpitch, st, z, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageScope sc(ctx, ST_SMOOTH, smooth_launch_count(sm));
        e = launch_sfoc_smooth(F, fpitch, H, W, sm, cube->c, ctx->stream);
    }
    if (e != cudaSuccess) {
        if (!reuse) sfoc_cube_free(cube);
        return cuda_fail(ctx, e, "sfoc kernels");
    }
    cube->c.integ_valid = false;
    *out = cube;
    return SFOC_OK;
}

}  // namespace

extern "C" {

sfoc_status sfoc_ctx_create(sfoc_ctx** out, int device, void* stream) {
    if (!out) return SFOC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return SFOC_ERR_CUDA;  // no driver or no device reachable
    if (device < 0 || device >= ndev) return SFOC_ERR_INVALID_ARG;
    sfoc_ctx* c = new (std::nothrow) sfoc_ctx();
    if (!c) return SFOC_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    DeviceGuard g(device);
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) {
        delete c;
        return SFOC_ERR_OOM;
    }
    cudaMemset(c->d_err, 0, sizeof(int));
    *out = c;
    return SFOC_OK;
}

sfoc_status sfoc_ctx_destroy(sfoc_ctx* ctx) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->pair_ref) sfoc_cube_free(ctx->pair_ref);
    if (ctx->pair_sen) sfoc_cube_free(ctx->pair_sen);
    cudaFree(ctx->ws);
    cudaFree(ctx->stage);
    cudaFree(ctx->d_err);
    for (auto& e : ctx->evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    if (ctx->ev_switch) cudaEventDestroy(ctx->ev_switch);
    for (auto ev : ctx->ev_wave)
        if (ev) cudaEventDestroy(ev);
    if (ctx->ev_hsfoc) cudaEventDestroy(ctx->ev_hsfoc);
    if (ctx->ev_hpts) cudaEventDestroy(ctx->ev_hpts);
    for (auto ev : ctx->ev_hdone)
        if (ev) cudaEventDestroy(ev);
    for (BatchPlan* p : ctx->plans) destroy_plan(p);
    cudaFree(ctx->hstage);
    delete ctx;
    return SFOC_OK;
}

sfoc_status sfoc_ctx_set_stream(sfoc_ctx* ctx, void* stream) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (static_cast<cudaStream_t>(stream) == ctx->stream) return SFOC_OK;
    // the workspace is reused (and regrown) by calls on the new stream: the
    // work still queued on the old one must be done with it first.  An event
    // recorded on the old stream orders it before the new one's work without
    // blocking the host; a stream being captured into a graph is refused
    // (the wait would pull the new stream into that capture)
    DeviceGuard g(ctx->device);
    cudaStreamCaptureStatus c0 = cudaStreamCaptureStatusNone, c1 = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &c0);
    cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &c1);
    if (c0 != cudaStreamCaptureStatusNone || c1 != cudaStreamCaptureStatusNone)
        return fail(ctx, SFOC_ERR_INVALID_ARG, "sfoc_ctx_set_stream during a stream capture");
    cudaError_t e = cudaSuccess;
    if (!ctx->ev_switch) e = cudaEventCreateWithFlags(&ctx->ev_switch, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_switch, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), ctx->ev_switch, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ordering the new stream after the previous one");
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SFOC_OK;
}

sfoc_status sfoc_ctx_sync(sfoc_ctx* ctx) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(error word)");
    if (h) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return fail(ctx, SFOC_ERR_TIMEOUT, "a bounded device wait expired (error word " + std::to_string(h) + ")");
    }
    return SFOC_OK;
}

sfoc_status sfoc_ctx_reserve(sfoc_ctx* ctx, size_t bytes) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return ensure_ws(ctx, bytes);
}

size_t sfoc_match_workspace_bytes(int n, int search_radius) {
    if (n < 0 || search_radius < 0) return 0;
    size_t P = (size_t)(2 * search_radius + 1) * (2 * search_radius + 1);
    return align256(sizeof(PointStat) * (size_t)n) + align256(sizeof(float) * P * (size_t)n);
}

const char* sfoc_last_error_string(const sfoc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t sfoc_ctx_launch_count(const sfoc_ctx* ctx) { return ctx ? ctx->launches : 0; }

sfoc_status sfoc_ctx_enable_timing(sfoc_ctx* ctx, int enable) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    ctx->timing = enable != 0;
    return SFOC_OK;
}

sfoc_status sfoc_ctx_stage_times(sfoc_ctx* ctx, double* ms_out, int64_t* launches_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    for (auto& ev : ctx->evs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) ctx->acc_ms[ev.stage] += ms;
        ctx->scope_ms[ev.stage].push_back(ms);
        ctx->acc_n[ev.stage] += ev.launches;
        ctx->pool.push_back(ev.a);
        ctx->pool.push_back(ev.b);
    }
    ctx->evs.clear();
    for (int i = 0; i < SFOC_NUM_STAGES; ++i) {
        if (ms_out) ms_out[i] = ctx->acc_ms[i];
        if (launches_out) launches_out[i] = ctx->acc_n[i];
    }
    return SFOC_OK;
}

sfoc_status sfoc_ctx_reset_timing(sfoc_ctx* ctx) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    double tmp[SFOC_NUM_STAGES];
    sfoc_status s = sfoc_ctx_stage_times(ctx, tmp, nullptr);
    for (int i = 0; i < SFOC_NUM_STAGES; ++i) {
        ctx->acc_ms[i] = 0.0;
        ctx->acc_n[i] = 0;
        ctx->scope_ms[i].clear();
    }
    return s;
}

sfoc_status sfoc_ctx_stage_scopes(sfoc_ctx* ctx, int stage, float* ms_out, int cap, int* n_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (stage < 0 || stage >= SFOC_NUM_STAGES || !n_out || cap < 0)
        return fail(ctx, SFOC_ERR_INVALID_ARG, "bad stage or output");
    double tmp[SFOC_NUM_STAGES];
    sfoc_status s = sfoc_ctx_stage_times(ctx, tmp, nullptr);  // collects the pending events
    if (s != SFOC_OK) return s;
    const std::vector<float>& v = ctx->scope_ms[stage];
    *n_out = (int)v.size();
    for (int i = 0; i < (int)v.size() && i < cap && ms_out; ++i) ms_out[i] = v[i];
    return SFOC_OK;
}

sfoc_status sfoc_measure_peaks(sfoc_ctx* ctx, sfoc_peaks* out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!out) return fail(ctx, SFOC_ERR_INVALID_ARG, "null output");
    DeviceGuard g(ctx->device);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceGetAttribute");
    sfoc_peaks r = {0.0, 0.0, 0.0, 0.0};
    ctx->launches += 4 * 6;
    e = measure_peaks(ctx->stream, sms, &r.fp32_tflops, &r.fp32x2_tflops, &r.fp64_tflops, &r.hbm_copy_gbs);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "peak microbenchmarks");
    *out = r;
    return SFOC_OK;
}

sfoc_status sfoc_ctx_selftest_timeout(sfoc_ctx* ctx, int limit_us) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (limit_us < 1 || limit_us > 100000) return fail(ctx, SFOC_ERR_INVALID_ARG, "limit_us must be in [1, 100000]");
    DeviceGuard g(ctx->device);
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, 1);
        e = launch_wait_selftest(ctx->d_err, limit_us, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "self-test launch");
    return SFOC_OK;
}

sfoc_status sfoc_params_default(sfoc_params* p) {
    if (!p) return SFOC_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->n_scales = 3;
    p->scales[0] = 0.6;
    p->scales[1] = 0.8;
    p->scales[2] = 1.0;
    p->sigma2 = 1.5;
    p->n_orient = 6;
    p->n_dil = 3;
    p->dil[0] = 1;
    p->dil[1] = 2;
    p->dil[2] = 3;
    p->sigma_d1 = 1.0;
    p->sigma_d2 = 1.5;
    p->eps = 1e-3;
    p->rectify = 1;
    p->radius_mult = 3.0;
    p->first_order_only = 0;
    p->cube_dtype = SFOC_DTYPE_F32;
    return SFOC_OK;
}

sfoc_status sfoc_build(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems, const double* scales,
                       int n_scales, int n_orient, const sfoc_params* pin, sfoc_cube** out) {
    return build_cube(ctx, d_image, H, W, pitch_elems, scales, n_scales, n_orient, pin, out);
}

sfoc_status sfoc_build_u16(sfoc_ctx* ctx, const uint16_t* d_image, int H, int W, size_t pitch_elems,
                           const sfoc_params* p, sfoc_cube** out) {
    return build_cube(ctx, d_image, H, W, pitch_elems, nullptr, 0, 0, p, out);
}

sfoc_status sfoc_cube_info(const sfoc_cube* cube, int* z, int* H, int* W, int* dtype) {
    if (!cube) return SFOC_ERR_INVALID_ARG;
    if (z) *z = cube->c.z;
    if (H) *H = cube->c.H;
    if (W) *W = cube->c.W;
    if (dtype) *dtype = cube->c.dtype;
    return SFOC_OK;
}

sfoc_status sfoc_cube_view(const sfoc_cube* cube, void** d_data, int* z, int* H, int* W, size_t* pitch, int* dtype) {
    if (!cube) return SFOC_ERR_INVALID_ARG;
    const Cube& c = cube->c;
    if (d_data) *d_data = c.dtype == SFOC_DTYPE_BF16 ? static_cast<void*>(c.rm) : static_cast<void*>(c.f32);
    if (z) *z = c.z;
    if (H) *H = c.H;
    if (W) *W = c.W;
    if (pitch) *pitch = c.dtype == SFOC_DTYPE_BF16 ? (size_t)c.W : c.pitch;
    if (dtype) *dtype = c.dtype;
    return SFOC_OK;
}

sfoc_status sfoc_cube_export(sfoc_ctx* ctx, const sfoc_cube* cube, float* d_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!cube || !d_out) return fail(ctx, SFOC_ERR_INVALID_ARG, "null cube or output");
    DeviceGuard g(ctx->device);
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, 1);
        e = launch_cube_export(cube->c, d_out, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "export launch");
    return SFOC_OK;
}

sfoc_status sfoc_fast_blocks(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems, float threshold,
                             int grid_y, int grid_x, int margin, int32_t* d_points, float* d_scores) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!d_image || !d_points || !d_scores) return fail(ctx, SFOC_ERR_INVALID_ARG, "null pointer");
    if (H < 1 || W < 1 || pitch_elems < (size_t)W) return fail(ctx, SFOC_ERR_INVALID_ARG, "bad image shape");
    if (grid_y < 1 || grid_y > H || grid_x < 1 || grid_x > W || grid_y > 65535)
        return fail(ctx, SFOC_ERR_INVALID_ARG, "grid sizes must be in [1, H] and [1, W]");
    if (margin < 0 || !(threshold >= 0.f) || !std::isfinite(threshold))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "margin >= 0 and a finite threshold >= 0 required");
    DeviceGuard g(ctx->device);
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, 1);
        e = launch_fast_blocks(d_image, H, W, pitch_elems, threshold, grid_y, grid_x, margin, d_points, d_scores,
                               ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fast launch");
    return SFOC_OK;
}

sfoc_status sfoc_rectify(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems, const double* d_model,
                         float fill, int out_h, int out_w, float* d_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!d_image || !d_model || !d_out) return fail(ctx, SFOC_ERR_INVALID_ARG, "null pointer");
    if (H < 1 || W < 1 || out_h < 1 || out_w < 1 || pitch_elems < (size_t)W || out_h > 65535 * 8)
        return fail(ctx, SFOC_ERR_INVALID_ARG, "bad image shape");
    DeviceGuard g(ctx->device);
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, 1);
        e = launch_rectify(d_image, H, W, pitch_elems, d_model, fill, out_h, out_w, d_out, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rectify launch");
    return SFOC_OK;
}

sfoc_status fastncc_points_from_results(sfoc_ctx* ctx, const int32_t* d_points, const fastncc_result* d_results,
                                        int n, double* d_src, double* d_dst, uint8_t* d_valid) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, SFOC_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!d_points || !d_results || !d_src || !d_dst || !d_valid))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "null pointer");
    if (n == 0) return SFOC_OK;
    DeviceGuard g(ctx->device);
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, 1);
        e = launch_results_to_points(d_points, d_results, n, d_src, d_dst, d_valid, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "points launch");
    return SFOC_OK;
}

sfoc_status fastncc_ransac(sfoc_ctx* ctx, const double* d_src, const double* d_dst, const uint8_t* d_valid, int n,
                           int model, const int32_t* d_samples, int n_hyp, double threshold, int refits,
                           double* d_model, uint8_t* d_inlier, int32_t* d_info, int32_t* d_scores) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (n < 0 || n_hyp < 0 || refits < 0) return fail(ctx, SFOC_ERR_INVALID_ARG, "n, n_hyp and refits must be >= 0");
    if (!(threshold >= 0.0) || !std::isfinite(threshold))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "threshold must be finite and >= 0");
    if (model != SFOC_MODEL_AFFINE && model != SFOC_MODEL_PROJECTIVE)
        return fail(ctx, SFOC_ERR_INVALID_ARG, "unknown model");
    if (!d_model || !d_info || (n > 0 && (!d_src || !d_dst || !d_inlier)) || (n_hyp > 0 && !d_samples))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "null pointer");
    DeviceGuard g(ctx->device);
    sfoc_status s = ensure_ws(ctx, ransac_workspace_bytes(n_hyp));
    if (s != SFOC_OK) return s;
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, n_hyp > 0 ? 3 : 2);
        int nl = 0;
        e = launch_ransac(d_src, d_dst, d_valid, n, model == SFOC_MODEL_PROJECTIVE ? 1 : 0, d_samples, n_hyp,
                          threshold, refits, d_model, d_inlier, d_info, d_scores, ctx->ws, ctx->stream, &nl);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ransac launch");
    return SFOC_OK;
}

sfoc_status sfoc_cube_export_integral(sfoc_ctx* ctx, sfoc_cube* cube, double* d_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!cube || !d_out) return fail(ctx, SFOC_ERR_INVALID_ARG, "null cube or output");
    DeviceGuard g(ctx->device);
    sfoc_status s = build_integral(ctx, cube->c);
    if (s != SFOC_OK) return s;
    const Cube& c = cube->c;
    s = ensure_ws(ctx, integral_export_scratch_bytes(c.H, c.W));
    if (s != SFOC_OK) return s;
    cudaError_t e;
    {
        StageScope sc(ctx, ST_OTHER, 3);
        e = launch_integral_export(c, ctx->ws, d_out, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "integral export launch");
    return SFOC_OK;
}

sfoc_status sfoc_cube_free(sfoc_cube* cube) {
    if (!cube) return SFOC_ERR_INVALID_ARG;
    DeviceGuard g(cube->c.device);
    free_cube_mem(cube->c);
    delete cube;
    return SFOC_OK;
}

sfoc_status fastncc_match(sfoc_ctx* ctx, sfoc_cube* ref, sfoc_cube* sen, const int32_t* d_points, int n,
                          int template_size, int search_radius, const fastncc_opts* opts, fastncc_result* d_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!ref || !sen) return fail(ctx, SFOC_ERR_INVALID_ARG, "null cube");
    if (n < 0) return fail(ctx, SFOC_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!d_points || !d_out)) return fail(ctx, SFOC_ERR_INVALID_ARG, "null points or output");
    if (template_size < 1 || search_radius < 0) return fail(ctx, SFOC_ERR_INVALID_ARG, "m >= 1 and R >= 0 required");
    if (template_size > kMaxTemplate || search_radius > kMaxRadius)
        return fail(ctx, SFOC_ERR_UNSUPPORTED, "m <= 128 and R <= 63");
    if (ref->c.z != sen->c.z) return fail(ctx, SFOC_ERR_SHAPE, "cubes have different channel counts");
    if (ref->c.dtype != sen->c.dtype) return fail(ctx, SFOC_ERR_SHAPE, "cubes have different dtypes");
    int path = opts ? opts->corr_path : SFOC_CORR_AUTO;
    if (path < SFOC_CORR_AUTO || path > SFOC_CORR_FFT) return fail(ctx, SFOC_ERR_INVALID_ARG, "unknown corr_path");
    const int dtype = ref->c.dtype;
    const bool f32_cube = dtype == SFOC_DTYPE_F32;
    const int m = template_size, R = search_radius;
    if (path == SFOC_CORR_IGEMM_TC) {
        if (f32_cube) return fail(ctx, SFOC_ERR_UNSUPPORTED, "tensor-core paths need BF16 cubes");
        if (auto_rule(SFOC_DTYPE_BF16, m, R, 1) < 0)
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "no tensor-core form runs for this m / R");
    } else if (path == SFOC_CORR_AUTO) {
        if (auto_rule(dtype, m, R, 0) < 0) return fail(ctx, SFOC_ERR_UNSUPPORTED, "no correlation form runs for this m / R");
    } else if (!path_serves(path, dtype)) {
        return fail(ctx, SFOC_ERR_UNSUPPORTED,
                    f32_cube ? "tensor-core paths need BF16 cubes" : "DIRECT_F32 needs F32 cubes");
    }
    DeviceGuard g(ctx->device);
    if (n == 0) return SFOC_OK;

    // integral images of the searched (reference) cube; the template sums
    // come straight from the sensed cube's sum planes
    sfoc_status s = build_integral(ctx, ref->c);
    if (s != SFOC_OK) return s;
    s = ensure_ws(ctx, sfoc_match_workspace_bytes(n, search_radius));
    if (s != SFOC_OK) return s;
    char* w = static_cast<char*>(ctx->ws);
    PointStat* stats = reinterpret_cast<PointStat*>(w);
    float* maps = reinterpret_cast<float*>(w + align256(sizeof(PointStat) * (size_t)n));
    MatchJob one = make_job(ref->c, sen->c, d_points, n, m, R, stats, maps, opts ? opts->d_maps : nullptr, d_out);
    const ItemSet none;
    cudaError_t e;
    {
        StageScope sc(ctx, ST_STATS, 1);
        e = launch_template_stats(one, none, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "template stats launch");
    // AUTO / IGEMM_TC: the measured choice for (dtype, m, R), looked up or
    // measured now on this call's points (not inside a capture: the
    // measurement waits for its events); the fixed rule where there is neither
    int option = 0;
    path = resolve_path(ctx, path, dtype, &one, true, &option);
    if (path < 0) return fail(ctx, SFOC_ERR_UNSUPPORTED, "no correlation form runs for this m / R");
    one.centered = centered_path(path) ? 1 : 0;
    {
        StageScope sc(ctx, ST_CORR, 1);
        e = launch_corr_path(ctx, path, option, one);
    }
    if (e == cudaErrorInvalidValue || e == cudaErrorNotSupported) {
        (void)cudaGetLastError();  // a refused attribute or launch leaves no error for later calls
        return fail(ctx, SFOC_ERR_UNSUPPORTED, "correlation kernel does not support this m / R");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "correlation launch");
    {
        StageScope sc(ctx, ST_NCC, 1);
        e = launch_ncc_argmax(one, none, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ncc launch");
    return SFOC_OK;
}

sfoc_status fastncc_register_pair(sfoc_ctx* ctx, const float* d_ref, int Hr, int Wr, const float* d_sen, int Hs,
                                  int Ws, const int32_t* d_points, int n, int template_size, int search_radius,
                                  const sfoc_params* p, const fastncc_opts* opts, fastncc_result* d_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    sfoc_status s = sfoc_build(ctx, d_ref, Hr, Wr, (size_t)Wr, nullptr, 0, 0, p, &ctx->pair_ref);
    if (s != SFOC_OK) return s;
    s = sfoc_build(ctx, d_sen, Hs, Ws, (size_t)Ws, nullptr, 0, 0, p, &ctx->pair_sen);
    if (s != SFOC_OK) return s;
    return fastncc_match(ctx, ctx->pair_ref, ctx->pair_sen, d_points, n, template_size, search_radius, opts, d_out);
}

sfoc_status fastncc_register_pair_host(sfoc_ctx* ctx, const float* h_ref, int Hr, int Wr, const float* h_sen,
                                       int Hs, int Ws, const int32_t* h_points, int n, int template_size,
                                       int search_radius, const sfoc_params* p, const fastncc_opts* opts,
                                       fastncc_result* h_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!h_ref || !h_sen || (n > 0 && (!h_points || !h_out)))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "null host buffer");
    if (Hr <= 0 || Wr <= 0 || Hs <= 0 || Ws <= 0 || n < 0) return fail(ctx, SFOC_ERR_SHAPE, "bad sizes");
    DeviceGuard g(ctx->device);
    size_t b_ref = align256(sizeof(float) * (size_t)Hr * Wr), b_sen = align256(sizeof(float) * (size_t)Hs * Ws);
    size_t b_pts = align256(sizeof(int32_t) * 2 * (size_t)n), b_out = align256(sizeof(fastncc_result) * (size_t)n);
    size_t need = b_ref + b_sen + b_pts + b_out;
    if (need > ctx->stage_bytes) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
        cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        e = cudaMalloc(&ctx->stage, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(staging)");
        ctx->stage_bytes = need;
    }
    char* b = static_cast<char*>(ctx->stage);
    float* d_ref = reinterpret_cast<float*>(b);
    float* d_sen = reinterpret_cast<float*>(b + b_ref);
    int32_t* d_pts = reinterpret_cast<int32_t*>(b + b_ref + b_sen);
    fastncc_result* d_out = reinterpret_cast<fastncc_result*>(b + b_ref + b_sen + b_pts);
    cudaError_t e = cudaSuccess;
    // each created on first use (the batched host path shares the stream)
    if (!ctx->copy_stream) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->ev_start) e = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->ev_copied) e = cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
    // the reference image on the context stream, the sensed image and the
    // points on the copy stream (after everything queued before this call):
    // the sensed copy lands while the reference cube is built
    e = cudaEventRecord(ctx->ev_start, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_start, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ref, h_ref, sizeof(float) * (size_t)Hr * Wr, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_sen, h_sen, sizeof(float) * (size_t)Hs * Ws, cudaMemcpyHostToDevice, ctx->copy_stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(d_pts, h_points, sizeof(int32_t) * 2 * (size_t)n, cudaMemcpyHostToDevice,
                            ctx->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copied, ctx->copy_stream);
    // the call is synchronous on every path: once copies from the caller's
    // buffers are queued, a failure still waits for them before returning
    auto drained = [&](sfoc_status st) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamSynchronize(ctx->stream);
        (void)cudaGetLastError();
        return st;
    };
    if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "host to device copy"));
    sfoc_status s = sfoc_build(ctx, d_ref, Hr, Wr, (size_t)Wr, nullptr, 0, 0, p, &ctx->pair_ref);
    if (s != SFOC_OK) return drained(s);
    e = cudaStreamWaitEvent(ctx->stream, ctx->ev_copied, 0);
    if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "cudaStreamWaitEvent"));
    s = sfoc_build(ctx, d_sen, Hs, Ws, (size_t)Ws, nullptr, 0, 0, p, &ctx->pair_sen);
    if (s == SFOC_OK)
        s = fastncc_match(ctx, ctx->pair_ref, ctx->pair_sen, d_pts, n, template_size, search_radius, opts, d_out);
    if (s != SFOC_OK) return drained(s);
    if (n > 0) {
        e = cudaMemcpyAsync(h_out, d_out, sizeof(fastncc_result) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "device to host copy"));
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    return SFOC_OK;
}

sfoc_status sfoc_ctx_set_autotune(sfoc_ctx* ctx, int enable) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    ctx->autotune = enable != 0;
    return SFOC_OK;
}

sfoc_status sfoc_ctx_autotune_entry(const sfoc_ctx* ctx, int dtype, int m, int R, int family, int* corr_path,
                                    int* option, int* n_cand, int* cand_path, int* cand_option, float* cand_ms,
                                    int* sample) {
    if (!ctx || !corr_path) return SFOC_ERR_INVALID_ARG;
    auto it = ctx->tune.find(TuneKey{dtype, m, R, family});
    if (it == ctx->tune.end()) {
        *corr_path = -1;
        if (n_cand) *n_cand = 0;
        return SFOC_OK;
    }
    const TuneEntry& t = it->second;
    *corr_path = t.path;
    if (option) *option = t.option;
    if (n_cand) *n_cand = t.n_cand;
    if (sample) *sample = t.sample;
    for (int i = 0; i < t.n_cand; ++i) {
        if (cand_path) cand_path[i] = t.cand_path[i];
        if (cand_option) cand_option[i] = t.cand_option[i];
        if (cand_ms) cand_ms[i] = t.cand_ms[i];
    }
    return SFOC_OK;
}

sfoc_status sfoc_ctx_autotune_export(const sfoc_ctx* ctx, char* buf, size_t cap, size_t* len) {
    if (!ctx || !len) return SFOC_ERR_INVALID_ARG;
    std::string j = "{\"sfoc_autotune\": 1, \"entries\": [";
    bool first = true;
    char tmp[256];
    for (const auto& kv : ctx->tune) {
        const TuneEntry& t = kv.second;
        snprintf(tmp, sizeof(tmp), "%s{\"dtype\": %d, \"family\": %d, \"m\": %d, \"R\": %d, \"path\": %d, "
                 "\"option\": %d, \"sample\": %d, \"candidates\": [", first ? "" : ", ", kv.first.dtype,
                 kv.first.family, kv.first.m, kv.first.R, t.path, t.option, t.sample);
        j += tmp;
        for (int i = 0; i < t.n_cand; ++i) {
            snprintf(tmp, sizeof(tmp), "%s[%d, %d, %.6g]", i ? ", " : "", t.cand_path[i], t.cand_option[i],
                     (double)t.cand_ms[i]);
            j += tmp;
        }
        j += "]}";
        first = false;
    }
    j += "]}";
    *len = j.size() + 1;
    if (!buf) return SFOC_OK;
    if (cap < j.size() + 1) return SFOC_ERR_INVALID_ARG;
    memcpy(buf, j.c_str(), j.size() + 1);
    return SFOC_OK;
}

namespace {

// the integer after `"key":` inside [p, end); false when absent
bool json_int(const char* p, const char* end, const char* key, int* out) {
    std::string k = std::string("\"") + key + "\"";
    const char* q = std::search(p, end, k.begin(), k.end());
    if (q == end) return false;
    q += k.size();
    while (q < end && (*q == ' ' || *q == ':')) ++q;
    char* e = nullptr;
    long v = strtol(q, &e, 10);
    if (e == q) return false;
    *out = (int)v;
    return true;
}

}  // namespace

sfoc_status sfoc_ctx_autotune_import(sfoc_ctx* ctx, const char* text) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!text) return fail(ctx, SFOC_ERR_INVALID_ARG, "null text");
    const char* p = strstr(text, "\"entries\"");
    if (!p) return fail(ctx, SFOC_ERR_INVALID_ARG, "no entries in the autotune text");
    std::map<TuneKey, TuneEntry> got;
    // each entry is an object from "{" to the "]}" that closes its candidates
    while ((p = strstr(p, "{\"dtype\"")) != nullptr) {
        const char* end = strstr(p, "]}");
        if (!end) return fail(ctx, SFOC_ERR_INVALID_ARG, "unterminated autotune entry");
        TuneEntry t;
        memset(&t, 0, sizeof(t));
        int dtype, m, R, family = 0;
        if (!json_int(p, end, "dtype", &dtype) || !json_int(p, end, "m", &m) || !json_int(p, end, "R", &R) ||
            !json_int(p, end, "path", &t.path) || !json_int(p, end, "option", &t.option))
            return fail(ctx, SFOC_ERR_INVALID_ARG, "autotune entry without dtype, m, R, path or option");
        json_int(p, end, "sample", &t.sample);
        json_int(p, end, "family", &family);
        const bool ok_path = t.path == SFOC_CORR_DIRECT_F32 || t.path == SFOC_CORR_FFT || t.path == SFOC_CORR_TC_TOEPLITZ ||
                             t.path == SFOC_CORR_TC_COLUMN || t.path == SFOC_CORR_TC_BAND;
        if (!ok_path || (dtype != SFOC_DTYPE_F32 && dtype != SFOC_DTYPE_BF16) || !path_serves(t.path, dtype) ||
            (family != 0 && family != 1) || (family == 1 && (dtype != SFOC_DTYPE_BF16 || centered_path(t.path))) ||
            m < 1 || m > kMaxTemplate || R < 0 || R > kMaxRadius)
            return fail(ctx, SFOC_ERR_INVALID_ARG, "autotune entry out of range");
        const int opt = t.path == SFOC_CORR_FFT ? t.option : 0;
        if (t.path == SFOC_CORR_FFT && (opt != 64 && opt != 128)) return fail(ctx, SFOC_ERR_INVALID_ARG, "bad FFT side");
        // the entry must name a form that runs for (m, R)
        if (t.path == SFOC_CORR_FFT ? (!corr_fft_supported(m, R) || m + 2 * R > opt)
            : t.path == SFOC_CORR_DIRECT_F32 ? !corr_f32_supported(m, R)
                                             : corr_tc_class(t.path == SFOC_CORR_TC_TOEPLITZ ? 1
                                                             : t.path == SFOC_CORR_TC_COLUMN ? 2 : 3, m, R) == 0)
            return fail(ctx, SFOC_ERR_INVALID_ARG, "autotune entry names a form that does not run for its m / R");
        got[TuneKey{dtype, m, R, family}] = t;
        p = end + 2;
    }
    for (const auto& kv : got) ctx->tune[kv.first] = kv.second;
    return SFOC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sfoc_build_static: the SFOC build with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory at the moment they need a
// descriptor: a service that sizes every allocation up front and holds a
// hard memory cap, or a real-time loop that must not take cudaMalloc's
// device-wide synchronisation.  This entry point serves them: the
// steering responses (the only scratch of the build) go to the array below,
// the cube goes to the caller's buffer, and nothing is allocated.
//
// The array is 2^24 floats (64 MiB).  It holds the z steering planes
// (rows padded to 32 floats) followed by the two per-pixel sum planes the
// smoothing pass writes; nothing in it has to start at zero, because the
// steering pass writes every element the smoothing pass reads and the sum
// planes are stored, not accumulated.  There is one array per device, so
// calls that overlap in time (two streams, two threads) race on it, and it
// keeps the last call's contents until the next call.
// ---------------------------------------------------------------------------
static __device__ __align__(256) float g_static_scratch[SFOC_STATIC_SCRATCH_FLOATS];

namespace {

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
float* g_static_ptr[kMaxStaticDevices] = {nullptr};

// Address of this device's array; the first call on a device looks it up
// (with that device current) and remembers it.
cudaError_t static_scratch(int device, float** out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[device] = static_cast<float*>(ptr);
    }
    *out = g_static_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" {

sfoc_status sfoc_build_static(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems,
                              const sfoc_params* pin, float* d_out) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!d_image || !d_out) return fail(ctx, SFOC_ERR_INVALID_ARG, "null image or output pointer");
    if (H <= 0 || W <= 0) return fail(ctx, SFOC_ERR_SHAPE, "image must be at least 1 x 1");
    if (pitch_elems < (size_t)W) return fail(ctx, SFOC_ERR_SHAPE, "pitch_elems < W");
    if (ctx->device < 0 || ctx->device >= kMaxStaticDevices)
        return fail(ctx, SFOC_ERR_UNSUPPORTED, "device index beyond the static scratch table");
    sfoc_params p;
    if (pin) p = *pin;
    else sfoc_params_default(&p);
    if (p.cube_dtype != SFOC_DTYPE_F32) return fail(ctx, SFOC_ERR_UNSUPPORTED, "sfoc_build_static writes F32 cubes only");
    sfoc_status s = check_params(ctx, p);
    if (s != SFOC_OK) return s;
    const int z = p.first_order_only ? p.n_orient : 2 * p.n_orient;
    const size_t fpitch = roundup((size_t)W, 32);
    const size_t f_floats = fpitch * (size_t)H * z;
    const size_t need = f_floats + 2 * (size_t)H * W;
    if ((size_t)H * W > ((size_t)1 << 31) || need > (size_t)SFOC_STATIC_SCRATCH_FLOATS)
        return fail(ctx, SFOC_ERR_UNSUPPORTED,
                    "image too large for the static scratch: needs " + std::to_string(need) + " floats, holds " +
                        std::to_string((size_t)SFOC_STATIC_SCRATCH_FLOATS));
    DeviceGuard g(ctx->device);
    float* F = nullptr;
    cudaError_t e = static_scratch(ctx->device, &F);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(static scratch)");
    Cube c;
    c.H = H;
    c.W = W;
    c.z = z;
    c.dtype = SFOC_DTYPE_F32;
    c.pitch = (size_t)W;  // dense [z][H][W], the layout sfoc_cube_export writes
    c.ipitch = (size_t)W + 1;
    c.device = ctx->device;
    c.f32 = d_out;
    c.s1 = F + f_floats;
    c.s2 = c.s1 + (size_t)H * W;
    const SteerTaps st = make_steer(p);
    const SmoothTaps sm = make_smooth(p);
    ctx->launches += 1 + smooth_launch_count(sm);
    e = launch_sfoc_steer(d_image, H, W, pitch_elems, F, fpitch, st, z, ctx->stream);
    if (e == cudaSuccess) e = launch_sfoc_smooth(F, fpitch, H, W, sm, c, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sfoc kernels");
    return SFOC_OK;
}

}  // extern "C"
