// Batched forms of the path over many image pairs of uneven size, point
// count, template size and search radius (the per-point loop of Sec. 3.2.2
// and the per-pair loop around it, as launches over all of them at once).
//
// A plan holds everything one distinct call needs: the device tables of
// images (SFOC), cubes (integral images) and match jobs, the list of all
// (pair, point) items (template statistics, NCC), and per correlation class
// (one kernel instance: the Fourier side, the direct kernel's tile class or
// a tensor-core form's instance) the items it takes, sorted by decreasing
// cost per point.  Each stage is then one launch over the whole batch and
// each correlation class one persistent launch (the Fourier kernel's CTAs
// take items from an atomic counter; the tensor-core kernels stride over
// the cost-sorted list).  The first call with a new signature runs its
// stages eagerly (measuring the correlation form of every (m, R) that has
// no autotuned entry yet, on that pair's own points) and captures the same
// launches into a CUDA graph, on a private stream; later calls with the same
// signature replay the graph on the context's stream.  Plans live in the
// context (the most recent few) and point into its workspace, so a
// workspace that has to grow drops them.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "host.h"

namespace sfoc {

namespace {

constexpr size_t kFBudget = (size_t)4 << 30;  // steering planes of one SFOC wave

struct Wave {
    int img0 = 0, n_img = 0;
    int steer_ctas = 0, smooth_ctas = 0;
    size_t tab = 0, steer_begin = 0, smooth_begin = 0;  // offsets in the plan's device buffer
};

struct CorrClass {
    int path = 0, cls = 0;          // concrete sfoc_corr_path and its kernel class (FFT: side, direct: tiles)
    std::vector<int> ms, Rs;        // distinct (m, R) of its pairs
    std::vector<int> pairs;         // its pairs, by decreasing cost per point
    size_t items = 0;               // offset of its item list in the device buffer
    int n_items = 0;
    int max_m = 0, max_R = 0, max_lw = 0;
    int queue = -1;                 // its counter (Fourier form), or -1
    int msplit = 0;                 // tensor-core forms: the template size of its pairs
};

}  // namespace

struct BatchPlan {
    int kind = 0;  // 0 build, 1 match, 2 register
    std::vector<uint64_t> key;
    char* dbuf = nullptr;
    size_t dbuf_bytes = 0;
    // SFOC build
    std::vector<sfoc_cube*> own;     // cubes owned by the plan (register)
    std::vector<sfoc_cube*> cubes;   // cubes built (build, register)
    SteerTaps st;
    SmoothTaps sm;
    bool build_batched = true;
    std::vector<ImgJob> img;         // host copies (per-image fallback)
    std::vector<Wave> waves;
    // integral images
    std::vector<Cube*> int_cubes;
    size_t int_blob = 0;
    int int_ctas[4] = {0, 0, 0, 0};
    // match
    std::vector<MatchJob> jobs;      // host copies (Toeplitz launches take them by value)
    size_t d_jobs = 0, d_items = 0, d_queues = 0;
    int n_items = 0, max_R = 0, n_queues = 0;
    std::vector<CorrClass> classes;
    int dtype = 0;                   // the cubes' dtype (every pair alike)
    // graph of the whole call
    cudaGraphExec_t exec = nullptr;
    int launches = 0;                // kernel launches per run
};

void destroy_plan(BatchPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (sfoc_cube* c : p->own) sfoc_cube_free(c);
    if (p->dbuf) cudaFree(p->dbuf);
    delete p;
}

namespace {

// ---- plan keys -------------------------------------------------------------

struct KeyWriter {
    std::vector<uint64_t> k;
    void u(uint64_t v) { k.push_back(v); }
    void p(const void* v) { k.push_back((uint64_t)(uintptr_t)v); }
};

BatchPlan* find_plan(sfoc_ctx* ctx, const std::vector<uint64_t>& key) {
    for (size_t i = 0; i < ctx->plans.size(); ++i)
        if (ctx->plans[i]->key == key) {
            BatchPlan* p = ctx->plans[i];  // most recently used goes last
            ctx->plans.erase(ctx->plans.begin() + i);
            ctx->plans.push_back(p);
            return p;
        }
    return nullptr;
}

void keep_plan(sfoc_ctx* ctx, BatchPlan* p) {
    while (ctx->plans.size() >= ctx->max_plans && !ctx->plans.empty()) {
        // the oldest plan may still be in use by queued work
        cudaStreamSynchronize(ctx->stream);
        destroy_plan(ctx->plans.front());
        ctx->plans.erase(ctx->plans.begin());
    }
    ctx->plans.push_back(p);
}

// ---- device buffer layout ----------------------------------------------------

struct Layout {
    size_t bytes = 0;
    size_t add(size_t n, size_t align = 256) {
        bytes = roundup(bytes, align);
        const size_t at = bytes;
        bytes += n;
        return at;
    }
};

// per-point cost of a pair in its form (a relative figure: items are sorted
// by it, largest first)
double point_cost(int m, int R) { return (double)m * m * (2.0 * R + 1) * (2.0 * R + 1); }

int tc_form(int path) {
    return path == SFOC_CORR_TC_TOEPLITZ ? 1 : path == SFOC_CORR_TC_COLUMN ? 2 : path == SFOC_CORR_TC_BAND ? 3 : 0;
}

// kernel class of a pair in a concrete form (0 = the form does not run)
int class_of(int path, int option, int m, int R) {
    switch (path) {
        case SFOC_CORR_FFT:
            if (!corr_fft_supported(m, R)) return 0;
            return option ? option : corr_fft_side(m, R);
        case SFOC_CORR_DIRECT_F32: return corr_f32_supported(m, R) ? corr_f32_class(R) : 0;
        default: return corr_tc_class(tc_form(path), m, R);
    }
}

// ---- stages ------------------------------------------------------------------

cudaError_t enqueue_build(sfoc_ctx* ctx, BatchPlan* p, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (p->build_batched) {
        for (const Wave& w : p->waves) {
            StageScope sc(ctx, ST_STEER, 3);
            e = launch_sfoc_batch(reinterpret_cast<const ImgJob*>(p->dbuf + w.tab), w.n_img,
                                  reinterpret_cast<const int*>(p->dbuf + w.steer_begin), w.steer_ctas,
                                  reinterpret_cast<const int*>(p->dbuf + w.smooth_begin), w.smooth_ctas, p->st, p->sm,
                                  s);
            if (e != cudaSuccess) return e;
        }
        return e;
    }
    for (size_t i = 0; i < p->img.size(); ++i) {  // parameters without a batched kernel: one image at a time
        const ImgJob& j = p->img[i];
        StageScope sc(ctx, ST_STEER, 1 + smooth_launch_count(p->sm));
        e = launch_sfoc_steer(static_cast<const float*>(j.img), j.H, j.W, j.pitch, j.F, j.fpitch, p->st, 0, s);
        if (e == cudaSuccess) e = launch_sfoc_smooth(j.F, j.fpitch, j.H, j.W, p->sm, p->cubes[i]->c, s);
        if (e != cudaSuccess) return e;
    }
    return e;
}

cudaError_t enqueue_match_head(sfoc_ctx* ctx, BatchPlan* p, cudaStream_t s) {
    cudaError_t e;
    {
        StageScope sc(ctx, ST_INTEGRAL, 4);
        e = launch_integral_batch(p->dbuf + p->int_blob, (int)p->int_cubes.size(), p->int_ctas, s);
    }
    if (e != cudaSuccess) return e;
    for (Cube* c : p->int_cubes) c->integ_valid = true;
    ItemSet all;
    all.jobs = reinterpret_cast<const MatchJob*>(p->dbuf + p->d_jobs);
    all.items = reinterpret_cast<const int2*>(p->dbuf + p->d_items);
    all.n = p->n_items;
    MatchJob none;
    memset(&none, 0, sizeof(none));
    StageScope sc(ctx, ST_STATS, 1);
    return launch_template_stats(none, all, s);
}

cudaError_t enqueue_match_tail(sfoc_ctx* ctx, BatchPlan* p, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    MatchJob none;
    memset(&none, 0, sizeof(none));
    const MatchJob* d_jobs = reinterpret_cast<const MatchJob*>(p->dbuf + p->d_jobs);
    if (p->n_queues > 0) {
        e = cudaMemsetAsync(p->dbuf + p->d_queues, 0, sizeof(int) * (size_t)p->n_queues, s);
        if (e != cudaSuccess) return e;
    }
    for (CorrClass& c : p->classes) {
        ItemSet is;
        is.jobs = d_jobs;
        is.items = reinterpret_cast<const int2*>(p->dbuf + c.items);
        is.n = c.n_items;
        is.max_m = c.max_m;
        is.max_R = c.max_R;
        is.max_lw = c.max_lw;
        is.queue = c.queue >= 0 ? reinterpret_cast<int*>(p->dbuf + p->d_queues) + c.queue : nullptr;
        if (c.path == SFOC_CORR_TC_TOEPLITZ) {  // one launch per pair
            for (int pi : c.pairs) {
                StageScope sc(ctx, ST_CORR, 1);
                const ItemSet single;
                const MatchJob& j = p->jobs[pi];
                e = launch_corr_tc(1, c.cls, j, single, &j.m, &j.R, 1, ctx->d_err, s);
                if (e != cudaSuccess) return e;
            }
            continue;
        }
        StageScope sc(ctx, ST_CORR, 1);
        if (c.path == SFOC_CORR_FFT) e = launch_corr_fft(none, is, c.cls, p->dtype == SFOC_DTYPE_BF16, s);
        else if (c.path == SFOC_CORR_DIRECT_F32) e = launch_corr_f32(none, is, c.cls, s);
        else e = launch_corr_tc(tc_form(c.path), c.cls, none, is, c.ms.data(), c.Rs.data(), (int)c.ms.size(),
                                ctx->d_err, s);
        if (e != cudaSuccess) return e;
    }
    ItemSet all;
    all.jobs = d_jobs;
    all.items = reinterpret_cast<const int2*>(p->dbuf + p->d_items);
    all.n = p->n_items;
    all.max_R = p->max_R;
    StageScope sc(ctx, ST_NCC, 1);
    return launch_ncc_argmax(none, all, s);
}

cudaError_t enqueue_all(sfoc_ctx* ctx, BatchPlan* p, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (p->kind != 1) e = enqueue_build(ctx, p, s);
    if (e == cudaSuccess && p->kind != 0) e = enqueue_match_head(ctx, p, s);
    if (e == cudaSuccess && p->kind != 0) e = enqueue_match_tail(ctx, p, s);
    return e;
}

// Captures the plan's launches into a graph (on a private stream; nothing
// runs during the capture).  Launch counts of the capture are not counted.
sfoc_status capture_plan(sfoc_ctx* ctx, BatchPlan* p) {
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
    const int64_t l0 = ctx->launches;
    const bool timing = ctx->timing;
    ctx->timing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_all(ctx, p, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e2 != cudaSuccess) e = e2;
    }
    ctx->timing = timing;
    p->launches = (int)(ctx->launches - l0);
    ctx->launches = l0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        p->exec = nullptr;
        return cuda_fail(ctx, e, "graph capture");
    }
    return SFOC_OK;
}

// Runs a plan: its graph when it has one and per-stage timing is off (the
// stage events need separate launches), else its launches one by one.
sfoc_status run_plan(sfoc_ctx* ctx, BatchPlan* p) {
    cudaError_t e;
    if (p->exec && !ctx->timing) {
        e = cudaGraphLaunch(p->exec, ctx->stream);
        ctx->launches += p->launches;
    } else {
        e = enqueue_all(ctx, p, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch launch");
    return SFOC_OK;
}

// ---- plan construction ---------------------------------------------------------

struct BuildIn {
    int n;
    const float* const* images;
    const int* H;
    const int* W;
    const size_t* pitch;  // may be null (dense)
};

// Allocates (or reuses) the cubes and lays out the SFOC waves; the tables
// are written into `host` at the offsets recorded in the plan.
sfoc_status plan_build(sfoc_ctx* ctx, BatchPlan* p, const BuildIn& in, const sfoc_params& prm, sfoc_cube** cubes,
                       bool own, char* ws_scratch, size_t scratch_bytes, Layout& lay) {
    p->st = make_steer(prm);
    p->sm = make_smooth(prm);
    p->build_batched = sfoc_batch_supported(p->st, p->sm);
    const int z = prm.first_order_only ? prm.n_orient : 2 * prm.n_orient;
    for (int i = 0; i < in.n; ++i) {
        sfoc_cube* c = cubes[i];
        const bool reuse = c && c->c.H == in.H[i] && c->c.W == in.W[i] && c->c.z == z && c->c.dtype == prm.cube_dtype &&
                           c->c.device == ctx->device;
        if (!reuse) {
            c = new (std::nothrow) sfoc_cube();
            if (!c) return fail(ctx, SFOC_ERR_OOM, "host allocation");
            sfoc_status s = alloc_cube(ctx, c->c, in.H[i], in.W[i], z, prm.cube_dtype);
            if (s != SFOC_OK) {
                delete c;
                return s;
            }
            if (own) p->own.push_back(c);
            cubes[i] = c;
        }
        c->c.integ_valid = false;
        p->cubes.push_back(c);
    }
    // waves of images whose steering planes fit the scratch region
    p->img.resize(in.n);
    size_t used = 0;
    Wave w;
    for (int i = 0; i < in.n; ++i) {
        const size_t fpitch = roundup((size_t)in.W[i], 32);
        const size_t fb = align256(sizeof(float) * fpitch * (size_t)in.H[i] * z);
        if (fb > scratch_bytes) return fail(ctx, SFOC_ERR_OOM, "workspace too small for one image's steering planes");
        if (used + fb > scratch_bytes && w.n_img > 0) {
            p->waves.push_back(w);
            w = Wave();
            w.img0 = i;
            used = 0;
        }
        ImgJob& j = p->img[i];
        memset(&j, 0, sizeof(j));
        const Cube& c = p->cubes[i]->c;
        j.img = in.images[i];
        j.pitch = in.pitch ? in.pitch[i] : (size_t)in.W[i];
        j.H = in.H[i];
        j.W = in.W[i];
        j.F = reinterpret_cast<float*>(ws_scratch + used);
        j.fpitch = fpitch;
        j.c32 = c.f32;
        j.cpitch = c.pitch;
        j.rm = c.rm;
        j.cm = c.cm;
        j.s1 = c.s1;
        j.s2 = c.s2;
        used += fb;
        int sc = 0, mc = 0;
        sfoc_batch_tiles(in.H[i], in.W[i], &sc, &mc);
        w.steer_ctas += sc;
        w.smooth_ctas += mc;
        ++w.n_img;
    }
    if (w.n_img > 0) p->waves.push_back(w);
    for (Wave& wv : p->waves) {
        wv.tab = lay.add(sizeof(ImgJob) * (size_t)wv.n_img);
        wv.steer_begin = lay.add(sizeof(int) * (size_t)(wv.n_img + 1));
        wv.smooth_begin = lay.add(sizeof(int) * (size_t)(wv.n_img + 1));
    }
    return SFOC_OK;
}

void write_build_tables(BatchPlan* p, char* host) {
    for (const Wave& w : p->waves) {
        memcpy(host + w.tab, p->img.data() + w.img0, sizeof(ImgJob) * (size_t)w.n_img);
        int* sb = reinterpret_cast<int*>(host + w.steer_begin);
        int* mb = reinterpret_cast<int*>(host + w.smooth_begin);
        int a = 0, b = 0;
        for (int i = 0; i < w.n_img; ++i) {
            const ImgJob& j = p->img[w.img0 + i];
            int sc = 0, mc = 0;
            sfoc_batch_tiles(j.H, j.W, &sc, &mc);
            sb[i] = a;
            mb[i] = b;
            a += sc;
            b += mc;
        }
        sb[w.n_img] = a;
        mb[w.n_img] = b;
    }
}

struct MatchIn {
    int n;
    sfoc_cube* const* refs;
    sfoc_cube* const* sens;
    const int32_t* const* pts;
    const int* npts;
    const int* m;
    const int* R;
    fastncc_result* const* outs;
};

sfoc_status check_match(sfoc_ctx* ctx, const MatchIn& in, int path) {
    int dtype = -1, z = -1;
    for (int i = 0; i < in.n; ++i) {
        const sfoc_cube* r = in.refs[i];
        const sfoc_cube* s = in.sens[i];
        if (!r || !s) return fail(ctx, SFOC_ERR_INVALID_ARG, "null cube in the batch");
        if (in.npts[i] < 0) return fail(ctx, SFOC_ERR_INVALID_ARG, "n < 0 in the batch");
        if (in.npts[i] > 0 && (!in.pts[i] || !in.outs[i])) return fail(ctx, SFOC_ERR_INVALID_ARG, "null points or output");
        if (in.m[i] < 1 || in.R[i] < 0) return fail(ctx, SFOC_ERR_INVALID_ARG, "m >= 1 and R >= 0 required");
        if (in.m[i] > kMaxTemplate || in.R[i] > kMaxRadius) return fail(ctx, SFOC_ERR_UNSUPPORTED, "m <= 128 and R <= 63");
        if (r->c.z != s->c.z || r->c.dtype != s->c.dtype) return fail(ctx, SFOC_ERR_SHAPE, "cubes of a pair differ");
        if (dtype < 0) {
            dtype = r->c.dtype;
            z = r->c.z;
        } else if (r->c.dtype != dtype || r->c.z != z) {
            return fail(ctx, SFOC_ERR_SHAPE, "every pair of a batch has the same cube dtype and channels");
        }
        if (path == SFOC_CORR_AUTO || path == SFOC_CORR_IGEMM_TC) {
            const int family = path == SFOC_CORR_AUTO ? 0 : 1;
            if (auto_rule(dtype, in.m[i], in.R[i], family) < 0)
                return fail(ctx, SFOC_ERR_UNSUPPORTED, "no correlation form of the path runs for a pair's m / R");
        } else {
            if (!path_serves(path, dtype))
                return fail(ctx, SFOC_ERR_UNSUPPORTED, "the correlation path does not serve the batch's cubes");
            if (class_of(path, 0, in.m[i], in.R[i]) == 0)
                return fail(ctx, SFOC_ERR_UNSUPPORTED, "the correlation form does not run for a pair's m / R");
        }
    }
    return SFOC_OK;
}

size_t match_ws_bytes(const MatchIn& in, size_t* maps_off, int* total) {
    size_t items = 0, maps = 0;
    for (int i = 0; i < in.n; ++i) {
        items += (size_t)in.npts[i];
        maps += (size_t)in.npts[i] * (size_t)(2 * in.R[i] + 1) * (2 * in.R[i] + 1);
    }
    *total = (int)items;
    *maps_off = align256(sizeof(PointStat) * items);
    return *maps_off + align256(sizeof(float) * maps);
}

// Jobs, the item list and the integral table (the classes come later,
// once every pair's form is known).
void plan_match_jobs(BatchPlan* p, const MatchIn& in, char* ws, size_t maps_off, char* int_scratch, Layout& lay) {
    PointStat* stats = reinterpret_cast<PointStat*>(ws);
    float* maps = reinterpret_cast<float*>(ws + maps_off);
    size_t so = 0, mo = 0;
    p->jobs.resize(in.n);
    p->n_items = 0;
    p->max_R = 0;
    for (int i = 0; i < in.n; ++i) {
        p->jobs[i] = make_job(in.refs[i]->c, in.sens[i]->c, in.pts[i], in.npts[i], in.m[i], in.R[i], stats + so,
                              maps + mo, nullptr, in.outs[i]);
        so += (size_t)in.npts[i];
        mo += (size_t)in.npts[i] * (size_t)(2 * in.R[i] + 1) * (2 * in.R[i] + 1);
        p->n_items += in.npts[i];
        if (in.npts[i] > 0 && in.R[i] > p->max_R) p->max_R = in.R[i];
    }
    // integral images of the distinct reference cubes
    for (int i = 0; i < in.n; ++i) {
        Cube* c = &in.refs[i]->c;
        if (std::find(p->int_cubes.begin(), p->int_cubes.end(), c) == p->int_cubes.end()) p->int_cubes.push_back(c);
    }
    (void)int_scratch;
    p->d_jobs = lay.add(sizeof(MatchJob) * (size_t)in.n, 128);
    p->d_items = lay.add(sizeof(int2) * (size_t)p->n_items);
    p->int_blob = lay.add(integral_batch_blob_bytes((int)p->int_cubes.size()));
}

void write_match_head(BatchPlan* p, char* host, char* int_scratch) {
    int2* it = reinterpret_cast<int2*>(host + p->d_items);
    size_t k = 0;
    for (size_t i = 0; i < p->jobs.size(); ++i)
        for (int q = 0; q < p->jobs[i].n; ++q) it[k++] = make_int2((int)i, q);
    integral_batch_blob(const_cast<const Cube* const*>(p->int_cubes.data()), (int)p->int_cubes.size(), int_scratch,
                        host + p->int_blob, p->int_ctas);
}

// The correlation form of every pair, then the classes and their item lists.
// False when a tensor map cannot be encoded for a pair.
bool plan_classes(sfoc_ctx* ctx, BatchPlan* p, int path, int dtype, Layout& lay) {
    struct Pick {
        int path, cls;
    };
    std::vector<Pick> pick(p->jobs.size());
    p->dtype = dtype;
    for (size_t i = 0; i < p->jobs.size(); ++i) {
        MatchJob& j = p->jobs[i];
        int opt = 0;
        const int pp = resolve_path(ctx, path, dtype, &j, false, &opt);
        j.centered = centered_path(pp) ? 1 : 0;
        pick[i] = {pp, class_of(pp, opt, j.m, j.R)};
    }
    // a tensor-core launch lays its shared memory out for its largest item,
    // so its classes are split by template size too: a launch of smaller
    // templates keeps smaller window tiles and a deeper template-slab ring
    p->classes.clear();
    for (size_t i = 0; i < p->jobs.size(); ++i) {
        if (p->jobs[i].n == 0) continue;
        const int msplit = tc_form(pick[i].path) ? p->jobs[i].m : 0;
        CorrClass* c = nullptr;
        for (CorrClass& cc : p->classes)
            if (cc.path == pick[i].path && cc.cls == pick[i].cls && cc.msplit == msplit) c = &cc;
        if (!c) {
            p->classes.push_back(CorrClass());
            c = &p->classes.back();
            c->path = pick[i].path;
            c->cls = pick[i].cls;
            c->msplit = msplit;
        }
        c->pairs.push_back((int)i);
    }
    p->n_queues = 0;
    for (CorrClass& c : p->classes) {
        std::stable_sort(c.pairs.begin(), c.pairs.end(), [&](int a, int b) {
            return point_cost(p->jobs[a].m, p->jobs[a].R) > point_cost(p->jobs[b].m, p->jobs[b].R);
        });
        c.n_items = 0;
        for (int pi : c.pairs) {
            MatchJob& j = p->jobs[pi];
            c.n_items += j.n;
            c.max_m = std::max(c.max_m, j.m);
            c.max_R = std::max(c.max_R, j.R);
            c.max_lw = std::max(c.max_lw, j.m + 2 * j.R);
            bool seen = false;
            for (size_t q = 0; q < c.ms.size(); ++q) seen = seen || (c.ms[q] == j.m && c.Rs[q] == j.R);
            if (!seen) {
                c.ms.push_back(j.m);
                c.Rs.push_back(j.R);
            }
            if (tc_form(c.path) && !corr_tc_maps(tc_form(c.path), j)) return false;
        }
        c.items = lay.add(sizeof(int2) * (size_t)c.n_items);
        if (c.path == SFOC_CORR_FFT) c.queue = p->n_queues++;
    }
    p->d_queues = lay.add(sizeof(int) * (size_t)(p->n_queues > 0 ? p->n_queues : 1));
    return true;
}

void write_classes(BatchPlan* p, char* host) {
    memcpy(host + p->d_jobs, p->jobs.data(), sizeof(MatchJob) * p->jobs.size());
    for (const CorrClass& c : p->classes) {
        int2* it = reinterpret_cast<int2*>(host + c.items);
        size_t k = 0;
        for (int pi : c.pairs)
            for (int q = 0; q < p->jobs[pi].n; ++q) it[k++] = make_int2(pi, q);
    }
}

sfoc_status upload(sfoc_ctx* ctx, BatchPlan* p, const std::vector<char>& host, size_t from, size_t to) {
    if (to <= from) return SFOC_OK;
    // a fresh buffer: nothing on any stream uses it yet
    cudaError_t e = cudaMemcpy(p->dbuf + from, host.data() + from, to - from, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch table upload");
    return SFOC_OK;
}

// Makes a plan for a match over `in` (and, kind 2, the build of its images
// first): tables, eager first run with the autotuner, graph.
// Workspace of a plan: [stats][maps][scratch: SFOC waves / integral scratch].
// *scratch_out (may be null) receives the scratch part.
size_t plan_ws_bytes(const BuildIn* bin, const sfoc_params* prm, const MatchIn* min, size_t* scratch_out) {
    size_t ws_match = 0, maps_off = 0;
    int total_items = 0;
    if (min) ws_match = match_ws_bytes(*min, &maps_off, &total_items);
    size_t f_need = 0, f_max = 0;
    if (bin) {
        const int z = prm->first_order_only ? prm->n_orient : 2 * prm->n_orient;
        for (int i = 0; i < bin->n; ++i) {
            const size_t fb = align256(sizeof(float) * roundup((size_t)bin->W[i], 32) * (size_t)bin->H[i] * z);
            f_need += fb;
            f_max = std::max(f_max, fb);
        }
    }
    size_t int_need = 0;
    if (min) {
        std::vector<const Cube*> rc;
        for (int i = 0; i < min->n; ++i) {
            if (!min->refs[i]) continue;
            const Cube* c = &min->refs[i]->c;
            if (std::find(rc.begin(), rc.end(), c) == rc.end()) rc.push_back(c);
        }
        int_need = integral_batch_scratch_bytes(rc.data(), (int)rc.size());
    }
    const size_t f_bytes = std::min(f_need, std::max(f_max, kFBudget));
    const size_t scratch = std::max(f_bytes, int_need);
    if (scratch_out) *scratch_out = scratch;
    return align256(ws_match) + scratch;
}

sfoc_status make_and_run(sfoc_ctx* ctx, int kind, std::vector<uint64_t>&& key, const BuildIn* bin,
                         const sfoc_params* prm, sfoc_cube** build_cubes, const MatchIn* min, int path,
                         BatchPlan** out) {
    // workspace: [stats][maps][scratch: SFOC waves / integral scratch]
    size_t ws_match = 0, maps_off = 0;
    int total_items = 0;
    if (min) ws_match = match_ws_bytes(*min, &maps_off, &total_items);
    size_t scratch = 0;
    const size_t ws_total = plan_ws_bytes(bin, prm, min, &scratch);
    sfoc_status s = ensure_ws(ctx, ws_total);
    if (s != SFOC_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    char* scr = ws + align256(ws_match);

    BatchPlan* p = new (std::nothrow) BatchPlan();
    if (!p) return fail(ctx, SFOC_ERR_OOM, "host allocation");
    p->kind = kind;
    ++ctx->plans_built;
    p->key = std::move(key);
    Layout lay;
    if (bin) {
        s = plan_build(ctx, p, *bin, *prm, build_cubes, kind == 2, scr, scratch, lay);
        if (s != SFOC_OK) {
            destroy_plan(p);
            return s;
        }
    }
    MatchIn mi;
    std::vector<sfoc_cube*> rv, sv;
    if (min) {
        mi = *min;
        if (kind == 2) {  // the pairs' cubes are the ones just laid out: ref 2i, sensed 2i + 1
            for (int i = 0; i < min->n; ++i) {
                rv.push_back(p->cubes[2 * i]);
                sv.push_back(p->cubes[2 * i + 1]);
            }
            mi.refs = rv.data();
            mi.sens = sv.data();
        }
        plan_match_jobs(p, mi, ws, maps_off, scr, lay);
    }
    const size_t head_end = lay.bytes;
    // allocate the buffer for everything but the class tables, upload, and run
    // the stages the autotuner needs
    const int dtype = min ? mi.refs[0]->c.dtype : 0;
    bool need_tune = false;
    const int family = path == SFOC_CORR_AUTO ? 0 : 1;
    if (min && (path == SFOC_CORR_AUTO || path == SFOC_CORR_IGEMM_TC) && ctx->autotune)
        for (int i = 0; i < mi.n; ++i)
            if (mi.npts[i] > 0 && !ctx->tune.count(TuneKey{dtype, mi.m[i], mi.R[i], family})) need_tune = true;
    std::vector<char> host;
    if (min) {
        // classes need the forms, which may need measurements: lay them out after
        if (need_tune) {
            host.assign(roundup(head_end, 256), 0);
            if (bin) write_build_tables(p, host.data());
            write_match_head(p, host.data(), scr);
            // the jobs table (tensor maps are set later, per class)
            const size_t djobs_end = p->d_jobs + sizeof(MatchJob) * p->jobs.size();
            memcpy(host.data() + p->d_jobs, p->jobs.data(), djobs_end - p->d_jobs);
            cudaError_t e = cudaMalloc(&p->dbuf, roundup(head_end, 256) + 4096);
            if (e != cudaSuccess) {
                destroy_plan(p);
                return cuda_fail(ctx, e, "cudaMalloc(batch tables)");
            }
            p->dbuf_bytes = roundup(head_end, 256) + 4096;
            s = upload(ctx, p, host, 0, head_end);
            cudaError_t e2 = cudaSuccess;
            if (s == SFOC_OK && bin) e2 = enqueue_build(ctx, p, ctx->stream);
            if (s == SFOC_OK && e2 == cudaSuccess) e2 = enqueue_match_head(ctx, p, ctx->stream);
            if (e2 != cudaSuccess) s = cuda_fail(ctx, e2, "batch launch");
            if (s != SFOC_OK) {
                destroy_plan(p);
                return s;
            }
            // measure each (m, R) without an entry on the first pair that has it
            for (int i = 0; i < mi.n; ++i) {
                if (mi.npts[i] == 0 || ctx->tune.count(TuneKey{dtype, mi.m[i], mi.R[i], family})) continue;
                if (!autotune_pair(ctx, dtype, family, p->jobs[i])) {
                    destroy_plan(p);
                    return fail(ctx, SFOC_ERR_UNSUPPORTED, "no correlation form ran for a pair's m / R");
                }
            }
            cudaFree(p->dbuf);  // re-laid out with the classes below (the head stays identical)
            p->dbuf = nullptr;
        }
        if (!plan_classes(ctx, p, path, dtype, lay)) {
            destroy_plan(p);
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "tensor map of a pair could not be encoded");
        }
    }
    host.assign(roundup(lay.bytes, 256), 0);
    if (bin) write_build_tables(p, host.data());
    if (min) {
        write_match_head(p, host.data(), scr);
        write_classes(p, host.data());
    }
    cudaError_t e = cudaMalloc(&p->dbuf, host.size() + 256);
    if (e != cudaSuccess) {
        destroy_plan(p);
        return cuda_fail(ctx, e, "cudaMalloc(batch tables)");
    }
    p->dbuf_bytes = host.size() + 256;
    s = upload(ctx, p, host, 0, host.size());
    if (s == SFOC_OK) s = capture_plan(ctx, p);
    if (s != SFOC_OK) {
        destroy_plan(p);
        return s;
    }
    keep_plan(ctx, p);
    *out = p;
    return run_plan(ctx, p);
}

// field by field: the struct's padding bytes (and the unused tails of its
// arrays) hold whatever the caller's copy left there, so hashing its raw
// bytes could key two equal parameter sets apart
void key_params(KeyWriter& k, const sfoc_params& p) {
    auto dbl = [&](double v) {
        uint64_t w;
        memcpy(&w, &v, sizeof(w));
        k.u(w);
    };
    k.u((uint64_t)(uint32_t)p.n_scales);
    for (int i = 0; i < p.n_scales && i < 8; ++i) dbl(p.scales[i]);
    dbl(p.sigma2);
    k.u((uint64_t)(uint32_t)p.n_orient << 32 | (uint32_t)p.n_dil);
    for (int i = 0; i < p.n_dil && i < 4; ++i) k.u((uint64_t)(uint32_t)p.dil[i]);
    dbl(p.sigma_d1);
    dbl(p.sigma_d2);
    dbl(p.eps);
    dbl(p.radius_mult);
    k.u((uint64_t)(uint32_t)p.rectify << 32 | (uint32_t)p.first_order_only);
    k.u((uint64_t)(uint32_t)p.cube_dtype);
}

void key_cube(KeyWriter& k, const sfoc_cube* c) {
    k.p(c);
    if (!c) return;
    k.p(c->c.f32);
    k.p(c->c.rm);
    k.p(c->c.cm);
    k.p(c->c.s1);
    k.p(c->c.s2);
    k.p(c->c.integ);
    k.u((uint64_t)c->c.H << 32 | (uint32_t)c->c.W);
    k.u((uint64_t)c->c.z << 32 | (uint32_t)c->c.dtype);
}

sfoc_status resolve_params(sfoc_ctx* ctx, const sfoc_params* pin, sfoc_params* p) {
    if (pin) *p = *pin;
    else sfoc_params_default(p);
    return check_params(ctx, *p);
}

// the signature of a fastncc_register_batch call (its plan's key)
void register_key(KeyWriter& k, int n_pairs, int path, const sfoc_params& prm, const float* const* d_refs,
                  const int* Hr, const int* Wr, const float* const* d_sens, const int* Hs, const int* Ws,
                  const int32_t* const* d_points, const int* n_points, const int* template_size,
                  const int* search_radius, fastncc_result* const* d_outs) {
    k.u(2);
    k.u((uint64_t)n_pairs);
    k.u((uint64_t)path);
    key_params(k, prm);
    for (int i = 0; i < n_pairs; ++i) {
        k.p(d_refs[i]);
        k.p(d_sens[i]);
        k.u((uint64_t)(uint32_t)Hr[i] << 32 | (uint32_t)Wr[i]);
        k.u((uint64_t)(uint32_t)Hs[i] << 32 | (uint32_t)Ws[i]);
        k.p(d_points[i]);
        k.p(d_outs[i]);
        k.u((uint64_t)(uint32_t)n_points[i] << 32 | (uint32_t)template_size[i]);
        k.u((uint64_t)search_radius[i]);
    }
}

}  // namespace

}  // namespace sfoc

using namespace sfoc;

extern "C" {

sfoc_status sfoc_build_batch(sfoc_ctx* ctx, int n_img, const float* const* d_images, const int* H, const int* W,
                             const size_t* pitch_elems, const sfoc_params* pin, sfoc_cube** outs) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (n_img < 0 || (n_img > 0 && (!d_images || !H || !W || !outs)))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "bad batch arguments");
    if (n_img == 0) return SFOC_OK;
    sfoc_params prm;
    sfoc_status s = resolve_params(ctx, pin, &prm);
    if (s != SFOC_OK) return s;
    for (int i = 0; i < n_img; ++i) {
        if (!d_images[i]) return fail(ctx, SFOC_ERR_INVALID_ARG, "null image in the batch");
        if (H[i] <= 0 || W[i] <= 0) return fail(ctx, SFOC_ERR_SHAPE, "image must be at least 1 x 1");
        if (pitch_elems && pitch_elems[i] < (size_t)W[i]) return fail(ctx, SFOC_ERR_SHAPE, "pitch_elems < W");
        if ((size_t)H[i] * (size_t)W[i] > ((size_t)1 << 31))
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "image larger than 2^31 pixels");
    }
    DeviceGuard g(ctx->device);
    // the cubes first (allocated or reused as sfoc_build does), so the key
    // holds their addresses
    const int z = prm.first_order_only ? prm.n_orient : 2 * prm.n_orient;
    for (int i = 0; i < n_img; ++i) {
        sfoc_cube* c = outs[i];
        if (c && c->c.H == H[i] && c->c.W == W[i] && c->c.z == z && c->c.dtype == prm.cube_dtype &&
            c->c.device == ctx->device)
            continue;
        c = new (std::nothrow) sfoc_cube();
        if (!c) return fail(ctx, SFOC_ERR_OOM, "host allocation");
        s = alloc_cube(ctx, c->c, H[i], W[i], z, prm.cube_dtype);
        if (s != SFOC_OK) {
            delete c;
            return s;
        }
        outs[i] = c;
    }
    KeyWriter k;
    k.u(0);
    k.u((uint64_t)n_img);
    key_params(k, prm);
    for (int i = 0; i < n_img; ++i) {
        k.p(d_images[i]);
        k.u((uint64_t)H[i] << 32 | (uint32_t)W[i]);
        k.u(pitch_elems ? pitch_elems[i] : (size_t)W[i]);
        key_cube(k, outs[i]);
    }
    BatchPlan* p = find_plan(ctx, k.k);
    if (p) {
        for (sfoc_cube* c : p->cubes) c->c.integ_valid = false;
        return run_plan(ctx, p);
    }
    BuildIn bin{n_img, d_images, H, W, pitch_elems};
    return make_and_run(ctx, 0, std::move(k.k), &bin, &prm, outs, nullptr, SFOC_CORR_AUTO, &p);
}

sfoc_status fastncc_match_batch(sfoc_ctx* ctx, int n_pairs, sfoc_cube* const* refs, sfoc_cube* const* sens,
                                const int32_t* const* d_points, const int* n_points, const int* template_size,
                                const int* search_radius, const fastncc_opts* opts, fastncc_result* const* d_outs) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (n_pairs < 0 || (n_pairs > 0 && (!refs || !sens || !d_points || !n_points || !template_size || !search_radius ||
                                        !d_outs)))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "bad batch arguments");
    const int path = opts ? opts->corr_path : SFOC_CORR_AUTO;
    if (path < SFOC_CORR_AUTO || path > SFOC_CORR_FFT) return fail(ctx, SFOC_ERR_INVALID_ARG, "unknown corr_path");
    if (n_pairs == 0) return SFOC_OK;
    MatchIn mi{n_pairs, refs, sens, d_points, n_points, template_size, search_radius, d_outs};
    sfoc_status s = check_match(ctx, mi, path);
    if (s != SFOC_OK) return s;
    DeviceGuard g(ctx->device);
    KeyWriter k;
    k.u(1);
    k.u((uint64_t)n_pairs);
    k.u((uint64_t)path);
    for (int i = 0; i < n_pairs; ++i) {
        key_cube(k, refs[i]);
        key_cube(k, sens[i]);
        k.p(d_points[i]);
        k.p(d_outs[i]);
        k.u((uint64_t)(uint32_t)n_points[i] << 32 | (uint32_t)template_size[i]);
        k.u((uint64_t)search_radius[i]);
    }
    BatchPlan* p = find_plan(ctx, k.k);
    if (p) return run_plan(ctx, p);
    return make_and_run(ctx, 1, std::move(k.k), nullptr, nullptr, nullptr, &mi, path, &p);
}

sfoc_status fastncc_register_batch(sfoc_ctx* ctx, int n_pairs, const float* const* d_refs, const int* Hr,
                                   const int* Wr, const float* const* d_sens, const int* Hs, const int* Ws,
                                   const int32_t* const* d_points, const int* n_points, const int* template_size,
                                   const int* search_radius, const sfoc_params* pin, const fastncc_opts* opts,
                                   fastncc_result* const* d_outs) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (n_pairs < 0 || (n_pairs > 0 && (!d_refs || !Hr || !Wr || !d_sens || !Hs || !Ws || !d_points || !n_points ||
                                        !template_size || !search_radius || !d_outs)))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "bad batch arguments");
    const int path = opts ? opts->corr_path : SFOC_CORR_AUTO;
    if (path < SFOC_CORR_AUTO || path > SFOC_CORR_FFT) return fail(ctx, SFOC_ERR_INVALID_ARG, "unknown corr_path");
    if (n_pairs == 0) return SFOC_OK;
    sfoc_params prm;
    sfoc_status s = resolve_params(ctx, pin, &prm);
    if (s != SFOC_OK) return s;
    std::vector<const float*> imgs(2 * (size_t)n_pairs);
    std::vector<int> H(2 * (size_t)n_pairs), W(2 * (size_t)n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        imgs[2 * i] = d_refs[i];
        imgs[2 * i + 1] = d_sens[i];
        H[2 * i] = Hr[i];
        W[2 * i] = Wr[i];
        H[2 * i + 1] = Hs[i];
        W[2 * i + 1] = Ws[i];
    }
    for (size_t i = 0; i < imgs.size(); ++i) {
        if (!imgs[i]) return fail(ctx, SFOC_ERR_INVALID_ARG, "null image in the batch");
        if (H[i] <= 0 || W[i] <= 0) return fail(ctx, SFOC_ERR_SHAPE, "image must be at least 1 x 1");
        if ((size_t)H[i] * (size_t)W[i] > ((size_t)1 << 31))
            return fail(ctx, SFOC_ERR_UNSUPPORTED, "image larger than 2^31 pixels");
    }
    // the match checks on stand-in cubes of the right shape and dtype
    const int z = prm.first_order_only ? prm.n_orient : 2 * prm.n_orient;
    std::vector<sfoc_cube> shape(2 * (size_t)n_pairs);
    std::vector<sfoc_cube*> rp(n_pairs), sp(n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        for (int q = 0; q < 2; ++q) {
            Cube& c = shape[2 * i + q].c;
            c.H = H[2 * i + q];
            c.W = W[2 * i + q];
            c.z = z;
            c.dtype = prm.cube_dtype;
        }
        rp[i] = &shape[2 * i];
        sp[i] = &shape[2 * i + 1];
    }
    MatchIn mi{n_pairs, rp.data(), sp.data(), d_points, n_points, template_size, search_radius, d_outs};
    s = check_match(ctx, mi, path);
    if (s != SFOC_OK) return s;
    DeviceGuard g(ctx->device);
    KeyWriter k;
    register_key(k, n_pairs, path, prm, d_refs, Hr, Wr, d_sens, Hs, Ws, d_points, n_points, template_size,
                 search_radius, d_outs);
    BatchPlan* p = find_plan(ctx, k.k);
    if (p) return run_plan(ctx, p);
    std::vector<sfoc_cube*> cubes(2 * (size_t)n_pairs, nullptr);
    BuildIn bin{2 * n_pairs, imgs.data(), H.data(), W.data(), nullptr};
    return make_and_run(ctx, 2, std::move(k.k), &bin, &prm, cubes.data(), &mi, path, &p);
}

namespace {

// The host-buffer batch, enqueued without waiting: the point sets and images
// copied into the context's staging buffer on the copy stream, the batch's
// launches and the copies of the results into h_outs on the context stream.
// Against the previous submission it is ordered by events alone: its images
// are overwritten once that submission's SFOC launches are done with them,
// its point sets once its results are out, so a submission's copies run
// while the one before it is still matching.  *ticket = the submission's
// number (0 when nothing was enqueued: an empty batch).
sfoc_status host_batch_enqueue(sfoc_ctx* ctx, int n_pairs, const float* const* h_refs, const int* Hr, const int* Wr,
                               const float* const* h_sens, const int* Hs, const int* Ws,
                               const int32_t* const* h_points, const int* n_points, const int* template_size,
                               const int* search_radius, const sfoc_params* pin, const fastncc_opts* opts,
                               fastncc_result* const* h_outs, int64_t* ticket) {
    *ticket = 0;
    if (n_pairs < 0 || (n_pairs > 0 && (!h_refs || !Hr || !Wr || !h_sens || !Hs || !Ws || !h_points || !n_points ||
                                        !template_size || !search_radius || !h_outs)))
        return fail(ctx, SFOC_ERR_INVALID_ARG, "bad batch arguments");
    if (n_pairs == 0) return SFOC_OK;
    const int path = opts ? opts->corr_path : SFOC_CORR_AUTO;
    if (path < SFOC_CORR_AUTO || path > SFOC_CORR_FFT) return fail(ctx, SFOC_ERR_INVALID_ARG, "unknown corr_path");
    sfoc_params prm;
    sfoc_status s = resolve_params(ctx, pin, &prm);
    if (s != SFOC_OK) return s;
    size_t need = 0;
    for (int i = 0; i < n_pairs; ++i) {
        if (!h_refs[i] || !h_sens[i] || n_points[i] < 0 || (n_points[i] > 0 && (!h_points[i] || !h_outs[i])))
            return fail(ctx, SFOC_ERR_INVALID_ARG, "null host buffer in the batch");
        if (Hr[i] <= 0 || Wr[i] <= 0 || Hs[i] <= 0 || Ws[i] <= 0) return fail(ctx, SFOC_ERR_SHAPE, "bad sizes");
        need += align256(sizeof(float) * (size_t)Hr[i] * Wr[i]) + align256(sizeof(float) * (size_t)Hs[i] * Ws[i]) +
                align256(sizeof(int32_t) * 2 * (size_t)n_points[i]) +
                align256(sizeof(fastncc_result) * (size_t)n_points[i]);
    }
    DeviceGuard g(ctx->device);
    // the whole batch's workspace before the staging buffer, so a later
    // growth of either does not drop the plan built below
    {
        const int z = prm.first_order_only ? prm.n_orient : 2 * prm.n_orient;
        std::vector<const float*> imgs(2 * (size_t)n_pairs, nullptr);
        std::vector<int> H(2 * (size_t)n_pairs), W(2 * (size_t)n_pairs);
        std::vector<sfoc_cube> shape(2 * (size_t)n_pairs);
        std::vector<sfoc_cube*> rp(n_pairs), sp(n_pairs);
        for (int i = 0; i < n_pairs; ++i) {
            H[2 * i] = Hr[i];
            W[2 * i] = Wr[i];
            H[2 * i + 1] = Hs[i];
            W[2 * i + 1] = Ws[i];
            for (int q = 0; q < 2; ++q) {
                Cube& c = shape[2 * i + q].c;
                c.H = H[2 * i + q];
                c.W = W[2 * i + q];
                c.z = z;
                c.dtype = prm.cube_dtype;
            }
            rp[i] = &shape[2 * i];
            sp[i] = &shape[2 * i + 1];
        }
        BuildIn bin{2 * n_pairs, imgs.data(), H.data(), W.data(), nullptr};
        MatchIn mi{n_pairs, rp.data(), sp.data(), h_points, n_points, template_size, search_radius, h_outs};
        s = ensure_ws(ctx, plan_ws_bytes(&bin, &prm, &mi, nullptr));
        if (s != SFOC_OK) return s;
    }
    if (need > ctx->hstage_bytes) {
        // the staging buffer moves: every submission in flight ends first, and
        // plans keyed on the old buffer are dropped
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess && ctx->copy_stream) e = cudaStreamSynchronize(ctx->copy_stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
        for (BatchPlan* bp : ctx->plans) destroy_plan(bp);
        ctx->plans.clear();
        cudaFree(ctx->hstage);
        ctx->hstage = nullptr;
        ctx->hstage_bytes = 0;
        e = cudaMalloc(&ctx->hstage, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(batch staging)");
        ctx->hstage_bytes = need;
    }
    cudaError_t e = cudaSuccess;
    if (!ctx->copy_stream) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->ev_hsfoc) e = cudaEventCreateWithFlags(&ctx->ev_hsfoc, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->ev_hpts) e = cudaEventCreateWithFlags(&ctx->ev_hpts, cudaEventDisableTiming);
    for (int r = 0; r < sfoc_ctx::kHostRing && e == cudaSuccess; ++r)
        if (!ctx->ev_hdone[r]) e = cudaEventCreateWithFlags(&ctx->ev_hdone[r], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
    // staging layout, pair by pair: reference image, sensed image, points, results
    std::vector<const float*> dr(n_pairs), ds(n_pairs);
    std::vector<const int32_t*> dp(n_pairs);
    std::vector<fastncc_result*> dout(n_pairs);
    {
        char* b = static_cast<char*>(ctx->hstage);
        for (int i = 0; i < n_pairs; ++i) {
            dr[i] = reinterpret_cast<const float*>(b);
            b += align256(sizeof(float) * (size_t)Hr[i] * Wr[i]);
            ds[i] = reinterpret_cast<const float*>(b);
            b += align256(sizeof(float) * (size_t)Hs[i] * Ws[i]);
            dp[i] = reinterpret_cast<const int32_t*>(b);
            b += align256(sizeof(int32_t) * 2 * (size_t)n_points[i]);
            dout[i] = reinterpret_cast<fastncc_result*>(b);
            b += align256(sizeof(fastncc_result) * (size_t)n_points[i]);
        }
    }
    KeyWriter k;
    register_key(k, n_pairs, path, prm, dr.data(), Hr, Wr, ds.data(), Hs, Ws, dp.data(), n_points, template_size,
                 search_radius, dout.data());
    BatchPlan* plan = find_plan(ctx, k.k);
    const bool by_wave = plan && plan->build_batched && plan->kind == 2;
    const size_t n_ev = by_wave ? plan->waves.size() : 1;
    while (ctx->ev_wave.size() < n_ev && e == cudaSuccess) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) ctx->ev_wave.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy events");
    // on a failure after the first copy: everything in flight ends before the
    // caller's buffers go back to it
    auto drained = [&](sfoc_status st) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamSynchronize(ctx->stream);
        (void)cudaGetLastError();
        return st;
    };
    const int64_t prev = ctx->host_ticket;  // the previous submission (0: none)
    // the images, in the plan's image order (reference of pair i = image 2i,
    // sensed = 2i + 1) with an event after each SFOC wave's last image, once
    // the previous submission's SFOC launches have read the staged images
    if (prev > 0) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_hsfoc, 0);
    auto copy_image = [&](int im) {
        const int i = im >> 1;
        if (im & 1)
            return cudaMemcpyAsync(const_cast<float*>(ds[i]), h_sens[i], sizeof(float) * (size_t)Hs[i] * Ws[i],
                                   cudaMemcpyHostToDevice, ctx->copy_stream);
        return cudaMemcpyAsync(const_cast<float*>(dr[i]), h_refs[i], sizeof(float) * (size_t)Hr[i] * Wr[i],
                               cudaMemcpyHostToDevice, ctx->copy_stream);
    };
    if (by_wave) {
        for (size_t w = 0; w < plan->waves.size() && e == cudaSuccess; ++w) {
            const Wave& wv = plan->waves[w];
            for (int im = wv.img0; im < wv.img0 + wv.n_img && e == cudaSuccess; ++im) e = copy_image(im);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_wave[w], ctx->copy_stream);
        }
    } else {
        for (int im = 0; im < 2 * n_pairs && e == cudaSuccess; ++im) e = copy_image(im);
    }
    // then the point sets, once the previous submission's results are out
    // (its matching is the last to read them)
    if (prev > 0 && e == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_hdone[prev % sfoc_ctx::kHostRing], 0);
    for (int i = 0; i < n_pairs && e == cudaSuccess; ++i)
        if (n_points[i] > 0)
            e = cudaMemcpyAsync(const_cast<int32_t*>(dp[i]), h_points[i], sizeof(int32_t) * 2 * (size_t)n_points[i],
                                cudaMemcpyHostToDevice, ctx->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_hpts, ctx->copy_stream);
    if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "host to device copy"));
    if (by_wave) {
        // the plan's stages launched one by one, each SFOC wave after its images
        for (size_t w = 0; w < plan->waves.size() && e == cudaSuccess; ++w) {
            const Wave& wv = plan->waves[w];
            e = cudaStreamWaitEvent(ctx->stream, ctx->ev_wave[w], 0);
            if (e != cudaSuccess) break;
            StageScope sc(ctx, ST_STEER, 3);
            e = launch_sfoc_batch(reinterpret_cast<const ImgJob*>(plan->dbuf + wv.tab), wv.n_img,
                                  reinterpret_cast<const int*>(plan->dbuf + wv.steer_begin), wv.steer_ctas,
                                  reinterpret_cast<const int*>(plan->dbuf + wv.smooth_begin), wv.smooth_ctas,
                                  plan->st, plan->sm, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_hsfoc, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_hpts, 0);
        if (e == cudaSuccess) e = enqueue_match_head(ctx, plan, ctx->stream);
        if (e == cudaSuccess) e = enqueue_match_tail(ctx, plan, ctx->stream);
        if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "batch launch"));
    } else {
        // first call with this signature: everything copied, then the plan is
        // built and run (and its graph captured) as fastncc_register_batch does
        e = cudaStreamWaitEvent(ctx->stream, ctx->ev_hpts, 0);
        if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "cudaStreamWaitEvent"));
        sfoc_status s2 = fastncc_register_batch(ctx, n_pairs, dr.data(), Hr, Wr, ds.data(), Hs, Ws, dp.data(),
                                                n_points, template_size, search_radius, &prm, opts, dout.data());
        if (s2 != SFOC_OK) return drained(s2);
        e = cudaEventRecord(ctx->ev_hsfoc, ctx->stream);
        if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "cudaEventRecord"));
    }
    for (int i = 0; i < n_pairs && e == cudaSuccess; ++i)
        if (n_points[i] > 0)
            e = cudaMemcpyAsync(h_outs[i], dout[i], sizeof(fastncc_result) * (size_t)n_points[i],
                                cudaMemcpyDeviceToHost, ctx->stream);
    const int64_t t = prev + 1;
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_hdone[t % sfoc_ctx::kHostRing], ctx->stream);
    if (e != cudaSuccess) return drained(cuda_fail(ctx, e, "device to host copy"));
    ctx->host_ticket = t;
    *ticket = t;
    return SFOC_OK;
}

}  // namespace

sfoc_status fastncc_submit_batch_host(sfoc_ctx* ctx, int n_pairs, const float* const* h_refs, const int* Hr,
                                      const int* Wr, const float* const* h_sens, const int* Hs, const int* Ws,
                                      const int32_t* const* h_points, const int* n_points, const int* template_size,
                                      const int* search_radius, const sfoc_params* p, const fastncc_opts* opts,
                                      fastncc_result* const* h_outs, int64_t* ticket) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (!ticket) return fail(ctx, SFOC_ERR_INVALID_ARG, "ticket is NULL");
    return host_batch_enqueue(ctx, n_pairs, h_refs, Hr, Wr, h_sens, Hs, Ws, h_points, n_points, template_size,
                              search_radius, p, opts, h_outs, ticket);
}

sfoc_status fastncc_wait_batch_host(sfoc_ctx* ctx, int64_t ticket) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    if (ticket == 0) return SFOC_OK;  // an empty batch
    if (ticket < 0 || ticket > ctx->host_ticket) return fail(ctx, SFOC_ERR_INVALID_ARG, "unknown batch ticket");
    DeviceGuard g(ctx->device);
    // a later submission in the same ring slot ends after this one
    cudaError_t e = cudaEventSynchronize(ctx->ev_hdone[ticket % sfoc_ctx::kHostRing]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
    return SFOC_OK;
}

sfoc_status fastncc_register_batch_host(sfoc_ctx* ctx, int n_pairs, const float* const* h_refs, const int* Hr,
                                        const int* Wr, const float* const* h_sens, const int* Hs, const int* Ws,
                                        const int32_t* const* h_points, const int* n_points, const int* template_size,
                                        const int* search_radius, const sfoc_params* p, const fastncc_opts* opts,
                                        fastncc_result* const* h_outs) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    int64_t t = 0;
    sfoc_status s = host_batch_enqueue(ctx, n_pairs, h_refs, Hr, Wr, h_sens, Hs, Ws, h_points, n_points,
                                       template_size, search_radius, p, opts, h_outs, &t);
    if (s != SFOC_OK) return s;
    return fastncc_wait_batch_host(ctx, t);
}

int sfoc_ctx_plan_count(const sfoc_ctx* ctx) { return ctx ? (int)ctx->plans.size() : 0; }

sfoc_status sfoc_ctx_plan_info(const sfoc_ctx* ctx, char* buf, size_t cap, size_t* len) {
    if (!ctx || !len) return SFOC_ERR_INVALID_ARG;
    std::string j = "{\"plans_built\": " + std::to_string((long long)ctx->plans_built) + "}";
    if (!ctx->plans.empty()) {
        const BatchPlan* p = ctx->plans.back();
        char t[256];
        snprintf(t, sizeof(t),
                 "{\"plans_built\": %lld, \"kind\": %d, \"pairs\": %d, \"items\": %d, \"graph\": %s, "
                 "\"launches\": %d, ",
                 (long long)ctx->plans_built, p->kind, (int)p->jobs.size(), p->n_items, p->exec ? "true" : "false",
                 p->launches);
        j = t;
        j += "\"build_batched\": ";
        j += p->build_batched ? "true" : "false";
        j += ", \"waves\": [";
        for (size_t i = 0; i < p->waves.size(); ++i) {
            snprintf(t, sizeof(t), "%s{\"images\": %d, \"steer_ctas\": %d, \"smooth_ctas\": %d}", i ? ", " : "",
                     p->waves[i].n_img, p->waves[i].steer_ctas, p->waves[i].smooth_ctas);
            j += t;
        }
        j += "], \"classes\": [";
        for (size_t i = 0; i < p->classes.size(); ++i) {
            const CorrClass& c = p->classes[i];
            snprintf(t, sizeof(t), "%s{\"path\": %d, \"cls\": %d, \"items\": %d, \"launches\": %d, \"pairs\": [",
                     i ? ", " : "", c.path, c.cls, c.n_items,
                     c.path == SFOC_CORR_TC_TOEPLITZ ? (int)c.pairs.size() : 1);
            j += t;
            for (size_t q = 0; q < c.pairs.size(); ++q) {
                snprintf(t, sizeof(t), "%s%d", q ? ", " : "", c.pairs[q]);
                j += t;
            }
            j += "]}";
        }
        j += "]}";
    }
    *len = j.size() + 1;
    if (!buf) return SFOC_OK;
    if (cap < j.size() + 1) return SFOC_ERR_INVALID_ARG;
    memcpy(buf, j.c_str(), j.size() + 1);
    return SFOC_OK;
}

sfoc_status sfoc_ctx_release_plans(sfoc_ctx* ctx) {
    if (!ctx) return SFOC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    for (BatchPlan* p : ctx->plans) destroy_plan(p);
    ctx->plans.clear();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    return SFOC_OK;
}

}  // extern "C"
