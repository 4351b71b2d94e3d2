/*
 * sfoc.h - C ABI of the GB300 (sm_103a) library for the fine-registration
 * hot path of Ye et al., arXiv 2202.13347: building the SFOC feature cube
 * (Sec. 2.1) and Fast-NCC_SFOC template matching (Sec. 2.2, Sec. 3.2.2).
 *
 * Conventions
 *  - Images are H rows x W columns; x is the column (right), y the row (down).
 *  - Every pointer named d_* is CUDA device memory owned by the caller unless
 *    stated otherwise; h_* is host memory.  Nothing is freed by the library
 *    that it did not allocate.
 *  - All calls are asynchronous on the context's stream unless stated
 *    otherwise and return an sfoc_status.  Nothing throws across the ABI.
 *    On a negative status sfoc_last_error_string() describes the failure.
 *  - A context is not thread-safe: use one per host thread.
 *  - Calls check their arguments before enqueuing work; kernel-side failures
 *    (bounded waits that expired, bad points) are reported per point in
 *    fastncc_result.status or by sfoc_ctx_sync().
 */
#ifndef SFOC_GB300_H
#define SFOC_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SFOC_API __attribute__((visibility("default")))
#else
#define SFOC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfoc_ctx sfoc_ctx;
typedef struct sfoc_cube sfoc_cube;

typedef enum {
    SFOC_OK = 0,
    SFOC_ERR_INVALID_ARG = -1, /* null pointer, negative size, bad enum */
    SFOC_ERR_SHAPE = -2,       /* shapes or channel counts that do not fit together */
    SFOC_ERR_OOM = -3,         /* a device allocation failed */
    SFOC_ERR_CUDA = -4,        /* a CUDA runtime/driver call failed */
    SFOC_ERR_TIMEOUT = -5,     /* a bounded device wait expired */
    SFOC_ERR_UNSUPPORTED = -6  /* valid but outside what the kernels implement */
} sfoc_status;

/* Per-point status in fastncc_result.status. */
enum {
    SFOC_PT_OK = 0,
    SFOC_PT_OUT_OF_BOUNDS = 1, /* template or a candidate window leaves its image; nothing computed */
    SFOC_PT_FLAT_TEMPLATE = 2, /* template variance <= 1e-6 * m*m*z; offsets 0, ncc 0 */
    SFOC_PT_PEAK_ON_EDGE = 3,  /* best |dx| or |dy| equals R; no sub-pixel on that axis */
    SFOC_PT_NAN = 4            /* NaN in the template or in some candidate's score */
};

typedef enum { SFOC_DTYPE_F32 = 0, SFOC_DTYPE_BF16 = 1 } sfoc_dtype;

/* Correlation kernel for R_ST (Eq. 10). */
typedef enum {
    SFOC_CORR_AUTO = 0,       /* the form the autotuner measured fastest for (cube dtype, m, R)
                               * (see the autotuner section below) */
    SFOC_CORR_DIRECT_F32 = 1, /* FP32 CUDA-core direct correlation (F32 cubes) */
    SFOC_CORR_IGEMM_TC = 2,   /* tcgen05 BF16 implicit GEMM, FP32 accumulate (BF16 cubes): the
                               * tensor-core form the autotuner measured fastest (family 1) */
    SFOC_CORR_TC_TOEPLITZ = 3, /* the Toeplitz form of the tcgen05 kernel for any m, R */
    SFOC_CORR_TC_COLUMN = 4,  /* the column form: m + 2R <= 128, else SFOC_ERR_UNSUPPORTED */
    SFOC_CORR_TC_BAND = 5,    /* the band form (bands of 16 window rows x 8 offsets):
                               * R <= 40 and its shared memory fits, else SFOC_ERR_UNSUPPORTED */
    SFOC_CORR_FFT = 6         /* Eq. 13: FP32 Fourier transforms of the zero-padded window and
                               * zero-mean template, summed over channels (F32 cubes, or BF16
                               * cubes widened to FP32 as they are read; m + 2R <= 128, else
                               * SFOC_ERR_UNSUPPORTED) */
} sfoc_corr_path;

/*
 * Descriptor parameters (Sec. 2.1; Table 2).  sfoc_params_default() fills:
 *   scales = {0.6, 0.8, 1.0} first-order STDs, sigma2 = 1.5 second-order STD
 *   (Table 2); n_orient = 6 (theta_k = k*pi/6, Sec. 2.1); dilations {1,2,3}
 *   (Sec. 2.1); sigma_d1 = 1.0 and sigma_d2 = 1.5, the smoothing STDs of the
 *   first- and second-order groups (the paper only says the second is
 *   larger); eps = 1e-3 in v/(||v||+eps); rectify = 1 (|.| of each steered
 *   response); radius_mult = 3 (kernel radius ceil(3 sigma));
 *   first_order_only = 0 (1 gives the F-SFOC variant of Sec. 4.2);
 *   cube_dtype = SFOC_DTYPE_F32.
 * The smoothing variants that Sec. 2.1 compares in Fig. 3: n_dil = 1 with
 * dil = {1} smooths with a plain Gaussian; sigma_d1 or sigma_d2 = 0 leaves
 * that group unsmoothed (the steered channels go straight to the group
 * normalisation).  Negative STDs are SFOC_ERR_INVALID_ARG.
 * Limits: n_scales 1..4, each radius <= 9; sigma2 radius <= 9; n_orient 1..8;
 * n_dil 1..3 with rates 1..3; smoothing radii <= 6; cube_dtype BF16 needs
 * n_orient == 6 and first_order_only == 0 (12 channels).
 */
typedef struct {
    int n_scales;
    double scales[8];
    double sigma2;
    int n_orient;
    int n_dil;
    int dil[4];
    double sigma_d1;
    double sigma_d2;
    double eps;
    int rectify;
    double radius_mult;
    int first_order_only;
    int cube_dtype; /* sfoc_dtype */
} sfoc_params;

/* One matched control point (Sec. 3.2.2: the most similar position is the CP).
 * The template is cut from the sensed cube around p; the candidate window is
 * the reference cube around p + (dx, dy).  For a sensed image that is the
 * reference shifted by s, the answer is (dx, dy) = -s. */
typedef struct {
    int32_t dx, dy;       /* integer offset in [-R, R] of the best NCC */
    float ncc;            /* NCC_SFOC at that offset (Eq. 8) */
    float sub_dx, sub_dy; /* offset refined by a 3-point parabola per axis */
    int32_t status;       /* SFOC_PT_* */
} fastncc_result;

typedef struct {
    int corr_path;  /* sfoc_corr_path */
    float* d_maps;  /* optional: n x (2R+1) x (2R+1) NCC maps (rows dy, cols dx) */
} fastncc_opts;

/* ---- context -------------------------------------------------------- */

/* Creates a context on CUDA device `device` issuing work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The context owns its
 * workspace (grown on demand, freed by sfoc_ctx_destroy).  *out is NULL on
 * failure: SFOC_ERR_INVALID_ARG for a NULL `out` or a device index out of
 * range, SFOC_ERR_CUDA when no CUDA device can be reached, SFOC_ERR_OOM when
 * the context's error word cannot be allocated.
 * Every call below that takes a context returns SFOC_ERR_INVALID_ARG for a
 * NULL one (sfoc_last_error_string returns "null context",
 * sfoc_ctx_launch_count 0). */
SFOC_API sfoc_status sfoc_ctx_create(sfoc_ctx** out, int device, void* stream);
SFOC_API sfoc_status sfoc_ctx_destroy(sfoc_ctx* ctx);
/* Issues later calls on `stream`.  The work already queued on the previous
 * stream shares the context's workspace, so the new stream is made to wait
 * for it on the device (an event recorded on the previous stream; the host
 * does not block).  SFOC_ERR_INVALID_ARG while either stream is being
 * captured into a CUDA graph. */
SFOC_API sfoc_status sfoc_ctx_set_stream(sfoc_ctx* ctx, void* stream);
/* Blocks until the context's stream is idle; reports deferred device errors
 * (SFOC_ERR_CUDA, or SFOC_ERR_TIMEOUT when a bounded device wait expired). */
SFOC_API sfoc_status sfoc_ctx_sync(sfoc_ctx* ctx);
/* Self-test of the failure path (not part of the paper's method): enqueues
 * one kernel that allocates tensor memory, waits on a barrier nothing
 * arrives on with the bounded wait the tensor-core kernels use, limited to
 * limit_us microseconds (1..100000), and then takes their abort path (frees
 * the tensor memory, sets the context's device error word, returns).  The
 * next sfoc_ctx_sync returns SFOC_ERR_TIMEOUT and clears the word; the
 * context stays usable.  SFOC_ERR_INVALID_ARG for a limit out of range. */
SFOC_API sfoc_status sfoc_ctx_selftest_timeout(sfoc_ctx* ctx, int limit_us);
/* Grows the workspace to hold at least `bytes` (so later calls, e.g. inside
 * a CUDA-graph capture, allocate nothing). */
SFOC_API sfoc_status sfoc_ctx_reserve(sfoc_ctx* ctx, size_t bytes);
/* Bytes of workspace fastncc_match needs for n points of radius R. */
SFOC_API size_t sfoc_match_workspace_bytes(int n, int search_radius);
/* Last error message of this context (never NULL; "" when none). */
SFOC_API const char* sfoc_last_error_string(const sfoc_ctx* ctx);
/* Number of kernel launches this context has issued so far. */
SFOC_API int64_t sfoc_ctx_launch_count(const sfoc_ctx* ctx);

/* Per-stage device timing (tracing).  When enabled, every kernel launch of
 * the context is bracketed by CUDA events on the context stream.  Stages:
 * 0 steer (Eq. 2-7), 1 smooth+normalise, 2 integral images (Eq. 14-15),
 * 3 template statistics (Eq. 12), 4 correlation R_ST (Eq. 10),
 * 5 NCC + argmax + sub-pixel (Eq. 9), 6 other (exports, copies). */
#define SFOC_NUM_STAGES 7
SFOC_API sfoc_status sfoc_ctx_enable_timing(sfoc_ctx* ctx, int enable);
/* Synchronises the stream and returns, per stage, the summed milliseconds
 * and the number of launches since the last reset. */
SFOC_API sfoc_status sfoc_ctx_stage_times(sfoc_ctx* ctx, double* ms_out, int64_t* launches_out);
SFOC_API sfoc_status sfoc_ctx_reset_timing(sfoc_ctx* ctx);
/* The timed scopes of one stage since the last reset, in order (a scope is
 * one launch, or the launches of one step of a stage: the four integral
 * kernels, a batched SFOC wave); *n_out = their number, the first `cap`
 * written to ms_out (milliseconds).  Synchronises the stream. */
SFOC_API sfoc_status sfoc_ctx_stage_scopes(sfoc_ctx* ctx, int stage, float* ms_out, int cap, int* n_out);

/* Peaks of this device measured by the library's own microbenchmarks (the
 * denominators of roofline fractions): FP32 FMA chains as scalar FFMA and
 * as paired FFMA2 (float2) instructions and FP64 FMA chains, in TFLOP/s
 * (2 flop per FMA), and a float4 copy of 1 GiB to another 1 GiB, in GB/s
 * of bytes read + written.  Each figure is the best of five timed launches
 * (CUDA events) after a warm-up.  Synchronous; allocates 2 GiB (plus a
 * small sink) for the copy and frees them before returning.  Not part of
 * the paper's method.  SFOC_ERR_INVALID_ARG for a NULL output,
 * SFOC_ERR_OOM / SFOC_ERR_CUDA when a buffer or a launch fails. */
typedef struct {
    double fp32_tflops;
    double fp32x2_tflops;
    double fp64_tflops;
    double hbm_copy_gbs;
} sfoc_peaks;
SFOC_API sfoc_status sfoc_measure_peaks(sfoc_ctx* ctx, sfoc_peaks* out);

/* ---- descriptor ----------------------------------------------------- */

SFOC_API sfoc_status sfoc_params_default(sfoc_params* p);

/*
 * sfoc_build - SFOC cube of one image (Sec. 2.1, Eq. 1-7, dilated Gaussian
 * smoothing and group normalisation).
 *   d_image      float32 image, row-major, pitch `pitch_elems` >= W elements.
 *   scales       host array of n_scales first-order STDs (overrides p->scales;
 *                NULL = take p->scales / n_scales from p).
 *   n_orient     orientations per group (overrides p->n_orient; <= 0 = p's).
 *   p            NULL = sfoc_params_default().
 *   out          receives a cube owned by the library (free with
 *                sfoc_cube_free).  On entry *out is NULL or a cube from an
 *                earlier build: a cube of the same H, W, channel count,
 *                dtype and device is rebuilt in place and no memory is
 *                allocated; any other cube is left as it is (the caller
 *                still frees it) and *out receives a new one.  On failure
 *                *out is unchanged.
 * The cube holds z = 2*n_orient channels (first-order then second-order
 * orientations), each normalised per group, plus per-pixel sums over
 * channels of g and g^2 used for the integral images of Eq. 14.
 */
SFOC_API sfoc_status sfoc_build(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems,
                       const double* scales, int n_scales, int n_orient, const sfoc_params* p,
                       sfoc_cube** out);

/*
 * sfoc_build_static - sfoc_build into a caller-owned F32 cube, allocating
 * nothing.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory when they build a descriptor (a fixed
 * memory budget set at start-up, or a loop that must not take cudaMalloc's
 * device-wide synchronisation).  It computes the same cube as sfoc_build
 * (same kernels, same values).
 *   d_image      float32 image, row-major, pitch `pitch_elems` >= W elements.
 *   p            NULL = sfoc_params_default(); cube_dtype must be F32.
 *   d_out        caller-owned float32 [z][H][W] (dense), z = 2*n_orient (or
 *                n_orient with first_order_only); receives the cube.
 * Scratch: one library-owned device array of SFOC_STATIC_SCRATCH_FLOATS
 * floats (64 MiB) per device.  A call needs z*roundup(W,32)*H + 2*H*W
 * floats of it (12 channels at H = 1024: W up to 1152, while W = 1153
 * already needs 16,910,336); larger images return SFOC_ERR_UNSUPPORTED
 * with the sizes in the error string.
 * The first call on a device looks up the array's address (this may load
 * the library's device code); make that first call before any stream
 * capture.  Calls that overlap in time on one device (several streams or
 * threads) share the array and race; it keeps the last call's contents.
 * Asynchronous on the context's stream.
 */
#define SFOC_STATIC_SCRATCH_FLOATS (1u << 24)
SFOC_API sfoc_status sfoc_build_static(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems,
                                       const sfoc_params* p, float* d_out);

/*
 * sfoc_build_u16 - sfoc_build of a 16-bit image: each sample v is taken as
 * the intensity v / 65535 (in float32, correctly rounded) while the tile is
 * loaded, so no converted copy of the image is made.  Same cube, params and
 * ownership rules as sfoc_build (the scales come from p).
 */
SFOC_API sfoc_status sfoc_build_u16(sfoc_ctx* ctx, const uint16_t* d_image, int H, int W, size_t pitch_elems,
                                    const sfoc_params* p, sfoc_cube** out);

/* Shape and dtype of a cube (any pointer may be NULL). */
SFOC_API sfoc_status sfoc_cube_info(const sfoc_cube* cube, int* z, int* H, int* W, int* dtype);
/*
 * Device view of a cube's values (any pointer may be NULL; the data stay
 * owned by the cube and valid until it is rebuilt or freed):
 *   F32 cube:  *d_data = float [z][H][pitch] (planar, pitch in elements);
 *   BF16 cube: *d_data = bf16 [z/6][H][W][8] (chunk g = the six channels of
 *              group g then two zeros, pixels row-major), *pitch = W.
 */
SFOC_API sfoc_status sfoc_cube_view(const sfoc_cube* cube, void** d_data, int* z, int* H, int* W, size_t* pitch,
                                    int* dtype);
/* Writes the cube as float32 [z][H][W] (dense) into d_out. */
SFOC_API sfoc_status sfoc_cube_export(sfoc_ctx* ctx, const sfoc_cube* cube, float* d_out);
/* Builds (if needed) and writes the two integral planes of Eq. 14 as
 * float64 [2][H+1][W+1] (exclusive prefix of sum_c g and of sum_c g^2).
 * The library keeps them as exact sums of the per-pixel values rounded to
 * multiples of 2^-28; an entry whose prefix rectangle holds a non-finite
 * value is NaN.  Uses the context workspace (4 bytes per entry). */
SFOC_API sfoc_status sfoc_cube_export_integral(sfoc_ctx* ctx, sfoc_cube* cube, double* d_out);
SFOC_API sfoc_status sfoc_cube_free(sfoc_cube* cube);

/* ---- matching ------------------------------------------------------- */

/*
 * fastncc_match - Fast-NCC_SFOC (Sec. 2.2, Eq. 8-16) for n interest points.
 *   ref, sen        cubes of the reference and sensed images (same z/dtype).
 *   d_points        int32 n x 2 (x, y) pairs in sensed coordinates.
 *   template_size   m >= 1 (odd: +-(m-1)/2 around p; even: [p-m/2, p+m/2-1]).
 *   search_radius   R >= 0: candidates d in [-R, R]^2.
 *   opts            NULL = defaults (AUTO path, no maps).
 *   d_out           caller-owned array of n fastncc_result.
 * NCC is the Eq. 8 value computed through Eq. 9: R_ST by a correlation
 * kernel (opts->corr_path), R_S and R_SS from the reference cube's integral
 * images (Eq. 14-16: exact 64-bit sums of the per-pixel channel sums rounded
 * to multiples of 2^-28, built on first use and kept with the cube), R_T and
 * R_TT from the same sums over the template, the variances in FP64.  Ties go
 * to the smallest dy, then the smallest dx.  The workspace grows to
 * sfoc_match_workspace_bytes(n, R) if it is smaller.
 * Errors: SFOC_ERR_INVALID_ARG for a NULL cube, NULL points or output with
 * n > 0, n < 0, m < 1, R < 0 or an unknown corr_path; SFOC_ERR_SHAPE when
 * the cubes' channel counts or dtypes differ; SFOC_ERR_UNSUPPORTED beyond
 * m <= 128, R <= 63, for a path the cube dtype does not serve (DIRECT_F32
 * needs F32 cubes, the tensor-core paths BF16 cubes) or a forced
 * form outside its limits; SFOC_ERR_OOM when the workspace cannot grow.
 * Points whose template or windows leave an image get status OUT_OF_BOUNDS.
 */
SFOC_API sfoc_status fastncc_match(sfoc_ctx* ctx, sfoc_cube* ref, sfoc_cube* sen, const int32_t* d_points, int n,
                          int template_size, int search_radius, const fastncc_opts* opts,
                          fastncc_result* d_out);

/*
 * fastncc_register_pair - the whole fine-registration path for one pair:
 * sfoc_build of both images, then fastncc_match.  Device buffers.  The two
 * cubes are cached in the context and reused while the shapes stay equal.
 */
SFOC_API sfoc_status fastncc_register_pair(sfoc_ctx* ctx, const float* d_ref, int Hr, int Wr, const float* d_sen,
                                  int Hs, int Ws, const int32_t* d_points, int n, int template_size,
                                  int search_radius, const sfoc_params* p, const fastncc_opts* opts,
                                  fastncc_result* d_out);

/* Same with host buffers: copies the images and points to the device,
 * runs the path and copies the results back before returning (synchronous).
 * h_out receives n fastncc_result. */
SFOC_API sfoc_status fastncc_register_pair_host(sfoc_ctx* ctx, const float* h_ref, int Hr, int Wr, const float* h_sen,
                                       int Hs, int Ws, const int32_t* h_points, int n, int template_size,
                                       int search_radius, const sfoc_params* p, const fastncc_opts* opts,
                                       fastncc_result* h_out);

/* ---- batched forms -------------------------------------------------- */
/*
 * Many image pairs of uneven size, each with its own points, m and R, in one
 * launch per stage instead of the per-point loop of Sec. 3.2.2 run pair after
 * pair: the SFOC kernels run over the tiles of every image at once (in
 * waves whose steering planes fit 4 GiB of workspace), the integral images
 * over every reference cube, the template statistics and the NCC stage over
 * every (pair, point) item, and the correlation as one persistent launch per
 * kernel instance ("class": the Fourier side, the direct kernel's tile
 * class, or a tensor-core form's instance; the Toeplitz form runs one launch
 * per pair) over its items, largest template and radius first.  Every pair
 * gets the correlation form opts->corr_path names, or with AUTO the one the
 * autotuner measured fastest for its (cube dtype, m, R).
 * A call's tables (a "plan") are built on its first use and kept in the
 * context (the two most recent), keyed by every pointer, size and parameter
 * of the call; that first call runs the stages one by one (measuring the
 * forms of any (m, R) that have no autotuned entry yet, which waits for the
 * device) and captures them into a CUDA graph; a later call with the same
 * arguments launches that graph on the context's stream.  With per-stage
 * timing on, plans run stage by stage instead (the stage events need their
 * own launches).  Plans point into the workspace: a workspace that grows
 * drops them.  Not thread-safe (like every call on a context).
 * All pairs of a batch have the same cube dtype and channel count.  Errors
 * as fastncc_match, checked for every pair before any work is queued.
 */

/* Builds n_img cubes; images[i] is H[i] x W[i] with pitch pitch_elems[i]
 * (NULL = dense).  outs[i] follows sfoc_build's in/out rule. */
SFOC_API sfoc_status sfoc_build_batch(sfoc_ctx* ctx, int n_img, const float* const* d_images, const int* H, const int* W,
                             const size_t* pitch_elems, const sfoc_params* p, sfoc_cube** outs);

/* Matches n_pairs (refs[i], sens[i]) pairs; pair i has n_points[i] points
 * d_points[i], template_size[i], search_radius[i] and writes d_outs[i]
 * (per-pair NCC maps are not returned). */
SFOC_API sfoc_status fastncc_match_batch(sfoc_ctx* ctx, int n_pairs, sfoc_cube* const* refs, sfoc_cube* const* sens,
                                const int32_t* const* d_points, const int* n_points, const int* template_size,
                                const int* search_radius, const fastncc_opts* opts, fastncc_result* const* d_outs);

/* The whole path for n_pairs pairs of dense float images on the device
 * (d_refs[i]: Hr[i] x Wr[i], d_sens[i]: Hs[i] x Ws[i]): SFOC of all
 * 2 n_pairs images, then the batched match.  The cubes belong to the plan
 * (freed with it).  Same plan and graph rules as above. */
SFOC_API sfoc_status fastncc_register_batch(sfoc_ctx* ctx, int n_pairs, const float* const* d_refs, const int* Hr,
                                            const int* Wr, const float* const* d_sens, const int* Hs, const int* Ws,
                                            const int32_t* const* d_points, const int* n_points,
                                            const int* template_size, const int* search_radius, const sfoc_params* p,
                                            const fastncc_opts* opts, fastncc_result* const* d_outs);

/* fastncc_register_batch from host buffers: copies every image and point
 * set into a device staging buffer kept by the context, runs the batch and
 * copies every pair's results to h_outs[i] before returning (synchronous:
 * fastncc_submit_batch_host, then fastncc_wait_batch_host).
 * The first call with a signature copies everything, then builds the plan
 * (as fastncc_register_batch does); later calls copy the images in the
 * order of the plan's SFOC waves on a second stream, then the point sets,
 * and each wave's SFOC launch waits only for its own images, so the copies
 * of the later waves run while the earlier waves are built.  (Pinned host
 * buffers let the copies overlap.)  These runs launch the plan's kernels
 * one by one rather than replaying its graph.  A staging buffer that has to
 * grow waits for every submission in flight and drops the context's plans. */
SFOC_API sfoc_status fastncc_register_batch_host(sfoc_ctx* ctx, int n_pairs, const float* const* h_refs,
                                                 const int* Hr, const int* Wr, const float* const* h_sens,
                                                 const int* Hs, const int* Ws, const int32_t* const* h_points,
                                                 const int* n_points, const int* template_size,
                                                 const int* search_radius, const sfoc_params* p,
                                                 const fastncc_opts* opts, fastncc_result* const* h_outs);

/* The same batch, enqueued without waiting, for a stream of batches (the
 * paper's per-point loop of Sec. 3.2.2 over many image pairs, fed from host
 * memory).  Arguments as fastncc_register_batch_host; *ticket receives the
 * submission's number (1, 2, ...; 0 for an empty batch, which enqueues
 * nothing).  The submission is ordered against the previous one by events
 * only: its images are copied in once the previous submission's SFOC
 * launches have read the staged ones, its point sets once the previous
 * results are out, so its copies run while the previous batch is still
 * being matched.  The host buffers (inputs unchanged, outputs unread) must
 * stay valid until fastncc_wait_batch_host(ticket) returns; they must be
 * pinned for the call to return before the copies end (pageable buffers
 * make the runtime copy synchronously).  The first submission with a
 * signature builds its plan and runs as the synchronous call does.
 * Errors: as fastncc_register_batch_host, SFOC_ERR_INVALID_ARG for a NULL
 * ticket; on an error every copy and launch in flight has ended and no
 * ticket is issued. */
SFOC_API sfoc_status fastncc_submit_batch_host(sfoc_ctx* ctx, int n_pairs, const float* const* h_refs,
                                               const int* Hr, const int* Wr, const float* const* h_sens,
                                               const int* Hs, const int* Ws, const int32_t* const* h_points,
                                               const int* n_points, const int* template_size,
                                               const int* search_radius, const sfoc_params* p,
                                               const fastncc_opts* opts, fastncc_result* const* h_outs,
                                               int64_t* ticket);
/* Blocks until submission `ticket` has copied its results to its h_outs
 * (when more than four submissions are outstanding it may also wait for a
 * later one).  Ticket 0 returns at once; a ticket not yet issued by this
 * context is SFOC_ERR_INVALID_ARG.  A bounded device wait that expired is
 * reported by sfoc_ctx_sync, as for the other calls. */
SFOC_API sfoc_status fastncc_wait_batch_host(sfoc_ctx* ctx, int64_t ticket);

/* Number of batch plans the context holds; frees them all (waits for the
 * context's stream first). */
SFOC_API int sfoc_ctx_plan_count(const sfoc_ctx* ctx);
SFOC_API sfoc_status sfoc_ctx_release_plans(sfoc_ctx* ctx);
/* The most recently used plan as JSON text: kind (0 build, 1 match, 2 both),
 * pairs, items, whether it has a graph and how many kernels one run
 * launches, the SFOC waves, and per correlation class (in launch order) its
 * sfoc_corr_path, kernel class, items, launches and pairs (indices into the
 * call's arrays, in the order its items are listed); plans_built: the batch
 * plans the context has built so far.  Without a plan only plans_built.
 * *len receives the bytes needed (with the zero); buf NULL writes nothing
 * else; SFOC_ERR_INVALID_ARG when cap is smaller. */
SFOC_API sfoc_status sfoc_ctx_plan_info(const sfoc_ctx* ctx, char* buf, size_t cap, size_t* len);

/* ---- autotuner -------------------------------------------------------- */
/*
 * With SFOC_CORR_AUTO (family 0) and SFOC_CORR_IGEMM_TC (family 1) the
 * correlation form of a (cube dtype, m, R) is measured, not ruled: on the
 * first match of that key (outside a stream capture) every form of the
 * family that runs for it is launched on the first min(n, 2 x SMs) points
 * of that call (one warm-up launch, then the better of two timed with CUDA
 * events), and the fastest is kept in the context and used from then on.
 *   family 0, F32 cubes:  the Fourier correlation (where m + 2R <= 64 also
 *                         with its 128-point transform) and the direct kernel;
 *   family 0, BF16 cubes: the band, column and Toeplitz tensor-core forms and
 *                         the Fourier correlation (reading the bf16 cube);
 *   family 1 (BF16):      the tensor-core forms only.
 * The paper weighs its FFT against spatial correlation by operation counts
 * (Eq. 17-19); on this device the choice is made by measurement.  Without
 * an entry (autotuning off, or inside a capture) the fixed rule: F32 cubes
 * the Fourier form when m + 2R <= 128, else the direct kernel; BF16 cubes
 * the tensor-core form with the fewest MMAs.
 */
SFOC_API sfoc_status sfoc_ctx_set_autotune(sfoc_ctx* ctx, int enable);
/* The entry of (dtype, m, R): *corr_path = the chosen sfoc_corr_path (-1 when
 * there is none), *option = its FFT side (else 0), and per candidate timed
 * (*n_cand <= 6) its path, option and milliseconds (-1 = it failed to run);
 * *sample = the points timed.  Output pointers other than corr_path may be
 * NULL. */
SFOC_API sfoc_status sfoc_ctx_autotune_entry(const sfoc_ctx* ctx, int dtype, int m, int R, int family,
                                             int* corr_path, int* option, int* n_cand, int* cand_path,
                                             int* cand_option, float* cand_ms, int* sample);
/* The context's entries as JSON text ({"sfoc_autotune": 1, "entries":
 * [...]}).  *len receives the bytes needed including the terminating zero;
 * with buf NULL nothing else is written; SFOC_ERR_INVALID_ARG when cap is
 * smaller than that. */
SFOC_API sfoc_status sfoc_ctx_autotune_export(const sfoc_ctx* ctx, char* buf, size_t cap, size_t* len);
/* Adds (or replaces) the entries of text written by sfoc_ctx_autotune_export.
 * SFOC_ERR_INVALID_ARG, with nothing added, for text that does not parse or
 * an entry whose form does not run for its m / R. */
SFOC_API sfoc_status sfoc_ctx_autotune_import(sfoc_ctx* ctx, const char* text);

/* ---- interest points (Sec. 3.1.1) --------------------------------------- */

/*
 * Block-based FAST interest points (Sec. 3.1.1): FAST-9 on the 16 pixels of
 * the radius-3 circle, one point per block of a grid_y x grid_x partition of
 * the image (rows [by H / grid_y, (by + 1) H / grid_y), columns likewise).
 * A pixel's score is the largest threshold for which 9 contiguous circle
 * pixels are all brighter (or all darker) than it by more (FP32 differences
 * of the stored values); it is a corner when the score exceeds `threshold`.
 * Pixels closer than 3 to the border score 0.  Corners survive 3 x 3
 * non-maximum suppression when they are at least every neighbour and above
 * the neighbours before them in raster order.  Each block keeps its
 * strongest surviving corner at least `margin` pixels from the border
 * (ties: smaller y, then x).
 *   d_image   float32 image (finite values), row-major, pitch >= W elements.
 *   d_points  grid_y * grid_x x 2 int32 (x, y) per block, (-1, -1) when a
 *             block has no corner; d_scores grid_y * grid_x float32 (0 then).
 * Device memory owned by the caller; asynchronous on the context stream.
 * INVALID_ARG for null pointers, H or W < 1, pitch < W, grid sizes outside
 * [1, H] / [1, W], margin < 0 or a threshold that is negative or not finite.
 */
SFOC_API sfoc_status sfoc_fast_blocks(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems,
                                      float threshold, int grid_y, int grid_x, int margin, int32_t* d_points,
                                      float* d_scores);

/* ---- outlier rejection over the control points (Sec. 3.2.3) ------------- */

typedef enum { SFOC_MODEL_AFFINE = 0, SFOC_MODEL_PROJECTIVE = 1 } sfoc_model;

/*
 * Control-point pairs from one match.  For point k (sensed-image coordinates
 * p_k = (d_points[2k], d_points[2k+1])): d_src[2k..] = p_k, d_dst[2k..] =
 * p_k + (sub_dx, sub_dy) (its match in the reference image at the refined offset),
 * d_valid[k] = 1 when its status is SFOC_PT_OK, else 0.  d_src, d_dst: n x 2
 * doubles; d_valid: n bytes; all device memory owned by the caller.
 * Asynchronous on the context stream.  INVALID_ARG for a null pointer with
 * n > 0 or n < 0.
 */
SFOC_API sfoc_status fastncc_points_from_results(sfoc_ctx* ctx, const int32_t* d_points,
                                                 const fastncc_result* d_results, int n, double* d_src,
                                                 double* d_dst, uint8_t* d_valid);

/*
 * RANSAC (Sec. 3.2.3) with the projective transformation of the paper or an
 * affine model, in FP64 on the device:
 *   x' = (h0 x + h1 y + h2) / (h6 x + h7 y + 1),
 *   y' = (h3 x + h4 y + h5) / (h6 x + h7 y + 1)      (affine: h6 = h7 = 0).
 * d_src, d_dst: n x 2 doubles (pixels; src -> dst); d_valid: n bytes or NULL
 * (all valid).  d_samples: n_hyp x k int32 point indices, k = 4 (projective)
 * or 3 (affine): the random draws, supplied by the caller.  Coordinates are
 * normalised (the valid points' centroid to the origin, mean distance
 * sqrt(2)); each hypothesis is the exact solution on its sample and scores
 * the number of valid points within `threshold` pixels of the model's image
 * (-1 for a singular sample or an index outside [0, n)).  The highest score
 * wins (ties: the lower index); its inliers are refitted by least squares
 * and recounted, `refits` times.
 * Outputs (device memory owned by the caller): d_model 9 doubles (row-major
 * 3 x 3, d_model[8] = 1; identity when no hypothesis scored), d_inlier n
 * bytes, d_info 2 int32 (winning hypothesis or -1, inlier count), d_scores
 * n_hyp int32 per-hypothesis scores or NULL.  Uses the context workspace.
 * Asynchronous on the context stream.  INVALID_ARG for null pointers, n < 0,
 * n_hyp < 0, threshold < 0 or not finite, refits < 0 or an unknown model.
 */
SFOC_API sfoc_status fastncc_ransac(sfoc_ctx* ctx, const double* d_src, const double* d_dst, const uint8_t* d_valid,
                                    int n, int model, const int32_t* d_samples, int n_hyp, double threshold,
                                    int refits, double* d_model, uint8_t* d_inlier, int32_t* d_info,
                                    int32_t* d_scores);

/*
 * Rectification (Sec. 3.2.3, last paragraph): the sensed image resampled
 * into the reference frame with a model H (sensed -> reference, 9 doubles
 * row-major in device memory, e.g. fastncc_ransac's d_model): output pixel
 * (x, y) of the out_h x out_w image d_out takes the bilinear sample of
 * d_image at H^-1 (x, y), or `fill` outside [0, W-1] x [0, H-1].  Mapping in
 * FP64, blend in FP32.  A singular model gives an all-fill image.  Device
 * memory owned by the caller; asynchronous on the context stream.
 * INVALID_ARG for null pointers, H, W, out_h or out_w < 1, pitch < W.
 */
SFOC_API sfoc_status sfoc_rectify(sfoc_ctx* ctx, const float* d_image, int H, int W, size_t pitch_elems,
                                  const double* d_model, float fill, int out_h, int out_w, float* d_out);

#ifdef __cplusplus
}
#endif

#endif /* SFOC_GB300_H */
