/*
 * tfn.h -- C ABI of the GB300 Three-Filters-to-Normal library (libtfn.so).
 *
 * The library computes per-pixel unit surface normals and a validity mask
 * from a depth or disparity image, following Fan et al., "Three-Filters-to-
 * Normal: An Accurate and Ultrafast Surface Normal Estimator" (RA-L 2021):
 *
 *   Sec. III, Eq. (intrinsic matrix)   pinhole back-projection with fx, fy, u0, v0;
 *   Sec. III, Eq. (d1/z_to_du_dv) and the text after it: a horizontal and a
 *                                      vertical gradient filter on 1/Z;
 *   Sec. III, Eq. (nx2_ny2_nz2)        nx = fx d(1/Z)/du, ny = fy d(1/Z)/dv,
 *                                      n_z = -Phi{(dx_j nx + dy_j ny)/dz_j}, j = 1..8,
 *                                      Phi = mean or median (the third filter);
 *   Sec. III, special case             equal depths -> n = [0, 0, -1];
 *   Sec. III, Eqs. (z_d), (nx2_ny2_nz3) the same estimator on a disparity image.
 *
 * Readings where the paper is silent (holes, borders, orientation, the
 * median of an even count) are fixed as follows and are identical in the
 * CPU reference used by the tests:
 *   - a sample is a hole unless it is finite and 2^-16 <= value <= 2^16
 *     (TFN_DISP_U16: unless the raw value is non-zero);
 *   - a pixel is evaluable iff it and every tap with a non-zero weight in
 *     either gradient filter are inside the image and not holes (FD: the 4
 *     axis neighbours; Sobel, Scharr, Prewitt: all 8; the 5x5 filters: up to
 *     2 pixels out); other pixels get normal (0,0,0), mask 0;
 *   - neighbours that are holes or have the centre's depth give no candidate;
 *   - the median of an even count is the mean of the two middle candidates;
 *   - if both gradients are exactly zero, or no neighbour gives a candidate
 *     (every valid neighbour at the centre's depth), the normal is [0, 0, -1];
 *   - the normal is n = -n'/|n'|, n' = (nx, ny, n_z): it faces the camera.
 *
 * Memory.  Every image pointer in a tfn_frame is a DEVICE pointer owned by
 * the caller; the library never frees it.  Rows of every image must start on
 * 16-byte boundaries (pointer and pitches multiples of 16 bytes), else
 * TFN_ERR_MISALIGNED.  The context owns only its scratch (frame descriptors,
 * TMA tensor maps, the list of pixels to refine, staging buffers of the
 * host-buffer path, a status word).  A launch may enqueue a second, small
 * kernel after the main one (the double-float redo of the rare pixels whose
 * FP32 error bound is too loose); both are on the caller's stream.
 *
 * Streams and errors.  Calls that take a stream validate their arguments
 * synchronously, return a status, and then enqueue work on that stream
 * (NULL = legacy default stream); outputs are valid once the stream reaches
 * that point.  No C++ exception crosses the ABI.  A context is not
 * thread-safe: use one per host thread or lock around it.  A context uses the
 * CUDA device that was current when it was created; calls switch to that
 * device for their duration.
 */
#ifndef TFN_H
#define TFN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tfn_stream; /* a cudaStream_t */
typedef struct tfn_ctx tfn_ctx;

typedef enum tfn_status {
    TFN_OK = 0,
    TFN_ERR_INVALID_ARG = 1,   /* null pointer, bad size, non-finite intrinsics, bad enum */
    TFN_ERR_UNSUPPORTED = 2,   /* a valid but unsupported combination (disparity with fx != fy) */
    TFN_ERR_MISALIGNED = 3,    /* a pointer or pitch not a multiple of 16 bytes */
    TFN_ERR_OUT_OF_MEMORY = 4, /* scratch would exceed the context's memory budget */
    TFN_ERR_CUDA = 5,          /* a CUDA runtime/driver call failed (see tfn_last_cuda_error) */
    TFN_ERR_TIMEOUT = 6,       /* a host-side wait ran out of time */
    TFN_ERR_CANCELLED = 7,     /* a request was cancelled before it ran */
    TFN_ERR_BUSY = 8,          /* admission refused: no slot or memory free right now */
    TFN_ERR_DEVICE = 9,        /* a kernel reported a failed bounded wait (tfn_device_status) */
    TFN_ERR_IO = 10            /* a file could not be opened, read or written */
} tfn_status;

/* Input sample types. */
typedef enum tfn_input {
    TFN_DEPTH_F32 = 0, /* depth Z, any length unit, float32 */
    TFN_DEPTH_F16 = 1, /* depth Z, IEEE binary16 */
    TFN_DISP_U16 = 2,  /* stereo disparity, unsigned 16-bit fixed point (0 = hole) */
    TFN_DISP_F32 = 3   /* stereo disparity in pixels, float32 */
} tfn_input;

/* Gradient filters (Sec. III; Sec. IV-B compares them): correlation with
 * [-1 0 1] horizontally (its transpose vertically), row weights
 * FD (0 1 0), Sobel (1 2 1), Scharr (3 10 3), Prewitt (1 1 1), or any row
 * weights (w0 w1 w2) given in tfn_method.weights (TFN_GRAD_WEIGHTED: the 3x3
 * kernels of the paper's brute-force kernel search, Sec. IV-B).
 *
 * 5x5 filters (Fig. 2 compares filter types and sizes): separable, an
 * antisymmetric derivative profile (d1 at offsets +-1, d2 at +-2) along the
 * filter's axis times a symmetric smoothing profile (s0 at 0, s1 at +-1, s2 at
 * +-2) across it; TFN_GRAD_SEP5 takes (d1 d2 s0 s1 s2) in tfn_method.weights
 * (d1 + 2 d2 and s0 + 2 s1 + 2 s2 must be non-zero), and the named members
 * fix them: FD5 (8 -1 | 1 0 0), the fourth-order central difference, Sobel5
 * (2 1 | 6 4 1) and Prewitt5 (1 2 | 1 1 1).  The candidates and Phi keep the
 * 8-connected neighbourhood.
 *
 * A pixel is evaluable when it and every tap with a non-zero weight in either
 * filter are valid (a 5x5 filter with d2 or s2 non-zero leaves a 2-pixel
 * border). */
typedef enum tfn_grad {
    TFN_GRAD_FD = 0,
    TFN_GRAD_SOBEL = 1,
    TFN_GRAD_SCHARR = 2,
    TFN_GRAD_PREWITT = 3,
    TFN_GRAD_WEIGHTED = 4,
    TFN_GRAD_SEP5 = 5,
    TFN_GRAD_FD5 = 6,
    TFN_GRAD_SOBEL5 = 7,
    TFN_GRAD_PREWITT5 = 8
} tfn_grad;

/* Phi of Eq. (nx2_ny2_nz2). */
typedef enum tfn_phi { TFN_PHI_MEAN = 0, TFN_PHI_MEDIAN = 1 } tfn_phi;

/* Output layouts.  Planar: three planes (x, y, z) of H rows each, element
 * type float32 / float16 / bfloat16.  Packed: one plane of 4 x 16-bit per
 * pixel (x, y, z, 0). */
typedef enum tfn_output {
    TFN_OUT_F32 = 0,
    TFN_OUT_F16 = 1,
    TFN_OUT_BF16 = 2,
    TFN_OUT_F16X4 = 3,
    TFN_OUT_BF16X4 = 4,
    TFN_OUT_OCT16 = 5 /* one plane of 2 x int16 per pixel: the octahedral code of the unit
                         normal (see below) */
} tfn_output;

/* TFN_OUT_OCT16: the octahedral map of Cigolle et al. ("A Survey of Efficient
 * Representations for Independent Unit Vectors", JCGT 3(2), 2014): for the
 * unit normal (x, y, z), p = (x, y) / (|x| + |y| + |z|), and where z < 0,
 * p = ((1 - |p_y|) s(p_x), (1 - |p_x|) s(p_y)) with s(t) = +1 for t >= 0, else
 * -1; each component is stored as round-to-nearest-even(p * 32767).  Decode:
 * v = (p_x, p_y, 1 - |p_x| - |p_y|), unfold where v_z < 0 the same way,
 * normalise.  Non-evaluable pixels store (0, 0).  16-bit codes keep every
 * direction within 0.005 degrees. */

/* Pinhole intrinsics (Sec. III, Eq. intrinsic matrix), in pixels.  For
 * disparity input fx must equal fy (= f of Eq. z_d) and `baseline` is the
 * stereo baseline t_c (> 0); both cancel from the normal's direction. */
typedef struct tfn_camera {
    float fx, fy, u0, v0;
    float baseline;
} tfn_camera;

/* One image and where its results go.  All pointers are device pointers. */
typedef struct tfn_frame {
    const void *input;            /* height rows of input_pitch bytes */
    int64_t input_pitch;          /* bytes, multiple of 16, >= width * sample size */
    int32_t height, width;        /* each >= 1 and <= 32768 */
    int32_t input_type;           /* tfn_input */
    float disp_scale;             /* pixels per raw unit for TFN_DISP_U16 (e.g. 1/16) */
    tfn_camera cam;
    void *normals;                /* planar: plane c at normals + c * normals_plane_stride */
    int64_t normals_pitch;        /* bytes per row, multiple of 16 */
    int64_t normals_plane_stride; /* bytes between planes (planar layouts), multiple of 16 */
    uint8_t *mask;                /* height rows of mask_pitch bytes: 1 = evaluable, 0 = not */
    int64_t mask_pitch;           /* bytes, multiple of 16 */
    /* Optional point cloud written in the same pass (NULL: none): three float32
     * planes (X, Y, Z) at points + c * points_plane_stride, height rows of
     * points_pitch bytes; every valid sample's back-projection p = (Z (u -
     * u0)/fx, Z (v - v0)/fy, Z) (Sec. III, Eq. intrinsic matrix; disparity
     * input: Z = f t_c / d, Eq. z_d), holes (0, 0, 0). */
    void *points;
    int64_t points_pitch;         /* bytes, multiple of 16, >= width * 4 */
    int64_t points_plane_stride;  /* bytes, multiple of 16, >= points_pitch * height */
} tfn_frame;

/* Estimators.  TFN_EST_3F2N is the paper's method (Sec. III).  TFN_EST_PLANEPCA
 * is the comparison estimator of Sec. II, item 2 (Eq. planepca): the 9 back-projected
 * points of the 3x3 neighbourhood (Eq. intrinsic matrix) have their mean
 * removed, and the normal is the principal component of smallest variance,
 * turned to face the camera (n . p < 0).  A pixel is evaluable when it and
 * its 8 neighbours are valid.  It has no gradient filter and no Phi: grad,
 * phi and weights are ignored.  FP32 arithmetic; its direction error grows
 * as the two smallest eigenvalues of the scatter matrix approach each other
 * (the estimator itself is ill-conditioned there). */
typedef enum tfn_estimator { TFN_EST_3F2N = 0, TFN_EST_PLANEPCA = 1 } tfn_estimator;

/* Method selection. */
typedef struct tfn_method {
    int32_t grad;      /* tfn_grad */
    int32_t phi;       /* tfn_phi */
    int32_t output;    /* tfn_output */
    int32_t flags;     /* TFN_FLAG_* */
    float weights[5];  /* TFN_GRAD_WEIGHTED: row weights (w0 w1 w2), finite, not all 0;
                          TFN_GRAD_SEP5: (d1 d2 s0 s1 s2), finite; else ignored */
    int32_t estimator; /* tfn_estimator (0: the paper's 3F2N) */
} tfn_method;

/* Compute every pixel on the compensated (double-float) path instead of only
 * the rare pixels whose FP32 error bound is too loose.  For testing. */
#define TFN_FLAG_REFINE_ALL 1
/* Test hook for the failure path: the first warp of each launch, before it
 * issues any copy, waits on a barrier that nothing completes, gives up after
 * about 1 ms through the same bounded wait that a TMA copy that never lands
 * would run out, sets the failed-wait bit in the status word and leaves its
 * work items unprocessed.  The launch then reports the failure as a real one
 * would (tfn_device_status, a server batch's TFN_ERR_DEVICE) and the context
 * stays usable.  For testing. */
#define TFN_FLAG_TEST_WAIT_TIMEOUT 2
/* FP16 depth with the FD filter: compute each pixel's FP32 error bound and
 * refinement test even where the frames' binary16 sample spacing already
 * proves that no pixel can fail it (there the library otherwise runs a kernel
 * without them: the same normals and masks, bit for bit, with fewer
 * instructions).  For testing and for measuring the bound's cost. */
#define TFN_FLAG_FULL_BOUND 4

/* ---- status and context ------------------------------------------------ */

/* Static string for a status code. */
const char *tfn_status_string(tfn_status status);

/* Library version string. */
const char *tfn_version(void);

/* Text of the last CUDA error seen by this thread (static storage). */
const char *tfn_last_cuda_error(void);

/* Creates a context on `device` (-1: the current device).  Scratch that the
 * context allocates never exceeds `mem_budget_bytes` (0: no limit).  On
 * failure *ctx is NULL. */
tfn_status tfn_create(tfn_ctx **ctx, int device, size_t mem_budget_bytes);

/* Releases the context's scratch; waits for its work to finish. NULL is a no-op. */
tfn_status tfn_destroy(tfn_ctx *ctx);

/* ---- the estimator --------------------------------------------------------- */

/* Normals of one frame: Sec. III end to end, one fused kernel launch. */
tfn_status tfn_normals(tfn_ctx *ctx, const tfn_frame *frame, const tfn_method *method, tfn_stream stream);

/* Normals of n frames (any mix of sizes, input types and intrinsics) in one
 * persistent launch that walks a tile queue spanning all frames.  Frame
 * descriptors are uploaded through the context's scratch; a call with the
 * same frames and method as the previous one reuses them. */
tfn_status tfn_normals_batch(tfn_ctx *ctx, const tfn_frame *frames, int n, const tfn_method *method,
                             tfn_stream stream);

/* ---- tile shapes ------------------------------------------------------------ */

/* Number of tile shapes the kernels are compiled for. */
int tfn_tile_shape_count(void);

/* Tile width and height in pixels and pixel rows per thread of shape `index`
 * (each thread computes 4 columns x rows_per_thread pixels). */
tfn_status tfn_tile_shape_info(int index, int *tile_w, int *tile_h, int *rows_per_thread);

/* Warps per thread block (CTA) of shape `index`: for the 3x3 filters (FD,
 * Sobel, Scharr, Prewitt, the weighted family: *warps_3x3) and for the 5x5
 * filters and PlanePCA (*warps_other).  Shapes that share a height differ in
 * these widths; a work item is always one warp's.  (An interface of this
 * library: the paper has no counterpart.) */
tfn_status tfn_tile_shape_warps(int index, int *warps_3x3, int *warps_other);

/* Forces the tile shape used by later calls of this context; index -1 (the
 * default) uses the context's tune table (see tfn_autotune), and for
 * combinations the table does not hold, shape 1 (the tallest items), or a
 * shape of short work items when a launch has too few items to occupy the
 * GPU (one or a few small frames).  Results do not depend on the shape; speed does.  Plans and
 * batches built before the call keep their shape. */
tfn_status tfn_set_tile_shape(tfn_ctx *ctx, int index);

/* Autotuner.  Times every compiled tile shape on the caller's batch (`reps`
 * timed runs of tfn_normals_batch each, after one untimed run; CUDA events on
 * `stream`; the outputs are written as by tfn_normals_batch) and records the
 * fastest in the context's tune table for each input type in the batch with
 * the method's gradient, phi and output.  Returns the chosen index in *best
 * and, if ms_per_shape is not NULL, the mean milliseconds per run of each
 * shape in ms_per_shape[0 .. tfn_tile_shape_count()).  Synchronises `stream`.
 * A forced shape (tfn_set_tile_shape >= 0) stays forced. */
tfn_status tfn_autotune(tfn_ctx *ctx, const tfn_frame *frames, int n, const tfn_method *method, int reps,
                        tfn_stream stream, int *best, float *ms_per_shape);

/* The tune table's shape for (input_type, method's grad/phi/output), or -1
 * in *index if the table holds none. */
tfn_status tfn_tuned_shape(tfn_ctx *ctx, int input_type, const tfn_method *method, int *index);

/* Writes the tune table to a text file: a version line, a line naming the
 * device (name, SM count, compute capability), one line per entry with the
 * tile geometry and the time measured.  TFN_ERR_IO if the file cannot be
 * written. */
tfn_status tfn_tune_cache_save(tfn_ctx *ctx, const char *path);

/* Reads a file written by tfn_tune_cache_save into the tune table (entries
 * replace existing ones; shapes this build does not compile are skipped).
 * TFN_ERR_IO: cannot be read; TFN_ERR_INVALID_ARG: not a well-formed cache
 * (nothing is loaded); TFN_ERR_UNSUPPORTED: tuned on another kind of device
 * (nothing is loaded). */
tfn_status tfn_tune_cache_load(tfn_ctx *ctx, const char *path);

/* ---- plans: a frozen batch replayed as a CUDA graph ---------------------- */

typedef struct tfn_plan tfn_plan;

/* Freezes a batch (frames, pointers, shapes, intrinsics, method): validates it
 * as tfn_normals_batch does, uploads its frame descriptors and TMA tensor maps
 * once into scratch the plan owns (counted against the context's budget;
 * this call synchronises), and captures its kernel launches into a CUDA
 * graph.  The images themselves are not copied: the plan reads and writes the
 * caller's buffers each time it is launched. */
tfn_status tfn_plan_create(tfn_ctx *ctx, const tfn_frame *frames, int n, const tfn_method *method, tfn_plan **plan);

/* Replays the plan's graph on `stream`: the whole estimator over the batch,
 * with no host work beyond one graph launch. */
tfn_status tfn_plan_launch(tfn_plan *plan, tfn_stream stream);

/* Number of kernel launches one tfn_plan_launch runs (per input kind of the
 * batch: normals_kernel, and the refinement kernel where the launch can flag
 * pixels and refines them in a second kernel: not for the FD mean, whose
 * kernel refines its own, nor for the short items of small launches). */
tfn_status tfn_plan_kernels(const tfn_plan *plan, int32_t *count);

/* The name of kernel `index` (0 .. tfn_plan_kernels - 1, in the order the
 * plan's graph lists its kernel nodes) as the compiler emitted it: a mangled
 * C++ name whose template arguments give the instance (input kind, filter,
 * Phi, tile shape, and whether it is the form without the error bound), as a
 * profiler lists it.  `*name` points into the CUDA runtime's own storage and
 * stays valid while the library is loaded.  No counterpart in the paper:
 * introspection of which compiled kernel a plan replays.  Errors:
 * TFN_ERR_INVALID_ARG for a NULL argument or an index out of range,
 * TFN_ERR_CUDA if the runtime cannot name the kernel. */
tfn_status tfn_plan_kernel_name(const tfn_plan *plan, int32_t index, const char **name);

/* Waits for the device, releases the plan's scratch and graph. NULL is a no-op. */
tfn_status tfn_plan_destroy(tfn_plan *plan);

/* Same as tfn_normals_batch, but every pointer in `frames` is a HOST pointer
 * (page-locked memory is fastest).  The context stages the frames through
 * device buffers in chunks, overlapping host-to-device copies, kernels and
 * device-to-host copies; returns after every output is in host memory. */
tfn_status tfn_normals_batch_host(tfn_ctx *ctx, const tfn_frame *frames, int n, const tfn_method *method,
                                  tfn_stream stream);

/* Reads and clears the device status word that kernels of this context set
 * when a bounded wait gave up (0: none).  Synchronises `stream`. */
tfn_status tfn_device_status(tfn_ctx *ctx, uint32_t *bits, tfn_stream stream);

/* Reads and clears the number of pixels that kernels of this context sent to
 * the double-float path (whose FP32 error bound was too loose; see the
 * accuracy notes of the kernel).  Diagnostics; counts wrap at 2^32.
 * Synchronises `stream`. */
tfn_status tfn_refined_pixels(tfn_ctx *ctx, uint64_t *count, tfn_stream stream);

/* ---- serving: a request server with continuous batching ------------------- */

/* A thread-safe server that takes single frames from any number of client
 * threads and runs them in batches: requests queue up while earlier batches
 * run, and each time one of its pipelines frees up the server admits as many
 * queued requests as fit -- in arrival order, at most max_batch_frames, with
 * their device staging inside the memory budget -- and computes them with one
 * persistent launch per input type (the tfn_normals_batch path).  A
 * request's result does not depend on which other requests share its batch.
 * (The paper has no serving layer; this is the library's.) */
typedef struct tfn_server tfn_server;

typedef struct tfn_server_opts {
    tfn_method method;        /* gradient, phi, output layout and flags of every request */
    size_t mem_budget_bytes;  /* device memory for staging host-buffer requests (0: 1 GiB); allocated once */
    int32_t max_batch_frames; /* most requests per batch (0: 256) */
    int32_t max_queue;        /* most requests waiting for admission (0: 65536) */
    int32_t max_delay_us;     /* hold a partial batch up to this long after its oldest request
                                 arrived while the device is busy (0: never hold) */
    int32_t pipelines;        /* batches in flight at once, 1..4 (0: 2) */
    int32_t flags;            /* TFN_SERVER_* */
} tfn_server_opts;

/* tfn_server_opts flag: launch each batch's kernels directly instead of
 * replaying them from the pipeline's CUDA graphs (for comparison). */
#define TFN_SERVER_NO_GRAPHS 1

/* tfn_submit flag: the frame's pointers are HOST pointers (page-locked
 * memory is fastest); the server copies the input into device staging memory
 * and the results back.  Without it they are device pointers, used in place. */
#define TFN_REQ_HOST 1
/* tfn_submit flag: the request's batch is launched with
 * TFN_FLAG_TEST_WAIT_TIMEOUT, so that batch fails with TFN_ERR_DEVICE.  For
 * testing. */
#define TFN_REQ_TEST_WAIT_TIMEOUT 2

typedef struct tfn_serving_stats {
    uint64_t submitted, completed, failed, cancelled;
    uint64_t rejected;           /* submissions refused with TFN_ERR_BUSY */
    uint64_t batches;            /* batches launched */
    uint64_t pixels;             /* pixels of completed requests */
    double elapsed_s;            /* since creation or the last reset */
    double frames_per_s;         /* completed / elapsed_s */
    double mean_batch_frames;
    double latency_p50_us;       /* submit -> results in the client's buffers, over the */
    double latency_p99_us;       /* last latency_samples (at most 65536) completions */
    double latency_max_us;
    uint64_t latency_samples;
    int32_t queued;              /* requests waiting for admission */
    int32_t in_flight;           /* requests admitted and not yet complete */
    size_t staging_bytes_in_use;
    size_t staging_bytes_capacity;
    uint64_t graph_launches;        /* batches whose kernels were replayed from a CUDA graph */
    uint64_t max_batches_in_flight; /* most batches launched and not yet retired at once */
    uint64_t admitted_while_busy;   /* requests admitted while an earlier batch was in flight */
    uint64_t device_overlaps;       /* batches whose kernels started on the device before the
                                       previous batch's kernels had finished (CUDA events) */
    uint64_t graph_captures;        /* of graph_launches, those whose graph was captured first
                                       (a new combination of input kinds and tile shapes, or one
                                       evicted from the pipeline's 64 graphs since) */
} tfn_serving_stats;

/* Creates a server on ctx's device.  The server owns a context of its own
 * (copying ctx's tune table and forced tile shape), two threads, its streams
 * and the staging memory; ctx stays free for other use.  On failure *srv is
 * NULL. */
tfn_status tfn_server_create(tfn_ctx *ctx, const tfn_server_opts *opts, tfn_server **srv);

/* Queues one frame; on success *ticket identifies it for tfn_wait.  The
 * frame is validated here (as tfn_normals_batch does; host-buffer requests
 * need no alignment).  TFN_ERR_BUSY: the queue is full (nothing queued);
 * TFN_ERR_OUT_OF_MEMORY: the frame's staging is larger than the whole budget.
 * The server runs on streams of its own: a device-buffer input must be
 * complete (the work that produced it synchronised) before the call, and the
 * caller's buffers must stay valid until the request completes. */
tfn_status tfn_submit(tfn_server *srv, const tfn_frame *frame, int flags, uint64_t *ticket);

/* Waits at most timeout_ms (>= 0; 0 polls) for the request.  TFN_OK: it
 * finished and *result holds its status (TFN_OK: outputs written;
 * TFN_ERR_CANCELLED: the server was destroyed before it was admitted;
 * TFN_ERR_DEVICE: a kernel of its batch gave up a bounded wait (each batch
 * reports only its own kernels' waits); TFN_ERR_CUDA); the ticket is then
 * released.  TFN_ERR_TIMEOUT: not finished yet (wait again).
 * TFN_ERR_INVALID_ARG: unknown or already released ticket.  Never blocks
 * longer than the limit. */
tfn_status tfn_wait(tfn_server *srv, uint64_t ticket, int32_t timeout_ms, tfn_status *result);

/* Counters and latency percentiles; reset != 0 restarts them after reading. */
tfn_status tfn_server_stats(tfn_server *srv, tfn_serving_stats *stats, int reset);

/* Stops admitting, cancels queued requests, waits for the batches in flight,
 * joins the threads and frees everything.  No call on srv may be running or
 * follow.  NULL is a no-op. */
tfn_status tfn_server_destroy(tfn_server *srv);

/* ---- without any allocation ------------------------------------------------- */

/* Largest n that tfn_normals_noalloc accepts. */
#define TFN_NOALLOC_MAX_FRAMES 64

/* Same result as tfn_normals_batch (the same kernels, bit for bit), for
 * callers that may not allocate device memory at all:
 *   - a host framework or plugin interface that owns every device byte: its
 *     memory plan is fixed before it calls plugins, so a plugin's own
 *     cudaMalloc would overrun that plan or fail;
 *   - a loop with a latency budget: cudaMalloc and cudaFree can synchronise
 *     the whole device, stalling every stream, not only the caller's;
 *   - a caller that cannot keep a context (tfn_create allocates its scratch).
 * (The paper has no counterpart: this is an interface concern of this
 * library.)
 *
 * It takes no context.  The scratch the kernels need (frame descriptors, TMA
 * tensor maps, a status word, the list of pixels to refine; about 540 KB, of
 * which 512 KB is the refinement list) lives in one fixed array compiled into
 * the library, which every device that loads the library keeps until the
 * process exits.  Limits and behaviour:
 *   - n > TFN_NOALLOC_MAX_FRAMES returns TFN_ERR_INVALID_ARG before anything
 *     is enqueued; otherwise arguments are validated as for tfn_normals_batch;
 *   - works on the current CUDA device; the first call on each device looks
 *     up the array's device address there;
 *   - it calls no cudaMalloc, cudaFree or other allocating routine; the
 *     descriptors are staged in thread-local host storage and copied into the
 *     array on `stream` from that pageable memory, which the CUDA runtime may
 *     stage by first waiting for the work already queued on `stream`: the call
 *     can block the host until that work is done;
 *   - each call zeroes the refinement list's header on `stream` before its
 *     kernels, so a call never sees an earlier call's list;
 *   - every call reuses the same array and overwrites the previous call's
 *     contents, so calls whose GPU work overlaps (other streams, or earlier
 *     work still running on another stream) race and must be serialised by
 *     the caller;
 *   - TFN_ERR_UNSUPPORTED: `stream` is in a state in which the staged copy
 *     cannot be enqueued for this call alone; nothing is enqueued;
 *   - kernel-side wait failures are not reported (there is no context to
 *     hold them); use tfn_normals_batch where that matters. */
tfn_status tfn_normals_noalloc(const tfn_frame *frames, int n, const tfn_method *method, tfn_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TFN_H */
