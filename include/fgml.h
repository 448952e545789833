/*
 * fgml — multi-level foreground estimation on GB300 (sm_103a).
 *
 * C ABI of the library libfgml.so. The method is the multi-level foreground/background
 * estimation of Germer, Uelwer, Conrad and Harmeling, "Fast Multi-Level Foreground
 * Estimation": given an RGB image I and an alpha matte alpha it computes a foreground F
 * and a background B by running, on an image pyramid from 1x1 up to the input size,
 * a fixed number of per-pixel closed-form 2x2 solves per level (Algorithm 1; the solve
 * is the g = (U U^T + R^T V R)^{-1} (I U + R^T V h) of Section III-C).
 *
 * Conventions shared by every entry point
 *  - Images are row-major, y outer, x inner. I, F and B hold 3 interleaved channels per
 *    pixel, alpha one. row_pitch_bytes is the distance between rows in bytes; it must be
 *    at least w * channels * element size and a multiple of the element size.
 *  - Values are in [0, 1]. Elements are float32, bfloat16 or float16 (fg_dtype); the
 *    solves always run in float32. All images of one call share one dtype.
 *  - Pointers named "device" are CUDA device memory of the current device; the caller
 *    owns them. The library owns its workspace (intermediate pyramid levels), one per
 *    (device, stream), allocated on first use and kept until fg_release_workspace().
 *  - Calls that take a stream are asynchronous on that stream (NULL = legacy default
 *    stream) unless stated otherwise; errors of the launch itself are returned, errors
 *    of the running kernels surface at the next synchronisation.
 *  - Every entry point returns an fg_status; nothing is thrown across the ABI. The
 *    message of the last error of the calling thread is fg_last_error().
 *  - Widths and heights are in [1, 32767].
 */
#ifndef FGML_H
#define FGML_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FG_OK = 0,
    FG_ERR_INVALID_ARG = 1,   /* null pointer, bad size, pitch, dtype or parameter */
    FG_ERR_OOM = 2,           /* workspace allocation failed */
    FG_ERR_CUDA = 3,          /* a CUDA runtime call failed; see fg_last_error() */
    FG_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    FG_ERR_RANGE = 5,         /* input outside [0, 1] or NaN (only when FGML_DEBUG=1) */
    FG_ERR_BUSY = 6,          /* a resource is in use (server full, etc.) */
    FG_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} fg_status;

typedef enum { FG_F32 = 0, FG_BF16 = 1, FG_F16 = 2 } fg_dtype;

/*
 * Update orders of the per-pixel solves of one iteration (Algorithm 1 iterates the
 * closed-form update of Section III-C; the order of the updates inside an iteration is
 * not fixed by the method's result, only by its convergence).
 *  FG_ORDER_JACOBI:   every pixel of iteration t+1 reads iteration t (the default).
 *  FG_ORDER_REDBLACK: an iteration updates the pixels with x + y even, then those with
 *                     x + y odd, each reading the latest values; a pixel reads only
 *                     pixels of the other colour (or itself at a clamped border), so the
 *                     result does not depend on the order inside a colour. Levels run in
 *                     tiles with a halo of 2 cells per iteration; fg_estimate_batch and
 *                     the server run red-black image by image.
 */
typedef enum { FG_ORDER_JACOBI = 0, FG_ORDER_REDBLACK = 1 } fg_order;

/*
 * Parameters of Algorithm 1. fg_params_default() fills the paper's values:
 * eps_r = 5e-3 and omega = 0.1 (Section IV-F), 10 iterations on levels that fit in
 * 32 x 32 and 2 on the others (Section III-D), clamping to [0, 1] (Algorithm 1), and a
 * 1x1 starting F = B = 0 (Algorithm 1).
 */
typedef struct {
    float eps_r;       /* regularisation epsilon_r > 0 */
    float omega;       /* alpha-gradient weight omega >= 0 */
    int small_size;    /* a level is "small" if w_l <= small_size and h_l <= small_size */
    int small_iters;   /* sweeps on small levels, >= 0 */
    int big_iters;     /* sweeps on the other levels, >= 0 */
    int order;         /* fg_order: FG_ORDER_JACOBI or FG_ORDER_REDBLACK */
    int clamp;         /* nonzero: clamp F and B to [0, 1] after each solve */
    float init;        /* value of the 1x1 starting F and B */
} fg_params;

/* An image in memory (see the conventions above for layout and pitch). */
typedef struct {
    void *ptr;
    int w;
    int h;
    long long row_pitch_bytes;
    fg_dtype dtype;
} fg_image;

/* Fills *p with the paper's parameters. */
void fg_params_default(fg_params *p);

/*
 * Level schedule of Algorithm 1 for a w x h input: n_l = max(1, ceil(log2(max(w, h))))
 * levels; level l (1-based) is round(w^(l/n_l)) x round(h^(l/n_l)) with round(x) =
 * floor(x + 0.5); its sweep count is small_iters if it fits in small_size x small_size,
 * else big_iters. Writes level l to ws[l-1], hs[l-1], ks[l-1] (any of them may be
 * NULL). Returns n_l, or -1 if w or h is out of range or n_l > cap. Host-only.
 */
int fg_schedule(int w, int h, const fg_params *p, int *ws, int *hs, int *ks, int cap);

/*
 * Multi-level foreground estimation (Algorithm 1) of one image, on the GPU.
 *  I:     device, w x h x 3; alpha: device, w x h (same w, h, dtype as I).
 *  F, B:  device, w x h x 3 outputs, same dtype; must not overlap the inputs.
 *  params: NULL for the paper's defaults.
 *  stream: cudaStream_t (NULL = default stream). Asynchronous.
 * Update order: params->order (Jacobi by default). Levels whose F/B fit in one SM's shared
 * memory run in one persistent block; each larger level runs as one pass (two sweeps fused)
 * through HBM. Inputs are not validated on this path; with the environment variable
 * FGML_DEBUG=1 the call first checks that I and alpha are in [0, 1] without NaN
 * (synchronising the stream) and returns FG_ERR_RANGE otherwise. Large inputs whose rows
 * are not on the 16-byte grid are copied once into a row-aligned workspace copy.
 * Errors: FG_ERR_INVALID_ARG for bad images/params, FG_ERR_OOM if the workspace cannot
 * be allocated, FG_ERR_CUDA for a failed launch, FG_ERR_RANGE (checked inputs only).
 */
fg_status fg_estimate(const fg_image *I, const fg_image *alpha, const fg_params *params,
                      fg_image *F, fg_image *B, void *stream);

/*
 * fg_estimate followed by compositing the foreground onto a new background (Section I,
 * the compositing equation I = alpha F + (1 - alpha) B, applied with a new background):
 *   I_new = alpha F + (1 - alpha) B_new   at every pixel,
 * written by the last level's pass as it stores F, so F is never read back.
 *  I, alpha, params, F, B: as fg_estimate (F and B are still written).
 *  B_new: device, w x h x 3, the new background; I_new: device, w x h x 3 output.
 *  One dtype for all images; the composite is formed in float32 from F's float32
 *  value (before F itself is rounded to the storage type) and rounded once.
 *  I_new must not overlap any other image; F and B must not overlap B_new.
 * Asynchronous on `stream`, like fg_estimate.
 */
fg_status fg_estimate_composite(const fg_image *I, const fg_image *alpha, const fg_params *params,
                                fg_image *F, fg_image *B, const fg_image *B_new, fg_image *I_new,
                                void *stream);

/*
 * As fg_estimate, but I, alpha, F and B are HOST memory (tightly packed, element type
 * dtype). The library copies the inputs to its device staging buffers, runs the
 * method and copies F and B back, all on `stream`, and returns when F and B are in host
 * memory. Page-locked host buffers give the fastest copies.
 */
fg_status fg_estimate_host(const void *I, const void *alpha, int w, int h, fg_dtype dtype,
                           const fg_params *params, void *F, void *B, void *stream);

/*
 * As fg_estimate_host, but returns once the copies and the solve are enqueued on `stream`
 * (no synchronisation; the paper has no counterpart). For a sequence of images: calls on
 * two or more streams overlap one image's copy back with the next image's copy in and
 * solve, since the host link carries both directions at once. The host buffers must stay
 * valid and unchanged until the stream has passed the call (fg_sync, an event);
 * page-locked buffers are needed for the copies to run asynchronously. Each stream has its
 * own staging buffers; calls on one stream run in order.
 */
fg_status fg_estimate_host_async(const void *I, const void *alpha, int w, int h, fg_dtype dtype,
                                 const fg_params *params, void *F, void *B, void *stream);

/*
 * One pass of the level update, for testing a level in isolation:
 * the level is w x h; I_l and alpha_l are the nearest resize of the full-resolution I
 * and alpha (Algorithm 1: resize from the input); the starting F and B are the nearest
 * resize of (F_src, B_src) (a previous level, or this level itself); `iters` Jacobi
 * sweeps (1..2 per pass, >2 runs several passes through the workspace) are written to
 * (F_dst, B_dst), which must be w x h and must not overlap F_src/B_src. F_src and B_src
 * must each be readable over h x row_pitch_bytes bytes (the last row's padding too, as
 * with a pitched allocation).
 */
fg_status fg_level_pass(const fg_image *I, const fg_image *alpha,
                        const fg_image *F_src, const fg_image *B_src,
                        int iters, const fg_params *params,
                        fg_image *F_dst, fg_image *B_dst, void *stream);

/*
 * fg_estimate without any device allocation. The paper has no counterpart: this entry
 * point exists for callers that cannot let the library call cudaMalloc, such as a
 * process whose device memory is all reserved up front by its own pool or budget, or a
 * latency-critical loop that cannot absorb cudaMalloc's implicit device synchronisation.
 * Arguments, layout, results and errors are those of fg_estimate (FGML_DEBUG=1 input
 * range check included), except:
 *  - the intermediate pyramid levels live in a fixed array of 64 MiB + 256 bytes inside
 *    the library (two 32 MiB level buffers and the range check's counter), held by every
 *    device that loads the library until the process exits; an image whose largest
 *    intermediate level needs more (FP32 beyond about 5.6 megapixels with the default
 *    schedule) is rejected with FG_ERR_INVALID_ARG and a message giving both sizes;
 *  - inputs whose rows are off the 16-byte grid are read in place (fg_estimate first
 *    copies them to aligned rows in its workspace), which is slower but gives the same
 *    results;
 *  - the first call on a device (and the first after a cudaDeviceReset) looks up the
 *    array's device address with that device current, so make that first call before
 *    any stream capture;
 *  - all calls share the one array: calls whose work overlaps on the GPU (different
 *    streams, or several host threads) race and corrupt each other's results; order
 *    them on one stream or serialise them. Nothing in the array needs to start at zero:
 *    each call writes every byte it later reads.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 */
fg_status fg_estimate_noalloc(const fg_image *I, const fg_image *alpha,
                              const fg_params *params, fg_image *F, fg_image *B,
                              void *stream);

/*
 * Multi-level foreground estimation of n images of any sizes (Algorithm 1 on each), as
 * one batch: one launch runs the coarse levels of every image (one block per image),
 * then one persistent launch runs every remaining level pass of every image from a work
 * list of (image, level pass, strip) items. An item waits until the pass it reads from
 * (the previous level or pass of the same image) is complete; the wait is bounded
 * (2 s) and a timeout is reported by fg_sync() as FG_ERR_TIMEOUT. Results equal those
 * of fg_estimate on each image within float32 rounding.
 *  I, alpha, F, B: arrays of n device images (F[i], B[i] the outputs of image i); one
 *  dtype for the whole batch; outputs must not overlap their own inputs.
 *  Asynchronous on `stream`; the work list and the per-image levels live in the
 *  stream's workspace.
 */
fg_status fg_estimate_batch(int n, const fg_image *I, const fg_image *alpha,
                            const fg_params *params, fg_image *F, fg_image *B, void *stream);

/*
 * Chooses the strip shape of fg_estimate_batch's work list by measurement (the paper has
 * no counterpart): runs the given batch once per candidate shape (a handful of
 * strips-per-SM / rows-per-strip settings), times two calls of each with events on
 * `stream`, and keeps the fastest as the process-wide setting of later batches (results do
 * not depend on it: every strip computes the same per-pixel updates). Arguments as
 * fg_estimate_batch (F and B are overwritten). *chosen (may be NULL): index of the chosen
 * candidate; *ms (may be NULL): its time per call. Synchronous. The environment variable
 * FGML_BATCH_STRIPS="per_sm,lo,hi" sets the starting shape instead; with
 * FGML_TUNE_CACHE=path the chosen shape is also written to that file (one line per GPU
 * model) and later processes start from it.
 */
fg_status fg_autotune_batch(int n, const fg_image *I, const fg_image *alpha,
                            const fg_params *params, fg_image *F, fg_image *B, void *stream,
                            int *chosen, float *ms);

/*
 * Diagnostic of the device-side bounded waits (not part of the method): runs the work-list
 * kernel on one item that waits for a count nothing ever reaches, with a 20 ms bound, and
 * checks that the kernel gives up, reports it through the device error word and leaves
 * the context usable. Returns FG_ERR_TIMEOUT when that happened as intended; any other
 * status is a failure. Synchronises `stream`.
 */
fg_status fg_selftest_bounded_wait(void *stream);

/* ------------------------------------------------------------------ serving
 * A server runs jobs submitted at any time with continuous batching on the current
 * device. A scheduler thread admits queued jobs in arrival order while a slot is free and
 * the job's device bytes fit in the HBM budget and the device's free memory at that
 * moment; an admitted job's pyramid (its intermediate levels) stays device-resident until
 * it completes. Host inputs are copied up and host outputs back in pieces of at most 8 MB,
 * the job with the fewest bytes left first (device inputs on the 16-byte row grid are read
 * in place). Each launch merges the next level passes of every admitted job (of one dtype)
 * whose inputs are on the device and that no running launch holds, up to step_work
 * pixel-sweeps, into one work list on an idle compute stream, so a large job advances level
 * by level across launches while later jobs join the next launches on the other streams.
 * A job completes when its last pass is done and its outputs are in place. The paper has
 * no serving layer; the method run for each job is Algorithm 1. Parameter sets the work
 * list does not run (red-black order, a level without sweeps) are served whole jobs per
 * launch.
 */
typedef struct fg_server fg_server;

typedef struct {
    int max_inflight_jobs;       /* admitted and unfinished jobs at most (default 256) */
    long long hbm_budget_bytes;  /* device bytes jobs may hold (<= 0: half the free memory at
                                    creation); admission also keeps what jobs hold below the
                                    device's free memory read at that moment, less a reserve */
    int streams;                 /* batches in flight at most, 1..16 (default 2) */
    int max_batch;               /* jobs per launch at most (default 64) */
    fg_params params;            /* method parameters for every job */
    long long step_work;         /* pixel-sweeps of level passes per launch at most (<= 0:
                                    default 16 Mi); a single larger pass runs alone */
} fg_server_cfg;

typedef struct {
    const void *I;       /* w x h x 3, packed, element type dtype (host, or device: see flags) */
    const void *alpha;   /* w x h, packed */
    int w, h;
    fg_dtype dtype;
    void *F, *B;         /* w x h x 3 outputs, written when the job is done */
    int flags;           /* FG_REQ_DEVICE_INPUT: I and alpha are device memory of the server's
                            device (read in place, no copy up); FG_REQ_DEVICE_OUTPUT: F and B
                            are device memory (written in place, no copy back) */
    void *ready_event;   /* optional cudaEvent_t: device inputs are complete once it has
                            fired (the job's launch waits for it); NULL: already complete */
} fg_request;

enum { FG_REQ_DEVICE_INPUT = 1, FG_REQ_DEVICE_OUTPUT = 2 };

typedef struct {
    long long submitted, completed, failed, batches;
    long long pixels;        /* full-resolution pixels of completed jobs */
    long long max_inflight;  /* most jobs admitted at once */
    long long max_bytes;     /* most device bytes held by jobs at once */
    long long budget_bytes;  /* the HBM budget in force */
} fg_server_stats;

/* Fills *c with defaults. */
void fg_server_cfg_default(fg_server_cfg *c);
/* Creates a server (NULL cfg: defaults) bound to the current device. */
fg_status fg_server_create(const fg_server_cfg *cfg, fg_server **out);
/* Queues a job; the host buffers must stay valid until the job is done. A job larger
 * than the whole budget is rejected with FG_ERR_INVALID_ARG. Thread-safe. */
fg_status fg_server_submit(fg_server *s, const fg_request *r, uint64_t *ticket);
/* *done = 1 once the job's outputs are in its host buffers; a failed job returns its
 * error status. */
fg_status fg_server_poll(fg_server *s, uint64_t ticket, int *done);
/* Blocks until the job is done (timeout_ms < 0: no limit); FG_ERR_TIMEOUT on timeout. */
fg_status fg_server_wait(fg_server *s, uint64_t ticket, int timeout_ms);
/* Submit and completion times of a finished job, seconds since the server started. */
fg_status fg_server_times(fg_server *s, uint64_t ticket, double *submit_s, double *done_s);
/* Forgets a finished job's record. */
fg_status fg_server_release(fg_server *s, uint64_t ticket);
/* Counters since creation. */
fg_status fg_server_get_stats(fg_server *s, fg_server_stats *out);
/* Finishes every queued and running job, then frees the server. */
void fg_server_destroy(fg_server *s);
/* Message of the calling thread's last server error. */
const char *fg_server_last_error(void);

/*
 * Converged reference (not part of the method): the minimiser of the global cost whose
 * per-pixel minimisation Algorithm 1 iterates, at full resolution and without the clamp.
 * Summing the local cost of Section III-C over the pixels, each 4-neighbour edge once:
 *   E = sum_i sum_c (alpha_i F_i + (1 - alpha_i) B_i - I_i)^2
 *     + sum_{edges {i,j}} (eps_r + omega |alpha_i - alpha_j|) sum_c [(F_i - F_j)^2 + (B_i - B_j)^2],
 * whose stationary point is the fixed point of the unclamped update. Solved by conjugate
 * gradients on grad E = 0 in float64, preconditioned by the inverse of each pixel's 2x2
 * diagonal block; E is strictly convex (a unique minimiser) when alpha is not constant.
 *  I, alpha: device images (one dtype); params: eps_r and omega are used.
 *  F, B: device float64 arrays of h x w x 3, tightly packed: the starting point on entry
 *        (zeros, or the method's output converted), the solution on return.
 *  Stops when |b - H x| <= rel_tol |b| (b = (alpha I, (1 - alpha) I)) or after max_iters
 *  iterations (checked every 32). *iters (may be NULL): iterations run;
 *  *rel_residual (may be NULL): |b - H x| / |b| recomputed from the returned x.
 * Synchronous on `stream`. Workspace: 36 doubles per pixel.
 * Errors: FG_ERR_RANGE if the iteration diverges (constant alpha).
 */
fg_status fg_minimiser_cg(const fg_image *I, const fg_image *alpha, const fg_params *params,
                          double *F, double *B, int max_iters, double rel_tol, int *iters,
                          double *rel_residual, void *stream);

/*
 * Error measures of a foreground estimate against a known foreground (Section IV-C),
 * over the pixels with 0 < alpha_gt < 1, each weighted by alpha_gt:
 *   out[0] = SAD  = sum alpha_gt |F_est - F_gt|_1
 *   out[1] = MSE  = sum alpha_gt |F_est - F_gt|_2^2
 *   out[2] = GRAD = sum alpha_gt |grad F_est - grad F_gt|_2^2
 * The norms run over the three channels (and, for GRAD, both gradient components); the
 * gradient is taken with first-order Gaussian derivative filters of sigma = 1.4 on taps
 * -6..6 (the Gaussian sampled and normalised to sum 1), image borders repeated.
 *  F_est, F_gt: device, w x h x 3; alpha_gt: device, w x h; one dtype for all three.
 *  out: host array of 3 doubles. Sums are per-block doubles added in a fixed order.
 * Synchronises `stream` (the result is on the host when the call returns).
 */
fg_status fg_quality(const fg_image *F_est, const fg_image *F_gt, const fg_image *alpha_gt,
                     double *out, void *stream);

/* Waits for `stream` and reports any device-side error of the library's kernels. */
fg_status fg_sync(void *stream);

/* Frees the workspace held for (current device, stream); the stream must be idle. */
fg_status fg_release_workspace(void *stream);

/* Message of the calling thread's last error ("" if none). Valid until its next call. */
const char *fg_last_error(void);

/* Version string of the library build. */
const char *fg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FGML_H */
