/*
 * mrirecon -- GB300 (sm_103a) library for TV-regularised multi-coil MRI
 * reconstruction with ADMM, after Lu et al., "Accelerating MRI Reconstruction
 * on TPUs" (arXiv 2006.14080).
 *
 * The non-uniform DFT of Eq. 1 is evaluated in separable form as dense
 * complex matrix products:
 *     y_c = rowsum((A_x (S_c . X)) . A_y),          A_x[k][i] = exp(-i 2 pi kx_k x_i)
 *     X   = sum_c conj(S_c) . (A_x^H diag(y_c) conj(A_y)),  A_y[k][j] = exp(-i 2 pi ky_k y_j)
 * with pixel coordinates x_i = i - nx/2, y_j = j - ny/2 (integer division) and
 * k in cycles/pixel.  The DFT is unnormalised.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Array pointers are DEVICE pointers owned by the caller unless a call says
 *    otherwise; the library never frees them and never keeps them after the
 *    call returns.  Arrays must not overlap unless a call allows it.
 *  - Complex values are interleaved complex64 (mri_c64: re, im floats), C
 *    row-major:
 *        image       [nx][ny]      (the first index is the one A_x multiplies)
 *        coil_maps   [nc][nx][ny]
 *        kspace      [nc][nk]
 *        traj        [nk][2] float (kx, ky) in cycles/pixel, nominally [-0.5, 0.5)
 *        TV fields   [2][nx][ny]   (differences along x, then along y)
 *  - Every call that takes a stream enqueues its work on that stream and
 *    returns without synchronising (except where stated).  Deferred device
 *    failures (a bounded device-side wait that gave up) are reported by
 *    mri_plan_sync_status().
 *  - Return value: MRI_OK (0) or a negative MRI_ERR_* code; the calling
 *    thread's mri_last_error() then describes the failure.  On error no
 *    output is guaranteed to be written.
 *  - A plan (mri_plan) owns the DFT factors for one trajectory and all
 *    workspace; calls on one plan must be serialised by the caller (one
 *    stream at a time).  Different plans are independent.
 */
#ifndef MRIRECON_H
#define MRIRECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MRI_API __attribute__((visibility("default")))
#else
#define MRI_API
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *mri_stream_t;

typedef struct { float re, im; } mri_c64;

typedef struct mri_plan mri_plan;

/* Status codes. */
#define MRI_OK               0
#define MRI_ERR_INVALID     -1  /* null pointer, dimension <= 0, non-finite parameter, bad enum */
#define MRI_ERR_NOMEM       -2  /* device allocation failed or a memory budget would be exceeded */
#define MRI_ERR_CUDA        -3  /* a CUDA runtime call failed */
#define MRI_ERR_TIMEOUT     -4  /* a bounded device-side wait gave up */
#define MRI_ERR_UNSUPPORTED -5  /* precision / shape combination not available */

/* Arithmetic of the two dense products inside the DFT operators. */
#define MRI_FP32   0  /* FP32 FFMA on the CUDA cores */
#define MRI_TF32   1  /* tcgen05 TF32 tensor cores: operands rounded to TF32
                         (10-bit mantissa, nearest), one product, FP32 accumulation */
#define MRI_BF16X3 2  /* tcgen05 BF16 tensor cores, hi+lo split operands, three
                         products (hi*hi + hi*lo + lo*hi), FP32 accumulation */

/* Text of the last failure on the calling thread ("" if none). */
MRI_API const char *mri_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
MRI_API int mri_version(void);

/*
 * Create a plan for an nx x ny image, nc coils and nk samples per coil, and
 * generate the DFT factors A_x, A_y for traj (device, [nk][2] float) -- the
 * per-core operator generation of Alg. 1, in separable form.  The phase
 * k*x is formed and reduced to [-1/2, 1/2] in FP64 before the FP32 sine and
 * cosine.  traj is read during the call (stream-ordered on `stream`) and not
 * kept.  precision is MRI_FP32, MRI_TF32 or MRI_BF16X3.  Allocates device memory (the
 * factors plus workspace, O(nk*(nx+ny)) + O(nc*nx*ny)); *plan receives the
 * handle, or NULL on error.
 */
MRI_API int mri_plan_create(mri_plan **plan, int nx, int ny, int nk, int nc,
                            const float *traj, int precision, mri_stream_t stream);

/* Regenerate the factors of an existing plan for a new trajectory of the
 * same nk (Alg. 1).  No allocation. */
MRI_API int mri_plan_set_trajectory(mri_plan *plan, const float *traj, mri_stream_t stream);

/* Release a plan and everything it owns.  Synchronises the device first.
 * NULL is accepted. */
MRI_API int mri_plan_destroy(mri_plan *plan);

/* Wait for all work on `stream` and report deferred device-side failures of
 * this plan (MRI_ERR_TIMEOUT when a bounded wait gave up); clears them. */
MRI_API int mri_plan_sync_status(mri_plan *plan, mri_stream_t stream);

/* Bytes of device memory the plan holds. */
MRI_API size_t mri_plan_device_bytes(const mri_plan *plan);

/* Bytes mri_plan_create would allocate for this shape on the current
 * device (0 for invalid arguments); allocates nothing. */
MRI_API size_t mri_plan_estimate_bytes(int nx, int ny, int nk, int nc, int precision);

/*
 * Forward operator F of Eq. 1-2:
 *   kspace[c][k] = sum_{i,j} coil_maps[c][i][j] image[i][j] exp(-i 2 pi (kx_k x_i + ky_k y_j))
 * image [nx][ny], coil_maps [nc][nx][ny] -> kspace [nc][nk].
 */
MRI_API int mri_nudft_forward(mri_plan *plan, const mri_c64 *image, const mri_c64 *coil_maps,
                              mri_c64 *kspace, mri_stream_t stream);

/*
 * Adjoint F^H (the inverse-DFT step of Alg. 3 followed by the coil
 * combination; the paper's cross-core partial-image sum becomes an on-chip
 * fixed-order reduction over k-space splits):
 *   image[i][j] = sum_c conj(coil_maps[c][i][j]) sum_k kspace[c][k] exp(+i 2 pi (kx_k x_i + ky_k y_j))
 * kspace [nc][nk], coil_maps [nc][nx][ny] -> image [nx][ny].
 */
MRI_API int mri_nudft_adjoint(mri_plan *plan, const mri_c64 *kspace, const mri_c64 *coil_maps,
                              mri_c64 *image, mri_stream_t stream);

/*
 * Normal operator of the x-update, Eq. 11 (linear_op of Alg. 2 / Alg. 3):
 *   out = F^H F image + (beta/2) Theta^H Theta image
 * beta = 0 gives F^H F alone.  image and out are [nx][ny] and must differ.
 */
MRI_API int mri_normal_op(mri_plan *plan, const mri_c64 *image, const mri_c64 *coil_maps,
                          float beta, mri_c64 *out, mri_stream_t stream);

/*
 * Sparsifying transform Theta (first-order finite differences, the conv1d of
 * Section IV-B, zero past the last pixel):
 *   grad[0][i][j] = image[i+1][j] - image[i][j],  grad[1][i][j] = image[i][j+1] - image[i][j]
 * image [nx][ny] -> grad [2][nx][ny].  Needs no plan.
 */
MRI_API int mri_tv_forward(int nx, int ny, const mri_c64 *image, mri_c64 *grad, mri_stream_t stream);

/* Theta^H, the exact transpose of mri_tv_forward:
 *   image[i][j] = grad[0][i-1][j] - grad[0][i][j] + grad[1][i][j-1] - grad[1][i][j]  (grad[.][-1] = 0)
 * grad [2][nx][ny] -> image [nx][ny]. */
MRI_API int mri_tv_adjoint(int nx, int ny, const mri_c64 *grad, mri_c64 *image, mri_stream_t stream);

/* Soft threshold of Eq. 8-9 applied to complex values (magnitude shrink):
 *   out = in * (1 - t/|in|) where |in| > t, else 0.   n elements; in == out allowed. */
MRI_API int mri_soft_threshold(int n, float t, const mri_c64 *in, mri_c64 *out, mri_stream_t stream);

/* ADMM parameters (Eq. 5-12, Alg. 2 and Alg. 4; the paper's Table I lists one set). */
typedef struct {
    float lambda;     /* regularisation weight of Eq. 3 (>= 0) */
    float beta;       /* augmented-Lagrangian parameter of Eq. 5 (> 0) */
    int admm_iters;   /* maximum outer iterations (>= 0) */
    int cg_iters;     /* maximum CG iterations per x-update (>= 0) */
    double rtol;      /* Alg. 4: stop when ||x'-x||^2/||x'||^2 <= rtol^2 (0: fixed count) */
    double atol;      /* Alg. 2: stop CG when ||r||^2 <= atol^2 (0: fixed count) */
} mri_admm_params;

/*
 * Full reconstruction (Alg. 4): starting from x = 0 and eta = 0, each outer
 * step computes mu = S_{lambda/beta}(Theta x + eta), b = F^H d +
 * (beta/2) Theta^H (mu - eta), solves A x' = b by CG warm-started from x
 * (A = F^H F + (beta/2) Theta^H Theta), then eta += Theta x' - mu.
 * kspace [nc][nk] and coil_maps [nc][nx][ny] are device inputs; image_out
 * [nx][ny] receives the final image.  objective_hist and alpha_hist are
 * nullable DEVICE arrays of admm_iters doubles receiving, after each outer
 * step, the Eq. 3 objective (costs one extra forward operator per step) and
 * the relative change; entries of steps not taken (early stop) are left as
 * they were.  Tolerances are evaluated on the device: the call never
 * synchronises.  CG scalars (alpha, beta, residual norms) are reduced in FP64.
 */
MRI_API int mri_admm_reconstruct(mri_plan *plan, const mri_c64 *kspace, const mri_c64 *coil_maps,
                                 const mri_admm_params *params, mri_c64 *image_out,
                                 double *objective_hist, double *alpha_hist, mri_stream_t stream);

/*
 * Checkpoint and resume (not in the paper): Alg. 4 started from a saved state
 * instead of x^0 = 0, eta^0 = 0.  x0 [nx][ny] and eta0 [2][nx][ny] (device,
 * nullable: zero) are the image and the dual variable to start from; on
 * return image_out holds x and eta_out ([2][nx][ny], nullable) the dual
 * variable, which must not alias x0 or eta0.  The ADMM state is exactly
 * (x, eta) -- mu is recomputed from them at the start of each step -- so with
 * fixed counts (rtol = atol = 0) a reconstruction split into two calls, the
 * second resuming from the first one's (x, eta), computes bit for bit the
 * iterates of one call with the summed admm_iters.  objective_hist and
 * alpha_hist count the steps of this call.
 */
MRI_API int mri_admm_resume(mri_plan *plan, const mri_c64 *kspace, const mri_c64 *coil_maps,
                            const mri_admm_params *params, const mri_c64 *x0, const mri_c64 *eta0,
                            mri_c64 *image_out, mri_c64 *eta_out, double *objective_hist, double *alpha_hist,
                            mri_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched reconstructions (not in the paper, which reconstructs one image
 * at a time): many independent problems of different shapes in one launch.
 * ------------------------------------------------------------------------- */

/* One reconstruction of a batch: its own plan (created for its shape and
 * trajectory; plans may not be shared between requests of a batch), device
 * inputs and output as for mri_admm_reconstruct, and its parameters. */
typedef struct {
    mri_plan *plan;
    const mri_c64 *kspace;     /* [nc][nk] */
    const mri_c64 *coil_maps;  /* [nc][nx][ny] */
    mri_c64 *image_out;        /* [nx][ny] */
    mri_admm_params params;
} mri_request;

typedef struct mri_batch mri_batch;

/* A batch object caches the combined launch of one request list. */
MRI_API int mri_batch_create(mri_batch **batch);
MRI_API int mri_batch_destroy(mri_batch *batch);

/*
 * Reconstruct n independent problems (Alg. 4 each).  Every request's whole
 * reconstruction is captured into a child CUDA graph; the children are
 * independent nodes of one parent graph, launched with one
 * cudaGraphLaunch on `stream`, so their kernels overlap on the GPU.  The
 * parent graph is cached and replayed while the request list (plans,
 * pointers, parameters) repeats.  Each result is identical to the one the
 * request produces alone (same kernels, tiles and summation order).
 * Requests may not use timing-enabled plans.  The first call on a request
 * list captures (host work proportional to the number of launches).
 */
MRI_API int mri_batch_reconstruct(mri_batch *batch, int n, const mri_request *reqs, mri_stream_t stream);

/* Kernels in one replay of the cached batch launch. */
MRI_API long long mri_batch_launch_count(const mri_batch *batch);

/* ---------------------------------------------------------------------------
 * Serving loop (not in the paper): reconstruction requests arriving over
 * time from host memory, admitted under a device-memory budget and run
 * concurrently (continuous batching).
 *
 * A server owns a scheduler thread, `max_inflight` CUDA streams, a device
 * memory pool and a cache of entries: an entry is a plan for one shape and
 * trajectory (its DFT factors) with fixed device buffers for that shape's
 * k-space, coil maps and image, which stay resident between requests.  A
 * request whose trajectory equals an idle entry's (byte for byte) reuses
 * the entry's factors; if its coil maps also equal the entry's, they are
 * not uploaded again.  From the first request that finds an entry holding
 * its trajectory, the entry's reconstruction runs as a CUDA graph captured
 * once over its buffers and then replayed.  The scheduler starts the oldest waiting
 * request (first in, first out) as soon as a stream is free and its device
 * bytes -- a new entry's (mri_plan_estimate_bytes plus the three buffers)
 * and the trajectory upload, or nothing beyond the trajectory upload for a
 * cached entry -- fit under `hbm_budget_bytes` together with everything
 * resident; idle entries are evicted least-recently-used to make room, and
 * when nothing else fits an idle entry of the request's shape is given the
 * new trajectory in place.  A request whose bytes exceed the whole budget
 * fails with MRI_ERR_NOMEM; one whose shape the precision does not support
 * fails with MRI_ERR_NOMEM too (estimate 0).  Every request runs Alg. 4
 * with its own plan and buffers, so its image is bit-identical to the one
 * mri_admm_reconstruct produces for it alone with a plan of the same
 * precision, whatever else is in flight.
 * ------------------------------------------------------------------------- */

typedef struct mri_server mri_server;

/* One request: shape, HOST arrays (copied at submit; the caller may reuse
 * them as soon as mri_server_submit returns) and parameters.
 * traj [nk][2] float in cycles/pixel, kspace [nc][nk], coil_maps [nc][nx][ny]. */
typedef struct {
    int nx, ny, nk, nc;
    const float *traj;
    const mri_c64 *kspace;
    const mri_c64 *coil_maps;
    mri_admm_params params;
} mri_server_request;

/* Start a server on the current device.  precision: MRI_FP32, MRI_TF32
 * or MRI_BF16X3 for all its plans; max_inflight in 1..64. */
MRI_API int mri_server_create(mri_server **server, size_t hbm_budget_bytes, int max_inflight, int precision);

/* Queue a request; *ticket identifies it in poll/wait.  Thread-safe. */
MRI_API int mri_server_submit(mri_server *server, const mri_server_request *request, uint64_t *ticket);

/* *done = 1 once the request has finished (successfully or not). */
MRI_API int mri_server_poll(mri_server *server, uint64_t ticket, int *done);

/* Wait for a request (timeout_s <= 0: no limit; else MRI_ERR_TIMEOUT after
 * timeout_s seconds, and the ticket stays valid), copy its image [nx][ny]
 * to host `image` (nullable) and its submit-to-finish latency in ms to
 * `latency_ms` (nullable), and retire the ticket.  Returns the request's
 * own status: MRI_OK, MRI_ERR_NOMEM (does not fit the budget),
 * MRI_ERR_TIMEOUT (a bounded device-side wait gave up), or the error of
 * plan creation or launch. */
MRI_API int mri_server_wait(mri_server *server, uint64_t ticket, mri_c64 *image, double *latency_ms,
                            double timeout_s);

/* Latency percentiles (ms, nearest-rank) over all requests completed so
 * far, counts of completed and failed requests, and the device bytes held
 * now and at most so far by cached plans and in-flight requests. */
MRI_API int mri_server_stats(mri_server *server, double *p50_ms, double *p99_ms, uint64_t *completed,
                             uint64_t *failed, size_t *resident_bytes, size_t *peak_resident_bytes);

/* Cache counters since creation (each nullable): requests that found an
 * idle entry with their trajectory (factors reused), requests that gave an
 * idle entry of their shape a new trajectory in place, requests whose coil
 * maps were already resident in their entry, and requests run by replaying
 * their entry's captured graph. */
MRI_API int mri_server_cache_stats(mri_server *server, uint64_t *plan_hits, uint64_t *plan_retargets,
                                   uint64_t *maps_reused, uint64_t *graph_replays);

/* Finish in-flight requests, fail the waiting ones, free everything.  No
 * other call on the server may be in progress or follow. */
MRI_API int mri_server_destroy(mri_server *server);

/* ---------------------------------------------------------------------------
 * Allocation-free adjoint (the paper has no counterpart; it is a convenience
 * for callers that cannot allocate device memory -- code running where the
 * CUDA allocator must not be touched, such as a real-time loop, a host
 * callback, or a process whose device memory is reserved up front).
 *
 * Same result as mri_nudft_adjoint with an MRI_FP32 plan, but needs no plan
 * and allocates nothing: the DFT factors are formed on the fly from traj
 * (device, [nk][2] float) and the k-space-split partial images live in a
 * fixed 16 MiB device buffer that the library holds on every GPU that loads
 * it, until the process exits.  kspace [nc][nk], coil_maps [nc][nx][ny] and
 * image [nx][ny] are device arrays owned by the caller.
 *   - nc * nx * ny must not exceed 2097152 (16 MiB of complex64), else
 *     MRI_ERR_INVALID with a message naming the limit.
 *   - all calls on a device share the buffer and it keeps the last call's
 *     contents; calls that overlap on the GPU (unordered streams) race on
 *     it, so serialise them.
 *   - nc must not exceed 65535, else MRI_ERR_INVALID.
 *   - the first call on a device looks up the buffer's address; make it
 *     before any stream capture.  The address is kept for the life of the
 *     process: calls after a cudaDeviceReset of that device are not supported.
 * ------------------------------------------------------------------------- */
MRI_API int mri_nudft_adjoint_noalloc(int nx, int ny, int nk, int nc, const float *traj, const mri_c64 *kspace,
                                      const mri_c64 *coil_maps, mri_c64 *image, mri_stream_t stream);

/* ---------------------------------------------------------------------------
 * Diagnostics (not in the paper): kernel accounting used by benchmarks.
 * ------------------------------------------------------------------------- */

/* Enable (1) or disable (0) CUDA-event timing of the two product kernels of
 * this plan (forward Eq. 1 and adjoint) and of the adjoint's reduction:
 * every launch is bracketed by events on the launching stream. */
MRI_API int mri_plan_set_timing(mri_plan *plan, int enable);

/* Total milliseconds and launch counts of the timed forward and adjoint
 * product kernels and of the adjoint's split-sum/coil-combine kernel since
 * the last read (nullable outputs); waits for the recorded events and then
 * forgets them. */
MRI_API int mri_plan_read_timing(mri_plan *plan, double *fwd_ms, long long *fwd_launches, double *adj_ms,
                                 long long *adj_launches, double *red_ms, long long *red_launches);

/* Number of kernels this plan has enqueued since creation. */
MRI_API long long mri_plan_launch_count(const mri_plan *plan);

/* Self-test of failure detection: enqueue one thread that waits on a
 * device barrier nothing completes, through the same bounded wait the
 * tensor-core kernels use; after limit_ms (0 < limit_ms <= 1000) it gives up
 * and records the timeout in the plan's deferred status, so that the next
 * mri_plan_sync_status returns MRI_ERR_TIMEOUT (and clears it).  The device
 * context stays usable. */
MRI_API int mri_plan_selftest_wait(mri_plan *plan, double limit_ms, mri_stream_t stream);

/* ---------------------------------------------------------------------------
 * Scheduling of the tensor-core products (not in the paper).  The forward
 * and adjoint kernels are persistent (one CTA per SM); their tile
 * configuration is the number of coils per forward N tile (the UMMA N is
 * coils x ny_pad, at most 256) and the number of operand stages of each
 * product's shared-memory ring (2..4, as shared memory and tensor memory
 * allow).  It changes the schedule only, never the arithmetic or its order.
 * Every CTA loads its own operand tiles (no cluster multicast).
 * ------------------------------------------------------------------------- */

/* Current configuration (nullable outputs): coils per forward tile, forward
 * and adjoint operand stages, number of k-space splits of the adjoint (set
 * by the shape and SM count, not tunable: it fixes the summation order). */
MRI_API int mri_plan_get_config(const mri_plan *plan, int *fwd_coils_per_tile, int *fwd_stages, int *adj_stages,
                                int *adj_ksplit);

/* Set the tile configuration (0 keeps the current value): coils per forward
 * tile in 1..min(4, nc, 256 / ny_pad), stage counts in 2..4.  MRI_ERR_INVALID
 * when the shape or the on-chip memory does not allow it; MRI_ERR_UNSUPPORTED
 * on an FP32 plan. */
MRI_API int mri_plan_set_tiles(mri_plan *plan, int fwd_coils_per_tile, int fwd_stages, int adj_stages);

/* mri_admm_reconstruct captures its whole launch sequence into a CUDA graph
 * on first use and replays it while the stream is not the legacy default
 * stream and the arguments (pointers, parameters) are the same; enable = 0
 * launches kernels directly.  On by default.  A plan with timing enabled
 * always launches directly (per-kernel events are not readable from graph
 * replays). */
MRI_API int mri_plan_set_graphs(mri_plan *plan, int enable);

/* Autotuner: time every valid tile configuration of both products on this
 * plan's shape (forward: coils per tile x stages; adjoint: stages;
 * `repeats` launches each, default 3) and keep the fastest.  The
 * choice is also recorded in the process-wide tuning table (below), keyed by
 * precision, shape and SM count.  Synchronises `stream`; allocates a
 * temporary buffer.  No-op for FP32 plans. */
MRI_API int mri_plan_autotune(mri_plan *plan, int repeats, mri_stream_t stream);

/* Persistent tuning table.  Plans created for a (precision, nx, ny, nk, nc,
 * SM count) that the table holds start with its tile configuration.
 *   mri_tuning_save: write the table to `path` as JSON
 *     {"format": "mrirecon-tuning", "version": 1, "entries": [{"precision",
 *      "nx", "ny", "nk", "nc", "sms", "fwd_coils_per_tile", "fwd_stages",
 *      "adj_stages"}, ...]}
 *   mri_tuning_load: merge such a file into the table (MRI_ERR_INVALID, and
 *     no change, for a file that is missing, not a tuning file, or has an
 *     entry without one of those integer keys, with coils per tile outside
 *     1..4 or a stage count outside 2..4)
 *   mri_tuning_clear / mri_tuning_count: empty the table / its entry count.
 * No GPU is needed; the table is guarded for use from several threads. */
MRI_API int mri_tuning_save(const char *path);
MRI_API int mri_tuning_load(const char *path);
MRI_API int mri_tuning_clear(void);
MRI_API int mri_tuning_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MRIRECON_H */
