/*
 * occ_serve.h -- serving loop over the hot path of occ.h (liboccreuse.so).
 *
 * The paper computes one frame at a time (Alg. 1 and Alg. 2); it has no
 * request loop.  This header adds one around the same trace and reuse calls:
 * frames of mixed size, effect (AO / shadow), neighbour pattern, estimator
 * and storage format arrive as requests, are admitted while their device
 * memory fits a budget, and run in batches -- small views together in the
 * persistent batched kernels of occ_frame_batch, large views through the
 * per-view trace and reuse kernels -- with up to `max_inflight` batches on
 * the device at once, each on its own stream.  A request's result does not
 * depend on the requests it is batched with: the kernels a view runs through
 * are chosen from the view alone, and every view has its own buffers.
 *
 * Two layers:
 *   occ_sched_*   the admission scheduler: host-only bookkeeping (no CUDA
 *                 call), FIFO admission under a byte budget, a limit on
 *                 batches in flight, queue limit, admission deadlines.  It is
 *                 exported on its own so that its policy can be driven and
 *                 tested without a GPU;
 *   occ_server_*  the server: a native worker thread that owns the streams,
 *                 a stream-ordered device memory pool and one occ_ctx per
 *                 in-flight slot, uses occ_sched_* for admission, and reports
 *                 per-request timestamps (submit, admission, result ready).
 *
 * Status codes are those of occ.h.  All occ_sched_* and occ_server_* calls
 * are thread-safe except the *_destroy calls, which must not race any other
 * call on the same object.
 */
#ifndef OCC_SERVE_H
#define OCC_SERVE_H

#include <stdint.h>

#include "occ.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- admission scheduler (host only) ------------------------------------ */

typedef struct occ_sched occ_sched;

typedef struct {
    int64_t budget_bytes;         /* device bytes the admitted requests may hold at once, > 0 */
    int32_t max_views_per_batch;  /* 1 .. 256 */
    int32_t max_inflight;         /* batches on the device at once, 1 .. 16 */
    int32_t max_queued;           /* waiting requests, >= 1; a submit beyond it is refused */
} occ_sched_config;

typedef struct {
    int64_t queued, inflight_batches, reserved_bytes, peak_reserved_bytes;
    int64_t submitted, admitted, completed_batches, expired, refused;
} occ_sched_stats;

occ_status occ_sched_create(const occ_sched_config* cfg, occ_sched** out);
occ_status occ_sched_destroy(occ_sched* s);

/* Queues request `id` needing `bytes` of device memory.  deadline_ns > 0 is the
 * absolute time (same clock as now_ns) after which it is dropped if it has not
 * been admitted; 0 = no deadline.  Returns OCC_ERR_INVALID_ARG for bytes <= 0
 * or a repeated id still queued or running, OCC_ERR_OOM if bytes exceeds the
 * budget (it could never be admitted), OCC_ERR_BUSY if the queue is full;
 * nothing is queued then. */
occ_status occ_sched_submit(occ_sched* s, uint64_t id, int64_t bytes, int64_t now_ns,
                            int64_t deadline_ns);

/* One scheduling decision at time now_ns.
 *  1. Queued requests past their deadline are removed and listed in
 *     expired[0 .. *n_expired) (at most exp_cap per call; when more are due,
 *     step 2 is skipped and the caller calls again).
 *  2. If fewer than max_inflight batches run, requests are admitted in
 *     submission order while their bytes fit the budget beside the bytes of
 *     the running batches, up to max_views_per_batch and `cap`; the first
 *     request that does not fit stops admission (no overtaking, so a large
 *     request is not starved).  Admitted ids go to ids[0 .. *n) and *slot
 *     receives the batch slot in [0, max_inflight); with nothing admitted
 *     *n = 0 and *slot = -1. */
occ_status occ_sched_next(occ_sched* s, int64_t now_ns, uint64_t* ids, int32_t cap, int32_t* n,
                          int32_t* slot, uint64_t* expired, int32_t exp_cap, int32_t* n_expired);

/* The batch in `slot` finished: its bytes and slot are free again.
 * OCC_ERR_INVALID_ARG if the slot is not running a batch. */
occ_status occ_sched_complete(occ_sched* s, int32_t slot);

/* Removes every queued request (not the running ones) into ids[0 .. *n), at
 * most cap; call again while *n == cap. */
occ_status occ_sched_drain(occ_sched* s, uint64_t* ids, int32_t cap, int32_t* n);

occ_status occ_sched_get_stats(const occ_sched* s, occ_sched_stats* out);

/* ---- server --------------------------------------------------------------- */

typedef struct occ_server occ_server;

typedef struct {
    int64_t budget_bytes;         /* 0: 80% of the device memory free at creation */
    int32_t max_views_per_batch;  /* 0: 64 (<= 256) */
    int32_t max_inflight;         /* 0: 2 (<= 16); one stream and context each */
    int32_t max_queued;           /* 0: 4096 */
    int32_t poll_us;              /* 0: the worker spins (yielding) while batches run;
                                     > 0: it sleeps this long between polls */
    int64_t batch_max_px;         /* views of at most this many pixels (and K <= 16) share
                                     the batched kernels; larger ones run the per-view
                                     kernels.  0: 1,048,576 */
    int64_t batch_window_us;      /* 0: a free slot takes whatever is queued at once; > 0: it
                                     waits until max_views_per_batch requests are queued or
                                     the oldest has waited this long */
    int32_t inject_alloc_failures; /* host-side fault injection: the first N batches find the
                                      device memory pool exhausted; their requests finish with
                                      OCC_ERR_OOM and the server goes on (0 in production) */
    int32_t reserved;
} occ_server_config;

/* One frame to serve.  The G-buffer comes either from a pinhole camera
 * rendered on the device (pos4_host == NULL; camera = eye[3], target[3],
 * up[3], vfov_deg; eps as in occ_gbuffer_pinhole) or from host memory
 * (pos4_host and nrm4_host: FP32 float4 planes; with packed = 1 pos4_host is
 * the packed plane and nrm4_host is NULL), copied at run time: host buffers
 * must stay valid until the request's result is polled.  The estimate goes to
 * exactly one of out_host (float[H][W], pinned memory recommended) or
 * out_device (device float[H][W] on the server's device).  Pattern offsets
 * are copied at submit.  deadline_ns > 0: dropped with OCC_ERR_TIMEOUT if not
 * admitted within this many nanoseconds of the submit. */
typedef struct {
    int32_t W, H;
    int32_t effect;
    float radius;
    occ_rect_light light;
    uint64_t seed;
    uint32_t sample;
    occ_pattern pattern;
    int32_t K, estimator;
    int32_t packed;               /* 0: FP32 G-buffer and records; 1: packed formats */
    float camera[10];
    float eps;
    const float* pos4_host;
    const float* nrm4_host;
    float* out_host;
    float* out_device;
    int64_t deadline_ns;
} occ_request;

typedef struct {
    uint64_t id;
    int32_t status;               /* OCC_OK; OCC_ERR_TIMEOUT (deadline passed in the queue);
                                     OCC_ERR_CANCELLED (still queued at a cancelling shutdown);
                                     otherwise the
                                     error of the batch's launch or OCC_ERR_DEVICE_CHECK */
    int32_t batch_views;          /* views in the batch it ran in (0 if it never ran) */
    int64_t t_submit_ns, t_admit_ns, t_done_ns;  /* monotonic clock, ns since creation */
} occ_result;

typedef struct {
    occ_sched_stats sched;
    int64_t budget_bytes;
    int64_t batches, views_batched, views_single;
    int64_t pool_reserved_bytes;  /* device memory the pool holds */
} occ_server_stats;

/* Starts a server on ctx's device for scene `bvh` (which must outlive it); the
 * server copies ctx's tuning (occ_set_tuning).  Returns OCC_ERR_OOM if the
 * budget exceeds the free device memory. */
occ_status occ_server_create(occ_ctx* ctx, const occ_bvh* bvh, const occ_server_config* cfg,
                             occ_server** out);

/* Validates and queues a request; *id receives its id (> 0).  Argument
 * errors, OCC_ERR_OOM (larger than the budget) and OCC_ERR_BUSY (queue full)
 * queue nothing; err_msg (err_len bytes, may be NULL) receives the reason. */
occ_status occ_server_submit(occ_server* srv, const occ_request* req, uint64_t* id,
                             char* err_msg, int32_t err_len);

/* Moves up to cap finished results into out[0 .. *n), oldest first, waiting
 * up to timeout_us (0: do not wait; < 0: wait until one is there) for the
 * first.  A result is ready when its estimate is in out_host / out_device. */
occ_status occ_server_poll(occ_server* srv, occ_result* out, int32_t cap, int64_t timeout_us,
                           int32_t* n);

occ_status occ_server_get_stats(occ_server* srv, occ_server_stats* out);

/* Stops accepting requests and returns when the worker has finished: with
 * cancel_queued = 0 every queued request still runs; otherwise queued
 * requests finish as OCC_ERR_CANCELLED.  Running batches always complete.
 * Results stay available to occ_server_poll.  A second call does nothing. */
occ_status occ_server_shutdown(occ_server* srv, int32_t cancel_queued);

/* occ_server_shutdown(srv, cancel_queued) if not done yet, then releases the
 * device memory pool, streams and contexts; unpolled results are discarded. */
occ_status occ_server_destroy(occ_server* srv, int32_t cancel_queued);

#ifdef __cplusplus
}
#endif

#endif /* OCC_SERVE_H */
