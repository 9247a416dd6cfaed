/*
 * occ.h -- C ABI of the GB300 occlusion-point reuse library (liboccreuse.so).
 *
 * The library computes the data-parallel hot path of "Occlusion-Point Reuse
 * for Ray-Traced Ambient Occlusion and Shadow" on one GPU:
 *
 *   1. trace  (Alg. 1 and Alg. 2, step 1): one cosine-weighted AO ray (Eq. 2)
 *      or one uniform area-light shadow ray (Eq. 5) per receiver, traced to
 *      its closest hit; the hit point and its normal, turned toward the
 *      receiver, form the receiver's occluder record;
 *   2. reuse  (Alg. 1 and Alg. 2, steps 2-3): every receiver combines the
 *      occluder records of its neighbour set N_i (Eq. 8) with balance-
 *      heuristic MIS weights (Eqs. 10-12), giving the unbiased estimators of
 *      Eq. 17 (AO) and Eq. 23 (shadow) with first-hit validation (Eq. 7), or
 *      the biased estimators of Eq. 18 and Eq. 24 without it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named *_host are host memory; every other buffer pointer is
 *    device memory on the context's device.  The caller owns all G-buffer,
 *    occluder and output buffers; the library owns BVHs and its workspace.
 *  - Device buffers holding float4 data must be 16-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Compute calls are asynchronous on that stream.
 *  - Argument errors are detected before anything is launched and return
 *    OCC_ERR_INVALID_ARG (or OCC_ERR_UNSUPPORTED); the message is available
 *    from occ_last_error().  A launch failure returns OCC_ERR_CUDA.  Faults a
 *    kernel detects itself (a traversal stack overflow, a bounded wait that
 *    ran out) are recorded in a device status word and returned as
 *    OCC_ERR_DEVICE_CHECK by the next occ_sync().  No entry point aborts,
 *    traps or throws across the ABI.
 *  - A context may be used by one host thread at a time.  Its AO trace calls share one
 *    device work counter and its unbiased group reuse calls one validation workspace, so
 *    they must not overlap on the device: use one context per stream that traces or
 *    reuses concurrently.
 *
 * Images are row-major, pixel (x, y) at linear index y * W + x.
 */
#ifndef OCC_H
#define OCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OCC_OK = 0,
    OCC_ERR_INVALID_ARG = 1,
    OCC_ERR_CUDA = 2,
    OCC_ERR_OOM = 3,
    OCC_ERR_TIMEOUT = 4,
    OCC_ERR_UNSUPPORTED = 5,
    OCC_ERR_DEVICE_CHECK = 6,
    OCC_ERR_BUSY = 7,        /* a serving queue is full (include/occ_serve.h) */
    OCC_ERR_CANCELLED = 8    /* a queued request dropped when its server shut down */
} occ_status;

enum { OCC_EFFECT_AO = 0, OCC_EFFECT_SHADOW = 1 };

/* Estimators (Sec. 4.3-4.4): NOREUSE is Eq. 3 / Eq. 6 with one sample; BIASED
 * is Eq. 18 / Eq. 24 (shadow adds the all-blocked guard); UNBIASED is Eq. 17 /
 * Eq. 23 with first-hit validation rays; BOXMEAN averages the binary
 * visibility of N_i (final-value filtering / light-sample averaging, the biased
 * baselines Filter(N) and Light(N) of Sec. 6).  LIGHT_UNBIASED (shadows only) is
 * the unbiased light-sample reuse baseline Light(N U) of Sec. 6.2: receiver i
 * traces a segment to every member's light sample (drawn from the member's own
 * random numbers of the records' seed and sample) and averages the visibility;
 * the uniform area sampler gives every sample the same balance-heuristic weight. */
enum { OCC_EST_NOREUSE = 0, OCC_EST_BIASED = 1, OCC_EST_UNBIASED = 2, OCC_EST_BOXMEAN = 3,
       OCC_EST_LIGHT_UNBIASED = 4 };

/* Neighbour patterns N_i (Eq. 8, Sec. 5 "Reuse Implementation", App. I):
 *  GROUP:   the screen is partitioned into gw x gh blocks; N_i is i's block.
 *  BOX:     the gw x gh window centred on i (dx in [-(gw-1)/2, gw/2]).
 *  OFFSETS: i plus i + (dx, dy) for each of n_offsets shared offsets.
 *  RANDOM:  i plus n_offsets offsets drawn for each receiver and sample (the per-receiver
 *           form of Eq. 8): slot s (1 .. n_offsets) of receiver pixel p takes the first
 *           attempt a (0 .. 31) of Philox4x32-10 with counter (p, sample, 2, 32 s + a), key
 *           (seed low 32 bits, seed high 32 bits), whose words w0, w1 give
 *           dx = floor(w0 (2R + 1) / 2^32) - R, dy = floor(w1 (2R + 1) / 2^32) - R with
 *           dx^2 + dy^2 <= R^2, (dx, dy) != (0, 0) and not drawn by an earlier slot of p
 *           (R = radius_px; `sample` is the occluder records' sample); a slot without such
 *           an attempt stays empty.
 * Members outside the image or with an invalid G-buffer entry are dropped. */
enum { OCC_PAT_GROUP = 0, OCC_PAT_BOX = 1, OCC_PAT_OFFSETS = 2, OCC_PAT_RANDOM = 3 };

/* Storage formats.  FP32: as described at occ_gbuffer / occ_occluders.  PACKED (16 bytes
 * per pixel each, FP32 arithmetic on the unpacked values):
 *  - G-buffer: one float4 plane (x.xyz, normal as octahedral 2 x 16-bit snorm code in the
 *    w bits; code 0x80008000 marks an invalid pixel);
 *  - records: one 16-byte plane: words 0-1 (a 64-bit little-endian word) hold
 *    d = z - x_source as three 19-bit two's-complement mantissas m (bits 0-18, 19-37,
 *    38-56) with a shared exponent E (bits 57-62), d = m * 2^(E - 60), and bit 63 =
 *    occluder present; word 2 the octahedral n_z code; word 3 the triangle id or -1.
 *    The writer takes E = floor(log2 max|d_i|) + 43 (clamped to 0..63) and rounds
 *    d_i * 2^(60 - E) to nearest (even), clamped to +-(2^18 - 1); the reader rebuilds each
 *    coordinate as fmaf(m, 2^(E - 60), x_source) in FP32 (one rounding), x_source being
 *    the source receiver's G-buffer point.
 * Octahedral normals: Cigolle et al., "A Survey of Efficient Representations for
 * Independent Unit Vectors", JCGT 2014. */
enum { OCC_GB_FP32 = 0, OCC_GB_PACKED = 1 };
enum { OCC_REC_FP32 = 0, OCC_REC_PACKED = 1 };

typedef struct occ_ctx occ_ctx;   /* opaque: device, status word, workspace */
typedef struct occ_bvh occ_bvh;   /* opaque: device-resident wide BVH */

/* G-buffer of receivers.  pos4[q] = (x.xyz, valid): x is the receiver point
 * (the visible surface point already offset along its normal), valid is 1
 * for a receiver and 0 for background.  nrm4[q] = (n.xyz, unused): the unit
 * geometric normal facing the viewer.  Two layouts of the float4 planes:
 *   OCC_LAYOUT_LINEAR (0): row-major, pixel (x, y) at q = y * pitch_px + x, pitch_px >= W
 *     (0 means W), so a G-buffer may be a window of a wider render target;
 *   OCC_LAYOUT_TILED (1): 8 x 8-pixel tiles, tiles_x = ceil(W / 8) per tile row; tile
 *     (x / 8, y / 8) holds the 64 entries from ((y / 8) * tiles_x + x / 8) * 64 on, the
 *     pixel (u, v) = (x mod 8, y mod 8) at its Morton index u0 | v0 << 1 | u1 << 2 |
 *     v1 << 3 | u2 << 4 | v2 << 5 (u_i, v_i the bits of u, v).  Each plane holds
 *     ceil(W / 8) * ceil(H / 8) * 64 entries; entries of tile pixels outside the image are
 *     never read.  pitch_px must be 0.  occ_tile_gbuffer writes this layout.
 * Records and outputs stay dense row-major (W per row) whatever the G-buffer layout. */
enum { OCC_LAYOUT_LINEAR = 0, OCC_LAYOUT_TILED = 1 };
typedef struct {
    int32_t W, H;
    const float* pos4;         /* FP32: pos4 plane; PACKED: the packed plane */
    const float* nrm4;         /* FP32: nrm4 plane; PACKED: unused (NULL) */
    int32_t format;            /* OCC_GB_FP32 (0) or OCC_GB_PACKED */
    int32_t layout;            /* OCC_LAYOUT_LINEAR (0) or OCC_LAYOUT_TILED */
    int64_t pitch_px;          /* LINEAR: row pitch of the planes in pixels (0: W); TILED: 0 */
} occ_gbuffer;

/* Rectangle light c + a eu + b ev, a, b in [-1/2, 1/2], eu orthogonal to ev.
 * It emits along n_L = normalize(eu x ev); every receiver and occluder must lie
 * on that side of its plane (Eqs. 4-5, 19-21). */
typedef struct { float c[3], eu[3], ev[3]; } occ_rect_light;

/* Occluder records (Alg. 1/2 step 1: "store hit position and oriented hit
 * normal").  `data` is caller-owned device memory.  FP32: 32 * W * H bytes holding
 * two float4 planes: plane 0 [p] = (z.xyz, triangle id as int bits, -1 = no
 * occluder), plane 1 [W*H + p] = (n_z.xyz facing the source receiver, t).
 * PACKED: 16 * W * H bytes (see the formats above).  The trace calls write the
 * format given in `format` and fill the remaining fields; the reuse calls read them. */
typedef struct {
    int32_t W, H;
    int32_t format;            /* OCC_REC_FP32 or OCC_REC_PACKED */
    void* data;
    int32_t effect;            /* written by trace */
    float radius;              /* AO radius R (AO) */
    occ_rect_light light;      /* light (shadow) */
    uint64_t seed;
    uint32_t sample;
} occ_occluders;

typedef struct {
    int32_t kind;              /* OCC_PAT_* */
    int32_t gw, gh;            /* GROUP / BOX extent */
    int32_t n_offsets;         /* OFFSETS / RANDOM: number of offsets, K - 1 */
    const int32_t* offsets_host;   /* OFFSETS: 2 * n_offsets ints, copied at call time */
    int32_t radius_px;         /* RANDOM: disk radius R in pixels, 1 .. 64 */
    uint64_t seed;             /* RANDOM: key of the offset draws */
} occ_pattern;

typedef struct {
    int64_t num_tris, num_nodes, num_leaves;
    int32_t depth, max_leaf_tris;
    int64_t bytes;             /* device bytes of nodes + triangles */
    double build_seconds;
} occ_bvh_stats;

/* ---- context ------------------------------------------------------------- */

/* Creates a context on CUDA device `device` (made current on the calling
 * thread).  OCC_ERR_UNSUPPORTED if the device is not sm_103. */
occ_status occ_create(int device, occ_ctx** out);
occ_status occ_destroy(occ_ctx* ctx);
/* Message of the last non-OK status of this context ("" if none). */
const char* occ_last_error(const occ_ctx* ctx);
/* Waits for `stream`, then reports launch errors and device-side check flags
 * (and clears the flags). */
occ_status occ_sync(occ_ctx* ctx, void* stream);
const char* occ_version(void);

/* ---- scene ---------------------------------------------------------------- */

/* Builds a 4-wide BVH (binned SAH, collapsed from a binary tree) over
 * tris_host: T triangles of 3 float xyz vertices (row-major [T][3][3]); the
 * array is copied.  Triangle ids are the input order.  Synchronous. */
occ_status occ_bvh_build(occ_ctx* ctx, const float* tris_host, int64_t T, occ_bvh** out);
occ_status occ_bvh_free(occ_ctx* ctx, occ_bvh* bvh);
occ_status occ_bvh_info(const occ_bvh* bvh, occ_bvh_stats* out);

/* Input stage (not part of the paper's method, which takes a raster
 * G-buffer): pinhole primary rays.  cam_host = eye[3], target[3], up[3],
 * vfov_deg.  Writes pos4/nrm4 (W*H float4 each); pos4 is the hit point moved
 * `eps` along the geometric normal turned toward the camera.  With nrm4 NULL
 * it writes the PACKED G-buffer (one float4 plane, as occ_pack_gbuffer makes)
 * into pos4. */
occ_status occ_gbuffer_pinhole(occ_ctx* ctx, const occ_bvh* bvh, const float* cam_host,
                               float eps, int32_t W, int32_t H, float* pos4, float* nrm4,
                               void* stream);

/* Packs an FP32 G-buffer (either layout) into the PACKED format (16 bytes per pixel):
 * receiver point kept in FP32, normal octahedral-encoded; invalid pixels get the invalid
 * code.  packed_out: W*H float4, row-major (OCC_LAYOUT_LINEAR, pitch W), device, 16-byte
 * aligned. */
occ_status occ_pack_gbuffer(occ_ctx* ctx, const occ_gbuffer* gb, float* packed_out, void* stream);

/* Copies a G-buffer (either format, either layout) into OCC_LAYOUT_TILED (see
 * occ_gbuffer), same format: pos_out (and nrm_out for FP32; NULL for PACKED) hold
 * ceil(W/8) * ceil(H/8) * 64 float4 each, device, 16-byte aligned, owned by the caller;
 * they must not overlap the input.  The G-buffer to pass on is {W, H, pos_out, nrm_out,
 * format, OCC_LAYOUT_TILED, 0}.  Asynchronous on `stream`.  Every kernel takes either
 * layout; the TMA window kernel needs row-major planes, so window patterns on a tiled
 * G-buffer run the per-receiver kernel (the same estimates as reuse_window_path 2). */
occ_status occ_tile_gbuffer(occ_ctx* ctx, const occ_gbuffer* gb, float* pos_out, float* nrm_out,
                            void* stream);

/* ---- hot path ------------------------------------------------------------- */

/* Alg. 1 step 1 (Eq. 2): per receiver, the cosine-weighted direction from
 * Philox4x32-10(counter = (pixel, sample, 0, 0), key = seed) and its closest
 * hit on (0, radius].  out->W/H/data must be set; the call fills the rest. */
occ_status occ_trace_ao(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh, float radius,
                        uint64_t seed, uint32_t sample, occ_occluders* out, void* stream);

/* Alg. 2 step 1 (Eq. 5): per receiver, y uniform on the light (counter =
 * (pixel, sample, 1, 0)) and the closest hit on the segment toward y. */
occ_status occ_trace_shadow(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                            const occ_rect_light* light, uint64_t seed, uint32_t sample,
                            occ_occluders* out, void* stream);

/* Alg. 1 steps 2-3: AO estimate per receiver into out (device float[H][W]).
 * K must equal the pattern's size (gw*gh, or n_offsets + 1), 1 <= K <= 64.
 * bvh_or_null is required for OCC_EST_UNBIASED (and, for shadows,
 * OCC_EST_LIGHT_UNBIASED) and must be NULL otherwise.  Invalid receivers get 1.
 * Estimates are not clamped.  The batched and served paths take estimators 0-3.
 * UNBIASED over GROUP patterns of up to 16 members queues its first-hit validation rays
 * (Eq. 7) in a context workspace of 4 K bytes per pixel, allocated on first use and
 * grown with the image (the estimate is the same as tracing them inline). */
occ_status occ_reuse_ao(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* occ,
                        const occ_pattern* pattern, int32_t K, int32_t estimator,
                        const occ_bvh* bvh_or_null, float* out, void* stream);

/* Alg. 2 steps 2-3: shadow visibility per receiver (Eq. 23 / Eq. 24 with the
 * all-blocked guard of Sec. 4.4).  Same arguments as occ_reuse_ao; the light
 * comes from the occluder records. */
occ_status occ_reuse_shadow(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* occ,
                            const occ_pattern* pattern, int32_t K, int32_t estimator,
                            const occ_bvh* bvh_or_null, float* out, void* stream);

/* Alg. 1 steps 1-3 in one kernel for a shared-group pattern (Sec. 5, "Reuse
 * Implementation": a group's rays run in neighbouring lanes of a warp and exchange their
 * occluders there).  The estimate equals occ_trace_ao followed by occ_reuse_ao with FP32
 * records, without storing the records in device memory.  pattern: OCC_PAT_GROUP with
 * gw x gh = 2x1, 2x2, 4x2 or 4x4 (K = gw * gh), anything else OCC_ERR_UNSUPPORTED;
 * estimator NOREUSE, BIASED, UNBIASED or BOXMEAN (UNBIASED traces its validation rays
 * in the same kernel).  occ_or_null: NULL, or a record buffer (W/H/format/data set as for
 * occ_trace_ao) that also receives the step-1 records, header filled; the estimate
 * uses the FP32 occluders either way.  out: device float[H][W].  Uses the context's work
 * counter like occ_trace_ao. */
occ_status occ_trace_reuse_ao(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                              float radius, uint64_t seed, uint32_t sample,
                              const occ_pattern* pattern, int32_t K, int32_t estimator,
                              occ_occluders* occ_or_null, float* out, void* stream);

/* Alg. 2 steps 1-3 in one kernel (shadow counterpart of occ_trace_reuse_ao; BIASED keeps
 * the all-blocked guard of Sec. 4.4). */
occ_status occ_trace_reuse_shadow(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                                  const occ_rect_light* light, uint64_t seed, uint32_t sample,
                                  const occ_pattern* pattern, int32_t K, int32_t estimator,
                                  occ_occluders* occ_or_null, float* out, void* stream);

/* Several rectangular lights (Sec. 6.2, "Multiple Lights"): out = sum over l of
 * weights_host[l] * V_l, where V_l is light l's shadow visibility from its own step-1
 * trace (key seed + l, sample `sample`) into recs[l] and its own reuse with `estimator`
 * over `pattern` into vis + l * W * H.  recs: n_lights caller-owned occluder buffers
 * (W/H/format/data set, either format); vis: device float[n_lights][H][W]; out: device
 * float[H][W]; 1 <= n_lights <= 16.  The per-light visibilities stay in vis. */
occ_status occ_shadow_lights(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                             const occ_rect_light* lights_host, const float* weights_host,
                             int32_t n_lights, uint64_t seed, uint32_t sample,
                             const occ_pattern* pattern, int32_t K, int32_t estimator,
                             occ_occluders* recs, float* vis, float* out, void* stream);

/* One whole frame from host memory: copies pos4_host/nrm4_host (pinned host
 * memory recommended) to library-owned device buffers, traces (effect AO with
 * `radius`, or SHADOW with `light`), reuses, and copies the estimate to
 * out_host (float[H][W]), all on `stream`; returns after the stream finished. */
occ_status occ_frame_host(occ_ctx* ctx, const occ_bvh* bvh, int32_t effect,
                          const float* pos4_host, const float* nrm4_host, int32_t W, int32_t H,
                          float radius, const occ_rect_light* light, uint64_t seed,
                          uint32_t sample, const occ_pattern* pattern, int32_t K,
                          int32_t estimator, float* out_host, void* stream);

/* occ_frame_host without the final wait: enqueues the same copies and launches on
 * `stream` and returns.  out_host holds the estimate once `stream` has completed;
 * occ_sync(ctx, stream) waits for it and reports device checks.  The context's frame
 * workspace stays in use until then, so one context carries one such frame at a time: to
 * overlap consecutive frames (the copies of one with the kernels of the other), give each
 * frame in flight its own context and stream.  The host buffers must stay valid (pinned,
 * for the copies to run asynchronously) until the stream completes. */
occ_status occ_frame_host_async(occ_ctx* ctx, const occ_bvh* bvh, int32_t effect,
                                const float* pos4_host, const float* nrm4_host, int32_t W,
                                int32_t H, float radius, const occ_rect_light* light,
                                uint64_t seed, uint32_t sample, const occ_pattern* pattern,
                                int32_t K, int32_t estimator, float* out_host, void* stream);

/* ---- batched frames, captured batches and tuning ----------------------------- */

/* One view of a batched frame.  gb and rec describe caller-owned buffers (either
 * format; rec.W/H/format/data set by the caller, the rest of rec is written as by the
 * trace calls); effect with radius (AO) or light (shadow); Philox seed and sample;
 * neighbour pattern with K <= 16 and estimator (the unbiased one uses the batch's
 * BVH); out: device float[H][W]. */
typedef struct {
    occ_gbuffer gb;
    occ_occluders rec;
    int32_t effect;
    float radius;
    occ_rect_light light;
    uint64_t seed;
    uint32_t sample;
    occ_pattern pattern;
    int32_t K, estimator;
    float* out;
} occ_view;

/* Trace and reuse of n_views (<= 256) views of any sizes, effects, patterns and
 * estimators as one persistent trace launch and one persistent reuse launch over the
 * views' concatenated 16x8 tiles (uneven views share the GPU without a launch each).
 * Results equal the per-view calls'. */
occ_status occ_frame_batch(occ_ctx* ctx, const occ_bvh* bvh, occ_view* views, int32_t n_views,
                           void* stream);

/* A batched frame captured as a CUDA graph: the views' buffers, sizes, patterns and
 * parameters are fixed at capture; each launch replays it with new per-view seeds and
 * samples (uploaded before the replay on the launch stream). */
typedef struct occ_batch occ_batch;
occ_status occ_batch_capture(occ_ctx* ctx, const occ_bvh* bvh, occ_view* views, int32_t n_views,
                             occ_batch** out);
occ_status occ_batch_launch(occ_ctx* ctx, occ_batch* batch, const uint64_t* seeds_host,
                            const uint32_t* samples_host, void* stream);
occ_status occ_batch_free(occ_ctx* ctx, occ_batch* batch);

/* Launch choices an autotuner may change (0 = built-in default everywhere). */
typedef struct {
    int32_t reuse_tile_rows;     /* TMA window kernel: receiver rows per tile (4, 8, 16) */
    int32_t reuse_window_path;   /* window patterns: 1 TMA tile kernel (one thread per receiver),
                                    2 per-receiver kernel, 3 TMA tile kernel with two threads
                                    per receiver; 0: TMA tile kernel, two threads per receiver
                                    for AO windows of more than 9 members */
    int32_t batch_ctas_per_sm;   /* persistent batched kernels: CTAs per SM (1 .. 16) */
    int32_t fused_ao_path;       /* occ_trace_reuse_ao: 1 one CTA per 16 x 8 tile, 2 persistent
                                    CTAs refilling whole groups from the context's counter */
    int32_t group_prefetch;      /* GROUP reuse kernel: 1 no prefetch, 2 each CTA prefetches into
                                    L2 the G-buffer and record plane 0 of the CTA one wave of
                                    resident CTAs later, 3 also its hit-normal plane */
    int32_t trace_path;          /* step-1 trace: 1 one CTA per 16 x 8 tile, 2 persistent CTAs
                                    taking rays from the context's counter; 0: persistent for AO,
                                    per tile for shadows */
    int32_t trace_ctas_per_sm;   /* persistent trace: CTAs per SM (1 .. 16; 0 all that fit) */
    int32_t trace_refill;        /* persistent trace: a warp takes new rays once this many of its
                                    lanes are idle (1 .. 32; 0: 16) */
    int32_t trace_order;         /* persistent trace: order in which rays are handed out by 16 x 8
                                    tile: 1 tiles row-major, 2 blocks of 8 x 8 tiles row-major with
                                    the tiles of a block in Morton order (0: row-major) */
} occ_tuning;
occ_status occ_set_tuning(occ_ctx* ctx, const occ_tuning* t);
occ_status occ_get_tuning(const occ_ctx* ctx, occ_tuning* t);

/* ---- allocation-free frame -------------------------------------------------- */

/* The paper has no counterpart to this call; it serves callers that cannot allocate
 * device memory: plugins whose host application owns every device allocation, and
 * real-time frame loops that cannot afford the device-wide synchronisation that
 * cudaMalloc / cudaFree may cause.  Such callers cannot create an occ_ctx (which
 * allocates its status word) nor provide a record workspace.
 *
 * One frame on the current device: the step-1 trace of `effect` (AO with `radius`,
 * or SHADOW with `light`) for every receiver of gb, then the reuse of `estimator`
 * over `pattern` into out (device float[H][W]).  The caller passes the G-buffer
 * (either format), the BVH and `out`; the occluder records, the device status word
 * and the trace's work counter live in a static device array inside the library
 * (calls no cudaMalloc, cudaFree or other allocating routine).  Limits and behaviour:
 *  - estimator NOREUSE, BIASED, UNBIASED (validation rays traced inline) or BOXMEAN;
 *    LIGHT_UNBIASED returns OCC_ERR_INVALID_ARG;
 *  - the records are always FP32 (32 bytes per pixel), whatever the G-buffer format;
 *  - frames of at most 1,048,576 pixels (e.g. 1280x720, 1024x1024); larger ones
 *    return OCC_ERR_INVALID_ARG with a message and launch nothing;
 *  - the array (32 MiB) is held by every GPU that loads the library until exit;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the life of the
 *    process: make that first call before any stream capture, and do not call this
 *    entry point again on a device after cudaDeviceReset (the kept address is stale);
 *  - every call shares the array and overwrites the previous call's records; calls
 *    that overlap on the GPU (other streams or host threads) race on it;
 *  - the status word is cleared at the start of each call; if flags_host is not
 *    NULL the call waits for `stream`, stores the flags there and returns
 *    OCC_ERR_DEVICE_CHECK when any is set; with NULL the call stays asynchronous;
 *  - err_msg (err_len bytes, may be NULL) receives the message of a failure. */
occ_status occ_frame_noalloc(const occ_gbuffer* gb, const occ_bvh* bvh, int32_t effect,
                             float radius, const occ_rect_light* light, uint64_t seed,
                             uint32_t sample, const occ_pattern* pattern, int32_t K,
                             int32_t estimator, float* out, uint32_t* flags_host, char* err_msg,
                             int32_t err_len, void* stream);

/* ---- test and debugging aids ---------------------------------------------- */

/* Philox4x32-10 of n (counter[4], key[2]) items: in_dev holds 6 uint32 per
 * item, out_dev receives 4 uint32 per item. */
occ_status occ_debug_philox(occ_ctx* ctx, const uint32_t* in_dev, int64_t n, uint32_t* out_dev,
                            void* stream);

/* Exercises the bounded-wait failure path of the TMA reuse kernel without a fault: one
 * thread polls an mbarrier that nothing completes, gives up after `spins` polls
 * (1 .. 2^24) and sets the wait-timeout flag, so that the next occ_sync() returns
 * OCC_ERR_DEVICE_CHECK ("wait timeout") and clears it; the context stays usable. */
occ_status occ_debug_wait_timeout(occ_ctx* ctx, uint32_t spins, void* stream);

/* Measurement aid (not part of the method): a throughput probe of the FP32 pipe, the peak
 * that FP32-bound kernels (the window reuse with its K^2 pair densities) are rated against.
 * `blocks` CTAs of 256 threads each run 16 independent chains of `iters` (1 .. 2^24) fused
 * multiply-adds: paired = 0 scalar fma.rn.f32, paired = 1 fma.rn.f32x2 (two FMAs per
 * instruction).  sink_dev (device float[blocks * 256], caller-owned) receives one value per
 * thread so that nothing is optimised away; *flop_host receives the launch's FLOP count
 * (2 per FMA).  Asynchronous on `stream`: time it with events there. */
occ_status occ_debug_fp32_peak(occ_ctx* ctx, int32_t paired, int32_t iters, int32_t blocks,
                               float* sink_dev, double* flop_host, void* stream);

/* Measurement aid (not part of the method): the streaming ceiling of the GROUP reuse
 * kernel's memory pattern at 4 x 2 groups.  Reads what that kernel reads from gb and occ
 * (FP32 formats only: G-buffer position and normal and record plane 0 of every pixel,
 * record plane 1 of the pixels whose ray hit) with the same CTA shape, and writes one float
 * per pixel into out (device float[H][W]) that is a checksum, not an estimate.
 * Asynchronous on `stream`. */
occ_status occ_debug_stream_ceiling(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* occ,
                                    float* out, void* stream);

/* Measurement aid for the instrumented library only (built with OCC_COUNTERS=1; the product
 * library returns OCC_ERR_UNSUPPORTED): what the traversal of every launch since the last
 * reset did on `bvh` (Alg. 1/2 step 1 and the Eq. 7 validation rays).  out_host[5] =
 * {node visits, triangle tests, distinct nodes touched, distinct triangles touched, bytes of
 * those distinct nodes and triangles}.  Waits for the device; reset = 1 then zeroes the
 * counters. */
occ_status occ_debug_bvh_counters(occ_ctx* ctx, const occ_bvh* bvh, int32_t reset,
                                  uint64_t* out_host);

/* The builder alone, on the host (no context, no device): builds the BVH of tris_host
 * ([T][3][3] floats) as occ_bvh_build does and copies the tree out.  nodes_out receives
 * n_nodes nodes of 32 floats (128 bytes: planes lo_x, hi_x, lo_y, hi_y, lo_z, hi_z of the
 * four children as 6 x 4 floats, then the four child references as uint32 bits, then 4
 * floats of padding); tris_out receives T triangles of 12 floats (v0.xyz, input id bits,
 * v1.xyz, 0, v2.xyz, 0) in leaf order.  A child reference is an internal node index, the
 * empty marker 0x7FFFFFFF, or a leaf: bit 31 set, bits 26..30 = count - 1, bits 0..25 = the
 * first triangle.  With nodes_out NULL only n_nodes and depth are written; otherwise
 * nodes_cap (nodes) and tris_cap (triangles) must hold the tree.  OCC_ERR_INVALID_ARG on
 * invalid input, a tree too deep for the traversal stack, or capacities too small.
 * The builder test (tests/test_bvh_host.py) checks the tree on the CPU. */
occ_status occ_debug_bvh_host(const float* tris_host, int64_t T, float* nodes_out,
                              int64_t nodes_cap, float* tris_out, int64_t tris_cap,
                              int64_t* n_nodes, int32_t* depth);

/* The traversal on arbitrary rays: rays_dev holds 8 floats per ray (o.xyz, tmax,
 * d.xyz, unused), t in units of |d| on (0, tmax].  any = 0: tri_dev[i] = the closest
 * hit's input triangle id (-1 none) and t_dev[i] its t (-1 none); any = 1: tri_dev[i] = 1
 * if some triangle is hit, else 0. */
occ_status occ_debug_closest_hit(occ_ctx* ctx, const occ_bvh* bvh, const float* rays_dev,
                                 int64_t n, int32_t any, int32_t* tri_dev, float* t_dev,
                                 void* stream);

/* The step-1 ray of every receiver: out_dev[p] = (direction.xyz, tmax). */
occ_status occ_debug_rays(occ_ctx* ctx, const occ_gbuffer* gb, int32_t effect, float radius,
                          const occ_rect_light* light, uint64_t seed, uint32_t sample,
                          float* out_dev, void* stream);

/* Balance-heuristic weights seen by n receivers pix_host[i] (linear index):
 * w_host[i*64*64 + a*64 + b] = p(z_a | x_b) / sum_e p(z_a | x_e) over the
 * receiver's members in order, members_host[i*64 + a] = member pixel (or -1).
 * Synchronous. */
occ_status occ_debug_mis(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* occ,
                         const occ_pattern* pattern, int32_t K, int32_t estimator,
                         const occ_bvh* bvh_or_null, const int32_t* pix_host, int32_t n,
                         int32_t* members_host, float* w_host);

#ifdef __cplusplus
}
#endif

#endif /* OCC_H */
