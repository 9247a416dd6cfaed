// occ_kernels.h -- host-side launchers of the CUDA kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "occ_layout.h"

namespace occ {

struct GBufView {
    int32_t W, H;
    const float4* pos;   // FP32: (x.xyz, valid); packed: (x.xyz, octahedral normal code)
    const float4* nrm;   // FP32: (n.xyz, -); packed: unused
    int32_t packed;
    int32_t pitch;       // row pitch of the planes in pixels (>= W); pixel p = y W + x sits at
                         // y pitch + x
    int32_t tiled;       // 8 x 8 tiles, Morton order inside a tile (pitch unused; see gb_index)
};

// Occluder records.  FP32: plane 0 (z.xyz, tri id bits), plane 1 (n_z.xyz, t).
// Packed: plane 0 only, 16 bytes per pixel: the 64-bit offset word (z - x_source as three
// 19-bit mantissas with a shared exponent, bit 63 = occluder present), the octahedral n_z
// code and the tri id.
struct RecView {
    float4* r0;
    float4* r1;
    int32_t packed;
};

struct LightParams {
    float c[3], eu[3], ev[3];
};

constexpr int kMaxMembers = 64;

struct PatternParams {
    int32_t kind;       // 0 group, 1 box, 2 offsets, 3 random per receiver
    int32_t gw, gh;
    int32_t n_off;      // offsets / random: count
    int32_t K;          // members incl. the receiver
    int2 off[kMaxMembers - 1];
    int32_t halo[4];    // offsets: max extent left, right, up, down
    int32_t radius;     // random: disk radius in pixels
    uint32_t sample;    // random: the records' sample (counter word 1 of the draws)
    uint64_t seed;      // random: key of the draws
};

enum Effect { kAO = 0, kShadow = 1 };

// One view of a batched frame (device-resident work table; see occ_frame_batch).
constexpr int kMaxBatchViews = 256;
struct BatchView {
    GBufView gb;
    RecView rec;
    int32_t effect, estimator;
    float radius;
    LightParams light;
    PatternParams pat;
    float R2s;            // AO: R^2 (1 + 2^-16), rounded to float on the host
    float* out;
    int32_t tiles_x;      // 16 x 8 tiles per row of this view
    int32_t first_tile;   // offset of this view in the batch's tile space
};
// Per-frame values of a view, kept apart so a captured batch can be replayed with new ones.
struct BatchDyn {
    uint64_t seed;
    uint32_t sample;
    uint32_t pad;
};
enum Estimator { kNoReuse = 0, kBiased = 1, kUnbiased = 2, kBoxMean = 3, kLightUnbiased = 4 };

cudaError_t launch_gbuffer(const DevBVH& bvh, const float* cam, float eps, int W, int H,
                           float4* pos, float4* nrm, unsigned* status, cudaStream_t s);
struct Tuning;
// counter: a device word for the persistent dynamic-fetch kernel (reset on `s` before the
// launch); nullptr selects the one-CTA-per-tile kernel.  tune: trace launch choices
// (nullptr: defaults).
cudaError_t launch_trace(int effect, const GBufView& gb, const DevBVH& bvh, float radius,
                         const LightParams& light, uint64_t seed, uint32_t sample, RecView rec,
                         unsigned* status, cudaStream_t s, unsigned* counter = nullptr,
                         const Tuning* tune = nullptr);
cudaError_t launch_pack_gbuffer(const GBufView& gb, float4* out, cudaStream_t s);
constexpr int kMaxLights = 16;
struct LightWeights {
    float w[kMaxLights];
    int n;
};
cudaError_t launch_weighted_sum(const float* vis, int64_t P, const LightWeights& w, float* out,
                                cudaStream_t s);
cudaError_t launch_debug_philox(const uint32_t* in, int64_t n, uint32_t* out, cudaStream_t s);
cudaError_t launch_debug_wait_timeout(uint32_t spins, unsigned* status, cudaStream_t s);
cudaError_t launch_debug_closest_hit(const DevBVH& bvh, const float4* rays, int64_t n, int any,
                                     int32_t* tri, float* t, unsigned* status, cudaStream_t s);
cudaError_t launch_debug_rays(int effect, const GBufView& gb, float radius,
                              const LightParams& light, uint64_t seed, uint32_t sample,
                              float4* out, cudaStream_t s);
// Streaming ceiling of the group reuse kernel's memory pattern (kernels_probe.cu).
// G-buffer (either format, either layout) -> the same format in the tiled layout
cudaError_t launch_tile_gbuffer(const GBufView& gb, float4* pos_out, float4* nrm_out,
                                cudaStream_t s);
cudaError_t launch_stream_ceiling(const GBufView& gb, const RecView& rec, float* out,
                                  cudaStream_t s);
// FP32 throughput probe (kernels_probe.cu): *flop = FLOPs of the launch.
cudaError_t launch_fp32_peak(int paired, int iters, int blocks, float* sink, double* flop,
                             cudaStream_t s);

// Launch choices (0 = default); see occ_tuning.
struct Tuning {
    int tile_rows = 0;
    int window_path = 0;
    int batch_per_sm = 0;
    int fused_ao_path = 0;
    int group_prefetch = 0;   // group kernel L2 prefetch: 0 default, 1 none, 2 / 3 planes
    int trace_path = 0;       // 0 default (AO persistent, shadow per tile), 1 per tile, 2 persistent
    int trace_ctas_per_sm = 0;   // persistent trace: CTAs per SM (0: all that fit)
    int trace_refill = 0;     // persistent trace: idle lanes that trigger a refill (0: default)
    int trace_order = 0;      // persistent trace: 0 / 1 tiles row-major, 2 Morton blocks
};

// Workspace of the queued first-hit validation (unbiased group reuse): up to (K - 1) W H
// query words, W H validation words, two counters.  Without it the group kernel traces
// its validation rays inline.
struct ValidateWs {
    uint32_t* queue;
    size_t queue_cap;
    uint32_t* bits;
    size_t bits_cap;
    unsigned* counters;
};

cudaError_t launch_reuse(int effect, int estimator, const GBufView& gb, const RecView& rec,
                         const PatternParams& pat, float radius, const LightParams& light,
                         const DevBVH* bvh, float* out, unsigned* status, cudaStream_t s,
                         const Tuning& tune = Tuning(), uint64_t seed = 0, uint32_t sample = 0,
                         const ValidateWs* vws = nullptr);
// Batched frame over several views (persistent kernels over the concatenated tiles).
cudaError_t launch_trace_batch(const BatchView* views, const BatchDyn* dyn, int n_views, int n_tiles,
                               const DevBVH& bvh, int ctas, unsigned* status, cudaStream_t s);
int trace_batch_ctas(int per_sm_wanted);
cudaError_t launch_reuse_batch(const BatchView* views, const BatchDyn* dyn, int n_views,
                               int n_tiles, int max_k,
                               const DevBVH& bvh, int per_sm_wanted, unsigned* status,
                               cudaStream_t s);

// TMA-staged biased reuse for box / offset patterns; returns false (nothing launched) when
// the pattern or its staging does not fit that kernel.
bool launch_reuse_tile(int effect, const GBufView& gb, const RecView& rec, const PatternParams& pat,
                       float R2s, const LightParams& light, float* out, unsigned* status,
                       cudaStream_t s, cudaError_t* err, int tile_rows, bool pairs);

// Steps 1-3 in one kernel for GROUP patterns gw x gh in {2x1, 2x2, 4x2, 4x4}
// (frame_group_shape) and estimators NOREUSE, BIASED, UNBIASED, BOXMEAN; rec.r0 == nullptr
// stores no records.  mode (AO): 0 default, 1 one CTA per tile, 2 persistent group refill
// (needs `counter`, reset on `s` before the launch; unbiased always takes mode 1).
bool frame_group_shape(int gw, int gh);
cudaError_t launch_trace_reuse(int effect, int estimator, const GBufView& gb, const DevBVH& bvh,
                               float radius, const LightParams& light, uint64_t seed,
                               uint32_t sample, int gw, int gh, RecView rec, float* out,
                               unsigned* status, cudaStream_t s, unsigned* counter, int mode);

cudaError_t launch_debug_mis(int effect, int estimator, const GBufView& gb, const RecView& rec,
                             const PatternParams& pat, float radius, const LightParams& light,
                             const DevBVH* bvh, const int32_t* pix, int32_t n, int32_t* members,
                             float* w, unsigned* status, cudaStream_t s);

}  // namespace occ
