// kernels_trace.cu -- step 1 of Algorithms 1 and 2 (occluder generation) and the
// pinhole G-buffer input stage.
//
// One thread per receiver.  A CTA of 128 threads covers a 16 x 8 pixel tile and
// each warp an 8 x 4 sub-tile, so neighbouring rays start from neighbouring
// receivers and touch the same BVH nodes (short AO rays stay local).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "occ_device.cuh"
#include "occ_kernels.h"
#include "occ_path.cuh"

namespace occ {
namespace {

constexpr int kTileW = 16, kTileH = 8;

// Minimum resident CTAs per SM requested from the register allocator for the trace
// kernel (8 -> 64 registers, 10 -> 48, 12 -> 40).
#ifndef OCC_TRACE_MIN_BLOCKS
#define OCC_TRACE_MIN_BLOCKS 8
#endif

__device__ __forceinline__ void tile_pixel(int* x, int* y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    *x = blockIdx.x * kTileW + (warp & 1) * 8 + (lane & 7);
    *y = blockIdx.y * kTileH + (warp >> 1) * 4 + (lane >> 3);
}

// Step 1 for pixel (x, y) of a view.  Warp-collective (the warp shares its start node):
// every lane of the warp must call it, with pixels of the same view.
template <int EFFECT>
__device__ __forceinline__ void trace_pixel(const GBufView& gb, const DevBVH& bvh, float radius,
                                            const LightParams& lp, uint64_t seed, uint32_t sample,
                                            const RecView& rec, unsigned* status, int x, int y) {
    const bool inside = x < gb.W && y < gb.H;
    const uint32_t p = inside ? (uint32_t)y * (uint32_t)gb.W + (uint32_t)x : 0u;
    float3 xo = make_float3(0.0f, 0.0f, 0.0f), n = xo;
    const bool valid = inside && gb_fetch(gb, (int)p, &xo, &n);
    // AO segments are short: start below the part of the tree they cannot leave
    const uint32_t start = EFFECT == kAO ? warp_start_node(bvh, valid, xo, radius) : 0u;
    if (!inside) return;
    if (!valid) {
        write_record(rec, p, xo, xo, xo, 0.0f, -1);
        return;
    }
    RectLight L;
    if (EFFECT == kShadow) L = make_light(lp);
    float tmax;
    const float3 d = step1_ray<EFFECT>(xo, n, p, radius, L, seed, sample, &tmax);
    const Hit h = closest_hit(bvh, xo, d, tmax, status, start);
    if (h.id == kNoHit) {
        write_record(rec, p, xo, xo, xo, 0.0f, -1);
        return;
    }
    const float3 nz = hit_normal(bvh, h.slot, d);
    const float3 z = make_float3(fmaf(h.t, d.x, xo.x), fmaf(h.t, d.y, xo.y), fmaf(h.t, d.z, xo.z));
    write_record(rec, p, xo, z, nz, h.t, (int)h.id);
}

template <int EFFECT>
__global__ void __launch_bounds__(128, OCC_TRACE_MIN_BLOCKS) k_trace(GBufView gb, DevBVH bvh, float radius,
                                               LightParams lp, uint64_t seed, uint32_t sample,
                                               RecView rec, unsigned* status) {
    int x, y;
    tile_pixel(&x, &y);
    trace_pixel<EFFECT>(gb, bvh, radius, lp, seed, sample, rec, status, x, y);
}

// Persistent step 1 with dynamic ray fetching (AO): each warp keeps its lanes busy by
// taking new ray indices from a global counter (one atomic per warp refill) once at least
// OCC_TRACE_DYN_MIN_IDLE lanes have finished, instead of idling until the warp's longest
// ray ends (Aila and Laine, "Understanding the Efficiency of Ray Traversal on GPUs", HPG
// 2009).  Ray index i covers the same 16 x 8 tiles and 8 x 4 warp sub-tiles as k_trace,
// so a refill takes neighbouring pixels.  Rays start at the root.  Measured at 1080p on
// the 1M-triangle scene: 0.387 ms against 0.473 ms for k_trace<AO> (refill thresholds
// 16-24 equal, 1 lane: 0.411 ms; a per-ray start node did not help, nor did one start node
// per refill, the deepest node holding every refilled segment: 0.387 against 0.354 ms
// with the 128-bin tree).  Shadow rays of a
// tile head for one small light and stay coherent in k_trace, which refills would break
// (0.341 against 0.284 ms), so they keep the one-CTA-per-tile kernel.
#ifndef OCC_TRACE_DYN
#define OCC_TRACE_DYN 1
#endif
#ifndef OCC_TRACE_DYN_MIN_IDLE
#define OCC_TRACE_DYN_MIN_IDLE 16
#endif
// AO rays in the persistent kernel visit nodes with the scalar slab test (0) or the paired
// one (1, as the shadow rays)
#ifndef OCC_TRACE_AO_PAIRED
#define OCC_TRACE_AO_PAIRED 0
#endif
// 7 resident CTAs per SM (70 registers, no spill) measured 0.371 against 0.374 ms with 8
// (64 registers); 6: 0.373 ms.
#ifndef OCC_TRACE_DYN_MIN_BLOCKS
#define OCC_TRACE_DYN_MIN_BLOCKS 7
#endif

// Ray index i -> pixel: 128 rays per 16 x 8 tile (warp sub-tiles of 8 x 4).  order 0: tiles
// row-major (tiles_x per row); order 1: blocks of 8 x 8 tiles row-major (tiles_x rounded up
// to a multiple of 8), the tiles of a block in Morton order, so that the rays in flight cover
// compact regions of the image.  Indices of tiles outside the image give x >= W or y >= H.
__device__ __forceinline__ void index_pixel(uint32_t i, int tiles_x, int order, int* x, int* y) {
    const uint32_t tile = i >> 7, within = i & 127u;
    const uint32_t w = within >> 5, l = within & 31u;
    uint32_t tx, ty;
    if (order == 1) {
        const uint32_t bx = ((uint32_t)tiles_x + 7u) >> 3, blk = tile >> 6, m = tile & 63u;
        tx = (blk % bx) * 8u + ((m & 1u) | ((m >> 1) & 2u) | ((m >> 2) & 4u));
        ty = (blk / bx) * 8u + (((m >> 1) & 1u) | ((m >> 2) & 2u) | ((m >> 3) & 4u));
    } else {
        tx = tile % (uint32_t)tiles_x;
        ty = tile / (uint32_t)tiles_x;
    }
    *x = (int)tx * kTileW + (int)(w & 1u) * 8 + (int)(l & 7u);
    *y = (int)ty * kTileH + (int)(w >> 1) * 4 + (int)(l >> 3);
}

template <int EFFECT>
__global__ void __launch_bounds__(128, OCC_TRACE_DYN_MIN_BLOCKS)
    k_trace_dyn(GBufView gb, DevBVH bvh, float radius, LightParams lp, uint64_t seed,
                uint32_t sample, RecView rec, unsigned* status, unsigned* counter, int tiles_x,
                uint32_t n_idx, int min_idle, int order) {
    RectLight L;
    if (EFFECT == kShadow) L = make_light(lp);
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    Traversal t;
    StackEntry stack[kStackSize];
    trav_clear(t);
    t.overflow = false;
    t.bad = false;
    bool have = false, exhausted = false, overflow = false, bad = false;
    uint32_t p = 0;
    for (;;) {
        // lanes without a ray take the next indices (warp-uniform loop; ends when every
        // lane holds a ray or the counter ran past the last index)
        while (!exhausted) {
            const unsigned need = __ballot_sync(0xFFFFFFFFu, !have);
            if (!need) break;
            if (__popc(need) < min_idle && need != 0xFFFFFFFFu) break;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(counter, (unsigned)__popc(need));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base >= n_idx) {
                exhausted = true;
                break;
            }
            bool fresh = false;   // this lane took a valid receiver in this refill
            float3 xo = make_float3(0.0f, 0.0f, 0.0f), n = xo;
            if (!have) {
                const uint32_t idx = base + (uint32_t)__popc(need & below);
                int x, y;
                index_pixel(idx, tiles_x, order, &x, &y);
                if (idx < n_idx && x < gb.W && y < gb.H) {
                    p = (uint32_t)y * (uint32_t)gb.W + (uint32_t)x;
                    if (gb_fetch(gb, (int)p, &xo, &n))
                        fresh = true;
                    else
                        write_record(rec, p, xo, xo, xo, 0.0f, -1);
                }
            }
            if (fresh) {
                float tmax;
                const float3 d = step1_ray<EFFECT>(xo, n, p, radius, L, seed, sample, &tmax);
                trav_init(t, xo, d, tmax, 0u);
                have = true;
            }
        }
        if (!__any_sync(0xFFFFFFFFu, have)) break;
        if (have) {
            trav_round<false, EFFECT != kAO || OCC_TRACE_AO_PAIRED>(t, bvh, stack);
            if (trav_done(t)) {
                overflow |= t.overflow;
                bad |= t.bad;
                const float3 o = t.r.o, d = t.r.d;
                if (t.best_id == kNoHit) {
                    write_record(rec, p, o, o, o, 0.0f, -1);
                } else {
                    const float3 nz = hit_normal(bvh, t.best_slot, d);
                    const float3 z = make_float3(fmaf(t.tbest, d.x, o.x), fmaf(t.tbest, d.y, o.y),
                                                 fmaf(t.tbest, d.z, o.z));
                    write_record(rec, p, o, z, nz, t.tbest, (int)t.best_id);
                }
                have = false;
            }
        }
    }
    if (overflow && status) atomicOr(status, kStatusStackOverflowBit);
    if (OCC_CHECKS && bad && status) atomicOr(status, kStatusBadIndexBit);
}

// ---------------------------------------------------------------------------------------
// Batched step 1 over views of different sizes and effects: persistent CTAs stride over
// the concatenated 16 x 8 tiles of all views (view of a tile found by binary search on
// the tile offsets, staged in shared memory).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, OCC_TRACE_MIN_BLOCKS)
    k_trace_batch(const BatchView* views, const BatchDyn* dyn, int n_views, int n_tiles, DevBVH bvh,
                  unsigned* status) {
    __shared__ int s_first[kMaxBatchViews + 1];
    for (int v = threadIdx.x; v <= n_views; v += blockDim.x)
        s_first[v] = v < n_views ? views[v].first_tile : n_tiles;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int lo = 0, hi = n_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        const BatchView& v = views[lo];
        const int t = tile - s_first[lo];
        const int x = (t % v.tiles_x) * kTileW + (warp & 1) * 8 + (lane & 7);
        const int y = (t / v.tiles_x) * kTileH + (warp >> 1) * 4 + (lane >> 3);
        const BatchDyn d = dyn[lo];
        if (v.effect == kAO)
            trace_pixel<kAO>(v.gb, bvh, v.radius, v.light, d.seed, d.sample, v.rec, status, x, y);
        else
            trace_pixel<kShadow>(v.gb, bvh, v.radius, v.light, d.seed, d.sample, v.rec, status, x, y);
    }
}

__global__ void __launch_bounds__(128) k_gbuffer(DevBVH bvh, float3 eye, float3 f, float3 rt,
                                                 float3 up, float th, float aspect, float eps,
                                                 int W, int H, float4* pos, float4* nrm,
                                                 unsigned* status) {
    int x, y;
    tile_pixel(&x, &y);
    if (x >= W || y >= H) return;
    const uint32_t p = (uint32_t)y * (uint32_t)W + (uint32_t)x;
    const float sx = (2.0f * ((float)x + 0.5f) / (float)W - 1.0f) * th * aspect;
    const float sy = (1.0f - 2.0f * ((float)y + 0.5f) / (float)H) * th;
    const float3 d = normalize3(make_float3(f.x + sx * rt.x + sy * up.x, f.y + sx * rt.y + sy * up.y,
                                            f.z + sx * rt.z + sy * up.z));
    const Hit h = closest_hit(bvh, eye, d, 3.0e38f, status);
    // nrm == nullptr: one packed plane (point, octahedral normal code in w)
    if (h.id == kNoHit) {
        if (nrm) {
            pos[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            nrm[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
            pos[p] = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(kOctInvalid));
        }
        return;
    }
    const float3 n = hit_normal(bvh, h.slot, d);
    const float3 hp = make_float3(fmaf(h.t, d.x, eye.x) + eps * n.x, fmaf(h.t, d.y, eye.y) + eps * n.y,
                                  fmaf(h.t, d.z, eye.z) + eps * n.z);
    if (nrm) {
        pos[p] = make_float4(hp.x, hp.y, hp.z, 1.0f);
        nrm[p] = make_float4(n.x, n.y, n.z, 0.0f);
    } else {
        pos[p] = make_float4(hp.x, hp.y, hp.z, __uint_as_float(oct_encode(n)));
    }
}

__global__ void k_debug_philox(const uint32_t* in, int64_t n, uint32_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t* q = in + 6 * i;
    const uint4 w = philox4x32_10(make_uint4(q[0], q[1], q[2], q[3]), make_uint2(q[4], q[5]));
    out[4 * i + 0] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

// Closest (or any) hit of arbitrary rays: rays[2i] = (o.xyz, tmax), rays[2i+1] = (d.xyz, -).
__global__ void k_debug_closest_hit(DevBVH bvh, const float4* rays, int64_t n, int any, int32_t* tri,
                                    float* t, unsigned* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rays[2 * i], b = rays[2 * i + 1];
    if (any) {
        tri[i] = any_hit(bvh, f3(a), f3(b), a.w, status) ? 1 : 0;
        t[i] = 0.0f;
        return;
    }
    const Hit h = closest_hit(bvh, f3(a), f3(b), a.w, status);
    tri[i] = h.id == kNoHit ? -1 : (int32_t)h.id;
    t[i] = h.id == kNoHit ? -1.0f : h.t;
}

template <int EFFECT>
__global__ void k_debug_rays(GBufView gb, float radius, LightParams lp, uint64_t seed,
                             uint32_t sample, float4* out) {
    int x, y;
    tile_pixel(&x, &y);
    if (x >= gb.W || y >= gb.H) return;
    const uint32_t p = (uint32_t)y * (uint32_t)gb.W + (uint32_t)x;
    float3 xo, n;
    if (!gb_fetch(gb, (int)p, &xo, &n)) {
        out[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    RectLight L;
    if (EFFECT == kShadow) L = make_light(lp);
    float tmax;
    const float3 d = step1_ray<EFFECT>(xo, n, p, radius, L, seed, sample, &tmax);
    out[p] = make_float4(d.x, d.y, d.z, tmax);
}

// FP32 G-buffer -> packed G-buffer (receiver point kept, normal octahedral-encoded).
__global__ void k_pack_gbuffer(GBufView gb, float4* out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)gb.W * gb.H) return;
    const int g = gb_at(gb, (int)p);
    const float4 P = __ldg(gb.pos + g);
    const uint32_t code = P.w != 0.0f ? oct_encode(f3(__ldg(gb.nrm + g))) : kOctInvalid;
    out[p] = make_float4(P.x, P.y, P.z, __uint_as_float(code));
}

// G-buffer -> the same format in the tiled layout: pixel p's entries move from gb_at to
// their tiled index.
__global__ void k_tile_gbuffer(GBufView gb, float4* pos_out, float4* nrm_out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)gb.W * gb.H) return;
    const int y = (int)(p / gb.W), x = (int)(p - (int64_t)y * gb.W);
    const int g = gb_at(gb, (int)p);
    GBufView t = gb;
    t.tiled = 1;
    const int d = gb_index(t, x, y);
    pos_out[d] = __ldg(gb.pos + g);
    if (nrm_out) nrm_out[d] = __ldg(gb.nrm + g);
}

dim3 tile_grid(int W, int H) {
    return dim3((unsigned)((W + kTileW - 1) / kTileW), (unsigned)((H + kTileH - 1) / kTileH));
}

}  // namespace

cudaError_t launch_trace(int effect, const GBufView& gb, const DevBVH& bvh, float radius,
                         const LightParams& light, uint64_t seed, uint32_t sample, RecView rec,
                         unsigned* status, cudaStream_t s, unsigned* counter, const Tuning* tune) {
    if (gb.W <= 0 || gb.H <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(gb.W, gb.H);
    // persistent kernel by default for AO; the tuning may pick either kernel for either effect
    const int path = tune ? tune->trace_path : 0;
    const bool persistent = path == 2 || (path == 0 && effect == kAO);
    if (OCC_TRACE_DYN && counter && persistent) {
        const int order = tune && tune->trace_order == 2 ? 1 : 0;
        const uint32_t n_idx = order == 1 ? ((grid.x + 7u) / 8u) * ((grid.y + 7u) / 8u) * 64u * 128u
                                          : grid.x * grid.y * 128u;
        // persistent grid: resident CTAs per SM x SMs (computed once; threads that race
        // here compute the same value)
        static std::atomic<int> ctas[2];
        const int ei = effect == kAO ? 0 : 1;
        int n = ctas[ei].load(std::memory_order_relaxed);
        if (!n) {
            int dev = 0, sms = 1, per_sm = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, effect == kAO ? k_trace_dyn<kAO> : k_trace_dyn<kShadow>, 128, 0);
            n = (per_sm > 0 ? per_sm : 1) * sms;
            ctas[ei].store(n, std::memory_order_relaxed);
        }
        int want = n;
        if (tune && tune->trace_ctas_per_sm > 0) {
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            want = std::min(n, tune->trace_ctas_per_sm * sms);
        }
        const int min_idle = tune && tune->trace_refill > 0 ? tune->trace_refill : OCC_TRACE_DYN_MIN_IDLE;
        const unsigned blocks = (unsigned)want < grid.x * grid.y ? (unsigned)want : grid.x * grid.y;
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        if (effect == kAO)
            k_trace_dyn<kAO><<<blocks, 128, 0, s>>>(gb, bvh, radius, light, seed, sample, rec, status,
                                                   counter, (int)grid.x, n_idx, min_idle, order);
        else
            k_trace_dyn<kShadow><<<blocks, 128, 0, s>>>(gb, bvh, radius, light, seed, sample, rec,
                                                       status, counter, (int)grid.x, n_idx, min_idle,
                                                       order);
        return cudaGetLastError();
    }
    if (effect == kAO)
        k_trace<kAO><<<grid, 128, 0, s>>>(gb, bvh, radius, light, seed, sample, rec, status);
    else
        k_trace<kShadow><<<grid, 128, 0, s>>>(gb, bvh, radius, light, seed, sample, rec, status);
    return cudaGetLastError();
}

cudaError_t launch_gbuffer(const DevBVH& bvh, const float* cam, float eps, int W, int H,
                           float4* pos, float4* nrm, unsigned* status, cudaStream_t s) {
    if (W <= 0 || H <= 0) return cudaSuccess;
    // camera basis in FP32: forward, right = forward x up, up' = right x forward
    auto norm = [](float3 a) {
        const float l = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
        return make_float3(a.x / l, a.y / l, a.z / l);
    };
    auto cr = [](float3 a, float3 b) {
        return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
    };
    const float3 eye = make_float3(cam[0], cam[1], cam[2]);
    const float3 f = norm(make_float3(cam[3] - cam[0], cam[4] - cam[1], cam[5] - cam[2]));
    const float3 rt = norm(cr(f, make_float3(cam[6], cam[7], cam[8])));
    const float3 up = cr(rt, f);
    const float th = tanf(0.5f * cam[9] * 3.14159265358979f / 180.0f);
    k_gbuffer<<<tile_grid(W, H), 128, 0, s>>>(bvh, eye, f, rt, up, th, (float)W / (float)H, eps,
                                              W, H, pos, nrm, status);
    return cudaGetLastError();
}

cudaError_t launch_tile_gbuffer(const GBufView& gb, float4* pos_out, float4* nrm_out,
                                cudaStream_t s) {
    const int64_t P = (int64_t)gb.W * gb.H;
    if (P <= 0) return cudaSuccess;
    k_tile_gbuffer<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(gb, pos_out, gb.packed ? nullptr : nrm_out);
    return cudaGetLastError();
}

cudaError_t launch_trace_batch(const BatchView* views, const BatchDyn* dyn, int n_views, int n_tiles,
                               const DevBVH& bvh, int ctas, unsigned* status, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    k_trace_batch<<<ctas < n_tiles ? ctas : n_tiles, 128, 0, s>>>(views, dyn, n_views, n_tiles, bvh,
                                                                  status);
    return cudaGetLastError();
}

int trace_batch_ctas(int per_sm_wanted) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_batch, 128, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (per_sm_wanted > 0 && per_sm_wanted < per_sm) per_sm = per_sm_wanted;
    return per_sm * sms;
}

// out[p] = sum_l w[l] vis[l][p], accumulated in light order (one FMA per light).
__global__ void k_weighted_sum(const float* vis, int64_t P, LightWeights w, float* out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float acc = 0.0f;
    for (int l = 0; l < w.n; ++l) acc = fmaf(w.w[l], __ldg(vis + (size_t)l * P + p), acc);
    out[p] = acc;
}

cudaError_t launch_weighted_sum(const float* vis, int64_t P, const LightWeights& w, float* out,
                                cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    k_weighted_sum<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(vis, P, w, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_gbuffer(const GBufView& gb, float4* out, cudaStream_t s) {
    const int64_t n = (int64_t)gb.W * gb.H;
    if (n <= 0) return cudaSuccess;
    k_pack_gbuffer<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gb, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_closest_hit(const DevBVH& bvh, const float4* rays, int64_t n, int any,
                                     int32_t* tri, float* t, unsigned* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_debug_closest_hit<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(bvh, rays, n, any, tri, t, status);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint32_t* in, int64_t n, uint32_t* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_debug_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_rays(int effect, const GBufView& gb, float radius,
                              const LightParams& light, uint64_t seed, uint32_t sample,
                              float4* out, cudaStream_t s) {
    if (gb.W <= 0 || gb.H <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(gb.W, gb.H);
    if (effect == kAO)
        k_debug_rays<kAO><<<grid, 128, 0, s>>>(gb, radius, light, seed, sample, out);
    else
        k_debug_rays<kShadow><<<grid, 128, 0, s>>>(gb, radius, light, seed, sample, out);
    return cudaGetLastError();
}

}  // namespace occ
